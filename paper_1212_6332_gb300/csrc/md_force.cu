// Density pass (Sec. 3.3, Fig. 5) and force pass (Fig. 6, Eq. 3), float64.
//
// Both passes walk the full neighbour list of each atom (both i->j and j->i
// are stored), so every atom's sums are private to one thread and no atomic
// update is needed (the paper does the same on the GPU; its CPU code uses
// Newton's third law instead, Sec. 4.3). The list is column-major, so a warp
// of 32 consecutive atoms loads one 128-byte row of indices per neighbour
// slot; neighbour positions are gathered from the Morton-sorted array,
// mostly from L1/L2.
//
// GB300 executes float64 at 1/64 of the float32 rate while its HBM sits
// idle in this kernel pair, so the work is split to evaluate every pair
// function once per step and to move bytes instead of float64 instructions:
//   density: for each list entry inside r_cut, V, rho, A = V'/r and
//            B = rho'/r from one rsqrt and two table-driven exponentials;
//            rho_i = sum rho, 1/2 sum V; F(rho_i), F'(rho_i); the pair
//            (A, B) is stored per list slot (zero outside r_cut);
//   force:   F_i = sum_j [A + (F'_i + F'_j) B] (x_j - x_i)   [Eq. (3)]
//            i.e. 5 float64 operations per pair after the separation,
//            optionally followed by v_i += dt/2 F_i/m (second half-kick).
#include "md_device.cuh"

namespace mdk {

constexpr int kFNT = 128;

template <int KIND, bool SINGLE>
__global__ void __launch_bounds__(kFNT) k_density(int64_t N, int64_t Np, Geo g, Pot P,
                                                  const double4_32a* __restrict__ x, const int* __restrict__ nn,
                                                  const int* __restrict__ nl, int max_nb,
                                                  double2* __restrict__ ab, double* __restrict__ rho,
                                                  double* __restrict__ Fp, double* __restrict__ e_atom,
                                                  const Ctl* ctl) {
    if (load_status(ctl)) return;
    __shared__ double sT[kExpTable];
    if (KIND == MD_POT_RGL) load_exp_table(sT, P.exp_T);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double L[3];
    int b = SINGLE ? 0 : g.atom_box[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
    const double4_32a xi = x[i];
    const int n = min(nn[i], max_nb);
    double r_i = 0.0, ep = 0.0;
    for (int k = 0; k < n; ++k) {
        const int64_t slot = (int64_t)k * Np + i;
        const int e = nl[slot];
        const double4_32a xj = x[entry_slot(e)];
        double dx, dy, dz;
        sep_entry(xi, xj, entry_code(e), L, dx, dy, dz);
        double r2 = dx * dx + dy * dy + dz * dz;
        double2 c = make_double2(0.0, 0.0);
        if (r2 < P.rc2) {
            double phi, fr;
            pair_eval<KIND>(P, sT, r2, phi, fr, c.x, c.y);
            r_i += fr;
            ep += phi;
        }
        ab[slot] = c;
    }
    double F, Fpi;
    embed<KIND>(P, r_i, F, Fpi);
    rho[i] = r_i;
    Fp[i] = Fpi;
    e_atom[i] = F + 0.5 * ep;
}

template <bool SINGLE>
__global__ void __launch_bounds__(kFNT) k_force(int64_t N, int64_t Np, Geo g, const double4_32a* __restrict__ x,
                                                const int* __restrict__ nn, const int* __restrict__ nl, int max_nb,
                                                const double2* __restrict__ ab, const double* __restrict__ Fp,
                                                double* __restrict__ f, double* __restrict__ v, double c_kick,
                                                const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double L[3];
    int b = SINGLE ? 0 : g.atom_box[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
    const double4_32a xi = x[i];
    const double Fpi = Fp[i];
    const int n = min(nn[i], max_nb);
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int k = 0; k < n; ++k) {
        const int64_t slot = (int64_t)k * Np + i;
        double2 c = ab[slot];
        // entries outside r_cut carry (0, 0): skip them with an integer test
        if ((__double_as_longlong(c.x) | __double_as_longlong(c.y)) == 0) continue;
        const int e = nl[slot];
        const int j = entry_slot(e);
        const double4_32a xj = x[j];
        double dx, dy, dz;
        sep_entry(xi, xj, entry_code(e), L, dx, dy, dz);
        double s = fma(Fpi + Fp[j], c.y, c.x);
        fx = fma(s, dx, fx);
        fy = fma(s, dy, fy);
        fz = fma(s, dz, fz);
    }
    f[i] = fx;
    f[Np + i] = fy;
    f[2 * Np + i] = fz;
    if (v) {
        v[i] += c_kick * fx;
        v[Np + i] += c_kick * fy;
        v[2 * Np + i] += c_kick * fz;
    }
}

void launch_forces_mixed(Engine& e, int kick, cudaStream_t s);

template <int KIND, bool SINGLE>
static void run_fp64(Engine& e, int kick, cudaStream_t s) {
    Geo g = make_geo(e);
    int nb = (int)((e.N + kFNT - 1) / kFNT);
    double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    e.launches += 2;
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        k_density<KIND, SINGLE><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.ab, e.rho,
                                                   e.Fp, e.e_atom, e.ctl);
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    k_force<SINGLE><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.nn, e.nl, e.max_nb, e.ab, e.Fp, e.f,
                                        kick ? e.v : nullptr, c_kick, e.ctl);
}

template <int KIND>
static void run_fp64_k(Engine& e, int kick, cudaStream_t s) {
    if (e.B == 1)
        run_fp64<KIND, true>(e, kick, s);
    else
        run_fp64<KIND, false>(e, kick, s);
}

void launch_forces(Engine& e, int kick, cudaStream_t s) {
    if (e.N == 0) return;
    if (e.cfg.precision == MD_MIXED) {
        launch_forces_mixed(e, kick, s);
        return;
    }
    switch (e.pot.kind) {
        case MD_POT_RGL: run_fp64_k<MD_POT_RGL>(e, kick, s); break;
        case MD_POT_SC: run_fp64_k<MD_POT_SC>(e, kick, s); break;
        default: run_fp64_k<MD_POT_SPLINE>(e, kick, s); break;
    }
}

}  // namespace mdk
