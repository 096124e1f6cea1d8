// Density pass (Sec. 3.3, Fig. 5) and force pass (Fig. 6, Eq. 3), float64.
//
// Both passes walk the full neighbour list of each atom (both i->j and j->i
// are stored), so every atom's sums are private to one thread and no atomic
// update is needed (the paper does the same on the GPU; its CPU code uses
// Newton's third law instead, Sec. 4.3). The list is column-major, so a warp
// of 32 consecutive atoms loads one 128-byte row of indices per neighbour
// slot; neighbour positions are gathered from the Morton-sorted array,
// mostly from L1/L2.
//   density: rho_i = sum_{j, r<rc} rho(r_ij); then F(rho_i), F'(rho_i)
//   force:   F_i = sum_{j, r<rc} [V'(r) + (F'_i + F'_j) rho'(r)] (x_j - x_i)/r
//            E_i = F(rho_i) + 1/2 sum_j V(r)
//            optionally v_i += dt/2 F_i/m (second half-kick, fused)
#include "md_device.cuh"

namespace mdk {

constexpr int kFNT = 128;

template <int KIND, bool SINGLE>
__global__ void __launch_bounds__(kFNT) k_density(int64_t N, int64_t Np, Geo g, Pot P,
                                                  const double4_32a* __restrict__ x, const int* __restrict__ nn,
                                                  const int* __restrict__ nl, int max_nb, double* __restrict__ rho,
                                                  double* __restrict__ Fp, double* __restrict__ e_atom,
                                                  const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double L[3], h[3];
    int b = SINGLE ? 0 : g.atom_box[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
        h[a] = 0.5 * L[a];
    }
    const double4_32a xi = x[i];
    const int n = min(nn[i], max_nb);
    double r_i = 0.0;
    for (int k = 0; k < n; ++k) {
        int j = nl[(int64_t)k * Np + i];
        double4_32a xj = x[j];
        double dx = minimg(xj.x - xi.x, L[0], h[0]);
        double dy = minimg(xj.y - xi.y, L[1], h[1]);
        double dz = minimg(xj.z - xi.z, L[2], h[2]);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < P.rc2) r_i += dens_f<KIND>(P, sqrt(r2));
    }
    double F, Fpi;
    embed<KIND>(P, r_i, F, Fpi);
    rho[i] = r_i;
    Fp[i] = Fpi;
    e_atom[i] = F;
}

template <int KIND, bool SINGLE>
__global__ void __launch_bounds__(kFNT) k_force(int64_t N, int64_t Np, Geo g, Pot P,
                                                const double4_32a* __restrict__ x, const int* __restrict__ nn,
                                                const int* __restrict__ nl, int max_nb, const double* __restrict__ Fp,
                                                double* __restrict__ f, double* __restrict__ e_atom,
                                                double* __restrict__ v, double c_kick, const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double L[3], h[3];
    int b = SINGLE ? 0 : g.atom_box[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
        h[a] = 0.5 * L[a];
    }
    const double4_32a xi = x[i];
    const double Fpi = Fp[i];
    const int n = min(nn[i], max_nb);
    double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
    for (int k = 0; k < n; ++k) {
        int j = nl[(int64_t)k * Np + i];
        double4_32a xj = x[j];
        double dx = minimg(xj.x - xi.x, L[0], h[0]);
        double dy = minimg(xj.y - xi.y, L[1], h[1]);
        double dz = minimg(xj.z - xi.z, L[2], h[2]);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < P.rc2) {
            double r = sqrt(r2);
            double phi, dphi, fr, dfr;
            pair_all<KIND>(P, r, phi, dphi, fr, dfr);
            double s = (dphi + (Fpi + Fp[j]) * dfr) / r;
            fx += s * dx;
            fy += s * dy;
            fz += s * dz;
            ep += phi;
        }
    }
    f[i] = fx;
    f[Np + i] = fy;
    f[2 * Np + i] = fz;
    e_atom[i] += 0.5 * ep;
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
    k_density<KIND, SINGLE><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.rho, e.Fp,
                                               e.e_atom, e.ctl);
    k_force<KIND, SINGLE><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.Fp, e.f,
                                             e.e_atom, kick ? e.v : nullptr, c_kick, e.ctl);
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
