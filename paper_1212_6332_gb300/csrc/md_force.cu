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
// idle in this kernel pair, so the work is split to evaluate every pair's
// functions once per step and to move bytes instead of float64 instructions:
//   pairs:   the lower slot of each pair (j > i in i's list) evaluates V,
//            rho, A = V'/r and B = rho'/r (one rsqrt, two table-driven
//            exponentials) and writes them into both lists' slots (the
//            partner's position comes from the reverse index built with the
//            list); all four are functions of r alone, so both slots get
//            the same bits the partner would have computed;
//   density: rho_i = sum rho, 1/2 sum V over i's slots in list order;
//            F(rho_i), F'(rho_i);
//   force:   F_i = sum_j [A + (F'_i + F'_j) B] (x_j - x_i)   [Eq. (3)]
//            i.e. 5 float64 operations per pair after the separation,
//            optionally followed by v_i += dt/2 F_i/m (second half-kick).
// The sums run over each list in list order, as a full evaluation per atom
// does (the block-per-box schedule evaluates every entry from its own
// side), so both give identical results.
#include "md_device.cuh"

namespace mdk {

constexpr int kFNT = 128;

// Pair pass. Lanes walk their own lists (coalesced rows, cheap separation
// and r^2), and the in-cutoff pairs are compacted through a per-warp queue
// in shared memory: every batch of 32 queued pairs is evaluated with all 32
// lanes active. On GB300 a masked lane still costs the float64 pipe its
// cycles, and without compaction half the lanes of a warp would idle (list
// lengths, the cutoff test).
constexpr int kQueue = 64;

template <int KIND>
__device__ __forceinline__ void eval_pair_item(const Pot& P, const double* __restrict__ sT, double r2, int64_t own,
                                               int64_t mir, double2* __restrict__ ab, double2* __restrict__ fv) {
    double2 c, w;
    pair_eval<KIND>(P, sT, r2, w.y, w.x, c.x, c.y);
    ab[own] = c;
    fv[own] = w;
    ab[mir] = c;
    fv[mir] = w;
}

template <int KIND, bool SINGLE>
__global__ void __launch_bounds__(kFNT) k_pairs_half(int64_t N, int64_t Np, Geo g, Pot P,
                                                     const double4_32a* __restrict__ x, const int* __restrict__ nn,
                                                     const int* __restrict__ nl, const int* __restrict__ rev,
                                                     const int* __restrict__ n_up, int max_nb,
                                                     double2* __restrict__ ab, double2* __restrict__ fv,
                                                     const Ctl* ctl) {
    if (load_status(ctl)) return;
    __shared__ double sT[kExpTable];
    // two queues per warp: pairs inside r_taper (no taper) and beyond it,
    // so each evaluated batch takes one branch of pair_eval
    __shared__ double q_r2[kFNT / 32][2][kQueue];
    __shared__ long long q_own[kFNT / 32][2][kQueue];
    __shared__ long long q_mir[kFNT / 32][2][kQueue];
    if (KIND == MD_POT_RGL) load_exp_table(sT, P.exp_T);
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < N;
    double L[3] = {0.0, 0.0, 0.0};
    double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    int kend = 0;
    if (active) {
        int b = SINGLE ? 0 : g.atom_box[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
        xi = x[i];
        const int n = min(nn[i], max_nb);
        // lists are [upper | lower]: the upper entries (j > i) are rows
        // 0..n_up-1; the lower ones are written by the partners' threads (a
        // list kept unrotated, n_up < 0, is scanned whole)
        const int nup = n_up[i];
        kend = nup < 0 ? n : nup;
    }
    const int kmax = warp_max(kend);
    int qn[2] = {0, 0};
    for (int k = 0; k < kmax; ++k) {
        bool in = false;
        double r2 = 0.0;
        int64_t own = 0, mir = 0;
        if (k < kend) {
            own = (int64_t)k * Np + i;
            const int e = nl[own];
            const int j = entry_slot(e);
            if (j > i) {
                double dx, dy, dz;
                sep_entry(xi, x[j], entry_code(e), L, dx, dy, dz);
                r2 = dx * dx + dy * dy + dz * dz;
                mir = (int64_t)rev[own] * Np + j;
                if (r2 < P.rc2) {
                    in = true;
                } else {
                    const double2 z = make_double2(0.0, 0.0);
                    ab[own] = z;
                    fv[own] = z;
                    ab[mir] = z;
                    fv[mir] = z;
                }
            }
        }
        const bool tq = r2 > P.rs2;
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
            const bool mine = in && (tq == (qq == 1));
            const unsigned m = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                const int p = qn[qq] + __popc(m & lt_mask);
                q_r2[wq][qq][p] = r2;
                q_own[wq][qq][p] = own;
                q_mir[wq][qq][p] = mir;
            }
            qn[qq] += __popc(m);
        }
        __syncwarp();
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
            if (qn[qq] >= 32) {
                qn[qq] -= 32;
                const int p = qn[qq] + lane;
                eval_pair_item<KIND>(P, sT, q_r2[wq][qq][p], q_own[wq][qq][p], q_mir[wq][qq][p], ab, fv);
                __syncwarp();
            }
        }
    }
#pragma unroll
    for (int qq = 0; qq < 2; ++qq)
        if (lane < qn[qq]) eval_pair_item<KIND>(P, sT, q_r2[wq][qq][lane], q_own[wq][qq][lane], q_mir[wq][qq][lane], ab, fv);
}

template <int KIND>
__global__ void __launch_bounds__(kFNT) k_rho_sum(int64_t N, int64_t Np, Pot P, const int* __restrict__ nn,
                                                  int max_nb, const double2* __restrict__ fv, double* __restrict__ rho,
                                                  double* __restrict__ Fp, double* __restrict__ e_atom,
                                                  const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = min(nn[i], max_nb);
    // explicit round-to-nearest adds: the block-per-box schedule sums the
    // same values in the same order and must not fuse them differently
    double r_i = 0.0, ep = 0.0;
    for (int k = 0; k < n; ++k) {
        double2 w = fv[(int64_t)k * Np + i];
        r_i = __dadd_rn(r_i, w.x);
        ep = __dadd_rn(ep, w.y);
    }
    double F, Fpi;
    embed<KIND>(P, r_i, F, Fpi);
    rho[i] = r_i;
    Fp[i] = Fpi;
    e_atom[i] = fma(0.5, ep, F);
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
    e.launches += 3;
    {
        PhaseScope scope(e, MD_PHASE_PAIRS, s);
        k_pairs_half<KIND, SINGLE><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.rev, e.n_up,
                                                      e.max_nb, e.ab, e.fv, e.ctl);
    }
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        k_rho_sum<KIND><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, e.pot, e.nn, e.max_nb, e.fv, e.rho, e.Fp, e.e_atom, e.ctl);
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
