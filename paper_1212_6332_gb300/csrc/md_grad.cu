// Adjoint of the force evaluation with respect to the potential parameters
// (no counterpart in the paper; it turns the force kernels into a
// force-matching gradient).
//
// Given g_i = dL/dF_i and g_E(b) = dL/dE_b for every atom i and box b, and
// the forces of Eq. (3) F_i = sum_j s_ij d_ij with d_ij = x_j - x_i,
// s_ij = [V'(r) + (F'_i + F'_j) rho'(r)] / r (symmetric in i, j):
//   dL/dtheta = sum_i sum_j { w_ij [dV' + (F'_i + F'_j) drho']
//                             + (u_i F''_i + g_E F'_i) drho + g_E dV / 2 }
//             + sum_i { u_i d_theta F'(rho_i) + g_E d_theta F(rho_i) },
// where d = d/dtheta at fixed r and rho, w_ij = g_i . d_ij / r, and
//   u_i = sum_j (g_i - g_j) . d_ij rho'(r_ij) / r_ij
// is a per-atom adjoint scalar (a gather of g_j over the list). The two
// passes of the forward pass become three:
//   k_grad_rho    recompute rho_i, F'_i and F''_i (or, when the float64
//                 forward values are current, k_grad_embed: F''_i from rho_i)
//   k_grad_u      u_i (k_grad_u_cached: rho'/r from the pair cache)
//   k_grad_param  per-pair terms into per-block parameter partials (RGL
//                 from the cached V, V', rho, rho' when current)
//                 (RGL: block reduction of 5 sums; spline: shared-memory
//                 histogram over the cubic coefficients of each interval)
// then a fixed-order reduction and, for splines, the transpose of the
// knot-value -> coefficient map (one more tridiagonal solve per spline).
// In mixed precision the adjoint evaluates its pair geometry and pair
// functions in float32 (cell-local offsets, as the mixed forward pass) and
// sums the parameter terms in float64 (RGL: per-thread sums; splines: the
// float64 coefficient histogram at the float32 pair distance).
#include <cstring>

#include "md_device.cuh"

namespace mdk {

constexpr int kGNT = 128;
constexpr int kRglParams = 5;

__device__ __forceinline__ double box_gE(const Geo& g, const double* gE, int64_t i) {
    if (!gE) return 0.0;
    return gE[g.B == 1 ? 0 : g.atom_box[i]];
}

__device__ __forceinline__ void sep(const Geo& g, const double4_32a* __restrict__ x, int64_t i, int j, double& dx,
                                    double& dy, double& dz) {
    int b = g.B == 1 ? 0 : g.atom_box[i];
    double Lx = g.L[3 * b], Ly = g.L[3 * b + 1], Lz = g.L[3 * b + 2];
    double4_32a xi = x[i], xj = x[j];
    dx = minimg(xj.x - xi.x, Lx, 0.5 * Lx);
    dy = minimg(xj.y - xi.y, Ly, 0.5 * Ly);
    dz = minimg(xj.z - xi.z, Lz, 0.5 * Lz);
}

// Species of atom i and type-pair table of (i, j) from the positions' pad
// lanes (splines with several species; 0 otherwise).
template <int KIND>
__device__ __forceinline__ int atom_tab(const Pot& P, const double4_32a* __restrict__ x, int64_t i) {
    return KIND == MD_POT_SPLINE && P.n_types > 1 ? pos_type(x[i]) : 0;
}
template <int KIND>
__device__ __forceinline__ int pair_tab(const Pot& P, const double4_32a* __restrict__ x, int64_t i, int j) {
    return KIND == MD_POT_SPLINE && P.n_types > 1 ? pair_table(P.n_types, pos_type(x[i]), pos_type(x[j])) : 0;
}

// rho_i, F'(rho_i) and F''(rho_i) into the per-atom arrays (F'' of the
// spline is that of its cubic piece; 0 on the linear extensions).
template <int KIND>
__device__ __forceinline__ void store_embedding(const Pot& P, double r_i, int64_t i, double* __restrict__ rho,
                                                double* __restrict__ Fp, double* __restrict__ Fpp, int a = 0) {
    double F, Fpi, Fppi = 0.0;
    embed<KIND>(P, r_i, F, Fpi, a);
    if (KIND == MD_POT_SPLINE) {
        double s = (r_i - P.st0[2]) * P.sinvh[2];
        int k = (int)s;
        if (s >= 0.0 && k < P.sn[2] - 1) {
            double u = r_i - (P.st0[2] + P.sh[2] * k);
            double4_32a c = P.sp[2][(int64_t)a * P.sn[2] + k];
            Fppi = 2.0 * c.z + 6.0 * c.w * u;
        }
    } else if (r_i > 0.0) {
        Fppi = 0.25 * P.F_scale / (r_i * sqrt(r_i));
    }
    rho[i] = r_i;
    Fp[i] = Fpi;
    Fpp[i] = Fppi;
}

// rho_i, F'(rho_i), F''(rho_i) recomputed from the list.
template <int KIND>
__global__ void __launch_bounds__(kGNT) k_grad_rho(int64_t N, int64_t Np, Geo g, Pot P,
                                                   const double4_32a* __restrict__ x, const int* __restrict__ nn,
                                                   const int* __restrict__ nl, int max_nb, double* __restrict__ rho,
                                                   double* __restrict__ Fp, double* __restrict__ Fpp) {
    __shared__ double sT[kExpTable];
    if (KIND == MD_POT_RGL) load_exp_table(sT, P.exp_T);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = min(nn[i], max_nb);
    double r_i = 0.0;
    for (int k = 0; k < n; ++k) {
        const int e = nl[(int64_t)k * Np + i];
        int j = entry_slot(e);
        double dx, dy, dz;
        sep(g, x, i, j, dx, dy, dz);
        double r2 = norm2(dx, dy, dz);
        if (r2 >= P.rc2) continue;
        double phi, fr, A, B;
        pair_eval<KIND>(P, sT, r2, phi, fr, A, B, pair_tab<KIND>(P, x, i, j));
        r_i += fr;
    }
    store_embedding<KIND>(P, r_i, i, rho, Fp, Fpp, atom_tab<KIND>(P, x, i));
}

// u_i = sum_j (g_i - g_j) . d_ij rho'(r)/r
template <int KIND>
__global__ void __launch_bounds__(kGNT) k_grad_u(int64_t N, int64_t Np, Geo g, Pot P,
                                                 const double4_32a* __restrict__ x, const int* __restrict__ nn,
                                                 const int* __restrict__ nl, int max_nb, const double* __restrict__ gs,
                                                 double* __restrict__ u) {
    __shared__ double sT[kExpTable];
    if (KIND == MD_POT_RGL) load_exp_table(sT, P.exp_T);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = min(nn[i], max_nb);
    const double gx = gs[i], gy = gs[Np + i], gz = gs[2 * Np + i];
    double acc = 0.0;
    for (int k = 0; k < n; ++k) {
        const int e = nl[(int64_t)k * Np + i];
        int j = entry_slot(e);
        double dx, dy, dz;
        sep(g, x, i, j, dx, dy, dz);
        double r2 = norm2(dx, dy, dz);
        if (r2 >= P.rc2) continue;
        double phi, fr, A, B;
        pair_eval<KIND>(P, sT, r2, phi, fr, A, B, pair_tab<KIND>(P, x, i, j));
        acc += ((gx - gs[j]) * dx + (gy - gs[Np + j]) * dy + (gz - gs[2 * Np + j]) * dz) * B;
    }
    u[i] = acc;
}

// ---------------------------------------------------------------- from the forward pass
//
// When the float64 pair cache, rho and F' are those of the current positions
// and potential (the forward pass that produced the forces being fitted),
// the adjoint reads them instead of evaluating the pair functions again:
// F'' from the stored rho, u_i with rho'/r from the cache (the same bits as
// recomputing them), and the RGL parameter terms from the cached V, V',
// rho and rho' alone (every derivative of Eq. (1)-(3) with respect to
// (A, xi, p, q, r0) is a multiple of these four at fixed r).

// F''(rho_i) from the stored rho_i
template <int KIND>
__global__ void __launch_bounds__(kGNT) k_grad_embed(int64_t N, Pot P, const double4_32a* __restrict__ x,
                                                     const double* __restrict__ rho, double* __restrict__ Fpp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double r_i = rho[i];
    double Fppi = 0.0;
    if (KIND == MD_POT_SPLINE) {
        const int a = atom_tab<KIND>(P, x, i);
        double s = (r_i - P.st0[2]) * P.sinvh[2];
        int k = (int)s;
        if (s >= 0.0 && k < P.sn[2] - 1) {
            double u = r_i - (P.st0[2] + P.sh[2] * k);
            double4_32a c = P.sp[2][(int64_t)a * P.sn[2] + k];
            Fppi = 2.0 * c.z + 6.0 * c.w * u;
        }
    } else if (r_i > 0.0) {
        Fppi = 0.25 * P.F_scale / (r_i * sqrt(r_i));
    }
    Fpp[i] = Fppi;
}

__device__ __forceinline__ bool zero_entry(double2 c) {
    return (__double_as_longlong(c.x) | __double_as_longlong(c.y)) == 0;
}

// u_i = sum_j (g_i - g_j) . d_ij rho'(r)/r with rho'/r from the cache and
// d_ij from the entry's image (zero cache entries lie beyond r_cut). Every
// entry in turn, the next cache value and list entry loaded ahead; zero
// entries skip the arithmetic (stepping each lane to its next non-zero
// entry kept the lanes converged at one dependent load per skipped
// entry); the sum keeps its order.
__global__ void __launch_bounds__(kGNT) k_grad_u_cached(int64_t N, int64_t Np, Geo g,
                                                        const double4_32a* __restrict__ x,
                                                        const int* __restrict__ nn, const int* __restrict__ nl,
                                                        int max_nb, const double4_32a* __restrict__ pc,
                                                        const double* __restrict__ gs, double* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < N;
    double L[3] = {0.0, 0.0, 0.0};
    double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    double gx = 0.0, gy = 0.0, gz = 0.0;
    int n = 0;
    if (active) {
        const int b = g.B == 1 ? 0 : g.atom_box[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) L[a] = g.L[3 * b + a];
        xi = x[i];
        n = min(nn[i], max_nb);
        gx = gs[i];
        gy = gs[Np + i];
        gz = gs[2 * Np + i];
    }
    const double2 zero = make_double2(0.0, 0.0);
    double acc = 0.0;
    double2 c = n > 0 ? cache_ab(pc, i) : zero;
    int e = n > 0 ? nl[i] : 0;
    const int kmax = warp_max(n);
    for (int k = 0; k < kmax; ++k) {
        const int64_t slot = (int64_t)k * Np + i;
        const bool more = k + 1 < n;
        const double2 cn = more ? cache_ab(pc, slot + Np) : zero;
        const int en = more ? nl[slot + Np] : 0;
        if (k < n && !zero_entry(c)) {
            const int j = entry_slot(e);
            double dx, dy, dz;
            sep_entry(xi, x[j], entry_code(e), L, dx, dy, dz);
            acc += ((gx - gs[j]) * dx + (gy - gs[Np + j]) * dy + (gz - gs[2 * Np + j]) * dz) * c.y;
        }
        c = cn;
        e = en;
    }
    if (active) u[i] = acc;
}

// RGL parameter terms from the cached values: with u = r/r0 - 1,
//   dV/dA = V/A, dV'/dA = V'/A;  drho/dxi = 2 rho/xi, drho'/dxi = 2 rho'/xi;
//   dV/dp = -u V, dV'/dp = -u V' - V/r0;  drho/dq = -2u rho, drho'/dq = -2u rho' - 2 rho/r0;
//   dV/dr0 = p (r/r0^2) V, dV'/dr0 = p (r/r0^2) V' + p V/r0^2 (likewise rho with 2q);
// the taper S(r) does not depend on the parameters and rides in V, rho.
__global__ void __launch_bounds__(kGNT) k_grad_param_rgl_cached(int64_t N, int64_t Np, Geo g, Pot P,
                                                                const double4_32a* __restrict__ x,
                                                                const int* __restrict__ nn,
                                                                const int* __restrict__ nl, int max_nb,
                                                                const double4_32a* __restrict__ pc,
                                                                const double* __restrict__ gs,
                                                                const double* __restrict__ gE,
                                                                const double* __restrict__ Fp,
                                                                const double* __restrict__ Fpp,
                                                                const double* __restrict__ u,
                                                                double inv_A, double two_inv_xi,
                                                                double* __restrict__ partial) {
    __shared__ double sh[kGNT / 32];
    const double inv_r0 = 1.0 / P.r0, inv_r02 = inv_r0 * inv_r0, pp = P.p, q2 = P.q2;
    double acc[kRglParams] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = g.B == 1 ? 0 : g.atom_box[i];
        const double L[3] = {g.L[3 * b], g.L[3 * b + 1], g.L[3 * b + 2]};
        const double4_32a xi = x[i];
        const int n = min(nn[i], max_nb);
        const double gx = gs[i], gy = gs[Np + i], gz = gs[2 * Np + i];
        const double ge = box_gE(g, gE, i);
        const double Fpi = Fp[i];
        const double aF = u[i] * Fpp[i] + ge * Fpi;
        const double aV = 0.5 * ge;
        for (int k = 0; k < n; ++k) {
            const int64_t slot = (int64_t)k * Np + i;
            const double2 c = cache_ab(pc, slot);
            if ((__double_as_longlong(c.x) | __double_as_longlong(c.y)) == 0) continue;
            const double2 fv = cache_fv(pc, slot);
            const int e = nl[slot];
            const int j = entry_slot(e);
            double dx, dy, dz;
            sep_entry(xi, x[j], entry_code(e), L, dx, dy, dz);
            const double r2 = norm2(dx, dy, dz);
            const double rinv = rsqrt_nr(r2);
            const double r = r2 * rinv;
            const double aVp = (gx * dx + gy * dy + gz * dz) * rinv;  // w
            const double aFp = aVp * (Fpi + Fp[j]);
            const double V = fv.y, rh = fv.x, Vp = c.x * r, rhp = c.y * r;
            const double uu = fma(r, inv_r0, -1.0), c0 = r * inv_r02;
            const double tV = aVp * Vp + aV * V, tR = aFp * rhp + aF * rh;
            acc[0] += tV * inv_A;
            acc[1] += tR * two_inv_xi;
            acc[2] += -uu * tV - aVp * V * inv_r0;
            acc[3] += -2.0 * uu * tR - 2.0 * aFp * rh * inv_r0;
            acc[4] += pp * (c0 * tV + aVp * V * inv_r02) + q2 * (c0 * tR + aFp * rh * inv_r02);
        }
    }
    for (int k = 0; k < kRglParams; ++k) {
        double t = block_sum<kGNT>(acc[k], sh);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kRglParams + k] = t;
    }
}

// The same sums with every pair visited once, from the atom of the lower
// slot (the upper rows of its rotated list, or its entries j > i when the
// list was kept ascending). The terms above are linear in the weights
// (w, 1/2 g_E, w (F'_i + F'_j), u F'' + g_E F'), so the two ordered pairs
// (i, j) and (j, i) add up to one term with the summed weights: w_i + w_j =
// (g_i - g_j) . d / r, a_F,i + a_F,j; the cached values of both slots are
// the same. Half the separations, square roots and parameter terms.
// The five parameter terms are linear combinations of four sums per thread,
// T1 = sum tV, T4 = sum tR, T23 = sum (r tV + w V), T56 = sum (r tR + a_F' rho)
// (with u = r/r0 - 1 and c0 = r/r0^2 expanded), combined once at the end:
// d/dA = T1/A, d/dxi = 2 T4/xi, d/dp = T1 - T23/r0, d/dq = 2 T4 - 2 T56/r0,
// d/dr0 = (p T23 + 2q T56)/r0^2; 1/r and r come from the integer pipe
// (rsqrt_sqrt). About 30 float64 instructions per pair instead of 53.
__global__ void __launch_bounds__(kGNT) k_grad_param_rgl_pairs(int64_t N, int64_t Np, Geo g, Pot P,
                                                               const double4_32a* __restrict__ x,
                                                               const int* __restrict__ nn,
                                                               const int* __restrict__ nl,
                                                               const int* __restrict__ n_up, int max_nb,
                                                               const double4_32a* __restrict__ pc,
                                                               const double* __restrict__ gs,
                                                               const double* __restrict__ gE,
                                                               const double* __restrict__ Fp,
                                                               const double* __restrict__ Fpp,
                                                               const double* __restrict__ u, double inv_A,
                                                               double two_inv_xi, double* __restrict__ partial) {
    __shared__ double sh[kGNT / 32];
    const double inv_r0 = 1.0 / P.r0, inv_r02 = inv_r0 * inv_r0, pp = P.p, q2 = P.q2;
    const double2 zero = make_double2(0.0, 0.0);
    double t1 = 0.0, t4 = 0.0, t23 = 0.0, t56 = 0.0;
    // warp-uniform outer loop (all lanes take part in the vote below); each
    // lane steps to its own next non-zero upper entry, as k_grad_u_cached
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < N; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool active = i < N;
        double L[3] = {0.0, 0.0, 0.0};
        double4_32a xi = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        double gx = 0.0, gy = 0.0, gz = 0.0, ge = 0.0, Fpi = 0.0, aFi = 0.0;
        int n = 0;
        if (active) {
            const int b = g.B == 1 ? 0 : g.atom_box[i];
#pragma unroll
            for (int a = 0; a < 3; ++a) L[a] = g.L[3 * b + a];
            xi = x[i];
            const int nup = n_up[i];
            n = nup < 0 ? min(nn[i], max_nb) : nup;
            gx = gs[i];
            gy = gs[Np + i];
            gz = gs[2 * Np + i];
            ge = box_gE(g, gE, i);
            Fpi = Fp[i];
            aFi = u[i] * Fpp[i] + ge * Fpi;
        }
        const double aV2 = ge;  // 1/2 g_E from each side
        // every row in turn (the next cache value and list entry loaded
        // ahead); zero entries and, in an unrotated list, entries j < i
        // skip the arithmetic
        double2 c = n > 0 ? cache_ab(pc, i) : zero;
        int e = n > 0 ? nl[i] : 0;
        const int kmax = warp_max(n);
        for (int k = 0; k < kmax; ++k) {
            const int64_t slot = (int64_t)k * Np + i;
            const bool more = k + 1 < n;
            const double2 cn = more ? cache_ab(pc, slot + Np) : zero;
            const int en = more ? nl[slot + Np] : 0;
            const int j = entry_slot(e);
            if (k < n && !zero_entry(c) && j > i) {
                const double2 fv = cache_fv(pc, slot);
                double dx, dy, dz;
                sep_entry(xi, x[j], entry_code(e), L, dx, dy, dz);
                const double r2 = norm2(dx, dy, dz);
                double rinv, r;
                rsqrt_sqrt(r2, rinv, r);
                const double W = ((gx - gs[j]) * dx + (gy - gs[Np + j]) * dy + (gz - gs[2 * Np + j]) * dz) * rinv;
                const double AFp = W * (Fpi + Fp[j]);
                const double AF = aFi + (u[j] * Fpp[j] + ge * Fp[j]);
                const double V = fv.y, rh = fv.x, Vp = c.x * r, rhp = c.y * r;
                const double tV = W * Vp + aV2 * V, tR = AFp * rhp + AF * rh;
                t1 += tV;
                t4 += tR;
                t23 = fma(r, tV, fma(W, V, t23));
                t56 = fma(r, tR, fma(AFp, rh, t56));
            }
            c = cn;
            e = en;
        }
    }
    double acc[kRglParams];
    acc[0] = t1 * inv_A;
    acc[1] = t4 * two_inv_xi;
    acc[2] = t1 - inv_r0 * t23;
    acc[3] = 2.0 * t4 - 2.0 * inv_r0 * t56;
    acc[4] = inv_r02 * (pp * t23 + q2 * t56);
    for (int k = 0; k < kRglParams; ++k) {
        double t = block_sum<kGNT>(acc[k], sh);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kRglParams + k] = t;
    }
}

// ---------------------------------------------------------------- RGL

// Derivatives of V, V', rho, rho' with respect to (A, xi, p, q, r0) at r,
// combined with the adjoint weights:
//   a_dV' = w, a_drho' = w (F'_i + F'_j), a_drho = u_i F''_i + gE F'_i, a_dV = gE/2.
__device__ __forceinline__ void rgl_param_terms(const Pot& P, const double* T, double r, double aVp, double aFp,
                                                double aF, double aV, double* acc) {
    double S, dS;
    taper(P, r, S, dS);
    const double p_r0 = P.p_r0, q2_r0 = P.q2_r0, r0 = P.r0;
    const double u = r / r0 - 1.0;
    const double E1 = exp_tab(P.p - p_r0 * r, T, P.ek);   // exp(-p u)
    const double E2 = exp_tab(P.q2 - q2_r0 * r, T, P.ek);  // exp(-2q u)
    const double gV = S, gVp = dS - p_r0 * S;    // V = 2A E1 gV, V' = 2A E1 gVp
    const double gf = S, gfp = dS - q2_r0 * S;   // rho = xi^2 E2 gf, rho' = xi^2 E2 gfp
    const double e1 = P.A2 * E1, e2 = P.xi2 * E2;
    const double V = e1 * gV, Vp = e1 * gVp, f = e2 * gf, fp = e2 * gfp;
    const double inv_r02 = 1.0 / (r0 * r0);
    // d/dA: V = 2A E1 S
    double dV_A = 2.0 * E1 * gV, dVp_A = 2.0 * E1 * gVp;
    // d/dxi: rho = xi^2 E2 S
    double df_xi = 2.0 * P.xi * E2 * gf, dfp_xi = 2.0 * P.xi * E2 * gfp;
    // d/dp: dE1/dp = -u E1, d(p/r0)/dp = 1/r0
    double dV_p = -u * V, dVp_p = -u * Vp - e1 * S / r0;
    // d/dq: dE2/dq = -2u E2, d(2q/r0)/dq = 2/r0
    double df_q = -2.0 * u * f, dfp_q = -2.0 * u * fp - 2.0 * e2 * S / r0;
    // d/dr0: du/dr0 = -r/r0^2, d(p/r0)/dr0 = -p/r0^2
    double c0 = r * inv_r02;
    double dV_r0 = P.p * c0 * V, dVp_r0 = P.p * c0 * Vp + e1 * P.p * S * inv_r02;
    double df_r0 = P.q2 * c0 * f, dfp_r0 = P.q2 * c0 * fp + e2 * P.q2 * S * inv_r02;
    acc[0] += aVp * dVp_A + aV * dV_A;
    acc[1] += aFp * dfp_xi + aF * df_xi;
    acc[2] += aVp * dVp_p + aV * dV_p;
    acc[3] += aFp * dfp_q + aF * df_q;
    acc[4] += aVp * dVp_r0 + aV * dV_r0 + aFp * dfp_r0 + aF * df_r0;
}

__global__ void __launch_bounds__(kGNT) k_grad_param_rgl(int64_t N, int64_t Np, Geo g, Pot P,
                                                         const double4_32a* __restrict__ x,
                                                         const int* __restrict__ nn, const int* __restrict__ nl,
                                                         int max_nb, const double* __restrict__ gs,
                                                         const double* __restrict__ gE,
                                                         const double* __restrict__ Fp,
                                                         const double* __restrict__ Fpp,
                                                         const double* __restrict__ u,
                                                         double* __restrict__ partial) {
    __shared__ double sT[kExpTable];
    __shared__ double sh[kGNT / 32];
    load_exp_table(sT, P.exp_T);
    double acc[kRglParams] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int n = min(nn[i], max_nb);
        const double gx = gs[i], gy = gs[Np + i], gz = gs[2 * Np + i];
        const double ge = box_gE(g, gE, i);
        const double Fpi = Fp[i];
        const double aF = u[i] * Fpp[i] + ge * Fpi;
        for (int k = 0; k < n; ++k) {
            const int e = nl[(int64_t)k * Np + i];
            int j = entry_slot(e);
            double dx, dy, dz;
            sep(g, x, i, j, dx, dy, dz);
            double r2 = norm2(dx, dy, dz);
            if (r2 >= P.rc2) continue;
            double r = sqrt(r2);
            double w = (gx * dx + gy * dy + gz * dz) / r;
            rgl_param_terms(P, sT, r, w, w * (Fpi + Fp[j]), aF, 0.5 * ge, acc);
        }
    }
    for (int k = 0; k < kRglParams; ++k) {
        double t = block_sum<kGNT>(acc[k], sh);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kRglParams + k] = t;
    }
}

// fixed-order sum of per-block partials, one block per output:
// out[k] = sum_b partial[b * np + k]
__global__ void __launch_bounds__(256) k_sum_partials(int nblocks, int np, const double* __restrict__ partial,
                                                      double* __restrict__ out) {
    __shared__ double sh[8];
    int k = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += partial[(int64_t)b * np + k];
    double t = block_sum<256>(s, sh);
    if (threadIdx.x == 0) out[k] = t;
}

// ---------------------------------------------------------------- splines

// Adjoint weights of one cubic piece c0 + c1 t + c2 t^2 + c3 t^3 (local
// t): value weight aval, slope weight aslope -> coefficient gradients.
__device__ __forceinline__ void piece_adj(double* sg, int k, double t, double aval, double aslope) {
    double t2 = t * t;
    atomicAdd(&sg[4 * k + 0], aval);
    atomicAdd(&sg[4 * k + 1], aval * t + aslope);
    atomicAdd(&sg[4 * k + 2], aval * t2 + 2.0 * t * aslope);
    atomicAdd(&sg[4 * k + 3], aval * t2 * t + 3.0 * t2 * aslope);
}

// Adjoint of spline_eval for spline w at argument s (value weight aval,
// slope weight aslope) into the coefficient gradients of spline w (layout:
// per interval 4 values; the extrapolation entry above the range is mapped
// onto the last interval: value c0+c1 h+c2 h^2+c3 h^3 and slope c1+2c2 h+3c3 h^2
// at t = h, so the same piece adjoint with t = h covers it, plus the slope
// weight times (s - t_end) on the value).
__device__ __forceinline__ void spline_adj(const Pot& P, int w, double s, double aval, double aslope, double* sg) {
    int n = P.sn[w];
    double t0 = P.st0[w], h = P.sh[w];
    double q = (s - t0) * P.sinvh[w];
    if (q < 0.0) {
        // value = c0 + c1 (s - t0) on interval 0, slope = c1
        double t = s - t0;
        atomicAdd(&sg[0], aval);
        atomicAdd(&sg[1], aval * t + aslope);
        return;
    }
    int k = (int)q;
    if (k >= n - 1) {
        // value = v_end + slope_end (s - t_end), slope = slope_end (last piece at t = h)
        double te = s - (t0 + h * (n - 1));
        piece_adj(sg, n - 2, h, aval, aslope + aval * te);
        return;
    }
    piece_adj(sg, k, s - (t0 + h * k), aval, aslope);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_grad_param_spline(int64_t N, int64_t Np, Geo g, Pot P,
                                                          const double4_32a* __restrict__ x,
                                                          const int* __restrict__ nn, const int* __restrict__ nl,
                                                          int max_nb, const double* __restrict__ gs,
                                                          const double* __restrict__ gE,
                                                          const double* __restrict__ rho,
                                                          const double* __restrict__ Fp,
                                                          const double* __restrict__ Fpp,
                                                          const double* __restrict__ u, int ncoef,
                                                          double* __restrict__ partial) {
    // [ncoef] coefficient gradients of this block (V pieces, rho pieces, F
    // pieces): its own slice of partial, added to by native float64 atomics
    // in L2. (A shared-memory histogram made the float64 atomics retry under
    // the contention of a shell's pairs meeting the same spline pieces,
    // each retry a float64 add: the spline loss + gradient ran at 231 per
    // second.)
    double* sg = partial + (int64_t)blockIdx.x * ncoef;
    for (int k = threadIdx.x; k < ncoef; k += NT) sg[k] = 0.0;
    __syncthreads();
    // per table 4 (n - 1) coefficients: V pair tables, rho pair tables, F tables
    const int np_ = P.n_types * (P.n_types + 1) / 2;
    const int cV = 4 * (P.sn[0] - 1), cR = 4 * (P.sn[1] - 1), cF = 4 * (P.sn[2] - 1);
    double* gV = sg;
    double* gR = sg + np_ * cV;
    double* gF = gR + np_ * cR;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int n = min(nn[i], max_nb);
        const double gx = gs[i], gy = gs[Np + i], gz = gs[2 * Np + i];
        const double ge = box_gE(g, gE, i);
        const double Fpi = Fp[i];
        const double aF = u[i] * Fpp[i] + ge * Fpi;
        for (int k = 0; k < n; ++k) {
            const int e = nl[(int64_t)k * Np + i];
            int j = entry_slot(e);
            double dx, dy, dz;
            sep(g, x, i, j, dx, dy, dz);
            double r2 = norm2(dx, dy, dz);
            if (r2 >= P.rc2) continue;
            double r = sqrt(r2);
            if (r >= P.rc) continue;
            double w = (gx * dx + gy * dy + gz * dz) / r;
            const int pt = pair_tab<MD_POT_SPLINE>(P, x, i, j);
            spline_adj(P, 0, r, 0.5 * ge, w, gV + pt * cV);
            spline_adj(P, 1, r, aF, w * (Fpi + Fp[j]), gR + pt * cR);
        }
        // embedding: u_i dF'/dtheta + gE dF/dtheta at rho_i
        spline_adj(P, 2, rho[i], ge, u[i], gF + atom_tab<MD_POT_SPLINE>(P, x, i) * cF);
    }
}

// Transpose of the knot-value -> coefficient map of one natural spline
// (coefficients c0 = y_k, c1 = (y_{k+1}-y_k)/h - h(2M_k + M_{k+1})/6,
// c2 = M_k/2, c3 = (M_{k+1}-M_k)/(6h), M = T^{-1} D y with T the symmetric
// tridiagonal (h/6, 2h/3, h/6) on interior knots and (D y)_k =
// (y_{k+1} - 2 y_k + y_{k-1})/h): gy = (d coef/d y)^T gc.
// One thread per table: np_ V tables (n0 knots), np_ rho tables (n1), nt F
// tables (n2), in the knot order.
__global__ void k_spline_adjoint(const double* __restrict__ gc_all, double* __restrict__ work,
                                 double* __restrict__ gy_all, int n0, int n1, int n2, double h0, double h1,
                                 double h2, int np_, int nt) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= 2 * np_ + nt) return;
    const int kind = w < np_ ? 0 : (w < 2 * np_ ? 1 : 2);
    const int n = kind == 0 ? n0 : (kind == 1 ? n1 : n2);
    const int t = kind == 0 ? w : (kind == 1 ? w - np_ : w - 2 * np_);  // table within its kind
    const int koff = kind == 0 ? t * n0 : (kind == 1 ? np_ * n0 + t * n1 : np_ * (n0 + n1) + t * n2);
    const int coff = kind == 0 ? t * 4 * (n0 - 1)
                               : (kind == 1 ? np_ * 4 * (n0 - 1) + t * 4 * (n1 - 1)
                                            : np_ * 4 * (n0 - 1 + n1 - 1) + t * 4 * (n2 - 1));
    const double h = kind == 0 ? h0 : (kind == 1 ? h1 : h2);
    const double* gc = gc_all + coff;
    double* gy = gy_all + koff;
    double* gM = work + 3 * koff;  // [n]
    double* cp = gM + n;           // Thomas scratch
    double* dp = cp + n;
    for (int k = 0; k < n; ++k) {
        gy[k] = 0.0;
        gM[k] = 0.0;
    }
    for (int k = 0; k < n - 1; ++k) {
        double g0 = gc[4 * k], g1 = gc[4 * k + 1], g2 = gc[4 * k + 2], g3 = gc[4 * k + 3];
        gy[k] += g0 - g1 / h;
        gy[k + 1] += g1 / h;
        gM[k] += -g1 * h / 3.0 + 0.5 * g2 - g3 / (6.0 * h);
        gM[k + 1] += -g1 * h / 6.0 + g3 / (6.0 * h);
    }
    // z = T^{-1} gM on the interior knots (T symmetric), Thomas algorithm
    double a = h / 6.0, bd = 2.0 * h / 3.0, cu = h / 6.0;
    for (int k = 1; k <= n - 2; ++k) {
        double den = k == 1 ? bd : bd - a * cp[k - 1];
        cp[k] = cu / den;
        dp[k] = (k == 1 ? gM[k] : gM[k] - a * dp[k - 1]) / den;
    }
    for (int k = n - 2; k >= 1; --k) gM[k] = dp[k] - (k < n - 2 ? cp[k] * gM[k + 1] : 0.0);
    // gy += D^T z
    for (int k = 1; k <= n - 2; ++k) {
        double z = gM[k] / h;
        gy[k - 1] += z;
        gy[k] -= 2.0 * z;
        gy[k + 1] += z;
    }
}

// ---------------------------------------------------------------- host

__global__ void k_gather_g(int64_t N, int64_t Np, const double* __restrict__ g_f, const int* __restrict__ perm,
                           double* __restrict__ gs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int64_t c = perm[t];
    gs[t] = g_f ? g_f[3 * c] : 0.0;
    gs[Np + t] = g_f ? g_f[3 * c + 1] : 0.0;
    gs[2 * Np + t] = g_f ? g_f[3 * c + 2] : 0.0;
}

// ---------------------------------------------------------------- mixed precision
//
// The same three passes with float32 pair math from the cell-local offsets
// (as in the mixed force kernels), float32 sums grouped per 16 list entries
// and compensated, and the per-thread parameter sums in float64.

template <int KIND, bool WIDE>
__global__ void __launch_bounds__(kGNT) k_grad_rho_mixed(int64_t N, int64_t Np, Geo g, Pot P,
                                                         const float4* __restrict__ xo, const int* __restrict__ nn,
                                                         const int* __restrict__ nl, int max_nb,
                                                         double* __restrict__ rho, double* __restrict__ Fp,
                                                         double* __restrict__ Fpp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CellSep cs = cell_sep<false>(g, CellSep{}, i);
    const float4 oi = xo[i];
    const int n = min(nn[i], max_nb);
    GSum acc;
    for (int k = 0; k < n; ++k) {
        const int e = nl[(int64_t)k * Np + i];
        int j = entry_slot(e);
        float dx, dy, dz;
        sep_mixed_entry<WIDE>(cs, oi, xo[j], e, dx, dy, dz);
        float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < P.f_rc2) acc.add(dens_ff<KIND>(P, r2 * rsqrtf(r2), species_pair<KIND>(P, oi, xo[j])));
        if ((k & kGroupMask) == kGroupMask) acc.flush();
    }
    store_embedding<KIND>(P, acc.value(), i, rho, Fp, Fpp, KIND == MD_POT_SPLINE ? off_type(oi) : 0);
}

template <int KIND, bool WIDE>
__global__ void __launch_bounds__(kGNT) k_grad_u_mixed(int64_t N, int64_t Np, Geo g, Pot P,
                                                       const float4* __restrict__ xo, const int* __restrict__ nn,
                                                       const int* __restrict__ nl, int max_nb,
                                                       const double* __restrict__ gs, double* __restrict__ u) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CellSep cs = cell_sep<false>(g, CellSep{}, i);
    const float4 oi = xo[i];
    const int n = min(nn[i], max_nb);
    const double gx = gs[i], gy = gs[Np + i], gz = gs[2 * Np + i];
    GSum acc;
    for (int k = 0; k < n; ++k) {
        const int e = nl[(int64_t)k * Np + i];
        int j = entry_slot(e);
        float dx, dy, dz;
        sep_mixed_entry<WIDE>(cs, oi, xo[j], e, dx, dy, dz);
        float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < P.f_rc2) {
            float rinv = rsqrtf(r2);
            float phi, dphi, fr, dfr;
            pair_allf<KIND>(P, r2 * rinv, phi, dphi, fr, dfr, species_pair<KIND>(P, oi, xo[j]));
            float w = (float)(gx - gs[j]) * dx + (float)(gy - gs[Np + j]) * dy + (float)(gz - gs[2 * Np + j]) * dz;
            acc.add(w * dfr * rinv);
        }
        if ((k & kGroupMask) == kGroupMask) acc.flush();
    }
    u[i] = acc.value();
}

__device__ __forceinline__ void rgl_param_terms_f(const Pot& P, float r, float aVp, float aFp, float aF, float aV,
                                                  double* acc) {
    float S, dS;
    taperf(P, r, S, dS);
    const float p_r0 = P.f_p_r0, q2_r0 = P.f_q2_r0, r0 = (float)P.r0;
    const float u = r / r0 - 1.0f;
    const float E1 = __expf(P.f_p - p_r0 * r), E2 = __expf(P.f_q2 - q2_r0 * r);
    const float gV = S, gVp = dS - p_r0 * S, gf = S, gfp = dS - q2_r0 * S;
    const float e1 = P.f_A2 * E1, e2 = P.f_xi2 * E2;
    const float V = e1 * gV, Vp = e1 * gVp, f = e2 * gf, fp = e2 * gfp;
    const float inv_r02 = 1.0f / (r0 * r0), c0 = r * inv_r02, pp = P.f_p, q2 = P.f_q2, xi = (float)P.xi;
    acc[0] += (double)(aVp * (2.0f * E1 * gVp) + aV * (2.0f * E1 * gV));
    acc[1] += (double)(aFp * (2.0f * xi * E2 * gfp) + aF * (2.0f * xi * E2 * gf));
    acc[2] += (double)(aVp * (-u * Vp - e1 * S / r0) + aV * (-u * V));
    acc[3] += (double)(aFp * (-2.0f * u * fp - 2.0f * e2 * S / r0) + aF * (-2.0f * u * f));
    acc[4] += (double)(aVp * (pp * c0 * Vp + e1 * pp * S * inv_r02) + aV * (pp * c0 * V) +
                       aFp * (q2 * c0 * fp + e2 * q2 * S * inv_r02) + aF * (q2 * c0 * f));
}

template <bool WIDE>
__global__ void __launch_bounds__(kGNT) k_grad_param_rgl_mixed(int64_t N, int64_t Np, Geo g, Pot P,
                                                               const float4* __restrict__ xo,
                                                               const int* __restrict__ nn,
                                                               const int* __restrict__ nl, int max_nb,
                                                               const double* __restrict__ gs,
                                                               const double* __restrict__ gE,
                                                               const double* __restrict__ Fp,
                                                               const double* __restrict__ Fpp,
                                                               const double* __restrict__ u,
                                                               double* __restrict__ partial) {
    __shared__ double sh[kGNT / 32];
    double acc[kRglParams] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const CellSep cs = cell_sep<false>(g, CellSep{}, i);
        const float4 oi = xo[i];
        const int n = min(nn[i], max_nb);
        const float gx = (float)gs[i], gy = (float)gs[Np + i], gz = (float)gs[2 * Np + i];
        const double ge = box_gE(g, gE, i);
        const double Fpi = Fp[i];
        const float aF = (float)(u[i] * Fpp[i] + ge * Fpi);
        // every ordered pair from its own side: the lists of the mixed path
        // are not rotated, so visiting each pair once would only mask the
        // lanes of the other half (measured slower: 0.445 -> 0.603 ms per
        // 221,184-atom gradient, the partner gathers added)
        for (int k = 0; k < n; ++k) {
            const int e = nl[(int64_t)k * Np + i];
            int j = entry_slot(e);
            float dx, dy, dz;
            sep_mixed_entry<WIDE>(cs, oi, xo[j], e, dx, dy, dz);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= P.f_rc2) continue;
            float rinv = rsqrtf(r2);
            float r = r2 * rinv;
            float w = (gx * dx + gy * dy + gz * dz) * rinv;
            rgl_param_terms_f(P, r, w, w * (float)(Fpi + Fp[j]), aF, (float)(0.5 * ge), acc);
        }
    }
    for (int k = 0; k < kRglParams; ++k) {
        double t = block_sum<kGNT>(acc[k], sh);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kRglParams + k] = t;
    }
}

// Spline parameter terms with the pair geometry in float32 (cell-local
// offsets): the adjoint weights and the coefficient histogram stay float64.
template <int NT, bool WIDE>
__global__ void __launch_bounds__(NT) k_grad_param_spline_mixed(int64_t N, int64_t Np, Geo g, Pot P,
                                                                const float4* __restrict__ xo,
                                                                const int* __restrict__ nn,
                                                                const int* __restrict__ nl, int max_nb,
                                                                const double* __restrict__ gs,
                                                                const double* __restrict__ gE,
                                                                const double* __restrict__ rho,
                                                                const double* __restrict__ Fp,
                                                                const double* __restrict__ Fpp,
                                                                const double* __restrict__ u, int ncoef,
                                                                double* __restrict__ partial) {
    double* sg = partial + (int64_t)blockIdx.x * ncoef;  // as in k_grad_param_spline
    for (int k = threadIdx.x; k < ncoef; k += NT) sg[k] = 0.0;
    __syncthreads();
    const int np_ = P.n_types * (P.n_types + 1) / 2;
    const int cV = 4 * (P.sn[0] - 1), cR = 4 * (P.sn[1] - 1), cF = 4 * (P.sn[2] - 1);
    double* gV = sg;
    double* gR = sg + np_ * cV;
    double* gF = gR + np_ * cR;
    const float rcf = (float)P.rc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const CellSep cs = cell_sep<false>(g, CellSep{}, i);
        const float4 oi = xo[i];
        const int n = min(nn[i], max_nb);
        const float gx = (float)gs[i], gy = (float)gs[Np + i], gz = (float)gs[2 * Np + i];
        const double ge = box_gE(g, gE, i);
        const double Fpi = Fp[i];
        const double aF = u[i] * Fpp[i] + ge * Fpi;
        for (int k = 0; k < n; ++k) {
            const int e = nl[(int64_t)k * Np + i];
            int j = entry_slot(e);
            float dx, dy, dz;
            sep_mixed_entry<WIDE>(cs, oi, xo[j], e, dx, dy, dz);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 >= P.f_rc2) continue;
            float rinv = rsqrtf(r2);
            float r = r2 * rinv;
            if (r >= rcf) continue;
            const double w = (double)((gx * dx + gy * dy + gz * dz) * rinv);
            const int pt = species_pair<MD_POT_SPLINE>(P, oi, xo[j]);
            spline_adj(P, 0, (double)r, 0.5 * ge, w, gV + pt * cV);
            spline_adj(P, 1, (double)r, aF, w * (Fpi + Fp[j]), gR + pt * cR);
        }
        spline_adj(P, 2, rho[i], ge, u[i], gF + off_type(oi) * cF);
    }
}

// The same histogram with every pair visited once, from the atom of the
// lower slot (the upper rows of its rotated list, or its entries j > i when
// the list was kept ascending): the adjoint weights of (i, j) and (j, i)
// add up (values 2 (g_E / 2) and a_F,i + a_F,j, slopes w_i + w_j =
// (g_i - g_j) . d / r), the type pair and r are the same from both sides,
// so one visit adds their sum. Half the geometry and the shared-memory
// atomics.
template <int NT>
__global__ void __launch_bounds__(NT) k_grad_param_spline_pairs(int64_t N, int64_t Np, Geo g, Pot P,
                                                                const double4_32a* __restrict__ x,
                                                                const int* __restrict__ nn,
                                                                const int* __restrict__ nl,
                                                                const int* __restrict__ n_up, int max_nb,
                                                                const double* __restrict__ gs,
                                                                const double* __restrict__ gE,
                                                                const double* __restrict__ rho,
                                                                const double* __restrict__ Fp,
                                                                const double* __restrict__ Fpp,
                                                                const double* __restrict__ u, int ncoef,
                                                                double* __restrict__ partial) {
    double* sg = partial + (int64_t)blockIdx.x * ncoef;  // as in k_grad_param_spline
    for (int k = threadIdx.x; k < ncoef; k += NT) sg[k] = 0.0;
    __syncthreads();
    const int np_ = P.n_types * (P.n_types + 1) / 2;
    const int cV = 4 * (P.sn[0] - 1), cR = 4 * (P.sn[1] - 1), cF = 4 * (P.sn[2] - 1);
    double* gV = sg;
    double* gR = sg + np_ * cV;
    double* gF = gR + np_ * cR;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int nup = n_up[i];
        const int n = nup < 0 ? min(nn[i], max_nb) : nup;
        const double gx = gs[i], gy = gs[Np + i], gz = gs[2 * Np + i];
        const double ge = box_gE(g, gE, i);
        const double Fpi = Fp[i];
        const double aFi = u[i] * Fpp[i] + ge * Fpi;
        for (int k = 0; k < n; ++k) {
            const int e = nl[(int64_t)k * Np + i];
            const int j = entry_slot(e);
            if (j <= i) continue;
            double dx, dy, dz;
            sep(g, x, i, j, dx, dy, dz);
            double r2 = norm2(dx, dy, dz);
            if (r2 >= P.rc2) continue;
            double r = sqrt(r2);
            if (r >= P.rc) continue;
            const double W = ((gx - gs[j]) * dx + (gy - gs[Np + j]) * dy + (gz - gs[2 * Np + j]) * dz) / r;
            const double AF = aFi + (u[j] * Fpp[j] + ge * Fp[j]);
            const int pt = pair_tab<MD_POT_SPLINE>(P, x, i, j);
            spline_adj(P, 0, r, ge, W, gV + pt * cV);
            spline_adj(P, 1, r, AF, W * (Fpi + Fp[j]), gR + pt * cR);
        }
        // embedding: u_i dF'/dtheta + gE dF/dtheta at rho_i
        spline_adj(P, 2, rho[i], ge, u[i], gF + atom_tab<MD_POT_SPLINE>(P, x, i) * cF);
    }
}

// Spline coefficient count over all tables: P pair tables each for V and rho,
// T embedding tables, 4 (n - 1) coefficients per table.
static int spline_ncoef(const Engine& e) {
    const md_potential& p = e.pot_host;
    const int T = e.pot.n_types, P = T * (T + 1) / 2;
    return 4 * (P * (p.n_phi - 1) + P * (p.n_f - 1) + T * (p.n_F - 1));
}
static int spline_nknots(const Engine& e) {
    const md_potential& p = e.pot_host;
    const int T = e.pot.n_types, P = T * (T + 1) / 2;
    return P * p.n_phi + P * p.n_f + T * p.n_F;
}
static void launch_spline_adjoint(Engine& e, double* grad, cudaStream_t s) {
    const md_potential& p = e.pot_host;
    const int T = e.pot.n_types, P = T * (T + 1) / 2;
    k_spline_adjoint<<<1, 32, 0, s>>>(e.grad_coef, e.spline_work, grad, p.n_phi, p.n_f, p.n_F, e.pot.sh[0],
                                      e.pot.sh[1], e.pot.sh[2], P, T);
}

template <int KIND, bool WIDE>
static int grad_mixed_impl(Engine& e, const double* g_f, const double* g_e, double* grad, cudaStream_t s) {
    Geo g = make_geo(e);
    int nb = (int)((e.N + kGNT - 1) / kGNT);
    k_gather_g<<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g_f, e.perm, e.grad_g);
    // rho and F' of the forward pass are current (it sums the same float32
    // terms in the same groups): F'' from rho alone
    if (e.forces_ok)
        k_grad_embed<KIND><<<nb, kGNT, 0, s>>>(e.N, e.pot, e.x, e.rho, e.grad_Fpp);
    else
        k_grad_rho_mixed<KIND, WIDE><<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.xo, e.nn, e.nl, e.max_nb,
                                                         e.rho, e.Fp, e.grad_Fpp);
    k_grad_u_mixed<KIND, WIDE><<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.xo, e.nn, e.nl, e.max_nb, e.grad_g,
                                                   e.grad_u);
    e.launches += 3;
    if (KIND == MD_POT_RGL) {
        k_grad_param_rgl_mixed<WIDE><<<e.grad_blocks, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.xo, e.nn, e.nl,
                                                                   e.max_nb, e.grad_g, g_e, e.Fp, e.grad_Fpp,
                                                                   e.grad_u, e.grad_partial);
        k_sum_partials<<<kRglParams, 256, 0, s>>>(e.grad_blocks, kRglParams, e.grad_partial, grad);
        e.launches += 2;
    } else {
        int ncoef = spline_ncoef(e);
        k_grad_param_spline_mixed<kGNT, WIDE><<<e.grad_blocks, kGNT, 0, s>>>(
            e.N, e.N_pad, g, e.pot, e.xo, e.nn, e.nl, e.max_nb, e.grad_g, g_e, e.rho, e.Fp, e.grad_Fpp, e.grad_u,
            ncoef, e.grad_partial);
        k_sum_partials<<<ncoef, 256, 0, s>>>(e.grad_blocks, ncoef, e.grad_partial, e.grad_coef);
        launch_spline_adjoint(e, grad, s);
        e.launches += 3;
    }
    return MD_OK;
}

template <int KIND>
static int grad_impl(Engine& e, const double* g_f, const double* g_e, double* grad, cudaStream_t s) {
    Geo g = make_geo(e);
    int nb = (int)((e.N + kGNT - 1) / kGNT);
    int npb = e.grad_blocks;
    // the forward pass's cache, rho and F' are those of these positions and
    // this potential: read them (the Newton's-third-law variant leaves the
    // lower cache slots unwritten)
    const bool cached = e.forces_ok && !e.newton3 && e.pc;
    k_gather_g<<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g_f, e.perm, e.grad_g);
    if (cached) {
        k_grad_embed<KIND><<<nb, kGNT, 0, s>>>(e.N, e.pot, e.x, e.rho, e.grad_Fpp);
        k_grad_u_cached<<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.nn, e.nl, e.max_nb, e.pc, e.grad_g, e.grad_u);
    } else {
        k_grad_rho<KIND><<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.rho, e.Fp,
                                             e.grad_Fpp);
        k_grad_u<KIND><<<nb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.grad_g, e.grad_u);
    }
    e.launches += 3;
    if (KIND == MD_POT_RGL) {
        if (cached && e.pot.A2 != 0.0 && e.pot.xi != 0.0 && e.n_up)
            k_grad_param_rgl_pairs<<<npb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.n_up, e.max_nb,
                                                        e.pc, e.grad_g, g_e, e.Fp, e.grad_Fpp, e.grad_u,
                                                        2.0 / e.pot.A2, 2.0 / e.pot.xi, e.grad_partial);
        else if (cached && e.pot.A2 != 0.0 && e.pot.xi != 0.0)
            k_grad_param_rgl_cached<<<npb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.pc,
                                                         e.grad_g, g_e, e.Fp, e.grad_Fpp, e.grad_u,
                                                         2.0 / e.pot.A2, 2.0 / e.pot.xi, e.grad_partial);
        else
            k_grad_param_rgl<<<npb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb, e.grad_g, g_e,
                                                 e.Fp, e.grad_Fpp, e.grad_u, e.grad_partial);
        k_sum_partials<<<kRglParams, 256, 0, s>>>(npb, kRglParams, e.grad_partial, grad);
        e.launches += 2;
    } else {
        int ncoef = spline_ncoef(e);
        if (e.n_up)
            k_grad_param_spline_pairs<kGNT><<<npb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.n_up,
                                                                    e.max_nb, e.grad_g, g_e, e.rho, e.Fp, e.grad_Fpp,
                                                                    e.grad_u, ncoef, e.grad_partial);
        else
            k_grad_param_spline<kGNT><<<npb, kGNT, 0, s>>>(e.N, e.N_pad, g, e.pot, e.x, e.nn, e.nl, e.max_nb,
                                                              e.grad_g, g_e, e.rho, e.Fp, e.grad_Fpp, e.grad_u, ncoef,
                                                              e.grad_partial);
        k_sum_partials<<<ncoef, 256, 0, s>>>(npb, ncoef, e.grad_partial, e.grad_coef);
        launch_spline_adjoint(e, grad, s);
        e.launches += 3;
    }
    return MD_OK;
}

int launch_param_grad(Engine& e, const double* g_f, const double* g_e, double* grad, cudaStream_t s) {
    if (e.N == 0)
        return cudaMemsetAsync(grad, 0, sizeof(double) * (e.pot.kind == MD_POT_SPLINE ? spline_nknots(e) : 5), s) ==
                       cudaSuccess ? MD_OK : MD_ERR_CUDA;
    // mixed precision: float32 pair geometry and pair functions in the
    // adjoint as in the forward pass
    const bool mixed = e.cfg.precision == MD_MIXED;
    if (e.pot.kind == MD_POT_RGL) {
        if (mixed)
            return e.wide ? grad_mixed_impl<MD_POT_RGL, true>(e, g_f, g_e, grad, s)
                          : grad_mixed_impl<MD_POT_RGL, false>(e, g_f, g_e, grad, s);
        return grad_impl<MD_POT_RGL>(e, g_f, g_e, grad, s);
    }
    if (e.pot.kind == MD_POT_SPLINE) {
        int ncoef = spline_ncoef(e);
        if ((size_t)ncoef * sizeof(double) > 200 * 1024) return MD_ERR_UNSUPPORTED;
        if (mixed)
            return e.wide ? grad_mixed_impl<MD_POT_SPLINE, true>(e, g_f, g_e, grad, s)
                          : grad_mixed_impl<MD_POT_SPLINE, false>(e, g_f, g_e, grad, s);
        if ((size_t)ncoef * sizeof(double) > 48 * 1024) {
            cudaFuncSetAttribute(k_grad_param_spline<kGNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(ncoef * sizeof(double)));
            cudaFuncSetAttribute(k_grad_param_spline_pairs<kGNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(ncoef * sizeof(double)));
        }
        return grad_impl<MD_POT_SPLINE>(e, g_f, g_e, grad, s);
    }
    return MD_ERR_UNSUPPORTED;
}

}  // namespace mdk
