// Mixed-precision density and force passes.
//
// Positions, velocities and the integrator stay float64. For the pair math
// each atom carries a float32 offset from the origin of the cell it was
// binned into at the last list build (xo, refreshed after every drift), so
// a separation is
//     d = (c_j - c_i) * cell_side + (o_j - o_i)
// with the cell difference taken as a minimum image in whole cells (exact)
// and both offsets below one cell side plus the skin: the float32 rounding
// error of d is ~1e-7 of a cell side, not of the box length. V, rho and
// their derivatives are evaluated in float32 (hardware exp2 / rsqrt); the
// per-atom sums rho_i, F_i and the pair energy add each group of 16 list
// entries in plain float32 and combine the groups with compensated float32
// accumulation (Neumaier), and F(rho_i), F'(rho_i) are taken in float64.
// The paper's own precedent is float32 positions inside its neighbour-list
// kernel (Sec. 4).
#include "md_device.cuh"

namespace mdk {

constexpr int kMNT = 128;
// List entries whose partner data (offset, F') are loaded together before
// their pair math: more loads in flight per thread, the sums in the same
// order and groups (4 entries: the 4M-atom step 1.98 -> 1.74 ms, 2 entries:
// 1.92 ms; the compiler's float32 contractions may differ between batch
// sizes, so results differ by float32 rounding).
#ifndef MD_MIXED_BATCH
#define MD_MIXED_BATCH 4
#endif
constexpr int kMB = MD_MIXED_BATCH;

// ---------------------------------------------------------------- packed RGL
//
// sm_100 and later issue two float32 multiply-adds, adds or multiplies on a
// register pair as one instruction (FFMA2 / FADD2 / FMUL2). The RGL passes
// take the list entries of a batch two at a time in that form: one
// instruction stream carries both entries' separation, r, taper and
// exponentials. The exponentials are 2^(g0 + g1 r) on the hardware base-2
// unit (the base change folded into the constants), and the taper variable
// is clamped to [0, 1] by the saturating FMA, so that an entry past r_cut
// gets S = dS = 0 exactly and no cutoff branch is needed (without a taper,
// S is the cutoff mask and dS = 0). Entries of the same group of 16 go to
// two float32 partial sums (even and odd entries), added at the group end.
// This cut the instructions per list entry from 93 to 61 (force) and 67 to
// 44 (density) on the 1M-atom Cu box (ncu instruction counters); with the
// loops no longer issue-bound, the loads below are software-pipelined.
// The packed loops serve atoms whose box has 3 or more cells per axis (the
// separation from the cell offset of the list entry); other atoms, and the
// other potentials, take the scalar loops.
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// separation of two list entries (a, b) of an atom whose box has 3 or more
// cells per axis, from the cell offsets the entries carry: sep_mixed_code's
// arithmetic for each
__device__ __forceinline__ void sep_code_pair(const CellSep& cs, float4 oi, float4 oa, float4 ob, int ea, int eb,
                                              float2& dx, float2& dy, float2& dz) {
    const unsigned ca = entry_code(ea), cb = entry_code(eb);
    const float2 bias = pk(-8388609.0f);
    const float2 kx = add2(make_float2(__int_as_float(0x4B000000 | (int)(ca & 3u)),
                                       __int_as_float(0x4B000000 | (int)(cb & 3u))), bias);
    const float2 ky = add2(make_float2(__int_as_float(0x4B000000 | (int)((ca >> 2) & 3u)),
                                       __int_as_float(0x4B000000 | (int)((cb >> 2) & 3u))), bias);
    const float2 kz = add2(make_float2(__int_as_float(0x4B000000 | (int)((ca >> 4) & 3u)),
                                       __int_as_float(0x4B000000 | (int)((cb >> 4) & 3u))), bias);
    dx = fma2(kx, pk(cs.lx), add2(make_float2(oa.x, ob.x), pk(-oi.x)));
    dy = fma2(ky, pk(cs.ly), add2(make_float2(oa.y, ob.y), pk(-oi.y)));
    dz = fma2(kz, pk(cs.lz), add2(make_float2(oa.z, ob.z), pk(-oi.z)));
}

// taper S(r) and dS/dr of two entries; TAPER false: S = [r^2 < rc^2], dS = 0
template <bool TAPER>
__device__ __forceinline__ void taper_pair(const Pot& P, float2 r, float2 r2, float2& S, float2& dS) {
    if (TAPER) {
        const float2 x = make_float2(__saturatef(fmaf(r.x, P.f_inv_w, P.f_x0)),
                                     __saturatef(fmaf(r.y, P.f_inv_w, P.f_x0)));
        const float2 x2 = mul2(x, x);
        const float2 t = fma2(x, fma2(x, pk(-6.0f), pk(15.0f)), pk(-10.0f));
        S = fma2(mul2(x2, x), t, pk(1.0f));
        dS = mul2(x2, fma2(x, fma2(x, pk(P.f_dS[2]), pk(P.f_dS[1])), pk(P.f_dS[0])));
    } else {
        S = make_float2(r2.x < P.f_rc2 ? 1.0f : 0.0f, r2.y < P.f_rc2 ? 1.0f : 0.0f);
        dS = pk(0.0f);
    }
}

// 2^(g0 + g1 r) of two entries
__device__ __forceinline__ float2 exp_pair(const float* g, float2 r) {
    const float2 a = fma2(r, pk(g[1]), pk(g[0]));
    return make_float2(ex2a(a.x), ex2a(a.y));
}

// Plain float32 partial sums of the even and odd entries of a group,
// folded into a compensated total at group ends.
struct GSum2 {
    float2 part = make_float2(0.0f, 0.0f);
    KSum tot;
    __device__ __forceinline__ void flush() {
        tot.add(part.x + part.y);
        part = make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ double value() {
        flush();
        return tot.value();
    }
};

// the cell offset of a list entry gives the separation (boxes of 3 or more
// cells per axis)
template <bool WIDE>
__device__ __forceinline__ bool code_sep(const CellSep& cs) {
    return WIDE || (cs.nx >= 3 && cs.ny >= 3 && cs.nz >= 3);
}

// F'_j of the density pass, float32, in the w lane of j's record
__device__ __forceinline__ float fp_of(const float4* __restrict__ xf, int64_t j) {
    return reinterpret_cast<const float*>(xf)[4 * j + 3];
}

// Software pipeline of the packed loops: the list entries of the next
// batch (PIPE 1), or of the batch after next with the partners' data of the
// next batch (PIPE 2), are in flight while a batch is evaluated. Slots past
// the end of the list hold atom i's own slot and a partner half an angstrom
// away (finite arithmetic), whose terms a 0/1 mask removes, so that every
// entry of a list, the last ones included, takes the same arithmetic (a
// pair gets the same bits from both of its atoms). Measured on the 4M-atom
// Cu box (ms per pass, density / force): scalar loops 0.450 / 0.678; packed
// with a scalar tail and no pipeline 0.514 / 0.695; PIPE 1 0.414 (52
// registers) / 0.546 (7 blocks per SM, a few registers spilled); PIPE 2
// 0.459 (72 registers) / 0.587 (5 blocks). Fewer registers for more
// resident warps did not pay (density at 48 or 40 registers: 0.448, 0.564;
// force at 64: 0.832), nor did batches of 2 entries (0.514 / 0.640).
#ifndef MD_MIXED_PIPE_DENSITY
#define MD_MIXED_PIPE_DENSITY 1
#endif
#ifndef MD_MIXED_PIPE_FORCE
#define MD_MIXED_PIPE_FORCE 1
#endif

__device__ __forceinline__ void load_entries(const int* __restrict__ row, int k0, int n, int64_t Np, int self,
                                             int (&e)[kMB]) {
#pragma unroll
    for (int u = 0; u < kMB; ++u) e[u] = k0 + u < n ? row[(int64_t)u * Np] : self;
}

__device__ __forceinline__ void load_partners(const float4* __restrict__ src, const int (&e)[kMB], int k0, int n,
                                              float4 pad, float4 (&o)[kMB]) {
#pragma unroll
    for (int u = 0; u < kMB; ++u) o[u] = k0 + u < n ? src[entry_slot(e[u])] : pad;
}

template <int N_, typename T>
__device__ __forceinline__ void copy_arr(T (&d)[N_], const T (&s)[N_]) {
#pragma unroll
    for (int u = 0; u < N_; ++u) d[u] = s[u];
}

// rho of one batch; FULL false: the first nv entries are real
template <bool TAPER, bool FULL>
__device__ __forceinline__ void rho_batch(const Pot& P, const CellSep& cs, float4 oi, const int (&e)[kMB],
                                          const float4 (&o)[kMB], int nv, float2& part) {
#pragma unroll
    for (int u = 0; u < kMB; u += 2) {
        float2 dx, dy, dz;
        sep_code_pair(cs, oi, o[u], o[u + 1], e[u], e[u + 1], dx, dy, dz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 r = mul2(r2, make_float2(rsqrtf(r2.x), rsqrtf(r2.y)));
        float2 S, dS;
        taper_pair<TAPER>(P, r, r2, S, dS);
        if (!FULL) S = mul2(S, make_float2(u < nv ? 1.0f : 0.0f, u + 1 < nv ? 1.0f : 0.0f));
        part = fma2(mul2(pk(P.f_xi2), exp_pair(P.f_g2, r)), S, part);
    }
}

// rho_i of the RGL density pass, packed (boxes of 3 or more cells per axis)
template <bool TAPER>
__device__ __forceinline__ double rho_rgl_packed(const Pot& P, const CellSep& cs, float4 oi,
                                                 const float4* __restrict__ xo, const int* __restrict__ nl,
                                                 int64_t Np, int64_t i, int n) {
    GSum2 acc;
    const int self = (int)((unsigned)i | (kNoShift << kSlotBits));
    const float4 pad = make_float4(oi.x + 0.5f, oi.y, oi.z, oi.w);
    const int64_t step = (int64_t)kMB * Np;
    const int* ra = nl + i;
    int e0[kMB], e1[kMB];
    float4 o0[kMB];
    load_entries(ra, 0, n, Np, self, e0);
    ra += step;
    if (MD_MIXED_PIPE_DENSITY == 2) {
        load_entries(ra, kMB, n, Np, self, e1);
        ra += step;
        load_partners(xo, e0, 0, n, pad, o0);
    }
    for (int k0 = 0; k0 < n; k0 += kMB) {
        if (MD_MIXED_PIPE_DENSITY == 2) {
            int e2[kMB];
            float4 o1[kMB];
            load_entries(ra, k0 + 2 * kMB, n, Np, self, e2);
            load_partners(xo, e1, k0 + kMB, n, pad, o1);
            if (k0 && !(k0 & kGroupMask)) acc.flush();
            if (k0 + kMB <= n)
                rho_batch<TAPER, true>(P, cs, oi, e0, o0, kMB, acc.part);
            else
                rho_batch<TAPER, false>(P, cs, oi, e0, o0, n - k0, acc.part);
            copy_arr(e0, e1);
            copy_arr(e1, e2);
            copy_arr(o0, o1);
        } else {
            load_entries(ra, k0 + kMB, n, Np, self, e1);
            load_partners(xo, e0, k0, n, pad, o0);
            if (k0 && !(k0 & kGroupMask)) acc.flush();
            if (k0 + kMB <= n)
                rho_batch<TAPER, true>(P, cs, oi, e0, o0, kMB, acc.part);
            else
                rho_batch<TAPER, false>(P, cs, oi, e0, o0, n - k0, acc.part);
            copy_arr(e0, e1);
        }
        ra += step;
    }
    return acc.value();
}

// F_i, the pair energy and the virial of one batch; partner data (offset,
// F' in w); FULL false: the first nv entries are real
template <bool TAPER, bool FULL, bool VIR>
__device__ __forceinline__ void force_batch(const Pot& P, const CellSep& cs, float4 oi, float Fpi,
                                            const int (&e)[kMB], const float4 (&o)[kMB], int nv, GSum2& ax,
                                            GSum2& ay, GSum2& az, GSum2& ae, GSum2& aw) {
#pragma unroll
    for (int u = 0; u < kMB; u += 2) {
        float2 dx, dy, dz;
        sep_code_pair(cs, oi, o[u], o[u + 1], e[u], e[u + 1], dx, dy, dz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 r = mul2(r2, rinv);
        float2 S, dS;
        taper_pair<TAPER>(P, r, r2, S, dS);
        if (!FULL) {
            const float2 v = make_float2(u < nv ? 1.0f : 0.0f, u + 1 < nv ? 1.0f : 0.0f);
            S = mul2(S, v);
            dS = mul2(dS, v);
        }
        const float2 e1 = mul2(pk(P.f_A2), exp_pair(P.f_g1, r));
        const float2 e2 = mul2(pk(P.f_xi2), exp_pair(P.f_g2, r));
        const float2 dphi = mul2(e1, fma2(S, pk(-P.f_p_r0), dS));
        const float2 dfr = mul2(e2, fma2(S, pk(-P.f_q2_r0), dS));
        const float2 sv = mul2(fma2(add2(pk(Fpi), make_float2(o[u].w, o[u + 1].w)), dfr, dphi), rinv);
        ax.part = fma2(sv, dx, ax.part);
        ay.part = fma2(sv, dy, ay.part);
        az.part = fma2(sv, dz, az.part);
        ae.part = fma2(e1, S, ae.part);
        if (VIR) aw.part = fma2(sv, r2, aw.part);
    }
}

// the RGL force pass, packed (boxes of 3 or more cells per axis); xf holds
// each atom's offset with F' in w
template <bool TAPER, bool VIR>
__device__ __forceinline__ void force_rgl_packed(const Pot& P, const CellSep& cs, float4 oi, float Fpi,
                                                 const float4* __restrict__ xf, const int* __restrict__ nl,
                                                 int64_t Np, int64_t i, int n, GSum2& ax, GSum2& ay, GSum2& az,
                                                 GSum2& ae, GSum2& aw) {
    const int self = (int)((unsigned)i | (kNoShift << kSlotBits));
    const float4 pad = make_float4(oi.x + 0.5f, oi.y, oi.z, 0.0f);
    const int64_t step = (int64_t)kMB * Np;
    const int* ra = nl + i;
    int e0[kMB], e1[kMB];
    float4 o0[kMB];
    load_entries(ra, 0, n, Np, self, e0);
    ra += step;
    if (MD_MIXED_PIPE_FORCE == 2) {
        load_entries(ra, kMB, n, Np, self, e1);
        ra += step;
        load_partners(xf, e0, 0, n, pad, o0);
    }
    for (int k0 = 0; k0 < n; k0 += kMB) {
        if (MD_MIXED_PIPE_FORCE == 2) {
            int e2[kMB];
            float4 o1[kMB];
            load_entries(ra, k0 + 2 * kMB, n, Np, self, e2);
            load_partners(xf, e1, k0 + kMB, n, pad, o1);
            if (k0 && !(k0 & kGroupMask)) {
                ax.flush();
                ay.flush();
                az.flush();
                ae.flush();
                if (VIR) aw.flush();
            }
            if (k0 + kMB <= n)
                force_batch<TAPER, true, VIR>(P, cs, oi, Fpi, e0, o0, kMB, ax, ay, az, ae, aw);
            else
                force_batch<TAPER, false, VIR>(P, cs, oi, Fpi, e0, o0, n - k0, ax, ay, az, ae, aw);
            copy_arr(e0, e1);
            copy_arr(e1, e2);
            copy_arr(o0, o1);
        } else {
            load_entries(ra, k0 + kMB, n, Np, self, e1);
            load_partners(xf, e0, k0, n, pad, o0);
            if (k0 && !(k0 & kGroupMask)) {
                ax.flush();
                ay.flush();
                az.flush();
                ae.flush();
                if (VIR) aw.flush();
            }
            if (k0 + kMB <= n)
                force_batch<TAPER, true, VIR>(P, cs, oi, Fpi, e0, o0, kMB, ax, ay, az, ae, aw);
            else
                force_batch<TAPER, false, VIR>(P, cs, oi, Fpi, e0, o0, n - k0, ax, ay, az, ae, aw);
            copy_arr(e0, e1);
        }
        ra += step;
    }
}

// (no minimum of resident blocks: with one, the compiler takes 62 registers
// instead of 52, and the pass runs 0.414 instead of 0.388 ms)
template <int KIND, bool SINGLE, bool WIDE, bool TAPER>
__global__ void __launch_bounds__(kMNT) k_density_mixed(int64_t N, int64_t Np, Geo g, CellSep cs0, Pot P,
                                                        const float4* __restrict__ xo, const int* __restrict__ nn,
                                                        const int* __restrict__ nl, int max_nb,
                                                        double* __restrict__ rho, double* __restrict__ Fp,
                                                        float4* __restrict__ xf, double* __restrict__ e_atom,
                                                        const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CellSep cs = cell_sep<SINGLE>(g, cs0, i);
    const float4 oi = xo[i];
    const int n = min(nn[i], max_nb);
    double r_i;
    if (KIND == MD_POT_RGL && code_sep<WIDE>(cs)) {
        r_i = rho_rgl_packed<TAPER>(P, cs, oi, xo, nl, Np, i, n);
    } else {
    GSum acc;
    for (int k0 = 0; k0 < n; k0 += kMB) {
        int eb[kMB];
        float4 ob[kMB];
#pragma unroll
        for (int u = 0; u < kMB; ++u) eb[u] = k0 + u < n ? nl[(int64_t)(k0 + u) * Np + i] : 0;
#pragma unroll
        for (int u = 0; u < kMB; ++u) ob[u] = k0 + u < n ? xo[entry_slot(eb[u])] : oi;
#pragma unroll
        for (int u = 0; u < kMB; ++u) {
            const int k = k0 + u;
            if (k >= n) break;
            float dx, dy, dz;
            sep_mixed_entry<WIDE>(cs, oi, ob[u], eb[u], dx, dy, dz);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.f_rc2) acc.add(dens_ff<KIND>(P, r2 * rsqrtf(r2), species_pair<KIND>(P, oi, ob[u])));
            if ((k & kGroupMask) == kGroupMask) acc.flush();
        }
    }
    r_i = acc.value();
    }
    double F, Fpi;
    embed<KIND>(P, r_i, F, Fpi, KIND == MD_POT_SPLINE ? off_type(oi) : 0);
    rho[i] = r_i;
    Fp[i] = Fpi;
    xf[i] = make_float4(oi.x, oi.y, oi.z, (float)Fpi);
    e_atom[i] = F;
}

// Resident blocks per multiprocessor: with one entry in flight per thread
// the pass waits on gathered offsets and F', and 12 blocks (40 registers, a
// few spilled to L1) hid more of that than the spills cost (8% faster than
// 54 registers); with a batch of entries in flight the registers go to the
// batch instead.
#ifndef MD_MIXED_FORCE_BLOCKS
#define MD_MIXED_FORCE_BLOCKS (kMB == 1 ? 12 : 8)
#endif
// the packed RGL force loop holds two entries' float32 state and its packed
// constants in register pairs: 72 registers at 7 blocks (some spilled to
// L1), faster than 80 registers at 6 blocks or 64 at 8
#ifndef MD_MIXED_FORCE_BLOCKS_RGL
#define MD_MIXED_FORCE_BLOCKS_RGL 7
#endif
template <int KIND, bool SINGLE, bool WIDE, bool TAPER, bool VIR>
__global__ void __launch_bounds__(kMNT, KIND == MD_POT_RGL ? MD_MIXED_FORCE_BLOCKS_RGL : MD_MIXED_FORCE_BLOCKS) k_force_mixed(int64_t N, int64_t Np, Geo g, CellSep cs0, Pot P,
                                                      const float4* __restrict__ xo, const int* __restrict__ nn,
                                                      const int* __restrict__ nl, int max_nb,
                                                      const float4* __restrict__ xf, double* __restrict__ f,
                                                      double* __restrict__ e_atom, double* __restrict__ v,
                                                      double c_kick, Bath bath, double* __restrict__ w_atom,
                                                      const Ctl* ctl) {
    if (load_status(ctl)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const CellSep cs = cell_sep<SINGLE>(g, cs0, i);
    const float4 oi = xo[i];
    const float Fpi = fp_of(xf, i);
    const int n = min(nn[i], max_nb);
    // w_atom (pressure users only): per-atom virial -1/2 sum_j s_ij r_ij^2
    const bool vir = VIR;
    double fx, fy, fz, epair, wsum;
    if (KIND == MD_POT_RGL && code_sep<WIDE>(cs)) {
        GSum2 ax, ay, az, ae, aw;
        force_rgl_packed<TAPER, VIR>(P, cs, oi, Fpi, xf, nl, Np, i, n, ax, ay, az, ae, aw);
        fx = ax.value();
        fy = ay.value();
        fz = az.value();
        epair = ae.value();
        wsum = vir ? aw.value() : 0.0;
    } else {
    GSum ax, ay, az, ae, aw;
    for (int k0 = 0; k0 < n; k0 += kMB) {
        int eb[kMB];
        float4 ob[kMB];
        float fb[kMB];
#pragma unroll
        for (int u = 0; u < kMB; ++u) eb[u] = k0 + u < n ? nl[(int64_t)(k0 + u) * Np + i] : 0;
#pragma unroll
        for (int u = 0; u < kMB; ++u) {
            const bool ok = k0 + u < n;
            ob[u] = ok ? xo[entry_slot(eb[u])] : oi;
            fb[u] = ok ? fp_of(xf, entry_slot(eb[u])) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kMB; ++u) {
            const int k = k0 + u;
            if (k >= n) break;
            if ((k & kGroupMask) == 0 && k) {
                ax.flush();
                ay.flush();
                az.flush();
                ae.flush();
                if (vir) aw.flush();
            }
            float dx, dy, dz;
            sep_mixed_entry<WIDE>(cs, oi, ob[u], eb[u], dx, dy, dz);
            float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.f_rc2) {
                float rinv = rsqrtf(r2);
                float r = r2 * rinv;
                float phi, dphi, fr, dfr;
                pair_allf<KIND>(P, r, phi, dphi, fr, dfr, species_pair<KIND>(P, oi, ob[u]));
                float s = (dphi + (Fpi + fb[u]) * dfr) * rinv;
                ax.add(s * dx);
                ay.add(s * dy);
                az.add(s * dz);
                ae.add(phi);
                if (vir) aw.add(s * r2);
            }
        }
    }
    fx = ax.value();
    fy = ay.value();
    fz = az.value();
    epair = ae.value();
    wsum = vir ? aw.value() : 0.0;
    }
    f[i] = fx;
    f[Np + i] = fy;
    f[2 * Np + i] = fz;
    e_atom[i] += 0.5 * epair;
    if (vir) w_atom[i] = -0.5 * wsum;
    if (v) {
        double vx = v[i] + c_kick * fx, vy = v[Np + i] + c_kick * fy, vz = v[2 * Np + i] + c_kick * fz;
        bath_half(bath, vx, vy, vz);  // friction half step after the kick
        v[i] = vx;
        v[Np + i] = vy;
        v[2 * Np + i] = vz;
    }
}

CellSep single_cell_sep(const Engine& e) {
    CellSep cs{};
    if (e.B != 1) return cs;
    cs.lx = (float)(e.L_h[0] / e.nc_h[0]);
    cs.ly = (float)(e.L_h[1] / e.nc_h[1]);
    cs.lz = (float)(e.L_h[2] / e.nc_h[2]);
    cs.nx = e.nc_h[0];
    cs.ny = e.nc_h[1];
    cs.nz = e.nc_h[2];
    cs.Lx = (float)e.L_h[0];
    cs.Ly = (float)e.L_h[1];
    cs.Lz = (float)e.L_h[2];
    return cs;
}

template <int KIND, bool SINGLE, bool WIDE, bool TAPER>
static void run_mixed(Engine& e, int kick, cudaStream_t s, bool virial) {
    Geo g = make_geo(e);
    const CellSep cs = single_cell_sep(e);
    int nb = (int)((e.N + kMNT - 1) / kMNT);
    double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    e.launches += 2;
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        k_density_mixed<KIND, SINGLE, WIDE, TAPER><<<nb, kMNT, 0, s>>>(e.N, e.N_pad, g, cs, e.pot, e.xo, e.nn, e.nl,
                                                                    e.max_nb, e.rho, e.Fp, e.xf, e.e_atom, e.ctl);
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    double* vk = kick ? e.v : nullptr;
    if (virial)
        k_force_mixed<KIND, SINGLE, WIDE, TAPER, true><<<nb, kMNT, 0, s>>>(
            e.N, e.N_pad, g, cs, e.pot, e.xo, e.nn, e.nl, e.max_nb, e.xf, e.f, e.e_atom, vk, c_kick, e.bath,
            e.w_atom, e.ctl);
    else
        k_force_mixed<KIND, SINGLE, WIDE, TAPER, false><<<nb, kMNT, 0, s>>>(
            e.N, e.N_pad, g, cs, e.pot, e.xo, e.nn, e.nl, e.max_nb, e.xf, e.f, e.e_atom, vk, c_kick, e.bath,
            nullptr, e.ctl);
}

template <int KIND, bool TAPER>
static void run_mixed_k(Engine& e, int kick, cudaStream_t s, bool virial) {
    if (single_fast(e))
        e.wide ? run_mixed<KIND, true, true, TAPER>(e, kick, s, virial)
               : run_mixed<KIND, true, false, TAPER>(e, kick, s, virial);
    else
        e.wide ? run_mixed<KIND, false, true, TAPER>(e, kick, s, virial)
               : run_mixed<KIND, false, false, TAPER>(e, kick, s, virial);
}

void launch_forces_mixed(Engine& e, int kick, cudaStream_t s, bool virial) {
    switch (e.pot.kind) {
        case MD_POT_RGL:
            // the packed RGL loops take the taper's clamp as the cutoff test
            if (e.pot.f_inv_w > 0.0f)
                run_mixed_k<MD_POT_RGL, true>(e, kick, s, virial);
            else
                run_mixed_k<MD_POT_RGL, false>(e, kick, s, virial);
            break;
        case MD_POT_SC: run_mixed_k<MD_POT_SC, false>(e, kick, s, virial); break;
        default: run_mixed_k<MD_POT_SPLINE, false>(e, kick, s, virial); break;
    }
}

}  // namespace mdk
