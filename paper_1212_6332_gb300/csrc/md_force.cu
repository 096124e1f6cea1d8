// Density pass (Sec. 3.3, Fig. 5) and force pass (Fig. 6, Eq. 3), float64.
//
// The force pass walks the full neighbour list of each atom (both i->j and
// j->i are stored), so every atom's force sum is private to one thread and
// no atomic update is needed (the paper does the same on the GPU; its CPU
// code uses Newton's third law instead, Sec. 4.3). The list is column-major, so a warp
// of 32 consecutive atoms loads one 128-byte row of indices per neighbour
// slot; neighbour positions are gathered from the Morton-sorted array,
// mostly from L1/L2.
//
// GB300 executes float64 at 1/64 of the float32 rate while its HBM sits
// idle in this kernel pair, so the work is split to evaluate every pair's
// functions once per step and to move bytes instead of float64 instructions:
//   pairs:   the lower slot of each pair (j > i in i's list) evaluates V,
//            rho, A = V'/r and B = rho'/r (one rsqrt; RGL: both
//            exponentials from one reduction over an r table; splines: one
//            interval record) and writes them as one 32-byte entry into
//            both lists' slots (the partner's slot comes from the reverse
//            index built with the list); all four are functions of r
//            alone, so both slots get the same bits the partner would have
//            computed; the same pass adds rho(r) and V(r) to both atoms'
//            64-bit fixed-point totals by atomic integer adds (exact and
//            order-free, so every run gives the same bits: see sum_fixed);
//   density: rho_i and 1/2 sum V from those totals; F(rho_i), F'(rho_i)
//            (the pass no longer reads the cache entries);
//   force:   F_i = sum_j s_ij x_j - x_i sum_j s_ij with
//            s_ij = A + (F'_i + F'_j) B   [Eq. (3) regrouped]
//            i.e. 6 float64 operations per entry and no separation,
//            optionally followed by v_i += dt/2 F_i/m (second half-kick).
// The force sums run over each list in list order, as a full evaluation per
// atom does (the block-per-box schedule evaluates every entry from its own
// side), and the density totals are integer sums of the same terms, so both
// give identical results.
#include "md_device.cuh"

namespace mdk {

constexpr int kFNT = 128;

// Pair pass. Each warp owns groups of 32 consecutive atoms in turn
// (persistent warps, so queue tails are paid once per warp, not once per
// group). Lanes walk their own lists (coalesced rows) and screen every upper
// entry with a float32 r^2 from the cell-local offsets: an entry whose
// float32 r^2 lies above rc^2 (1 + 1e-4) is outside r_cut in any image (the
// float32 error of r^2 is below 1e-4 A^2, the margin 25 times more for
// rc = 5 A) and gets zeros. For the rest the lane forms the exact float64
// separation (x_j is loaded beside its offset, so this adds no latency) and
// queues it in shared memory, in one of two per-warp queues split at
// r_taper so that a batch takes one branch of pair_eval. Every batch of 32
// takes r^2, the exact test r^2 < rc^2 (which alone decides, as in the list
// build) and the pair functions with all 32 lanes active: on GB300 a masked
// lane still costs the float64 pipe its cycles. The exponential table is
// read through L1 (one 16 KB copy per multiprocessor instead of one per
// block in shared memory, which leaves L1 room for the list streams).
constexpr int kQueue = 64;
constexpr double kScreen = 1e-4;  // relative r^2 margin of the float32 screen

// ST: the type of a list-slot index, 32-bit when every slot of the list
// array fits (less queue traffic in shared memory), 64-bit otherwise.
template <typename ST>
struct PairQueue {
    double r2[2][kQueue];    // exact r^2 of the pair, per region
    ST own[2][kQueue];       // slot of the entry in i's list
    ST mir[2][kQueue];       // slot of the mirror entry in j's list
    int pt[2][kQueue];       // type-pair table (several species)
    int ai[2][kQueue];       // the pair's atoms (the fixed-point density sums)
    int aj[2][kQueue];
};

// The fixed-point sums of a pair (DENS): rho(r) and V(r) added to both
// atoms' totals by atomic integer adds (the high words only when a term
// needs them).
struct SumOut {
    long long* sq;  // [kSumWords N_pad] fixed-point totals, zeroed before the pass
    int64_t Np;
    int S;          // sum_split(list capacity)
    bool with_v;    // also the pair-energy totals (Engine::pair_energy)
    Ctl* ctl;
};

__device__ __forceinline__ void red_pair(unsigned long long* w, int i, int j, long long v) {
    if (v) {
        atomicAdd(w + i, (unsigned long long)v);
        atomicAdd(w + j, (unsigned long long)v);
    }
}

__device__ __forceinline__ void add_pair_sums(const SumOut& so, int i, int j, double fr, double V) {
    long long hr, lr, hv = 0, lv = 0;
    const bool ok = split_fixed(fr, so.S, hr, lr) & (!so.with_v || split_fixed(V, so.S, hv, lv));
    if (!ok) {
        atomicOr(&so.ctl->status, kStNonFinite);
        return;
    }
    unsigned long long* u = reinterpret_cast<unsigned long long*>(so.sq);
    red_pair(u, i, j, lr);
    if (so.with_v) red_pair(u + so.Np, i, j, lv);
    if (hr | hv) {
        red_pair(u + 2 * so.Np, i, j, hr);
        red_pair(u + 3 * so.Np, i, j, hv);
    }
}

template <int KIND, bool MIRROR, bool DENS, typename ST>
__device__ __forceinline__ void eval_queued(const Pot& P, const PairQueue<ST>& q, int r, int p,
                                            double4_32a* __restrict__ pc, const SumOut& so) {
    const double r2 = q.r2[r][p];
    double A = 0.0, B = 0.0, V = 0.0, fr = 0.0;
    const int pt = KIND == MD_POT_SPLINE ? q.pt[r][p] : 0;
    if (below(r2, P.rc2)) {
        pair_eval<KIND>(P, P.exp_T, r2, V, fr, A, B, pt);
        if (DENS) add_pair_sums(so, q.ai[r][p], q.aj[r][p], fr, V);
    }
    const double4_32a c = make_double4_32a(A, B, fr, V);
    pc[(int64_t)q.own[r][p]] = c;
    if (MIRROR) pc[(int64_t)q.mir[r][p]] = c;
}

// The positions in fixed point (x 2^kq, kq of the atom's box) with the
// species label, gathered by the pair pass for its exact r^2: one
// conversion per atom and step instead of one per list entry.
// With sq, also clears the fixed-point sums that the pair pass adds into.
template <bool SINGLE>
__global__ void __launch_bounds__(kFNT) k_fixed_positions(int64_t N, int64_t Np, Geo g,
                                                          const double4_32a* __restrict__ x,
                                                          longlong4_32a* __restrict__ xq, long long* __restrict__ sq,
                                                          const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (sq) {
#pragma unroll
        for (int w = 0; w < kSumWords; ++w) sq[w * Np + i] = 0;
    }
    const int b = SINGLE ? 0 : g.atom_box[i];
    const int kq = SINGLE ? box_kq(g.L0[0], g.L0[1], g.L0[2]) : box_kq(g.L[3 * b], g.L[3 * b + 1], g.L[3 * b + 2]);
    xq[i] = fixed_pos(x[i], kq);
}

// One list row of a lane: the entry and, for an upper entry (j > i), the
// partner's offset and fixed-point position and the row of the mirror entry.
struct PairRow {
    float4 oj;
    longlong4_32a qj;
    int e, rv;
    bool upper;
};

template <bool MIRROR>
__device__ __forceinline__ PairRow load_pair_row(int e, bool valid, int64_t i, const float4* __restrict__ xo,
                                                 const longlong4_32a* __restrict__ xq, const int* __restrict__ rev,
                                                 int64_t Np, int k) {
    PairRow r;
    r.e = e;
    r.upper = valid && entry_slot(e) > i;
    r.oj = make_float4(0.f, 0.f, 0.f, 0.f);
    r.qj = longlong4_32a{0, 0, 0, 0};
    r.rv = 0;
    if (r.upper) {
        const int j = entry_slot(e);
        r.oj = xo[j];
        r.qj = xq[j];
        if (MIRROR) r.rv = rev[(int64_t)k * Np + i];
    }
    return r;
}

// MIRROR = false (Newton's third law variant): only the upper slot of each
// pair is written; the lower slots are never read.
// (a minimum of 6 or 8 resident blocks, 80 or 64 registers, measured
// slower: 4M-atom pair pass 3.41 -> 3.45 / 3.82 ms)
#ifdef MD_PAIR_MIN_BLOCKS
#define MD_PAIR_BOUNDS __launch_bounds__(kFNT, MD_PAIR_MIN_BLOCKS)
#else
// 5 resident blocks: the single-box pass fits them unbounded (92
// registers); boxes of a batch (per-atom box geometry) would take 110
// registers and 4 blocks. (An explicit minimum of one block lets the
// compiler take 172 registers: 0.99 -> 1.64 ms per 1M atoms.)
#define MD_PAIR_BOUNDS __launch_bounds__(kFNT, 5)
#endif
template <int KIND, bool SINGLE, bool MIRROR, bool DENS, typename ST>
__global__ void MD_PAIR_BOUNDS k_pairs_half(int64_t N, int64_t Np, Geo g, CellSep cs0, Pot P, float rc2f,
                                                     float rs2f, const longlong4_32a* __restrict__ xq,
                                                     const float4* __restrict__ xo, const int* __restrict__ nn,
                                                     const int* __restrict__ nl, const int* __restrict__ rev,
                                                     const int* __restrict__ n_up, int max_nb,
                                                     double4_32a* __restrict__ pc, SumOut so, const Ctl* ctl) {
    if (load_status(ctl)) return;
    __shared__ PairQueue<ST> queues[kFNT / 32];
    const int lane = threadIdx.x & 31;
    PairQueue<ST>& q = queues[threadIdx.x >> 5];
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n_groups = (N + 31) >> 5, stride = (int64_t)gridDim.x * (kFNT / 32);
    int qn[2] = {0, 0};
    for (int64_t grp = (int64_t)blockIdx.x * (kFNT / 32) + (threadIdx.x >> 5); grp < n_groups; grp += stride) {
        const int64_t i = grp * 32 + lane;
        CellSep cs = cs0;
        float4 oi = make_float4(0.f, 0.f, 0.f, 0.f);
        int ti = 0;
        long long qi[3] = {0, 0, 0}, qL[3] = {0, 0, 0};
        int kq = 0;
        int kend = 0;
        if (i < N) {
            cs = cell_sep<SINGLE>(g, cs0, i);
            const int b = SINGLE ? 0 : g.atom_box[i];
            double L[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
            kq = box_kq(L[0], L[1], L[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) qL[a] = to_fixed(L[a], kq);
            oi = xo[i];
            const longlong4_32a q = xq[i];
            qi[0] = q.x;
            qi[1] = q.y;
            qi[2] = q.z;
            ti = (int)q.w;
            // lists are [upper | lower]: the upper entries (j > i) are rows
            // 0..n_up-1; the lower ones are written by the partners' lanes (a
            // list kept unrotated, n_up < 0, is scanned whole)
            const int nup = n_up[i];
            kend = nup < 0 ? min(nn[i], max_nb) : nup;
        }
        const int kmax = warp_max(kend);
        // software pipeline: the list entry two rows ahead and the partner
        // data (offset, position, mirror row) one row ahead are in flight
        // while a row is screened, so the loop does not wait on L2 / HBM
        PairRow cur = load_pair_row<MIRROR>(0 < kend ? nl[i] : 0, 0 < kend, i, xo, xq, rev, Np, 0);
        int e_ahead = 1 < kend ? nl[Np + i] : 0;
        for (int k = 0; k < kmax; ++k) {
            const PairRow nxt = load_pair_row<MIRROR>(e_ahead, k + 1 < kend, i, xo, xq, rev, Np, k + 1);
            e_ahead = k + 2 < kend ? nl[(int64_t)(k + 2) * Np + i] : 0;
            bool in = false, tq = false;
            double r2 = 0.0;
            const ST own = (ST)((long long)k * Np + i);
            const int j_cur = entry_slot(cur.e);
            const ST mir = (ST)((long long)cur.rv * Np + j_cur);
            const int pt = KIND == MD_POT_SPLINE && P.n_types > 1
                               ? pair_table(P.n_types, ti, (int)cur.qj.w)
                               : 0;
            if (cur.upper) {
                float fx, fy, fz;
                sep_mixed<false>(cs, oi, cur.oj, fx, fy, fz);
                const float r2f = fmaf(fz, fz, fmaf(fy, fy, fx * fx));
                if (r2f < rc2f) {
                    in = true;
                    tq = r2f > rs2f;
                    r2 = r2_exact(qi, cur.qj.x, cur.qj.y, cur.qj.z, entry_code(cur.e), qL, kq);
                } else {
                    const double4_32a z = make_double4_32a(0.0, 0.0, 0.0, 0.0);
                    pc[own] = z;
                    if (MIRROR) pc[mir] = z;
                }
            }
            cur = nxt;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const bool mine = in && (tq == (r == 1));
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (mine) {
                    const int p = qn[r] + __popc(m & lt_mask);
                    q.r2[r][p] = r2;
                    q.own[r][p] = own;
                    q.mir[r][p] = mir;
                    if (KIND == MD_POT_SPLINE) q.pt[r][p] = pt;
                    if (DENS) {
                        q.ai[r][p] = (int)i;
                        q.aj[r][p] = j_cur;
                    }
                }
                qn[r] += __popc(m);
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (qn[r] >= 32) {
                    qn[r] -= 32;
                    eval_queued<KIND, MIRROR, DENS, ST>(P, q, r, qn[r] + lane, pc, so);
                    __syncwarp();
                }
            }
        }
    }
    // tails: one batch when both fit (lanes of the two regions diverge in
    // pair_eval, which still costs less than two part-empty batches)
    if (qn[0] + qn[1] <= 32) {
        if (lane < qn[0])
            eval_queued<KIND, MIRROR, DENS, ST>(P, q, 0, lane, pc, so);
        else if (lane < qn[0] + qn[1])
            eval_queued<KIND, MIRROR, DENS, ST>(P, q, 1, lane - qn[0], pc, so);
    } else {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (lane < qn[r]) eval_queued<KIND, MIRROR, DENS, ST>(P, q, r, lane, pc, so);
    }
}

// Both sums below skip the list entries that the pair pass zeroed (outside
// r_cut). Each lane steps to its own next non-zero entry, so the float64
// instructions of an iteration run with nearly all lanes active (in list-row
// lockstep about a fifth of the lanes would idle on zero entries), and the
// next entry's cache value is loaded one iteration ahead. Adding an exact
// zero never changes a sum that starts at +0, so the sums are bit-identical
// to adding every entry in list order.
__device__ __forceinline__ bool is_zero2(double2 c) {
    return (__double_as_longlong(c.x) | __double_as_longlong(c.y)) == 0;
}

// rho_i and the pair energy from the fixed-point totals the pair pass added
// (see split_fixed), then F(rho_i), F'(rho_i) and E_i = F(rho_i) + 1/2 sum V
// (with_v false: the pair pass formed no pair-energy totals, E_i = F(rho_i)
// until a later evaluation forms them).
template <int KIND>
__global__ void __launch_bounds__(kFNT) k_embed_sums(int64_t N, int64_t Np, Pot P, const long long* __restrict__ sq,
                                                     int S, bool with_v, const int* __restrict__ nn, int max_nb,
                                                     const double4_32a* __restrict__ pc,
                                                     const double4_32a* __restrict__ x,
                                                     double* __restrict__ rho, double* __restrict__ Fp,
                                                     double* __restrict__ e_atom, const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    FixedSum qr, qv;
    load_sums(sq, Np, i, qr, qv);
    if (!with_v) qv = FixedSum{};
    double r_i, Fpi, E;
    embed_sums<KIND>(P, qr, qv, S, KIND == MD_POT_SPLINE && P.n_types > 1 ? pos_type(x[i]) : 0, pc, Np, i,
                     min(nn[i], max_nb), r_i, Fpi, E);
    rho[i] = r_i;
    Fp[i] = Fpi;
    e_atom[i] = E;
}

// VIR: also the per-atom virial w_i = -1/2 sum_j s_ij r_ij^2 (the pair
// virial of Eq. (6) split evenly between the two atoms of each pair), r_ij^2
// exact from the fixed-point difference as in the pair pass.
// Resident blocks: 10 for one box (48 registers; with 12, 40 registers, the
// walk below spills: 1.368 against 1.431 ms per 4M-atom step), 8 for
// batches, whose box constants are per thread (64 registers; with 10 they
// spill: 4096-box force phase 2.434 against 2.603 ms).
template <bool SINGLE, bool VIR>
__global__ void __launch_bounds__(kFNT, SINGLE ? 10 : 8) k_force(int64_t N, int64_t Np, Geo g, const longlong4_32a* __restrict__ xq,
                                                const int* __restrict__ nn, const int* __restrict__ nl, int max_nb,
                                                const double4_32a* __restrict__ pc, const double* __restrict__ Fp,
                                                double* __restrict__ f, double* __restrict__ v, double c_kick,
                                                Bath bath, double* __restrict__ w_atom, int cb, const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < N;
    // the box's constants (for one box, the same in every thread)
    const int b = SINGLE || !active ? 0 : g.atom_box[i];
    double L[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
    const int kq = box_kq(L[0], L[1], L[2]);
    const DSplit D = dsplit_init(kq, cb);
    long long qL[3], qi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) qL[a] = to_fixed(L[a], kq);
    double Fpi = 0.0;
    int n = 0;
    if (active) {
        const longlong4_32a q = xq[i];
        // x_i less the pre-shift's rounding constant: x_j - that = d + rnd
        qi[0] = q.x - D.rnd;
        qi[1] = q.y - D.rnd;
        qi[2] = q.z - D.rnd;
        Fpi = Fp[i];
        n = min(nn[i], max_nb);
    }
    const double2 zero = make_double2(0.0, 0.0);
    // f_i = sum_j s_ij (x_j - x_i) (Eq. 3 with the separation exact in
    // fixed point, the entry's image added as an integer): per entry F'_i +
    // F'_j and s in float64, the rest in float32 pieces (ForceSumF)
    // Every entry in turn, the next entry's cache value and list entry
    // loaded one ahead; the entries beyond r_cut (zero cache values, about a
    // fifth) skip the arithmetic. Stepping each lane to its next non-zero
    // entry instead kept the float64 work of the earlier sums converged, at
    // one dependent load per skipped entry: force phase 2.016 -> 1.368 ms
    // per 4M-atom step with this walk.
    ForceSumF fs;
    double w = 0.0;
    double2 c = n > 0 ? cache_ab(pc, i) : zero;
    int e = n > 0 ? nl[i] : 0;
    const int kmax = warp_max(n);
    for (int k = 0; k < kmax; ++k) {
        const int64_t slot = (int64_t)k * Np + i;
        const bool more = k + 1 < n;
        const double2 cn = more ? cache_ab(pc, slot + Np) : zero;
        const int en = more ? nl[slot + Np] : 0;
        if (k < n && !is_zero2(c)) {
            const int j = entry_slot(e);
            const unsigned code = entry_code(e);
            const double s = fma(Fpi + Fp[j], c.y, c.x);
            const longlong4_32a qj = xq[j];
            long long rx = qj.x - qi[0], ry = qj.y - qi[1], rz = qj.z - qi[2];
            if (code != kNoShift) {
                rx += qshift(code, 0, qL[0]);
                ry += qshift(code, 1, qL[1]);
                rz += qshift(code, 2, qL[2]);
            }
            fs.add(s, rx, ry, rz, D);
            if (VIR) w = fma(s, r2_fixed(rx - D.rnd, ry - D.rnd, rz - D.rnd, 2 * kq), w);
        }
        c = cn;
        e = en;
    }
    if (!active) return;
    const double fx = fs.value(0), fy = fs.value(1), fz = fs.value(2);
    f[i] = fx;
    f[Np + i] = fy;
    f[2 * Np + i] = fz;
    if (VIR) w_atom[i] = -0.5 * w;
    if (v) {
        double vx = v[i] + c_kick * fx, vy = v[Np + i] + c_kick * fy, vz = v[2 * Np + i] + c_kick * fz;
        bath_half(bath, vx, vy, vz);  // friction half step after the kick
        v[i] = vx;
        v[Np + i] = vy;
        v[2 * Np + i] = vz;
    }
}

// ---------------------------------------------------------------- small systems
//
// For a few thousand atoms the passes above are latency-bound: the pair
// pass gives each warp 32 atoms of float64 work on one scheduler, and each
// thread of the two sums walks its list with one load in flight. The
// variants below do the same arithmetic with more parallelism:
//   k_pairs_flat: one thread per atom and upper list row (32 row slots per
//     atom, each looping over rows 32 apart), the screen and the pair
//     functions of k_pairs_half with the same operands (the bits of a pair
//     depend on r alone, not on the lane that evaluates it); it beats the
//     queued pass up to about 20,000 atoms (measured), the sums up to
//     32,768 at least;
//   k_rho_small / k_force_small: 128 threads per 32 atoms stage a chunk of
//     32 list rows of their atoms in shared memory (all loads in flight, and
//     for the force pass s_ij and the partner's image position formed at the
//     same time), then one lane per atom adds them: the density terms in
//     the fixed point of k_pairs_half's atomic adds (exact integer sums),
//     the force terms in list order with the operations of k_force. The
//     results are therefore bit-identical to the passes above.
#ifndef MD_SMALL_ATOMS
#define MD_SMALL_ATOMS 32768
#endif
#ifndef MD_SMALL_PAIR_ATOMS
#define MD_SMALL_PAIR_ATOMS 16384
#endif
constexpr int kSmallAtoms = MD_SMALL_ATOMS;            // largest system whose sums take these kernels
constexpr int kSmallPairAtoms = MD_SMALL_PAIR_ATOMS;   // ... whose pair pass takes k_pairs_flat
constexpr int kSmallRows = 32;  // list rows staged per chunk; row slots per atom in k_pairs_flat

// One upper list row k of atom i: the screen and, inside it, the pair
// functions, written to the entry's slot and its mirror.
template <int KIND, bool SINGLE, bool MIRROR>
__device__ __forceinline__ void pair_flat_row(int64_t i, int64_t k, int64_t Np, const Geo& g, const CellSep& cs0,
                                              const Pot& P, float rc2f, const double4_32a* __restrict__ x,
                                              const float4* __restrict__ xo, const int* __restrict__ nl,
                                              const int* __restrict__ rev, double4_32a* __restrict__ pc) {
    const int64_t own = k * Np + i;
    const int e = nl[own];
    const int j = entry_slot(e);
    if (j <= i) return;  // lower entries of an unrotated list
    const CellSep cs = cell_sep<SINGLE>(g, cs0, i);
    const int b = SINGLE ? 0 : g.atom_box[i];
    const float4 oi = xo[i], oj = xo[j];
    const long long mir = MIRROR ? (long long)rev[own] * Np + j : 0;
    float fx, fy, fz;
    sep_mixed<false>(cs, oi, oj, fx, fy, fz);
    const float r2f = fmaf(fz, fz, fmaf(fy, fy, fx * fx));
    double A = 0.0, B = 0.0, V = 0.0, fr = 0.0;
    if (r2f < rc2f) {
        const double4_32a xi = x[i], xj = x[j];
        double L[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
        const int kq = box_kq(L[0], L[1], L[2]);
        long long qi[3], qL[3];
        qi[0] = to_fixed(xi.x, kq);
        qi[1] = to_fixed(xi.y, kq);
        qi[2] = to_fixed(xi.z, kq);
#pragma unroll
        for (int a = 0; a < 3; ++a) qL[a] = to_fixed(L[a], kq);
        const double r2 = r2_exact(qi, xj, entry_code(e), qL, kq);
        const int pt = KIND == MD_POT_SPLINE && P.n_types > 1 ? pair_table(P.n_types, pos_type(xi), pos_type(xj)) : 0;
        if (below(r2, P.rc2)) pair_eval<KIND>(P, P.exp_T, r2, V, fr, A, B, pt);
    }
    const double4_32a c = make_double4_32a(A, B, fr, V);
    pc[own] = c;
    if (MIRROR) pc[mir] = c;
}

template <int KIND, bool SINGLE, bool MIRROR>
__global__ void __launch_bounds__(kFNT) k_pairs_flat(int64_t N, int64_t Np, Geo g, CellSep cs0, Pot P, float rc2f,
                                                     const double4_32a* __restrict__ x, const float4* __restrict__ xo,
                                                     const int* __restrict__ nn, const int* __restrict__ nl,
                                                     const int* __restrict__ rev, const int* __restrict__ n_up,
                                                     int max_nb, double4_32a* __restrict__ pc, const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t % N;
    const int64_t k0 = t / N;
    if (k0 >= kSmallRows) return;
    const int nup = n_up[i];
    const int kend = nup < 0 ? min(nn[i], max_nb) : nup;
    for (int64_t k = k0; k < kend; k += kSmallRows) pair_flat_row<KIND, SINGLE, MIRROR>(i, k, Np, g, cs0, P, rc2f, x, xo, nl, rev, pc);
}

template <int KIND>
__global__ void __launch_bounds__(kFNT) k_rho_small(int64_t N, int64_t Np, Pot P, const int* __restrict__ nn,
                                                    int max_nb, const double4_32a* __restrict__ pc,
                                                    const double4_32a* __restrict__ x, double* __restrict__ rho,
                                                    double* __restrict__ Fp, double* __restrict__ e_atom, int S,
                                                    Ctl* ctl) {
    if (load_status(ctl)) return;
    // each warp adds the fixed-point terms of its rows (every fourth row of
    // the 32 atoms' lists, all loads in flight), the warps' partial totals
    // then meet in shared memory: integer sums, so the bits of the pair
    // pass's atomic adds in any split
    __shared__ long long part[kFNT / 32][4][32];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    const bool active = i < N;
    const int n = active ? min(nn[i], max_nb) : 0;
    FixedSum qr, qv;
    bool ok = true;
    for (int k = wq; k < n; k += kFNT / 32) {
        const double2 w = cache_fv(pc, (int64_t)k * Np + i);
        ok &= qr.add(w.x, S) & qv.add(w.y, S);
    }
    part[wq][0][lane] = qr.lo;
    part[wq][1][lane] = qr.hi;
    part[wq][2][lane] = qv.lo;
    part[wq][3][lane] = qv.hi;
    if (!ok) atomicOr(&ctl->status, kStNonFinite);
    __syncthreads();
    if (wq != 0 || !active) return;
#pragma unroll
    for (int w = 1; w < kFNT / 32; ++w) {
        qr.lo += part[w][0][lane];
        qr.hi += part[w][1][lane];
        qv.lo += part[w][2][lane];
        qv.hi += part[w][3][lane];
    }
    double r_i, Fpi, E;
    embed_sums<KIND>(P, qr, qv, S, KIND == MD_POT_SPLINE && P.n_types > 1 ? pos_type(x[i]) : 0, pc, Np, i, n, r_i,
                     Fpi, E);
    rho[i] = r_i;
    Fp[i] = Fpi;
    e_atom[i] = E;
}

template <bool SINGLE, bool VIR>
__global__ void __launch_bounds__(kFNT) k_force_small(int64_t N, int64_t Np, Geo g, const double4_32a* __restrict__ x,
                                                      const int* __restrict__ nn, const int* __restrict__ nl,
                                                      int max_nb, const double4_32a* __restrict__ pc,
                                                      const double* __restrict__ Fp, double* __restrict__ f,
                                                      double* __restrict__ v, double c_kick, Bath bath,
                                                      double* __restrict__ w_atom, int cb, const Ctl* ctl) {
    if (load_status(ctl)) return;
    // the float32 pieces of each term: (s_h, s_l, d_h x, d_h y), (d_h z, d_l x, d_l y, d_l z)
    __shared__ float4 sp[kSmallRows][2][32];
    __shared__ double2 sw[VIR ? kSmallRows : 1][32];  // (s_ij, r_ij^2)
    __shared__ unsigned char sok[kSmallRows][32];     // 1: a term
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * 32 + lane;
    const bool active = i < N;
    const int b = SINGLE || !active ? 0 : g.atom_box[i];
    double L[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
    const int kq = box_kq(L[0], L[1], L[2]);
    const DSplit D = dsplit_init(kq, cb);
    long long qL[3], qi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) qL[a] = to_fixed(L[a], kq);
    double Fpi = 0.0;
    int n = 0;
    if (active) {
        const double4_32a xi = x[i];
        // the fixed point of k_fixed_positions, less the rounding constant
        qi[0] = to_fixed(xi.x, kq) - D.rnd;
        qi[1] = to_fixed(xi.y, kq) - D.rnd;
        qi[2] = to_fixed(xi.z, kq) - D.rnd;
        Fpi = Fp[i];
        n = min(nn[i], max_nb);
    }
    const int kmax = warp_max(n);
    ForceSumF fs;
    double w = 0.0;
    for (int k0 = 0; k0 < kmax; k0 += kSmallRows) {
#pragma unroll 4
        for (int r = wq; r < kSmallRows; r += kFNT / 32) {
            const int k = k0 + r;
            unsigned char ok = 0;
            if (k < n) {
                const int64_t slot = (int64_t)k * Np + i;
                const double2 c = cache_ab(pc, slot);
                if (!is_zero2(c)) {
                    const int e = nl[slot];
                    const int j = entry_slot(e);
                    const double4_32a xj = x[j];
                    const double sij = fma(Fpi + Fp[j], c.y, c.x);
                    const unsigned code = entry_code(e);
                    long long rx = to_fixed(xj.x, kq) - qi[0], ry = to_fixed(xj.y, kq) - qi[1],
                              rz = to_fixed(xj.z, kq) - qi[2];
                    if (code != kNoShift) {
                        rx += qshift(code, 0, qL[0]);
                        ry += qshift(code, 1, qL[1]);
                        rz += qshift(code, 2, qL[2]);
                    }
                    float sh, sl, dh[3], dl[3];
                    ssplit(sij, sh, sl);
                    dsplit(rx, D, dh[0], dl[0]);
                    dsplit(ry, D, dh[1], dl[1]);
                    dsplit(rz, D, dh[2], dl[2]);
                    sp[r][0][lane] = make_float4(sh, sl, dh[0], dh[1]);
                    sp[r][1][lane] = make_float4(dh[2], dl[0], dl[1], dl[2]);
                    if (VIR) sw[r][lane] = make_double2(sij, r2_fixed(rx - D.rnd, ry - D.rnd, rz - D.rnd, 2 * kq));
                    ok = 1;
                }
            }
            sok[r][lane] = ok;
        }
        __syncthreads();
        if (wq == 0) {
            // the operations and order of k_force
            const int kend = min(n - k0, kSmallRows);
            for (int r = 0; r < kend; ++r) {
                if (!sok[r][lane]) continue;
                const float4 p0 = sp[r][0][lane], p1 = sp[r][1][lane];
                fs.add(p0.x, p0.y, {p0.z, p0.w, p1.x}, {p1.y, p1.z, p1.w});
                if (VIR) {
                    const double2 q = sw[r][lane];
                    w = fma(q.x, q.y, w);
                }
            }
        }
        __syncthreads();
    }
    if (wq != 0 || !active) return;
    const double fx = fs.value(0), fy = fs.value(1), fz = fs.value(2);
    f[i] = fx;
    f[Np + i] = fy;
    f[2 * Np + i] = fz;
    if (VIR) w_atom[i] = -0.5 * w;
    if (v) {
        double vx = v[i] + c_kick * fx, vy = v[Np + i] + c_kick * fy, vz = v[2 * Np + i] + c_kick * fz;
        bath_half(bath, vx, vy, vz);  // friction half step after the kick
        v[i] = vx;
        v[Np + i] = vy;
        v[2 * Np + i] = vz;
    }
}

// ---------------------------------------------------------------- Newton's third law
//
// Float64 variant in the style of the paper's CPU code (Sec. 4.3): the pair
// pass writes only the upper slot of each pair, and the density and force
// passes walk only the upper entries of each list, adding every pair's term
// to both atoms, to the partner by an atomic add (rho_j and V_ij into the
// fixed-point totals, -s_ij d_ij into the float64 force). That halves the
// cache bytes and the float64 work of both sums at the price of one atomic
// per pair and component. The density totals are exact integer sums, the
// same bits as the full-list path (but for densities below kSumSmall, which
// the full-list path takes in float64 from its lower slots, that this
// variant does not write); the order in which the float64 force
// atomics land varies, so the last bits of F vary from run to run (the
// full-list passes are reproducible). The totals and f are zeroed before
// their passes.

// Upper entries of a list: rows 0..n_up-1 of a rotated list, else (a list
// kept ascending) the entries with j > i among all rows.
__device__ __forceinline__ int upper_rows(const int* __restrict__ nn, const int* __restrict__ n_up, int max_nb,
                                          int64_t i) {
    const int nup = n_up[i];
    return nup < 0 ? min(nn[i], max_nb) : nup;
}

__global__ void __launch_bounds__(kFNT) k_rho_n3(int64_t N, int64_t Np, const int* __restrict__ nn,
                                                 const int* __restrict__ nl, const int* __restrict__ n_up, int max_nb,
                                                 const double4_32a* __restrict__ pc, long long* __restrict__ sq,
                                                 int S, Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = upper_rows(nn, n_up, max_nb, i);
    unsigned long long* u = reinterpret_cast<unsigned long long*>(sq);
    FixedSum qr, qv;
    bool ok = true;
    for (int k = 0; k < n; ++k) {
        const int64_t slot = (int64_t)k * Np + i;
        const double2 w = cache_fv(pc, slot);
        if (is_zero2(w)) continue;
        const int j = entry_slot(nl[slot]);
        if (j <= i) continue;
        long long hr, lr, hv, lv;
        ok &= split_fixed(w.x, S, hr, lr) & split_fixed(w.y, S, hv, lv);
        qr.lo += lr;
        qr.hi += hr;
        qv.lo += lv;
        qv.hi += hv;
        atomicAdd(u + j, (unsigned long long)lr);
        atomicAdd(u + Np + j, (unsigned long long)lv);
        if (hr | hv) {
            atomicAdd(u + 2 * Np + j, (unsigned long long)hr);
            atomicAdd(u + 3 * Np + j, (unsigned long long)hv);
        }
    }
    if (!ok) atomicOr(&ctl->status, kStNonFinite);
    atomicAdd(u + i, (unsigned long long)qr.lo);
    atomicAdd(u + Np + i, (unsigned long long)qv.lo);
    atomicAdd(u + 2 * Np + i, (unsigned long long)qr.hi);
    atomicAdd(u + 3 * Np + i, (unsigned long long)qv.hi);
}

// rho_i, F(rho_i), F'(rho_i) and E_i from the fixed-point totals
template <int KIND>
__global__ void __launch_bounds__(kFNT) k_embed_n3(int64_t N, int64_t Np, Pot P, const double4_32a* __restrict__ x,
                                                   const long long* __restrict__ sq, int S, double* __restrict__ rho,
                                                   double* __restrict__ Fp, double* __restrict__ e_atom,
                                                   const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    FixedSum qr, qv;
    load_sums(sq, Np, i, qr, qv);
    double r_i, Fpi, E;
    embed_sums<KIND>(P, qr, qv, S, KIND == MD_POT_SPLINE && P.n_types > 1 ? pos_type(x[i]) : 0, nullptr, Np, i, 0,
                     r_i, Fpi, E);
    rho[i] = r_i;
    Fp[i] = Fpi;
    e_atom[i] = E;
}

// VIR: w_atom[i] = -sum over i's upper pairs of s_ij r_ij^2 (each pair
// counted once, at its lower slot; the box sums are those of k_force).
template <bool SINGLE, bool VIR>
__global__ void __launch_bounds__(kFNT) k_force_n3(int64_t N, int64_t Np, Geo g, const double4_32a* __restrict__ x,
                                                   const int* __restrict__ nn, const int* __restrict__ nl,
                                                   const int* __restrict__ n_up, int max_nb,
                                                   const double4_32a* __restrict__ pc, const double* __restrict__ Fp,
                                                   double* __restrict__ f, double* __restrict__ w_atom,
                                                   const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double L[3];
    const int b = SINGLE ? 0 : g.atom_box[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) L[a] = SINGLE ? g.L0[a] : g.L[3 * b + a];
    const double4_32a xi = x[i];
    const double Fpi = Fp[i];
    const int n = upper_rows(nn, n_up, max_nb, i);
    double fx = 0.0, fy = 0.0, fz = 0.0, w = 0.0;
    for (int k = 0; k < n; ++k) {
        const int64_t slot = (int64_t)k * Np + i;
        const double2 c = cache_ab(pc, slot);
        if (is_zero2(c)) continue;
        const int e = nl[slot];
        const int j = entry_slot(e);
        if (j <= i) continue;
        double dx, dy, dz;
        sep_entry(xi, x[j], entry_code(e), L, dx, dy, dz);
        const double s = fma(Fpi + Fp[j], c.y, c.x);
        fx = fma(s, dx, fx);
        fy = fma(s, dy, fy);
        fz = fma(s, dz, fz);
        atomicAdd(&f[j], -s * dx);
        atomicAdd(&f[Np + j], -s * dy);
        atomicAdd(&f[2 * Np + j], -s * dz);
        if (VIR) w = fma(s, norm2(dx, dy, dz), w);
    }
    atomicAdd(&f[i], fx);
    atomicAdd(&f[Np + i], fy);
    atomicAdd(&f[2 * Np + i], fz);
    if (VIR) w_atom[i] = -w;
}

// second half-kick (and friction half step) once all force atomics landed
__global__ void __launch_bounds__(kFNT) k_kick_n3(int64_t N, int64_t Np, const double* __restrict__ f,
                                                  double* __restrict__ v, double c_kick, Bath bath, const Ctl* ctl) {
    if (load_status(ctl)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double vx = v[i] + c_kick * f[i], vy = v[Np + i] + c_kick * f[Np + i], vz = v[2 * Np + i] + c_kick * f[2 * Np + i];
    bath_half(bath, vx, vy, vz);
    v[i] = vx;
    v[Np + i] = vy;
    v[2 * Np + i] = vz;
}

void launch_forces_mixed(Engine& e, int kick, cudaStream_t s, bool virial);

// float32 screen threshold: rc^2 (1 + margin), rounded up
static float screen_r2f(double rc2) { return nextafterf((float)(rc2 * (1.0 + kScreen)), INFINITY); }

// persistent pair pass: all resident blocks of this instantiation on every
// SM, at most one 32-atom group per warp
template <int KIND, bool SINGLE, bool MIRROR, bool DENS, typename ST>
static int pair_blocks(const Engine& e) {
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pairs_half<KIND, SINGLE, MIRROR, DENS, ST>, kFNT, 0);
        per_sm = std::max(per_sm, 1);
    }
    const int64_t groups = (e.N + 31) / 32, per_block = kFNT / 32;
    return (int)std::max<int64_t>(1, std::min<int64_t>((groups + per_block - 1) / per_block, (int64_t)per_sm * e.n_sm));
}

// The queued pair pass with list-slot indices as narrow as the list array
// allows, after the fixed-point copy of the positions it gathers. DENS: the
// pass also adds rho(r) and V(r) of every pair into both atoms' fixed-point
// totals (cleared by the position copy), which k_embed_sums turns into rho_i.
template <int KIND, bool SINGLE, bool MIRROR, bool DENS>
static void launch_pairs_half(Engine& e, const Geo& g, cudaStream_t s) {
    e.launches += 1;
    k_fixed_positions<SINGLE><<<(int)((e.N + kFNT - 1) / kFNT), kFNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.xq,
                                                                             DENS ? e.sum_q : nullptr, e.ctl);
    const SumOut so{e.sum_q, e.N_pad, sum_split(e.max_nb), e.pair_energy, e.ctl};
    // 32-bit slots: 85 instead of 89 registers, 18 instead of 22.5 KB of
    // queues per block (4M-atom step 8.69 -> 8.63 ms; the same bits);
    // 6 blocks per SM forced (80 registers, spills) measured slower
    const bool narrow = (int64_t)e.N_pad * e.max_nb <= (int64_t)0xffffffffll;
    if (narrow)
        k_pairs_half<KIND, SINGLE, MIRROR, DENS, unsigned>
            <<<pair_blocks<KIND, SINGLE, MIRROR, DENS, unsigned>(e), kFNT, 0, s>>>(
                e.N, e.N_pad, g, single_cell_sep(e), e.pot, screen_r2f(e.pot.rc2), (float)e.pot.rs2, e.xq, e.xo,
                e.nn, e.nl, e.rev, e.n_up, e.max_nb, e.pc, so, e.ctl);
    else
        k_pairs_half<KIND, SINGLE, MIRROR, DENS, long long>
            <<<pair_blocks<KIND, SINGLE, MIRROR, DENS, long long>(e), kFNT, 0, s>>>(
                e.N, e.N_pad, g, single_cell_sep(e), e.pot, screen_r2f(e.pot.rc2), (float)e.pot.rs2, e.xq, e.xo,
                e.nn, e.nl, e.rev, e.n_up, e.max_nb, e.pc, so, e.ctl);
}

// The small-system kernels: same results, more parallelism (see above).
template <int KIND, bool SINGLE>
static void run_fp64_small(Engine& e, int kick, cudaStream_t s, bool virial) {
    Geo g = make_geo(e);
    const int nb32 = (int)((e.N + 31) / 32);
    const int64_t flat = e.N * (int64_t)kSmallRows;
    const double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    e.launches += 3;
    {
        PhaseScope scope(e, MD_PHASE_PAIRS, s);
        if (e.N <= kSmallPairAtoms)
            k_pairs_flat<KIND, SINGLE, true><<<(int)((flat + kFNT - 1) / kFNT), kFNT, 0, s>>>(
                e.N, e.N_pad, g, single_cell_sep(e), e.pot, screen_r2f(e.pot.rc2), e.x, e.xo, e.nn, e.nl, e.rev,
                e.n_up, e.max_nb, e.pc, e.ctl);
        else
            launch_pairs_half<KIND, SINGLE, true, false>(e, g, s);
    }
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        k_rho_small<KIND><<<nb32, kFNT, 0, s>>>(e.N, e.N_pad, e.pot, e.nn, e.max_nb, e.pc, e.x, e.rho, e.Fp,
                                                e.e_atom, sum_split(e.max_nb), e.ctl);
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    if (virial)
        k_force_small<SINGLE, true><<<nb32, kFNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.nn, e.nl, e.max_nb, e.pc, e.Fp,
                                                          e.f, kick ? e.v : nullptr, c_kick, e.bath, e.w_atom,
                                                          cut_bits(e.pot.rc), e.ctl);
    else
        k_force_small<SINGLE, false><<<nb32, kFNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.nn, e.nl, e.max_nb, e.pc, e.Fp,
                                                           e.f, kick ? e.v : nullptr, c_kick, e.bath, nullptr,
                                                           cut_bits(e.pot.rc), e.ctl);
}

template <int KIND, bool SINGLE>
static void run_fp64(Engine& e, int kick, cudaStream_t s, bool virial) {
    if (e.N <= kSmallAtoms) {
        run_fp64_small<KIND, SINGLE>(e, kick, s, virial);
        return;
    }
    Geo g = make_geo(e);
    int nb = (int)((e.N + kFNT - 1) / kFNT);
    double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    e.launches += 3;
    {
        PhaseScope scope(e, MD_PHASE_PAIRS, s);
        launch_pairs_half<KIND, SINGLE, true, true>(e, g, s);
    }
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        k_embed_sums<KIND><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, e.pot, e.sum_q, sum_split(e.max_nb), e.pair_energy,
                                               e.nn, e.max_nb, e.pc, e.x, e.rho, e.Fp, e.e_atom, e.ctl);
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    if (virial)
        k_force<SINGLE, true><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.xq, e.nn, e.nl, e.max_nb, e.pc, e.Fp, e.f,
                                                  kick ? e.v : nullptr, c_kick, e.bath, e.w_atom,
                                                  cut_bits(e.pot.rc), e.ctl);
    else
        k_force<SINGLE, false><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.xq, e.nn, e.nl, e.max_nb, e.pc, e.Fp, e.f,
                                                   kick ? e.v : nullptr, c_kick, e.bath, nullptr,
                                                   cut_bits(e.pot.rc), e.ctl);
}

template <int KIND, bool SINGLE>
static void run_fp64_n3(Engine& e, int kick, cudaStream_t s, bool virial) {
    Geo g = make_geo(e);
    const int nb = (int)((e.N + kFNT - 1) / kFNT);
    const double c_kick = 0.5 * e.cfg.dt / (e.cfg.mass * kMVV);
    e.launches += 4 + (kick ? 1 : 0);
    {
        PhaseScope scope(e, MD_PHASE_PAIRS, s);
        launch_pairs_half<KIND, SINGLE, false, false>(e, g, s);
    }
    {
        PhaseScope scope(e, MD_PHASE_DENSITY, s);
        cudaMemsetAsync(e.sum_q, 0, sizeof(long long) * kSumWords * e.N_pad, s);
        k_rho_n3<<<nb, kFNT, 0, s>>>(e.N, e.N_pad, e.nn, e.nl, e.n_up, e.max_nb, e.pc, e.sum_q,
                                     sum_split(e.max_nb), e.ctl);
        k_embed_n3<KIND><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, e.pot, e.x, e.sum_q, sum_split(e.max_nb), e.rho, e.Fp,
                                             e.e_atom, e.ctl);
    }
    PhaseScope scope(e, MD_PHASE_FORCE, s);
    cudaMemsetAsync(e.f, 0, sizeof(double) * 3 * e.N_pad, s);
    if (virial)
        k_force_n3<SINGLE, true><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.nn, e.nl, e.n_up, e.max_nb, e.pc, e.Fp,
                                                     e.f, e.w_atom, e.ctl);
    else
        k_force_n3<SINGLE, false><<<nb, kFNT, 0, s>>>(e.N, e.N_pad, g, e.x, e.nn, e.nl, e.n_up, e.max_nb, e.pc,
                                                      e.Fp, e.f, nullptr, e.ctl);
    if (kick) k_kick_n3<<<nb, kFNT, 0, s>>>(e.N, e.N_pad, e.f, e.v, c_kick, e.bath, e.ctl);
}

template <int KIND>
static void run_fp64_k(Engine& e, int kick, cudaStream_t s, bool virial) {
    if (e.newton3)
        single_fast(e) ? run_fp64_n3<KIND, true>(e, kick, s, virial) : run_fp64_n3<KIND, false>(e, kick, s, virial);
    else if (single_fast(e))
        run_fp64<KIND, true>(e, kick, s, virial);
    else
        run_fp64<KIND, false>(e, kick, s, virial);
}

void launch_forces(Engine& e, int kick, cudaStream_t s, bool virial) {
    if (e.N == 0) return;
    if (e.cfg.precision == MD_MIXED) {
        launch_forces_mixed(e, kick, s, virial);
        return;
    }
    switch (e.pot.kind) {
        case MD_POT_RGL: run_fp64_k<MD_POT_RGL>(e, kick, s, virial); break;
        case MD_POT_SC: run_fp64_k<MD_POT_SC>(e, kick, s, virial); break;
        default: run_fp64_k<MD_POT_SPLINE>(e, kick, s, virial); break;
    }
}

}  // namespace mdk
