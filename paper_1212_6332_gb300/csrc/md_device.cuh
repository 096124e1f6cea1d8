// Device-side helpers: periodic geometry, the taper, and the pair and
// embedding functions of Eq. (1) in float64 and float32.
#pragma once

#include <cmath>

#include "md_engine.cuh"
#include "md_math.cuh"

namespace mdk {

// Minimum image of one separation component d = x_j - x_i in a box of
// length L (h = L/2): one shift of +-L at most.
__device__ __forceinline__ double minimg(double d, double L, double h) {
    if (d > h) return d - L;
    if (d < -h) return d + L;
    return d;
}

__device__ __forceinline__ float minimgf(float d, float L, float h) {
    if (d > h) return d - L;
    if (d < -h) return d + L;
    return d;
}

// Wraps a coordinate into [0, L): x - L*floor(x/L) rounded after each
// operation (no fused multiply-add); +L if rounding left it negative (x just
// below k*L with |k| >= 2, where L*k rounds above x), then -L if it is L.
__device__ __forceinline__ double wrap_coord(double x, double L) {
    double k = floor(__ddiv_rn(x, L));
    double y = __dsub_rn(x, __dmul_rn(L, k));
    if (y < 0.0) y = __dadd_rn(y, L);
    if (y >= L) y = __dsub_rn(y, L);
    return y;
}

// The same result as wrap_coord without a division when -L <= x < 2L (one
// step of drift): for x in [L, 2L) the rule gives x - L (exact), for x in
// [-L, 0) it gives x + L, then -L if that rounded to L.
__device__ __forceinline__ double wrap_step(double x, double L) {
    if (x >= 0.0 && x < L) return x;
    if (x >= L && x < 2.0 * L) return x - L;
    if (x < 0.0 && x >= -L) {
        double y = x + L;
        return y >= L ? y - L : y;
    }
    return wrap_coord(x, L);
}

// A neighbour-list entry holds the neighbour's slot in its low 26 bits and
// the periodic image of the pair in its top 6 bits (2 bits per axis, shift
// + 1): x_j + shift * L is the image of atom j within the list radius of
// atom i. Positions are not wrapped between list builds, so the image stays
// valid for the life of the list and no minimum-image test is needed.
constexpr int kSlotBits = 26;
constexpr int kSlotMask = (1 << kSlotBits) - 1;
constexpr unsigned kNoShift = 0x15u;  // shifts (0, 0, 0)

__device__ __forceinline__ int entry_slot(int e) { return e & kSlotMask; }
__device__ __forceinline__ unsigned entry_code(int e) { return (unsigned)e >> kSlotBits; }
__device__ __forceinline__ int make_entry(int j, int sx, int sy, int sz) {
    unsigned code = (unsigned)(sx + 1) | ((unsigned)(sy + 1) << 2) | ((unsigned)(sz + 1) << 4);
    return (int)((unsigned)j | (code << kSlotBits));
}

// Species: the type of an atom rides in the w lane of its position (an
// exact small integer), and in bits 30-31 of the packed cell coordinates of
// its float32 offset; the tables of a type pair are in row-major upper
// triangle order.
__device__ __forceinline__ int pos_type(const double4_32a& p) { return (int)p.w; }
__device__ __forceinline__ int off_type(const float4& o) { return (int)((unsigned)__float_as_int(o.w) >> 30); }
__device__ __forceinline__ int pair_table(int T, int a, int b) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * T - lo * (lo - 1) / 2 + (hi - lo);
}
// type-pair table of two atoms from their float32 offsets (splines only)
template <int KIND>
__device__ __forceinline__ int species_pair(const Pot& P, const float4& oi, const float4& oj) {
    if (KIND != MD_POT_SPLINE || P.n_types <= 1) return 0;
    return pair_table(P.n_types, off_type(oi), off_type(oj));
}

__device__ __forceinline__ double image_shift(unsigned c2, double L) {
    return c2 == 1u ? 0.0 : (c2 == 0u ? -L : L);
}

// separation x_j - x_i of a list entry with its stored image
__device__ __forceinline__ void sep_entry(const double4_32a& xi, const double4_32a& xj, unsigned code,
                                          const double* L, double& dx, double& dy, double& dz) {
    dx = xj.x - xi.x;
    dy = xj.y - xi.y;
    dz = xj.z - xi.z;
    if (code != kNoShift) {
        dx += image_shift(code & 3u, L[0]);
        dy += image_shift((code >> 2) & 3u, L[1]);
        dz += image_shift((code >> 4) & 3u, L[2]);
    }
}

// Float64 pair cache entry (V'/r, rho'/r, rho(r), V(r)): written as one
// 32-byte sector, read by the sums as its (V'/r, rho'/r) or (rho, V) half.
__device__ __forceinline__ double2 cache_ab(const double4_32a* __restrict__ pc, int64_t slot) {
    return reinterpret_cast<const double2*>(pc)[2 * slot];
}
__device__ __forceinline__ double2 cache_fv(const double4_32a* __restrict__ pc, int64_t slot) {
    return reinterpret_cast<const double2*>(pc)[2 * slot + 1];
}

// |d|^2 with a fixed contraction, so every kernel that evaluates a pair
// gets the same bits
__device__ __forceinline__ double norm2(double dx, double dy, double dz) {
    return fma(dz, dz, fma(dy, dy, dx * dx));
}

// ---------------------------------------------------------------- exact r^2
//
// GB300 issues float64 at 1/64 of its float32 and integer rate, so the
// squared separation that the pair functions take is formed on the integer
// pipe: each coordinate as a 64-bit fixed-point number x 2^kq (exact for
// |x| >= 2^(52 - kq); below that the bits under 2^-kq are dropped, under
// 2^-50 A), the separation including its periodic image and the sum of its
// squares exact in 128-bit integers, and r^2 rounded once to the nearest
// double. This takes 6 float64 instructions (3 subtractions, the 3
// operations of |d|^2) off every pair, and the result is at least as
// accurate as the float64 form, which rounds up to four times. The scale
// kq is a function of the box alone (box_kq), so a box gives the same bits
// alone and inside a batch.

// Fixed-point scale of a box with sides L: every position lies within a few
// box lengths of its box (wrapped at each list build, drifting less than the
// skin in between), |x| < 4 L < 2^(ex + 2) for the longest side L < 2^ex,
// so kq = 60 - ex keeps |x| 2^kq below 2^62; separations below 8 A keep the
// sum of three squares below 2^(2 kq + 8) <= 2^126 (L is taken as at least
// 1 A, so kq <= 59).
__device__ __forceinline__ int box_kq(double Lx, double Ly, double Lz) {
    const double L = fmax(fmax(Lx, Ly), fmax(Lz, 1.0));
    const int ex = (int)((__double_as_longlong(L) >> 52) & 0x7ff) - 1022;  // L = f 2^ex, f in [1/2, 1)
    return 60 - ex;
}

// x 2^kq as a 64-bit integer, toward zero, formed from the bit pattern
__device__ __forceinline__ long long to_fixed(double x, int kq) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu);
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = e - 1075 + kq;  // x = m 2^(e - 1075)
    unsigned long long v = 0;
    if (e != 0) v = sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0ull);
    return (b >> 63) ? -(long long)v : (long long)v;
}

// (hi 2^64 + lo) 2^-scale rounded to the nearest double (ties to even),
// from the bit patterns
__device__ __forceinline__ double round_u128(unsigned long long hi, unsigned long long lo, int scale) {
    if (hi == 0ull) {
        if (lo == 0ull) return 0.0;
        hi = lo;
        lo = 0ull;
        scale += 64;
    }
    const int lz = __clzll((long long)hi);
    const unsigned long long top = (hi << lz) | ((lo >> 1) >> (63 - lz));  // leading one at bit 63
    const unsigned long long rest = lo << lz;
    unsigned long long m = top >> 11;  // 53 bits
    const unsigned long long rb = top & 0x7ffull;
    if (rb > 0x400ull || (rb == 0x400ull && (rest != 0ull || (m & 1ull)))) ++m;
    // the leading one of the result is 2^(127 - lz - scale); m carries the
    // implicit bit, so a carry out of the rounding moves the exponent up
    const long long E = 127 - lz - scale;
    return __longlong_as_double((long long)(((unsigned long long)(E + 1022) << 52) + m));
}

// (lo, hi) += (blo, bhi) in 128 bits
__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi, unsigned long long blo,
                                       unsigned long long bhi) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(blo), "l"(bhi));
}

// d^2 of a fixed-point difference |d| < 2^58 in 29-bit limbs, d = h 2^29 + l:
// d^2 = h^2 2^58 + (h l) 2^30 + l^2, each product below 2^58
__device__ __forceinline__ void sq_parts(long long d, unsigned long long& shh, unsigned long long& shl,
                                         unsigned long long& sll) {
    const unsigned long long u = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
    const unsigned h = (unsigned)(u >> 29), l = (unsigned)u & 0x1fffffffu;
    shh += (unsigned long long)h * h;
    shl += (unsigned long long)h * l;
    sll += (unsigned long long)l * l;
}

// (dx^2 + dy^2 + dz^2) 2^-scale of fixed-point differences, exact in 128
// bits and rounded once
__device__ __forceinline__ double r2_fixed(long long dx, long long dy, long long dz, int scale) {
    unsigned long long shh = 0ull, shl = 0ull, sll = 0ull;
    sq_parts(dx, shh, shl, sll);
    sq_parts(dy, shh, shl, sll);
    sq_parts(dz, shh, shl, sll);
    unsigned long long lo = shh << 58, hi = shh >> 6;
    add128(lo, hi, shl << 30, shl >> 34);
    add128(lo, hi, sll, 0ull);
    return round_u128(hi, lo, scale);
}

// 1/sqrt(x) and sqrt(x) of a positive normal double on the integer pipe
// (the float64 form, a Newton step and r = x / sqrt(x), takes 6 float64
// instructions). With x = m' 2^(2h), m' in [1, 4): a float32 estimate y0 of
// 1/sqrt(m') (hardware rsqrt of m' truncated to float32), then in fixed
// point e = 1 - m' y0^2 and the third-order step
//     y1 = y0 (1 + e/2 + 3 e^2 / 8)
// (truncation 5 e^3 / 16 < 2^-62 for |e| < 2^-21), sqrt(m') = m' y1, each
// rounded once to the nearest double and scaled by 2^-h, 2^h. The fixed-
// point steps keep 63 fractional bits or more, so either result lies within
// 0.51 ulp of the true value (correctly rounded but for near-ties), against
// up to about one ulp for the float64 form.
__device__ __forceinline__ void rsqrt_sqrt(double x, double& y, double& r) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)(b >> 52) - 1023;  // x = m 2^e, m in [1, 2)
    const int odd = e & 1;
    const int h = (e - odd) / 2;
    const unsigned long long M = ((b & 0xfffffffffffffull) | (1ull << 52)) << odd;  // m' 2^52
    // m' in float32 (fraction truncated), its rsqrt in (1/2, 1]
    const float mf = __uint_as_float(((unsigned)(127 + odd) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    const unsigned yb = __float_as_uint(rsqrtf(mf));
    const int ey = (int)(yb >> 23) - 127;                                                  // -1 or 0
    const unsigned long long Y0 = (unsigned long long)((yb & 0x7fffffu) | 0x800000u) << (8 + ey);  // y0 2^31
    // e 2^64 = (2^114 - m' y0^2 2^114) 2^-50; |e| < 2^-20, so the bits of
    // the product above 2^114 cancel and its low 114 bits decide
    const unsigned long long Y2 = Y0 * Y0;  // y0^2 2^62
    const unsigned long long plo = M * Y2, phi = __umul64hi(M, Y2);
    unsigned long long dlo = 0ull, dhi = 1ull << 50;  // 2^114
    asm("sub.cc.u64 %0, %0, %2;\n\tsubc.u64 %1, %1, %3;" : "+l"(dlo), "+l"(dhi) : "l"(plo), "l"(phi));
    const long long E = (long long)((dhi << 14) | (dlo >> 50));
    const long long C = (E >> 1) + (3 * __mul64hi(E, E) >> 3);  // (e/2 + 3e^2/8) 2^64
    // y1 2^95 = Y0 2^64 + Y0 C, in two's complement over 128 bits
    unsigned long long ylo = (unsigned long long)((long long)Y0 * C);
    unsigned long long yhi = (unsigned long long)__mul64hi((long long)Y0, C) + Y0;
    y = round_u128(yhi, ylo, 95 + h);
    const unsigned long long Y1h = (yhi << 32) | (ylo >> 32);  // y1 2^63
    r = round_u128(__umul64hi(M, Y1h), M * Y1h, 115 - h);
}

// |x_j + shift L - x_i|^2 of a list entry from fixed-point coordinates (q_i,
// q_j, q_L: x_i, x_j and L through to_fixed)
__device__ __forceinline__ double r2_exact(const long long (&qi)[3], long long qjx, long long qjy, long long qjz,
                                           unsigned code, const long long (&qL)[3], int kq) {
    long long d[3] = {qjx - qi[0], qjy - qi[1], qjz - qi[2]};
    if (code != kNoShift) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned c = (code >> (2 * a)) & 3u;
            d[a] += c == 0u ? -qL[a] : (c == 2u ? qL[a] : 0ll);
        }
    }
    return r2_fixed(d[0], d[1], d[2], 2 * kq);
}

// the same from x_j in float64
__device__ __forceinline__ double r2_exact(const long long (&qi)[3], const double4_32a& xj, unsigned code,
                                           const long long (&qL)[3], int kq) {
    return r2_exact(qi, to_fixed(xj.x, kq), to_fixed(xj.y, kq), to_fixed(xj.z, kq), code, qL, kq);
}

// Fixed-point copy of a position for the pair passes: (x, y, z) 2^kq and the
// species label
__device__ __forceinline__ longlong4_32a fixed_pos(const double4_32a& p, int kq) {
    longlong4_32a q;
    q.x = to_fixed(p.x, kq);
    q.y = to_fixed(p.y, kq);
    q.z = to_fixed(p.z, kq);
    q.w = (long long)pos_type(p);
    return q;
}

// ---------------------------------------------------------------- fixed-point sums
//
// The float64 density and pair-energy sums of Eq. (1)-(2) are taken in
// fixed point: every term rounded once to the nearest multiple of 2^-kSumQ
// (on the integer pipe, from its bit pattern), the terms added as integers,
// the total rounded once to a double. Integer addition is exact and
// associative, so the total does not depend on the order of the terms: the
// pair pass adds each pair's rho(r) and V(r) to both of its atoms with
// atomic adds and still gets the same bits on every run, and every kernel
// that forms the sums in another order (small systems, the block-per-box
// schedule, the Newton's-third-law variant) gets those bits too. Error: at
// most K 2^-(kSumQ+1) = K 4.4e-16 for K terms, plus the final rounding
// (a float64 sum rounds up to K times by half an ulp of its running total:
// 4.4e-16 for totals in [4, 8), 1.8e-15 for the ~20 of a Cu density).
//
// Range: a term q = x 2^kSumQ is split as q = hi 2^S + lo with lo in
// [-2^(S-1), 2^(S-1)) and a total keeps two 64-bit words, sum(lo) and
// sum(hi). S = 62 - ceil(log2(list capacity)) keeps the low word of a full
// list inside 64 bits; for the terms of ordinary configurations (|x| below
// 2^(S-1-kSumQ), 16 eV for a capacity of 96) hi is 0 and only the low word
// is touched. The total hi 2^S + lo is exact in 128 bits, so no term size
// short of ~2^60 eV loses range.
//
// Small totals: the resolution is absolute, and F'(rho) = -1/(2 sqrt(rho))
// turns an absolute error of rho into a relative one of 1/(2 rho) times
// it. An atom whose fixed-point density is below kSumSmall (an atom with
// almost no neighbours inside r_cut: a gas, a dimer near its cutoff; a
// crystal's densities are ~10-100) therefore takes both of its sums again
// in float64, over its cached pair values in list order (list_sums_f64),
// in every kernel that finishes the density: the same rule on the same exact
// total picks the same path everywhere.
constexpr int kSumQ = 50;

// S for lists of capacity cap (at most 2^20)
__host__ __device__ inline int sum_split(int cap) {
    int c = 0;
    while (c < 20 && (1 << c) < cap) ++c;
    return 62 - c;
}

// round(x 2^kSumQ) to the nearest integer (ties to even), split into
// (hi, lo) at S; false for a non-finite x or |x| 2^kSumQ >= 2^(2S) (then
// |hi| could reach 2^S, and a full list of such terms the 64-bit range)
__device__ __forceinline__ bool split_fixed(double x, int S, long long& hi, long long& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu);
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = e - 1075 + kSumQ;  // |x| 2^kSumQ = m 2^sh
    hi = 0;
    lo = 0;
    if (e == 0) return true;  // zero or subnormal: far below the resolution
    if (sh >= 0) {
        if (sh + 53 > 2 * S) return false;  // Inf, NaN or |x| >= 2^(2S - kSumQ) (~2^60 eV)
        __int128 q = (__int128)m << sh;
        if (b >> 63) q = -q;
        const __int128 h = (q + ((__int128)1 << (S - 1))) >> S;
        hi = (long long)h;
        lo = (long long)(q - h * ((__int128)1 << S));
        return true;
    }
    if (sh <= -54) return true;  // |x| 2^kSumQ < 1/2
    const int r = -sh;
    unsigned long long v = m >> r;
    const unsigned long long rem = m & ((1ull << r) - 1ull), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (v & 1ull))) ++v;
    // v < 2^53 <= 2^(S-1): the whole term is the low word
    lo = (b >> 63) ? -(long long)v : (long long)v;
    return true;
}

// (hi 2^S + lo) 2^-kSumQ rounded once to the nearest double
__device__ __forceinline__ double sum_value(long long hi, long long lo, int S) {
    const __int128 t = (__int128)hi * ((__int128)1 << S) + (__int128)lo;
    const unsigned __int128 u = t < 0 ? (unsigned __int128)(-t) : (unsigned __int128)t;
    const double a = round_u128((unsigned long long)(u >> 64), (unsigned long long)u, kSumQ);
    return t < 0 ? -a : a;
}

// One fixed-point total.
struct FixedSum {
    long long lo = 0, hi = 0;
    __device__ __forceinline__ bool add(double x, int S) {
        long long h, l;
        const bool ok = split_fixed(x, S, h, l);
        lo += l;
        hi += h;
        return ok;
    }
    __device__ __forceinline__ double value(int S) const { return sum_value(hi, lo, S); }
};

// whether a density total is below kSumSmall = 2 (then its float64 list
// sum serves instead)
__device__ __forceinline__ bool sums_small(const FixedSum& qr) {
    return qr.hi == 0 && qr.lo < (2ll << kSumQ);
}

// rho_i and sum_j V_ij in float64 from the cached pair values of atom i's
// list, in list order (round-to-nearest adds)
__device__ __forceinline__ void list_sums_f64(const double4_32a* __restrict__ pc, int64_t Np, int64_t i, int n,
                                              double& r_i, double& ep) {
    r_i = 0.0;
    ep = 0.0;
    for (int k = 0; k < n; ++k) {
        const double2 w = reinterpret_cast<const double2*>(pc)[2 * ((int64_t)k * Np + i) + 1];
        r_i = __dadd_rn(r_i, w.x);
        ep = __dadd_rn(ep, w.y);
    }
}

// ---------------------------------------------------------------- force sums in float32 pieces
//
// The force of Eq. (3) as f_i = sum_j s_ij d_ij over the list, d_ij = x_j -
// x_i from the fixed-point positions (exact, the entry's image shift added
// as an integer), with float32 arithmetic only: float64 issues at about 1/64
// of the float32 rate on this part, so four float64 instructions per entry
// cost more than the ~100 float32 and integer ones below.
//   d: the fixed-point difference (pre-shifted by sh bits with rounding
//     where the box's scale would put more than 54 bits below r_cut) cut
//     into three exact float32 values formed from the bits (an integer add
//     or or with an exponent-scaled 1.5 2^23 or 2^23, then one exact
//     subtraction): a = its high word (signed, below 2^22), b = the next
//     23 bits, c = the last 9; then d_h = RN(a + b) with its exact
//     remainder (Dekker's Fast2Sum), d_l = RN(remainder + c): d_h + d_l is
//     d to about 2^-48 of |d|, whatever |d|;
//   s: s_h = s truncated to 24 significant bits, s_l = the remaining 29
//     bits rounded to 23 (both from the float64 bit pattern), relative
//     error 2^-48;
//   s d = p + e with p = s_h d_h rounded, e = its exact error (one FMA) +
//     s_l d_h + s_h d_l (s_l d_l, 2^-47 of the term, is left out);
//   the total is a float-float pair (A, c): A + p by Knuth's TwoSum (the
//     rounding error of the addition exactly), that error and e added to c,
//     then (A, c) renormalised by Fast2Sum so that |c| <= ulp(A)/2.
// The error of a term is at most about 2^-46 of |s| |d| (the rounding of
// its small parts e, up to 2^-22 of p); the total adds about 2^-48 of
// itself per term. The result A + c is exact in float64. Every operation is one IEEE rounding in a fixed
// order (no contraction) and every rounding is to nearest, so the bits
// depend on the list order alone and the errors carry no bias.
struct DSplit {
    long long rnd;  // 2^(sh - 1) if sh > 0, else 0: the pre-shift rounds to nearest
    int sh;
    int mh, mm, ml;  // bit patterns of 1.5 2^23 2^(32 + sh - kq), 2^23 2^(9 + sh - kq), 2^23 2^(sh - kq)
    float ch, cm, cl;  // the same as float32 values
};

// cb: 2^cb > r_cut (entries with nonzero cached terms lie within r_cut)
__device__ __forceinline__ DSplit dsplit_init(int kq, int cb) {
    DSplit D;
    D.sh = max(0, kq + cb - 54);
    D.rnd = D.sh > 0 ? 1ll << (D.sh - 1) : 0ll;
    D.mh = 0x4b400000 + (32 + D.sh - kq) * (1 << 23);
    D.mm = 0x4b000000 + (9 + D.sh - kq) * (1 << 23);
    D.ml = 0x4b000000 + (D.sh - kq) * (1 << 23);
    D.ch = __int_as_float(D.mh);
    D.cm = __int_as_float(D.mm);
    D.cl = __int_as_float(D.ml);
    return D;
}

// d + rnd (d in units of 2^-kq, the rounding constant already added) ->
// d_h + d_l
__device__ __forceinline__ void dsplit(long long dr, const DSplit& D, float& dh, float& dl) {
    const int hi = (int)(dr >> 32);
    const unsigned lo = (unsigned)dr;
    const int k = hi >> D.sh;                                                      // bits 32 + sh and up
    const unsigned t = __funnelshift_r(lo, (unsigned)hi, 9 + D.sh) & 0x7fffffu;  // bits 9 + sh .. 31 + sh
    const unsigned u = (lo >> D.sh) & 0x1ffu;                                     // bits sh .. 8 + sh
    const float a = __fsub_rn(__int_as_float(D.mh + k), D.ch);
    const float b = __fsub_rn(__uint_as_float((unsigned)D.mm | t), D.cm);  // 0 <= b < one unit of a
    const float c = __fsub_rn(__uint_as_float((unsigned)D.ml | u), D.cl);  // 0 <= c < one unit of b
    dh = __fadd_rn(a, b);
    const float r = __fsub_rn(b, __fsub_rn(dh, a));  // a + b = dh + r exactly (a = 0 or |a| > b)
    dl = __fadd_rn(r, c);
}

// s -> s_h + s_l from the float64 bits (2^-100 <= |s| < 2^128; zero, other
// magnitudes and non-finite values go through the conversion, s_l = 0)
__device__ __forceinline__ void ssplit(double s, float& sh, float& sl) {
    const unsigned hi = (unsigned)__double2hiint(s), lo = (unsigned)__double2loint(s);
    const unsigned ab = hi & 0x7fffffffu;
    if (ab - (923u << 20) < ((1151u - 923u) << 20)) {
        const unsigned sg = hi & 0x80000000u;
        const unsigned fb = __funnelshift_l(lo, ab - (896u << 20), 3);  // |s| truncated to 24 bits
        sh = __uint_as_float(fb | sg);
        const unsigned F = ((fb & 0x7f800000u) - (23u << 23)) | sg;   // 2^23 at the residual's scale
        // the residual's 29 bits rounded to 23 (a carry to 2^23 steps the
        // exponent of the added pattern: still the exact value)
        sl = __fsub_rn(__uint_as_float(F + (((lo & 0x1fffffffu) + 32u) >> 6)), __uint_as_float(F));
    } else {
        sh = __double2float_rn(s);
        sl = 0.f;
    }
}

struct ForceSumF {
    float A[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
    // one component: A + c += s d with s = sh + sl, d = dh + dl
    __device__ __forceinline__ void add(int ax, float sh, float sl, float dh, float dl) {
        const float p = __fmul_rn(sh, dh);
        float e = __fmaf_rn(sh, dh, -p);  // the product's rounding error, exactly
        e = __fmaf_rn(sl, dh, e);
        e = __fmaf_rn(sh, dl, e);
        const float S = __fadd_rn(A[ax], p);  // TwoSum: S + err = A + p exactly
        const float bp = __fsub_rn(S, A[ax]);
        const float err = __fadd_rn(__fsub_rn(A[ax], __fsub_rn(S, bp)), __fsub_rn(p, bp));
        const float t = __fadd_rn(c[ax], __fadd_rn(err, e));
        // renormalised (Dekker's Fast2Sum), |c| <= ulp(A) / 2: the low part
        // stays small, so its roundings stay ~2^-48 of the running total
        A[ax] = __fadd_rn(S, t);
        c[ax] = __fsub_rn(t, __fsub_rn(A[ax], S));
    }
    // one entry from its pieces (sh, sl; dh, dl per axis)
    __device__ __forceinline__ void add(float sh, float sl, const float (&dh)[3], const float (&dl)[3]) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) add(ax, sh, sl, dh[ax], dl[ax]);
    }
    // one entry: s and the rounded difference (x, y, z)
    __device__ __forceinline__ void add(double s, long long rx, long long ry, long long rz, const DSplit& D) {
        float sh, sl, dh[3], dl[3];
        ssplit(s, sh, sl);
        dsplit(rx, D, dh[0], dl[0]);
        dsplit(ry, D, dh[1], dl[1]);
        dsplit(rz, D, dh[2], dl[2]);
        add(sh, sl, dh, dl);
    }
    __device__ __forceinline__ double value(int ax) const { return (double)A[ax] + (double)c[ax]; }
};

// the fixed-point image shift of a list entry along one axis
__device__ __forceinline__ long long qshift(unsigned code, int ax, long long qL) {
    const unsigned c = (code >> (2 * ax)) & 3u;
    return c == 0u ? -qL : (c == 2u ? qL : 0ll);
}

// 2^cb > rc, for dsplit_init (host side)
inline int cut_bits(double rc) {
    int ex = 0;
    std::frexp(rc, &ex);  // rc = f 2^ex, f in [1/2, 1)
    return ex;
}

// The per-atom totals live in kSumWords = 4 words per atom, word w of atom
// i at sq[w N_pad + i]: rho low, V low, rho high, V high.

// r^2 < c^2 for non-negative, non-NaN doubles, as an integer compare
__device__ __forceinline__ bool below(double r2, double c2) {
    return __double_as_longlong(r2) < __double_as_longlong(c2);
}

// One friction half step of Eq. (4) on a velocity (see Bath); an atom at
// rest stays at rest.
__device__ __forceinline__ void bath_half(const Bath& B, double& vx, double& vy, double& vz) {
    if (!B.on) return;
    const double v2 = vx * vx + vy * vy + vz * vz;
    if (!(v2 > 0.0)) return;
    const double Ti = B.m_3kb * v2;
    const double lam = sqrt((B.T_e + (Ti - B.T_e) * B.decay) / Ti);
    vx *= lam;
    vy *= lam;
    vz *= lam;
}

__device__ __forceinline__ int load_status(const Ctl* c) {
    return *((volatile const int*)&c->status);
}

// Whether box b rebuilds in this call: always when mode is 1, else when its
// largest displacement since its last build exceeds skin/2 (boxes decide
// independently). The caller reads the status word once: an error raised
// by an earlier kernel skips the whole build.
__device__ __forceinline__ bool box_due(const unsigned long long* disp, int b, int mode, unsigned long long thr) {
    return mode || disp[b] > thr;
}


// Float32 offset of each atom from the origin of the cell it was binned
// into (minimum image), w = packed cell coordinates: the list build's
// prefilter and the mixed-precision pair math use it.
__device__ __forceinline__ float4 cell_local(const Geo& g, int b, int gc, double4_32a p) {
    int xyz = g.cell_xyz[gc];
    int c[3] = {xyz & 1023, (xyz >> 10) & 1023, (xyz >> 20) & 1023};
    double pc[3] = {p.x, p.y, p.z};
    float o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double L = g.L[3 * b + a];
        double d = pc[a] - c[a] * g.cell_len[3 * b + a];
        o[a] = (float)minimg(d, L, 0.5 * L);
    }
    return make_float4(o[0], o[1], o[2], __int_as_float(xyz | (pos_type(p) << 30)));
}

// The (de-duplicated) 27-cell stencil of cell (cx, cy, cz) of box b, as
// global cell ids in ascending order: atoms are sorted by cell id, so
// visiting the stencil in this order lists neighbours by ascending slot,
// which lets the partner's position in a list be found by binary search.
__device__ __forceinline__ int stencil_sorted(const Geo& g, int b, int cx, int cy, int cz, int* q) {
    const int ncx = g.nc[3 * b], ncy = g.nc[3 * b + 1], ncz = g.nc[3 * b + 2];
    const int nx = ncx >= 3 ? 3 : ncx, ny = ncy >= 3 ? 3 : ncy, nz = ncz >= 3 ? 3 : ncz;
    int k = 0;
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy)
            for (int iz = 0; iz < nz; ++iz) {
                int ox = ncx >= 3 ? ix - 1 : ix, oy = ncy >= 3 ? iy - 1 : iy, oz = ncz >= 3 ? iz - 1 : iz;
                int qx = (cx + ox + ncx) % ncx, qy = (cy + oy + ncy) % ncy, qz = (cz + oz + ncz) % ncz;
                q[k++] = g.cell_rank[g.cell_off[b] + (qx * ncy + qy) * ncz + qz];
            }
    for (int a = 1; a < k; ++a) {
        int v = q[a], j = a - 1;
        while (j >= 0 && q[j] > v) {
            q[j + 1] = q[j];
            --j;
        }
        q[j + 1] = v;
    }
    return k;
}

// Minimum image of a cell-index difference on an axis of n cells.
__device__ __forceinline__ int cell_delta(int cj, int ci, int n) {
    int d = cj - ci;
    if (2 * d > n) return d - n;
    if (2 * d < -n) return d + n;
    return d;
}

// Candidate test. A float32 separation from the cell-local offsets (exact
// cell difference times the cell side plus the offset difference) decides
// every candidate whose r^2 lies farther than `margin` from rl^2; the float32
// error of that r^2 is below 2e-4 A^2 for the cell sides used here, and
// margin = 4e-4 * rl A^2 covers it with a wide factor. The few candidates
// inside the band (~0.01 per atom) take the exact float64 test, which alone
// decides membership, so the list equals the oracle's bit for bit.

// The float64 list test, the definition both the oracle and the GPU lists
// follow: d = x_j - x_i with one minimum-image shift per axis, r^2 rounded
// after every operation (no fused multiply-add), accepted when r^2 < rl^2;
// (sx, sy, sz) is the shift in box lengths.
__device__ __forceinline__ bool exact_candidate(const double4_32a& xi, const double4_32a& xj, double Lx, double Ly,
                                                double Lz, double rl2, int& sx, int& sy, int& sz) {
    const double hx = 0.5 * Lx, hy = 0.5 * Ly, hz = 0.5 * Lz;
    double ex = __dsub_rn(xj.x, xi.x), ey = __dsub_rn(xj.y, xi.y), ez = __dsub_rn(xj.z, xi.z);
    sx = ex > hx ? -1 : (ex < -hx ? 1 : 0);
    sy = ey > hy ? -1 : (ey < -hy ? 1 : 0);
    sz = ez > hz ? -1 : (ez < -hz ? 1 : 0);
    ex = minimg(ex, Lx, hx);
    ey = minimg(ey, Ly, hy);
    ez = minimg(ez, Lz, hz);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
    return r2 < rl2;
}

__device__ __forceinline__ bool list_candidate(const float4& oi, const float4& oj, const double4_32a& xi,
                                               const double4_32a* __restrict__ xall, int j, int cix, int ciy, int ciz,
                                               int ncx, int ncy, int ncz, float lfx, float lfy, float lfz, float Lfx,
                                               float Lfy, float Lfz, double Lx, double Ly, double Lz, double rl2,
                                               float rl2f_lo, float rl2f_hi, int& sx, int& sy, int& sz) {
    int cj = __float_as_int(oj.w);
    // cell difference as a minimum image in whole cells; the wrap it needed
    // is a shift of one box length
    int rx = (cj & 1023) - cix, ry = ((cj >> 10) & 1023) - ciy, rz = ((cj >> 20) & 1023) - ciz;
    int wx = cell_delta(cj & 1023, cix, ncx), wy = cell_delta((cj >> 10) & 1023, ciy, ncy),
        wz = cell_delta((cj >> 20) & 1023, ciz, ncz);
    // w - r is -n, 0 or n: its sign is the shift in box lengths
    sx = (wx > rx) - (wx < rx);
    sy = (wy > ry) - (wy < ry);
    sz = (wz > rz) - (wz < rz);
    float dx = fmaf((float)wx, lfx, oj.x - oi.x);
    float dy = fmaf((float)wy, lfy, oj.y - oi.y);
    float dz = fmaf((float)wz, lfz, oj.z - oi.z);
    // one more box shift when the cell image is not the nearest (fewer than
    // 3 cells on an axis)
    if (dx > 0.5f * Lfx) { dx -= Lfx; sx -= 1; } else if (dx < -0.5f * Lfx) { dx += Lfx; sx += 1; }
    if (dy > 0.5f * Lfy) { dy -= Lfy; sy -= 1; } else if (dy < -0.5f * Lfy) { dy += Lfy; sy += 1; }
    if (dz > 0.5f * Lfz) { dz -= Lfz; sz -= 1; } else if (dz < -0.5f * Lfz) { dz += Lfz; sz += 1; }
    float r2f = dx * dx + dy * dy + dz * dz;
    // components within 1e-3 A of half a box take the exact path too, so the
    // stored image is the float64 one
    bool near_half =
        fabsf(dx) > 0.5f * Lfx - 1e-3f || fabsf(dy) > 0.5f * Lfy - 1e-3f || fabsf(dz) > 0.5f * Lfz - 1e-3f;
    if (r2f < rl2f_lo && !near_half) return true;
    if (r2f > rl2f_hi && !near_half) return false;
    return exact_candidate(xi, xall[j], Lx, Ly, Lz, rl2, sx, sy, sz);
}

// Each list leaves the build ascending by neighbour slot. It is rotated to
// [upper entries (j > i) | lower entries (j < i)], both parts ascending, so
// the pair pass reads row k of all lists together (coalesced) while it
// walks only the upper entries, and the partner of an upper entry is found
// by binary search in the partner's lower part. n_up[i] counts the upper
// entries; lists longer than kRotMax keep the ascending order and
// n_up = -1 (the pair pass then scans them whole). The lower part (or the
// whole list when it is not rotated) is also copied row-major into
// nl_lo[i * max_nb + m], so that the search reads a few contiguous sectors
// of the partner's list instead of one column-major row per probe.
constexpr int kRotMax = 320;

__device__ __forceinline__ int rotate_list(int64_t Np, int64_t i, int n, int* __restrict__ nl,
                                           int* __restrict__ nl_lo, int max_nb) {
    int* lo_out = nl_lo + i * (int64_t)max_nb;
    if (n > kRotMax) {
        for (int k = 0; k < n; ++k) lo_out[k] = nl[(int64_t)k * Np + i];
        return -1;
    }
    int lo = 0;
    while (lo < n && entry_slot(nl[(int64_t)lo * Np + i]) < i) {
        lo_out[lo] = nl[(int64_t)lo * Np + i];
        ++lo;
    }
    if (lo == 0 || lo == n) return n - lo;
    int buf[kRotMax];
    for (int k = 0; k < n; ++k) buf[k] = nl[(int64_t)k * Np + i];
    for (int k = 0; k < n; ++k) nl[(int64_t)k * Np + i] = buf[(k + lo) % n];
    return n - lo;
}

// The same rotation for the kernel-built lists, which the list build wrote
// into a scratch array of the same layout (raw): each row is gathered from
// its rotated source row, so no per-thread staging is needed.
__device__ __forceinline__ int rotate_list_from(int64_t Np, int64_t i, int n, const int* __restrict__ raw,
                                                int* __restrict__ nl, int* __restrict__ nl_lo, int max_nb) {
    int* lo_out = nl_lo + i * (int64_t)max_nb;
    if (n > kRotMax) {
        for (int k = 0; k < n; ++k) {
            const int v = raw[(int64_t)k * Np + i];
            lo_out[k] = v;
            nl[(int64_t)k * Np + i] = v;
        }
        return -1;
    }
    int lo = 0;
    while (lo < n && entry_slot(raw[(int64_t)lo * Np + i]) < i) {
        lo_out[lo] = raw[(int64_t)lo * Np + i];
        ++lo;
    }
    for (int k = 0; k < n; ++k) {
        const int src = k + lo < n ? k + lo : k + lo - n;
        nl[(int64_t)k * Np + i] = raw[(int64_t)src * Np + i];
    }
    return n - lo;
}

__device__ __forceinline__ void reverse_index(int64_t Np, int64_t i, int n, int nup, const int* __restrict__ nn,
                                              const int* __restrict__ nl, const int* __restrict__ nl_lo,
                                              const int* __restrict__ n_up, int max_nb, int* __restrict__ rev) {
    const int kmax = nup < 0 ? n : nup;
    for (int k = 0; k < kmax; ++k) {
        const int j = entry_slot(nl[(int64_t)k * Np + i]);
        if (j <= i) continue;
        const int nj = min(nn[j], max_nb);
        const int uj = n_up[j];
        // j's lower part (or its whole ascending list), row-major
        const int* lst = nl_lo + (int64_t)j * max_nb;
        int lo = 0, hi = uj < 0 ? nj : nj - uj;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (entry_slot(lst[mid]) < i)
                lo = mid + 1;
            else
                hi = mid;
        }
        rev[(int64_t)k * Np + i] = (uj < 0 ? 0 : uj) + lo;
    }
}

// ---------------------------------------------------------------- float64

// C2 smoothstep taper S(r) = 1 - 10x^3 + 15x^4 - 6x^5 on [rs, rc), x = (r - rs)/(rc - rs),
// and dS/dr. The caller guarantees r < rc. Branch-free (x clamped at 0 gives
// S = 1, dS = 0 exactly): the perturbed third fcc shell straddles r_taper, so
// a branch would split most warps.
__device__ __forceinline__ void taper(const Pot& P, double r, double& S, double& dS) {
    double x = fmax((r - P.rs) * P.inv_w, 0.0);
    double x2 = x * x;
    S = 1.0 + x2 * x * (-10.0 + x * (15.0 - 6.0 * x));
    dS = x2 * (-30.0 + x * (60.0 - 30.0 * x)) * P.inv_w;
}

// Spline w (0: V, 1: rho, 2: F) of table tab (a type pair for V and rho,
// a type for F): every table of w has n = P.sn[w] coefficient entries.
__device__ __forceinline__ void spline_eval(const Pot& P, int w, double t, double& v, double& dv, int tab = 0) {
    double s = (t - P.st0[w]) * P.sinvh[w];
    int n = P.sn[w];
    const double4_32a* c = P.sp[w] + (int64_t)tab * n;
    if (s < 0.0) {
        double4_32a c0 = c[0];
        v = c0.x + (t - P.st0[w]) * c0.y;
        dv = c0.y;
        return;
    }
    int k = (int)s;
    if (k >= n - 1) {  // beyond the last knot: coefficient n-1 holds (value, slope) at the end
        double4_32a ce = c[n - 1];
        double u = t - (P.st0[w] + P.sh[w] * (n - 1));
        v = ce.x + u * ce.y;
        dv = ce.y;
        return;
    }
    double u = t - (P.st0[w] + P.sh[w] * k);
    double4_32a ck = c[k];
    v = ck.x + u * (ck.y + u * (ck.z + u * ck.w));
    dv = ck.y + u * (2.0 * ck.z + 3.0 * u * ck.w);
}

// integer power for the Sutton-Chen exponents when they are whole numbers
__device__ __forceinline__ double powr(double b, double e) {
    int k = (int)e;
    if ((double)k == e && k >= 0 && k <= 16) {
        double r = 1.0, p = b;
        while (k) {
            if (k & 1) r *= p;
            p *= p;
            k >>= 1;
        }
        return r;
    }
    return pow(b, e);
}

// Pair functions at r^2 < rc^2: V(r), rho(r), and A = V'(r)/r, B = rho'(r)/r
// (the force pass needs only these two ratios). T: the exponential table in
// shared memory.
template <int KIND>
__device__ __forceinline__ void pair_eval(const Pot& P, const double* __restrict__ T, double r2, double& phi,
                                          double& fr, double& A, double& B, int pt = 0) {
    double rinv, r;
    rsqrt_sqrt(r2, rinv, r);
    // pairs inside r_taper (r^2 <= r_taper^2) skip the taper (S = 1, S' = 0);
    // non-negative doubles order like their bit patterns, so the test runs
    // on the integer pipe
    const bool tap = __double_as_longlong(r2) > __double_as_longlong(P.rs2);
    if (KIND == MD_POT_RGL) {
        double e1, e2;
        // r = k h + d with k an integer next to r/h, chosen in float32 from
        // a float32 copy of r (integer and float32 pipes; k may be the
        // neighbour of the nearest one next to a half point, |d| <= h/2 +
        // 1e-6 A), d exact from one fused multiply-add; both exponentials
        // share it
        const int k = __float2int_rn(narrow_f32(r) * (float)kRxPerA);
        const int kk = k - P.rx_k0;
        if (P.rx && (unsigned)kk < (unsigned)P.rx_n) {
            const double d = fma(widen_f32((float)k), -1.0 / kRxPerA, r);
            const double2 E = P.rx[kk];
            // e^(-b d) = 1 + d (c0 + c1 d) + d^3 (c2 + c3 d): the first two
            // orders in float64, the rest (below |b d|^3/6 < 6e-9 for
            // |d| <= 1/2048 A and b <= 7 / A) in float32, whose error of a few
            // 1e-7 of that term stays below 1e-15 of the result; d and the
            // term cross between the precisions on the integer pipe
            const float df = narrow_f32_signed(d);
            const float d3 = df * df * df;
            const double h1 = widen_f32(d3 * fmaf(P.rx_f1[1], df, P.rx_f1[0]));
            const double h2 = widen_f32(d3 * fmaf(P.rx_f2[1], df, P.rx_f2[0]));
            e1 = fma(E.x, fma(d, fma(P.rx_c1[1], d, P.rx_c1[0]), h1), E.x);
            e2 = fma(E.y, fma(d, fma(P.rx_c2[1], d, P.rx_c2[0]), h2), E.y);
        } else {
            // the prefactors 2A and xi^2 ride in the exponent when both are positive
            e1 = P.fold ? exp_tab(P.pA - P.p_r0 * r, T, P.ek) : P.A2 * exp_tab(P.p - P.p_r0 * r, T, P.ek);
            e2 = P.fold ? exp_tab(P.qX - P.q2_r0 * r, T, P.ek) : P.xi2 * exp_tab(P.q2 - P.q2_r0 * r, T, P.ek);
        }
        if (tap) {
            double S, dS;
            taper(P, r, S, dS);
            phi = e1 * S;
            fr = e2 * S;
            A = e1 * (dS - P.p_r0 * S) * rinv;
            B = e2 * (dS - P.q2_r0 * S) * rinv;
        } else {
            phi = e1;
            fr = e2;
            A = e1 * (-P.p_r0) * rinv;
            B = e2 * (-P.q2_r0) * rinv;
        }
    } else if (KIND == MD_POT_SC) {
        double ar = P.a * rinv;
        double an, am;
        if (P.sc96) {
            // the Sutton-Chen Cu exponents: a^2, a^3, a^6 = (a^3)^2, a^9 =
            // a^6 a^3, four float64 multiplies where the two general
            // integer-power loops take eleven
            const double a2 = ar * ar, a3 = a2 * ar, a6 = a3 * a3;
            am = a6;
            an = P.eps * (a6 * a3);
        } else {
            an = P.eps * powr(ar, P.n);
            am = powr(ar, P.m);
        }
        if (tap) {
            double S, dS;
            taper(P, r, S, dS);
            phi = an * S;
            fr = am * S;
            A = an * (dS - P.n * rinv * S) * rinv;
            B = am * (dS - P.m * rinv * S) * rinv;
        } else {
            phi = an;
            fr = am;
            A = an * (-(P.n * rinv)) * rinv;
            B = am * (-(P.m * rinv)) * rinv;
        }
    } else {
        if (__double_as_longlong(r) >= __double_as_longlong(P.rc)) {  // r >= rc (both non-negative)
            phi = fr = A = B = 0.0;
            return;
        }
        double dphi, dfr;
        if (P.sq) {
            // the record is chosen from r in float32 (integer-formed copy):
            // next to a knot the neighbouring interval may be taken, whose
            // cubic agrees there in value and first two derivatives (C2),
            // so V and rho change by rounding only; the clamp keeps any r
            // (also a non-finite one) inside the table
            const float sf = fmaf(narrow_f32(r), P.sq_invhf, P.sq_c0f);
            const int kk = min(max(__float2int_rd(sf) + 1, 0), P.sq_n);
            const double4_32a* q = P.sq + ((int64_t)pt * (P.sq_n + 1) + kk) * 4;
            const double4_32a q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
            const double u = r - q0.x;
            phi = fma(u, fma(u, fma(u, q1.x, q0.w), q0.z), q0.y);
            dphi = fma(u, fma(u, q1.z, q1.y), q0.z);
            fr = fma(u, fma(u, fma(u, q2.z, q2.y), q2.x), q1.w);
            dfr = fma(u, fma(u, q3.x, q2.w), q2.x);
        } else {
            spline_eval(P, 0, r, phi, dphi, pt);
            spline_eval(P, 1, r, fr, dfr, pt);
        }
        A = dphi * rinv;
        B = dfr * rinv;
    }
}

// Loads the exponential table into shared memory (whole block).
__device__ __forceinline__ void load_exp_table(double* sT, const double* __restrict__ gT) {
    for (int k = threadIdx.x; k < kExpTable; k += blockDim.x) sT[k] = gT[k];
    __syncthreads();
}

// F(rho) and F'(rho); F = F' = 0 for rho <= 0 (RGL, SC)
template <int KIND>
__device__ __forceinline__ void embed(const Pot& P, double rho, double& F, double& Fp, int a = 0) {
    if (KIND == MD_POT_SPLINE) {
        spline_eval(P, 2, rho, F, Fp, a);
    } else {
        if (rho <= 0.0) {
            F = 0.0;
            Fp = 0.0;
            return;
        }
        // sqrt(rho) and 1/sqrt(rho) on the integer pipe (rsqrt_sqrt, within
        // 0.51 ulp each; float64 sqrt and division take ~20 float64
        // instructions); rho below the normal range keeps the library forms
        double y, s;
        if (rho >= 0x1p-1022) {
            rsqrt_sqrt(rho, y, s);
        } else {
            s = sqrt(rho);
            y = 1.0 / s;
        }
        F = -P.F_scale * s;
        Fp = (-0.5 * P.F_scale) * y;
    }
}

// rho_i, F'(rho_i) and E_i = F(rho_i) + 1/2 sum_j V_ij from the fixed-point
// totals of rho(r_ij) and V(r_ij) (type: the atom's species, splines)
// For a total below kSumSmall, pc (the pair cache), Np and n (the list
// length) give the float64 list sums instead (pc null: no such fallback,
// for the Newton's-third-law variant, whose lower slots hold no values).
template <int KIND>
__device__ __forceinline__ void embed_sums(const Pot& P, const FixedSum& qr, const FixedSum& qv, int S, int type,
                                           const double4_32a* __restrict__ pc, int64_t Np, int64_t i, int n,
                                           double& rho, double& Fp, double& E) {
    double ep;
    if (pc && sums_small(qr)) {
        list_sums_f64(pc, Np, i, n, rho, ep);
    } else {
        rho = qr.value(S);
        ep = qv.value(S);
    }
    double F;
    embed<KIND>(P, rho, F, Fp, type);
    E = fma(0.5, ep, F);
}

// the totals of atom i from the four words of sq
__device__ __forceinline__ void load_sums(const long long* __restrict__ sq, int64_t Np, int64_t i, FixedSum& qr,
                                          FixedSum& qv) {
    qr.lo = sq[i];
    qv.lo = sq[Np + i];
    qr.hi = sq[2 * Np + i];
    qv.hi = sq[3 * Np + i];
}

// ---------------------------------------------------------------- float32

// Branch-free: x clamped at 0 gives S = 1, dS = 0 exactly (pairs inside
// r_taper), without a branch that splits warps at r_taper (the 4M-atom mixed
// step 1.66 -> 1.58 ms against an early return for r <= r_taper, the same
// results).
__device__ __forceinline__ void taperf(const Pot& P, float r, float& S, float& dS) {
    const float x = fmaxf((r - P.f_rs) * P.f_inv_w, 0.0f);
    const float x2 = x * x;
    S = 1.0f + x2 * x * (-10.0f + x * (15.0f - 6.0f * x));
    dS = x2 * (-30.0f + x * (60.0f - 30.0f * x)) * P.f_inv_w;
}

__device__ __forceinline__ float powrf(float b, float e) {
    int k = (int)e;
    if ((float)k == e && k >= 0 && k <= 16) {
        float r = 1.0f, p = b;
        while (k) {
            if (k & 1) r *= p;
            p *= p;
            k >>= 1;
        }
        return r;
    }
    return powf(b, e);
}

__device__ __forceinline__ void spline_evalf(const Pot& P, int w, float t, float& v, float& dv, int tab = 0) {
    // float32 copies of the coefficient tables; u from the interval position
    const float s = (t - P.st0f[w]) * P.sinvhf[w];
    const int n = P.sn[w];
    const float4* c = P.spf[w] + (int64_t)tab * n;
    if (s < 0.0f) {
        const float4 c0 = c[0];
        v = c0.x + (t - P.st0f[w]) * c0.y;
        dv = c0.y;
        return;
    }
    const int k = (int)s;
    if (k >= n - 1) {
        const float4 ce = c[n - 1];
        const float u = (s - (float)(n - 1)) * P.shf[w];
        v = ce.x + u * ce.y;
        dv = ce.y;
        return;
    }
    const float u = (s - (float)k) * P.shf[w];
    const float4 ck = c[k];
    v = ck.x + u * (ck.y + u * (ck.z + u * ck.w));
    dv = ck.y + u * (2.0f * ck.z + 3.0f * u * ck.w);
}

template <int KIND>
__device__ __forceinline__ float dens_ff(const Pot& P, float r, int pt = 0) {
    if (KIND == MD_POT_RGL) {
        float S, dS;
        taperf(P, r, S, dS);
        return P.f_xi2 * __expf(P.f_q2 - P.f_q2_r0 * r) * S;
    } else if (KIND == MD_POT_SC) {
        float S, dS;
        taperf(P, r, S, dS);
        return powrf(P.f_a / r, P.f_m) * S;
    } else {
        if (r >= (float)P.rc) return 0.0f;
        float v, dv;
        spline_evalf(P, 1, r, v, dv, pt);
        return v;
    }
}

template <int KIND>
__device__ __forceinline__ void pair_allf(const Pot& P, float r, float& phi, float& dphi, float& fr,
                                          float& dfr, int pt = 0) {
    if (KIND == MD_POT_RGL) {
        float S, dS;
        taperf(P, r, S, dS);
        float e1 = P.f_A2 * __expf(P.f_p - P.f_p_r0 * r);
        float e2 = P.f_xi2 * __expf(P.f_q2 - P.f_q2_r0 * r);
        phi = e1 * S;
        dphi = e1 * (dS - P.f_p_r0 * S);
        fr = e2 * S;
        dfr = e2 * (dS - P.f_q2_r0 * S);
    } else if (KIND == MD_POT_SC) {
        float S, dS;
        taperf(P, r, S, dS);
        float rinv = 1.0f / r;
        float ar = P.f_a * rinv;
        float an = P.f_eps * powrf(ar, P.f_n), am = powrf(ar, P.f_m);
        phi = an * S;
        dphi = an * (dS - P.f_n * rinv * S);
        fr = am * S;
        dfr = am * (dS - P.f_m * rinv * S);
    } else {
        if (r >= (float)P.rc) {
            phi = dphi = fr = dfr = 0.0f;
            return;
        }
        spline_evalf(P, 0, r, phi, dphi, pt);
        spline_evalf(P, 1, r, fr, dfr, pt);
    }
}

// Compensated float32 accumulator (Kahan-Babuska / Neumaier): s + c carries
// about twice the float32 precision over the few hundred terms of one atom.
struct KSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        if (fabsf(s) >= fabsf(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// ---------------------------------------------------------------- mixed-precision separation

__device__ __forceinline__ int wrap_cells(int d, int n) {
    if (2 * d > n) return d - n;
    if (2 * d < -n) return d + n;
    return d;
}

// WIDE: every box has at least 3 cells per axis, so the nearest cell image
// is the nearest atom image and no box-length correction can be needed.
template <bool WIDE>
__device__ __forceinline__ void sep_mixed(const CellSep& cs, float4 oi, float4 oj, float& dx, float& dy, float& dz) {
    int ci = __float_as_int(oi.w), cj = __float_as_int(oj.w);
    int ddx = wrap_cells((cj & 1023) - (ci & 1023), cs.nx);
    int ddy = wrap_cells(((cj >> 10) & 1023) - ((ci >> 10) & 1023), cs.ny);
    int ddz = wrap_cells(((cj >> 20) & 1023) - ((ci >> 20) & 1023), cs.nz);
    dx = fmaf((float)ddx, cs.lx, oj.x - oi.x);
    dy = fmaf((float)ddy, cs.ly, oj.y - oi.y);
    dz = fmaf((float)ddz, cs.lz, oj.z - oi.z);
    if (!WIDE) {
        dx = minimgf(dx, cs.Lx, 0.5f * cs.Lx);
        dy = minimgf(dy, cs.Ly, 0.5f * cs.Ly);
        dz = minimgf(dz, cs.Lz, 0.5f * cs.Lz);
    }
}

// The same separation when every box has at least 3 cells per axis and
// the list entry carries the cell offset (-1, 0, 1 per axis, stored as
// 0..2: lists built for float32 pair math): no decoding of the packed cell
// coordinates. The offset becomes a float by the 2^23 bias (exact for small
// integers), and the arithmetic is that of sep_mixed<true>: the same bits.
__device__ __forceinline__ void sep_mixed_code(const CellSep& cs, float4 oi, float4 oj, unsigned code, float& dx,
                                               float& dy, float& dz) {
    const float kx = __int_as_float(0x4B000000 | (int)(code & 3u)) - 8388609.0f;
    const float ky = __int_as_float(0x4B000000 | (int)((code >> 2) & 3u)) - 8388609.0f;
    const float kz = __int_as_float(0x4B000000 | (int)((code >> 4) & 3u)) - 8388609.0f;
    dx = fmaf(kx, cs.lx, oj.x - oi.x);
    dy = fmaf(ky, cs.ly, oj.y - oi.y);
    dz = fmaf(kz, cs.lz, oj.z - oi.z);
}

// Separation of list entry e in a mixed-precision kernel: from the entry's
// cell offset when the atom's box has 3 or more cells per axis (every box,
// WIDE), else from the packed coordinates.
template <bool WIDE>
__device__ __forceinline__ void sep_mixed_entry(const CellSep& cs, float4 oi, float4 oj, int e, float& dx, float& dy,
                                                float& dz) {
    if (WIDE || (cs.nx >= 3 && cs.ny >= 3 && cs.nz >= 3))
        sep_mixed_code(cs, oi, oj, entry_code(e), dx, dy, dz);
    else
        sep_mixed<false>(cs, oi, oj, dx, dy, dz);
}

// Plain float32 partial sum over a group of list entries, folded into a
// compensated total at group ends.
struct GSum {
    float part = 0.0f;
    KSum tot;
    __device__ __forceinline__ void add(float x) { part += x; }
    __device__ __forceinline__ void flush() {
        tot.add(part);
        part = 0.0f;
    }
    __device__ __forceinline__ double value() {
        flush();
        return tot.value();
    }
};
constexpr int kGroupMask = 15;

template <bool SINGLE>
__device__ __forceinline__ CellSep cell_sep(const Geo& g, const CellSep& cs0, int64_t i) {
    if (SINGLE) return cs0;
    int b = g.atom_box[i];
    CellSep cs;
    cs.lx = g.cell_len_f[3 * b];
    cs.ly = g.cell_len_f[3 * b + 1];
    cs.lz = g.cell_len_f[3 * b + 2];
    cs.nx = g.nc[3 * b];
    cs.ny = g.nc[3 * b + 1];
    cs.nz = g.nc[3 * b + 2];
    cs.Lx = (float)g.L[3 * b];
    cs.Ly = (float)g.L[3 * b + 1];
    cs.Lz = (float)g.L[3 * b + 2];
    return cs;
}

// ---------------------------------------------------------------- reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Block-wide sum in a fixed order (deterministic). Result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < NT / 32; ++k) r += sh[k];
    return r;
}

}  // namespace mdk
