// Float64 elementary functions with few float64 instructions.
//
// On GB300 the float64 pipe issues 2 FMA per clock per SM (float32: 128), so
// the float64 path is bound by float64 instruction count. These replace the
// general-purpose library calls on the hot path; both stay within a few ulp
// (checked against CUDA's exp and rsqrt by the GPU tests through
// md_eval_math).
#pragma once

#include <cuda_runtime.h>

namespace mdk {

// Constants of the table-driven exponential, computed on the host at set-up
// from long-double arithmetic: inv_l = 2048/ln 2, l1 + l2 = ln 2 / 2048 (l1
// the nearest double, l2 the remainder).
struct ExpConst {
    double inv_l, l1, l2;
};

constexpr int kExpBits = 11;
constexpr double kRxPerA = 1024.0;  // r-table points per Angstrom (RGL pair path)
constexpr int kExpTable = 1 << kExpBits;  // 16 KB of shared memory per block

// e^y by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989), with a 2048-entry table:
//   n = round(y * 2048/ln2), y = n ln2/2048 + r, |r| <= ln2/4096,
//   e^y = 2^(n >> 11) * T[n & 2047] * (1 + r + r^2/2 + r^3/6),
// T[j] = 2^(j/2048); the neglected r^4/24 term is below 3.5e-17 (the larger
// table buys one polynomial degree: a float64 instruction per call). The
// rounding to an integer uses the 1.5 * 2^52 shift (the integer lands in the
// low word); the reduction uses two fused multiply-adds with the two-part
// constant; the power of two is added to the exponent field. Requires
// |y| < 700 (callers guarantee it); 8 float64 instructions.
__device__ __forceinline__ double exp_tab(double y, const double* __restrict__ T, const ExpConst& K) {
    const double shift = 6755399441055744.0;  // 1.5 * 2^52
    double t = fma(y, K.inv_l, shift);
    int n = __double2loint(t);
    double nd = t - shift;
    double r = fma(-nd, K.l1, y);
    r = fma(-nd, K.l2, r);
    double b = fma(fma(r, 1.0 / 6.0, 0.5), r, 1.0);  // 1 + r/2 + r^2/6
    double tj = T[n & (kExpTable - 1)];
    double res = fma(tj * r, b, tj);
    return __hiloint2double(__double2hiint(res) + ((n >> kExpBits) << 20), __double2loint(res));
}

// 1/sqrt(x) for x in the float32 normal range: a float32 hardware
// estimate refined by one third-order Newton step,
//   e = 1 - x y^2,  y' = y (1 + e/2 + 3e^2/8),
// whose error is O(e^3) (~1e-20 for a float32 start), i.e. rounding-limited.
// The float32 argument and the widened estimate are formed from the bit
// patterns by integer arithmetic (exponent re-biased, mantissa truncated or
// zero-padded), so no conversion instruction occupies the float64 pipe.
// float32 copy of a positive double in the float32 normal range, mantissa
// truncated, formed on the integer pipe
__device__ __forceinline__ float narrow_f32(double x) {
    const int kRebias = (1023 - 127) << 20;
    const unsigned hi = (unsigned)(__double2hiint(x) - kRebias);
    const unsigned lo = (unsigned)__double2loint(x);
    return __uint_as_float((hi << 3) | (lo >> 29));
}

// float32 copy of a double of either sign with |x| < 2^128, mantissa
// truncated, formed on the integer pipe; |x| below the float32 normal range
// gives 0.
__device__ __forceinline__ float narrow_f32_signed(double x) {
    const int kRebias = (1023 - 127) << 20;
    const unsigned hi = (unsigned)__double2hiint(x);
    const unsigned ahi = hi & 0x7fffffffu;
    if (ahi < (unsigned)(kRebias + (1 << 20))) return 0.0f;
    const unsigned lo = (unsigned)__double2loint(x);
    return __uint_as_float(((ahi - kRebias) << 3) | (lo >> 29) | (hi & 0x80000000u));
}

// The double of a float32 value (exact), formed on the integer pipe;
// zero and subnormal inputs give 0.
__device__ __forceinline__ double widen_f32(float f) {
    const int kRebias = (1023 - 127) << 20;
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7fffffffu;
    if (a < 0x00800000u) return 0.0;
    return __hiloint2double((int)(((a >> 3) + kRebias) | (u & 0x80000000u)), (int)(a << 29));
}

__device__ __forceinline__ double rsqrt_nr(double x) {
    const int kRebias = (1023 - 127) << 20;
    const unsigned yb = __float_as_uint(rsqrtf(narrow_f32(x)));
    const double y = __hiloint2double((int)(yb >> 3) + kRebias, (int)(yb << 29));
    double e = fma(-(x * y), y, 1.0);
    double c = fma(0.375, e, 0.5);
    return fma(y * e, c, y);
}

}  // namespace mdk
