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
// from long-double arithmetic: inv_l = 256/ln 2, l1 + l2 = ln 2 / 256 (l1 the
// nearest double, l2 the remainder).
struct ExpConst {
    double inv_l, l1, l2;
};

constexpr int kExpTable = 256;

// e^y by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989), with a 256-entry table:
//   n = round(y * 256/ln2), y = n ln2/256 + r, |r| <= ln2/512,
//   e^y = 2^(n >> 8) * 2^((n & 255)/256) * (1 + r + r^2/2 + r^3/6 + r^4/24),
// the neglected r^5/120 term is below 4e-17. The rounding to an integer uses
// the 1.5 * 2^52 shift (the integer lands in the low word); the reduction
// uses two fused multiply-adds with the two-part constant; the power of two
// is added to the exponent field. T[j] = 2^(j/256). Requires |y| < 700
// (callers guarantee it); 9 float64 instructions.
__device__ __forceinline__ double exp_tab(double y, const double* __restrict__ T, const ExpConst& K) {
    const double shift = 6755399441055744.0;  // 1.5 * 2^52
    double t = fma(y, K.inv_l, shift);
    int n = __double2loint(t);
    double nd = t - shift;
    double r = fma(-nd, K.l1, y);
    r = fma(-nd, K.l2, r);
    double r2 = r * r;
    double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r2, p, r);
    double tj = T[n & (kExpTable - 1)];
    double res = fma(tj, p, tj);
    return __hiloint2double(__double2hiint(res) + ((n >> 8) << 20), __double2loint(res));
}

// 1/sqrt(x) for x > 0 (normal, below float range): a float32 hardware
// estimate refined by one third-order Newton step,
//   e = 1 - x y^2,  y' = y (1 + e/2 + 3e^2/8),
// whose error is O(e^3) (~1e-20 for a float32 start), i.e. rounding-limited.
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y = (double)rsqrtf((float)x);
    double e = fma(-(x * y), y, 1.0);
    double c = fma(0.375, e, 0.5);
    return fma(y * e, c, y);
}

}  // namespace mdk
