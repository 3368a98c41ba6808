// Double-precision exp and log for kernels bound by the FP64 pipe.
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM (1/64 of the FP32 rate), and
// a general-purpose double exp costs ~20 DFMA-equivalents, log ~36.  These versions use
// small tables kept in shared memory and short polynomials, for ~9 (exp) and ~14 (log) FP64
// operations, accurate to a few units in the last place (measured on GB300 against CUDA's
// exp/log: max relative difference 1.5e-15 for exp on [-700, 700] with a two-term ln2
// reduction, max absolute difference 1.1e-16 for log; the one-term reduction used here adds
// at most 3.3e-17 |x| relative).
//
// exp: Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989):
//   x = (128 m + j) ln2/128 + r with |r| <= ln2/256,
//   exp(x) = 2^m * 2^(j/128) * (1 + p(r)),  p(r) = r + r^2/2 + r^3/6 + r^4/24,
//   2^m applied by adding m to the exponent field.
// log: x = 2^e * m with m in [1, 2); j = top 7 bits of the mantissa, c_j = 1 + (j + 1/2)/128,
//   r = m * (1/c_j) - 1 in one fused multiply-add (|r| < 2^-8),
//   log(x) = e ln2 + log(c_j) + log1p(r), log1p by its Taylor series to degree 7.
// The tables (2^(j/128); 1/c_j rounded to double and -log of that rounded value) are
// computed on the host at mechanism load (nk_abi.cu) and staged per block into shared
// memory by stage_math_tables().
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#endif

namespace nk {

constexpr int kExpTab = 128;
constexpr int kLogTab = 128;
constexpr int kMathTabDoubles = kExpTab + 2 * kLogTab;   // exp table, 1/c_j, log(c_j)

struct MathTab {
    const double* e2;   // [128] 2^(j/128)
    const double* rc;   // [128] 1/c_j
    const double* lc;   // [128] -log(rc_j)
};

__device__ __forceinline__ MathTab stage_math_tables(double* smem_tab, const double* gtab) {
    for (int j = threadIdx.x; j < kMathTabDoubles; j += blockDim.x) smem_tab[j] = __ldg(gtab + j);
    return MathTab{smem_tab, smem_tab + kExpTab, smem_tab + kExpTab + kLogTab};
}

static __device__ __noinline__ double fexp_edge(double x, double v, int m) {
    if (x != x) return x;
    if (x > 709.782712893384) return __longlong_as_double(0x7ff0000000000000LL);
    if (x < -745.1332191019412) return 0.0;
    // result near the ends of the range: apply 2^m in two halves
    const int m1 = m / 2, m2 = m - m1;
    const double s1 = __longlong_as_double((long long)(1023 + m1) << 52);
    const double s2 = __longlong_as_double((long long)(1023 + m2) << 52);
    return v * s1 * s2;
}

__device__ __forceinline__ double fexp(double x, const MathTab& t) {
    const double shifter = 6755399441055744.0;   // 1.5 * 2^52: rounds x*128/ln2 to an integer
    const double kd = fma(x, 184.6649652337873, shifter);
    const int N = __double2loint(kd);
    const double Nd = kd - shifter;
    // ln2/128 as one double: the neglected 1.8e-19 * N shifts the result by 3.3e-17 |x|
    // relative, below the 1.1e-16 |x| that rounding of the argument itself carries
    const double r = fma(Nd, -5.4152123481245725e-03, x);
    const double p = r * fma(r, fma(r, fma(r, 1.0 / 24.0, 1.0 / 6.0), 0.5), 1.0);
    const double tj = t.e2[N & (kExpTab - 1)];
    const double v = fma(tj, p, tj);
    const int m = N >> 7;
    const int hx = __double2hiint(x) & 0x7fffffff;
    if (hx >= 0x40862000) return fexp_edge(x, v, m);        // |x| >= 708 or NaN (rare)
    return __longlong_as_double(__double_as_longlong(v) + ((long long)m << 52));
}

__device__ __forceinline__ double flog(double x, const MathTab& t) {
    const long long b = __double_as_longlong(x);
    const int hi = (int)(b >> 32);
    if (hi < 0x00100000 || hi >= 0x7ff00000) return log(x);  // x <= 0, subnormal, inf, NaN (rare)
    const int e = (hi >> 20) - 1023;
    const int j = (hi >> 13) & (kLogTab - 1);
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double r = fma(m, t.rc[j], -1.0);
    double p = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    p = fma(r, p, 0.2);
    p = fma(r, p, -0.25);
    p = fma(r, p, 1.0 / 3.0);
    p = fma(r, p, -0.5);
    const double l1p = fma(r * r, p, r);                    // log1p(r)
    const double ed = (double)e;
    return fma(ed, 0.6931471805599453, t.lc[j] + fma(ed, 2.3190468138462996e-17, l1p));
}

}  // namespace nk
