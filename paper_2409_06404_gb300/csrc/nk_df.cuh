// Double-float ("f32x2") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, carrying 48
// significand bits (relative rounding ~2^-46 per operation for the add/multiply below).
// On GB300 the FP32 pipe retires ~58x more operations per clock than the FP64 pipe, so sums
// of positive, bounded terms -- the transport pair sums -- are evaluated here at FP64-class
// accuracy.  The error-free transformations are the classical ones: Knuth's two-sum,
// Dekker's fast two-sum (|a| >= |b|), and the FMA two-product (exact product a*b = p + e).
// Every step uses round-to-nearest intrinsics so the compiler cannot contract or reorder
// the compensation terms.
#pragma once

#include <cuda_runtime.h>

namespace nk {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {   // requires |a| >= |b| (or a == 0)
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a double as a pair with the conversion instructions (F2F, on the FP64 pipe)
__device__ __forceinline__ dfl df_split_cvt(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
static __device__ __noinline__ dfl df_split_edge(double x) { return df_split_cvt(x); }

// float of a double's bits whose low 29 significand bits are zero and whose exponent lies in
// the normal float range (exact: sign, rebiased exponent, top 23 significand bits)
__device__ __forceinline__ float d2f_exact_bits(unsigned long long u) {
    return __uint_as_float(((unsigned int)(u >> 32) & 0x80000000u) | (((unsigned int)(u >> 52) & 0x7ffu) - 896u) << 23 |
                           ((unsigned int)(u >> 29) & 0x7fffffu));
}

// a double as a pair by integer operations: h = x rounded to 24 significant bits on its bit
// pattern (half-way cases away from zero), l = x - h (exact in double) rounded the same way.
// For 2^-73 <= |x| < 2^127, where any nonzero l is a normal float; other x (zero, tiny, huge,
// non-finite) take the conversion instructions out of line.  This keeps the FP64 pipe to the
// one subtraction.
__device__ __forceinline__ dfl df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int e = (unsigned int)(b >> 52) & 0x7ffu;
    if (e < 1023u - 73u || e > 1023u + 126u) return df_split_edge(x);
    constexpr unsigned long long kHalf = 1ULL << 28, kMask = ~((1ULL << 29) - 1);
    const unsigned long long hb = (b + kHalf) & kMask;           // a carry may raise the exponent by one
    const double ld = x - __longlong_as_double((long long)hb);
    const unsigned long long lb = (unsigned long long)__double_as_longlong(ld);
    const float l = (lb << 1) == 0 ? 0.0f : d2f_exact_bits((lb + kHalf) & kMask);
    return {d2f_exact_bits(hb), l};
}

__device__ __forceinline__ double df_value(dfl a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    dfl s = two_sum(x.h, y.h);
    s.l = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return fast_two_sum(p, e);
}

// s + a * x
__device__ __forceinline__ dfl df_fma(dfl a, dfl x, dfl s) {
    const float p = __fmul_rn(a.h, x.h);
    float e = __fmaf_rn(a.h, x.h, -p);
    e = __fmaf_rn(a.h, x.l, __fmaf_rn(a.l, x.h, e));
    dfl u = two_sum(s.h, p);
    u.l = __fadd_rn(u.l, __fadd_rn(e, s.l));
    return fast_two_sum(u.h, u.l);
}

// x / y (y > 0): quotient of the high parts, corrected once by the pair residual
__device__ __forceinline__ dfl df_div(dfl x, dfl y) {
    const float q1 = __fdiv_rn(x.h, y.h);
    const float p = __fmul_rn(q1, y.h);
    float e = __fmaf_rn(q1, y.h, -p);
    e = __fmaf_rn(q1, y.l, e);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p), e), x.l);
    return fast_two_sum(q1, __fdiv_rn(r, y.h));
}

// a * 2^m for |m| <= 126 (exact)
__device__ __forceinline__ dfl df_ldexp(dfl a, int m) {
    const float s = __int_as_float((m + 127) << 23);
    return {__fmul_rn(a.h, s), __fmul_rn(a.l, s)};
}

// exp(x) for a double-float x with |x| <= 22, by Tang's table-driven method in pairs:
//   x = (128 m + j) ln2/128 + r, |r| <= ln2/256, ln2/128 split into three floats (the first
//   with 12 significant bits, so N * C1 is exact for |N| < 2^12);
//   exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24 with r and r^2/2 carried in pairs and the two
//   small terms in float; result 2^m * T_j * (1 + (exp(r) - 1)), T_j = 2^(j/128) as a pair.
//   Relative error <= 3.2e-14 on [-22, 22] (checked against 200-bit exp).
__device__ __forceinline__ dfl df_exp(dfl x, const float2* tab) {
    constexpr float kInvC = 184.6649652337873f;          // 128 / ln2
    constexpr float C1 = 5.4149627685546875e-03f;        // ln2/128, 12 significant bits
    constexpr float C2 = 2.495795570212067e-07f;         // next 24 bits
    constexpr float C3 = 1.2864023201156725e-14f;        // remainder
    // N = nearest integer to x.h * 128/ln2 by the 1.5 * 2^23 shifter (|N| < 2^22), read from
    // the float's bits: FP32 and integer pipe only
    const float kd = __fmaf_rn(x.h, kInvC, 12582912.0f);
    const int N = __float_as_int(kd) - 0x4B400000;
    const float Nf = __fsub_rn(kd, 12582912.0f);
    const float rh = __fmaf_rn(-Nf, C1, x.h);            // exact
    const float p2 = __fmul_rn(-Nf, C2);
    const float p2e = __fmaf_rn(-Nf, C2, -p2);
    dfl r = two_sum(rh, p2);
    r.l = __fadd_rn(r.l, __fadd_rn(__fadd_rn(x.l, p2e), __fmul_rn(-Nf, C3)));
    r = fast_two_sum(r.h, r.l);
    // r^2/2 as a pair, then the float tail
    const float q = __fmul_rn(r.h, r.h);
    float qe = __fmaf_rn(r.h, r.h, -q);
    qe = __fmaf_rn(2.0f * r.h, r.l, qe);
    const float tail = __fmul_rn(__fmul_rn(q, r.h), __fmaf_rn(r.h, 1.0f / 24.0f, 1.0f / 6.0f));
    dfl em1 = two_sum(r.h, 0.5f * q);
    em1.l = __fadd_rn(em1.l, __fadd_rn(r.l, __fmaf_rn(0.5f, qe, tail)));
    em1 = fast_two_sum(em1.h, em1.l);
    const float2 t = tab[N & 127];
    const dfl tj{t.x, t.y};
    const dfl v = df_fma(tj, em1, tj);
    return df_ldexp(v, N >> 7);
}

// ------------------------------------------------------------------ conversions by integer ops
// The F2F conversion instructions run at the FP64 rate on GB300; rebuilding the bit pattern
// with integer operations keeps them off the FP64 pipe.  Normal floats and zero only (a
// subnormal float converts to a signed zero; the kernels never produce one that matters).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)sign);
    const unsigned long long bits =
        sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// A float widened to double with integer operations.  Exact for normal floats, infinities and
// NaN; a subnormal float (|f| < 1.2e-38) becomes a signed zero.
__device__ __forceinline__ double widen(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long ee = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
    const unsigned long long bits = e == 0u ? sign : sign | (ee << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// A double rounded to float with integer operations (half-way cases away from zero).  Results
// in the normal float range are correctly rounded otherwise; |x| < 2^-126 gives a signed zero
// (no subnormals), larger than the float range gives +-inf, NaN stays NaN.
__device__ __forceinline__ float narrow(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned int e = (unsigned int)(b >> 52) & 0x7ffu;
    if (e < 897u) return __uint_as_float(sign);
    if (e > 1150u) return __uint_as_float(sign | 0x7f800000u | (e == 0x7ffu && (b << 12) != 0 ? 0x400000u : 0u));
    return d2f_exact_bits((b + (1ULL << 28)) & ~((1ULL << 29) - 1));   // a carry at the top rounds to inf
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

// x * s for a float s (pair result)
__device__ __forceinline__ dfl df_mul_f(dfl x, float s) {
    const float p = __fmul_rn(x.h, s);
    float e = __fmaf_rn(x.h, s, -p);
    e = __fmaf_rn(x.l, s, e);
    return fast_two_sum(p, e);
}

// ---------------------------------------------------------------- exp / log over the full range
// exp(x) returned in double for a pair x with |x| < 708 (NaN and larger |x| fall back to the
// double exp of x.h + x.l).  Same method as df_exp with ln2/128 split as C1 (7 significant
// bits, so N*C1 is exact for |N| < 2^17) + C2 + C3; the pair T_j (1 + (e^r - 1)) in [1, 2)
// becomes a double with one FP64 add and 2^m goes into the exponent field.  Relative error
// <= 1.7e-13 for |x| <= 100, 2.2e-12 at |x| = 700 (the pair carries x to 2^-48 |x|).
// Out of line, so the rare paths' conversions to double stay off the common path.
static __device__ __noinline__ double exp_df_d_edge(float h, float l) { return exp((double)h + (double)l); }
static __device__ __noinline__ dfl log_df_edge(double x) { return df_split_cvt(log(x)); }

// The common part: exp(x) = v 2^(N >> 7) with the pair v = T_j (1 + (e^r - 1)) in [1, 2).
__device__ __forceinline__ dfl exp_df_core(dfl x, const float2* tab, int& N) {
    constexpr float kInvC = 184.6649652337873f;          // 128 / ln2
    constexpr float C1 = 5.43212890625e-03f;
    constexpr float C2 = -1.691655779723078e-05f;
    constexpr float C3 = -3.281964814933619e-13f;
    // N = nearest integer to x.h * 128/ln2 by the 1.5 * 2^23 shifter (|N| < 2^22), read from
    // the float's bits: FP32 and integer pipe only
    const float kd = __fmaf_rn(x.h, kInvC, 12582912.0f);
    N = __float_as_int(kd) - 0x4B400000;
    const float Nf = __fsub_rn(kd, 12582912.0f);
    const float rh = __fmaf_rn(-Nf, C1, x.h);            // exact
    const float p2 = __fmul_rn(-Nf, C2);
    const float p2e = __fmaf_rn(-Nf, C2, -p2);
    dfl r = two_sum(rh, p2);
    r.l = __fadd_rn(r.l, __fadd_rn(__fadd_rn(x.l, p2e), __fmul_rn(-Nf, C3)));
    r = fast_two_sum(r.h, r.l);
    const float q = __fmul_rn(r.h, r.h);
    float qe = __fmaf_rn(r.h, r.h, -q);
    qe = __fmaf_rn(2.0f * r.h, r.l, qe);
    const float tail = __fmul_rn(__fmul_rn(q, r.h), __fmaf_rn(r.h, 1.0f / 24.0f, 1.0f / 6.0f));
    dfl em1 = two_sum(r.h, 0.5f * q);
    em1.l = __fadd_rn(em1.l, __fadd_rn(r.l, __fmaf_rn(0.5f, qe, tail)));
    em1 = fast_two_sum(em1.h, em1.l);
    const float2 t = tab[N & 127];
    const dfl tj{t.x, t.y};
    return df_fma(tj, em1, tj);
}

__device__ __forceinline__ double exp_df_d(dfl x, const float2* tab) {
    if (!(fabsf(x.h) < 708.0f)) return exp_df_d_edge(x.h, x.l);
    int N;
    const dfl v = exp_df_core(x, tab, N);
    const double d = f2d_bits(v.h) + f2d_bits(v.l);     // the one FP64 operation
    return __longlong_as_double(__double_as_longlong(d) + ((long long)(N >> 7) << 52));
}

// exp(x) as a pair, for results in the normal float range: 0 below it (x < -87), +inf above it
// (x >= 88) and NaN for NaN.  No FP64 operation.
__device__ __forceinline__ dfl exp_df_pair(dfl x, const float2* tab) {
    if (!(x.h > -87.0f && x.h < 88.0f)) {
        const float z = x.h > 0.0f ? __int_as_float(0x7f800000) : 0.0f;
        return x.h != x.h ? dfl{x.h, x.h} : dfl{z, 0.0f};
    }
    int N;
    const dfl v = exp_df_core(x, tab, N);
    return df_ldexp(v, N >> 7);
}

// log(2^e m) for a pair m in about [1, 2) (m.h in [1, 2)) whose top 7 fraction bits are j: the
// part of log_df after the decomposition, shared with log_df_pair
__device__ __forceinline__ dfl log_df_tail(dfl m, int e, int j, const float2* rc, const float2* lc) {
    const float2 rcj = rc[j];
    dfl r = df_mul(m, dfl{rcj.x, rcj.y});
    r = df_add(r, dfl{-1.0f, 0.0f});
    const float q = __fmul_rn(r.h, r.h);
    float qe = __fmaf_rn(r.h, r.h, -q);
    qe = __fmaf_rn(2.0f * r.h, r.l, qe);
    const float P = __fmaf_rn(r.h, __fmaf_rn(r.h, __fmaf_rn(r.h, __fmaf_rn(r.h, 1.0f / 7.0f, -1.0f / 6.0f), 0.2f),
                                             -0.25f), 1.0f / 3.0f);
    const float cub = __fmul_rn(__fmul_rn(q, r.h), P);
    dfl l1 = two_sum(r.h, -0.5f * q);
    l1.l = __fadd_rn(l1.l, __fadd_rn(r.l, __fmaf_rn(-0.5f, qe, cub)));
    l1 = fast_two_sum(l1.h, l1.l);
    const float ef = (float)e;
    constexpr float LN2H = 0.693147182464599609375f, LN2L = -1.9046542121259336e-09f;
    const float p = __fmul_rn(ef, LN2H);
    float pe = __fmaf_rn(ef, LN2H, -p);
    pe = __fmaf_rn(ef, LN2L, pe);
    const dfl el = two_sum(p, pe);
    const float2 lcj = lc[j];
    return df_add(df_add(el, dfl{lcj.x, lcj.y}), l1);
}

// log(x) as a pair for a positive normal double x (others fall back to the double log):
// x = 2^e m, j = top 7 bits of m, r = m / c_j - 1 with the pair 1/c_j, log1p(r) with r and
// r^2/2 in pairs and the cubic tail in float, plus e ln2 and log(c_j) as pairs.  Absolute
// error ~1e-14 for |log x| <= 10, 5e-12 at |log x| = 700.
__device__ __forceinline__ dfl log_df(double x, const float2* rc, const float2* lc) {
    const long long b = __double_as_longlong(x);
    const int hi = (int)(b >> 32);
    if (hi < 0x00100000 || hi >= 0x7ff00000) return log_df_edge(x);
    const int e = (hi >> 20) - 1023;
    const int j = (hi >> 13) & 127;
    const unsigned long long mant = (unsigned long long)b & 0x000fffffffffffffULL;
    const dfl m{__uint_as_float(0x3f800000u | (unsigned int)(mant >> 29)),
                (float)(unsigned int)(mant & 0x1fffffffULL) * 2.220446049250313e-16f};   // * 2^-52
    return log_df_tail(m, e, j, rc, lc);
}

// log(x) as a pair for a pair x with x.h in [2^-126, 2^126): x = 2^e m with m = x 2^-e exact
// (m.h in [1, 2)), then the steps of log_df.  No FP64 operation.
__device__ __forceinline__ dfl log_df_pair(dfl x, const float2* rc, const float2* lc) {
    const unsigned int b = __float_as_uint(x.h);
    const int e = (int)((b >> 23) & 0xffu) - 127;
    const float s = __uint_as_float((unsigned int)(127 - e) << 23);     // 2^-e
    const dfl m{__uint_as_float((b & 0x7fffffu) | 0x3f800000u), __fmul_rn(x.l, s)};
    return log_df_tail(m, e, (int)((b >> 16) & 127u), rc, lc);
}

}  // namespace nk
