// Device pieces shared by the reaction kernels (rates, JVP, VJP): the reaction record as the
// kernels hold it, the double-float tables and constants, the per-point temperature terms and
// the reaction thermo groups (sum_k nu_k g_k/RT, h_k/RT, c_p,k/R of one reaction; see
// kGrpPairs in nk_internal.cuh).
#pragma once

#include "nk_internal.cuh"

namespace nk {

constexpr double kLnP0overR = 9.408091968961747;   // ln(101325 Pa / (8.314462618 J/mol/K))

// double constants of the definitions as float pairs (hi = nearest float, lo = remainder)
__device__ __forceinline__ dfl dfc_lnp0r() { return {9.40809154510498f, 4.2385676124467864e-07f}; }
__device__ __forceinline__ dfl dfc_invln10() { return {0.4342944920063019f, -1.0103049952192578e-08f}; }
__device__ __forceinline__ dfl dfc_ln10() { return {2.3025851249694824f, -3.1975435632602967e-08f}; }
__device__ __forceinline__ dfl dfc_m0_4() { return {-0.4000000059604645f, 5.9604645663569045e-09f}; }
__device__ __forceinline__ dfl dfc_m0_67() { return {-0.6700000166893005f, 1.668930060816365e-08f}; }
__device__ __forceinline__ dfl dfc_m1_27() { return {-1.2699999809265137f, -1.907348590179936e-08f}; }
__device__ __forceinline__ dfl dfc_m0_14() { return {-0.14000000059604645f, 5.9604643443123e-10f}; }
__device__ __forceinline__ dfl dfl_of(float2 v) { return {v.x, v.y}; }

// a pair as a double: both halves widened by integer operations, one FP64 add
__device__ __forceinline__ double df_to_d(dfl a) { return f2d_bits(a.h) + f2d_bits(a.l); }

// double-float tables staged in shared memory
struct DfTab {
    const float2* e2;   // 2^(j/128)
    const float2* rc;   // 1/c_j
    const float2* lc;   // -log(1/c_j)
};

// Stage the three 128-entry pair tables (3 KB) at `t`; the caller synchronises.
__device__ __forceinline__ DfTab stage_df_tables(float2* t, const DevMech& m) {
    for (int j = threadIdx.x; j < kExpTab; j += blockDim.x) {
        t[j] = __ldg(m.df_exp_tab + j);
        t[kExpTab + j] = __ldg(m.df_log_rc + j);
        t[2 * kExpTab + j] = __ldg(m.df_log_lc + j);
    }
    return DfTab{t, t + kExpTab, t + 2 * kExpTab};
}
constexpr size_t kDfTabBytes = 3 * kExpTab * sizeof(float2);

// exp and log of doubles through the pair routines (relative error ~1e-13 for the moderate
// arguments of the falloff terms)
__device__ __forceinline__ double dexp_df(double x, const DfTab& dt) { return exp_df_d(df_split(x), dt.e2); }
__device__ __forceinline__ double dlog_df(double x, const DfTab& dt) { return df_to_d(log_df(x, dt.rc, dt.lc)); }

struct Rxn {
    double lnA, beta, EaR, dnu;
    double nud[2 * kMaxSide];
    int type, nr, np, aux, orig, eff0, eff1, thermo;
    int sp[2 * kMaxSide];
    int nu[2 * kMaxSide];
};

__device__ __forceinline__ Rxn load_rxn(const RxnRec* rec) {
    Rxn x;
    const double2* d = reinterpret_cast<const double2*>(rec);
    const double2 a = __ldg(d), b = __ldg(d + 1);
    x.lnA = a.x;
    x.beta = a.y;
    x.EaR = b.x;
    x.dnu = b.y;
#pragma unroll
    for (int j = 0; j < kMaxSide; ++j) {
        const double2 v = __ldg(d + 2 + j);
        x.nud[2 * j] = v.x;
        x.nud[2 * j + 1] = v.y;
    }
    const int4* q = reinterpret_cast<const int4*>(rec) + 6;
    const int4 h = __ldg(q), h2 = __ldg(q + 1), s0 = __ldg(q + 2), s1 = __ldg(q + 3), u0 = __ldg(q + 4),
               u1 = __ldg(q + 5);
    x.type = h.x;
    x.nr = h.y;
    x.np = h.z;
    x.aux = h.w;
    x.orig = h2.x;
    x.eff0 = h2.y;
    x.eff1 = h2.z;
    x.thermo = h2.w;
    x.sp[0] = s0.x; x.sp[1] = s0.y; x.sp[2] = s0.z; x.sp[3] = s0.w;
    x.sp[4] = s1.x; x.sp[5] = s1.y; x.sp[6] = s1.z; x.sp[7] = s1.w;
    x.nu[0] = u0.x; x.nu[1] = u0.y; x.nu[2] = u0.z; x.nu[3] = u0.w;
    x.nu[4] = u1.x; x.nu[5] = u1.y; x.nu[6] = u1.z; x.nu[7] = u1.w;
    return x;
}

// Temperature terms of a point as pairs.
struct TPairs {
    double T;
    dfl Td, invTd, lnTd, omlnTd, lnP0RTd;   // T, 1/T, ln T, 1 - ln T, ln(p0/(R T))
};

__device__ __forceinline__ TPairs make_tpairs(double T, double invT, const DfTab& dt) {
    TPairs P;
    P.T = T;
    P.Td = df_split(T);
    P.invTd = df_split(invT);
    P.lnTd = log_df(T, dt.rc, dt.lc);
    P.omlnTd = df_add(dfl{1.0f, 0.0f}, df_neg(P.lnTd));
    P.lnP0RTd = df_add(dfc_lnp0r(), df_neg(P.lnTd));
    return P;
}

// Thermo sums of one reaction (kGrpPairs layout): g = sum nu g/RT always; h = sum nu h/RT when
// H; cp = sum nu c_p/R when CP.
template <bool H, bool CP>
__device__ __forceinline__ void rxn_thermo(const DevMech& m, int thermo, const TPairs& P, dfl& g, dfl& h, dfl& cp) {
    const int g0 = thermo & 0xffffff, ng = thermo >> 24;
    g = h = cp = dfl{0.0f, 0.0f};
    for (int j = 0; j < ng; ++j) {
        const int grp = g0 + j;
        // T <= T_mid on the bit patterns (T_mid > 0: signed 64-bit order is the order of the
        // doubles; NaN T takes the high range as the double comparison would)
        const bool lo = __double_as_longlong(P.T) <= __ldg(reinterpret_cast<const long long*>(m.grp_Tmid) + grp);
        const float4* c4 = reinterpret_cast<const float4*>(m.grp_df + ((size_t)grp * 2 + (lo ? 0 : 1)) * kGrpPairs);
        float2 c[kGrpPairs];
#pragma unroll
        for (int v = 0; v < kGrpPairs / 2; ++v) {
            const float4 w = __ldg(c4 + v);
            c[2 * v] = make_float2(w.x, w.y);
            c[2 * v + 1] = make_float2(w.z, w.w);
        }
        dfl a = dfl_of(c[4]);
        a = df_fma(a, P.Td, dfl_of(c[3]));
        a = df_fma(a, P.Td, dfl_of(c[2]));
        a = df_fma(a, P.Td, dfl_of(c[1]));
        a = df_mul(a, P.Td);
        a = df_fma(dfl_of(c[0]), P.omlnTd, a);
        a = df_fma(dfl_of(c[5]), P.invTd, a);
        a = df_add(a, dfl_of(c[6]));
        g = j == 0 ? a : df_add(g, a);
        if (H) {
            dfl b = dfl_of(c[11]);
            b = df_fma(b, P.Td, dfl_of(c[10]));
            b = df_fma(b, P.Td, dfl_of(c[9]));
            b = df_fma(b, P.Td, dfl_of(c[8]));
            b = df_fma(b, P.Td, dfl_of(c[7]));
            b = df_fma(dfl_of(c[12]), P.invTd, b);
            h = j == 0 ? b : df_add(h, b);
        }
        if (CP) {
            dfl e = dfl_of(c[17]);
            e = df_fma(e, P.Td, dfl_of(c[16]));
            e = df_fma(e, P.Td, dfl_of(c[15]));
            e = df_fma(e, P.Td, dfl_of(c[14]));
            e = df_fma(e, P.Td, dfl_of(c[13]));
            cp = j == 0 ? e : df_add(cp, e);
        }
    }
}

// ln k_f = ln A + beta ln T - (Ea/R)/T of reaction r (device order) as a pair, with the
// caller's ln A shift.
__device__ __forceinline__ dfl ln_kf_df(const DevMech& m, int r, const TPairs& P, const dfl& shift, bool shifted) {
    const float4 a0 = __ldg(m.rxn_df + 2 * r), a1 = __ldg(m.rxn_df + 2 * r + 1);
    dfl l = df_fma(dfl{a0.z, a0.w}, P.lnTd, dfl{a0.x, a0.y});
    l = df_fma(dfl{-a1.x, -a1.y}, P.invTd, l);
    return shifted ? df_add(l, shift) : l;
}

// sum_k nu_k of reaction r (device order) as a float, from the pair record (converting the
// double in the reaction record would take an F2F instruction on the FP64 pipe per reaction)
__device__ __forceinline__ float dnu_f(const DevMech& m, int r) {
    return __ldg(reinterpret_cast<const float*>(m.rxn_df + 2 * r + 1) + 2);
}

// Part `part` of NP takes the contiguous slice [a + len*part/NP, a + len*(part+1)/NP) of the
// range [a, b).
template <int NP>
__device__ __forceinline__ void slice(int a, int b, int part, int& r0, int& r1) {
    const int len = b - a;
    r0 = a + (len * part) / NP;
    r1 = a + (len * (part + 1)) / NP;
}

}  // namespace nk
