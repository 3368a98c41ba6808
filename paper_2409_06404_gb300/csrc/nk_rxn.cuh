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

// c = beta + (Ea/R)/T = T d ln k / dT of reaction r (device order) as a pair
__device__ __forceinline__ dfl arrh_slope_df(const DevMech& m, int r, const TPairs& P) {
    const float4 a0 = __ldg(m.rxn_df + 2 * r), a1 = __ldg(m.rxn_df + 2 * r + 1);
    return df_fma(dfl{a1.x, a1.y}, P.invTd, dfl{a0.z, a0.w});
}

// ---------------------------------------------------------------- Troe falloff in pairs
// ln x for a pair x > 0: the pair logarithm for x.h in [2^-100, 2^100), the double log out of
// line otherwise (concentrations and falloff centres that small or large do not occur in the
// workloads; the edge keeps the result defined)
static __device__ __noinline__ dfl log_pair_edge(float h, float l) { return df_split_cvt(log((double)h + (double)l)); }
__device__ __forceinline__ dfl log_pos_pair(dfl x, const DfTab& dt) {
    if (!(x.h >= 7.888609052210118e-31f && x.h < 1.2676506002282294e30f)) return log_pair_edge(x.h, x.l);
    return log_df_pair(x, dt.rc, dt.lc);
}

// L = log10 F_cent and LT = T dL/dT of a Troe reaction, with
//   F_cent = (1 - a) exp(-T/T3) + a exp(-T/T1) + exp(-T2/T)     (the last term when T2 > 0),
//   T dF_cent/dT = -(1 - a)(T/T3) exp(-T/T3) - a (T/T1) exp(-T/T1) + (T2/T) exp(-T2/T),
// in pairs (terms below the float range drop out; an F_cent below 2^-100 takes the double
// edge path out of line).
struct TroeCent {
    dfl L, LT;
};
static __device__ __noinline__ TroeCent troe_cent_edge(const TroeRec* t, double T) {
    const double a = t->a, x3 = T * t->invT3, x1 = T * t->invT1, x2 = t->hasT2 != 0.0 ? t->T2 / T : 0.0;
    const double e3 = (1.0 - a) * exp(-x3), e1 = a * exp(-x1), e2 = t->hasT2 != 0.0 ? exp(-x2) : 0.0;
    const double Fc = e3 + e1 + e2, FT = e2 * x2 - e3 * x3 - e1 * x1;
    return TroeCent{df_split_cvt(log10(Fc)), df_split_cvt(FT / (Fc * 2.302585092994046))};
}
__device__ __forceinline__ TroeCent troe_cent(const DevMech& m, int aux, const TPairs& P, const DfTab& dt) {
    const float4 t1 = __ldg(m.troe_df + kTroeDf * aux + 1);    // (Ea0/R, 1/T3)
    const float4 t2 = __ldg(m.troe_df + kTroeDf * aux + 2);    // (1/T1, T2)
    const float4 t3 = __ldg(m.troe_df + kTroeDf * aux + 3);    // (a, 1 - a)
    const dfl x3 = df_mul(P.Td, dfl{t1.z, t1.w}), x1 = df_mul(P.Td, dfl{t2.x, t2.y});
    const dfl e3 = df_mul(dfl{t3.z, t3.w}, exp_df_pair(df_neg(x3), dt.e2));
    const dfl e1 = df_mul(dfl{t3.x, t3.y}, exp_df_pair(df_neg(x1), dt.e2));
    dfl Fc = df_add(e3, e1);
    dfl FT = df_neg(df_fma(e3, x3, df_mul(e1, x1)));
    if (t2.z != 0.0f) {
        const dfl x2 = df_mul(dfl{t2.z, t2.w}, P.invTd);
        const dfl e2 = exp_df_pair(df_neg(x2), dt.e2);
        Fc = df_add(Fc, e2);
        FT = df_fma(e2, x2, FT);
    }
    if (!(Fc.h >= 7.888609052210118e-31f)) return troe_cent_edge(m.troe + aux, P.T);
    return TroeCent{df_mul(log_df_pair(Fc, dt.rc, dt.lc), dfc_invln10()), df_mul(df_div(FT, Fc), dfc_invln10())};
}

// The Troe falloff factor in logarithmic form: for x = ln P_r and L = log10 F_cent,
//   u = x/ln10 - 0.4 - 0.67 L,  v = 0.75 - 1.27 L - 0.14 u,  f1 = u/v,
//   log10 F_T = L/(1 + f1^2),  ln F = ln(P_r/(1 + P_r)) + ln10 log10 F_T,
// and its partial derivatives Px = d ln F/dx = 1/(1 + P_r) + ln10 d log10 F_T/dx and
// PL = d ln F/dL = ln10 d log10 F_T/dL, from
//   d f1 = (du - f1 dv)/v,  d log10 F_T = (dL - 2 log10 F_T f1 d f1)/(1 + f1^2)
// with du/dx = 1/ln10, dv/dx = -0.14/ln10, du/dL = -0.67, dv/dL = -1.27 + 0.14 * 0.67.
// ln(P_r/(1 + P_r)) = -log(1 + e^-x) for x >= 0 and x - log(1 + e^x) below, from z = e^-|x|
// (z underflows to 0 past |x| = 87, dropping terms below 2^-125).  All in pairs.
struct TroeLog {
    dfl lnF, Px, PL;
};
__device__ __forceinline__ TroeLog troe_log(dfl x, dfl L, const DfTab& dt) {
    const dfl one{1.0f, 0.0f};
    const dfl u = df_add(df_fma(L, dfc_m0_67(), dfc_m0_4()), df_mul(x, dfc_invln10()));
    const dfl v = df_fma(u, dfc_m0_14(), df_fma(L, dfc_m1_27(), dfl{0.75f, 0.0f}));
    const dfl iv = df_div(one, v);
    const dfl f1 = df_mul(u, iv);
    const dfl iden = df_div(one, df_fma(f1, f1, one));
    const dfl lF = df_mul(L, iden);
    const dfl t = df_mul(df_mul(lF, f1), dfl{-2.0f, 0.0f});                              // -2 log10 F_T f1
    const dfl f1x = df_mul(df_mul(df_fma(f1, df_neg(dfc_m0_14()), one), iv), dfc_invln10());
    const dfl f1L = df_mul(df_fma(f1, dfl{1.17620003223419189453125f, -3.2234190427971043e-08f}, dfc_m0_67()), iv);
    const bool neg = x.h < 0.0f;
    const dfl z = exp_df_pair(neg ? x : df_neg(x), dt.e2);
    const dfl opz = df_add(one, z);
    const dfl s = log_df_pair(opz, dt.rc, dt.lc);
    TroeLog o;
    o.lnF = df_fma(lF, dfc_ln10(), neg ? df_add(x, df_neg(s)) : df_neg(s));
    o.Px = df_fma(df_mul(df_mul(t, f1x), iden), dfc_ln10(), df_div(neg ? one : z, opz));
    o.PL = df_mul(df_mul(df_fma(t, f1L, one), iden), dfc_ln10());
    return o;
}

// ln P_r = ln k_0 - ln k_inf + ln [M] of Troe reaction r (aux its Troe row) as a pair, with
// ln k_0 = ln A_0 + beta_0 ln T - (Ea_0/R)/T (+ the caller's shift of ln A) and the pair ln k_inf
// (which carries the same shift), for [M] > 0 as a pair; c0 = beta_0 + (Ea_0/R)/T.
__device__ __forceinline__ dfl troe_lnPr(const DevMech& m, int aux, const TPairs& P, dfl lnkinf, dfl shift,
                                         bool shifted, dfl Mp, const DfTab& dt, dfl* c0) {
    const float4 t0 = __ldg(m.troe_df + kTroeDf * aux);        // (lnA0, beta0)
    const float4 t1 = __ldg(m.troe_df + kTroeDf * aux + 1);    // (Ea0/R, 1/T3)
    dfl lnk0 = df_fma(dfl{t0.z, t0.w}, P.lnTd, dfl{t0.x, t0.y});
    lnk0 = df_fma(dfl{-t1.x, -t1.y}, P.invTd, lnk0);
    if (shifted) lnk0 = df_add(lnk0, shift);
    if (c0) *c0 = df_fma(dfl{t1.x, t1.y}, P.invTd, dfl{t0.z, t0.w});
    return df_add(df_add(lnk0, df_neg(lnkinf)), log_pos_pair(Mp, dt));
}

// sum_k nu_k of reaction r (device order) as a float, from the pair record (converting the
// double in the reaction record would take an F2F instruction on the FP64 pipe per reaction)
__device__ __forceinline__ float dnu_f(const DevMech& m, int r) {
    return __ldg(reinterpret_cast<const float*>(m.rxn_df + 2 * r + 1) + 2);
}

// sum_e nu_e l_e over one side of a reaction (ne entries, species sp[e], coefficients nu[e]) for
// pair values l_k at l[k * BLK]: the logarithm of a concentration product, or its tangent
template <int BLK>
__device__ __forceinline__ dfl side_sum_df(const float2* l, const int* sp, const int* nu, int ne) {
    dfl s = dfl_of(l[sp[0] * BLK]);
    if (nu[0] != 1) s = df_mul_f(s, (float)nu[0]);
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e)
        if (e < ne) {
            dfl t = dfl_of(l[sp[e] * BLK]);
            if (nu[e] != 1) t = df_mul_f(t, (float)nu[e]);
            s = df_add(s, t);
        }
    return s;
}

// w[sp[e] * BLK] += nud[e] q over one side's ne entries (1..kMaxSide).  A switch on the
// (warp-uniform) entry count, each case unrolled exactly: guarding an unrolled loop by e < ne
// instead leaves the compiler predicated FP64 instructions that occupy the FP64 pipe with every
// lane off (a third of the rates kernel's FP64-pipe time, measured).
template <int BLK, int N>
__device__ __forceinline__ void scatter_n(const int* sp, const double* nud, double* w, double q) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
        double* t = w + sp[e] * BLK;
        *t = fma(nud[e], q, *t);
    }
}
template <int BLK>
__device__ __forceinline__ void scatter_side(const int* sp, const double* nud, int ne, double* w, double q) {
    switch (ne) {
        case 1: scatter_n<BLK, 1>(sp, nud, w, q); break;
        case 2: scatter_n<BLK, 2>(sp, nud, w, q); break;
        case 3: scatter_n<BLK, 3>(sp, nud, w, q); break;
        default: scatter_n<BLK, kMaxSide>(sp, nud, w, q); break;
    }
}

// The logarithmic form holds for a mass fraction y when y is a positive double of at least
// 2^-100 (finite): its logarithm and the pair quotients dY/Y then stay within the float range of
// the pairs.  Integer operations on the exponent field.
__device__ __forceinline__ bool log_form_ok(double y) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(y);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    return (b >> 63) == 0 && e >= 1023u - 100u && e < 1023u + 100u;
}

// 1/y for a positive double within 2^+-100: the float reciprocal refined by one Newton step in
// double (relative error ~2^-46; two FP64 operations instead of a division)
__device__ __forceinline__ double recip_nr(double y) {
    const double r0 = widen(__frcp_rn(narrow(y)));
    return fma(r0, fma(-y, r0, 1.0), r0);
}

// sum_e nud[e] w[sp[e] * BLK] over one side's ne entries (1..kMaxSide), a switch on the count
// with each case unrolled exactly (as scatter_side)
template <int BLK, int N>
__device__ __forceinline__ double gather_n(const int* sp, const double* nud, const double* w) {
    double a = nud[0] * w[sp[0] * BLK];
#pragma unroll
    for (int e = 1; e < N; ++e) a = fma(nud[e], w[sp[e] * BLK], a);
    return a;
}
template <int BLK>
__device__ __forceinline__ double gather_side(const int* sp, const double* nud, int ne, const double* w) {
    switch (ne) {
        case 1: return gather_n<BLK, 1>(sp, nud, w);
        case 2: return gather_n<BLK, 2>(sp, nud, w);
        case 3: return gather_n<BLK, 3>(sp, nud, w);
        default: return gather_n<BLK, kMaxSide>(sp, nud, w);
    }
}
// |v| in [2^-100, 2^100) or v == 0 (a direction or cotangent value the pairs can carry)
__device__ __forceinline__ bool pair_range_ok(double v) {
    const unsigned e = (unsigned)(__double_as_longlong(v) >> 52) & 0x7ffu;
    return e == 0 ? (__double_as_longlong(v) << 1) == 0 : (e >= 1023u - 100u && e < 1023u + 100u);
}

// v / y within 2^+-120 (exponent fields; y a normal double, v == 0 allowed): the quotient a pair
// can carry
__device__ __forceinline__ bool quot_range_ok(double v, double y) {
    const int ev = (int)((__double_as_longlong(v) >> 52) & 0x7ff), ey = (int)((__double_as_longlong(y) >> 52) & 0x7ff);
    return ev == 0 ? (__double_as_longlong(v) << 1) == 0 : (ev - ey >= -120 && ev - ey <= 120);
}

// Part `part` of NP takes the contiguous slice [a + len*part/NP, a + len*(part+1)/NP) of the
// range [a, b).
template <int NP>
__device__ __forceinline__ void slice(int a, int b, int part, int& r0, int& r1) {
    const int len = b - a;
    r0 = a + (len * part) / NP;
    r1 = a + (len * (part + 1)) / NP;
}

// Part `part`'s reactions of kind g (0 elementary, 1 third-body, 2 Troe), round by round, for
// NP = 2 or 4 parts per point: f(r) for the part's reaction r of each round (none when the round
// leaves it idle), the block synchronised after every round.  Within a round the parts'
// reactions share no species (DevMech::rsched2/4), so they may add into one row per point.
// EFF: the VJP's schedule (the parts' reactions of a round also share no species with a
// third-body efficiency).
template <int NP, bool EFF = false, class Fn>
__device__ __forceinline__ void for_rounds(const DevMech& m, int g, int part, Fn&& f) {
    static_assert(NP == 2 || NP == 4, "reaction rounds exist for 2 and 4 parts");
    const int32_t* S = EFF ? (NP == 2 ? m.rschedv2 : m.rschedv4) : (NP == 2 ? m.rsched2 : m.rsched4);
    const int rd0 = EFF ? (NP == 2 ? m.rrndv2[g] : m.rrndv4[g]) : (NP == 2 ? m.rrnd2[g] : m.rrnd4[g]);
    const int rd1 = EFF ? (NP == 2 ? m.rrndv2[g + 1] : m.rrndv4[g + 1]) : (NP == 2 ? m.rrnd2[g + 1] : m.rrnd4[g + 1]);
    int r = rd0 < rd1 ? __ldg(S + rd0 * NP + part) : -1;
    for (int rd = rd0; rd < rd1; ++rd) {
        const int rn = rd + 1 < rd1 ? __ldg(S + (rd + 1) * NP + part) : -1;   // the next round's, early
        if (r >= 0) f(r);
        __syncthreads();
        r = rn;
    }
}

// As for_rounds (NP = 2 or 4, the rates kernel's schedule) for passes that read stored data per
// reaction: ld(r) issues the loads the reaction needs, ap(r, v) uses them; the part's next
// reaction's loads are issued before the current one is applied, so they stay in flight across
// the round's barrier.
template <int NP, class Ld, class Ap>
__device__ __forceinline__ void for_rounds_prefetch(const DevMech& m, int g, int part, Ld&& ld, Ap&& ap) {
    static_assert(NP == 2 || NP == 4, "reaction rounds exist for 2 and 4 parts");
    const int32_t* S = NP == 2 ? m.rsched2 : m.rsched4;
    const int rd0 = NP == 2 ? m.rrnd2[g] : m.rrnd4[g], rd1 = NP == 2 ? m.rrnd2[g + 1] : m.rrnd4[g + 1];
    if (rd0 >= rd1) return;
    using V = decltype(ld(0));
    int r = __ldg(S + rd0 * NP + part);
    V cur{};
    if (r >= 0) cur = ld(r);
    for (int rd = rd0; rd < rd1; ++rd) {
        const int rn = rd + 1 < rd1 ? __ldg(S + (rd + 1) * NP + part) : -1;
        V nxt{};
        if (rn >= 0) nxt = ld(rn);
        if (r >= 0) ap(r, cur);
        __syncthreads();
        r = rn;
        cur = nxt;
    }
}

}  // namespace nk
