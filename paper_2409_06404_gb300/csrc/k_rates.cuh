// Kernels of the net species production rates omega_k and heat release per point (the "rates" kernel of
// the paper, Tab. 3-4; omega_k of Eq. 1a, heat release of Eq. 1b).
//
// Layout: a point is worked on by NP warps ("parts"), one lane per point in each.  All lanes
// of a warp walk the same reaction at the same time, so reaction records are broadcast loads
// and control flow is uniform.  The device copy of the mechanism groups reactions by kind
// (elementary, third-body, Troe); each part walks its own contiguous slice of every kind.
// The per-point species state (C_k and g_k/RT, shared by the parts, and one row of omega_k
// partials per part) lives in shared memory as [species][point]; the partials are added in
// part order at the end.  NP and the points per block come from CUDA's occupancy calculator:
// shared memory per point bounds the resident warps, and splitting a point's reactions over
// warps raises them (5 -> 8 warps per SM at K = 53, 2 -> 4 at K = 120), which this
// latency-bound walk needs.
//
// Three arithmetic forms (template PREC):
//  kNative (NK_FP64_NATIVE): every operation in double (exp/log from nk_math.cuh), with the
//    per-species g_k/RT in shared memory.
//  kDF (NK_FP64): the exponent chains -- the reaction's Gibbs sum (from its thermo groups),
//    ln k_f, ln K_c, the Troe falloff -- in double-float pairs on the FP32 pipe (nk_df.cuh),
//    each exponential returned as a double with one FP64 add; the concentrations enter the
//    rate terms' exponents as pair logarithms (their signs beside them), and the rate terms,
//    the forward-minus-reverse difference and the omega accumulation stay in double.  Results
//    match the double-precision definition to ~1e-12 (the pairs carry 48 bits).
//  kMixed (NK_MIXED): the Arrhenius argument ln A + beta ln T - Ea/(RT), k_f and the whole
//    Troe falloff in single precision; the Gibbs sum and K_c as in the kDF form (pairs), the
//    forward-minus-reverse difference and the omega accumulation in double.
#pragma once

#include <mutex>
#include <utility>
#include <vector>

#include "nk_rxn.cuh"

namespace nk {
namespace {

enum { kNative = 0, kMixed = 1, kDF = 2 };

// Per-point quantities shared by all reactions.
struct Pt {
    double T, lnT, invT, pRT, lnP0RT;
    float Tf, lnTf, invTf;
    TPairs tp;                       // kDF form
    dfl pRTd;                        // kDF form: p/(RT) as a pair
};

// sum_k nu_k g_k/RT (products minus reactants) and the concentration products of each side;
// every reaction has at least one entry per side, which initialises the product.
template <int BLK>
__device__ __forceinline__ void gibbs_products(const Rxn& x, const double* sC, const double* sG, double& sumg,
                                               double& fw, double& rv) {
    {
        const int k = x.sp[0];
        const double c = sC[k * BLK];
        fw = c;
        for (int j = 1; j < x.nu[0]; ++j) fw *= c;
        sumg = x.nud[0] * sG[k * BLK];
    }
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e) {
        if (e < x.nr) {
            const int k = x.sp[e];
            const double c = sC[k * BLK];
            for (int j = 0; j < x.nu[e]; ++j) fw *= c;
            sumg = fma(x.nud[e], sG[k * BLK], sumg);
        }
    }
    {
        const int k = x.sp[kMaxSide];
        const double c = sC[k * BLK];
        rv = c;
        for (int j = 1; j < x.nu[kMaxSide]; ++j) rv *= c;
        sumg = fma(x.nud[kMaxSide], sG[k * BLK], sumg);
    }
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e) {
        if (e < x.np) {
            const int k = x.sp[kMaxSide + e];
            const double c = sC[k * BLK];
            for (int j = 0; j < x.nu[kMaxSide + e]; ++j) rv *= c;
            sumg = fma(x.nud[kMaxSide + e], sG[k * BLK], sumg);
        }
    }
}

// Troe falloff factor F * P_r/(1+P_r) in double precision, given ln k_inf, ln k_0 and [M].
__device__ __forceinline__ double troe_factor(const TroeRec* t, double lnkinf, double lnk0, double M, const Pt& P,
                                              const MathTab& mt) {
    const double lnPr = lnk0 - lnkinf + flog(M, mt);
    const double a = __ldg(&t->a);
    double Fc = (1.0 - a) * fexp(-P.T * __ldg(&t->invT3), mt) + a * fexp(-P.T * __ldg(&t->invT1), mt);
    if (__ldg(&t->hasT2) != 0.0) Fc += fexp(-__ldg(&t->T2) * P.invT, mt);
    const double lFc = flog(Fc, mt) * kInvLn10;
    const double c = fma(-0.67, lFc, -0.4);
    const double nn = fma(-1.27, lFc, 0.75);
    const double u = fma(lnPr, kInvLn10, c);
    const double f1 = u / fma(-0.14, u, nn);
    const double lF = lFc / fma(f1, f1, 1.0);
    return fexp(lF * kLn10, mt) / (1.0 + fexp(-lnPr, mt));   // P_r/(1+P_r) = 1/(1+1/P_r)
}

// Rate of progress q of one reaction of kind KIND (0 elementary, 1 third-body, 2 Troe);
// r is the reaction's position in the device order.  Native form: everything in double.
template <int BLK, int KIND>
__device__ __forceinline__ double rate_of_progress(const DevMech& m, const Rxn& x, const double* sC,
                                                   const double* sG, const Pt& P, const double* dlnA,
                                                   const MathTab& mt) {
    double sumg, fw, rv;
    gibbs_products<BLK>(x, sC, sG, sumg, fw, rv);
    const double lnKc = fma(x.dnu, P.lnP0RT, -sumg);   // ln K_c = -sum nu g/RT + sum nu ln(p0/RT)
    double lnA = x.lnA;                                  // ln A + shift (uniform branch)
    double shift = 0.0;
    if (dlnA) {
        shift = __ldg(dlnA + x.orig);
        lnA += shift;
    }
    double M = 0.0;
    if (KIND != 0) {
        M = P.pRT;                                       // sum_k C_k = p/(R T)
        for (int j = x.eff0; j < x.eff1; ++j) M = fma(__ldg(m.eff_m1 + j), sC[__ldg(m.eff_sp + j) * BLK], M);
    }
    double kf, kr;
    const double lnkf = fma(-x.EaR, P.invT, fma(x.beta, P.lnT, lnA));
    if constexpr (KIND == 2) {
        const TroeRec* t = m.troe + x.aux;
        const double lnk0 = fma(-__ldg(&t->Ea0R), P.invT, fma(__ldg(&t->beta0), P.lnT, __ldg(&t->lnA0) + shift));
        kf = M == 0.0 ? 0.0 : fexp(lnkf, mt) * troe_factor(t, lnkf, lnk0, M, P, mt);
        kr = kf * fexp(-lnKc, mt);
    } else {
        kf = fexp(lnkf, mt);
        kr = fexp(lnkf - lnKc, mt);
    }
    double q = fma(kf, fw, -kr * rv);
    if (KIND == 1) q *= M;
    return q;
}

// kDF form: the concentration products of each side in double (the Gibbs sum comes from the
// reaction's thermo groups).
template <int BLK>
__device__ __forceinline__ void products(const Rxn& x, const double* sC, double& fw, double& rv) {
    {
        const double c = sC[x.sp[0] * BLK];
        fw = c;
        for (int j = 1; j < x.nu[0]; ++j) fw *= c;
    }
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e)
        if (e < x.nr) {
            const double c = sC[x.sp[e] * BLK];
            for (int j = 0; j < x.nu[e]; ++j) fw *= c;
        }
    {
        const double c = sC[x.sp[kMaxSide] * BLK];
        rv = c;
        for (int j = 1; j < x.nu[kMaxSide]; ++j) rv *= c;
    }
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e)
        if (e < x.np) {
            const double c = sC[x.sp[kMaxSide + e] * BLK];
            for (int j = 0; j < x.nu[kMaxSide + e]; ++j) rv *= c;
        }
}

// Logarithmic form of the concentration products (kDF and kMixed forms).  The C_k row holds
// ln |C_k| as pairs (a zero concentration as -2^100, whose exponential is 0), and each side's
// product enters its rate term through the exponent:
//   q_f = exp(ln k_f + sum_reactants nu ln C),  q_r = exp(ln k_f - ln K_c + sum_products nu ln C),
// one pair exponential each (as k_f and k_r alone took), so no concentration product is formed
// in double: the FP64 pipe keeps the exponentials' final additions, the forward-minus-reverse
// difference, [M] and the scatter.  A negative concentration (a negative mass fraction) enters
// by its magnitude, with its sign in a byte row beside the logarithms (SG, the kernel's second
// pass): a side's product changes sign with every factor of odd exponent that is negative, and
// [M] takes the signed C_j.

// the sign of one side's concentration product: 1 if an odd number of its factors (counted with
// their integer exponents) are negative
template <int BLK>
__device__ __forceinline__ int side_sign(const uint8_t* sg, const int* sp, const int* nu, int ne) {
    int s = sg[sp[0] * BLK] & nu[0];
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e)
        if (e < ne) s ^= sg[sp[e] * BLK] & nu[e];
    return s & 1;
}

// [M] = p/(RT) + sum (eps - 1) C_j as a pair from the logarithms ln |C_j| (and, SG, the signs;
// terms below the float range drop out: they are under 1e-37 against p/(RT))
template <int BLK, bool SG>
__device__ __forceinline__ dfl third_body_pair(const DevMech& m, const Rxn& x, const float2* sL, const uint8_t* sg,
                                               const Pt& P, const DfTab& dt) {
    dfl M = P.pRTd;
    for (int j = x.eff0; j < x.eff1; ++j) {
        const int k = __ldg(m.eff_sp + j);
        dfl c = exp_df_pair(dfl_of(sL[k * BLK]), dt.e2);
        if (SG && sg[k * BLK]) c = df_neg(c);
        M = df_fma(dfl_of(__ldg(m.df_eff_m1 + j)), c, M);
    }
    return M;
}

// FP64 form.  The exponent of each rate term, ln k_f (+ ln F, the Troe falloff factor, whose
// whole chain runs in pairs: troe_log) + the concentration logarithms - ln K_c, in pairs; the
// terms (signed by the sides' concentration signs, SG), their difference and the [M] factor of
// third-body reactions in double.
template <int BLK, int KIND, bool SG>
__device__ __forceinline__ double rate_of_progress_df(const DevMech& m, const Rxn& x, int r, const float2* sL,
                                                      const uint8_t* sg, const Pt& P, const double* dlnA,
                                                      const DfTab& dt) {
    dfl sumg, unused_h, unused_cp;
    rxn_thermo<false, false>(m, x.thermo, P.tp, sumg, unused_h, unused_cp);
    const dfl lnKc = df_add(df_mul_f(P.tp.lnP0RTd, dnu_f(m, r)), df_neg(sumg));   // ln K_c
    dfl shift{0.0f, 0.0f};
    if (dlnA) shift = df_split(__ldg(dlnA + x.orig));
    const dfl lnkf = ln_kf_df(m, r, P.tp, shift, dlnA != nullptr);
    double M = 0.0;
    dfl Mp{0.0f, 0.0f};
    if constexpr (KIND != 0) {
        Mp = third_body_pair<BLK, SG>(m, x, sL, sg, P, dt);
        if (KIND == 1) M = df_to_d(Mp);
    }
    dfl lnkF = lnkf;                                             // ln k_f + ln F
    bool noF = false;                                            // Troe with [M] = 0: no rate
    if constexpr (KIND == 2) {
        if (Mp.h == 0.0f) {
            noF = true;
        } else {
            const dfl lnPr = troe_lnPr(m, x.aux, P.tp, lnkf, shift, dlnA != nullptr, Mp, dt, nullptr);
            lnkF = df_add(lnkf, troe_log(lnPr, troe_cent(m, x.aux, P.tp, dt).L, dt).lnF);
        }
    }
    const dfl sf = side_sum_df<BLK>(sL, x.sp, x.nu, x.nr);
    const dfl sb = side_sum_df<BLK>(sL, x.sp + kMaxSide, x.nu + kMaxSide, x.np);
    double qf = exp_df_d(df_add(lnkF, sf), dt.e2), qr = exp_df_d(df_add(df_add(lnkF, df_neg(lnKc)), sb), dt.e2);
    if constexpr (SG) {
        if (side_sign<BLK>(sg, x.sp, x.nu, x.nr)) qf = -qf;
        if (side_sign<BLK>(sg, x.sp + kMaxSide, x.nu + kMaxSide, x.np)) qr = -qr;
    }
    double q = qf - qr;
    if (KIND == 2 && noF) q = 0.0;
    if (KIND == 1) q *= M;
    return q;
}

// Mixed form: k_f and the whole Troe falloff in single precision; the Gibbs sum and K_c from
// the reaction's thermo groups in pairs, the exponent sums of the rate terms in pairs (the
// single-precision ln k_f enters both terms alike, so q keeps the FP64 difference of
// K_c-consistent terms), the difference in double.
template <int BLK, int KIND, bool SG>
__device__ __forceinline__ double rate_of_progress_mixed(const DevMech& m, const Rxn& x, int r, const float2* sL,
                                                         const uint8_t* sg, const Pt& P, const double* dlnA,
                                                         const DfTab& dt) {
    dfl sumg, unused_h, unused_cp;
    rxn_thermo<false, false>(m, x.thermo, P.tp, sumg, unused_h, unused_cp);
    const dfl lnKc = df_add(df_mul_f(P.tp.lnP0RTd, dnu_f(m, r)), df_neg(sumg));   // ln K_c
    const float shf = dlnA ? (float)__ldg(dlnA + x.orig) : 0.0f;
    double M = 0.0;                                              // [M] in double (third-body rows)
    float Mf = 0.0f;                                             // and in float (the falloff)
    if constexpr (KIND != 0) {
        const dfl Mp = third_body_pair<BLK, SG>(m, x, sL, sg, P, dt);
        Mf = Mp.h;
        if (KIND == 1) M = df_to_d(Mp);
    }
    const float4 xf = __ldg(reinterpret_cast<const float4*>(m.rxnf + r));   // lnA, beta, EaR
    const float lnkf = fmaf(-xf.z, P.invTf, fmaf(xf.y, P.lnTf, xf.x + shf));
    float Ff = 1.0f;                                             // Troe: F P_r/(1 + P_r)
    if constexpr (KIND == 2) {
        const float4 t0 = __ldg(reinterpret_cast<const float4*>(m.troef + x.aux));       // lnA0, beta0, Ea0R, a
        const float4 t1 = __ldg(reinterpret_cast<const float4*>(m.troef + x.aux) + 1);   // 1/T3, 1/T1, T2, has
        if (Mf == 0.0f) {
            Ff = 0.0f;
        } else {
            const float lnk0 = fmaf(-t0.z, P.invTf, fmaf(t0.y, P.lnTf, t0.x + shf));
            const float lnPr = lnk0 - lnkf + logf(Mf);
            float Fc = (1.0f - t0.w) * expf(-P.Tf * t1.x) + t0.w * expf(-P.Tf * t1.y);
            if (t1.w != 0.0f) Fc += expf(-t1.z * P.invTf);
            const float lFc = log10f(Fc);
            const float c = fmaf(-0.67f, lFc, -0.4f);
            const float nn = fmaf(-1.27f, lFc, 0.75f);
            const float u = fmaf(lnPr, (float)kInvLn10, c);
            const float f1 = u / fmaf(-0.14f, u, nn);
            const float lF = lFc / fmaf(f1, f1, 1.0f);
            Ff = exp10f(lF) / (1.0f + expf(-lnPr));
        }
    }
    const dfl lkf{lnkf, 0.0f};
    const dfl sf = side_sum_df<BLK>(sL, x.sp, x.nu, x.nr);
    const dfl sb = side_sum_df<BLK>(sL, x.sp + kMaxSide, x.nu + kMaxSide, x.np);
    double qf = exp_df_d(df_add(lkf, sf), dt.e2), qr = exp_df_d(df_add(df_add(lkf, df_neg(lnKc)), sb), dt.e2);
    if constexpr (SG) {
        if (side_sign<BLK>(sg, x.sp, x.nu, x.nr)) qf = -qf;
        if (side_sign<BLK>(sg, x.sp + kMaxSide, x.nu + kMaxSide, x.np)) qr = -qr;
    }
    double q = qf - qr;
    if (KIND == 2) q *= widen(Ff);
    if (KIND == 1) q *= M;
    return q;
}

template <int BLK>
__device__ __forceinline__ void scatter(const Rxn& x, double* sW, double q) {
    scatter_side<BLK>(x.sp, x.nud, x.nr, sW, q);
    scatter_side<BLK>(x.sp + kMaxSide, x.nud + kMaxSide, x.np, sW, q);
}

template <int BLK, int PREC, int KIND, bool SG>
__device__ __forceinline__ double q_of(const DevMech& m, const Rxn& x, int r, const double* sC, const double* sG,
                                       const uint8_t* sg, const Pt& P, const double* dlnA, const MathTab& mt,
                                       const DfTab& dt) {
    const float2* sL = reinterpret_cast<const float2*>(sC);
    if constexpr (PREC == kDF)
        return rate_of_progress_df<BLK, KIND, SG>(m, x, r, sL, sg, P, dlnA, dt);
    else if constexpr (PREC == kMixed)
        return rate_of_progress_mixed<BLK, KIND, SG>(m, x, r, sL, sg, P, dlnA, dt);
    else
        return rate_of_progress<BLK, KIND>(m, x, sC, sG, P, dlnA, mt);
}

// Reactions [r0, r1) of one kind, scattered in reaction order (one part per point).
// (Unrolling by two or four reactions per iteration measured slower once several warps share a
// point.)  SG: the concentrations' signs enter (kDF and kMixed, second pass).
template <int BLK, int PREC, int KIND, bool SG>
__device__ __forceinline__ void reaction_group(const DevMech& m, int r0, int r1, const double* sC, const double* sG,
                                               double* sW, const uint8_t* sg, const Pt& P, const double* dlnA,
                                               const MathTab& mt, const DfTab& dt) {
    for (int r = r0; r < r1; ++r) {
        const Rxn a = load_rxn(m.rxn + r);
        scatter<BLK>(a, sW, q_of<BLK, PREC, KIND, SG>(m, a, r, sC, sG, sg, P, dlnA, mt, dt));
    }
}

// The reactions of one kind for NP > 1 parts per point, round by round (for_rounds): the parts'
// reactions of a round share no species, so all scatter into the point's one omega_k row.
template <int BLK, int NP, int PREC, int KIND, bool SG>
__device__ __forceinline__ void reaction_rounds(const DevMech& m, int part, const double* sC, const double* sG,
                                                double* sW, const uint8_t* sg, const Pt& P, const double* dlnA,
                                                const MathTab& mt, const DfTab& dt) {
    for_rounds<NP>(m, KIND, part, [&](int r) {
        const Rxn a = load_rxn(m.rxn + r);
        scatter<BLK>(a, sW, q_of<BLK, PREC, KIND, SG>(m, a, r, sC, sG, sg, P, dlnA, mt, dt));
    });
}

// Per-point species arrays: C_k, then g_k/RT (native form only), then the omega_k row.
template <int PREC>
__host__ __device__ constexpr int shared_rows() {
    return PREC == kNative ? 2 : 1;
}

// BLK points per block, NP parts (warps) per point: thread (part, slot) works on point
// blockIdx.x * BLK + slot.  The parts of a point share its C_k (and g_k/RT) and its omega_k row;
// they take the reactions in rounds whose reactions share no species (for_rounds), so every
// omega_k is summed in an order fixed by the mechanism's schedule, whatever the scheduling of
// the warps.
//
// RHS: write the implicit-stage sources instead: omega -> W_k omega_k / rho, hrr -> hrr/(rho c_p).
//
// PASS (kDF and kMixed): 0 takes the blocks without a negative concentration and skips the
// others, 1 takes only those, with the concentrations' signs in a byte row after the omega_k row
// (rates_smem_signs); so the common pass carries no sign work.  The second pass leaves at once
// where no mass fraction of the block is negative.  The native form has one pass (0) over every
// block.
template <int BLK, int NP, int PREC, bool RHS, int PASS>
__global__ void __launch_bounds__(BLK * NP, (PREC != kNative ? 768 : 640) / (BLK * NP))
    rates_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                         const double* __restrict__ T, const double* __restrict__ p,
                                                         const double* __restrict__ Y,
                                                         const double* __restrict__ dlnA,
                                                         double* __restrict__ omega, double* __restrict__ hrr) {
    extern __shared__ double smem[];
    MathTab mt{};
    DfTab dt{};
    if constexpr (PREC == kNative)
        mt = stage_math_tables(smem, m.mtab);
    else
        dt = stage_df_tables(reinterpret_cast<float2*>(smem), m);
    __syncthreads();
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no block barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;         // idle slots of the last block recompute point n-1
    if constexpr (PREC != kNative && PASS == 1) {
        // no negative mass fraction and positive T and p in the block (its warp for NP = 1): no
        // concentration is negative (rho > 0), the logarithmic pass took it; anything else goes
        // on to the exact vote below
        bool anyneg = !(T[i] > 0.0 && p[i] > 0.0);
        for (int k = part; k < K; k += NP) anyneg |= Y[(int64_t)k * ld + i] < 0.0;
        const bool some = NP > 1 ? __syncthreads_or(anyneg) != 0 : __any_sync(__activemask(), anyneg);
        if (!some) return;
    }
    double* sC = smem + kMathTabDoubles + slot;                       // C_k       at sC[k * BLK]
    double* sG = smem + kMathTabDoubles + (size_t)K * BLK + slot;     // g_k / RT (native form)
    double* sW0 = smem + kMathTabDoubles + (size_t)shared_rows<PREC>() * K * BLK + slot;
    double* sW = sW0;                                                  // omega_k
    constexpr bool SG = PREC != kNative && PASS == 1;
    uint8_t* sg = reinterpret_cast<uint8_t*>(sW0 - slot + (size_t)K * BLK) + slot;   // (SG) sign of C_k

    Pt P;
    P.T = T[i];
    P.invT = 1.0 / P.T;
    P.pRT = p[i] * P.invT * kInvR;                     // p/(RT) = sum_k C_k
    if constexpr (PREC == kNative) {
        P.lnT = flog(P.T, mt);
        P.lnP0RT = kLnP0overR - P.lnT;                 // ln(p0/(R T))
    } else {
        P.tp = make_tpairs(P.T, P.invT, dt);
        P.Tf = P.tp.Td.h;
        P.lnTf = P.tp.lnTd.h + P.tp.lnTd.l;
        P.invTf = P.tp.invTd.h;
        P.pRTd = df_split(P.pRT);
    }
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double rho_w = P.pRT / s;                    // rho = p Wbar/(RT) with Wbar = 1/s
    bool neg = false;
    for (int k = part; k < K; k += NP) {
        const double c = Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * rho_w;   // C_k = rho Y_k / W_k
        if constexpr (PREC == kNative) {
            sC[k * BLK] = c;
            sG[k * BLK] = nasa_gRT(nasa_range(m, k, P.T), P.T, P.lnT, P.invT);
        } else {
            // ln |C_k| as a pair in the C_k row (zero: -2^100), and in the second pass its sign
            neg |= c < 0.0;
            const dfl l = c == 0.0 ? dfl{-0x1p100f, 0.0f} : log_df(SG ? fabs(c) : c, dt.rc, dt.lc);
            reinterpret_cast<float2*>(sC)[k * BLK] = make_float2(l.h, l.l);
            if constexpr (SG) sg[k * BLK] = c < 0.0;
        }
    }
    for (int k = part; k < K; k += NP) sW[k * BLK] = 0.0;
    bool vote = false;
    if constexpr (NP > 1) {
        if constexpr (PREC == kNative)
            __syncthreads();
        else
            vote = __syncthreads_or(neg) != 0;
    } else if constexpr (PREC != kNative) {
        vote = __any_sync(__activemask(), neg);
    }
    if constexpr (PREC != kNative) {
        if (PASS == 0 ? vote : !vote) return;     // the other pass takes this block
    }

    if constexpr (NP == 1) {
        const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
        reaction_group<BLK, PREC, 0, SG>(m, 0, e1, sC, sG, sW, sg, P, dlnA, mt, dt);
        reaction_group<BLK, PREC, 1, SG>(m, e1, t1, sC, sG, sW, sg, P, dlnA, mt, dt);
        reaction_group<BLK, PREC, 2, SG>(m, t1, m.R, sC, sG, sW, sg, P, dlnA, mt, dt);
    } else {
        // (each round ends with a barrier: the omega_k row is complete after the last one)
        reaction_rounds<BLK, NP, PREC, 0, SG>(m, part, sC, sG, sW, sg, P, dlnA, mt, dt);
        reaction_rounds<BLK, NP, PREC, 1, SG>(m, part, sC, sG, sW, sg, P, dlnA, mt, dt);
        reaction_rounds<BLK, NP, PREC, 2, SG>(m, part, sC, sG, sW, sg, P, dlnA, mt, dt);
    }

    // omega_k (or the source W_k omega_k / rho), sum_k h_k/RT omega_k and, for the sources,
    // c_p/R = sum_k Y_k/W_k c_p,k/R of this part's species
    double h = 0.0, cpm = 0.0, inv_rho = 0.0;
    if constexpr (RHS) inv_rho = 1.0 / rho_w;
    for (int k = part; k < K; k += NP) {
        double w = sW0[k * BLK];
        const double* c = nasa_range(m, k, P.T);
        h = fma(nasa_hRT(c, P.T, P.invT), w, h);
        if constexpr (RHS) {
            cpm = fma(Y[(int64_t)k * ld + i] * __ldg(m.invW + k), nasa_cpR(c, P.T), cpm);
            w *= __ldg(m.W + k) * inv_rho;
        }
        if (live) omega[(int64_t)k * ld + i] = w;
    }
    if constexpr (NP > 1) {
        // C_k is dead: rows q (and NP + q for the sources; (1 + RHS) NP <= K) take part q's
        // sums, added in part order
        sC[part * BLK] = h;
        if constexpr (RHS) sC[(NP + part) * BLK] = cpm;
        __syncthreads();
        if (part != 0) return;
        h = sC[0];
        if constexpr (RHS) cpm = sC[NP * BLK];
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            h += sC[q * BLK];
            if constexpr (RHS) cpm += sC[(NP + q) * BLK];
        }
    }
    const double hr = -kR * P.T * h;                   // heat release -sum_k h_k omega_k
    if constexpr (RHS) {
        if (live) hrr[i] = hr * inv_rho / (kR * cpm);  // dT/dt = hrr / (rho c_p)
    } else {
        if (live) hrr[i] = hr;
    }
}

struct Shape {
    int blk, np;
};

// Launch shapes the library instantiates (points per block, parts per point).
constexpr Shape kShapes[] = {{32, 1}, {64, 1}, {128, 1}, {32, 2}, {64, 2}, {32, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <int PREC, bool RHS, int S, int PASS = 0>
constexpr auto kernel_of() {
    return rates_kernel<kShapes[S].blk, kShapes[S].np, PREC, RHS, PASS>;
}

template <int PREC, bool RHS, int... S>
const void* kernel_ptr(int idx, std::integer_sequence<int, S...>) {
    const void* ptrs[] = {(const void*)kernel_of<PREC, RHS, S>()...};
    return ptrs[idx];
}

// Shared bytes of a block: the staged tables, then the per-point species arrays; the second pass
// adds the byte row of the concentrations' signs.
template <int PREC>
size_t rates_smem(int K, const Shape& sh) {
    return (size_t)kMathTabDoubles * sizeof(double) +
           (size_t)(shared_rows<PREC>() + 1) * K * sh.blk * sizeof(double);
}
inline size_t rates_smem_signs(int K, const Shape& sh) { return ((size_t)K * sh.blk + 7) / 8 * 8; }

// The shape's first pass, then (kDF, kMixed) its second pass on the same stream.
template <int PREC, bool RHS, int... S>
cudaError_t launch_idx(int idx, std::integer_sequence<int, S...>, const DevMech& m, int64_t n, int64_t ld,
                       const double* T, const double* p, const double* Y, const double* dlnA, double* omega,
                       double* hrr, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaErrorInvalidConfiguration;
    ((S == idx ? (void)(e = [&] {
        constexpr Shape sh = kShapes[S];
        const unsigned grid = (unsigned)((n + sh.blk - 1) / sh.blk);
        auto kern = kernel_of<PREC, RHS, S, 0>();
        cudaError_t r = ensure_smem((const void*)kern, smem);
        if (r != cudaSuccess) return r;
        kern<<<grid, sh.blk * sh.np, smem, st>>>(m, n, ld, T, p, Y, dlnA, omega, hrr);
        r = cudaGetLastError();
        if (r != cudaSuccess || PREC == kNative) return r;
        auto kern1 = kernel_of<PREC, RHS, S, 1>();
        const size_t smem1 = smem + rates_smem_signs(m.K, sh);
        r = ensure_smem((const void*)kern1, smem1);
        if (r != cudaSuccess) return r;
        kern1<<<grid, sh.blk * sh.np, smem1, st>>>(m, n, ld, T, p, Y, dlnA, omega, hrr);
        return cudaGetLastError();
    }())
               : (void)0),
     ...);
    return e;
}


// The shape with the most resident warps per SM (CUDA's occupancy calculator: shared memory,
// registers, threads), fewer parts on ties.  Cached per
// (device, K, form).
struct Plan {
    int dev, K, prec, rhs, idx;
};
std::mutex g_plan_mu;
std::vector<Plan> g_plans;

template <int PREC, bool RHS>
int plan_shape(int K) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const Plan& q : g_plans)
            if (q.dev == dev && q.K == K && q.prec == PREC && q.rhs == (int)RHS) return q.idx;
    }
    int per_block = 0;
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const auto seq = std::make_integer_sequence<int, kNumShapes>{};
    int best = -1, best_warps = 0;
    for (int c = 0; c < kNumShapes; ++c) {
        const Shape& sh = kShapes[c];
        if ((RHS ? 2 : 1) * sh.np > K && sh.np > 1) continue;
        const size_t bytes = rates_smem<PREC>(K, sh);
        if (bytes > (size_t)per_block) continue;
        const void* kern = kernel_ptr<PREC, RHS>(c, seq);
        if (ensure_smem(kern, bytes) != cudaSuccess) continue;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, sh.blk * sh.np, bytes) != cudaSuccess)
            continue;
        const int warps = blocks * sh.blk * sh.np / 32;
        if (warps > best_warps) {
            best_warps = warps;
            best = c;
        }
    }
    if (best >= 0) {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        g_plans.push_back({dev, K, PREC, (int)RHS, best});
    }
    return best;
}

template <int PREC, bool RHS>
cudaError_t launch_form(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                        const double* dlnA, double* omega, double* hrr, cudaStream_t s) {
    const int idx = plan_shape<PREC, RHS>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx<PREC, RHS>(idx, std::make_integer_sequence<int, kNumShapes>{}, m, n, ld, T, p, Y, dlnA, omega,
                                 hrr, rates_smem<PREC>(m.K, kShapes[idx]), s);
}

}  // namespace

}  // namespace nk
