// Kernels of the exact Jacobian-vector product of (omega_k, heat release) with respect to (T, Y_k) at fixed
// p: the product the Newton-GMRES stage of the paper approximates by difference quotients
// (Sec. 2, Sec. 4).  Forward-mode differentiation written out by hand, rates of progress
// recomputed in registers (nothing per reaction is stored).
//
// Tangents: with y_k = Y_k/W_k, s = sum y_k, rho = p/(R T s), C_k = rho y_k:
//   d rho/rho = -dT/T - ds/s,  dC_k = C_k d rho/rho + rho dY_k/W_k,
//   d ln k_f = (beta + Ea/(R T)) dT/T,
//   d ln K_c = (dT/T) (sum_k nu_k h_k/RT - sum_k nu_k)     (d(g/RT)/dT = -(h/RT)/T),
// Troe: d ln k = d ln k_inf + d ln P_r/(1+P_r) + ln10 d log10 F with F from the chain rule
// through F_cent(T), c, n, f1.  Heat release is accumulated per reaction, which needs no
// omega_k storage:
//   hrr = -R T sum_r q_r (sum_k nu_kr h_k/RT),
//   d hrr = -R sum_r [dT q_r (sum_k nu_kr c_p,k/R) + T dq_r (sum_k nu_kr h_k/RT)].
//
// FP64 form as the rates kernel: the exponent chains (ln k_f, the reaction's Gibbs and
// enthalpy sums, ln K_c) in double-float pairs on the FP32 pipe, concentrations, their
// products and every tangent in double.  The falloff chain runs in double with pair-based
// exp/log.  Layout as the rates kernel: NP warps per point share C_k and dC_k in shared
// memory and its d omega_k (and omega_k when asked for) rows, into which they scatter in rounds
// of reactions that share no species (for_rounds): every sum in an order fixed by the schedule.
#pragma once

#include <mutex>
#include <utility>
#include <vector>

#include "nk_rxn.cuh"

namespace nk {
namespace {

struct JvpPoint {
    TPairs P;
    double invT, lnT, tT, dT, pRT, dpRT, arho;   // arho = d rho / rho
    dfl tTd, pRTd, dpRTd;                        // the logarithmic form's pairs
};

struct JvpAcc {
    double h = 0.0;    // sum_r q_r dH_r/RT
    double cp = 0.0;   // sum_r q_r dCp_r/R
    double dh = 0.0;   // sum_r dq_r dH_r/RT
};

template <int BLK, int KIND, bool OMEGA, bool RHS>
__device__ __forceinline__ void jvp_reaction(const DevMech& m, int r, const double* sC, const double* sdC, double* sW,
                                             double* sD, const JvpPoint& Q, const double* dlnA, const DfTab& dt,
                                             JvpAcc& acc) {
    const Rxn x = load_rxn(m.rxn + r);
    double fw, dfw, rv, drv;                      // dual-number concentration products
    {
        const int k = x.sp[0];
        const double c = sC[k * BLK], dc = sdC[k * BLK];
        fw = c;
        dfw = dc;
        for (int j = 1; j < x.nu[0]; ++j) {
            dfw = fma(dfw, c, fw * dc);
            fw *= c;
        }
    }
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e)
        if (e < x.nr) {
            const int k = x.sp[e];
            const double c = sC[k * BLK], dc = sdC[k * BLK];
            for (int j = 0; j < x.nu[e]; ++j) {
                dfw = fma(dfw, c, fw * dc);
                fw *= c;
            }
        }
    {
        const int k = x.sp[kMaxSide];
        const double c = sC[k * BLK], dc = sdC[k * BLK];
        rv = c;
        drv = dc;
        for (int j = 1; j < x.nu[kMaxSide]; ++j) {
            drv = fma(drv, c, rv * dc);
            rv *= c;
        }
    }
#pragma unroll
    for (int e = 1; e < kMaxSide; ++e)
        if (e < x.np) {
            const int k = x.sp[kMaxSide + e];
            const double c = sC[k * BLK], dc = sdC[k * BLK];
            for (int j = 0; j < x.nu[kMaxSide + e]; ++j) {
                drv = fma(drv, c, rv * dc);
                rv *= c;
            }
        }
    dfl dG, dH, dCp;
    rxn_thermo<true, true>(m, x.thermo, Q.P, dG, dH, dCp);
    const double sumh = df_to_d(dH), sumcp = df_to_d(dCp);
    const dfl lnKc = df_add(df_mul_f(Q.P.lnP0RTd, dnu_f(m, r)), df_neg(dG));
    const double dlnKc = Q.tT * (sumh - x.dnu);

    double shift = 0.0;
    dfl shiftd{0.0f, 0.0f};
    if (dlnA) {
        shift = __ldg(dlnA + x.orig);
        shiftd = df_split(shift);
    }
    const dfl lnkf = ln_kf_df(m, r, Q.P, shiftd, dlnA != nullptr);
    double dlnkf = fma(x.EaR, Q.invT, x.beta) * Q.tT;

    double M = 0.0, dM = 0.0;
    if (KIND != 0) {
        M = Q.pRT;
        dM = Q.dpRT;
        for (int j = x.eff0; j < x.eff1; ++j) {
            const int k = __ldg(m.eff_sp + j);
            const double em1 = __ldg(m.eff_m1 + j);
            M = fma(em1, sC[k * BLK], M);
            dM = fma(em1, sdC[k * BLK], dM);
        }
    }
    double kf, kr;
    if constexpr (KIND == 2) {
        if (M == 0.0) {
            kf = kr = 0.0;
            dlnkf = 0.0;
        } else {
            const TroeRec* t = m.troe + x.aux;
            const double beta0 = __ldg(&t->beta0), Ea0R = __ldg(&t->Ea0R);
            const double lnk0 = fma(-Ea0R, Q.invT, fma(beta0, Q.lnT, __ldg(&t->lnA0) + shift));
            const double dlnk0 = fma(Ea0R, Q.invT, beta0) * Q.tT;
            const double lnPr = lnk0 - df_to_d(lnkf) + dlog_df(M, dt);
            const double dlnPr = dlnk0 - dlnkf + dM / M;
            const double a = __ldg(&t->a), i3 = __ldg(&t->invT3), i1 = __ldg(&t->invT1);
            const double e3 = dexp_df(-Q.P.T * i3, dt), e1 = dexp_df(-Q.P.T * i1, dt);
            double Fc = (1.0 - a) * e3 + a * e1;
            double dFc = -((1.0 - a) * i3 * e3 + a * i1 * e1) * Q.dT;
            if (__ldg(&t->hasT2) != 0.0) {
                const double T2 = __ldg(&t->T2), e2 = dexp_df(-T2 * Q.invT, dt);
                Fc += e2;
                dFc = fma(T2 * Q.invT * e2, Q.tT, dFc);
            }
            const double lFc = dlog_df(Fc, dt) * kInvLn10, dlFc = dFc / Fc * kInvLn10;
            const double c = fma(-0.67, lFc, -0.4), nn = fma(-1.27, lFc, 0.75);
            const double u = fma(lnPr, kInvLn10, c), du = fma(dlnPr, kInvLn10, -0.67 * dlFc);
            const double v = fma(-0.14, u, nn), dv = fma(-0.14, du, -1.27 * dlFc);
            const double f1 = u / v, df1 = fma(-f1, dv, du) / v;
            const double den = fma(f1, f1, 1.0);
            const double lF = lFc / den;
            const double dlF = fma(-2.0 * lF * f1, df1, dlFc) / den;
            const double g = 1.0 / (1.0 + dexp_df(-lnPr, dt));       // P_r / (1 + P_r)
            kf = exp_df_d(lnkf, dt.e2) * g * dexp_df(lF * kLn10, dt);
            dlnkf = dlnkf + dlnPr * (1.0 - g) + kLn10 * dlF;
            kr = kf * exp_df_d(df_neg(lnKc), dt.e2);
        }
    } else {
        kf = exp_df_d(lnkf, dt.e2);
        kr = exp_df_d(df_add(lnkf, df_neg(lnKc)), dt.e2);
    }
    const double dkf = kf * dlnkf, dkr = kr * (dlnkf - dlnKc);
    double q = fma(kf, fw, -kr * rv);
    double dq = fma(dkf, fw, kf * dfw) - fma(dkr, rv, kr * drv);
    if (KIND == 1) {
        dq = fma(dq, M, q * dM);
        q *= M;
    }
    // the sources' tangent W_k (d omega_k - omega_k d rho/rho) / rho is linear in the
    // reactions: scatter dq - q d rho/rho and no omega_k row is needed
    const double dqs = RHS ? fma(-Q.arho, q, dq) : dq;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.nr) {
            const int k = x.sp[e];
            sD[k * BLK] = fma(x.nud[e], dqs, sD[k * BLK]);
            if (OMEGA) sW[k * BLK] = fma(x.nud[e], q, sW[k * BLK]);
        }
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.np) {
            const int k = x.sp[kMaxSide + e];
            sD[k * BLK] = fma(x.nud[kMaxSide + e], dqs, sD[k * BLK]);
            if (OMEGA) sW[k * BLK] = fma(x.nud[kMaxSide + e], q, sW[k * BLK]);
        }
    if constexpr (OMEGA || RHS) acc.h = fma(q, sumh, acc.h);     // the primal heat release
    acc.cp = fma(q, sumcp, acc.cp);
    acc.dh = fma(dq, sumh, acc.dh);
}

// The logarithmic form (blocks whose mass fractions are all at least 2^-100 and whose direction
// the pairs can carry; see the kernel).  The point's rows hold ln C_k and r_k = dC_k/C_k =
// d rho/rho + dY_k/Y_k as pairs, and with F the falloff factor (1 but for Troe reactions)
//   q_f = exp(ln k_f + ln F + sum_reac nu ln C),   q_r = exp(ln k_f + ln F - ln K_c + sum_prod nu ln C),
//   dq  = q_f (d ln k_f + d ln F + sum_reac nu r) - q_r (d ln k_f + d ln F - d ln K_c + sum_prod nu r),
// the exponent and tangent sums (with the whole falloff chain) in pairs; the exponentials'
// results, the difference, dq, [M] scaling, the scatter and the heat-release sums in double.
// No concentration product is formed.
template <int BLK, int KIND, bool OMEGA, bool RHS>
__device__ __forceinline__ void jvp_reaction_log(const DevMech& m, int r, const float2* sL, const float2* sR,
                                                 double* sW, double* sD, const JvpPoint& Q, const double* dlnA,
                                                 const DfTab& dt, JvpAcc& acc) {
    const Rxn x = load_rxn(m.rxn + r);
    const dfl sf = side_sum_df<BLK>(sL, x.sp, x.nu, x.nr);
    const dfl sb = side_sum_df<BLK>(sL, x.sp + kMaxSide, x.nu + kMaxSide, x.np);
    const dfl gf = side_sum_df<BLK>(sR, x.sp, x.nu, x.nr);
    const dfl gb = side_sum_df<BLK>(sR, x.sp + kMaxSide, x.nu + kMaxSide, x.np);
    dfl dG, dH, dCp;
    rxn_thermo<true, true>(m, x.thermo, Q.P, dG, dH, dCp);
    const float dnu = dnu_f(m, r);
    const dfl lnKc = df_add(df_mul_f(Q.P.lnP0RTd, dnu), df_neg(dG));
    dfl shiftd{0.0f, 0.0f};
    if (dlnA) shiftd = df_split(__ldg(dlnA + x.orig));
    const dfl lnkf = ln_kf_df(m, r, Q.P, shiftd, dlnA != nullptr);
    const dfl dlnkf = df_mul(arrh_slope_df(m, r, Q.P), Q.tTd);                               // (beta + Ea/RT) dT/T
    const dfl dlnKc = df_mul(Q.tTd, df_add(dH, dfl{-dnu, 0.0f}));                            // (sum nu h/RT - sum nu) dT/T

    double M = 0.0, dM = 0.0;
    dfl Mp{0.0f, 0.0f}, dMp{0.0f, 0.0f};
    if (KIND != 0) {
        Mp = Q.pRTd;
        dMp = Q.dpRTd;
        for (int j = x.eff0; j < x.eff1; ++j) {
            const int k = __ldg(m.eff_sp + j);
            const dfl ec = df_mul(dfl_of(__ldg(m.df_eff_m1 + j)), exp_df_pair(dfl_of(sL[k * BLK]), dt.e2));
            Mp = df_add(Mp, ec);
            dMp = df_fma(ec, dfl_of(sR[k * BLK]), dMp);
        }
        if (KIND == 1) {
            M = df_to_d(Mp);
            dM = df_to_d(dMp);
        }
    }
    // Troe: ln F and its tangent in pairs, folded into the exponents and the tangent sums
    //   d ln F = Px d ln P_r + PL dL,  d ln P_r = (c0 - c1) dT/T + d[M]/[M],  dL = LT dT/T
    dfl lnF{0.0f, 0.0f}, dlnF{0.0f, 0.0f};
    bool noF = false;                             // [M] = 0: no falloff term
    if constexpr (KIND == 2) {
        if (Mp.h == 0.0f) {
            noF = true;
        } else {
            dfl c0;
            const dfl lnPr = troe_lnPr(m, x.aux, Q.P, lnkf, shiftd, dlnA != nullptr, Mp, dt, &c0);
            const TroeCent c = troe_cent(m, x.aux, Q.P, dt);
            const TroeLog f = troe_log(lnPr, c.L, dt);
            lnF = f.lnF;
            const dfl dx = df_add(df_add(df_mul(c0, Q.tTd), df_neg(dlnkf)), df_div(dMp, Mp));
            dlnF = df_fma(f.Px, dx, df_mul(f.PL, df_mul(c.LT, Q.tTd)));
        }
    }
    const dfl lnkF = KIND == 2 ? df_add(lnkf, lnF) : lnkf;
    const dfl dlnkF = KIND == 2 ? df_add(dlnkf, dlnF) : dlnkf;
    double qf = exp_df_d(df_add(lnkF, sf), dt.e2);
    double qr = exp_df_d(df_add(df_add(lnkF, df_neg(lnKc)), sb), dt.e2);
    const double Gf = df_to_d(df_add(dlnkF, gf));
    const double Gb = df_to_d(df_add(df_add(dlnkF, df_neg(dlnKc)), gb));
    if (KIND == 2 && noF) qf = qr = 0.0;
    double q = qf - qr;
    double dq = fma(qf, Gf, -qr * Gb);
    if (KIND == 1) {
        dq = fma(dq, M, q * dM);
        q *= M;
    }
    const double dqs = RHS ? fma(-Q.arho, q, dq) : dq;
    scatter_side<BLK>(x.sp, x.nud, x.nr, sD, dqs);
    scatter_side<BLK>(x.sp + kMaxSide, x.nud + kMaxSide, x.np, sD, dqs);
    if (OMEGA) {
        scatter_side<BLK>(x.sp, x.nud, x.nr, sW, q);
        scatter_side<BLK>(x.sp + kMaxSide, x.nud + kMaxSide, x.np, sW, q);
    }
    const double sumh = df_to_d(dH);
    if constexpr (OMEGA || RHS) acc.h = fma(q, sumh, acc.h);     // the primal heat release
    acc.cp = fma(q, df_to_d(dCp), acc.cp);
    acc.dh = fma(dq, sumh, acc.dh);
}

template <int BLK, int KIND, bool OMEGA, bool RHS>
__device__ __forceinline__ void jvp_group_log(const DevMech& m, int r0, int r1, const double* sC, const double* sdC,
                                              double* sW, double* sD, const JvpPoint& Q, const double* dlnA,
                                              const DfTab& dt, JvpAcc& acc) {
    const float2* sL = reinterpret_cast<const float2*>(sC);
    const float2* sR = reinterpret_cast<const float2*>(sdC);
    for (int r = r0; r < r1; ++r) jvp_reaction_log<BLK, KIND, OMEGA, RHS>(m, r, sL, sR, sW, sD, Q, dlnA, dt, acc);
}

template <int BLK, int KIND, bool OMEGA, bool RHS>
__device__ __forceinline__ void jvp_group(const DevMech& m, int r0, int r1, const double* sC, const double* sdC,
                                          double* sW, double* sD, const JvpPoint& Q, const double* dlnA,
                                          const DfTab& dt, JvpAcc& acc) {
    for (int r = r0; r < r1; ++r) jvp_reaction<BLK, KIND, OMEGA, RHS>(m, r, sC, sdC, sW, sD, Q, dlnA, dt, acc);
}

// The reactions of one kind for NP > 1 parts per point, round by round (for_rounds): the parts'
// reactions of a round share no species, so all scatter into the point's one d omega_k (and
// omega_k) row.
template <int BLK, int NP, int KIND, bool OMEGA, bool RHS>
__device__ __forceinline__ void jvp_rounds(const DevMech& m, int part, bool direct, const double* sC,
                                           const double* sdC, double* sW, double* sD, const JvpPoint& Q,
                                           const double* dlnA, const DfTab& dt, JvpAcc& acc) {
    if (direct) {
        for_rounds<NP>(m, KIND, part,
                       [&](int r) { jvp_reaction<BLK, KIND, OMEGA, RHS>(m, r, sC, sdC, sW, sD, Q, dlnA, dt, acc); });
    } else {
        const float2* sL = reinterpret_cast<const float2*>(sC);
        const float2* sR = reinterpret_cast<const float2*>(sdC);
        for_rounds<NP>(m, KIND, part, [&](int r) {
            jvp_reaction_log<BLK, KIND, OMEGA, RHS>(m, r, sL, sR, sW, sD, Q, dlnA, dt, acc);
        });
    }
}

// Per-point species rows: C_k, dC_k, the d omega_k row and, with OMEGA, the omega_k row.
__host__ __device__ constexpr int jvp_rows(bool omega) { return omega ? 4 : 3; }

// RHS: the JVP of the implicit-stage sources (omega -> W_k omega_k / rho, hrr -> hrr/(rho c_p)
// and their tangents in d_omega, d_hrr).
template <int BLK, int NP, bool OMEGA, bool RHS>
__global__ void __launch_bounds__(BLK * NP, 512 / (BLK * NP)) jvp_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                       const double* __restrict__ T, const double* __restrict__ p,
                                                       const double* __restrict__ Y, const double* __restrict__ dlnA,
                                                       const double* __restrict__ vT, const double* __restrict__ vY,
                                                       double* __restrict__ omega, double* __restrict__ hrr,
                                                       double* __restrict__ d_omega, double* __restrict__ d_hrr) {
    extern __shared__ double smem[];
    const DfTab dt = stage_df_tables(reinterpret_cast<float2*>(smem), m);
    __syncthreads();
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;         // idle slots of the last block recompute point n-1
    double* base = smem + kMathTabDoubles + slot;
    double* sC = base;                                   // C_k
    double* sdC = base + (size_t)K * BLK;                // dC_k
    double* sD0 = base + (size_t)2 * K * BLK;            // d omega_k
    double* sW0 = base + (size_t)3 * K * BLK;            // omega_k (OMEGA)
    double* sD = sD0;
    double* sW = sW0;

    JvpPoint Q;
    const double Ti = T[i];
    Q.dT = vT[i];
    Q.invT = 1.0 / Ti;
    Q.tT = Q.dT * Q.invT;                                // dT/T
    Q.pRT = p[i] * Q.invT * kInvR;
    Q.dpRT = -Q.pRT * Q.tT;
    Q.P = make_tpairs(Ti, Q.invT, dt);
    Q.lnT = df_to_d(Q.P.lnTd);
    double s = 0.0, ds = 0.0;
    for (int k = 0; k < K; ++k) {
        const double iw = __ldg(m.invW + k);
        s += Y[(int64_t)k * ld + i] * iw;
        ds = fma(vY[(int64_t)k * ld + i], iw, ds);
    }
    const double rho = Q.pRT / s;
    const double arho = -Q.tT - ds / s;                  // d rho / rho
    Q.arho = arho;
    // The logarithmic form needs every Y_k >= 2^-100 (positive, finite) and direction values the
    // pairs can carry (dY_k/Y_k, dT/T and d rho/rho within 2^+-100 or zero); a block with a point
    // that has neither takes the dual products in double (C_k, dC_k in the rows) instead.
    bool bad = !(pair_range_ok(Q.tT) && pair_range_ok(arho));
    for (int k = part; k < K; k += NP) {
        const double y = Y[(int64_t)k * ld + i], v = vY[(int64_t)k * ld + i];
        bad |= !(log_form_ok(y) && pair_range_ok(v) && quot_range_ok(v, y));
    }
    bool direct;
    if constexpr (NP > 1)
        direct = __syncthreads_or(bad) != 0;
    else
        direct = __any_sync(__activemask(), bad);
    if (direct) {
        for (int k = part; k < K; k += NP) {
            const double iw = __ldg(m.invW + k);
            const double c = Y[(int64_t)k * ld + i] * iw * rho;
            sC[k * BLK] = c;
            sdC[k * BLK] = fma(c, arho, rho * vY[(int64_t)k * ld + i] * iw);
        }
    } else {
        Q.tTd = df_split(Q.tT);
        Q.pRTd = df_split(Q.pRT);
        Q.dpRTd = df_neg(df_mul(Q.pRTd, Q.tTd));
        const dfl ar = df_split(arho);
        for (int k = part; k < K; k += NP) {
            const double y = Y[(int64_t)k * ld + i];
            const dfl l = log_df(y * __ldg(m.invW + k) * rho, dt.rc, dt.lc);
            const dfl rk = df_add(ar, df_div(df_split(vY[(int64_t)k * ld + i]), df_split(y)));
            reinterpret_cast<float2*>(sC)[k * BLK] = make_float2(l.h, l.l);
            reinterpret_cast<float2*>(sdC)[k * BLK] = make_float2(rk.h, rk.l);
        }
    }
    for (int k = part; k < K; k += NP) {
        sD[k * BLK] = 0.0;
        if (OMEGA) sW[k * BLK] = 0.0;
    }
    if (NP > 1) __syncthreads();

    JvpAcc acc;
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    if constexpr (NP == 1) {
        if (direct) {
            jvp_group<BLK, 0, OMEGA, RHS>(m, 0, e1, sC, sdC, sW, sD, Q, dlnA, dt, acc);
            jvp_group<BLK, 1, OMEGA, RHS>(m, e1, t1, sC, sdC, sW, sD, Q, dlnA, dt, acc);
            jvp_group<BLK, 2, OMEGA, RHS>(m, t1, m.R, sC, sdC, sW, sD, Q, dlnA, dt, acc);
        } else {
            jvp_group_log<BLK, 0, OMEGA, RHS>(m, 0, e1, sC, sdC, sW, sD, Q, dlnA, dt, acc);
            jvp_group_log<BLK, 1, OMEGA, RHS>(m, e1, t1, sC, sdC, sW, sD, Q, dlnA, dt, acc);
            jvp_group_log<BLK, 2, OMEGA, RHS>(m, t1, m.R, sC, sdC, sW, sD, Q, dlnA, dt, acc);
        }
    } else {
        // (each round ends with a barrier: the rows are complete after the last one)
        jvp_rounds<BLK, NP, 0, OMEGA, RHS>(m, part, direct, sC, sdC, sW, sD, Q, dlnA, dt, acc);
        jvp_rounds<BLK, NP, 1, OMEGA, RHS>(m, part, direct, sC, sdC, sW, sD, Q, dlnA, dt, acc);
        jvp_rounds<BLK, NP, 2, OMEGA, RHS>(m, part, direct, sC, sdC, sW, sD, Q, dlnA, dt, acc);
    }

    // Implicit-stage sources (RHS): fY_k = W_k omega_k / rho, fT = hrr / (rho c_p) with
    // c_p = R sum_k Y_k/W_k c_p,k/R; tangents dfY_k = W_k (d omega_k - omega_k d rho/rho) / rho
    // (the shifted scatter above), dfT = (d hrr - hrr (d rho/rho + d c_p/c_p)) / (rho c_p).
    double cpm = 0.0, dcpm = 0.0, inv_rho = 0.0;
    if constexpr (RHS) inv_rho = 1.0 / rho;
    for (int k = part; k < K; k += NP) {
        double dw = sD0[k * BLK];
        double w = 0.0;
        if constexpr (OMEGA) w = sW0[k * BLK];
        if constexpr (RHS) {
            const double* c = nasa_range(m, k, Ti);
            const double iw = __ldg(m.invW + k), cpk = nasa_cpR(c, Ti);
            const double yk = Y[(int64_t)k * ld + i] * iw, vk = vY[(int64_t)k * ld + i] * iw;
            cpm = fma(yk, cpk, cpm);
            dcpm = fma(vk, cpk, fma(yk * nasa_dcpR_dT(c, Ti), Q.dT, dcpm));
            const double wr = __ldg(m.W + k) * inv_rho;
            dw *= wr;
            w *= wr;
        }
        if (live) {
            d_omega[(int64_t)k * ld + i] = dw;
            if (OMEGA && omega) omega[(int64_t)k * ld + i] = w;
        }
    }
    if constexpr (NP > 1) {
        // C_k and dC_k are dead: rows 3q .. 3q+2 of C and 2q, 2q+1 of dC (3 NP <= K) take part
        // q's sums, added in part order
        sC[(3 * part) * BLK] = acc.h;
        sC[(3 * part + 1) * BLK] = acc.cp;
        sC[(3 * part + 2) * BLK] = acc.dh;
        if constexpr (RHS) {
            sdC[(2 * part) * BLK] = cpm;
            sdC[(2 * part + 1) * BLK] = dcpm;
        }
        __syncthreads();
        if (part != 0) return;
        acc.h = sC[0];
        acc.cp = sC[BLK];
        acc.dh = sC[2 * BLK];
        if constexpr (RHS) {
            cpm = sdC[0];
            dcpm = sdC[BLK];
        }
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            acc.h += sC[(3 * q) * BLK];
            acc.cp += sC[(3 * q + 1) * BLK];
            acc.dh += sC[(3 * q + 2) * BLK];
            if constexpr (RHS) {
                cpm += sdC[(2 * q) * BLK];
                dcpm += sdC[(2 * q + 1) * BLK];
            }
        }
    }
    if (live) {
        const double dhr = -kR * fma(Q.dT, acc.cp, Ti * acc.dh), hr = -kR * Ti * acc.h;
        if constexpr (RHS) {
            const double irc = inv_rho / (kR * cpm);                 // 1 / (rho c_p)
            d_hrr[i] = irc * fma(-hr, arho + dcpm / cpm, dhr);
            if (hrr) hrr[i] = hr * irc;
        } else {
            d_hrr[i] = dhr;
            if (hrr) hrr[i] = hr;
        }
    }
}

// ---------------------------------------------------------------- launch shapes
struct Shape {
    int blk, np;
};
constexpr Shape kShapes[] = {{32, 1}, {64, 1}, {128, 1}, {32, 2}, {64, 2}, {32, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <bool OMEGA, bool RHS, int S>
constexpr auto kernel_of() {
    return jvp_kernel<kShapes[S].blk, kShapes[S].np, OMEGA, RHS>;
}

template <bool OMEGA, bool RHS, int... S>
const void* kernel_ptr(int idx, std::integer_sequence<int, S...>) {
    const void* ptrs[] = {(const void*)kernel_of<OMEGA, RHS, S>()...};
    return ptrs[idx];
}

size_t jvp_smem(int K, const Shape& sh, bool omega) {
    return (size_t)kMathTabDoubles * sizeof(double) + (size_t)jvp_rows(omega) * K * sh.blk * sizeof(double);
}

struct Plan {
    int dev, K;
    bool omega, rhs;
    int idx;
};
std::mutex g_plan_mu;
std::vector<Plan> g_plans;

// The shape with the most resident warps per SM, fewer parts on ties (cached per device, K
// and output set).
template <bool OMEGA, bool RHS>
int plan_shape(int K) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const Plan& q : g_plans)
            if (q.dev == dev && q.K == K && q.omega == OMEGA && q.rhs == RHS) return q.idx;
    }
    int per_block = 0;
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = -1, best_warps = 0;
    for (int c = 0; c < kNumShapes; ++c) {
        const Shape& sh = kShapes[c];
        if (3 * sh.np > K && sh.np > 1) continue;
        const size_t bytes = jvp_smem(K, sh, OMEGA);
        if (bytes > (size_t)per_block) continue;
        const void* kern = kernel_ptr<OMEGA, RHS>(c, std::make_integer_sequence<int, kNumShapes>{});
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
        g_plans.push_back({dev, K, OMEGA, RHS, best});
    }
    return best;
}

template <bool OMEGA, bool RHS, int... S>
cudaError_t launch_idx(int idx, std::integer_sequence<int, S...>, const DevMech& m, int64_t n, int64_t ld,
                       const double* T, const double* p, const double* Y, const double* dlnA, const double* vT,
                       const double* vY, double* omega, double* hrr, double* d_omega, double* d_hrr,
                       cudaStream_t st) {
    cudaError_t e = cudaErrorInvalidConfiguration;
    ((S == idx ? (void)(e = [&] {
        constexpr Shape sh = kShapes[S];
        auto kern = kernel_of<OMEGA, RHS, S>();
        const size_t smem = jvp_smem(m.K, sh, OMEGA);
        cudaError_t r = ensure_smem((const void*)kern, smem);
        if (r != cudaSuccess) return r;
        kern<<<(unsigned)((n + sh.blk - 1) / sh.blk), sh.blk * sh.np, smem, st>>>(m, n, ld, T, p, Y, dlnA, vT, vY,
                                                                                  omega, hrr, d_omega, d_hrr);
        return cudaGetLastError();
    }())
               : (void)0),
     ...);
    return e;
}

template <bool OMEGA, bool RHS>
cudaError_t launch_o(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     const double* dlnA, const double* vT, const double* vY, double* omega, double* hrr,
                     double* d_omega, double* d_hrr, cudaStream_t s) {
    const int idx = plan_shape<OMEGA, RHS>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx<OMEGA, RHS>(idx, std::make_integer_sequence<int, kNumShapes>{}, m, n, ld, T, p, Y, dlnA, vT,
                                  vY, omega, hrr, d_omega, d_hrr, s);
}

}  // namespace

}  // namespace nk
