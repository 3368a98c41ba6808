// State-only terms of a reaction's rate of progress and of its tangent, shared by the two
// stored linearizations of the rates (the per-entry form of k_lin.cu and the per-reaction form
// of k_linc.cu).  At fixed p, with tT = dT/T:
//   d ln k_f = aT tT + aM d[M]        (aM only for Troe reactions: the falloff chain)
//   d ln K_c = D tT,  D = sum_k nu_k h_k/RT - sum_k nu_k
// and the rate constants themselves, k_f (with the falloff factor for Troe reactions) and
// k_r = k_f / K_c.  The exponent chains, the falloff chain and its two tangents run in
// double-float pairs as in the FP64 rates kernel.
#pragma once

#include "nk_rxn.cuh"

namespace nk {

struct LinPoint {
    TPairs P;
    double invT, lnT, pRT;
};

struct RateTerms {
    double kf, kr;    // forward and reverse rate constants (without [M] for third-body rows)
    double aT, aM;    // d ln k_f / (dT/T), d ln k_f / d[M]
    double D;         // d ln K_c / (dT/T)
    double sumcp;     // sum_k nu_k c_p,k/R
    double M;         // [M] (third-body and Troe rows; 0 for elementary ones)
};

// sC: the point's concentrations C_k at sC[k * BLK]
template <int BLK, int KIND>
__device__ __forceinline__ RateTerms rate_terms(const DevMech& m, int r, const Rxn& x, const double* sC,
                                                const LinPoint& Q, const double* dlnA, const DfTab& dt) {
    RateTerms o;
    dfl dG, dH, dCp;
    rxn_thermo<true, true>(m, x.thermo, Q.P, dG, dH, dCp);
    const double sumh = df_to_d(dH);
    o.sumcp = df_to_d(dCp);
    const dfl lnKc = df_add(df_mul_f(Q.P.lnP0RTd, dnu_f(m, r)), df_neg(dG));
    dfl shiftd{0.0f, 0.0f};
    if (dlnA) shiftd = df_split(__ldg(dlnA + x.orig));
    const dfl lnkf = ln_kf_df(m, r, Q.P, shiftd, dlnA != nullptr);
    const double c1 = fma(x.EaR, Q.invT, x.beta);     // d ln k_inf / (dT/T)

    double M = 0.0;
    if (KIND != 0) {
        M = Q.pRT;
        for (int j = x.eff0; j < x.eff1; ++j) M = fma(__ldg(m.eff_m1 + j), sC[__ldg(m.eff_sp + j) * BLK], M);
    }
    double kf, kr, aT = c1, aM = 0.0;
    if constexpr (KIND == 2) {
        if (M == 0.0) {
            kf = kr = aT = 0.0;
        } else {
            // the falloff chain in pairs: ln F, and d ln k_f = (c1 + Px (c0 - c1) + PL LT) dT/T + (Px/[M]) d[M]
            const dfl Mp = df_split(M);
            dfl c0;
            const dfl lnPr = troe_lnPr(m, x.aux, Q.P, lnkf, shiftd, dlnA != nullptr, Mp, dt, &c0);
            const TroeCent c = troe_cent(m, x.aux, Q.P, dt);
            const TroeLog f = troe_log(lnPr, c.L, dt);
            const dfl lnkF = df_add(lnkf, f.lnF), c1d = arrh_slope_df(m, r, Q.P);
            kf = exp_df_d(lnkF, dt.e2);
            kr = exp_df_d(df_add(lnkF, df_neg(lnKc)), dt.e2);
            aT = df_to_d(df_add(df_fma(f.Px, df_add(c0, df_neg(c1d)), c1d), df_mul(f.PL, c.LT)));
            aM = df_to_d(df_div(f.Px, Mp));
        }
    } else {
        kf = exp_df_d(lnkf, dt.e2);
        kr = exp_df_d(df_add(lnkf, df_neg(lnKc)), dt.e2);
    }
    o.kf = kf;
    o.kr = kr;
    o.aT = aT;
    o.aM = aM;
    o.D = sumh - x.dnu;
    o.M = M;
    return o;
}

// The point terms of both linearization passes: T pairs, 1/T, ln T, p/(R T).
__device__ __forceinline__ LinPoint make_lin_point(double Ti, double pi, const DfTab& dt) {
    LinPoint Q;
    Q.invT = 1.0 / Ti;
    Q.pRT = pi * Q.invT * kInvR;
    Q.P = make_tpairs(Ti, Q.invT, dt);
    Q.lnT = df_to_d(Q.P.lnTd);
    return Q;
}

// The end of a product pass from stored data (both linearizations): d omega_k summed over the
// parts' partial rows in part order, d hrr = -R (dT S1 + T sum_k (h_k/RT) d omega_k) with S1 and
// h_k/RT read from the stored slots (hRT[k ldl], *S1p of point i).  With RHS the tangents of the
// implicit-stage sources instead, given the sources fT, fY at the same state:
//   dfY_k = (W_k/rho) d omega_k - fY_k d rho/rho,  dfT = d hrr/(rho c_p) - fT (d rho/rho + d c_p/c_p)
// (written to d_omega and d_hrr).  sX: per-point shared rows no longer in use, at least
// (1 + 2 RHS) NP of them, for the parts' scalar sums.  Part 0 writes the point terms.  NR: the
// rows of d omega_k partials in sD0 (NP, or 1 when the parts share one row).
template <int BLK, int NP, bool RHS, int NR = NP>
__device__ __forceinline__ void lin_epilogue(const DevMech& m, int part, bool live, int64_t i, double Ti, double dT,
                                             double rho, double arho, const double* sD0, double* sX,
                                             const double* __restrict__ hRT, const double* __restrict__ S1p,
                                             int64_t ldl, const double* __restrict__ Y,
                                             const double* __restrict__ vY, int64_t ld,
                                             const double* __restrict__ fT, const double* __restrict__ fY,
                                             int64_t ldf, double* __restrict__ d_omega,
                                             double* __restrict__ d_hrr) {
    const int K = m.K;
    double hsum = 0.0, cpm = 0.0, dcpm = 0.0, inv_rho = 0.0;
    if constexpr (RHS) inv_rho = 1.0 / rho;
    for (int k = part; k < K; k += NP) {
        double dw = sD0[k * BLK];
#pragma unroll
        for (int q = 1; q < NR; ++q) dw += sD0[((size_t)q * K + k) * BLK];
        hsum = fma(hRT[(int64_t)k * ldl], dw, hsum);
        if constexpr (RHS) {
            const double* c = nasa_range(m, k, Ti);
            const double iw = __ldg(m.invW + k), cpk = nasa_cpR(c, Ti);
            const double yk = Y[(int64_t)k * ld + i] * iw, vk = vY[(int64_t)k * ld + i] * iw;
            cpm = fma(yk, cpk, cpm);
            dcpm = fma(vk, cpk, fma(yk * nasa_dcpR_dT(c, Ti), dT, dcpm));
            dw = fma(__ldg(m.W + k) * inv_rho, dw, -fY[(int64_t)k * ldf + i] * arho);
        }
        if (live) d_omega[(int64_t)k * ld + i] = dw;
    }
    if constexpr (NP > 1) {
        // rows q, NP + q, 2 NP + q of sX take part q's sums
        sX[part * BLK] = hsum;
        if constexpr (RHS) {
            sX[(NP + part) * BLK] = cpm;
            sX[(2 * NP + part) * BLK] = dcpm;
        }
        __syncthreads();
        if (part != 0) return;
        hsum = sX[0];
        if constexpr (RHS) {
            cpm = sX[NP * BLK];
            dcpm = sX[2 * NP * BLK];
        }
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            hsum += sX[q * BLK];
            if constexpr (RHS) {
                cpm += sX[(NP + q) * BLK];
                dcpm += sX[(2 * NP + q) * BLK];
            }
        }
    }
    if (live) {
        const double dhr = -kR * fma(dT, *S1p, Ti * hsum);
        if constexpr (RHS)
            d_hrr[i] = fma(dhr, inv_rho / (kR * cpm), -fT[i] * (arho + dcpm / cpm));
        else
            d_hrr[i] = dhr;
    }
}

}  // namespace nk
