// Vector-Jacobian product of (omega_k, heat release): reverse-mode differentiation written
// out by hand, the exact transpose of the JVP (gradients for mechanism calibration and for
// adjoint solves).  Rates of progress are recomputed in registers, nothing per reaction is
// stored.
//
// Single pass over the reactions: with hrr = -sum_k h_k omega_k and omega_k = sum_r nu_kr q_r,
//   qbar_r = sum_k nu_kr bar_omega_k - bar_hrr R T (sum_k nu_kr h_k/RT),
//   Tbar  += -bar_hrr R q_r (sum_k nu_kr c_p,k/R)          (temperature dependence of h_k),
// so the forward values omega_k are never needed, and the reaction sums of h/RT and c_p/R
// come from the reaction's thermo groups.  The ln A gradient of a point is qbar_r q_r (a shift
// of ln A_r scales k_f and k_r alike, and both limits of a Troe reaction); it is summed over
// the points of a warp by shuffles, over the point tiles of a block in shared memory and over
// blocks by a second kernel in a fixed order: deterministic, no atomics.
//
// FP64 form as the rates kernel (exponent chains and, in the logarithmic form, the falloff
// chain in double-float pairs, everything else in double).  Layout: blocks of 32 points, NP
// warps per point sharing C_k, bar_omega_k and the Cbar_k row in shared memory, into which they
// add in rounds of reactions that share no species (the logarithmic form on the rates kernel's
// rounds, its efficiency terms deferred to per-species sums after each kind; the double-product
// form on rounds that also keep efficiency species apart): every sum in an order fixed by the
// schedule.  A persistent grid walks the point tiles.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "nk_rxn.cuh"

namespace nk {
namespace {

constexpr int kVjpBlk = 32;   // points per block: one warp per part

// prod of p[0..n) (returned) and, in ex[e], the product of all entries but e (n <= 4, uniform)
__device__ __forceinline__ double exclusive_products(const double* p, int n, double* ex) {
    switch (n) {
        case 1:
            ex[0] = 1.0;
            return p[0];
        case 2:
            ex[0] = p[1];
            ex[1] = p[0];
            return p[0] * p[1];
        case 3: {
            const double a = p[0] * p[1];
            ex[0] = p[1] * p[2];
            ex[1] = p[0] * p[2];
            ex[2] = a;
            return a * p[2];
        }
        default: {
            const double a = p[0] * p[1], b = p[2] * p[3];
            ex[0] = p[1] * b;
            ex[1] = p[0] * b;
            ex[2] = a * p[3];
            ex[3] = a * p[2];
            return a * b;
        }
    }
}

struct VjpPoint {
    TPairs P;
    double invT, lnT, pRT, hb, hbRT;
    dfl pRTd;
    bool valid;
};

template <int KIND, bool WANT_G, bool HB>
__device__ __forceinline__ void vjp_reaction(const DevMech& m, int r, const double* sC, const double* sWb, double* sB,
                                             double* gw, const VjpPoint& Q, const double* dlnA, const DfTab& dt,
                                             double& Tbar) {
    constexpr int BLK = kVjpBlk;
    const Rxn x = load_rxn(m.rxn + r);
    // concentration powers of the entries and sum_k nu_k bar_omega_k
    double wsum = 0.0;
    double cR[kMaxSide], pR[kMaxSide], cP[kMaxSide], pP[kMaxSide];
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        cR[e] = pR[e] = cP[e] = pP[e] = 1.0;
        if (e < x.nr) {
            const int k = x.sp[e];
            const double c = sC[k * BLK];
            double pw = c;
            for (int j = 1; j < x.nu[e]; ++j) pw *= c;
            cR[e] = c;
            pR[e] = pw;
            wsum = fma(x.nud[e], sWb[k * BLK], wsum);
        }
        if (e < x.np) {
            const int k = x.sp[kMaxSide + e];
            const double c = sC[k * BLK];
            double pw = c;
            for (int j = 1; j < x.nu[kMaxSide + e]; ++j) pw *= c;
            cP[e] = c;
            pP[e] = pw;
            wsum = fma(x.nud[kMaxSide + e], sWb[k * BLK], wsum);
        }
    }
    double exR[kMaxSide], exP[kMaxSide];
    const double fw = exclusive_products(pR, x.nr, exR);
    const double rv = exclusive_products(pP, x.np, exP);

    dfl dG, dH, dCp;
    rxn_thermo<true, HB>(m, x.thermo, Q.P, dG, dH, dCp);
    const double sumh = df_to_d(dH);
    const dfl lnKc = df_add(df_mul_f(Q.P.lnP0RTd, dnu_f(m, r)), df_neg(dG));
    double shift = 0.0;
    dfl shiftd{0.0f, 0.0f};
    if (dlnA) {
        shift = __ldg(dlnA + x.orig);
        shiftd = df_split(shift);
    }
    const dfl lnkf = ln_kf_df(m, r, Q.P, shiftd, dlnA != nullptr);

    double M = 0.0;
    if (KIND != 0) {
        M = Q.pRT;
        for (int j = x.eff0; j < x.eff1; ++j) M = fma(__ldg(m.eff_m1 + j), sC[__ldg(m.eff_sp + j) * BLK], M);
    }

    // ---- primal (values kept for the adjoint)
    double kf;
    double tr_g = 0.0, tr_lF = 0.0, tr_f1 = 0.0, tr_den = 1.0, tr_u = 0.0, tr_v = 1.0, tr_nn = 0.0, tr_Fc = 1.0,
           tr_dFc = 0.0;
    const TroeRec* t = nullptr;
    if constexpr (KIND == 2) {
        t = m.troe + x.aux;
        if (M == 0.0) {
            kf = 0.0;
        } else {
            const double lnk0 = fma(-__ldg(&t->Ea0R), Q.invT, fma(__ldg(&t->beta0), Q.lnT, __ldg(&t->lnA0) + shift));
            const double lnPr = lnk0 - df_to_d(lnkf) + dlog_df(M, dt);
            const double a = __ldg(&t->a), i3 = __ldg(&t->invT3), i1 = __ldg(&t->invT1);
            const double e3 = dexp_df(-Q.P.T * i3, dt), e1 = dexp_df(-Q.P.T * i1, dt);
            tr_Fc = (1.0 - a) * e3 + a * e1;
            tr_dFc = -((1.0 - a) * i3 * e3 + a * i1 * e1);
            if (__ldg(&t->hasT2) != 0.0) {
                const double T2 = __ldg(&t->T2), e2 = dexp_df(-T2 * Q.invT, dt);
                tr_Fc += e2;
                tr_dFc = fma(T2 * Q.invT * Q.invT, e2, tr_dFc);
            }
            const double lFc = dlog_df(tr_Fc, dt) * kInvLn10;
            const double c = fma(-0.67, lFc, -0.4);
            tr_nn = fma(-1.27, lFc, 0.75);
            tr_u = fma(lnPr, kInvLn10, c);
            tr_v = fma(-0.14, tr_u, tr_nn);
            tr_f1 = tr_u / tr_v;
            tr_den = fma(tr_f1, tr_f1, 1.0);
            tr_lF = lFc / tr_den;
            tr_g = 1.0 / (1.0 + dexp_df(-lnPr, dt));
            kf = exp_df_d(lnkf, dt.e2) * tr_g * dexp_df(tr_lF * kLn10, dt);
        }
    } else {
        kf = exp_df_d(lnkf, dt.e2);
    }
    const double E = exp_df_d(df_neg(lnKc), dt.e2);
    const double kr = kf * E;
    const double qc = fma(kf, fw, -kr * rv);
    const double q = KIND == 1 ? qc * M : qc;

    // ---- adjoint
    const double qbar = HB ? fma(-Q.hbRT, sumh, wsum) : wsum;   // sum nu (bar_omega - bar_hrr h)
    if (HB) Tbar = fma(-Q.hb * kR * q, df_to_d(dCp), Tbar);
    if (WANT_G) {
        double gl = Q.valid ? qbar * q : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gl += __shfl_xor_sync(0xffffffffu, gl, o);
        if ((threadIdx.x & 31) == 0) gw[r] += gl;
    }
    double Mbar = 0.0, qcbar = qbar;
    if (KIND == 1) {
        qcbar = qbar * M;
        Mbar = qbar * qc;
    }
    const double krbar = -qcbar * rv;
    const double kfbar = fma(krbar, E, qcbar * fw);
    const double fwbar = qcbar * kf, rvbar = -qcbar * kr;
    const double lnKcbar = -krbar * kr;
    Tbar = fma(lnKcbar * Q.invT, sumh - x.dnu, Tbar);           // through g_k/RT(T) and ln(p0/RT)
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        if (e < x.nr) {
            double d = exR[e];                                  // d fw / d C_e = nu C_e^(nu-1) prod_{f!=e}
            if (x.nu[e] > 1) {
                d *= -x.nud[e];
                for (int j = 1; j < x.nu[e]; ++j) d *= cR[e];
            }
            double* b = sB + x.sp[e] * BLK;
            *b = fma(fwbar, d, *b);
        }
        if (e < x.np) {
            double d = exP[e];
            if (x.nu[kMaxSide + e] > 1) {
                d *= x.nud[kMaxSide + e];
                for (int j = 1; j < x.nu[kMaxSide + e]; ++j) d *= cP[e];
            }
            double* b = sB + x.sp[kMaxSide + e] * BLK;
            *b = fma(rvbar, d, *b);
        }
    }
    const double Lbar = kfbar * kf;                              // cotangent of ln k_f
    if constexpr (KIND == 2) {
        if (M != 0.0) {
            const double lnf = fma(__ldg(&t->Ea0R), Q.invT, __ldg(&t->beta0)) * Q.invT;
            // d lF / d log10 Pr and d lF / d log10 F_cent
            const double dlF_du = -2.0 * tr_lF * tr_f1 * (tr_nn / (tr_v * tr_v)) / tr_den;
            const double df1_dlFc = fma(1.1762, tr_u, -0.67 * tr_v) / (tr_v * tr_v);
            const double dlF_dlFc = (1.0 - 2.0 * tr_lF * tr_f1 * df1_dlFc) / tr_den;
            const double lnPrbar = Lbar * (1.0 - tr_g + dlF_du);
            const double lnkinfbar = Lbar - lnPrbar;
            Mbar = fma(lnPrbar, 1.0 / M, Mbar);
            Tbar = fma(Lbar * dlF_dlFc, tr_dFc / tr_Fc, Tbar);
            Tbar = fma(lnPrbar, lnf, Tbar);
            Tbar = fma(lnkinfbar, fma(x.EaR, Q.invT, x.beta) * Q.invT, Tbar);
        }
    } else {
        Tbar = fma(Lbar, fma(x.EaR, Q.invT, x.beta) * Q.invT, Tbar);
    }
    if (KIND != 0 && Mbar != 0.0) {
        Tbar = fma(-Mbar * Q.pRT, Q.invT, Tbar);                 // sum_k C_k = p/(RT)
        for (int j = x.eff0; j < x.eff1; ++j) {
            double* b = sB + __ldg(m.eff_sp + j) * BLK;
            *b = fma(Mbar, __ldg(m.eff_m1 + j), *b);
        }
    }
}

// The logarithmic form (tiles whose mass fractions are all within 2^+-100; see the kernel).  The C_k
// row holds ln C_k as pairs; with F the falloff factor (1 but for Troe reactions)
//   q_f = exp(ln k_f + ln F + sum_reac nu ln C),  q_r = exp(ln k_f + ln F - ln K_c + sum_prod nu ln C),
// so d q_c / d ln C_k = nu (q_f or -q_r), d q_c / d (ln k_f + ln F) = q_c and d q_c / d ln K_c = q_r.
// The bar_omega_k row holds the cotangents as pairs (the reaction's sum nu bar_omega in pairs).
// The species rows accumulate S_k = Cbar_k C_k (the cotangent of ln C_k), turned into
// Cbar_k = S_k/C_k once per point at the end; the third-body terms Mbar (eps - 1) enter as
// Mbar (eps - 1) C_k.  The temperature cotangent is accumulated times T (TbarT), term by term:
// Lbar kT through ln k_f + ln F (Lbar = qcbar q_c; kT = T d(ln k_f + ln F)/dT at fixed [M], which
// is c1 = beta + Ea/(RT) but for Troe reactions), qcbar q_r (sum nu h/RT - sum nu) through ln K_c,
// -Mbar p/(RT) through sum_k C_k and -bar_hrr R T q sum nu c_p/R through h_k.  The falloff chain
// runs in pairs (troe_log).
// DEFER: the efficiency terms wait: Mbar goes to this reaction's slot *sMb (deferred_eff adds
// them after the kind's rounds).
// Returns this point's term qbar_r q_r of the ln A gradient (0 without WANT_G); the caller sums
// it over the warp.
template <int KIND, bool WANT_G, bool HB, bool DEFER = false>
__device__ __forceinline__ double vjp_reaction_log(const DevMech& m, int r, const float2* sL, const double* sWb,
                                                   double* sS, const VjpPoint& Q, const double* dlnA,
                                                   const DfTab& dt, double& TbarT, double* sMb = nullptr) {
    constexpr int BLK = kVjpBlk;
    const Rxn x = load_rxn(m.rxn + r);
    // sum_k nu_k bar_omega_k (products minus reactants) from the pair row, one conversion
    const float2* sW2 = reinterpret_cast<const float2*>(sWb);
    const double wsum = df_to_d(df_add(side_sum_df<BLK>(sW2, x.sp + kMaxSide, x.nu + kMaxSide, x.np),
                                       df_neg(side_sum_df<BLK>(sW2, x.sp, x.nu, x.nr))));
    const dfl sf = side_sum_df<BLK>(sL, x.sp, x.nu, x.nr);
    const dfl sb = side_sum_df<BLK>(sL, x.sp + kMaxSide, x.nu + kMaxSide, x.np);
    dfl dG, dH, dCp;
    rxn_thermo<true, HB>(m, x.thermo, Q.P, dG, dH, dCp);
    const float dnu = dnu_f(m, r);
    const dfl lnKc = df_add(df_mul_f(Q.P.lnP0RTd, dnu), df_neg(dG));
    dfl shiftd{0.0f, 0.0f};
    if (dlnA) shiftd = df_split(__ldg(dlnA + x.orig));
    const dfl lnkf = ln_kf_df(m, r, Q.P, shiftd, dlnA != nullptr);
    const dfl c1 = arrh_slope_df(m, r, Q.P);
    dfl Mp{0.0f, 0.0f};
    if (KIND != 0) {
        Mp = Q.pRTd;
        for (int j = x.eff0; j < x.eff1; ++j)
            Mp = df_fma(dfl_of(__ldg(m.df_eff_m1 + j)), exp_df_pair(dfl_of(sL[__ldg(m.eff_sp + j) * BLK]), dt.e2), Mp);
    }

    // ---- primal; for Troe reactions ln F and the coefficients of its adjoint in pairs:
    //   kT = c1 + Px (c0 - c1) + PL LT (T d(ln k_f + ln F)/dT at fixed [M]), kM = Px/[M]
    dfl lnkF = lnkf, kT = c1, kM{0.0f, 0.0f};
    bool noF = false;
    if constexpr (KIND == 2) {
        if (Mp.h == 0.0f) {
            noF = true;
        } else {
            dfl c0;
            const dfl lnPr = troe_lnPr(m, x.aux, Q.P, lnkf, shiftd, dlnA != nullptr, Mp, dt, &c0);
            const TroeCent c = troe_cent(m, x.aux, Q.P, dt);
            const TroeLog f = troe_log(lnPr, c.L, dt);
            lnkF = df_add(lnkf, f.lnF);
            kT = df_add(df_fma(f.Px, df_add(c0, df_neg(c1)), c1), df_mul(f.PL, c.LT));
            kM = df_div(f.Px, Mp);
        }
    }
    double qf = exp_df_d(df_add(lnkF, sf), dt.e2);
    double qr = exp_df_d(df_add(df_add(lnkF, df_neg(lnKc)), sb), dt.e2);
    if (KIND == 2 && noF) qf = qr = 0.0;
    const double qc = qf - qr;
    double M = 0.0;
    if (KIND == 1) M = df_to_d(Mp);
    const double q = KIND == 1 ? qc * M : qc;

    // ---- adjoint
    const double qbar = HB ? fma(-Q.hbRT, df_to_d(dH), wsum) : wsum;   // sum nu (bar_omega - bar_hrr h)
    if (HB) TbarT = fma(-Q.hbRT * q, df_to_d(dCp), TbarT);
    const double gl = WANT_G && Q.valid ? qbar * q : 0.0;
    double Mbar = 0.0, qcbar = qbar;
    if (KIND == 1) {
        qcbar = qbar * M;
        Mbar = qbar * qc;
    }
    // S_k += nu_k (q_f or -q_r) qcbar: with the signed coefficients nud (-nu for reactants)
    scatter_side<BLK>(x.sp, x.nud, x.nr, sS, -qcbar * qf);
    scatter_side<BLK>(x.sp + kMaxSide, x.nud + kMaxSide, x.np, sS, -qcbar * qr);
    // through ln K_c (g_k/RT(T) and ln(p0/RT)) and through ln k_f + ln F
    const double Lbar = qcbar * qc;
    TbarT = fma(qcbar * qr, df_to_d(df_add(dH, dfl{-dnu, 0.0f})), TbarT);
    TbarT = fma(Lbar, df_to_d(kT), TbarT);
    if constexpr (KIND == 2) Mbar = Lbar * df_to_d(kM);
    if constexpr (KIND != 0 && DEFER) *sMb = Mbar;
    if (KIND != 0 && Mbar != 0.0) {
        TbarT = fma(-Mbar, Q.pRT, TbarT);                       // sum_k C_k = p/(RT)
        for (int j = x.eff0; !DEFER && j < x.eff1; ++j) {
            const int k = __ldg(m.eff_sp + j);
            double* b = sS + k * BLK;
            const dfl ec = df_mul(dfl_of(__ldg(m.df_eff_m1 + j)), exp_df_pair(dfl_of(sL[k * BLK]), dt.e2));
            *b = fma(Mbar, df_to_d(ec), *b);
        }
    }
    return gl;
}

// gw[r_j] += the warp sum of a_j for the first nv of four reactions r_0..r_3: one transposed
// butterfly (the lanes trade halves of the four values, then of the two left, then reduce
// within groups of eight), so lane 8 j ends with the sum of a_j.  Every sum is the same
// pairwise tree as a butterfly all-reduce of a_j alone (bit-identical), at 7 FP64 additions for
// the four instead of 24.
__device__ __forceinline__ void warp_sum4_add(double* gw, double a0, double a1, double a2, double a3, int r0, int r1,
                                              int r2, int r3, int nv) {
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool hi = (lane & 16) != 0, b3 = (lane & 8) != 0;
    double k0 = hi ? a2 : a0, k1 = hi ? a3 : a1;
    const double s0 = hi ? a0 : a2, s1 = hi ? a1 : a3;
    k0 += __shfl_xor_sync(kAll, s0, 16);
    k1 += __shfl_xor_sync(kAll, s1, 16);
    double k = b3 ? k1 : k0;
    k += __shfl_xor_sync(kAll, b3 ? k0 : k1, 8);
    k += __shfl_xor_sync(kAll, k, 4);
    k += __shfl_xor_sync(kAll, k, 2);
    k += __shfl_xor_sync(kAll, k, 1);
    const int j = lane >> 3;
    const int rj = j == 0 ? r0 : (j == 1 ? r1 : (j == 2 ? r2 : r3));
    if ((lane & 7) == 0 && j < nv) gw[rj] += k;
}

// The ln A gradient terms of a warp's reactions, held three at a time and summed over the warp
// with the fourth (warp_sum4_add); flush() sends the last one to three with the other slots zero.
struct GradBatch {
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    int r0 = 0, r1 = 0, r2 = 0, nb = 0;          // the held terms' reactions and count (warp-uniform)
    __device__ __forceinline__ void add(double* gw, int r, double g) {
        if (nb == 3) {
            warp_sum4_add(gw, g0, g1, g2, g, r0, r1, r2, r, 4);
            nb = 0;
        } else {
            if (nb == 0) {
                g0 = g;
                r0 = r;
            } else if (nb == 1) {
                g1 = g;
                r1 = r;
            } else {
                g2 = g;
                r2 = r;
            }
            ++nb;
        }
    }
    __device__ __forceinline__ void flush(double* gw) {
        if (nb > 0) warp_sum4_add(gw, g0, nb > 1 ? g1 : 0.0, nb > 2 ? g2 : 0.0, 0.0, r0, r1, r2, 0, nb);
        nb = 0;
    }
};

// Reactions [r0, r1) of one kind in order (one part per point).
template <int KIND, bool WANT_G, bool HB>
__device__ __forceinline__ void vjp_group_log(const DevMech& m, int r0, int r1, const double* sC, const double* sWb,
                                              double* sB, double* gw, const VjpPoint& Q, const double* dlnA,
                                              const DfTab& dt, double& Tbar) {
    const float2* sL = reinterpret_cast<const float2*>(sC);
    GradBatch gb;
    for (int r = r0; r < r1; ++r) {
        const double g = vjp_reaction_log<KIND, WANT_G, HB>(m, r, sL, sWb, sB, Q, dlnA, dt, Tbar);
        if (WANT_G) gb.add(gw, r, g);
    }
    if (WANT_G) gb.flush(gw);
}

// The deferred efficiency terms of kind KIND (1, 2) after its rounds: species k of this part
// (k = part, part + NP, ...) takes C_k sum Mbar_slot (eps - 1) over its entries, in round order.
template <int NP, int KIND>
__device__ __forceinline__ void deferred_eff(const DevMech& m, int part, const float2* sL, double* sS,
                                             const double* sMb, const DfTab& dt) {
    constexpr int BLK = kVjpBlk;
    const int K = m.K;
    const int32_t* ptr = (NP == 2 ? m.mt_ptr2 : m.mt_ptr4) + (size_t)(KIND - 1) * (K + 1);
    const int32_t* sl = NP == 2 ? m.mt_slot2 : m.mt_slot4;
    const double* ev = NP == 2 ? m.mt_eps2 : m.mt_eps4;
    for (int k = part; k < K; k += NP) {
        const int e0 = __ldg(ptr + k), e1 = __ldg(ptr + k + 1);
        if (e0 == e1) continue;
        double acc = 0.0;
        for (int e = e0; e < e1; ++e) acc = fma(sMb[__ldg(sl + e) * BLK], __ldg(ev + e), acc);
        sS[k * BLK] = fma(acc, exp_df_d(dfl_of(sL[k * BLK]), dt.e2), sS[k * BLK]);
    }
}

// The reactions of one kind for NP > 1 parts per point, round by round, all parts adding into
// the point's one row of S_k (or Cbar_k).  The double-product form (direct) takes the VJP's
// schedule (for_rounds with EFF: the parts' reactions of a round share no species, efficiencies
// included).  The logarithmic form takes the plain schedule of the rates kernel and defers the
// efficiency terms of third-body and Troe reactions: each leaves its Mbar in the slot of its
// round and part (sMb), and deferred_eff adds them per species after the kind's rounds.
template <int NP, int KIND, bool WANT_G, bool HB>
__device__ __forceinline__ void vjp_rounds(const DevMech& m, int part, bool direct, const double* sC,
                                           const double* sWb, double* sB, double* gw, const VjpPoint& Q,
                                           const double* dlnA, const DfTab& dt, double& Tbar, double* sMb) {
    if (direct) {
        for_rounds<NP, true>(m, KIND, part, [&](int r) {
            vjp_reaction<KIND, WANT_G, HB>(m, r, sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
        });
    } else {
        constexpr int BLK = kVjpBlk;
        const float2* sL = reinterpret_cast<const float2*>(sC);
        const int32_t* S = NP == 2 ? m.rsched2 : m.rsched4;
        const int rd0 = NP == 2 ? m.rrnd2[KIND] : m.rrnd4[KIND], rd1 = NP == 2 ? m.rrnd2[KIND + 1] : m.rrnd4[KIND + 1];
        GradBatch gb;
        int r = rd0 < rd1 ? __ldg(S + rd0 * NP + part) : -1;
        for (int rd = rd0; rd < rd1; ++rd) {
            const int rn = rd + 1 < rd1 ? __ldg(S + (rd + 1) * NP + part) : -1;   // the next round's, early
            if (r >= 0) {
                const double g = vjp_reaction_log<KIND, WANT_G, HB, true>(m, r, sL, sWb, sB, Q, dlnA, dt, Tbar,
                                                                          sMb + ((rd - rd0) * NP + part) * BLK);
                if (WANT_G) gb.add(gw, r, g);
            }
            __syncthreads();
            r = rn;
        }
        if (WANT_G) gb.flush(gw);
        if constexpr (KIND != 0) {
            if (rd0 < rd1) {
                deferred_eff<NP, KIND>(m, part, sL, sB, sMb, dt);
                __syncthreads();                                  // before the next kind's rounds
            }
        }
    }
}

template <int KIND, bool WANT_G, bool HB>
__device__ __forceinline__ void vjp_group(const DevMech& m, int r0, int r1, const double* sC, const double* sWb,
                                          double* sB, double* gw, const VjpPoint& Q, const double* dlnA,
                                          const DfTab& dt, double& Tbar) {
    for (int r = r0; r < r1; ++r) vjp_reaction<KIND, WANT_G, HB>(m, r, sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
}

// Shared memory of a block: the pair tables, the ln A sums [R] (WANT_G), then per point C_k,
// bar_omega_k, the Cbar_k row and (NP > 1) the deferred [M] cotangents' slots.
int vjp_mslots(const DevMech& m, int np) { return np == 2 ? m.mslots2 : (np == 4 ? m.mslots4 : 0); }
size_t vjp_smem(int K, int R, int mslots, bool want_g) {
    return (size_t)kMathTabDoubles * sizeof(double) + (want_g ? (size_t)((R + 1) & ~1) * sizeof(double) : 0) +
           ((size_t)3 * K + mslots) * kVjpBlk * sizeof(double);
}

// PASS 0 takes the tiles of the logarithmic form and skips the others; PASS 1 takes only those
// (products in double).  Each pass alone compiles to fewer registers than both paths together:
// the logarithmic pass runs four blocks of 4 warps per SM, the fallback pass three.
template <int NP, bool WANT_G, bool HB, int PASS>
__global__ void __launch_bounds__(kVjpBlk * NP, (PASS == 0 ? 512 : 384) / (kVjpBlk * NP)) vjp_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                           const double* __restrict__ T, const double* __restrict__ p,
                                                           const double* __restrict__ Y,
                                                           const double* __restrict__ dlnA,
                                                           const double* __restrict__ bar_omega,
                                                           const double* __restrict__ bar_hrr,
                                                           double* __restrict__ gT, double* __restrict__ gY,
                                                           double* __restrict__ ws) {
    constexpr int BLK = kVjpBlk, NT = BLK * NP;
    extern __shared__ double smem[];
    const DfTab dt = stage_df_tables(reinterpret_cast<float2*>(smem), m);
    const int K = m.K, R = m.R;
    double* gw = smem + kMathTabDoubles;                          // ln A sums of this block, device order
    if (WANT_G)
        for (int r = threadIdx.x; r < R; r += NT) gw[r] = 0.0;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    double* base = smem + kMathTabDoubles + (WANT_G ? ((R + 1) & ~1) : 0) + slot;
    double* sC = base;                                            // C_k
    double* sWb = base + (size_t)K * BLK;                         // bar_omega_k
    double* sB0 = base + (size_t)2 * K * BLK;                     // Cbar_k (S_k in the logarithmic form)
    double* sB = sB0;
    double* sMb = base + (size_t)3 * K * BLK;                     // (NP > 1) deferred Mbar slots
    int ra[3], rb[3];
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    slice<NP>(0, e1, part, ra[0], rb[0]);
    slice<NP>(e1, t1, part, ra[1], rb[1]);
    slice<NP>(t1, R, part, ra[2], rb[2]);
    __syncthreads();

    for (int64_t tile = blockIdx.x; tile * BLK < n; tile += gridDim.x) {
        const int64_t i0 = tile * BLK + slot;
        VjpPoint Q;
        Q.valid = i0 < n;
        const int64_t i = Q.valid ? i0 : n - 1;                   // idle lanes shadow the last point
        // logarithmic form unless a point of the tile has a mass fraction outside 2^+-100 (zero,
        // negative, tiny or non-finite): then the products in double (C_k in the row)
        // (and the logarithmic form sums the cotangents bar_omega_k in pairs: each within 2^+-100
        // or zero).  Decided first, so a pass skips a tile after these loads alone.
        bool bad = false;
        for (int k = part; k < K; k += NP)
            bad |= !log_form_ok(Y[(int64_t)k * ld + i]) || !pair_range_ok(bar_omega[(int64_t)k * ld + i]);
        const bool dvote = __syncthreads_or(bad) != 0;
        if (PASS == 0 ? dvote : !dvote) continue;                 // the other pass takes this tile
        constexpr bool direct = PASS == 1;
        const double Ti = T[i];
        Q.invT = 1.0 / Ti;
        Q.pRT = p[i] * Q.invT * kInvR;
        Q.P = make_tpairs(Ti, Q.invT, dt);
        Q.lnT = df_to_d(Q.P.lnTd);
        Q.hb = HB ? bar_hrr[i] : 0.0;
        Q.hbRT = Q.hb * kR * Ti;
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
        const double rho = Q.pRT / s;
        Q.pRTd = df_split(Q.pRT);
        for (int k = part; k < K; k += NP) {
            const double c = Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * rho;
            const double wb = bar_omega[(int64_t)k * ld + i];
            if (direct) {
                sC[k * BLK] = c;
                sWb[k * BLK] = wb;
            } else {
                const dfl l = log_df(c, dt.rc, dt.lc), w = df_split(wb);
                reinterpret_cast<float2*>(sC)[k * BLK] = make_float2(l.h, l.l);
                reinterpret_cast<float2*>(sWb)[k * BLK] = make_float2(w.h, w.l);
            }
        }
        for (int k = part; k < K; k += NP) sB[k * BLK] = 0.0;
        __syncthreads();

        double Tbar = 0.0;
        if constexpr (NP == 1) {
            if (direct) {
                vjp_group<0, WANT_G, HB>(m, ra[0], rb[0], sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
                vjp_group<1, WANT_G, HB>(m, ra[1], rb[1], sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
                vjp_group<2, WANT_G, HB>(m, ra[2], rb[2], sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
            } else {
                vjp_group_log<0, WANT_G, HB>(m, ra[0], rb[0], sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
                vjp_group_log<1, WANT_G, HB>(m, ra[1], rb[1], sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
                vjp_group_log<2, WANT_G, HB>(m, ra[2], rb[2], sC, sWb, sB, gw, Q, dlnA, dt, Tbar);
            }
        } else {
            // (each round ends with a barrier: the row is complete after the last one)
            vjp_rounds<NP, 0, WANT_G, HB>(m, part, direct, sC, sWb, sB, gw, Q, dlnA, dt, Tbar, sMb);
            vjp_rounds<NP, 1, WANT_G, HB>(m, part, direct, sC, sWb, sB, gw, Q, dlnA, dt, Tbar, sMb);
            vjp_rounds<NP, 2, WANT_G, HB>(m, part, direct, sC, sWb, sB, gw, Q, dlnA, dt, Tbar, sMb);
        }
        if (!direct) Tbar *= Q.invT;                              // the logarithmic form sums T Tbar
        __syncthreads();

        // this part's share of sum_k Cbar_k C_k (in the logarithmic form the row holds
        // S_k = Cbar_k C_k)
        double cc = 0.0;
        for (int k = part; k < K; k += NP) {
            const double cb = sB0[k * BLK];
            cc = direct ? fma(cb, sC[k * BLK], cc) : cc + cb;
        }
        if (NP > 1) {
            // bar_omega is dead: rows 2q, 2q+1 (2 NP <= K) take part q's sums, added in part order
            sWb[(2 * part) * BLK] = cc;
            sWb[(2 * part + 1) * BLK] = Tbar;
            __syncthreads();
            cc = sWb[0];
            Tbar = sWb[BLK];
#pragma unroll
            for (int q = 1; q < NP; ++q) {
                cc += sWb[(2 * q) * BLK];
                Tbar += sWb[(2 * q + 1) * BLK];
            }
        }
        // C_k = rho y_k, rho = p/(R T s), s = sum y_k, y_k = Y_k / W_k:
        // rhobar = sum_k Cbar_k y_k = cc / rho, sbar = -rhobar rho / s, Tbar -= rhobar rho / T
        const double sbar = -cc / s;
        if (Q.valid) {
            if (part == 0) gT[i] = fma(-cc, Q.invT, Tbar);
            for (int k = part; k < K; k += NP) {
                // rho Cbar_k / W_k = S_k / Y_k in the logarithmic form (C_k = rho Y_k / W_k)
                const double iw = __ldg(m.invW + k);
                gY[(int64_t)k * ld + i] = direct ? iw * fma(rho, sB0[k * BLK], sbar)
                                                 : fma(sB0[k * BLK], recip_nr(Y[(int64_t)k * ld + i]), iw * sbar);
            }
        }
        __syncthreads();                                          // before the next tile reuses the rows
    }

    if (WANT_G)
        for (int r = threadIdx.x; r < R; r += NT) ws[(size_t)blockIdx.x * R + r] = gw[r];
}

// g[orig(r)] = sum over blocks of ws[b][r], blocks in order
__global__ void reduce_blocks_kernel(const double* __restrict__ ws, int nblocks, const RxnRec* __restrict__ rxn,
                                     int R, double* __restrict__ g) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += ws[(size_t)b * R + r];
    g[__ldg(&rxn[r].orig)] = acc;
}

// ---------------------------------------------------------------- launch plan
constexpr int kParts[] = {1, 2, 4};

template <bool WANT_G, bool HB, int PASS>
const void* kernel_ptr(int c) {
    switch (c) {
        case 0: return (const void*)vjp_kernel<1, WANT_G, HB, PASS>;
        case 1: return (const void*)vjp_kernel<2, WANT_G, HB, PASS>;
        default: return (const void*)vjp_kernel<4, WANT_G, HB, PASS>;
    }
}

// Per pass: the parts per point with the most resident warps and a grid of resident blocks (the
// fallback pass finds work only in tiles with mass fractions or cotangents outside the pairs'
// range; it reads the rest's Y and bar_omega once to see that).  The ln A partial sums of the two
// passes' blocks lie one after the other in the workspace.
struct VjpPlan {
    int dev, K, R, ms2, ms4, variant;
    int parts_idx[2];   // index into kParts, per pass
    int grid_cap[2];    // blocks of each pass
};
std::mutex g_plan_mu;
std::vector<VjpPlan> g_plans;

template <bool WANT_G, bool HB, int PASS>
bool plan_pass(const DevMech& m, int sms, int per_block, int& parts_idx, int& blocks_per_sm) {
    int best = -1, best_warps = 0;
    for (int c = 0; c < 3; ++c) {
        const int np = kParts[c];
        if (np > 1 && 2 * np > m.K) continue;
        const size_t bytes = vjp_smem(m.K, m.R, vjp_mslots(m, np), WANT_G);
        if (bytes > (size_t)per_block) continue;
        const void* kern = kernel_ptr<WANT_G, HB, PASS>(c);
        if (ensure_smem(kern, bytes) != cudaSuccess) continue;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kVjpBlk * np, bytes) != cudaSuccess)
            continue;
        if (blocks * np > best_warps) {
            best_warps = blocks * np;
            blocks_per_sm = blocks;
            best = c;
        }
    }
    parts_idx = best;
    (void)sms;
    return best >= 0;
}

template <bool WANT_G, bool HB>
bool plan_variant(const DevMech& m, VjpPlan& out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const int variant = (WANT_G ? 1 : 0) | (HB ? 2 : 0);
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const VjpPlan& q : g_plans)
            if (q.dev == dev && q.K == m.K && q.R == m.R && q.ms2 == m.mslots2 && q.ms4 == m.mslots4 &&
                q.variant == variant) {
                out = q;
                return true;
            }
    }
    int per_block = 0, sms = 0;
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int p0 = -1, p1 = -1, b0 = 0, b1 = 0;
    if (!plan_pass<WANT_G, HB, 0>(m, sms, per_block, p0, b0)) return false;
    if (!plan_pass<WANT_G, HB, 1>(m, sms, per_block, p1, b1)) return false;
    out = VjpPlan{dev, m.K, m.R, m.mslots2, m.mslots4, variant, {p0, p1}, {sms * b0, sms * b1}};
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.push_back(out);
    return true;
}

bool plan_for(const DevMech& m, bool want_g, bool hb, VjpPlan& out) {
    if (want_g) return hb ? plan_variant<true, true>(m, out) : plan_variant<true, false>(m, out);
    return hb ? plan_variant<false, true>(m, out) : plan_variant<false, false>(m, out);
}

int64_t vjp_grid(const VjpPlan& pl, int pass, int64_t n) {
    const int64_t tiles = (n + kVjpBlk - 1) / kVjpBlk;
    return tiles < pl.grid_cap[pass] ? tiles : pl.grid_cap[pass];
}

// blocks of both passes, the ln A partial sums' rows in the workspace
int64_t vjp_blocks(const VjpPlan& pl, int64_t n) { return vjp_grid(pl, 0, n) + vjp_grid(pl, 1, n); }

template <bool WANT_G, bool HB, int PASS>
cudaError_t launch_pass(const VjpPlan& pl, const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                        const double* Y, const double* dlnA, const double* bar_omega, const double* bar_hrr,
                        double* gT, double* gY, double* ws, cudaStream_t s) {
    const int np = kParts[pl.parts_idx[PASS]];
    const size_t smem = vjp_smem(m.K, m.R, vjp_mslots(m, np), WANT_G);
    const void* kp = kernel_ptr<WANT_G, HB, PASS>(pl.parts_idx[PASS]);
    cudaError_t e = ensure_smem(kp, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)vjp_grid(pl, PASS, n);
    switch (np) {
        case 1:
            vjp_kernel<1, WANT_G, HB, PASS><<<grid, kVjpBlk, smem, s>>>(m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr,
                                                                        gT, gY, ws);
            break;
        case 2:
            vjp_kernel<2, WANT_G, HB, PASS><<<grid, 2 * kVjpBlk, smem, s>>>(m, n, ld, T, p, Y, dlnA, bar_omega,
                                                                            bar_hrr, gT, gY, ws);
            break;
        default:
            vjp_kernel<4, WANT_G, HB, PASS><<<grid, 4 * kVjpBlk, smem, s>>>(m, n, ld, T, p, Y, dlnA, bar_omega,
                                                                            bar_hrr, gT, gY, ws);
    }
    return cudaGetLastError();
}

template <bool WANT_G, bool HB>
cudaError_t launch_v(const VjpPlan& pl, const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                     const double* Y, const double* dlnA, const double* bar_omega, const double* bar_hrr, double* gT,
                     double* gY, double* ws, cudaStream_t s) {
    cudaError_t e = launch_pass<WANT_G, HB, 0>(pl, m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, ws, s);
    if (e != cudaSuccess) return e;
    double* ws1 = ws ? ws + (size_t)vjp_grid(pl, 0, n) * m.R : nullptr;
    return launch_pass<WANT_G, HB, 1>(pl, m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, ws1, s);
}

}  // namespace

// ---------------------------------------------------------------- no-allocation variant
// Scratch for the per-block ln A partial sums of nk_rates_vjp_noalloc: a fixed device array in
// this library's module, present on every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {
std::mutex g_noalloc_mu;
// device address of the array, per device ordinal, for the life of the process (a device reset
// would invalidate it; the entry point's documentation says not to call it after one)
void* g_noalloc_ptr[64] = {};
}  // namespace

cudaError_t noalloc_scratch(void** ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        // host code may not use the array's name as a device address: ask the runtime once
        // per device, with that device current
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}


size_t vjp_workspace_bytes(const DevMech& m, int64_t n) {
    VjpPlan pl;
    if (!plan_for(m, true, false, pl)) return 0;
    VjpPlan pl2;
    if (!plan_for(m, true, true, pl2)) return 0;
    const int64_t blocks = std::max(vjp_blocks(pl, n), vjp_blocks(pl2, n));   // either cotangent set
    return (size_t)blocks * m.R * sizeof(double);
}

cudaError_t launch_vjp(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                       const double* dlnA, const double* bar_omega, const double* bar_hrr, double* gT, double* gY,
                       double* g_lnA, void* ws, cudaStream_t s) {
    static_assert(kDfTabBytes <= kMathTabDoubles * sizeof(double), "table space");
    const bool want_g = g_lnA != nullptr, hb = bar_hrr != nullptr;
    VjpPlan pl;
    if (!plan_for(m, want_g, hb, pl)) return cudaErrorInvalidConfiguration;
    double* wsd = static_cast<double*>(ws);
    cudaError_t e;
    if (want_g)
        e = hb ? launch_v<true, true>(pl, m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, wsd, s)
               : launch_v<true, false>(pl, m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, wsd, s);
    else
        e = hb ? launch_v<false, true>(pl, m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, nullptr, s)
               : launch_v<false, false>(pl, m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, nullptr, s);
    if (e != cudaSuccess || !want_g) return e;
    reduce_blocks_kernel<<<(m.R + 127) / 128, 128, 0, s>>>(wsd, (int)vjp_blocks(pl, n), m.rxn, m.R, g_lnA);
    return cudaGetLastError();
}

}  // namespace nk
