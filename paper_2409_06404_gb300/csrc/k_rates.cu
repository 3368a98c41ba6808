// Net species production rates omega_k and heat release per point (the "rates" kernel of
// the paper, Tab. 3-4; omega_k of Eq. 1a, heat release of Eq. 1b).
//
// Layout: one thread per point.  Every thread of a warp walks the same reaction at the same
// time, so reaction records are broadcast loads and control flow is uniform.  The device
// copy of the mechanism groups reactions by kind (elementary, third-body, Troe); each kind
// has its own branch-free loop that takes two reactions per iteration, giving the FP64 pipe
// two independent dependency chains per warp.  The per-point species state (C_k, g_k/RT and
// the omega_k accumulators) lives in shared memory as [species][thread].
//
// FP64 form: every operation in double precision (exp/log from nk_math.cuh).
// Mixed form: the Arrhenius argument ln A + beta ln T - Ea/(RT), k_f and the whole Troe
// falloff in single precision; equilibrium constants (the sum of nu_k g_k/RT and its
// exponential), the forward-minus-reverse difference and the omega accumulation in double.
#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr double kLnP0overR = 9.408091968961747;   // ln(101325 Pa / (8.314462618 J/mol/K))

// exp of a single-precision argument, returned in double: x = n ln2 + r (Cody-Waite two-term
// split of ln 2), expf(r) with |r| <= ln2/2, and 2^n added to the exponent field of the
// double, so results beyond the single-precision range stay representable.
__device__ __forceinline__ double exp_f32_to_f64(float x) {
    if (x < -700.0f) return 0.0;
    if (x > 700.0f) return __longlong_as_double(0x7ff0000000000000LL);
    const float nf = rintf(x * 1.44269504089f);
    float r = fmaf(nf, -0.693359375f, x);
    r = fmaf(nf, 2.12194440054690583e-4f, r);
    const double e = (double)expf(r);
    return __longlong_as_double(__double_as_longlong(e) + ((long long)(int)nf << 52));
}

struct Rxn {
    double lnA, beta, EaR, dnu;
    double nud[2 * kMaxSide];
    int type, nr, np, aux, orig, eff0, eff1;
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
    x.sp[0] = s0.x; x.sp[1] = s0.y; x.sp[2] = s0.z; x.sp[3] = s0.w;
    x.sp[4] = s1.x; x.sp[5] = s1.y; x.sp[6] = s1.z; x.sp[7] = s1.w;
    x.nu[0] = u0.x; x.nu[1] = u0.y; x.nu[2] = u0.z; x.nu[3] = u0.w;
    x.nu[4] = u1.x; x.nu[5] = u1.y; x.nu[6] = u1.z; x.nu[7] = u1.w;
    return x;
}

// Per-point quantities shared by all reactions.
struct Pt {
    double T, lnT, invT, pRT, lnP0RT;
    float Tf, lnTf, invTf;
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
// r is the reaction's position in the device order.
template <int BLK, bool MIXED, int KIND>
__device__ __forceinline__ double rate_of_progress(const DevMech& m, const Rxn& x, int r, const double* sC,
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
    if constexpr (!MIXED) {
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
    } else {
        const float4 xf = __ldg(reinterpret_cast<const float4*>(m.rxnf + r));   // lnA, beta, EaR
        const float shf = (float)shift;
        const float lnkf = fmaf(-xf.z, P.invTf, fmaf(xf.y, P.lnTf, xf.x + shf));
        if constexpr (KIND == 2) {
            const float4 t0 = __ldg(reinterpret_cast<const float4*>(m.troef + x.aux));       // lnA0, beta0, Ea0R, a
            const float4 t1 = __ldg(reinterpret_cast<const float4*>(m.troef + x.aux) + 1);   // 1/T3, 1/T1, T2, has
            if (M == 0.0) {
                kf = 0.0;
            } else {
                const float lnk0 = fmaf(-t0.z, P.invTf, fmaf(t0.y, P.lnTf, t0.x + shf));
                const float lnPr = lnk0 - lnkf + logf((float)M);
                float Fc = (1.0f - t0.w) * expf(-P.Tf * t1.x) + t0.w * expf(-P.Tf * t1.y);
                if (t1.w != 0.0f) Fc += expf(-t1.z * P.invTf);
                const float lFc = log10f(Fc);
                const float c = fmaf(-0.67f, lFc, -0.4f);
                const float nn = fmaf(-1.27f, lFc, 0.75f);
                const float u = fmaf(lnPr, (float)kInvLn10, c);
                const float f1 = u / fmaf(-0.14f, u, nn);
                const float lF = lFc / fmaf(f1, f1, 1.0f);
                kf = exp_f32_to_f64(lnkf) * (double)(exp10f(lF) / (1.0f + expf(-lnPr)));
            }
        } else {
            kf = exp_f32_to_f64(lnkf);
        }
        kr = kf * fexp(-lnKc, mt);
    }
    double q = fma(kf, fw, -kr * rv);
    if (KIND == 1) q *= M;
    return q;
}

template <int BLK>
__device__ __forceinline__ void scatter(const Rxn& x, double* sW, double q) {
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.nr) {
            double* w = sW + x.sp[e] * BLK;
            *w = fma(x.nud[e], q, *w);
        }
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.np) {
            double* w = sW + x.sp[kMaxSide + e] * BLK;
            *w = fma(x.nud[kMaxSide + e], q, *w);
        }
}

// All reactions of one kind, two per iteration.
template <int BLK, bool MIXED, int KIND>
__device__ __forceinline__ void reaction_group(const DevMech& m, int r0, int r1, const double* sC, const double* sG,
                                               double* sW, const Pt& P, const double* dlnA, const MathTab& mt) {
    for (int r = r0; r < r1; r += 2) {
        const Rxn a = load_rxn(m.rxn + r);
        if (r + 1 < r1) {
            const Rxn b = load_rxn(m.rxn + r + 1);
            const double qa = rate_of_progress<BLK, MIXED, KIND>(m, a, r, sC, sG, P, dlnA, mt);
            const double qb = rate_of_progress<BLK, MIXED, KIND>(m, b, r + 1, sC, sG, P, dlnA, mt);
            scatter<BLK>(a, sW, qa);
            scatter<BLK>(b, sW, qb);
        } else {
            scatter<BLK>(a, sW, rate_of_progress<BLK, MIXED, KIND>(m, a, r, sC, sG, P, dlnA, mt));
        }
    }
}

template <int BLK, bool MIXED>
__global__ void __launch_bounds__(BLK) rates_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                    const double* __restrict__ T, const double* __restrict__ p,
                                                    const double* __restrict__ Y,
                                                    const double* __restrict__ dlnA,
                                                    double* __restrict__ omega, double* __restrict__ hrr) {
    extern __shared__ double smem[];
    const MathTab mt = stage_math_tables(smem, m.mtab);
    __syncthreads();
    const int K = m.K;
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    double* sC = smem + kMathTabDoubles + tid;                       // C_k       at sC[k * BLK]
    double* sG = smem + kMathTabDoubles + (size_t)K * BLK + tid;     // g_k / RT
    double* sW = smem + kMathTabDoubles + (size_t)2 * K * BLK + tid; // omega_k accumulators

    Pt P;
    P.T = T[i];
    P.lnT = flog(P.T, mt);
    P.invT = 1.0 / P.T;
    P.pRT = p[i] * P.invT * kInvR;                     // p/(RT) = sum_k C_k
    P.lnP0RT = kLnP0overR - P.lnT;                     // ln(p0/(R T))
    P.Tf = (float)P.T;
    P.lnTf = (float)P.lnT;
    P.invTf = (float)P.invT;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double yw = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
        sC[k * BLK] = yw;
        s += yw;
    }
    const double rho_w = P.pRT / s;                    // rho = p Wbar/(RT) with Wbar = 1/s
    for (int k = 0; k < K; ++k) {
        sC[k * BLK] *= rho_w;                          // C_k = rho Y_k / W_k
        sG[k * BLK] = nasa_gRT(nasa_range(m, k, P.T), P.T, P.lnT, P.invT);
        sW[k * BLK] = 0.0;
    }
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    reaction_group<BLK, MIXED, 0>(m, 0, e1, sC, sG, sW, P, dlnA, mt);
    reaction_group<BLK, MIXED, 1>(m, e1, t1, sC, sG, sW, P, dlnA, mt);
    reaction_group<BLK, MIXED, 2>(m, t1, m.R, sC, sG, sW, P, dlnA, mt);

    double h = 0.0;
    for (int k = 0; k < K; ++k) {
        const double w = sW[k * BLK];
        omega[(int64_t)k * ld + i] = w;
        h = fma(nasa_hRT(nasa_range(m, k, P.T), P.T, P.invT), w, h);
    }
    hrr[i] = -kR * P.T * h;                            // -sum_k h_k omega_k
}

template <int BLK, bool MIXED>
cudaError_t launch_t(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     const double* dlnA, double* omega, double* hrr, size_t smem, cudaStream_t s) {
    auto kern = rates_kernel<BLK, MIXED>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + BLK - 1) / BLK;
    kern<<<(unsigned)grid, BLK, smem, s>>>(m, n, ld, T, p, Y, dlnA, omega, hrr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rates(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                         const double* Y, const double* dlnA, double* omega, double* hrr, int precision,
                         cudaStream_t s) {
    const size_t per_thread = (size_t)3 * m.K * sizeof(double);
    const size_t tab = kMathTabDoubles * sizeof(double);
    const int blk = pick_block_occupancy(per_thread, tab);
    if (!blk) return cudaErrorInvalidConfiguration;
    const size_t smem = per_thread * blk + tab;
    const bool mixed = precision == NK_MIXED;
#define NK_RATES_CASE(B)                                                                                   \
    case B:                                                                                                \
        return mixed ? launch_t<B, true>(m, n, ld, T, p, Y, dlnA, omega, hrr, smem, s)                     \
                     : launch_t<B, false>(m, n, ld, T, p, Y, dlnA, omega, hrr, smem, s);
    switch (blk) {
        NK_RATES_CASE(128)
        NK_RATES_CASE(64)
        NK_RATES_CASE(32)
    }
#undef NK_RATES_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace nk
