// Net species production rates omega_k and heat release per point (the "rates" kernel of
// the paper, Tab. 3-4; omega_k of Eq. 1a, heat release of Eq. 1b).
//
// Layout: one thread per point.  Every thread of a warp walks the same reaction at the same
// time, so the reaction record is a broadcast load and all control flow is uniform (no
// divergence from reaction types or stoichiometry).  The per-point species state
// (concentrations C_k, g_k/RT and the omega_k accumulators) lives in shared memory as
// [species][thread], so that the runtime species indices of a reaction hit one bank row.
//
// FP64 form: every operation in double precision.
// Mixed form: the Arrhenius argument ln A + beta ln T - Ea/(RT), k_f and the whole Troe
// falloff in single precision; equilibrium constants (the sum of nu_k g_k/RT and its
// exponential), the forward-minus-reverse difference and the omega accumulation in double.
#include "nk_internal.cuh"

namespace nk {
namespace {

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
    int type, nr, np, aux;
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
    const int4* q = reinterpret_cast<const int4*>(rec) + 2;
    const int4 h = __ldg(q), s0 = __ldg(q + 1), s1 = __ldg(q + 2), u0 = __ldg(q + 3), u1 = __ldg(q + 4);
    x.type = h.x;
    x.nr = h.y;
    x.np = h.z;
    x.aux = h.w;
    x.sp[0] = s0.x; x.sp[1] = s0.y; x.sp[2] = s0.z; x.sp[3] = s0.w;
    x.sp[4] = s1.x; x.sp[5] = s1.y; x.sp[6] = s1.z; x.sp[7] = s1.w;
    x.nu[0] = u0.x; x.nu[1] = u0.y; x.nu[2] = u0.z; x.nu[3] = u0.w;
    x.nu[4] = u1.x; x.nu[5] = u1.y; x.nu[6] = u1.z; x.nu[7] = u1.w;
    return x;
}

template <int BLK, bool MIXED>
__global__ void __launch_bounds__(BLK) rates_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                    const double* __restrict__ T, const double* __restrict__ p,
                                                    const double* __restrict__ Y,
                                                    const double* __restrict__ dlnA,
                                                    double* __restrict__ omega, double* __restrict__ hrr) {
    extern __shared__ double smem[];
    const int K = m.K;
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    double* sC = smem + tid;                          // C_k       at sC[k * BLK]
    double* sG = smem + (size_t)K * BLK + tid;        // g_k / RT
    double* sW = smem + (size_t)2 * K * BLK + tid;    // omega_k accumulators

    const double Ti = T[i], pi = p[i];
    const double lnT = log(Ti), invT = 1.0 / Ti;
    const double pRT = pi * invT * kInvR;             // p/(RT) = sum_k C_k
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double yw = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
        sC[k * BLK] = yw;
        s += yw;
    }
    const double rho_w = pRT / s;                     // rho = p Wbar/(RT) with Wbar = 1/s
    for (int k = 0; k < K; ++k) {
        sC[k * BLK] *= rho_w;                         // C_k = rho Y_k / W_k
        sG[k * BLK] = nasa_gRT(nasa_range(m, k, Ti), Ti, lnT, invT);
        sW[k * BLK] = 0.0;
    }
    const double lnP0RT = log(kP0 * kInvR) - lnT;    // ln(p0/(R T))
    const float lnTf = (float)lnT, invTf = (float)invT, Tf = (float)Ti;

    for (int r = 0; r < m.R; ++r) {
        const Rxn x = load_rxn(m.rxn + r);
        const double shift = dlnA ? __ldg(dlnA + r) : 0.0;
        // Gibbs sum and concentration products over the reaction's entries
        double sumg = 0.0, fw = 1.0, rv = 1.0;
#pragma unroll
        for (int e = 0; e < kMaxSide; ++e) {
            if (e < x.nr) {
                const int k = x.sp[e];
                const double c = sC[k * BLK], g = sG[k * BLK];
                if (x.nu[e] == 1) {
                    sumg -= g;
                    fw *= c;
                } else {
                    sumg = fma(-(double)x.nu[e], g, sumg);
                    fw *= ipow(c, x.nu[e]);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < kMaxSide; ++e) {
            if (e < x.np) {
                const int k = x.sp[kMaxSide + e];
                const double c = sC[k * BLK], g = sG[k * BLK];
                if (x.nu[kMaxSide + e] == 1) {
                    sumg += g;
                    rv *= c;
                } else {
                    sumg = fma((double)x.nu[kMaxSide + e], g, sumg);
                    rv *= ipow(c, x.nu[kMaxSide + e]);
                }
            }
        }
        const double lnKc = fma(x.dnu, lnP0RT, -sumg);   // ln K_c = -sum nu g/RT + sum nu ln(p0/RT)

        double M = 0.0;
        if (x.type != NK_RXN_ELEMENTARY) {
            M = pRT;
            const int e0 = __ldg(m.eff_ptr + r), e1 = __ldg(m.eff_ptr + r + 1);
            for (int j = e0; j < e1; ++j) M = fma(__ldg(m.eff_m1 + j), sC[__ldg(m.eff_sp + j) * BLK], M);
        }

        double kf, kr;
        if constexpr (!MIXED) {
            const double lnkf = fma(-x.EaR, invT, fma(x.beta, lnT, x.lnA + shift));
            if (x.type == NK_RXN_TROE) {
                const TroeRec* t = m.troe + x.aux;
                const double lnk0 = fma(-__ldg(&t->Ea0R), invT, fma(__ldg(&t->beta0), lnT, __ldg(&t->lnA0) + shift));
                if (M == 0.0) {
                    kf = 0.0;                              // P_r = 0: falloff rate vanishes
                } else {
                    const double lnPr = lnk0 - lnkf + log(M);
                    const double a = __ldg(&t->a);
                    double Fcent = (1.0 - a) * exp(-Ti * __ldg(&t->invT3)) + a * exp(-Ti * __ldg(&t->invT1));
                    if (__ldg(&t->hasT2) != 0.0) Fcent += exp(-__ldg(&t->T2) * invT);
                    const double lFc = log(Fcent) * kInvLn10;
                    const double c = -0.4 - 0.67 * lFc;
                    const double nn = 0.75 - 1.27 * lFc;
                    const double u = fma(lnPr, kInvLn10, c);
                    const double f1 = u / fma(-0.14, u, nn);
                    const double lF = lFc / fma(f1, f1, 1.0);
                    kf = exp(lnkf) * (1.0 / (1.0 + exp(-lnPr))) * exp(lF * kLn10);   // P_r/(1+P_r) = 1/(1+1/P_r)
                }
                kr = kf * exp(-lnKc);
            } else {
                kf = exp(lnkf);
                kr = exp(lnkf - lnKc);
            }
        } else {
            const float4 xf4 = __ldg(reinterpret_cast<const float4*>(m.rxnf + r));
            const RxnRecF xf{xf4.x, xf4.y, xf4.z, xf4.w};
            const float shf = (float)shift;
            const float lnkf = fmaf(-xf.EaR, invTf, fmaf(xf.beta, lnTf, xf.lnA + shf));
            if (x.type == NK_RXN_TROE) {
                const TroeRecF* t = m.troef + x.aux;
                const float4 t0 = __ldg(reinterpret_cast<const float4*>(t));
                const float4 t1 = __ldg(reinterpret_cast<const float4*>(t) + 1);
                // t0 = (lnA0, beta0, Ea0R, a), t1 = (invT3, invT1, T2, hasT2)
                const float lnk0 = fmaf(-t0.z, invTf, fmaf(t0.y, lnTf, t0.x + shf));
                if (M == 0.0) {
                    kf = 0.0;
                } else {
                    const float lnPr = lnk0 - lnkf + logf((float)M);
                    const float a = t0.w;
                    float Fcent = (1.0f - a) * expf(-Tf * t1.x) + a * expf(-Tf * t1.y);
                    if (t1.w != 0.0f) Fcent += expf(-t1.z * invTf);
                    const float lFc = log10f(Fcent);
                    const float c = -0.4f - 0.67f * lFc;
                    const float nn = 0.75f - 1.27f * lFc;
                    const float u = fmaf(lnPr, (float)kInvLn10, c);
                    const float f1 = u / fmaf(-0.14f, u, nn);
                    const float lF = lFc / fmaf(f1, f1, 1.0f);
                    const float g = 1.0f / (1.0f + expf(-lnPr));          // P_r / (1 + P_r)
                    kf = exp_f32_to_f64(lnkf) * (double)(g * exp10f(lF));
                }
            } else {
                kf = exp_f32_to_f64(lnkf);
            }
            kr = kf * exp(-lnKc);
        }
        double q = fma(kf, fw, -kr * rv);
        if (x.type == NK_RXN_THIRD_BODY) q *= M;

#pragma unroll
        for (int e = 0; e < kMaxSide; ++e) {
            if (e < x.nr) {
                const int k = x.sp[e];
                sW[k * BLK] -= (x.nu[e] == 1) ? q : (double)x.nu[e] * q;
            }
        }
#pragma unroll
        for (int e = 0; e < kMaxSide; ++e) {
            if (e < x.np) {
                const int k = x.sp[kMaxSide + e];
                sW[k * BLK] += (x.nu[kMaxSide + e] == 1) ? q : (double)x.nu[kMaxSide + e] * q;
            }
        }
    }

    double h = 0.0;
    for (int k = 0; k < K; ++k) {
        const double w = sW[k * BLK];
        omega[(int64_t)k * ld + i] = w;
        h = fma(nasa_hRT(nasa_range(m, k, Ti), Ti, invT), w, h);
    }
    hrr[i] = -kR * Ti * h;                            // -sum_k h_k omega_k
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
    const size_t lim = smem_limit();
    int blk = pick_block(per_thread, lim / 2);
    if (!blk) blk = pick_block(per_thread, lim);
    if (!blk) return cudaErrorInvalidConfiguration;
    const size_t smem = per_thread * blk;
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
