// Exact Jacobian-vector product of (omega_k, heat release) with respect to (T, Y_k) at fixed
// p: the product the Newton-GMRES stage of the paper approximates by difference quotients
// (Sec. 2, Sec. 4).  Forward-mode differentiation written out by hand, one thread per point,
// rates of progress recomputed in registers (nothing per reaction is stored).
//
// Tangents: with y_k = Y_k/W_k, s = sum y_k, rho = p/(R T s), C_k = rho y_k:
//   d rho/rho = -dT/T - ds/s,  dC_k = C_k d rho/rho + rho dY_k/W_k,
//   d(g_k/RT) = -(h_k/RT) dT/T,  d ln k_f = (beta + Ea/(R T)) dT/T,
//   d ln K_c = -sum nu d(g/RT) - (sum nu) dT/T,
//   d hrr = -sum_k (c_p,k dT omega_k + h_k d omega_k).
// Troe: d ln k = d ln k_inf + d ln P_r/(1+P_r) + ln10 d log10 F with F from the chain rule
// through F_cent(T), c, n, f1.
#include "nk_internal.cuh"

namespace nk {
namespace {

template <int BLK>
__global__ void __launch_bounds__(BLK) jvp_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                  const double* __restrict__ T, const double* __restrict__ p,
                                                  const double* __restrict__ Y, const double* __restrict__ dlnA,
                                                  const double* __restrict__ vT, const double* __restrict__ vY,
                                                  double* __restrict__ omega, double* __restrict__ hrr,
                                                  double* __restrict__ d_omega, double* __restrict__ d_hrr) {
    extern __shared__ double smem_all[];
    const MathTab mt = stage_math_tables(smem_all, m.mtab);
    __syncthreads();
    double* smem = smem_all + kMathTabDoubles;
    const int K = m.K;
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    double* sC = smem + tid;                          // C_k
    double* sG = smem + (size_t)K * BLK + tid;        // g_k/RT
    double* sH = smem + (size_t)2 * K * BLK + tid;    // h_k/RT
    double* sW = smem + (size_t)3 * K * BLK + tid;    // omega_k
    double* sD = smem + (size_t)4 * K * BLK + tid;    // d omega_k

    const double Ti = T[i], pi = p[i], dT = vT[i];
    const double lnT = flog(Ti, mt), invT = 1.0 / Ti;
    const double tT = dT * invT;                      // dT/T
    const double pRT = pi * invT * kInvR;
    double s = 0.0, ds = 0.0;
    for (int k = 0; k < K; ++k) {
        const double iw = __ldg(m.invW + k);
        const double yw = Y[(int64_t)k * ld + i] * iw;
        ds = fma(vY[(int64_t)k * ld + i], iw, ds);
        sC[k * BLK] = yw;
        s += yw;
    }
    const double rho = pRT / s;
    const double arho = -tT - ds / s;                 // d rho / rho
    for (int k = 0; k < K; ++k) {
        const double* c = nasa_range(m, k, Ti);
        sC[k * BLK] *= rho;
        sG[k * BLK] = nasa_gRT(c, Ti, lnT, invT);
        sH[k * BLK] = nasa_hRT(c, Ti, invT);
        sW[k * BLK] = 0.0;
        sD[k * BLK] = 0.0;
    }
    const double lnP0RT = 9.408091968961747 - lnT;   // ln(p0/(R T)), ln(101325/8.314462618) = 9.408...
    const double dpRT = -pRT * tT;

    // dC_k on demand: C_k d rho/rho + rho vY_k / W_k
    auto dC = [&](int k, double Ck) {
        return fma(Ck, arho, rho * vY[(int64_t)k * ld + i] * __ldg(m.invW + k));
    };

    for (int r = 0; r < m.R; ++r) {
        const RxnRec* rec = m.rxn + r;
        const int type = __ldg(&rec->type), nr = __ldg(&rec->nr), np = __ldg(&rec->np);
        const double shift = dlnA ? __ldg(dlnA + __ldg(&rec->orig)) : 0.0;
        double sumg, dsumh;                           // sum nu g/RT, sum nu h/RT
        double fw, dfw, rv, drv;                      // dual-number concentration products
        {
            const int k = __ldg(&rec->sp[0]), nu = __ldg(&rec->nu[0]);
            const double nd = __ldg(&rec->nud[0]);
            const double c = sC[k * BLK], dc = dC(k, c);
            sumg = nd * sG[k * BLK];
            dsumh = nd * sH[k * BLK];
            fw = c;
            dfw = dc;
            for (int j = 1; j < nu; ++j) {
                dfw = fma(dfw, c, fw * dc);
                fw *= c;
            }
        }
#pragma unroll
        for (int e = 1; e < kMaxSide; ++e) {
            if (e < nr) {
                const int k = __ldg(&rec->sp[e]), nu = __ldg(&rec->nu[e]);
                const double nd = __ldg(&rec->nud[e]);
                const double c = sC[k * BLK], dc = dC(k, c);
                sumg = fma(nd, sG[k * BLK], sumg);
                dsumh = fma(nd, sH[k * BLK], dsumh);
                for (int j = 0; j < nu; ++j) {
                    dfw = fma(dfw, c, fw * dc);
                    fw *= c;
                }
            }
        }
        {
            const int k = __ldg(&rec->sp[kMaxSide]), nu = __ldg(&rec->nu[kMaxSide]);
            const double nd = __ldg(&rec->nud[kMaxSide]);
            const double c = sC[k * BLK], dc = dC(k, c);
            sumg = fma(nd, sG[k * BLK], sumg);
            dsumh = fma(nd, sH[k * BLK], dsumh);
            rv = c;
            drv = dc;
            for (int j = 1; j < nu; ++j) {
                drv = fma(drv, c, rv * dc);
                rv *= c;
            }
        }
#pragma unroll
        for (int e = 1; e < kMaxSide; ++e) {
            if (e < np) {
                const int k = __ldg(&rec->sp[kMaxSide + e]), nu = __ldg(&rec->nu[kMaxSide + e]);
                const double nd = __ldg(&rec->nud[kMaxSide + e]);
                const double c = sC[k * BLK], dc = dC(k, c);
                sumg = fma(nd, sG[k * BLK], sumg);
                dsumh = fma(nd, sH[k * BLK], dsumh);
                for (int j = 0; j < nu; ++j) {
                    drv = fma(drv, c, rv * dc);
                    rv *= c;
                }
            }
        }
        const double dnu = __ldg(&rec->dnu);
        const double lnKc = fma(dnu, lnP0RT, -sumg);
        // d(sum nu g/RT) = -(dT/T) sum nu h/RT;  d ln(p0/RT) = -dT/T
        const double dlnKc = fma(tT, dsumh, -dnu * tT);

        const double beta = __ldg(&rec->beta), EaR = __ldg(&rec->EaR);
        const double lnkf = fma(-EaR, invT, fma(beta, lnT, dlnA ? __ldg(&rec->lnA) + shift : __ldg(&rec->lnA)));
        double dlnkf = fma(EaR, invT, beta) * tT;

        double M = 0.0, dM = 0.0;
        if (type != NK_RXN_ELEMENTARY) {
            M = pRT;
            dM = dpRT;
            const int e0 = __ldg(&rec->eff0), e1 = __ldg(&rec->eff1);
            for (int j = e0; j < e1; ++j) {
                const int k = __ldg(m.eff_sp + j);
                const double em1 = __ldg(m.eff_m1 + j), c = sC[k * BLK];
                M = fma(em1, c, M);
                dM = fma(em1, dC(k, c), dM);
            }
        }

        double kf;
        if (type == NK_RXN_TROE) {
            const TroeRec* t = m.troe + __ldg(&rec->aux);
            const double beta0 = __ldg(&t->beta0), Ea0R = __ldg(&t->Ea0R);
            const double lnk0 = fma(-Ea0R, invT, fma(beta0, lnT, __ldg(&t->lnA0) + shift));
            const double dlnk0 = fma(Ea0R, invT, beta0) * tT;
            if (M == 0.0) {
                kf = 0.0;
                dlnkf = 0.0;
            } else {
                const double lnPr = lnk0 - lnkf + flog(M, mt);
                const double dlnPr = dlnk0 - dlnkf + dM / M;
                const double a = __ldg(&t->a), i3 = __ldg(&t->invT3), i1 = __ldg(&t->invT1);
                const double e3 = fexp(-Ti * i3, mt), e1 = fexp(-Ti * i1, mt);
                double Fc = (1.0 - a) * e3 + a * e1;
                double dFc = -((1.0 - a) * i3 * e3 + a * i1 * e1) * dT;
                if (__ldg(&t->hasT2) != 0.0) {
                    const double T2 = __ldg(&t->T2), e2 = fexp(-T2 * invT, mt);
                    Fc += e2;
                    dFc = fma(T2 * invT * e2, tT, dFc);
                }
                const double lFc = flog(Fc, mt) * kInvLn10, dlFc = dFc / Fc * kInvLn10;
                const double c = -0.4 - 0.67 * lFc, nn = 0.75 - 1.27 * lFc;
                const double u = fma(lnPr, kInvLn10, c), du = fma(dlnPr, kInvLn10, -0.67 * dlFc);
                const double v = fma(-0.14, u, nn), dv = fma(-0.14, du, -1.27 * dlFc);
                const double f1 = u / v, df1 = fma(-f1, dv, du) / v;
                const double den = fma(f1, f1, 1.0);
                const double lF = lFc / den;
                const double dlF = fma(-2.0 * lF * f1, df1, dlFc) / den;
                const double g = 1.0 / (1.0 + fexp(-lnPr, mt));     // P_r / (1 + P_r)
                kf = fexp(lnkf, mt) * g * fexp(lF * kLn10, mt);
                dlnkf = dlnkf + dlnPr * (1.0 - g) + kLn10 * dlF;
            }
        } else {
            kf = fexp(lnkf, mt);
        }
        const double kr = kf * fexp(-lnKc, mt);
        const double dkf = kf * dlnkf, dkr = kr * (dlnkf - dlnKc);
        double q = fma(kf, fw, -kr * rv);
        double dq = fma(dkf, fw, kf * dfw) - fma(dkr, rv, kr * drv);
        if (type == NK_RXN_THIRD_BODY) {
            dq = fma(dq, M, q * dM);
            q *= M;
        }
#pragma unroll
        for (int e = 0; e < kMaxSide; ++e) {
            if (e < nr) {
                const int k = __ldg(&rec->sp[e]);
                const double nd = __ldg(&rec->nud[e]);
                sW[k * BLK] = fma(nd, q, sW[k * BLK]);
                sD[k * BLK] = fma(nd, dq, sD[k * BLK]);
            }
        }
#pragma unroll
        for (int e = 0; e < kMaxSide; ++e) {
            if (e < np) {
                const int k = __ldg(&rec->sp[kMaxSide + e]);
                const double nd = __ldg(&rec->nud[kMaxSide + e]);
                sW[k * BLK] = fma(nd, q, sW[k * BLK]);
                sD[k * BLK] = fma(nd, dq, sD[k * BLK]);
            }
        }
    }

    double h = 0.0, dh = 0.0;
    for (int k = 0; k < K; ++k) {
        const double w = sW[k * BLK], dw = sD[k * BLK];
        const double cpR = nasa_cpR(nasa_range(m, k, Ti), Ti);
        h = fma(sH[k * BLK], w, h);
        dh = fma(sH[k * BLK] * Ti, dw, fma(cpR * dT, w, dh));
        d_omega[(int64_t)k * ld + i] = dw;
        if (omega) omega[(int64_t)k * ld + i] = w;
    }
    d_hrr[i] = -kR * dh;                              // -sum (c_p,k dT omega_k + h_k d omega_k)
    if (hrr) hrr[i] = -kR * Ti * h;
}

template <int BLK>
cudaError_t launch_t(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     const double* dlnA, const double* vT, const double* vY, double* omega, double* hrr,
                     double* d_omega, double* d_hrr, size_t smem, cudaStream_t s) {
    auto kern = jvp_kernel<BLK>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + BLK - 1) / BLK;
    kern<<<(unsigned)grid, BLK, smem, s>>>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_jvp(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* vT, const double* vY, double* omega,
                       double* hrr, double* d_omega, double* d_hrr, cudaStream_t s) {
    const size_t per_thread = (size_t)5 * m.K * sizeof(double);
    const size_t tab = kMathTabDoubles * sizeof(double);
    const int blk = pick_block_occupancy(per_thread, tab);
    if (!blk) return cudaErrorInvalidConfiguration;
    const size_t smem = per_thread * blk + tab;
    switch (blk) {
        case 128: return launch_t<128>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, smem, s);
        case 64: return launch_t<64>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, smem, s);
        case 32: return launch_t<32>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, smem, s);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace nk
