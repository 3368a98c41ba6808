// Vector-Jacobian product of (omega_k, heat release): reverse-mode differentiation written
// out by hand, the exact transpose of the JVP (gradients for mechanism calibration and for
// adjoint solves).  One thread per point, rates of progress recomputed in registers.
//
// Single pass over the reactions: with hrr = -sum_k h_k omega_k and omega_k = sum_r nu_kr q_r,
//   qbar_r = sum_k nu_kr (bar_omega_k - bar_hrr h_k)
//   Tbar  += -bar_hrr R q_r sum_k nu_kr c_p,k/R          (temperature dependence of h_k)
// so the forward values omega_k are never needed.  The ln A gradient of a point is
// qbar_r q_r (a shift of ln A_r scales k_f and k_r alike, and both limits of a Troe reaction);
// it is summed over the points of a warp by shuffles, over the warps of a block in shared
// memory, and over blocks by a second kernel in a fixed order: deterministic, no atomics.
#include <mutex>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kVjpMaxBlocks = 1024;

int vjp_block(const DevMech& m) {
    const size_t per_thread = (size_t)5 * m.K * sizeof(double);
    // per block the math tables, per warp its ln A accumulators
    return pick_block_occupancy(per_thread, kMathTabDoubles * sizeof(double), (size_t)m.R * sizeof(double));
}

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

template <int BLK, bool WANT_G>
__global__ void __launch_bounds__(BLK) vjp_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                  const double* __restrict__ T, const double* __restrict__ p,
                                                  const double* __restrict__ Y, const double* __restrict__ dlnA,
                                                  const double* __restrict__ bar_omega,
                                                  const double* __restrict__ bar_hrr, double* __restrict__ gT,
                                                  double* __restrict__ gY, double* __restrict__ ws) {
    extern __shared__ double smem_all[];
    const MathTab mt = stage_math_tables(smem_all, m.mtab);
    __syncthreads();
    double* smem = smem_all + kMathTabDoubles;
    const int K = m.K, R = m.R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* sC = smem + tid;                          // C_k
    double* sG = smem + (size_t)K * BLK + tid;        // g_k/RT
    double* sH = smem + (size_t)2 * K * BLK + tid;    // h_k/RT
    double* sP = smem + (size_t)3 * K * BLK + tid;    // c_p,k/R
    double* sB = smem + (size_t)4 * K * BLK + tid;    // Cbar_k
    double* gw = smem + (size_t)5 * K * BLK + (size_t)warp * R;   // per-warp ln A partial sums
    if (WANT_G) {
        for (int r = lane; r < R; r += 32) gw[r] = 0.0;
        __syncwarp();
    }

    for (int64_t base = (int64_t)blockIdx.x * BLK; base < n; base += (int64_t)gridDim.x * BLK) {
        const int64_t i0 = base + tid;
        const bool valid = i0 < n;
        const int64_t i = valid ? i0 : n - 1;         // idle lanes shadow the last point
        const double Ti = T[i], pi = p[i];
        const double lnT = flog(Ti, mt), invT = 1.0 / Ti;
        const double pRT = pi * invT * kInvR;
        const bool hb_any = bar_hrr != nullptr;            // uniform: heat-release cotangent given
        const double hb = hb_any ? bar_hrr[i] : 0.0;
        const double hbRT = hb * kR * Ti;
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double yw = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
            sC[k * BLK] = yw;
            s += yw;
        }
        const double rho = pRT / s;
        for (int k = 0; k < K; ++k) {
            const double* c = nasa_range(m, k, Ti);
            sC[k * BLK] *= rho;
            sG[k * BLK] = nasa_gRT(c, Ti, lnT, invT);
            sH[k * BLK] = nasa_hRT(c, Ti, invT);
            if (hb_any) sP[k * BLK] = nasa_cpR(c, Ti);
            sB[k * BLK] = 0.0;
        }
        const double lnP0RT = 9.408091968961747 - lnT;   // ln(p0/(R T)), ln(101325/8.314462618) = 9.408...
        double Tbar = 0.0;

        for (int r = 0; r < R; ++r) {
            const RxnRec* rec = m.rxn + r;
            const int type = __ldg(&rec->type), nr = __ldg(&rec->nr), np = __ldg(&rec->np);
            const int orig = __ldg(&rec->orig);
            double lnA = __ldg(&rec->lnA), shift = 0.0;
            if (dlnA) {
                shift = __ldg(dlnA + orig);
                lnA += shift;
            }
            // sums over the entries (signed coefficients) and the concentration powers
            double sumg = 0.0, sumh = 0.0, sumcp = 0.0, wsum = 0.0;
            double cR[kMaxSide], pR[kMaxSide], cP[kMaxSide], pP[kMaxSide];
#pragma unroll
            for (int e = 0; e < kMaxSide; ++e) {
                cR[e] = pR[e] = cP[e] = pP[e] = 1.0;
                if (e < nr) {
                    const int k = __ldg(&rec->sp[e]), nu = __ldg(&rec->nu[e]);
                    const double nd = __ldg(&rec->nud[e]);
                    sumg = fma(nd, sG[k * BLK], sumg);
                    sumh = fma(nd, sH[k * BLK], sumh);
                    if (hb_any) sumcp = fma(nd, sP[k * BLK], sumcp);
                    wsum = fma(nd, bar_omega[(int64_t)k * ld + i], wsum);
                    const double c = sC[k * BLK];
                    double pw = c;
                    for (int j = 1; j < nu; ++j) pw *= c;
                    cR[e] = c;
                    pR[e] = pw;
                }
                if (e < np) {
                    const int k = __ldg(&rec->sp[kMaxSide + e]), nu = __ldg(&rec->nu[kMaxSide + e]);
                    const double nd = __ldg(&rec->nud[kMaxSide + e]);
                    sumg = fma(nd, sG[k * BLK], sumg);
                    sumh = fma(nd, sH[k * BLK], sumh);
                    if (hb_any) sumcp = fma(nd, sP[k * BLK], sumcp);
                    wsum = fma(nd, bar_omega[(int64_t)k * ld + i], wsum);
                    const double c = sC[k * BLK];
                    double pw = c;
                    for (int j = 1; j < nu; ++j) pw *= c;
                    cP[e] = c;
                    pP[e] = pw;
                }
            }
            // products of all entries but one: exR[e] = prod_{f != e} pR[f] (uniform switch)
            double exR[kMaxSide], exP[kMaxSide];
            double fw = exclusive_products(pR, nr, exR);
            double rv = exclusive_products(pP, np, exP);
            const double dnu = __ldg(&rec->dnu);
            const double lnKc = fma(dnu, lnP0RT, -sumg);
            const double beta = __ldg(&rec->beta), EaR = __ldg(&rec->EaR);
            const double lnkf = fma(-EaR, invT, fma(beta, lnT, lnA));

            double M = 0.0;
            if (type != NK_RXN_ELEMENTARY) {
                M = pRT;
                const int e0 = __ldg(&rec->eff0), e1 = __ldg(&rec->eff1);
                for (int j = e0; j < e1; ++j) M = fma(__ldg(m.eff_m1 + j), sC[__ldg(m.eff_sp + j) * BLK], M);
            }

            // ---- primal (kept values for the adjoint)
            double kf;
            double tr_g = 0.0, tr_lF = 0.0, tr_f1 = 0.0, tr_den = 1.0, tr_u = 0.0, tr_v = 1.0, tr_nn = 0.0,
                   tr_Fc = 1.0, tr_dFc = 0.0;
            const TroeRec* t = nullptr;
            if (type == NK_RXN_TROE) {
                t = m.troe + __ldg(&rec->aux);
                const double lnk0 =
                    fma(-__ldg(&t->Ea0R), invT, fma(__ldg(&t->beta0), lnT, __ldg(&t->lnA0) + shift));
                if (M == 0.0) {
                    kf = 0.0;
                } else {
                    const double lnPr = lnk0 - lnkf + flog(M, mt);
                    const double a = __ldg(&t->a), i3 = __ldg(&t->invT3), i1 = __ldg(&t->invT1);
                    const double e3 = fexp(-Ti * i3, mt), e1 = fexp(-Ti * i1, mt);
                    tr_Fc = (1.0 - a) * e3 + a * e1;
                    tr_dFc = -((1.0 - a) * i3 * e3 + a * i1 * e1);
                    if (__ldg(&t->hasT2) != 0.0) {
                        const double T2 = __ldg(&t->T2), e2 = fexp(-T2 * invT, mt);
                        tr_Fc += e2;
                        tr_dFc = fma(T2 * invT * invT, e2, tr_dFc);
                    }
                    const double lFc = flog(tr_Fc, mt) * kInvLn10;
                    const double c = fma(-0.67, lFc, -0.4);
                    tr_nn = fma(-1.27, lFc, 0.75);
                    tr_u = fma(lnPr, kInvLn10, c);
                    tr_v = fma(-0.14, tr_u, tr_nn);
                    tr_f1 = tr_u / tr_v;
                    tr_den = fma(tr_f1, tr_f1, 1.0);
                    tr_lF = lFc / tr_den;
                    tr_g = 1.0 / (1.0 + fexp(-lnPr, mt));
                    kf = fexp(lnkf, mt) * tr_g * fexp(tr_lF * kLn10, mt);
                }
            } else {
                kf = fexp(lnkf, mt);
            }
            const double E = fexp(-lnKc, mt);
            const double kr = kf * E;
            const double qc = fma(kf, fw, -kr * rv);
            const double q = (type == NK_RXN_THIRD_BODY) ? qc * M : qc;

            // ---- adjoint
            const double qbar = hb_any ? fma(-hbRT, sumh, wsum) : wsum;   // sum nu (bar_omega - bar_hrr h)
            if (hb_any) Tbar = fma(-hb * kR * q, sumcp, Tbar);
            if (WANT_G) {
                double gl = valid ? qbar * q : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) gl += __shfl_xor_sync(0xffffffffu, gl, o);
                if (lane == 0) gw[orig] += gl;
            }
            double Mbar = 0.0, qcbar = qbar;
            if (type == NK_RXN_THIRD_BODY) {
                qcbar = qbar * M;
                Mbar = qbar * qc;
            }
            const double krbar = -qcbar * rv;
            const double kfbar = fma(krbar, E, qcbar * fw);
            const double fwbar = qcbar * kf, rvbar = -qcbar * kr;
            const double lnKcbar = -krbar * kr;
            Tbar = fma(lnKcbar * invT, sumh - dnu, Tbar);        // through g_k/RT(T) and ln(p0/RT)
#pragma unroll
            for (int e = 0; e < kMaxSide; ++e) {
                if (e < nr) {
                    const int nu = __ldg(&rec->nu[e]);
                    double d = exR[e];                           // d fw / d C_e = nu C_e^(nu-1) prod_{f!=e}
                    if (nu > 1) {
                        d *= -__ldg(&rec->nud[e]);
                        for (int j = 1; j < nu; ++j) d *= cR[e];
                    }
                    const int k = __ldg(&rec->sp[e]);
                    sB[k * BLK] = fma(fwbar, d, sB[k * BLK]);
                }
                if (e < np) {
                    const int nu = __ldg(&rec->nu[kMaxSide + e]);
                    double d = exP[e];
                    if (nu > 1) {
                        d *= __ldg(&rec->nud[kMaxSide + e]);
                        for (int j = 1; j < nu; ++j) d *= cP[e];
                    }
                    const int k = __ldg(&rec->sp[kMaxSide + e]);
                    sB[k * BLK] = fma(rvbar, d, sB[k * BLK]);
                }
            }
            const double Lbar = kfbar * kf;                       // cotangent of ln k_f
            if (type == NK_RXN_TROE) {
                if (M != 0.0) {
                    const double lnf = fma(__ldg(&t->Ea0R), invT, __ldg(&t->beta0)) * invT;
                    // d lF / d log10 Pr and d lF / d log10 F_cent
                    const double dlF_du = -2.0 * tr_lF * tr_f1 * (tr_nn / (tr_v * tr_v)) / tr_den;
                    const double df1_dlFc = fma(1.1762, tr_u, -0.67 * tr_v) / (tr_v * tr_v);
                    const double dlF_dlFc = (1.0 - 2.0 * tr_lF * tr_f1 * df1_dlFc) / tr_den;
                    const double lnPrbar = Lbar * (1.0 - tr_g + dlF_du);
                    const double lnkinfbar = Lbar - lnPrbar;
                    Mbar = fma(lnPrbar, 1.0 / M, Mbar);
                    Tbar = fma(Lbar * dlF_dlFc, tr_dFc / tr_Fc, Tbar);
                    Tbar = fma(lnPrbar, lnf, Tbar);
                    Tbar = fma(lnkinfbar, fma(EaR, invT, beta) * invT, Tbar);
                }
            } else {
                Tbar = fma(Lbar, fma(EaR, invT, beta) * invT, Tbar);
            }
            if (type != NK_RXN_ELEMENTARY && Mbar != 0.0) {
                Tbar = fma(-Mbar * pRT, invT, Tbar);             // sum_k C_k = p/(RT)
                const int e0 = __ldg(&rec->eff0), e1 = __ldg(&rec->eff1);
                for (int j = e0; j < e1; ++j) {
                    const int k = __ldg(m.eff_sp + j);
                    sB[k * BLK] = fma(Mbar, __ldg(m.eff_m1 + j), sB[k * BLK]);
                }
            }
        }

        // C_k = rho y_k, rho = p/(R T s), s = sum y_k, y_k = Y_k / W_k
        double rhobar = 0.0;
        for (int k = 0; k < K; ++k) rhobar = fma(sB[k * BLK], sC[k * BLK], rhobar);
        rhobar /= rho;                                          // sum_k Cbar_k y_k
        const double sbar = -rhobar * rho / s;
        Tbar = fma(-rhobar * rho, invT, Tbar);
        if (valid) {
            gT[i] = Tbar;
            for (int k = 0; k < K; ++k)
                gY[(int64_t)k * ld + i] = __ldg(m.invW + k) * fma(rho, sB[k * BLK], sbar);
        }
    }

    if (WANT_G) {
        __syncthreads();
        const double* g0 = smem + (size_t)5 * K * BLK;   // per-warp sums, indexed by caller order
        for (int r = tid; r < R; r += BLK) {
            double acc = 0.0;
            for (int w = 0; w < BLK / 32; ++w) acc += g0[(size_t)w * R + r];
            ws[(size_t)blockIdx.x * R + r] = acc;
        }
    }
}

__global__ void reduce_blocks_kernel(const double* __restrict__ ws, int nblocks, int R, double* __restrict__ g) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += ws[(size_t)b * R + r];
    g[r] = acc;
}

template <int BLK>
cudaError_t launch_t(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     const double* dlnA, const double* bar_omega, const double* bar_hrr, double* gT, double* gY,
                     double* g_lnA, void* ws, cudaStream_t s) {
    const size_t smem = kMathTabDoubles * sizeof(double) + (size_t)5 * m.K * BLK * sizeof(double) +
                        (g_lnA ? (size_t)(BLK / 32) * m.R * sizeof(double) : 0);
    const int64_t need = (n + BLK - 1) / BLK;
    cudaError_t e;
    if (g_lnA) {
        auto kern = vjp_kernel<BLK, true>;
        if ((e = ensure_smem((const void*)kern, smem)) != cudaSuccess) return e;
        const int grid = (int)(need < kVjpMaxBlocks ? need : kVjpMaxBlocks);
        double* wsd = static_cast<double*>(ws);
        kern<<<grid, BLK, smem, s>>>(m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, wsd);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        reduce_blocks_kernel<<<(m.R + 127) / 128, 128, 0, s>>>(wsd, grid, m.R, g_lnA);
    } else {
        auto kern = vjp_kernel<BLK, false>;
        if ((e = ensure_smem((const void*)kern, smem)) != cudaSuccess) return e;
        kern<<<(unsigned)need, BLK, smem, s>>>(m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, nullptr);
    }
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- no-allocation variant
// Scratch for the per-block ln A partial sums of nk_rates_vjp_noalloc: a fixed device array in
// this library's module, present on every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};   // device address of the array, per device ordinal
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
    const int blk = vjp_block(m);
    if (!blk) return 0;
    const int64_t need = (n + blk - 1) / blk;
    const int64_t grid = need < kVjpMaxBlocks ? need : kVjpMaxBlocks;
    return (size_t)grid * m.R * sizeof(double);
}

cudaError_t launch_vjp(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                       const double* dlnA, const double* bar_omega, const double* bar_hrr, double* gT, double* gY,
                       double* g_lnA, void* ws, cudaStream_t s) {
    switch (vjp_block(m)) {
        case 128: return launch_t<128>(m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, g_lnA, ws, s);
        case 64: return launch_t<64>(m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, g_lnA, ws, s);
        case 32: return launch_t<32>(m, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, g_lnA, ws, s);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace nk
