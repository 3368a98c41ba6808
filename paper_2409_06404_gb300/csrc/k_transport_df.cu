// Mixture-averaged transport properties, FP64 form, evaluated in double-float arithmetic on
// the FP32 pipe (nk_df.cuh): Wilke viscosity, Mathur-Saxena conductivity and
// Hirschfelder-Curtiss diffusion coefficients (D_k of Eq. 2, mu of Eq. 4, lambda of Eq. 1b).
//
// Every sum here has positive, bounded terms (binary diffusion coefficients, Wilke weights,
// mole fractions), so 48-bit pairs give FP64-class results: the error bound of the pair
// arithmetic (~2^-46 per operation, 3e-14 for df_exp) stays below the 1e-10 the FP64 form
// promises by three orders of magnitude.  The FP64 pipe (1/58 of the FP32 rate on GB300) only
// converts inputs and outputs and forms ln T, the mole fractions and the mass-fraction sums
// of the diffusion numerators.
//
// Same reformulations as the FP64-native kernel (k_transport.cu): the Wilke denominators as
// three dot products with the constant matrix A_kj, one exponential per species pair, the
// factor p/p_ref applied to the finished sums, numerators from prefix and suffix sums.  The
// cubic fits are evaluated in u = ln T - kLnT0 with coefficients re-expanded on the host,
// which shrinks the cancellation between the terms of the monomial form.
#include "nk_internal.cuh"

namespace nk {
namespace {

__device__ __forceinline__ dfl ld2(const float2* p) {
    const float2 v = __ldg(p);
    return {v.x, v.y};
}
__device__ __forceinline__ dfl as_df(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 as_f2(dfl a) { return make_float2(a.h, a.l); }
__device__ __forceinline__ dfl dneg(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfl dscale(dfl a, float s) { return {a.h * s, a.l * s}; }   // s a power of 2

// c0 + u (c1 + u (c2 + u c3)) in pairs
__device__ __forceinline__ dfl poly3_df(const float2* c, dfl u) {
    dfl acc = ld2(c + 3);
    acc = df_fma(acc, u, ld2(c + 2));
    acc = df_fma(acc, u, ld2(c + 1));
    return df_fma(acc, u, ld2(c + 0));
}

template <int BLK>
__global__ void __launch_bounds__(BLK) transport_df_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                           const double* __restrict__ T,
                                                           const double* __restrict__ p,
                                                           const double* __restrict__ Y,
                                                           double* __restrict__ mu_out,
                                                           double* __restrict__ lam_out,
                                                           double* __restrict__ Dmix) {
    extern __shared__ double smem_all[];
    const MathTab mt = stage_math_tables(smem_all, m.mtab);
    float2* etab = reinterpret_cast<float2*>(smem_all + kMathTabDoubles);
    for (int j = threadIdx.x; j < kExpTab; j += BLK) etab[j] = __ldg(m.df_exp_tab + j);
    __syncthreads();
    const int K = m.K;
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    float2* base = reinterpret_cast<float2*>(smem_all + kMathTabDoubles + kExpTab);
    float2* sX = base + tid;                                  // X_k
    float2* sA = base + (size_t)K * BLK + tid;                // D denominators, then X_k tau_k
    float2* sB = base + (size_t)2 * K * BLK + tid;            // Y prefix sums (as double), then X_k tau_k^2
    double* sBd = reinterpret_cast<double*>(sB);

    const double Ti = T[i];
    const dfl u = df_split(flog(Ti, mt) - kLnT0);
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double Wbar = 1.0 / s;
    for (int k = 0; k < K; ++k) sX[k * BLK] = as_f2(df_split(Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * Wbar));

    // ---- diffusion: sum_{j != k} X_j / D_jk(p_ref), one exponential per pair
    if (Dmix) {
        for (int k = 0; k < K; ++k) sA[k * BLK] = make_float2(0.0f, 0.0f);
        const float2* Dc = m.df_D_fit;
        int pi = 0;
        for (int j = 0; j < K; ++j) {
            const dfl xj = as_df(sX[j * BLK]);
            dfl acc0{0.0f, 0.0f}, acc1{0.0f, 0.0f};
            int k = j + 1;
            for (; k + 1 < K; k += 2, pi += 2) {
                const dfl i0 = df_exp(dneg(poly3_df(Dc + 4 * pi, u)), etab);
                const dfl i1 = df_exp(dneg(poly3_df(Dc + 4 * pi + 4, u)), etab);
                sA[k * BLK] = as_f2(df_fma(xj, i0, as_df(sA[k * BLK])));
                sA[(k + 1) * BLK] = as_f2(df_fma(xj, i1, as_df(sA[(k + 1) * BLK])));
                acc0 = df_fma(as_df(sX[k * BLK]), i0, acc0);
                acc1 = df_fma(as_df(sX[(k + 1) * BLK]), i1, acc1);
            }
            if (k < K) {
                const dfl i0 = df_exp(dneg(poly3_df(Dc + 4 * pi, u)), etab);
                sA[k * BLK] = as_f2(df_fma(xj, i0, as_df(sA[k * BLK])));
                acc0 = df_fma(as_df(sX[k * BLK]), i0, acc0);
                ++pi;
            }
            sA[j * BLK] = as_f2(df_add(as_df(sA[j * BLK]), df_add(acc0, acc1)));
        }
        // numerators sum_{j != k} Y_j from prefix and suffix sums (no 1 - Y_k cancellation)
        const double pscale = p[i] / m.p_ref;
        double pre = 0.0;
        for (int k = 0; k < K; ++k) {
            sBd[k * BLK] = pre;
            pre += Y[(int64_t)k * ld + i];
        }
        double suf = 0.0;
        for (int k = K - 1; k >= 0; --k) {
            const double num = sBd[k * BLK] + suf;
            double den = df_value(as_df(sA[k * BLK])) * pscale;
            if (den < 2.2250738585072014e-308) den = 2.2250738585072014e-308;
            Dmix[(int64_t)k * ld + i] = num == 0.0 ? 0.0 : num / den;
            suf += Y[(int64_t)k * ld + i];
        }
    }

    // ---- conductivity (Mathur-Saxena) and the Wilke weights X tau, X tau^2
    dfl s1{0.0f, 0.0f}, s2{0.0f, 0.0f};
    for (int k = 0; k < K; ++k) {
        const dfl x = as_df(sX[k * BLK]);
        const dfl lnlam = poly3_df(m.df_lam_fit + 4 * k, u);
        s1 = df_fma(x, df_exp(lnlam, etab), s1);
        s2 = df_fma(x, df_exp(dneg(lnlam), etab), s2);
        const dfl lnmu = poly3_df(m.df_mu_fit + 4 * k, u);
        const dfl tau = df_exp(df_add(ld2(m.df_qlnW + k), dscale(lnmu, -0.5f)), etab);   // W^1/4 / mu^1/2
        const dfl xt = df_mul(x, tau);
        sA[k * BLK] = as_f2(xt);
        sB[k * BLK] = as_f2(df_mul(xt, tau));
    }
    if (lam_out) lam_out[i] = 0.5 * (df_value(s1) + 1.0 / df_value(s2));

    // ---- Wilke viscosity
    if (mu_out) {
        dfl mu{0.0f, 0.0f};
        for (int k = 0; k < K; ++k) {
            const dfl lnmu = poly3_df(m.df_mu_fit + 4 * k, u);
            const dfl sig = df_exp(df_add(dscale(lnmu, 0.5f), dneg(ld2(m.df_qlnW + k))), etab);   // mu^1/2 W^-1/4
            const float2* Ak = m.df_wilkeA + (size_t)k * K;
            dfl S0{0.0f, 0.0f}, S1{0.0f, 0.0f}, S2{0.0f, 0.0f};
            for (int j = 0; j < K; ++j) {
                const dfl a = ld2(Ak + j);
                S0 = df_fma(a, as_df(sX[j * BLK]), S0);
                S1 = df_fma(a, as_df(sA[j * BLK]), S1);
                S2 = df_fma(a, as_df(sB[j * BLK]), S2);
            }
            const dfl den = df_fma(sig, df_fma(sig, S2, dscale(S1, 2.0f)), S0);
            const dfl muk = df_exp(lnmu, etab);
            mu = df_add(mu, df_div(df_mul(as_df(sX[k * BLK]), muk), den));
        }
        mu_out[i] = df_value(mu);
    }
}

template <int BLK>
cudaError_t launch_t(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     double* mu, double* lam, double* D, size_t smem, cudaStream_t s) {
    auto kern = transport_df_kernel<BLK>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + BLK - 1) / BLK;
    kern<<<(unsigned)grid, BLK, smem, s>>>(m, n, ld, T, p, Y, mu, lam, D);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transport_df(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, double* mu, double* lam, double* Dmix, cudaStream_t s) {
    const size_t per_thread = (size_t)3 * m.K * 8;
    const size_t fixed = (kMathTabDoubles + kExpTab) * sizeof(double);
    const int blk = pick_block_occupancy(per_thread, fixed);
    if (!blk) return cudaErrorInvalidConfiguration;
    const size_t smem = per_thread * blk + fixed;
    switch (blk) {
        case 128: return launch_t<128>(m, n, ld, T, p, Y, mu, lam, Dmix, smem, s);
        case 64: return launch_t<64>(m, n, ld, T, p, Y, mu, lam, Dmix, smem, s);
        case 32: return launch_t<32>(m, n, ld, T, p, Y, mu, lam, Dmix, smem, s);
    }
    return cudaErrorInvalidConfiguration;
}

}  // namespace nk
