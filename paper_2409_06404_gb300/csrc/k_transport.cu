// Mixture-averaged transport properties per point (the "properties" kernel of the paper,
// Tab. 3; D_k of Eq. 2, mu of Eq. 4, lambda of Eq. 1b):
//   Wilke viscosity, Mathur-Saxena conductivity, Hirschfelder-Curtiss diffusion coefficients.
//
// Arithmetic type F = double (FP64 form) or float (mixed form: fits, mixture rules and all
// sums in single precision; the sums of mass fractions in the diffusion numerators stay in
// double because they carry the 1 - Y_k cancellation).
//
// Reformulations used here (same mathematics as the definitions):
//  * Wilke: Phi_kj = A_kj (1 + sigma_k tau_j)^2 with A_kj = 8^-1/2 (1 + W_k/W_j)^-1/2
//    (mechanism constant), sigma_k = mu_k^1/2 W_k^-1/4, tau_j = 1/sigma_j.  The denominator
//    sum_j X_j Phi_kj = S0_k + 2 sigma_k S1_k + sigma_k^2 S2_k with S0 = sum_j A_kj X_j,
//    S1 = sum_j A_kj X_j tau_j, S2 = sum_j A_kj X_j tau_j^2: three dot products per species,
//    all terms positive (no cancellation).
//  * D_km = (sum_{j!=k} Y_j) / (sum_{j!=k} X_j/D_jk), since X_j W_j = Y_j Wbar; the
//    numerator is formed from prefix and suffix sums, never as 1 - Y_k.
//  * each binary coefficient exp(-ln D_jk) is evaluated once per pair and used for both
//    species of the pair; the factor p/p_ref of D_jk(p) multiplies the finished sums.
//  * double exp/log are the table-driven versions of nk_math.cuh.
#include "nk_internal.cuh"

namespace nk {
namespace {

template <class F> struct Tab;
template <> struct Tab<double> {
    static __device__ __forceinline__ const double* mu(const DevMech& m) { return m.mu_fit; }
    static __device__ __forceinline__ const double* lam(const DevMech& m) { return m.lam_fit; }
    static __device__ __forceinline__ const double* D(const DevMech& m) { return m.D_fit; }
    static __device__ __forceinline__ const double* A(const DevMech& m) { return m.wilkeA; }
    static __device__ __forceinline__ const double* qrtW(const DevMech& m) { return m.qrtW; }
    static __device__ __forceinline__ const double* sqrtW(const DevMech& m) { return m.sqrtW; }
    static __device__ __forceinline__ const double* invW(const DevMech& m) { return m.invW; }
};
template <> struct Tab<float> {
    static __device__ __forceinline__ const float* mu(const DevMech& m) { return m.f_mu_fit; }
    static __device__ __forceinline__ const float* lam(const DevMech& m) { return m.f_lam_fit; }
    static __device__ __forceinline__ const float* D(const DevMech& m) { return m.f_D_fit; }
    static __device__ __forceinline__ const float* A(const DevMech& m) { return m.f_wilkeA; }
    static __device__ __forceinline__ const float* qrtW(const DevMech& m) { return m.f_qrtW; }
    static __device__ __forceinline__ const float* sqrtW(const DevMech& m) { return m.f_sqrtW; }
    static __device__ __forceinline__ const float* invW(const DevMech& m) { return m.f_invW; }
};

template <class F>
__device__ __forceinline__ F poly3(const F* c, F L) {
    return fma(L, fma(L, fma(L, __ldg(c + 3), __ldg(c + 2)), __ldg(c + 1)), __ldg(c + 0));
}

// exp in the arithmetic type: the table-driven double exp, or single-precision expf
__device__ __forceinline__ double texp(double x, const MathTab& mt) { return fexp(x, mt); }
__device__ __forceinline__ float texp(float x, const MathTab&) { return expf(x); }

template <int BLK, class F>
__global__ void __launch_bounds__(BLK) transport_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                        const double* __restrict__ T, const double* __restrict__ p,
                                                        const double* __restrict__ Y, double* __restrict__ mu_out,
                                                        double* __restrict__ lam_out, double* __restrict__ Dmix) {
    extern __shared__ double smem_d[];
    const MathTab mt = stage_math_tables(smem_d, m.mtab);
    __syncthreads();
    F* smem = reinterpret_cast<F*>(smem_d + kMathTabDoubles);
    const int K = m.K;
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * BLK + tid;
    if (i >= n) return;
    F* sX = smem + tid;                        // X_k
    F* sA = smem + (size_t)K * BLK + tid;      // D denominators, then X_k tau_k
    F* sB = smem + (size_t)2 * K * BLK + tid;  // prefix sums of Y, then X_k tau_k^2
    using Tb = Tab<F>;

    const double Ti = T[i];
    const F L = (F)flog(Ti, mt);
    // mole fractions
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double Wbar = 1.0 / s;
    for (int k = 0; k < K; ++k) sX[k * BLK] = (F)(Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * Wbar);

    // ---- diffusion: sum_{j != k} X_j / D_jk(p_ref), one exponential per pair; the pressure
    // factor p/p_ref multiplies the finished sums
    if (Dmix) {
        for (int k = 0; k < K; ++k) sA[k * BLK] = F(0);
        const F* Dc = Tb::D(m);
        int pi = 0;
        for (int j = 0; j < K; ++j) {
            const F xj = sX[j * BLK];
            F acc0 = F(0), acc1 = F(0);
            int k = j + 1;
            for (; k + 1 < K; k += 2, pi += 2) {
                const F i0 = texp(-poly3(Dc + 4 * pi, L), mt);
                const F i1 = texp(-poly3(Dc + 4 * pi + 4, L), mt);
                sA[k * BLK] = fma(xj, i0, sA[k * BLK]);
                sA[(k + 1) * BLK] = fma(xj, i1, sA[(k + 1) * BLK]);
                acc0 = fma(sX[k * BLK], i0, acc0);
                acc1 = fma(sX[(k + 1) * BLK], i1, acc1);
            }
            if (k < K) {
                const F i0 = texp(-poly3(Dc + 4 * pi, L), mt);
                sA[k * BLK] = fma(xj, i0, sA[k * BLK]);
                acc0 = fma(sX[k * BLK], i0, acc0);
                ++pi;
            }
            sA[j * BLK] += acc0 + acc1;
        }
        // numerators sum_{j != k} Y_j from prefix and suffix sums (no 1 - Y_k cancellation)
        const double pscale = p[i] / m.p_ref;
        double pre = 0.0;
        for (int k = 0; k < K; ++k) {
            sB[k * BLK] = (F)pre;
            pre += Y[(int64_t)k * ld + i];
        }
        double suf = 0.0;
        for (int k = K - 1; k >= 0; --k) {
            const double num = (double)sB[k * BLK] + suf;
            double den = (double)sA[k * BLK] * pscale;
            if (den < 2.2250738585072014e-308) den = 2.2250738585072014e-308;
            Dmix[(int64_t)k * ld + i] = num == 0.0 ? 0.0 : num / den;
            suf += Y[(int64_t)k * ld + i];
        }
    }

    // ---- conductivity (Mathur-Saxena) and the Wilke weights
    F s1 = F(0), s2 = F(0);
    const F* lamc = Tb::lam(m);
    const F* muc = Tb::mu(m);
    for (int k = 0; k < K; ++k) {
        const F x = sX[k * BLK];
        const F lnlam = poly3(lamc + 4 * k, L);
        s1 = fma(x, texp(lnlam, mt), s1);
        s2 = fma(x, texp(-lnlam, mt), s2);
        const F tau = __ldg(Tb::qrtW(m) + k) * texp(F(-0.5) * poly3(muc + 4 * k, L), mt);   // W^1/4 / mu^1/2
        const F xt = x * tau;
        sA[k * BLK] = xt;
        sB[k * BLK] = xt * tau;
    }
    if (lam_out) lam_out[i] = (double)(F(0.5) * (s1 + F(1) / s2));

    // ---- Wilke viscosity
    if (mu_out) {
        const F* A = Tb::A(m);
        F mu = F(0);
        for (int k = 0; k < K; ++k) {
            const F hs = texp(F(0.5) * poly3(muc + 4 * k, L), mt);     // mu_k^1/2
            const F sig = hs / __ldg(Tb::qrtW(m) + k);                  // sigma_k
            const F* Ak = A + (size_t)k * K;
            F S0 = F(0), S1 = F(0), S2 = F(0);
            for (int j = 0; j < K; ++j) {
                const F a = __ldg(Ak + j);
                S0 = fma(a, sX[j * BLK], S0);
                S1 = fma(a, sA[j * BLK], S1);
                S2 = fma(a, sB[j * BLK], S2);
            }
            const F den = fma(sig, fma(sig, S2, F(2) * S1), S0);
            mu = fma(sX[k * BLK], hs * hs / den, mu);
        }
        mu_out[i] = (double)mu;
    }
}

template <int BLK, class F>
cudaError_t launch_t(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     double* mu, double* lam, double* D, size_t smem, cudaStream_t s) {
    auto kern = transport_kernel<BLK, F>;
    cudaError_t e = ensure_smem((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (n + BLK - 1) / BLK;
    kern<<<(unsigned)grid, BLK, smem, s>>>(m, n, ld, T, p, Y, mu, lam, D);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transport(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, double* mu, double* lam, double* Dmix, int precision,
                             cudaStream_t s) {
    const bool mixed = precision == NK_MIXED;
    const size_t per_thread = (size_t)3 * m.K * (mixed ? sizeof(float) : sizeof(double));
    const size_t tab = kMathTabDoubles * sizeof(double);
    const int blk = pick_block_occupancy(per_thread, tab);
    if (!blk) return cudaErrorInvalidConfiguration;
    const size_t smem = per_thread * blk + tab;
#define NK_TR_CASE(B)                                                                 \
    case B:                                                                           \
        return mixed ? launch_t<B, float>(m, n, ld, T, p, Y, mu, lam, Dmix, smem, s)  \
                     : launch_t<B, double>(m, n, ld, T, p, Y, mu, lam, Dmix, smem, s);
    switch (blk) {
        NK_TR_CASE(128)
        NK_TR_CASE(64)
        NK_TR_CASE(32)
    }
#undef NK_TR_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace nk
