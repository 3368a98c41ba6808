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
#include <mutex>
#include <utility>
#include <vector>

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

// The species-pair triangle of the diffusion sums in G = 2 NP contiguous species groups, taken
// by the NP parts of a point in rounds of group pairs that share no species (the circle method
// of a round-robin schedule; the last round pairs each part's two groups with themselves), so
// every part adds straight into the one row of sums, in an order fixed by the schedule.
template <int NP>
__device__ __forceinline__ void round_groups(int r, int part, int& ga, int& gb) {
    constexpr int G = 2 * NP;
    if (part == 0) {
        ga = r;
        gb = G - 1;
    } else {
        ga = (r + part) % (G - 1);
        gb = (r - part + G - 1) % (G - 1);
    }
    if (ga > gb) {
        const int t = ga;
        ga = gb;
        gb = t;
    }
}

// The pairs (j, k), j in [j0, j1), k in [k0, k1), k > j (k0 = j0, k1 = j1 for a group with itself):
// S_j += X_k / D_jk in registers and S_k += X_j / D_jk in the row, one exponential per pair, two
// pairs per iteration.
template <int BLK, class F>
__device__ __forceinline__ void diffusion_pairs(int K, int j0, int j1, int k0, int k1, bool same, const F* Dc, F L,
                                                const MathTab& mt, const F* sX, F* sS) {
    for (int j = j0; j < j1; ++j) {
        const int kb = same ? j + 1 : k0;
        int pi = j * (2 * K - j - 1) / 2 + (kb - j - 1);       // index of the pair (j, kb)
        const F xj = sX[j * BLK];
        F acc0 = F(0), acc1 = F(0);
        int k = kb;
        for (; k + 1 < k1; k += 2, pi += 2) {
            const F i0 = texp(-poly3(Dc + 4 * pi, L), mt);
            const F i1 = texp(-poly3(Dc + 4 * pi + 4, L), mt);
            sS[k * BLK] = fma(xj, i0, sS[k * BLK]);
            sS[(k + 1) * BLK] = fma(xj, i1, sS[(k + 1) * BLK]);
            acc0 = fma(sX[k * BLK], i0, acc0);
            acc1 = fma(sX[(k + 1) * BLK], i1, acc1);
        }
        if (k < k1) {
            const F i0 = texp(-poly3(Dc + 4 * pi, L), mt);
            sS[k * BLK] = fma(xj, i0, sS[k * BLK]);
            acc0 = fma(sX[k * BLK], i0, acc0);
        }
        sS[j * BLK] += acc0 + acc1;
    }
}

// BLK points per block, NP parts (warps) per point: the parts split the species-pair triangle
// of the diffusion sums by the rounds above, then the species of the conductivity, the diffusion
// outputs and the Wilke sums; the parts' scalar sums are added in part order.  Shared rows per
// point: X_k, the diffusion sums (then X_k tau_k), the mass-fraction prefix sums (then
// X_k tau_k^2).
template <int BLK, int NP, class F>
__global__ void __launch_bounds__(BLK * NP) transport_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                             const double* __restrict__ T,
                                                             const double* __restrict__ p,
                                                             const double* __restrict__ Y,
                                                             double* __restrict__ mu_out,
                                                             double* __restrict__ lam_out,
                                                             double* __restrict__ Dmix) {
    extern __shared__ double smem_d[];
    const MathTab mt = stage_math_tables(smem_d, m.mtab);
    __syncthreads();
    F* smem = reinterpret_cast<F*>(smem_d + kMathTabDoubles);
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;         // idle slots of the last block recompute point n-1
    F* sX = smem + slot;                         // X_k
    F* sA = smem + (size_t)K * BLK + slot;       // D denominators, then X_k tau_k
    F* sB = smem + (size_t)2 * K * BLK + slot;   // prefix sums of Y, then X_k tau_k^2
    using Tb = Tab<F>;

    // The mixed form (F = float) keeps every step in single precision: inputs rounded to float and
    // outputs widened by integer operations, the mole fractions, numerators and quotients in
    // float, so it issues no FP64-pipe instruction (the double form keeps its sums in double).
    constexpr bool kF32 = sizeof(F) == sizeof(float);
    const double Ti = T[i];
    F L;
    if constexpr (kF32)
        L = logf(narrow(Ti));
    else
        L = flog(Ti, mt);
    // mole fractions
    if constexpr (kF32) {
        float s = 0.0f;
        for (int k = 0; k < K; ++k) s = fmaf(narrow(Y[(int64_t)k * ld + i]), __ldg(m.f_invW + k), s);
        const float Wbar = 1.0f / s;
        for (int k = part; k < K; k += NP) sX[k * BLK] = narrow(Y[(int64_t)k * ld + i]) * __ldg(m.f_invW + k) * Wbar;
    } else {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
        const double Wbar = 1.0 / s;
        for (int k = part; k < K; k += NP) sX[k * BLK] = (F)(Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * Wbar);
    }

    // ---- diffusion: sum_{j != k} X_j / D_jk(p_ref), one exponential per pair; the pressure
    // factor p/p_ref multiplies the finished sums
    if (Dmix) {
        for (int k = part; k < K; k += NP) sA[k * BLK] = F(0);
        if (NP > 1) __syncthreads();
        const F* Dc = Tb::D(m);
        constexpr int G = 2 * NP;
        for (int r = 0; r < G - 1; ++r) {
            int ga, gb;
            round_groups<NP>(r, part, ga, gb);
            diffusion_pairs<BLK, F>(K, K * ga / G, K * (ga + 1) / G, K * gb / G, K * (gb + 1) / G, false, Dc, L, mt,
                                    sX, sA);
            if (NP > 1) __syncthreads();
        }
        for (int g = 2 * part; g < 2 * part + 2; ++g)
            diffusion_pairs<BLK, F>(K, K * g / G, K * (g + 1) / G, K * g / G, K * (g + 1) / G, true, Dc, L, mt, sX,
                                    sA);
        if (NP > 1) __syncthreads();
        // numerators sum_{j != k} Y_j from prefix and suffix sums (no 1 - Y_k cancellation)
        if constexpr (kF32) {
            const float pscale = narrow(p[i]) / narrow(m.p_ref);
            float pre = 0.0f;
            for (int k = 0; k < K; ++k) {
                if (NP == 1 || k % NP == part) sB[k * BLK] = pre;
                pre += narrow(Y[(int64_t)k * ld + i]);
            }
            float suf = 0.0f;
            for (int k = K - 1; k >= 0; --k) {
                if (NP == 1 || k % NP == part) {
                    const float num = sB[k * BLK] + suf;
                    float den = sA[k * BLK] * pscale;
                    if (den < 1.17549435e-38f) den = 1.17549435e-38f;
                    if (live) Dmix[(int64_t)k * ld + i] = num == 0.0f ? 0.0 : widen(num / den);
                }
                suf += narrow(Y[(int64_t)k * ld + i]);
            }
        } else {
            const double pscale = p[i] / m.p_ref;
            double pre = 0.0;
            for (int k = 0; k < K; ++k) {
                if (NP == 1 || k % NP == part) sB[k * BLK] = (F)pre;
                pre += Y[(int64_t)k * ld + i];
            }
            double suf = 0.0;
            for (int k = K - 1; k >= 0; --k) {
                if (NP == 1 || k % NP == part) {
                    const double num = (double)sB[k * BLK] + suf;
                    double den = (double)sA[k * BLK] * pscale;
                    if (den < 2.2250738585072014e-308) den = 2.2250738585072014e-308;
                    if (live) Dmix[(int64_t)k * ld + i] = num == 0.0 ? 0.0 : num / den;
                }
                suf += Y[(int64_t)k * ld + i];
            }
        }
    }

    // ---- conductivity (Mathur-Saxena) and the Wilke weights of this part's species
    F s1 = F(0), s2 = F(0);
    const F* lamc = Tb::lam(m);
    const F* muc = Tb::mu(m);
    for (int k = part; k < K; k += NP) {
        const F x = sX[k * BLK];
        const F lnlam = poly3(lamc + 4 * k, L);
        s1 = fma(x, texp(lnlam, mt), s1);
        s2 = fma(x, texp(-lnlam, mt), s2);
        const F tau = __ldg(Tb::qrtW(m) + k) * texp(F(-0.5) * poly3(muc + 4 * k, L), mt);   // W^1/4 / mu^1/2
        const F xt = x * tau;
        sA[k * BLK] = xt;
        sB[k * BLK] = xt * tau;
    }

    // ---- Wilke viscosity over this part's species
    F mu = F(0);
    if (mu_out) {
        if (NP > 1) __syncthreads();
        const F* A = Tb::A(m);
        for (int k = part; k < K; k += NP) {
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
    }
    if constexpr (NP > 1) {
        // the parts' sums in part order, through the (dead) X row: rows 3q .. 3q+2 (3 NP <= K)
        __syncthreads();
        sX[(3 * part) * BLK] = s1;
        sX[(3 * part + 1) * BLK] = s2;
        sX[(3 * part + 2) * BLK] = mu;
        __syncthreads();
        if (part != 0) return;
        s1 = sX[0];
        s2 = sX[BLK];
        mu = sX[2 * BLK];
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            s1 += sX[(3 * q) * BLK];
            s2 += sX[(3 * q + 1) * BLK];
            mu += sX[(3 * q + 2) * BLK];
        }
    }
    if (live) {
        if constexpr (kF32) {
            if (lam_out) lam_out[i] = widen(0.5f * (s1 + 1.0f / s2));
            if (mu_out) mu_out[i] = widen(mu);
        } else {
            if (lam_out) lam_out[i] = (double)(F(0.5) * (s1 + F(1) / s2));
            if (mu_out) mu_out[i] = (double)mu;
        }
    }
}

// ---------------------------------------------------------------- launch shapes
struct Shape {
    int blk, np;
};
constexpr Shape kShapes[] = {{32, 1}, {64, 1}, {128, 1}, {32, 2}, {64, 2}, {32, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <class F, int S>
constexpr auto kernel_of() {
    return transport_kernel<kShapes[S].blk, kShapes[S].np, F>;
}

template <class F, int... S>
const void* kernel_ptr(int idx, std::integer_sequence<int, S...>) {
    const void* ptrs[] = {(const void*)kernel_of<F, S>()...};
    return ptrs[idx];
}

template <class F>
size_t transport_smem(int K, const Shape& sh) {
    return (size_t)kMathTabDoubles * sizeof(double) + (size_t)3 * K * sh.blk * sizeof(F);
}

struct Plan {
    int dev, K, mixed, idx;
};
std::mutex g_plan_mu;
std::vector<Plan> g_plans;

// The shape with the most resident warps per SM, fewer parts on ties (cached per device, K and
// arithmetic type).
template <class F>
int plan_shape(int K) {
    constexpr int mixed = sizeof(F) == sizeof(float);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const Plan& q : g_plans)
            if (q.dev == dev && q.K == K && q.mixed == mixed) return q.idx;
    }
    int per_block = 0;
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = -1, best_warps = 0;
    for (int c = 0; c < kNumShapes; ++c) {
        const Shape& sh = kShapes[c];
        if (sh.np > 1 && 3 * sh.np > K) continue;
        const size_t bytes = transport_smem<F>(K, sh);
        if (bytes > (size_t)per_block) continue;
        const void* kern = kernel_ptr<F>(c, std::make_integer_sequence<int, kNumShapes>{});
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
        g_plans.push_back({dev, K, mixed, best});
    }
    return best;
}

template <class F, int... S>
cudaError_t launch_idx(int idx, std::integer_sequence<int, S...>, const DevMech& m, int64_t n, int64_t ld,
                       const double* T, const double* p, const double* Y, double* mu, double* lam, double* D,
                       cudaStream_t st) {
    cudaError_t e = cudaErrorInvalidConfiguration;
    ((S == idx ? (void)(e = [&] {
        constexpr Shape sh = kShapes[S];
        auto kern = kernel_of<F, S>();
        const size_t smem = transport_smem<F>(m.K, sh);
        cudaError_t r = ensure_smem((const void*)kern, smem);
        if (r != cudaSuccess) return r;
        kern<<<(unsigned)((n + sh.blk - 1) / sh.blk), sh.blk * sh.np, smem, st>>>(m, n, ld, T, p, Y, mu, lam, D);
        return cudaGetLastError();
    }())
               : (void)0),
     ...);
    return e;
}

template <class F>
cudaError_t launch_f(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     double* mu, double* lam, double* Dmix, cudaStream_t s) {
    const int idx = plan_shape<F>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx<F>(idx, std::make_integer_sequence<int, kNumShapes>{}, m, n, ld, T, p, Y, mu, lam, Dmix, s);
}

}  // namespace

cudaError_t launch_transport(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, double* mu, double* lam, double* Dmix, int precision,
                             cudaStream_t s) {
    return precision == NK_MIXED ? launch_f<float>(m, n, ld, T, p, Y, mu, lam, Dmix, s)
                                 : launch_f<double>(m, n, ld, T, p, Y, mu, lam, Dmix, s);
}

}  // namespace nk
