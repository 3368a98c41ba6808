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
#include <mutex>
#include <utility>
#include <vector>

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

// A sum of products a_j x_j of positive pairs kept as an unevaluated float sum hi + lo that is
// not renormalised per term: hi collects the high products by two-sum, lo the two-sums' rounding
// errors, the products' own errors and the cross terms (each about 2^-24 of its term, so a float
// carries them), and dot_value renormalises once.  12 FP32 operations per term instead of the 15
// of df_fma; for positive terms the result keeps the pair's ~2^-46 relative error.
struct DotAcc {
    float hi = 0.0f, lo = 0.0f;
};
__device__ __forceinline__ void dot_add(DotAcc& s, dfl a, dfl x) {
    const float p = __fmul_rn(a.h, x.h);
    float e = __fmaf_rn(a.h, x.h, -p);
    e = __fmaf_rn(a.h, x.l, e);
    e = __fmaf_rn(a.l, x.h, e);
    const float t = __fadd_rn(s.hi, p);
    const float bb = __fsub_rn(t, s.hi);
    const float err = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ dfl dot_value(const DotAcc& s) { return fast_two_sum(s.hi, s.lo); }

// c0 + u (c1 + u (c2 + u c3)) in pairs
__device__ __forceinline__ dfl poly3_df(const float2* c, dfl u) {
    dfl acc = ld2(c + 3);
    acc = df_fma(acc, u, ld2(c + 2));
    acc = df_fma(acc, u, ld2(c + 1));
    return df_fma(acc, u, ld2(c + 0));
}

// Shared rows per point (8 bytes per species): X_k, the diffusion sums (later X_k tau_k) and
// one row for the mass-fraction prefix sums (later X_k tau_k^2).
constexpr int kTransportRows = 3;

// The species-pair triangle of the diffusion sums in G = kGroupsPerPart NP contiguous species
// groups.  In each of the first G - 1 rounds the G/2 group pairs of a round-robin schedule (the
// circle method: group G - 1 meets group r, groups (r + q) and (r - q) mod (G - 1) meet for
// q = 1 .. G/2 - 1) share no species; part q takes pairs q kGroupsPerPart/2 .. (q + 1)
// kGroupsPerPart/2 - 1 of the round.  In the last round part q takes the pairs within its own
// kGroupsPerPart groups.  So within a round no two parts touch one species, every part adds
// straight into the one row of sums, and the order of each sum is fixed by the schedule.
constexpr int kGroupsPerPart = 2;

template <int G>
__device__ __forceinline__ void round_pair(int r, int q, int& ga, int& gb) {
    if (q == 0) {
        ga = r;
        gb = G - 1;
    } else {
        ga = (r + q) % (G - 1);
        gb = (r - q + G - 1) % (G - 1);
    }
    if (ga > gb) {
        const int t = ga;
        ga = gb;
        gb = t;
    }
}

// The pairs (j, k) with j in [j0, j1) and k in [k0, k1), k > j (k0 = j0, k1 = j1 for a group with
// itself): S_j += X_k / D_jk in registers, S_k += X_j / D_jk in the row, one exponential per pair,
// four pairs per iteration (four independent exponential chains per thread).
template <int BLK>
__device__ __forceinline__ void diffusion_pairs(int K, int j0, int j1, int k0, int k1, bool same, const float2* Dc,
                                                dfl u, const float2* etab, const float2* sX, float2* sS) {
    for (int j = j0; j < j1; ++j) {
        const int kb = same ? j + 1 : k0;
        int pi = j * (2 * K - j - 1) / 2 + (kb - j - 1);       // index of the pair (j, kb)
        const dfl xj = as_df(sX[j * BLK]);
        dfl acc0{0.0f, 0.0f}, acc1{0.0f, 0.0f}, acc2{0.0f, 0.0f}, acc3{0.0f, 0.0f};
        int k = kb;
        for (; k + 3 < k1; k += 4, pi += 4) {
            const dfl i0 = df_exp(dneg(poly3_df(Dc + 4 * pi, u)), etab);
            const dfl i1 = df_exp(dneg(poly3_df(Dc + 4 * pi + 4, u)), etab);
            const dfl i2 = df_exp(dneg(poly3_df(Dc + 4 * pi + 8, u)), etab);
            const dfl i3 = df_exp(dneg(poly3_df(Dc + 4 * pi + 12, u)), etab);
            sS[k * BLK] = as_f2(df_fma(xj, i0, as_df(sS[k * BLK])));
            sS[(k + 1) * BLK] = as_f2(df_fma(xj, i1, as_df(sS[(k + 1) * BLK])));
            sS[(k + 2) * BLK] = as_f2(df_fma(xj, i2, as_df(sS[(k + 2) * BLK])));
            sS[(k + 3) * BLK] = as_f2(df_fma(xj, i3, as_df(sS[(k + 3) * BLK])));
            acc0 = df_fma(as_df(sX[k * BLK]), i0, acc0);
            acc1 = df_fma(as_df(sX[(k + 1) * BLK]), i1, acc1);
            acc2 = df_fma(as_df(sX[(k + 2) * BLK]), i2, acc2);
            acc3 = df_fma(as_df(sX[(k + 3) * BLK]), i3, acc3);
        }
        for (; k < k1; ++k, ++pi) {
            const dfl i0 = df_exp(dneg(poly3_df(Dc + 4 * pi, u)), etab);
            sS[k * BLK] = as_f2(df_fma(xj, i0, as_df(sS[k * BLK])));
            acc0 = df_fma(as_df(sX[k * BLK]), i0, acc0);
        }
        sS[j * BLK] = as_f2(df_add(as_df(sS[j * BLK]), df_add(df_add(acc0, acc1), df_add(acc2, acc3))));
    }
}

// BLK points per block, NP parts (warps) per point, as in the rates kernel: the parts split the
// species-pair triangle of the diffusion sums by the round schedule above and then the species
// of the conductivity, diffusion outputs and Wilke sums.
template <int BLK, int NP>
__global__ void __launch_bounds__(BLK * NP) transport_df_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                                const double* __restrict__ T,
                                                                const double* __restrict__ p,
                                                                const double* __restrict__ Y,
                                                                double* __restrict__ mu_out,
                                                                double* __restrict__ lam_out,
                                                                double* __restrict__ Dmix) {
    extern __shared__ double smem_all[];
    const MathTab mt = stage_math_tables(smem_all, m.mtab);
    float2* etab = reinterpret_cast<float2*>(smem_all + kMathTabDoubles);
    for (int j = threadIdx.x; j < kExpTab; j += BLK * NP) etab[j] = __ldg(m.df_exp_tab + j);
    __syncthreads();
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;         // idle slots of the last block recompute point n-1
    float2* base = reinterpret_cast<float2*>(smem_all + kMathTabDoubles + kExpTab) + slot;
    float2* sX = base;                                        // X_k
    float2* sA0 = base + (size_t)K * BLK;                     // diffusion sums, then X_k tau_k
    float2* sB = base + (size_t)2 * K * BLK;                  // Y prefix sums (as double), then X_k tau_k^2
    double* sBd = reinterpret_cast<double*>(sB);

    const double Ti = T[i];
    const dfl u = df_split(flog(Ti, mt) - kLnT0);
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double Wbar = 1.0 / s;
    for (int k = part; k < K; k += NP)
        sX[k * BLK] = as_f2(df_split(Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * Wbar));

    // ---- diffusion: sum_{j != k} X_j / D_jk(p_ref), one exponential per pair
    if (Dmix) {
        for (int k = part; k < K; k += NP) sA0[k * BLK] = make_float2(0.0f, 0.0f);
        if (NP > 1) __syncthreads();
        const float2* Dc = m.df_D_fit;
        constexpr int G = kGroupsPerPart * NP, H = kGroupsPerPart / 2;
        for (int r = 0; r < G - 1; ++r) {
#pragma unroll 1
            for (int h = 0; h < H; ++h) {
                int ga, gb;
                round_pair<G>(r, part * H + h, ga, gb);
                diffusion_pairs<BLK>(K, K * ga / G, K * (ga + 1) / G, K * gb / G, K * (gb + 1) / G, false, Dc, u,
                                     etab, sX, sA0);
            }
            if (NP > 1) __syncthreads();
        }
        for (int g = kGroupsPerPart * part; g < kGroupsPerPart * (part + 1); ++g)
            diffusion_pairs<BLK>(K, K * g / G, K * (g + 1) / G, K * g / G, K * (g + 1) / G, true, Dc, u, etab, sX,
                                 sA0);
        if (NP > 1) __syncthreads();
        // numerators sum_{j != k} Y_j from prefix and suffix sums (no 1 - Y_k cancellation)
        const double pscale = p[i] / m.p_ref;
        double pre = 0.0;
        for (int k = 0; k < K; ++k) {
            if (NP == 1 || k % NP == part) sBd[k * BLK] = pre;
            pre += Y[(int64_t)k * ld + i];
        }
        double suf = 0.0;
        for (int k = K - 1; k >= 0; --k) {
            if (NP == 1 || k % NP == part) {
                const double num = sBd[k * BLK] + suf;
                double den = df_value(as_df(sA0[k * BLK])) * pscale;
                if (den < 2.2250738585072014e-308) den = 2.2250738585072014e-308;
                if (live) Dmix[(int64_t)k * ld + i] = num == 0.0 ? 0.0 : num / den;
            }
            suf += Y[(int64_t)k * ld + i];
        }
    }

    // ---- conductivity (Mathur-Saxena) and the Wilke weights X tau, X tau^2 of this part's species
    dfl s1{0.0f, 0.0f}, s2{0.0f, 0.0f};
    for (int k = part; k < K; k += NP) {
        const dfl x = as_df(sX[k * BLK]);
        const dfl lnlam = poly3_df(m.df_lam_fit + 4 * k, u);
        s1 = df_fma(x, df_exp(lnlam, etab), s1);
        s2 = df_fma(x, df_exp(dneg(lnlam), etab), s2);
        const dfl lnmu = poly3_df(m.df_mu_fit + 4 * k, u);
        const dfl tau = df_exp(df_add(ld2(m.df_qlnW + k), dscale(lnmu, -0.5f)), etab);   // W^1/4 / mu^1/2
        const dfl xt = df_mul(x, tau);
        sA0[k * BLK] = as_f2(xt);
        sB[k * BLK] = as_f2(df_mul(xt, tau));
    }

    // ---- Wilke viscosity over this part's species
    dfl mu{0.0f, 0.0f};
    if (mu_out) {
        if (NP > 1) __syncthreads();
        for (int k = part; k < K; k += NP) {
            const dfl lnmu = poly3_df(m.df_mu_fit + 4 * k, u);
            const dfl sig = df_exp(df_add(dscale(lnmu, 0.5f), dneg(ld2(m.df_qlnW + k))), etab);   // mu^1/2 W^-1/4
            const float2* Ak = m.df_wilkeA + (size_t)k * K;
            // j in two interleaved sums of each of the three: six independent chains per thread
            DotAcc S0, S1, S2, T0, T1, T2;
            int j = 0;
            for (; j + 1 < K; j += 2) {
                const dfl a = ld2(Ak + j), b = ld2(Ak + j + 1);
                dot_add(S0, a, as_df(sX[j * BLK]));
                dot_add(T0, b, as_df(sX[(j + 1) * BLK]));
                dot_add(S1, a, as_df(sA0[j * BLK]));
                dot_add(T1, b, as_df(sA0[(j + 1) * BLK]));
                dot_add(S2, a, as_df(sB[j * BLK]));
                dot_add(T2, b, as_df(sB[(j + 1) * BLK]));
            }
            if (j < K) {
                const dfl a = ld2(Ak + j);
                dot_add(S0, a, as_df(sX[j * BLK]));
                dot_add(S1, a, as_df(sA0[j * BLK]));
                dot_add(S2, a, as_df(sB[j * BLK]));
            }
            const dfl W0 = df_add(dot_value(S0), dot_value(T0));
            const dfl W1 = df_add(dot_value(S1), dot_value(T1));
            const dfl W2 = df_add(dot_value(S2), dot_value(T2));
            const dfl den = df_fma(sig, df_fma(sig, W2, dscale(W1, 2.0f)), W0);
            const dfl muk = df_exp(lnmu, etab);
            mu = df_add(mu, df_div(df_mul(as_df(sX[k * BLK]), muk), den));
        }
    }
    if constexpr (NP > 1) {
        // the parts' sums in part order, through the (dead) X row: rows 3q .. 3q+2 (3 NP <= K)
        __syncthreads();
        float2* r1 = sX;
        r1[(3 * part) * BLK] = as_f2(s1);
        r1[(3 * part + 1) * BLK] = as_f2(s2);
        r1[(3 * part + 2) * BLK] = as_f2(mu);
        __syncthreads();
        if (part != 0) return;
        s1 = as_df(r1[0]);
        s2 = as_df(r1[BLK]);
        mu = as_df(r1[2 * BLK]);
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            s1 = df_add(s1, as_df(r1[(3 * q) * BLK]));
            s2 = df_add(s2, as_df(r1[(3 * q + 1) * BLK]));
            mu = df_add(mu, as_df(r1[(3 * q + 2) * BLK]));
        }
    }
    if (live) {
        if (lam_out) lam_out[i] = 0.5 * (df_value(s1) + 1.0 / df_value(s2));
        if (mu_out) mu_out[i] = df_value(mu);
    }
}

// ---------------------------------------------------------------- launch shapes
struct Shape {
    int blk, np;
};
constexpr Shape kShapes[] = {{32, 1}, {64, 1}, {32, 2}, {64, 2}, {32, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

template <int S>
constexpr auto kernel_of() {
    return transport_df_kernel<kShapes[S].blk, kShapes[S].np>;
}

template <int... S>
const void* kernel_ptr(int idx, std::integer_sequence<int, S...>) {
    const void* ptrs[] = {(const void*)kernel_of<S>()...};
    return ptrs[idx];
}

size_t transport_smem(int K, const Shape& sh) {
    return (size_t)(kMathTabDoubles + kExpTab) * sizeof(double) +
           (size_t)kTransportRows * K * sh.blk * sizeof(double);
}

struct Plan {
    int dev, K, idx;
};
std::mutex g_plan_mu;
std::vector<Plan> g_plans;

// The shape with the most resident warps per SM, fewer parts on ties (cached per device and K).
int plan_shape(int K) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const Plan& q : g_plans)
            if (q.dev == dev && q.K == K) return q.idx;
    }
    int per_block = 0;
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = -1, best_warps = 0;
    for (int c = 0; c < kNumShapes; ++c) {
        const Shape& sh = kShapes[c];
        if (sh.np > 1 && 3 * sh.np > K) continue;
        const size_t bytes = transport_smem(K, sh);
        if (bytes > (size_t)per_block) continue;
        const void* kern = kernel_ptr(c, std::make_integer_sequence<int, kNumShapes>{});
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
        g_plans.push_back({dev, K, best});
    }
    return best;
}

template <int... S>
cudaError_t launch_idx(int idx, std::integer_sequence<int, S...>, const DevMech& m, int64_t n, int64_t ld,
                       const double* T, const double* p, const double* Y, double* mu, double* lam, double* D,
                       cudaStream_t st) {
    cudaError_t e = cudaErrorInvalidConfiguration;
    ((S == idx ? (void)(e = [&] {
        constexpr Shape sh = kShapes[S];
        auto kern = kernel_of<S>();
        const size_t smem = transport_smem(m.K, sh);
        cudaError_t r = ensure_smem((const void*)kern, smem);
        if (r != cudaSuccess) return r;
        kern<<<(unsigned)((n + sh.blk - 1) / sh.blk), sh.blk * sh.np, smem, st>>>(m, n, ld, T, p, Y, mu, lam, D);
        return cudaGetLastError();
    }())
               : (void)0),
     ...);
    return e;
}

}  // namespace

cudaError_t launch_transport_df(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, double* mu, double* lam, double* Dmix, cudaStream_t s) {
    const int idx = plan_shape(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx(idx, std::make_integer_sequence<int, kNumShapes>{}, m, n, ld, T, p, Y, mu, lam, Dmix, s);
}

}  // namespace nk
