// Dense Jacobian of the implicit-stage sources (the production and heat-release terms of
// Eq. 1a-b at fixed p) with respect to x = (T, Y_k), assembled per point from a stored
// linearization of the rates (k_lin.cu) and the sources at the same state.  It feeds the
// per-point block-Jacobi preconditioner of the implicit stage's GMRES solve (the paper runs
// that solve unpreconditioned, Sec. 2; with large steps the per-point blocks of I - dt J carry
// the stiffness).
//
// With s = sum Y_k/W_k, rho = p/(R T s), C_k = rho Y_k/W_k, a_j = -1/(W_j s) (d ln rho/dY_j)
// and the linearization dq_r = A_r dT/T + sum_e B_re dC_e + L_r d[M] of every rate of progress:
//   G_kj  = sum_r nu_kr (B_rj + L_r (eps_rj - 1))    (terms listed per mechanism, DevMech::jac_*)
//   U_k   = sum_j G_kj C_j,  V_k = sum_r nu_kr A_r,  Lam_k = sum_r nu_kr L_r
//   d omega_k/dY_j = a_j U_k + (rho/W_j) G_kj,   d omega_k/dT = (V_k - U_k - (p/RT) Lam_k)/T
// (the third-body concentration moves with T through p/(RT) and with the density through the
// listed efficiencies).  Then, with fY_k = W_k omega_k/rho and fT = hrr/(rho c_p):
//   J[Y_k, Y_j] = (W_k/W_j) (G_kj - c_k),  c_k = (U_k - omega_k) (RT/p)
//   J[Y_k, T]   = W_k/(rho T) (V_k - U_k - (p/RT) Lam_k + omega_k)
//   J[T, Y_j]   = (dhrr/dY_j - hrr (a_j + c_p,j/(W_j c_p))) / (rho c_p),
//                 dhrr/dY_j = -RT (a_j sum_k (h_k/RT) U_k + (rho/W_j) sum_k (h_k/RT) G_kj)
//   J[T, T]     = (dhrr/dT - hrr (dc_p/dT / c_p - 1/T)) / (rho c_p),
//                 dhrr/dT = -RT sum_k (h_k/RT) d omega_k/dT - sum_k c_p,k omega_k
// with omega_k and hrr recovered from the given sources.  Plain double arithmetic.
//
// One warp per point, the point's block in shared memory (row stride N + 1): rows k + 1 belong
// to lanes (k = lane, lane + 32, ...), which gather G_kj of their rows (the structural nonzeros,
// from the stored linearization in global memory, whose sectors the block's neighbouring points
// share), then lanes over columns form sum_k (h_k/RT) G_kj; mixture sums are warp reductions
// (fixed order).  Per point in shared memory: the block, 6K + 8 doubles of vectors, 2N ints.
// Two outputs:
//   the Jacobian itself, entry (r, c) at J[(r (K+1) + c) ldJ + i] (r, c in the order T, Y_0..);
//   the preconditioner block P = I - dt diag(w) J diag(1/w), w the error weights of the Newton
//   solve, each row r scaled by 2^-e_r so that its largest entry lies in [1/2, 1) (the pivoting
//   then compares scaled rows) and factored in place (nk_lu.cuh), written in pivot order with
//   the pivot words (row | e_row << 16).
// The block of `pts` points is written entry by entry for all its points at once.
#include <algorithm>

#include "nk_lu.cuh"

namespace nk {
namespace {

// 2^-e with the largest |entry| m = f 2^e, f in [1/2, 1); e = 0 for a zero or non-finite m
__device__ __forceinline__ int row_exponent(double m) {
    int e = 0;
    if (m > 0.0 && m <= 1.7976931348623157e308) frexp(m, &e);
    return e;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// doubles of shared memory per point: N (N + 1) block entries, 6K + 8 of vectors, 2N ints
__host__ __device__ inline int64_t point_doubles(int K) {
    const int N = K + 1;
    return (int64_t)N * (N + 1) + 6 * K + 8 + N;
}

struct BlockOut {
    double* J;            // !PREC: the Jacobian
    double* F;            // PREC: the factors
    int32_t* piv;         // PREC: pivot words
    int64_t ld;           // of J or F and piv
    const double* w;      // PREC: error weights, row r at w + r ldw
    int64_t ldw;
    double dt;
};

template <bool PREC>
__global__ void block_kernel(const DevMech m, const int64_t n, const int64_t ld, const double* __restrict__ T,
                             const double* __restrict__ p, const double* __restrict__ Y,
                             const double* __restrict__ lin, const int64_t ldl, const double* __restrict__ fT,
                             const double* __restrict__ fY, const int64_t ldf, const BlockOut out, const int pts) {
    extern __shared__ double sm[];
    const int K = m.K, N = K + 1, S = N + 1;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * pts;
    const int np = (int)(n - i0 < pts ? n - i0 : pts);
    const int64_t per = point_doubles(K);
    double* a = sm + (int64_t)q * per;                         // the block, row stride S
    double* yw = a + (int64_t)N * S;                           // Y_j / W_j
    double* HG = yw + K;                                       // sum_k (h_k/RT) G_kj
    double* colf = HG + K;                                     // PREC: 1 / (W_j w_(j+1))
    double* Uv = colf + K;                                     // U_k
    double* dW = Uv + K;                                       // d omega_k / dT
    double* hk = dW + K;                                       // h_k / RT
    int32_t* perm = reinterpret_cast<int32_t*>(hk + K + 8);    // PREC: [N] original rows, pivot order
    int32_t* ex = perm + N;                                    // PREC: [N] row exponents
    if (q < np) {
        const int64_t i = i0 + q;
        const double* Li = lin + i;                            // slot s at Li[s ldl]
        const double Ti = T[i], invT = 1.0 / Ti;
        const double pRT = p[i] * invT * kInvR, RTp = 1.0 / pRT;
        double s = 0.0, cpm = 0.0, dcpm = 0.0;
        for (int k = lane; k < K; k += 32) {
            const double y = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
            const double* c = nasa_range(m, k, Ti);
            yw[k] = y;
            s += y;
            cpm = fma(y, nasa_cpR(c, Ti), cpm);
            dcpm = fma(y, nasa_dcpR_dT(c, Ti), dcpm);
            hk[k] = Li[(m.R + m.lin_nb + (m.R - m.R_el) + 1 + k) * ldl];
            if (PREC) colf[k] = __ldg(m.invW + k) / out.w[(int64_t)(k + 1) * out.ldw + i];
        }
        s = warp_sum(s);
        cpm = warp_sum(cpm) * kR;
        dcpm = warp_sum(dcpm) * kR;
        const double rho = pRT / s, irho = 1.0 / rho;
        const double hrr = fT[i] * rho * cpm;
        const int64_t sH = m.R + m.lin_nb + (m.R - m.R_el) + 1;    // h_k/RT; sum_k c_p,k omega_k/R before
        __syncwarp();
        // rows k + 1: the raw G_kj first, V_k and Lam_k in the row's first and padding entries
        // (one flat pass over the row's terms, eight loads in flight per lane)
        for (int k = lane; k < K; k += 32) {
            double* ar = a + (k + 1) * S;
            for (int j = 0; j <= N; ++j) ar[j] = 0.0;
            const int t0 = __ldg(m.jac_row + k), t1 = __ldg(m.jac_row + k + 1);
            const int4* tr = reinterpret_cast<const int4*>(m.jac_term);
#pragma unroll 8
            for (int t = t0; t < t1; ++t) {
                const int4 x = __ldg(tr + t);                  // coef (lo, hi), slot, dst
                ar[x.w] = fma(__hiloint2double(x.y, x.x), Li[(int64_t)x.z * ldl], ar[x.w]);
            }
            double U = 0.0;
            for (int j = 0; j < K; ++j) U = fma(ar[j + 1], yw[j], U);
            U *= rho;                                          // sum_j G_kj C_j
            Uv[k] = U;
            dW[k] = (ar[0] - U - pRT * ar[N]) * invT;          // d omega_k / dT
        }
        __syncwarp();
        double hU = 0.0, hJT = 0.0;
        for (int j = lane; j < K; j += 32) {
            const double hj = hk[j];
            double hg = 0.0;
            for (int k = 0; k < K; ++k) hg = fma(hk[k], a[(k + 1) * S + j + 1], hg);
            HG[j] = hg;
            hU = fma(hj, Uv[j], hU);
            hJT = fma(hj, dW[j], hJT);
        }
        hU = warp_sum(hU);
        hJT = warp_sum(hJT);
        __syncwarp();
        // species rows: J[Y_k, Y_j] = (W_k/W_j) (G_kj - c_k), J[Y_k, T] = W_k/rho (dw_k/dT + w_k/T)
        const double iw0 = PREC ? 1.0 / out.w[i] : 1.0;
        for (int k = lane; k < K; k += 32) {
            double* ar = a + (k + 1) * S;
            const double Wk = __ldg(m.W + k);
            const double om = fY[(int64_t)k * ldf + i] * rho * __ldg(m.invW + k);
            const double ck = (Uv[k] - om) * RTp;
            const double jT = Wk * irho * fma(om, invT, dW[k]);
            if constexpr (PREC) {
                const double rw = out.dt * out.w[(int64_t)(k + 1) * out.ldw + i];   // dt w_(k+1)
                const double vT = -rw * jT * iw0, rf = rw * Wk;
                double mx = fabs(vT);
                ar[0] = vT;
                for (int j = 0; j < K; ++j) {
                    const double v = (k == j ? 1.0 : 0.0) - rf * (ar[j + 1] - ck) * colf[j];
                    ar[j + 1] = v;
                    mx = fmax(mx, fabs(v));
                }
                const int e = row_exponent(mx);
                const double sc = ldexp(1.0, -e);
                for (int j = 0; j < N; ++j) ar[j] *= sc;
                ex[k + 1] = e;
            } else {
                ar[0] = jT;
                for (int j = 0; j < K; ++j) ar[j + 1] = Wk * (ar[j + 1] - ck) * __ldg(m.invW + j);
            }
        }
        // temperature row
        const double RT = kR * Ti, icp = irho / cpm, icpm = 1.0 / cpm, is = 1.0 / s;
        const double rT = PREC ? out.dt * out.w[i] : 1.0;
        double mx = 0.0;
        for (int j = lane; j < K; j += 32) {
            const double iw = __ldg(m.invW + j);
            const double aj = -iw * is;
            const double cpj = kR * nasa_cpR(nasa_range(m, j, Ti), Ti);
            const double dh = -RT * fma(aj, hU, rho * iw * HG[j]);
            const double v = icp * fma(-hrr, fma(cpj * iw, icpm, aj), dh);   // J[T, Y_j]
            if constexpr (PREC) {
                const double qv = -rT * v * __ldg(m.W + j) * colf[j];
                a[j + 1] = qv;
                mx = fmax(mx, fabs(qv));
            } else {
                a[j + 1] = v;
            }
        }
        const double S1 = Li[(sH - 1) * ldl];
        const double dhT = fma(-RT, hJT, -kR * S1);
        const double jTT = icp * fma(-hrr, fma(dcpm, icpm, -invT), dhT);
        if constexpr (PREC) {
            const double vTT = 1.0 - out.dt * jTT;
            mx = fmax(warp_max(mx), fabs(vTT));
            const int e0 = row_exponent(mx);
            const double sc0 = ldexp(1.0, -e0);
            for (int j = lane; j < K; j += 32) a[j + 1] *= sc0;
            if (lane == 0) {
                a[0] = vTT * sc0;
                ex[0] = e0;
            }
            __syncwarp();
            warp_lu(a, N, S, lane, perm);
        } else if (lane == 0) {
            a[0] = jTT;
        }
    }
    __syncthreads();
    const int64_t NN = (int64_t)N * N;
    double* dst = PREC ? out.F : out.J;
    for (int64_t f = threadIdx.x; f < NN * np; f += blockDim.x) {
        const int64_t e = f / np;
        const int qq = (int)(f - e * np);
        const int r = (int)(e / N), c = (int)(e % N);
        dst[e * out.ld + i0 + qq] = sm[(int64_t)qq * per + r * S + c];
    }
    if constexpr (PREC) {
        for (int f = threadIdx.x; f < N * np; f += blockDim.x) {
            const int k = f / np, qq = f % np;
            const int32_t* pq = reinterpret_cast<const int32_t*>(sm + (int64_t)qq * per + (int64_t)N * S + 6 * K + 8);
            const int r = pq[k];
            out.piv[(int64_t)k * out.ld + i0 + qq] = (r & 0xffff) | (int32_t)((uint32_t)pq[N + r] << 16);
        }
    }
}

template <bool PREC>
cudaError_t launch_blocks(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                          const double* lin, int64_t ldl, const double* fT, const double* fY, int64_t ldf,
                          const BlockOut& out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (m.K + 1 > kMaxPrecondN) return cudaErrorInvalidValue;
    const size_t per = (size_t)point_doubles(m.K) * sizeof(double);
    const int pts = (int)std::min<size_t>(8, smem_limit() / per);
    if (pts < 1) return cudaErrorInvalidConfiguration;
    const size_t bytes = per * pts;
    cudaError_t e = ensure_smem((const void*)block_kernel<PREC>, bytes);
    if (e != cudaSuccess) return e;
    block_kernel<PREC><<<(unsigned)((n + pts - 1) / pts), 32 * pts, bytes, s>>>(m, n, ld, T, p, Y, lin, ldl, fT, fY,
                                                                              ldf, out, pts);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rhs_jacobian(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                double* J, int64_t ldJ, cudaStream_t s) {
    const BlockOut out{J, nullptr, nullptr, ldJ, nullptr, 0, 0.0};
    return launch_blocks<false>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ld, out, s);
}

cudaError_t launch_precond_setup(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                 int64_t ldf, const double* w, int64_t ldw, double dt, double* F, int32_t* piv,
                                 int64_t ldF, cudaStream_t s) {
    const BlockOut out{nullptr, F, piv, ldF, w, ldw, dt};
    return launch_blocks<true>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ldf, out, s);
}

}  // namespace nk
