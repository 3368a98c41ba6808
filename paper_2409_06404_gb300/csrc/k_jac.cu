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
// with omega_k and hrr recovered from the given sources.  One thread per point; G_kj of one row
// is gathered into a shared-memory row (the structural nonzeros only), then the whole row is
// written; sum_k (h_k/RT) G_kj accumulates in a second shared row for the temperature row,
// written last.  Plain double arithmetic.
//
// Two outputs: the Jacobian itself (entry (r, c) at J[(r (K+1) + c) ldJ + i], r and c in the
// order T, Y_0..Y_{K-1}), or the preconditioner block P = I - dt diag(w) J diag(1/w), w the
// error weights of the Newton solve (same entry layout), each row r scaled by 2^-e_r so that
// its largest entry lies in [1/2, 1) (the pivoting then compares scaled rows), e_r to
// piv[r ldq + i].
#include <algorithm>
#include <mutex>
#include <vector>

#include "nk_lu.cuh"

namespace nk {
namespace {

template <bool PREC>
struct JacSink {
    double* J;            // !PREC
    double* P;            // PREC
    int32_t* piv;         // PREC: row exponents e_r
    int64_t ld;
    const double* w;      // PREC: error weights, row r at w + r ldw
    int64_t ldw;
    double dt;
};

// 2^-e with the largest |entry| m = f 2^e, f in [1/2, 1); e = 0 for a zero or non-finite m
__device__ __forceinline__ int row_exponent(double m) {
    int e = 0;
    if (m > 0.0 && m <= 1.7976931348623157e308) frexp(m, &e);
    return e;
}

// scaled row r of P from its values in sRow (reset to 0 on the way)
template <int BLK>
__device__ __forceinline__ void put_scaled_row(const JacSink<true>& out, int64_t i, int r, int N, double* sRow,
                                               double vT, double mx) {
    const int e = row_exponent(mx);
    const double sc = ldexp(1.0, -e);
    const int64_t o = (int64_t)r * N * out.ld + i;
    out.P[o] = vT * sc;
    for (int j = 0; j + 1 < N; ++j) {
        out.P[o + (int64_t)(j + 1) * out.ld] = sRow[j * BLK] * sc;
        sRow[j * BLK] = 0.0;
    }
    out.piv[(int64_t)r * out.ld + i] = e;
}

template <int BLK, bool PREC>
__global__ void __launch_bounds__(BLK) jac_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                  const double* __restrict__ T, const double* __restrict__ p,
                                                  const double* __restrict__ Y, const double* __restrict__ lin,
                                                  const int64_t ldl, const double* __restrict__ fT,
                                                  const double* __restrict__ fY, const int64_t ldf,
                                                  const JacSink<PREC> out) {
    extern __shared__ double smem[];
    const int K = m.K, N = K + 1;
    const int64_t i = (int64_t)blockIdx.x * BLK + threadIdx.x;
    if (i >= n) return;                                        // (no barrier in this kernel)
    double* sRow = smem + threadIdx.x;                         // G_kj of the current row k
    double* sHG = smem + (size_t)K * BLK + threadIdx.x;        // sum_k (h_k/RT) G_kj
    double* sCol = smem + (size_t)2 * K * BLK + threadIdx.x;  // PREC: 1/(W_j w_j)

    const double Ti = T[i], invT = 1.0 / Ti;
    const double pRT = p[i] * invT * kInvR, RTp = 1.0 / pRT;
    double s = 0.0, cpm = 0.0, dcpm = 0.0;
    for (int k = 0; k < K; ++k) {
        const double yw = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
        const double* c = nasa_range(m, k, Ti);
        s += yw;
        cpm = fma(yw, nasa_cpR(c, Ti), cpm);
        dcpm = fma(yw, nasa_dcpR_dT(c, Ti), dcpm);
        sRow[k * BLK] = 0.0;
        sHG[k * BLK] = 0.0;
    }
    cpm *= kR;
    dcpm *= kR;
    const double rho = pRT / s;
    const double hrr = fT[i] * rho * cpm;
    const double irho = 1.0 / rho;
    double iw0 = 1.0;                                          // PREC: 1/w_0
    if constexpr (PREC) {
        iw0 = 1.0 / out.w[i];
        for (int j = 0; j < K; ++j) sCol[j * BLK] = __ldg(m.invW + j) / out.w[(int64_t)(j + 1) * out.ldw + i];
    }

    const double* H = lin + (int64_t)(m.R + m.lin_nb + (m.R - m.R_el) + 1) * ldl + i;   // h_k/RT
    double hU = 0.0, hJT = 0.0;
    for (int k = 0; k < K; ++k) {
        const double Wk = __ldg(m.W + k);
        const double om = fY[(int64_t)k * ldf + i] * rho * __ldg(m.invW + k);
        const double hk = H[(int64_t)k * ldl];
        double U = 0.0, V = 0.0, Lam = 0.0;
        const int e0 = __ldg(m.jac_row + k), e1 = __ldg(m.jac_row + k + 1);
        for (int e = e0; e < e1; ++e) {
            const int col = __ldg(m.jac_col + e);
            const int t0 = __ldg(m.jac_ent + e), t1 = __ldg(m.jac_ent + e + 1);
            double g = 0.0;
#pragma unroll 4
            for (int t = t0; t < t1; ++t) {
                const double coef = __ldg(&m.jac_term[t].coef);
                const int slot = __ldg(&m.jac_term[t].slot);
                g = fma(coef, lin[(int64_t)slot * ldl + i], g);
            }
            if (col >= 0) {
                sRow[col * BLK] = g;
                sHG[col * BLK] = fma(hk, g, sHG[col * BLK]);
                U = fma(g, Y[(int64_t)col * ld + i] * __ldg(m.invW + col), U);
            } else if (col == -1) {
                V = g;
            } else {
                Lam = g;
            }
        }
        U *= rho;                                              // sum_j G_kj C_j
        const double ck = (U - om) * RTp;
        const double dwT = (V - U - pRT * Lam) * invT;         // d omega_k / dT
        hU = fma(hk, U, hU);
        hJT = fma(hk, dwT, hJT);
        const double jT = Wk * irho * fma(om, invT, dwT);      // J[Y_k, T]
        const int64_t o = (int64_t)(k + 1) * N * out.ld + i;  // entry (k + 1, 0)
        if constexpr (PREC) {
            const double rw = out.dt * out.w[(int64_t)(k + 1) * out.ldw + i];   // dt w_(k+1)
            const double vT = -rw * jT * iw0, rf = rw * Wk;
            double mx = fabs(vT);
            for (int j = 0; j < K; ++j) {
                const double v = (k == j ? 1.0 : 0.0) - rf * (sRow[j * BLK] - ck) * sCol[j * BLK];
                sRow[j * BLK] = v;
                mx = fmax(mx, fabs(v));
            }
            put_scaled_row<BLK>(out, i, k + 1, N, sRow, vT, mx);
        } else {
            out.J[o] = jT;
            for (int j = 0; j < K; ++j)
                out.J[o + (int64_t)(j + 1) * out.ld] = Wk * (sRow[j * BLK] - ck) * __ldg(m.invW + j);
            for (int e = e0; e < e1; ++e) {
                const int col = __ldg(m.jac_col + e);
                if (col >= 0) sRow[col * BLK] = 0.0;
            }
        }
    }
    // temperature row
    const double RT = kR * Ti, icp = irho / cpm, icpm = 1.0 / cpm, is = 1.0 / s;
    const double rT = PREC ? out.dt * out.w[i] : 1.0;        // PREC: dt w_0
    double mx = 0.0;
    for (int j = 0; j < K; ++j) {
        const double iw = __ldg(m.invW + j);
        const double aj = -iw * is;
        const double cpj = kR * nasa_cpR(nasa_range(m, j, Ti), Ti);
        const double dh = -RT * fma(aj, hU, rho * iw * sHG[j * BLK]);
        const double v = icp * fma(-hrr, fma(cpj * iw, icpm, aj), dh);   // J[T, Y_j]
        if constexpr (PREC) {
            const double q = -rT * v * __ldg(m.W + j) * sCol[j * BLK];
            sRow[j * BLK] = q;
            mx = fmax(mx, fabs(q));
        } else {
            out.J[(int64_t)(j + 1) * out.ld + i] = v;
        }
    }
    const double S1 = lin[(int64_t)(m.R + m.lin_nb + (m.R - m.R_el)) * ldl + i];   // sum_k c_p,k omega_k / R
    const double dhT = fma(-RT, hJT, -kR * S1);
    const double jTT = icp * fma(-hrr, fma(dcpm, icpm, -invT), dhT);
    if constexpr (PREC) {
        const double vT = 1.0 - out.dt * jTT;
        put_scaled_row<BLK>(out, i, 0, N, sRow, vT, fmax(mx, fabs(vT)));
    } else {
        out.J[i] = jTT;
    }
}

// ---------------------------------------------------------------- fused block set-up
// The preconditioner's set-up for points whose stored linearization and block fit in shared
// memory together: one warp per point assembles P (the formulas above, the same expressions)
// from the point's linearization, staged into shared memory by the whole block with coalesced
// loads, and factors it in place (nk_lu.cuh); the block then writes the factors of its points
// entry by entry.  Rows are owned by lanes (k + 1 for species k = lane, lane + 32, ...), the
// column sums sum_k (h_k/RT) G_kj by lanes over columns; the per-point sums run in species
// order in every lane, so that the blocks equal the assembly kernel's bit for bit.  Shared
// memory per point: the slots, N (N + 1) block entries, 5K + 8 doubles of vectors, 2N ints.
__host__ __device__ inline int64_t fused_point_doubles(int K, int64_t slots) {
    const int N = K + 1;
    return slots + (int64_t)N * (N + 1) + 5 * K + 8 + N;     // (the last N doubles hold 2N ints)
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void precond_setup_kernel(const DevMech m, const int64_t n, const int64_t ld, const double* __restrict__ T,
                                     const double* __restrict__ p, const double* __restrict__ Y,
                                     const double* __restrict__ lin, const int64_t ldl, const int slots,
                                     const double* __restrict__ fT, const double* __restrict__ fY, const int64_t ldf,
                                     const double* __restrict__ w, const int64_t ldw, const double dt,
                                     double* __restrict__ F, int32_t* __restrict__ piv, const int64_t ldF,
                                     const int pts) {
    extern __shared__ double sm[];
    const int K = m.K, N = K + 1, S = N + 1;
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * pts;
    const int np = (int)(n - i0 < pts ? n - i0 : pts);
    const int64_t per = fused_point_doubles(K, slots);
    double* base = sm + (int64_t)q * per;
    double* L = base;                                          // stored linearization
    double* a = L + slots;                                     // the block, row stride S
    double* yw = a + (int64_t)N * S;                           // Y_j / W_j
    double* HG = yw + K;                                       // sum_k (h_k/RT) G_kj
    double* colf = HG + K;                                     // 1 / (W_j w_(j+1))
    double* Uv = colf + K;                                     // U_k
    double* dW = Uv + K;                                       // d omega_k / dT
    int32_t* perm = reinterpret_cast<int32_t*>(dW + K + 8);    // [N] pivot rows
    int32_t* ex = perm + N;                                    // [N] row exponents
    for (int64_t f = threadIdx.x; f < (int64_t)slots * np; f += blockDim.x) {
        const int64_t s = f / np;
        const int qq = (int)(f - s * np);
        sm[(int64_t)qq * per + s] = lin[s * ldl + i0 + qq];
    }
    __syncthreads();
    if (q < np) {
        const int64_t i = i0 + q;
        const double Ti = T[i], invT = 1.0 / Ti;
        const double pRT = p[i] * invT * kInvR, RTp = 1.0 / pRT;
        for (int k = lane; k < K; k += 32) {
            yw[k] = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
            colf[k] = __ldg(m.invW + k) / w[(int64_t)(k + 1) * ldw + i];
        }
        __syncwarp();
        double s = 0.0, cpm = 0.0, dcpm = 0.0;                 // (every lane, in species order)
        for (int k = 0; k < K; ++k) {
            const double y = yw[k];
            const double* c = nasa_range(m, k, Ti);
            s += y;
            cpm = fma(y, nasa_cpR(c, Ti), cpm);
            dcpm = fma(y, nasa_dcpR_dT(c, Ti), dcpm);
        }
        cpm *= kR;
        dcpm *= kR;
        const double rho = pRT / s, irho = 1.0 / rho;
        const double hrr = fT[i] * rho * cpm;
        const double iw0 = 1.0 / w[i];
        const double* H = L + (m.R + m.lin_nb + (m.R - m.R_el) + 1);   // h_k/RT
        __syncwarp();
        // species rows k + 1: the raw G_kj first
        double ckr[kMaxRowsPerLane], jTr[kMaxRowsPerLane];
#pragma unroll
        for (int b = 0; b < kMaxRowsPerLane; ++b) {
            const int k = lane + 32 * b;
            ckr[b] = jTr[b] = 0.0;
            if (k >= K) continue;
            double* ar = a + (k + 1) * S;
            for (int j = 0; j < N; ++j) ar[j] = 0.0;
            const double om = fY[(int64_t)k * ldf + i] * rho * __ldg(m.invW + k);
            double U = 0.0, V = 0.0, Lam = 0.0;
            const int e0 = __ldg(m.jac_row + k), e1 = __ldg(m.jac_row + k + 1);
            for (int e = e0; e < e1; ++e) {
                const int col = __ldg(m.jac_col + e);
                const int t0 = __ldg(m.jac_ent + e), t1 = __ldg(m.jac_ent + e + 1);
                double g = 0.0;
                for (int t = t0; t < t1; ++t) g = fma(__ldg(&m.jac_term[t].coef), L[__ldg(&m.jac_term[t].slot)], g);
                if (col >= 0) {
                    ar[col + 1] = g;
                    U = fma(g, yw[col], U);
                } else if (col == -1) {
                    V = g;
                } else {
                    Lam = g;
                }
            }
            U *= rho;
            const double dwT = (V - U - pRT * Lam) * invT;
            Uv[k] = U;
            dW[k] = dwT;
            ckr[b] = (U - om) * RTp;
            jTr[b] = __ldg(m.W + k) * irho * fma(om, invT, dwT);
        }
        __syncwarp();
        for (int j = lane; j < K; j += 32) {
            double hg = 0.0;
            for (int k = 0; k < K; ++k) hg = fma(H[k], a[(k + 1) * S + j + 1], hg);
            HG[j] = hg;
        }
        double hU = 0.0, hJT = 0.0;                            // (every lane, the same order)
        for (int k = 0; k < K; ++k) {
            hU = fma(H[k], Uv[k], hU);
            hJT = fma(H[k], dW[k], hJT);
        }
        __syncwarp();
        // species rows of P, scaled
#pragma unroll
        for (int b = 0; b < kMaxRowsPerLane; ++b) {
            const int k = lane + 32 * b;
            if (k >= K) continue;
            double* ar = a + (k + 1) * S;
            const double rw = dt * w[(int64_t)(k + 1) * ldw + i];
            const double vT = -rw * jTr[b] * iw0, rf = rw * __ldg(m.W + k), ck = ckr[b];
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
        }
        // temperature row
        const double RT = kR * Ti, icp = irho / cpm, icpm = 1.0 / cpm, is = 1.0 / s;
        const double rT = dt * w[i];
        double mx = 0.0;
        for (int j = lane; j < K; j += 32) {
            const double iw = __ldg(m.invW + j);
            const double aj = -iw * is;
            const double cpj = kR * nasa_cpR(nasa_range(m, j, Ti), Ti);
            const double dh = -RT * fma(aj, hU, rho * iw * HG[j]);
            const double v = icp * fma(-hrr, fma(cpj * iw, icpm, aj), dh);
            const double qv = -rT * v * __ldg(m.W + j) * colf[j];
            a[j + 1] = qv;
            mx = fmax(mx, fabs(qv));
        }
        const double S1 = L[m.R + m.lin_nb + (m.R - m.R_el)];
        const double dhT = fma(-RT, hJT, -kR * S1);
        const double jTT = icp * fma(-hrr, fma(dcpm, icpm, -invT), dhT);
        const double vTT = 1.0 - dt * jTT;
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
    }
    __syncthreads();
    const int64_t NN = (int64_t)N * N;
    for (int64_t f = threadIdx.x; f < NN * np; f += blockDim.x) {
        const int64_t e = f / np;
        const int qq = (int)(f - e * np);
        const int k = (int)(e / N), j = (int)(e % N);
        const double* bq = sm + (int64_t)qq * per;
        const int32_t* pq = reinterpret_cast<const int32_t*>(bq + slots + (int64_t)N * S + 5 * K + 8);
        F[e * ldF + i0 + qq] = bq[slots + (int64_t)pq[k] * S + j];
    }
    for (int f = threadIdx.x; f < N * np; f += blockDim.x) {
        const int k = f / np, qq = f % np;
        const int32_t* pq = reinterpret_cast<const int32_t*>(sm + (int64_t)qq * per + slots + (int64_t)N * S + 5 * K + 8);
        const int r = pq[k];
        piv[(int64_t)k * ldF + i0 + qq] = (r & 0xffff) | (int32_t)((uint32_t)pq[N + r] << 16);
    }
}

struct Plan {
    int dev, K, blk;
    bool prec;
};
std::mutex g_mu;
std::vector<Plan> g_plans;

size_t jac_smem(int K, int blk) { return (size_t)blk * 3 * K * sizeof(double); }

template <bool PREC>
const void* kern_of(int blk) {
    switch (blk) {
        case 32: return (const void*)jac_kernel<32, PREC>;
        case 64: return (const void*)jac_kernel<64, PREC>;
        default: return (const void*)jac_kernel<128, PREC>;
    }
}

// the block size with the most resident warps
template <bool PREC>
int plan_blk(int K) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (const Plan& q : g_plans)
            if (q.dev == dev && q.K == K && q.prec == PREC) return q.blk;
    }
    int best = -1, best_warps = 0;
    for (int blk : {32, 64, 128}) {
        const size_t bytes = jac_smem(K, blk);
        if (bytes > smem_limit()) continue;
        const void* k = kern_of<PREC>(blk);
        if (ensure_smem(k, bytes) != cudaSuccess) continue;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, blk, bytes) != cudaSuccess) continue;
        if (blocks * blk / 32 > best_warps) {
            best_warps = blocks * blk / 32;
            best = blk;
        }
    }
    if (best > 0) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_plans.push_back({dev, K, best, PREC});
    }
    return best;
}

template <bool PREC>
cudaError_t launch(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                   const double* lin, int64_t ldl, const double* fT, const double* fY, int64_t ldf,
                   const JacSink<PREC>& out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blk = plan_blk<PREC>(m.K);
    if (blk < 0) return cudaErrorInvalidConfiguration;
    const size_t bytes = jac_smem(m.K, blk);
    const unsigned grid = (unsigned)((n + blk - 1) / blk);
    switch (blk) {
        case 32: jac_kernel<32, PREC><<<grid, 32, bytes, s>>>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ldf, out); break;
        case 64: jac_kernel<64, PREC><<<grid, 64, bytes, s>>>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ldf, out); break;
        default: jac_kernel<128, PREC><<<grid, 128, bytes, s>>>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ldf, out); break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rhs_jacobian(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                double* J, int64_t ldJ, cudaStream_t s) {
    JacSink<false> out{J, nullptr, nullptr, ldJ, nullptr, 0, 0.0};
    return launch<false>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ld, out, s);
}

cudaError_t launch_precond_setup(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                 int64_t ldf, const double* w, int64_t ldw, double dt, double* F, int32_t* piv,
                                 int64_t ldF, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int N = m.K + 1;
    const int64_t slots = lin_slots(m);
    const size_t per = (size_t)fused_point_doubles(m.K, slots) * sizeof(double);
    const size_t lim = smem_limit();
    int pts = (int)std::min<size_t>(8, lim / per);
    if (pts >= 1) {
        const size_t bytes = per * pts;
        cudaError_t e = ensure_smem((const void*)precond_setup_kernel, bytes);
        if (e != cudaSuccess) return e;
        precond_setup_kernel<<<(unsigned)((n + pts - 1) / pts), 32 * pts, bytes, s>>>(
            m, n, ld, T, p, Y, lin, ldl, (int)slots, fT, fY, ldf, w, ldw, dt, F, piv, ldF, pts);
        return cudaGetLastError();
    }
    // the point does not fit: blocks by the assembly kernel, then the factorization kernel
    cudaError_t e = launch_precond_blocks(m, n, ld, T, p, Y, lin, ldl, fT, fY, ldf, w, ldw, dt, F, piv, ldF, s);
    if (e != cudaSuccess) return e;
    return launch_precond_factor(N, n, F, ldF, piv, ldF, s);
}

cudaError_t launch_precond_blocks(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                  const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                  int64_t ldf, const double* w, int64_t ldw, double dt, double* P, int32_t* piv,
                                  int64_t ldP, cudaStream_t s) {
    JacSink<true> out{nullptr, P, piv, ldP, w, ldw, dt};
    return launch<true>(m, n, ld, T, p, Y, lin, ldl, fT, fY, ldf, out, s);
}

}  // namespace nk
