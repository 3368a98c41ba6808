// Application of the per-point block-Jacobi preconditioner of the implicit stage's GMRES
// solve: z = P^-1 v from the LU factors that k_jac.cu leaves (double precision: the blocks of
// stiff chemistry in the solver's weights are so ill-conditioned that single-precision factors,
// even of row- and column-equilibrated blocks, missed the solution by orders of magnitude in
// testing, while double-precision ones stay within tens of per cent -- enough to steer GMRES).
//
// Storage, entry (r, c) of point i at F[(r N + c) ldF + i] (N = K + 1, all points of one entry
// contiguous), rows in pivot order: row k holds L_k,0..k-1 (unit lower part) and U_k,k..N-1 of
// the row-scaled block D P, with 1/U_kk in place of U_kk; piv[k ldq + i] holds that row's
// original index (low 16 bits) and its exponent e (high 16 bits, signed), D = diag(2^-e).  P z = v
// is then L U z = (D v) in pivot order.  One thread per point, forward then backward
// substitution with the vector in shared memory and the factors read once, in order, streamed
// into shared memory ahead of use (coalesced across the warp's points).
#include <algorithm>
#include <cstdint>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kApplyPts = 32;   // points (threads) per block

// Asynchronous 8-byte copy global -> shared (cp.async, completion tracked per thread in commit
// groups), its group commit and the wait for all but the newest N groups.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Step s of the two substitutions: the forward row k = s (entries 0..k-1 of L) for s < N, then
// the backward row k = 2N - 1 - s (entries k..N-1 of U, the first being 1/U_kk).
__device__ __forceinline__ void step_row(int s, int N, int& k, int& j0, int& j1) {
    if (s < N) {
        k = s;
        j0 = 0;
        j1 = s;
    } else {
        k = 2 * N - 1 - s;
        j0 = k;
        j1 = N;
    }
}

// z = P^-1 v per point: v and z rows of ldv / ldz (row r of point i at r ld + i), of type TI and
// TO, arithmetic in double.  One thread per point; the factor entries each step needs are copied
// into shared memory asynchronously two steps ahead (cp.async into two row buffers), so each
// thread keeps up to two factor rows of loads in flight instead of stalling on every row's first
// load.  Every thread works on its own columns of the shared arrays only (no block barrier).  z
// may alias v: each thread reads its point's entries of v before it writes z.
template <class TI, class TO>
__global__ void __launch_bounds__(kApplyPts) lu_apply_kernel(const int N, const int64_t n, const double* __restrict__ F,
                                                             const int64_t ldF, const int32_t* __restrict__ piv,
                                                             const int64_t ldq, const TI* v, const int64_t ldv, TO* z,
                                                             const int64_t ldz) {
    extern __shared__ double sm[];
    const int64_t i = (int64_t)blockIdx.x * kApplyPts + threadIdx.x;
    if (i >= n) return;
    double* y = sm + threadIdx.x;                                  // y[j * kApplyPts]
    double* const buf0 = sm + (size_t)N * kApplyPts + threadIdx.x;   // the two row buffers
    double* const buf1 = buf0 + (size_t)N * kApplyPts;
    const double* f = F + i;
    const int S = 2 * N;
    auto issue = [&](int s, double* b) {
        int k, j0, j1;
        step_row(s, N, k, j0, j1);
        const double* fk = f + (int64_t)k * N * ldF;
        for (int j = j0; j < j1; ++j) cp_async8(b + j * kApplyPts, fk + (int64_t)j * ldF);
        cp_async_commit();
    };
    issue(0, buf0);
    if (S > 1) issue(1, buf1);
    for (int s = 0; s < S; ++s) {
        double* b = (s & 1) ? buf1 : buf0;
        cp_async_wait<1>();                                        // step s's copies have landed
        int k, j0, j1;
        step_row(s, N, k, j0, j1);
        if (s < N) {                                               // L y = (D v)(perm), unit diagonal
            double d0 = 0.0, d1 = 0.0;
            int j = 0;
            for (; j + 1 < k; j += 2) {
                d0 = fma(b[j * kApplyPts], y[j * kApplyPts], d0);
                d1 = fma(b[(j + 1) * kApplyPts], y[(j + 1) * kApplyPts], d1);
            }
            if (j < k) d0 = fma(b[j * kApplyPts], y[j * kApplyPts], d0);
            const int32_t pk = piv[(int64_t)k * ldq + i];
            y[k * kApplyPts] = ldexp((double)v[(int64_t)(pk & 0xffff) * ldv + i], -(pk >> 16)) - (d0 + d1);
        } else {                                                   // U x = y, 1/U_kk stored
            double d0 = 0.0, d1 = 0.0;
            int j = k + 1;
            for (; j + 1 < N; j += 2) {
                d0 = fma(b[j * kApplyPts], y[j * kApplyPts], d0);
                d1 = fma(b[(j + 1) * kApplyPts], y[(j + 1) * kApplyPts], d1);
            }
            if (j < N) d0 = fma(b[j * kApplyPts], y[j * kApplyPts], d0);
            y[k * kApplyPts] = (y[k * kApplyPts] - (d0 + d1)) * b[k * kApplyPts];
        }
        if (s + 2 < S)
            issue(s + 2, b);                                       // (b's entries of step s are used)
        else
            cp_async_commit();                                     // an empty group keeps the count
    }
    for (int k = 0; k < N; ++k) z[(int64_t)k * ldz + i] = (TO)y[k * kApplyPts];
}

template <class TI, class TO>
cudaError_t apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq, const TI* v,
                  int64_t ldv, TO* z, int64_t ldz, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t bytes = (size_t)3 * N * kApplyPts * sizeof(double);
    auto kern = lu_apply_kernel<TI, TO>;
    cudaError_t e = ensure_smem((const void*)kern, bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((n + kApplyPts - 1) / kApplyPts), kApplyPts, bytes, s>>>(N, n, F, ldF, piv, ldq, v, ldv, z,
                                                                              ldz);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_precond_apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq,
                                 const double* v, int64_t ldv, double* z, int64_t ldz, cudaStream_t s) {
    return apply<double, double>(N, n, F, ldF, piv, ldq, v, ldv, z, ldz, s);
}

}  // namespace nk
