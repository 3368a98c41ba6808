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
// substitution with the vector in shared memory and the factors read once, in order (coalesced
// across the warp's points).
#include <algorithm>
#include <cstdint>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kApplyBlk = 128;

// sum_{j0 <= j < j1} f[j ldF] y[j]: four independent partial sums, so that four factor loads
// per thread are in flight (the loads, not the arithmetic, bound the substitutions; eight
// measured slower)
__device__ __forceinline__ double dot_run(const double* __restrict__ f, int64_t ldF, const double* y, int j0, int j1) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int j = j0;
    for (; j + 3 < j1; j += 4) {
        const double f0 = f[(int64_t)j * ldF], f1 = f[(int64_t)(j + 1) * ldF], f2 = f[(int64_t)(j + 2) * ldF],
                     f3 = f[(int64_t)(j + 3) * ldF];
        s0 = fma(f0, y[j * kApplyBlk], s0);
        s1 = fma(f1, y[(j + 1) * kApplyBlk], s1);
        s2 = fma(f2, y[(j + 2) * kApplyBlk], s2);
        s3 = fma(f3, y[(j + 3) * kApplyBlk], s3);
    }
    for (; j < j1; ++j) s0 = fma(f[(int64_t)j * ldF], y[j * kApplyBlk], s0);
    return (s0 + s1) + (s2 + s3);
}

// z = P^-1 v per point: v and z rows of ldv / ldz (row r of point i at r ld + i), of type TI and
// TO, arithmetic in double.  z may alias v: every thread reads its point's entries of v before
// it writes z.
template <class TI, class TO>
__global__ void __launch_bounds__(kApplyBlk) lu_apply_kernel(const int N, const int64_t n, const double* __restrict__ F,
                                                             const int64_t ldF, const int32_t* __restrict__ piv,
                                                             const int64_t ldq, const TI* v, const int64_t ldv, TO* z,
                                                             const int64_t ldz) {
    extern __shared__ double sy[];
    const int64_t i = (int64_t)blockIdx.x * kApplyBlk + threadIdx.x;
    if (i >= n) return;
    double* y = sy + threadIdx.x;
    const double* f = F + i;
    for (int k = 0; k < N; ++k) {                              // L y = (D v)(perm), unit diagonal
        const int32_t pk = piv[(int64_t)k * ldq + i];
        const double* fk = f + (int64_t)k * N * ldF;
        y[k * kApplyBlk] = ldexp((double)v[(int64_t)(pk & 0xffff) * ldv + i], -(pk >> 16)) -
                           dot_run(fk, ldF, y, 0, k);
    }
    for (int k = N - 1; k >= 0; --k) {                         // U x = y, 1/U_kk stored
        const double* fk = f + (int64_t)k * N * ldF;
        y[k * kApplyBlk] = (y[k * kApplyBlk] - dot_run(fk, ldF, y, k + 1, N)) * fk[(int64_t)k * ldF];
    }
    for (int k = 0; k < N; ++k) z[(int64_t)k * ldz + i] = (TO)y[k * kApplyBlk];
}

template <class TI, class TO>
cudaError_t apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq, const TI* v,
                  int64_t ldv, TO* z, int64_t ldz, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t bytes = (size_t)N * kApplyBlk * sizeof(double);
    auto kern = lu_apply_kernel<TI, TO>;
    cudaError_t e = ensure_smem((const void*)kern, bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((n + kApplyBlk - 1) / kApplyBlk), kApplyBlk, bytes, s>>>(N, n, F, ldF, piv, ldq, v, ldv, z, ldz);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_precond_apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq,
                                 const double* v, int64_t ldv, double* z, int64_t ldz, cudaStream_t s) {
    return apply<double, double>(N, n, F, ldF, piv, ldq, v, ldv, z, ldz, s);
}

}  // namespace nk
