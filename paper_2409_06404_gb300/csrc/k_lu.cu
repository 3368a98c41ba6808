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
// is then L U z = (D v) in pivot order.  Four threads per point, forward then backward
// substitution with the vector in shared memory and the factors read once, in order (each warp
// reads eight points' consecutive entries: whole 32-byte sectors).
#include <algorithm>
#include <cstdint>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kApplyBlk = 128;

// TPP threads per point (adjacent lanes): thread t sums the terms j = j0 + t, j0 + t + TPP, ...
// of sum_{j0 <= j < j1} f[j ldF] y[j] in two independent partial sums, and the point's threads
// combine theirs by shuffles, so each gets the whole dot product.  Splitting a point over
// threads divides its vector's shared memory among them (more resident warps) and multiplies
// the factor loads in flight per point.  y: the point's vector at y[j * PPB].
template <int TPP, int PPB>
__device__ __forceinline__ double dot_run(const double* __restrict__ f, int64_t ldF, const double* y, int j0, int j1,
                                          int t) {
    double s0 = 0.0, s1 = 0.0;
    int j = j0 + t;
    for (; j + TPP < j1; j += 2 * TPP) {
        const double f0 = f[(int64_t)j * ldF], f1 = f[(int64_t)(j + TPP) * ldF];
        s0 = fma(f0, y[j * PPB], s0);
        s1 = fma(f1, y[(j + TPP) * PPB], s1);
    }
    if (j < j1) s0 = fma(f[(int64_t)j * ldF], y[j * PPB], s0);
    double sum = s0 + s1;
#pragma unroll
    for (int o = 1; o < TPP; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    return sum;
}

// z = P^-1 v per point: v and z rows of ldv / ldz (row r of point i at r ld + i), of type TI and
// TO, arithmetic in double.  z may alias v: every point's threads read its entries of v before
// they write z (the row of y each thread reads at step k was written by the point's thread 0
// before the shuffles of step k, which order it).  Threads past the last point shadow point
// n - 1 without writing (the shuffles need the whole warp).
template <class TI, class TO, int TPP>
__global__ void __launch_bounds__(kApplyBlk) lu_apply_kernel(const int N, const int64_t n, const double* __restrict__ F,
                                                             const int64_t ldF, const int32_t* __restrict__ piv,
                                                             const int64_t ldq, const TI* v, const int64_t ldv, TO* z,
                                                             const int64_t ldz) {
    constexpr int PPB = kApplyBlk / TPP;                       // points per block
    extern __shared__ double sy[];
    const int pt = threadIdx.x / TPP, t = threadIdx.x % TPP;
    const int64_t i0 = (int64_t)blockIdx.x * PPB + pt;
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;
    double* y = sy + pt;
    const double* f = F + i;
    for (int k = 0; k < N; ++k) {                              // L y = (D v)(perm), unit diagonal
        const double* fk = f + (int64_t)k * N * ldF;
        const double d = dot_run<TPP, PPB>(fk, ldF, y, 0, k, t);
        if (t == 0) {
            const int32_t pk = piv[(int64_t)k * ldq + i];
            y[k * PPB] = ldexp((double)v[(int64_t)(pk & 0xffff) * ldv + i], -(pk >> 16)) - d;
        }
        __syncwarp();
    }
    for (int k = N - 1; k >= 0; --k) {                         // U x = y, 1/U_kk stored
        const double* fk = f + (int64_t)k * N * ldF;
        const double d = dot_run<TPP, PPB>(fk, ldF, y, k + 1, N, t);
        if (t == 0) y[k * PPB] = (y[k * PPB] - d) * fk[(int64_t)k * ldF];
        __syncwarp();
    }
    if (live)
        for (int k = t; k < N; k += TPP) z[(int64_t)k * ldz + i] = (TO)y[k * PPB];
}

template <class TI, class TO>
cudaError_t apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq, const TI* v,
                  int64_t ldv, TO* z, int64_t ldz, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    constexpr int TPP = 4, PPB = kApplyBlk / TPP;
    const size_t bytes = (size_t)N * PPB * sizeof(double);
    auto kern = lu_apply_kernel<TI, TO, TPP>;
    cudaError_t e = ensure_smem((const void*)kern, bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((n + PPB - 1) / PPB), kApplyBlk, bytes, s>>>(N, n, F, ldF, piv, ldq, v, ldv, z, ldz);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_precond_apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq,
                                 const double* v, int64_t ldv, double* z, int64_t ldz, cudaStream_t s) {
    return apply<double, double>(N, n, F, ldF, piv, ldq, v, ldv, z, ldz, s);
}

}  // namespace nk
