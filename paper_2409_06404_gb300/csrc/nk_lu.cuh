// LU factorization with partial pivoting of one N x N block in shared memory by one warp, the
// step shared by the block-Jacobi kernels (k_lu.cu, k_jac.cu).
//
// The block a has row stride S.  At step k the warp picks the largest |a_rk| over the rows
// r >= k not yet eliminated (lowest position on ties, NaN counted as +inf so that the order is
// total; lane 0's choice is broadcast), swaps that row into position k, and the lanes update
// rows k + 1 + lane, k + 33 + lane, ... against it (the pivot row read as a broadcast), so the
// remaining rows stay contiguous and every lane has work while 32 or more are left.  On return
// row k holds L_k,0..k-1 (unit lower part) and U_k,k.. of the k-th pivot row with 1/U_kk in
// place of U_kk, and perm[k] the original index of that row.  A zero pivot (a singular block)
// is replaced by 1: the factors stay finite and GMRES, which only uses them as a
// preconditioner, still converges, more slowly.
#pragma once
#include "nk_internal.cuh"

namespace nk {

__device__ __forceinline__ void warp_lu(double* a, const int N, const int S, const int lane, int32_t* perm) {
    for (int r = lane; r < N; r += 32) perm[r] = r;
    __syncwarp();
    for (int k = 0; k < N; ++k) {
        double bv = -1.0;
        int best = N;
        for (int r = k + lane; r < N; r += 32) {
            double v = fabs(a[r * S + k]);
            if (v != v) v = __longlong_as_double(0x7ff0000000000000LL);   // NaN as +inf
            if (best == N || v > bv) {
                bv = v;
                best = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int ob = __shfl_xor_sync(0xffffffffu, best, o);
            if (ob < N && (best == N || ov > bv || (ov == bv && ob < best))) {
                bv = ov;
                best = ob;
            }
        }
        // lane 0 holds a valid row (rows k..N-1 remain, and a lane holding one never gives it
        // up for none); its choice, broadcast, is the warp's
        const int pr = __shfl_sync(0xffffffffu, best, 0);
        if (pr != k) {
            for (int j = lane; j < N; j += 32) {
                const double t = a[k * S + j];
                a[k * S + j] = a[pr * S + j];
                a[pr * S + j] = t;
            }
            if (lane == 0) {
                const int32_t t = perm[k];
                perm[k] = perm[pr];
                perm[pr] = t;
            }
            __syncwarp();
        }
        double pv = a[k * S + k];
        if (pv == 0.0) pv = 1.0;
        const double inv = 1.0 / pv;
        const double* ap = a + k * S;
        for (int r = k + 1 + lane; r < N; r += 32) {
            double* ar = a + r * S;
            const double l = ar[k] * inv;
            ar[k] = l;
#pragma unroll 4
            for (int j = k + 1; j < N; ++j) ar[j] = fma(-l, ap[j], ar[j]);
        }
        __syncwarp();
        if (lane == 0) a[k * S + k] = inv;
        __syncwarp();
    }
}

}  // namespace nk
