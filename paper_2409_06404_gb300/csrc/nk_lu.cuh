// LU factorization with partial pivoting of one N x N block in shared memory by one warp, the
// step shared by the block-Jacobi kernels (k_lu.cu, k_jac.cu).
//
// The block a has row stride S; lane l owns rows l, l + 32, ...  At step k the warp picks the
// largest |a_rk| among rows not yet used (lowest row on ties, NaN counted as +inf so that the
// order is total; lane 0's choice is broadcast), each lane scales and updates its unused rows
// against the pivot row (read as a broadcast).  Rows stay in place: perm[k] receives the k-th
// pivot row, whose entries then hold L_k,0..k-1 (unit lower part) and U_k,k.. with 1/U_kk in
// place of U_kk.  A zero pivot (a singular block) is replaced by 1: the factors stay finite and
// GMRES, which only uses them as a preconditioner, still converges, more slowly.
#pragma once
#include "nk_internal.cuh"

namespace nk {

constexpr int kMaxRowsPerLane = (kMaxPrecondN + 31) / 32;

__device__ __forceinline__ void warp_lu(double* a, const int N, const int S, const int lane, int32_t* perm) {
    uint32_t used = 0;                                         // bit b: row lane + 32 b is a pivot row
    for (int k = 0; k < N; ++k) {
        double bv = -1.0;
        int best = N;
#pragma unroll
        for (int b = 0; b < kMaxRowsPerLane; ++b) {
            const int r = lane + 32 * b;
            if (r < N && !((used >> b) & 1u)) {
                double v = fabs(a[r * S + k]);
                if (v != v) v = __longlong_as_double(0x7ff0000000000000LL);   // NaN as +inf
                if (best == N || v > bv) {
                    bv = v;
                    best = r;
                }
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
        // lane 0 holds a valid row (some row is unused while k < N, and a lane holding one never
        // gives it up for none); its choice, broadcast, is the warp's
        const int pr = __shfl_sync(0xffffffffu, best, 0);
        if ((pr & 31) == lane) used |= 1u << (pr >> 5);
        double pv = a[pr * S + k];
        if (pv == 0.0) pv = 1.0;
        const double inv = 1.0 / pv;
        const double* ap = a + pr * S;
#pragma unroll
        for (int b = 0; b < kMaxRowsPerLane; ++b) {
            const int r = lane + 32 * b;
            if (r < N && !((used >> b) & 1u)) {
                double* ar = a + r * S;
                const double l = ar[k] * inv;
                ar[k] = l;
#pragma unroll 4
                for (int j = k + 1; j < N; ++j) ar[j] = fma(-l, ap[j], ar[j]);
            }
        }
        __syncwarp();
        if (lane == 0) {
            a[pr * S + k] = inv;
            perm[k] = pr;
        }
        __syncwarp();
    }
}

}  // namespace nk
