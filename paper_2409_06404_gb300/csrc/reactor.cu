// One implicit Euler step of the homogeneous constant-pressure reactor at every point, by
// Newton's method with a GMRES solve over all points together: the structure of the paper's
// implicit thermochemistry stage (Sec. 2), with the exact JVP of the sources (nk_rhs_jvp) in
// place of difference quotients, the Krylov basis kept in single precision and classical
// Gram-Schmidt: all projections of the new vector in one reduction, then its orthogonalised
// norm in a second one.  (The paper's single-reduction form takes that norm as
// sqrt(|w|^2 - |h|^2); with stiff chemistry w is dominated by its stiff modes and the
// difference keeps too few digits, which ended the Krylov cycles early in testing.)
//
// Unknowns x = (T, Y_k) per point, scaled by the error weights W_i = 1/(rtol |x0_i| + atol_i)
// so that the Krylov solve and the convergence tests work in the weighted RMS norm of a stiff
// ODE solver.  Newton: G(x) = x - x0 - dt f(x), (I - dt J) d = -G, solved for z = W d with
// A z = W (I - dt J) (z / W) by GMRES (one cycle of at most m iterations, stopping at a
// residual reduction lin_tol); x += d; converged by the update test of a stiff ODE solver
// (weighted RMS norm of d times min(1, contraction rate) below newton_tol).  A cycle that stops
// short still updates x, and the next Newton iteration restarts GMRES at the new residual.
//
// Optional left preconditioning by the per-point blocks P of I - dt W J W^-1 (block Jacobi,
// k_jac.cu and k_lu.cu), made once per step at x0 from a stored linearization (filled chunk by
// chunk) and the sources there, or kept from an earlier call (as a stiff ODE solver reuses its
// Newton matrix over steps): GMRES then solves P^-1 A z = P^-1 r and its stopping test
// measures P^-1 (r - A z), close to the error of the update.  (With stiff chemistry the
// unpreconditioned residual is dominated by its stiff components -- many orders of magnitude
// above the update -- so a test on it, as right preconditioning keeps, says little about the
// update's accuracy.)
//
// Products: recomputed from the state per direction (nk_rhs_jvp), or from a linearization
// stored once per Newton iteration (nk_rhs_jvp_linearized), or from that linearization
// rounded to float with single-precision arithmetic (linearized = 2): the basis is FP32, so
// products rounded at that level change the Krylov solve about as much as the basis itself
// does, while the residual -- and with it the converged state -- stays double.
//
// Vectors of the workspace hold (K+1) rows of n doubles (row 0 = T, rows 1..K = Y_k); the
// basis m+1 rows of (K+1) n floats.  Reductions go through per-block partial sums added in a
// fixed order (deterministic).  The host keeps the (m+1) x m Hessenberg matrix and the Givens
// rotations; each GMRES iteration reads j+2 and then 1 double back from the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kElemBlk = 256;
constexpr int kRedBlk = 256;
constexpr int kRedPerSM = 4;                 // resident reduction blocks per SM (the grid's size)
constexpr int kMaxDots = NK_REACTOR_MAX_KRYLOV + 2;

// row (0 = T, k + 1 = Y_k) and point of entry e of a (K+1)-row vector of n points
__device__ __forceinline__ int64_t row_of(int64_t e, int64_t n, int64_t& i) {
    const int64_t r = e / n;
    i = e - r * n;
    return r;
}

// x0, the weights W = 1/(rtol |x0| + atol) and their reciprocals iW = rtol |x0| + atol
__global__ void init_kernel(int64_t n, int64_t N, int64_t ld, const double* __restrict__ T,
                            const double* __restrict__ Y, double rtol, double atolT, double atolY,
                            double* __restrict__ x0, double* __restrict__ W, double* __restrict__ iW) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        const int64_t r = row_of(e, n, i);
        const double v = r == 0 ? T[i] : Y[(r - 1) * ld + i];
        const double d = rtol * fabs(v) + (r == 0 ? atolT : atolY);
        x0[e] = v;
        W[e] = 1.0 / d;
        iW[e] = d;
    }
}

// r = -W (x - x0 - dt f), and per-block partial sums of r^2
__global__ void __launch_bounds__(kRedBlk) residual_kernel(int64_t n, int64_t N, int64_t ld,
                                                           const double* __restrict__ T,
                                                           const double* __restrict__ Y,
                                                           const double* __restrict__ x0,
                                                           const double* __restrict__ f,
                                                           const double* __restrict__ W, double dt,
                                                           double* __restrict__ r, double* __restrict__ part) {
    __shared__ double red[kRedBlk / 32];
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i;
        const int64_t row = row_of(e, n, i);
        const double x = row == 0 ? T[i] : Y[(row - 1) * ld + i];
        const double v = -W[e] * (x - x0[e] - dt * f[e]);
        r[e] = v;
        acc = fma(v, v, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kRedBlk / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// v0 = (float)(r / beta)
__global__ void start_kernel(int64_t N, const double* __restrict__ r, double inv_beta, float* __restrict__ v0) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        v0[e] = (float)(r[e] * inv_beta);
}

// u = v / W (the unweighted direction)
__global__ void unscale_kernel(int64_t N, const float* __restrict__ v, const double* __restrict__ iW,
                               double* __restrict__ u) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        u[e] = widen(v[e]) * iW[e];
}

// w = A v_j = v_j - dt W (J u), u = v_j / W
__global__ void form_kernel(int64_t N, const float* __restrict__ vj, const double* __restrict__ Ju,
                            const double* __restrict__ W, double dt, double* __restrict__ w) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        w[e] = fma(-dt * W[e], Ju[e], widen(vj[e]));
}

// Dots <v_q, w> for q in [q0, q0 + nq) (nq <= NVC): per-block partial sums into part[b][q].
// FORM: this launch first forms w = A v_j = v_j - dt W (J u) (u = v_j / W); else w is read.
// NORM: also the partial sums of |w|^2, into part[b][nv] (nv = j + 1 basis vectors in all).
// The dots of a GMRES iteration take ceil(nv / 8) launches of at most 8 vectors each, which
// keeps the accumulators few and the SMs full (predicated-off double FMAs would still take the
// FP64 pipe, so the loop bound is NVC, nq rounded up to 4 or 8).  (Double-float products on
// the FP32 pipe measured no faster here: the kernel is not bound by the FP64 pipe alone.)
template <bool FORM, bool NORM, int NVC>
__global__ void __launch_bounds__(kRedBlk, kRedPerSM) apply_dots_kernel(int64_t N, const float* __restrict__ V,
                                                                        int64_t vstride, int q0, int nq, int nv,
                                                                        const double* __restrict__ Ju,
                                                                        const double* __restrict__ W, double dt,
                                                                        double* __restrict__ w,
                                                                        double* __restrict__ part) {
    __shared__ double red[kRedBlk / 32][NVC + 1];
    double acc[NVC + 1];
#pragma unroll
    for (int q = 0; q <= NVC; ++q) acc[q] = 0.0;
    const float* Vq = V + (int64_t)q0 * vstride;
    const float* vj = V + (int64_t)(nv - 1) * vstride;         // the vector the operator was applied to
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        double we;
        if constexpr (FORM) {
            we = fma(-dt * W[e], Ju[e], widen(vj[e]));
            w[e] = we;
        } else {
            we = w[e];
        }
        if constexpr (NORM) acc[NVC] = fma(we, we, acc[NVC]);
#pragma unroll
        for (int q = 0; q < NVC; ++q)
            if (q < nq) acc[q] = fma(widen(Vq[(int64_t)q * vstride + e]), we, acc[q]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q <= NVC; ++q) {
        if (q < NVC ? q >= nq : !NORM) continue;
        double a = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[warp][q] = a;
    }
    __syncthreads();
    const int nout = nq + (NORM ? 1 : 0);
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
        const int src = t < nq ? t : NVC;
        double sum = 0.0;
        for (int w2 = 0; w2 < kRedBlk / 32; ++w2) sum += red[w2][src];
        part[(int64_t)blockIdx.x * kMaxDots + (t < nq ? q0 + t : nv)] = sum;
    }
}

template <bool FORM, bool NORM>
void dots_launch(int nq, unsigned grid, cudaStream_t s, int64_t N, const float* V, int64_t vstride, int q0, int nv,
                 const double* Ju, const double* W, double dt, double* w, double* part) {
    if (nq > 4)
        apply_dots_kernel<FORM, NORM, 8><<<grid, kRedBlk, 0, s>>>(N, V, vstride, q0, nq, nv, Ju, W, dt, w, part);
    else
        apply_dots_kernel<FORM, NORM, 4><<<grid, kRedBlk, 0, s>>>(N, V, vstride, q0, nq, nv, Ju, W, dt, w, part);
}

// every dot of iteration j (nv = j + 1 basis vectors) and |w|^2 with the first group;
// FORM: w = A v_j formed by the first launch, else w as given
template <bool FORM>
cudaError_t apply_dots(int nv, unsigned grid, cudaStream_t s, int64_t N, const float* V, int64_t vstride,
                       const double* Ju, const double* W, double dt, double* w, double* part) {
    for (int q0 = 0; q0 < nv; q0 += 8) {
        const int nq = std::min(8, nv - q0);
        if (q0 == 0)
            dots_launch<FORM, true>(nq, grid, s, N, V, vstride, q0, nv, Ju, W, dt, w, part);
        else
            dots_launch<false, false>(nq, grid, s, N, V, vstride, q0, nv, Ju, W, dt, w, part);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// out[q] = sum over blocks of part[b][q], blocks in order (q < nq)
__global__ void reduce_kernel(const double* __restrict__ part, int nblocks, int stride, int nq,
                              double* __restrict__ out) {
    const int q = threadIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * stride + q];
    out[q] = s;
}

// w -= sum_{q < nv} h_q v_q in place, and per-block partial sums of the result's |w|^2
__global__ void __launch_bounds__(kRedBlk) orth_kernel(int64_t N, const float* __restrict__ V, int64_t vstride, int nv,
                                                       const double* __restrict__ h, double* __restrict__ w,
                                                       double* __restrict__ part) {
    __shared__ double hs[kMaxDots];
    __shared__ double red[kRedBlk / 32];
    for (int q = threadIdx.x; q < nv; q += blockDim.x) hs[q] = h[q];
    __syncthreads();
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        double we = w[e];
        for (int q = 0; q < nv; ++q) we = fma(-hs[q], widen(V[(int64_t)q * vstride + e]), we);
        w[e] = we;
        acc = fma(we, we, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < kRedBlk / 32; ++q) s += red[q];
        part[blockIdx.x] = s;
    }
}

// v_next = (float)(w / hn)
__global__ void normalize_kernel(int64_t N, const double* __restrict__ w, double inv_hn, float* __restrict__ vnext) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        vnext[e] = (float)(w[e] * inv_hn);
}

// d = (sum_q y_q v_q) / W; x += d; per-block partial sums of (W d)^2
__global__ void __launch_bounds__(kRedBlk) update_kernel(int64_t n, int64_t N, int64_t ld, const float* __restrict__ V,
                                                         int64_t vstride, int nv, const double* __restrict__ y,
                                                         const double* __restrict__ iW, double* __restrict__ T,
                                                         double* __restrict__ Y, double* __restrict__ part) {
    __shared__ double ys[kMaxDots];
    __shared__ double red[kRedBlk / 32];
    for (int q = threadIdx.x; q < nv; q += blockDim.x) ys[q] = y[q];
    __syncthreads();
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        double z = 0.0;
        for (int q = 0; q < nv; ++q) z = fma(ys[q], widen(V[(int64_t)q * vstride + e]), z);
        int64_t i;
        const int64_t row = row_of(e, n, i);
        const double d = z * iW[e];
        if (row == 0)
            T[i] += d;
        else
            Y[(row - 1) * ld + i] += d;
        acc = fma(z, z, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kRedBlk / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------- workspace
struct Work {
    double *x0, *W, *iW, *f, *r, *u, *Ju, *w, *part, *dots;
    float* V;
    double* F;                // block factors (precond only)
    int32_t* piv;             // pivot rows and row exponents of the factors
    double* lin;              // stored linearization of one chunk of points (all points for
                              // double linearized products)
    float* linf;              // the linearization rounded to float (single-precision products)
    int64_t N, vstride, nchunk;
    int nred;
};

int reduction_blocks() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, sms * kRedPerSM);
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// points per chunk of the stored (double) linearization: all of them for double linearized
// products, else about 2 GB (whole warps) for the preconditioner's set-up
int64_t lin_chunk(const DevMech& mech, int64_t n, int linearized) {
    if (linearized == 1) return n;
    const int64_t per = lin_slots(mech) * (int64_t)sizeof(double);
    const int64_t c = std::max<int64_t>(128, ((int64_t(2) << 30) / per) / 128 * 128);
    return std::min(n, c);
}

size_t work_bytes(const DevMech& mech, int64_t n, int m, int nred, int precond, int linearized) {
    const int64_t N = (int64_t)(mech.K + 1) * n;
    size_t b = 8 * align256((size_t)N * sizeof(double)) + align256((size_t)(m + 1) * N * sizeof(float)) +
               align256((size_t)nred * kMaxDots * sizeof(double)) + align256(kMaxDots * sizeof(double));
    if (precond)
        b += align256((size_t)(mech.K + 1) * N * sizeof(double)) + align256((size_t)N * sizeof(int32_t));
    if (precond || linearized == 1)
        b += align256((size_t)lin_slots(mech) * lin_chunk(mech, n, linearized) * sizeof(double));
    if (linearized == 2) b += align256((size_t)lin_slots_f32(mech) * n * sizeof(float));
    return b;
}

Work carve(const DevMech& mech, void* ws, int64_t n, int m, int nred, int precond, int linearized) {
    const int64_t N = (int64_t)(mech.K + 1) * n;
    Work w;
    char* b = static_cast<char*>(ws);
    auto take = [&](size_t bytes) {
        char* q = b;
        b += align256(bytes);
        return q;
    };
    const size_t vb = (size_t)N * sizeof(double);
    w.x0 = reinterpret_cast<double*>(take(vb));
    w.W = reinterpret_cast<double*>(take(vb));
    w.iW = reinterpret_cast<double*>(take(vb));
    w.f = reinterpret_cast<double*>(take(vb));
    w.r = reinterpret_cast<double*>(take(vb));
    w.u = reinterpret_cast<double*>(take(vb));
    w.Ju = reinterpret_cast<double*>(take(vb));
    w.w = reinterpret_cast<double*>(take(vb));
    w.V = reinterpret_cast<float*>(take((size_t)(m + 1) * N * sizeof(float)));
    w.part = reinterpret_cast<double*>(take((size_t)nred * kMaxDots * sizeof(double)));
    w.dots = reinterpret_cast<double*>(take(kMaxDots * sizeof(double)));
    w.F = nullptr;
    w.piv = nullptr;
    w.lin = nullptr;
    w.linf = nullptr;
    w.nchunk = 0;
    if (precond) {
        w.F = reinterpret_cast<double*>(take((size_t)(mech.K + 1) * N * sizeof(double)));
        w.piv = reinterpret_cast<int32_t*>(take((size_t)N * sizeof(int32_t)));
    }
    if (precond || linearized == 1) {
        w.nchunk = lin_chunk(mech, n, linearized);
        w.lin = reinterpret_cast<double*>(take((size_t)lin_slots(mech) * w.nchunk * sizeof(double)));
    }
    if (linearized == 2) w.linf = reinterpret_cast<float*>(take((size_t)lin_slots_f32(mech) * n * sizeof(float)));
    w.N = N;
    w.vstride = N;
    w.nred = nred;
    return w;
}

}  // namespace

size_t reactor_workspace_bytes(const DevMech& m, int64_t n, int krylov_dim, int precond, int linearized) {
    // (the reduction-block count depends on the device's SM count)
    return work_bytes(m, n, krylov_dim, reduction_blocks(), precond, linearized);
}

// One implicit Euler step (contiguous state: Y rows of stride n).  Returns cudaSuccess and
// fills the statistics; a step that does not converge is reported there, not as an error.
cudaError_t reactor_step(const DevMech& m, int64_t n, double* T, const double* p, double* Y, double dt,
                         const nk_reactor_opts& o, nk_reactor_stats& st, void* ws, cudaStream_t s) {
    const int K = m.K;
    const int64_t ld = n;
    const int64_t N = (int64_t)(K + 1) * n;
    const int mk = o.krylov_dim;
    const int nred = reduction_blocks();
    Work w = carve(m, ws, n, mk, nred, o.precond, o.linearized);
    const int eg = (int)std::min<int64_t>((N + kElemBlk - 1) / kElemBlk, (int64_t)nred * 8);
    cudaError_t e;
    std::vector<double> hbuf(kMaxDots);
    // sum of the per-block partials (stride values apart, nq of them) to the host
    auto fetch = [&](int stride, int nq, double* dev_out, double* host) -> cudaError_t {
        reduce_kernel<<<1, 64, 0, s>>>(w.part, nred, stride, nq, dev_out);
        cudaError_t r = cudaMemcpyAsync(host, dev_out, nq * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (r != cudaSuccess) return r;
        return cudaStreamSynchronize(s);
    };
    std::memset(&st, 0, sizeof st);
    init_kernel<<<eg, kElemBlk, 0, s>>>(n, N, ld, T, Y, o.rtol, o.atol_T, o.atol_Y, w.x0, w.W, w.iW);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double sqrtN = std::sqrt((double)N);
    std::vector<double> H((size_t)(mk + 1) * mk), cs(mk), sn(mk), g(mk + 1), yv(mk);
    double crate = 1.0;                              // estimated Newton contraction rate
    for (int it = 0; it < o.max_newton; ++it) {
        // residual r = -W (x - x0 - dt f(x)) of the implicit Euler system (f as rows of w.f)
        if ((e = launch_rates(m, n, ld, T, p, Y, nullptr, w.f + n, w.f, NK_FP64, s, 1)) != cudaSuccess) return e;
        residual_kernel<<<nred, kRedBlk, 0, s>>>(n, N, ld, T, Y, w.x0, w.f, w.W, dt, w.r, w.part);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = fetch(1, 1, w.dots, hbuf.data())) != cudaSuccess) return e;
        const double beta = std::sqrt(hbuf[0]);
        st.residual_wrms = beta / sqrtN;
        if (!(beta > 0.0)) {                       // exact solution (or a non-finite residual)
            st.converged = beta == 0.0;
            return cudaSuccess;
        }
        if (o.linearized == 1 &&                   // the rates' tangent data at this iterate
            (e = launch_linearize(m, n, ld, T, p, Y, nullptr, w.lin, n, s)) != cudaSuccess)
            return e;
        if (o.linearized == 2 &&                   // the same, rounded to float
            (e = launch_linearize_f32(m, n, ld, T, p, Y, nullptr, w.linf, n, s)) != cudaSuccess)
            return e;
        if (o.precond == 1 && it == 0) {           // blocks of I - dt W J W^-1 at x0, factored
            for (int64_t c0 = 0; c0 < n; c0 += w.nchunk) {
                const int64_t nc = std::min(w.nchunk, n - c0);
                const bool full = o.linearized == 1;    // the full double data: stride n
                if (!full &&
                    (e = launch_linearize(m, nc, ld, T + c0, p + c0, Y + c0, nullptr, w.lin, nc, s)) != cudaSuccess)
                    return e;
                const double* lc = full ? w.lin + c0 : w.lin;
                if ((e = launch_precond_setup(m, nc, ld, T + c0, p + c0, Y + c0, lc, full ? n : nc, w.f + c0,
                                              w.f + n + c0, n, w.W + c0, n, dt, w.F + c0, w.piv + c0, n, s)) !=
                    cudaSuccess)
                    return e;
            }
        }
        // GMRES: A z = r with A z = z - dt W J (z / W) (preconditioned: P^-1 A z = P^-1 r); one
        // cycle of at most m iterations
        double beta_lin = beta;                    // norm of the (preconditioned) initial residual
        if (o.precond) {
            if ((e = launch_precond_apply(K + 1, n, w.F, n, w.piv, n, w.r, n, w.r, n, s)) != cudaSuccess) return e;
            orth_kernel<<<nred, kRedBlk, 0, s>>>(N, w.V, w.vstride, 0, w.dots, w.r, w.part);   // |P^-1 r|^2
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = fetch(1, 1, w.dots + kMaxDots - 1, hbuf.data())) != cudaSuccess) return e;
            beta_lin = std::sqrt(hbuf[0]);
            if (!(beta_lin > 0.0)) {               // the preconditioned residual vanished
                st.converged = beta_lin == 0.0;
                return cudaSuccess;
            }
        }
        start_kernel<<<eg, kElemBlk, 0, s>>>(N, w.r, 1.0 / beta_lin, w.V);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta_lin;
        int j = 0;
        while (j < mk) {
            const float* vj = w.V + (int64_t)j * w.vstride;
            unscale_kernel<<<eg, kElemBlk, 0, s>>>(N, vj, w.iW, w.u);
            if (o.linearized == 1)
                e = launch_rhs_jvp_linearized(m, n, ld, T, p, Y, w.lin, n, w.f, w.f + n, n, w.u, w.u + n, w.Ju,
                                              w.Ju + n, s);
            else if (o.linearized == 2)
                e = launch_jvp_linearized_f32(m, n, ld, T, p, Y, w.linf, n, w.f, w.f + n, n, w.u, w.u + n, w.Ju,
                                              w.Ju + n, s, 1);
            else
                e = launch_jvp(m, n, ld, T, p, Y, nullptr, w.u, w.u + n, nullptr, nullptr, w.Ju + n, w.Ju, s, 1);
            if (e != cudaSuccess) return e;
            if (o.precond) {                          // w = P^-1 A v_j
                form_kernel<<<eg, kElemBlk, 0, s>>>(N, vj, w.Ju, w.W, dt, w.w);
                if ((e = launch_precond_apply(K + 1, n, w.F, n, w.piv, n, w.w, n, w.w, n, s)) != cudaSuccess)
                    return e;
                e = apply_dots<false>(j + 1, nred, s, N, w.V, w.vstride, w.Ju, w.W, dt, w.w, w.part);
            } else {
                e = apply_dots<true>(j + 1, nred, s, N, w.V, w.vstride, w.Ju, w.W, dt, w.w, w.part);
            }
            if (e != cudaSuccess) return e;
            if ((e = fetch(kMaxDots, j + 2, w.dots, hbuf.data())) != cudaSuccess) return e;
            ++st.krylov_iters;
            // column j of the Hessenberg matrix: the projections, then the norm of the
            // orthogonalised vector from a second reduction (with a stiff operator w = A v is
            // dominated by its stiff modes and |w|^2 - |h|^2 would keep too few digits)
            double hh = 0.0;
            for (int q = 0; q <= j; ++q) {
                H[(size_t)q * mk + j] = hbuf[q];
                hh += hbuf[q] * hbuf[q];
            }
            orth_kernel<<<nred, kRedBlk, 0, s>>>(N, w.V, w.vstride, j + 1, w.dots, w.w, w.part);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = fetch(1, 1, w.dots + kMaxDots - 1, hbuf.data() + kMaxDots - 1)) != cudaSuccess) return e;
            const double hn = std::sqrt(hbuf[kMaxDots - 1]);
            const bool lost = !(hn > 1e-14 * std::sqrt(hh + hn * hn));   // breakdown: w in the basis
            H[(size_t)(j + 1) * mk + j] = lost ? 0.0 : hn;
            if (!lost && j + 1 < mk) {
                normalize_kernel<<<eg, kElemBlk, 0, s>>>(N, w.w, 1.0 / hn, w.V + (int64_t)(j + 1) * w.vstride);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            for (int q = 0; q < j; ++q) {             // earlier Givens rotations
                const double a = H[(size_t)q * mk + j], b = H[(size_t)(q + 1) * mk + j];
                H[(size_t)q * mk + j] = cs[q] * a + sn[q] * b;
                H[(size_t)(q + 1) * mk + j] = -sn[q] * a + cs[q] * b;
            }
            const double a = H[(size_t)j * mk + j], b = H[(size_t)(j + 1) * mk + j];
            const double rr = std::hypot(a, b);
            cs[j] = rr > 0.0 ? a / rr : 1.0;
            sn[j] = rr > 0.0 ? b / rr : 0.0;
            H[(size_t)j * mk + j] = rr;
            H[(size_t)(j + 1) * mk + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++j;
            if (std::fabs(g[j]) <= o.lin_tol * beta_lin) break;   // relative to this iteration's residual
            if (lost) break;
        }
        // y = R^{-1} g (j columns), then x += (V y) / W
        for (int q = j - 1; q >= 0; --q) {
            double acc = g[q];
            for (int c = q + 1; c < j; ++c) acc -= H[(size_t)q * mk + c] * yv[c];
            yv[q] = H[(size_t)q * mk + q] != 0.0 ? acc / H[(size_t)q * mk + q] : 0.0;
        }
        if ((e = cudaMemcpyAsync(w.dots, yv.data(), j * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return e;
        update_kernel<<<nred, kRedBlk, 0, s>>>(n, N, ld, w.V, w.vstride, j, w.dots, w.iW, T, Y, w.part);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = fetch(1, 1, w.dots + kMaxDots - 1, hbuf.data())) != cudaSuccess) return e;
        ++st.newton_iters;
        const double del = std::sqrt(hbuf[0]) / sqrtN;
        // convergence test of a stiff ODE solver on the updates (the residual of a stiff
        // system is dominated by rounding long before the iterate stops moving): converged when
        // del * min(1, rate) <= newton_tol with rate the contraction of successive updates;
        // diverging when an update more than doubles
        if (it > 0) crate = std::max(0.3 * crate, del / st.update_wrms);
        const bool diverging = it > 0 && del > 2.0 * st.update_wrms;
        st.update_wrms = del;
        if (del * std::min(1.0, crate) <= o.newton_tol) {
            st.converged = 1;
            return cudaSuccess;
        }
        if (diverging) return cudaSuccess;
    }
    return cudaSuccess;
}

}  // namespace nk
