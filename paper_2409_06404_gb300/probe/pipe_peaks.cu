// Throughput of the arithmetic pipes that bound the library's kernels: the denominators of their
// per-pipe rooflines.  Each thread runs CH independent streams of one operation (double or float
// fused multiply-add, multiply or add), every SM filled with resident blocks, timed with CUDA
// events on the launching stream.  Built as its own library (libnkprobe.so) for the benchmark; it
// is not part of the nkchem interface.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;

template <class T>
__device__ __forceinline__ T op(int kind, T a, T b, T c);

template <>
__device__ __forceinline__ double op<double>(int kind, double a, double b, double c) {
    return kind == 0 ? fma(a, b, c) : (kind == 1 ? a * b : a + c);
}
template <>
__device__ __forceinline__ float op<float>(int kind, float a, float b, float c) {
    return kind == 0 ? fmaf(a, b, c) : (kind == 1 ? a * b : a + c);
}

// KIND 0: multiply-add, 1: multiply, 2: add; CH independent streams per thread
template <class T, int KIND, int CH>
__global__ void __launch_bounds__(kThreads) stream_kernel(int iters, T b, T c, T* sink) {
    T a[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) a[j] = (T)(threadIdx.x + 1) * (T)(j + 1) * c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < CH; ++j) a[j] = op<T>(KIND, a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) s += a[j];
    if (s == (T)-1) sink[threadIdx.x] = s;     // keeps the streams live; never true for these inputs
}

template <class T, int KIND, int CH>
int run(int blocks_per_sm, int iters, int reps, double* ops_per_s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    T* sink = nullptr;
    if (cudaMalloc(&sink, kThreads * sizeof(T)) != cudaSuccess) return 2;
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    const T b = (T)0.9999999, c = (T)1e-7;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    stream_kernel<T, KIND, CH><<<grid, kThreads>>>(iters, b, c, sink);     // warm-up
    float best = 0.0f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        stream_kernel<T, KIND, CH><<<grid, kThreads>>>(iters, b, c, sink);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess || best <= 0.0f) return 3;
    *ops_per_s = (double)grid * kThreads * CH * (double)iters / (best * 1e-3);
    return 0;
}

}  // namespace

extern "C" {

// Thread-level operations per second of one pipe on the current device, the best of `reps`
// timed launches of sms x blocks_per_sm blocks of 256 threads (after one untimed launch).
//   kind 0: double multiply-add (FP64 pipe), 1: double multiply, 2: double add,
//        3: float multiply-add (FMA pipes), 4: float multiply, 5: float add
// Returns 0 on success, nonzero on a CUDA error or a bad kind.
int nkp_pipe_rate(int kind, int blocks_per_sm, int iters, int reps, double* ops_per_s) {
    if (!ops_per_s || blocks_per_sm < 1 || iters < 1 || reps < 1) return 4;
    switch (kind) {
        case 0: return run<double, 0, 8>(blocks_per_sm, iters, reps, ops_per_s);
        case 1: return run<double, 1, 8>(blocks_per_sm, iters, reps, ops_per_s);
        case 2: return run<double, 2, 8>(blocks_per_sm, iters, reps, ops_per_s);
        case 3: return run<float, 0, 16>(blocks_per_sm, iters, reps, ops_per_s);
        case 4: return run<float, 1, 16>(blocks_per_sm, iters, reps, ops_per_s);
        case 5: return run<float, 2, 16>(blocks_per_sm, iters, reps, ops_per_s);
        default: return 4;
    }
}

}  // extern "C"
