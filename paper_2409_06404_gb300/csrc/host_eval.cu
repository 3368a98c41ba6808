// Rates and transport of host-resident fields, pipelined: the points are cut into chunks that
// cycle over kStreams streams, each with its own device buffers, so that the host-to-device
// copy of one chunk, the kernels of another and the device-to-host copy of a third run at the
// same time (one copy engine per direction, the SMs for the kernels).  The species rows of a
// chunk are one strided 2-D copy per direction.  With page-locked host memory the copies are
// asynchronous; pageable memory still works, with the driver's staging.
#include <algorithm>

#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kStreams = 3;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// device buffers of one stream: T, p, Y (K rows), omega (K rows), hrr, mu, lambda, Dmix (K rows)
size_t slot_bytes(int K, int64_t chunk) {
    const size_t v = (size_t)chunk * sizeof(double);
    return 5 * align256(v) + 3 * align256((size_t)K * v);
}

struct Slot {
    double *T, *p, *Y, *w, *hrr, *mu, *lam, *D;
};

Slot carve(void* base, int K, int64_t chunk) {
    char* b = static_cast<char*>(base);
    const size_t v = (size_t)chunk * sizeof(double);
    auto take = [&](size_t bytes) {
        char* q = b;
        b += align256(bytes);
        return reinterpret_cast<double*>(q);
    };
    Slot s;
    s.T = take(v);
    s.p = take(v);
    s.Y = take((size_t)K * v);
    s.w = take((size_t)K * v);
    s.hrr = take(v);
    s.mu = take(v);
    s.lam = take(v);
    s.D = take((size_t)K * v);
    return s;
}

}  // namespace

size_t host_eval_workspace_bytes(const DevMech& m, int64_t chunk) { return kStreams * slot_bytes(m.K, chunk); }

cudaError_t host_eval(const DevMech& m, int64_t n, const double* T, const double* p, const double* Y, double* omega,
                      double* hrr, double* mu, double* lam, double* Dmix, int precision, int64_t chunk, void* ws,
                      cudaStream_t caller) {
    const int K = m.K;
    const size_t row = (size_t)n * sizeof(double);
    cudaStream_t st[kStreams] = {};
    cudaEvent_t start = nullptr, done[kStreams] = {};
    cudaError_t e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    for (int q = 0; q < kStreams && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&st[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[q], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventRecord(start, caller);   // after the caller's earlier work
    for (int q = 0; q < kStreams && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(st[q], start, 0);
    const bool rates = omega || hrr, transport = mu || lam || Dmix;
    int64_t c = 0;
    for (int64_t c0 = 0; c0 < n && e == cudaSuccess; c0 += chunk, ++c) {
        const int64_t nc = std::min(chunk, n - c0);
        const int q = (int)(c % kStreams);
        const cudaStream_t s = st[q];
        Slot b = carve(static_cast<char*>(ws) + q * slot_bytes(K, chunk), K, chunk);
        const size_t w = (size_t)nc * sizeof(double), pitch = (size_t)chunk * sizeof(double);
        e = cudaMemcpyAsync(b.T, T + c0, w, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.p, p + c0, w, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpy2DAsync(b.Y, pitch, Y + c0, row, w, K, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && rates)
            e = launch_rates(m, nc, chunk, b.T, b.p, b.Y, nullptr, b.w, b.hrr, precision, s);
        if (e == cudaSuccess && transport)
            e = precision == NK_FP64 ? launch_transport_df(m, nc, chunk, b.T, b.p, b.Y, b.mu, b.lam, b.D, s)
                                     : launch_transport(m, nc, chunk, b.T, b.p, b.Y, b.mu, b.lam, b.D, precision, s);
        if (e == cudaSuccess && omega) e = cudaMemcpy2DAsync(omega + c0, row, b.w, pitch, w, K, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && hrr) e = cudaMemcpyAsync(hrr + c0, b.hrr, w, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && mu) e = cudaMemcpyAsync(mu + c0, b.mu, w, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && lam) e = cudaMemcpyAsync(lam + c0, b.lam, w, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && Dmix) e = cudaMemcpy2DAsync(Dmix + c0, row, b.D, pitch, w, K, cudaMemcpyDeviceToHost, s);
    }
    // the caller's stream continues after every chunk; the call returns with the outputs on
    // the host
    for (int q = 0; q < kStreams; ++q) {
        if (st[q] && done[q]) {
            const cudaError_t r = cudaEventRecord(done[q], st[q]);
            if (r == cudaSuccess) cudaStreamWaitEvent(caller, done[q], 0);
            if (e == cudaSuccess) e = r;
        }
    }
    for (int q = 0; q < kStreams; ++q) {
        if (st[q]) {
            const cudaError_t r = cudaStreamSynchronize(st[q]);
            if (e == cudaSuccess) e = r;
            cudaStreamDestroy(st[q]);
        }
        if (done[q]) cudaEventDestroy(done[q]);
    }
    if (start) cudaEventDestroy(start);
    return e;
}

}  // namespace nk
