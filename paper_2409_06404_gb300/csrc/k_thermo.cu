// Thermodynamic properties per point: NASA-7 species c_p, h, g and the mass-based mixture
// c_p and h, mean molar mass and ideal-gas density (Eq. 1b-1d of the paper).
// One thread per point; species rows are read coalesced across the warp (SoA layout).
#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kBlk = 128;

__global__ void __launch_bounds__(kBlk) thermo_kernel(DevMech m, int64_t n, int64_t ld,
                                                      const double* __restrict__ T, const double* __restrict__ p,
                                                      const double* __restrict__ Y, double* __restrict__ cp_mix,
                                                      double* __restrict__ h_mix, double* __restrict__ Wbar,
                                                      double* __restrict__ rho, double* __restrict__ cp_k,
                                                      double* __restrict__ h_k, double* __restrict__ g_k) {
    const int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x;
    if (i >= n) return;
    const double Ti = T[i];
    const double lnT = log(Ti), invT = 1.0 / Ti, RT = kR * Ti;
    double s = 0.0, cp = 0.0, h = 0.0;
    for (int k = 0; k < m.K; ++k) {
        const double yw = Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
        const double* c = nasa_range(m, k, Ti);
        const double cpR = nasa_cpR(c, Ti);
        const double hRT = nasa_hRT(c, Ti, invT);
        s += yw;
        cp = fma(yw, cpR, cp);
        h = fma(yw, hRT, h);
        if (cp_k) cp_k[(int64_t)k * ld + i] = kR * cpR;
        if (h_k) h_k[(int64_t)k * ld + i] = RT * hRT;
        if (g_k) g_k[(int64_t)k * ld + i] = RT * nasa_gRT(c, Ti, lnT, invT);
    }
    const double wb = 1.0 / s;
    if (cp_mix) cp_mix[i] = kR * cp;
    if (h_mix) h_mix[i] = RT * h;
    if (Wbar) Wbar[i] = wb;
    if (rho) rho[i] = p[i] * wb * invT * kInvR;
}

}  // namespace

cudaError_t launch_thermo(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                          const double* Y, double* cp_mix, double* h_mix, double* Wbar, double* rho,
                          double* cp_k, double* h_k, double* g_k, cudaStream_t s) {
    const int64_t grid = (n + kBlk - 1) / kBlk;
    thermo_kernel<<<(unsigned)grid, kBlk, 0, s>>>(m, n, ld, T, p, Y, cp_mix, h_mix, Wbar, rho, cp_k, h_k, g_k);
    return cudaGetLastError();
}

}  // namespace nk
