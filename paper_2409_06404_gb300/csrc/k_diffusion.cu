// Mixture-averaged diffusion fluxes (Eq. 2 of the paper with the correction velocity defined
// below it) from the mixture-averaged coefficients D_k and the mole-fraction gradients:
//   V_k = -(D_k/X_k) grad X_k + V_c,  V_c = -sum_k Y_k V'_k  (V'_k the uncorrected velocity),
//   j_k = rho Y_k V_k,  and sum_k c_p,k j_k (the factor of the enthalpy-flux term of Eq. 1b).
// With Y_k/X_k = W_k/Wbar the uncorrected flux rho Y_k V'_k = a_k grad X_k,
// a_k = -rho (W_k/Wbar) D_k, has no division by X_k; with S = sum_k a_k grad X_k,
// V_c = -S/rho and j_k = a_k grad X_k - Y_k S.  One thread per point, two passes over the
// species (the second re-reads D_k and grad X_k, which the first brought into L2).
// Plain double arithmetic; the pass reads 3K + 2K + 2 and writes 3K + 6 doubles per point.
#include "nk_internal.cuh"

namespace nk {
namespace {

constexpr int kBlk = 128;

__global__ void __launch_bounds__(kBlk) diffusion_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                         const double* __restrict__ T, const double* __restrict__ p,
                                                         const double* __restrict__ Y, const double* __restrict__ D,
                                                         const double* __restrict__ G, double* __restrict__ j,
                                                         double* __restrict__ Vc, double* __restrict__ hf) {
    const int64_t i = (int64_t)blockIdx.x * kBlk + threadIdx.x;
    if (i >= n) return;
    const int K = m.K;
    const int64_t cs = (int64_t)K * ld;                       // component stride of grad X and j
    const double Ti = T[i];
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double rho = p[i] / (kR * Ti * s);                  // rho = p Wbar/(R T), Wbar = 1/s
    const double c0 = -rho * s;                               // a_k = c0 W_k D_k = -rho (W_k/Wbar) D_k
    double S0 = 0.0, S1 = 0.0, S2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const int64_t o = (int64_t)k * ld + i;
        const double a = c0 * __ldg(m.W + k) * D[o];
        S0 = fma(a, G[o], S0);
        S1 = fma(a, G[o + cs], S1);
        S2 = fma(a, G[o + 2 * cs], S2);
    }
    if (Vc) {
        const double ir = -1.0 / rho;
        Vc[i] = S0 * ir;
        Vc[ld + i] = S1 * ir;
        Vc[2 * ld + i] = S2 * ir;
    }
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;
    for (int k = 0; k < K; ++k) {
        const int64_t o = (int64_t)k * ld + i;
        const double a = c0 * __ldg(m.W + k) * D[o], y = Y[o];
        const double j0 = fma(a, G[o], -y * S0), j1 = fma(a, G[o + cs], -y * S1), j2 = fma(a, G[o + 2 * cs], -y * S2);
        j[o] = j0;
        j[o + cs] = j1;
        j[o + 2 * cs] = j2;
        if (hf) {
            const double cpk = kR * nasa_cpR(nasa_range(m, k, Ti), Ti) * __ldg(m.invW + k);   // J/(kg K)
            h0 = fma(cpk, j0, h0);
            h1 = fma(cpk, j1, h1);
            h2 = fma(cpk, j2, h2);
        }
    }
    if (hf) {
        hf[i] = h0;
        hf[ld + i] = h1;
        hf[2 * ld + i] = h2;
    }
}

}  // namespace

cudaError_t launch_diffusion(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* D, const double* gradX, double* j, double* Vc,
                             double* hf, cudaStream_t s) {
    diffusion_kernel<<<(unsigned)((n + kBlk - 1) / kBlk), kBlk, 0, s>>>(m, n, ld, T, p, Y, D, gradX, j, Vc, hf);
    return cudaGetLastError();
}

}  // namespace nk
