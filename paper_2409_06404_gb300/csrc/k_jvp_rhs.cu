// The implicit-stage sources' JVP variants of the JVP kernel (k_jvp.cuh), compiled apart from the
// rates' variants (k_jvp.cu) so the two build in parallel.
#include "k_jvp.cuh"

namespace nk {

cudaError_t launch_jvp_rhs(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                           const double* Y, const double* dlnA, const double* vT, const double* vY, double* omega,
                           double* hrr, double* d_omega, double* d_hrr, cudaStream_t s) {
    if (omega) return launch_o<true, true>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, s);
    return launch_o<false, true>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, s);
}

}  // namespace nk
