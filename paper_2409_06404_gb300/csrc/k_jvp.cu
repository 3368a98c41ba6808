// Exact Jacobian-vector product of (omega_k, heat release) and of the implicit-stage sources: the
// launch entry (kernels and launch shapes in k_jvp.cuh).  The sources' variants are compiled in
// k_jvp_rhs.cu, a translation unit of their own, so the two halves build in parallel.
#include "k_jvp.cuh"

namespace nk {

cudaError_t launch_jvp_rhs(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                           const double* Y, const double* dlnA, const double* vT, const double* vY, double* omega,
                           double* hrr, double* d_omega, double* d_hrr, cudaStream_t s);

cudaError_t launch_jvp(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* vT, const double* vY, double* omega,
                       double* hrr, double* d_omega, double* d_hrr, cudaStream_t s, int rhs) {
    static_assert(kDfTabBytes <= kMathTabDoubles * sizeof(double), "table space");
    if (rhs) return launch_jvp_rhs(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, s);
    // the primal outputs (either one) take the variant that sums them; without them the kernel
    // skips the heat-release sum
    if (omega || hrr) return launch_o<true, false>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, s);
    return launch_o<false, false>(m, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr, s);
}

}  // namespace nk
