// Net production rates and heat release (and the implicit-stage sources): the launch entry
// (kernels and launch shapes in k_rates.cuh).  The sources' variants are compiled in
// k_rates_rhs.cu, a translation unit of their own, so the two halves build in parallel.
#include "k_rates.cuh"

namespace nk {

cudaError_t launch_rates_rhs(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* dlnA, double* omega, double* hrr, int precision,
                             cudaStream_t s);

cudaError_t launch_rates(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                         const double* Y, const double* dlnA, double* omega, double* hrr, int precision,
                         cudaStream_t s, int rhs) {
    // the staged tables (kMathTabDoubles doubles) cover the kDF tables too (3 x 128 pairs)
    static_assert(kDfTabBytes <= kMathTabDoubles * sizeof(double), "table space");
    if (rhs) return launch_rates_rhs(m, n, ld, T, p, Y, dlnA, omega, hrr, precision, s);
    if (precision == NK_MIXED) return launch_form<kMixed, false>(m, n, ld, T, p, Y, dlnA, omega, hrr, s);
    if (precision == NK_FP64_NATIVE) return launch_form<kNative, false>(m, n, ld, T, p, Y, dlnA, omega, hrr, s);
    return launch_form<kDF, false>(m, n, ld, T, p, Y, dlnA, omega, hrr, s);
}

}  // namespace nk
