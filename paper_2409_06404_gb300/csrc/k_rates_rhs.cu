// The implicit-stage sources' variants of the rates kernel (k_rates.cuh), compiled apart from the
// rates' variants (k_rates.cu) so the two build in parallel.
#include "k_rates.cuh"

namespace nk {

cudaError_t launch_rates_rhs(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* dlnA, double* omega, double* hrr, int precision,
                             cudaStream_t s) {
    if (precision == NK_MIXED) return launch_form<kMixed, true>(m, n, ld, T, p, Y, dlnA, omega, hrr, s);
    if (precision == NK_FP64_NATIVE) return launch_form<kNative, true>(m, n, ld, T, p, Y, dlnA, omega, hrr, s);
    return launch_form<kDF, true>(m, n, ld, T, p, Y, dlnA, omega, hrr, s);
}

}  // namespace nk
