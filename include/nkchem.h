/*
 * nkchem — pointwise thermochemistry for spectral-element reacting-flow solvers, on GB300.
 *
 * C ABI of the library (libnkchem.so).  It evaluates, independently at every grid point,
 * the right-hand-side quantities that the implicit thermochemistry stage of a low-Mach
 * reacting-flow solver needs (nekCRF, arXiv 2409.06404, Sec. 2, Eq. 1-4 and the "rates" and
 * "properties" kernels of Tab. 3-4): NASA-7 thermodynamics, net species production rates
 * omega_k with heat release, mixture-averaged transport, and exact Jacobian-vector and
 * vector-Jacobian products of (omega_k, heat release).
 *
 * Conventions shared by every entry point
 *  - Units are SI: K, Pa, kg/mol, J/mol, mol/m^3, s.
 *  - State arrays are structure-of-arrays in DEVICE memory, owned by the caller:
 *      T[n], p[n]                  point temperature and pressure
 *      Y[K*ld]                     mass fractions, species k of point i at Y[k*ld + i]
 *    Per-species outputs use the same [K][ld] layout; per-point outputs are [n].
 *    ld >= n is the row stride, so a chunk of a larger field is passed as (ptr + offset, ld).
 *  - Every double array must be 8-byte aligned (else NK_EALIGN).
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *    return after enqueueing.  Only argument errors and launch failures are reported
 *    synchronously; kernels never trap.  Non-finite or non-physical inputs (T <= 0, all
 *    Y = 0) propagate NaN/Inf to that point's outputs only.
 *  - Mass fractions are used as given: no clipping and no renormalisation; negative Y_k
 *    give negative concentrations and are evaluated as such.
 *  - On failure a thread-local message is available from nk_last_error().
 *  - One nk_mech may be used from several streams and host threads concurrently.
 */
#ifndef NKCHEM_H
#define NKCHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NKCHEM_VERSION 1

typedef struct CUstream_st* nk_stream; /* identical to cudaStream_t */

typedef enum {
    NK_OK = 0,
    NK_EINVAL = 1,        /* bad argument: null pointer, n < 0, ld < n, bad enum, bad table */
    NK_EALIGN = 2,        /* an array is not 8-byte aligned */
    NK_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    NK_ENOMEM = 4,        /* device allocation failed (mechanism load only) */
    NK_EUNSUPPORTED = 5   /* mechanism beyond the library's limits (see nk_mechanism_load) */
} nk_status;

typedef enum {
    NK_FP64 = 0,        /* results to double precision (1e-10 of the FP64 definition, typically
                           1e-13): exponent chains of the rates (ln k_f, Gibbs sums, ln K_c,
                           falloff) and all of transport in double-float (pairs of floats,
                           48-bit significands) on the FP32 pipe; concentrations, products,
                           the forward-minus-reverse difference and every accumulation in
                           double; inputs and outputs in double */
    NK_MIXED = 1,       /* rates: Arrhenius/Troe arguments and k_f in single precision,
                           equilibrium constants (pairs), forward-minus-reverse difference and
                           omega accumulation in double; transport: fits, mixture rules and
                           sums in single precision (1e-5) */
    NK_FP64_NATIVE = 2, /* every operation in native double precision (reference form) */
    NK_JIT = 3          /* nk_rates_eval only: NK_FP64_NATIVE's arithmetic in a kernel generated
                           for the loaded mechanism (straight-line code, the mechanism's data as
                           literals) and compiled at first use with NVRTC, as the paper generates
                           its kernels from the mechanism (Sec. 2); see nk_mechanism_jit */
} nk_precision;

/* Reaction kinds of nk_mech_desc.rtype */
enum { NK_RXN_ELEMENTARY = 0, NK_RXN_THIRD_BODY = 1, NK_RXN_TROE = 2 };

/* Opaque, immutable device copy of a mechanism; owned by the library. */
typedef struct nk_mech nk_mech;

/*
 * Host-side description of a mechanism (read during nk_mechanism_load, then no longer
 * referenced).  This is the data a Cantera-format mechanism carries (Sec. 2: species
 * thermodynamics, reactions, transport fits), as flat arrays:
 *   K species, R reactions, n_elem elements.
 *   W[K]                  molar masses (kg/mol)
 *   atoms[K*n_elem]       element counts (informational; not used in evaluation)
 *   nasa_lo[K*7], nasa_hi[K*7]   NASA-7 coefficients a1..a7, low range used for T <= T_mid[k]
 *   T_mid[K]
 *   reac_ptr[R+1], reac_sp[], reac_nu[]  reactant entries of reaction r in
 *                         [reac_ptr[r], reac_ptr[r+1]): species index, stoichiometric
 *                         coefficient (positive integer); products likewise (prod_*).
 *                         Every reaction is reversible.
 *   rtype[R]              NK_RXN_* kind
 *   lnA[R], beta[R], Ea[R]       Arrhenius k = exp(lnA) T^beta exp(-Ea/(R T)); for Troe rows
 *                         this is the high-pressure limit k_inf
 *   lnA0[R], beta0[R], Ea0[R]    Troe low-pressure limit k_0 (read for Troe rows only)
 *   troe[R*4]             Troe a, T3, T1, T2 (T2 <= 0: the exp(-T2/T) term is absent)
 *   eff[R*K]              third-body efficiencies (read for third-body and Troe rows)
 *   mu_fit[K*4], lam_fit[K*4]    ln(mu_k / Pa s), ln(lambda_k / W/m/K) as cubics in ln T,
 *                         lowest order first
 *   D_fit[K*(K-1)/2*4]    ln(D_jk / m^2/s) at p_ref as cubics in ln T, for pairs j<k packed
 *                         row-major: pair (j,k) at j*K - j*(j+1)/2 + (k-j-1)
 *   p_ref                 reference pressure of D_fit (Pa)
 */
typedef struct {
    int32_t K, R, n_elem;
    const double* W;
    const int32_t* atoms;
    const double* nasa_lo;
    const double* nasa_hi;
    const double* T_mid;
    const int32_t* reac_ptr;
    const int32_t* reac_sp;
    const int32_t* reac_nu;
    const int32_t* prod_ptr;
    const int32_t* prod_sp;
    const int32_t* prod_nu;
    const int32_t* rtype;
    const double* lnA;
    const double* beta;
    const double* Ea;
    const double* lnA0;
    const double* beta0;
    const double* Ea0;
    const double* troe;
    const double* eff;
    const double* mu_fit;
    const double* lam_fit;
    const double* D_fit;
    double p_ref;
} nk_mech_desc;

/*
 * Copy a mechanism to the current CUDA device and build the kernels' coefficient tables.
 * The mechanism input the paper feeds its generated kernels (Sec. 2, "Cantera format").
 * Limits: 1 <= K <= 256, 1 <= R <= 8192, at most 4 reactant and 4 product entries per
 * reaction, stoichiometric coefficients 1..8 (else NK_EUNSUPPORTED).  Synchronous.
 * On success *out owns device memory until nk_mechanism_free.
 */
nk_status nk_mechanism_load(const nk_mech_desc* desc, nk_mech** out);

/* Release a mechanism (NULL is accepted).  The caller ensures no call using it is running. */
nk_status nk_mechanism_free(nk_mech* mech);

/* Number of species and reactions of a loaded mechanism (either pointer may be NULL). */
nk_status nk_mechanism_info(const nk_mech* mech, int32_t* K, int32_t* R);

/*
 * Thermodynamic properties (Eq. 1b-1d: c_p, c_p,k, h_k, and p0 = rho R T / Wbar).
 * Outputs (NULL = not wanted):
 *   cp_mix[n]  mixture heat capacity, J/(kg K)      h_mix[n]  mixture enthalpy, J/kg
 *   Wbar[n]    mean molar mass, kg/mol              rho[n]    density, kg/m^3
 *   cp_k, h_k, g_k [K*ld]  species molar c_p (J/(mol K)), enthalpy and Gibbs energy (J/mol)
 * Double precision.
 */
nk_status nk_thermo_eval(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                         const double* p, const double* Y, double* cp_mix, double* h_mix,
                         double* Wbar, double* rho, double* cp_k, double* h_k, double* g_k,
                         nk_stream stream);

/*
 * Net production rates and heat release (the "rates" kernel, Tab. 3-4; omega_k of Eq. 1a
 * and the heat release of Eq. 1b / iHRR of Sec. 3.3):
 *   omega[K*ld]  omega_k = sum_r nu_kr q_r, mol/(m^3 s)
 *   hrr[n]       -sum_k h_k(T) omega_k, W/m^3 (positive when exothermic)
 * dlnA: NULL or device [R] shift added to ln A_r (to both limits of a Troe reaction).
 * precision: NK_FP64, NK_FP64_NATIVE, NK_MIXED or NK_JIT.
 */
nk_status nk_rates_eval(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                        const double* p, const double* Y, const double* dlnA, double* omega,
                        double* hrr, nk_precision precision, nk_stream stream);

/*
 * Mixture-averaged transport properties (the "properties" kernel, Tab. 3; Eq. 2 and 4):
 *   mu[n]      mixture viscosity (Wilke), Pa s
 *   lambda[n]  mixture conductivity (Mathur-Saxena average), W/(m K)
 *   Dmix[K*ld] mixture-averaged diffusion coefficients D_k of Eq. 2, m^2/s
 *              (D_km = sum_{j!=k} X_j W_j / (Wbar sum_{j!=k} X_j/D_jk); 0 for a pure species)
 * Any output may be NULL.  precision: NK_FP64, NK_FP64_NATIVE or NK_MIXED.
 */
nk_status nk_transport_eval(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                            const double* p, const double* Y, double* mu, double* lambda,
                            double* Dmix, nk_precision precision, nk_stream stream);

/*
 * Mixture-averaged diffusion fluxes (Eq. 2 with its correction velocity, Sec. 2), the
 * species and enthalpy fluxes whose divergences enter Eq. 1a-b:
 *   Dmix[K*ld]      mixture-averaged coefficients D_k (from nk_transport_eval), m^2/s
 *   gradX[3*K*ld]   mole-fraction gradients: component c of species k at (c*K + k)*ld + i, 1/m
 *   j[3*K*ld]       species mass fluxes rho Y_k V_k, kg/(m^2 s), same layout, with
 *                   V_k = -(D_k/X_k) grad X_k + V_c and V_c = -sum_k Y_k V'_k (V'_k uncorrected)
 *   Vc[3*ld]        correction velocity V_c, m/s (NULL: not written)
 *   hf[3*ld]        sum_k c_p,k j_k with mass-based c_p,k, W/(m^2 K) (NULL: not written)
 * Y_k/X_k is taken as W_k/Wbar, so absent species (X_k = 0) have finite fluxes.  Double
 * precision; the gradients come from the caller's discretisation (not part of this library).
 */
nk_status nk_diffusion_fluxes(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                              const double* Y, const double* Dmix, const double* gradX, double* j, double* Vc,
                              double* hf, nk_stream stream);

/*
 * Exact Jacobian-vector product of (omega_k, hrr) with respect to (T, Y_k) at fixed p: the
 * product the Newton-GMRES stage of the paper forms by difference quotients (Sec. 2 and 4).
 *   vT[n], vY[K*ld]        direction
 *   d_omega[K*ld], d_hrr[n]  J v
 *   omega[K*ld], hrr[n]    NULL, or also return the primal values
 * Rates of progress are recomputed per point, never stored.  Double precision.
 */
nk_status nk_rates_jvp(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                       const double* p, const double* Y, const double* dlnA, const double* vT,
                       const double* vY, double* omega, double* hrr, double* d_omega,
                       double* d_hrr, nk_stream stream);

/*
 * Chemistry sources of the implicit thermochemistry stage: the production and heat-release
 * terms of Eq. 1a-b at fixed pressure (Sec. 2; no dp0/dt term), the right-hand side the
 * stage's Newton iterations evaluate at every point:
 *   fT[n]      dT/dt = hrr / (rho c_p), K/s (c_p the mass-based mixture heat capacity)
 *   fY[K*ld]   dY_k/dt = W_k omega_k / rho, 1/s
 * with omega_k, hrr as in nk_rates_eval and rho = p Wbar/(R T).  dlnA as in nk_rates_eval.
 * precision: NK_FP64, NK_FP64_NATIVE or NK_MIXED.
 */
nk_status nk_rhs_eval(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                      const double* Y, const double* dlnA, double* fT, double* fY,
                      nk_precision precision, nk_stream stream);

/*
 * Exact Jacobian-vector product of those sources with respect to (T, Y_k) at fixed p: the
 * product the stage's GMRES solve forms by difference quotients (Sec. 2).
 *   vT[n], vY[K*ld]      direction
 *   dfT[n], dfY[K*ld]    J v
 *   fT[n], fY[K*ld]      NULL, or also return the sources
 * Rates of progress recomputed per point, never stored; FP64 form (as NK_FP64).
 */
nk_status nk_rhs_jvp(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                     const double* Y, const double* dlnA, const double* vT, const double* vY,
                     double* fT, double* fY, double* dfT, double* dfY, nk_stream stream);

/*
 * Stored linearization of (omega_k, hrr) at one state, for several Jacobian-vector products
 * at that state (the Newton-Krylov stage issues several per step, Sec. 2 and 4).  The
 * state-only part of nk_rates_jvp -- exponentials, thermo polynomials, concentration
 * products -- is evaluated once and kept per point:
 *   *slots   doubles per point of the stored data (depends on the mechanism only)
 *   lin      device [slots][ldl], ldl >= n, caller-owned; written by nk_rates_linearize
 * nk_rates_jvp_linearized then forms (d_omega, d_hrr) = J (vT, vY) from lin and the state,
 * which must be the one lin was made at (same T, p, Y, dlnA).  Results agree with
 * nk_rates_jvp to rounding (FP64 form).  Use it when slots * ldl * 8 bytes fit beside the
 * fields; otherwise nk_rates_jvp recomputes everything per direction.
 */
nk_status nk_rates_linearization_slots(const nk_mech* mech, int64_t* slots);
nk_status nk_rates_linearize(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* dlnA, double* lin, int64_t ldl, nk_stream stream);
nk_status nk_rates_jvp_linearized(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                                  const double* p, const double* Y, const double* lin, int64_t ldl,
                                  const double* vT, const double* vY, double* d_omega, double* d_hrr,
                                  nk_stream stream);

/*
 * The same stored linearization in single precision, and products from it in single
 * precision (FP32 pipe).  For Krylov solvers whose basis is single precision (as the paper's
 * GMRES, Sec. 2): the products then carry rounding of the order the basis already has.
 *   *slots   32-bit words per point (nk_rates_linearization_slots_f32; about half the bytes)
 *   lin      device float [slots][ldl], ldl >= n, caller-owned; written by nk_rates_linearize_f32
 * Each reaction's coefficients are stored rounded to float after scaling by a power of two
 * per reaction and point, and each species' tangent is summed at a power-of-two scale of its
 * own (both kept beside the coefficients), so rates of any magnitude fit; coefficients below
 * 2^-126 of their reaction's largest, and terms below 2^-126 of their species' scale, drop
 * out.  Result k is within about (terms_k + 8) 2^-24 of the sum of the magnitudes of the
 * terms it adds, terms_k the reactions species k takes part in (against 2^-53 for the double
 * entries); the inputs are rounded to float without subnormals, the heat-release and source
 * epilogues run in double.  The rhs form takes the sources at the state, as
 * nk_rhs_jvp_linearized.
 */
nk_status nk_rates_linearization_slots_f32(const nk_mech* mech, int64_t* slots);
nk_status nk_rates_linearize_f32(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* dlnA, float* lin, int64_t ldl, nk_stream stream);
nk_status nk_rates_jvp_linearized_f32(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                                      const double* p, const double* Y, const float* lin, int64_t ldl,
                                      const double* vT, const double* vY, double* d_omega, double* d_hrr,
                                      nk_stream stream);
nk_status nk_rhs_jvp_linearized_f32(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                                    const double* Y, const float* lin, int64_t ldl, const double* fT,
                                    const double* fY, const double* vT, const double* vY, double* dfT,
                                    double* dfY, nk_stream stream);

/*
 * The stored linearization in a per-reaction ("compact") form, for fields whose per-entry data
 * (nk_rates_linearize) would not fit: the Newton-Krylov stage's several products at one state
 * (Sec. 2 and 4) on the largest fields.  Kept per point: per reaction the forward and reverse
 * terms (k_f prod C^nu' and k_r prod C^nu'', times [M] for third-body reactions), the
 * coefficient of dT/T and, for third-body and Troe reactions, of d[M]; per species h_k/RT, 1/Y_k
 * and C_k -- about half the per-entry form's doubles (1,180 per point at 53 species and 325
 * reactions, against 2,112).  The products then need no concentration product: each side's
 * tangent is its term times sum_e nu_e dC_e/C_e, with dC_e/C_e = d rho/rho + dY_e/Y_e.  Sides
 * with a mass fraction below 2^-200 in magnitude, zero or non-finite keep k without the
 * product and are formed by exclusive products instead, so zero and absent species are exact.
 *   *slots   doubles per point (nk_rates_linearization_slots_compact; depends on the mechanism)
 *   lin      device [slots][ldl], ldl >= n, caller-owned; written by nk_rates_linearize_compact
 *   omega[K*ld], hrr[n]   both NULL, or also written: the rates at the state, as nk_rates_eval
 *            (NK_FP64) computes them, from the same pass (NK_EINVAL if only one is given)
 * nk_rates_jvp_linearized_compact forms (d_omega, d_hrr) = J (vT, vY) from lin and the state lin
 * was made at (same T, p, Y, dlnA); nk_rhs_jvp_linearized_compact the sources' JVP given the
 * sources there, as nk_rhs_jvp_linearized.  Results agree with nk_rates_jvp to rounding (the
 * FP64 form's linearization, plain double products).
 */
nk_status nk_rates_linearization_slots_compact(const nk_mech* mech, int64_t* slots);
nk_status nk_rates_linearize_compact(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                                     const double* Y, const double* dlnA, double* lin, int64_t ldl, double* omega,
                                     double* hrr, nk_stream stream);
nk_status nk_rates_jvp_linearized_compact(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                                          const double* p, const double* Y, const double* lin, int64_t ldl,
                                          const double* vT, const double* vY, double* d_omega, double* d_hrr,
                                          nk_stream stream);
nk_status nk_rhs_jvp_linearized_compact(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                                        const double* p, const double* Y, const double* lin, int64_t ldl,
                                        const double* fT, const double* fY, const double* vT, const double* vY,
                                        double* dfT, double* dfY, nk_stream stream);

/*
 * Rates (nk_rates_eval) and transport (nk_transport_eval) of fields that live in host memory,
 * the library's end-to-end entry: the points are cut into chunks of `chunk`, each copied to
 * the device, evaluated and copied back, the chunks cycling over three internal streams so that
 * both copy directions overlap the kernels.
 *   T[n], p[n], Y[K*n]                       host, contiguous SoA (species rows of n)
 *   omega[K*n], hrr[n], mu[n], lambda[n], Dmix[K*n]   host outputs, any may be NULL
 *   workspace   device, nk_host_eval_workspace(mech, min(chunk, n)) bytes
 * Page-locked host memory makes the copies asynchronous.  The caller's stream is ordered
 * before and after the evaluation; the call returns when the outputs are in host memory.
 * precision: NK_FP64, NK_FP64_NATIVE or NK_MIXED (both kernels).
 */
nk_status nk_host_eval_workspace(const nk_mech* mech, int64_t chunk, size_t* bytes);
nk_status nk_host_eval(const nk_mech* mech, int64_t n, const double* T, const double* p, const double* Y,
                       double* omega, double* hrr, double* mu, double* lambda, double* Dmix,
                       nk_precision precision, int64_t chunk, void* workspace, size_t workspace_bytes,
                       nk_stream stream);

/*
 * The mechanism-specialised rates kernel behind NK_JIT.  nk_mechanism_jit compiles it now
 * (otherwise the first NK_JIT call does): NVRTC (libnvrtc.so.13, loaded at run time) builds a
 * cubin for the current device's architecture, which the runtime loads; NK_EUNSUPPORTED with
 * the compiler's message when NVRTC is missing or the compilation fails.  nk_jit_source writes
 * the generated CUDA source for a mechanism description (host only, no device needed): *len is
 * the buffer size on entry and the size needed (with the terminating NUL) on return; the text
 * is copied when it fits, else NK_EINVAL.
 */
nk_status nk_mechanism_jit(nk_mech* mech);
nk_status nk_jit_source(const nk_mech_desc* desc, char* buf, size_t* len);

/*
 * Dense Jacobian of the sources of nk_rhs_eval with respect to x = (T, Y_0..Y_{K-1}) at fixed p,
 * assembled from a stored linearization (nk_rates_linearize, dlnA = NULL) and the sources
 * (nk_rhs_eval, NK_FP64) at the same state: the per-point blocks of the Jacobian of the
 * paper's implicit thermochemistry stage (Sec. 2), exact to rounding.
 *   lin[slots*ldl]        stored linearization at (T, p, Y)
 *   fT[n], fY[K*ld]       the sources at (T, p, Y)
 *   J[(K+1)*(K+1)*ldJ]    out: entry (r, c) of point i at J[(r (K+1) + c) ldJ + i]; r, c = 0 for T,
 *                         k + 1 for Y_k (row = source, column = variable); ldJ >= n
 * Double precision; K + 1 <= 160 (a point's block is assembled in shared memory).
 */
nk_status nk_rhs_jacobian(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                          const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                          double* J, int64_t ldJ, nk_stream stream);

/*
 * Per-point block-Jacobi preconditioner of an implicit stage's Newton-Krylov solve (an option
 * beside the paper's unpreconditioned GMRES, Sec. 2): with w the error weights of the solve,
 * the blocks P = I - dt diag(w) J diag(1/w) (J as in nk_rhs_jacobian) are formed and factored
 * in place, LU with partial pivoting per point, in double precision (the blocks of stiff
 * chemistry in these weights are far too ill-conditioned for single-precision factors).  Each
 * row r of P is first scaled by 2^-e_r, its largest entry then in [1/2, 1).
 *   w[(K+1)*ldw]          weights, row 0 for T, row k + 1 for Y_k
 *   F[(K+1)*(K+1)*ldF]    out: the factors of the scaled block, entry (r, c) of point i at
 *                         F[(r (K+1) + c) ldF + i], in pivot order: row k holds the
 *                         unit-lower part L_k,0..k-1 and U_k,k+1.. of the k-th pivot row, with
 *                         1/U_kk at (k, k) (a zero pivot is replaced by 1)
 *   piv[(K+1)*ldF]        out: for the k-th pivot row of point i, piv[k ldF + i] = its row
 *                         index (low 16 bits) | e_row << 16 (signed)
 * nk_block_jacobi_apply then computes z = P^-1 v for vectors v, z of (K+1) rows of ldv / ldz
 * (row r of point i at r ld + i; z may alias v).  K + 1 <= 160; ldF >= n.
 */
nk_status nk_block_jacobi_factor(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* lin, int64_t ldl, const double* fT,
                                 const double* fY, const double* w, int64_t ldw, double dt, double* F,
                                 int32_t* piv, int64_t ldF, nk_stream stream);
nk_status nk_block_jacobi_apply(const nk_mech* mech, int64_t n, const double* F, const int32_t* piv, int64_t ldF,
                                const double* v, int64_t ldv, double* z, int64_t ldz, nk_stream stream);

/*
 * The JVP of nk_rhs_jvp from a stored linearization (nk_rates_linearize at the same state,
 * dlnA = NULL) and the sources there (nk_rhs_eval, NK_FP64): the cheap per-direction pass for a
 * Newton-Krylov solve that forms several products at one state.
 *   fT[n], fY[K*ld]   the sources at (T, p, Y);  vT, vY the direction;  dfT[n], dfY[K*ld] out
 */
nk_status nk_rhs_jvp_linearized(const nk_mech* mech, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, const double* lin, int64_t ldl, const double* fT,
                                const double* fY, const double* vT, const double* vY, double* dfT, double* dfY,
                                nk_stream stream);

/*
 * One implicit (backward) Euler step of dt seconds of the homogeneous constant-pressure
 * reactor at every point: solves x1 - x0 - dt f(x1) = 0, x = (T, Y_k), f the sources of
 * nk_rhs_eval, the nonlinear system of the paper's implicit thermochemistry stage (Sec. 2),
 * here without the transport terms.  Newton's method with one GMRES solve over all points per
 * iteration, as the paper's stage: exact Jacobian-vector products (nk_rhs_jvp) instead of
 * difference quotients, the Krylov basis in single precision, classical Gram-Schmidt with the
 * projections in one reduction and the new vector's norm in a second.  Norms are weighted RMS
 * norms with weights 1/(rtol |x0_i| + atol_i).
 *   T[n], Y[K*n]   in: the state x0; out: the step's result (contiguous: Y rows of stride n)
 *   workspace      device, nk_reactor_workspace bytes for the same options (holds (K+1) n
 *                  doubles x 8 and (krylov_dim + 1) (K+1) n floats; with the preconditioner
 *                  also (K+1)^2 n doubles of factors, (K+1) n pivot words and a stored
 *                  linearization of up to about 2 GB, filled chunk by chunk; with linearized
 *                  products the full stored linearization, nk_rates_linearization_slots x n
 *                  doubles, or floats for linearized = 2)
 * With precond = 1 the solve is left-preconditioned by the per-point blocks of
 * nk_block_jacobi_factor, made once per step at x0: GMRES minimises P^-1 (r - A z), which
 * tracks the error of the update (the unpreconditioned residual of stiff chemistry is dominated
 * by its stiff components), and lin_tol applies to it.  precond = 2 reuses the factors left in
 * the workspace by the last call with precond 1 (same mechanism, n and workspace), as a stiff
 * ODE solver keeps its Newton matrix over several steps; the caller refreshes them (precond 1)
 * when the state or dt has moved far.
 * The call returns when the step is done (it reads a few scalars back per GMRES iteration);
 * non-convergence is reported in stats, not as an error.
 */
#define NK_REACTOR_MAX_KRYLOV 30
typedef struct {
    double rtol;          /* relative tolerance of the error weights */
    double atol_T;        /* absolute tolerance for T, K */
    double atol_Y;        /* absolute tolerance for the mass fractions */
    double newton_tol;    /* converged when (weighted RMS norm of the Newton update) x
                             min(1, its contraction rate) is below this, the update test of a
                             stiff ODE solver */
    double lin_tol;       /* each GMRES solve stops when its residual has fallen by this factor
                             (or after krylov_dim iterations; the partial solution is used) */
    int32_t max_newton;   /* Newton iterations at most */
    int32_t krylov_dim;   /* GMRES iterations per Newton iteration, 1..NK_REACTOR_MAX_KRYLOV */
    int32_t precond;      /* 0: none (the paper's stage); 1: per-point block Jacobi made at x0;
                             2: block Jacobi from the factors of an earlier call (K + 1 <= 160) */
    int32_t linearized;   /* 0: every GMRES product recomputes the rates (nk_rhs_jvp); 1: the rates
                             are linearized once per Newton iteration and the products come from
                             the stored data (nk_rhs_jvp_linearized): cheaper once a Newton
                             iteration takes more than one or two GMRES iterations; 2: as 1 with
                             the linearization in single precision and the products from it
                             (nk_rhs_jvp_linearized_f32), matching the FP32 basis; the residuals,
                             and so the converged state, stay double.  2 needs precond = 0: the
                             preconditioned operator P^-1 A would amplify the products' rounding
                             by the blocks' condition numbers (~1e29 for stiff chemistry) */
} nk_reactor_opts;
typedef struct {
    int32_t converged;    /* 1 when the update test was met (0: max_newton reached, or the
                             updates grew: diverging) */
    int32_t newton_iters;
    int32_t krylov_iters; /* summed over the Newton iterations */
    double update_wrms;   /* weighted RMS norm of the last Newton update */
    double residual_wrms; /* weighted RMS norm of the residual before the last update */
} nk_reactor_stats;
nk_status nk_reactor_workspace(const nk_mech* mech, int64_t n, const nk_reactor_opts* opts, size_t* bytes);
nk_status nk_reactor_step(const nk_mech* mech, int64_t n, double* T, const double* p, double* Y, double dt,
                          const nk_reactor_opts* opts, nk_reactor_stats* stats, void* workspace,
                          size_t workspace_bytes, nk_stream stream);

/*
 * Bytes of device workspace nk_rates_vjp needs for n points when g_lnA is requested
 * (per-block partial sums of the ln A gradient, reduced in a fixed order).
 */
nk_status nk_rates_vjp_workspace(const nk_mech* mech, int64_t n, size_t* bytes);

/*
 * Vector-Jacobian product of (omega_k, hrr) (gradients for mechanism calibration and for
 * adjoint solves; the exact transpose of nk_rates_jvp):
 *   bar_omega[K*ld], bar_hrr[n] (NULL = 0)   cotangents
 *   gT[n], gY[K*ld]                          J^T (bar_omega, bar_hrr) with respect to T, Y
 *   g_lnA[R] (NULL = not wanted)  sum over the n points of d/d lnA_r; overwritten.  Needs
 *            workspace of nk_rates_vjp_workspace bytes; the sum is deterministic for a
 *            given n (fixed partition and summation order, no atomics).
 * Double precision.
 */
nk_status nk_rates_vjp(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                       const double* p, const double* Y, const double* dlnA,
                       const double* bar_omega, const double* bar_hrr, double* gT, double* gY,
                       double* g_lnA, void* workspace, size_t workspace_bytes, nk_stream stream);

/*
 * nk_rates_vjp without a workspace argument; it allocates no device memory.  (No counterpart
 * in the paper: this is a convenience of the library.)
 *
 * For callers that cannot allocate device memory or hand one in: for example a right-hand-
 * side or Jacobian-product callback of an ODE or nonlinear solver whose fixed signature has
 * no place for a workspace, or code inside a framework whose memory pool owns the whole
 * device and forbids direct cudaMalloc.  cudaMalloc/cudaFree may also synchronize the device,
 * which a caller in the middle of asynchronous work on several streams must avoid.
 *
 * Same arguments, results and errors as nk_rates_vjp, except that the per-block ln A partial
 * sums go to a fixed scratch array compiled into the library (2^20 doubles = 8 MiB, held on
 * every GPU that loads the library until the process exits).  g_lnA needs one R-vector per
 * block of the VJP's two persistent passes (SMs x resident blocks of each, at most the blocks n
 * needs): on a 152-SM GB300 that allows about 980 reactions with 4 + 3 resident blocks per SM
 * (53 species).  nk_rates_vjp_workspace gives the exact bytes a call
 * needs; above 8 MiB the call returns NK_EUNSUPPORTED and enqueues nothing.  The first call on
 * a device looks up the scratch address on that device (make that first call before any
 * stream capture); later calls read the cached pointer.  The cache lives as long as the
 * process: after cudaDeviceReset (or anything else that destroys the device's primary
 * context) the cached address is stale, so do not call this entry again in that process.
 * All calls share the one scratch array: calls that overlap on the GPU (on different
 * streams, or from different host threads without ordering) race and corrupt each other's
 * g_lnA; order them on one stream.  Every call overwrites the partial sums it reads, so
 * nothing needs clearing between calls.
 */
nk_status nk_rates_vjp_noalloc(const nk_mech* mech, int64_t n, int64_t ld, const double* T,
                               const double* p, const double* Y, const double* dlnA,
                               const double* bar_omega, const double* bar_hrr, double* gT,
                               double* gY, double* g_lnA, nk_stream stream);

/* Message of the last failing call on this host thread ("" if none). */
const char* nk_last_error(void);

/* NKCHEM_VERSION of the built library. */
int32_t nk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NKCHEM_H */
