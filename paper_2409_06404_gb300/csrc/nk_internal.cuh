// Internal declarations of the nkchem CUDA library: device-side mechanism tables, the
// launch interface between the C-ABI layer and the kernels, and device helpers shared by
// the kernels.  Not part of the public ABI (see include/nkchem.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "nkchem.h"
#include "nk_math.cuh"
#include "nk_df.cuh"

namespace nk {

// Physical constants of the evaluated model (SI).
constexpr double kR = 8.314462618;          // molar gas constant, J/(mol K)
constexpr double kInvR = 1.0 / 8.314462618;
constexpr double kP0 = 101325.0;            // standard-state pressure of K_c (1 atm)
constexpr double kLn10 = 2.302585092994045684;
constexpr double kInvLn10 = 0.434294481903251828;

constexpr int kMaxK = 256;
constexpr int kMaxR = 8192;
constexpr int kMaxSide = 4;                 // reactant / product entries per reaction
constexpr int kMaxNu = 8;

// One reaction, read by every thread of a warp at the same address (a broadcast load).
// The device copy orders reactions by kind (elementary, third-body, Troe) so that each kind
// runs in its own branch-free loop; `orig` is the caller's reaction index (for ln A shifts
// and the ln A gradient).
struct __align__(16) RxnRec {
    double lnA;        // ln A (high-pressure limit for Troe)
    double beta;
    double EaR;        // Ea / R, kelvin
    double dnu;        // sum of net stoichiometric coefficients (products - reactants)
    double nud[2 * kMaxSide];   // signed coefficients of the entries as doubles: -nu for
                                // reactants, +nu for products (no int-to-double conversion,
                                // which runs on the FP64 pipe)
    int32_t type;      // NK_RXN_*
    int32_t nr, np;    // reactant / product entry counts
    int32_t aux;       // Troe record index (type 2), else -1
    int32_t orig;      // index of the reaction in the caller's description
    int32_t eff0, eff1;// third-body efficiencies != 1 in [eff0, eff1) of eff_sp / eff_m1
    int32_t thermo;    // thermo groups of the reaction: first (low 24 bits), count (high 8)
    int32_t sp[2 * kMaxSide];   // species of entries: reactants at [0, nr),
                                // products at [kMaxSide, kMaxSide + np)
    int32_t nu[2 * kMaxSide];   // stoichiometric coefficients of the entries
};
static_assert(sizeof(RxnRec) == 192, "reaction record layout");

// Single-precision copy of the Arrhenius data for the mixed form.
struct __align__(16) RxnRecF {
    float lnA, beta, EaR, pad;
};

struct __align__(16) TroeRec {
    double lnA0, beta0, Ea0R;   // low-pressure limit
    double a, invT3, invT1, T2; // broadening parameters (T2 <= 0: term absent)
    double hasT2;               // 1.0 or 0.0
};

struct __align__(16) TroeRecF {
    float lnA0, beta0, Ea0R, a, invT3, invT1, T2, hasT2;
};

// NASA-7 coefficients of one temperature range, with the derived forms the kernels use:
//   c[0..6] = a1..a7; c[7..10] = a2/2, a3/3, a4/4, a5/5 (h/RT);
//   c[11..14] = -a2/2, -a3/6, -a4/12, -a5/20 (g/RT); c[15] unused.
constexpr int kNasaStride = 16;   // per range; species k: [k][2][16] (low, high)

// Reaction thermo groups.  The net coefficients nu_k of a reaction (products minus
// reactants) combine the NASA-7 polynomials of its species into polynomials of the reaction:
// with da_j = sum_k nu_k a_j,k over species that share one T_mid (a group; almost always the
// whole reaction),
//   sum_k nu_k g_k/RT  = da1 (1 - ln T) - da2 T/2 - da3 T^2/6 - da4 T^3/12 - da5 T^4/20 + da6/T - da7,
//   sum_k nu_k h_k/RT  = da1 + da2 T/2 + da3 T^2/3 + da4 T^3/4 + da5 T^4/5 + da6/T,
//   sum_k nu_k cp_k/R  = da1 + da2 T + da3 T^2 + da4 T^3 + da5 T^4,
// each range picked per group by T <= T_mid, as for the species.  Per group and range the
// pairs hold: [0..6] da1, -da2/2, -da3/6, -da4/12, -da5/20, da6, -da7; [7..12] da1, da2/2,
// da3/3, da4/4, da5/5, da6; [13..17] da1..da5.  The kernels then need no per-species g, h or
// c_p in shared memory.
constexpr int kGrpPairs = 18;

// One term of the dense Jacobian assembly from a stored linearization (k_jac.cu): coefficient
// times stored slot, added to position dst of the row.  Entry (k, j) of
// G_kj = sum_r nu_kr (B_rj + L_r (eps_rj - 1)) (the concentration Jacobian of omega_k at fixed
// T, with [M] = p/(RT) + sum_j (eps_j - 1) C_j) goes to dst = j + 1, the row sums
// V_k = sum_r nu_kr A_r to dst = 0 and Lam_k = sum_r nu_kr L_r to dst = K + 1.
struct __align__(16) JacTerm {
    double coef;
    int32_t slot, dst;
};

constexpr int kTroeDf = 4;       // float4 records per Troe reaction in DevMech::troe_df

// Device view of a loaded mechanism (passed by value to every kernel).
struct DevMech {
    int32_t K, R, P;              // species, reactions, species pairs K(K-1)/2
    int32_t n_troe;
    int32_t R_el, R_tb;           // reactions [0, R_el) elementary, [R_el, R_el+R_tb) third-body,
                                  // [R_el+R_tb, R) Troe (device order)
    double p_ref;
    const double* mtab;           // exp/log tables (kMathTabDoubles, see nk_math.cuh)
    const double* invW;           // [K] 1/W
    const double* W;              // [K] W, kg/mol
    const double* Tmid;           // [K]
    const double* nasa;           // [K][2][16]
    const RxnRec* rxn;            // [R]
    const RxnRecF* rxnf;          // [R]
    const TroeRec* troe;          // [n_troe]
    const TroeRecF* troef;        // [n_troe]
    const int32_t* eff_sp;        // third-body efficiencies != 1, ranges given by RxnRec::eff0/eff1:
    const double* eff_m1;         //   species and eps - 1 (all other species have eps = 1)
    // transport
    const double* mu_fit;         // [K][4]
    const double* lam_fit;        // [K][4]
    const double* D_fit;          // [P][4]
    const double* wilkeA;         // [K][K] A_kj = 8^-1/2 (1 + W_k/W_j)^-1/2
    const double* qrtW;           // [K] W^(1/4)
    const double* sqrtW;          // [K] W^(1/2)
    const float* f_mu_fit;        // single-precision copies for the mixed form
    const float* f_lam_fit;
    const float* f_D_fit;
    const float* f_wilkeA;
    const float* f_qrtW;
    const float* f_sqrtW;
    const float* f_invW;
    // double-float tables of the FP64 transport kernel: fits re-expanded in u = ln T - kLnT0
    const float2* df_mu_fit;      // [K][4]
    const float2* df_lam_fit;     // [K][4]
    const float2* df_D_fit;       // [P][4]
    const float2* df_wilkeA;      // [K][K]
    const float2* df_qlnW;        // [K] ln(W)/4
    const float2* df_sqrtW;       // [K]
    const float2* df_exp_tab;     // [128] 2^(j/128)
    const float2* df_log_rc;      // [128] 1/c_j (see nk_math.cuh)
    const float2* df_log_lc;      // [128] -log(1/c_j)
    // double-float tables of the FP64 rates kernel (exponent arithmetic on the FP32 pipe)
    const float2* nasa_df;        // [K][2][8] g/RT coefficients a1, -a2/2, -a3/6, -a4/12, -a5/20, a6, -a7
    const float4* rxn_df;         // [R][2] (lnA, beta) and (Ea/R, dnu, -) as pairs, device order
    const float4* troe_df;        // [n_troe][kTroeDf] (lnA0, beta0), (Ea0/R, 1/T3), (1/T1, T2), (a, 1 - a) as pairs
    const float2* grp_df;         // [groups][2][kGrpPairs] reaction thermo groups (below), pairs
    const double* grp_Tmid;       // [groups] the group's T_mid
    const int32_t* lin_boff;      // [R] first entry slot of each reaction in a stored linearization
    int32_t lin_nb;               // entry slots of all reactions (sum of nr + np)
    // reaction rounds for 2 and 4 parts per point (rates and JVP kernels): rsched[round * NP + q]
    // is part q's reaction (device order) in that round or -1; within a round the parts'
    // reactions share no species; kind g (elementary, third-body, Troe) has rounds
    // [rrnd[g], rrnd[g + 1])
    const int32_t* rsched2;
    const int32_t* rsched4;
    int32_t rrnd2[4], rrnd4[4];
    // the same for the VJP, whose rounds also keep the species with a third-body efficiency apart
    const int32_t* rschedv2;
    const int32_t* rschedv4;
    int32_t rrndv2[4], rrndv4[4];
    // the VJP's logarithmic pass takes the plain rounds above for every kind and defers the
    // [M] cotangents' efficiency terms: each third-body or Troe reaction leaves its Mbar in a
    // per-point slot (round - first round of its kind) * NP + part, and after the kind's rounds
    // species k takes sum Mbar_slot (eps - 1) over the entries [mt_ptr[(g - 1)(K + 1) + k],
    // mt_ptr[(g - 1)(K + 1) + k + 1]) of kind g (1, 2): slots mt_slot, values mt_eps, in round
    // order.  mslots: the slots per point (the larger kind's rounds x NP).
    const int32_t* mt_ptr2;
    const int32_t* mt_ptr4;
    const int32_t* mt_slot2;
    const int32_t* mt_slot4;
    const double* mt_eps2;
    const double* mt_eps4;
    int32_t mslots2, mslots4;
    // single-precision products from an FP32 linearization: signed coefficients of each
    // reaction's entries (RxnRec::nud order, device order), efficiencies - 1 (eff_m1 order),
    // c_p/R coefficients a1..a5 per species and range ([K][2][8], low then high)
    const float* f_nud;           // [R][2 kMaxSide]
    const float* f_eff_m1;
    const float* f_cp;
    // Jacobian assembly: species row k has the terms [jac_row[k], jac_row[k+1]) of jac_term,
    // grouped by destination in increasing order, each group in reaction order
    const int32_t* jac_row;       // [K+1]
    const JacTerm* jac_term;      // [terms]
    // per-reaction stored linearization (k_linc.cu): entry weights nu_e / nu_first of each side
    // (reactants at [0, nr), products at [kMaxSide, kMaxSide + np); nu_first the side's first entry)
    const double* lc_w;           // [R][2 kMaxSide]
    const float2* df_eff_m1;      // efficiencies - 1 as pairs (eff_m1 order)
};

// Centre of the re-expanded transport fits (ln T about 1100 K).
constexpr double kLnT0 = 7.0;

}  // namespace nk

namespace nk {
// A run-time compiled, mechanism-specialised kernel (jit.cu).
struct JitModule {
    void* lib = nullptr;    // cudaLibrary_t
    void* kern = nullptr;   // cudaKernel_t
};
}  // namespace nk

// The opaque handle of the public ABI.
struct nk_mech {
    nk::DevMech d;
    int device;
    void* block;        // single device allocation holding every table
    size_t bytes;
    // the mechanism-specialised rates kernel: source written at load, compiled at first use
    std::string jit_src;
    nk::JitModule jit;
    int jit_state = 0;  // 0 not built, 1 built, -1 failed (jit_err says why)
    std::string jit_err;
    std::mutex jit_mu;
};

namespace nk {

// Launchers (one per kernel family); each returns cudaGetLastError() after the launch.
cudaError_t launch_thermo(const DevMech& m, int64_t n, int64_t ld, const double* T,
                          const double* p, const double* Y, double* cp_mix, double* h_mix,
                          double* Wbar, double* rho, double* cp_k, double* h_k, double* g_k,
                          cudaStream_t s);
// rhs = 1: write the implicit-stage sources instead (omega -> dY/dt, hrr -> dT/dt).
cudaError_t launch_rates(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                         const double* Y, const double* dlnA, double* omega, double* hrr,
                         int precision, cudaStream_t s, int rhs = 0);
cudaError_t launch_transport(const DevMech& m, int64_t n, int64_t ld, const double* T,
                             const double* p, const double* Y, double* mu, double* lam,
                             double* Dmix, int precision, cudaStream_t s);
cudaError_t launch_transport_df(const DevMech& m, int64_t n, int64_t ld, const double* T,
                                const double* p, const double* Y, double* mu, double* lam,
                                double* Dmix, cudaStream_t s);
// rhs = 1: the JVP of the implicit-stage sources (omega, hrr -> dY/dt, dT/dt, both nullable;
// d_omega, d_hrr -> their tangents).
cudaError_t launch_jvp(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* vT, const double* vY,
                       double* omega, double* hrr, double* d_omega, double* d_hrr, cudaStream_t s,
                       int rhs = 0);
size_t vjp_workspace_bytes(const DevMech& m, int64_t n);
size_t reactor_workspace_bytes(const DevMech& m, int64_t n, int krylov_dim, int precond, int linearized);
cudaError_t reactor_step(const DevMech& m, int64_t n, double* T, const double* p, double* Y, double dt,
                         const nk_reactor_opts& o, nk_reactor_stats& st, void* ws, cudaStream_t s);
// Dense Jacobian of the sources from a stored linearization and the sources (k_jac.cu).
cudaError_t launch_rhs_jacobian(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                double* J, int64_t ldJ, cudaStream_t s);
// Block-Jacobi preconditioner (k_jac.cu, k_lu.cu): the blocks P = I - dt diag(w) J diag(1/w)
// with power-of-two row scales, factored (pivot rows and row exponents to piv), and z = P^-1 v
// (z may alias v).  N = K + 1 <= kMaxPrecondN (one block must fit in shared memory).
constexpr int kMaxPrecondN = 160;
cudaError_t launch_precond_setup(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                 int64_t ldf, const double* w, int64_t ldw, double dt, double* F, int32_t* piv,
                                 int64_t ldF, cudaStream_t s);
cudaError_t launch_precond_apply(int N, int64_t n, const double* F, int64_t ldF, const int32_t* piv, int64_t ldq,
                                 const double* v, int64_t ldv, double* z, int64_t ldz, cudaStream_t s);
cudaError_t launch_diffusion(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* D, const double* gradX, double* j, double* Vc,
                             double* hf, cudaStream_t s);
// Rates and transport of host-resident fields, chunked over streams (host_eval.cu).
size_t host_eval_workspace_bytes(const DevMech& m, int64_t chunk);
cudaError_t host_eval(const DevMech& m, int64_t n, const double* T, const double* p, const double* Y, double* omega,
                      double* hrr, double* mu, double* lam, double* Dmix, int precision, int64_t chunk, void* ws,
                      cudaStream_t caller);
// The implicit-stage sources' JVP from a stored linearization and the sources at the state
// (k_lin.cu).
cudaError_t launch_rhs_jvp_linearized(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                      const double* Y, const double* lin, int64_t ldl, const double* fT,
                                      const double* fY, int64_t ldf, const double* vT, const double* vY, double* dfT,
                                      double* dfY, cudaStream_t s);
// Mechanism-specialised rates kernel (jit.cu): source from the host description, NVRTC
// compilation and loading, launch (all-double form, results as nk_rates_eval's).
std::string jit_source(const nk_mech_desc* d);
cudaError_t jit_build(const std::string& src, int device, JitModule& mod, std::string& why);
void jit_unload(JitModule& mod);
cudaError_t jit_launch_rates(const JitModule& mod, const DevMech& m, int device, int64_t n, int64_t ld,
                             const double* T, const double* p, const double* Y, const double* dlnA, double* omega,
                             double* hrr, cudaStream_t s);
// Stored linearization of the rates (k_lin.cu): per-point slots, see lin_slots().
int64_t lin_slots(const DevMech& m);
int64_t lin_slots_f32(const DevMech& m);   // the float format's 32-bit words per point
cudaError_t launch_linearize(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* dlnA, double* lin, int64_t ldl, cudaStream_t s);
cudaError_t launch_jvp_linearized(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                  const double* Y, const double* lin, int64_t ldl, const double* vT,
                                  const double* vY, double* d_omega, double* d_hrr, cudaStream_t s);
// The same linearization rounded to float, and the products from it in single precision
// (results widened to double): rhs = 0 the rates' JVP, rhs = 1 the sources' (fT, fY given).
cudaError_t launch_linearize_f32(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* dlnA, float* lin, int64_t ldl, cudaStream_t s);
cudaError_t launch_jvp_linearized_f32(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                      const double* Y, const float* lin, int64_t ldl, const double* fT,
                                      const double* fY, int64_t ldf, const double* vT, const double* vY,
                                      double* d_T, double* d_Y, cudaStream_t s, int rhs);
// Per-reaction (compact) stored linearization (k_linc.cu): per reaction the rate constants and
// the coefficients of their tangents, per species 1/Y_k and C_k; the concentration products are
// formed again per direction.  omega, hrr: NULL, or also the rates at the state (FP64 form).
// rhs = 1 in the product: the sources' JVP (fT, fY given), as launch_rhs_jvp_linearized.
int64_t linc_slots(const DevMech& m);
cudaError_t launch_linearize_compact(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                     const double* Y, const double* dlnA, double* lin, int64_t ldl, double* omega,
                                     double* hrr, cudaStream_t s);
cudaError_t launch_jvp_linearized_compact(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                          const double* Y, const double* lin, int64_t ldl, const double* fT,
                                          const double* fY, int64_t ldf, const double* vT, const double* vY,
                                          double* d_T, double* d_Y, cudaStream_t s, int rhs);
cudaError_t launch_vjp(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* bar_omega,
                       const double* bar_hrr, double* gT, double* gY, double* g_lnA,
                       void* ws, cudaStream_t s);

// Capacity of the fixed device scratch of nk_rates_vjp_noalloc (8 MiB of doubles).
constexpr size_t kNoallocScratchDoubles = (size_t)1 << 20;
// Device address of that scratch on the current device (looked up once per device).
cudaError_t noalloc_scratch(void** ptr);

// Largest block size in {128, 64, 32} whose per-thread shared-memory scratch
// (bytes_per_thread * block) stays within the budget; 0 if none fits.
int pick_block(size_t bytes_per_thread, size_t budget);
// Block size in {128, 64, 32} that maximises resident threads per SM for a kernel using
// bytes_per_thread of shared memory per thread, fixed_bytes per block and bytes_per_warp per
// warp; 0 if none fits.
int pick_block_occupancy(size_t bytes_per_thread, size_t fixed_bytes, size_t bytes_per_warp = 0);
// Opt a kernel into `bytes` of dynamic shared memory on the current device (cached).
cudaError_t ensure_smem(const void* kernel, size_t bytes);
// Opt-in shared-memory limit per block of the current device.
size_t smem_limit();

// ------------------------------------------------------------------ device helpers
// NASA-7 polynomials of species k at (T, lnT, 1/T); c points at the chosen range.
__device__ __forceinline__ const double* nasa_range(const DevMech& m, int k, double T) {
    const double* base = m.nasa + (size_t)k * 2 * kNasaStride;
    return (T <= __ldg(m.Tmid + k)) ? base : base + kNasaStride;
}
__device__ __forceinline__ double nasa_gRT(const double* c, double T, double lnT, double invT) {
    const double poly = T * fma(T, fma(T, fma(T, __ldg(c + 14), __ldg(c + 13)), __ldg(c + 12)), __ldg(c + 11));
    return fma(__ldg(c + 0), 1.0 - lnT, fma(__ldg(c + 5), invT, poly - __ldg(c + 6)));
}
__device__ __forceinline__ double nasa_hRT(const double* c, double T, double invT) {
    const double poly = T * fma(T, fma(T, fma(T, __ldg(c + 10), __ldg(c + 9)), __ldg(c + 8)), __ldg(c + 7));
    return __ldg(c + 0) + fma(__ldg(c + 5), invT, poly);
}
__device__ __forceinline__ double nasa_cpR(const double* c, double T) {
    return fma(T, fma(T, fma(T, fma(T, __ldg(c + 4), __ldg(c + 3)), __ldg(c + 2)), __ldg(c + 1)), __ldg(c + 0));
}
// d(c_p/R)/dT = a2 + 2 a3 T + 3 a4 T^2 + 4 a5 T^3
__device__ __forceinline__ double nasa_dcpR_dT(const double* c, double T) {
    return fma(T, fma(T, fma(T, 4.0 * __ldg(c + 4), 3.0 * __ldg(c + 3)), 2.0 * __ldg(c + 2)), __ldg(c + 1));
}

// x^nu for a small positive integer nu (uniform across the warp)
__device__ __forceinline__ double ipow(double x, int nu) {
    double r = x;
    for (int j = 1; j < nu; ++j) r *= x;
    return r;
}

}  // namespace nk
