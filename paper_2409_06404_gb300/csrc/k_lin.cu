// Stored linearization of the net production rates: the JVP of (omega_k, heat release) split
// into a pass that evaluates everything that depends on the state only, and a cheap pass per
// direction.  The Newton-Krylov stage of the paper (Sec. 2) asks for several Jacobian-vector
// products at one state (about 7 per step, Sec. 4); when the per-point data fit in device
// memory, the exponentials, thermo polynomials and concentration products are evaluated once.
//
// At fixed p, with tT = dT/T, the tangent of a rate of progress is linear in (tT, dC, d[M]):
//   dq_r = A_r tT + sum_e B_re dC_e + L_r d[M],
// elementary:  A = (q_f - q_r) a_T + q_r D_r,  B_e = k_f dfw/dC_e (reactants), -k_r drv/dC_e
//              (products), with a_T = beta + Ea/(R T) and D_r = sum_k nu_k h_k/RT - sum_k nu_k
//              (d ln k_f = a_T tT, d ln K_c = D_r tT);
// third body:  q = q_c [M]: A, B scaled by [M] and L = q_c;
// Troe:        d ln k_f = a_T tT + a_M d[M] (the falloff chain of the JVP kernel taken for
//              the two unit tangents), A as above with that a_T, L = (q_f - q_r) a_M.
// The concentration derivatives are exclusive products (no division), so zero concentrations
// are exact.  Per direction: dC_k = C_k d rho/rho + rho dY_k/W_k, d[M] = -p/(RT) tT +
// sum (eps - 1) dC, dq_r from the stored coefficients, d omega_k = sum_r nu_kr dq_r and
//   d hrr = -R (dT sum_r q_r (sum_k nu_kr c_p,k/R) + T sum_k (h_k/RT) d omega_k),
// the first sum and h_k/RT also stored.
//
// Per-point slots (double, stored as [slot][ldl] so the points of a warp are contiguous):
//   [0, R)                    A_r (device order)
//   [R, R + NB)               B entries: reaction r at R + lin_boff[r], reactants then products
//   [R + NB, R + NB + R - R_el)  L_r of the third-body and Troe reactions
//   R + NB + R - R_el         sum_r q_r (sum_k nu_kr c_p,k/R)
//   then K slots              h_k/RT
// The linearization pass uses the FP64 form of the rates kernel (exponent chains in
// double-float pairs, the falloff chain in double); the apply pass is plain double.
#include <mutex>
#include <utility>
#include <vector>

#include "nk_lin.cuh"

namespace nk {
namespace {

__host__ __device__ inline int64_t slot_M(const DevMech& m) { return (int64_t)m.R + m.lin_nb; }
__host__ __device__ inline int64_t slot_S(const DevMech& m) { return slot_M(m) + (m.R - m.R_el); }
__host__ __device__ inline int64_t slot_H(const DevMech& m) { return slot_S(m) + 1; }
// the float format: S1 as the two 32-bit words of its double, h_k/RT, one exponent word per
// reaction (the reaction's coefficients are stored scaled by 2^-e_r), then one per species
// (E_k = the largest e_r of the reactions it takes part in, the scale of its tangent sums)
__host__ __device__ inline int64_t slot_H32(const DevMech& m) { return slot_S(m) + 2; }
__host__ __device__ inline int64_t slot_E32(const DevMech& m) { return slot_H32(m) + m.K; }
__host__ __device__ inline int64_t slot_EK32(const DevMech& m) { return slot_E32(m) + m.R; }
constexpr int kNoExp = -2000;                  // E_k of a species without reactions

// prod of p[0..n) (returned) and, in ex[e], the product of all entries but e (n <= 4, uniform)
__device__ __forceinline__ double exclusive_products(const double* p, int n, double* ex) {
    switch (n) {
        case 1:
            ex[0] = 1.0;
            return p[0];
        case 2:
            ex[0] = p[1];
            ex[1] = p[0];
            return p[0] * p[1];
        case 3: {
            const double a = p[0] * p[1];
            ex[0] = p[1] * p[2];
            ex[1] = p[0] * p[2];
            ex[2] = a;
            return a * p[2];
        }
        default: {
            const double a = p[0] * p[1], b = p[2] * p[3];
            ex[0] = p[1] * b;
            ex[1] = p[0] * b;
            ex[2] = a * p[3];
            ex[3] = a * p[2];
            return a * b;
        }
    }
}

// a stored value: as is, or rounded to float (integer operations: no FP64-pipe conversion)
__device__ __forceinline__ void put(double* q, double v) { *q = v; }
__device__ __forceinline__ void put(float* q, double v) { *q = narrow(v); }

// biased exponent field of a double (0 for zero and subnormals)
__device__ __forceinline__ int bexp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7ff); }

// v 2^-e rounded to float, by integer operations on the bits (v's exponent field minus e; below
// the normal float range a signed zero; infinities and NaN as they are)
__device__ __forceinline__ float narrow_scaled(double v, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int field = (int)((b >> 52) & 0x7ff);
    if (field == 0x7ff) return narrow(v);
    const int ex = field - e;
    if (field == 0 || ex < 897) return __uint_as_float((unsigned int)(b >> 32) & 0x80000000u);
    return narrow(__longlong_as_double((long long)((b & ~(0x7ffULL << 52)) | ((unsigned long long)ex << 52))));
}

// The coefficients of reaction r at point i: A (slot r), the entries' B (reactants at Bv[e],
// products at Bv[kMaxSide + e]), L (third-body and Troe).  Double storage as computed; float
// storage scaled by 2^-e_r, e_r the largest binary exponent among them (so they fit the float
// range whatever the reaction's magnitude -- rates of progress of stiff mechanisms span far more
// than it), with e_r in the reaction's exponent word.
template <int BLK, int KIND>
__device__ __forceinline__ void store_coef(const DevMech& m, int r, double* lin, int64_t ldl, int64_t i, int nr,
                                           int np, const int*, int*, double Av, const double* Bv, double Lv) {
    lin[(int64_t)r * ldl + i] = Av;
    double* B = lin + ((int64_t)m.R + __ldg(m.lin_boff + r)) * ldl + i;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        if (e < nr) B[(int64_t)e * ldl] = Bv[e];
        if (e < np) B[(int64_t)(nr + e) * ldl] = Bv[kMaxSide + e];
    }
    if (KIND != 0) lin[(slot_M(m) + (r - m.R_el)) * ldl + i] = Lv;
}

template <int BLK, int KIND>
__device__ __forceinline__ void store_coef(const DevMech& m, int r, float* lin, int64_t ldl, int64_t i, int nr,
                                           int np, const int* sp, int* sE, double Av, const double* Bv, double Lv) {
    int mx = bexp(Av);
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        if (e < nr) mx = max(mx, bexp(Bv[e]));
        if (e < np) mx = max(mx, bexp(Bv[kMaxSide + e]));
    }
    if (KIND != 0) mx = max(mx, bexp(Lv));
    const int er = mx == 0 ? 0 : mx - 1023;           // largest |coefficient| in [1, 2) after scaling
    lin[(int64_t)r * ldl + i] = narrow_scaled(Av, er);
    float* B = lin + ((int64_t)m.R + __ldg(m.lin_boff + r)) * ldl + i;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        if (e < nr) B[(int64_t)e * ldl] = narrow_scaled(Bv[e], er);
        if (e < np) B[(int64_t)(nr + e) * ldl] = narrow_scaled(Bv[kMaxSide + e], er);
    }
    if (KIND != 0) lin[(slot_M(m) + (r - m.R_el)) * ldl + i] = narrow_scaled(Lv, er);
    reinterpret_cast<int32_t*>(lin)[(slot_E32(m) + r) * ldl + i] = er;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {               // the species' scales (parts share them)
        if (e < nr) atomicMax(sE + sp[e] * BLK, er);
        if (e < np) atomicMax(sE + sp[kMaxSide + e] * BLK, er);
    }
}

// ---------------------------------------------------------------- linearization pass
template <int BLK, int KIND, class TS>
__device__ __forceinline__ void lin_reaction(const DevMech& m, int r, const double* sC, const LinPoint& Q,
                                             const double* dlnA, const DfTab& dt, TS* __restrict__ lin,
                                             int64_t ldl, int64_t i, bool live, double& S1, int* sE) {
    const Rxn x = load_rxn(m.rxn + r);
    double cR[kMaxSide], pR[kMaxSide], cP[kMaxSide], pP[kMaxSide];
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        cR[e] = pR[e] = cP[e] = pP[e] = 1.0;
        if (e < x.nr) {
            const double c = sC[x.sp[e] * BLK];
            double pw = c;
            for (int j = 1; j < x.nu[e]; ++j) pw *= c;
            cR[e] = c;
            pR[e] = pw;
        }
        if (e < x.np) {
            const double c = sC[x.sp[kMaxSide + e] * BLK];
            double pw = c;
            for (int j = 1; j < x.nu[kMaxSide + e]; ++j) pw *= c;
            cP[e] = c;
            pP[e] = pw;
        }
    }
    double exR[kMaxSide], exP[kMaxSide];
    const double fw = exclusive_products(pR, x.nr, exR);
    const double rv = exclusive_products(pP, x.np, exP);

    const RateTerms rt = rate_terms<BLK, KIND>(m, r, x, sC, Q, dlnA, dt);
    const double kf = rt.kf, kr = rt.kr, aT = rt.aT, aM = rt.aM, M = rt.M, sumcp = rt.sumcp;
    const double qr = kr * rv;
    const double qc = fma(kf, fw, -qr);
    const double D = rt.D;
    const double sc = KIND == 1 ? M : 1.0;              // third body: q = q_c [M]
    S1 = fma(qc * sc, sumcp, S1);
    if (!live) return;
    double Bv[2 * kMaxSide];
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        Bv[e] = Bv[kMaxSide + e] = 0.0;
        if (e < x.nr) {
            double d = exR[e];                            // d fw / d C_e = nu C_e^(nu-1) prod_{f!=e}
            if (x.nu[e] > 1) {
                d *= -x.nud[e];
                for (int j = 1; j < x.nu[e]; ++j) d *= cR[e];
            }
            Bv[e] = sc * kf * d;
        }
        if (e < x.np) {
            double d = exP[e];
            if (x.nu[kMaxSide + e] > 1) {
                d *= x.nud[kMaxSide + e];
                for (int j = 1; j < x.nu[kMaxSide + e]; ++j) d *= cP[e];
            }
            Bv[kMaxSide + e] = -sc * kr * d;
        }
    }
    store_coef<BLK, KIND>(m, r, lin, ldl, i, x.nr, x.np, x.sp, sE, sc * fma(qc, aT, qr * D), Bv,
                          KIND == 1 ? qc : (KIND == 2 ? qc * aM : 0.0));
}

template <int BLK, int KIND, class TS>
__device__ __forceinline__ void lin_group(const DevMech& m, int r0, int r1, const double* sC, const LinPoint& Q,
                                          const double* dlnA, const DfTab& dt, TS* lin, int64_t ldl, int64_t i,
                                          bool live, double& S1, int* sE) {
    for (int r = r0; r < r1; ++r) lin_reaction<BLK, KIND>(m, r, sC, Q, dlnA, dt, lin, ldl, i, live, S1, sE);
}

// TS: the stored type (double, or float for the single-precision products)
template <int BLK, int NP, class TS>
__global__ void __launch_bounds__(BLK * NP, 512 / (BLK * NP)) linearize_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                             const double* __restrict__ T,
                                                             const double* __restrict__ p,
                                                             const double* __restrict__ Y,
                                                             const double* __restrict__ dlnA,
                                                             TS* __restrict__ lin, const int64_t ldl) {
    constexpr bool F32 = sizeof(TS) == sizeof(float);
    extern __shared__ double smem[];
    const DfTab dt = stage_df_tables(reinterpret_cast<float2*>(smem), m);
    __syncthreads();
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;
    double* sC = smem + kMathTabDoubles + slot;
    // float format: the species' exponent scales E_k (K ints per point after C_k)
    int* sE = F32 ? reinterpret_cast<int*>(smem + kMathTabDoubles + (size_t)K * BLK) + slot : nullptr;

    const double Ti = T[i];
    const LinPoint Q = make_lin_point(Ti, p[i], dt);
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double rho = Q.pRT / s;
    for (int k = part; k < K; k += NP) {
        sC[k * BLK] = Y[(int64_t)k * ld + i] * __ldg(m.invW + k) * rho;
        if (live)
            put(lin + ((F32 ? slot_H32(m) : slot_H(m)) + k) * ldl + i, nasa_hRT(nasa_range(m, k, Ti), Ti, Q.invT));
        if constexpr (F32) sE[k * BLK] = kNoExp;
    }
    if (NP > 1) __syncthreads();

    double S1 = 0.0;
    int a, b;
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    slice<NP>(0, e1, part, a, b);
    lin_group<BLK, 0>(m, a, b, sC, Q, dlnA, dt, lin, ldl, i, live, S1, sE);
    slice<NP>(e1, t1, part, a, b);
    lin_group<BLK, 1>(m, a, b, sC, Q, dlnA, dt, lin, ldl, i, live, S1, sE);
    slice<NP>(t1, m.R, part, a, b);
    lin_group<BLK, 2>(m, a, b, sC, Q, dlnA, dt, lin, ldl, i, live, S1, sE);
    if (NP > 1) __syncthreads();
    if constexpr (F32)
        if (live)
            for (int k = part; k < K; k += NP)
                reinterpret_cast<int32_t*>(lin)[(slot_EK32(m) + k) * ldl + i] = sE[k * BLK];
    if constexpr (NP > 1) {
        sC[part * BLK] = S1;                       // C_k is dead; rows 0..NP-1 (NP <= K)
        __syncthreads();
        if (part != 0) return;
        S1 = sC[0];
#pragma unroll
        for (int q = 1; q < NP; ++q) S1 += sC[q * BLK];
    }
    if (!live) return;
    if constexpr (F32) {                           // S1 in full: the two words of the double
        const unsigned long long b = (unsigned long long)__double_as_longlong(S1);
        reinterpret_cast<uint32_t*>(lin)[slot_S(m) * ldl + i] = (uint32_t)b;
        reinterpret_cast<uint32_t*>(lin)[(slot_S(m) + 1) * ldl + i] = (uint32_t)(b >> 32);
    } else {
        lin[slot_S(m) * ldl + i] = S1;
    }
}

// ---------------------------------------------------------------- apply pass (one direction)
// The stored coefficients of a reaction (A, its entries' B, L): read for the next reaction
// while the current one is contracted, so each warp keeps two reactions' HBM loads in flight.
struct LinCoef {
    double A, L;
    double Br[kMaxSide], Bp[kMaxSide];   // reactant and product entries
};

template <int KIND>
__device__ __forceinline__ LinCoef load_coef(const DevMech& m, int r, const double* __restrict__ lin, int64_t ldl,
                                             int64_t i, int nr, int np) {
    LinCoef c;
    c.A = lin[(int64_t)r * ldl + i];
    const double* B = lin + ((int64_t)m.R + __ldg(m.lin_boff + r)) * ldl + i;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        c.Br[e] = e < nr ? B[(int64_t)e * ldl] : 0.0;
        c.Bp[e] = e < np ? B[(int64_t)(nr + e) * ldl] : 0.0;
    }
    c.L = KIND != 0 ? lin[(slot_M(m) + (r - m.R_el)) * ldl + i] : 0.0;
    return c;
}

// One reaction of the double product pass: dq from its stored coefficients and dC, then its
// scatter into d omega_k.
template <int BLK, int KIND>
__device__ __forceinline__ void apply_one(const DevMech& m, const Rxn& x, const LinCoef& c, const double* sdC,
                                          double* sD, double tT, double dpRT) {
    double dq = c.A * tT;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.nr) dq = fma(c.Br[e], sdC[x.sp[e] * BLK], dq);
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.np) dq = fma(c.Bp[e], sdC[x.sp[kMaxSide + e] * BLK], dq);
    if (KIND != 0) {
        double dM = dpRT;
        for (int j = x.eff0; j < x.eff1; ++j) dM = fma(__ldg(m.eff_m1 + j), sdC[__ldg(m.eff_sp + j) * BLK], dM);
        dq = fma(c.L, dM, dq);
    }
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.nr) {
            double* w = sD + x.sp[e] * BLK;
            *w = fma(x.nud[e], dq, *w);
        }
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.np) {
            double* w = sD + x.sp[kMaxSide + e] * BLK;
            *w = fma(x.nud[kMaxSide + e], dq, *w);
        }
}

struct RxnLin {
    Rxn x;
    LinCoef c;
};

// Reactions [r0, r1) of one kind in order (one part per point).
template <int BLK, int KIND>
__device__ __forceinline__ void apply_group(const DevMech& m, int r0, int r1, const double* sdC, double* sD,
                                            const double* __restrict__ lin, int64_t ldl, int64_t i, double tT,
                                            double dpRT) {
    if (r0 >= r1) return;
    Rxn x = load_rxn(m.rxn + r0);
    LinCoef c = load_coef<KIND>(m, r0, lin, ldl, i, x.nr, x.np);
    for (int r = r0; r < r1; ++r) {
        Rxn xn;
        LinCoef cn;
        if (r + 1 < r1) {
            xn = load_rxn(m.rxn + r + 1);
            cn = load_coef<KIND>(m, r + 1, lin, ldl, i, xn.nr, xn.np);
        }
        apply_one<BLK, KIND>(m, x, c, sdC, sD, tT, dpRT);
        if (r + 1 < r1) {
            x = xn;
            c = cn;
        }
    }
}

// The reactions of one kind for NP > 1 parts per point in the rates kernel's rounds, all parts
// adding into the point's one d omega_k row.
template <int BLK, int NP, int KIND>
__device__ __forceinline__ void apply_rounds(const DevMech& m, int part, const double* sdC, double* sD,
                                             const double* __restrict__ lin, int64_t ldl, int64_t i, double tT,
                                             double dpRT) {
    for_rounds_prefetch<NP>(
        m, KIND, part,
        [&](int r) {
            RxnLin v;
            v.x = load_rxn(m.rxn + r);
            v.c = load_coef<KIND>(m, r, lin, ldl, i, v.x.nr, v.x.np);
            return v;
        },
        [&](int, const RxnLin& v) { apply_one<BLK, KIND>(m, v.x, v.c, sdC, sD, tT, dpRT); });
}

// RHS: the tangent of the implicit-stage sources instead, given the sources fT, fY at the same
// state: dfY_k = (W_k/rho) d omega_k - fY_k d rho/rho, dfT = d hrr/(rho c_p) - fT (d rho/rho +
// d c_p/c_p) (d_omega, d_hrr then receive dfY, dfT).
template <int BLK, int NP, bool RHS>
__global__ void __launch_bounds__(BLK * NP, 512 / (BLK * NP)) jvp_lin_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                           const double* __restrict__ T,
                                                           const double* __restrict__ p,
                                                           const double* __restrict__ Y,
                                                           const double* __restrict__ lin, const int64_t ldl,
                                                           const double* __restrict__ vT,
                                                           const double* __restrict__ vY,
                                                           double* __restrict__ d_omega, double* __restrict__ d_hrr,
                                                           const double* __restrict__ fT,
                                                           const double* __restrict__ fY, const int64_t ldf) {
    extern __shared__ double smem[];
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;
    double* sdC = smem + slot;                                   // dC_k
    double* sD0 = smem + (size_t)K * BLK + slot;                 // d omega_k
    double* sD = sD0;

    const double Ti = T[i], dT = vT[i];
    const double invT = 1.0 / Ti, tT = dT * invT;
    const double pRT = p[i] * invT * kInvR;
    double s = 0.0, ds = 0.0;
    for (int k = 0; k < K; ++k) {
        const double iw = __ldg(m.invW + k);
        s += Y[(int64_t)k * ld + i] * iw;
        ds = fma(vY[(int64_t)k * ld + i], iw, ds);
    }
    const double rho = pRT / s;
    const double arho = -tT - ds / s;                            // d rho / rho
    for (int k = part; k < K; k += NP) {
        const double iw = __ldg(m.invW + k);
        sdC[k * BLK] = fma(Y[(int64_t)k * ld + i] * iw * rho, arho, rho * vY[(int64_t)k * ld + i] * iw);
    }
    for (int k = part; k < K; k += NP) sD[k * BLK] = 0.0;
    if (NP > 1) __syncthreads();

    const double dpRT = -pRT * tT;
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    if constexpr (NP == 1) {
        apply_group<BLK, 0>(m, 0, e1, sdC, sD, lin, ldl, i, tT, dpRT);
        apply_group<BLK, 1>(m, e1, t1, sdC, sD, lin, ldl, i, tT, dpRT);
        apply_group<BLK, 2>(m, t1, m.R, sdC, sD, lin, ldl, i, tT, dpRT);
    } else {
        // (each round ends with a barrier: the row is complete after the last one)
        apply_rounds<BLK, NP, 0>(m, part, sdC, sD, lin, ldl, i, tT, dpRT);
        apply_rounds<BLK, NP, 1>(m, part, sdC, sD, lin, ldl, i, tT, dpRT);
        apply_rounds<BLK, NP, 2>(m, part, sdC, sD, lin, ldl, i, tT, dpRT);
    }

    lin_epilogue<BLK, NP, RHS, 1>(m, part, live, i, Ti, dT, rho, arho, sD0, sdC, lin + slot_H(m) * ldl + i,
                                  lin + slot_S(m) * ldl + i, ldl, Y, vY, ld, fT, fY, ldf, d_omega, d_hrr);
}

// ---------------------------------------------------------------- FP32 apply pass
// The same contraction from the float linearization, on the FP32 pipe (about 60 times the FP64
// pipe's rate on GB300) and from half the bytes: each reaction's dq_r' = dq_r 2^-e_r in single
// precision from its scaled coefficients, scattered into species sums kept at the species'
// scale, omega_k' = sum_r nu_kr dq_r' 2^(e_r - E_k) (powers of two built by integer operations;
// e_r <= E_k, so nothing overflows, and terms below 2^-126 of the species' scale drop out),
// and each sum brought to double with its E_k at the end.  Meant for Krylov solvers whose
// basis is FP32 anyway: the products carry rounding of the order the basis already has.  The
// point terms (rho, d rho/rho, dC_k, c_p) are formed in float from the double inputs, rounded
// by integer operations; the heat-release and source epilogues run in double.
constexpr float kInvRf = (float)(1.0 / 8.314462618);

struct Rxn32 {
    int nr, np, eff0, eff1;
    int sp[2 * kMaxSide];
    float nud[2 * kMaxSide];
};

__device__ __forceinline__ Rxn32 load_rxn32(const DevMech& m, int r) {
    Rxn32 x;
    const int4* q = reinterpret_cast<const int4*>(m.rxn + r) + 6;
    const int4 h = __ldg(q), h2 = __ldg(q + 1), s0 = __ldg(q + 2), s1 = __ldg(q + 3);
    x.nr = h.y;
    x.np = h.z;
    x.eff0 = h2.y;
    x.eff1 = h2.z;
    x.sp[0] = s0.x; x.sp[1] = s0.y; x.sp[2] = s0.z; x.sp[3] = s0.w;
    x.sp[4] = s1.x; x.sp[5] = s1.y; x.sp[6] = s1.z; x.sp[7] = s1.w;
    const float4* f = reinterpret_cast<const float4*>(m.f_nud + (size_t)r * 2 * kMaxSide);
    const float4 a = __ldg(f), b = __ldg(f + 1);
    x.nud[0] = a.x; x.nud[1] = a.y; x.nud[2] = a.z; x.nud[3] = a.w;
    x.nud[4] = b.x; x.nud[5] = b.y; x.nud[6] = b.z; x.nud[7] = b.w;
    return x;
}

struct LinCoef32 {
    float A, L;
    float Br[kMaxSide], Bp[kMaxSide];
    int e;                                  // the reaction's exponent: coefficients x 2^e
};

template <int KIND>
__device__ __forceinline__ LinCoef32 load_coef32(const DevMech& m, int r, const float* __restrict__ lin, int64_t ldl,
                                                 int64_t i, int nr, int np) {
    LinCoef32 c;
    c.A = lin[(int64_t)r * ldl + i];
    const float* B = lin + ((int64_t)m.R + __ldg(m.lin_boff + r)) * ldl + i;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        c.Br[e] = e < nr ? B[(int64_t)e * ldl] : 0.0f;
        c.Bp[e] = e < np ? B[(int64_t)(nr + e) * ldl] : 0.0f;
    }
    c.L = KIND != 0 ? lin[(slot_M(m) + (r - m.R_el)) * ldl + i] : 0.0f;
    c.e = reinterpret_cast<const int32_t*>(lin)[(slot_E32(m) + r) * ldl + i];
    return c;
}

// v 2^e for a double v, by adding e to its exponent field (zero stays zero; the result flushes to
// a signed zero below the normal range and becomes inf above it)
__device__ __forceinline__ double scale2(double v, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int field = (int)((b >> 52) & 0x7ff);
    if (field == 0 || field == 0x7ff) return v;
    const int ex = field + e;
    const unsigned long long sign = b & 0x8000000000000000ULL;
    if (ex <= 0) return __longlong_as_double((long long)sign);
    if (ex >= 0x7ff) return __longlong_as_double((long long)(sign | (0x7ffULL << 52)));
    return __longlong_as_double((long long)((b & ~(0x7ffULL << 52)) | ((unsigned long long)ex << 52)));
}

// 2^d as a float for an integer d <= 0 (zero below -126)
__device__ __forceinline__ float pow2f(int d) { return d >= -126 ? __int_as_float((127 + d) << 23) : 0.0f; }

// One reaction of the single-precision product pass: dq' from its scaled coefficients and dC,
// scattered into the species sums at the species' scales.
template <int BLK, int KIND>
__device__ __forceinline__ void apply_one32(const DevMech& m, const Rxn32& x, const LinCoef32& c, const float* sdC,
                                            float* sD, const int* sE, float tT, float dpRT) {
    float dq = c.A * tT;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.nr) dq = fmaf(c.Br[e], sdC[x.sp[e] * BLK], dq);
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.np) dq = fmaf(c.Bp[e], sdC[x.sp[kMaxSide + e] * BLK], dq);
    if (KIND != 0) {
        float dM = dpRT;
        for (int j = x.eff0; j < x.eff1; ++j) dM = fmaf(__ldg(m.f_eff_m1 + j), sdC[__ldg(m.eff_sp + j) * BLK], dM);
        dq = fmaf(c.L, dM, dq);
    }
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.nr) {
            const int k = x.sp[e] * BLK;
            sD[k] = fmaf(x.nud[e] * pow2f(c.e - sE[k]), dq, sD[k]);
        }
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e)
        if (e < x.np) {
            const int k = x.sp[kMaxSide + e] * BLK;
            sD[k] = fmaf(x.nud[kMaxSide + e] * pow2f(c.e - sE[k]), dq, sD[k]);
        }
}

struct RxnLin32 {
    Rxn32 x;
    LinCoef32 c;
};

// Reactions [r0, r1) of one kind in order (one part per point).
template <int BLK, int KIND>
__device__ __forceinline__ void apply_group32(const DevMech& m, int r0, int r1, const float* sdC, float* sD,
                                              const int* sE, const float* __restrict__ lin, int64_t ldl, int64_t i,
                                              float tT, float dpRT) {
    if (r0 >= r1) return;
    Rxn32 x = load_rxn32(m, r0);
    LinCoef32 c = load_coef32<KIND>(m, r0, lin, ldl, i, x.nr, x.np);
    for (int r = r0; r < r1; ++r) {
        Rxn32 xn;
        LinCoef32 cn;
        if (r + 1 < r1) {
            xn = load_rxn32(m, r + 1);
            cn = load_coef32<KIND>(m, r + 1, lin, ldl, i, xn.nr, xn.np);
        }
        apply_one32<BLK, KIND>(m, x, c, sdC, sD, sE, tT, dpRT);
        if (r + 1 < r1) {
            x = xn;
            c = cn;
        }
    }
}

// The reactions of one kind for NP > 1 parts per point in the rates kernel's rounds, all parts
// adding into the point's one row of scaled sums.
template <int BLK, int NP, int KIND>
__device__ __forceinline__ void apply_rounds32(const DevMech& m, int part, const float* sdC, float* sD,
                                               const int* sE, const float* __restrict__ lin, int64_t ldl, int64_t i,
                                               float tT, float dpRT) {
    for_rounds_prefetch<NP>(
        m, KIND, part,
        [&](int r) {
            RxnLin32 v;
            v.x = load_rxn32(m, r);
            v.c = load_coef32<KIND>(m, r, lin, ldl, i, v.x.nr, v.x.np);
            return v;
        },
        [&](int, const RxnLin32& v) { apply_one32<BLK, KIND>(m, v.x, v.c, sdC, sD, sE, tT, dpRT); });
}

// Shared memory: 3 NP sums per point (double), the row of scaled d omega_k sums, dC_k, E_k
// (4-byte words).
__host__ __device__ constexpr size_t lin32_smem(int K, int blk, int np) {
    return (size_t)3 * np * blk * sizeof(double) + (size_t)3 * K * blk * sizeof(float);
}

template <int BLK, int NP, bool RHS>
__global__ void __launch_bounds__(BLK * NP, 768 / (BLK * NP)) jvp_lin32_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                             const double* __restrict__ T,
                                                             const double* __restrict__ p,
                                                             const double* __restrict__ Y,
                                                             const float* __restrict__ lin, const int64_t ldl,
                                                             const double* __restrict__ vT,
                                                             const double* __restrict__ vY,
                                                             double* __restrict__ d_omega,
                                                             double* __restrict__ d_hrr,
                                                             const double* __restrict__ fT,
                                                             const double* __restrict__ fY, const int64_t ldf) {
    extern __shared__ double smd[];
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;
    double* sR = smd + slot;                                     // part sums
    float* sD0 = reinterpret_cast<float*>(smd + (size_t)3 * NP * BLK) + slot;   // scaled d omega_k sums
    float* sD = sD0;
    float* sdC = sD0 + (size_t)K * BLK;                          // dC_k
    int* sE = reinterpret_cast<int*>(sdC + (size_t)K * BLK);     // E_k
    const int32_t* linE = reinterpret_cast<const int32_t*>(lin) + slot_EK32(m) * ldl + i;

    const double Td = T[i], dTd = vT[i];
    const float Ti = narrow(Td), dT = narrow(dTd);
    const float invT = 1.0f / Ti, tT = dT * invT;
    const float pRT = narrow(p[i]) * invT * kInvRf;
    float s = 0.0f, ds = 0.0f;
    for (int k = 0; k < K; ++k) {
        const float iw = __ldg(m.f_invW + k);
        s = fmaf(narrow(Y[(int64_t)k * ld + i]), iw, s);
        ds = fmaf(narrow(vY[(int64_t)k * ld + i]), iw, ds);
    }
    const float rho = pRT / s;
    const float arho = -tT - ds / s;                             // d rho / rho
    for (int k = part; k < K; k += NP) {
        const float iw = __ldg(m.f_invW + k);
        sdC[k * BLK] = fmaf(narrow(Y[(int64_t)k * ld + i]) * iw * rho, arho, rho * narrow(vY[(int64_t)k * ld + i]) * iw);
        sE[k * BLK] = linE[(int64_t)k * ldl];
    }
    for (int k = part; k < K; k += NP) sD[k * BLK] = 0.0f;
    if (NP > 1) __syncthreads();

    const float dpRT = -pRT * tT;
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    if constexpr (NP == 1) {
        apply_group32<BLK, 0>(m, 0, e1, sdC, sD, sE, lin, ldl, i, tT, dpRT);
        apply_group32<BLK, 1>(m, e1, t1, sdC, sD, sE, lin, ldl, i, tT, dpRT);
        apply_group32<BLK, 2>(m, t1, m.R, sdC, sD, sE, lin, ldl, i, tT, dpRT);
    } else {
        // (each round ends with a barrier: the row is complete after the last one)
        apply_rounds32<BLK, NP, 0>(m, part, sdC, sD, sE, lin, ldl, i, tT, dpRT);
        apply_rounds32<BLK, NP, 1>(m, part, sdC, sD, sE, lin, ldl, i, tT, dpRT);
        apply_rounds32<BLK, NP, 2>(m, part, sdC, sD, sE, lin, ldl, i, tT, dpRT);
    }

    double hsum = 0.0;
    float cpm = 0.0f, dcpm = 0.0f;
    const float inv_rho = RHS ? 1.0f / rho : 0.0f;
    const double arho_d = widen(arho);
    for (int k = part; k < K; k += NP) {
        const float dws = sD0[k * BLK];
        double dw = scale2(widen(dws), sE[k * BLK]);
        hsum = fma(widen(lin[(slot_H32(m) + k) * ldl + i]), dw, hsum);
        if constexpr (RHS) {
            // NASA range on the doubles' bit patterns (T, T_mid > 0), as the double kernels choose it
            const bool lo = __double_as_longlong(Td) <= __ldg(reinterpret_cast<const long long*>(m.Tmid) + k);
            const float* cf = m.f_cp + ((size_t)k * 2 + (lo ? 0 : 1)) * 8;
            const float4 c = __ldg(reinterpret_cast<const float4*>(cf));
            const float a5 = __ldg(cf + 4);
            const float cpk = fmaf(Ti, fmaf(Ti, fmaf(Ti, fmaf(Ti, a5, c.w), c.z), c.y), c.x);
            const float dcpk = fmaf(Ti, fmaf(Ti, fmaf(Ti, 4.0f * a5, 3.0f * c.w), 2.0f * c.z), c.y);
            const float iw = __ldg(m.f_invW + k);
            const float yk = narrow(Y[(int64_t)k * ld + i]) * iw, vk = narrow(vY[(int64_t)k * ld + i]) * iw;
            cpm = fmaf(yk, cpk, cpm);
            dcpm = fmaf(vk, cpk, fmaf(yk * dcpk, dT, dcpm));
            dw = fma(widen(inv_rho / iw), dw, -fY[(int64_t)k * ldf + i] * arho_d);
        }
        if (live) d_omega[(int64_t)k * ld + i] = dw;
    }
    if constexpr (NP > 1) {
        sR[part * BLK] = hsum;
        if constexpr (RHS) {
            sR[(NP + part) * BLK] = widen(cpm);
            sR[(2 * NP + part) * BLK] = widen(dcpm);
        }
        __syncthreads();
        if (part != 0) return;
        hsum = sR[0];
        double cpd = RHS ? sR[NP * BLK] : 0.0, dcpd = RHS ? sR[2 * NP * BLK] : 0.0;
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            hsum += sR[q * BLK];
            if constexpr (RHS) {
                cpd += sR[(NP + q) * BLK];
                dcpd += sR[(2 * NP + q) * BLK];
            }
        }
        cpm = narrow(cpd);
        dcpm = narrow(dcpd);
    }
    if (live) {
        const uint32_t lo = reinterpret_cast<const uint32_t*>(lin)[slot_S(m) * ldl + i];
        const uint32_t hi = reinterpret_cast<const uint32_t*>(lin)[(slot_S(m) + 1) * ldl + i];
        const double S1 = __hiloint2double((int)hi, (int)lo);
        const double dhr = -kR * fma(dTd, S1, Td * hsum);
        if constexpr (RHS)
            d_hrr[i] = fma(dhr, widen(inv_rho / (8.314462618f * cpm)), -fT[i] * widen(arho + dcpm / cpm));
        else
            d_hrr[i] = dhr;
    }
}

// ---------------------------------------------------------------- launch shapes
struct Shape {
    int blk, np;
};
constexpr Shape kShapes[] = {{32, 1}, {64, 1}, {128, 1}, {32, 2}, {64, 2}, {32, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// MODE 0: the linearization pass; 1: the JVP from it; 2: the sources' JVP from it; 3, 4: the
// same two in single precision from 5: the linearization rounded to float
template <int MODE, int S>
constexpr auto kernel_of() {
    if constexpr (MODE == 1)
        return jvp_lin_kernel<kShapes[S].blk, kShapes[S].np, false>;
    else if constexpr (MODE == 2)
        return jvp_lin_kernel<kShapes[S].blk, kShapes[S].np, true>;
    else if constexpr (MODE == 3)
        return jvp_lin32_kernel<kShapes[S].blk, kShapes[S].np, false>;
    else if constexpr (MODE == 4)
        return jvp_lin32_kernel<kShapes[S].blk, kShapes[S].np, true>;
    else if constexpr (MODE == 5)
        return linearize_kernel<kShapes[S].blk, kShapes[S].np, float>;
    else
        return linearize_kernel<kShapes[S].blk, kShapes[S].np, double>;
}

template <int MODE, int... S>
const void* kernel_ptr(int idx, std::integer_sequence<int, S...>) {
    const void* ptrs[] = {(const void*)kernel_of<MODE, S>()...};
    return ptrs[idx];
}

// linearization: the pair tables and C_k; apply: dC_k and the d omega_k row (and the part sums
// of the single-precision apply)
size_t lin_smem(int K, const Shape& sh, int mode) {
    if (mode == 0 || mode == 5)
        return (size_t)kMathTabDoubles * sizeof(double) + (size_t)K * sh.blk * (mode == 5 ? 12 : 8);
    if (mode == 3 || mode == 4) return lin32_smem(K, sh.blk, sh.np);
    return (size_t)2 * K * sh.blk * sizeof(double);
}

struct Plan {
    int dev, K, mode;
    int idx;
};
std::mutex g_plan_mu;
std::vector<Plan> g_plans;

template <int MODE>
int plan_shape(int K) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (const Plan& q : g_plans)
            if (q.dev == dev && q.K == K && q.mode == MODE) return q.idx;
    }
    int per_block = 0;
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = -1, best_warps = 0;
    for (int c = 0; c < kNumShapes; ++c) {
        const Shape& sh = kShapes[c];
        if ((MODE == 2 ? 3 : 1) * sh.np > K) continue;
        const size_t bytes = lin_smem(K, sh, MODE);
        if (bytes > (size_t)per_block) continue;
        const void* kern = kernel_ptr<MODE>(c, std::make_integer_sequence<int, kNumShapes>{});
        if (ensure_smem(kern, bytes) != cudaSuccess) continue;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, sh.blk * sh.np, bytes) != cudaSuccess)
            continue;
        const int warps = blocks * sh.blk * sh.np / 32;
        if (warps > best_warps) {
            best_warps = warps;
            best = c;
        }
    }
    if (best >= 0) {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        g_plans.push_back({dev, K, MODE, best});
    }
    return best;
}

template <int MODE, class... Args, int... S>
cudaError_t launch_idx(int idx, std::integer_sequence<int, S...>, int K, int64_t n, cudaStream_t st,
                       Args... args) {
    cudaError_t e = cudaErrorInvalidConfiguration;
    ((S == idx ? (void)(e = [&] {
        constexpr Shape sh = kShapes[S];
        auto kern = kernel_of<MODE, S>();
        const size_t smem = lin_smem(K, sh, MODE);
        cudaError_t r = ensure_smem((const void*)kern, smem);
        if (r != cudaSuccess) return r;
        kern<<<(unsigned)((n + sh.blk - 1) / sh.blk), sh.blk * sh.np, smem, st>>>(args...);
        return cudaGetLastError();
    }())
               : (void)0),
     ...);
    return e;
}

}  // namespace

int64_t lin_slots(const DevMech& m) { return slot_H(m) + m.K; }
int64_t lin_slots_f32(const DevMech& m) { return slot_EK32(m) + m.K; }

cudaError_t launch_linearize(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* dlnA, double* lin, int64_t ldl, cudaStream_t s) {
    static_assert(kDfTabBytes <= kMathTabDoubles * sizeof(double), "table space");
    const int idx = plan_shape<0>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx<0>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, dlnA,
                         lin, ldl);
}

cudaError_t launch_jvp_linearized(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                  const double* Y, const double* lin, int64_t ldl, const double* vT,
                                  const double* vY, double* d_omega, double* d_hrr, cudaStream_t s) {
    const int idx = plan_shape<1>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    const double* none = nullptr;
    return launch_idx<1>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, lin, ldl,
                         vT, vY, d_omega, d_hrr, none, none, (int64_t)0);
}

cudaError_t launch_linearize_f32(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* dlnA, float* lin, int64_t ldl, cudaStream_t s) {
    const int idx = plan_shape<5>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx<5>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, dlnA,
                         lin, ldl);
}

cudaError_t launch_jvp_linearized_f32(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                      const double* Y, const float* lin, int64_t ldl, const double* fT,
                                      const double* fY, int64_t ldf, const double* vT, const double* vY,
                                      double* d_T, double* d_Y, cudaStream_t s, int rhs) {
    if (rhs) {
        const int idx = plan_shape<4>(m.K);
        if (idx < 0) return cudaErrorInvalidConfiguration;
        return launch_idx<4>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, lin,
                             ldl, vT, vY, d_Y, d_T, fT, fY, ldf);
    }
    const int idx = plan_shape<3>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    const double* none = nullptr;
    return launch_idx<3>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, lin, ldl,
                         vT, vY, d_Y, d_T, none, none, (int64_t)0);
}

cudaError_t launch_rhs_jvp_linearized(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                      const double* Y, const double* lin, int64_t ldl, const double* fT,
                                      const double* fY, int64_t ldf, const double* vT, const double* vY, double* dfT,
                                      double* dfY, cudaStream_t s) {
    const int idx = plan_shape<2>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    return launch_idx<2>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, lin, ldl,
                         vT, vY, dfY, dfT, fT, fY, ldf);
}

}  // namespace nk
