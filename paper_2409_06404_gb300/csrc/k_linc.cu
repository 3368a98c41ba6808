// Per-reaction ("compact") stored linearization of the net production rates.  Like k_lin.cu it
// splits the JVP of (omega_k, heat release) into a pass over the state-only terms and a cheap
// pass per direction, for the several products a Newton-Krylov stage forms at one state (Sec. 2;
// about 7 per step, Sec. 4); but it keeps per point only what each reaction needs, not one
// coefficient per reaction entry: about half the bytes, so that the stored data of a
// 16.8M-point field of a 53-species mechanism fit beside the field in device memory.
//
// At fixed p, with tT = dT/T and the logarithmic tangents of the concentrations
//   r_k = dC_k / C_k = d rho/rho + dY_k / Y_k,
// the tangent of a rate of progress q_r = F_r (k_f prod C^nu' - k_r prod C^nu'') is
//   dq_r = A_r tT + F_r k_f prod C^nu' sum_{reactants} nu_e r_e
//                 - F_r k_r prod C^nu'' sum_{products} nu_e r_e + L_r d[M],
// (F_r = [M] for third-body reactions, else 1; A_r, L_r as in the per-entry form:
// A = F ((q_f - q_r) a_T + q_r D), L = q_c for third-body and q_c a_M for Troe reactions), since
// d(prod C^nu) = prod C^nu sum nu dC/C.  Where a mass fraction of a side is zero or tiny
// (|Y_e| < 2^-200, zero, or not finite) the logarithmic form does not apply: such a side keeps
// F k without the concentration product and the product pass forms its tangent by exclusive
// products of C_e^nu_e and dC_e (exact at C_e = 0, as the recomputing JVP), so absent species
// and pure mixtures stay exact.  The per-direction work is then one gather per entry (a sum of
// r_e), one multiply-add per side and the scatter: no concentration product is formed again.
//
// Per-point slots (double, [slot][ldl], the points of a warp contiguous):
//   [0, R)              A_r (device order)
//   [R, 2R)             V^f_r = F k_f prod C^nu' nu_1 (nu_1: the first reactant's coefficient;
//                       the sum then runs over nu_e/nu_1 weights, 1 for the first), or F k_f
//                       for a side with a tiny mass fraction
//   [2R, 3R)            V^b_r = -F k_r prod C^nu'' nu_1, likewise for the products
//   [3R, 4R - R_el)     L_r of the third-body and Troe reactions
//   4R - R_el           S1 = sum_r q_r (sum_k nu_kr c_p,k/R)
//   then K slots        h_k/RT
//   then K slots        1/Y_k (a quiet NaN for a tiny, zero or non-finite Y_k)
//   then K slots        C_k
// The linearization pass takes the FP64 form's arithmetic (rate_terms: exponent chains in
// double-float pairs); it can also write omega_k and the heat release at the state.  The
// product pass is plain double.
#include <mutex>
#include <utility>
#include <vector>

#include "nk_lin.cuh"

namespace nk {
namespace {

__host__ __device__ inline int64_t cs_Vf(const DevMech& m) { return m.R; }
__host__ __device__ inline int64_t cs_Vb(const DevMech& m) { return 2 * (int64_t)m.R; }
__host__ __device__ inline int64_t cs_L(const DevMech& m) { return 3 * (int64_t)m.R; }
__host__ __device__ inline int64_t cs_S(const DevMech& m) { return cs_L(m) + (m.R - m.R_el); }
__host__ __device__ inline int64_t cs_H(const DevMech& m) { return cs_S(m) + 1; }
__host__ __device__ inline int64_t cs_iY(const DevMech& m) { return cs_H(m) + m.K; }
__host__ __device__ inline int64_t cs_C(const DevMech& m) { return cs_iY(m) + m.K; }

// |y| < 2^-200, zero, subnormal, infinite or NaN: on the exponent field (integer operations)
__device__ __forceinline__ bool tiny_y(double y) {
    const unsigned e = (unsigned)(__double_as_longlong(y) >> 52) & 0x7ffu;
    return e < 1023u - 200u || e == 0x7ffu;
}
// NaN or infinite (an exponent field of all ones)
__device__ __forceinline__ bool nonfinite(double v) {
    return ((unsigned)__double2hiint(v) & 0x7ff00000u) == 0x7ff00000u;
}
__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000LL); }

// ---------------------------------------------------------------- linearization pass
template <int BLK, int KIND, bool OUT>
__device__ __forceinline__ void linc_reaction(const DevMech& m, int r, const double* sC, const uint8_t* sTiny,
                                              double* sW, const LinPoint& Q, const double* dlnA, const DfTab& dt,
                                              double* __restrict__ lin, int64_t ldl, int64_t i, bool live,
                                              double& S1) {
    const Rxn x = load_rxn(m.rxn + r);
    double fw = 1.0, rv = 1.0;
    bool tf = false, tb = false;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        if (e < x.nr) {
            fw *= ipow(sC[x.sp[e] * BLK], x.nu[e]);
            tf |= sTiny[x.sp[e] * BLK] != 0;
        }
        if (e < x.np) {
            rv *= ipow(sC[x.sp[kMaxSide + e] * BLK], x.nu[kMaxSide + e]);
            tb |= sTiny[x.sp[kMaxSide + e] * BLK] != 0;
        }
    }
    const RateTerms rt = rate_terms<BLK, KIND>(m, r, x, sC, Q, dlnA, dt);
    const double qr = rt.kr * rv;
    const double qc = fma(rt.kf, fw, -qr);
    const double sc = KIND == 1 ? rt.M : 1.0;              // third body: q = q_c [M]
    S1 = fma(qc * sc, rt.sumcp, S1);
    if constexpr (OUT) {
        const double q = qc * sc;
        scatter_side<BLK>(x.sp, x.nud, x.nr, sW, q);
        scatter_side<BLK>(x.sp + kMaxSide, x.nud + kMaxSide, x.np, sW, q);
    }
    if (!live) return;
    const double skf = sc * rt.kf, skr = sc * rt.kr;
    lin[(int64_t)r * ldl + i] = sc * fma(qc, rt.aT, qr * rt.D);
    lin[(cs_Vf(m) + r) * ldl + i] = tf ? skf : skf * fw * (-x.nud[0]);
    lin[(cs_Vb(m) + r) * ldl + i] = tb ? -skr : -(skr * rv * x.nud[kMaxSide]);
    if (KIND != 0) lin[(cs_L(m) + (r - m.R_el)) * ldl + i] = KIND == 1 ? qc : qc * rt.aM;
}

template <int BLK, int KIND, bool OUT>
__device__ __forceinline__ void linc_group(const DevMech& m, int r0, int r1, const double* sC, const uint8_t* sTiny,
                                           double* sW, const LinPoint& Q, const double* dlnA, const DfTab& dt,
                                           double* lin, int64_t ldl, int64_t i, bool live, double& S1) {
    for (int r = r0; r < r1; ++r)
        linc_reaction<BLK, KIND, OUT>(m, r, sC, sTiny, sW, Q, dlnA, dt, lin, ldl, i, live, S1);
}

// Shared memory: pair tables, C_k, with OUT NP rows of omega_k partials, and one byte per
// species for the tiny flags.
__host__ __device__ constexpr size_t linc_smem(int K, int blk, int np, bool out) {
    return (size_t)kMathTabDoubles * sizeof(double) + (size_t)(1 + (out ? np : 0)) * K * blk * sizeof(double) +
           (size_t)K * blk;
}

template <int BLK, int NP, bool OUT>
__global__ void __launch_bounds__(BLK * NP) linc_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                        const double* __restrict__ T, const double* __restrict__ p,
                                                        const double* __restrict__ Y,
                                                        const double* __restrict__ dlnA, double* __restrict__ lin,
                                                        const int64_t ldl, double* __restrict__ omega,
                                                        double* __restrict__ hrr) {
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
    double* sW0 = smem + kMathTabDoubles + (size_t)K * BLK + slot;          // OUT: omega_k partials
    double* sW = sW0 + (size_t)part * K * BLK;
    uint8_t* sTiny = reinterpret_cast<uint8_t*>(smem + kMathTabDoubles + (size_t)(1 + (OUT ? NP : 0)) * K * BLK) + slot;

    const double Ti = T[i];
    const LinPoint Q = make_lin_point(Ti, p[i], dt);
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += Y[(int64_t)k * ld + i] * __ldg(m.invW + k);
    const double rho = Q.pRT / s;
    for (int k = part; k < K; k += NP) {
        const double y = Y[(int64_t)k * ld + i];
        const double c = y * __ldg(m.invW + k) * rho;
        const bool tiny = tiny_y(y);
        sC[k * BLK] = c;
        sTiny[k * BLK] = tiny ? 1 : 0;
        if (live) {
            lin[(cs_H(m) + k) * ldl + i] = nasa_hRT(nasa_range(m, k, Ti), Ti, Q.invT);
            lin[(cs_iY(m) + k) * ldl + i] = tiny ? qnan() : 1.0 / y;
            lin[(cs_C(m) + k) * ldl + i] = c;
        }
    }
    if constexpr (OUT)
        for (int k = 0; k < K; ++k) sW[k * BLK] = 0.0;
    if (NP > 1) __syncthreads();

    double S1 = 0.0;
    int a, b;
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    slice<NP>(0, e1, part, a, b);
    linc_group<BLK, 0, OUT>(m, a, b, sC, sTiny, sW, Q, dlnA, dt, lin, ldl, i, live, S1);
    slice<NP>(e1, t1, part, a, b);
    linc_group<BLK, 1, OUT>(m, a, b, sC, sTiny, sW, Q, dlnA, dt, lin, ldl, i, live, S1);
    slice<NP>(t1, m.R, part, a, b);
    linc_group<BLK, 2, OUT>(m, a, b, sC, sTiny, sW, Q, dlnA, dt, lin, ldl, i, live, S1);
    if (NP > 1) __syncthreads();

    // omega_k (partials in part order) and the heat release -R T sum_k (h_k/RT) omega_k
    double hsum = 0.0;
    if constexpr (OUT) {
        for (int k = part; k < K; k += NP) {
            double w = sW0[k * BLK];
#pragma unroll
            for (int q = 1; q < NP; ++q) w += sW0[((size_t)q * K + k) * BLK];
            hsum = fma(nasa_hRT(nasa_range(m, k, Ti), Ti, Q.invT), w, hsum);
            if (live) omega[(int64_t)k * ld + i] = w;
        }
    }
    if constexpr (NP > 1) {
        // C_k is dead: rows q and NP + q take part q's S1 and heat-release sums (2 NP <= K)
        sC[part * BLK] = S1;
        if constexpr (OUT) sC[(NP + part) * BLK] = hsum;
        __syncthreads();
        if (part != 0) return;
        S1 = sC[0];
        if constexpr (OUT) hsum = sC[NP * BLK];
#pragma unroll
        for (int q = 1; q < NP; ++q) {
            S1 += sC[q * BLK];
            if constexpr (OUT) hsum += sC[(NP + q) * BLK];
        }
    }
    if (!live) return;
    lin[cs_S(m) * ldl + i] = S1;
    if constexpr (OUT) hrr[i] = -kR * Ti * hsum;
}

// ---------------------------------------------------------------- product pass (one direction)
// The fields of a reaction record the product pass holds (species, signed coefficients, entry
// counts, efficiency range): two reactions' worth stay in registers.
struct RxnC {
    int nr, np, eff0, eff1;
    int sp[2 * kMaxSide];
    double nud[2 * kMaxSide];
};

__device__ __forceinline__ RxnC load_rxnc(const RxnRec* rec) {
    RxnC x;
    const double2* d = reinterpret_cast<const double2*>(rec);
#pragma unroll
    for (int j = 0; j < kMaxSide; ++j) {
        const double2 v = __ldg(d + 2 + j);
        x.nud[2 * j] = v.x;
        x.nud[2 * j + 1] = v.y;
    }
    const int4* q = reinterpret_cast<const int4*>(rec) + 6;
    const int4 h = __ldg(q), h2 = __ldg(q + 1), s0 = __ldg(q + 2), s1 = __ldg(q + 3);
    x.nr = h.y;
    x.np = h.z;
    x.eff0 = h2.y;
    x.eff1 = h2.z;
    x.sp[0] = s0.x; x.sp[1] = s0.y; x.sp[2] = s0.z; x.sp[3] = s0.w;
    x.sp[4] = s1.x; x.sp[5] = s1.y; x.sp[6] = s1.z; x.sp[7] = s1.w;
    return x;
}

struct CoefC {
    double A, Vf, Vb, L;
};

template <int KIND>
__device__ __forceinline__ CoefC load_coefc(const DevMech& m, int r, const double* __restrict__ lin, int64_t ldl,
                                            int64_t i) {
    CoefC c;
    c.A = lin[(int64_t)r * ldl + i];
    c.Vf = lin[(cs_Vf(m) + r) * ldl + i];
    c.Vb = lin[(cs_Vb(m) + r) * ldl + i];
    c.L = KIND != 0 ? lin[(cs_L(m) + (r - m.R_el)) * ldl + i] : 0.0;
    return c;
}

// The point's state for the exact sides and the tiny species of the efficiency sums.
struct ExactCtx {
    const double* C;     // stored C_k of the point: C[k ldl]
    const double* vY;    // direction of the point: vY[k ld]
    int64_t ldl, ld;
    double rho, arho;
};

// dC_k = C_k d rho/rho + rho dY_k / W_k (as the recomputing JVP forms it)
__device__ __forceinline__ double dconc(const double* __restrict__ invW, int k, const ExactCtx& c) {
    return fma(c.C[(int64_t)k * c.ldl], c.arho, c.rho * c.vY[(int64_t)k * c.ld] * __ldg(invW + k));
}

// The tangent of prod_e C_e^nu_e over one side (ne <= 4 entries) by exclusive products: exact
// where a C_e is zero.  Out of line: only points with tiny mass fractions take it.
__device__ __noinline__ double side_tangent_exact(const double* __restrict__ invW, int ne, int4 sp, int4 nu,
                                                  ExactCtx c) {
    const int s4[kMaxSide] = {sp.x, sp.y, sp.z, sp.w}, n4[kMaxSide] = {nu.x, nu.y, nu.z, nu.w};
    double pw[kMaxSide], dp[kMaxSide];
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        pw[e] = 1.0;
        dp[e] = 0.0;
        if (e < ne) {
            const double ce = c.C[(int64_t)s4[e] * c.ldl];
            double d = 1.0;                                  // nu C^(nu-1)
            for (int j = 1; j < n4[e]; ++j) d *= ce;
            dp[e] = d * (double)n4[e] * dconc(invW, s4[e], c);
            pw[e] = d * ce;
        }
    }
    double t = 0.0;
#pragma unroll
    for (int e = 0; e < kMaxSide; ++e) {
        if (e >= ne) continue;
        double ex = dp[e];
#pragma unroll
        for (int f = 0; f < kMaxSide; ++f)
            if (f != e && f < ne) ex *= pw[f];
        t += ex;
    }
    return t;
}

// sum_e w_e r_e over one side (w_0 = 1, w_e = nu_e/nu_0: the stored V carries nu_0); a switch on
// the entry count with each case unrolled exactly (no predicated-off FP64 instructions)
template <int BLK, int N>
__device__ __forceinline__ double side_sum_n(const double* w, const double* sR, const int* sp) {
    double g = sR[sp[0] * BLK];
#pragma unroll
    for (int e = 1; e < N; ++e) g = fma(__ldg(w + e), sR[sp[e] * BLK], g);
    return g;
}
template <int BLK>
__device__ __forceinline__ double side_sum(const DevMech& m, int r, int side, const double* sR, const int* sp,
                                           int ne) {
    const double* w = m.lc_w + ((size_t)r * 2 + side) * kMaxSide;
    switch (ne) {
        case 1: return sR[sp[0] * BLK];
        case 2: return side_sum_n<BLK, 2>(w, sR, sp);
        case 3: return side_sum_n<BLK, 3>(w, sR, sp);
        default: return side_sum_n<BLK, kMaxSide>(w, sR, sp);
    }
}

// One side's contribution V g, or, where g is not finite, the exact tangent of a side with a tiny
// mass fraction (when a 1/Y_e of it is NaN: V then holds F k) -- else V g as it is (a non-finite
// direction or state).  The coefficients nu_e are read from the reaction record (rare path).
__device__ __forceinline__ double side_term(const DevMech& m, int r, int side, double V, double g, int ne,
                                            const int* sp, const double* __restrict__ iY, const ExactCtx& c) {
    if (!nonfinite(g)) return V * g;
    bool tiny = false;
    for (int e = 0; e < ne; ++e) tiny |= nonfinite(iY[(int64_t)sp[e] * c.ldl]);
    if (!tiny) return V * g;
    const int4 nu = __ldg(reinterpret_cast<const int4*>(m.rxn + r) + 10 + side);
    return V * side_tangent_exact(m.invW, ne, make_int4(sp[0], sp[1], sp[2], sp[3]), nu, c);
}

template <int BLK, int KIND>
__device__ __forceinline__ void applyc_group(const DevMech& m, int r0, int r1, const double* sR, double* sD,
                                             const double* __restrict__ lin, int64_t ldl, int64_t i, double tT,
                                             double dpRT, const double* __restrict__ iY, const ExactCtx& ec) {
    if (r0 >= r1) return;
    RxnC x = load_rxnc(m.rxn + r0);
    CoefC c = load_coefc<KIND>(m, r0, lin, ldl, i);
    for (int r = r0; r < r1; ++r) {
        RxnC xn;
        CoefC cn;
        if (r + 1 < r1) {                          // the next reaction's loads in flight
            xn = load_rxnc(m.rxn + r + 1);
            cn = load_coefc<KIND>(m, r + 1, lin, ldl, i);
        }
        const double gf = side_sum<BLK>(m, r, 0, sR, x.sp, x.nr);
        const double gb = side_sum<BLK>(m, r, 1, sR, x.sp + kMaxSide, x.np);
        double dq;
        if (!nonfinite(gf) && !nonfinite(gb)) {
            dq = fma(c.Vf, gf, fma(c.Vb, gb, c.A * tT));
        } else {
            dq = c.A * tT + side_term(m, r, 0, c.Vf, gf, x.nr, x.sp, iY, ec) +
                 side_term(m, r, 1, c.Vb, gb, x.np, x.sp + kMaxSide, iY, ec);
        }
        if (KIND != 0) {
            double dM = dpRT;
            for (int j = x.eff0; j < x.eff1; ++j) {
                const int k = __ldg(m.eff_sp + j);
                const double rk = sR[k * BLK];
                const double dC = nonfinite(rk) ? dconc(m.invW, k, ec) : ec.C[(int64_t)k * ldl] * rk;
                dM = fma(__ldg(m.eff_m1 + j), dC, dM);
            }
            dq = fma(c.L, dM, dq);
        }
        scatter_side<BLK>(x.sp, x.nud, x.nr, sD, dq);
        scatter_side<BLK>(x.sp + kMaxSide, x.nud + kMaxSide, x.np, sD, dq);
        if (r + 1 < r1) {
            x = xn;
            c = cn;
        }
    }
}

// Shared memory: r_k and NP rows of d omega_k partials per point.
__host__ __device__ constexpr size_t jvpc_smem(int K, int blk, int np) {
    return (size_t)(1 + np) * K * blk * sizeof(double);
}

template <int BLK, int NP, bool RHS>
__global__ void __launch_bounds__(BLK * NP) jvpc_kernel(const DevMech m, const int64_t n, const int64_t ld,
                                                        const double* __restrict__ T, const double* __restrict__ p,
                                                        const double* __restrict__ Y,
                                                        const double* __restrict__ lin, const int64_t ldl,
                                                        const double* __restrict__ vT,
                                                        const double* __restrict__ vY, double* __restrict__ d_omega,
                                                        double* __restrict__ d_hrr, const double* __restrict__ fT,
                                                        const double* __restrict__ fY, const int64_t ldf) {
    extern __shared__ double smem[];
    const int K = m.K;
    const int slot = threadIdx.x % BLK, part = threadIdx.x / BLK;
    const int64_t i0 = (int64_t)blockIdx.x * BLK + slot;
    if (NP == 1 && i0 >= n) return;              // (NP = 1 has no barrier below)
    const bool live = i0 < n;
    const int64_t i = live ? i0 : n - 1;
    double* sR = smem + slot;                                    // r_k
    double* sD0 = smem + (size_t)K * BLK + slot;                 // d omega_k partials, part q at row q
    double* sD = sD0 + (size_t)part * K * BLK;
    const double* iY = lin + cs_iY(m) * ldl + i;

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
    for (int k = part; k < K; k += NP) sR[k * BLK] = fma(vY[(int64_t)k * ld + i], iY[(int64_t)k * ldl], arho);
    for (int k = 0; k < K; ++k) sD[k * BLK] = 0.0;
    if (NP > 1) __syncthreads();

    const ExactCtx ec{lin + cs_C(m) * ldl + i, vY + i, ldl, ld, rho, arho};
    const double dpRT = -pRT * tT;
    int a, b;
    const int e1 = m.R_el, t1 = m.R_el + m.R_tb;
    slice<NP>(0, e1, part, a, b);
    applyc_group<BLK, 0>(m, a, b, sR, sD, lin, ldl, i, tT, dpRT, iY, ec);
    slice<NP>(e1, t1, part, a, b);
    applyc_group<BLK, 1>(m, a, b, sR, sD, lin, ldl, i, tT, dpRT, iY, ec);
    slice<NP>(t1, m.R, part, a, b);
    applyc_group<BLK, 2>(m, a, b, sR, sD, lin, ldl, i, tT, dpRT, iY, ec);
    if (NP > 1) __syncthreads();

    // r_k is dead: its rows take the parts' sums
    lin_epilogue<BLK, NP, RHS>(m, part, live, i, Ti, dT, rho, arho, sD0, sR, lin + cs_H(m) * ldl + i,
                               lin + cs_S(m) * ldl + i, ldl, Y, vY, ld, fT, fY, ldf, d_omega, d_hrr);
}

// ---------------------------------------------------------------- launch shapes
struct Shape {
    int blk, np;
};
constexpr Shape kShapes[] = {{32, 1}, {64, 1}, {128, 1}, {32, 2}, {64, 2}, {32, 4}};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// MODE 0: the linearization pass; 1: it with omega and the heat release; 2: the rates' JVP from
// it; 3: the sources' JVP from it
template <int MODE, int S>
constexpr auto kernel_of() {
    if constexpr (MODE == 0)
        return linc_kernel<kShapes[S].blk, kShapes[S].np, false>;
    else if constexpr (MODE == 1)
        return linc_kernel<kShapes[S].blk, kShapes[S].np, true>;
    else if constexpr (MODE == 2)
        return jvpc_kernel<kShapes[S].blk, kShapes[S].np, false>;
    else
        return jvpc_kernel<kShapes[S].blk, kShapes[S].np, true>;
}

template <int MODE, int... S>
const void* kernel_ptr(int idx, std::integer_sequence<int, S...>) {
    const void* ptrs[] = {(const void*)kernel_of<MODE, S>()...};
    return ptrs[idx];
}

size_t mode_smem(int K, const Shape& sh, int mode) {
    return mode <= 1 ? linc_smem(K, sh.blk, sh.np, mode == 1) : jvpc_smem(K, sh.blk, sh.np);
}

// parts whose scalar sums the dead rows must hold: 2 NP rows of C_k (S1 and the heat release),
// (1 + 2 RHS) NP rows of r_k
int rows_needed(int mode, int np) { return mode == 0 ? np : (mode == 1 ? 2 * np : (mode == 3 ? 3 * np : np)); }

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
        if (rows_needed(MODE, sh.np) > K) continue;
        const size_t bytes = mode_smem(K, sh, MODE);
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
        const size_t smem = mode_smem(K, sh, MODE);
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

int64_t linc_slots(const DevMech& m) { return cs_C(m) + m.K; }

cudaError_t launch_linearize_compact(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                     const double* Y, const double* dlnA, double* lin, int64_t ldl, double* omega,
                                     double* hrr, cudaStream_t s) {
    static_assert(kDfTabBytes <= kMathTabDoubles * sizeof(double), "table space");
    if (omega) {
        const int idx = plan_shape<1>(m.K);
        if (idx < 0) return cudaErrorInvalidConfiguration;
        return launch_idx<1>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, dlnA,
                             lin, ldl, omega, hrr);
    }
    const int idx = plan_shape<0>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    double* none = nullptr;
    return launch_idx<0>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, dlnA, lin,
                         ldl, none, none);
}

cudaError_t launch_jvp_linearized_compact(const DevMech& m, int64_t n, int64_t ld, const double* T, const double* p,
                                          const double* Y, const double* lin, int64_t ldl, const double* fT,
                                          const double* fY, int64_t ldf, const double* vT, const double* vY,
                                          double* d_T, double* d_Y, cudaStream_t s, int rhs) {
    if (rhs) {
        const int idx = plan_shape<3>(m.K);
        if (idx < 0) return cudaErrorInvalidConfiguration;
        return launch_idx<3>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, lin,
                             ldl, vT, vY, d_Y, d_T, fT, fY, ldf);
    }
    const int idx = plan_shape<2>(m.K);
    if (idx < 0) return cudaErrorInvalidConfiguration;
    const double* none = nullptr;
    return launch_idx<2>(idx, std::make_integer_sequence<int, kNumShapes>{}, m.K, n, s, m, n, ld, T, p, Y, lin, ldl,
                         vT, vY, d_Y, d_T, none, none, (int64_t)0);
}

}  // namespace nk
