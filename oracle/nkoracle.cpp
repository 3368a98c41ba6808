/*
 * CPU oracle for the pointwise thermochemistry of a low-Mach reacting-flow solver
 * (nekCRF, arXiv 2409.06404: the "rates" and "properties" kernels of Sec. 2 and Tab. 3-4).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct double precision code that
 * *defines* the results the CUDA library must reproduce.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline / reference legs may build, load or call it; the
 * library itself never does.  It shares no code, header, table or constant with the CUDA
 * path; its only common input is the seeded generator output.
 *
 * The paper names the quantities (species production rates omega_k, heat release
 * sum_k h_k omega_k in Eq. 1b, c_p, mixture-averaged transport D_k in Eq. 2, viscosity mu in
 * Eq. 4, conductivity lambda in Eq. 1b) but prints no chemistry formula: the mechanism comes
 * "in Cantera format" (Sec. 2) and results are validated against Chemkin and Cantera
 * (Sec. 3.1-3.2).  Each function below therefore writes out the standard Chemkin/Cantera
 * definition of its quantity, step by step, in that order:
 *
 *   1. mixture: Wbar = 1/sum_k(Y_k/W_k); rho = p Wbar/(R T) (Eq. 1d); C_k = rho Y_k/W_k;
 *      X_k = Y_k Wbar/W_k
 *   2. NASA-7 polynomials (low range for T <= T_mid)
 *   3. Arrhenius k = A T^beta exp(-Ea/(R T))
 *   4. third-body concentration [M] = sum_k eps_k C_k
 *   5. Troe falloff (k_0, k_inf, P_r = k_0 [M]/k_inf, F_cent, F)
 *   6. K_c = exp(-sum_k nu_k g_k/(R T)) (p0/(R T))^(sum_k nu_k), k_r = k_f/K_c, p0 = 1 atm
 *   7. q = k_f prod C^nu' - k_r prod C^nu'' (times [M] for third-body reactions)
 *   8. omega_k = sum_r nu_kr q_r;  hrr = -sum_k h_k omega_k  (molar h_k(T))
 *   9. mixture-averaged transport: Wilke viscosity, Mathur conductivity, Hirschfelder-Curtiss
 *      diffusion coefficients D_km = sum_{j!=k} X_j W_j / (Wbar sum_{j!=k} X_j/D_jk)
 *  10. derivatives by complex step (h = 1e-100) through the same templated code: Im f(x + i h v)/h
 *      equals the directional derivative up to a third-derivative term times h^2/6, negligible
 *      at h = 1e-100 even at pure or nearly pure mixtures, where third derivatives in the
 *      concentrations reach ~1e80 and a step of 1e-30 would bias the result by ~1e20.
 *  11. implicit-stage chemistry sources of Eq. 1a-b at fixed p: dY_k/dt = W_k omega_k / rho,
 *      dT/dt = hrr / (rho c_p), c_p the mass-based mixture heat capacity; their directional
 *      derivatives and their dense Jacobian (one unit direction per column) by complex step as
 *      in 10.
 *  12. mixture-averaged diffusion fluxes of Eq. 2: V_k = -(D_k/X_k) grad X_k + V_c with
 *      V_c = -sum_k Y_k V'_k; j_k = rho Y_k V_k and sum_k c_p,k j_k.
 *  13. one implicit Euler step of the homogeneous constant-pressure reactor, x1 - x0 - dt f(x1)
 *      = 0 with the sources of 11, by dense Newton per point.
 *
 * Everything is templated on the scalar type S: double, std::complex<double> (complex-step
 * derivatives) and Cnt (counts the floating-point operations the definition performs).
 */
#include <cfloat>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
/* The oracle's own copy of the mechanism description (host arrays, same field meanings as
 * the generator's output). */
typedef struct {
    int32_t K, R, n_elem;
    const double* W;          /* [K] kg/mol */
    const int32_t* atoms;     /* [K][n_elem] */
    const double* nasa_lo;    /* [K][7] */
    const double* nasa_hi;    /* [K][7] */
    const double* T_mid;      /* [K] */
    const int32_t* reac_ptr;  /* [R+1] */
    const int32_t* reac_sp;
    const int32_t* reac_nu;
    const int32_t* prod_ptr;  /* [R+1] */
    const int32_t* prod_sp;
    const int32_t* prod_nu;
    const int32_t* rtype;     /* [R] 0 elementary, 1 third body, 2 Troe */
    const double* lnA;        /* [R] */
    const double* beta;
    const double* Ea;         /* J/mol */
    const double* lnA0;       /* [R] (Troe rows) */
    const double* beta0;
    const double* Ea0;
    const double* troe;       /* [R][4] a, T3, T1, T2 (T2 <= 0: absent) */
    const double* eff;        /* [R][K] */
    const double* mu_fit;     /* [K][4] */
    const double* lam_fit;    /* [K][4] */
    const double* D_fit;      /* [K(K-1)/2][4], pairs j<k */
    double p_ref;
} or_mech;
}

namespace {

const double RU = 8.314462618;   /* molar gas constant, J/(mol K) */
const double P0 = 101325.0;      /* standard-state pressure of K_c, Pa (1 atm) */

/* ---------------------------------------------------------------- operation counter */
struct OpCount {
    double add = 0, mul = 0, div = 0, exp = 0, log = 0, pow = 0, sqrt = 0;
};
thread_local OpCount* g_cnt = nullptr;

struct Cnt {
    double v;
    Cnt(double x = 0.0) : v(x) {}
};
inline Cnt tick(double v, double OpCount::*f) {
    if (g_cnt) g_cnt->*f += 1;
    return Cnt(v);
}
inline Cnt operator+(Cnt a, Cnt b) { return tick(a.v + b.v, &OpCount::add); }
inline Cnt operator-(Cnt a, Cnt b) { return tick(a.v - b.v, &OpCount::add); }
inline Cnt operator*(Cnt a, Cnt b) { return tick(a.v * b.v, &OpCount::mul); }
inline Cnt operator/(Cnt a, Cnt b) { return tick(a.v / b.v, &OpCount::div); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline Cnt exp(Cnt a) { return tick(std::exp(a.v), &OpCount::exp); }
inline Cnt log(Cnt a) { return tick(std::log(a.v), &OpCount::log); }
inline Cnt log10(Cnt a) { return tick(std::log10(a.v), &OpCount::log); }
inline Cnt sqrt(Cnt a) { return tick(std::sqrt(a.v), &OpCount::sqrt); }
inline Cnt pow(Cnt a, double b) { return tick(std::pow(a.v, b), &OpCount::pow); }
inline Cnt pow(double a, Cnt b) { return tick(std::pow(a, b.v), &OpCount::pow); }
inline double re(Cnt x) { return x.v; }

/* ---------------------------------------------------------------- scalar helpers */
using cplx = std::complex<double>;
using std::exp;
using std::log;
using std::log10;
using std::pow;
using std::sqrt;
inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }
inline double im(double) { return 0.0; }
inline double im(const cplx& x) { return x.imag(); }
inline double im(Cnt) { return 0.0; }

/* x^n for integer n by repeated multiplication (negative n: reciprocal) */
template <class S>
S ipow(S x, int n) {
    S r = S(1.0);
    int m = n < 0 ? -n : n;
    for (int i = 0; i < m; ++i) r = r * x;
    if (n < 0) r = S(1.0) / r;
    return r;
}

template <class S>
S poly3(const double* a, S x) {
    return S(a[0]) + S(a[1]) * x + S(a[2]) * x * x + S(a[3]) * x * x * x;
}

/* ---------------------------------------------------------------- step 1: mixture */
template <class S>
struct Mixture {
    S Wbar, rho;
    std::vector<S> C, X;
};

template <class S>
void mixture(const or_mech& m, S T, double p, const S* Y, Mixture<S>& mx) {
    const int K = m.K;
    S inv = S(0.0);
    for (int k = 0; k < K; ++k) inv += Y[k] / S(m.W[k]);
    mx.Wbar = S(1.0) / inv;
    mx.rho = S(p) * mx.Wbar / (S(RU) * T);             /* Eq. 1d: p0 = rho R T / Wbar */
    mx.C.assign(K, S(0.0));
    mx.X.assign(K, S(0.0));
    for (int k = 0; k < K; ++k) {
        mx.C[k] = mx.rho * Y[k] / S(m.W[k]);
        mx.X[k] = Y[k] * mx.Wbar / S(m.W[k]);
    }
}

/* ---------------------------------------------------------------- step 2: NASA-7 */
template <class S>
void nasa7(const or_mech& m, int k, S T, S& cpR, S& hRT, S& sR) {
    const double* a = (re(T) <= m.T_mid[k]) ? m.nasa_lo + 7 * k : m.nasa_hi + 7 * k;
    S T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    cpR = S(a[0]) + S(a[1]) * T + S(a[2]) * T2 + S(a[3]) * T3 + S(a[4]) * T4;
    hRT = S(a[0]) + S(a[1]) * T / S(2.0) + S(a[2]) * T2 / S(3.0) + S(a[3]) * T3 / S(4.0) +
          S(a[4]) * T4 / S(5.0) + S(a[5]) / T;
    sR = S(a[0]) * log(T) + S(a[1]) * T + S(a[2]) * T2 / S(2.0) + S(a[3]) * T3 / S(3.0) +
         S(a[4]) * T4 / S(4.0) + S(a[6]);
}

/* ---------------------------------------------------------------- step 3: Arrhenius */
template <class S>
S arrhenius(double lnA, double beta, double Ea, S T, S shift) {
    return exp(S(lnA) + shift) * pow(T, beta) * exp(S(-Ea) / (S(RU) * T));
}

/* ---------------------------------------------------------------- step 5: Troe F */
template <class S>
S troe_F(const double* tp, S T, S Pr) {
    const double a = tp[0], T3 = tp[1], T1 = tp[2], T2 = tp[3];
    S Fcent = S(1.0 - a) * exp(-T / S(T3)) + S(a) * exp(-T / S(T1));
    if (T2 > 0.0) Fcent += exp(S(-T2) / T);
    S lFc = log10(Fcent);
    S c = S(-0.4) - S(0.67) * lFc;
    S nn = S(0.75) - S(1.27) * lFc;
    S lPr = log10(Pr);
    S f1 = (lPr + c) / (nn - S(0.14) * (lPr + c));
    S lF = lFc / (S(1.0) + f1 * f1);
    return pow(10.0, lF);
}

/* ---------------------------------------------------------------- steps 3-7: one reaction */
template <class S>
struct RxnOut {
    S q, fwd, rev;
};

template <class S>
RxnOut<S> reaction(const or_mech& m, int r, S T, const S* C, const S* gRT, S shift) {
    const int K = m.K;
    S kf = arrhenius(m.lnA[r], m.beta[r], m.Ea[r], T, shift);
    S M = S(0.0);
    if (m.rtype[r] != 0)
        for (int k = 0; k < K; ++k) M += S(m.eff[(size_t)r * K + k]) * C[k];
    if (m.rtype[r] == 2) {
        S k0 = arrhenius(m.lnA0[r], m.beta0[r], m.Ea0[r], T, shift);
        S Pr = k0 * M / kf;
        if (re(Pr) == 0.0)
            kf = S(0.0);                                   /* P_r -> 0 limit: k -> 0 */
        else
            kf = kf * (Pr / (S(1.0) + Pr)) * troe_F(m.troe + 4 * r, T, Pr);
    }
    S sum_nu_g = S(0.0);
    int sum_nu = 0;
    for (int i = m.prod_ptr[r]; i < m.prod_ptr[r + 1]; ++i) {
        sum_nu_g += S((double)m.prod_nu[i]) * gRT[m.prod_sp[i]];
        sum_nu += m.prod_nu[i];
    }
    for (int i = m.reac_ptr[r]; i < m.reac_ptr[r + 1]; ++i) {
        sum_nu_g -= S((double)m.reac_nu[i]) * gRT[m.reac_sp[i]];
        sum_nu -= m.reac_nu[i];
    }
    S Kc = exp(-sum_nu_g) * ipow(S(P0) / (S(RU) * T), sum_nu);
    S kr = kf / Kc;
    S fwd = kf, rev = kr;
    for (int i = m.reac_ptr[r]; i < m.reac_ptr[r + 1]; ++i) fwd = fwd * ipow(C[m.reac_sp[i]], m.reac_nu[i]);
    for (int i = m.prod_ptr[r]; i < m.prod_ptr[r + 1]; ++i) rev = rev * ipow(C[m.prod_sp[i]], m.prod_nu[i]);
    if (m.rtype[r] == 1) {
        fwd = fwd * M;
        rev = rev * M;
    }
    return {fwd - rev, fwd, rev};
}

/* ---------------------------------------------------------------- steps 1-8: one point */
template <class S>
struct SpeciesThermo {
    std::vector<S> cpR, hRT, sR, gRT;
};

template <class S>
void species_thermo(const or_mech& m, S T, SpeciesThermo<S>& th) {
    const int K = m.K;
    th.cpR.resize(K);
    th.hRT.resize(K);
    th.sR.resize(K);
    th.gRT.resize(K);
    for (int k = 0; k < K; ++k) {
        nasa7(m, k, T, th.cpR[k], th.hRT[k], th.sR[k]);
        th.gRT[k] = th.hRT[k] - th.sR[k];
    }
}

/* scale_k/scale_h (nullable): magnitudes sum_r |nu_kr| (|fwd_r| + |rev_r|) and sum_k |h_k| scale_k;
 * dscale_k/dscale_h (nullable, complex step only): the same with the imaginary parts, i.e. the
 * magnitudes of the forward and reverse terms' directional derivatives (times the step). */
template <class S>
void rates_point(const or_mech& m, S T, double p, const S* Y, const S* shift, S* omega, S& hrr,
                 double* scale_k, double* scale_h, double* dscale_k = nullptr, double* dscale_h = nullptr) {
    const int K = m.K, R = m.R;
    Mixture<S> mx;
    mixture(m, T, p, Y, mx);
    SpeciesThermo<S> th;
    species_thermo(m, T, th);
    for (int k = 0; k < K; ++k) omega[k] = S(0.0);
    if (scale_k)
        for (int k = 0; k < K; ++k) scale_k[k] = 0.0;
    if (dscale_k)
        for (int k = 0; k < K; ++k) dscale_k[k] = 0.0;
    for (int r = 0; r < R; ++r) {
        RxnOut<S> o = reaction(m, r, T, mx.C.data(), th.gRT.data(), shift ? shift[r] : S(0.0));
        for (int i = m.reac_ptr[r]; i < m.reac_ptr[r + 1]; ++i)
            omega[m.reac_sp[i]] -= S((double)m.reac_nu[i]) * o.q;
        for (int i = m.prod_ptr[r]; i < m.prod_ptr[r + 1]; ++i)
            omega[m.prod_sp[i]] += S((double)m.prod_nu[i]) * o.q;
        if (scale_k) {
            double mag = std::fabs(re(o.fwd)) + std::fabs(re(o.rev));
            for (int i = m.reac_ptr[r]; i < m.reac_ptr[r + 1]; ++i) scale_k[m.reac_sp[i]] += m.reac_nu[i] * mag;
            for (int i = m.prod_ptr[r]; i < m.prod_ptr[r + 1]; ++i) scale_k[m.prod_sp[i]] += m.prod_nu[i] * mag;
        }
        if (dscale_k) {
            double mag = std::fabs(im(o.fwd)) + std::fabs(im(o.rev));
            for (int i = m.reac_ptr[r]; i < m.reac_ptr[r + 1]; ++i) dscale_k[m.reac_sp[i]] += m.reac_nu[i] * mag;
            for (int i = m.prod_ptr[r]; i < m.prod_ptr[r + 1]; ++i) dscale_k[m.prod_sp[i]] += m.prod_nu[i] * mag;
        }
    }
    hrr = S(0.0);
    double sh = 0.0, dsh = 0.0;
    for (int k = 0; k < K; ++k) {
        S h = S(RU) * T * th.hRT[k];                       /* molar enthalpy h_k(T) */
        hrr -= h * omega[k];
        if (scale_k) sh += std::fabs(re(h)) * scale_k[k];
        if (dscale_k && scale_k) dsh += std::fabs(re(h)) * dscale_k[k] + std::fabs(im(h)) * scale_k[k];
    }
    if (scale_h) *scale_h = sh;
    if (dscale_h) *dscale_h = dsh;
}

/* ---------------------------------------------------------------- implicit-stage sources
 * The chemistry source terms of Eq. 1a-b at fixed p: dY_k/dt = W_k omega_k / rho (omega_k is
 * molar, so W_k omega_k is the mass production rate) and dT/dt = hrr / (rho c_p) with the
 * heat release hrr = -sum_k h_k omega_k and the mass-based mixture c_p.
 * scale_Y/scale_T (nullable): the omega and hrr magnitudes of rates_point carried through the
 * same factors; with complex S the imaginary parts (dscale_*) give the magnitudes of the
 * directional derivatives: W_k (|d omega_k| + |omega_k| |d rho|/rho) / rho and
 * (|d hrr| + |hrr| (|d rho|/rho + |d c_p|/c_p)) / (rho c_p), each term by its own magnitude. */
template <class S>
void rhs_point(const or_mech& m, S T, double p, const S* Y, S* fY, S& fT, double* scale_Y, double* scale_T,
               double* dscale_Y = nullptr, double* dscale_T = nullptr) {
    const int K = m.K;
    std::vector<S> w(K);
    std::vector<double> sc(K), dsc(K);
    double sh = 0.0, dsh = 0.0;
    S hrr;
    const bool want = scale_Y != nullptr;
    rates_point<S>(m, T, p, Y, nullptr, w.data(), hrr, want ? sc.data() : nullptr, want ? &sh : nullptr,
                   dscale_Y ? dsc.data() : nullptr, dscale_Y ? &dsh : nullptr);
    Mixture<S> mx;
    mixture(m, T, p, Y, mx);
    S cp = S(0.0);
    for (int k = 0; k < K; ++k) {
        S cpR, hRT, sR;
        nasa7(m, k, T, cpR, hRT, sR);
        cp += Y[k] * S(RU) * cpR / S(m.W[k]);
    }
    for (int k = 0; k < K; ++k) fY[k] = S(m.W[k]) * w[k] / mx.rho;
    fT = hrr / (mx.rho * cp);
    if (want) {
        const double rho = std::fabs(re(mx.rho)), c = std::fabs(re(cp));
        for (int k = 0; k < K; ++k) scale_Y[k] = m.W[k] * sc[k] / rho;
        *scale_T = sh / (rho * c);
        if (dscale_Y) {
            const double drr = std::fabs(im(mx.rho)) / rho, dcc = std::fabs(im(cp)) / c;
            for (int k = 0; k < K; ++k) dscale_Y[k] = m.W[k] * (dsc[k] + std::fabs(re(w[k])) * drr) / rho;
            *dscale_T = (dsh + std::fabs(re(hrr)) * (drr + dcc)) / (rho * c);
        }
    }
}

/* ---------------------------------------------------------------- step 9: transport */
inline int pair_index(int K, int j, int k) { /* j < k */
    return j * K - j * (j + 1) / 2 + (k - j - 1);
}

template <class S>
void transport_point(const or_mech& m, S T, double p, const S* Y, S& mu, S& lam, S* Dmix) {
    const int K = m.K;
    Mixture<S> mx;
    mixture(m, T, p, Y, mx);
    const S L = log(T);
    std::vector<S> mu_k(K), lam_k(K);
    for (int k = 0; k < K; ++k) {
        mu_k[k] = exp(poly3(m.mu_fit + 4 * k, L));
        lam_k[k] = exp(poly3(m.lam_fit + 4 * k, L));
    }
    /* Wilke mixture viscosity */
    mu = S(0.0);
    for (int k = 0; k < K; ++k) {
        S den = S(0.0);
        for (int j = 0; j < K; ++j) {
            S t = S(1.0) + sqrt(mu_k[k] / mu_k[j]) * pow(S(m.W[j] / m.W[k]), 0.25);
            S phi = S(1.0) / sqrt(S(8.0)) / sqrt(S(1.0) + S(m.W[k] / m.W[j])) * t * t;
            den += mx.X[j] * phi;
        }
        mu += mx.X[k] * mu_k[k] / den;
    }
    /* Mathur-Saxena combination rule for the conductivity */
    S s1 = S(0.0), s2 = S(0.0);
    for (int k = 0; k < K; ++k) {
        s1 += mx.X[k] * lam_k[k];
        s2 += mx.X[k] / lam_k[k];
    }
    lam = S(0.5) * (s1 + S(1.0) / s2);
    /* mixture-averaged diffusion coefficients */
    for (int k = 0; k < K; ++k) {
        S num = S(0.0), den = S(0.0);
        for (int j = 0; j < K; ++j) {
            if (j == k) continue;
            const int pi = j < k ? pair_index(K, j, k) : pair_index(K, k, j);
            S Djk = exp(poly3(m.D_fit + 4 * pi, L)) * S(m.p_ref / p);
            num += mx.X[j] * S(m.W[j]);
            den += mx.X[j] / Djk;
        }
        if (re(num) == 0.0)
            Dmix[k] = S(0.0);
        else {
            if (re(den) < DBL_MIN) den = S(DBL_MIN);
            Dmix[k] = num / (mx.Wbar * den);
        }
    }
}

int nthreads_of(int requested) {
#ifdef _OPENMP
    return requested > 0 ? requested : omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/* ---------------------------------------------------------------- step 12: diffusion fluxes
 * Eq. 2 with the correction velocity defined below it: V_k = -(D_k/X_k) grad X_k + V_c and
 * V_c = -sum_k Y_k V'_k over the uncorrected velocities V'_k = -(D_k/X_k) grad X_k.  Outputs
 * per Cartesian component c: the species mass fluxes j_k = rho Y_k V_k, the correction velocity
 * V_c and sum_k c_p,k j_k (c_p,k mass based; the factor of the enthalpy-flux term of Eq. 1b).
 * Y_k/X_k is evaluated as written; at X_k = 0 its limit W_k/Wbar is used.
 * D, gradX: [K] and [3][K]; j: [3][K]; Vc, hf: [3]. */
void diffusion_point(const or_mech& m, double T, double p, const double* Y, const double* D, const double* gradX,
                     double* j, double* Vc, double* hf) {
    const int K = m.K;
    Mixture<double> mx;
    mixture(m, T, p, Y, mx);
    std::vector<double> cpk(K), yv(K);
    for (int k = 0; k < K; ++k) {
        double cpR, hRT, sR;
        nasa7(m, k, T, cpR, hRT, sR);
        cpk[k] = RU * cpR / m.W[k];
    }
    for (int c = 0; c < 3; ++c) {
        double sum = 0.0;
        for (int k = 0; k < K; ++k) {
            const double y_over_x = mx.X[k] != 0.0 ? Y[k] / mx.X[k] : m.W[k] / mx.Wbar;
            yv[k] = -y_over_x * D[k] * gradX[c * K + k];   /* Y_k V'_k */
            sum += yv[k];
        }
        Vc[c] = -sum;
        double h = 0.0;
        for (int k = 0; k < K; ++k) {
            j[c * K + k] = mx.rho * (yv[k] + Y[k] * Vc[c]);
            h += cpk[k] * j[c * K + k];
        }
        hf[c] = h;
    }
}

/* ---------------------------------------------------------------- step 13: implicit reactor step
 * One implicit (backward) Euler step of a homogeneous constant-pressure reactor, the
 * nonlinear system the paper's implicit thermochemistry stage solves at every point (Sec. 2,
 * there by Newton-GMRES over the whole mesh): x1 - x0 - dt f(x1) = 0 with x = (T, Y_k) and f
 * the sources of step 11.  Solved per point by Newton's method on the dense system with the
 * complex-step Jacobian of f and Gaussian elimination with partial pivoting, until the update
 * is below 1e-14 of (|x| + atol) in every component.  Returns the iterations used (negative:
 * not converged in 100). */
int reactor_point(const or_mech& m, double T0, double p, const double* Y0, double dt, double atolT,
                  double atolY, double* x1) {
    const int K = m.K, N = K + 1;
    const double hstep = 1e-100;
    std::vector<double> x0(N), x(N), G(N), A((size_t)N * N), d(N);
    x0[0] = T0;
    for (int k = 0; k < K; ++k) x0[k + 1] = Y0[k];
    x = x0;
    std::vector<cplx> yc(K), fY(K);
    for (int it = 1; it <= 100; ++it) {
        // f(x) and its Jacobian, one complex-step evaluation per input
        for (int j = 0; j < N; ++j) {
            for (int k = 0; k < K; ++k) yc[k] = cplx(x[k + 1], j == k + 1 ? hstep : 0.0);
            cplx fT;
            rhs_point<cplx>(m, cplx(x[0], j == 0 ? hstep : 0.0), p, yc.data(), fY.data(), fT, nullptr, nullptr);
            if (j == 0) {
                G[0] = x[0] - x0[0] - dt * fT.real();
                for (int k = 0; k < K; ++k) G[k + 1] = x[k + 1] - x0[k + 1] - dt * fY[k].real();
            }
            A[(size_t)0 * N + j] = (j == 0 ? 1.0 : 0.0) - dt * fT.imag() / hstep;
            for (int k = 0; k < K; ++k) A[(size_t)(k + 1) * N + j] = (j == k + 1 ? 1.0 : 0.0) - dt * fY[k].imag() / hstep;
        }
        // solve A d = -G
        for (int i = 0; i < N; ++i) d[i] = -G[i];
        for (int c = 0; c < N; ++c) {
            int piv = c;
            for (int r = c + 1; r < N; ++r)
                if (std::fabs(A[(size_t)r * N + c]) > std::fabs(A[(size_t)piv * N + c])) piv = r;
            if (piv != c) {
                for (int q = 0; q < N; ++q) std::swap(A[(size_t)c * N + q], A[(size_t)piv * N + q]);
                std::swap(d[c], d[piv]);
            }
            for (int r = c + 1; r < N; ++r) {
                const double f = A[(size_t)r * N + c] / A[(size_t)c * N + c];
                for (int q = c; q < N; ++q) A[(size_t)r * N + q] -= f * A[(size_t)c * N + q];
                d[r] -= f * d[c];
            }
        }
        for (int c = N - 1; c >= 0; --c) {
            double acc = d[c];
            for (int q = c + 1; q < N; ++q) acc -= A[(size_t)c * N + q] * d[q];
            d[c] = acc / A[(size_t)c * N + c];
        }
        double worst = 0.0;
        for (int i = 0; i < N; ++i) {
            x[i] += d[i];
            worst = std::fmax(worst, std::fabs(d[i]) / (std::fabs(x[i]) + (i == 0 ? atolT : atolY)));
        }
        if (worst <= 1e-14) {
            for (int i = 0; i < N; ++i) x1[i] = x[i];
            return it;
        }
    }
    for (int i = 0; i < N; ++i) x1[i] = x[i];
    return -100;
}

}  // namespace

/* ====================================================================== C entry points */
extern "C" {

int or_max_threads(void) { return nthreads_of(0); }

/* Species and mixture thermodynamics at n points.  Mixture outputs are mass based
 * (J/kg/K, J/kg); per-species outputs are molar (J/mol/K, J/mol).  Nullable outputs. */
void or_thermo(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
               const double* Y, double* cp_mix, double* h_mix, double* Wbar, double* rho,
               double* cp_k, double* h_k, double* g_k, int nthreads) {
    const int K = m->K;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K);
        for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
        Mixture<double> mx;
        mixture(*m, T[i], p[i], y.data(), mx);
        double cp = 0.0, h = 0.0;
        for (int k = 0; k < K; ++k) {
            double cpR, hRT, sR;
            nasa7(*m, k, T[i], cpR, hRT, sR);
            const double cpk = RU * cpR, hk = RU * T[i] * hRT, gk = RU * T[i] * (hRT - sR);
            cp += y[k] * cpk / m->W[k];
            h += y[k] * hk / m->W[k];
            if (cp_k) cp_k[k * ld + i] = cpk;
            if (h_k) h_k[k * ld + i] = hk;
            if (g_k) g_k[k * ld + i] = gk;
        }
        if (cp_mix) cp_mix[i] = cp;
        if (h_mix) h_mix[i] = h;
        if (Wbar) Wbar[i] = mx.Wbar;
        if (rho) rho[i] = mx.rho;
    }
}

/* Species cp, h and s (molar) and their temperature derivatives dh/dT, ds/dT by complex step
 * through the same NASA-7 code, at n temperatures, for species k. */
void or_nasa7_cs(const or_mech* m, int k, int64_t n, const double* T, double* cp, double* h,
                 double* s, double* dh_dT, double* ds_dT) {
    const double hstep = 1e-100;
    for (int64_t i = 0; i < n; ++i) {
        cplx Tc(T[i], hstep), cpR, hRT, sR;
        nasa7(*m, k, Tc, cpR, hRT, sR);
        cplx hc = RU * Tc * hRT, sc = RU * sR;
        cp[i] = RU * cpR.real();
        h[i] = hc.real();
        s[i] = sc.real();
        dh_dT[i] = hc.imag() / hstep;
        ds_dT[i] = sc.imag() / hstep;
    }
}

/* Net production rates omega [K][ld] (mol/m^3/s) and heat release hrr [n] (W/m^3).
 * dlnA: nullable [R] shift added to ln A (both limits of a Troe reaction).
 * omega_scale/hrr_scale (nullable): sum_r |nu_kr| (|fwd_r| + |rev_r|) and sum_k |h_k| omega_scale_k,
 * the magnitudes against which cancellation-aware tolerances are measured. */
void or_rates(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
              const double* Y, const double* dlnA, double* omega, double* hrr, double* omega_scale,
              double* hrr_scale, int nthreads) {
    const int K = m->K;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K), w(K), sc(K);
        for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
        double h, sh;
        rates_point<double>(*m, T[i], p[i], y.data(), dlnA, w.data(), h, omega_scale ? sc.data() : nullptr, &sh);
        for (int k = 0; k < K; ++k) omega[k * ld + i] = w[k];
        hrr[i] = h;
        if (omega_scale)
            for (int k = 0; k < K; ++k) omega_scale[k * ld + i] = sc[k];
        if (hrr_scale) hrr_scale[i] = omega_scale ? sh : 0.0;
    }
}

/* Per-reaction forward and reverse terms (fwd_r, rev_r) at n points, [R][ld]. */
void or_rates_of_progress(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                          const double* Y, const double* dlnA, double* fwd, double* rev, int nthreads) {
    const int K = m->K, R = m->R;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K);
        for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
        Mixture<double> mx;
        mixture(*m, T[i], p[i], y.data(), mx);
        SpeciesThermo<double> th;
        species_thermo(*m, T[i], th);
        for (int r = 0; r < R; ++r) {
            RxnOut<double> o = reaction(*m, r, T[i], mx.C.data(), th.gRT.data(), dlnA ? dlnA[r] : 0.0);
            fwd[r * ld + i] = o.fwd;
            rev[r * ld + i] = o.rev;
        }
    }
}

/* Mixture viscosity mu [n] (Pa s), conductivity lam [n] (W/m/K), and mixture-averaged
 * diffusion coefficients Dmix [K][ld] (m^2/s). */
void or_transport(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                  const double* Y, double* mu, double* lam, double* Dmix, int nthreads) {
    const int K = m->K;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K), d(K);
        for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
        double a, b;
        transport_point<double>(*m, T[i], p[i], y.data(), a, b, d.data());
        mu[i] = a;
        lam[i] = b;
        for (int k = 0; k < K; ++k) Dmix[k * ld + i] = d[k];
    }
}

/* Dense Jacobian d(omega_0..omega_{K-1}, hrr)/d(T, Y_0..Y_{K-1}) at fixed p, by complex step.
 * J: [n][(K+1)*(K+1)], row = output, column = input.
 * Js (nullable), same shape: sum_r |nu_kr| (|d fwd_r/dx| + |d rev_r/dx|) and the heat-release
 * analogue, the magnitudes behind each entry for cancellation-aware tolerances. */
void or_rates_jacobian(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, double* J, double* Js, int nthreads) {
    const int K = m->K, R = m->R, N = K + 1;
    const double hstep = 1e-100;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<cplx> y(K), w(K), sh(R);
        for (int r = 0; r < R; ++r) sh[r] = cplx(dlnA ? dlnA[r] : 0.0, 0.0);
        for (int j = 0; j < N; ++j) {
            for (int k = 0; k < K; ++k) y[k] = cplx(Y[k * ld + i], (j == k + 1) ? hstep : 0.0);
            cplx Tc(T[i], j == 0 ? hstep : 0.0), h;
            std::vector<double> sc(K), dsc(K);
            double sh_, dsh_;
            rates_point<cplx>(*m, Tc, p[i], y.data(), sh.data(), w.data(), h, sc.data(), &sh_, dsc.data(), &dsh_);
            double* Ji = J + (size_t)i * N * N;
            for (int k = 0; k < K; ++k) Ji[k * N + j] = w[k].imag() / hstep;
            Ji[K * N + j] = h.imag() / hstep;
            if (Js) {
                double* Si = Js + (size_t)i * N * N;
                for (int k = 0; k < K; ++k) Si[k * N + j] = dsc[k] / hstep;
                Si[K * N + j] = dsh_ / hstep;
            }
        }
    }
}

/* Jacobian-vector product along (vT, vY) by one complex-step evaluation per point.
 * d_omega_scale/d_hrr_scale (nullable): sum_r |nu_kr| (|d fwd_r| + |d rev_r|) along v, and the
 * matching heat-release magnitude, the scales of cancellation-aware tolerances on J v. */
void or_rates_jvp(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                  const double* Y, const double* dlnA, const double* vT, const double* vY,
                  double* d_omega, double* d_hrr, double* d_omega_scale, double* d_hrr_scale, int nthreads) {
    const int K = m->K, R = m->R;
    const double hstep = 1e-100;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<cplx> y(K), w(K), sh(R);
        for (int r = 0; r < R; ++r) sh[r] = cplx(dlnA ? dlnA[r] : 0.0, 0.0);
        for (int k = 0; k < K; ++k) y[k] = cplx(Y[k * ld + i], hstep * vY[k * ld + i]);
        cplx Tc(T[i], hstep * vT[i]), h;
        std::vector<double> sc(K), dsc(K);
        double sh_, dsh_;
        rates_point<cplx>(*m, Tc, p[i], y.data(), sh.data(), w.data(), h, sc.data(), &sh_, dsc.data(), &dsh_);
        for (int k = 0; k < K; ++k) d_omega[k * ld + i] = w[k].imag() / hstep;
        d_hrr[i] = h.imag() / hstep;
        if (d_omega_scale)
            for (int k = 0; k < K; ++k) d_omega_scale[k * ld + i] = dsc[k] / hstep;
        if (d_hrr_scale) d_hrr_scale[i] = dsh_ / hstep;
    }
}

/* Gradient of L = sum_points [ sum_k wbar_k omega_k + hbar hrr ] with respect to ln A_r.
 * Only q_r depends on ln A_r, so d omega_k/d lnA_r = nu_kr dq_r/dlnA_r and
 * d hrr/d lnA_r = -sum_k h_k nu_kr dq_r/dlnA_r; dq_r/dlnA_r is taken by complex step on that
 * reaction alone.  Per-thread partial sums are added in thread order.  hbar nullable. */
void or_rates_grad_lnA(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* wbar, const double* hbar,
                       double* g, int nthreads) {
    const int K = m->K, R = m->R;
    const int nt = nthreads_of(nthreads);
    const double hstep = 1e-100;
    std::vector<double> part((size_t)nt * R, 0.0);
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
        const int tid = omp_get_thread_num();
#else
        const int tid = 0;
#endif
        double* acc = part.data() + (size_t)tid * R;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            std::vector<double> y(K);
            for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
            Mixture<double> mx;
            mixture(*m, T[i], p[i], y.data(), mx);
            SpeciesThermo<double> th;
            species_thermo(*m, T[i], th);
            std::vector<cplx> C(K), gRT(K);
            for (int k = 0; k < K; ++k) {
                C[k] = mx.C[k];
                gRT[k] = th.gRT[k];
            }
            const double hb = hbar ? hbar[i] : 0.0;
            for (int r = 0; r < R; ++r) {
                cplx shift(dlnA ? dlnA[r] : 0.0, hstep);
                RxnOut<cplx> o = reaction(*m, r, cplx(T[i], 0.0), C.data(), gRT.data(), shift);
                const double dq = o.q.imag() / hstep;
                double s = 0.0;
                for (int e = m->reac_ptr[r]; e < m->reac_ptr[r + 1]; ++e) {
                    const int k = m->reac_sp[e];
                    const double hk = RU * T[i] * th.hRT[k];
                    s -= m->reac_nu[e] * (wbar[k * ld + i] - hb * hk);
                }
                for (int e = m->prod_ptr[r]; e < m->prod_ptr[r + 1]; ++e) {
                    const int k = m->prod_sp[e];
                    const double hk = RU * T[i] * th.hRT[k];
                    s += m->prod_nu[e] * (wbar[k * ld + i] - hb * hk);
                }
                acc[r] += s * dq;
            }
        }
    }
    for (int r = 0; r < R; ++r) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += part[(size_t)t * R + r];
        g[r] = s;
    }
}

/* Implicit-stage chemistry sources (rhs_point): fT [n] (K/s) and fY [K][ld] (1/s); the scales
 * (nullable) are the magnitudes behind cancellation-aware tolerances. */
void or_rhs(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
            double* fT, double* fY, double* fT_scale, double* fY_scale, int nthreads) {
    const int K = m->K;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K), f(K), sc(K);
        for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
        double ft, st;
        rhs_point<double>(*m, T[i], p[i], y.data(), f.data(), ft, fY_scale ? sc.data() : nullptr, &st);
        fT[i] = ft;
        for (int k = 0; k < K; ++k) fY[k * ld + i] = f[k];
        if (fY_scale)
            for (int k = 0; k < K; ++k) fY_scale[k * ld + i] = sc[k];
        if (fT_scale) fT_scale[i] = fY_scale ? st : 0.0;
    }
}

/* Their directional derivative along (vT, vY) at fixed p by one complex-step evaluation per
 * point, with the derivative magnitudes (nullable) for cancellation-aware tolerances. */
void or_rhs_jvp(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                const double* vT, const double* vY, double* dfT, double* dfY, double* dfT_scale, double* dfY_scale,
                int nthreads) {
    const int K = m->K;
    const double hstep = 1e-100;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<cplx> y(K), f(K);
        std::vector<double> sc(K), dsc(K);
        for (int k = 0; k < K; ++k) y[k] = cplx(Y[k * ld + i], hstep * vY[k * ld + i]);
        cplx Tc(T[i], hstep * vT[i]), ft;
        double st, dst;
        rhs_point<cplx>(*m, Tc, p[i], y.data(), f.data(), ft, sc.data(), &st, dsc.data(), &dst);
        dfT[i] = ft.imag() / hstep;
        for (int k = 0; k < K; ++k) dfY[k * ld + i] = f[k].imag() / hstep;
        if (dfY_scale)
            for (int k = 0; k < K; ++k) dfY_scale[k * ld + i] = dsc[k] / hstep;
        if (dfT_scale) dfT_scale[i] = dst / hstep;
    }
}

/* Dense Jacobian of the sources of 11 with respect to (T, Y_0..Y_{K-1}) at fixed p, one complex
 * step per column.  J: [n][(K+1)*(K+1)], row = output (0: dT/dt, k+1: dY_k/dt), column = input
 * (0: T, j+1: Y_j), the ordering of the reactor unknowns of 13.  Js (nullable), same shape: the
 * derivative magnitudes of or_rhs_jvp along each unit direction. */
void or_rhs_jacobian(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     double* J, double* Js, int nthreads) {
    const int K = m->K, N = K + 1;
    const double hstep = 1e-100;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<cplx> y(K), f(K);
        std::vector<double> sc(K), dsc(K);
        double* Ji = J + (size_t)i * N * N;
        double* Si = Js ? Js + (size_t)i * N * N : nullptr;
        for (int j = 0; j < N; ++j) {
            for (int k = 0; k < K; ++k) y[k] = cplx(Y[k * ld + i], j == k + 1 ? hstep : 0.0);
            cplx ft;
            double st, dst;
            rhs_point<cplx>(*m, cplx(T[i], j == 0 ? hstep : 0.0), p[i], y.data(), f.data(), ft, sc.data(), &st,
                            dsc.data(), &dst);
            Ji[j] = ft.imag() / hstep;
            for (int k = 0; k < K; ++k) Ji[(size_t)(k + 1) * N + j] = f[k].imag() / hstep;
            if (Si) {
                Si[j] = dst / hstep;
                for (int k = 0; k < K; ++k) Si[(size_t)(k + 1) * N + j] = dsc[k] / hstep;
            }
        }
    }
}

/* Diffusion fluxes (diffusion_point) at n points: D [K][ld], gradX [3][K][ld] in; j [3][K][ld],
 * Vc [3][ld], hf [3][ld] out. */
void or_diffusion(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                  const double* D, const double* gradX, double* j, double* Vc, double* hf, int nthreads) {
    const int K = m->K;
#pragma omp parallel for schedule(static) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K), d(K), g(3 * K), jj(3 * K);
        double vc[3], h[3];
        for (int k = 0; k < K; ++k) {
            y[k] = Y[k * ld + i];
            d[k] = D[k * ld + i];
        }
        for (int q = 0; q < 3 * K; ++q) g[q] = gradX[q * ld + i];
        diffusion_point(*m, T[i], p[i], y.data(), d.data(), g.data(), jj.data(), vc, h);
        for (int q = 0; q < 3 * K; ++q) j[q * ld + i] = jj[q];
        for (int c = 0; c < 3; ++c) {
            Vc[c * ld + i] = vc[c];
            hf[c * ld + i] = h[c];
        }
    }
}

/* One implicit Euler step of dt at every point (reactor_point): T1 [n], Y1 [K][ld] out, the
 * Newton iterations per point in iters [n] (negative: not converged). */
void or_reactor_step(const or_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     double dt, double atolT, double atolY, double* T1, double* Y1, int* iters, int nthreads) {
    const int K = m->K;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads_of(nthreads))
    for (int64_t i = 0; i < n; ++i) {
        std::vector<double> y(K), x1(K + 1);
        for (int k = 0; k < K; ++k) y[k] = Y[k * ld + i];
        iters[i] = reactor_point(*m, T[i], p[i], y.data(), dt, atolT, atolY, x1.data());
        T1[i] = x1[0];
        for (int k = 0; k < K; ++k) Y1[k * ld + i] = x1[k + 1];
    }
}

/* Floating-point operations performed by the definitions above for one point:
 * counts[0..6] = add/sub, mul, div, exp, log (incl. log10), pow, sqrt;
 * which = 0: rates (steps 1-8), 1: transport (steps 1 and 9). */
void or_count_ops(const or_mech* m, double T, double p, const double* Y, int which, double* counts) {
    const int K = m->K, R = m->R;
    OpCount c;
    std::vector<Cnt> y(K), w(K), d(K), sh(R, Cnt(0.0));
    for (int k = 0; k < K; ++k) y[k] = Cnt(Y[k]);
    g_cnt = &c;
    if (which == 0) {
        Cnt h;
        rates_point<Cnt>(*m, Cnt(T), p, y.data(), sh.data(), w.data(), h, nullptr, nullptr);
    } else {
        Cnt a, b;
        transport_point<Cnt>(*m, Cnt(T), p, y.data(), a, b, d.data());
    }
    g_cnt = nullptr;
    counts[0] = c.add;
    counts[1] = c.mul;
    counts[2] = c.div;
    counts[3] = c.exp;
    counts[4] = c.log;
    counts[5] = c.pow;
    counts[6] = c.sqrt;
}

}  /* extern "C" */
