// C-ABI layer of nkchem: argument checking, error reporting, mechanism upload and the
// dispatch to the kernel launchers.  Every entry point declared in include/nkchem.h is
// defined here.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <map>
#include <vector>

#include "nk_internal.cuh"

namespace {

thread_local char g_err[512] = "";

nk_status fail(nk_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

nk_status ok() {
    g_err[0] = '\0';
    return NK_OK;
}

nk_status cuda_fail(cudaError_t e, const char* what) {
    return fail(NK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool misaligned(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 7u); }

// Bump allocator over one host staging buffer mirrored by one device allocation.
struct Layout {
    size_t bytes = 0;
    size_t add(size_t n) {
        size_t off = (bytes + 255) & ~size_t(255);
        bytes = off + n;
        return off;
    }
};

nk_status check_mech_desc(const nk_mech_desc* d) {
    if (!d) return fail(NK_EINVAL, "desc is NULL");
    if (d->K < 1 || d->R < 1) return fail(NK_EINVAL, "K and R must be >= 1 (K=%d, R=%d)", d->K, d->R);
    if (d->K > nk::kMaxK) return fail(NK_EUNSUPPORTED, "K=%d exceeds %d species", d->K, nk::kMaxK);
    if (d->R > nk::kMaxR) return fail(NK_EUNSUPPORTED, "R=%d exceeds %d reactions", d->R, nk::kMaxR);
    const void* req[] = {d->W, d->nasa_lo, d->nasa_hi, d->T_mid, d->reac_ptr, d->reac_sp, d->reac_nu,
                         d->prod_ptr, d->prod_sp, d->prod_nu, d->rtype, d->lnA, d->beta, d->Ea,
                         d->lnA0, d->beta0, d->Ea0, d->troe, d->eff, d->mu_fit, d->lam_fit};
    for (const void* p : req)
        if (!p) return fail(NK_EINVAL, "a required mechanism array is NULL");
    if (d->K > 1 && !d->D_fit) return fail(NK_EINVAL, "D_fit is NULL");
    if (!(d->p_ref > 0.0)) return fail(NK_EINVAL, "p_ref must be > 0");
    for (int k = 0; k < d->K; ++k) {
        if (!(d->W[k] > 0.0)) return fail(NK_EINVAL, "W[%d] must be > 0", k);
        if (!(d->T_mid[k] > 0.0)) return fail(NK_EINVAL, "T_mid[%d] must be > 0", k);
    }
    const int32_t* ptrs[2] = {d->reac_ptr, d->prod_ptr};
    const int32_t* sps[2] = {d->reac_sp, d->prod_sp};
    const int32_t* nus[2] = {d->reac_nu, d->prod_nu};
    for (int side = 0; side < 2; ++side) {
        if (ptrs[side][0] != 0) return fail(NK_EINVAL, "stoichiometry pointer arrays must start at 0");
        for (int r = 0; r < d->R; ++r) {
            const int c = ptrs[side][r + 1] - ptrs[side][r];
            if (c < 1) return fail(NK_EINVAL, "reaction %d has an empty side", r);
            if (c > nk::kMaxSide)
                return fail(NK_EUNSUPPORTED, "reaction %d has %d entries on one side (max %d)", r, c, nk::kMaxSide);
            for (int e = ptrs[side][r]; e < ptrs[side][r + 1]; ++e) {
                if (sps[side][e] < 0 || sps[side][e] >= d->K)
                    return fail(NK_EINVAL, "reaction %d: species index %d out of range", r, sps[side][e]);
                if (nus[side][e] < 1 || nus[side][e] > nk::kMaxNu)
                    return fail(NK_EUNSUPPORTED, "reaction %d: stoichiometric coefficient %d not in 1..%d", r,
                                nus[side][e], nk::kMaxNu);
            }
        }
    }
    for (int r = 0; r < d->R; ++r)
        if (d->rtype[r] < 0 || d->rtype[r] > 2) return fail(NK_EINVAL, "rtype[%d]=%d", r, d->rtype[r]);
    return NK_OK;
}

}  // namespace

namespace nk {

int pick_block(size_t bytes_per_thread, size_t budget) {
    for (int b : {128, 64, 32})
        if (bytes_per_thread * (size_t)b <= budget) return b;
    return 0;
}

int pick_block_occupancy(size_t bytes_per_thread, size_t fixed_bytes, size_t bytes_per_warp) {
    int dev = 0, per_sm = 0, per_block = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = 0, best_threads = 0;
    for (int b : {128, 64, 32}) {
        const size_t blk_bytes = bytes_per_thread * (size_t)b + fixed_bytes + bytes_per_warp * (size_t)(b / 32);
        if (blk_bytes > (size_t)per_block) continue;
        const int blocks = (int)((size_t)per_sm / (blk_bytes + 1024));   // 1 KB reserved per block
        const int threads = blocks * b;
        if (threads > best_threads) {
            best_threads = threads;
            best = b;
        }
    }
    return best;
}

namespace {
struct SmemEntry {
    const void* kernel;
    int device;
    size_t bytes;
};
std::mutex g_smem_mu;
std::vector<SmemEntry> g_smem;
}  // namespace

cudaError_t ensure_smem(const void* kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_smem_mu);
    for (const SmemEntry& s : g_smem)
        if (s.kernel == kernel && s.device == dev && s.bytes >= bytes) return cudaSuccess;
    const size_t lim = smem_limit();
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    if (e != cudaSuccess) return e;
    g_smem.push_back({kernel, dev, lim});
    return cudaSuccess;
}

size_t smem_limit() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 48 * 1024;
    return (size_t)v;
}

}  // namespace nk

extern "C" {

int32_t nk_version(void) { return NKCHEM_VERSION; }

const char* nk_last_error(void) { return g_err; }

nk_status nk_mechanism_load(const nk_mech_desc* d, nk_mech** out) {
    if (!out) return fail(NK_EINVAL, "out is NULL");
    *out = nullptr;
    nk_status st = check_mech_desc(d);
    if (st != NK_OK) return st;
    const int K = d->K, R = d->R, P = K * (K - 1) / 2;

    // ---- build host tables
    std::vector<double> invW(K), Tmid(K), nasa((size_t)K * 2 * nk::kNasaStride, 0.0);
    for (int k = 0; k < K; ++k) {
        invW[k] = 1.0 / d->W[k];
        Tmid[k] = d->T_mid[k];
        for (int range = 0; range < 2; ++range) {
            const double* a = (range == 0 ? d->nasa_lo : d->nasa_hi) + 7 * k;
            double* c = nasa.data() + ((size_t)k * 2 + range) * nk::kNasaStride;
            for (int j = 0; j < 7; ++j) c[j] = a[j];
            c[7] = a[1] / 2.0;
            c[8] = a[2] / 3.0;
            c[9] = a[3] / 4.0;
            c[10] = a[4] / 5.0;
            c[11] = -a[1] / 2.0;
            c[12] = -a[2] / 6.0;
            c[13] = -a[3] / 12.0;
            c[14] = -a[4] / 20.0;
        }
    }
    // device order of the reactions: elementary, then third-body, then Troe (stable)
    std::vector<int> order;
    for (int kind = 0; kind < 3; ++kind)
        for (int r = 0; r < R; ++r)
            if (d->rtype[r] == kind) order.push_back(r);
    int R_el = 0, R_tb = 0;
    for (int r = 0; r < R; ++r) {
        R_el += d->rtype[r] == NK_RXN_ELEMENTARY;
        R_tb += d->rtype[r] == NK_RXN_THIRD_BODY;
    }
    std::vector<nk::RxnRec> rxn(R);
    std::vector<nk::RxnRecF> rxnf(R);
    std::vector<nk::TroeRec> troe;
    std::vector<nk::TroeRecF> troef;
    std::vector<int32_t> eff_sp;
    std::vector<double> eff_m1;
    for (int q = 0; q < R; ++q) {
        const int r = order[q];
        nk::RxnRec& x = rxn[q];
        std::memset(&x, 0, sizeof x);
        x.lnA = d->lnA[r];
        x.beta = d->beta[r];
        x.EaR = d->Ea[r] / nk::kR;
        x.type = d->rtype[r];
        x.orig = r;
        x.nr = d->reac_ptr[r + 1] - d->reac_ptr[r];
        x.np = d->prod_ptr[r + 1] - d->prod_ptr[r];
        int dnu = 0, e = 0;
        for (int i = d->reac_ptr[r]; i < d->reac_ptr[r + 1]; ++i, ++e) {
            x.sp[e] = d->reac_sp[i];
            x.nu[e] = d->reac_nu[i];
            x.nud[e] = -(double)d->reac_nu[i];
            dnu -= d->reac_nu[i];
        }
        e = nk::kMaxSide;
        for (int i = d->prod_ptr[r]; i < d->prod_ptr[r + 1]; ++i, ++e) {
            x.sp[e] = d->prod_sp[i];
            x.nu[e] = d->prod_nu[i];
            x.nud[e] = (double)d->prod_nu[i];
            dnu += d->prod_nu[i];
        }
        x.dnu = (double)dnu;
        x.aux = -1;
        rxnf[q] = nk::RxnRecF{(float)x.lnA, (float)x.beta, (float)x.EaR, 0.0f};
        if (x.type == NK_RXN_TROE) {
            const double* t = d->troe + 4 * r;
            if (!(t[1] > 0.0) || !(t[2] > 0.0))
                return fail(NK_EINVAL, "reaction %d: Troe T3 and T1 must be > 0", r);
            nk::TroeRec tr;
            tr.lnA0 = d->lnA0[r];
            tr.beta0 = d->beta0[r];
            tr.Ea0R = d->Ea0[r] / nk::kR;
            tr.a = t[0];
            tr.invT3 = 1.0 / t[1];
            tr.invT1 = 1.0 / t[2];
            tr.T2 = t[3] > 0.0 ? t[3] : 0.0;
            tr.hasT2 = t[3] > 0.0 ? 1.0 : 0.0;
            x.aux = (int32_t)troe.size();
            troe.push_back(tr);
            troef.push_back(nk::TroeRecF{(float)tr.lnA0, (float)tr.beta0, (float)tr.Ea0R, (float)tr.a,
                                         (float)tr.invT3, (float)tr.invT1, (float)tr.T2, (float)tr.hasT2});
        }
        x.eff0 = (int32_t)eff_sp.size();
        if (x.type != NK_RXN_ELEMENTARY) {
            for (int k = 0; k < K; ++k) {
                const double eps = d->eff[(size_t)r * K + k];
                if (eps != 1.0) {
                    eff_sp.push_back(k);
                    eff_m1.push_back(eps - 1.0);
                }
            }
        }
        x.eff1 = (int32_t)eff_sp.size();
    }
    // exp/log tables (nk_math.cuh), from their definitions in extended precision
    std::vector<double> mtab(nk::kMathTabDoubles);
    for (int j = 0; j < nk::kExpTab; ++j) mtab[j] = (double)exp2l((long double)j / nk::kExpTab);
    for (int j = 0; j < nk::kLogTab; ++j) {
        const long double c = 1.0L + ((long double)j + 0.5L) / nk::kLogTab;
        const double rc = (double)(1.0L / c);
        mtab[nk::kExpTab + j] = rc;
        mtab[nk::kExpTab + nk::kLogTab + j] = (double)(-logl((long double)rc));
    }
    std::vector<double> wilkeA((size_t)K * K), qrtW(K), sqrtW(K);
    for (int k = 0; k < K; ++k) {
        qrtW[k] = std::pow(d->W[k], 0.25);
        sqrtW[k] = std::sqrt(d->W[k]);
        for (int j = 0; j < K; ++j) wilkeA[(size_t)k * K + j] = 1.0 / std::sqrt(8.0 * (1.0 + d->W[k] / d->W[j]));
    }
    // double-float tables: cubic fits re-expanded about ln T = kLnT0, split into float pairs
    auto split = [](long double v) {
        const float h = (float)v;
        return float2{h, (float)(v - (long double)h)};
    };
    auto reexpand = [&](const double* a, float2* out) {   // b_i = sum_{m>=i} a_m C(m,i) L0^(m-i)
        static const int C[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
        for (int i = 0; i < 4; ++i) {
            long double b = 0.0L;
            for (int m2 = i; m2 < 4; ++m2) b += (long double)a[m2] * C[m2][i] * powl((long double)nk::kLnT0, m2 - i);
            out[i] = split(b);
        }
    };
    std::vector<float2> df_mu((size_t)K * 4), df_lam((size_t)K * 4), df_D((size_t)P * 4 + 4), df_A((size_t)K * K),
        df_qlnW(K), df_sqrtW(K), df_exp(nk::kExpTab);
    for (int k = 0; k < K; ++k) {
        reexpand(d->mu_fit + 4 * k, df_mu.data() + 4 * k);
        reexpand(d->lam_fit + 4 * k, df_lam.data() + 4 * k);
        df_qlnW[k] = split(0.25L * logl((long double)d->W[k]));
        df_sqrtW[k] = split(sqrtl((long double)d->W[k]));
        for (int j = 0; j < K; ++j)
            df_A[(size_t)k * K + j] = split(1.0L / sqrtl(8.0L * (1.0L + (long double)d->W[k] / d->W[j])));
    }
    for (int q = 0; q < P; ++q) reexpand(d->D_fit + 4 * q, df_D.data() + 4 * q);
    for (int j = 0; j < nk::kExpTab; ++j) df_exp[j] = split(exp2l((long double)j / nk::kExpTab));
    std::vector<float2> df_rc(nk::kLogTab), df_lc(nk::kLogTab);
    for (int j = 0; j < nk::kLogTab; ++j) {
        const long double c = 1.0L + ((long double)j + 0.5L) / nk::kLogTab;
        const double rc = (double)(1.0L / c);
        df_rc[j] = split(rc);
        df_lc[j] = split(-logl((long double)rc));
    }
    // rates: NASA g/RT coefficients, Arrhenius and Troe parameters as pairs (device order)
    std::vector<float2> nasa_df((size_t)K * 2 * 8, float2{0.0f, 0.0f});
    for (int k = 0; k < K; ++k)
        for (int range = 0; range < 2; ++range) {
            const double* a = (range == 0 ? d->nasa_lo : d->nasa_hi) + 7 * k;
            float2* c = nasa_df.data() + ((size_t)k * 2 + range) * 8;
            c[0] = split(a[0]);
            c[1] = split(-(long double)a[1] / 2.0L);
            c[2] = split(-(long double)a[2] / 6.0L);
            c[3] = split(-(long double)a[3] / 12.0L);
            c[4] = split(-(long double)a[4] / 20.0L);
            c[5] = split(a[5]);
            c[6] = split(-(long double)a[6]);
        }
    std::vector<float4> rxn_df((size_t)R * 2), troe_df;
    for (int q = 0; q < R; ++q) {
        const int r = order[q];
        const float2 lA = split(d->lnA[r]), be = split(d->beta[r]), ea = split((long double)d->Ea[r] / nk::kR);
        rxn_df[2 * q] = float4{lA.x, lA.y, be.x, be.y};
        rxn_df[2 * q + 1] = float4{ea.x, ea.y, (float)rxn[q].dnu, 0.0f};
        if (d->rtype[r] == NK_RXN_TROE) {
            const double* t = d->troe + 4 * r;
            const float2 a0 = split(d->lnA0[r]), b0 = split(d->beta0[r]), e0 = split((long double)d->Ea0[r] / nk::kR),
                         i3 = split(1.0L / t[1]), i1 = split(1.0L / t[2]), t2 = split(t[3] > 0.0 ? t[3] : 0.0);
            troe_df.push_back(float4{a0.x, a0.y, b0.x, b0.y});
            troe_df.push_back(float4{e0.x, e0.y, i3.x, i3.y});
            troe_df.push_back(float4{i1.x, i1.y, t2.x, t2.y});
            const float2 ta = split(t[0]), tb = split(1.0L - (long double)t[0]);
            troe_df.push_back(float4{ta.x, ta.y, tb.x, tb.y});
        }
    }

    // entry slots of a stored linearization (k_lin.cu): reactants then products, device order
    std::vector<int32_t> lin_boff(R);
    int32_t lin_nb = 0;
    for (int q = 0; q < R; ++q) {
        lin_boff[q] = lin_nb;
        lin_nb += rxn[q].nr + rxn[q].np;
    }
    // Reaction rounds of the rates and JVP kernels for NP = 2 and 4 parts per point: per kind, rows
    // of NP reactions (device order; -1 idle) whose species (reactants and products) are pairwise
    // disjoint, so the parts of a point add into one omega_k row without a conflict between the
    // barriers that separate the rounds.  Greedy in device order.
    // Schedules 2 and 3 are the VJP's: its reverse pass also adds into the rows of the species with
    // a third-body efficiency, which therefore count as the reaction's species there.
    std::vector<int32_t> rsched[4];
    int32_t rrnd[4][4];
    {
        const int words = (K + 63) / 64;
        std::vector<uint64_t> spb((size_t)R * words, 0), spe;
        for (int q = 0; q < R; ++q)
            for (int a = 0; a < rxn[q].nr + rxn[q].np; ++a) {
                const int k = rxn[q].sp[a < rxn[q].nr ? a : nk::kMaxSide + (a - rxn[q].nr)];
                spb[(size_t)q * words + k / 64] |= 1ULL << (k % 64);
            }
        spe = spb;
        for (int q = 0; q < R; ++q)
            for (int j = rxn[q].eff0; j < rxn[q].eff1; ++j) {
                const int k = eff_sp[j];
                spe[(size_t)q * words + k / 64] |= 1ULL << (k % 64);
            }
        const int bounds[4] = {0, R_el, R_el + R_tb, R};
        for (int v = 0; v < 4; ++v) {
            const int NP = v % 2 == 0 ? 2 : 4;
            const std::vector<uint64_t>& spv = v < 2 ? spb : spe;
            std::vector<int32_t>& S = rsched[v];
            std::vector<uint64_t> used(words);
            for (int g = 0; g < 3; ++g) {
                rrnd[v][g] = (int32_t)(S.size() / NP);
                std::vector<int> pool, rest, row;
                for (int q = bounds[g]; q < bounds[g + 1]; ++q) pool.push_back(q);
                while (!pool.empty()) {
                    std::fill(used.begin(), used.end(), 0ULL);
                    row.clear();
                    rest.clear();
                    for (int q : pool) {
                        bool take = (int)row.size() < NP;
                        for (int w = 0; take && w < words; ++w) take = (used[w] & spv[(size_t)q * words + w]) == 0;
                        if (take) {
                            row.push_back(q);
                            for (int w = 0; w < words; ++w) used[w] |= spv[(size_t)q * words + w];
                        } else {
                            rest.push_back(q);
                        }
                    }
                    for (int j = 0; j < NP; ++j) S.push_back(j < (int)row.size() ? row[j] : -1);
                    pool.swap(rest);
                }
            }
            rrnd[v][3] = (int32_t)(S.size() / NP);
        }
    }
    // The VJP's deferred efficiency terms on the plain rounds (nk_internal.cuh: mt_*), NP = 2, 4.
    std::vector<int32_t> mt_ptr[2], mt_slot[2];
    std::vector<double> mt_eps[2];
    int32_t mslots[2] = {0, 0};
    for (int v = 0; v < 2; ++v) {
        const int NP = v == 0 ? 2 : 4;
        const std::vector<int32_t>& S = rsched[v];
        mt_ptr[v].assign((size_t)2 * (K + 1), 0);
        for (int g = 1; g <= 2; ++g) {
            const int rd0 = rrnd[v][g], rd1 = rrnd[v][g + 1];
            mslots[v] = std::max(mslots[v], (rd1 - rd0) * NP);
            std::vector<std::vector<std::pair<int32_t, double>>> by_k(K);
            for (int rd = rd0; rd < rd1; ++rd)
                for (int pt = 0; pt < NP; ++pt) {
                    const int q = S[(size_t)rd * NP + pt];
                    if (q < 0) continue;
                    for (int j = rxn[q].eff0; j < rxn[q].eff1; ++j)
                        by_k[eff_sp[j]].push_back({(rd - rd0) * NP + pt, eff_m1[j]});
                }
            int32_t* ptr = mt_ptr[v].data() + (size_t)(g - 1) * (K + 1);
            for (int k = 0; k < K; ++k) {
                ptr[k] = (int32_t)mt_slot[v].size();
                for (const auto& e : by_k[k]) {
                    mt_slot[v].push_back(e.first);
                    mt_eps[v].push_back(e.second);
                }
            }
            ptr[K] = (int32_t)mt_slot[v].size();
        }
    }
    // Jacobian assembly terms (nk_internal.cuh): for every entry a of reaction q (species k,
    // signed coefficient nu), V_k gets nu A_q; G_k,j gets nu B_q,b for every entry b (species j)
    // and, for third-body and Troe reactions, Lam_k gets nu L_q and G_k,j nu (eps_j - 1) L_q for
    // every listed efficiency.  Per row, terms by destination, each destination in reaction order.
    std::vector<int32_t> jac_row(K + 1);
    std::vector<nk::JacTerm> jac_term;
    {
        std::map<std::pair<int, int>, std::vector<nk::JacTerm>> ent;      // (row, dst) -> terms
        for (int q = 0; q < R; ++q) {
            const nk::RxnRec& x = rxn[q];
            const int32_t sB = R + lin_boff[q], sL = R + lin_nb + (q - R_el);
            for (int a = 0; a < x.nr + x.np; ++a) {
                const int ia = a < x.nr ? a : nk::kMaxSide + (a - x.nr);
                const int k = x.sp[ia];
                const double nu = x.nud[ia];
                ent[{k, 0}].push_back({nu, q, 0});
                for (int b = 0; b < x.nr + x.np; ++b) {
                    const int ib = b < x.nr ? b : nk::kMaxSide + (b - x.nr);
                    ent[{k, x.sp[ib] + 1}].push_back({nu, sB + b, x.sp[ib] + 1});
                }
                if (x.type != NK_RXN_ELEMENTARY) {
                    ent[{k, K + 1}].push_back({nu, sL, K + 1});
                    for (int j = x.eff0; j < x.eff1; ++j)
                        ent[{k, eff_sp[j] + 1}].push_back({nu * eff_m1[j], sL, eff_sp[j] + 1});
                }
            }
        }
        int row = 0;
        for (const auto& kv : ent) {
            while (row <= kv.first.first) jac_row[row++] = (int32_t)jac_term.size();
            jac_term.insert(jac_term.end(), kv.second.begin(), kv.second.end());
        }
        while (row <= K) jac_row[row++] = (int32_t)jac_term.size();
    }
    // reaction thermo groups (nk_internal.cuh): net coefficients of each reaction, grouped by
    // the species' T_mid, combined in extended precision
    std::vector<float2> grp_df;
    std::vector<double> grp_Tmid;
    for (int q = 0; q < R; ++q) {
        const int r = order[q];
        std::vector<int> net(K, 0);
        for (int i = d->reac_ptr[r]; i < d->reac_ptr[r + 1]; ++i) net[d->reac_sp[i]] -= d->reac_nu[i];
        for (int i = d->prod_ptr[r]; i < d->prod_ptr[r + 1]; ++i) net[d->prod_sp[i]] += d->prod_nu[i];
        std::vector<double> tm;
        for (int k = 0; k < K; ++k)
            if (net[k] != 0 && std::find(tm.begin(), tm.end(), Tmid[k]) == tm.end()) tm.push_back(Tmid[k]);
        const int g0 = (int)grp_Tmid.size();
        if (g0 + (int)tm.size() >= (1 << 24)) return fail(NK_EINVAL, "too many reaction thermo groups");
        rxn[q].thermo = g0 | ((int32_t)tm.size() << 24);
        for (double t : tm) {
            grp_Tmid.push_back(t);
            for (int range = 0; range < 2; ++range) {
                long double da[7] = {0, 0, 0, 0, 0, 0, 0};
                for (int k = 0; k < K; ++k)
                    if (net[k] != 0 && Tmid[k] == t) {
                        const double* a = (range == 0 ? d->nasa_lo : d->nasa_hi) + 7 * k;
                        for (int j = 0; j < 7; ++j) da[j] += (long double)net[k] * a[j];
                    }
                const long double c[nk::kGrpPairs] = {da[0], -da[1] / 2, -da[2] / 6, -da[3] / 12, -da[4] / 20, da[5],
                                                      -da[6], da[0], da[1] / 2, da[2] / 3, da[3] / 4, da[4] / 5,
                                                      da[5], da[0], da[1], da[2], da[3], da[4]};
                for (int j = 0; j < nk::kGrpPairs; ++j) grp_df.push_back(split(c[j]));
            }
        }
    }

    auto to_f = [](const double* s, size_t n) {
        std::vector<float> v(n);
        for (size_t i = 0; i < n; ++i) v[i] = (float)s[i];
        return v;
    };
    std::vector<float> f_mu = to_f(d->mu_fit, (size_t)K * 4), f_lam = to_f(d->lam_fit, (size_t)K * 4),
                       f_D = to_f(P ? d->D_fit : nullptr, (size_t)P * 4), f_A = to_f(wilkeA.data(), wilkeA.size()),
                       f_q = to_f(qrtW.data(), K), f_s = to_f(sqrtW.data(), K), f_iw = to_f(invW.data(), K);
    std::vector<float> f_nud((size_t)R * 2 * nk::kMaxSide, 0.0f), f_effm1 = to_f(eff_m1.data(), eff_m1.size()),
                       f_cp((size_t)K * 2 * 8, 0.0f);
    for (int q = 0; q < R; ++q)
        for (int e = 0; e < 2 * nk::kMaxSide; ++e) f_nud[(size_t)q * 2 * nk::kMaxSide + e] = (float)rxn[q].nud[e];
    std::vector<float2> df_effm1(eff_m1.size());
    for (size_t j = 0; j < eff_m1.size(); ++j) df_effm1[j] = split((long double)eff_m1[j]);
    std::vector<double> lc_w((size_t)R * 2 * nk::kMaxSide, 0.0);
    for (int q = 0; q < R; ++q)
        for (int side = 0; side < 2; ++side) {
            const int ne = side ? rxn[q].np : rxn[q].nr, b = side * nk::kMaxSide;
            for (int e = 0; e < ne; ++e)
                lc_w[(size_t)q * 2 * nk::kMaxSide + b + e] = (double)rxn[q].nu[b + e] / (double)rxn[q].nu[b];
        }
    for (int k = 0; k < K; ++k)
        for (int range = 0; range < 2; ++range)
            for (int j = 0; j < 5; ++j)
                f_cp[((size_t)k * 2 + range) * 8 + j] = (float)nasa[((size_t)k * 2 + range) * nk::kNasaStride + j];

    // ---- one device block for everything
    Layout L;
    const size_t o_W = L.add(K * 8), o_invW = L.add(K * 8), o_Tmid = L.add(K * 8), o_nasa = L.add(nasa.size() * 8),
                 o_rxn = L.add(R * sizeof(nk::RxnRec)), o_rxnf = L.add(R * sizeof(nk::RxnRecF)),
                 o_troe = L.add(troe.size() * sizeof(nk::TroeRec) + 16),
                 o_troef = L.add(troef.size() * sizeof(nk::TroeRecF) + 16), o_mtab = L.add(mtab.size() * 8),
                 o_effs = L.add(eff_sp.size() * 4 + 16), o_effv = L.add(eff_m1.size() * 8 + 16),
                 o_mu = L.add(K * 32), o_lam = L.add(K * 32), o_D = L.add((size_t)P * 32 + 16),
                 o_A = L.add((size_t)K * K * 8), o_q = L.add(K * 8), o_s = L.add(K * 8),
                 o_fmu = L.add(K * 16), o_flam = L.add(K * 16), o_fD = L.add((size_t)P * 16 + 16),
                 o_fA = L.add((size_t)K * K * 4), o_fq = L.add(K * 4), o_fs = L.add(K * 4), o_fiw = L.add(K * 4),
                 o_dmu = L.add(df_mu.size() * 8), o_dlam = L.add(df_lam.size() * 8), o_dD = L.add(df_D.size() * 8),
                 o_dA = L.add(df_A.size() * 8), o_dq = L.add(df_qlnW.size() * 8), o_ds = L.add(df_sqrtW.size() * 8),
                 o_dexp = L.add(df_exp.size() * 8), o_drc = L.add(df_rc.size() * 8), o_dlc = L.add(df_lc.size() * 8),
                 o_ndf = L.add(nasa_df.size() * 8), o_rdf = L.add(rxn_df.size() * 16),
                 o_tdf = L.add(troe_df.size() * 16 + 16), o_gdf = L.add(grp_df.size() * 8 + 16),
                 o_gT = L.add(grp_Tmid.size() * 8 + 16), o_lb = L.add((size_t)R * 4 + 16),
                 o_jr = L.add(jac_row.size() * 4 + 16), o_jt = L.add(jac_term.size() * sizeof(nk::JacTerm) + 16),
                 o_fnud = L.add(f_nud.size() * 4), o_feff = L.add(f_effm1.size() * 4 + 16),
                 o_fcp = L.add(f_cp.size() * 4 + 16), o_lcw = L.add(lc_w.size() * 8),
                 o_dfe = L.add(df_effm1.size() * 8 + 16), o_rs2 = L.add(rsched[0].size() * 4 + 16),
                 o_rs4 = L.add(rsched[1].size() * 4 + 16), o_rv2 = L.add(rsched[2].size() * 4 + 16),
                 o_rv4 = L.add(rsched[3].size() * 4 + 16), o_mp2 = L.add(mt_ptr[0].size() * 4 + 16),
                 o_mp4 = L.add(mt_ptr[1].size() * 4 + 16), o_ms2 = L.add(mt_slot[0].size() * 4 + 16),
                 o_ms4 = L.add(mt_slot[1].size() * 4 + 16), o_me2 = L.add(mt_eps[0].size() * 8 + 16),
                 o_me4 = L.add(mt_eps[1].size() * 8 + 16);
    std::vector<unsigned char> host(L.bytes, 0);
    auto put = [&](size_t off, const void* src, size_t n) {
        if (n) std::memcpy(host.data() + off, src, n);
    };
    put(o_W, d->W, K * 8);
    put(o_invW, invW.data(), K * 8);
    put(o_Tmid, Tmid.data(), K * 8);
    put(o_nasa, nasa.data(), nasa.size() * 8);
    put(o_rxn, rxn.data(), R * sizeof(nk::RxnRec));
    put(o_rxnf, rxnf.data(), R * sizeof(nk::RxnRecF));
    put(o_troe, troe.data(), troe.size() * sizeof(nk::TroeRec));
    put(o_troef, troef.data(), troef.size() * sizeof(nk::TroeRecF));
    put(o_mtab, mtab.data(), mtab.size() * 8);
    put(o_effs, eff_sp.data(), eff_sp.size() * 4);
    put(o_effv, eff_m1.data(), eff_m1.size() * 8);
    put(o_mu, d->mu_fit, K * 32);
    put(o_lam, d->lam_fit, K * 32);
    if (P) put(o_D, d->D_fit, (size_t)P * 32);
    put(o_A, wilkeA.data(), (size_t)K * K * 8);
    put(o_q, qrtW.data(), K * 8);
    put(o_s, sqrtW.data(), K * 8);
    put(o_fmu, f_mu.data(), K * 16);
    put(o_flam, f_lam.data(), K * 16);
    put(o_fD, f_D.data(), (size_t)P * 16);
    put(o_fA, f_A.data(), (size_t)K * K * 4);
    put(o_fq, f_q.data(), K * 4);
    put(o_fs, f_s.data(), K * 4);
    put(o_fiw, f_iw.data(), K * 4);
    put(o_dmu, df_mu.data(), df_mu.size() * 8);
    put(o_dlam, df_lam.data(), df_lam.size() * 8);
    put(o_dD, df_D.data(), df_D.size() * 8);
    put(o_dA, df_A.data(), df_A.size() * 8);
    put(o_dq, df_qlnW.data(), df_qlnW.size() * 8);
    put(o_ds, df_sqrtW.data(), df_sqrtW.size() * 8);
    put(o_dexp, df_exp.data(), df_exp.size() * 8);
    put(o_drc, df_rc.data(), df_rc.size() * 8);
    put(o_dlc, df_lc.data(), df_lc.size() * 8);
    put(o_ndf, nasa_df.data(), nasa_df.size() * 8);
    put(o_rdf, rxn_df.data(), rxn_df.size() * 16);
    put(o_tdf, troe_df.data(), troe_df.size() * 16);
    put(o_gdf, grp_df.data(), grp_df.size() * 8);
    put(o_gT, grp_Tmid.data(), grp_Tmid.size() * 8);
    put(o_lb, lin_boff.data(), (size_t)R * 4);
    put(o_jr, jac_row.data(), jac_row.size() * 4);
    put(o_jt, jac_term.data(), jac_term.size() * sizeof(nk::JacTerm));
    put(o_rs2, rsched[0].data(), rsched[0].size() * 4);
    put(o_rs4, rsched[1].data(), rsched[1].size() * 4);
    put(o_rv2, rsched[2].data(), rsched[2].size() * 4);
    put(o_rv4, rsched[3].data(), rsched[3].size() * 4);
    put(o_mp2, mt_ptr[0].data(), mt_ptr[0].size() * 4);
    put(o_mp4, mt_ptr[1].data(), mt_ptr[1].size() * 4);
    put(o_ms2, mt_slot[0].data(), mt_slot[0].size() * 4);
    put(o_ms4, mt_slot[1].data(), mt_slot[1].size() * 4);
    put(o_me2, mt_eps[0].data(), mt_eps[0].size() * 8);
    put(o_me4, mt_eps[1].data(), mt_eps[1].size() * 8);
    put(o_fnud, f_nud.data(), f_nud.size() * 4);
    put(o_feff, f_effm1.data(), f_effm1.size() * 4);
    put(o_fcp, f_cp.data(), f_cp.size() * 4);
    put(o_lcw, lc_w.data(), lc_w.size() * 8);
    put(o_dfe, df_effm1.data(), df_effm1.size() * 8);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    void* block = nullptr;
    e = cudaMalloc(&block, L.bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NK_ENOMEM : NK_ECUDA, "cudaMalloc(%zu): %s", L.bytes,
                    cudaGetErrorString(e));
    }
    e = cudaMemcpy(block, host.data(), L.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(block);
        return cuda_fail(e, "cudaMemcpy(mechanism tables)");
    }
    nk_mech* m = new nk_mech;
    m->device = dev;
    m->block = block;
    m->bytes = L.bytes;
    m->jit_src = nk::jit_source(d);
    unsigned char* b = static_cast<unsigned char*>(block);
    nk::DevMech& dm = m->d;
    dm.K = K;
    dm.R = R;
    dm.P = P;
    dm.n_troe = (int32_t)troe.size();
    dm.R_el = R_el;
    dm.R_tb = R_tb;
    dm.mtab = reinterpret_cast<const double*>(b + o_mtab);
    dm.p_ref = d->p_ref;
    dm.invW = reinterpret_cast<const double*>(b + o_invW);
    dm.W = reinterpret_cast<const double*>(b + o_W);
    dm.Tmid = reinterpret_cast<const double*>(b + o_Tmid);
    dm.nasa = reinterpret_cast<const double*>(b + o_nasa);
    dm.rxn = reinterpret_cast<const nk::RxnRec*>(b + o_rxn);
    dm.rxnf = reinterpret_cast<const nk::RxnRecF*>(b + o_rxnf);
    dm.troe = reinterpret_cast<const nk::TroeRec*>(b + o_troe);
    dm.troef = reinterpret_cast<const nk::TroeRecF*>(b + o_troef);
    dm.eff_sp = reinterpret_cast<const int32_t*>(b + o_effs);
    dm.eff_m1 = reinterpret_cast<const double*>(b + o_effv);
    dm.mu_fit = reinterpret_cast<const double*>(b + o_mu);
    dm.lam_fit = reinterpret_cast<const double*>(b + o_lam);
    dm.D_fit = reinterpret_cast<const double*>(b + o_D);
    dm.wilkeA = reinterpret_cast<const double*>(b + o_A);
    dm.qrtW = reinterpret_cast<const double*>(b + o_q);
    dm.sqrtW = reinterpret_cast<const double*>(b + o_s);
    dm.f_mu_fit = reinterpret_cast<const float*>(b + o_fmu);
    dm.f_lam_fit = reinterpret_cast<const float*>(b + o_flam);
    dm.f_D_fit = reinterpret_cast<const float*>(b + o_fD);
    dm.f_wilkeA = reinterpret_cast<const float*>(b + o_fA);
    dm.f_qrtW = reinterpret_cast<const float*>(b + o_fq);
    dm.f_sqrtW = reinterpret_cast<const float*>(b + o_fs);
    dm.f_invW = reinterpret_cast<const float*>(b + o_fiw);
    dm.df_mu_fit = reinterpret_cast<const float2*>(b + o_dmu);
    dm.df_lam_fit = reinterpret_cast<const float2*>(b + o_dlam);
    dm.df_D_fit = reinterpret_cast<const float2*>(b + o_dD);
    dm.df_wilkeA = reinterpret_cast<const float2*>(b + o_dA);
    dm.df_qlnW = reinterpret_cast<const float2*>(b + o_dq);
    dm.df_sqrtW = reinterpret_cast<const float2*>(b + o_ds);
    dm.df_exp_tab = reinterpret_cast<const float2*>(b + o_dexp);
    dm.df_log_rc = reinterpret_cast<const float2*>(b + o_drc);
    dm.df_log_lc = reinterpret_cast<const float2*>(b + o_dlc);
    dm.nasa_df = reinterpret_cast<const float2*>(b + o_ndf);
    dm.rxn_df = reinterpret_cast<const float4*>(b + o_rdf);
    dm.troe_df = reinterpret_cast<const float4*>(b + o_tdf);
    dm.grp_df = reinterpret_cast<const float2*>(b + o_gdf);
    dm.grp_Tmid = reinterpret_cast<const double*>(b + o_gT);
    dm.lin_boff = reinterpret_cast<const int32_t*>(b + o_lb);
    dm.lin_nb = lin_nb;
    dm.jac_row = reinterpret_cast<const int32_t*>(b + o_jr);
    dm.jac_term = reinterpret_cast<const nk::JacTerm*>(b + o_jt);
    dm.f_nud = reinterpret_cast<const float*>(b + o_fnud);
    dm.f_eff_m1 = reinterpret_cast<const float*>(b + o_feff);
    dm.f_cp = reinterpret_cast<const float*>(b + o_fcp);
    dm.lc_w = reinterpret_cast<const double*>(b + o_lcw);
    dm.df_eff_m1 = reinterpret_cast<const float2*>(b + o_dfe);
    dm.rsched2 = reinterpret_cast<const int32_t*>(b + o_rs2);
    dm.rsched4 = reinterpret_cast<const int32_t*>(b + o_rs4);
    dm.rschedv2 = reinterpret_cast<const int32_t*>(b + o_rv2);
    dm.rschedv4 = reinterpret_cast<const int32_t*>(b + o_rv4);
    dm.mt_ptr2 = reinterpret_cast<const int32_t*>(b + o_mp2);
    dm.mt_ptr4 = reinterpret_cast<const int32_t*>(b + o_mp4);
    dm.mt_slot2 = reinterpret_cast<const int32_t*>(b + o_ms2);
    dm.mt_slot4 = reinterpret_cast<const int32_t*>(b + o_ms4);
    dm.mt_eps2 = reinterpret_cast<const double*>(b + o_me2);
    dm.mt_eps4 = reinterpret_cast<const double*>(b + o_me4);
    dm.mslots2 = mslots[0];
    dm.mslots4 = mslots[1];
    for (int g = 0; g < 4; ++g) {
        dm.rrnd2[g] = rrnd[0][g];
        dm.rrnd4[g] = rrnd[1][g];
        dm.rrndv2[g] = rrnd[2][g];
        dm.rrndv4[g] = rrnd[3][g];
    }
    *out = m;
    return ok();
}

nk_status nk_mechanism_free(nk_mech* m) {
    if (!m) return ok();
    nk::jit_unload(m->jit);
    cudaError_t e = cudaFree(m->block);
    delete m;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    return ok();
}

nk_status nk_mechanism_info(const nk_mech* m, int32_t* K, int32_t* R) {
    if (!m) return fail(NK_EINVAL, "mech is NULL");
    if (K) *K = m->d.K;
    if (R) *R = m->d.R;
    return ok();
}

}  // extern "C"

namespace {

// Checks shared by the evaluation entry points.  Returns NK_OK with *skip = true for n == 0.
nk_status check_eval(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                     const double* Y, bool* skip) {
    *skip = false;
    if (!m) return fail(NK_EINVAL, "mech is NULL");
    if (n < 0) return fail(NK_EINVAL, "n=%lld < 0", (long long)n);
    if (ld < n) return fail(NK_EINVAL, "ld=%lld < n=%lld", (long long)ld, (long long)n);
    if (n == 0) {
        *skip = true;
        return NK_OK;
    }
    if (ld > ((int64_t)1 << 40) || n > ((int64_t)1 << 36))
        return fail(NK_EINVAL, "n=%lld / ld=%lld too large", (long long)n, (long long)ld);
    if (!T || !p || !Y) return fail(NK_EINVAL, "T, p and Y must not be NULL");
    if (misaligned(T) || misaligned(p) || misaligned(Y)) return fail(NK_EALIGN, "T, p, Y must be 8-byte aligned");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != m->device)
        return fail(NK_EINVAL, "mechanism lives on device %d but device %d is current", m->device, dev);
    return NK_OK;
}

nk_status check_out(std::initializer_list<const void*> ptrs) {
    for (const void* q : ptrs)
        if (misaligned(q)) return fail(NK_EALIGN, "output arrays must be 8-byte aligned");
    return NK_OK;
}

nk_status launched(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return cuda_fail(e, what);
    return ok();
}

// g_lnA of a VJP over no points: zero, after the checks the other calls make (the mechanism's
// device is current, the array aligned).  NULL g_lnA: nothing to do.
nk_status zero_grad(const nk_mech* m, double* g_lnA, nk_stream stream) {
    if (!g_lnA) return ok();
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != m->device)
        return fail(NK_EINVAL, "mechanism lives on device %d but device %d is current", m->device, dev);
    nk_status st = check_out({g_lnA});
    if (st != NK_OK) return st;
    return launched(cudaMemsetAsync(g_lnA, 0, sizeof(double) * m->d.R, (cudaStream_t)stream),
                    "cudaMemsetAsync(g_lnA)");
}

}  // namespace

extern "C" {

nk_status nk_thermo_eval(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                         const double* Y, double* cp_mix, double* h_mix, double* Wbar, double* rho,
                         double* cp_k, double* h_k, double* g_k, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if ((st = check_out({cp_mix, h_mix, Wbar, rho, cp_k, h_k, g_k})) != NK_OK) return st;
    return launched(nk::launch_thermo(m->d, n, ld, T, p, Y, cp_mix, h_mix, Wbar, rho, cp_k, h_k, g_k,
                                      (cudaStream_t)stream),
                    "thermo kernel launch");
}

// builds the mechanism-specialised kernel once (the handle caches it; the build is serialised)
nk_status ensure_jit(nk_mech* m) {
    std::lock_guard<std::mutex> lk(m->jit_mu);
    if (m->jit_state == 0) {
        int dev = -1;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        e = nk::jit_build(m->jit_src, dev, m->jit, m->jit_err);
        m->jit_state = e == cudaSuccess ? 1 : -1;
    }
    if (m->jit_state < 0) return fail(NK_EUNSUPPORTED, "mechanism-specialised kernel: %s", m->jit_err.c_str());
    return NK_OK;
}

nk_status nk_mechanism_jit(nk_mech* m) {
    if (!m) return fail(NK_EINVAL, "mech is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != m->device)
        return fail(NK_EINVAL, "mechanism lives on device %d but device %d is current", m->device, dev);
    nk_status st = ensure_jit(m);
    return st == NK_OK ? ok() : st;
}

nk_status nk_jit_source(const nk_mech_desc* d, char* buf, size_t* len) {
    if (!len) return fail(NK_EINVAL, "len must not be NULL");
    nk_status st = check_mech_desc(d);
    if (st != NK_OK) return st;
    const std::string src = nk::jit_source(d);
    const size_t need = src.size() + 1;
    const size_t have = *len;
    *len = need;
    if (!buf || have < need) return fail(NK_EINVAL, "the source needs %zu bytes", need);
    std::memcpy(buf, src.c_str(), need);
    return ok();
}

nk_status nk_rates_eval(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                        const double* Y, const double* dlnA, double* omega, double* hrr,
                        nk_precision precision, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (precision != NK_FP64 && precision != NK_MIXED && precision != NK_FP64_NATIVE && precision != NK_JIT)
        return fail(NK_EINVAL, "bad precision %d", (int)precision);
    if (!omega || !hrr) return fail(NK_EINVAL, "omega and hrr must not be NULL");
    if ((st = check_out({omega, hrr, dlnA})) != NK_OK) return st;
    if (precision == NK_JIT) {
        // (the handle is logically const: the compiled kernel is a cache of its source)
        nk_mech* mm = const_cast<nk_mech*>(m);
        if ((st = ensure_jit(mm)) != NK_OK) return st;
        return launched(nk::jit_launch_rates(mm->jit, m->d, m->device, n, ld, T, p, Y, dlnA, omega, hrr,
                                             (cudaStream_t)stream),
                        "specialised rates kernel launch");
    }
    return launched(nk::launch_rates(m->d, n, ld, T, p, Y, dlnA, omega, hrr, (int)precision, (cudaStream_t)stream),
                    "rates kernel launch");
}

nk_status nk_host_eval_workspace(const nk_mech* m, int64_t chunk, size_t* bytes) {
    if (!m || !bytes) return fail(NK_EINVAL, "mech and bytes must not be NULL");
    if (chunk < 1) return fail(NK_EINVAL, "chunk=%lld < 1", (long long)chunk);
    *bytes = nk::host_eval_workspace_bytes(m->d, chunk);
    return ok();
}

nk_status nk_host_eval(const nk_mech* m, int64_t n, const double* T, const double* p, const double* Y,
                       double* omega, double* hrr, double* mu, double* lambda, double* Dmix, nk_precision precision,
                       int64_t chunk, void* workspace, size_t workspace_bytes, nk_stream stream) {
    if (!m) return fail(NK_EINVAL, "mech is NULL");
    if (n < 0) return fail(NK_EINVAL, "n=%lld < 0", (long long)n);
    if (n == 0) return ok();
    if (!T || !p || !Y) return fail(NK_EINVAL, "T, p and Y must not be NULL");
    if (precision != NK_FP64 && precision != NK_MIXED && precision != NK_FP64_NATIVE)
        return fail(NK_EINVAL, "bad precision %d", (int)precision);
    if (chunk < 1) return fail(NK_EINVAL, "chunk=%lld < 1", (long long)chunk);
    if (misaligned(T) || misaligned(p) || misaligned(Y)) return fail(NK_EALIGN, "T, p, Y must be 8-byte aligned");
    nk_status st = check_out({omega, hrr, mu, lambda, Dmix, workspace});
    if (st != NK_OK) return st;
    const int64_t c = std::min(chunk, n);
    const size_t need = nk::host_eval_workspace_bytes(m->d, c);
    if (!workspace || workspace_bytes < need)
        return fail(NK_EINVAL, "nk_host_eval needs %zu bytes of workspace for chunks of %lld, got %zu", need,
                    (long long)c, workspace ? workspace_bytes : (size_t)0);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != m->device)
        return fail(NK_EINVAL, "mechanism lives on device %d but device %d is current", m->device, dev);
    return launched(nk::host_eval(m->d, n, T, p, Y, omega, hrr, mu, lambda, Dmix, (int)precision, c, workspace,
                                  (cudaStream_t)stream),
                    "host evaluation");
}

nk_status nk_transport_eval(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                            const double* Y, double* mu, double* lambda, double* Dmix,
                            nk_precision precision, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (precision != NK_FP64 && precision != NK_MIXED && precision != NK_FP64_NATIVE)
        return fail(NK_EINVAL, "bad precision %d", (int)precision);
    if ((st = check_out({mu, lambda, Dmix})) != NK_OK) return st;
    if (!mu && !lambda && !Dmix) return ok();
    if (precision == NK_FP64)
        return launched(nk::launch_transport_df(m->d, n, ld, T, p, Y, mu, lambda, Dmix, (cudaStream_t)stream),
                        "transport kernel launch");
    return launched(nk::launch_transport(m->d, n, ld, T, p, Y, mu, lambda, Dmix, (int)precision,
                                         (cudaStream_t)stream),
                    "transport kernel launch");
}

nk_status nk_diffusion_fluxes(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                              const double* Y, const double* Dmix, const double* gradX, double* j, double* Vc,
                              double* hf, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!Dmix || !gradX || !j) return fail(NK_EINVAL, "Dmix, gradX and j must not be NULL");
    if ((st = check_out({Dmix, gradX, j, Vc, hf})) != NK_OK) return st;
    return launched(nk::launch_diffusion(m->d, n, ld, T, p, Y, Dmix, gradX, j, Vc, hf, (cudaStream_t)stream),
                    "diffusion kernel launch");
}

nk_status check_precond(const nk_mech* m, int32_t precond) {
    if (precond < 0 || precond > 2) return fail(NK_EINVAL, "precond=%d is not 0, 1 or 2", precond);
    if (precond && m->d.K + 1 > nk::kMaxPrecondN)
        return fail(NK_EUNSUPPORTED, "dense per-point blocks take K + 1 <= %d (K=%d)", nk::kMaxPrecondN, m->d.K);
    return NK_OK;
}

nk_status nk_reactor_workspace(const nk_mech* m, int64_t n, const nk_reactor_opts* o, size_t* bytes) {
    if (!m || !bytes || !o) return fail(NK_EINVAL, "mech, opts and bytes must not be NULL");
    if (n < 0) return fail(NK_EINVAL, "n < 0");
    if (o->krylov_dim < 1 || o->krylov_dim > NK_REACTOR_MAX_KRYLOV)
        return fail(NK_EINVAL, "krylov_dim=%d outside 1..%d", o->krylov_dim, NK_REACTOR_MAX_KRYLOV);
    nk_status st = check_precond(m, o->precond);
    if (st != NK_OK) return st;
    if (o->linearized < 0 || o->linearized > 2)
        return fail(NK_EINVAL, "linearized=%d is not 0, 1 or 2", o->linearized);
    if (o->linearized == 2 && o->precond != 0)
        return fail(NK_EINVAL, "single-precision products (linearized=2) need precond=0");
    *bytes = n == 0 ? 0 : nk::reactor_workspace_bytes(m->d, n, o->krylov_dim, o->precond, o->linearized);
    return ok();
}

nk_status nk_rhs_jvp_linearized(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                const double* vT, const double* vY, double* dfT, double* dfY, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !fT || !fY || !vT || !vY || !dfT || !dfY)
        return fail(NK_EINVAL, "lin, fT, fY, vT, vY, dfT and dfY must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, fT, fY, vT, vY, dfT, dfY})) != NK_OK) return st;
    return launched(nk::launch_rhs_jvp_linearized(m->d, n, ld, T, p, Y, lin, ldl, fT, fY, ld, vT, vY, dfT, dfY,
                                                  (cudaStream_t)stream),
                    "linearized sources jvp kernel launch");
}

nk_status nk_rhs_jacobian(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                          const double* lin, int64_t ldl, const double* fT, const double* fY, double* J, int64_t ldJ,
                          nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !fT || !fY || !J) return fail(NK_EINVAL, "lin, fT, fY and J must not be NULL");
    if ((st = check_precond(m, 1)) != NK_OK) return st;        // (the same block size limit)
    if (ldl < n || ldJ < n) return fail(NK_EINVAL, "ldl and ldJ must be >= n=%lld", (long long)n);
    if ((st = check_out({lin, fT, fY, J})) != NK_OK) return st;
    return launched(nk::launch_rhs_jacobian(m->d, n, ld, T, p, Y, lin, ldl, fT, fY, J, ldJ, (cudaStream_t)stream),
                    "jacobian kernel launch");
}

nk_status nk_block_jacobi_factor(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* lin, int64_t ldl, const double* fT, const double* fY,
                                 const double* w, int64_t ldw, double dt, double* F, int32_t* piv, int64_t ldF,
                                 nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if ((st = check_precond(m, 1)) != NK_OK) return st;
    if (!lin || !fT || !fY || !w || !F || !piv) return fail(NK_EINVAL, "lin, fT, fY, w, F and piv must not be NULL");
    if (ldl < n || ldw < n || ldF < n) return fail(NK_EINVAL, "ldl, ldw and ldF must be >= n=%lld", (long long)n);
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(NK_EINVAL, "dt must be finite and >= 0");
    if ((st = check_out({lin, fT, fY, w, F})) != NK_OK) return st;
    if (reinterpret_cast<uintptr_t>(piv) & 3u) return fail(NK_EALIGN, "piv must be 4-byte aligned");
    const cudaStream_t s = (cudaStream_t)stream;
    return launched(nk::launch_precond_setup(m->d, n, ld, T, p, Y, lin, ldl, fT, fY, ld, w, ldw, dt, F, piv, ldF, s),
                    "block-Jacobi factor kernel launch");
}

nk_status nk_block_jacobi_apply(const nk_mech* m, int64_t n, const double* F, const int32_t* piv, int64_t ldF,
                                const double* v, int64_t ldv, double* z, int64_t ldz, nk_stream stream) {
    if (!m) return fail(NK_EINVAL, "mech is NULL");
    if (n < 0) return fail(NK_EINVAL, "n=%lld < 0", (long long)n);
    if (n == 0) return ok();
    nk_status st = check_precond(m, 1);
    if (st != NK_OK) return st;
    if (!F || !piv || !v || !z) return fail(NK_EINVAL, "F, piv, v and z must not be NULL");
    if (ldF < n || ldv < n || ldz < n) return fail(NK_EINVAL, "ldF, ldv and ldz must be >= n=%lld", (long long)n);
    if ((st = check_out({F, v, z})) != NK_OK) return st;
    if (reinterpret_cast<uintptr_t>(piv) & 3u) return fail(NK_EALIGN, "piv must be 4-byte aligned");
    return launched(nk::launch_precond_apply(m->d.K + 1, n, F, ldF, piv, ldF, v, ldv, z, ldz, (cudaStream_t)stream),
                    "block-Jacobi apply kernel launch");
}

nk_status nk_reactor_step(const nk_mech* m, int64_t n, double* T, const double* p, double* Y, double dt,
                          const nk_reactor_opts* opts, nk_reactor_stats* stats, void* workspace,
                          size_t workspace_bytes, nk_stream stream) {
    if (!opts || !stats) return fail(NK_EINVAL, "opts and stats must not be NULL");
    bool skip;
    nk_status st = check_eval(m, n, n, T, p, Y, &skip);
    if (st != NK_OK) return st;
    if (skip) {
        std::memset(stats, 0, sizeof *stats);
        stats->converged = 1;
        return ok();
    }
    const nk_reactor_opts& o = *opts;
    if (o.krylov_dim < 1 || o.krylov_dim > NK_REACTOR_MAX_KRYLOV)
        return fail(NK_EINVAL, "krylov_dim=%d outside 1..%d", o.krylov_dim, NK_REACTOR_MAX_KRYLOV);
    if (!(o.rtol >= 0.0) || !(o.atol_T > 0.0) || !(o.atol_Y > 0.0) || !(o.newton_tol > 0.0) || !(o.lin_tol > 0.0) ||
        o.max_newton < 1 || !(dt >= 0.0) || !std::isfinite(dt))
        return fail(NK_EINVAL, "bad reactor options (tolerances > 0, max_newton >= 1, finite dt >= 0)");
    if ((st = check_precond(m, o.precond)) != NK_OK) return st;
    if (o.linearized < 0 || o.linearized > 2) return fail(NK_EINVAL, "linearized=%d is not 0, 1 or 2", o.linearized);
    if (o.linearized == 2 && o.precond != 0)
        return fail(NK_EINVAL, "single-precision products (linearized=2) need precond=0");
    const size_t need = nk::reactor_workspace_bytes(m->d, n, o.krylov_dim, o.precond, o.linearized);
    if (!workspace || workspace_bytes < need)
        return fail(NK_EINVAL, "the reactor step needs %zu bytes of workspace, got %zu", need,
                    workspace ? workspace_bytes : (size_t)0);
    if (misaligned(workspace)) return fail(NK_EALIGN, "workspace must be 8-byte aligned");
    return launched(nk::reactor_step(m->d, n, T, p, Y, dt, o, *stats, workspace, (cudaStream_t)stream),
                    "reactor step");
}

nk_status nk_rates_jvp(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* vT, const double* vY,
                       double* omega, double* hrr, double* d_omega, double* d_hrr, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!vT || !vY || !d_omega || !d_hrr) return fail(NK_EINVAL, "vT, vY, d_omega and d_hrr must not be NULL");
    if ((st = check_out({vT, vY, d_omega, d_hrr, omega, hrr, dlnA})) != NK_OK) return st;
    return launched(nk::launch_jvp(m->d, n, ld, T, p, Y, dlnA, vT, vY, omega, hrr, d_omega, d_hrr,
                                   (cudaStream_t)stream),
                    "jvp kernel launch");
}

nk_status nk_rhs_eval(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                      const double* dlnA, double* fT, double* fY, nk_precision precision, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (precision != NK_FP64 && precision != NK_MIXED && precision != NK_FP64_NATIVE)
        return fail(NK_EINVAL, "bad precision %d", (int)precision);
    if (!fT || !fY) return fail(NK_EINVAL, "fT and fY must not be NULL");
    if ((st = check_out({fT, fY, dlnA})) != NK_OK) return st;
    return launched(nk::launch_rates(m->d, n, ld, T, p, Y, dlnA, fY, fT, (int)precision, (cudaStream_t)stream, 1),
                    "rates kernel launch");
}

nk_status nk_rhs_jvp(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p, const double* Y,
                     const double* dlnA, const double* vT, const double* vY, double* fT, double* fY, double* dfT,
                     double* dfY, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!vT || !vY || !dfT || !dfY) return fail(NK_EINVAL, "vT, vY, dfT and dfY must not be NULL");
    if ((st = check_out({vT, vY, dfT, dfY, fT, fY, dlnA})) != NK_OK) return st;
    return launched(nk::launch_jvp(m->d, n, ld, T, p, Y, dlnA, vT, vY, fY, fT, dfY, dfT, (cudaStream_t)stream, 1),
                    "jvp kernel launch");
}

nk_status nk_rates_linearization_slots(const nk_mech* m, int64_t* slots) {
    if (!m || !slots) return fail(NK_EINVAL, "mech and slots must not be NULL");
    *slots = nk::lin_slots(m->d);
    return ok();
}

nk_status nk_rates_linearize(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                             const double* Y, const double* dlnA, double* lin, int64_t ldl, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin) return fail(NK_EINVAL, "lin must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, dlnA})) != NK_OK) return st;
    return launched(nk::launch_linearize(m->d, n, ld, T, p, Y, dlnA, lin, ldl, (cudaStream_t)stream),
                    "linearize kernel launch");
}

nk_status nk_rates_jvp_linearized(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                  const double* Y, const double* lin, int64_t ldl, const double* vT,
                                  const double* vY, double* d_omega, double* d_hrr, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !vT || !vY || !d_omega || !d_hrr)
        return fail(NK_EINVAL, "lin, vT, vY, d_omega and d_hrr must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, vT, vY, d_omega, d_hrr})) != NK_OK) return st;
    return launched(nk::launch_jvp_linearized(m->d, n, ld, T, p, Y, lin, ldl, vT, vY, d_omega, d_hrr,
                                              (cudaStream_t)stream),
                    "linearized jvp kernel launch");
}

nk_status nk_rates_linearization_slots_compact(const nk_mech* m, int64_t* slots) {
    if (!m || !slots) return fail(NK_EINVAL, "mech and slots must not be NULL");
    *slots = nk::linc_slots(m->d);
    return ok();
}

nk_status nk_rates_linearize_compact(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                     const double* Y, const double* dlnA, double* lin, int64_t ldl, double* omega,
                                     double* hrr, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin) return fail(NK_EINVAL, "lin must not be NULL");
    if ((omega == nullptr) != (hrr == nullptr)) return fail(NK_EINVAL, "omega and hrr are both given or both NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, dlnA, omega, hrr})) != NK_OK) return st;
    return launched(nk::launch_linearize_compact(m->d, n, ld, T, p, Y, dlnA, lin, ldl, omega, hrr,
                                                 (cudaStream_t)stream),
                    "compact linearize kernel launch");
}

nk_status nk_rates_jvp_linearized_compact(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                          const double* Y, const double* lin, int64_t ldl, const double* vT,
                                          const double* vY, double* d_omega, double* d_hrr, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !vT || !vY || !d_omega || !d_hrr)
        return fail(NK_EINVAL, "lin, vT, vY, d_omega and d_hrr must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, vT, vY, d_omega, d_hrr})) != NK_OK) return st;
    return launched(nk::launch_jvp_linearized_compact(m->d, n, ld, T, p, Y, lin, ldl, nullptr, nullptr, 0, vT, vY,
                                                      d_hrr, d_omega, (cudaStream_t)stream, 0),
                    "compact linearized jvp kernel launch");
}

nk_status nk_rhs_jvp_linearized_compact(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                        const double* Y, const double* lin, int64_t ldl, const double* fT,
                                        const double* fY, const double* vT, const double* vY, double* dfT,
                                        double* dfY, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !fT || !fY || !vT || !vY || !dfT || !dfY)
        return fail(NK_EINVAL, "lin, fT, fY, vT, vY, dfT and dfY must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, fT, fY, vT, vY, dfT, dfY})) != NK_OK) return st;
    return launched(nk::launch_jvp_linearized_compact(m->d, n, ld, T, p, Y, lin, ldl, fT, fY, ld, vT, vY, dfT, dfY,
                                                      (cudaStream_t)stream, 1),
                    "compact linearized sources jvp kernel launch");
}

nk_status nk_rates_linearization_slots_f32(const nk_mech* m, int64_t* slots) {
    if (!m || !slots) return fail(NK_EINVAL, "mech and slots must not be NULL");
    *slots = nk::lin_slots_f32(m->d);
    return ok();
}

nk_status nk_rates_linearize_f32(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                 const double* Y, const double* dlnA, float* lin, int64_t ldl, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin) return fail(NK_EINVAL, "lin must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, dlnA})) != NK_OK) return st;
    return launched(nk::launch_linearize_f32(m->d, n, ld, T, p, Y, dlnA, lin, ldl, (cudaStream_t)stream),
                    "linearize (float) kernel launch");
}

nk_status nk_rates_jvp_linearized_f32(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                      const double* Y, const float* lin, int64_t ldl, const double* vT,
                                      const double* vY, double* d_omega, double* d_hrr, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !vT || !vY || !d_omega || !d_hrr)
        return fail(NK_EINVAL, "lin, vT, vY, d_omega and d_hrr must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, vT, vY, d_omega, d_hrr})) != NK_OK) return st;
    return launched(nk::launch_jvp_linearized_f32(m->d, n, ld, T, p, Y, lin, ldl, nullptr, nullptr, 0, vT, vY, d_hrr,
                                                  d_omega, (cudaStream_t)stream, 0),
                    "linearized jvp (float) kernel launch");
}

nk_status nk_rhs_jvp_linearized_f32(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                                    const double* Y, const float* lin, int64_t ldl, const double* fT,
                                    const double* fY, const double* vT, const double* vY, double* dfT, double* dfY,
                                    nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK || skip) return st == NK_OK ? ok() : st;
    if (!lin || !fT || !fY || !vT || !vY || !dfT || !dfY)
        return fail(NK_EINVAL, "lin, fT, fY, vT, vY, dfT and dfY must not be NULL");
    if (ldl < n) return fail(NK_EINVAL, "ldl=%lld < n=%lld", (long long)ldl, (long long)n);
    if ((st = check_out({lin, fT, fY, vT, vY, dfT, dfY})) != NK_OK) return st;
    return launched(nk::launch_jvp_linearized_f32(m->d, n, ld, T, p, Y, lin, ldl, fT, fY, ld, vT, vY, dfT, dfY,
                                                  (cudaStream_t)stream, 1),
                    "linearized sources jvp (float) kernel launch");
}

nk_status nk_rates_vjp_workspace(const nk_mech* m, int64_t n, size_t* bytes) {
    if (!m || !bytes) return fail(NK_EINVAL, "mech and bytes must not be NULL");
    if (n < 0) return fail(NK_EINVAL, "n < 0");
    *bytes = n == 0 ? 0 : nk::vjp_workspace_bytes(m->d, n);
    return ok();
}

nk_status nk_rates_vjp(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                       const double* Y, const double* dlnA, const double* bar_omega, const double* bar_hrr,
                       double* gT, double* gY, double* g_lnA, void* workspace, size_t workspace_bytes,
                       nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK) return st;
    if (skip) return zero_grad(m, g_lnA, stream);           // the gradient of an empty sum is zero
    if (!bar_omega || !gT || !gY) return fail(NK_EINVAL, "bar_omega, gT and gY must not be NULL");
    if ((st = check_out({bar_omega, bar_hrr, gT, gY, g_lnA, dlnA, workspace})) != NK_OK) return st;
    if (g_lnA) {
        const size_t need = nk::vjp_workspace_bytes(m->d, n);
        if (!workspace || workspace_bytes < need)
            return fail(NK_EINVAL, "g_lnA needs %zu bytes of workspace, got %zu", need,
                        workspace ? workspace_bytes : (size_t)0);
    }
    return launched(nk::launch_vjp(m->d, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, g_lnA, workspace,
                                   (cudaStream_t)stream),
                    "vjp kernel launch");
}

nk_status nk_rates_vjp_noalloc(const nk_mech* m, int64_t n, int64_t ld, const double* T, const double* p,
                               const double* Y, const double* dlnA, const double* bar_omega,
                               const double* bar_hrr, double* gT, double* gY, double* g_lnA, nk_stream stream) {
    bool skip;
    nk_status st = check_eval(m, n, ld, T, p, Y, &skip);
    if (st != NK_OK) return st;
    if (skip) return zero_grad(m, g_lnA, stream);
    if (!bar_omega || !gT || !gY) return fail(NK_EINVAL, "bar_omega, gT and gY must not be NULL");
    if ((st = check_out({bar_omega, bar_hrr, gT, gY, g_lnA, dlnA})) != NK_OK) return st;
    void* scratch = nullptr;
    if (g_lnA) {
        const size_t need = nk::vjp_workspace_bytes(m->d, n);
        const size_t cap = nk::kNoallocScratchDoubles * sizeof(double);
        if (need > cap)
            return fail(NK_EUNSUPPORTED,
                        "nk_rates_vjp_noalloc: the ln A partial sums need %zu bytes, more than its fixed %zu-byte "
                        "scratch (R=%d reactions); use nk_rates_vjp with a workspace", need, cap, m->d.R);
        cudaError_t e = nk::noalloc_scratch(&scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    }
    return launched(nk::launch_vjp(m->d, n, ld, T, p, Y, dlnA, bar_omega, bar_hrr, gT, gY, g_lnA, scratch,
                                   (cudaStream_t)stream),
                    "vjp kernel launch");
}

}  // extern "C"
