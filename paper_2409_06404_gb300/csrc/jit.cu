// Per-mechanism specialisation of the rates kernel: the library writes CUDA source for the
// loaded mechanism -- every reaction as straight-line code with its species indices,
// stoichiometric coefficients, Arrhenius and Troe constants and third-body efficiencies as
// literals, its Gibbs sum as one polynomial in T per NASA range with the net coefficients
// combined at generation -- compiles it at run time (NVRTC, loaded with dlopen) to a cubin for
// the device's architecture and loads it through the runtime's library API.  The paper's
// production code is generated this way from the Cantera-format mechanism (Sec. 2); here it is
// the comparison point for the table-driven kernels, in the all-double form (NK_FP64_NATIVE's
// arithmetic: the same table-driven exp and log, nk_math.cuh, whose text is compiled into the
// program).
//
// The generated kernel: one thread per point, C_k in shared memory as [species][point], the
// omega_k accumulators as locals (registers, literal indices), h_k/RT per species at the end.
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <sstream>
#include <string>
#include <vector>

#include "nk_internal.cuh"

namespace nk {
namespace {

// the text of nk_math.cuh (written into the build directory at build time)
#include "nk_math_src.inc"

constexpr int kJitBlk = 64;

std::string lit(double v) {
    char b[48];
    if (!std::isfinite(v)) {                                   // as its bits
        long long bits;
        std::memcpy(&bits, &v, sizeof bits);
        std::snprintf(b, sizeof b, "__longlong_as_double(%lldLL)", bits);
        return b;
    }
    std::snprintf(b, sizeof b, "%.17g", v);
    std::string s(b);
    if (s.find_first_of(".eEn") == std::string::npos) s += ".0";
    return s;
}

// g/RT of a net-coefficient combination da[0..6] of NASA-7 coefficients, as an expression in
// Ti, lnT, invT
std::string gpoly(const long double* da) {
    std::ostringstream o;
    o << "(fma(" << lit((double)da[0]) << ", 1.0 - lnT, Ti * fma(Ti, fma(Ti, fma(Ti, " << lit((double)(-da[4] / 20))
      << ", " << lit((double)(-da[3] / 12)) << "), " << lit((double)(-da[2] / 6)) << "), " << lit((double)(-da[1] / 2))
      << ")) + fma(" << lit((double)da[5]) << ", invT, " << lit((double)(-da[6])) << "))";
    return o.str();
}

// h/RT of one species' coefficients a[0..6]
std::string hpoly(const double* a) {
    std::ostringstream o;
    o << "fma(Ti, fma(Ti, fma(Ti, fma(Ti, " << lit((double)((long double)a[4] / 5)) << ", "
      << lit((double)((long double)a[3] / 4)) << "), " << lit((double)((long double)a[2] / 3)) << "), "
      << lit((double)((long double)a[1] / 2)) << "), " << lit(a[0]) << ") + " << lit(a[5]) << " * invT";
    return o.str();
}

// product of C^nu over one side's entries
std::string side_product(const int32_t* sp, const int32_t* nu, int a, int b) {
    std::ostringstream o;
    bool first = true;
    for (int i = a; i < b; ++i)
        for (int j = 0; j < nu[i]; ++j) {
            o << (first ? "" : " * ") << "C[" << sp[i] << " * B]";
            first = false;
        }
    return first ? std::string("1.0") : o.str();
}

}  // namespace

std::string jit_source(const nk_mech_desc* d) {
    const int K = d->K, R = d->R;
    std::ostringstream o;
    o << "// generated for a mechanism of " << K << " species and " << R << " reactions\n"
      << "#include \"nk_math.cuh\"\n"
      << "namespace {\n"
      << "constexpr int B = " << kJitBlk << ";\n"
      << "__device__ __forceinline__ double troe(double lnkinf, double lnk0, double M, double Ti, double invT,\n"
      << "                                      double a, double iT3, double iT1, double T2, const nk::MathTab& mt) {\n"
      << "    const double lnPr = lnk0 - lnkinf + nk::flog(M, mt);\n"
      << "    double Fc = (1.0 - a) * nk::fexp(-Ti * iT3, mt) + a * nk::fexp(-Ti * iT1, mt);\n"
      << "    if (T2 > 0.0) Fc += nk::fexp(-T2 * invT, mt);\n"
      << "    const double lFc = nk::flog(Fc, mt) * " << lit(1.0 / std::log(10.0)) << ";\n"
      << "    const double c = fma(-0.67, lFc, -0.4), nn = fma(-1.27, lFc, 0.75);\n"
      << "    const double u = fma(lnPr, " << lit(1.0 / std::log(10.0)) << ", c);\n"
      << "    const double f1 = u / fma(-0.14, u, nn);\n"
      << "    const double lF = lFc / fma(f1, f1, 1.0);\n"
      << "    return nk::fexp(lF * " << lit(std::log(10.0)) << ", mt) / (1.0 + nk::fexp(-lnPr, mt));\n"
      << "}\n"
      << "}  // namespace\n\n"
      << "extern \"C\" __global__ void __launch_bounds__(B) nk_jit_rates(long long n, long long ld,\n"
      << "        const double* __restrict__ T, const double* __restrict__ p, const double* __restrict__ Y,\n"
      << "        const double* __restrict__ dlnA, double* __restrict__ omega, double* __restrict__ hrr,\n"
      << "        const double* __restrict__ gtab) {\n"
      << "    extern __shared__ double sm[];\n"
      << "    const nk::MathTab mt = nk::stage_math_tables(sm, gtab);\n"
      << "    __syncthreads();\n"
      << "    const long long i = (long long)blockIdx.x * B + threadIdx.x;\n"
      << "    if (i >= n) return;\n"
      << "    double* C = sm + nk::kMathTabDoubles + threadIdx.x;\n"
      << "    const double Ti = T[i], invT = 1.0 / Ti, lnT = nk::flog(Ti, mt);\n"
      << "    const double pRT = p[i] * invT * " << lit(1.0 / 8.314462618) << ";\n"
      << "    const double lnP0RT = " << lit((double)logl(101325.0L / 8.314462618L)) << " - lnT;\n"
      << "    double s = 0.0;\n";
    std::vector<long double> invW(K);
    for (int k = 0; k < K; ++k) invW[k] = 1.0L / d->W[k];
    for (int k = 0; k < K; ++k) o << "    s += Y[" << k << " * ld + i] * " << lit((double)invW[k]) << ";\n";
    o << "    const double rho = pRT / s;\n";
    for (int k = 0; k < K; ++k)
        o << "    C[" << k << " * B] = Y[" << k << " * ld + i] * " << lit((double)invW[k]) << " * rho;\n";
    o << "    double w[" << K << "];\n"
      << "#pragma unroll\n"
      << "    for (int k = 0; k < " << K << "; ++k) w[k] = 0.0;\n";
    for (int r = 0; r < R; ++r) {
        const int ra = d->reac_ptr[r], rb = d->reac_ptr[r + 1], pa = d->prod_ptr[r], pb = d->prod_ptr[r + 1];
        std::vector<int> net(K, 0);
        int dnu = 0;
        for (int i = ra; i < rb; ++i) {
            net[d->reac_sp[i]] -= d->reac_nu[i];
            dnu -= d->reac_nu[i];
        }
        for (int i = pa; i < pb; ++i) {
            net[d->prod_sp[i]] += d->prod_nu[i];
            dnu += d->prod_nu[i];
        }
        o << "    {   // reaction " << r << "\n"
          << "        const double sh = dlnA ? __ldg(dlnA + " << r << ") : 0.0;\n"
          << "        const double lnkf = fma(" << lit(-d->Ea[r] / 8.314462618) << ", invT, fma(" << lit(d->beta[r])
          << ", lnT, " << lit(d->lnA[r]) << " + sh));\n";
        // sum_k nu_k g_k/RT, one polynomial per T_mid group and range
        std::vector<double> tm;
        for (int k = 0; k < K; ++k)
            if (net[k] != 0 && std::find(tm.begin(), tm.end(), d->T_mid[k]) == tm.end()) tm.push_back(d->T_mid[k]);
        o << "        double dG = 0.0;\n";
        for (double t : tm) {
            long double lo[7] = {0, 0, 0, 0, 0, 0, 0}, hi[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int k = 0; k < K; ++k)
                if (net[k] != 0 && d->T_mid[k] == t)
                    for (int j = 0; j < 7; ++j) {
                        lo[j] += (long double)net[k] * d->nasa_lo[7 * k + j];
                        hi[j] += (long double)net[k] * d->nasa_hi[7 * k + j];
                    }
            o << "        dG += Ti <= " << lit(t) << " ? " << gpoly(lo) << " : " << gpoly(hi) << ";\n";
        }
        o << "        const double lnKc = fma(" << lit((double)dnu) << ", lnP0RT, -dG);\n"
          << "        const double fw = " << side_product(d->reac_sp, d->reac_nu, ra, rb) << ";\n"
          << "        const double rv = " << side_product(d->prod_sp, d->prod_nu, pa, pb) << ";\n";
        const int type = d->rtype[r];
        if (type != NK_RXN_ELEMENTARY) {
            o << "        double M = pRT;\n";
            for (int k = 0; k < K; ++k) {
                const double e = d->eff[(size_t)r * K + k];
                if (e != 1.0) o << "        M = fma(" << lit(e - 1.0) << ", C[" << k << " * B], M);\n";
            }
        }
        if (type == NK_RXN_TROE) {
            const double* t = d->troe + 4 * r;
            o << "        const double lnk0 = fma(" << lit(-d->Ea0[r] / 8.314462618) << ", invT, fma(" << lit(d->beta0[r])
              << ", lnT, " << lit(d->lnA0[r]) << " + sh));\n"
              << "        const double kf = M == 0.0 ? 0.0 : nk::fexp(lnkf, mt) * troe(lnkf, lnk0, M, Ti, invT, "
              << lit(t[0]) << ", " << lit((double)(1.0L / t[1])) << ", " << lit((double)(1.0L / t[2])) << ", "
              << lit(t[3] > 0.0 ? t[3] : 0.0) << ", mt);\n"
              << "        const double kr = kf * nk::fexp(-lnKc, mt);\n";
        } else {
            o << "        const double kf = nk::fexp(lnkf, mt), kr = nk::fexp(lnkf - lnKc, mt);\n";
        }
        o << "        const double q = fma(kf, fw, -kr * rv)" << (type == NK_RXN_THIRD_BODY ? " * M" : "") << ";\n";
        for (int k = 0; k < K; ++k) {
            if (net[k] == 0) continue;
            if (net[k] == 1)
                o << "        w[" << k << "] += q;\n";
            else if (net[k] == -1)
                o << "        w[" << k << "] -= q;\n";
            else
                o << "        w[" << k << "] = fma(" << lit((double)net[k]) << ", q, w[" << k << "]);\n";
        }
        o << "    }\n";
    }
    o << "    if (omega) {\n";
    for (int k = 0; k < K; ++k) o << "        omega[" << k << " * ld + i] = w[" << k << "];\n";
    o << "    }\n"
      << "    if (hrr) {\n"
      << "        double h = 0.0;\n";
    for (int k = 0; k < K; ++k)
        o << "        h = fma(Ti <= " << lit(d->T_mid[k]) << " ? " << hpoly(d->nasa_lo + 7 * k) << " : "
          << hpoly(d->nasa_hi + 7 * k) << ", w[" << k << "], h);\n";
    o << "        hrr[i] = " << lit(-8.314462618) << " * Ti * h;\n"
      << "    }\n"
      << "}\n";
    return o.str();
}

namespace {

// NVRTC, resolved at run time (no link-time dependency of the library on it)
struct Nvrtc {
    void* h = nullptr;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
    nvrtcResult (*log_size)(nvrtcProgram, size_t*);
    nvrtcResult (*log)(nvrtcProgram, char*);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
    nvrtcResult (*cubin)(nvrtcProgram, char*);
    nvrtcResult (*destroy)(nvrtcProgram*);
    const char* (*err)(nvrtcResult);
};

bool load_nvrtc(Nvrtc& f, std::string& why) {
    static const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                                  "/usr/local/cuda/targets/sbsa-linux/lib/libnvrtc.so.13",
                                  "/usr/local/cuda/targets/x86_64-linux/lib/libnvrtc.so.13"};
    for (const char* nm : names)
        if ((f.h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!f.h) {
        why = "NVRTC (libnvrtc.so.13) not found";
        return false;
    }
    auto sym = [&](const char* s) { return dlsym(f.h, s); };
    f.create = reinterpret_cast<decltype(f.create)>(sym("nvrtcCreateProgram"));
    f.compile = reinterpret_cast<decltype(f.compile)>(sym("nvrtcCompileProgram"));
    f.log_size = reinterpret_cast<decltype(f.log_size)>(sym("nvrtcGetProgramLogSize"));
    f.log = reinterpret_cast<decltype(f.log)>(sym("nvrtcGetProgramLog"));
    f.cubin_size = reinterpret_cast<decltype(f.cubin_size)>(sym("nvrtcGetCUBINSize"));
    f.cubin = reinterpret_cast<decltype(f.cubin)>(sym("nvrtcGetCUBIN"));
    f.destroy = reinterpret_cast<decltype(f.destroy)>(sym("nvrtcDestroyProgram"));
    f.err = reinterpret_cast<decltype(f.err)>(sym("nvrtcGetErrorString"));
    if (!f.create || !f.compile || !f.log_size || !f.log || !f.cubin_size || !f.cubin || !f.destroy || !f.err) {
        why = "NVRTC lacks an entry point";
        return false;
    }
    return true;
}

}  // namespace

cudaError_t jit_build(const std::string& src, int device, JitModule& mod, std::string& why) {
    Nvrtc f;
    if (!load_nvrtc(f, why)) return cudaErrorNotSupported;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major * 10 + minor) + "a";
    const char* hdr_src[] = {kNkMathSrc};
    const char* hdr_name[] = {"nk_math.cuh"};
    nvrtcProgram prog;
    nvrtcResult r = f.create(&prog, src.c_str(), "nk_jit_rates.cu", 1, hdr_src, hdr_name);
    if (r != NVRTC_SUCCESS) {
        why = std::string("nvrtcCreateProgram: ") + f.err(r);
        return cudaErrorNotSupported;
    }
    const char* opts[] = {arch.c_str(), "-std=c++17", "--fmad=true"};
    r = f.compile(prog, 3, opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        f.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) f.log(prog, &log[0]);
        why = std::string("NVRTC compile failed: ") + f.err(r) + "\n" + log;
        f.destroy(&prog);
        return cudaErrorNotSupported;
    }
    size_t nb = 0;
    f.cubin_size(prog, &nb);
    std::vector<char> cubin(nb);
    f.cubin(prog, cubin.data());
    f.destroy(&prog);
    cudaLibrary_t lib;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        why = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
        return e;
    }
    cudaKernel_t kern;
    e = cudaLibraryGetKernel(&kern, lib, "nk_jit_rates");
    if (e != cudaSuccess) {
        cudaLibraryUnload(lib);
        why = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
        return e;
    }
    mod.lib = lib;
    mod.kern = kern;
    return cudaSuccess;
}

void jit_unload(JitModule& mod) {
    if (mod.lib) cudaLibraryUnload(static_cast<cudaLibrary_t>(mod.lib));
    mod.lib = nullptr;
    mod.kern = nullptr;
}

cudaError_t jit_launch_rates(const JitModule& mod, const DevMech& m, int device, int64_t n, int64_t ld,
                             const double* T, const double* p, const double* Y, const double* dlnA, double* omega,
                             double* hrr, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t bytes = ((size_t)kMathTabDoubles + (size_t)m.K * kJitBlk) * sizeof(double);
    cudaKernel_t kern = static_cast<cudaKernel_t>(mod.kern);
    cudaError_t e = cudaKernelSetAttributeForDevice(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes,
                                                    device);
    if (e != cudaSuccess) return e;
    long long nn = n, lld = ld;
    const double* tab = m.mtab;
    void* args[] = {&nn, &lld, (void*)&T, (void*)&p, (void*)&Y, (void*)&dlnA, (void*)&omega, (void*)&hrr, (void*)&tab};
    return cudaLaunchKernel((const void*)kern, dim3((unsigned)((n + kJitBlk - 1) / kJitBlk)), dim3(kJitBlk), args,
                            bytes, s);
}

}  // namespace nk
