// Shape-specialised sweep kernels.
//
// Every distinct BDD shape (structure of nodes and arcs, independent of the
// variables and multipliers) gets process-wide id.  For a set of shape ids the
// generator below emits one straight-line device function per shape and
// sweep mode -- the four operations of the static kernels (ascending pass
// with Eq. 5 updates, descending pass, min-marginals by Eq. 6, energies) --
// with every successor choice resolved at generation time, and NVRTC compiles
// them together with the embedded kernel skeleton for sm_103a.  Modules are
// cached per id set for the life of the process.
//
// The arithmetic is the same sequence of float additions and minima as in the
// static kernels: an arc to the top terminal contributes +0 and is written
// without the addition, an arc to the bottom terminal is left out of the
// minimum (it would contribute +inf).
#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "fdog_internal.h"
#include "jit_sources.inc"  // generated by the build: kJitAbi, kJitSkeleton

namespace fdog {
namespace {

std::mutex g_mu;
std::condition_variable g_cv;
std::set<std::string> g_building;  // module keys being compiled
std::unordered_map<std::string, int> g_ids;
std::vector<HostShape> g_shapes;
std::map<std::string, JitKernels> g_modules;
std::map<std::string, std::vector<char>> g_cubins;
std::string generate_module(const std::vector<int>& ids);

std::string id_key(std::vector<int>& ids) {
    std::sort(ids.begin(), ids.end());
    ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
    std::string key;
    for (int id : ids) key += std::to_string(id) + ",";
    return key;
}

// NVRTC compile of the module for `ids` (sorted, unique).  Compiles run
// outside the registry lock, so threads planning different instances compile
// in parallel; a thread that needs a module another thread is compiling waits
// for it instead of compiling it again.
int compile_module(const std::vector<int>& ids, const std::string& key, std::string& err) {
    std::string src;
    {
        std::unique_lock<std::mutex> lk(g_mu);
        g_cv.wait(lk, [&] { return !g_building.count(key); });
        if (g_cubins.count(key)) return FDOG_OK;
        g_building.insert(key);
        src = generate_module(ids);
    }
    std::vector<char> cubin;
    int rc = FDOG_OK;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "fdog_shapes.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        err = "nvrtcCreateProgram failed";
        rc = FDOG_EUNSUPPORTED;
    } else {
        const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo"};
        if (nvrtcCompileProgram(prog, 3, opts) != NVRTC_SUCCESS) {
            size_t n = 0;
            nvrtcGetProgramLogSize(prog, &n);
            std::string log(n, '\0');
            nvrtcGetProgramLog(prog, &log[0]);
            err = "NVRTC: " + log.substr(0, 2000);
            rc = FDOG_EUNSUPPORTED;
        } else {
            size_t n = 0;
            nvrtcGetCUBINSize(prog, &n);
            cubin.resize(n);
            nvrtcGetCUBIN(prog, cubin.data());
        }
        nvrtcDestroyProgram(&prog);
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (rc == FDOG_OK) g_cubins.emplace(key, std::move(cubin));
        g_building.erase(key);
    }
    g_cv.notify_all();
    return rc;
}

std::string structure_key(const HostShape& s) {
    std::string key;
    auto put = [&](const std::vector<int>& v) {
        const int32_t n = static_cast<int32_t>(v.size());
        key.append(reinterpret_cast<const char*>(&n), 4);
        key.append(reinterpret_cast<const char*>(v.data()), 4 * v.size());
    };
    put(s.lstart);
    put(s.lo);
    put(s.hi);
    return key;
}

std::string fmin_all(const std::vector<std::string>& terms) {
    if (terms.empty()) return "FDOG_INF";
    std::string r = terms.back();
    for (int q = static_cast<int>(terms.size()) - 2; q >= 0; --q) r = "fminf(" + terms[q] + ", " + r + ")";
    return r;
}

std::string nm(const char* p, int t, int v) { return std::string(p) + std::to_string(t) + "_" + std::to_string(v); }
std::string nm(const char* p, int t) { return std::string(p) + std::to_string(t); }

// Emits shp_<id>_<mode>(I, base, valid, flags) -> this BDD's share of the bound.
void emit_shape(std::ostringstream& o, const HostShape& s, int id, int mode) {
    const int k = s.k;
    auto width = [&](int t) { return s.lstart[t + 1] - s.lstart[t]; };
    // successor of node v (local) of layer t through arc beta: -1 TOP, -2 BOT, else local index in layer t+1
    auto succ = [&](int t, int v, int beta) {
        const int x = beta ? s.hi[s.lstart[t] + v] : s.lo[s.lstart[t] + v];
        return x >= 0 ? x - s.lstart[t + 1] : x;
    };
    o << "__device__ __forceinline__ float shp_" << id << "_" << mode
      << "(const InstDev* __restrict__ I, long long base, bool valid, int flags, bool local, float* ep_lam, "
         "int* ep_var) {\n";
    o << "  (void)local; (void)ep_lam; (void)ep_var;\n";
    o << "  float* __restrict__ lam = I->lam;\n  const float omega = I->omega;\n  (void)omega; (void)flags;\n";
    for (int t = 0; t < k; ++t) o << "  float " << nm("l", t) << " = 0.f, " << nm("u", t) << " = 0.f;\n";
    o << "  if (valid) {\n";
    for (int t = 0; t < k; ++t) o << "    " << nm("l", t) << " = lam[base + " << 32 * t << "];\n";
    const char* need_u = mode <= 1 ? "true" : "(flags & 1)";
    o << "    if (" << need_u << ") {\n";
    for (int t = 0; t < k; ++t) {
        o << "      { const int v = __ldcs(I->var + base + " << 32 * t << "); " << nm("u", t) << " = I->T[v];";
        if (mode <= 1) o << " if (local) ep_var[" << 32 * t << "] = v;";
        o << " }\n";
    }
    if (mode >= 2)
        for (int t = 0; t < k; ++t) o << "      " << nm("l", t) << " += " << nm("u", t) << ";\n";
    o << "    }\n  }\n";

    // b<t>_<v> = SP(node, TOP) at the current multipliers for layers [from, k)
    auto emit_backward_labels = [&](int from) {
        for (int t = k - 1; t >= from; --t)
            for (int v = 0; v < width(t); ++v) {
                std::vector<std::string> terms;
                const int lo = succ(t, v, 0), hi = succ(t, v, 1);
                if (lo == -1) terms.push_back("0.f");
                else if (lo >= 0) terms.push_back(nm("b", t + 1, lo));
                if (hi == -1) terms.push_back(nm("l", t));
                else if (hi >= 0) terms.push_back("(" + nm("b", t + 1, hi) + " + " + nm("l", t) + ")");
                o << "  const float " << nm("b", t, v) << " = " << fmin_all(terms) << ";\n";
            }
    };
    // f<t+1>_<w> from layer t with multiplier l<t>
    auto emit_push = [&](int t) {
        for (int w = 0; w < width(t + 1); ++w) {
            std::vector<std::string> terms;
            for (int v = 0; v < width(t); ++v) {
                if (succ(t, v, 0) == w) terms.push_back(nm("f", t, v));
                if (succ(t, v, 1) == w) terms.push_back("(" + nm("f", t, v) + " + " + nm("l", t) + ")");
            }
            o << "  const float " << nm("f", t + 1, w) << " = " << fmin_all(terms) << ";\n";
        }
    };
    // m0 / m1 of layer t from f<t> and the successor labels b<t+1> (Eq. 6)
    auto marg_terms = [&](int t, int beta) {
        std::vector<std::string> terms;
        for (int v = 0; v < width(t); ++v) {
            const int x = succ(t, v, beta);
            if (x == -1) terms.push_back(nm("f", t, v));
            else if (x >= 0) terms.push_back("(" + nm("f", t, v) + " + " + nm("b", t + 1, x) + ")");
        }
        return fmin_all(terms);
    };
    auto emit_update = [&](int t) {
        o << "  {\n    const float m0 = " << marg_terms(t, 0) << ";\n";
        o << "    const float m1 = " << marg_terms(t, 1) << " + " << nm("l", t) << ";\n";
        o << "    const float d = m1 - m0;\n";
        o << "    " << nm("l", t) << " = fmaf(-omega, d, " << nm("l", t) << ") + " << nm("u", t) << ";\n";
        o << "    neg += fmaxf(-d, 0.f);\n  }\n";
    };
    auto last_energy = [&](int t) {
        std::vector<std::string> terms;
        for (int v = 0; v < width(t); ++v) {
            if (succ(t, v, 0) == -1) terms.push_back(nm("f", t, v));
            if (succ(t, v, 1) == -1) terms.push_back("(" + nm("f", t, v) + " + " + nm("l", t) + ")");
        }
        return fmin_all(terms);
    };

    if (mode == 0 || mode == 2) {
        emit_backward_labels(1);
        o << "  const float f0_0 = 0.f;\n  float neg = 0.f;\n  (void)neg;\n";
        for (int t = 0; t < k; ++t) {
            if (mode == 0) {
                emit_update(t);
            } else {
                o << "  {\n    const float m0 = " << marg_terms(t, 0) << ";\n";
                o << "    const float m1 = " << marg_terms(t, 1) << " + " << nm("l", t) << ";\n";
                o << "    if (valid) {\n      const long long p = base + " << 32 * t << ";\n";
                o << "      if (flags & 2) { I->mm0[p] = m0; I->mm1[p] = m1; } else { I->mm0[p] = m1 - m0; }\n";
                o << "    }\n  }\n";
            }
            if (t + 1 < k) emit_push(t);
        }
        o << "  const float E = " << last_energy(k - 1) << ";\n";
        if (mode == 0) o << "  const float term = fmaf(-omega, neg, E);\n";
        else o << "  const float term = E;\n";
    } else if (mode == 1) {
        o << "  const float f0_0 = 0.f;\n";
        for (int t = 0; t + 1 < k; ++t) emit_push(t);
        o << "  float neg = 0.f;\n";
        for (int t = k - 1; t >= 0; --t) {
            emit_update(t);
            for (int v = 0; v < width(t); ++v) {
                std::vector<std::string> terms;
                const int lo = succ(t, v, 0), hi = succ(t, v, 1);
                if (lo == -1) terms.push_back("0.f");
                else if (lo >= 0) terms.push_back(nm("b", t + 1, lo));
                if (hi == -1) terms.push_back(nm("l", t));
                else if (hi >= 0) terms.push_back("(" + nm("b", t + 1, hi) + " + " + nm("l", t) + ")");
                o << "  const float " << nm("b", t, v) << " = " << fmin_all(terms) << ";\n";
            }
        }
        o << "  const float term = fmaf(-omega, neg, b0_0);\n";
    } else {
        emit_backward_labels(0);
        o << "  const float term = b0_0;\n";
    }
    if (mode <= 1) {
        o << "  if (valid) {\n";
        for (int t = 0; t < k; ++t) o << "    lam[base + " << 32 * t << "] = " << nm("l", t) << ";\n";
        o << "  }\n  if (local) {\n";
        for (int t = 0; t < k; ++t) o << "    ep_lam[" << 32 * t << "] = " << nm("l", t) << ";\n";
        o << "  }\n";
    }
    o << "  return term;\n}\n\n";
}

std::string generate_module(const std::vector<int>& ids) {
    std::ostringstream o;
    o << "typedef int int32_t;\ntypedef unsigned int uint32_t;\ntypedef unsigned short uint16_t;\n"
         "typedef unsigned char uint8_t;\ntypedef long long int64_t;\ntypedef unsigned long long uint64_t;\n"
         "#define FDOG_INF __int_as_float(0x7f800000)\n";
    o << kJitAbi << "\n";
    for (int id : ids)
        for (int mode = 0; mode < 4; ++mode) emit_shape(o, g_shapes[id], id, mode);
    o << "#define FDOG_DISPATCH(MODE) \\\n";
    for (int mode = 0; mode < 4; ++mode) {
        o << "  " << (mode ? "else " : "") << "if (MODE == " << mode << ") { switch (jit) { \\\n";
        for (int id : ids)
            o << "    case " << id << ": term = shp_" << id << "_" << mode
              << "(I, base, valid, a.flags, local, ep_lam + lane, ep_var + lane); break; \\\n";
        o << "    default: break; } } \\\n";
    }
    o << "\n" << kJitSkeleton;
    return o.str();
}

}  // namespace

int jit_register_shape(const HostShape& s) {
    std::lock_guard<std::mutex> lk(g_mu);
    std::string key = structure_key(s);
    auto it = g_ids.find(key);
    if (it != g_ids.end()) return it->second;
    const int id = static_cast<int>(g_shapes.size());
    g_shapes.push_back(s);
    g_ids.emplace(std::move(key), id);
    return id;
}

int jit_compile(const std::vector<int>& ids_in, std::string& err) {
    if (ids_in.empty()) return FDOG_OK;
    std::vector<int> ids = ids_in;
    const std::string key = id_key(ids);
    return compile_module(ids, key, err);
}

int jit_kernels(const std::vector<int>& ids_in, JitKernels& out, std::string& err) {
    out = JitKernels();
    if (ids_in.empty()) return FDOG_OK;
    std::vector<int> ids = ids_in;
    const std::string key = id_key(ids);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_modules.find(key);
        if (it != g_modules.end()) { out = it->second; return FDOG_OK; }
    }
    int rc = compile_module(ids, key, err);
    if (rc != FDOG_OK) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_modules.find(key);
    if (it != g_modules.end()) { out = it->second; return FDOG_OK; }
    const std::vector<char>& cubin = g_cubins.at(key);
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
        return FDOG_ECUDA;
    }
    const char* names[4] = {"fdog_jit_fwd", "fdog_jit_bwd", "fdog_jit_mm", "fdog_jit_eval"};
    JitKernels kk;
    for (int m = 0; m < 4; ++m) {
        cudaKernel_t kern = nullptr;
        e = cudaLibraryGetKernel(&kern, lib, names[m]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
            return FDOG_ECUDA;
        }
        kk.fn[m] = reinterpret_cast<const void*>(kern);
    }
    g_modules.emplace(key, kk);  // the library stays loaded for the life of the process
    out = kk;
    return FDOG_OK;
}

std::string jit_source(const std::vector<int>& ids_in) {
    std::vector<int> ids = ids_in;
    id_key(ids);
    std::lock_guard<std::mutex> lk(g_mu);
    return generate_module(ids);
}

}  // namespace fdog
