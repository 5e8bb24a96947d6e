// fdog_bound_reduce_noalloc: the lower-bound reduction for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc where they need a bound: plug-ins that
// live inside a host framework which owns every device allocation through its
// own pool (a direct cudaMalloc would bypass its accounting), and real-time
// loops that forbid allocation after start-up (cudaMalloc may synchronise the
// device and has no latency bound).  They already hold the per-subproblem
// energies E_j in their own device buffer and only need the deterministic
// compensated sum.  This entry
// point uses the same two-stage compensated reduction as the library's
// lower-bound kernels -- per-block partials, then a Neumaier sum of them by
// the last block -- over FP64 inputs, 256 values per block, and keeps its
// scratch -- the block partials and the last-block ticket -- in one
// file-scope static device array instead of memory owned by an instance.
#include <cuda.h>  // CUcontext / CUresult types of the two driver calls fetched at run time
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/fastdog.h"

namespace {

constexpr int kChunk = 256;          // values per block, one per thread
constexpr int kMaxChunks = 32768;    // scratch partials: 32768 doubles = 256 KiB
constexpr int64_t kMaxValues = static_cast<int64_t>(kChunk) * kMaxChunks;  // 8,388,608 values per call
constexpr int kMaxDevices = 64;

struct Scratch {
    double chunk[kMaxChunks];
    int ticket;
};

// Held by every GPU that loads this library until the process exits.  In host
// code this name is only a host-side stand-in: the device address comes from
// cudaGetSymbolAddress, once per device, with that device current.
static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mu;
// per device: the scratch address and the id of the context it was looked up in
Scratch* g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};

__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
}

__device__ __forceinline__ void block_reduce(double* ss, double* sc, double s, double c) {
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int w = kChunk / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double x = ss[threadIdx.x], cc = sc[threadIdx.x] + sc[threadIdx.x + w];
            neumaier(x, cc, ss[threadIdx.x + w]);
            ss[threadIdx.x] = x;
            sc[threadIdx.x] = cc;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kChunk) bound_reduce_noalloc_kernel(const double* __restrict__ v, int64_t n,
                                                                        int n_chunks, double constant,
                                                                        double* __restrict__ out, Scratch* scr) {
    __shared__ double ss[kChunk], sc[kChunk];
    __shared__ int last;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * kChunk + threadIdx.x;
    block_reduce(ss, sc, t < n ? v[t] : 0.0, 0.0);
    if (threadIdx.x == 0) {
        scr->chunk[blockIdx.x] = ss[0] + sc[0];
        __threadfence();
        last = atomicAdd(&scr->ticket, 1) == n_chunks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0, c = 0.0;
    for (int q = threadIdx.x; q < n_chunks; q += kChunk) neumaier(s, c, __ldcg(scr->chunk + q));
    block_reduce(ss, sc, s, c);
    if (threadIdx.x == 0) {
        double S = ss[0], C = sc[0];
        neumaier(S, C, constant);
        *out = S + C;
        scr->ticket = 0;
    }
}

// Unique id of the calling thread's current CUDA context (0 if there is
// none), from cuCtxGetCurrent / cuCtxGetId fetched through the runtime, so
// the library needs no link against the driver library.  The id changes when
// cudaDeviceReset destroys a device's primary context and a later call
// creates a new one, in which the module -- and g_scratch -- may be loaded at
// another address.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_scratch on the current device.  Set-up (the
// cudaGetSymbolAddress lookup, with the device current) runs on the first
// call on a device and again whenever the current context is not the one the
// cached address was looked up in (after cudaDeviceReset).
Scratch* scratch_for_current_device(int* status) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        *status = FDOG_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);  // creates the primary context if needed
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            g_addr[dev] = nullptr;
            *status = FDOG_ECUDA;
            return nullptr;
        }
        g_addr[dev] = static_cast<Scratch*>(p);
        g_ctx[dev] = current_context_id();
    }
    *status = FDOG_OK;
    return g_addr[dev];
}

}  // namespace

extern "C" int fdog_bound_reduce_noalloc(const double* dev_values, int64_t n, double constant, double* dev_out,
                                         void* cuda_stream) {
    if (n < 0 || n > kMaxValues || (n > 0 && !dev_values) || !dev_out) return FDOG_EINVAL;
    int status = FDOG_OK;
    Scratch* scr = scratch_for_current_device(&status);
    if (!scr) return status;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the ticket must start at zero; a call that was interrupted may have left it set
    cudaError_t e = cudaMemsetAsync(&scr->ticket, 0, sizeof(int), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FDOG_ECUDA;
    }
    const int n_chunks = n > 0 ? static_cast<int>((n + kChunk - 1) / kChunk) : 1;
    bound_reduce_noalloc_kernel<<<n_chunks, kChunk, 0, s>>>(dev_values, n, n_chunks, constant, dev_out, scr);
    e = cudaGetLastError();
    return e == cudaSuccess ? FDOG_OK : FDOG_ECUDA;
}
