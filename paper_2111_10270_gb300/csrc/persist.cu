// Persistent iteration kernel: a chunk of dual iterations of a batch view as
// one cooperative launch.
//
// Alg. 1's passes need device-wide barriers: the deferred sums of a pass read
// the multipliers of every tile, and the next pass reads every deferred term
// (Eq. 5).  The per-pass kernels of kernels.cu get those barriers from kernel
// boundaries inside a CUDA graph; here one kernel, with every block resident
// (cooperative launch), runs the same phases -- ascending sweep, deferred
// sums, descending sweep, deferred sums and the chunk partials of the bound,
// bound totals and the stopping test -- separated by a grid barrier of its
// own.  Every phase calls the same device code as the per-pass kernels
// (sweep.cuh, reduce.cuh) in the same order per tile, variable and chunk, so
// results are bitwise those of the graph path.
//
// The barrier waits are bounded: a block that waits longer than the limit
// raises the error flag and every block leaves at its next barrier; the
// members' control blocks then carry the error, which the engine reports as
// FDOG_ETIMEOUT, and the context stays usable.
//
// Scope: views whose tiles are all in the generic width-2 classes (register
// and segmented), which covers the MRF, matching and cell-tracking
// workloads when the shape-specialised kernels are off (params.jit = -1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "reduce.cuh"

namespace fdog {
namespace {

using namespace dev;

constexpr int kPersistThreads = 256;
constexpr int kRegClass = 0;  // class_of(2, k <= kRegK): width 2, registers
constexpr int kSegClass = 1;  // class_of(2, k > kRegK): width 2, segments of kRegK layers

struct PersistArgs {
    SweepArgs fwd[2], bwd[2];  // [0] register class, [1] segmented class (same arguments for both passes)
    int32_t n_reg, n_seg;      // tiles of each class
    FlatArgs work, wide;       // deferred sums: thread per variable, warp per variable
    LbArgs lb;                 // chunks of the bound reduction
    int32_t lb_chunks;
    int32_t iters;
    int64_t warp_floats;       // shared memory stride of a warp (the larger class's need)
    unsigned* bar;             // [0] arrivals, [1] generation, [2] error flag
    unsigned long long wait_ns;  // a block leaves a barrier wait after this many nanoseconds
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier with a bounded wait.  Returns false (in every thread) once any
// block has given up waiting.  The fences on both sides make the writes of
// every block before the barrier visible to every block after it, L1
// included.
__device__ bool grid_barrier(const PersistArgs& a) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vb = a.bar;
        const unsigned gen = vb[1];
        __threadfence();
        if (atomicAdd(a.bar, 1u) == gridDim.x - 1) {
            atomicExch(a.bar, 0u);
            __threadfence();
            atomicAdd(a.bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (vb[1] == gen && vb[2] == 0u) {
                if (global_ns() - t0 > a.wait_ns) {
                    atomicExch(a.bar + 2, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = vb[2] == 0u;
    }
    __syncthreads();
    return ok != 0;
}

template <int MODE>
__device__ __forceinline__ void sweep_pass(const SweepArgs (&c)[2], int n_reg, int n_seg, int gw, int nw, float* wsm,
                                           int lane) {
    // segmented tiles first: they are the longest walks
    for (int g = gw; g < n_seg + n_reg; g += nw) {
        const int gn = g + nw;
        if (g < n_seg) seg_tile<2, MODE>(c[kSegClass], g, gn < n_seg ? gn : n_seg, wsm, lane);
        else sweep_tile<2, true, MODE>(c[kRegClass], g - n_seg, gn - n_seg, wsm, lane);
    }
}

__device__ __forceinline__ void deferred_sums(const PersistArgs& a, int gt, int nt, int gw, int nw, int lane) {
    for (int g = gt; g < a.work.total; g += nt) reduce_T_one(a.work, g);
    for (int g = gw; g < a.wide.total; g += nw) reduce_T_wide_one(a.wide, g, lane);
}

__global__ void __launch_bounds__(kPersistThreads, 2) persist_iterations_kernel(PersistArgs a) {
    extern __shared__ float smem[];
    __shared__ double ss[8], sc[8];
    __shared__ float ssf[8], scf[8];
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5), nw = gridDim.x * wpb;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    float* wsm = smem + static_cast<int64_t>(threadIdx.x >> 5) * a.warp_floats;
    bool ok = true;
    for (int it = 0; it < a.iters && ok; ++it) {
        sweep_pass<kFwdUpdate>(a.fwd, a.n_reg, a.n_seg, gw, nw, wsm, lane);
        if (!(ok = grid_barrier(a))) break;
        deferred_sums(a, gt, nt, gw, nw, lane);
        if (!(ok = grid_barrier(a))) break;
        sweep_pass<kBwdUpdate>(a.bwd, a.n_reg, a.n_seg, gw, nw, wsm, lane);
        if (!(ok = grid_barrier(a))) break;
        deferred_sums(a, gt, nt, gw, nw, lane);
        // the bound: a block per chunk (lb_reduce_kernel's arithmetic)
        for (int g = blockIdx.x; g < a.lb_chunks; g += gridDim.x) {
            const int ii = find_inst(a.lb.prefix, a.lb.n_inst, g);
            const InstDev* __restrict__ I = a.lb.insts + ii;
            if (!FDOG_INACTIVE(I->ctl)) {
                const int c = g - __ldg(a.lb.prefix + ii);
                const double v = lb_chunk(I, c, ssf, scf);
                if (threadIdx.x == 0) I->chunk_lb[c] = v;
            }
            __syncthreads();
        }
        if (!(ok = grid_barrier(a))) break;
        // totals and the stopping test: a block per instance with chunks
        for (int ii = blockIdx.x; ii < a.lb.n_inst; ii += gridDim.x) {
            const InstDev* __restrict__ I = a.lb.insts + ii;
            if (__ldg(a.lb.prefix + ii + 1) == __ldg(a.lb.prefix + ii) || FDOG_INACTIVE(I->ctl)) continue;
            const double v = lb_total(I, ss, sc);
            if (threadIdx.x == 0) commit_iteration(I->ctl, v);
            __syncthreads();
        }
        ok = grid_barrier(a);
    }
    if (!ok && blockIdx.x == 0)
        for (int ii = threadIdx.x; ii < a.lb.n_inst; ii += blockDim.x) a.lb.insts[ii].ctl->error = 1;
}

// the update passes' launch arguments of a class, as launch_class forms them
SweepArgs class_args(const DevBatch& b, int cls) {
    const int kstride = class_is_seg(cls) ? (b.kmax[cls] + kRegK - 1) / kRegK : 0;
    const int epi = b.has_local[cls] ? std::min(b.kmax[cls], kEpiMaxK) : 0;
    return SweepArgs{b.insts, b.tile_prefix[cls], b.tile_first[cls], b.n_inst, b.tiles_total[cls], kstride, 0, epi};
}

}  // namespace

bool persist_supported(const DevBatch& b) {
    if (b.serial.inst) return false;
    for (int cls = 0; cls < kNumClasses; ++cls)
        if (b.tiles_total[cls] > 0 && cls != kRegClass && cls != kSegClass) return false;
    return persist_smem_bytes(b) <= 200 * 1024;
}

size_t persist_smem_bytes(const DevBatch& b) {
    const int64_t wf = std::max<int64_t>(static_cast<int64_t>(sweep_warp_floats<2, true>(class_args(b, kRegClass))),
                                          static_cast<int64_t>(seg_warp_floats<2>(class_args(b, kSegClass))));
    return static_cast<size_t>(wf) * sizeof(float) * (kPersistThreads / 32);
}

cudaError_t launch_persistent(const DevBatch& b, int iters, unsigned* bar, double wait_s, const LaunchCfg& cfg,
                              cudaStream_t s) {
    if (iters <= 0 || b.n_inst == 0) return cudaSuccess;
    PersistArgs a{};
    for (int c : {kRegClass, kSegClass}) a.fwd[c] = a.bwd[c] = class_args(b, c);
    a.n_reg = b.tiles_total[kRegClass];
    a.n_seg = b.tiles_total[kSegClass];
    a.work = FlatArgs{b.insts, b.work_prefix, b.n_inst, b.work_total};
    a.wide = FlatArgs{b.insts, b.wide_prefix, b.n_inst, b.wide_total};
    a.lb = LbArgs{b.insts, b.chunk_prefix, b.n_inst, kLbStage};
    a.lb_chunks = b.chunks_total;
    a.iters = iters;
    const size_t smem = persist_smem_bytes(b);
    a.warp_floats = static_cast<int64_t>(smem / sizeof(float) / (kPersistThreads / 32));
    a.bar = bar;
    a.wait_ns = static_cast<unsigned long long>(std::max(wait_s, 0.0) * 1e9);
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(persist_iterations_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_iterations_kernel, kPersistThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    void* args[] = {&a};
    cfg.count();
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(persist_iterations_kernel),
                                       dim3(per_sm * cfg.num_sms), dim3(kPersistThreads), args, smem, s);
}

}  // namespace fdog
