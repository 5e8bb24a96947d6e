// sm_103a kernels of the FastDOG dual hot path.
//
// Work decomposition
//   * sweep kernels: one warp per tile of 32 BDDs of one shape, one thread per
//     BDD.  All per-layer loads/stores of a warp are single 128-byte
//     transactions (interleaved slots).  The shape template (successor codes
//     per layer and node) is read with warp-uniform loads.  Shortest-path
//     labels of the direction opposite to the pass are recomputed on chip at
//     the start of each pass, so no per-node state ever goes to HBM; per-slot
//     multipliers are the only state the sweeps stream.
//   * deferred sums: one thread per variable with at most 8 copies (slot
//     positions bucketed by copy count, read column by column), one warp per
//     variable with more; copies summed in a fixed order (deterministic; no
//     floating-point atomics).
//   * lower bound: FP32 per BDD, compensated FP32 pairs per tile and per chunk
//     of tiles, FP64 Neumaier across chunks with a fixed chunking per
//     instance, so the bound of an instance does not depend on what else is
//     in the batch.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "reduce.cuh"
#include "sweep.cuh"

namespace fdog {
namespace {

using dev::FlatArgs;
using dev::LbArgs;
using dev::block_pair_reduce;
using dev::commit_iteration;
using dev::find_inst;
using dev::lb_chunk;
using dev::lb_total;
using dev::neumaier;
using dev::reduce_T_one;
using dev::reduce_T_wide_one;

// One block per chunk of kLbChunk tiles (chunk g of the flat batch), then the
// last block of the instance sums the chunk partials and stages the bound for
// lb_commit_kernel, or with `commit` commits the iteration itself.  The
// chunking depends only on the instance, so its bound is the same alone or in
// a batch.
__device__ __forceinline__ void lb_reduce_block(const LbArgs& a, int g, bool commit) {
    __shared__ double ss[8], sc[8];
    __shared__ float ssf[8], scf[8];
    __shared__ int last;
    const int ii = find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    InstCtl* ctl = I->ctl;
    if (FDOG_INACTIVE(ctl)) return;
    const int c = g - __ldg(a.prefix + ii);
    const double chunk = lb_chunk(I, c, ssf, scf);
    if (threadIdx.x == 0) {
        I->chunk_lb[c] = chunk;
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1) == I->n_chunks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double lb = lb_total(I, ss, sc);
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        if (commit) {
            commit_iteration(ctl, lb);
        } else {
            ctl->lb_staged = lb;
            ctl->staged = 1;
        }
    }
}

__global__ void __launch_bounds__(256) lb_reduce_kernel(LbArgs a) {
    dev::pdl_trigger();
    dev::pdl_wait();
    lb_reduce_block(a, blockIdx.x, false);
}

// One launch per deferred-sum step (Eq. 5's averaged term through Prop. 1).
// Blocks [0, chunks) (END only): the descending pass's bound, and the last of
// an instance's blocks commits the iteration (ring, counter, stopping test);
// the next wide_blocks blocks: a warp per variable with more than 8 copies;
// the rest: a thread per listed variable with at most 8 copies.  The parts
// read only the pass's output and write disjoint state.  END: a commit may
// land while the deferred sums run, so they test the instance's activity as
// the ascending step recorded it at the start of the iteration.
template <bool END>
__global__ void __launch_bounds__(256) deferred_sum_kernel(FlatArgs work, FlatArgs wide, LbArgs l, int chunks,
                                                           int wide_blocks) {
    dev::pdl_trigger();
    dev::pdl_wait();
    int blk = blockIdx.x;
    if (END) {
        if (blk < chunks) {
            lb_reduce_block(l, blk, true);
            return;
        }
        blk -= chunks;
    }
    if (blk < wide_blocks) {
        const int g = (blk * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x)) >> 5;
        if (g < wide.total) reduce_T_wide_one<END>(wide, g, threadIdx.x & 31);
        return;
    }
    const int g = (blk - wide_blocks) * static_cast<int>(blockDim.x) + static_cast<int>(threadIdx.x);
    if (g < work.total) reduce_T_one<END>(work, g);
}

// End of an iteration for every member whose bound was staged: ring, counter
// and the stopping test.  Runs after the deferred sums of the backward pass,
// which must still see the iteration as active (the shards of a split
// instance and the serial update of Eq. 4; the parallel update commits
// inside deferred_sum_kernel<true>).
__global__ void lb_commit_kernel(const InstDev* insts, int n) {
    dev::pdl_trigger();
    dev::pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    InstCtl* ctl = insts[i].ctl;
    if (!ctl->staged) return;
    ctl->staged = 0;
    commit_iteration(ctl, ctl->lb_staged);
}

// C_i = c_i, T_i = 0 (M-bar = 0)
__global__ void __launch_bounds__(256) init_vars_kernel(FlatArgs a) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += gridDim.x * blockDim.x) {
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        const int i = g - __ldg(a.prefix + ii);
        I->C[i] = static_cast<float>(I->cost[i]);
        I->T[i] = 0.f;
    }
}

// lambda^j_i = c_i / |J_i| (Alg. 1 initialisation); padding slots get 0
__global__ void __launch_bounds__(256) init_lam_kernel(FlatArgs a) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += gridDim.x * blockDim.x) {
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        const int p = g - __ldg(a.prefix + ii);
        const int v = I->var[p];
        float l = 0.f;
        if (v >= 0) l = I->C[v] / static_cast<float>(I->csr_off[v + 1] - I->csr_off[v]);
        I->lam[p] = l;
    }
}

// final loop of Alg. 1: lambda^j_i += T_i
__global__ void __launch_bounds__(256) addback_kernel(FlatArgs a) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += gridDim.x * blockDim.x) {
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        const int p = g - __ldg(a.prefix + ii);
        const int v = I->var[p];
        if (v >= 0) I->lam[p] += I->T[v];
    }
}

__global__ void __launch_bounds__(256) zero_T_kernel(FlatArgs a) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += gridDim.x * blockDim.x) {
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        I->T[g - __ldg(a.prefix + ii)] = 0.f;
    }
}

// SplitMix64 output function (Steele, Lea & Flood 2014) of one counter value
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct RoundArgs {
    FlatArgs f;
};

// Alg. 2 per variable: agreement test on M_ij and the perturbation of this round
__global__ void __launch_bounds__(256) round_test_kernel(RoundArgs a) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.f.total; g += gridDim.x * blockDim.x) {
        const int ii = find_inst(a.f.prefix, a.f.n_inst, g);
        const InstDev* __restrict__ I = a.f.insts + ii;
        const int i = g - __ldg(a.f.prefix + ii);
        const int b = I->csr_off[i], e = I->csr_off[i + 1];
        if (b == e) continue;
        int npos = 0, nneg = 0, nzero = 0;
        float sum = 0.f;
        for (int p = b; p < e; ++p) {
            const float m = I->mm0[I->csr_pos[p]];
            npos += m > 0.f;
            nneg += m < 0.f;
            nzero += m == 0.f;
            sum += m;
        }
        const int cnt = e - b;
        if (!(npos == cnt || nneg == cnt)) atomicAdd(&I->ctl->n_disagree, 1);
        I->x[i] = sum < 0.f ? 1 : 0;
        const int round = I->ctl->round;
        const double delta = I->ctl->delta;
        const uint64_t h = mix64(static_cast<uint64_t>(I->seed) ^
                                 (static_cast<uint64_t>(static_cast<uint32_t>(round)) << 32) ^
                                 static_cast<uint64_t>(static_cast<uint32_t>(i)));
        // r uniform in [-delta, delta) (Alg. 2); the tie and conflict pushes are r * delta
        const double r = (2.0 * (static_cast<double>(h >> 11) * 0x1.0p-53) - 1.0) * delta;
        double p;
        if (npos == cnt) p = delta;
        else if (nneg == cnt) p = -delta;
        else if (nzero == cnt) p = r * delta;
        else {
            const double sg = sum > 0.f ? 1.0 : (sum < 0.f ? -1.0 : (r >= 0.0 ? 1.0 : -1.0));
            p = sg * fabs(r) * delta;
        }
        I->pert[i] = static_cast<float>(p);
    }
}

// Alg. 2: lambda^j_i += p_i for all j in J_i (only if some variable disagrees)
__global__ void __launch_bounds__(256) round_apply_kernel(FlatArgs a) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += gridDim.x * blockDim.x) {
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        if (I->ctl->n_disagree == 0) continue;
        const int i = g - __ldg(a.prefix + ii);
        const int b = I->csr_off[i], e = I->csr_off[i + 1];
        if (b == e) continue;
        const float p = I->pert[i];
        for (int q = b; q < e; ++q) I->lam[I->csr_pos[q]] += p;
        I->C[i] += p * static_cast<float>(e - b);
        I->T[i] = 0.f;
    }
}

// Exact feasibility of the rounded solution: each thread follows its BDD
// along x (Def. of constraint set correspondence: x is in X_j iff its path
// ends at TOP) and counts the BDDs that reject it.  Rows removed by presolve
// are satisfied by construction, so this checks every row of the ILP.
__global__ void __launch_bounds__(256) accept_kernel(FlatArgs a) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < a.total; g += warps) {
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        const TileDev tile = I->tiles[g - __ldg(a.prefix + ii)];
        if (lane >= tile.n_valid) continue;
        const ShapeDev sh = I->shapes[tile.shape];
        const uint16_t* __restrict__ tpl = I->tpl + sh.tpl_off;
        uint32_t node = 0;
        bool ok = true;
        for (int t = 0; t < sh.k && ok; ++t) {
            const int v = I->var[static_cast<size_t>(tile.slot_base) + static_cast<size_t>(t) * kTile + lane];
            const uint32_t code = tpl[t * sh.width + node];
            const uint32_t next = I->x[v] ? (code >> 8) : (code & 0xFFu);
            if (next == kCodeBot) ok = false;
            else if (next == kCodeTop) ok = (t == sh.k - 1);
            else node = next;
        }
        if (!ok) atomicAdd(&I->ctl->n_rejected, 1);
    }
}

// c^T x over the variables inside BDDs, FP64 Neumaier with fixed chunking
__global__ void __launch_bounds__(256) objective_kernel(LbArgs a) {
    __shared__ double ss[256], sc[256];
    const int g = blockIdx.x;
    const int ii = find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    InstCtl* ctl = I->ctl;
    const int c = g - __ldg(a.prefix + ii);
    const int v0 = c * kObjChunk, v1 = min(v0 + kObjChunk, I->n_vars);
    double s = 0.0, cp = 0.0;
    for (int i = v0 + threadIdx.x; i < v1; i += blockDim.x)
        if (I->csr_off[i + 1] > I->csr_off[i] && I->x[i]) neumaier(s, cp, I->cost[i]);
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = cp;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double x = ss[threadIdx.x], y = ss[threadIdx.x + w], cc = sc[threadIdx.x] + sc[threadIdx.x + w];
            neumaier(x, cc, y);
            ss[threadIdx.x] = x;
            sc[threadIdx.x] = cc;
        }
        __syncthreads();
    }
    __shared__ int last;
    if (threadIdx.x == 0) {
        I->obj_chunk[c] = ss[0] + sc[0];
        __threadfence();
        last = atomicAdd(&ctl->obj_ticket, 1) == I->n_obj_chunks - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block sums the chunk totals, strided over its threads then a fixed-order tree
    __threadfence();
    s = 0.0;
    cp = 0.0;
    for (int q = threadIdx.x; q < I->n_obj_chunks; q += blockDim.x) neumaier(s, cp, __ldcg(I->obj_chunk + q));
    ss[threadIdx.x] = s;
    sc[threadIdx.x] = cp;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            double x = ss[threadIdx.x], y = ss[threadIdx.x + w], cc = sc[threadIdx.x] + sc[threadIdx.x + w];
            neumaier(x, cc, y);
            ss[threadIdx.x] = x;
            sc[threadIdx.x] = cc;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctl->objective = ss[0] + sc[0];
        ctl->obj_ticket = 0;
    }
}

// Control-block operations, one thread per instance of the batch.
__global__ void instance_op_kernel(const InstDev* insts, int n, int op, int arg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const InstDev& I = insts[i];
    InstCtl* c = I.ctl;
    switch (op) {
        case kOpLimit: c->iter_limit = c->iter + arg; break;
        case kOpLimitReopt: c->iter_limit = c->iter + I.reopt_iters; break;
        case kOpRoundBegin:
            c->stop_enabled = 0; c->done = 0; c->round = 0; c->delta = I.delta0; c->n_disagree = 0;
            break;
        case kOpRoundNext: c->round += 1; c->delta *= I.alpha; break;
        case kOpClearDisagree: c->n_disagree = 0; break;
        case kOpClearRejected: c->n_rejected = 0; break;
        case kOpStopRestore: c->stop_enabled = I.stop_param; c->done = 0; c->since_reset = 0; break;
        default: break;
    }
}

__global__ void status_kernel(const InstDev* insts, int n, InstStatus* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const InstCtl* c = insts[i].ctl;
    InstStatus s;
    s.iter = c->iter;
    s.done = c->done;
    s.iter_limit = c->iter_limit;
    s.n_disagree = c->n_disagree;
    s.n_rejected = c->n_rejected;
    s.round = c->round;
    s.error = c->error;
    s.pad = 0;
    s.lb_last = c->lb_last;
    s.objective = c->objective;
    s.lb_eval = c->lb_eval;
    out[i] = s;
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
inline int blocks_for(int total, int per_block, int cap) {
    int b = (total + per_block - 1) / per_block;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace

int smem_max_layers(int width) {
    // per warp: kTile columns x (lambda, T, W labels) floats per layer (staged kernels) or
    // W labels per segment of kRegK layers (segmented kernels); at least one warp per block
    if (width <= kRegW) return kRegK * ((200 * 1024 - kEpiMaxK * 2 * kTile * 4) / (kTile * 4 * width));
    return (200 * 1024 - kEpiMaxK * 2 * kTile * 4) / (kTile * 4 * (2 + width));
}

namespace {

// one class's sweep launch on stream s
cudaError_t launch_class(const DevBatch& b, int cls, int mode, int mm_flags, const LaunchCfg& cfg, cudaStream_t s,
                         bool dominant) {
    const int total = b.tiles_total[cls];
    const bool reg = class_is_reg(cls);
    const int W = class_width(cls);
    int wpb = cfg.warps_per_block;
    const bool seg = class_is_seg(cls);
    // staged kernels: one row of state per layer; segmented kernels: one checkpoint per kRegK layers
    const int kstride = reg ? 0 : (seg ? (b.kmax[cls] + kRegK - 1) / kRegK : b.kmax[cls]);
    const int epi = ((mode == kFwdUpdate || mode == kBwdUpdate) && b.has_local[cls])
                        ? (b.kmax[cls] < kEpiMaxK ? b.kmax[cls] : kEpiMaxK) : 0;
    const size_t per_warp =
        (static_cast<size_t>(kstride) * (seg ? W : 2 + W) + static_cast<size_t>(epi) * 2) * kTile * sizeof(float);
    while (wpb > 1 && per_warp * wpb > 200 * 1024) wpb >>= 1;
    const size_t smem = per_warp * wpb;
    SweepArgs args{b.insts, b.tile_prefix[cls], b.tile_first[cls], b.n_inst, total, kstride, mm_flags, epi};
    const int blocks = blocks_for(total, wpb, cfg.max_waves > 0 ? cfg.max_waves * cfg.num_sms * (2048 / (32 * wpb)) : (1 << 30));
    const bool timed = cfg.prof && cfg.prof->on && (mode == kFwdUpdate || mode == kBwdUpdate);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (timed) { ev0 = cfg.prof->take(); ev1 = cfg.prof->take(); cudaEventRecord(ev0, s); }
    // update passes of the dominant class keep the deferred terms they gather in L2
    const L2Window l2 = dominant && (mode == kFwdUpdate || mode == kBwdUpdate) ? b.l2 : L2Window();
    cudaError_t e;
    if (cls == kJitClass) {
        void* kargs[] = {&args};
        e = cudaSuccess;
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(b.jit.fn[mode], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem));
        if (e == cudaSuccess) e = launch_windowed(b.jit.fn[mode], blocks, 32 * wpb, kargs, smem, s, l2);
    } else switch (W) {
        case 2: e = launch_sweep_width<2>(reg, mode, blocks, 32 * wpb, smem, s, args, l2); break;
        case 4: e = launch_sweep_width<4>(reg, mode, blocks, 32 * wpb, smem, s, args, l2); break;
        case 8: e = launch_sweep_width<8>(reg, mode, blocks, 32 * wpb, smem, s, args, l2); break;
        default: e = launch_sweep_width<16>(reg, mode, blocks, 32 * wpb, smem, s, args, l2); break;
    }
    if (timed) { cudaEventRecord(ev1, s); cfg.prof->record(dominant ? 0 : 2, ev0, ev1); }
    cfg.count();
    return e;
}

// timing, when on, records each launch's events on the stream it runs on
bool can_fork(const LaunchCfg& cfg) { return cfg.side && cfg.side->ready; }

}  // namespace

cudaError_t launch_windowed(const void* fn, int blocks, int threads, void** args, size_t smem, cudaStream_t s,
                            const L2Window& l2) {
    cudaLaunchAttribute attr[2];
    int n = 0;
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
    if (l2.bytes > 0) {
        attr[n].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[n].val.accessPolicyWindow.base_ptr = l2.base;
        attr[n].val.accessPolicyWindow.num_bytes = l2.bytes;
        attr[n].val.accessPolicyWindow.hitRatio = l2.hit_ratio;
        attr[n].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[n].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        ++n;
    }
    cudaLaunchConfig_t c{};
    c.gridDim = dim3(blocks);
    c.blockDim = dim3(threads);
    c.dynamicSmemBytes = smem;
    c.stream = s;
    c.attrs = attr;
    c.numAttrs = n;
    return cudaLaunchKernelExC(&c, fn, args);
}

L2Window l2_window_for(int device, void* base, size_t bytes) {
    L2Window w;
    int pmax = 0, wmax = 0;
    if (bytes == 0 || cudaDeviceGetAttribute(&pmax, cudaDevAttrMaxPersistingL2CacheSize, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&wmax, cudaDevAttrMaxAccessPolicyWindowSize, device) != cudaSuccess || pmax <= 0 ||
        wmax <= 0) {
        cudaGetLastError();
        return w;
    }
    const size_t want = std::min<size_t>(bytes, static_cast<size_t>(pmax));
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) cur = 0;
    if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) cur = want;
    cudaGetLastError();
    if (cur == 0) return w;
    w.base = base;
    w.bytes = std::min<size_t>(bytes, static_cast<size_t>(wmax));
    w.hit_ratio = std::min(1.0f, static_cast<float>(cur) / static_cast<float>(w.bytes));
    return w;
}

int SideStreams::create(int device) {
    if (ready) return cudaSuccess;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int j = 0; j < kSideStreams && e == cudaSuccess; ++j)
        e = cudaStreamCreateWithPriority(&s[j], cudaStreamNonBlocking, hi);  // small latency-bound work first
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int j = 0; j < kSideStreams && e == cudaSuccess; ++j) e = cudaEventCreateWithFlags(&join[j], cudaEventDisableTiming);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy();
        return e;
    }
    ready = true;
    return cudaSuccess;
}

void SideStreams::destroy() {
    for (int j = 0; j < kSideStreams; ++j) {
        if (s[j]) cudaStreamDestroy(s[j]);
        if (join[j]) cudaEventDestroy(join[j]);
        s[j] = nullptr;
        join[j] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
    ready = false;
}

// All classes of one pass.  With side streams, the minor classes are
// launched first on them (their blocks become resident before the dominant
// launch fills the GPU) and joined back before the pass ends.
cudaError_t launch_sweep(const DevBatch& b, int mode, int mm_flags, const LaunchCfg& cfg, cudaStream_t s) {
    int cls_list[kNumClasses], n = 0, dom = -1;
    long long best = -1;
    for (int cls = 0; cls < kNumClasses; ++cls) {
        if (b.tiles_total[cls] == 0) continue;
        cls_list[n++] = cls;
        const long long work = static_cast<long long>(b.tiles_total[cls]) * (b.kmax[cls] > 0 ? b.kmax[cls] : 1);
        if (work > best) { best = work; dom = cls; }
    }
    cudaError_t e = cudaSuccess;
    if (n <= 1 || !can_fork(cfg)) {
        for (int q = 0; q < n && e == cudaSuccess; ++q)
            e = launch_class(b, cls_list[q], mode, mm_flags, cfg, s, cls_list[q] == dom);
        return e;
    }
    const SideStreams& sd = *cfg.side;
    bool used[kSideStreams] = {};
    e = cudaEventRecord(sd.fork, s);
    int j = 0;
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
        if (cls_list[q] == dom) continue;
        const int k = j++ % kSideStreams;
        if (!used[k]) { e = cudaStreamWaitEvent(sd.s[k], sd.fork, 0); used[k] = true; }
        if (e == cudaSuccess) e = launch_class(b, cls_list[q], mode, mm_flags, cfg, sd.s[k], false);
    }
    if (e == cudaSuccess) e = launch_class(b, dom, mode, mm_flags, cfg, s, true);
    for (int k = 0; k < kSideStreams && e == cudaSuccess; ++k) {
        if (!used[k]) continue;
        e = cudaEventRecord(sd.join[k], sd.s[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, sd.join[k], 0);
    }
    return e;
}

static FlatArgs flat(const DevBatch& b, const int32_t* prefix, int total) {
    return FlatArgs{b.insts, prefix, b.n_inst, total};
}

// one deferred-sum step: END adds the bound reduction and the commit of the iteration
static cudaError_t launch_deferred(const DevBatch& b, bool end, const LaunchCfg& cfg, cudaStream_t s) {
    const int chunks = end ? b.chunks_total : 0;
    if (b.work_total == 0 && b.wide_total == 0 && chunks == 0) return cudaSuccess;
    const bool timed = cfg.prof && cfg.prof->on;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (timed) { ev0 = cfg.prof->take(); ev1 = cfg.prof->take(); cudaEventRecord(ev0, s); }
    FlatArgs work = flat(b, b.work_prefix, b.work_total);
    FlatArgs wide = flat(b, b.wide_prefix, b.wide_total);
    LbArgs la{b.insts, b.chunk_prefix, b.n_inst, kLbStage};
    int nc = chunks;
    int wide_blocks = (b.wide_total + 7) / 8;  // 8 warps per block
    void* args[] = {&work, &wide, &la, &nc, &wide_blocks};
    const int blocks = chunks + wide_blocks + (b.work_total + 255) / 256;
    const void* fn = end ? reinterpret_cast<const void*>(deferred_sum_kernel<true>)
                         : reinterpret_cast<const void*>(deferred_sum_kernel<false>);
    const cudaError_t e = launch_windowed(fn, blocks, 256, args, 0, s, L2Window());
    cfg.count();
    if (timed) { cudaEventRecord(ev1, s); cfg.prof->record(1, ev0, ev1); }
    return e;
}

cudaError_t launch_reduce_T(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    return launch_deferred(b, false, cfg, s);
}

cudaEvent_t Profiler::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Profiler::drain(int64_t& n_sweep, double& ms_sweep, int64_t& n_reduce, double& ms_reduce) {
    auto sum = [&](std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v, int64_t& n, double& ms) {
        for (auto& [a, b] : v) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, a, b) == cudaSuccess) { ms += t; ++n; }
            pool.push_back(a);
            pool.push_back(b);
        }
        v.clear();
    };
    sum(sweep, n_sweep, ms_sweep);
    sum(reduce, n_reduce, ms_reduce);
    int64_t n_minor = 0;
    double ms_minor = 0.0;
    sum(minor, n_minor, ms_minor);
    cudaGetLastError();
}

void Profiler::release() {
    for (auto& [a, b] : sweep) { pool.push_back(a); pool.push_back(b); }
    for (auto& [a, b] : reduce) { pool.push_back(a); pool.push_back(b); }
    for (auto& [a, b] : minor) { pool.push_back(a); pool.push_back(b); }
    sweep.clear();
    reduce.clear();
    minor.clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
}

cudaError_t launch_lb_reduce(const DevBatch& b, int target, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.chunks_total == 0) return cudaSuccess;
    cfg.count();
    LbArgs la{b.insts, b.chunk_prefix, b.n_inst, target};
    void* args[] = {&la};
    return launch_windowed(reinterpret_cast<const void*>(lb_reduce_kernel), b.chunks_total, 256, args, 0, s,
                           L2Window());
}

cudaError_t launch_init(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    cfg.count((b.vars_total > 0) + (b.slots_total > 0));
    if (b.vars_total > 0)
        init_vars_kernel<<<blocks_for(b.vars_total, 256, cfg.num_sms * 8), 256, 0, s>>>(
            flat(b, b.var_prefix, b.vars_total));
    if (b.slots_total > 0)
        init_lam_kernel<<<blocks_for(b.slots_total, 256, cfg.num_sms * 8), 256, 0, s>>>(
            flat(b, b.slot_prefix, b.slots_total));
    return cudaGetLastError();
}

cudaError_t launch_addback(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    cfg.count(b.slots_total > 0);
    if (b.slots_total > 0)
        addback_kernel<<<blocks_for(b.slots_total, 256, cfg.num_sms * 8), 256, 0, s>>>(
            flat(b, b.slot_prefix, b.slots_total));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_zero_T(b, cfg, s);
}

cudaError_t launch_zero_T(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    cfg.count(b.vars_total > 0);
    if (b.vars_total > 0)
        zero_T_kernel<<<blocks_for(b.vars_total, 256, cfg.num_sms * 8), 256, 0, s>>>(
            flat(b, b.var_prefix, b.vars_total));
    return cudaGetLastError();
}

cudaError_t launch_round_test(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.vars_total == 0) return cudaSuccess;
    cfg.count();
    round_test_kernel<<<blocks_for(b.vars_total, 256, cfg.num_sms * 8), 256, 0, s>>>(
        RoundArgs{flat(b, b.var_prefix, b.vars_total)});
    return cudaGetLastError();
}

cudaError_t launch_round_apply(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.vars_total == 0) return cudaSuccess;
    cfg.count();
    round_apply_kernel<<<blocks_for(b.vars_total, 256, cfg.num_sms * 8), 256, 0, s>>>(
        flat(b, b.var_prefix, b.vars_total));
    return cudaGetLastError();
}

cudaError_t launch_objective(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.objchunks_total == 0) return cudaSuccess;
    cfg.count();
    objective_kernel<<<b.objchunks_total, 256, 0, s>>>(LbArgs{b.insts, b.objchunk_prefix, b.n_inst, 0});
    return cudaGetLastError();
}

cudaError_t launch_accept(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.tiles_all_total == 0) return cudaSuccess;
    cfg.count();
    accept_kernel<<<blocks_for(b.tiles_all_total, 8, cfg.num_sms * 8), 256, 0, s>>>(
        flat(b, b.tile_all_prefix, b.tiles_all_total));
    return cudaGetLastError();
}

cudaError_t launch_instance_op(const DevBatch& b, int op, int arg, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.n_inst == 0) return cudaSuccess;
    cfg.count();
    instance_op_kernel<<<(b.n_inst + 127) / 128, 128, 0, s>>>(b.insts, b.n_inst, op, arg);
    return cudaGetLastError();
}

cudaError_t launch_status(const DevBatch& b, InstStatus* dev_out, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.n_inst == 0) return cudaSuccess;
    cfg.count();
    status_kernel<<<(b.n_inst + 127) / 128, 128, 0, s>>>(b.insts, b.n_inst, dev_out);
    return cudaGetLastError();
}

cudaError_t launch_lb_commit(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.n_inst == 0) return cudaSuccess;
    cfg.count();
    const InstDev* insts = b.insts;
    int n = b.n_inst;
    void* args[] = {&insts, &n};
    return launch_windowed(reinterpret_cast<const void*>(lb_commit_kernel), (b.n_inst + 127) / 128, 128, args, 0, s,
                           L2Window());
}

cudaError_t launch_iteration(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.serial.inst) return launch_iteration_serial(b, cfg, s);
    cudaError_t e;
    if ((e = launch_sweep(b, kFwdUpdate, 0, cfg, s)) != cudaSuccess) return e;
    if ((e = launch_reduce_T(b, cfg, s)) != cudaSuccess) return e;
    if ((e = launch_sweep(b, kBwdUpdate, 0, cfg, s)) != cudaSuccess) return e;
    // deferred sums, bound and the commit of the iteration: one launch
    return launch_deferred(b, true, cfg, s);
}

}  // namespace fdog
