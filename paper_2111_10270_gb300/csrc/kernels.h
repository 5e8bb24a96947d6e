// Launchers of the sm_103a kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "fdog_internal.h"

namespace fdog {

enum SweepMode : int {
    kFwdUpdate = 0,  // ascending pass of Alg. 1 (Alg. 3 shortest paths, Eq. 5 updates)
    kBwdUpdate = 1,  // descending pass of Alg. 1 (Alg. 4 shortest paths, Eq. 5 updates)
    kMinMarg = 2,    // min-marginals of every slot (Eq. 6), no update
    kEval = 3,       // energies E^j only, no update
};

// kMinMarg / kEval flags
constexpr int kMMAddT = 1;   // evaluate at lambda + T (the add-back of Alg. 1)
constexpr int kMMBoth = 2;   // write m0 and m1 (else M = m1 - m0 into mm0)

// lower-bound reduction target: the bound of an iteration into InstCtl::lb_staged (committed later);
// evaluations at a given state use launch_eval64
constexpr int kLbStage = 2;

constexpr int kLbChunk = FDOG_LB_CHUNK;  // tiles per chunk of the lower-bound reduction
constexpr int kObjChunk = 8192;  // variables per block of the objective reduction

// Device-side description of a batch of instances (one or many).  Work of
// every kernel is a flat index space over all instances; prefix arrays map a
// flat index back to (instance, local index).
// Level schedule of the serial update (Eq. 4) for a view of one instance.
struct SerialPlan {
    const InstDev* inst = nullptr;       // device descriptor of the member; null: parallel update (Alg. 1)
    const int32_t* lev_f_off = nullptr;  // host: first variable of each level, ascending sweep
    const int32_t* lev_b_off = nullptr;  // host: descending sweep
    int n_lev_f = 0, n_lev_b = 0;
    const int32_t* lev_f = nullptr;      // device: variables by level
    const int32_t* lev_b = nullptr;
};

// L2 access-policy window of a launch: lines of [base, base + bytes) are
// kept in the device's persisting L2 carve-out (0 bytes: no window).  Used
// for one instance's deferred terms T, which every update sweep gathers at
// scattered positions.
struct L2Window {
    void* base = nullptr;
    size_t bytes = 0;
    float hit_ratio = 0.f;
};

// Raises the device's persisting-L2 carve-out to hold `bytes` (capped by the
// device maximum; never lowered) and returns the window for [base, base + bytes).
L2Window l2_window_for(int device, void* base, size_t bytes);

struct FlatArgsS {
    const InstDev* I;
    int32_t total;
};

struct DevBatch {
    InstDev* insts = nullptr;
    int32_t* tile_prefix[kNumClasses] = {};  // [n_inst + 1] tiles of class c per instance
    int32_t* tile_first[kNumClasses] = {};   // [n_inst] first tile of class c in the instance
    int32_t tiles_total[kNumClasses] = {};
    int32_t kmax[kNumClasses] = {};
    int32_t* var_prefix = nullptr;           // [n_inst + 1]
    int32_t vars_total = 0;
    int32_t* tile_all_prefix = nullptr;      // [n_inst + 1] all tiles of every class
    int32_t tiles_all_total = 0;
    int32_t* work_prefix = nullptr;          // [n_inst + 1] deferred-sum variables with at most 8 copies
    int32_t work_total = 0;
    int32_t* wide_prefix = nullptr;          // [n_inst + 1] deferred-sum variables with more copies (warp each)
    int32_t wide_total = 0;
    bool has_local[kNumClasses] = {};        // some tile of the class has tile-local variables
    int32_t* slot_prefix = nullptr;          // [n_inst + 1] padded slots
    int32_t slots_total = 0;
    int32_t* chunk_prefix = nullptr;         // [n_inst + 1] lower-bound chunks
    int32_t chunks_total = 0;
    int32_t* objchunk_prefix = nullptr;      // [n_inst + 1]
    int32_t objchunks_total = 0;
    int32_t n_inst = 0;
    JitKernels jit;                          // kernels of the shape-specialised class
    SerialPlan serial;                       // serial update only
    L2Window l2;                             // update sweeps of a one-instance batch: its T array
};


// CUDA-event timing of the update sweeps and the deferred-sum kernel
struct Profiler {
    bool on = false;
    int64_t launches = 0;  // kernel launches of this instance (always counted)
    std::vector<cudaEvent_t> pool;
    // update sweeps of the dominant class of each pass, deferred-sum steps, other sweep launches
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> sweep, reduce, minor;
    cudaEvent_t take();
    void record(int kind, cudaEvent_t a, cudaEvent_t b) {
        (kind == 0 ? sweep : kind == 1 ? reduce : minor).emplace_back(a, b);
    }
    // sums and recycles the recorded pairs (the stream must be synchronised)
    void drain(int64_t& n_sweep, double& ms_sweep, int64_t& n_reduce, double& ms_reduce);
    void release();
};

// Streams beside the launching stream for the small launches of a pass
// (minor kernel classes, the warp-per-variable deferred sums): forked from
// and joined back into the launching stream around each pass, so that they
// run alongside the dominant launch, in eager mode and inside graphs alike.
constexpr int kSideStreams = 3;
struct SideStreams {
    cudaStream_t s[kSideStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kSideStreams] = {};
    bool ready = false;
    int create(int device);  // cudaError_t as int
    void destroy();
};

struct LaunchCfg {
    int warps_per_block = 4;  // sweep kernels
    int num_sms = 152;
    int max_waves = 1;        // sweep grid: at most this many waves of resident blocks (0: a block per
                              // warps_per_block tiles), the rest by a grid-stride loop
    Profiler* prof = nullptr;
    const SideStreams* side = nullptr;  // no side streams: every launch in order on the stream
    void count(int n = 1) const {
        if (prof) prof->launches += n;
    }
};

// maximum layers the shared-memory sweep kernels take for a width
int smem_max_layers(int width);

cudaError_t launch_sweep(const DevBatch& b, int mode, int mm_flags, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_reduce_T(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_lb_reduce(const DevBatch& b, int target, const LaunchCfg& cfg, cudaStream_t s);
// FP64 evaluation of every member's bound sum_j E^j at lambda (or lambda + T
// with add_t) into InstCtl::lb_eval (eval.cu)
cudaError_t launch_eval64(const DevBatch& b, bool add_t, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_init(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_addback(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_zero_T(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_round_test(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);

// per-instance control-block operations (instance_op_kernel)
enum InstanceOp : int {
    kOpLimit = 0,          // iter_limit = iter + arg
    kOpRoundBegin = 1,     // rounding state: stop rule off, round 0, delta = delta0
    kOpRoundNext = 2,      // round += 1, delta *= alpha
    kOpClearDisagree = 3,
    kOpClearRejected = 4,
    kOpStopRestore = 5,    // stopping rule back to the parameters, stop history cleared
    kOpLimitReopt = 6,     // iter_limit = iter + the instance's re-optimisation iterations
};

// snapshot of one instance's control block (status_kernel)
struct InstStatus {
    int32_t iter, done, iter_limit, n_disagree, n_rejected, round, error, pad;
    double lb_last, objective, lb_eval;
};

cudaError_t launch_instance_op(const DevBatch& b, int op, int arg, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_status(const DevBatch& b, InstStatus* dev_out, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_round_apply(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_objective(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_accept(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);

// The persistent iteration kernel (persist.cu): `iters` dual iterations of
// every member as one cooperative launch, phases separated by a grid barrier
// whose waits end after wait_s seconds (then every member's control block
// carries error 1).  bar: 3 device words of barrier state.  Views whose tiles
// all lie in the generic width-2 classes only (persist_supported).
bool persist_supported(const DevBatch& b);
size_t persist_smem_bytes(const DevBatch& b);
cudaError_t launch_persistent(const DevBatch& b, int iters, unsigned* bar, double wait_s, const LaunchCfg& cfg,
                              cudaStream_t s);

// one full dual iteration (forward pass, deferred sums, backward pass,
// deferred sums, lower bound) on every instance of the batch
cudaError_t launch_iteration(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
// one iteration of the serial update (Eq. 4) of a one-instance view (serial.cu)
cudaError_t launch_iteration_serial(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);
// ring, iteration counter and stopping test of every member whose bound is staged
cudaError_t launch_lb_commit(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s);

}  // namespace fdog
