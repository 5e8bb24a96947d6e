// Execution engine over sets of instances: one flat index space of tiles and
// variables for any set of built instances (ragged batching), iteration chunks
// captured in CUDA graphs, one status gather per decision point, and the
// per-instance state machine of Alg. 1 -> Alg. 2 used by the solo calls, the
// batch calls and the server alike.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "instance.h"
#include "kernels.h"

namespace fdog {

// A DevBatch over a set of instances together with the device memory behind
// its descriptor and prefix arrays, and a cached graph of iteration chunks.
struct BatchView {
    std::vector<fdog_instance*> members;
    std::vector<uint64_t> uids;  // identity of the members the device image was built for
    DevBatch b;
    void* dev = nullptr;
    size_t cap = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_chunk = 0;
    int graph_wpb = 0;
    int graph_waves = -1;
    bool graph_side = false;
    int64_t graph_launches_per_replay = 0;
    BatchView() = default;
    BatchView(const BatchView&) = delete;
    BatchView& operator=(const BatchView&) = delete;
    ~BatchView();
    void drop_graph();
};

struct Engine {
    // views reused across calls (their device buffers are kept)
    BatchView v_all, v_iter, v_move, v_test;
    int device = 0;
    cudaStream_t stream = nullptr;
    LaunchCfg cfg;
    Profiler* prof = nullptr;  // optional kernel timing (graphs are not used while it is on)
    int chunk = 8;             // iterations per graph launch (set by view_autotune)
    std::vector<int> jit_universe;  // if set: the shape ids every view's specialised module covers
    InstStatus* dev_status = nullptr;
    InstStatus* host_status = nullptr;  // pinned
    int status_cap = 0;
    SideStreams side;  // created by engine_use_side; cfg.side points here once they exist
    // dual iterations as one persistent cooperative kernel per chunk (persist.cu) instead of graph
    // replays of per-pass kernels, for views it supports; barrier waits end after persist_wait_s
    bool persistent = false;
    double persist_wait_s = 1.0;
    unsigned* dev_bar = nullptr;  // the persistent kernel's barrier state
    std::string err;
    ~Engine();
};

// Creates the engine's side streams on its device (once) and points cfg at
// them; without them every launch stays in order on the engine's stream.
void engine_use_side(Engine& e);

// Lays out `members` (built on the engine's device) as one batch.
int view_build(Engine& e, BatchView& v, const std::vector<fdog_instance*>& members);
// Status of every member (one gather kernel, one copy, one synchronisation).
int view_status(Engine& e, BatchView& v, std::vector<InstStatus>& out);
// `k` dual iterations of every member whose limit / stopping rule allows them.
int view_iterate(Engine& e, BatchView& v, int k);
// Control-block operation on every member.
int view_op(Engine& e, BatchView& v, int op, int arg);

// Phase of an instance in the engine's state machine.
constexpr int kPhaseDual = 0;   // Alg. 1 until the stopping rule or the iteration budget
constexpr int kPhaseTest = 1;   // Alg. 2 agreement test due
constexpr int kPhaseReopt = 2;  // Alg. 1 re-optimisation after a perturbation
constexpr int kPhaseDone = 3;   // solution, objective and acceptance available

struct Member {
    fdog_instance* inst = nullptr;
    int phase = kPhaseDual;
    int noconv = 0;
    int start_iter = 0;
    int dual_iters = 0;
};

// Prepares members [first, end) of `ms`: iteration budget max_iters (0: they
// go straight to Alg. 2, starting with the pending add-back).
int engine_admit(Engine& e, std::vector<Member>& ms, size_t first, int max_iters);
// One scheduling step over the members not yet done: a chunk of iterations
// for the iterating ones, then every phase change the status allows; members
// reaching kPhaseDone are finished (objective, acceptance, solution copied).
int engine_step(Engine& e, std::vector<Member>& ms);

// Picks the sweep kernels' warps per block and grid mode for this view by
// timing ascending and descending update passes (each member's multipliers
// and deferred terms are saved in scratch arrays and restored, so the dual
// state is unchanged), and the iterations per graph replay from the
// measured sweep time; results depend on none of the three.
int view_autotune(Engine& e, BatchView& v, bool tune_grid = true);

// Alg. 2 for every member (which must have finished their dual phase):
// add-back, rounds of test / perturb / re-optimise, objective, acceptance,
// solutions copied to each instance.  rounds / status per member (may be null).
int engine_round(Engine& e, const std::vector<fdog_instance*>& members, std::vector<int>* rounds,
                 std::vector<int>* status);

// Alg. 1 to each member's stopping rule (or max_iters more iterations), then
// Alg. 2, with members moving through their phases independently: an instance
// that stops early starts rounding while the others keep iterating.
int engine_solve(Engine& e, const std::vector<fdog_instance*>& members, int max_iters, std::vector<int>* iters,
                 std::vector<int>* rounds, std::vector<int>* status);

}  // namespace fdog
