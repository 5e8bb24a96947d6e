// The library-owned instance behind the opaque fdog_instance handle.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "fdog_internal.h"
#include "kernels.h"

namespace fdog {

template <class T>
using HostArray = std::vector<T, DefaultInitAlloc<T>>;

struct Engine;
struct BatchView;

// prefix ints of a one-instance batch: per class 3 (prefix[2], first[1]) + 4 x 2
constexpr int kPrefixInts = 3 * kNumClasses + 14;

struct DevArrays {
    InstDev* inst = nullptr;
    InstCtl* ctl = nullptr;
    TileDev* tiles = nullptr;
    ShapeDev* shapes = nullptr;
    uint16_t* tpl = nullptr;
    float* lam = nullptr;
    int32_t* var = nullptr;
    float* mm0 = nullptr;
    float* mm1 = nullptr;  // separate allocation, made on first use
    float* T = nullptr;
    float* C = nullptr;
    float* pert = nullptr;
    uint8_t* x = nullptr;
    double* cost = nullptr;
    int32_t* csr_off = nullptr;
    int32_t* csr_pos = nullptr;
    int32_t* patterns = nullptr;
    uint16_t* local_ent = nullptr;
    int32_t* work = nullptr;
    int32_t* wpos = nullptr;
    float* lab = nullptr;            // serial update: labels of every layer and the running labels, per tile
    int32_t* lab_off = nullptr;
    int32_t* tile_of_row = nullptr;
    int32_t* lev_f = nullptr;        // serial update: variables by level (ascending, descending sweeps)
    int32_t* lev_b = nullptr;
    float2* tile_lb = nullptr;
    double* chunk_lb = nullptr;
    double* obj_chunk = nullptr;
    int32_t* prefix = nullptr;
    int32_t* sh_vars = nullptr;      // shard of a split instance: its shared variables (ascending)
    int32_t* sh_copies = nullptr;    // and their copy counts over all shards
    int32_t* sh_slot = nullptr;      // and their index among all shared variables (the exchange buffer)
};

}  // namespace fdog

struct fdog_instance {
    uint64_t uid = 0;  // process-unique id (views compare ids, not addresses)
    // the ILP as given (copied at create)
    int32_t n_vars = 0;
    int32_t n_rows = 0;
    fdog::HostArray<double> cost;
    fdog::HostArray<int64_t> row_ptr;
    fdog::HostArray<int32_t> col, coef;
    fdog::HostArray<int8_t> sense;
    fdog::HostArray<int64_t> rhs;
    fdog_params params{};

    // decomposition and device state
    bool planned = false;
    bool planned_on_device = false;  // the plan came from the device builder (plan_device.cu)
    double plan_seconds = 0.0;       // wall time of building the decomposition
    bool built = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    fdog::Decomposition dec;
    void* arena = nullptr;
    size_t arena_bytes = 0;
    fdog::DevArrays dev;
    fdog::InstDev hdesc{};
    fdog::DevBatch batch;
    fdog::LaunchCfg cfg;
    fdog::InstCtl* host_ctl = nullptr;  // pinned
    uint8_t* host_x = nullptr;          // pinned staging of the rounded solution
    bool solution_pinned = false;       // the last solution lives in host_x (else in `solution`)
    fdog::Profiler prof;
    fdog::JitKernels jit;     // shape-specialised kernels of this instance's shapes
    bool jit_failed = false;  // NVRTC unavailable or failed: generic kernels only
    std::string jit_note;

    // shard of a split instance (fdog_shard_setup): which variables also have
    // copies in other shards, and every variable's copy count over all shards
    bool shard = false;
    std::vector<uint8_t> shard_shared;
    std::vector<int32_t> shard_copies;

    // host-side view of the dual state
    bool pending_T = false;  // deferred differences of the last pass not yet added back
    bool iterated = false;   // iterations ran since the last add-back (running bound available)

    // rounding result
    bool has_solution = false;
    std::vector<uint8_t> solution;
    double objective = 0.0;
    int32_t feasible = 0;
    int32_t rounds = 0;
    bool noconverge = false;

    // the engine that runs this instance's own calls, and its one-member view
    fdog::Engine* engine = nullptr;
    fdog::BatchView* self_view = nullptr;

    int64_t h2d_bytes = 0;  // host-to-device bytes copied by the library for this instance
    int64_t d2h_bytes = 0;

    std::string last_error;
};

namespace fdog {
int plan(fdog_instance* inst, bool compile_jit = true);
// device builder (plan_device.cu): FDOG_OK, plan_leave_to_host() when the
// instance needs the host builder, or an FDOG_* error
int plan_on_device(fdog_instance* inst, int jit_mode, bool fuse_local);
int plan_leave_to_host();
void free_device_plan(Decomposition& d, cudaStream_t s);
// downloads the arrays of a device-built plan that host calls read
int ensure_host_plan(fdog_instance* inst);
size_t arena_size(const fdog_instance* inst);
int fail_cuda(fdog_instance* inst, cudaError_t e, const char* where);
cudaError_t copy_async(fdog_instance* inst, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind);
int read_ctl(fdog_instance* inst, InstCtl& out);
int addback(fdog_instance* inst);
// shards of a split instance (shard.cu): the copy counts given at set-up
// against the plan, and the initial multipliers of the shared variables
int shard_check_copies(fdog_instance* inst);
cudaError_t launch_shard_init(fdog_instance* inst);
}  // namespace fdog
