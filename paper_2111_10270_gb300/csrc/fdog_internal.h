// Internal types shared by the host-side builder and the CUDA kernels.
#pragma once

#include <vector_types.h>  // float2 in the device descriptors

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <new>
#include <thread>
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fastdog.h"

namespace fdog {

// One warp processes one tile of kTile BDDs of the same shape; lane l owns
// BDD l of the tile (thread per BDD).  Slots of a tile are interleaved:
// slot (layer t, lane l) lives at slot_base + t * kTile + l, so every
// per-layer load and store of a warp is one coalesced 128-byte transaction.
constexpr int kTile = 32;

// Node-successor codes of the shape templates (one uint8 per arc).
constexpr uint8_t kCodeTop = 0xFE;
constexpr uint8_t kCodeBot = 0xFF;

// Kernel classes: maximum layer width W of the shape (register arrays of W
// shortest-path labels per layer) and whether all per-layer state fits in
// registers (W <= kRegW and k <= kRegK) or lives in shared memory.
constexpr int kRegK = 8;
constexpr int kRegW = 4;
constexpr int kWidths[4] = {2, 4, 8, 16};
constexpr int kNumWidths = 4;
constexpr int kMaxWidth = 16;
constexpr int kMaxLayersSmem = 256;  // longest row the staged shared-memory kernels take
constexpr int kMaxLayersSeg = 4096;  // longest row the segmented kernels (narrow BDDs) take
constexpr int kEpiMaxK = 16;         // longest row whose tile can form tile-local deferred terms
constexpr int kNumStaticClasses = 2 * kNumWidths;  // (width index) x (register | smem)
constexpr int kJitClass = kNumStaticClasses;         // shape-specialised kernels
constexpr int kNumClasses = kNumStaticClasses + 1;
constexpr int kJitMaxK = 16;                         // rows the shape-specialised code takes
constexpr int kJitMaxW = 4;
constexpr int64_t kJitMinBdds = 4096;  // jit mode 0: shapes with fewer BDDs stay on the generic kernels

inline int class_of(int width, int k) {
    int wi = 0;
    while (wi < kNumWidths && kWidths[wi] < width) ++wi;
    if (wi == kNumWidths) return -1;
    return wi * 2 + ((k <= kRegK && kWidths[wi] <= kRegW) ? 0 : 1);
}
inline int class_width(int cls) { return cls == kJitClass ? kJitMaxW : kWidths[cls / 2]; }
inline bool class_is_reg(int cls) { return cls == kJitClass || (cls % 2) == 0; }
// long rows of narrow BDDs: segments of kRegK layers in registers, checkpoints in shared memory
inline bool class_is_seg(int cls) { return !class_is_reg(cls) && kWidths[cls / 2] <= kRegW; }

// <jit-abi>  (this block is also compiled into the shape-specialised kernels)
struct ShapeDev {
    int32_t k;        // layers (= variables of the row)
    int32_t tpl_off;  // offset (in uint16 units) of the template: k * W entries
    int32_t width;    // W of its class
    int32_t jit;      // process-wide id of the shape-specialised code, -1 if none
};

struct TileDev {
    int32_t shape;
    int32_t slot_base;
    int32_t n_valid;   // BDDs in this tile (1..kTile)
    int32_t bdd_base;  // index of lane 0's BDD in the instance's BDD order
    int32_t pattern;   // tile-local variables: index into InstDev::patterns, -1 if none
    int32_t pad[3];
};

#define FDOG_LB_RING 64
#define FDOG_LB_CHUNK 256      // tiles per chunk of the lower-bound reduction

// Device-resident control block of one instance.
struct InstCtl {
    double lb_ring[FDOG_LB_RING];  // running lower bound after iteration t at [t % kLbRing]
    double lb_last;           // running lower bound after the last iteration
    double lb_eval;           // result of the last FP64 evaluation (eval.cu)
    double objective;         // c^T x of the last rounding (without presolve constants)
    int32_t iter;             // dual iterations completed since the build
    int32_t done;             // stopping rule met: update kernels become no-ops
    int32_t ticket;           // last-block ticket of the lower-bound reduction
    int32_t obj_ticket;
    int32_t n_disagree;       // rounding: variables whose M_ij do not share one strict sign
    int32_t error;
    int32_t stop_enabled;
    int32_t window;
    int32_t min_iters;
    int32_t since_reset;      // iterations since the stopping history was reset
    int32_t n_rejected;       // BDDs whose row the rounded solution violates
    int32_t iter_limit;       // update kernels skip the instance once iter reaches it
    int32_t round;            // rounding: current round of Alg. 2
    int32_t staged;           // this iteration's bound is reduced into lb_staged, not yet committed
    double tol;
    double delta;             // rounding: current perturbation strength
    double lb_staged;
    int32_t pass_active;      // the instance's activity at the start of the running iteration, recorded
                              // by its ascending pass's deferred sums for the end-of-iteration kernel
    int32_t pad;
};

// True when the update kernels must leave the instance alone: its stopping
// rule has fired or it has run the iterations it was given.
#define FDOG_INACTIVE(ctl) ((ctl)->done || (ctl)->iter >= (ctl)->iter_limit)

// Everything a kernel needs to know about one instance (device pointers).
// deferred-sum work buckets: copy counts 1 .. FDOG_WBUCKETS - 1, then one
// bucket for variables with more copies (a warp each, through csr_pos)
#define FDOG_WBUCKETS 9

struct InstDev {
    const TileDev* tiles;
    const ShapeDev* shapes;
    const uint16_t* tpl;     // per shape: k * W codes (lo | hi << 8)
    float* lam;              // [slots_pad] multipliers lambda^j_i
    const int32_t* var;      // [slots_pad] variable of each slot, -1 for padding
    float* mm0;              // [slots_pad] min-marginal outputs (m0, or M)
    float* mm1;              // [slots_pad] min-marginal output m1
    float* T;                // [n] deferred term  omega/|J_i| sum_k Mbar_ik
    float* C;                // [n] target sum_j lambda^j_i (= c_i, perturbed by rounding)
    const int32_t* csr_off;  // [n + 1]
    const int32_t* csr_pos;  // [slots] padded slot positions of each variable, ascending
    const int32_t* patterns; // [2 per pattern] {first entry, entries}: variables whose copies all lie in one tile
    const uint16_t* local_ent;  // [4 per entry] copy offsets (32 t + lane) within the tile, ascending, 0xFFFF unused
    const int32_t* work;     // [n_work] variables the deferred-sum kernel handles (copies in several tiles),
                             //          grouped into buckets by copy count (FDOG_WBUCKETS)
    float* lab;              // serial update (Eq. 4): per tile, labels of every layer [t][v][lane] then the
                             // running labels [v][lane] of the sweep, at lab_off[tile]
    const int32_t* lab_off;
    const int32_t* tile_of_row;  // tile of each row of 32 padded slots
    const int32_t* wpos;     // slot positions of the bucketed variables: bucket b (count c = b + 1, nb
                             // variables) holds copy q of its j-th variable at wpos[wb_pos[b] + q nb + j]
    const double* cost;      // [n]
    float* pert;             // [n] rounding perturbation of this round
    uint8_t* x;              // [n] rounded solution
    float2* tile_lb;         // [n_tiles] per-tile partial of the lower bound: compensated pair (sum, error)
    double* chunk_lb;        // [n_chunks] per-chunk partials of the lower-bound reduction
    double* obj_chunk;       // [n_obj_chunks]
    InstCtl* ctl;
    int32_t n_tiles;
    int32_t n_vars;
    int32_t n_chunks;
    int32_t n_obj_chunks;
    int32_t n_work;
    int32_t wb_start[FDOG_WBUCKETS + 1];  // first work index of each bucket; [FDOG_WBUCKETS] = n_work
    int32_t wb_pos[FDOG_WBUCKETS];        // offset of each bucket's columns in wpos
    float omega;
    double const_lb;
    double alpha;            // rounding: perturbation growth
    double delta0;           // rounding: initial perturbation strength
    unsigned long long seed; // rounding: seed of the perturbation draws
    int32_t stop_param;      // stopping rule enabled by the parameters
    int32_t reopt_iters;     // rounding: Alg. 1 iterations per re-optimisation
};

struct SweepArgs {
    const InstDev* insts;
    const int32_t* prefix;  // [n_inst + 1] tiles of this class per instance
    const int32_t* first;   // [n_inst] first tile of this class in the instance
    int32_t n_inst;
    int32_t total;
    int32_t kstride;        // shared-memory kernels: per-layer stride (>= longest row)
    int32_t flags;          // evaluate at lambda + T (1) | write m0 and m1 (2)
    int32_t epi;            // update passes: layer stride of the per-warp staging for tile-local
                            // deferred sums (0: no tile of this launch has local variables)
};

// </jit-abi>
constexpr int kLbRing = FDOG_LB_RING;

// ---------------------------------------------------------------------------
// host-side decomposition
// ---------------------------------------------------------------------------
constexpr int kArcTop = -1;
constexpr int kArcBot = -2;

struct HostShape {
    int k = 0;
    int width = 0;                 // maximum nodes in a layer
    std::vector<int> lstart;       // k + 1
    std::vector<int> lo, hi;       // per node: node index, kArcTop or kArcBot
};

struct Decomposition {
    // presolve
    std::vector<int8_t> fixed;     // -1 in a BDD, 0/1 fixed, 2 in no row
    std::vector<int32_t> outside;  // variables with fixed != -1 (their value is set on the host)
    double const_lb = 0.0;         // sum fixed c x + sum free min(c, 0)
    double const_obj = 0.0;        // sum fixed c x + sum free c [c < 0]
    // BDDs in layout order
    std::vector<HostShape> shapes;
    std::vector<int> shape_cls;    // kernel class of each shape
    std::vector<int32_t> bdd_row;  // original row of each BDD (layout order)
    std::vector<int32_t> bdd_shape;  // shape of each BDD
    std::vector<int32_t> bdd_slot0;  // padded slot of layer 0 of each BDD (layer t at + t * kTile)
    std::vector<int32_t> row_bdd;    // BDD of each original row, -1 if presolve removed it
    std::vector<TileDev> tiles;
    std::vector<int32_t> cls_tile_begin;  // kNumClasses + 1 (tiles sorted by class)
    std::vector<int32_t> var;      // padded slots
    std::vector<int32_t> csr_off, csr_pos;
    std::vector<int32_t> patterns;  // 2 ints per pattern (see InstDev::patterns)
    std::vector<uint16_t> local_ent;
    std::vector<int32_t> work;      // variables left to the deferred-sum kernel, bucketed by copy count
    std::vector<int32_t> wpos;      // bucketed slot positions (see InstDev::wpos)
    std::vector<int32_t> shared_vars;  // shard of a split instance: variables with copies in other shards
    // serial schedule (update = 1, Eq. 4); empty otherwise
    std::vector<int32_t> tile_of_row;          // tile of each row of 32 padded slots
    std::vector<int32_t> lab_off;              // per tile: first float of its label region
    int64_t lab_floats = 0;                    // sum over tiles of (k + 1) * W * 32
    std::vector<int32_t> lev_f_off, lev_f_vars;  // variables by level, ascending sweep
    std::vector<int32_t> lev_b_off, lev_b_vars;  // descending sweep
    int32_t wb_start[FDOG_WBUCKETS + 1] = {0};
    int32_t wb_pos[FDOG_WBUCKETS] = {0};
    int64_t n_local_vars = 0;
    int64_t n_work_slots = 0;       // copies of the variables in `work`
    int64_t n_work_overflow = 0;    // of those, copies of variables with more than 8 (a warp each)
    bool cls_has_local[kNumClasses] = {false};
    std::vector<ShapeDev> shape_dev;
    std::vector<uint16_t> tpl;
    int64_t n_bdds = 0, n_slots = 0, n_nodes = 0, slots_pad = 0;
    int64_t n_work = 0, n_wpos = 0, n_local_ent = 0;  // sizes of work, wpos, local_ent
    int kmax[kNumClasses] = {0};
    // Plan built on the device: var, csr_off, csr_pos, work, wpos, local_ent
    // and bdd_row exist only in device memory (d_* until the instance's arena
    // takes the first six; bdd_row stays in d_bdd_row) until a host consumer
    // downloads them; bdd_shape, bdd_slot0 and row_bdd are then derived from
    // tiles and bdd_row.
    bool on_device = false;
    int32_t* d_var = nullptr;
    int32_t* d_csr_off = nullptr;
    int32_t* d_csr_pos = nullptr;
    int32_t* d_work = nullptr;
    int32_t* d_wpos = nullptr;
    uint16_t* d_local_ent = nullptr;
    int32_t* d_bdd_row = nullptr;
};

// Process-wide cache of large host buffers (host_pool.cpp).  A buffer of at
// least kHostPoolMin bytes that an instance frees is kept (up to a total of
// kHostPoolCap bytes) and handed to the next request of the same rounded
// size, whose pages are then already mapped: creating an instance of the
// same size again costs its copy, not the page faults of fresh memory.
constexpr size_t kHostPoolMin = size_t(1) << 20;
constexpr size_t kHostPoolCap = size_t(2) << 30;
void* host_pool_get(size_t bytes);  // throws std::bad_alloc
void host_pool_put(void* p, size_t bytes) noexcept;
size_t host_pool_release() noexcept;  // frees every cached buffer, returns the bytes

// std::allocator whose value-less construct leaves trivial types
// uninitialised: resize() then costs no fill pass over arrays that are
// written right after (the instance's copy of the ILP); large buffers come
// from the host buffer cache.
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = DefaultInitAlloc<U>;
    };
    DefaultInitAlloc() = default;
    template <class U>
    DefaultInitAlloc(const DefaultInitAlloc<U>&) noexcept {}
    T* allocate(size_t n) {
        if (n * sizeof(T) >= kHostPoolMin) return static_cast<T*>(host_pool_get(n * sizeof(T)));
        return std::allocator<T>::allocate(n);
    }
    void deallocate(T* p, size_t n) noexcept {
        if (n * sizeof(T) >= kHostPoolMin) host_pool_put(p, n * sizeof(T));
        else std::allocator<T>::deallocate(p, n);
    }
    template <class U>
    void construct(U* p) noexcept {
        ::new (static_cast<void*>(p)) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
    }
};
// fn(begin, end) over [0, n) in contiguous chunks on up to 16 host threads.
// Callers give each chunk independent work and combine any per-chunk results
// in chunk order, so the plan does not depend on the thread count.
template <class F>
inline void parallel_chunks(int64_t n, F&& fn) {
    const unsigned hw = std::max(1u, std::min(std::thread::hardware_concurrency(), 16u));
    const int nt = static_cast<int>(std::min<int64_t>(hw, (n + 32767) / 32768));
    if (nt <= 1) {
        fn(int64_t(0), n);
        return;
    }
    std::atomic<bool> failed{false};
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            try {
                fn(n * t / nt, n * (t + 1) / nt);
            } catch (...) {
                failed = true;
            }
        });
    for (auto& x : th) x.join();
    if (failed) throw std::bad_alloc();
}

// Builds the decomposition: presolve, BDDs per row (shared per row
// signature), tiles, interleaved slots and the per-variable slot lists.
// jit_mode: -1 no shape-specialised class; 0 eligible shapes with at least
// kJitMinBdds BDDs; 1 every eligible shape.  shared (n_vars flags, may be
// null): the instance is one shard of a split instance and these variables
// also have copies in other shards; they are kept out of the tile-local and
// deferred-sum lists and listed in shared_vars, and a shard whose rows would
// need presolve is refused (FDOG_EUNSUPPORTED).  Returns an FDOG_* status.
int build_decomposition(int32_t n_vars, const double* cost, int32_t n_rows, const int64_t* row_ptr,
                        const int32_t* col, const int32_t* coef, const int8_t* sense, const int64_t* rhs,
                        int jit_mode, bool fuse_local, Decomposition& out, std::string& err,
                        const uint8_t* shared = nullptr);

// The schedule of the serial update (Eq. 4) on a built decomposition: a
// variable's ascending level is one more than the largest level of the
// variables before it in its BDDs (0 if it leads each of them), so variables
// of one level share no BDD and visiting levels in order matches visiting
// variables in ascending index order on every BDD; likewise descending.
void build_serial_schedule(int32_t n_vars, Decomposition& d);

// shape-specialised code (jit.cpp): process-wide shape registry and kernels
int jit_register_shape(const HostShape& s);  // id of the shape's structure
struct JitKernels {
    const void* fn[4] = {nullptr, nullptr, nullptr, nullptr};  // per sweep mode
};
// host-only NVRTC compile of the module for the given shape ids (cached)
int jit_compile(const std::vector<int>& ids, std::string& err);
// compiles if needed and loads the module; empty ids -> no kernels
int jit_kernels(const std::vector<int>& ids, JitKernels& out, std::string& err);
// the generated CUDA source of the module (for inspection)
std::string jit_source(const std::vector<int>& ids);

// The BDD of one row (coefficients of its non-zero entries in ascending
// variable order, no variable fixed); `presolve` is set when the row forces
// some variable or accepts every assignment (the host presolve then has work).
int analyse_row(const std::vector<int64_t>& a, int8_t sense, int64_t rhs, HostShape& shape, bool& presolve);
// kernel class of a shape with n_bdds BDDs under a jit mode, -1 if no kernel takes it
int shape_class(const HostShape& s, int jit_mode, int64_t n_bdds);
// per-shape device descriptors and successor-code templates of out.shapes / out.shape_cls
void build_templates(Decomposition& out);

// BDD of { x in {0,1}^k : lo_bound <= sum a_t x_t <= hi_bound } (either bound optional).
int build_row_shape(const std::vector<int64_t>& a, bool has_lo, int64_t lo_bound, bool has_hi, int64_t hi_bound,
                    HostShape& out);

}  // namespace fdog
