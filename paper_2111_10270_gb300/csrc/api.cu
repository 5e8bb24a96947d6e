// C ABI of the FastDOG GB300 library (include/fastdog.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "engine.h"
#include "instance.h"
#include "kernels.h"

using namespace fdog;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

namespace fdog {

cudaError_t copy_async(fdog_instance* inst, void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    if (kind == cudaMemcpyHostToDevice) inst->h2d_bytes += static_cast<int64_t>(bytes);
    if (kind == cudaMemcpyDeviceToHost) inst->d2h_bytes += static_cast<int64_t>(bytes);
    return cudaMemcpyAsync(dst, src, bytes, kind, inst->stream);
}

int fail_cuda(fdog_instance* inst, cudaError_t e, const char* where) {
    if (inst) inst->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return FDOG_ECUDA;
}

struct Item {
    void** ptr;
    size_t bytes;
};

// Every device array of the instance, in arena order.
static std::vector<Item> arena_items(const fdog_instance* inst, DevArrays& a) {
    const Decomposition& d = inst->dec;
    const int64_t n = inst->n_vars;
    const int64_t S = d.slots_pad;
    const int64_t nt = static_cast<int64_t>(d.tiles.size());
    const int64_t nchunks = std::max<int64_t>(1, (nt + kLbChunk - 1) / kLbChunk);
    const int64_t nobj = std::max<int64_t>(1, (n + kObjChunk - 1) / kObjChunk);
    auto sz = [](int64_t v) { return static_cast<size_t>(std::max<int64_t>(v, 1)); };
    return {
        {reinterpret_cast<void**>(&a.inst), sizeof(InstDev)},
        {reinterpret_cast<void**>(&a.ctl), sizeof(InstCtl)},
        {reinterpret_cast<void**>(&a.tiles), sizeof(TileDev) * sz(nt)},
        {reinterpret_cast<void**>(&a.shapes), sizeof(ShapeDev) * sz(static_cast<int64_t>(d.shape_dev.size()))},
        {reinterpret_cast<void**>(&a.tpl), sizeof(uint16_t) * std::max<size_t>(d.tpl.size(), 8)},
        {reinterpret_cast<void**>(&a.lam), sizeof(float) * sz(S)},
        {reinterpret_cast<void**>(&a.var), sizeof(int32_t) * sz(S)},
        {reinterpret_cast<void**>(&a.mm0), sizeof(float) * sz(S)},
        {reinterpret_cast<void**>(&a.T), sizeof(float) * sz(n)},
        {reinterpret_cast<void**>(&a.C), sizeof(float) * sz(n)},
        {reinterpret_cast<void**>(&a.pert), sizeof(float) * sz(n)},
        {reinterpret_cast<void**>(&a.x), sz(n)},
        {reinterpret_cast<void**>(&a.cost), sizeof(double) * sz(n)},
        {reinterpret_cast<void**>(&a.csr_off), sizeof(int32_t) * static_cast<size_t>(n + 1)},
        {reinterpret_cast<void**>(&a.csr_pos), sizeof(int32_t) * sz(d.n_slots)},
        {reinterpret_cast<void**>(&a.patterns), sizeof(int32_t) * std::max<size_t>(d.patterns.size(), 2)},
        {reinterpret_cast<void**>(&a.local_ent), sizeof(uint16_t) * static_cast<size_t>(std::max<int64_t>(d.n_local_ent, 4))},
        {reinterpret_cast<void**>(&a.work), sizeof(int32_t) * sz(d.n_work)},
        {reinterpret_cast<void**>(&a.wpos), sizeof(int32_t) * sz(d.n_wpos)},
        {reinterpret_cast<void**>(&a.lab), sizeof(float) * static_cast<size_t>(std::max<int64_t>(d.lab_floats, 1))},
        {reinterpret_cast<void**>(&a.lab_off), sizeof(int32_t) * std::max<size_t>(d.lab_off.size(), 1)},
        {reinterpret_cast<void**>(&a.tile_of_row), sizeof(int32_t) * std::max<size_t>(d.tile_of_row.size(), 1)},
        {reinterpret_cast<void**>(&a.lev_f), sizeof(int32_t) * std::max<size_t>(d.lev_f_vars.size(), 1)},
        {reinterpret_cast<void**>(&a.lev_b), sizeof(int32_t) * std::max<size_t>(d.lev_b_vars.size(), 1)},
        {reinterpret_cast<void**>(&a.tile_lb), sizeof(float2) * sz(nt)},
        {reinterpret_cast<void**>(&a.chunk_lb), sizeof(double) * static_cast<size_t>(nchunks)},
        {reinterpret_cast<void**>(&a.obj_chunk), sizeof(double) * static_cast<size_t>(nobj)},
        {reinterpret_cast<void**>(&a.prefix), sizeof(int32_t) * kPrefixInts},
        {reinterpret_cast<void**>(&a.sh_vars), sizeof(int32_t) * std::max<size_t>(d.shared_vars.size(), 1)},
        {reinterpret_cast<void**>(&a.sh_copies), sizeof(int32_t) * std::max<size_t>(d.shared_vars.size(), 1)},
        {reinterpret_cast<void**>(&a.sh_slot), sizeof(int32_t) * std::max<size_t>(d.shared_vars.size(), 1)},
    };
}

size_t arena_size(const fdog_instance* inst) {
    DevArrays tmp;
    size_t total = 0;
    for (const Item& it : arena_items(inst, tmp)) total = align_up(total + it.bytes, 256);
    return total;
}

// Upper bound of the device memory fdog_build_bdds needs for an unplanned
// instance that the device builder plans: the builder's temporaries (the
// uploaded rows, hash tables, keys and ranks) plus the instance's arena,
// bounded from the ILP's sizes alone (at most 1,024 shapes, each padding its
// last tile by at most 31 BDDs; at most 16 nodes per layer).
int64_t device_plan_bytes_bound(const fdog_instance* inst) {
    const int64_t n = inst->n_vars, m = inst->n_rows, nnz = inst->row_ptr[m];
    int64_t maxk = 0;
    for (int64_t j = 0; j < m; ++j) maxk = std::max<int64_t>(maxk, inst->row_ptr[j + 1] - inst->row_ptr[j]);
    const int64_t shapes = std::min<int64_t>(m, 1024);
    const int64_t nt = (m + kTile - 1) / kTile + shapes;
    const int64_t S = nnz + std::min<int64_t>(31 * shapes * maxk, 31 * nnz);
    const int64_t tpl = 2 * 16 * std::min<int64_t>(nnz, shapes * maxk);
    const int64_t arena = static_cast<int64_t>(sizeof(InstDev) + sizeof(InstCtl)) + 48 * nt + 16 * shapes + tpl +
                          12 * S + 29 * n + 4 + 8 * nnz + 8 * nt + 4 * (nt / kLbChunk + 1) * 2 +
                          8 * (n / kObjChunk + 1) + 4 * kPrefixInts + 40 * 256;
    const int64_t temporaries = 48 * nnz + 64 * m + (64 << 20);
    return arena + temporaries;
}

std::vector<int> jit_ids(const fdog_instance* inst) {
    std::vector<int> ids;
    for (const ShapeDev& s : inst->dec.shape_dev)
        if (s.jit >= 0) ids.push_back(s.jit);
    return ids;
}

// rows longer than the shared-memory sweep kernels take (either builder)
static int check_layer_limits(fdog_instance* inst) {
    for (int c = 0; c < kNumClasses; ++c)
        if (!class_is_reg(c) && inst->dec.kmax[c] > smem_max_layers(class_width(c))) {
            inst->last_error = "row longer than the shared-memory sweep kernels take";
            return FDOG_EUNSUPPORTED;
        }
    return FDOG_OK;
}

int plan(fdog_instance* inst, bool compile_jit) {
    if (inst->planned) return FDOG_OK;
    free_device_plan(inst->dec, inst->stream);
    const auto t0 = std::chrono::steady_clock::now();
    int rc;
    try {
        rc = build_decomposition(inst->n_vars, inst->cost.data(), inst->n_rows, inst->row_ptr.data(),
                                 inst->col.data(), inst->coef.data(), inst->sense.data(), inst->rhs.data(),
                                 inst->jit_failed ? -1 : inst->params.jit, inst->params.fuse >= 0, inst->dec,
                                 inst->last_error, inst->shard ? inst->shard_shared.data() : nullptr);
    } catch (const std::bad_alloc&) {
        rc = FDOG_ENOMEM;
    } catch (...) {
        rc = FDOG_EINVAL;
    }
    if (rc != FDOG_OK) return rc;
    if (inst->shard && (rc = shard_check_copies(inst)) != FDOG_OK) return rc;
    inst->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    inst->planned_on_device = false;
    if ((rc = check_layer_limits(inst)) != FDOG_OK) return rc;
    if (inst->params.update == 1) build_serial_schedule(inst->n_vars, inst->dec);
    std::vector<int> ids = jit_ids(inst);
    if (compile_jit && !ids.empty()) {
        std::string why;
        if (jit_compile(ids, why) != FDOG_OK) {
            // shape-specialised kernels unavailable: plan again for the generic kernels only
            inst->jit_note = why;
            inst->jit_failed = true;
            return plan(inst, true);
        }
    }
    inst->planned = true;
    return FDOG_OK;
}

// Planning at build time: the device builder where the instance allows it
// (parallel update, planner != 1), else the host builder.  Both give the
// same plan.
static int plan_for_build(fdog_instance* inst) {
    if (inst->planned) return FDOG_OK;
    const int mode = inst->params.planner;
    if (mode != 1 && inst->params.update == 0 && !inst->shard) {
        int rc = plan_on_device(inst, inst->jit_failed ? -1 : inst->params.jit, inst->params.fuse >= 0);
        if (rc == FDOG_OK) {
            if ((rc = check_layer_limits(inst)) != FDOG_OK) {
                free_device_plan(inst->dec, inst->stream);
                return rc;
            }
            std::vector<int> ids = jit_ids(inst);
            std::string why;
            if (!ids.empty() && jit_compile(ids, why) != FDOG_OK) {
                inst->jit_note = why;
                inst->jit_failed = true;
                free_device_plan(inst->dec, inst->stream);
                return plan_for_build(inst);
            }
            inst->planned = true;
            inst->planned_on_device = true;
            return FDOG_OK;
        }
        if (rc != plan_leave_to_host()) return rc;
    }
    if (mode == 2) {
        inst->last_error = "the device planner does not take this instance (presolve work, serial update, "
                           "a shard of a split instance, too many row signatures or copies)";
        return FDOG_EUNSUPPORTED;
    }
    return plan(inst);
}

int ensure_host_plan(fdog_instance* inst) {
    Decomposition& d = inst->dec;
    if (!d.on_device) return FDOG_OK;
    if (!inst->arena || !d.d_bdd_row) return FDOG_ESTATE;
    DeviceGuard g(inst->device);
    const int64_t n = inst->n_vars;
    try {
        d.var.resize(d.slots_pad);
        d.csr_off.resize(n + 1);
        d.csr_pos.resize(d.n_slots);
        d.work.resize(d.n_work);
        d.wpos.resize(d.n_wpos);
        d.local_ent.resize(d.n_local_ent);
        d.bdd_row.resize(d.n_bdds);
    } catch (const std::bad_alloc&) {
        return FDOG_ENOMEM;
    }
    cudaError_t e = cudaStreamSynchronize(inst->stream);
    auto down = [&](void* dst, const void* src, size_t bytes) {
        if (bytes > 0 && e == cudaSuccess) e = copy_async(inst, dst, src, bytes, cudaMemcpyDeviceToHost);
    };
    const DevArrays& a = inst->dev;
    down(d.var.data(), a.var, sizeof(int32_t) * d.var.size());
    down(d.csr_off.data(), a.csr_off, sizeof(int32_t) * d.csr_off.size());
    down(d.csr_pos.data(), a.csr_pos, sizeof(int32_t) * d.csr_pos.size());
    down(d.work.data(), a.work, sizeof(int32_t) * d.work.size());
    down(d.wpos.data(), a.wpos, sizeof(int32_t) * d.wpos.size());
    down(d.local_ent.data(), a.local_ent, sizeof(uint16_t) * d.local_ent.size());
    down(d.bdd_row.data(), d.d_bdd_row, sizeof(int32_t) * d.bdd_row.size());
    if (e == cudaSuccess) e = cudaStreamSynchronize(inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "plan download");
    d.bdd_shape.resize(d.n_bdds);
    d.bdd_slot0.resize(d.n_bdds);
    d.row_bdd.assign(inst->n_rows, -1);
    for (const TileDev& t : d.tiles)
        for (int l = 0; l < t.n_valid; ++l) {
            const int32_t b = t.bdd_base + l;
            d.bdd_shape[b] = t.shape;
            d.bdd_slot0[b] = t.slot_base + l;
            d.row_bdd[d.bdd_row[b]] = b;
        }
    free_device_plan(d, inst->stream);
    d.on_device = false;
    return FDOG_OK;
}

// Lay out every device array of the instance inside one allocation.
int allocate_and_upload(fdog_instance* inst) {
    Decomposition& d = inst->dec;
    const int64_t n = inst->n_vars;
    const int64_t S = d.slots_pad;
    const int64_t nt = static_cast<int64_t>(d.tiles.size());
    const int64_t nchunks = std::max<int64_t>(1, (nt + kLbChunk - 1) / kLbChunk);
    const int64_t nobj = std::max<int64_t>(1, (n + kObjChunk - 1) / kObjChunk);
    DevArrays& a = inst->dev;
    std::vector<Item> items = arena_items(inst, a);
    size_t total = 0;
    std::vector<size_t> offs(items.size());
    for (size_t q = 0; q < items.size(); ++q) {
        offs[q] = total;
        total = align_up(total + items[q].bytes, 256);
    }
    cudaError_t e = cudaMalloc(&inst->arena, total);
    if (e != cudaSuccess) {
        inst->arena = nullptr;
        inst->last_error = "cudaMalloc of " + std::to_string(total) + " bytes failed";
        cudaGetLastError();
        return FDOG_ENOMEM;
    }
    inst->arena_bytes = total;
    for (size_t q = 0; q < items.size(); ++q) *items[q].ptr = static_cast<char*>(inst->arena) + offs[q];

    // descriptor
    InstDev h{};
    h.tiles = a.tiles;
    h.shapes = a.shapes;
    h.tpl = a.tpl;
    h.lam = a.lam;
    h.var = a.var;
    h.mm0 = a.mm0;
    h.mm1 = nullptr;
    h.T = a.T;
    h.C = a.C;
    h.csr_off = a.csr_off;
    h.csr_pos = a.csr_pos;
    h.patterns = a.patterns;
    h.local_ent = a.local_ent;
    h.work = a.work;
    h.wpos = a.wpos;
    h.lab = a.lab;
    h.lab_off = a.lab_off;
    h.tile_of_row = a.tile_of_row;
    h.n_work = static_cast<int32_t>(d.n_work);
    for (int b = 0; b <= FDOG_WBUCKETS; ++b) h.wb_start[b] = d.wb_start[b];
    for (int b = 0; b < FDOG_WBUCKETS; ++b) h.wb_pos[b] = d.wb_pos[b];
    h.cost = a.cost;
    h.pert = a.pert;
    h.x = a.x;
    h.tile_lb = a.tile_lb;
    h.chunk_lb = a.chunk_lb;
    h.obj_chunk = a.obj_chunk;
    h.ctl = a.ctl;
    h.n_tiles = static_cast<int32_t>(nt);
    h.n_vars = static_cast<int32_t>(n);
    h.n_chunks = static_cast<int32_t>(nchunks);
    h.n_obj_chunks = static_cast<int32_t>(nobj);
    h.omega = static_cast<float>(inst->params.omega);
    h.const_lb = d.const_lb;
    h.alpha = inst->params.alpha;
    h.delta0 = inst->params.delta;
    h.seed = inst->params.seed;
    h.stop_param = inst->params.tol > 0 ? 1 : 0;
    h.reopt_iters = inst->params.rounding_dual_iters;
    inst->hdesc = h;

    // self-batch prefix arrays: per class (prefix[2], first[1]), then vars, slots, chunks, objective chunks
    std::vector<int32_t> pre(kPrefixInts, 0);
    DevBatch& b = inst->batch;
    b = DevBatch();
    b.insts = a.inst;
    b.n_inst = 1;
    b.jit = inst->jit;
    b.l2 = l2_window_for(inst->device, a.T, sizeof(float) * n);
    int q = 0;
    for (int c = 0; c < kNumClasses; ++c) {
        pre[q] = 0;
        pre[q + 1] = d.cls_tile_begin[c + 1] - d.cls_tile_begin[c];
        pre[q + 2] = d.cls_tile_begin[c];
        b.tile_prefix[c] = a.prefix + q;
        b.tile_first[c] = a.prefix + q + 2;
        b.tiles_total[c] = pre[q + 1];
        b.kmax[c] = d.kmax[c];
        q += 3;
    }
    auto two = [&](int32_t** dst, int32_t v) {
        pre[q] = 0;
        pre[q + 1] = v;
        *dst = a.prefix + q;
        q += 2;
    };
    two(&b.var_prefix, static_cast<int32_t>(n));
    b.vars_total = static_cast<int32_t>(n);
    two(&b.tile_all_prefix, static_cast<int32_t>(nt));
    b.tiles_all_total = static_cast<int32_t>(nt);
    two(&b.work_prefix, d.wb_start[FDOG_WBUCKETS - 1]);
    b.work_total = d.wb_start[FDOG_WBUCKETS - 1];
    two(&b.wide_prefix, d.wb_start[FDOG_WBUCKETS] - d.wb_start[FDOG_WBUCKETS - 1]);
    b.wide_total = d.wb_start[FDOG_WBUCKETS] - d.wb_start[FDOG_WBUCKETS - 1];
    for (int c = 0; c < kNumClasses; ++c) b.has_local[c] = d.cls_has_local[c];
    two(&b.slot_prefix, static_cast<int32_t>(S));
    b.slots_total = static_cast<int32_t>(S);
    two(&b.chunk_prefix, static_cast<int32_t>(nt > 0 ? nchunks : 0));
    b.chunks_total = static_cast<int32_t>(nt > 0 ? nchunks : 0);
    two(&b.objchunk_prefix, static_cast<int32_t>(n > 0 ? nobj : 0));
    b.objchunks_total = static_cast<int32_t>(n > 0 ? nobj : 0);

    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (bytes == 0 || e != cudaSuccess) return;
        e = copy_async(inst, dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(a.inst, &h, sizeof(h));
    up(a.tiles, d.tiles.data(), sizeof(TileDev) * nt);
    up(a.shapes, d.shape_dev.data(), sizeof(ShapeDev) * d.shape_dev.size());
    up(a.tpl, d.tpl.data(), sizeof(uint16_t) * d.tpl.size());
    up(a.cost, inst->cost.data(), sizeof(double) * n);
    up(a.patterns, d.patterns.data(), sizeof(int32_t) * d.patterns.size());
    if (d.on_device) {
        // arrays of a device-built plan: into the arena, then their buffers are released
        auto d2d = [&](void* dst, const void* src, int64_t bytes) {
            if (bytes > 0 && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, inst->stream);
        };
        d2d(a.var, d.d_var, sizeof(int32_t) * S);
        d2d(a.csr_off, d.d_csr_off, sizeof(int32_t) * (n + 1));
        d2d(a.csr_pos, d.d_csr_pos, sizeof(int32_t) * d.n_slots);
        d2d(a.local_ent, d.d_local_ent, sizeof(uint16_t) * d.n_local_ent);
        d2d(a.work, d.d_work, sizeof(int32_t) * d.n_work);
        d2d(a.wpos, d.d_wpos, sizeof(int32_t) * d.n_wpos);
        int32_t* keep = d.d_bdd_row;
        d.d_bdd_row = nullptr;
        free_device_plan(d, inst->stream);
        d.d_bdd_row = keep;
    } else {
        up(a.var, d.var.data(), sizeof(int32_t) * S);
        up(a.csr_off, d.csr_off.data(), sizeof(int32_t) * (n + 1));
        up(a.csr_pos, d.csr_pos.data(), sizeof(int32_t) * d.n_slots);
        up(a.local_ent, d.local_ent.data(), sizeof(uint16_t) * d.local_ent.size());
        up(a.work, d.work.data(), sizeof(int32_t) * d.work.size());
        up(a.wpos, d.wpos.data(), sizeof(int32_t) * d.wpos.size());
    }
    up(a.lab_off, d.lab_off.data(), sizeof(int32_t) * d.lab_off.size());
    up(a.tile_of_row, d.tile_of_row.data(), sizeof(int32_t) * d.tile_of_row.size());
    up(a.lev_f, d.lev_f_vars.data(), sizeof(int32_t) * d.lev_f_vars.size());
    up(a.lev_b, d.lev_b_vars.data(), sizeof(int32_t) * d.lev_b_vars.size());
    up(a.prefix, pre.data(), sizeof(int32_t) * kPrefixInts);
    if (!d.shared_vars.empty()) {
        // copy counts over all shards, and each variable's rank among all shared variables
        std::vector<int32_t> cnt(d.shared_vars.size()), slot(d.shared_vars.size());
        std::vector<int32_t> rank(static_cast<size_t>(n) + 1, 0);
        for (int64_t i = 0; i < n; ++i) rank[i + 1] = rank[i] + inst->shard_shared[i];
        for (size_t k = 0; k < cnt.size(); ++k) {
            cnt[k] = inst->shard_copies[d.shared_vars[k]];
            slot[k] = rank[d.shared_vars[k]];
        }
        // pageable sources: staged before each call returns
        up(a.sh_vars, d.shared_vars.data(), sizeof(int32_t) * d.shared_vars.size());
        up(a.sh_copies, cnt.data(), sizeof(int32_t) * cnt.size());
        up(a.sh_slot, slot.data(), sizeof(int32_t) * slot.size());
    }
    if (e != cudaSuccess) return fail_cuda(inst, e, "upload");
    return FDOG_OK;
}

// The engine and one-member view behind an instance's own calls.
int own_engine(fdog_instance* inst, Engine** eng, BatchView** view) {
    if (!inst->engine) {
        inst->engine = new (std::nothrow) Engine();
        inst->self_view = new (std::nothrow) BatchView();
        if (!inst->engine || !inst->self_view) return FDOG_ENOMEM;
    }
    Engine& e = *inst->engine;
    e.device = inst->device;
    e.stream = inst->stream;
    e.cfg = inst->cfg;
    e.prof = &inst->prof;
    engine_use_side(e);
    int rc = view_build(e, *inst->self_view, {inst});
    if (rc != FDOG_OK) {
        inst->last_error = e.err;
        return rc;
    }
    *eng = inst->engine;
    *view = inst->self_view;
    return FDOG_OK;
}

// Frees the instance's device memory; its plan, parameters and last solution
// stay on the host (a later fdog_build_bdds uploads it again).
int release_device(fdog_instance* inst) {
    if (!inst->built) return FDOG_OK;
    DeviceGuard g(inst->device);
    cudaStreamSynchronize(inst->stream);
    int rc = ensure_host_plan(inst);  // the plan stays on the host for a later build
    if (rc != FDOG_OK) return rc;
    delete inst->self_view;
    inst->self_view = nullptr;
    delete inst->engine;
    inst->engine = nullptr;
    if (inst->arena) cudaFree(inst->arena);
    if (inst->dev.mm1) cudaFree(inst->dev.mm1);
    if (inst->host_ctl) cudaFreeHost(inst->host_ctl);
    if (inst->solution_pinned && inst->host_x) {
        inst->solution.assign(inst->host_x, inst->host_x + inst->n_vars);  // keep the last solution
        inst->solution_pinned = false;
    }
    if (inst->host_x) cudaFreeHost(inst->host_x);
    inst->prof.release();
    cudaGetLastError();
    inst->arena = nullptr;
    inst->arena_bytes = 0;
    inst->host_ctl = nullptr;
    inst->host_x = nullptr;
    inst->dev = DevArrays();
    inst->built = false;
    inst->pending_T = false;
    inst->iterated = false;
    return FDOG_OK;
}

int reset_dual_state(fdog_instance* inst) {
    InstCtl c{};
    const fdog_params& p = inst->params;
    c.stop_enabled = p.tol > 0 ? 1 : 0;
    c.window = p.window;
    c.min_iters = p.min_iters;
    c.tol = p.tol;
    c.iter_limit = inst->shard ? INT32_MAX : 0;  // a shard's passes are driven by fdog_shard_pass
    c.delta = p.delta;
    cudaError_t e = copy_async(inst, inst->dev.ctl, &c, sizeof(c), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail_cuda(inst, e, "reset ctl");
    e = launch_init(inst->batch, inst->cfg, inst->stream);
    if (e == cudaSuccess && inst->shard) e = launch_shard_init(inst);
    if (e != cudaSuccess) return fail_cuda(inst, e, "init");
    inst->pending_T = false;
    inst->iterated = false;
    return FDOG_OK;
}

int read_ctl(fdog_instance* inst, InstCtl& out) {
    cudaError_t e = copy_async(inst, inst->host_ctl, inst->dev.ctl, sizeof(InstCtl), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaStreamSynchronize(inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "read control block");
    out = *inst->host_ctl;
    if (out.error != 0) {
        inst->last_error = "device-side error " + std::to_string(out.error);
        return FDOG_ETIMEOUT;
    }
    return FDOG_OK;
}

int set_ctl_field(fdog_instance* inst, size_t offset, const void* v, size_t bytes) {
    cudaError_t e = copy_async(inst, reinterpret_cast<char*>(inst->dev.ctl) + offset, v, bytes,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(inst->stream);  // v may be a stack temporary
    return e == cudaSuccess ? FDOG_OK : fail_cuda(inst, e, "write control block");
}

// Energy sum (+ presolve constant) at lambda, or at lambda + T (the add-back),
// with FP64 shortest-path labels and FP64 compensated sums (eval.cu).
int evaluate(fdog_instance* inst, bool add_t, double* out) {
    cudaError_t e = launch_eval64(inst->batch, add_t, inst->cfg, inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "evaluate");
    InstCtl c;
    int rc = read_ctl(inst, c);
    if (rc != FDOG_OK) return rc;
    *out = inst->dec.n_bdds > 0 ? c.lb_eval : inst->dec.const_lb;
    return FDOG_OK;
}

int addback(fdog_instance* inst) {
    if (!inst->pending_T) return FDOG_OK;
    cudaError_t e = launch_addback(inst->batch, inst->cfg, inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "add-back");
    inst->pending_T = false;
    inst->iterated = false;
    return FDOG_OK;
}

int ensure_mm1(fdog_instance* inst) {
    if (inst->dev.mm1) return FDOG_OK;
    void* p = nullptr;
    size_t bytes = sizeof(float) * std::max<int64_t>(inst->dec.slots_pad, 1);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return FDOG_ENOMEM; }
    inst->dev.mm1 = static_cast<float*>(p);
    inst->hdesc.mm1 = inst->dev.mm1;
    if (inst->self_view) inst->self_view->uids.clear();  // rebuild its descriptor copy on next use
    e = copy_async(inst, inst->dev.inst, &inst->hdesc, sizeof(InstDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(inst->stream);
    return e == cudaSuccess ? FDOG_OK : fail_cuda(inst, e, "descriptor update");
}

// Upload, initial dual state and (optionally) launch-shape tuning of a planned instance.
int build_instance(fdog_instance* inst, int32_t device, void* cuda_stream, bool autotune) {
    if (!inst) return FDOG_EINVAL;
    if (inst->built) return FDOG_ESTATE;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        inst->last_error = "no CUDA device " + std::to_string(device);
        return e != cudaSuccess ? FDOG_ECUDA : FDOG_EINVAL;
    }
    DeviceGuard g(device);
    inst->device = device;
    inst->stream = static_cast<cudaStream_t>(cuda_stream);
    int rc = plan_for_build(inst);
    if (rc != FDOG_OK) return rc;
    const std::vector<int> ids = jit_ids(inst);
    if (!ids.empty()) {
        std::string why;
        if (jit_kernels(ids, inst->jit, why) != FDOG_OK) {
            // shape-specialised kernels unavailable: plan again for the generic kernels
            inst->jit_note = why;
            inst->jit_failed = true;
            inst->planned = false;
            free_device_plan(inst->dec, inst->stream);
            if ((rc = plan_for_build(inst)) != FDOG_OK) return rc;
        }
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return fail_cuda(inst, e, "device properties");
    inst->cfg.num_sms = prop.multiProcessorCount;
    inst->cfg.warps_per_block = inst->params.block_threads > 0 ? inst->params.block_threads / 32 : 4;
    inst->cfg.max_waves = inst->params.grid_waves > 0 ? inst->params.grid_waves : (inst->params.grid_waves < 0 ? 0 : 1);
    inst->cfg.prof = &inst->prof;
    e = cudaMallocHost(reinterpret_cast<void**>(&inst->host_ctl), sizeof(InstCtl));
    if (e != cudaSuccess) { cudaGetLastError(); inst->host_ctl = nullptr; return FDOG_ENOMEM; }
    e = cudaMallocHost(reinterpret_cast<void**>(&inst->host_x), std::max<size_t>(inst->n_vars, 1));
    if (e != cudaSuccess) { cudaGetLastError(); inst->host_x = nullptr; return FDOG_ENOMEM; }
    rc = allocate_and_upload(inst);
    if (rc != FDOG_OK) return rc;
    rc = reset_dual_state(inst);
    if (rc != FDOG_OK) return rc;
    e = cudaStreamSynchronize(inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "build");
    inst->built = true;
    if (autotune && inst->dec.n_bdds > 0) {
        // launch shape of this instance's sweeps (results do not depend on it)
        Engine* eng;
        BatchView* v;
        if ((rc = own_engine(inst, &eng, &v)) != FDOG_OK) return rc;
        if ((rc = view_autotune(*eng, *v, inst->params.grid_waves == 0)) != FDOG_OK) {
            inst->last_error = eng->err;
            return rc;
        }
        inst->cfg.warps_per_block = eng->cfg.warps_per_block;
        inst->cfg.max_waves = eng->cfg.max_waves;
    }
    return FDOG_OK;
}

}  // namespace fdog

// ===========================================================================
// extern "C"
// ===========================================================================
extern "C" {

int fdog_params_default(fdog_params* p) {
    if (!p) return FDOG_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->omega = 0.5;
    p->delta = 1.0;
    p->alpha = 1.2;
    p->tol = 1e-4;
    p->window = 10;
    p->min_iters = 20;
    p->rounding_dual_iters = 20;
    p->max_rounds = 200;
    p->seed = 0;
    p->block_threads = 0;
    p->grid_waves = 0;
    p->update = 0;
    p->planner = 0;
    return FDOG_OK;
}

const char* fdog_status_string(int s) {
    switch (s) {
        case FDOG_OK: return "ok";
        case FDOG_EINVAL: return "invalid argument";
        case FDOG_ENOMEM: return "out of memory";
        case FDOG_EINFEASIBLE: return "infeasible row";
        case FDOG_ECUDA: return "CUDA error";
        case FDOG_ESTATE: return "call out of order";
        case FDOG_ETIMEOUT: return "device wait timed out";
        case FDOG_ENOCONVERGE: return "rounding did not converge";
        case FDOG_EUNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

int fdog_create(int32_t n_vars, const double* cost, int32_t n_rows, const int64_t* row_ptr, const int32_t* col,
                const int32_t* coef, const int8_t* sense, const int64_t* rhs, const fdog_params* params,
                fdog_instance** out) {
    if (!out) return FDOG_EINVAL;
    *out = nullptr;
    if (n_vars < 0 || n_rows < 0) return FDOG_EINVAL;
    if ((n_vars > 0 && !cost) || (n_rows > 0 && (!row_ptr || !sense || !rhs))) return FDOG_EINVAL;
    fdog_params p;
    if (params) p = *params; else fdog_params_default(&p);
    if (!(p.omega > 0.0 && p.omega <= 1.0) || !(p.delta > 0.0) || !(p.alpha >= 1.0) || p.window < 1 ||
        p.window >= kLbRing || p.min_iters < 0 || p.rounding_dual_iters < 0 || p.max_rounds < 0 ||
        p.block_threads < 0 || p.block_threads > 1024 || (p.block_threads % 32) != 0 || p.grid_waves < -1 ||
        p.update < 0 || p.update > 1 || p.planner < 0 || p.planner > 2)
        return FDOG_EINVAL;
    // copy and validate in one parallel pass per array (rows checked independently)
    fdog_instance* inst = new (std::nothrow) fdog_instance();
    if (!inst) return FDOG_ENOMEM;
    static std::atomic<uint64_t> next_uid{1};
    inst->uid = next_uid.fetch_add(1);
    inst->n_vars = n_vars;
    inst->n_rows = n_rows;
    inst->params = p;
    std::atomic<bool> bad{false};
    int rc = FDOG_OK;
    try {
        inst->cost.resize(n_vars);
        if (n_vars > 0) parallel_chunks(n_vars, [&](int64_t i0, int64_t i1) {
            std::memcpy(inst->cost.data() + i0, cost + i0, sizeof(double) * (i1 - i0));
            for (int64_t i = i0; i < i1; ++i)
                if (!std::isfinite(cost[i])) { bad = true; break; }
        });
        inst->row_ptr.resize(n_rows + 1);
        inst->row_ptr[0] = 0;
        if (n_rows > 0 && row_ptr[0] != 0) bad = true;
        inst->sense.resize(n_rows);
        inst->rhs.resize(n_rows);
        if (!bad && n_rows > 0) {
            parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
                std::memcpy(inst->row_ptr.data() + j0 + 1, row_ptr + j0 + 1, sizeof(int64_t) * (j1 - j0));
                std::memcpy(inst->sense.data() + j0, sense + j0, j1 - j0);
                std::memcpy(inst->rhs.data() + j0, rhs + j0, sizeof(int64_t) * (j1 - j0));
                for (int64_t j = j0; j < j1; ++j)
                    if (row_ptr[j + 1] < row_ptr[j] || sense[j] < -1 || sense[j] > 1) { bad = true; break; }
            });
        }
        const int64_t nnz = bad ? 0 : inst->row_ptr[n_rows];
        if (!bad && nnz > 0 && (!col || !coef)) bad = true;
        if (!bad && n_rows > 0) {
            inst->col.resize(nnz);
            inst->coef.resize(nnz);
            // columns in range and no column twice in a row (rows in ascending
            // column order pass without sorting)
            parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
                const int64_t q0 = row_ptr[j0], q1 = row_ptr[j1];
                std::memcpy(inst->col.data() + q0, col + q0, sizeof(int32_t) * (q1 - q0));
                std::memcpy(inst->coef.data() + q0, coef + q0, sizeof(int32_t) * (q1 - q0));
                std::vector<int32_t> cols;
                for (int64_t j = j0; j < j1 && !bad; ++j) {
                    bool ascending = true;
                    for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
                        if (col[q] < 0 || col[q] >= n_vars) { bad = true; break; }
                        if (q > row_ptr[j] && col[q] <= col[q - 1]) ascending = false;
                    }
                    if (ascending || bad) continue;
                    cols.assign(col + row_ptr[j], col + row_ptr[j + 1]);
                    std::sort(cols.begin(), cols.end());
                    if (std::adjacent_find(cols.begin(), cols.end()) != cols.end()) bad = true;
                }
            });
        }
    } catch (...) {
        rc = FDOG_ENOMEM;
    }
    if (rc == FDOG_OK && bad) rc = FDOG_EINVAL;
    if (rc != FDOG_OK) {
        delete inst;
        return rc;
    }
    *out = inst;
    return FDOG_OK;
}

int fdog_build_bdds(fdog_instance* inst, int32_t device, void* cuda_stream) {
    if (!inst) return FDOG_EINVAL;
    return build_instance(inst, device, cuda_stream, inst->params.block_threads == 0);
}

int fdog_plan(fdog_instance* inst, int64_t* device_bytes) {
    if (!inst) return FDOG_EINVAL;
    int rc = plan(inst);
    if (rc != FDOG_OK) return rc;
    if (device_bytes) *device_bytes = static_cast<int64_t>(arena_size(inst));
    return FDOG_OK;
}

int fdog_kernel_plan(fdog_instance* inst, int32_t* jit_shapes, int64_t* jit_tiles, int64_t* static_tiles,
                     int64_t* local_vars, int64_t* work_vars, int64_t* work_slots, char* note, int32_t note_cap) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->planned) return FDOG_ESTATE;
    const Decomposition& d = inst->dec;
    if (local_vars) *local_vars = d.n_local_vars;
    if (work_vars) *work_vars = d.n_work;
    if (work_slots) *work_slots = d.n_work_slots;
    if (jit_shapes) *jit_shapes = static_cast<int32_t>(jit_ids(inst).size());
    const int64_t jt = d.cls_tile_begin[kJitClass + 1] - d.cls_tile_begin[kJitClass];
    if (jit_tiles) *jit_tiles = jt;
    if (static_tiles) *static_tiles = static_cast<int64_t>(d.tiles.size()) - jt;
    if (note && note_cap > 0) {
        const std::string& s = inst->jit_note;
        const size_t n = std::min<size_t>(s.size(), static_cast<size_t>(note_cap - 1));
        std::memcpy(note, s.data(), n);
        note[n] = '\0';
    }
    return FDOG_OK;
}

int fdog_plan_stats(fdog_instance* inst, int32_t* on_device, double* seconds) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->planned) return FDOG_ESTATE;
    if (on_device) *on_device = inst->planned_on_device ? 1 : 0;
    if (seconds) *seconds = inst->plan_seconds;
    return FDOG_OK;
}

int fdog_plan_digest(fdog_instance* inst, uint64_t* digest) {
    if (!inst || !digest) return FDOG_EINVAL;
    if (!inst->planned) return FDOG_ESTATE;
    int rc = ensure_host_plan(inst);
    if (rc != FDOG_OK) return rc;
    const Decomposition& d = inst->dec;
    auto fnv = [](uint64_t h, const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t q = 0; q < n; ++q) { h ^= c[q]; h *= 0x100000001B3ull; }
        return h;
    };
    auto vec = [&](uint64_t h, const auto& v) {
        const uint64_t n = v.size();
        return fnv(fnv(h, &n, sizeof(n)), v.data(), v.size() * sizeof(v[0]));
    };
    auto val = [&](uint64_t h, const auto& x) { return fnv(h, &x, sizeof(x)); };
    const uint64_t h0 = 0xCBF29CE484222325ull;
    uint64_t h = h0;
    h = vec(h, d.fixed);
    h = vec(h, d.outside);
    h = val(val(h, d.const_lb), d.const_obj);
    digest[0] = h;
    h = h0;
    for (size_t s = 0; s < d.shapes.size(); ++s) {
        const HostShape& sh = d.shapes[s];
        h = val(val(h, sh.k), sh.width);
        h = vec(vec(vec(h, sh.lstart), sh.lo), sh.hi);
    }
    h = vec(h, d.shape_cls);
    h = vec(h, d.shape_dev);
    digest[1] = vec(h, d.tpl);
    h = vec(h0, d.tiles);
    h = vec(h, d.cls_tile_begin);
    h = fnv(h, d.kmax, sizeof(d.kmax));
    digest[2] = fnv(h, d.cls_has_local, sizeof(d.cls_has_local));
    digest[3] = vec(h0, d.var);
    digest[4] = vec(vec(h0, d.csr_off), d.csr_pos);
    digest[5] = vec(vec(h0, d.patterns), d.local_ent);
    h = vec(vec(h0, d.work), d.wpos);
    h = fnv(h, d.wb_start, sizeof(d.wb_start));
    digest[6] = fnv(h, d.wb_pos, sizeof(d.wb_pos));
    digest[7] = vec(vec(vec(vec(h0, d.bdd_row), d.bdd_shape), d.bdd_slot0), d.row_bdd);
    h = val(val(val(val(h0, d.n_bdds), d.n_slots), d.n_nodes), d.slots_pad);
    h = val(val(val(h, d.n_local_vars), d.n_work_slots), d.n_work_overflow);
    digest[8] = val(val(val(h, d.n_work), d.n_wpos), d.n_local_ent);
    return FDOG_OK;
}

int fdog_fixed_vars(fdog_instance* inst, int8_t* fixed) {
    if (!inst || !fixed) return FDOG_EINVAL;
    if (!inst->planned) return FDOG_ESTATE;
    std::memcpy(fixed, inst->dec.fixed.data(), inst->dec.fixed.size());
    return FDOG_OK;
}

int fdog_row_bdd(fdog_instance* inst, int32_t row, int32_t* k, int32_t* n_nodes, int32_t* vars, int32_t* lstart,
                 int32_t* lo, int32_t* hi) {
    if (!inst || !k || !n_nodes || row < 0 || row >= inst->n_rows) return FDOG_EINVAL;
    if (!inst->planned) return FDOG_ESTATE;
    int rc = ensure_host_plan(inst);
    if (rc != FDOG_OK) return rc;
    const Decomposition& d = inst->dec;
    const int32_t b = d.row_bdd[row];
    if (b < 0) { *k = 0; *n_nodes = 0; return FDOG_OK; }
    const HostShape& sh = d.shapes[d.bdd_shape[b]];
    *k = sh.k;
    *n_nodes = static_cast<int32_t>(sh.lo.size());
    if (vars)
        for (int t = 0; t < sh.k; ++t) vars[t] = d.var[d.bdd_slot0[b] + static_cast<int64_t>(t) * kTile];
    if (lstart) std::copy(sh.lstart.begin(), sh.lstart.end(), lstart);
    if (lo) std::copy(sh.lo.begin(), sh.lo.end(), lo);
    if (hi) std::copy(sh.hi.begin(), sh.hi.end(), hi);
    return FDOG_OK;
}

int fdog_reset_dual(fdog_instance* inst) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    DeviceGuard g(inst->device);
    int rc = reset_dual_state(inst);
    if (rc != FDOG_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(inst->stream);
    return e == cudaSuccess ? FDOG_OK : fail_cuda(inst, e, "reset");
}

int fdog_transfer_bytes(fdog_instance* inst, int64_t* h2d, int64_t* d2h) {
    if (!inst) return FDOG_EINVAL;
    if (h2d) *h2d = inst->h2d_bytes;
    if (d2h) *d2h = inst->d2h_bytes;
    return FDOG_OK;
}

int fdog_set_profiling(fdog_instance* inst, int32_t on) {
    if (!inst) return FDOG_EINVAL;
    inst->prof.on = on != 0;
    return FDOG_OK;
}

int fdog_profile_read(fdog_instance* inst, int64_t* sweep_launches, double* sweep_ms, int64_t* reduce_launches,
                      double* reduce_ms, int64_t* kernel_launches) {
    if (kernel_launches) *kernel_launches = inst ? inst->prof.launches : 0;
    if (!inst) return FDOG_EINVAL;
    int64_t ns = 0, nr = 0;
    double ms = 0.0, mr = 0.0;
    if (inst->built) {
        DeviceGuard g(inst->device);
        cudaError_t e = cudaStreamSynchronize(inst->stream);
        if (e != cudaSuccess) return fail_cuda(inst, e, "profile");
        inst->prof.drain(ns, ms, nr, mr);
    }
    if (sweep_launches) *sweep_launches = ns;
    if (sweep_ms) *sweep_ms = ms;
    if (reduce_launches) *reduce_launches = nr;
    if (reduce_ms) *reduce_ms = mr;
    return FDOG_OK;
}

int fdog_dual_iterate(fdog_instance* inst, int32_t k, int32_t* iters_done, double* lb) {
    if (!inst || k < 0) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    if (inst->shard) {
        inst->last_error = "a shard of a split instance iterates through fdog_shard_pass";
        return FDOG_ESTATE;
    }
    DeviceGuard g(inst->device);
    InstCtl before;
    int rc = read_ctl(inst, before);
    if (rc != FDOG_OK) return rc;
    if (inst->dec.n_bdds > 0 && k > 0) {
        Engine* e;
        BatchView* v;
        if ((rc = own_engine(inst, &e, &v)) != FDOG_OK) return rc;
        // the instance runs exactly k iterations unless its stopping rule fires
        // first; with the rule on, the status is polled every two graph chunks
        // so that launches stop soon after the device stops iterating
        rc = view_op(*e, *v, kOpLimit, k);
        const int poll = before.stop_enabled ? 2 * std::max(e->chunk, 1) : k;
        for (int left = k; rc == FDOG_OK && left > 0;) {
            const int step = std::min(left, poll);
            rc = view_iterate(*e, *v, step);
            left -= step;
            if (rc == FDOG_OK && left > 0) {
                std::vector<InstStatus> st;
                rc = view_status(*e, *v, st);
                if (rc == FDOG_OK && (st[0].done || st[0].iter >= st[0].iter_limit)) break;
            }
        }
        if (rc != FDOG_OK) {
            inst->last_error = e->err;
            return rc;
        }
    }
    InstCtl after;
    rc = read_ctl(inst, after);
    if (rc != FDOG_OK) return rc;
    const int32_t done = after.iter - before.iter;
    if (done > 0) { inst->pending_T = true; inst->iterated = true; }
    if (iters_done) *iters_done = done;
    if (lb) {
        if (inst->dec.n_bdds == 0) *lb = inst->dec.const_lb;
        else if (inst->iterated) *lb = after.lb_last;
        else return fdog_lower_bound(inst, lb, nullptr);
    }
    return FDOG_OK;
}

int fdog_finalize(fdog_instance* inst) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    DeviceGuard g(inst->device);
    int rc = addback(inst);
    if (rc != FDOG_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(inst->stream);
    return e == cudaSuccess ? FDOG_OK : fail_cuda(inst, e, "finalize");
}

int fdog_lower_bound(fdog_instance* inst, double* lb_running, double* lb_feasible) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    DeviceGuard g(inst->device);
    int rc;
    if (lb_running) {
        if (inst->iterated && inst->dec.n_bdds > 0) {
            InstCtl c;
            if ((rc = read_ctl(inst, c)) != FDOG_OK) return rc;
            *lb_running = c.lb_last;
        } else if ((rc = evaluate(inst, false, lb_running)) != FDOG_OK) {
            return rc;
        }
    }
    if (lb_feasible && (rc = evaluate(inst, inst->pending_T, lb_feasible)) != FDOG_OK) return rc;
    return FDOG_OK;
}

static int slot_table(fdog_instance* inst, int64_t* n_slots, int32_t* var, int32_t* row) {
    const Decomposition& d = inst->dec;
    if (!var) { *n_slots = d.n_slots; return FDOG_OK; }
    if (*n_slots < d.n_slots) return FDOG_EINVAL;
    int rc = ensure_host_plan(inst);
    if (rc != FDOG_OK) return rc;
    int64_t q = 0;
    for (const TileDev& t : d.tiles) {
        const int k = d.shapes[t.shape].k;
        for (int l = 0; l < t.n_valid; ++l)
            for (int layer = 0; layer < k; ++layer) {
                const int64_t p = t.slot_base + static_cast<int64_t>(layer) * kTile + l;
                var[q] = d.var[p];
                if (row) row[q] = d.bdd_row[t.bdd_base + l];
                ++q;
            }
    }
    *n_slots = q;
    return FDOG_OK;
}

static int gather_slots(fdog_instance* inst, const float* dev, float* out) {
    const Decomposition& d = inst->dec;
    std::vector<float> h(d.slots_pad);
    cudaError_t e = copy_async(inst, h.data(), dev, sizeof(float) * d.slots_pad, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaStreamSynchronize(inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "copy slots");
    int64_t q = 0;
    for (const TileDev& t : d.tiles) {
        const int k = d.shapes[t.shape].k;
        for (int l = 0; l < t.n_valid; ++l)
            for (int layer = 0; layer < k; ++layer) out[q++] = h[t.slot_base + static_cast<int64_t>(layer) * kTile + l];
    }
    return FDOG_OK;
}

int fdog_min_marginals(fdog_instance* inst, int64_t* n_slots, int32_t* var, int32_t* row, float* m0, float* m1) {
    if (!inst || !n_slots) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    if (!var) return slot_table(inst, n_slots, nullptr, nullptr);
    if (*n_slots < inst->dec.n_slots) return FDOG_EINVAL;
    DeviceGuard g(inst->device);
    int rc = ensure_mm1(inst);
    if (rc != FDOG_OK) return rc;
    if (inst->dec.n_bdds > 0) {
        cudaError_t e = launch_sweep(inst->batch, kMinMarg, kMMBoth, inst->cfg, inst->stream);
        if (e != cudaSuccess) return fail_cuda(inst, e, "min-marginals");
    }
    if ((rc = slot_table(inst, n_slots, var, row)) != FDOG_OK) return rc;
    if (m0 && (rc = gather_slots(inst, inst->dev.mm0, m0)) != FDOG_OK) return rc;
    if (m1 && (rc = gather_slots(inst, inst->dev.mm1, m1)) != FDOG_OK) return rc;
    return FDOG_OK;
}

int fdog_multipliers(fdog_instance* inst, int64_t* n_slots, int32_t* var, int32_t* row, float* lambda) {
    if (!inst || !n_slots) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    if (!var) return slot_table(inst, n_slots, nullptr, nullptr);
    if (*n_slots < inst->dec.n_slots) return FDOG_EINVAL;
    DeviceGuard g(inst->device);
    int rc = slot_table(inst, n_slots, var, row);
    if (rc == FDOG_OK && lambda) rc = gather_slots(inst, inst->dev.lam, lambda);
    return rc;
}

int fdog_primal_round(fdog_instance* inst, int32_t* rounds_used) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    if (inst->shard) {
        inst->last_error = "rounding a split instance needs every shard's min-marginals";
        return FDOG_EUNSUPPORTED;
    }
    DeviceGuard g(inst->device);
    Engine* e;
    BatchView* v;
    int rc = own_engine(inst, &e, &v);
    if (rc != FDOG_OK) return rc;
    std::vector<int> rounds, status;
    rc = engine_round(*e, {inst}, &rounds, &status);
    if (rc != FDOG_OK) {
        inst->last_error = e->err;
        return rc;
    }
    inst->iterated = false;  // the running bound of the perturbed problem is not an ILP bound
    inst->pending_T = false;
    if (rounds_used) *rounds_used = rounds[0];
    return status[0];
}

int fdog_solution(fdog_instance* inst, uint8_t* x, double* objective, int32_t* feasible) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->has_solution) return FDOG_ESTATE;
    if (x) std::memcpy(x, inst->solution_pinned ? inst->host_x : inst->solution.data(), static_cast<size_t>(inst->n_vars));
    if (objective) *objective = inst->objective;
    if (feasible) *feasible = inst->feasible;
    return FDOG_OK;
}

int fdog_info(fdog_instance* inst, int64_t* n_vars, int64_t* n_bdds, int64_t* n_slots, int64_t* n_nodes,
              int64_t* device_bytes) {
    if (!inst) return FDOG_EINVAL;
    if (n_vars) *n_vars = inst->n_vars;
    if (!inst->planned) {
        if (n_bdds || n_slots || n_nodes || device_bytes) return FDOG_ESTATE;
        return FDOG_OK;
    }
    if (n_bdds) *n_bdds = inst->dec.n_bdds;
    if (n_slots) *n_slots = inst->dec.n_slots;
    if (n_nodes) *n_nodes = inst->dec.n_nodes;
    if (device_bytes)
        *device_bytes = static_cast<int64_t>(inst->built ? inst->arena_bytes : arena_size(inst)) +
                        (inst->dev.mm1 ? static_cast<int64_t>(sizeof(float) * inst->dec.slots_pad) : 0);
    return FDOG_OK;
}

int fdog_release(fdog_instance* inst) {
    if (!inst) return FDOG_EINVAL;
    return release_device(inst);
}

void fdog_destroy(fdog_instance* inst) {
    if (!inst) return;
    const Decomposition& d = inst->dec;
    const bool device_plan = d.d_var || d.d_csr_off || d.d_csr_pos || d.d_work || d.d_wpos || d.d_local_ent ||
                             d.d_bdd_row;
    if (inst->built || inst->arena || inst->host_ctl || device_plan) {
        DeviceGuard g(inst->device);
        if (inst->stream || inst->arena) cudaStreamSynchronize(inst->stream);
        if (device_plan) {
            free_device_plan(inst->dec, inst->stream);
            cudaStreamSynchronize(inst->stream);
        }
        if (inst->arena) cudaFree(inst->arena);
        if (inst->dev.mm1) cudaFree(inst->dev.mm1);
        if (inst->host_ctl) cudaFreeHost(inst->host_ctl);
        if (inst->host_x) cudaFreeHost(inst->host_x);
        delete inst->self_view;
        delete inst->engine;
        inst->prof.release();
        cudaGetLastError();
    }
    delete inst;
}

}  // extern "C"
