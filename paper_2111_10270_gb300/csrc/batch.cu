// Ragged batching of instances (fdog_batch_*): the members' tiles and
// variables form one flat index space, every launch covers all members, and
// each member moves through Alg. 1 and Alg. 2 on its own schedule.
#include <cuda_runtime.h>

#include <new>
#include <string>
#include <vector>

#include "engine.h"

struct fdog_batch {
    std::vector<fdog_instance*> members;
    fdog::Engine engine;
    fdog::Profiler prof;  // launch counting for the batch's kernels
    int device = 0;
    std::string last_error;
};

using namespace fdog;

extern "C" {

int fdog_batch_create(fdog_instance* const* insts, int32_t n, void* cuda_stream, fdog_batch** out) {
    if (!out || !insts || n <= 0) return FDOG_EINVAL;
    *out = nullptr;
    const int dev = insts[0] ? insts[0]->device : -1;
    for (int32_t i = 0; i < n; ++i) {
        if (!insts[i]) return FDOG_EINVAL;
        if (!insts[i]->built) return FDOG_ESTATE;
        if (insts[i]->device != dev) return FDOG_EINVAL;
        for (int32_t j = 0; j < i; ++j)
            if (insts[j] == insts[i]) return FDOG_EINVAL;  // an instance may appear once
        if (n > 1 && insts[i]->params.update == 1) return FDOG_EUNSUPPORTED;  // the serial update runs alone
        if (insts[i]->shard) return FDOG_EUNSUPPORTED;  // a shard's passes wait on the other shards
    }
    fdog_batch* b = new (std::nothrow) fdog_batch();
    if (!b) return FDOG_ENOMEM;
    b->members.assign(insts, insts + n);
    b->device = dev;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    Engine& e = b->engine;
    e.device = dev;
    e.stream = static_cast<cudaStream_t>(cuda_stream);
    e.cfg = insts[0]->cfg;
    e.cfg.prof = &b->prof;
    e.prof = nullptr;
    engine_use_side(e);
    int rc = FDOG_OK;
    // members may have been built on other streams: their uploads must be complete
    for (fdog_instance* m : b->members)
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) { cudaGetLastError(); rc = FDOG_ECUDA; }
    if (rc == FDOG_OK && insts[0]->params.block_threads == 0) {
        BatchView v;
        rc = view_build(e, v, b->members);
        if (rc == FDOG_OK) rc = view_autotune(e, v, insts[0]->params.grid_waves == 0);
    }
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (rc != FDOG_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return FDOG_OK;
}

int fdog_batch_solve(fdog_batch* b, int32_t max_iters, int32_t* iters, int32_t* rounds, int32_t* status) {
    if (!b || max_iters < 0) return FDOG_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    std::vector<int> it, rd, st;
    int rc = engine_solve(b->engine, b->members, max_iters, &it, &rd, &st);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    if (rc != FDOG_OK) {
        b->last_error = b->engine.err;
        return rc;
    }
    for (size_t i = 0; i < b->members.size(); ++i) {
        b->members[i]->iterated = false;
        b->members[i]->pending_T = false;
        if (iters) iters[i] = it[i];
        if (rounds) rounds[i] = rd[i];
        if (status) status[i] = st[i];
    }
    return FDOG_OK;
}

int fdog_batch_set_persistent(fdog_batch* b, int32_t on, double barrier_wait_s) {
    if (!b || (on != 0 && on != 1) || barrier_wait_s < 0.0) return FDOG_EINVAL;
    if (on) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (prev != b->device) cudaSetDevice(b->device);
        BatchView v;
        int rc = view_build(b->engine, v, b->members);
        const bool ok = rc == FDOG_OK && persist_supported(v.b);
        if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
        if (rc != FDOG_OK) {
            b->last_error = b->engine.err;
            return rc;
        }
        if (!ok) {
            b->last_error = "the persistent kernel takes batches whose BDDs all have width <= 2 on the generic "
                            "kernels (params.jit = -1)";
            return FDOG_EUNSUPPORTED;
        }
    }
    b->engine.persistent = on != 0;
    b->engine.persist_wait_s = barrier_wait_s > 0.0 ? barrier_wait_s : 1.0;
    return FDOG_OK;
}

int fdog_batch_info(fdog_batch* b, int32_t* warps_per_block, int32_t* chunk, int64_t* kernel_launches) {
    if (!b) return FDOG_EINVAL;
    if (warps_per_block) *warps_per_block = b->engine.cfg.warps_per_block;
    if (chunk) *chunk = b->engine.chunk;
    if (kernel_launches) *kernel_launches = b->prof.launches;
    return FDOG_OK;
}

const char* fdog_batch_last_error(const fdog_batch* b) { return b ? b->last_error.c_str() : ""; }

void fdog_batch_destroy(fdog_batch* b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    if (b->engine.stream) cudaStreamSynchronize(b->engine.stream);
    const int dev = b->device;
    delete b;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    cudaGetLastError();
}

}  // extern "C"
