// Checkpoint / resume of the dual state (fdog_export_state, fdog_import_state).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "instance.h"

using namespace fdog;

namespace {

constexpr char kMagic[8] = {'F', 'D', 'O', 'G', 'S', 'T', '0', '1'};

struct StateHeader {
    char magic[8];
    uint32_t version;
    uint32_t flags;  // bit 0: deferred differences pending, bit 1: iterated since the last add-back
    int64_t n_vars;
    int64_t slots_pad;
    int64_t n_tiles;
    uint64_t layout_hash;
    double omega;
};

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t q = 0; q < n; ++q) { h ^= c[q]; h *= 0x100000001B3ull; }
    return h;
}

uint64_t layout_hash(const fdog_instance* inst) {
    uint64_t h = 0xCBF29CE484222325ull;
    h = fnv1a(h, inst->dec.var.data(), inst->dec.var.size() * sizeof(int32_t));
    h = fnv1a(h, inst->dec.tiles.data(), inst->dec.tiles.size() * sizeof(TileDev));
    h = fnv1a(h, inst->dec.tpl.data(), inst->dec.tpl.size() * sizeof(uint16_t));
    return h;
}

size_t state_bytes(const fdog_instance* inst) {
    return sizeof(StateHeader) + sizeof(float) * (inst->dec.slots_pad + 2 * static_cast<size_t>(inst->n_vars)) +
           sizeof(InstCtl);
}

}  // namespace

extern "C" {

int fdog_export_state(fdog_instance* inst, void* buf, size_t* bytes) {
    if (!inst || !bytes) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    const size_t need = state_bytes(inst);
    if (!buf) { *bytes = need; return FDOG_OK; }
    if (*bytes < need) return FDOG_EINVAL;
    int rc = ensure_host_plan(inst);  // the layout fingerprint reads the slot table
    if (rc != FDOG_OK) return rc;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != inst->device) cudaSetDevice(inst->device);
    StateHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.flags = (inst->pending_T ? 1u : 0u) | (inst->iterated ? 2u : 0u);
    h.n_vars = inst->n_vars;
    h.slots_pad = inst->dec.slots_pad;
    h.n_tiles = static_cast<int64_t>(inst->dec.tiles.size());
    h.layout_hash = layout_hash(inst);
    h.omega = inst->params.omega;
    char* out = static_cast<char*>(buf);
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    cudaStream_t s = inst->stream;
    cudaError_t e = copy_async(inst, out + off, inst->dev.lam, sizeof(float) * h.slots_pad, cudaMemcpyDeviceToHost);
    off += sizeof(float) * h.slots_pad;
    if (e == cudaSuccess) e = copy_async(inst, out + off, inst->dev.T, sizeof(float) * h.n_vars, cudaMemcpyDeviceToHost);
    off += sizeof(float) * h.n_vars;
    if (e == cudaSuccess) e = copy_async(inst, out + off, inst->dev.C, sizeof(float) * h.n_vars, cudaMemcpyDeviceToHost);
    off += sizeof(float) * h.n_vars;
    if (e == cudaSuccess) e = copy_async(inst, out + off, inst->dev.ctl, sizeof(InstCtl), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (prev >= 0 && prev != inst->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail_cuda(inst, e, "export state");
    *bytes = need;
    return FDOG_OK;
}

int fdog_import_state(fdog_instance* inst, const void* buf, size_t bytes) {
    if (!inst || !buf) return FDOG_EINVAL;
    if (!inst->built) return FDOG_ESTATE;
    if (bytes != state_bytes(inst)) return FDOG_EINVAL;
    int rc = ensure_host_plan(inst);
    if (rc != FDOG_OK) return rc;
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 || h.n_vars != inst->n_vars ||
        h.slots_pad != inst->dec.slots_pad || h.n_tiles != static_cast<int64_t>(inst->dec.tiles.size()) ||
        h.layout_hash != layout_hash(inst) || h.omega != inst->params.omega) {
        inst->last_error = "state does not belong to this instance";
        return FDOG_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != inst->device) cudaSetDevice(inst->device);
    const char* in = static_cast<const char*>(buf) + sizeof(h);
    cudaStream_t s = inst->stream;
    cudaError_t e = copy_async(inst, inst->dev.lam, in, sizeof(float) * h.slots_pad, cudaMemcpyHostToDevice);
    in += sizeof(float) * h.slots_pad;
    if (e == cudaSuccess) e = copy_async(inst, inst->dev.T, in, sizeof(float) * h.n_vars, cudaMemcpyHostToDevice);
    in += sizeof(float) * h.n_vars;
    if (e == cudaSuccess) e = copy_async(inst, inst->dev.C, in, sizeof(float) * h.n_vars, cudaMemcpyHostToDevice);
    in += sizeof(float) * h.n_vars;
    if (e == cudaSuccess) e = copy_async(inst, inst->dev.ctl, in, sizeof(InstCtl), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (prev >= 0 && prev != inst->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail_cuda(inst, e, "import state");
    inst->pending_T = (h.flags & 1u) != 0;
    inst->iterated = (h.flags & 2u) != 0;
    return FDOG_OK;
}

const char* fdog_last_error(const fdog_instance* inst) { return inst ? inst->last_error.c_str() : ""; }

}  // extern "C"
