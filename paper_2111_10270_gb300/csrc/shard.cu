// One instance split over several GPUs (the paper's conclusion names
// multi-GPU support as future work).
//
// Within one pass of Alg. 1 the BDDs are independent: every update of Eq. 5
// reads only the BDD's own multipliers and the deferred terms T_i fixed by the
// previous pass.  The only coupling between BDDs is T_i itself, which needs
// sum_j lambda^j_i over all copies of variable i (Prop. 1: right after a pass
// T_i = (c_i - sum_j lambda^j_i) / |J_i| = omega / |J_i| sum_k Mbar_ik).  So the
// rows are split into shards, each an ordinary instance of its own rows on
// its own GPU, and once per pass the shards exchange, for the variables whose
// copies lie in several shards, their partial sums of lambda (an all-reduce
// of one float per shared variable), plus one double per iteration for the
// lower bound.  Everything else stays local.  The exchange itself is the
// caller's (NCCL, or any all-reduce): these calls only produce and consume the
// per-shard sums, so the library stays one process on one GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "instance.h"
#include "kernels.h"

using namespace fdog;

namespace {

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~Guard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

struct ShardArgs {
    const InstDev* I;
    const int32_t* vars;    // shared variables with copies in this shard, ascending
    const int32_t* copies;  // their copy counts over all shards
    const int32_t* slot;    // their index in the exchange buffer (rank among all shared variables)
    int32_t n;
    float* sums;            // exchange buffer: partial sums out (pass) / sums over all shards in (apply)
};

// Alg. 1 initialisation for the shared variables: lambda^j_i = c_i / |J_i|
// with |J_i| counted over all shards, on every local copy.
__global__ void __launch_bounds__(256) shard_init_kernel(ShardArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
        const InstDev* __restrict__ I = a.I;
        const int i = a.vars[k];
        const float l = I->C[i] / static_cast<float>(a.copies[k]);
        for (int q = I->csr_off[i]; q < I->csr_off[i + 1]; ++q) I->lam[I->csr_pos[q]] = l;
    }
}

// After a pass: this shard's part of sum_j lambda^j_i, copies in ascending slot order.
__global__ void __launch_bounds__(256) shard_partial_kernel(ShardArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
        const InstDev* __restrict__ I = a.I;
        const int i = a.vars[k];
        float s = 0.f;
        for (int q = I->csr_off[i]; q < I->csr_off[i + 1]; ++q) s += I->lam[I->csr_pos[q]];
        a.sums[a.slot[k]] = s;
    }
}

// With the sums over all shards: T_i = (C_i - sum_j lambda^j_i) times 1 / |J_i|
// rounded to FP32, the deferred term of Eq. 5 as the other kernels form it.
__global__ void __launch_bounds__(256) shard_apply_kernel(ShardArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n; k += gridDim.x * blockDim.x) {
        const InstDev* __restrict__ I = a.I;
        const int i = a.vars[k];
        I->T[i] = (I->C[i] - a.sums[a.slot[k]]) * __frcp_rn(static_cast<float>(a.copies[k]));
    }
}

// the bound of the whole instance for this iteration, to be committed
__global__ void shard_stage_kernel(InstCtl* ctl, double lb) {
    ctl->lb_staged = lb;
    ctl->staged = 1;
}

ShardArgs shard_args(fdog_instance* inst, float* sums) {
    return ShardArgs{inst->dev.inst, inst->dev.sh_vars, inst->dev.sh_copies, inst->dev.sh_slot,
                     static_cast<int32_t>(inst->dec.shared_vars.size()), sums};
}

// length of the exchange buffer: every shared variable of the split instance
int32_t exchange_len(const fdog_instance* inst) {
    int32_t n = 0;
    for (uint8_t f : inst->shard_shared) n += f;
    return n;
}

int blocks_for(int n) { return n <= 0 ? 1 : std::min((n + 255) / 256, 152 * 8); }

int shard_ready(fdog_instance* inst) {
    if (!inst) return FDOG_EINVAL;
    if (!inst->shard) {
        inst->last_error = "not a shard (fdog_shard_setup)";
        return FDOG_ESTATE;
    }
    if (!inst->built) return FDOG_ESTATE;
    return FDOG_OK;
}

}  // namespace

namespace fdog {

int shard_check_copies(fdog_instance* inst) {
    const Decomposition& d = inst->dec;
    for (int32_t i = 0; i < inst->n_vars; ++i) {
        const int32_t local = d.csr_off[i + 1] - d.csr_off[i];
        const int32_t all = inst->shard_copies[i];
        if (inst->shard_shared[i] ? (local > all) : (local > 0 && local != all)) {
            inst->last_error = "variable " + std::to_string(i) + " has " + std::to_string(local) +
                               " copies in this shard and " + std::to_string(all) + " over all shards";
            return FDOG_EINVAL;
        }
    }
    return FDOG_OK;
}

cudaError_t launch_shard_init(fdog_instance* inst) {
    const ShardArgs a = shard_args(inst, nullptr);
    if (a.n == 0) return cudaSuccess;
    inst->cfg.count();
    shard_init_kernel<<<blocks_for(a.n), 256, 0, inst->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace fdog

extern "C" {

int fdog_shard_plan(int32_t n_vars, int32_t n_rows, const int64_t* row_ptr, const int32_t* col, const int32_t* coef,
                    int32_t n_shards, int32_t* row_shard, int32_t* copies, uint8_t* shared) {
    if (n_vars < 0 || n_rows < 0 || n_shards < 1 || !row_ptr || !row_shard || !copies || !shared) return FDOG_EINVAL;
    if (row_ptr[0] != 0) return FDOG_EINVAL;
    for (int32_t j = 0; j < n_rows; ++j)
        if (row_ptr[j + 1] < row_ptr[j]) return FDOG_EINVAL;
    const int64_t nnz = row_ptr[n_rows];
    if (nnz > 0 && !col) return FDOG_EINVAL;
    for (int64_t q = 0; q < nnz; ++q)
        if (col[q] < 0 || col[q] >= n_vars) return FDOG_EINVAL;
    // Rows in the order of their smallest variable (ties by row index), cut
    // into contiguous blocks of that order with about equal numbers of
    // non-zero entries: a row goes to the shard that holds the midpoint of its
    // entries.  Rows over nearby variables (a grid node's rows, a frame's
    // rows) land in one shard, so the shards share few variables when the
    // variables are numbered by locality.
    std::vector<int32_t> key(static_cast<size_t>(n_rows)), order(static_cast<size_t>(n_rows));
    std::vector<int64_t> len(static_cast<size_t>(n_rows));
    for (int32_t j = 0; j < n_rows; ++j) {
        int32_t k = n_vars;
        int64_t c = 0;
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q)
            if (!coef || coef[q] != 0) {
                k = std::min(k, col[q]);
                ++c;
            }
        key[j] = k;
        len[j] = c;
        order[j] = j;
    }
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    int64_t total = 0;
    for (int32_t j = 0; j < n_rows; ++j) total += len[j];
    int64_t before = 0;
    for (int32_t r = 0; r < n_rows; ++r) {
        const int32_t j = order[r];
        int64_t s = total > 0 ? (2 * before + len[j]) * n_shards / (2 * total)
                              : static_cast<int64_t>(r) * n_shards / std::max(n_rows, 1);
        row_shard[j] = static_cast<int32_t>(std::min<int64_t>(s, n_shards - 1));
        before += len[j];
    }
    std::vector<int32_t> first(static_cast<size_t>(n_vars), -1);
    for (int32_t i = 0; i < n_vars; ++i) {
        copies[i] = 0;
        shared[i] = 0;
    }
    for (int32_t j = 0; j < n_rows; ++j)
        for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) {
            if (coef && coef[q] == 0) continue;
            const int32_t i = col[q];
            ++copies[i];
            if (first[i] < 0) first[i] = row_shard[j];
            else if (first[i] != row_shard[j]) shared[i] = 1;
        }
    return FDOG_OK;
}

int fdog_shard_setup(fdog_instance* inst, const uint8_t* shared, const int32_t* copies) {
    if (!inst || !shared || !copies) return FDOG_EINVAL;
    if (inst->planned || inst->built) return FDOG_ESTATE;
    if (inst->params.update != 0) {
        inst->last_error = "a shard runs the parallel update of Alg. 1 (update = 0)";
        return FDOG_EUNSUPPORTED;
    }
    for (int32_t i = 0; i < inst->n_vars; ++i)
        if (shared[i] > 1 || copies[i] < 0) return FDOG_EINVAL;
    inst->shard_shared.assign(shared, shared + inst->n_vars);
    inst->shard_copies.assign(copies, copies + inst->n_vars);
    inst->shard = true;
    return FDOG_OK;
}

int fdog_shard_info(fdog_instance* inst, int32_t* n_shared) {
    if (!inst || !n_shared) return FDOG_EINVAL;
    if (!inst->shard) return FDOG_ESTATE;
    if (!inst->planned) {
        int rc = fdog::plan(inst);
        if (rc != FDOG_OK) return rc;
    }
    *n_shared = exchange_len(inst);
    return FDOG_OK;
}

int fdog_shard_pass(fdog_instance* inst, int32_t descending, float* dev_sums) {
    int rc = shard_ready(inst);
    if (rc != FDOG_OK) return rc;
    const ShardArgs a = shard_args(inst, dev_sums);
    const int32_t n_ex = exchange_len(inst);
    if ((descending != 0 && descending != 1) || (n_ex > 0 && !dev_sums)) return FDOG_EINVAL;
    Guard g(inst->device);
    const DevBatch& b = inst->batch;
    cudaError_t e = cudaSuccess;
    // shared variables this shard does not hold contribute 0 to the sums
    if (n_ex > 0) e = cudaMemsetAsync(dev_sums, 0, sizeof(float) * n_ex, inst->stream);
    if (e == cudaSuccess && inst->dec.n_bdds > 0) {
        e = launch_sweep(b, descending ? kBwdUpdate : kFwdUpdate, 0, inst->cfg, inst->stream);
        if (e == cudaSuccess) e = launch_reduce_T(b, inst->cfg, inst->stream);
        if (e == cudaSuccess && a.n > 0) {
            inst->cfg.count();
            shard_partial_kernel<<<blocks_for(a.n), 256, 0, inst->stream>>>(a);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && descending) e = launch_lb_reduce(b, kLbStage, inst->cfg, inst->stream);
    } else if (e == cudaSuccess && descending) {
        // no BDD in this shard: its part of the bound is its presolve constant alone
        inst->cfg.count();
        shard_stage_kernel<<<1, 1, 0, inst->stream>>>(inst->dev.ctl, inst->dec.const_lb);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail_cuda(inst, e, "shard pass");
    inst->pending_T = true;
    inst->iterated = true;
    return FDOG_OK;
}

int fdog_shard_apply(fdog_instance* inst, const float* dev_sums) {
    int rc = shard_ready(inst);
    if (rc != FDOG_OK) return rc;
    const ShardArgs a = shard_args(inst, const_cast<float*>(dev_sums));
    if (exchange_len(inst) > 0 && !dev_sums) return FDOG_EINVAL;
    if (a.n == 0) return FDOG_OK;
    Guard g(inst->device);
    inst->cfg.count();
    shard_apply_kernel<<<blocks_for(a.n), 256, 0, inst->stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FDOG_OK : fail_cuda(inst, e, "shard apply");
}

int fdog_shard_bound(fdog_instance* inst, double* lb_part) {
    int rc = shard_ready(inst);
    if (rc != FDOG_OK) return rc;
    if (!lb_part) return FDOG_EINVAL;
    Guard g(inst->device);
    InstCtl c;
    if ((rc = read_ctl(inst, c)) != FDOG_OK) return rc;
    if (!c.staged) {
        inst->last_error = "no descending pass since the last commit";
        return FDOG_ESTATE;
    }
    *lb_part = c.lb_staged;
    return FDOG_OK;
}

int fdog_shard_commit(fdog_instance* inst, double lb, int32_t* stop) {
    int rc = shard_ready(inst);
    if (rc != FDOG_OK) return rc;
    Guard g(inst->device);
    inst->cfg.count();
    shard_stage_kernel<<<1, 1, 0, inst->stream>>>(inst->dev.ctl, lb);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_lb_commit(inst->batch, inst->cfg, inst->stream);
    if (e != cudaSuccess) return fail_cuda(inst, e, "shard commit");
    InstCtl c;
    if ((rc = read_ctl(inst, c)) != FDOG_OK) return rc;
    if (stop) *stop = c.done;
    return FDOG_OK;
}

}  // extern "C"
