// Device code of the deferred sums and the lower-bound reduction, shared by
// the per-pass kernels (kernels.cu) and the persistent iteration kernel
// (persist.cu), so both run the same operations in the same order.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "sweep.cuh"

namespace fdog {
namespace dev {

struct FlatArgs {
    const InstDev* insts;
    const int32_t* prefix;
    int32_t n_inst;
    int32_t total;
};

// T_i = (C_i - sum_j lambda^j_i) / |J_i|.  Right after a pass, Prop. 1 gives
// sum_j lambda^j_i + omega sum_j M_ij = C_i, so T_i equals the averaged
// deferred term omega / |J_i| sum_k Mbar_ik of Eq. 5.
// One thread per listed variable with at most 8 copies (no grid-stride loop:
// the block scheduler keeps every warp slot busy); its slot positions come
// from the bucket of its copy count, one coalesced column per copy, so all of
// its multiplier gathers are issued together.
// one listed variable with at most 8 copies (work index g of the flat batch).
// Instances whose stopping rule or iteration limit has stopped them are left
// alone.  Without SNAPSHOT the test reads the control block and work index 0
// of each instance records its outcome in InstCtl::pass_active; with SNAPSHOT
// it reads that record instead of the control block's live state, which the
// end-of-iteration kernel's commit may change while this runs.
template <bool SNAPSHOT = false>
__device__ __forceinline__ void reduce_T_one(const FlatArgs& a, int g) {
    const int ii = find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    const int w = g - __ldg(a.prefix + ii);  // below wb_start[FDOG_WBUCKETS - 1]: at most 8 copies
    if (SNAPSHOT) {
        if (!I->ctl->pass_active) return;
    } else {
        const bool inactive = FDOG_INACTIVE(I->ctl);
        if (w == 0) I->ctl->pass_active = inactive ? 0 : 1;
        if (inactive) return;
    }
    const int i = __ldcs(I->work + w);  // a variable with copies in several tiles (list streamed once)
    int b = 0;
#pragma unroll
    for (int q = 1; q < FDOG_WBUCKETS - 1; ++q) b += w >= I->wb_start[q];
    // bucket of b + 1 copies: positions column by column, all loads independent;
    // copies summed in ascending slot order (as in csr_pos), a fixed order
    const int cnt = b + 1;
    const int nb = I->wb_start[b + 1] - I->wb_start[b];
    const int32_t* __restrict__ pos = I->wpos + I->wb_pos[b] + (w - I->wb_start[b]);
    const float* __restrict__ lam = I->lam;
    float l[FDOG_WBUCKETS - 1];
#pragma unroll
    for (int q = 0; q < FDOG_WBUCKETS - 1; ++q) l[q] = q < cnt ? lam[__ldcs(pos + q * nb)] : 0.f;
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < FDOG_WBUCKETS - 1; ++q)
        if (q < cnt) s += l[q];
    I->T[i] = (I->C[i] - s) * dev::inv_copies(cnt);
}


__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
}

struct LbArgs {
    const InstDev* insts;
    const int32_t* prefix;
    int32_t n_inst;
    int32_t target;
};

// (s, c) <- (s, c) + (x, y) for Neumaier pairs
__device__ __forceinline__ void neumaier_pair(double& s, double& c, double x, double y) {
    neumaier(s, c, x);
    c += y;
}

// (s, c) <- (s, c) + (x, y) for compensated FP32 pairs (TwoSum of the sums)
__device__ __forceinline__ void pair_add_f(float& s, float& c, float x, float y) {
    const float t = s + x;
    const float bp = t - s;
    const float e = (s - (t - bp)) + (x - bp);
    s = t;
    c = c + y + e;
}

// the same fixed-order block reduction for compensated FP32 pairs
__device__ __forceinline__ void block_pair_reduce_f(float* ss, float* sc, float& s, float& c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, s, off);
        const float oc = __shfl_xor_sync(0xffffffffu, c, off);
        pair_add_f(s, c, os, oc);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < 8 ? ss[threadIdx.x] : 0.f;
        c = threadIdx.x < 8 ? sc[threadIdx.x] : 0.f;
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, s, off);
            const float oc = __shfl_xor_sync(0xffffffffu, c, off);
            pair_add_f(s, c, os, oc);
        }
    }
}

// block-wide fixed-order reduction of one Neumaier pair per thread
// (blockDim.x == 256): butterfly within each warp, then warp 0 combines the
// eight warp results.  Every thread of warp 0 ends with the block total.
__device__ __forceinline__ void block_pair_reduce(double* ss, double* sc, double& s, double& c) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, s, off);
        const double oc = __shfl_xor_sync(0xffffffffu, c, off);
        neumaier_pair(s, c, os, oc);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = s;
        sc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < 8 ? ss[threadIdx.x] : 0.0;
        c = threadIdx.x < 8 ? sc[threadIdx.x] : 0.0;
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            const double os = __shfl_xor_sync(0xffffffffu, s, off);
            const double oc = __shfl_xor_sync(0xffffffffu, c, off);
            neumaier_pair(s, c, os, oc);
        }
    }
}

// bound of a finished iteration: ring, counter, stopping test (Alg. 1 text)
__device__ __forceinline__ void commit_iteration(InstCtl* ctl, double lb) {
    const int it = ctl->iter;
    ctl->lb_ring[it % kLbRing] = lb;
    ctl->lb_last = lb;
    ctl->iter = it + 1;
    const int since = ++ctl->since_reset;
    if (ctl->stop_enabled && since >= ctl->min_iters && since > ctl->window) {
        const double prev = ctl->lb_ring[(it - ctl->window) % kLbRing];
        if (lb - prev <= ctl->tol * fmax(fabs(lb), 1.0)) ctl->done = 1;
    }
}

// Variables with more than 8 copies (one assignment variable of a matching
// problem can sit in hundreds of rows): one warp per variable g, lane l
// summing copies l, l + 32, ... in ascending order, then a fixed butterfly.
// SNAPSHOT as in reduce_T_one (the first such variable of an instance records
// the activity when it is off).
template <bool SNAPSHOT = false>
__device__ __forceinline__ void reduce_T_wide_one(const FlatArgs& a, int g, int lane) {
    const int ii = find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    const int w = g - __ldg(a.prefix + ii);
    if (SNAPSHOT) {
        if (!I->ctl->pass_active) return;
    } else {
        const bool inactive = FDOG_INACTIVE(I->ctl);
        if (w == 0 && lane == 0) I->ctl->pass_active = inactive ? 0 : 1;
        if (inactive) return;
    }
    const int i = __ldcs(I->work + I->wb_start[FDOG_WBUCKETS - 1] + w);
    const int b = I->csr_off[i], cnt = I->csr_off[i + 1] - b;
    const int32_t* __restrict__ pos = I->csr_pos + b;
    const float* __restrict__ lam = I->lam;
    float s = 0.f;
    for (int q = lane; q < cnt; q += 32) s += lam[__ldcs(pos + q)];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) I->T[i] = (I->C[i] - s) * __frcp_rn(static_cast<float>(cnt));  // 1 / cnt rounded to FP32
}

// Bound of one chunk of kLbChunk tiles (thread t takes tile t of the chunk):
// the tiles' partials reduced as compensated FP32 pairs (FP64 is a small
// fraction of the FP32 rate here), exact in FP64 afterwards.  Every thread of
// the block calls it; the value is valid in thread 0.
__device__ __forceinline__ double lb_chunk(const InstDev* __restrict__ I, int c, float* ssf, float* scf) {
    const int t = c * kLbChunk + threadIdx.x;
    float2 p = t < I->n_tiles ? I->tile_lb[t] : make_float2(0.f, 0.f);
    block_pair_reduce_f(ssf, scf, p.x, p.y);
    return static_cast<double>(p.x) + static_cast<double>(p.y);
}

// Bound of one instance from its chunk values: thread-strided Neumaier sums,
// a fixed-order block reduction, then the presolve constant.  Every thread of
// the block calls it; the value is valid in thread 0.
__device__ __forceinline__ double lb_total(const InstDev* __restrict__ I, double* ss, double* sc) {
    double s = 0.0, cp = 0.0;
    for (int q = threadIdx.x; q < I->n_chunks; q += blockDim.x) neumaier(s, cp, __ldcg(I->chunk_lb + q));
    block_pair_reduce(ss, sc, s, cp);
    double S = s, Cc = cp;
    neumaier(S, Cc, I->const_lb);
    return S + Cc;
}

}  // namespace dev
}  // namespace fdog
