// FP64 evaluation of the lower bound sum_j E^j(lambda^j) (Eq. D, Prop. 1).
//
// The update sweeps keep the multipliers and every shortest-path label in
// FP32; the bound they report per iteration is summed from FP32 per-BDD
// energies.  The bound a caller reads at a given state (fdog_lower_bound)
// is instead evaluated here with FP64 labels from the same FP32 multipliers,
// so that the only FP32 error left in it is that of the multipliers
// themselves, which cannot make the bound invalid (any lambda with
// sum_j lambda^j_i = c_i gives a valid bound).
//
// One block of 256 threads per chunk of kLbChunk tiles (the chunking of the
// iteration bound): warp w visits tiles w, w + 8, ... of its chunk, lane l
// walks BDD l of the tile from its last layer to its root (backward labels,
// Alg. 4 without updates), each thread accumulates its energies with
// Neumaier, the block reduces in a fixed order, and the last block of an
// instance sums the chunk totals and the presolve constant.  The order is
// fixed, so the result is deterministic and equal alone or in a batch.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "sweep.cuh"

namespace fdog {
namespace {

using dev::find_inst;
using dev::load_codes;

__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000ll); }

__device__ __forceinline__ void neumaier64(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
}

// label of the successor with the given code: a node of the next layer, TOP (0) or BOT (inf)
template <int W>
__device__ __forceinline__ double pick64(const double (&x)[W], uint32_t code) {
    double r = (code == kCodeTop) ? 0.0 : dinf();
#pragma unroll
    for (int w = 0; w < W; ++w) r = (code == static_cast<uint32_t>(w)) ? x[w] : r;
    return r;
}

// E^j of the BDD in `lane` of a tile: SP(root, TOP) with arcs leaving layer t
// costing lambda_t on the 1-arc and 0 on the 0-arc (Def. 4, Fig. 3).  With
// add_t the multiplier of a slot is first formed as the FP32 sum lambda + T,
// exactly as the add-back (Alg. 1, last loop) stores it.
template <int W>
__device__ double bdd_energy64(const InstDev* __restrict__ I, const TileDev& tile, const ShapeDev& sh, int lane,
                               bool add_t) {
    const uint16_t* __restrict__ tpl = I->tpl + sh.tpl_off;
    const size_t base = static_cast<size_t>(tile.slot_base) + lane;
    double nx[W];
#pragma unroll
    for (int v = 0; v < W; ++v) nx[v] = dinf();
    for (int t = sh.k - 1; t >= 0; --t) {
        const size_t p = base + static_cast<size_t>(t) * kTile;
        float l = I->lam[p];
        if (add_t) l += I->T[I->var[p]];
        const double lt = static_cast<double>(l);
        uint32_t c[W];
        load_codes<W>(tpl + t * W, c);
        double cur[W];
#pragma unroll
        for (int v = 0; v < W; ++v) cur[v] = fmin(pick64<W>(nx, c[v] & 0xFFu), pick64<W>(nx, c[v] >> 8) + lt);
#pragma unroll
        for (int v = 0; v < W; ++v) nx[v] = cur[v];
    }
    return nx[0];
}

struct Eval64Args {
    const InstDev* insts;
    const int32_t* prefix;  // [n_inst + 1] lower-bound chunks per instance
    int32_t n_inst;
    int32_t add_t;
};

__global__ void __launch_bounds__(256) eval64_kernel(Eval64Args a) {
    __shared__ double ss[8], sc[8];
    __shared__ int last;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = blockIdx.x;
    const int ii = find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    InstCtl* ctl = I->ctl;
    const int c = g - __ldg(a.prefix + ii);
    const int t_end = min((c + 1) * kLbChunk, I->n_tiles);
    double s = 0.0, cp = 0.0;
    for (int ti = c * kLbChunk + wib; ti < t_end; ti += 8) {
        const TileDev tile = I->tiles[ti];
        if (lane >= tile.n_valid) continue;
        const ShapeDev sh = I->shapes[tile.shape];
        double e;
        switch (sh.width) {
            case 2: e = bdd_energy64<2>(I, tile, sh, lane, a.add_t != 0); break;
            case 4: e = bdd_energy64<4>(I, tile, sh, lane, a.add_t != 0); break;
            case 8: e = bdd_energy64<8>(I, tile, sh, lane, a.add_t != 0); break;
            default: e = bdd_energy64<16>(I, tile, sh, lane, a.add_t != 0); break;
        }
        neumaier64(s, cp, e);
    }
    // fixed-order block reduction: butterfly per warp, then warp 0 over the 8 warp totals
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double os = __shfl_xor_sync(0xffffffffu, s, off);
        const double oc = __shfl_xor_sync(0xffffffffu, cp, off);
        neumaier64(s, cp, os);
        cp += oc;
    }
    if (lane == 0) {
        ss[wib] = s;
        sc[wib] = cp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0, Cc = 0.0;
        for (int w = 0; w < 8; ++w) {
            neumaier64(S, Cc, ss[w]);
            Cc += sc[w];
        }
        I->chunk_lb[c] = S + Cc;
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1) == I->n_chunks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        // the last block: chunk totals in chunk order, then the presolve constant
        double S = 0.0, Cc = 0.0;
        for (int q = 0; q < I->n_chunks; ++q) neumaier64(S, Cc, __ldcg(I->chunk_lb + q));
        neumaier64(S, Cc, I->const_lb);
        ctl->lb_eval = S + Cc;
        ctl->ticket = 0;
    }
}

}  // namespace

cudaError_t launch_eval64(const DevBatch& b, bool add_t, const LaunchCfg& cfg, cudaStream_t s) {
    if (b.chunks_total == 0) return cudaSuccess;
    cfg.count();
    eval64_kernel<<<b.chunks_total, 256, 0, s>>>(Eval64Args{b.insts, b.chunk_prefix, b.n_inst, add_t ? 1 : 0});
    return cudaGetLastError();
}

}  // namespace fdog
