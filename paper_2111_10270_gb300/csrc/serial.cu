// The serial min-marginal averaging of Eq. 4, run level by level.
//
// One iteration is an ascending sweep over the variables and a descending
// one.  Before a sweep, serial_labels_kernel stores, for every BDD, the
// shortest-path labels of the direction opposite to the sweep at the current
// multipliers (SP(v, TOP) of every layer before an ascending sweep, SP(r, v)
// before a descending one) and initialises the BDD's running labels.  Then
// serial_level_kernel handles the sweep's levels in order: one thread per
// variable of the level computes the min-marginal difference of each copy
// (Eq. 6 from the running labels and the stored ones), averages them, sets
// every copy to lambda - M + average (Eq. 4) and advances that BDD's running
// labels past the layer.  Variables of one level share no BDD, and a BDD's
// layers are reached in its own order, so this equals visiting the variables
// one at a time in index order.  The bound is then evaluated at the new
// multipliers (evaluation sweep, staged reduction, commit).
#include <cuda_runtime.h>

#include "kernels.h"
#include "sweep.cuh"

namespace fdog {

namespace {

using dev::finf;
using dev::load_codes;
using dev::pick;
using dev::push;

struct SerialArgs {
    const InstDev* I;
    const int32_t* vars;  // the variables of one level
    int32_t n;
};

// Labels of one BDD (thread) for the sweep in direction ASC.  Layout of the
// tile's region: [t][v][lane] for t < k, then the running labels [v][lane].
template <int W, bool ASC>
__device__ void tile_labels(const InstDev* __restrict__ I, const TileDev& tile, const ShapeDev& sh, float* reg,
                            int lane) {
    const uint16_t* __restrict__ tpl = I->tpl + sh.tpl_off;
    const size_t base = static_cast<size_t>(tile.slot_base) + lane;
    const int k = sh.k;
    if constexpr (ASC) {
        // SP(v, TOP) of every layer, from the last layer up
        float nx[W];
#pragma unroll
        for (int v = 0; v < W; ++v) nx[v] = finf();
        for (int t = k - 1; t >= 0; --t) {
            uint32_t c[W];
            load_codes<W>(tpl + t * W, c);
            const float lt = I->lam[base + static_cast<size_t>(t) * kTile];
            float cur[W];
#pragma unroll
            for (int v = 0; v < W; ++v) cur[v] = fminf(pick<W>(nx, c[v] & 0xFFu), pick<W>(nx, c[v] >> 8) + lt);
#pragma unroll
            for (int v = 0; v < W; ++v) { nx[v] = cur[v]; reg[(t * W + v) * kTile + lane] = cur[v]; }
        }
#pragma unroll
        for (int v = 0; v < W; ++v) reg[(k * W + v) * kTile + lane] = v == 0 ? 0.f : finf();  // root labels
    } else {
        // SP(r, v) of every layer, from the root down
        float f[W];
#pragma unroll
        for (int v = 0; v < W; ++v) f[v] = v == 0 ? 0.f : finf();
        for (int t = 0; t < k; ++t) {
            uint32_t c[W];
            load_codes<W>(tpl + t * W, c);
            const float lt = I->lam[base + static_cast<size_t>(t) * kTile];
            float nf[W];
#pragma unroll
            for (int v = 0; v < W; ++v) { reg[(t * W + v) * kTile + lane] = f[v]; nf[v] = finf(); }
#pragma unroll
            for (int v = 0; v < W; ++v) {
                push<W>(nf, c[v] & 0xFFu, f[v]);
                push<W>(nf, c[v] >> 8, f[v] + lt);
            }
#pragma unroll
            for (int v = 0; v < W; ++v) f[v] = nf[v];
        }
#pragma unroll
        for (int v = 0; v < W; ++v) reg[(k * W + v) * kTile + lane] = finf();  // beyond the last layer: unused
    }
}

template <bool ASC>
__global__ void __launch_bounds__(256) serial_labels_kernel(FlatArgsS a) {
    const int lane = threadIdx.x & 31;
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= a.total) return;
    const InstDev* __restrict__ I = a.I;
    if (FDOG_INACTIVE(I->ctl)) return;
    const TileDev tile = I->tiles[g];
    if (lane >= tile.n_valid) return;
    const ShapeDev sh = I->shapes[tile.shape];
    float* reg = I->lab + I->lab_off[g];
    switch (sh.width) {
        case 2: tile_labels<2, ASC>(I, tile, sh, reg, lane); break;
        case 4: tile_labels<4, ASC>(I, tile, sh, reg, lane); break;
        case 8: tile_labels<8, ASC>(I, tile, sh, reg, lane); break;
        default: tile_labels<16, ASC>(I, tile, sh, reg, lane); break;
    }
}

// Min-marginal difference of one copy (Eq. 6) at the current labels; with
// `apply`, also sets the copy to lambda + (avg - M) (Eq. 4) and advances the
// running labels past its layer.
template <int W, bool ASC>
__device__ float copy_step(const InstDev* __restrict__ I, int32_t p, bool apply, float avg) {
    const int32_t row = p / kTile;
    const int lane = p % kTile;
    const int ti = I->tile_of_row[row];
    const TileDev tile = I->tiles[ti];
    const ShapeDev sh = I->shapes[tile.shape];
    const int t = row - tile.slot_base / kTile;
    const int k = sh.k;
    float* reg = I->lab + I->lab_off[ti];
    uint32_t c[W];
    load_codes<W>(I->tpl + sh.tpl_off + t * W, c);
    float f[W], b[W];
    // ascending: running SP(r, .) of layer t, stored SP(., TOP) of layer t + 1;
    // descending: stored SP(r, .) of layer t, running SP(., TOP) of layer t + 1
#pragma unroll
    for (int v = 0; v < W; ++v) {
        f[v] = ASC ? reg[(k * W + v) * kTile + lane] : reg[(t * W + v) * kTile + lane];
        b[v] = ASC ? (t + 1 < k ? reg[((t + 1) * W + v) * kTile + lane] : finf()) : reg[(k * W + v) * kTile + lane];
    }
    const float lt = I->lam[p];
    float m0 = finf(), m1 = finf();
#pragma unroll
    for (int v = 0; v < W; ++v) {
        m0 = fminf(m0, f[v] + pick<W>(b, c[v] & 0xFFu));
        m1 = fminf(m1, f[v] + lt + pick<W>(b, c[v] >> 8));
    }
    const float M = m1 - m0;
    if (apply) {
        const float ln = lt + (avg - M);
        I->lam[p] = ln;
        float nx[W];
        if constexpr (ASC) {
#pragma unroll
            for (int v = 0; v < W; ++v) nx[v] = finf();
#pragma unroll
            for (int v = 0; v < W; ++v) {
                push<W>(nx, c[v] & 0xFFu, f[v]);
                push<W>(nx, c[v] >> 8, f[v] + ln);
            }
        } else {
#pragma unroll
            for (int v = 0; v < W; ++v) nx[v] = fminf(pick<W>(b, c[v] & 0xFFu), pick<W>(b, c[v] >> 8) + ln);
        }
#pragma unroll
        for (int v = 0; v < W; ++v) reg[(k * W + v) * kTile + lane] = nx[v];
    }
    return M;
}

template <bool ASC>
__device__ float copy_step_any(const InstDev* __restrict__ I, int32_t p, bool apply, float avg) {
    switch (I->shapes[I->tiles[I->tile_of_row[p / kTile]].shape].width) {
        case 2: return copy_step<2, ASC>(I, p, apply, avg);
        case 4: return copy_step<4, ASC>(I, p, apply, avg);
        case 8: return copy_step<8, ASC>(I, p, apply, avg);
        default: return copy_step<16, ASC>(I, p, apply, avg);
    }
}

template <bool ASC>
__global__ void __launch_bounds__(256) serial_level_kernel(SerialArgs a) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n) return;
    const InstDev* __restrict__ I = a.I;
    if (FDOG_INACTIVE(I->ctl)) return;
    const int i = a.vars[g];
    const int b = I->csr_off[i], e = I->csr_off[i + 1];
    // copies in ascending slot order: sum of the differences, then the update
    float sum = 0.f;
    for (int q = b; q < e; ++q) sum += copy_step_any<ASC>(I, I->csr_pos[q], false, 0.f);
    const float avg = sum / static_cast<float>(e - b);
    for (int q = b; q < e; ++q) copy_step_any<ASC>(I, I->csr_pos[q], true, avg);
}

}  // namespace

cudaError_t launch_iteration_serial(const DevBatch& b, const LaunchCfg& cfg, cudaStream_t s) {
    const SerialPlan& sp = b.serial;
    const InstDev* I = sp.inst;
    const int tiles = b.tiles_all_total;
    for (int dir = 0; dir < 2; ++dir) {
        const bool asc = dir == 0;
        if (tiles > 0) {
            const FlatArgsS la{I, tiles};
            const int blocks = (tiles + 7) / 8;
            if (asc) serial_labels_kernel<true><<<blocks, 256, 0, s>>>(la);
            else serial_labels_kernel<false><<<blocks, 256, 0, s>>>(la);
            cfg.count();
        }
        const int32_t* off = asc ? sp.lev_f_off : sp.lev_b_off;
        const int n_lev = asc ? sp.n_lev_f : sp.n_lev_b;
        const int32_t* vars = asc ? sp.lev_f : sp.lev_b;
        for (int l = 0; l < n_lev; ++l) {
            const int n = off[l + 1] - off[l];
            if (n == 0) continue;
            const SerialArgs args{I, vars + off[l], n};
            if (asc) serial_level_kernel<true><<<(n + 255) / 256, 256, 0, s>>>(args);
            else serial_level_kernel<false><<<(n + 255) / 256, 256, 0, s>>>(args);
            cfg.count();
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the bound at the new multipliers: evaluation sweep, staged reduction, commit
    if ((e = launch_sweep(b, kEval, 0, cfg, s)) != cudaSuccess) return e;
    if ((e = launch_lb_reduce(b, kLbStage, cfg, s)) != cudaSuccess) return e;
    return launch_lb_commit(b, cfg, s);
}

}  // namespace fdog
