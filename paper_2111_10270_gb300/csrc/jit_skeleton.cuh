// Skeleton of the shape-specialised sweep kernels.  This file is not compiled
// by nvcc: the build embeds it as text, and at plan time jit.cpp appends the
// generated per-shape functions and dispatch tables and compiles the result
// for sm_103a with NVRTC.
//
// The tile loop, instance lookup and per-tile bound reduction are the same as
// in the static sweep kernels (sweep.cuh); only the per-BDD work differs: it
// is straight-line code for one known shape, with every successor choice
// resolved when the code was generated, so a thread spends its instructions
// on the min-plus arithmetic itself.

#define FDOG_INF __int_as_float(0x7f800000)
#define FDOG_FULL 0xffffffffu

__device__ __forceinline__ int fdog_find_inst(const int32_t* __restrict__ prefix, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Deferred terms of the tile-local variables, formed right after an update
// pass from the staged multipliers (same sum and order as the deferred-sum
// kernel); staging: layer t lane l at [32 t + l].
__device__ __forceinline__ void fdog_tile_local_sums(const InstDev* __restrict__ I, int pattern,
                                                     const float* ep_lam, const int* ep_var, int lane) {
    const int2 pat = reinterpret_cast<const int2*>(I->patterns)[pattern];
    for (int e = lane; e < pat.y; e += 32) {
        const ushort4 o = reinterpret_cast<const ushort4*>(I->local_ent)[pat.x + e];
        float s = 0.f + ep_lam[o.x];
        int c = 1;
        if (o.y != 0xFFFFu) { s += ep_lam[o.y]; ++c; }
        if (o.z != 0xFFFFu) { s += ep_lam[o.z]; ++c; }
        if (o.w != 0xFFFFu) { s += ep_lam[o.w]; ++c; }
        const int v = ep_var[o.x];
        // (C - sum) times 1 / c rounded to FP32, as in the deferred-sum kernel
        const float inv = c == 1 ? 1.f : c == 2 ? 0.5f : c == 3 ? 1.f / 3.f : 0.25f;
        I->T[v] = (I->C[v] - s) * inv;
    }
}

// L2 prefetch of the multiplier and variable rows of the tile this warp
// visits next (lane t takes layer t), issued before the current tile is
// computed so that the next tile's first loads hit L2.
__device__ __forceinline__ void fdog_prefetch_tile(const SweepArgs& a, int g, int lane) {
    if (g >= a.total) return;
    const int ii = fdog_find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    const TileDev tile = I->tiles[__ldg(a.first + ii) + (g - __ldg(a.prefix + ii))];
    const int k = I->shapes[tile.shape].k;
    if (lane < k) {
        const long long p = (long long)tile.slot_base + 32LL * lane;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(I->lam + p));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(I->var + p));
    }
}

// MODE: 0 ascending pass with updates, 1 descending pass with updates,
//       2 min-marginals, 3 energies only
template <int MODE>
__device__ __forceinline__ void fdog_jit_sweep(const SweepArgs& a) {
    extern __shared__ float fdog_smem[];
    // programmatic dependent launch (the launches allow it): let the next kernel be scheduled once every
    // block has started, and touch memory only after the kernel before this one has completed
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    float* ep_lam = fdog_smem + (long long)wib * a.epi * 32 * 2;
    int* ep_var = (int*)(ep_lam + (long long)a.epi * 32);
    for (int g = blockIdx.x * wpb + wib; g < a.total; g += gridDim.x * wpb) {
        fdog_prefetch_tile(a, g + gridDim.x * wpb, lane);
        const int ii = fdog_find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        if (MODE <= 1 && FDOG_INACTIVE(I->ctl)) continue;
        const int ti = __ldg(a.first + ii) + (g - __ldg(a.prefix + ii));
        const TileDev tile = I->tiles[ti];
        const int jit = I->shapes[tile.shape].jit;
        const bool valid = lane < tile.n_valid;
        const long long base = (long long)tile.slot_base + lane;
        const bool local = MODE <= 1 && a.epi > 0 && tile.pattern >= 0;
        float term = 0.f;
        FDOG_DISPATCH(MODE)
        if (local) {
            __syncwarp();
            fdog_tile_local_sums(I, tile.pattern, ep_lam, ep_var, lane);
            __syncwarp();
        }
        if (MODE == 1 || MODE == 3) {  // only the descending pass and the energy sweep feed a bound reduction
            float s = valid ? term : 0.f, comp = 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float o = __shfl_xor_sync(FDOG_FULL, s, off);
                const float oc = __shfl_xor_sync(FDOG_FULL, comp, off);
                const float sum = s + o;
                const float bp = sum - s;
                const float err = (s - (sum - bp)) + (o - bp);
                s = sum;
                comp = comp + oc + err;
            }
            if (lane == 0) I->tile_lb[ti] = make_float2(s, comp);
        }
    }
}

extern "C" __global__ void __launch_bounds__(256) fdog_jit_fwd(SweepArgs a) { fdog_jit_sweep<0>(a); }
extern "C" __global__ void __launch_bounds__(256) fdog_jit_bwd(SweepArgs a) { fdog_jit_sweep<1>(a); }
extern "C" __global__ void __launch_bounds__(256) fdog_jit_mm(SweepArgs a) { fdog_jit_sweep<2>(a); }
extern "C" __global__ void __launch_bounds__(256) fdog_jit_eval(SweepArgs a) { fdog_jit_sweep<3>(a); }
