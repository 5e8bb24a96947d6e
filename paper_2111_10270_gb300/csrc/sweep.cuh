// Sweep kernel template (included by the per-width translation units).
//
// One warp per tile of 32 BDDs of one shape, one thread per BDD.  All
// per-layer loads/stores of a warp are single 128-byte transactions
// (interleaved slots); the shape template is read with warp-uniform loads.
// Shortest-path labels of the direction opposite to the pass are recomputed
// on chip at the start of each pass, so no per-node state goes to HBM: the
// per-slot multipliers are the only state the sweeps stream.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace fdog {
namespace dev {

// Programmatic dependent launch.  The iteration kernels are launched with
// programmatic stream serialization: a kernel may be scheduled while the one
// before it on its stream drains.  pdl_wait() returns once that kernel has
// completed and its writes are visible (at once for a launch without the
// attribute), so every such kernel calls it before it touches memory;
// pdl_trigger() lets the next kernel be scheduled once every block of this
// one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

// largest instance index i with prefix[i] <= g (empty instances are skipped)
__device__ __forceinline__ int find_inst(const int32_t* __restrict__ prefix, int n, int g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int W>
__device__ __forceinline__ void load_codes(const uint16_t* __restrict__ p, uint32_t (&c)[W]) {
    if constexpr (W == 2) {
        const uint32_t u = __ldg(reinterpret_cast<const unsigned int*>(p));
        c[0] = u & 0xFFFFu; c[1] = u >> 16;
    } else if constexpr (W == 4) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        c[0] = u.x & 0xFFFFu; c[1] = u.x >> 16; c[2] = u.y & 0xFFFFu; c[3] = u.y >> 16;
    } else {
#pragma unroll
        for (int q = 0; q < W / 8; ++q) {
            const uint4 u = __ldg(reinterpret_cast<const uint4*>(p) + q);
            c[8 * q + 0] = u.x & 0xFFFFu; c[8 * q + 1] = u.x >> 16;
            c[8 * q + 2] = u.y & 0xFFFFu; c[8 * q + 3] = u.y >> 16;
            c[8 * q + 4] = u.z & 0xFFFFu; c[8 * q + 5] = u.z >> 16;
            c[8 * q + 6] = u.w & 0xFFFFu; c[8 * q + 7] = u.w >> 16;
        }
    }
}

// label of the successor with the given code: a node of the next layer, TOP (0) or BOT (inf)
template <int W>
__device__ __forceinline__ float pick(const float (&x)[W], uint32_t code) {
    float r = (code == kCodeTop) ? 0.f : finf();
#pragma unroll
    for (int w = 0; w < W; ++w) r = (code == static_cast<uint32_t>(w)) ? x[w] : r;
    return r;
}

template <int W>
__device__ __forceinline__ void push(float (&x)[W], uint32_t code, float val) {
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (code == static_cast<uint32_t>(w)) x[w] = fminf(x[w], val);
}

// per-layer state of one BDD: registers for short rows, shared memory otherwise
template <int W, bool REG>
struct Store;

template <int W>
struct Store<W, true> {
    float lam[kRegK], tb[kRegK], sp[kRegK][W];
    __device__ __forceinline__ float& L(int t) { return lam[t]; }
    __device__ __forceinline__ float& T(int t) { return tb[t]; }
    __device__ __forceinline__ float& S(int t, int v) { return sp[t][v]; }
};

template <int W>
struct Store<W, false> {
    float* base;  // this lane's column of the warp's region
    int stride;
    __device__ __forceinline__ float& L(int t) { return base[t * kTile]; }
    __device__ __forceinline__ float& T(int t) { return base[(stride + t) * kTile]; }
    __device__ __forceinline__ float& S(int t, int v) { return base[(2 * stride + t * W + v) * kTile]; }
};


// 1 / c rounded to FP32 for a copy count c <= 8 (constants folded at compile
// time); the deferred term of a variable is (C_i - sum_j lambda^j_i) times it
// in every kernel that forms one, so all of them agree bit for bit
__device__ __forceinline__ float inv_copies(int c) {
    return c == 1 ? 1.f : c == 2 ? 0.5f : c == 3 ? 1.f / 3.f : c == 4 ? 0.25f
         : c == 5 ? 1.f / 5.f : c == 6 ? 1.f / 6.f : c == 7 ? 1.f / 7.f : 0.125f;
}

// Deferred terms of the tile-local variables (every copy in this tile),
// formed right after the pass from the staged multipliers: the same sum, in
// the same ascending slot order, as the deferred-sum kernel uses.
// ep_lam / ep_var: this warp's staging, layer t lane l at [32 t + l].
__device__ __forceinline__ void tile_local_sums(const InstDev* __restrict__ I, int pattern, const float* ep_lam,
                                                const int* ep_var, int lane) {
    const int2 pat = reinterpret_cast<const int2*>(I->patterns)[pattern];
    for (int e = lane; e < pat.y; e += 32) {
        const ushort4 o = reinterpret_cast<const ushort4*>(I->local_ent)[pat.x + e];
        float s = 0.f + ep_lam[o.x];
        int c = 1;
        if (o.y != 0xFFFFu) { s += ep_lam[o.y]; ++c; }
        if (o.z != 0xFFFFu) { s += ep_lam[o.z]; ++c; }
        if (o.w != 0xFFFFu) { s += ep_lam[o.w]; ++c; }
        const int v = ep_var[o.x];
        I->T[v] = (I->C[v] - s) * inv_copies(c);
    }
}

// L2 prefetch of the multiplier and variable rows of the tile this warp
// visits next (lane t takes layer t), issued before the current tile is
// computed so that the next tile's first loads hit L2.
__device__ __forceinline__ void prefetch_tile(const SweepArgs& a, int g, int lane) {
    if (g >= a.total) return;
    const int ii = find_inst(a.prefix, a.n_inst, g);
    const InstDev* __restrict__ I = a.insts + ii;
    const TileDev tile = I->tiles[__ldg(a.first + ii) + (g - __ldg(a.prefix + ii))];
    const int k = I->shapes[tile.shape].k;
    for (int t = lane; t < k; t += kTile) {
        const long long p = static_cast<long long>(tile.slot_base) + static_cast<long long>(kTile) * t;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(I->lam + p));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(I->var + p));
    }
}

// Loops over layers.  With REG the trip count is the constant kRegK and the
// loops unroll completely, so every index into Store is a compile-time
// constant and the arrays stay in registers.
#define FD_UP(t) _Pragma("unroll") for (int t = 0; t < (REG ? kRegK : k); ++t)
#define FD_DOWN(t, tt) \
    _Pragma("unroll") for (int tt = 0; tt < (REG ? kRegK : k); ++tt) \
        if (const int t = (REG ? kRegK : k) - 1 - tt; t < k)

// shared-memory floats one warp of sweep_tile uses
template <int W, bool REG>
__host__ __device__ __forceinline__ size_t sweep_warp_floats(const SweepArgs& a) {
    return (REG ? 0 : static_cast<size_t>(a.kstride) * kTile * (2 + W)) + static_cast<size_t>(a.epi) * kTile * 2;
}

// One tile g of a class (lane = BDD), the warp's shared memory at wsm; the
// tile this warp visits next (g_next, if below a.total) is prefetched into L2.
template <int W, bool REG, int MODE>
__device__ __forceinline__ void sweep_tile(const SweepArgs& a, int g, int g_next, float* wsm, int lane) {
    {
        prefetch_tile(a, g_next, lane);
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        if constexpr (MODE == kFwdUpdate || MODE == kBwdUpdate) {
            if (FDOG_INACTIVE(I->ctl)) return;  // stopped, or out of iterations
        }
        const TileDev tile = I->tiles[__ldg(a.first + ii) + (g - __ldg(a.prefix + ii))];
        const ShapeDev sh = I->shapes[tile.shape];
        const int k = sh.k;
        const uint16_t* __restrict__ tpl = I->tpl + sh.tpl_off;
        const bool valid = lane < tile.n_valid;
        const float omega = I->omega;
        const size_t base = static_cast<size_t>(tile.slot_base) + lane;
        float* __restrict__ lam = I->lam;
        const bool need_t = (MODE == kFwdUpdate || MODE == kBwdUpdate) || (a.flags & kMMAddT);

        Store<W, REG> S;
        // per-warp shared memory: [Store arrays (shared-memory variants)] [staging for tile-local sums]
        if constexpr (!REG) {
            S.base = wsm + lane;
            S.stride = a.kstride;
        }
        float* ep_lam = wsm + (REG ? 0 : static_cast<size_t>(a.kstride) * kTile * (2 + W));
        int* ep_var = reinterpret_cast<int*>(ep_lam + static_cast<size_t>(a.epi) * kTile);
        const bool local = (MODE == kFwdUpdate || MODE == kBwdUpdate) && a.epi > 0 && tile.pattern >= 0;

        // multipliers and deferred terms of every layer (coalesced per layer)
        FD_UP(t) {
            if (t >= k) break;
            float l = 0.f, tb = 0.f;
            if (valid) {
                l = lam[base + static_cast<size_t>(t) * kTile];
                if (need_t) {
                    const int v = __ldcs(I->var + base + static_cast<size_t>(t) * kTile);  // streamed once per pass
                    tb = I->T[v];
                    if (local) ep_var[t * kTile + lane] = v;
                }
            }
            if constexpr (MODE == kMinMarg || MODE == kEval) {
                if (a.flags & kMMAddT) l += tb;
            }
            S.L(t) = l;
            S.T(t) = tb;
        }

        float term = 0.f;  // this BDD's share of the lower bound
        if constexpr (MODE == kFwdUpdate || MODE == kMinMarg || MODE == kEval) {
            // SP(v, TOP) of every node at the current multipliers (Alg. 4 without updates)
            float nx[W];
#pragma unroll
            for (int v = 0; v < W; ++v) nx[v] = finf();
            FD_DOWN(t, tt) {
                uint32_t c[W];
                load_codes<W>(tpl + t * W, c);
                const float lt = S.L(t);
                float cur[W];
#pragma unroll
                for (int v = 0; v < W; ++v) cur[v] = fminf(pick<W>(nx, c[v] & 0xFFu), pick<W>(nx, c[v] >> 8) + lt);
#pragma unroll
                for (int v = 0; v < W; ++v) { S.S(t, v) = cur[v]; nx[v] = cur[v]; }
            }
            if constexpr (MODE == kEval) term = nx[0];
        }

        if constexpr (MODE == kFwdUpdate || MODE == kMinMarg) {
            // ascending pass: SP(r, .) incrementally (Alg. 3) and Eq. 6 per layer
            float f[W];
#pragma unroll
            for (int v = 0; v < W; ++v) f[v] = v == 0 ? 0.f : finf();
            float negsum = 0.f, E = finf();
            float* __restrict__ mm0 = I->mm0;
            float* __restrict__ mm1 = I->mm1;
            FD_UP(t) {
                if (t >= k) break;
                uint32_t c[W];
                load_codes<W>(tpl + t * W, c);
                const int tn = REG ? ((t + 1 < kRegK) ? t + 1 : t) : ((t + 1 < k) ? t + 1 : t);
                float b[W];
#pragma unroll
                for (int v = 0; v < W; ++v) b[v] = S.S(tn, v);  // unused on the last layer (terminal codes)
                float m0 = finf(), m1 = finf();
#pragma unroll
                for (int v = 0; v < W; ++v) {
                    m0 = fminf(m0, f[v] + pick<W>(b, c[v] & 0xFFu));
                    m1 = fminf(m1, f[v] + pick<W>(b, c[v] >> 8));
                }
                const float lt = S.L(t);
                m1 += lt;
                float lt_new = lt;
                if constexpr (MODE == kFwdUpdate) {
                    const float d = m1 - m0;
                    lt_new = fmaf(-omega, d, lt) + S.T(t);  // Eq. 5
                    S.L(t) = lt_new;
                    negsum += fmaxf(-d, 0.f);
                } else {
                    if (valid) {
                        const size_t p = base + static_cast<size_t>(t) * kTile;
                        if (a.flags & kMMBoth) { mm0[p] = m0; mm1[p] = m1; }
                        else mm0[p] = m1 - m0;
                    }
                }
                float nf[W];
#pragma unroll
                for (int v = 0; v < W; ++v) nf[v] = finf();
#pragma unroll
                for (int v = 0; v < W; ++v) {
                    const uint32_t lo = c[v] & 0xFFu, hi = c[v] >> 8;
                    push<W>(nf, lo, f[v]);
                    push<W>(nf, hi, f[v] + lt_new);
                    E = fminf(E, lo == kCodeTop ? f[v] : finf());
                    E = fminf(E, hi == kCodeTop ? f[v] + lt_new : finf());
                }
#pragma unroll
                for (int v = 0; v < W; ++v) f[v] = nf[v];
            }
            term = fmaf(-omega, negsum, E);
        }

        if constexpr (MODE == kBwdUpdate) {
            // SP(r, v) of every node at the current multipliers (Alg. 3 without updates)
            float f[W];
#pragma unroll
            for (int v = 0; v < W; ++v) f[v] = v == 0 ? 0.f : finf();
            FD_UP(t) {
                if (t >= k) break;
                uint32_t c[W];
                load_codes<W>(tpl + t * W, c);
                const float lt = S.L(t);
                float nf[W];
#pragma unroll
                for (int v = 0; v < W; ++v) { S.S(t, v) = f[v]; nf[v] = finf(); }
#pragma unroll
                for (int v = 0; v < W; ++v) {
                    push<W>(nf, c[v] & 0xFFu, f[v]);
                    push<W>(nf, c[v] >> 8, f[v] + lt);
                }
#pragma unroll
                for (int v = 0; v < W; ++v) f[v] = nf[v];
            }
            // descending pass: SP(., TOP) incrementally (Alg. 4) and Eq. 6 per layer
            float b[W];
#pragma unroll
            for (int v = 0; v < W; ++v) b[v] = finf();
            float negsum = 0.f;
            FD_DOWN(t, tt) {
                uint32_t c[W];
                load_codes<W>(tpl + t * W, c);
                float m0 = finf(), m1 = finf();
#pragma unroll
                for (int v = 0; v < W; ++v) {
                    const float fv = S.S(t, v);
                    m0 = fminf(m0, fv + pick<W>(b, c[v] & 0xFFu));
                    m1 = fminf(m1, fv + pick<W>(b, c[v] >> 8));
                }
                const float lt = S.L(t);
                m1 += lt;
                const float d = m1 - m0;
                const float lt_new = fmaf(-omega, d, lt) + S.T(t);  // Eq. 5
                S.L(t) = lt_new;
                negsum += fmaxf(-d, 0.f);
                float nb[W];
#pragma unroll
                for (int v = 0; v < W; ++v) nb[v] = fminf(pick<W>(b, c[v] & 0xFFu), pick<W>(b, c[v] >> 8) + lt_new);
#pragma unroll
                for (int v = 0; v < W; ++v) b[v] = nb[v];
            }
            term = fmaf(-omega, negsum, b[0]);
        }

        if constexpr (MODE == kFwdUpdate || MODE == kBwdUpdate) {
            FD_UP(t) {
                if (t >= k) break;
                if (valid) lam[base + static_cast<size_t>(t) * kTile] = S.L(t);
                if (local) ep_lam[t * kTile + lane] = S.L(t);
            }
            if (local) {
                __syncwarp();
                tile_local_sums(I, tile.pattern, ep_lam, ep_var, lane);
                __syncwarp();
            }
        }

        // per-tile partial of the bound: compensated FP32 butterfly (all lanes end equal); only the
        // descending update pass and the energy sweep feed a bound reduction
        if constexpr (MODE == kBwdUpdate || MODE == kEval) {  // the passes whose bound is reduced
            float s = valid ? term : 0.f, comp = 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float o = __shfl_xor_sync(kFull, s, off);
                const float oc = __shfl_xor_sync(kFull, comp, off);
                const float sum = s + o;
                const float bp = sum - s;
                const float err = (s - (sum - bp)) + (o - bp);
                s = sum;
                comp = comp + oc + err;
            }
            if (lane == 0) I->tile_lb[__ldg(a.first + ii) + (g - __ldg(a.prefix + ii))] = make_float2(s, comp);
        }
    }
}

template <int W, bool REG, int MODE>
__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs a) {
    extern __shared__ float smem[];
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    float* wsm = smem + static_cast<size_t>(wib) * sweep_warp_floats<W, REG>(a);
    for (int g = blockIdx.x * wpb + wib; g < a.total; g += gridDim.x * wpb)
        sweep_tile<W, REG, MODE>(a, g, g + gridDim.x * wpb, wsm, lane);
}


// Long rows (more than kRegK layers) of narrow BDDs (W <= kRegW).  Staging
// every layer in shared memory would size each warp's region by the longest
// row of the launch and starve the SM of warps, so the layers are processed
// in segments of kRegK held in registers instead.  A first sweep over the
// whole row keeps only the labels at segment starts (checkpoints, in shared
// memory); the update sweep then visits the segments in its own direction,
// reloads each one's multipliers and recomputes its labels from the next
// checkpoint.  Every label and update is formed by the same operations in the
// same order as in sweep_kernel, so results are identical; the cost is one
// extra label sweep over data the warp has just read.
// Shared memory per warp: a.kstride checkpoints x W labels x 32 lanes, then
// the tile-local staging (a.epi layers).
// shared-memory floats one warp of seg_tile uses
template <int W>
__host__ __device__ __forceinline__ size_t seg_warp_floats(const SweepArgs& a) {
    return static_cast<size_t>(a.kstride) * W * kTile + static_cast<size_t>(a.epi) * kTile * 2;
}

template <int W, int MODE>
__device__ __forceinline__ void seg_tile(const SweepArgs& a, int g, int g_next, float* wsm, int lane) {
    constexpr int C = kRegK;
    float* cp = wsm + lane;  // checkpoint s, label v at cp[(s * W + v) * kTile]
    float* ep_lam = wsm + static_cast<size_t>(a.kstride) * W * kTile;
    int* ep_var = reinterpret_cast<int*>(ep_lam + static_cast<size_t>(a.epi) * kTile);
    {
        prefetch_tile(a, g_next, lane);
        const int ii = find_inst(a.prefix, a.n_inst, g);
        const InstDev* __restrict__ I = a.insts + ii;
        if constexpr (MODE == kFwdUpdate || MODE == kBwdUpdate) {
            if (FDOG_INACTIVE(I->ctl)) return;
        }
        const TileDev tile = I->tiles[__ldg(a.first + ii) + (g - __ldg(a.prefix + ii))];
        const ShapeDev sh = I->shapes[tile.shape];
        const int k = sh.k;
        const int nseg = (k + C - 1) / C;
        const uint16_t* __restrict__ tpl = I->tpl + sh.tpl_off;
        const bool valid = lane < tile.n_valid;
        const float omega = I->omega;
        const size_t base = static_cast<size_t>(tile.slot_base) + lane;
        float* __restrict__ lam = I->lam;
        const int32_t* __restrict__ varp = I->var;
        const float* __restrict__ Tv = I->T;
        constexpr bool update = MODE == kFwdUpdate || MODE == kBwdUpdate;
        const bool need_t = update || (a.flags & kMMAddT);
        const bool add_t = (MODE == kMinMarg || MODE == kEval) && (a.flags & kMMAddT);
        const bool local = update && a.epi > 0 && tile.pattern >= 0;

        // raw loads of one segment (multipliers, and variable ids if asked); independent of each other
        auto fetch = [&](int s, float (&L)[C], int (&V)[C], bool with_var) {
            const int t0 = s * C;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                L[c] = 0.f;
                V[c] = -1;
                if (valid && t0 + c < k) {
                    const size_t p = base + static_cast<size_t>(t0 + c) * kTile;
                    L[c] = lam[p];
                    if (with_var) V[c] = __ldcs(varp + p);  // streamed once per pass
                }
            }
        };
        // deferred terms of a fetched segment; with add_t the multipliers include them
        auto terms = [&](float (&L)[C], const int (&V)[C], float (&Tt)[C]) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                Tt[c] = V[c] >= 0 ? Tv[V[c]] : 0.f;
                if (add_t) L[c] += Tt[c];
            }
        };

        float term = 0.f;
        if constexpr (MODE == kFwdUpdate || MODE == kMinMarg || MODE == kEval) {
            // SP(v, TOP) over the whole row, one segment at a time from the last;
            // keep the labels at segment starts
            float nx[W];
#pragma unroll
            for (int v = 0; v < W; ++v) nx[v] = finf();
            for (int s = nseg - 1; s >= 0; --s) {
                const int t0 = s * C;
                const int kk = (k - t0 < C) ? k - t0 : C;
                float L[C], Tt[C];
                int V[C];
                fetch(s, L, V, add_t);
                if (add_t) terms(L, V, Tt);
#pragma unroll
                for (int cc = C - 1; cc >= 0; --cc) {
                    if (cc < kk) {
                        uint32_t c[W];
                        load_codes<W>(tpl + (t0 + cc) * W, c);
                        float cur[W];
#pragma unroll
                        for (int v = 0; v < W; ++v) cur[v] = fminf(pick<W>(nx, c[v] & 0xFFu), pick<W>(nx, c[v] >> 8) + L[cc]);
#pragma unroll
                        for (int v = 0; v < W; ++v) nx[v] = cur[v];
                    }
                }
#pragma unroll
                for (int v = 0; v < W; ++v) cp[(s * W + v) * kTile] = nx[v];
            }
            if constexpr (MODE == kEval) term = nx[0];
        }

        if constexpr (MODE == kFwdUpdate || MODE == kMinMarg) {
            float f[W];
#pragma unroll
            for (int v = 0; v < W; ++v) f[v] = v == 0 ? 0.f : finf();
            float negsum = 0.f, E = finf();
            float* __restrict__ mm0 = I->mm0;
            float* __restrict__ mm1 = I->mm1;
            float Ln[C];
            int Vn[C];
            fetch(0, Ln, Vn, need_t);
            for (int s = 0; s < nseg; ++s) {
                const int t0 = s * C;
                const int kk = (k - t0 < C) ? k - t0 : C;
                float L[C], Tt[C], Sg[C][W], nxt[W];
                int V[C];
#pragma unroll
                for (int c = 0; c < C; ++c) { L[c] = Ln[c]; V[c] = Vn[c]; }
                if (s + 1 < nseg) fetch(s + 1, Ln, Vn, need_t);  // in flight while this segment is swept
                terms(L, V, Tt);
                if (local && valid) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        if (c < kk) ep_var[(t0 + c) * kTile + lane] = V[c];
                }
                // labels of the segment's layers 1 .. kk-1, from the next checkpoint
#pragma unroll
                for (int v = 0; v < W; ++v) nxt[v] = (s + 1 < nseg) ? cp[((s + 1) * W + v) * kTile] : finf();
                {
                    float nx[W];
#pragma unroll
                    for (int v = 0; v < W; ++v) nx[v] = nxt[v];
#pragma unroll
                    for (int cc = C - 1; cc >= 1; --cc) {
                        if (cc < kk) {
                            uint32_t c[W];
                            load_codes<W>(tpl + (t0 + cc) * W, c);
                            float cur[W];
#pragma unroll
                            for (int v = 0; v < W; ++v)
                                cur[v] = fminf(pick<W>(nx, c[v] & 0xFFu), pick<W>(nx, c[v] >> 8) + L[cc]);
#pragma unroll
                            for (int v = 0; v < W; ++v) { Sg[cc][v] = cur[v]; nx[v] = cur[v]; }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    if (c < kk) {
                        const int t = t0 + c;
                        uint32_t cd[W];
                        load_codes<W>(tpl + t * W, cd);
                        float b[W];
#pragma unroll
                        for (int v = 0; v < W; ++v) b[v] = (c + 1 < kk) ? Sg[(c + 1 < C) ? c + 1 : c][v] : nxt[v];
                        float m0 = finf(), m1 = finf();
#pragma unroll
                        for (int v = 0; v < W; ++v) {
                            m0 = fminf(m0, f[v] + pick<W>(b, cd[v] & 0xFFu));
                            m1 = fminf(m1, f[v] + pick<W>(b, cd[v] >> 8));
                        }
                        const float lt = L[c];
                        m1 += lt;
                        float lt_new = lt;
                        if constexpr (MODE == kFwdUpdate) {
                            const float d = m1 - m0;
                            lt_new = fmaf(-omega, d, lt) + Tt[c];  // Eq. 5
                            L[c] = lt_new;
                            negsum += fmaxf(-d, 0.f);
                        } else {
                            if (valid) {
                                const size_t p = base + static_cast<size_t>(t) * kTile;
                                if (a.flags & kMMBoth) { mm0[p] = m0; mm1[p] = m1; }
                                else mm0[p] = m1 - m0;
                            }
                        }
                        float nf[W];
#pragma unroll
                        for (int v = 0; v < W; ++v) nf[v] = finf();
#pragma unroll
                        for (int v = 0; v < W; ++v) {
                            const uint32_t lo = cd[v] & 0xFFu, hi = cd[v] >> 8;
                            push<W>(nf, lo, f[v]);
                            push<W>(nf, hi, f[v] + lt_new);
                            E = fminf(E, lo == kCodeTop ? f[v] : finf());
                            E = fminf(E, hi == kCodeTop ? f[v] + lt_new : finf());
                        }
#pragma unroll
                        for (int v = 0; v < W; ++v) f[v] = nf[v];
                    }
                }
                if constexpr (MODE == kFwdUpdate) {
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        if (c < kk) {
                            if (valid) lam[base + static_cast<size_t>(t0 + c) * kTile] = L[c];
                            if (local) ep_lam[(t0 + c) * kTile + lane] = L[c];
                        }
                    }
                }
            }
            term = fmaf(-omega, negsum, E);
        }

        if constexpr (MODE == kBwdUpdate) {
            // SP(r, v) over the whole row, one segment at a time; keep the labels at segment starts
            {
                float f[W];
#pragma unroll
                for (int v = 0; v < W; ++v) f[v] = v == 0 ? 0.f : finf();
                for (int s = 0; s < nseg; ++s) {
                    const int t0 = s * C;
                    const int kk = (k - t0 < C) ? k - t0 : C;
                    float L[C];
                    int V[C];
                    fetch(s, L, V, false);
#pragma unroll
                    for (int v = 0; v < W; ++v) cp[(s * W + v) * kTile] = f[v];
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        if (c < kk) {
                            uint32_t cd[W];
                            load_codes<W>(tpl + (t0 + c) * W, cd);
                            float nf[W];
#pragma unroll
                            for (int v = 0; v < W; ++v) nf[v] = finf();
#pragma unroll
                            for (int v = 0; v < W; ++v) {
                                push<W>(nf, cd[v] & 0xFFu, f[v]);
                                push<W>(nf, cd[v] >> 8, f[v] + L[c]);
                            }
#pragma unroll
                            for (int v = 0; v < W; ++v) f[v] = nf[v];
                        }
                    }
                }
            }
            float b[W];
#pragma unroll
            for (int v = 0; v < W; ++v) b[v] = finf();
            float negsum = 0.f;
            float Ln[C];
            int Vn[C];
            fetch(nseg - 1, Ln, Vn, true);
            for (int s = nseg - 1; s >= 0; --s) {
                const int t0 = s * C;
                const int kk = (k - t0 < C) ? k - t0 : C;
                float L[C], Tt[C], Sg[C][W];
                int V[C];
#pragma unroll
                for (int c = 0; c < C; ++c) { L[c] = Ln[c]; V[c] = Vn[c]; }
                if (s > 0) fetch(s - 1, Ln, Vn, true);  // in flight while this segment is swept
                terms(L, V, Tt);
                if (local && valid) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        if (c < kk) ep_var[(t0 + c) * kTile + lane] = V[c];
                }
                // labels of the segment's layers, from its checkpoint
                {
                    float f[W];
#pragma unroll
                    for (int v = 0; v < W; ++v) f[v] = cp[(s * W + v) * kTile];
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        if (c < kk) {
                            uint32_t cd[W];
                            load_codes<W>(tpl + (t0 + c) * W, cd);
                            float nf[W];
#pragma unroll
                            for (int v = 0; v < W; ++v) { Sg[c][v] = f[v]; nf[v] = finf(); }
#pragma unroll
                            for (int v = 0; v < W; ++v) {
                                push<W>(nf, cd[v] & 0xFFu, f[v]);
                                push<W>(nf, cd[v] >> 8, f[v] + L[c]);
                            }
#pragma unroll
                            for (int v = 0; v < W; ++v) f[v] = nf[v];
                        }
                    }
                }
#pragma unroll
                for (int cc = C - 1; cc >= 0; --cc) {
                    if (cc < kk) {
                        uint32_t cd[W];
                        load_codes<W>(tpl + (t0 + cc) * W, cd);
                        float m0 = finf(), m1 = finf();
#pragma unroll
                        for (int v = 0; v < W; ++v) {
                            const float fv = Sg[cc][v];
                            m0 = fminf(m0, fv + pick<W>(b, cd[v] & 0xFFu));
                            m1 = fminf(m1, fv + pick<W>(b, cd[v] >> 8));
                        }
                        const float lt = L[cc];
                        m1 += lt;
                        const float d = m1 - m0;
                        const float lt_new = fmaf(-omega, d, lt) + Tt[cc];  // Eq. 5
                        L[cc] = lt_new;
                        negsum += fmaxf(-d, 0.f);
                        float nb[W];
#pragma unroll
                        for (int v = 0; v < W; ++v)
                            nb[v] = fminf(pick<W>(b, cd[v] & 0xFFu), pick<W>(b, cd[v] >> 8) + lt_new);
#pragma unroll
                        for (int v = 0; v < W; ++v) b[v] = nb[v];
                    }
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    if (c < kk) {
                        if (valid) lam[base + static_cast<size_t>(t0 + c) * kTile] = L[c];
                        if (local) ep_lam[(t0 + c) * kTile + lane] = L[c];
                    }
                }
            }
            term = fmaf(-omega, negsum, b[0]);
        }

        if constexpr (update) {
            if (local) {
                __syncwarp();
                tile_local_sums(I, tile.pattern, ep_lam, ep_var, lane);
                __syncwarp();
            }
        }

        if constexpr (MODE == kBwdUpdate || MODE == kEval) {  // the passes whose bound is reduced
            float s = valid ? term : 0.f, comp = 0.f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float o = __shfl_xor_sync(kFull, s, off);
                const float oc = __shfl_xor_sync(kFull, comp, off);
                const float sum = s + o;
                const float bp = sum - s;
                const float err = (s - (sum - bp)) + (o - bp);
                s = sum;
                comp = comp + oc + err;
            }
            if (lane == 0) I->tile_lb[__ldg(a.first + ii) + (g - __ldg(a.prefix + ii))] = make_float2(s, comp);
        }
    }
}

template <int W, int MODE>
__global__ void __launch_bounds__(256) sweep_seg_kernel(SweepArgs a) {
    extern __shared__ float smem[];
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    float* wsm = smem + static_cast<size_t>(wib) * seg_warp_floats<W>(a);
    for (int g = blockIdx.x * wpb + wib; g < a.total; g += gridDim.x * wpb)
        seg_tile<W, MODE>(a, g, g + gridDim.x * wpb, wsm, lane);
}

#undef FD_UP
#undef FD_DOWN

}  // namespace dev

// a kernel launch with programmatic stream serialization (the kernel calls
// pdl_wait before it touches memory) and an optional L2 access-policy window
// (kernels.cu)
cudaError_t launch_windowed(const void* fn, int blocks, int threads, void** args, size_t smem, cudaStream_t s,
                            const L2Window& l2);

// host-side dispatch of one width's instantiations (defined in sweep_w<W>.cu)
template <int W>
cudaError_t launch_sweep_width(bool reg, int mode, int blocks, int threads, size_t smem, cudaStream_t s,
                               const SweepArgs& a, const L2Window& l2);

#define FDOG_DEFINE_SWEEP_WIDTH(W, HAS_REG)                                                                    \
    template <>                                                                                                \
    cudaError_t launch_sweep_width<W>(bool reg, int mode, int blocks, int threads, size_t smem, cudaStream_t s, \
                                      const SweepArgs& a, const L2Window& l2) {                                \
        void (*fn)(SweepArgs) = nullptr;                                                                       \
        if (HAS_REG && reg) {                                                                                  \
            fn = mode == kFwdUpdate ? dev::sweep_kernel<W, HAS_REG, kFwdUpdate>                                \
               : mode == kBwdUpdate ? dev::sweep_kernel<W, HAS_REG, kBwdUpdate>                                \
               : mode == kMinMarg   ? dev::sweep_kernel<W, HAS_REG, kMinMarg>                                  \
                                    : dev::sweep_kernel<W, HAS_REG, kEval>;                                    \
        } else if (HAS_REG) {                                                                                  \
            fn = mode == kFwdUpdate ? dev::sweep_seg_kernel<W, kFwdUpdate>                                     \
               : mode == kBwdUpdate ? dev::sweep_seg_kernel<W, kBwdUpdate>                                     \
               : mode == kMinMarg   ? dev::sweep_seg_kernel<W, kMinMarg>                                       \
                                    : dev::sweep_seg_kernel<W, kEval>;                                         \
        } else {                                                                                               \
            fn = mode == kFwdUpdate ? dev::sweep_kernel<W, false, kFwdUpdate>                                  \
               : mode == kBwdUpdate ? dev::sweep_kernel<W, false, kBwdUpdate>                                  \
               : mode == kMinMarg   ? dev::sweep_kernel<W, false, kMinMarg>                                    \
                                    : dev::sweep_kernel<W, false, kEval>;                                      \
        }                                                                                                      \
        if (smem > 48 * 1024) {                                                                                \
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                                                 static_cast<int>(smem));                                      \
            if (e != cudaSuccess) return e;                                                                    \
        }                                                                                                      \
        void* args[] = {const_cast<SweepArgs*>(&a)};                                                           \
        return launch_windowed(reinterpret_cast<const void*>(fn), blocks, threads, args, smem, s, l2);         \
    }

}  // namespace fdog
