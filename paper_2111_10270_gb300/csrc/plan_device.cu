// Device-side construction of the decomposition: the same plan as the host
// builder (bdd_build.cpp) -- BDDs per row (Ex. 1, Def. 4) shared per row
// signature, tiles of kTile BDDs, interleaved slots, per-variable slot lists,
// tile-local variables and the deferred-sum buckets -- computed by
// data-parallel kernels on the instance's stream.
//
//  1. signatures: a thread per row hashes (sense, rhs, length, coefficients)
//     and checks that the row is sorted with non-zero coefficients;
//  2. rows with equal hashes meet in an open-addressing table whose slot keeps
//     the smallest row index (the group's representative); every row is then
//     compared with its representative entry by entry, so a hash collision
//     cannot merge different rows;
//  3. the host builds the BDD of each representative (a handful per instance)
//     and picks its kernel class; a stable multi-split (per-chunk histograms,
//     per-key scans, warp-level ranks with __match_any_sync) gives every row
//     its place in the layout order (class, shape, row);
//  4. a thread per row writes its variables into its interleaved slots;
//  5. copies are counted per variable, scanned into csr_off, scattered, and
//     each copy finds its rank among its variable's copies (ascending slots);
//  6. a warp per tile finds its tile-local variables in ascending slot order;
//     equal patterns are merged through a second table, first tile first;
//  7. the other variables are split by copy count into the deferred-sum
//     buckets (the same multi-split) and their slot positions transposed.
//
// An instance whose planning needs the host presolve (a row that forces a
// variable or accepts every assignment, an empty, unsorted or zero-coefficient
// row), has more than kMaxDevShapes distinct row signatures, or a variable
// with more than kMaxDevCopies copies, is left to the host builder, which
// gives the same plan.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <limits>
#include <vector>

#include "fdog_internal.h"
#include "instance.h"

namespace fdog {

namespace {

constexpr int kMaxDevShapes = 1024;   // distinct row signatures (also the multi-split's key bound)
constexpr int kMaxDevCopies = 4096;   // copies of one variable the slot-list ranking takes
constexpr int kSplitChunk = 1024;     // items per warp in the multi-split
constexpr int kSplitWarps = 4;        // warps per block of the multi-split
constexpr int kScanBlock = 1024;
constexpr unsigned kFull = 0xFFFFFFFFu;

// reasons to leave the instance to the host builder (PlanFlags::host bits)
constexpr int kHostRows = 1;       // empty, unsorted or zero-coefficient row
constexpr int kHostTable = 2;      // hash table full (cannot happen at load <= 1/2)
constexpr int kHostShapes = 4;     // more than kMaxDevShapes signatures
constexpr int kHostCollision = 8;  // two different rows (or patterns) with one hash
constexpr int kHostCopies = 16;    // a variable with more than kMaxDevCopies copies

struct PlanFlags {
    int32_t host;
    int32_t n_reps;
    int32_t n_outside;  // variables in no row
    int32_t pad;
    unsigned long long n_local;
    unsigned long long overflow_slots;
};

// SplitMix64 finaliser (Steele, Lea, Flood 2014) as the mixing step of the hashes
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

// ---- 1-2: row signatures and their representatives ------------------------

__global__ void row_signature_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     const int32_t* __restrict__ coef, const int8_t* __restrict__ sense,
                                     const int64_t* __restrict__ rhs, int32_t n_rows, uint64_t* __restrict__ key,
                                     PlanFlags* f) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_rows) return;
    const int64_t b = row_ptr[j], e = row_ptr[j + 1];
    uint64_t h = mix64(static_cast<uint64_t>(static_cast<int64_t>(sense[j]) + 2));
    h = mix64(h ^ static_cast<uint64_t>(rhs[j]));
    h = mix64(h ^ static_cast<uint64_t>(e - b));
    bool ok = e > b;
    int32_t prev = -1;
    for (int64_t q = b; q < e; ++q) {
        const int32_t c = col[q], a = coef[q];
        ok = ok && a != 0 && c > prev;
        prev = c;
        h = mix64(h ^ static_cast<uint32_t>(a));
    }
    if (!ok) atomicOr(&f->host, kHostRows);
    key[j] = h ? h : 1;
}

// Items with key 0 take no slot.  tval keeps the smallest item of each key.
// Lanes of a warp with equal keys insert once (their lowest lane, which holds
// the smallest item), and a slot is read before it is touched atomically, so
// that millions of rows sharing a handful of signatures do not serialise on
// one address.
__global__ void key_insert_kernel(const uint64_t* __restrict__ key, int32_t n, unsigned long long* tkey,
                                  int32_t* tval, int32_t* __restrict__ slot_of, uint32_t mask, PlanFlags* f) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned long long k = i < n ? key[i] : 0ull;
    const unsigned peers = __match_any_sync(kFull, k);
    const int leader = __ffs(peers) - 1;
    int32_t slot = -1;
    if (k != 0ull && lane == leader) {
        uint32_t s = static_cast<uint32_t>(k >> 20) & mask;
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(&tkey[s]);
            if (cur == 0ull) {
                cur = atomicCAS(&tkey[s], 0ull, k);
                if (cur == 0ull) cur = k;
            }
            if (cur == k) {
                // values only decrease, so a stale read is never below the current minimum
                if (i < *reinterpret_cast<volatile int32_t*>(&tval[s])) atomicMin(&tval[s], i);
                slot = static_cast<int32_t>(s);
                break;
            }
            s = (s + 1) & mask;
        }
        if (slot < 0) atomicOr(&f->host, kHostTable);
    }
    slot = __shfl_sync(kFull, slot, leader);
    if (i < n) slot_of[i] = k != 0ull ? slot : -1;
}

__global__ void row_verify_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ coef,
                                  const int8_t* __restrict__ sense, const int64_t* __restrict__ rhs,
                                  int32_t n_rows, const int32_t* __restrict__ slot_of,
                                  const int32_t* __restrict__ tval, int32_t* reps, PlanFlags* f) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_rows) return;
    const int32_t s = slot_of[j];
    if (s < 0) return;
    const int32_t r = tval[s];
    if (r == j) {
        const int32_t q = atomicAdd(&f->n_reps, 1);
        if (q < kMaxDevShapes) reps[q] = j;
        else atomicOr(&f->host, kHostShapes);
        return;
    }
    const int64_t bj = row_ptr[j], ej = row_ptr[j + 1], br = row_ptr[r], er = row_ptr[r + 1];
    bool same = sense[j] == sense[r] && rhs[j] == rhs[r] && ej - bj == er - br;
    for (int64_t q = 0; same && q < ej - bj; ++q) same = coef[bj + q] == coef[br + q];
    if (!same) atomicOr(&f->host, kHostCollision);
}

// id of every representative's slot (reps sorted ascending: ids in first-occurrence order)
__global__ void rep_ids_kernel(const int32_t* __restrict__ reps, int32_t n_reps, const int32_t* __restrict__ slot_of,
                               int32_t* __restrict__ tid) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n_reps) tid[slot_of[reps[r]]] = r;
}

__global__ void item_ids_kernel(int32_t n, const int32_t* __restrict__ slot_of, const int32_t* __restrict__ tid,
                                int32_t* __restrict__ id) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t s = slot_of[i];
    id[i] = s >= 0 ? tid[s] : -1;
}

// ---- stable multi-split ----------------------------------------------------
// keys[i] in [0, ns) or -1 (left out).  Chunk c holds items
// [c kSplitChunk, (c + 1) kSplitChunk), one warp per chunk, visited 32 at a
// time in index order.  RANK = false: hist[s][c] = items of key s in chunk c.
// RANK = true (hist scanned per key): out[i] = base[s] + items of key s
// before i, -1 for left-out items.
template <bool RANK>
__global__ void __launch_bounds__(kSplitWarps * 32) split_kernel(const int32_t* __restrict__ keys, int64_t n, int ns,
                                                                 int32_t nchunks, int32_t* __restrict__ hist,
                                                                 const int32_t* __restrict__ base,
                                                                 int32_t* __restrict__ out) {
    __shared__ int32_t cnt[kSplitWarps][kMaxDevShapes];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t c = blockIdx.x * kSplitWarps + w;
    if (c >= nchunks) return;  // warp-level work only: no block barrier below
    int32_t* my = cnt[w];
    for (int s = lane; s < ns; s += 32) my[s] = 0;
    __syncwarp();
    const int64_t i0 = static_cast<int64_t>(c) * kSplitChunk;
    for (int step = 0; step < kSplitChunk / 32; ++step) {
        const int64_t i = i0 + step * 32 + lane;
        const int32_t k = i < n ? keys[i] : -1;
        const unsigned peers = __match_any_sync(kFull, k);
        const int before = __popc(peers & lanemask_lt());
        if (RANK && i < n) out[i] = k >= 0 ? base[k] + hist[static_cast<int64_t>(k) * nchunks + c] + my[k] + before : -1;
        __syncwarp();
        if (k >= 0 && before == 0) my[k] += __popc(peers);
        __syncwarp();
    }
    if (!RANK)
        for (int s = lane; s < ns; s += 32) hist[static_cast<int64_t>(s) * nchunks + c] = my[s];
}

// inclusive block-wide scan of one value per thread (blockDim.x == kScanBlock)
__device__ int32_t block_scan_incl(int32_t v, int32_t* warp_sums) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
        int32_t s = warp_sums[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(kFull, s, d);
            if (lane >= d) s += o;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int32_t r = v + (w > 0 ? warp_sums[w - 1] : 0);
    __syncthreads();
    return r;
}

// per key (block): exclusive scan over its chunks, total into totals[s]
__global__ void __launch_bounds__(kScanBlock) split_scan_kernel(int32_t* __restrict__ hist, int32_t nchunks,
                                                                int32_t* __restrict__ totals) {
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry_sh;
    int32_t* h = hist + static_cast<int64_t>(blockIdx.x) * nchunks;
    if (threadIdx.x == 0) carry_sh = 0;
    __syncthreads();
    for (int32_t b = 0; b < nchunks; b += kScanBlock) {
        const int32_t i = b + threadIdx.x;
        const int32_t v = i < nchunks ? h[i] : 0;
        const int32_t incl = block_scan_incl(v, warp_sums);
        const int32_t carry = carry_sh;
        if (i < nchunks) h[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry_sh = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry_sh;
}

// ---- device-wide exclusive scan (in place) ---------------------------------
__global__ void __launch_bounds__(kScanBlock) scan_block_kernel(int32_t* __restrict__ d, int64_t n,
                                                                int32_t* __restrict__ bsum) {
    __shared__ int32_t warp_sums[32];
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanBlock + threadIdx.x;
    const int32_t v = i < n ? d[i] : 0;
    const int32_t incl = block_scan_incl(v, warp_sums);
    if (i < n) d[i] = incl - v;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = incl;
}

__global__ void __launch_bounds__(kScanBlock) scan_add_kernel(int32_t* __restrict__ d, int64_t n,
                                                              const int32_t* __restrict__ bsum) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanBlock + threadIdx.x;
    if (i < n) d[i] += bsum[blockIdx.x];
}

// ---- 4: slots ----------------------------------------------------------------
struct ShapePlace {
    int32_t bdd_base;    // first BDD of the shape in layout order
    int32_t slot_first;  // slot_base of its first tile
    int32_t k;
    int32_t pad;
};

__global__ void row_place_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                 int32_t n_rows, const int32_t* __restrict__ shape_of,
                                 const int32_t* __restrict__ pos, const ShapePlace* __restrict__ place,
                                 int32_t* __restrict__ var, int32_t* __restrict__ bdd_row) {
    const int32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_rows) return;
    const int32_t b = pos[j];
    const ShapePlace sp = place[shape_of[j]];
    const int32_t r = b - sp.bdd_base;
    const int64_t slot0 = static_cast<int64_t>(sp.slot_first) + static_cast<int64_t>(r >> 5) * sp.k * kTile + (r & 31);
    bdd_row[b] = j;
    const int64_t q0 = row_ptr[j];
    for (int t = 0; t < sp.k; ++t) var[slot0 + static_cast<int64_t>(t) * kTile] = col[q0 + t];
}

// ---- 5: per-variable slot lists ----------------------------------------------
__global__ void slot_count_kernel(const int32_t* __restrict__ var, int64_t S, int32_t* __restrict__ cnt,
                                  PlanFlags* f) {
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= S) return;
    const int32_t v = var[p];
    if (v < 0) return;
    if (atomicAdd(&cnt[v], 1) + 1 > kMaxDevCopies) atomicOr(&f->host, kHostCopies);
}

__global__ void outside_count_kernel(const int32_t* __restrict__ cnt, int32_t n, PlanFlags* f) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const int zeros = __syncthreads_count(i < n && cnt[i] == 0);
    if (threadIdx.x == 0 && zeros) atomicAdd(&f->n_outside, zeros);
}

__global__ void slot_scatter_kernel(const int32_t* __restrict__ var, int64_t S, const int32_t* __restrict__ off,
                                    int32_t* __restrict__ fill, int32_t* __restrict__ tmp) {
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= S) return;
    const int32_t v = var[p];
    if (v >= 0) tmp[off[v] + atomicAdd(&fill[v], 1)] = static_cast<int32_t>(p);
}

// each copy's rank among its variable's copies (slot positions are distinct)
__global__ void slot_rank_kernel(const int32_t* __restrict__ var, int64_t S, const int32_t* __restrict__ off,
                                 const int32_t* __restrict__ tmp, int32_t* __restrict__ pos) {
    const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= S) return;
    const int32_t v = var[p];
    if (v < 0) return;
    const int32_t b = off[v], e = off[v + 1];
    int32_t r = 0;
    for (int32_t q = b; q < e; ++q) r += tmp[q] < p;
    pos[b + r] = static_cast<int32_t>(p);
}

// ---- 6: tile-local variables -----------------------------------------------
// A variable is tile-local when all of its (at most four) copies lie in one
// tile of a row of at most kEpiMaxK layers; it is listed at its first copy.
// FILL: writes the entries and the tile's key, a sum over its entries of
// mix64(index, value) (order-dependent through the index; equal keys are
// verified entry by entry afterwards), 0 for a tile without entries.
template <bool FILL>
__global__ void tile_local_kernel(const TileDev* __restrict__ tiles, const int32_t* __restrict__ shape_k,
                                  int32_t nt, const int32_t* __restrict__ var, const int32_t* __restrict__ off,
                                  const int32_t* __restrict__ pos, int32_t* __restrict__ ent_cnt,
                                  const int32_t* __restrict__ ent_off, uint16_t* __restrict__ ents,
                                  uint8_t* __restrict__ local, uint64_t* __restrict__ key) {
    const int32_t ti = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ti >= nt) return;
    const TileDev t = tiles[ti];
    const int k = shape_k[t.shape];
    int32_t m = 0;
    uint64_t h = 0;
    if (k <= kEpiMaxK) {
        const int64_t lo = t.slot_base, hi = lo + static_cast<int64_t>(k) * kTile;
        for (int layer = 0; layer < k; ++layer) {
            const int64_t p = lo + static_cast<int64_t>(layer) * kTile + lane;
            const int32_t v = var[p];
            int32_t b = 0, c = 0;
            bool hit = false;
            if (v >= 0) {
                b = off[v];
                c = off[v + 1] - b;
                hit = c <= 4 && pos[b] == p && pos[b + c - 1] < hi;
            }
            const unsigned bal = __ballot_sync(kFull, hit);
            if (FILL && hit) {
                const int32_t idx = 4 * (m + __popc(bal & lanemask_lt()));
                uint16_t* dst = ents + ent_off[ti] + idx;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint16_t e = q < c ? static_cast<uint16_t>(pos[b + q] - lo) : uint16_t(0xFFFF);
                    dst[q] = e;
                    h += mix64((static_cast<uint64_t>(idx + q) << 16) | e);
                }
                local[v] = 1;
            }
            m += __popc(bal);
        }
    }
    if (!FILL && lane == 0) ent_cnt[ti] = 4 * m;
    if (FILL) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) h += __shfl_xor_sync(kFull, h, d);
        if (lane == 0) {
            h = m ? mix64(h ^ static_cast<uint64_t>(m)) : 0ull;
            key[ti] = m && h == 0ull ? 1ull : h;
        }
    }
}

// a warp per tile: representative tiles are listed, the others compared with theirs
__global__ void tile_verify_kernel(const int32_t* __restrict__ ent_off, int32_t nt, const uint16_t* __restrict__ ents,
                                   const int32_t* __restrict__ slot_of, const int32_t* __restrict__ tval,
                                   int32_t* reps, PlanFlags* f) {
    const int32_t ti = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ti >= nt) return;
    const int32_t s = slot_of[ti];
    if (s < 0) return;
    const int32_t r = tval[s];
    if (r == ti) {
        if (lane == 0) reps[atomicAdd(&f->n_reps, 1)] = ti;  // at most nt representatives
        return;
    }
    const int32_t len = ent_off[ti + 1] - ent_off[ti];
    bool same = len == ent_off[r + 1] - ent_off[r];
    for (int32_t q = lane; same && q < len; q += 32) same = ents[ent_off[ti] + q] == ents[ent_off[r] + q];
    if (!same) atomicOr(&f->host, kHostCollision);
}

// entries of pattern p (representative tile reps[p]) to local_ent at first[p] (uint16 units)
__global__ void pattern_gather_kernel(const int32_t* __restrict__ reps, const int32_t* __restrict__ first,
                                      int32_t n_pat, const int32_t* __restrict__ ent_off,
                                      const uint16_t* __restrict__ ents, uint16_t* __restrict__ local_ent) {
    const int32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n_pat) return;
    const int32_t b = ent_off[reps[p]], len = ent_off[reps[p] + 1] - b;
    for (int32_t q = lane; q < len; q += 32) local_ent[first[p] + q] = ents[b + q];
}

// ---- 7: deferred-sum buckets -------------------------------------------------
struct Buckets {
    int32_t start[FDOG_WBUCKETS + 1];
    int32_t pos[FDOG_WBUCKETS];
    int32_t count[FDOG_WBUCKETS];
};

__global__ void var_bucket_kernel(const int32_t* __restrict__ off, int32_t n, const uint8_t* __restrict__ local,
                                  int32_t* __restrict__ key, PlanFlags* f) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t k = -1, c = 0;
    bool loc = false;
    if (i < n) {
        c = off[i + 1] - off[i];
        loc = local[i] != 0;
        if (!loc && c > 0) k = min(c, FDOG_WBUCKETS) - 1;
        key[i] = k;
    }
    const int n_loc = __syncthreads_count(loc);
    if (threadIdx.x == 0 && n_loc) atomicAdd(&f->n_local, static_cast<unsigned long long>(n_loc));
    if (k == FDOG_WBUCKETS - 1) atomicAdd(&f->overflow_slots, static_cast<unsigned long long>(c));
}

__global__ void work_fill_kernel(const int32_t* __restrict__ off, const int32_t* __restrict__ csr_pos, int32_t n,
                                 const int32_t* __restrict__ key, const int32_t* __restrict__ wp, Buckets bk,
                                 int32_t* __restrict__ work, int32_t* __restrict__ wpos) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t p = wp[i];
    if (p < 0) return;
    work[p] = i;
    const int32_t b = key[i];
    if (b >= FDOG_WBUCKETS - 1) return;
    const int32_t nb = bk.count[b], jj = p - bk.start[b];
    for (int q = 0; q <= b; ++q) wpos[bk.pos[b] + static_cast<int64_t>(q) * nb + jj] = csr_pos[off[i] + q];
}

// ---- host side -----------------------------------------------------------------

inline unsigned grid_of(int64_t n, int threads) { return static_cast<unsigned>((n + threads - 1) / threads); }

// stream-ordered temporaries of one planning call
struct Scratch {
    cudaStream_t s;
    std::vector<void*> ptrs;
    cudaError_t err = cudaSuccess;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <class T>
    T* get(int64_t count) {
        void* p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = cudaMallocAsync(&p, static_cast<size_t>(std::max<int64_t>(count, 1)) * sizeof(T), s);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
};

// in-place exclusive scan of d[0, n) on the device (values and total fit int32)
cudaError_t device_scan(int32_t* d, int64_t n, Scratch& sc) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int32_t* bsum = sc.get<int32_t>(nb);
    if (!bsum) return sc.err;
    scan_block_kernel<<<static_cast<unsigned>(nb), kScanBlock, 0, sc.s>>>(d, n, bsum);
    if (nb > 1) {
        cudaError_t e = device_scan(bsum, nb, sc);
        if (e != cudaSuccess) return e;
        scan_add_kernel<<<static_cast<unsigned>(nb), kScanBlock, 0, sc.s>>>(d, n, bsum);
    }
    return cudaGetLastError();
}

// stable multi-split of keys[0, n) into ns groups: totals[s] (host) and the
// destination of every item (device), the groups placed at base[s]
cudaError_t device_split(const int32_t* keys, int64_t n, int ns, Scratch& sc, std::vector<int32_t>& totals,
                         const std::vector<int32_t>* base_or_null, int32_t* out, int32_t** hist_io) {
    const int32_t nchunks = static_cast<int32_t>((n + kSplitChunk - 1) / kSplitChunk);
    const unsigned blocks = grid_of(nchunks, kSplitWarps);
    cudaError_t e;
    if (!base_or_null) {
        int32_t* hist = sc.get<int32_t>(static_cast<int64_t>(ns) * nchunks);
        int32_t* tot = sc.get<int32_t>(ns);
        if (!hist || !tot) return sc.err;
        split_kernel<false><<<blocks, kSplitWarps * 32, 0, sc.s>>>(keys, n, ns, nchunks, hist, nullptr, nullptr);
        split_scan_kernel<<<ns, kScanBlock, 0, sc.s>>>(hist, nchunks, tot);
        totals.assign(ns, 0);
        if ((e = cudaMemcpyAsync(totals.data(), tot, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, sc.s)) != cudaSuccess)
            return e;
        *hist_io = hist;
        return cudaStreamSynchronize(sc.s);
    }
    int32_t* base = sc.get<int32_t>(ns);
    if (!base) return sc.err;
    if ((e = cudaMemcpyAsync(base, base_or_null->data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, sc.s)) !=
        cudaSuccess)
        return e;
    split_kernel<true><<<blocks, kSplitWarps * 32, 0, sc.s>>>(keys, n, ns, nchunks, *hist_io, base, out);
    return cudaGetLastError();
}

uint32_t table_mask(int64_t items) {
    uint32_t size = 1024;
    while (size < 2 * items) size <<= 1;
    return size - 1;
}

constexpr int kLeaveToHost = 1;  // positive: not a failure, the host builder plans the instance

#define PLAN_CHECK(expr)                          \
    do {                                          \
        cudaError_t e_ = (expr);                  \
        if (e_ != cudaSuccess) return fail(e_);   \
    } while (0)

}  // namespace

void free_device_plan(Decomposition& d, cudaStream_t s) {
    for (void* p : {static_cast<void*>(d.d_var), static_cast<void*>(d.d_csr_off), static_cast<void*>(d.d_csr_pos),
                    static_cast<void*>(d.d_work), static_cast<void*>(d.d_wpos), static_cast<void*>(d.d_local_ent),
                    static_cast<void*>(d.d_bdd_row)})
        if (p) cudaFreeAsync(p, s);
    d.d_var = d.d_csr_off = d.d_csr_pos = d.d_work = d.d_wpos = d.d_bdd_row = nullptr;
    d.d_local_ent = nullptr;
}

// Returns FDOG_OK (inst->dec planned, its large arrays in dec.d_*),
// kLeaveToHost, or an FDOG_* error.
int plan_on_device(fdog_instance* inst, int jit_mode, bool fuse_local) {
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = inst->stream;
    Decomposition& out = inst->dec;
    free_device_plan(out, st);
    out = Decomposition();
    const int32_t R = inst->n_rows, n = inst->n_vars;
    const int64_t nnz = inst->row_ptr[R];
    // (the hash tables hold twice the rows in 32-bit slot indices)
    if (R <= 0 || R > (1 << 28) || n <= 0 || 4 * static_cast<int64_t>(n) >= std::numeric_limits<int32_t>::max())
        return kLeaveToHost;
    Scratch sc(st);
    auto fail = [&](cudaError_t e) {
        free_device_plan(out, st);
        cudaGetLastError();
        return fail_cuda(inst, e, "device planning");
    };
    auto leave = [&]() {
        free_device_plan(out, st);
        out = Decomposition();
        return kLeaveToHost;
    };

    // raw rows on the device
    int64_t* d_row_ptr = sc.get<int64_t>(R + 1);
    int32_t* d_col = sc.get<int32_t>(nnz);
    int32_t* d_coef = sc.get<int32_t>(nnz);
    int8_t* d_sense = sc.get<int8_t>(R);
    int64_t* d_rhs = sc.get<int64_t>(R);
    PlanFlags* d_f = sc.get<PlanFlags>(1);
    if (sc.err != cudaSuccess) return fail(sc.err);
    PLAN_CHECK(copy_async(inst, d_row_ptr, inst->row_ptr.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice));
    PLAN_CHECK(copy_async(inst, d_col, inst->col.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    PLAN_CHECK(copy_async(inst, d_coef, inst->coef.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    PLAN_CHECK(copy_async(inst, d_sense, inst->sense.data(), R, cudaMemcpyHostToDevice));
    PLAN_CHECK(copy_async(inst, d_rhs, inst->rhs.data(), sizeof(int64_t) * R, cudaMemcpyHostToDevice));
    PLAN_CHECK(cudaMemsetAsync(d_f, 0, sizeof(PlanFlags), st));
    PlanFlags hf{};
    auto read_flags = [&]() {
        cudaError_t e = cudaMemcpyAsync(&hf, d_f, sizeof(PlanFlags), cudaMemcpyDeviceToHost, st);
        return e != cudaSuccess ? e : cudaStreamSynchronize(st);
    };

    // 1-2: signatures and representatives
    const uint32_t rmask = table_mask(R);
    uint64_t* d_key = sc.get<uint64_t>(R);
    unsigned long long* d_tkey = sc.get<unsigned long long>(static_cast<int64_t>(rmask) + 1);
    int32_t* d_tval = sc.get<int32_t>(static_cast<int64_t>(rmask) + 1);
    int32_t* d_tid = sc.get<int32_t>(static_cast<int64_t>(rmask) + 1);
    int32_t* d_slot_of = sc.get<int32_t>(R);
    int32_t* d_reps = sc.get<int32_t>(kMaxDevShapes);
    int32_t* d_shape_of = sc.get<int32_t>(R);
    if (sc.err != cudaSuccess) return fail(sc.err);
    PLAN_CHECK(cudaMemsetAsync(d_tkey, 0, sizeof(unsigned long long) * (static_cast<size_t>(rmask) + 1), st));
    PLAN_CHECK(cudaMemsetAsync(d_tval, 0x7F, sizeof(int32_t) * (static_cast<size_t>(rmask) + 1), st));
    row_signature_kernel<<<grid_of(R, 256), 256, 0, st>>>(d_row_ptr, d_col, d_coef, d_sense, d_rhs, R, d_key, d_f);
    key_insert_kernel<<<grid_of(R, 256), 256, 0, st>>>(d_key, R, d_tkey, d_tval, d_slot_of, rmask, d_f);
    row_verify_kernel<<<grid_of(R, 256), 256, 0, st>>>(d_row_ptr, d_coef, d_sense, d_rhs, R, d_slot_of, d_tval,
                                                         d_reps, d_f);
    PLAN_CHECK(cudaGetLastError());
    PLAN_CHECK(read_flags());
    if (hf.host) return leave();
    const int ns = hf.n_reps;
    std::vector<int32_t> reps(ns);
    PLAN_CHECK(cudaMemcpyAsync(reps.data(), d_reps, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, st));
    PLAN_CHECK(cudaStreamSynchronize(st));
    std::sort(reps.begin(), reps.end());

    // the BDD of each signature (host), in first-occurrence order
    std::vector<HostShape> shapes(ns);
    for (int s = 0; s < ns; ++s) {
        const int32_t j = reps[s];
        std::vector<int64_t> a(inst->coef.begin() + inst->row_ptr[j], inst->coef.begin() + inst->row_ptr[j + 1]);
        bool presolve = false;
        if (analyse_row(a, inst->sense[j], inst->rhs[j], shapes[s], presolve) != FDOG_OK || presolve) return leave();
    }
    PLAN_CHECK(cudaMemcpyAsync(d_reps, reps.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    rep_ids_kernel<<<grid_of(ns, 256), 256, 0, st>>>(d_reps, ns, d_slot_of, d_tid);
    item_ids_kernel<<<grid_of(R, 256), 256, 0, st>>>(R, d_slot_of, d_tid, d_shape_of);
    PLAN_CHECK(cudaGetLastError());
    std::vector<int32_t> count;
    int32_t* d_hist = nullptr;
    PLAN_CHECK(device_split(d_shape_of, R, ns, sc, count, nullptr, nullptr, &d_hist));

    // classes, layout order (class, shape), tiles
    out.fixed.assign(n, -1);
    out.shapes = std::move(shapes);
    out.shape_cls.resize(ns);
    for (int s = 0; s < ns; ++s)
        if ((out.shape_cls[s] = shape_class(out.shapes[s], jit_mode, count[s])) < 0) return leave();
    std::vector<int> order(ns);
    for (int s = 0; s < ns; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return out.shape_cls[x] < out.shape_cls[y]; });
    std::vector<int32_t> bdd_base(ns, 0);
    std::vector<ShapePlace> place(ns);
    out.cls_tile_begin.assign(kNumClasses + 1, 0);
    int64_t slot = 0, bdd = 0;
    for (int s : order) {
        const int k = out.shapes[s].k;
        bdd_base[s] = static_cast<int32_t>(bdd);
        place[s] = {static_cast<int32_t>(bdd), static_cast<int32_t>(slot), k, 0};
        for (int32_t q = 0; q < count[s]; q += kTile) {
            TileDev t{s, static_cast<int32_t>(slot), std::min<int32_t>(kTile, count[s] - q), static_cast<int32_t>(bdd + q),
                      -1, {0, 0, 0}};
            out.tiles.push_back(t);
            out.cls_tile_begin[out.shape_cls[s] + 1]++;
            out.kmax[out.shape_cls[s]] = std::max(out.kmax[out.shape_cls[s]], k);
            slot += static_cast<int64_t>(k) * kTile;
            if (slot > std::numeric_limits<int32_t>::max()) return leave();  // the host builder reports it
        }
        bdd += count[s];
        out.n_nodes += static_cast<int64_t>(count[s]) * out.shapes[s].lstart.back();
    }
    for (int c = 0; c < kNumClasses; ++c) out.cls_tile_begin[c + 1] += out.cls_tile_begin[c];
    out.slots_pad = slot;
    out.n_bdds = bdd;
    build_templates(out);
    const int64_t S = slot;
    const int32_t nt = static_cast<int32_t>(out.tiles.size());

    // 3-4: ranks within shapes, slots
    int32_t* d_pos = sc.get<int32_t>(R);
    ShapePlace* d_place = sc.get<ShapePlace>(ns);
    cudaError_t ae = sc.err;
    if (ae == cudaSuccess) ae = cudaMallocAsync(&out.d_var, sizeof(int32_t) * std::max<int64_t>(S, 1), st);
    if (ae == cudaSuccess) ae = cudaMallocAsync(&out.d_bdd_row, sizeof(int32_t) * std::max<int64_t>(bdd, 1), st);
    if (ae == cudaSuccess) ae = cudaMallocAsync(&out.d_csr_off, sizeof(int32_t) * (static_cast<size_t>(n) + 1), st);
    if (ae != cudaSuccess) return fail(ae);
    PLAN_CHECK(device_split(d_shape_of, R, ns, sc, count, &bdd_base, d_pos, &d_hist));
    PLAN_CHECK(cudaMemcpyAsync(d_place, place.data(), sizeof(ShapePlace) * ns, cudaMemcpyHostToDevice, st));
    PLAN_CHECK(cudaMemsetAsync(out.d_var, 0xFF, sizeof(int32_t) * S, st));
    row_place_kernel<<<grid_of(R, 256), 256, 0, st>>>(d_row_ptr, d_col, R, d_shape_of, d_pos, d_place, out.d_var,
                                                        out.d_bdd_row);
    PLAN_CHECK(cudaGetLastError());

    // 5: per-variable slot lists
    int32_t* cnt = out.d_csr_off;
    PLAN_CHECK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (static_cast<size_t>(n) + 1), st));
    slot_count_kernel<<<grid_of(S, 256), 256, 0, st>>>(out.d_var, S, cnt, d_f);
    outside_count_kernel<<<grid_of(n, 256), 256, 0, st>>>(cnt, n, d_f);
    PLAN_CHECK(cudaGetLastError());
    PLAN_CHECK(read_flags());
    if (hf.host) return leave();
    if (hf.n_outside > 0) {
        // variables in no row: fixed outside the BDDs (same loop as the host builder)
        std::vector<int32_t> c(n);
        PLAN_CHECK(cudaMemcpyAsync(c.data(), cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
        PLAN_CHECK(cudaStreamSynchronize(st));
        for (int32_t i = 0; i < n; ++i)
            if (c[i] == 0) {
                out.fixed[i] = 2;
                out.const_lb += std::min(inst->cost[i], 0.0);
                out.outside.push_back(i);
            }
    }
    out.const_obj = out.const_lb;
    PLAN_CHECK(device_scan(cnt, static_cast<int64_t>(n) + 1, sc));
    int32_t n_slots = 0;
    PLAN_CHECK(cudaMemcpyAsync(&n_slots, cnt + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PLAN_CHECK(cudaStreamSynchronize(st));
    out.n_slots = n_slots;
    int32_t* d_fill = sc.get<int32_t>(n);
    int32_t* d_tmp = sc.get<int32_t>(n_slots);
    if (sc.err != cudaSuccess) return fail(sc.err);
    if ((ae = cudaMallocAsync(&out.d_csr_pos, sizeof(int32_t) * std::max<int64_t>(n_slots, 1), st)) != cudaSuccess)
        return fail(ae);
    PLAN_CHECK(cudaMemsetAsync(d_fill, 0, sizeof(int32_t) * n, st));
    slot_scatter_kernel<<<grid_of(S, 256), 256, 0, st>>>(out.d_var, S, out.d_csr_off, d_fill, d_tmp);
    slot_rank_kernel<<<grid_of(S, 256), 256, 0, st>>>(out.d_var, S, out.d_csr_off, d_tmp, out.d_csr_pos);
    PLAN_CHECK(cudaGetLastError());

    // 6: tile-local variables and their patterns
    uint8_t* d_local = sc.get<uint8_t>(n);
    if (sc.err != cudaSuccess) return fail(sc.err);
    PLAN_CHECK(cudaMemsetAsync(d_local, 0, n, st));
    if (fuse_local && nt > 0) {
        TileDev* d_tiles = sc.get<TileDev>(nt);
        int32_t* d_shape_k = sc.get<int32_t>(ns);
        int32_t* d_ent_off = sc.get<int32_t>(static_cast<int64_t>(nt) + 1);
        if (sc.err != cudaSuccess) return fail(sc.err);
        std::vector<int32_t> shape_k(ns);
        for (int s = 0; s < ns; ++s) shape_k[s] = out.shapes[s].k;
        PLAN_CHECK(cudaMemcpyAsync(d_tiles, out.tiles.data(), sizeof(TileDev) * nt, cudaMemcpyHostToDevice, st));
        PLAN_CHECK(cudaMemcpyAsync(d_shape_k, shape_k.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
        PLAN_CHECK(cudaMemsetAsync(d_ent_off, 0, sizeof(int32_t) * (static_cast<size_t>(nt) + 1), st));
        const unsigned tgrid = grid_of(static_cast<int64_t>(nt) * 32, 256);
        tile_local_kernel<false><<<tgrid, 256, 0, st>>>(d_tiles, d_shape_k, nt, out.d_var, out.d_csr_off,
                                                        out.d_csr_pos, d_ent_off, nullptr, nullptr, nullptr, nullptr);
        PLAN_CHECK(cudaGetLastError());
        PLAN_CHECK(device_scan(d_ent_off, static_cast<int64_t>(nt) + 1, sc));
        std::vector<int32_t> ent_off(static_cast<size_t>(nt) + 1);
        PLAN_CHECK(cudaMemcpyAsync(ent_off.data(), d_ent_off, sizeof(int32_t) * (nt + 1), cudaMemcpyDeviceToHost, st));
        PLAN_CHECK(cudaStreamSynchronize(st));
        const int32_t n_ent = ent_off[nt];
        if (n_ent > 0) {
            uint16_t* d_ents = sc.get<uint16_t>(n_ent);
            const uint32_t tmask = table_mask(nt);
            uint64_t* d_tkey2 = sc.get<uint64_t>(nt);
            unsigned long long* d_ttab = sc.get<unsigned long long>(static_cast<int64_t>(tmask) + 1);
            int32_t* d_tval2 = sc.get<int32_t>(static_cast<int64_t>(tmask) + 1);
            int32_t* d_tid2 = sc.get<int32_t>(static_cast<int64_t>(tmask) + 1);
            int32_t* d_tslot = sc.get<int32_t>(nt);
            int32_t* d_treps = sc.get<int32_t>(nt);
            int32_t* d_tpat = sc.get<int32_t>(nt);
            if (sc.err != cudaSuccess) return fail(sc.err);
            tile_local_kernel<true><<<tgrid, 256, 0, st>>>(d_tiles, d_shape_k, nt, out.d_var, out.d_csr_off,
                                                           out.d_csr_pos, nullptr, d_ent_off, d_ents, d_local,
                                                           d_tkey2);
            PLAN_CHECK(cudaMemsetAsync(d_ttab, 0, sizeof(unsigned long long) * (static_cast<size_t>(tmask) + 1), st));
            PLAN_CHECK(cudaMemsetAsync(d_tval2, 0x7F, sizeof(int32_t) * (static_cast<size_t>(tmask) + 1), st));
            PLAN_CHECK(cudaMemsetAsync(&d_f->n_reps, 0, sizeof(int32_t), st));
            key_insert_kernel<<<grid_of(nt, 256), 256, 0, st>>>(d_tkey2, nt, d_ttab, d_tval2, d_tslot, tmask, d_f);
            tile_verify_kernel<<<tgrid, 256, 0, st>>>(d_ent_off, nt, d_ents, d_tslot, d_tval2, d_treps, d_f);
            PLAN_CHECK(cudaGetLastError());
            PLAN_CHECK(read_flags());
            if (hf.host) return leave();
            const int32_t np = hf.n_reps;
            std::vector<int32_t> treps(np);
            PLAN_CHECK(cudaMemcpyAsync(treps.data(), d_treps, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, st));
            PLAN_CHECK(cudaStreamSynchronize(st));
            std::sort(treps.begin(), treps.end());
            // patterns in tile order: {first entry group, entry groups}
            std::vector<int32_t> first(np);
            int64_t acc = 0;
            out.patterns.resize(2 * static_cast<size_t>(np));
            for (int32_t p = 0; p < np; ++p) {
                const int32_t len = ent_off[treps[p] + 1] - ent_off[treps[p]];
                first[p] = static_cast<int32_t>(acc);
                out.patterns[2 * p] = static_cast<int32_t>(acc / 4);
                out.patterns[2 * p + 1] = len / 4;
                acc += len;
            }
            out.n_local_ent = acc;
            int32_t* d_first = sc.get<int32_t>(np);
            if (sc.err != cudaSuccess) return fail(sc.err);
            if ((ae = cudaMallocAsync(&out.d_local_ent, sizeof(uint16_t) * std::max<int64_t>(acc, 4), st)) != cudaSuccess)
                return fail(ae);
            PLAN_CHECK(cudaMemcpyAsync(d_treps, treps.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st));
            PLAN_CHECK(cudaMemcpyAsync(d_first, first.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice, st));
            pattern_gather_kernel<<<grid_of(static_cast<int64_t>(np) * 32, 256), 256, 0, st>>>(
                d_treps, d_first, np, d_ent_off, d_ents, out.d_local_ent);
            rep_ids_kernel<<<grid_of(np, 256), 256, 0, st>>>(d_treps, np, d_tslot, d_tid2);
            item_ids_kernel<<<grid_of(nt, 256), 256, 0, st>>>(nt, d_tslot, d_tid2, d_tpat);
            PLAN_CHECK(cudaGetLastError());
            std::vector<int32_t> tpat(nt);
            PLAN_CHECK(cudaMemcpyAsync(tpat.data(), d_tpat, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, st));
            PLAN_CHECK(cudaStreamSynchronize(st));
            for (int32_t ti = 0; ti < nt; ++ti) {
                out.tiles[ti].pattern = tpat[ti];
                if (tpat[ti] < 0) continue;
                for (int c = 0; c < kNumClasses; ++c)
                    if (ti >= out.cls_tile_begin[c] && ti < out.cls_tile_begin[c + 1]) out.cls_has_local[c] = true;
            }
        }
    }

    // 7: deferred-sum buckets
    int32_t* d_vkey = sc.get<int32_t>(n);
    int32_t* d_vpos = sc.get<int32_t>(n);
    if (sc.err != cudaSuccess) return fail(sc.err);
    var_bucket_kernel<<<grid_of(n, 256), 256, 0, st>>>(out.d_csr_off, n, d_local, d_vkey, d_f);
    PLAN_CHECK(cudaGetLastError());
    std::vector<int32_t> bcount;
    PLAN_CHECK(device_split(d_vkey, n, FDOG_WBUCKETS, sc, bcount, nullptr, nullptr, &d_hist));
    PLAN_CHECK(read_flags());
    Buckets bk{};
    std::vector<int32_t> bstart(FDOG_WBUCKETS);
    int64_t nw = 0, nwp = 0;
    for (int b = 0; b < FDOG_WBUCKETS; ++b) {
        bstart[b] = bk.start[b] = out.wb_start[b] = static_cast<int32_t>(nw);
        bk.pos[b] = out.wb_pos[b] = static_cast<int32_t>(nwp);
        bk.count[b] = bcount[b];
        nw += bcount[b];
        if (b < FDOG_WBUCKETS - 1) {
            nwp += static_cast<int64_t>(b + 1) * bcount[b];
            out.n_work_slots += static_cast<int64_t>(b + 1) * bcount[b];
        }
    }
    bk.start[FDOG_WBUCKETS] = out.wb_start[FDOG_WBUCKETS] = static_cast<int32_t>(nw);
    out.n_work = nw;
    out.n_wpos = nwp;
    out.n_local_vars = static_cast<int64_t>(hf.n_local);
    out.n_work_overflow = static_cast<int64_t>(hf.overflow_slots);
    out.n_work_slots += out.n_work_overflow;
    ae = cudaMallocAsync(&out.d_work, sizeof(int32_t) * std::max<int64_t>(nw, 1), st);
    if (ae == cudaSuccess) ae = cudaMallocAsync(&out.d_wpos, sizeof(int32_t) * std::max<int64_t>(nwp, 1), st);
    if (ae != cudaSuccess) return fail(ae);
    PLAN_CHECK(device_split(d_vkey, n, FDOG_WBUCKETS, sc, bcount, &bstart, d_vpos, &d_hist));
    work_fill_kernel<<<grid_of(n, 256), 256, 0, st>>>(out.d_csr_off, out.d_csr_pos, n, d_vkey, d_vpos, bk, out.d_work,
                                                      out.d_wpos);
    PLAN_CHECK(cudaGetLastError());
    PLAN_CHECK(cudaStreamSynchronize(st));
    out.on_device = true;
    inst->plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return FDOG_OK;
}

int plan_leave_to_host() { return kLeaveToHost; }

}  // namespace fdog
