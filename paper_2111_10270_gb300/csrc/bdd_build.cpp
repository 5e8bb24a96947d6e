// Host-side decomposition of a 0-1 ILP into one BDD per row (Ex. 1, Def. 4),
// with presolve, per-signature shape sharing and the tiled device layout.
//
// A row's BDD depends only on its coefficient sequence (in ascending variable
// order), its sense and its right-hand side, so rows with equal signatures
// share one shape (the MRF encodings have two signatures for millions of
// rows).  Shapes are built once and instanced per row.
#include <algorithm>
#include <atomic>
#include <new>
#include <thread>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <unordered_map>
#include <utility>

#include "fdog_internal.h"

namespace fdog {

namespace {



constexpr int64_t kMaxShapeNodes = 1 << 20;

struct PairHash {
    size_t operator()(const std::pair<int, int>& p) const {
        return std::hash<int64_t>()((static_cast<int64_t>(p.first) << 32) ^ static_cast<uint32_t>(p.second));
    }
};

}  // namespace

// Top-down: the states of layer t are the reachable partial sums of the first
// t terms that can still be completed into [lo_bound, hi_bound] (interval
// test on the remaining minimum / maximum).  Bottom-up: a state whose two
// arcs both fail becomes the BOT terminal, and states of a layer with the same
// pair of successors are merged, which yields the reduced ordered BDD.
int build_row_shape(const std::vector<int64_t>& a, bool has_lo, int64_t lo_bound, bool has_hi, int64_t hi_bound,
                    HostShape& out) {
    const int k = static_cast<int>(a.size());
    if (k == 0) return FDOG_EINVAL;
    std::vector<int64_t> rest_min(k + 1, 0), rest_max(k + 1, 0);
    for (int t = k - 1; t >= 0; --t) {
        rest_min[t] = rest_min[t + 1] + std::min<int64_t>(a[t], 0);
        rest_max[t] = rest_max[t + 1] + std::max<int64_t>(a[t], 0);
    }
    auto can_finish = [&](int t, int64_t s) {
        return (!has_lo || s + rest_max[t] >= lo_bound) && (!has_hi || s + rest_min[t] <= hi_bound);
    };
    auto satisfied = [&](int64_t s) { return (!has_lo || s >= lo_bound) && (!has_hi || s <= hi_bound); };
    if (!can_finish(0, 0)) return FDOG_EINFEASIBLE;

    std::vector<std::vector<int64_t>> states(k);
    std::vector<std::unordered_map<int64_t, int>> where(k);
    states[0].push_back(0);
    where[0][0] = 0;
    int64_t total = 1;
    for (int t = 0; t + 1 < k; ++t) {
        for (int64_t s : states[t]) {
            for (int b = 0; b < 2; ++b) {
                int64_t s2 = s + (b ? a[t] : 0);
                if (!can_finish(t + 1, s2)) continue;
                if (where[t + 1].emplace(s2, static_cast<int>(states[t + 1].size())).second) {
                    states[t + 1].push_back(s2);
                    if (++total > kMaxShapeNodes) return FDOG_ENOMEM;
                }
            }
        }
    }

    // canon[t][q]: node id within layer t of state q, or kArcBot
    std::vector<std::vector<int>> canon(k);
    std::vector<std::vector<std::pair<int, int>>> layer_nodes(k);  // (lo, hi) per canonical node
    for (int t = k - 1; t >= 0; --t) {
        std::unordered_map<std::pair<int, int>, int, PairHash> seen;
        canon[t].assign(states[t].size(), kArcBot);
        for (size_t q = 0; q < states[t].size(); ++q) {
            int arcs[2];
            for (int b = 0; b < 2; ++b) {
                int64_t s2 = states[t][q] + (b ? a[t] : 0);
                if (t + 1 == k) {
                    arcs[b] = satisfied(s2) ? kArcTop : kArcBot;
                } else if (!can_finish(t + 1, s2)) {
                    arcs[b] = kArcBot;
                } else {
                    arcs[b] = canon[t + 1][where[t + 1].at(s2)];
                }
            }
            if (arcs[0] == kArcBot && arcs[1] == kArcBot) continue;
            auto key = std::make_pair(arcs[0], arcs[1]);
            auto it = seen.find(key);
            if (it == seen.end()) {
                it = seen.emplace(key, static_cast<int>(layer_nodes[t].size())).first;
                layer_nodes[t].push_back(key);
            }
            canon[t][q] = it->second;
        }
    }
    if (canon[0][0] == kArcBot) return FDOG_EINFEASIBLE;

    out = HostShape();
    out.k = k;
    out.lstart.resize(k + 1);
    int base = 0;
    for (int t = 0; t < k; ++t) {
        out.lstart[t] = base;
        base += static_cast<int>(layer_nodes[t].size());
        out.width = std::max<int>(out.width, static_cast<int>(layer_nodes[t].size()));
    }
    out.lstart[k] = base;
    out.lo.resize(base);
    out.hi.resize(base);
    for (int t = 0; t < k; ++t) {
        int next = (t + 1 < k) ? out.lstart[t + 1] : 0;
        for (size_t v = 0; v < layer_nodes[t].size(); ++v) {
            auto [l, h] = layer_nodes[t][v];
            out.lo[out.lstart[t] + v] = l >= 0 ? next + l : l;
            out.hi[out.lstart[t] + v] = h >= 0 ? next + h : h;
        }
    }
    return FDOG_OK;
}

namespace {

struct Analysis {
    int status = FDOG_OK;
    bool full_cube = false;
    std::vector<int8_t> forced;  // per layer: -1 free, 0 / 1 forced value
    HostShape shape;
};

Analysis analyse(const std::vector<int64_t>& a, int8_t sense, int64_t rhs) {
    Analysis an;
    an.status = build_row_shape(a, sense >= 0, rhs, sense <= 0, rhs, an.shape);
    if (an.status != FDOG_OK) return an;
    const HostShape& s = an.shape;
    an.full_cube = true;
    an.forced.assign(s.k, -1);
    for (int t = 0; t < s.k; ++t) {
        int b = s.lstart[t], e = s.lstart[t + 1];
        if (e - b != 1 || s.lo[b] != s.hi[b] || s.lo[b] == kArcBot) an.full_cube = false;
        bool no_one = true, no_zero = true;
        for (int v = b; v < e; ++v) {
            if (s.hi[v] != kArcBot) no_one = false;
            if (s.lo[v] != kArcBot) no_zero = false;
        }
        // every node lies on a root-TOP path, so a layer without 1-arcs forces 0
        if (no_one) an.forced[t] = 0;
        else if (no_zero) an.forced[t] = 1;
    }
    return an;
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) as the mixing step of the row hashes
inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The first presolve pass when it fixes nothing: every row's signature is
// hashed in parallel, signatures are numbered in order of first occurrence
// (per-chunk first occurrences merged in chunk order), every row is compared
// with its signature's first row, and each signature is analysed once.  This
// is what the sequential pass computes whenever no row forces a variable, is
// empty or fails; in any of those cases (or on a hash collision) it returns
// false and the sequential pass runs instead.
bool first_pass_parallel(int32_t n_rows, const std::vector<int64_t>& rb,
                         const std::vector<int64_t, DefaultInitAlloc<int64_t>>& ra,
                         const int8_t* sense, const int64_t* rhs, std::vector<Analysis>& analyses,
                         std::vector<int>& row_an, std::vector<uint8_t>& alive) {
    if (n_rows <= 0) return false;
    std::vector<uint64_t> hash(n_rows);
    std::atomic<bool> empty{false};
    parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; ++j) {
            if (rb[j] == rb[j + 1]) empty = true;
            uint64_t h = mix64(static_cast<uint64_t>(static_cast<int64_t>(sense[j]) + 2));
            h = mix64(h ^ static_cast<uint64_t>(rhs[j]));
            h = mix64(h ^ static_cast<uint64_t>(rb[j + 1] - rb[j]));
            for (int64_t q = rb[j]; q < rb[j + 1]; ++q) h = mix64(h ^ static_cast<uint64_t>(ra[q]));
            hash[j] = h;
        }
    });
    if (empty) return false;
    // first occurrences per chunk of rows, merged in row order: ids number the
    // signatures by first occurrence whatever the chunking
    std::mutex mu;
    std::vector<std::pair<int64_t, std::vector<std::pair<uint64_t, int32_t>>>> parts;
    parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
        std::unordered_map<uint64_t, int32_t> seen;
        std::vector<std::pair<uint64_t, int32_t>> firsts;
        for (int64_t j = j0; j < j1; ++j)
            if (seen.emplace(hash[j], static_cast<int32_t>(j)).second)
                firsts.emplace_back(hash[j], static_cast<int32_t>(j));
        std::lock_guard<std::mutex> lk(mu);
        parts.emplace_back(j0, std::move(firsts));
    });
    std::sort(parts.begin(), parts.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    std::unordered_map<uint64_t, int> id_of;
    std::vector<int32_t> rep;
    for (const auto& part : parts)
        for (const auto& [h, j] : part.second)
            if (id_of.emplace(h, static_cast<int>(rep.size())).second) rep.push_back(j);
    std::atomic<bool> collision{false};
    parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; ++j) {
            const int id = id_of.at(hash[j]);
            const int32_t r = rep[id];
            row_an[j] = id;
            if (r == j) continue;
            bool same = sense[j] == sense[r] && rhs[j] == rhs[r] && rb[j + 1] - rb[j] == rb[r + 1] - rb[r];
            for (int64_t q = 0; same && q < rb[j + 1] - rb[j]; ++q) same = ra[rb[j] + q] == ra[rb[r] + q];
            if (!same) collision = true;
        }
    });
    if (collision) return false;
    analyses.resize(rep.size());
    std::atomic<bool> presolve{false};
    parallel_chunks(static_cast<int64_t>(rep.size()), [&](int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; ++i) {
            const int32_t j = rep[i];
            std::vector<int64_t> a(ra.begin() + rb[j], ra.begin() + rb[j + 1]);
            analyses[i] = analyse(a, sense[j], rhs[j]);
            if (analyses[i].status != FDOG_OK) { presolve = true; continue; }
            for (int8_t f : analyses[i].forced)
                if (f >= 0) presolve = true;
        }
    });
    if (presolve) return false;
    parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; ++j) alive[j] = analyses[row_an[j]].full_cube ? 0 : 1;
    });
    return true;
}

std::string signature(int8_t sense, int64_t rhs, const std::vector<int64_t>& a) {
    std::string key(1 + 8 + 8 * a.size(), '\0');
    key[0] = static_cast<char>(sense);
    std::memcpy(&key[1], &rhs, 8);
    std::memcpy(&key[9], a.data(), 8 * a.size());
    return key;
}

}  // namespace

int analyse_row(const std::vector<int64_t>& a, int8_t sense, int64_t rhs, HostShape& shape, bool& presolve) {
    Analysis an = analyse(a, sense, rhs);
    if (an.status != FDOG_OK) return an.status;
    presolve = an.full_cube;
    for (int8_t f : an.forced) presolve = presolve || f >= 0;
    shape = std::move(an.shape);
    return FDOG_OK;
}

int shape_class(const HostShape& s, int jit_mode, int64_t n_bdds) {
    int cls = class_of(s.width, s.k);
    // a specialised kernel costs a compile; rare shapes stay generic in the default mode
    const bool often = jit_mode >= 1 || n_bdds >= kJitMinBdds;
    if (jit_mode >= 0 && often && s.width <= kJitMaxW && s.k <= kJitMaxK) cls = kJitClass;
    if (cls < 0 || (!class_is_reg(cls) && s.k > (class_is_seg(cls) ? kMaxLayersSeg : kMaxLayersSmem))) return -1;
    return cls;
}

void build_templates(Decomposition& out) {
    out.shape_dev.resize(out.shapes.size());
    for (size_t s = 0; s < out.shapes.size(); ++s) {
        const HostShape& h = out.shapes[s];
        int W = class_width(out.shape_cls[s]);
        while (out.tpl.size() % 8) out.tpl.push_back(0);  // 16-byte aligned vector loads
        const int jit = out.shape_cls[s] == kJitClass ? jit_register_shape(h) : -1;
        ShapeDev d{h.k, static_cast<int32_t>(out.tpl.size()), W, jit};
        out.shape_dev[s] = d;
        for (int t = 0; t < h.k; ++t) {
            int b = h.lstart[t], e = h.lstart[t + 1];
            int nb = (t + 1 < h.k) ? h.lstart[t + 1] : 0;
            for (int v = 0; v < W; ++v) {
                uint8_t lo = kCodeBot, hi = kCodeBot;
                if (b + v < e) {
                    int l = h.lo[b + v], u = h.hi[b + v];
                    lo = l == kArcTop ? kCodeTop : (l == kArcBot ? kCodeBot : static_cast<uint8_t>(l - nb));
                    hi = u == kArcTop ? kCodeTop : (u == kArcBot ? kCodeBot : static_cast<uint8_t>(u - nb));
                }
                out.tpl.push_back(static_cast<uint16_t>(lo | (hi << 8)));
            }
        }
    }
}

int build_decomposition(int32_t n_vars, const double* cost, int32_t n_rows, const int64_t* row_ptr,
                        const int32_t* col, const int32_t* coef, const int8_t* sense, const int64_t* rhs,
                        int jit_mode, bool fuse_local, Decomposition& out, std::string& err,
                        const uint8_t* shared) {
    out = Decomposition();
    out.fixed.assign(n_vars, -1);

    // rows with non-zero entries sorted by variable (Alg. 1 visits I_j ascending)
    std::vector<int64_t> rb(n_rows + 1, 0);
    parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
        for (int64_t j = j0; j < j1; ++j) {
            int64_t c = 0;
            for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q) c += coef[q] != 0;
            rb[j + 1] = c;
        }
    });
    for (int32_t j = 0; j < n_rows; ++j) rb[j + 1] += rb[j];
    std::vector<int32_t, DefaultInitAlloc<int32_t>> rv(static_cast<size_t>(rb[n_rows]));  // filled below
    std::vector<int64_t, DefaultInitAlloc<int64_t>> ra(static_cast<size_t>(rb[n_rows]));
    parallel_chunks(n_rows, [&](int64_t j0, int64_t j1) {
        std::vector<std::pair<int32_t, int32_t>> tmp;
        for (int64_t j = j0; j < j1; ++j) {
            tmp.clear();
            for (int64_t q = row_ptr[j]; q < row_ptr[j + 1]; ++q)
                if (coef[q] != 0) tmp.emplace_back(col[q], coef[q]);
            if (!std::is_sorted(tmp.begin(), tmp.end())) std::sort(tmp.begin(), tmp.end());
            int64_t o = rb[j];
            for (auto& [c, v] : tmp) { rv[o] = c; ra[o] = v; ++o; }
        }
    });

    std::unordered_map<std::string, int> cache;
    std::vector<Analysis> analyses;
    std::vector<int> row_an(n_rows, -1);
    std::vector<uint8_t> alive(n_rows, 1);
    std::vector<int64_t> a;
    auto residual = [&](int32_t j, std::vector<int64_t>& coefs, int64_t& b) {
        coefs.clear();
        b = rhs[j];
        for (int64_t q = rb[j]; q < rb[j + 1]; ++q) {
            int8_t f = out.fixed[rv[q]];
            if (f == 0 || f == 1) b -= ra[q] * f;
            else coefs.push_back(ra[q]);
        }
    };

    const bool parallel_done = first_pass_parallel(n_rows, rb, ra, sense, rhs, analyses, row_an, alive);
    if (!parallel_done) {
        // the sequential passes below start from scratch
        analyses.clear();
        std::fill(row_an.begin(), row_an.end(), -1);
        std::fill(alive.begin(), alive.end(), 1);
    }
    for (bool changed = !parallel_done; changed;) {
        changed = false;
        for (int32_t j = 0; j < n_rows; ++j) {
            if (!alive[j]) continue;
            int64_t b;
            residual(j, a, b);
            if (a.empty()) {
                bool ok = (sense[j] > 0 || 0 <= b) && (sense[j] < 0 || 0 >= b);
                if (!ok) { err = "row " + std::to_string(j) + " violated by fixed variables"; return FDOG_EINFEASIBLE; }
                alive[j] = 0;
                continue;
            }
            std::string key = signature(sense[j], b, a);
            auto it = cache.find(key);
            int id;
            if (it == cache.end()) {
                id = static_cast<int>(analyses.size());
                analyses.push_back(analyse(a, sense[j], b));
                cache.emplace(std::move(key), id);
            } else {
                id = it->second;
            }
            const Analysis& an = analyses[id];
            if (an.status == FDOG_EINFEASIBLE) { err = "row " + std::to_string(j) + " is infeasible"; return FDOG_EINFEASIBLE; }
            if (an.status != FDOG_OK) { err = "row " + std::to_string(j) + ": BDD too large"; return an.status; }
            row_an[j] = id;
            if (an.full_cube) { alive[j] = 0; continue; }
            int t = 0;
            for (int64_t q = rb[j]; q < rb[j + 1]; ++q) {
                int8_t f = out.fixed[rv[q]];
                if (f == 0 || f == 1) continue;
                if (an.forced[t] >= 0) { out.fixed[rv[q]] = an.forced[t]; changed = true; }
                ++t;
            }
        }
    }

    if (shared) {
        // a shard of a split instance: presolve would fix variables that other
        // shards' rows also hold, so a shard must not need it
        for (int32_t j = 0; j < n_rows; ++j)
            if (!alive[j]) { err = "shard row " + std::to_string(j) + " needs presolve"; return FDOG_EUNSUPPORTED; }
        for (int32_t i = 0; i < n_vars; ++i)
            if (out.fixed[i] == 0 || out.fixed[i] == 1) {
                err = "shard presolve fixes variable " + std::to_string(i);
                return FDOG_EUNSUPPORTED;
            }
    }

    // surviving rows: their analysis holds the final shape
    std::vector<int> shape_of_an(analyses.size(), -1);
    std::vector<int64_t> an_count(analyses.size(), 0);
    for (int32_t j = 0; j < n_rows; ++j)
        if (alive[j]) an_count[row_an[j]]++;
    struct Bdd { int cls; int shape; int32_t row; };
    std::vector<Bdd> bdds;
    for (int32_t j = 0; j < n_rows; ++j) {
        if (!alive[j]) continue;
        int id = row_an[j];
        if (shape_of_an[id] < 0) {
            const HostShape& s = analyses[id].shape;
            const int cls = shape_class(s, jit_mode, an_count[id]);
            if (cls < 0) {
                err = "row " + std::to_string(j) + ": BDD width " + std::to_string(s.width) + " / length " +
                      std::to_string(s.k) + " exceeds the sweep kernels' limits";
                return FDOG_EUNSUPPORTED;
            }
            shape_of_an[id] = static_cast<int>(out.shapes.size());
            out.shapes.push_back(s);
            out.shape_cls.push_back(cls);
        }
        int sh = shape_of_an[id];
        bdds.push_back({out.shape_cls[sh], sh, j});
    }
    {
        // stable counting sort by (class, shape): BDDs keep row order within a shape
        const int ns = static_cast<int>(out.shapes.size());
        std::vector<int> order(ns);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int x, int y) {
            return out.shape_cls[x] != out.shape_cls[y] ? out.shape_cls[x] < out.shape_cls[y] : x < y;
        });
        std::vector<int64_t> start(ns + 1, 0);
        for (const Bdd& d : bdds) start[d.shape + 1]++;
        std::vector<int64_t> at(ns, 0);
        int64_t acc = 0;
        for (int r = 0; r < ns; ++r) { at[order[r]] = acc; acc += start[order[r] + 1]; }
        std::vector<Bdd> sorted(bdds.size());
        for (const Bdd& d : bdds) sorted[at[d.shape]++] = d;
        bdds.swap(sorted);
    }

    // presolve constants
    std::vector<int32_t> cnt(n_vars, 0);
    for (const Bdd& d : bdds)
        for (int64_t q = rb[d.row]; q < rb[d.row + 1]; ++q)
            if (out.fixed[rv[q]] == -1) cnt[rv[q]]++;
    for (int32_t i = 0; i < n_vars; ++i) {
        if (out.fixed[i] == 0 || out.fixed[i] == 1) {
            out.const_lb += cost[i] * out.fixed[i];
        } else if (cnt[i] == 0) {
            out.fixed[i] = 2;
            out.const_lb += std::min(cost[i], 0.0);
        }
        if (out.fixed[i] != -1) out.outside.push_back(i);
    }
    out.const_obj = out.const_lb;

    build_templates(out);

    // tiles: runs of equal shape, kTile BDDs each, grouped by kernel class
    out.cls_tile_begin.assign(kNumClasses + 1, 0);
    int64_t slot = 0;
    for (size_t q = 0; q < bdds.size();) {
        size_t e = q;
        while (e < bdds.size() && e - q < static_cast<size_t>(kTile) && bdds[e].shape == bdds[q].shape) ++e;
        TileDev t{bdds[q].shape, static_cast<int32_t>(slot), static_cast<int32_t>(e - q), static_cast<int32_t>(q), -1,
                  {0, 0, 0}};
        int k = out.shapes[bdds[q].shape].k;
        slot += static_cast<int64_t>(k) * kTile;
        if (slot > INT32_MAX) { err = "more than 2^31 padded slots"; return FDOG_EUNSUPPORTED; }
        out.tiles.push_back(t);
        out.cls_tile_begin[bdds[q].cls + 1]++;
        int cls = bdds[q].cls;
        out.kmax[cls] = std::max(out.kmax[cls], k);
        q = e;
    }
    for (int c = 0; c < kNumClasses; ++c) out.cls_tile_begin[c + 1] += out.cls_tile_begin[c];
    out.slots_pad = slot;
    out.var.assign(slot, -1);
    out.bdd_row.resize(bdds.size());
    out.bdd_shape.resize(bdds.size());
    out.bdd_slot0.resize(bdds.size());
    out.row_bdd.assign(n_rows, -1);
    out.n_bdds = static_cast<int64_t>(bdds.size());
    for (const Bdd& d : bdds) out.n_nodes += out.shapes[d.shape].lstart.back();
    parallel_chunks(static_cast<int64_t>(out.tiles.size()), [&](int64_t t0, int64_t t1) {
        for (int64_t ti = t0; ti < t1; ++ti) {
            const TileDev& t = out.tiles[ti];
            for (int l = 0; l < t.n_valid; ++l) {
                const Bdd& d = bdds[t.bdd_base + l];
                out.bdd_row[t.bdd_base + l] = d.row;
                out.bdd_shape[t.bdd_base + l] = d.shape;
                out.bdd_slot0[t.bdd_base + l] = t.slot_base + l;
                out.row_bdd[d.row] = t.bdd_base + l;
                int layer = 0;
                for (int64_t q = rb[d.row]; q < rb[d.row + 1]; ++q) {
                    if (out.fixed[rv[q]] != -1) continue;
                    out.var[t.slot_base + static_cast<int64_t>(layer) * kTile + l] = rv[q];
                    ++layer;
                }
            }
        }
    });
    // per-variable slot lists (ascending padded position: a fixed summation order)
    out.csr_off.assign(n_vars + 1, 0);
    for (int32_t i = 0; i < n_vars; ++i) out.csr_off[i + 1] = out.csr_off[i] + cnt[i];
    out.n_slots = out.csr_off[n_vars];
    out.csr_pos.resize(out.n_slots);
    {
        // scattered in parallel, then each variable's few positions sorted
        std::vector<int32_t> fill(out.csr_off.begin(), out.csr_off.end() - 1);
        parallel_chunks(slot, [&](int64_t p0, int64_t p1) {
            for (int64_t p = p0; p < p1; ++p) {
                const int32_t v = out.var[p];
                if (v >= 0) out.csr_pos[__atomic_fetch_add(&fill[v], 1, __ATOMIC_RELAXED)] = static_cast<int32_t>(p);
            }
        });
        parallel_chunks(n_vars, [&](int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                int32_t* q = out.csr_pos.data() + out.csr_off[i];
                const int32_t c = out.csr_off[i + 1] - out.csr_off[i];
                for (int32_t x = 1; x < c; ++x)  // insertion sort: a variable has few copies
                    for (int32_t y = x; y > 0 && q[y - 1] > q[y]; --y) std::swap(q[y - 1], q[y]);
            }
        });
    }
    // Tile-local variables: every copy in one tile (at most four copies) of a
    // row of at most kEpiMaxK layers.  The
    // update sweep computes their deferred term itself; the deferred-sum
    // kernel keeps the rest.  Tiles with equal local-variable patterns share
    // one pattern.
    std::vector<uint8_t> local(n_vars, 0);
    if (fuse_local) {
        // per tile, in parallel: its local variables' copy offsets (a variable's
        // first copy lies in exactly one tile, so each is marked by one tile)
        const int64_t nt = static_cast<int64_t>(out.tiles.size());
        std::vector<int64_t> ent_off(nt + 1, 0);
        auto scan = [&](int64_t ti, uint16_t* dst) {
            const TileDev& t = out.tiles[ti];
            if (out.shapes[t.shape].k > kEpiMaxK) return int64_t(0);  // the sweep stages at most kEpiMaxK layers
            const int64_t lo = t.slot_base, hi = lo + static_cast<int64_t>(out.shapes[t.shape].k) * kTile;
            int64_t m = 0;
            for (int64_t p = lo; p < hi; ++p) {
                const int32_t v = out.var[p];
                if (v < 0 || (shared && shared[v])) continue;  // a shared variable's sum spans shards
                const int32_t b = out.csr_off[v], c = out.csr_off[v + 1] - b;
                if (c > 4 || out.csr_pos[b] != p || out.csr_pos[b + c - 1] >= hi) continue;  // p is the first copy
                if (dst) {
                    for (int q = 0; q < 4; ++q)
                        dst[4 * m + q] = q < c ? static_cast<uint16_t>(out.csr_pos[b + q] - lo) : uint16_t(0xFFFF);
                    local[v] = 1;
                }
                ++m;
            }
            return 4 * m;
        };
        parallel_chunks(nt, [&](int64_t t0, int64_t t1) {
            for (int64_t ti = t0; ti < t1; ++ti) ent_off[ti + 1] = scan(ti, nullptr);
        });
        for (int64_t ti = 0; ti < nt; ++ti) ent_off[ti + 1] += ent_off[ti];
        std::vector<uint16_t> ents(static_cast<size_t>(ent_off[nt]));
        parallel_chunks(nt, [&](int64_t t0, int64_t t1) {
            for (int64_t ti = t0; ti < t1; ++ti) scan(ti, ents.data() + ent_off[ti]);
        });
        // patterns in tile order (deduplicated)
        std::unordered_map<std::string, int> pat_ids;
        for (int64_t ti = 0; ti < nt; ++ti) {
            TileDev& t = out.tiles[ti];
            const uint16_t* e0 = ents.data() + ent_off[ti];
            const int64_t ne = ent_off[ti + 1] - ent_off[ti];
            if (ne == 0) continue;
            std::vector<uint16_t> ent(e0, e0 + ne);
            std::string key(reinterpret_cast<const char*>(ent.data()), ent.size() * sizeof(uint16_t));
            auto it = pat_ids.find(key);
            if (it == pat_ids.end()) {
                it = pat_ids.emplace(std::move(key), static_cast<int>(out.patterns.size() / 2)).first;
                out.patterns.push_back(static_cast<int32_t>(out.local_ent.size() / 4));
                out.patterns.push_back(static_cast<int32_t>(ent.size() / 4));
                out.local_ent.insert(out.local_ent.end(), ent.begin(), ent.end());
            }
            t.pattern = it->second;
            for (int c = 0; c < kNumClasses; ++c)
                if (static_cast<int32_t>(ti) >= out.cls_tile_begin[c] && static_cast<int32_t>(ti) < out.cls_tile_begin[c + 1])
                    out.cls_has_local[c] = true;
        }
    }
    // The other variables go to the deferred-sum kernel, bucketed by copy
    // count so that a warp reads its variables' slot positions column by
    // column (coalesced); more than FDOG_WBUCKETS - 1 copies: the last bucket.
    std::vector<std::vector<int32_t>> bucket(FDOG_WBUCKETS);
    for (int32_t i = 0; i < n_vars; ++i) {
        const int32_t c = out.csr_off[i + 1] - out.csr_off[i];
        if (local[i]) {
            ++out.n_local_vars;
        } else if (shared && shared[i]) {
            if (c > 0) out.shared_vars.push_back(i);  // deferred term from the sum over all shards
        } else if (c > 0) {
            bucket[std::min(c, FDOG_WBUCKETS) - 1].push_back(i);
            out.n_work_slots += c;
            if (c >= FDOG_WBUCKETS) out.n_work_overflow += c;
        }
    }
    for (int b = 0; b < FDOG_WBUCKETS; ++b) {
        out.wb_start[b] = static_cast<int32_t>(out.work.size());
        out.wb_pos[b] = static_cast<int32_t>(out.wpos.size());
        out.work.insert(out.work.end(), bucket[b].begin(), bucket[b].end());
        if (b == FDOG_WBUCKETS - 1) continue;
        const size_t nb = bucket[b].size();
        out.wpos.resize(out.wpos.size() + (b + 1) * nb);
        for (int q = 0; q <= b; ++q)
            for (size_t j = 0; j < nb; ++j)
                out.wpos[out.wb_pos[b] + q * nb + j] = out.csr_pos[out.csr_off[bucket[b][j]] + q];
    }
    out.wb_start[FDOG_WBUCKETS] = static_cast<int32_t>(out.work.size());
    out.n_work = static_cast<int64_t>(out.work.size());
    out.n_wpos = static_cast<int64_t>(out.wpos.size());
    out.n_local_ent = static_cast<int64_t>(out.local_ent.size());
    return FDOG_OK;
}

void build_serial_schedule(int32_t n_vars, Decomposition& d) {
    const int64_t rows = d.slots_pad / kTile;
    d.tile_of_row.assign(static_cast<size_t>(rows), -1);
    d.lab_off.resize(d.tiles.size());
    int64_t off = 0;
    for (size_t ti = 0; ti < d.tiles.size(); ++ti) {
        const TileDev& t = d.tiles[ti];
        const ShapeDev& sh = d.shape_dev[t.shape];
        for (int l = 0; l < sh.k; ++l) d.tile_of_row[t.slot_base / kTile + l] = static_cast<int32_t>(ti);
        d.lab_off[ti] = static_cast<int32_t>(off);
        off += static_cast<int64_t>(sh.k + 1) * sh.width * kTile;
    }
    d.lab_floats = off;
    // levels: predecessor / successor of a copy is the slot one layer up / down in its tile
    auto layer_of = [&](int32_t p) {
        const TileDev& t = d.tiles[d.tile_of_row[p / kTile]];
        return std::make_pair(p / kTile - t.slot_base / kTile, d.shape_dev[t.shape].k);
    };
    auto levels = [&](bool ascending, std::vector<int32_t>& loff, std::vector<int32_t>& lvars) {
        std::vector<int32_t> lev(n_vars, -1);
        int32_t top = -1;
        for (int32_t q = 0; q < n_vars; ++q) {
            const int32_t i = ascending ? q : n_vars - 1 - q;
            const int32_t b = d.csr_off[i], e = d.csr_off[i + 1];
            if (b == e) continue;
            int32_t l = 0;
            for (int32_t r = b; r < e; ++r) {
                const int32_t p = d.csr_pos[r];
                const auto [t, k] = layer_of(p);
                if (ascending ? t > 0 : t + 1 < k) l = std::max(l, lev[d.var[ascending ? p - kTile : p + kTile]] + 1);
            }
            lev[i] = l;
            top = std::max(top, l);
        }
        loff.assign(static_cast<size_t>(top + 2), 0);
        for (int32_t i = 0; i < n_vars; ++i)
            if (lev[i] >= 0) loff[lev[i] + 1]++;
        for (int32_t l = 0; l <= top; ++l) loff[l + 1] += loff[l];
        lvars.resize(static_cast<size_t>(loff[top + 1]));
        std::vector<int32_t> fill(loff.begin(), loff.end() - 1);
        for (int32_t i = 0; i < n_vars; ++i)
            if (lev[i] >= 0) lvars[fill[lev[i]]++] = i;
    };
    levels(true, d.lev_f_off, d.lev_f_vars);
    levels(false, d.lev_b_off, d.lev_b_vars);
}

}  // namespace fdog
