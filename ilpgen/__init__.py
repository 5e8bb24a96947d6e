"""Seeded synthetic 0-1 ILP generators shared by the tests, the benchmark and
the oracle's fixture scripts.

This module builds inputs only: sparse rows  L_j <= a_j^T x <= U_j  plus a
cost vector, in the form of Ex. 1 of the paper.  It holds none of the method's
arithmetic (no BDDs, no shortest paths, no dual updates).  The paper's
datasets are not available; the generators below produce instances with the
shapes and value distributions of its MRF, graph-matching and cell-tracking
workloads.

Sense convention: -1 means  a^T x <= b,  0 means  a^T x = b,  +1 means
a^T x >= b.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ILP:
    n_vars: int
    cost: np.ndarray      # float64 [n_vars]
    row_ptr: np.ndarray   # int64 [n_rows + 1]
    col: np.ndarray       # int32 [nnz]
    coef: np.ndarray      # int32 [nnz]
    sense: np.ndarray     # int8 [n_rows]
    rhs: np.ndarray       # int64 [n_rows]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_rows(self) -> int:
        return len(self.row_ptr) - 1

    def row(self, j):
        a, b = self.row_ptr[j], self.row_ptr[j + 1]
        return self.col[a:b], self.coef[a:b], int(self.sense[j]), int(self.rhs[j])

    def feasible(self, x) -> bool:
        """Exact integer check of every row for x in {0,1}^n."""
        x = np.asarray(x, dtype=np.int64)
        lhs = np.zeros(self.n_rows, np.int64)
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        np.add.at(lhs, rows, self.coef.astype(np.int64) * x[self.col])
        ok_le = (self.sense > 0) | (lhs <= self.rhs)
        ok_ge = (self.sense < 0) | (lhs >= self.rhs)
        return bool(np.all(ok_le & ok_ge))

    def objective(self, x) -> float:
        return float(np.dot(self.cost, np.asarray(x, dtype=np.float64)))


class _RowBuilder:
    def __init__(self):
        self.ptr = [0]
        self.col = []
        self.coef = []
        self.sense = []
        self.rhs = []

    def add(self, cols, coefs, sense, rhs):
        self.col.extend(int(c) for c in cols)
        self.coef.extend(int(a) for a in coefs)
        self.ptr.append(len(self.col))
        self.sense.append(int(sense))
        self.rhs.append(int(rhs))

    def finish(self, n_vars, cost, name, meta=None) -> ILP:
        return ILP(n_vars=int(n_vars), cost=np.asarray(cost, np.float64), row_ptr=np.asarray(self.ptr, np.int64),
                   col=np.asarray(self.col, np.int32), coef=np.asarray(self.coef, np.int32),
                   sense=np.asarray(self.sense, np.int8), rhs=np.asarray(self.rhs, np.int64), name=name,
                   meta=dict(meta or {}))


def fig2_example() -> ILP:
    """The worked example of the paper's Fig. 2:
    min -5x1 + x2 + 4x3 + 3x4  s.t.  x1 + x2 + x3 <= 2,  x2 + x3 - x4 = 0."""
    rb = _RowBuilder()
    rb.add([0, 1, 2], [1, 1, 1], -1, 2)
    rb.add([1, 2, 3], [1, 1, -1], 0, 0)
    return rb.finish(4, [-5.0, 1.0, 4.0, 3.0], "fig2")


def fig3_example() -> ILP:
    """The subproblem of the paper's Fig. 3:  a - b - c + d = 0  with costs
    (2, 3, 1, 4); one row, so the initial multipliers equal the costs."""
    rb = _RowBuilder()
    rb.add([0, 1, 2, 3], [1, -1, -1, 1], 0, 0)
    return rb.finish(4, [2.0, 3.0, 1.0, 4.0], "fig3")


def _grid_edges(h, w):
    edges = []
    for r in range(h):
        for c in range(w):
            u = r * w + c
            if c + 1 < w:
                edges.append((u, u + 1))
            if r + 1 < h:
                edges.append((u, u + w))
    return np.asarray(edges, dtype=np.int64).reshape(-1, 2)


def mrf_grid(h: int, w: int, labels: int, seed: int, potts_max: float = 1.0, unary_scale: float = 1.0,
             edges=None) -> ILP:
    """MAP-MRF on an h x w 4-connected grid as a 0-1 ILP (the one-hot local
    polytope encoding the paper's MRF datasets use).

    Variables: unary one-hot x_{u,l} (index u*L + l) first, then pairwise
    one-hot y_{e,l,l'} (index U*L + e*L^2 + l*L + l').  Rows: one simplex
    sum_l x_{u,l} = 1 per node, then per edge e = (u, v) the marginalisation
    rows  sum_{l'} y_{e,l,l'} - x_{u,l} = 0  (l = 0..L-1)  and
    sum_l y_{e,l,l'} - x_{v,l'} = 0  (l' = 0..L-1).
    Costs: unary ~ N(0, unary_scale^2); Potts y_{e,l,l'} = w_e [l != l'] with
    w_e ~ U(0, potts_max).  Seeded numpy PCG64."""
    rng = np.random.default_rng(seed)
    L = labels
    U = h * w
    E = _grid_edges(h, w) if edges is None else np.asarray(edges, np.int64)
    nE = len(E)
    n = U * L + nE * L * L
    unary = rng.standard_normal(U * L) * unary_scale
    wE = rng.uniform(0.0, potts_max, nE)
    cost = np.empty(n)
    cost[:U * L] = unary
    potts = (np.arange(L)[:, None] != np.arange(L)[None, :]).astype(np.float64).reshape(-1)
    cost[U * L:] = (wE[:, None] * potts[None, :]).reshape(-1)

    # vectorised row assembly (the large grid has millions of rows)
    n_simplex = U
    n_marg = nE * 2 * L
    row_len = np.concatenate([np.full(n_simplex, L), np.full(n_marg, L + 1)])
    row_ptr = np.zeros(n_simplex + n_marg + 1, np.int64)
    np.cumsum(row_len, out=row_ptr[1:])
    col = np.empty(row_ptr[-1], np.int32)
    coef = np.empty(row_ptr[-1], np.int32)
    # simplex rows
    s_end = n_simplex * L
    col[:s_end] = np.arange(U * L, dtype=np.int64)
    coef[:s_end] = 1
    # marginalisation rows: (e, side, l) -> [x, y...]
    e = np.repeat(np.arange(nE), 2 * L)
    side = np.tile(np.repeat(np.arange(2), L), nE)
    lab = np.tile(np.arange(L), 2 * nE)
    node = np.where(side == 0, E[e, 0], E[e, 1])
    xcol = node * L + lab
    base = U * L + e * L * L
    k = np.arange(L)
    # side 0: y_{e,l,k} = base + l*L + k ; side 1: y_{e,k,l} = base + k*L + l
    ycol = np.where(side[:, None] == 0, base[:, None] + lab[:, None] * L + k[None, :],
                    base[:, None] + k[None, :] * L + lab[:, None])
    block = np.concatenate([xcol[:, None], ycol], axis=1)
    bcoef = np.concatenate([-np.ones((n_marg, 1), np.int32), np.ones((n_marg, L), np.int32)], axis=1)
    col[s_end:] = block.reshape(-1)
    coef[s_end:] = bcoef.reshape(-1)
    sense = np.zeros(n_simplex + n_marg, np.int8)
    rhs = np.concatenate([np.ones(n_simplex, np.int64), np.zeros(n_marg, np.int64)])
    meta = {"kind": "mrf", "h": h, "w": w, "labels": L, "edges": E, "unary": unary.reshape(U, L), "potts": wE,
            "seed": seed}
    return ILP(n, cost, row_ptr, col, coef, sense, rhs, name=f"mrf{h}x{w}L{L}s{seed}", meta=meta)


def random_ilp(n: int, m: int, seed: int, max_row: int = 5, max_coef: int = 2, eq_frac: float = 0.25) -> ILP:
    """Small random feasible 0-1 ILP for brute-force checks: each row picks a
    random subset of variables and integer coefficients in
    [-max_coef, max_coef] \\ {0}; its right-hand side is set so that a random
    hidden point x* satisfies every row (the ILP is feasible).  Costs N(0,1)."""
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, 2, n)
    rb = _RowBuilder()
    for _ in range(m):
        k = int(rng.integers(1, min(max_row, n) + 1))
        cols = np.sort(rng.choice(n, size=k, replace=False))
        a = rng.integers(1, max_coef + 1, k) * rng.choice([-1, 1], k)
        ax = int(np.dot(a, xs[cols]))
        u = rng.random()
        if u < eq_frac:
            rb.add(cols, a, 0, ax)
        elif u < (1 + eq_frac) / 2:
            rb.add(cols, a, -1, ax + int(rng.integers(0, 2)))
        else:
            rb.add(cols, a, 1, ax - int(rng.integers(0, 2)))
    cost = rng.standard_normal(n)
    return rb.finish(n, cost, f"rand{n}x{m}s{seed}", {"kind": "random", "hidden": xs})


def _knn(src, dst, k):
    """indices of the k nearest points of dst for every point of src (Euclidean)."""
    from scipy.spatial import cKDTree

    k = min(k, len(dst))
    _, idx = cKDTree(dst).query(src, k=k)
    return np.asarray(idx).reshape(len(src), k)


def cell_tracking(seed: int, frames: int | None = None, det_lo: int = 200, det_hi: int = 2000, n_next: int = 5,
                  n_div: int = 2) -> ILP:
    """Cell-tracking-shaped 0-1 ILP (the structure of the paper's cell
    tracking datasets, with synthetic detections).  Frames ~ U{10..80} (or the
    given number), detections per frame ~ U{det_lo..det_hi}, points in
    U[0,1]^2.  Variables: one per detection d, then transitions t(d -> e) to
    the n_next nearest detections of the next frame, then one division per
    detection into its n_div nearest next-frame detections.  Rows:
      out-flow  sum_e t(d -> e) + div(d) - d <= 0
      in-flow   sum_c t(c -> d) + sum_{c divides into d} div(c) - d <= 0
      conflicts sum x <= 1 over disjoint triples of mutually close detections
                of one frame (greedy grouping).
    Costs N(0,1).  Seeded numpy PCG64."""
    rng = np.random.default_rng(seed)
    F = int(rng.integers(10, 81)) if frames is None else int(frames)
    counts = rng.integers(det_lo, det_hi + 1, F)
    pts = [rng.random((int(c), 2)) for c in counts]
    det_off = np.concatenate([[0], np.cumsum(counts)])
    n_det = int(det_off[-1])
    # transitions and divisions
    t_src, t_dst, dv_src, dv_dst = [], [], [], []
    for f in range(F - 1):
        nn = _knn(pts[f], pts[f + 1], n_next)
        src = np.repeat(np.arange(counts[f]) + det_off[f], nn.shape[1])
        t_src.append(src)
        t_dst.append((nn + det_off[f + 1]).reshape(-1))
        nd = _knn(pts[f], pts[f + 1], n_div)
        dv_src.append(np.arange(counts[f]) + det_off[f])
        dv_dst.append(nd + det_off[f + 1])
    t_src = np.concatenate(t_src) if t_src else np.zeros(0, np.int64)
    t_dst = np.concatenate(t_dst) if t_dst else np.zeros(0, np.int64)
    dv_src = np.concatenate(dv_src) if dv_src else np.zeros(0, np.int64)
    dv_dst = np.concatenate(dv_dst) if dv_dst else np.zeros((0, n_div), np.int64)
    n_t = len(t_src)
    n_dv = len(dv_src)
    t_var = n_det + np.arange(n_t)
    dv_var = n_det + n_t + np.arange(n_dv)
    n = n_det + n_t + n_dv
    cols_list, coef_list, len_list = [], [], []
    # out-flow rows: detections with successors, [d, its n_next transitions, its division]
    has_out = np.zeros(n_det, bool)
    has_out[dv_src] = True
    if n_t:
        k_next = n_t // max(len(dv_src), 1)
        out_d = dv_src  # detections of every frame but the last, in order
        block = np.concatenate([out_d[:, None], t_var.reshape(len(out_d), k_next), dv_var[:, None]], axis=1)
        cols_list.append(block.reshape(-1))
        coef_list.append(np.tile(np.concatenate([[-1], np.ones(k_next + 1, np.int64)]), len(out_d)))
        len_list.append(np.full(len(out_d), k_next + 2))
    # in-flow rows: [d, incoming transitions and divisions in ascending variable order]
    dst = np.concatenate([t_dst, dv_dst.reshape(-1)])
    src_var = np.concatenate([t_var, np.repeat(dv_var, dv_dst.shape[1] if n_dv else 0)])
    order = np.lexsort((src_var, dst))
    dst, src_var = dst[order], src_var[order]
    in_cnt = np.bincount(dst, minlength=n_det)
    in_d = np.nonzero(in_cnt)[0]
    starts = np.concatenate([[0], np.cumsum(in_cnt[in_d])])
    row_cols = np.empty(len(in_d) + len(src_var), np.int64)
    row_coef = np.ones(len(row_cols), np.int64)
    pos = starts[:-1] + np.arange(len(in_d))  # slot of d in each row
    row_cols[pos] = in_d
    row_coef[pos] = -1
    mask = np.ones(len(row_cols), bool)
    mask[pos] = False
    row_cols[mask] = src_var
    cols_list.append(row_cols)
    coef_list.append(row_coef)
    len_list.append(in_cnt[in_d] + 1)
    # conflict triples: greedy disjoint grouping of mutually close detections
    trip = []
    for f in range(F):
        c = int(counts[f])
        if c < 3:
            continue
        nn = _knn(pts[f], pts[f], 3)
        used = np.zeros(c, bool)
        for a in range(c):
            b_, c_ = int(nn[a, 1]), int(nn[a, 2])
            if used[a] or used[b_] or used[c_] or len({a, b_, c_}) < 3:
                continue
            used[[a, b_, c_]] = True
            trip.append(sorted([a + det_off[f], b_ + det_off[f], c_ + det_off[f]]))
    if trip:
        cols_list.append(np.asarray(trip, np.int64).reshape(-1))
        coef_list.append(np.ones(3 * len(trip), np.int64))
        len_list.append(np.full(len(trip), 3))
    lens = np.concatenate(len_list)
    row_ptr = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    n_rows = len(lens)
    sense = np.full(n_rows, -1, np.int8)
    rhs = np.zeros(n_rows, np.int64)
    if trip:
        rhs[-len(trip):] = 1
    cost = rng.standard_normal(n)
    return ILP(n, cost, row_ptr, np.concatenate(cols_list).astype(np.int32),
               np.concatenate(coef_list).astype(np.int32), sense, rhs, name=f"cell{seed}",
               meta={"kind": "cell", "frames": F, "detections": n_det, "transitions": n_t, "divisions": n_dv})


def qap(seed: int, n_left: int = 500, n_right: int = 1000, n_cand: int = 20, k_nn: int = 10,
        sparse: bool = False) -> ILP:
    """QAP-shaped graph matching as a 0-1 ILP.  Left and right nodes are
    points in U[0,1]^2; each left node p has n_cand distinct uniformly drawn
    right candidates a, with an assignment variable x_{p,a}.  Rows: sum_a
    x_{p,a} <= 1 per left node and sum_p x_{p,a} <= 1 per right node (rows with
    fewer than two variables dropped).  Quadratic terms: for every unordered
    pair {p, q} with q among the k_nn nearest left nodes of p, every candidate
    pair (a, b), a != b, gets a product variable z = x_{p,a} x_{q,b},
    linearised as  z - x_{p,a} <= 0,  z - x_{q,b} <= 0,
    x_{p,a} + x_{q,b} - z <= 1  (with sparse=True only pairs with b among the
    k_nn nearest right nodes of a).  All costs N(0,1).  Seeded PCG64."""
    rng = np.random.default_rng(seed)
    L = rng.random((n_left, 2))
    R = rng.random((n_right, 2))
    n_cand = min(n_cand, n_right)
    cand = np.stack([rng.choice(n_right, n_cand, replace=False) for _ in range(n_left)])
    x_index = np.arange(n_left * n_cand).reshape(n_left, n_cand)
    nn = _knn(L, L, k_nn + 1)[:, 1:]
    pp = np.repeat(np.arange(n_left), nn.shape[1])
    qq = nn.reshape(-1)
    keep = pp != qq
    pr = np.unique(np.stack([np.minimum(pp, qq), np.maximum(pp, qq)], axis=1)[keep], axis=0)
    A = cand[pr[:, 0]][:, :, None]  # [pairs, n_cand, 1]
    B = cand[pr[:, 1]][:, None, :]  # [pairs, 1, n_cand]
    ok = A != B
    if sparse:
        rnn = _knn(R, R, k_nn + 1)[:, 1:]
        near = np.zeros((n_right, n_right), bool)
        near[np.repeat(np.arange(n_right), rnn.shape[1]), rnn.reshape(-1)] = True
        ok &= near[A, B]
    pi, ia, ib = np.nonzero(ok)
    zs = np.stack([x_index[pr[pi, 0], ia], x_index[pr[pi, 1], ib]], axis=1)
    n_x = n_left * n_cand
    n_z = len(zs)
    n = n_x + n_z
    # rows: left uniqueness, right uniqueness (>= 2 variables), three rows per product
    left_cols = x_index.reshape(-1)
    left_len = np.full(n_left, n_cand)
    xr = cand.reshape(-1)  # right node of every x
    order = np.lexsort((left_cols, xr))
    r_cnt = np.bincount(xr, minlength=n_right)
    big = r_cnt >= 2
    # variables of right node a, ascending, for the nodes with >= 2 of them
    xs_sorted = left_cols[order]
    node_of = xr[order]
    sel = big[node_of]
    right_cols = xs_sorted[sel]
    right_len = r_cnt[big]
    z = n_x + np.arange(n_z)
    prod_cols = np.stack([zs[:, 0], z, zs[:, 1], z, zs[:, 0], zs[:, 1], z], axis=1).reshape(-1)
    prod_coef = np.tile(np.array([-1, 1, -1, 1, 1, 1, -1], np.int64), n_z)
    prod_len = np.tile(np.array([2, 2, 3]), n_z)
    lens = np.concatenate([left_len, right_len, prod_len])
    row_ptr = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    cols = np.concatenate([left_cols, right_cols, prod_cols]).astype(np.int32)
    coef = np.concatenate([np.ones(len(left_cols) + len(right_cols), np.int64), prod_coef]).astype(np.int32)
    n_rows = len(lens)
    sense = np.full(n_rows, -1, np.int8)
    rhs = np.ones(n_rows, np.int64)
    rhs[n_left + len(right_len):] = np.tile(np.array([0, 0, 1]), n_z)
    cost = rng.standard_normal(n)
    return ILP(n, cost, row_ptr, cols, coef, sense, rhs, name=f"qap{n_left}x{n_right}s{seed}",
               meta={"kind": "qap", "products": n_z, "pairs": len(pr)})


def _child_seeds(seed: int, n: int) -> list[int]:
    """n independent 63-bit seeds derived from one (numpy SeedSequence)."""
    return [int(s.generate_state(1, np.uint64)[0] >> np.uint64(1)) for s in np.random.SeedSequence(seed).spawn(n)]


def cell_tracking_batch(seed: int = 3, n: int = 64, **kw) -> list[ILP]:
    """The cell-tracking-shaped batch: n instances, each drawn by
    cell_tracking() from its own child seed (frames ~ U{10..80}, detections
    per frame ~ U{200..2000})."""
    return [cell_tracking(s, **kw) for s in _child_seeds(seed, n)]


def serving_stream(seed: int = 4, n: int = 10000, rate: float = 200.0) -> list[dict]:
    """Specs of a seeded request stream: Poisson arrivals at `rate` per second;
    half MRF grids (side ~ U{16..256}, labels ~ U{2..8}, Potts U(0,1)), half
    QAP (left ~ U{50..1000}, right = 2 left, candidates min(20, right), product
    terms between 10-NN neighbour matches on both sides: qap(..., sparse=True)).
    Each spec holds its arrival time and the arguments of its generator; build
    the instance with stream_instance(spec)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    kinds = rng.random(n) < 0.5
    sides = rng.integers(16, 257, n)
    labels = rng.integers(2, 9, n)
    lefts = rng.integers(50, 1001, n)
    seeds = _child_seeds(seed + 1, n)
    out = []
    for q in range(n):
        if kinds[q]:
            out.append({"arrival": float(t[q]), "kind": "mrf", "side": int(sides[q]), "labels": int(labels[q]),
                        "seed": seeds[q]})
        else:
            out.append({"arrival": float(t[q]), "kind": "qap", "left": int(lefts[q]), "seed": seeds[q]})
    return out


def stream_instance(spec: dict) -> ILP:
    if spec["kind"] == "mrf":
        return mrf_grid(spec["side"], spec["side"], spec["labels"], spec["seed"], potts_max=1.0)
    nl = spec["left"]
    return qap(spec["seed"], nl, 2 * nl, min(20, 2 * nl), sparse=True)
