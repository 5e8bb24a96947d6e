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
