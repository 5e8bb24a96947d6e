"""Long-row splitting (fdog_split_rows): an at-most-one / exactly-one row over
many variables becomes a chain of short rows joined by new binaries.

Pins, none of which uses the splitter's own reasoning:
  * brute force: the split ILP's feasible set, projected onto the original
    variables, is the original feasible set;
  * the LP relaxation (scipy's HiGHS) has the same value before and after
    splitting.  Every row here has +-1 coefficients, so each row alone is
    totally unimodular and its convex hull is its LP relaxation: the LP value
    is then the optimal bound of the Lagrange decomposition (Prop. 1's dual),
    so equal LP values are the exactness the splitting claims;
  * sizes and piece lengths follow the documented chain (first piece
    max_len - 1 variables, middle max_len - 2, last the rest).
"""
import itertools

import numpy as np
import pytest

import ilpgen


@pytest.fixture(scope="module")
def P():
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    return P


def split_ilp(P, g, max_len):
    nv, rp, col, coef, sense, rhs, orig = P.capi.split_rows(g.n_vars, g.row_ptr, g.col, g.coef, g.sense, g.rhs,
                                                           max_len)
    cost = np.concatenate([g.cost, np.zeros(nv - g.n_vars)])
    return ilpgen.ILP(nv, cost, rp, col, coef, sense, rhs, name=g.name + "-split"), orig


def small_mixed(seed, n=9):
    """At-most-one and exactly-one rows of 4..6 variables, plus a few other
    +-1 rows (left alone by the splitter); at most 9 new variables."""
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(3):
        k = int(rng.integers(4, 7))
        vs = np.sort(rng.choice(n, k, replace=False))
        rows.append((vs, np.ones(k, int), int(rng.choice([-1, 0])), 1))
    for _ in range(2):
        vs = np.sort(rng.choice(n, 3, replace=False))
        rows.append((vs, rng.choice([-1, 1], 3), 1, -1))
    row_ptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    return ilpgen.ILP(n, rng.normal(size=n), row_ptr, np.concatenate([r[0] for r in rows]).astype(np.int32),
                      np.concatenate([r[1] for r in rows]).astype(np.int32),
                      np.array([r[2] for r in rows], np.int8), np.array([r[3] for r in rows], np.int64),
                      name=f"mixed{seed}")


def feasible(g, X):
    """Rows of X (0/1 assignments) satisfying every row of g."""
    ok = np.ones(len(X), bool)
    for j in range(len(g.row_ptr) - 1):
        b, e = g.row_ptr[j], g.row_ptr[j + 1]
        s = X[:, g.col[b:e]] @ g.coef[b:e]
        ok &= (s <= g.rhs[j]) if g.sense[j] < 0 else (s >= g.rhs[j]) if g.sense[j] > 0 else (s == g.rhs[j])
    return ok


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("max_len", [3, 4])
def test_split_preserves_the_feasible_set(P, seed, max_len):
    g = small_mixed(seed)
    s, _ = split_ilp(P, g, max_len)
    assert np.diff(s.row_ptr).max() <= max(max_len, np.diff(g.row_ptr)[np.diff(g.row_ptr) <= max_len].max())
    X = np.array(list(itertools.product([0, 1], repeat=g.n_vars)), np.int64)
    Y = np.array(list(itertools.product([0, 1], repeat=s.n_vars - g.n_vars)), np.int64)
    orig = feasible(g, X)
    proj = np.zeros(len(X), bool)
    for y in Y:
        proj |= feasible(s, np.hstack([X, np.tile(y, (len(X), 1))]))
    assert np.array_equal(orig, proj)


def lp_value(g):
    opt = pytest.importorskip("scipy.optimize")
    A_ub, b_ub, A_eq, b_eq = [], [], [], []
    for j in range(len(g.row_ptr) - 1):
        a = np.zeros(g.n_vars)
        b, e = g.row_ptr[j], g.row_ptr[j + 1]
        a[g.col[b:e]] = g.coef[b:e]
        if g.sense[j] < 0:
            A_ub.append(a); b_ub.append(g.rhs[j])
        elif g.sense[j] > 0:
            A_ub.append(-a); b_ub.append(-g.rhs[j])
        else:
            A_eq.append(a); b_eq.append(g.rhs[j])
    r = opt.linprog(g.cost, A_ub=np.array(A_ub) if A_ub else None, b_ub=b_ub or None,
                    A_eq=np.array(A_eq) if A_eq else None, b_eq=b_eq or None, bounds=(0, 1), method="highs")
    assert r.status == 0, r.message
    return r.fun


@pytest.mark.parametrize("max_len", [3, 5, 8])
def test_split_keeps_the_lp_bound_of_a_matching_problem(P, max_len):
    g = ilpgen.qap(seed=5, n_left=12, n_right=20, n_cand=9, k_nn=3)
    s, _ = split_ilp(P, g, max_len)
    assert s.n_vars > g.n_vars  # some rows were split
    a, b = lp_value(g), lp_value(s)
    assert abs(a - b) <= 1e-7 * max(1.0, abs(a)), (a, b)


def test_split_sizes_and_row_origin(P):
    # one at-most-one row of 10 variables, one exactly-one row of 7, one row left alone
    row_ptr = np.array([0, 10, 17, 20], np.int64)
    col = np.concatenate([np.arange(10), np.arange(10, 17), [0, 5, 12]]).astype(np.int32)
    coef = np.concatenate([np.ones(17), [1, -1, 1]]).astype(np.int32)
    sense = np.array([-1, 0, -1], np.int8)
    rhs = np.array([1, 1, 1], np.int64)
    nv, rp, c, a, se, r, orig = P.capi.split_rows(17, row_ptr, col, coef, sense, rhs, 4)
    # row 0: pieces of 3, 2, 2, 3 variables; row 1: 3, 2, 2; row 2 as it was
    assert nv == 17 + 3 + 2
    assert list(orig) == [0] * 4 + [1] * 3 + [2]
    assert list(np.diff(rp)) == [4, 4, 4, 4, 4, 4, 3, 3]
    assert list(se) == [0, 0, 0, -1, 0, 0, 0, -1] and list(r) == [0, 0, 0, 1, 0, 0, 1, 1]
    piece = lambda q: (list(c[rp[q]:rp[q + 1]]), list(a[rp[q]:rp[q + 1]]))
    assert piece(0) == ([0, 1, 2, 17], [1, 1, 1, -1])
    assert piece(1) == ([3, 4, 17, 18], [1, 1, 1, -1])
    assert piece(3) == ([7, 8, 9, 19], [1, 1, 1, 1])
    assert piece(4) == ([10, 11, 12, 20], [1, 1, 1, -1])
    assert piece(5) == ([13, 14, 20, 21], [1, 1, 1, -1])
    assert piece(6) == ([15, 16, 21], [1, 1, 1])
    assert piece(7) == ([0, 5, 12], [1, -1, 1])
    with pytest.raises(P.FdogError):
        P.capi.split_rows(17, row_ptr, col, coef, sense, rhs, 2)
