"""Pins for the FP64 oracle: checks against values the paper prints, against
brute-force enumeration, closed forms, textbook special cases and the
invariants of Prop. 1.  None of these re-types the oracle's formulas; each
compares it with something computed another way."""
import itertools
import os

import networkx as nx
import numpy as np
import pytest

import ilpgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# brute-force helpers (independent of the oracle)
# ----------------------------------------------------------------------------
def row_feasible_set(coefs, sense, rhs):
    k = len(coefs)
    out = set()
    for x in itertools.product((0, 1), repeat=k):
        s = sum(a * b for a, b in zip(coefs, x))
        if (sense <= 0 and s > rhs) or (sense >= 0 and s < rhs):
            continue
        out.add(x)
    return out


def bdd_path_set(ls, lo, hi):
    """All assignments encoded by root-TOP paths (Def. of constraint set correspondence)."""
    k = len(ls) - 1
    out = set()

    def walk(v, t, acc):
        if v == -1:
            assert t == k
            out.add(tuple(acc))
            return
        if v == -2:
            return
        assert ls[t] <= v < ls[t + 1], "arc skips a layer"
        walk(lo[v], t + 1, acc + [0])
        walk(hi[v], t + 1, acc + [1])

    walk(0, 0, [])
    return out


def ordered_row(ilp, j, fixed=None):
    cols, coefs, sense, rhs = ilp.row(j)
    order = np.argsort(cols)
    return [int(c) for c in cols[order]], [int(a) for a in coefs[order]], sense, rhs


def bf_min_marginals(feas, lam):
    k = len(lam)
    m0 = [np.inf] * k
    m1 = [np.inf] * k
    for x in feas:
        e = sum(l for l, b in zip(lam, x) if b)
        for t in range(k):
            if x[t]:
                m1[t] = min(m1[t], e)
            else:
                m0[t] = min(m0[t], e)
    return np.array(m0), np.array(m1)


def bf_optimum(ilp):
    best, arg = np.inf, None
    for x in itertools.product((0, 1), repeat=ilp.n_vars):
        if ilp.feasible(x):
            v = ilp.objective(x)
            if v < best:
                best, arg = v, x
    return best, arg


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------------------
# the paper's worked examples
# ----------------------------------------------------------------------------
def test_fig3_structure_and_shortest_paths(oracle_mod):
    p = oracle_mod.Problem.from_ilp(ilpgen.fig3_example())
    assert (p.m, p.S, p.N) == (1, 4, 8)
    ls, lo, hi = p.bdd_nodes(0)
    f, g = p.shortest_paths(0)
    gold = read_golden("fig3_shortest_paths.txt")
    # name the oracle's nodes by following the figure's arcs from the root
    names = {0: "a"}
    by_name = {r[0]: r for r in gold}
    changed = True
    while changed:
        changed = False
        for v, nm in list(names.items()):
            for arcs, succ_name in ((lo, by_name[nm][2]), (hi, by_name[nm][3])):
                w = int(arcs[v])
                if succ_name in ("TOP", "BOT"):
                    assert w == (-1 if succ_name == "TOP" else -2), (nm, succ_name, w)
                elif w not in names:
                    names[w] = succ_name
                    changed = True
                else:
                    assert names[w] == succ_name
    assert sorted(names.values()) == sorted(by_name)
    for v, nm in names.items():
        r = by_name[nm]
        assert ls[int(r[1])] <= v < ls[int(r[1]) + 1], nm
        assert f[v] == float(r[4]), (nm, f[v])
        assert g[v] == float(r[5]), (nm, g[v])


def test_fig3_min_marginals_bruteforce(oracle_mod):
    ilp = ilpgen.fig3_example()
    p = oracle_mod.Problem.from_ilp(ilp)
    m0, m1 = p.min_marginals()
    feas = row_feasible_set([1, -1, -1, 1], 0, 0)
    b0, b1 = bf_min_marginals(feas, [2, 3, 1, 4])
    assert np.array_equal(m0, b0) and np.array_equal(m1, b1)
    assert np.array_equal(m1 - m0, [3, 5, 3, 5])
    assert p.lower_bounds() == (0.0, 0.0)


def test_fig2_initialisation_matches_printed_multipliers(oracle_mod):
    gold = {r[0]: [float(v) for v in r[1:]] for r in read_golden("fig2_example.txt")}
    p = oracle_mod.Problem.from_ilp(ilpgen.fig2_example())
    hi, lo, db0, db1 = p.state()
    assert np.array_equal(hi, gold["lambda_X1"] + gold["lambda_X2"])
    assert not lo.any() and not db0.any() and not db1.any()
    # the printed optimal assignments are the per-subproblem minimisers
    ilp = ilpgen.fig2_example()
    for j, key in ((0, "opt_X1"), (1, "opt_X2")):
        cols, coefs, sense, rhs = ordered_row(ilp, j)
        lam = hi[3 * j:3 * j + 3]
        feas = row_feasible_set(coefs, sense, rhs)
        best = min(feas, key=lambda x: np.dot(x, lam))
        assert list(best) == gold[key]


def test_fig2_first_forward_pass_by_hand(oracle_mod):
    """One ascending pass of Alg. 1 (omega = 1/2) on Fig. 2, derived by hand.

    X1 (x1,x2,x3), lambda = (-5, .5, 2):  M_x1 = -5 -> lo_x1 = -2.5;  with the
    new x1 costs M_x2 = -4.5 - (-5) = .5 -> hi_x2 = .25;  M_x3 = -3 - (-5) = 2
    -> hi_x3 = 1.
    X2 (x2,x3,x4), lambda = (.5, 2, 3):  M_x2 = 3.5 -> hi_x2 = -1.25;  then
    m1_x3 = 5, m0_x3 = min(0, -1.25 + 3) = 0 -> hi_x3 = -.5;  then
    m1_x4 = min(-1.25 + 3, -.5 + 3) = 1.75, m0_x4 = 0 -> hi_x4 = 2.125.
    Deferred sums (M-bar = 0 before the pass, so nothing is added back):
    D0 = (5, 0, 0, 0), D1 = (0, .5 + 3.5, 2 + 5, 1.75)."""
    p = oracle_mod.Problem.from_ilp(ilpgen.fig2_example())
    M = p.run_pass(True, 0.5)
    hi, lo, db0, db1 = p.state()
    assert np.array_equal(M, [-5, 0.5, 2, 3.5, 5, 1.75])
    assert np.array_equal(hi, [-5, 0.25, 1, -1.25, -0.5, 2.125])
    assert np.array_equal(lo, [-2.5, 0, 0, 0, 0, 0])
    assert np.array_equal(db0, [5, 0, 0, 0])
    assert np.array_equal(db1, [0, 4, 7, 1.75])


def test_fig2_bound_equals_optimum_and_rounding_stops_at_once(oracle_mod):
    ilp = ilpgen.fig2_example()
    opt, xopt = bf_optimum(ilp)
    assert opt == -5 and xopt == (1, 0, 0, 0)
    p = oracle_mod.Problem.from_ilp(ilp)
    assert p.lower_bounds() == (-5.0, -5.0)
    tr = p.iterate(40)
    assert np.all(tr == -5.0)  # monotone and bounded by OPT = initial bound
    r = p.round()
    assert r["status"] == 0 and r["rounds"] == 0
    assert list(r["x"]) == [1, 0, 0, 0] and r["objective"] == -5.0


# ----------------------------------------------------------------------------
# BDD construction and min-marginals against brute force
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(40))
def test_bdd_encodes_exactly_the_row(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    k = int(rng.integers(1, 9))
    a = [int(v) for v in rng.integers(1, 4, k) * rng.choice([-1, 1], k)]
    sense = int(rng.integers(-1, 2))
    x0 = rng.integers(0, 2, k)
    rhs = int(np.dot(a, x0)) + (0 if sense == 0 else int(rng.integers(-1, 2)))
    feas = row_feasible_set(a, sense, rhs)
    ilp = ilpgen.ILP(k, np.zeros(k), np.array([0, k]), np.arange(k, dtype=np.int32), np.array(a, np.int32),
                     np.array([sense], np.int8), np.array([rhs], np.int64))
    forced = [t for t in range(k) if len({x[t] for x in feas}) == 1]
    full = len(feas) == 2 ** k
    if not feas:
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.Problem.from_ilp(ilp)
        return
    p = oracle_mod.Problem.from_ilp(ilp)
    fixed = p.fixed()
    if full:
        assert p.m == 0 and np.all(fixed == 2)
        return
    if forced:
        # presolve fixes exactly the forced variables, to their forced value
        for t in forced:
            assert fixed[t] == next(iter(feas))[t]
        if p.m == 0:
            return
        # the remaining BDD encodes the projection on the free variables
        free = [t for t in range(k) if fixed[t] == -1]
        feas = {tuple(x[t] for t in free) for x in feas}
        a = [a[t] for t in free]
    ls, lo, hi = p.bdd_nodes(0)
    assert bdd_path_set(ls, lo, hi) == feas
    # reduced: no two nodes of a layer with the same successors, none dead
    for t in range(len(ls) - 1):
        pairs = [(lo[v], hi[v]) for v in range(ls[t], ls[t + 1])]
        assert len(set(pairs)) == len(pairs)
        assert all(pr != (-2, -2) for pr in pairs)


@pytest.mark.parametrize("seed", range(15))
def test_min_marginals_equal_bruteforce_at_random_multipliers(oracle_mod, seed):
    ilp = ilpgen.random_ilp(9, 6, seed, max_row=6)
    p = oracle_mod.Problem.from_ilp(ilp)
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(p.S)
    p.set_state(lam)
    m0, m1 = p.min_marginals()
    fixed = p.fixed()
    svar = p.slot_vars()
    for j in range(p.m):
        row, k, _, s0 = p.bdd_info(j)
        cols, coefs, sense, rhs = ordered_row(ilp, row)
        shift = sum(a * int(fixed[c]) for c, a in zip(cols, coefs) if fixed[c] in (0, 1))
        keep = [(c, a) for c, a in zip(cols, coefs) if fixed[c] == -1]
        assert [c for c, _ in keep] == list(svar[s0:s0 + k])
        feas = row_feasible_set([a for _, a in keep], sense, rhs - shift)
        b0, b1 = bf_min_marginals(feas, lam[s0:s0 + k])
        assert np.allclose(m0[s0:s0 + k], b0, rtol=0, atol=1e-12)
        assert np.allclose(m1[s0:s0 + k], b1, rtol=0, atol=1e-12)


def lifted_energy_bruteforce(p, ilp, hi, lo):
    fixed = p.fixed()
    total = p.const_lb
    for j in range(p.m):
        row, k, _, s0 = p.bdd_info(j)
        cols, coefs, sense, rhs = ordered_row(ilp, row)
        shift = sum(a * int(fixed[c]) for c, a in zip(cols, coefs) if fixed[c] in (0, 1))
        keep = [a for c, a in zip(cols, coefs) if fixed[c] == -1]
        feas = row_feasible_set(keep, sense, rhs - shift)
        h, l_ = hi[s0:s0 + k], lo[s0:s0 + k]
        total += min(sum(h[t] if x[t] else l_[t] for t in range(k)) for x in feas)
    return total


@pytest.mark.parametrize("seed", range(12))
def test_prop1_invariants_and_bounds(oracle_mod, seed):
    """Prop. 1: after every pass  sum_j lambda^j_i + omega M_ij = c_i  (here in
    the lifted form: sum_j hi + omega D1 = c_i and sum_j lo + omega D0 = 0),
    the lifted bound is non-decreasing, it equals the brute-force lifted
    energy, it never exceeds the enumerated optimum, and after the final
    add-back the multipliers are dual feasible."""
    ilp = ilpgen.random_ilp(10, 7, 100 + seed, max_row=5)
    opt, _ = bf_optimum(ilp)
    p = oracle_mod.Problem.from_ilp(ilp)
    svar = p.slot_vars()
    fixed = p.fixed()
    inb = fixed == -1
    omega = [0.5, 0.3, 1.0][seed % 3]
    prev = -np.inf
    for it in range(6):
        for fwd in (True, False):
            p.run_pass(fwd, omega)
            hi, lo, db0, db1 = p.state()
            shi = np.bincount(svar, hi, minlength=ilp.n_vars)
            slo = np.bincount(svar, lo, minlength=ilp.n_vars)
            assert np.allclose((shi + omega * db1)[inb], ilp.cost[inb], atol=1e-10)
            assert np.allclose((slo + omega * db0)[inb], 0.0, atol=1e-10)
            run, fea = p.lower_bounds(omega)
            assert run >= prev - 1e-10
            assert fea >= run - 1e-10
            assert run <= opt + 1e-9 and fea <= opt + 1e-9
            assert abs(run - lifted_energy_bruteforce(p, ilp, hi, lo)) < 1e-9
            prev = run
    run, fea = p.lower_bounds(omega)
    p.addback(omega)
    hi, lo, _, _ = p.state()
    lam = hi - lo
    assert np.allclose(np.bincount(svar, lam, minlength=ilp.n_vars)[inb], ilp.cost[inb], atol=1e-10)
    run2, fea2 = p.lower_bounds(omega)
    assert abs(run2 - fea) < 1e-9 and abs(fea2 - fea) < 1e-9


def test_subtracting_own_min_marginal_keeps_energy(oracle_mod):
    """The step of the Prop. 1 proof, in the lifted form: hi_t -= omega max(d, 0),
    lo_t -= omega max(-d, 0) with d = m1_t - m0_t leaves the lifted energy
    min_x sum_t (x_t hi_t + (1 - x_t) lo_t) unchanged (checked by enumeration)."""
    rng = np.random.default_rng(7)
    for trial in range(30):
        ilp = ilpgen.random_ilp(6, 1, 500 + trial, max_row=6)
        p = oracle_mod.Problem.from_ilp(ilp)
        if p.m == 0:
            continue
        lam = rng.standard_normal(p.S)
        p.set_state(lam)
        m0, m1 = p.min_marginals()
        row, k, _, s0 = p.bdd_info(0)
        cols, coefs, sense, rhs = ordered_row(ilp, row)
        fixed = p.fixed()
        shift = sum(a * int(fixed[c]) for c, a in zip(cols, coefs) if fixed[c] in (0, 1))
        feas = row_feasible_set([a for c, a in zip(cols, coefs) if fixed[c] == -1], sense, rhs - shift)

        def lifted(hi, lo):
            return min(sum(hi[t] if x[t] else lo[t] for t in range(k)) for x in feas)

        e = lifted(lam, np.zeros(k))
        for t in range(k):
            d = m1[t] - m0[t]
            for omega in (0.5, 1.0):
                hi, lo = lam.copy(), np.zeros(k)
                hi[t] -= omega * max(d, 0.0)
                lo[t] -= omega * max(-d, 0.0)
                assert abs(lifted(hi, lo) - e) < 1e-12
                # the plain multiplier moves by -omega d; its energy rises by omega max(-d, 0)
                lam2 = lam.copy()
                lam2[t] -= omega * d
                assert abs(min(np.dot(x, lam2) for x in feas) - (e + omega * max(-d, 0.0))) < 1e-12


def test_simplex_closed_form(oracle_mod):
    """One row sum_i x_i = 1: E = min_i c_i, m1_i = c_i, m0_i = min_{k != i} c_k."""
    rng = np.random.default_rng(3)
    for k in (2, 3, 7, 16):
        c = rng.standard_normal(k)
        ilp = ilpgen.ILP(k, c, np.array([0, k]), np.arange(k, dtype=np.int32), np.ones(k, np.int32),
                         np.array([0], np.int8), np.array([1], np.int64))
        p = oracle_mod.Problem.from_ilp(ilp)
        assert p.N == 1 + 2 * (k - 1)
        m0, m1 = p.min_marginals()
        assert np.array_equal(m1, c)
        assert np.array_equal(m0, [np.min(np.delete(c, i)) for i in range(k)])
        assert p.lower_bounds() == (c.min(), c.min())


@pytest.mark.parametrize("seed", range(3))
def test_chain_mrf_bound_reaches_viterbi_optimum(oracle_mod, seed):
    """A chain MRF's local polytope is tight, so the bound is at most the
    Viterbi optimum and the averaging reaches it."""
    W, L = 12, 4
    g = ilpgen.mrf_grid(1, W, L, seed, potts_max=2.0)
    un, wE = g.meta["unary"], g.meta["potts"]
    best = un[0].copy()
    for c in range(1, W):
        pen = wE[c - 1] * (np.arange(L)[:, None] != np.arange(L)[None, :])
        best = (best[:, None] + pen).min(0) + un[c]
    viterbi = best.min()
    p = oracle_mod.Problem.from_ilp(g)
    tr = p.iterate(300)
    assert np.all(np.diff(tr) >= -1e-12)
    assert tr[-1] <= viterbi + 1e-9
    assert tr[-1] >= viterbi - 1e-8


@pytest.mark.parametrize("seed", range(3))
def test_potts_grid_bound_reaches_min_cut(oracle_mod, seed):
    """2-label attractive Potts energies are submodular: the LP is tight and
    the optimum is a minimum s-t cut."""
    H = W = 5
    g = ilpgen.mrf_grid(H, W, 2, seed, potts_max=1.0)
    un, wE, E = g.meta["unary"], g.meta["potts"], g.meta["edges"]
    G = nx.DiGraph()
    const = 0.0
    for u in range(H * W):
        m = min(un[u, 0], un[u, 1])
        const += m
        G.add_edge("s", u, capacity=un[u, 1] - m)
        G.add_edge(u, "t", capacity=un[u, 0] - m)
    for (u, v), w in zip(E, wE):
        G.add_edge(int(u), int(v), capacity=w)
        G.add_edge(int(v), int(u), capacity=w)
    cut, _ = nx.minimum_cut(G, "s", "t")
    opt = cut + const
    p = oracle_mod.Problem.from_ilp(g)
    tr = p.iterate(500)
    assert tr[-1] <= opt + 1e-9
    assert tr[-1] >= opt - 1e-8
    r = p.round()
    assert r["status"] == 0 and g.feasible(r["x"])
    assert abs(r["objective"] - opt) < 1e-8


# ----------------------------------------------------------------------------
# rounding, presolve, RNG
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(12))
def test_rounding_returns_feasible_point_above_bound(oracle_mod, seed):
    ilp = ilpgen.random_ilp(11, 8, 300 + seed, max_row=4, max_coef=1)
    opt, _ = bf_optimum(ilp)
    p = oracle_mod.Problem.from_ilp(ilp)
    p.iterate(30)
    _, fea = p.lower_bounds()
    r = p.round(seed=seed)
    if r["status"] == 0:
        assert ilp.feasible(r["x"])
        assert r["objective"] >= opt - 1e-9 >= fea - 1e-6
        assert abs(r["objective"] - ilp.objective(r["x"])) < 1e-12
    else:
        assert r["status"] == oracle_mod.ENOCONVERGE


def _two_var_rounding_rounds(oracle_mod, seed, alpha=1.2):
    """Expected multipliers after two rounds of Alg. 2 on x0 + x1 <= 1 and
    x0 + x1 >= 1 with zero costs and no re-optimisation, worked out from the
    closed-form min-marginals of two-variable rows (lambda^j_i = p_i in both):
      x0 + x1 <= 1:  m1(x0) = p0,              m0(x0) = min(0, p1)
      x0 + x1 >= 1:  m1(x0) = p0 + min(0, p1), m0(x0) = p1
    Round 0 sees M = 0 everywhere (zero costs), so each variable moves by
    r delta with r drawn from [-delta, delta), delta = 1.  Round 1 has
    delta = alpha."""
    u = lambda rnd, i: oracle_mod.uniform_pm1(seed, rnd, i)
    p = [u(0, 0) * 1.0 * 1.0, u(0, 1) * 1.0 * 1.0]
    d1 = alpha
    q, conflict = [], []
    for i in (0, 1):
        a, b = p[i], p[1 - i]
        m_le = a - min(0.0, b)
        m_ge = a + min(0.0, b) - b
        ms = [m_le, m_ge]
        r = u(1, i) * d1
        if all(m > 0 for m in ms):
            q.append(d1); conflict.append(False)
        elif all(m < 0 for m in ms):
            q.append(-d1); conflict.append(False)
        elif all(m == 0 for m in ms):
            q.append(r * d1); conflict.append(False)
        else:
            tot = m_le + m_ge
            sg = 1.0 if tot > 0 else (-1.0 if tot < 0 else (1.0 if r >= 0 else -1.0))
            q.append(sg * abs(r) * d1); conflict.append(True)
    return p, q, conflict


def test_rounding_perturbation_worked_example(oracle_mod):
    """The perturbation step of Alg. 2, two rounds, with r drawn from
    [-delta, delta) and pushed as r delta: a conflicting variable in round 1
    moves by up to alpha^2 = 1.44 (a draw from [-1, 1) would give at most
    1.2).  Seeds are scanned for one whose round 1 has a conflict."""
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], -1, 1)
    rb.add([0, 1], [1, 1], 1, 1)
    ilp = rb.finish(2, np.zeros(2), "two-var")
    checked = 0
    for seed in range(64):
        p, q, conflict = _two_var_rounding_rounds(oracle_mod, seed)
        if not any(conflict):
            continue
        prob = oracle_mod.Problem.from_ilp(ilp)
        prob.round(omega=0.5, delta=1.0, alpha=1.2, kr=0, max_rounds=2, seed=seed)
        hi, lo, _, _ = prob.state()
        lam = hi - lo
        var = prob.slot_vars()
        want = np.array([p[v] + q[v] for v in var])
        assert np.allclose(lam, want, rtol=0, atol=1e-12), (seed, lam, want)
        checked += 1
        if any(c and abs(q[i]) > 1.2 for i, c in enumerate(conflict)):
            break
    assert checked > 0 and any(c and abs(q[i]) > 1.2 for i, c in enumerate(conflict))


# ----------------------------------------------------------------------------
# the serial min-marginal averaging of Eq. 4
# ----------------------------------------------------------------------------
def test_serial_averaging_worked_example(oracle_mod):
    """One iteration of Eq. 4 by hand on x0 + x1 <= 1 (BDD 0) and x0 + x1 >= 1
    (BDD 1), costs (2, -1), lambda = c / 2 initially.  Two-variable rows have
    closed-form min-marginals: for <= 1, m1(x0) = l0, m0(x0) = min(0, l1); for
    >= 1, m1(x0) = l0 + min(0, l1), m0(x0) = l1 (and symmetrically for x1).
    Ascending x0: M = (1.5, 1.0), average 1.25 -> lambda_0 = (0.75, 1.25);
    x1: M = (-0.5, -1.75), average -1.125 -> lambda_1 = (-1.125, 0.125);
    descending x1: M = (-1.125, -1.125), no change; x0: M = (1.875, 1.125),
    average 1.5 -> lambda_0 = (0.375, 1.625).  Bound -1.125 + 0.125 = -1 =
    OPT.  All values are dyadic, so exact."""
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], -1, 1)
    rb.add([0, 1], [1, 1], 1, 1)
    ilp = rb.finish(2, np.array([2.0, -1.0]), "serial-example")
    p = oracle_mod.Problem.from_ilp(ilp)
    tr = p.iterate_serial(1)
    hi, lo, _, _ = p.state()
    assert list(hi - lo) == [0.375, -1.125, 1.625, 0.125]
    assert tr[0] == -1.0


@pytest.mark.parametrize("seed", range(6))
def test_serial_averaging_invariants(oracle_mod, seed):
    """Eq. 4 keeps sum_j lambda^j_i = c_i, never lowers the bound (block
    coordinate ascent), stays below the brute-force optimum, and leaves the
    copies of the last variable it visits (variable 0, at the end of the
    descending sweep) with one common min-marginal difference."""
    ilp = ilpgen.random_ilp(11, 8, 500 + seed, max_row=4, max_coef=2)
    opt, _ = bf_optimum(ilp)
    p = oracle_mod.Problem.from_ilp(ilp)
    tr = p.iterate_serial(8)
    assert np.all(np.diff(tr) >= -1e-9 * max(1.0, abs(tr[-1])))
    assert tr[-1] <= opt + 1e-9
    hi, lo, _, _ = p.state()
    var = p.slot_vars()
    s = np.bincount(var, hi - lo, minlength=ilp.n_vars)
    inb = np.bincount(var, minlength=ilp.n_vars) > 0
    assert np.allclose(s[inb], np.asarray(ilp.cost)[inb], atol=1e-12)
    m0, m1 = p.min_marginals()
    d0 = (m1 - m0)[var == 0]
    if len(d0) > 1:
        assert np.allclose(d0, d0[0], atol=1e-9 * max(1.0, np.abs(d0).max()))


@pytest.mark.parametrize("seed", range(3))
def test_serial_averaging_chain_reaches_viterbi(oracle_mod, seed):
    """On a chain MRF (a tree, tight local polytope) the serial scheme reaches
    the Viterbi optimum computed by dynamic programming."""
    W, L = 12, 4
    g = ilpgen.mrf_grid(1, W, L, seed, potts_max=2.0)
    un, wE = g.meta["unary"], g.meta["potts"]
    best = un[0].copy()
    for c in range(1, W):
        pen = wE[c - 1] * (np.arange(L)[:, None] != np.arange(L)[None, :])
        best = (best[:, None] + pen).min(0) + un[c]
    viterbi = best.min()
    p = oracle_mod.Problem.from_ilp(g)
    tr = p.iterate_serial(60)
    assert np.all(np.diff(tr) >= -1e-9 * max(1.0, abs(tr[-1])))
    assert tr[-1] <= viterbi + 1e-9
    assert tr[-1] >= viterbi - 1e-8


def test_tiny_mrf_sizes_and_rounding(oracle_mod):
    g = ilpgen.mrf_grid(8, 8, 3, 0)
    p = oracle_mod.Problem.from_ilp(g)
    assert (g.n_vars, p.m, p.S, p.N) == (1200, 736, 2880, 5024)
    tr = p.iterate(200)
    assert np.all(np.diff(tr) >= -1e-12)
    r = p.round()
    assert r["status"] == 0 and g.feasible(r["x"]) and r["objective"] >= tr[-1] - 1e-9


def test_presolve_fixes_forced_variables(oracle_mod):
    # x0 + x1 = 2 forces x0 = x1 = 1; then x1 + x2 <= 1 forces x2 = 0;
    # x3 - x4 = 0 stays; x5 is in no row.
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], 0, 2)
    rb.add([1, 2], [1, 1], -1, 1)
    rb.add([3, 4], [1, -1], 0, 0)
    c = np.array([1.0, 2.0, -3.0, -1.0, 0.5, -0.25])
    ilp = rb.finish(6, c, "forced")
    p = oracle_mod.Problem.from_ilp(ilp)
    assert list(p.fixed()) == [1, 1, 0, -1, -1, 2]
    assert p.m == 1 and p.const_lb == 1.0 + 2.0 - 0.25
    tr = p.iterate(20)
    opt, xo = bf_optimum(ilp)
    assert tr[-1] <= opt + 1e-12
    r = p.round()
    assert r["status"] == 0 and list(r["x"]) == list(xo)


def test_infeasible_rows_are_reported(oracle_mod):
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], 0, 2)
    rb.add([0], [1], -1, 0)
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.Problem.from_ilp(rb.finish(2, [0.0, 0.0], "infeasible"))
    assert e.value.code == oracle_mod.EINFEASIBLE


def test_splitmix64_published_vector(oracle_mod):
    # first output of SplitMix64 seeded with 0 (published reference value)
    assert oracle_mod.splitmix64(0) == 0xE220A8397B1DCDAF


def test_uniform_draws_cover_the_interval(oracle_mod):
    r = np.array([oracle_mod.uniform_pm1(9, rd, v) for rd in range(4) for v in range(2000)])
    assert r.min() >= -1.0 and r.max() < 1.0
    assert abs(r.mean()) < 0.03 and abs(r.std() - 1 / np.sqrt(3)) < 0.02
    assert len(np.unique(r)) == len(r)


def test_energies_sum_to_the_running_bound(oracle_mod):
    ilp = ilpgen.random_ilp(9, 7, 4242, max_row=5)
    p = oracle_mod.Problem.from_ilp(ilp)
    p.iterate(3)
    run, _ = p.lower_bounds()
    assert abs(p.energies().sum() + p.const_lb - run) < 1e-12
    hi, lo, _, _ = p.state()
    assert abs(p.energies().sum() + p.const_lb - lifted_energy_bruteforce(p, ilp, hi, lo)) < 1e-9


def test_stored_lb_star_trajectory_is_monotone():
    """The stored 2,000-iteration oracle bound of the 512x512 grid (written by
    tests/golden/make_mrf512_lb_star.py): the lifted bound never decreases
    (Prop. 1), and LB* is the bound after the last iteration."""
    import os

    rec = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "mrf512_lb_star.txt")) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
    its = [100, 200, 500, 1000, 1500, 2000]
    tr = [float(rec[f"lb_after_{k}"]) for k in its]
    assert int(rec["iterations"]) == 2000
    assert all(b >= a for a, b in zip(tr, tr[1:]))
    assert float(rec["lb_star"]) == tr[-1]
