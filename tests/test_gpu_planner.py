"""Device-side BDD construction (params.planner): the decomposition the GPU
builds equals the host builder's part by part (plan digests: presolve,
shapes and templates, tiles, slot variables, slot lists, tile-local
patterns, deferred-sum buckets, BDD-row maps, counts), so every later
result is bit-identical; instances the device builder does not take are
planned on the host (planner 0) or refused (planner 2)."""
import dataclasses

import numpy as np
import pytest

import ilpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    return P


def built(P, ilp, planner, **kw):
    kw.setdefault("tol", 0.0)
    return P.Instance.from_ilp(ilp, planner=planner, **kw).build(0)


def with_free_variables(ilp, extra):
    """The ILP with `extra` variables that appear in no row (costs of both signs)."""
    cost = np.concatenate([ilp.cost, np.linspace(-1.5, 1.0, extra)])
    return dataclasses.replace(ilp, n_vars=ilp.n_vars + extra, cost=cost)


CASES = {
    "mrf8": lambda: ilpgen.mrf_grid(8, 8, 3, seed=0),
    "mrf48": lambda: ilpgen.mrf_grid(48, 48, 4, seed=5, potts_max=2.0),
    "mrf37_free": lambda: with_free_variables(ilpgen.mrf_grid(37, 29, 2, seed=6), 11),
    "qap": lambda: ilpgen.qap(seed=2, n_left=60, n_right=120, n_cand=8, k_nn=4),
    "cell": lambda: ilpgen.cell_tracking(seed=7, frames=6, det_lo=50, det_hi=120),
    "random": lambda: ilpgen.random_ilp(400, 300, seed=3),
}


@pytest.mark.parametrize("jit,fuse", [(0, 0), (1, 0), (-1, -1)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_device_plan_equals_host_plan(P, name, jit, fuse):
    ilp = CASES[name]()
    h = built(P, ilp, 1, jit=jit, fuse=fuse)
    d = built(P, ilp, 0, jit=jit, fuse=fuse)
    assert not h.plan_stats()[0]
    if name != "random":  # structured families need no presolve: the device builds them
        assert d.plan_stats()[0]
    dh, dd = h.plan_digest(), d.plan_digest()
    assert np.array_equal(dh, dd), [i for i in range(len(dh)) if dh[i] != dd[i]]
    assert h.kernel_plan() == d.kernel_plan()


@pytest.mark.parametrize("name", ["mrf48", "cell", "qap"])
def test_device_planned_solve_is_bit_identical(P, name):
    ilp = CASES[name]()
    h = built(P, ilp, 1)
    d = built(P, ilp, 2)
    assert d.plan_stats()[0]
    for k in (1, 7, 30):
        assert h.iterate(k) == d.iterate(k)
    assert h.lower_bound() == d.lower_bound()
    vh, rh, m0h, m1h = h.min_marginals()
    vd, rd, m0d, m1d = d.min_marginals()
    for a, b in ((vh, vd), (rh, rd), (m0h, m0d), (m1h, m1d)):
        assert np.array_equal(a, b)
    assert h.primal_round() == d.primal_round()
    xh, oh, fh = h.solution()
    xd, od, fd = d.solution()
    assert np.array_equal(xh, xd) and oh == od and fh == fd


def test_presolve_instances_fall_back_or_are_refused(P):
    # row 0 forces x0 = x1 = 1; the rest is a small MRF over other variables
    base = ilpgen.mrf_grid(4, 4, 2, seed=1)
    n = base.n_vars + 2
    row_ptr = np.concatenate([[0], base.row_ptr + 2]).astype(np.int64)
    col = np.concatenate([[base.n_vars, base.n_vars + 1], base.col]).astype(np.int32)
    coef = np.concatenate([[1, 1], base.coef]).astype(np.int32)
    sense = np.concatenate([[1], base.sense]).astype(np.int8)
    rhs = np.concatenate([[2], base.rhs]).astype(np.int64)
    ilp = dataclasses.replace(base, n_vars=n, cost=np.concatenate([base.cost, [0.5, -0.25]]), row_ptr=row_ptr,
                              col=col, coef=coef, sense=sense, rhs=rhs)
    h = built(P, ilp, 1)
    d = built(P, ilp, 0)
    assert not d.plan_stats()[0]
    assert np.array_equal(h.plan_digest(), d.plan_digest())
    with pytest.raises(P.FdogError) as err:
        built(P, ilp, 2)
    assert err.value.code == P.capi.FDOG_EUNSUPPORTED


def test_infeasible_row_reports_the_same_error(P):
    base = ilpgen.mrf_grid(4, 4, 2, seed=2)
    # the last row asks more than its variables can give
    rhs = base.rhs.copy()
    last = len(rhs) - 1
    k = int(base.row_ptr[last + 1] - base.row_ptr[last])
    ilp = dataclasses.replace(base, sense=np.concatenate([base.sense[:-1], [1]]).astype(np.int8),
                              rhs=np.concatenate([rhs[:-1], [k + 5]]).astype(np.int64))
    codes = []
    for planner in (1, 0):
        with pytest.raises(P.FdogError) as err:
            built(P, ilp, planner)
        codes.append(err.value.code)
    assert codes == [P.capi.FDOG_EINFEASIBLE] * 2


def test_release_rebuild_and_checkpoint_of_a_device_plan(P):
    ilp = CASES["mrf48"]()
    d = built(P, ilp, 2)
    d.iterate(5)
    blob = d.export_state()  # reads the plan back for the layout fingerprint
    lb = d.lower_bound()
    dig = d.plan_digest()
    d.release()
    d.build(0)
    assert np.array_equal(d.plan_digest(), dig)
    d.import_state(blob)
    assert d.lower_bound() == lb
    h = built(P, ilp, 1)
    h.import_state(blob)  # same layout fingerprint as the device plan
    assert d.iterate(3) == h.iterate(3)


def test_full_size_mrf_device_plan_equals_host_plan(P):
    ilp = ilpgen.mrf_grid(512, 512, 4, seed=1, potts_max=2.0)
    h = built(P, ilp, 1, tol=1e-4)
    d = built(P, ilp, 2, tol=1e-4)
    on_dev, sec = d.plan_stats()
    assert on_dev and sec > 0
    assert np.array_equal(h.plan_digest(), d.plan_digest())


def rows_ilp(n, rows, seed):
    """ILP from (cols, coefs, sense, rhs) rows with normal costs."""
    rng = np.random.default_rng(seed)
    row_ptr = np.cumsum([0] + [len(r[0]) for r in rows]).astype(np.int64)
    return ilpgen.ILP(n, rng.normal(size=n), row_ptr, np.concatenate([r[0] for r in rows]).astype(np.int32),
                      np.concatenate([r[1] for r in rows]).astype(np.int32),
                      np.array([r[2] for r in rows], np.int8), np.array([r[3] for r in rows], np.int64))


def many_signatures():
    """1,080 distinct row signatures (sum x <= b for every length k in 2..80
    and b in 1..min(15, k - 1)): more than the device builder takes."""
    rng = np.random.default_rng(7)
    rows = [(np.sort(rng.choice(3000, k, replace=False)), np.ones(k, int), -1, b)
            for k in range(2, 81) for b in range(1, min(15, k - 1) + 1)]
    return rows_ilp(3000, rows, 7)


def hub_variable():
    """x_0 + x_j <= 1 for j = 1..5000: x_0 has 5,000 copies."""
    return rows_ilp(5001, [(np.array([0, j]), np.ones(2, int), -1, 1) for j in range(1, 5001)], 8)


def unsorted_rows():
    """A small MRF with every row listed in descending column order."""
    g = ilpgen.mrf_grid(6, 6, 3, seed=9)
    col, coef = g.col.copy(), g.coef.copy()
    for j in range(len(g.row_ptr) - 1):
        b, e = g.row_ptr[j], g.row_ptr[j + 1]
        col[b:e], coef[b:e] = col[b:e][::-1], coef[b:e][::-1]
    return dataclasses.replace(g, col=col, coef=coef)


@pytest.mark.parametrize("make", [many_signatures, hub_variable, unsorted_rows],
                         ids=["signatures", "copies", "unsorted"])
def test_instances_beyond_the_device_builder_fall_back(P, make):
    ilp = make()
    h = built(P, ilp, 1)
    d = built(P, ilp, 0)
    assert not d.plan_stats()[0]
    assert np.array_equal(h.plan_digest(), d.plan_digest())
    assert h.iterate(5) == d.iterate(5)
    with pytest.raises(P.FdogError) as err:
        built(P, ilp, 2)
    assert err.value.code == P.capi.FDOG_EUNSUPPORTED
