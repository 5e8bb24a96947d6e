"""CPU tests of the C-ABI library: it loads, exports what include/fastdog.h
declares, validates inputs, and its host-side planning (presolve, BDD
construction, layout) agrees with the independent oracle and with brute
force.  No compute call needs a GPU here."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import ilpgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    return P


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fastdog.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdog_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(P):
    names = declared_symbols()
    assert len(names) >= 20
    L = P.lib()
    for n in names:
        assert hasattr(L, n), n
    # and the binding describes every one of them
    from paper_2111_10270_gb300.capi import SIGNATURES

    assert sorted(SIGNATURES) == names


def test_params_defaults(P):
    p = P.capi.default_params()
    assert (p.omega, p.delta, p.alpha, p.tol) == (0.5, 1.0, 1.2, 1e-4)
    assert (p.window, p.min_iters, p.rounding_dual_iters, p.max_rounds) == (10, 20, 20, 200)
    assert (p.update, p.planner) == (0, 0)


def test_create_rejects_malformed_input(P):
    g = ilpgen.fig2_example()
    cases = []
    bad = g.col.copy(); bad[0] = 99
    cases.append(dict(col=bad))
    bad = g.col.copy(); bad[1] = bad[0]
    cases.append(dict(col=bad))
    bad = g.sense.copy(); bad[0] = 3
    cases.append(dict(sense=bad))
    bad = g.row_ptr.copy(); bad[1] = 5; bad[2] = 4
    cases.append(dict(row_ptr=bad))
    bad = g.cost.copy(); bad[2] = np.nan
    cases.append(dict(cost=bad))
    for kw in cases:
        args = dict(n_vars=g.n_vars, cost=g.cost, row_ptr=g.row_ptr, col=g.col, coef=g.coef, sense=g.sense, rhs=g.rhs)
        args.update(kw)
        with pytest.raises(P.FdogError) as e:
            P.Instance(**args)
        assert e.value.code == P.FDOG_EINVAL
    # a row listed out of column order is valid; a repeat anywhere in it is not
    b0, b1 = int(g.row_ptr[0]), int(g.row_ptr[1])
    assert b1 - b0 >= 3
    perm = g.col.copy(); perm[b0:b1] = perm[b0:b1][::-1]
    P.Instance(n_vars=g.n_vars, cost=g.cost, row_ptr=g.row_ptr, col=perm, coef=g.coef, sense=g.sense, rhs=g.rhs)
    rep = perm.copy(); rep[b1 - 1] = rep[b0]
    with pytest.raises(P.FdogError) as e:
        P.Instance(n_vars=g.n_vars, cost=g.cost, row_ptr=g.row_ptr, col=rep, coef=g.coef, sense=g.sense, rhs=g.rhs)
    assert e.value.code == P.FDOG_EINVAL
    for kw in (dict(omega=0.0), dict(omega=1.5), dict(window=0), dict(block_threads=48), dict(planner=3)):
        with pytest.raises(P.FdogError) as e:
            P.Instance.from_ilp(g, **kw)
        assert e.value.code == P.FDOG_EINVAL


def test_calls_before_build_report_state_errors(P):
    inst = P.Instance.from_ilp(ilpgen.fig2_example())
    with pytest.raises(P.FdogError) as e:
        inst.iterate(1)
    assert e.value.code == P.FDOG_ESTATE
    with pytest.raises(P.FdogError) as e:
        inst.solution()
    assert e.value.code == P.FDOG_ESTATE


def path_set(ls, lo, hi):
    k = len(ls) - 1
    out = set()

    def walk(v, t, acc):
        if v == -1:
            out.add(tuple(acc))
        elif v >= 0:
            assert ls[t] <= v < ls[t + 1]
            walk(lo[v], t + 1, acc + [0])
            walk(hi[v], t + 1, acc + [1])

    walk(0, 0, [])
    return out


def feasible_set(coefs, sense, rhs):
    out = set()
    for x in itertools.product((0, 1), repeat=len(coefs)):
        s = int(np.dot(coefs, x))
        if (sense <= 0 and s > rhs) or (sense >= 0 and s < rhs):
            continue
        out.add(x)
    return out


@pytest.mark.parametrize("seed", range(25))
def test_planned_bdds_encode_rows_and_match_oracle(P, oracle_mod, seed):
    ilp = ilpgen.random_ilp(10, 8, 2000 + seed, max_row=7, max_coef=3)
    inst = P.Instance.from_ilp(ilp)
    inst.plan()
    orc = oracle_mod.Problem.from_ilp(ilp)
    fixed = inst.fixed_vars()
    assert np.array_equal(fixed, orc.fixed())
    info = inst.info()
    assert (info["n_bdds"], info["n_slots"], info["n_nodes"]) == (orc.m, orc.S, orc.N)
    for j in range(ilp.n_rows):
        got = inst.row_bdd(j)
        cols, coefs, sense, rhs = ilp.row(j)
        if got is None:
            continue
        vars_, ls, lo, hi = got
        assert list(vars_) == sorted(c for c in cols if fixed[c] == -1)
        shift = sum(int(a) * int(fixed[c]) for c, a in zip(cols, coefs) if fixed[c] in (0, 1))
        keep = [int(dict(zip(cols, coefs))[v]) for v in vars_]
        assert path_set(ls, lo, hi) == feasible_set(keep, sense, rhs - shift)


def test_tiny_mrf_plan_sizes(P):
    g = ilpgen.mrf_grid(8, 8, 3, 0)
    inst = P.Instance.from_ilp(g)
    dev_bytes = inst.plan()
    info = inst.info()
    assert (info["n_vars"], info["n_bdds"], info["n_slots"], info["n_nodes"]) == (1200, 736, 2880, 5024)
    assert dev_bytes > 0


def test_wide_and_long_rows_plan(P, oracle_mod):
    # widths beyond the register classes and rows longer than 8 variables
    rb = ilpgen._RowBuilder()
    rb.add(range(12), [1] * 12, -1, 5)       # cardinality <= 5: width 6
    rb.add(range(20), [1] * 20, 0, 1)        # simplex of 20
    rb.add(range(6), [3, -2, 2, 1, -1, 2], -1, 3)
    ilp = rb.finish(20, np.linspace(-1, 1, 20), "wide")
    inst = P.Instance.from_ilp(ilp)
    inst.plan()
    orc = oracle_mod.Problem.from_ilp(ilp)
    info = inst.info()
    assert (info["n_bdds"], info["n_slots"], info["n_nodes"]) == (orc.m, orc.S, orc.N)


def test_specialised_kernels_compile_on_the_host(P):
    """The shape-specialised kernels are generated and compiled with NVRTC
    while planning (no GPU needed): with jit=1 every narrow short shape gets
    one; in the default mode only shapes with at least 4096 BDDs do."""
    g = ilpgen.mrf_grid(8, 8, 3, 0)
    inst = P.Instance.from_ilp(g, jit=1)
    inst.plan()
    kp = inst.kernel_plan()
    assert kp["note"] == "" and kp["jit_shapes"] == 2 and kp["static_tiles"] == 0
    auto = P.Instance.from_ilp(g)
    auto.plan()
    assert auto.kernel_plan()["jit_shapes"] == 0
    # 48 x 48 grid, 3 labels: 2304 simplex rows stay generic, 4512 x 6 marginalisation rows are specialised
    big = P.Instance.from_ilp(ilpgen.mrf_grid(48, 48, 3, 0))
    big.plan()
    kb = big.kernel_plan()
    assert kb["jit_shapes"] == 1 and kb["jit_tiles"] == 4512 * 6 // 32 and kb["static_tiles"] == 2304 // 32
    # the 8 marginalisation rows of an edge share its 9 pairwise variables; 4 edges per tile
    assert kp["local_vars"] > 0
    off = P.Instance.from_ilp(g, jit=-1)
    off.plan()
    kp = off.kernel_plan()
    assert kp["jit_shapes"] == 0 and kp["jit_tiles"] == 0 and kp["static_tiles"] > 0
    # random rows of many shapes, including ones too wide or long for the specialised code
    ilp = ilpgen.random_ilp(60, 50, 77, max_row=20, max_coef=2)
    inst = P.Instance.from_ilp(ilp, jit=1)
    inst.plan()
    kp = inst.kernel_plan()
    assert kp["note"] == "" and kp["jit_shapes"] > 0


def test_infeasible_instance_is_reported(P):
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], 0, 2)
    rb.add([0], [1], -1, 0)
    inst = P.Instance.from_ilp(rb.finish(2, [0.0, 0.0], "infeasible"))
    with pytest.raises(P.FdogError) as e:
        inst.plan()
    assert e.value.code == P.FDOG_EINFEASIBLE


def test_build_without_gpu_fails_loudly(P):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    inst = P.Instance.from_ilp(ilpgen.fig2_example())
    with pytest.raises(P.FdogError):
        inst.build(0)


def test_plan_digest_and_stats_on_host_plans(P):
    g = ilpgen.mrf_grid(6, 5, 3, seed=4)
    a = P.Instance.from_ilp(g)
    a.plan()
    b = P.Instance.from_ilp(g)
    b.plan()
    on_dev, sec = a.plan_stats()
    assert not on_dev and sec > 0
    da, db = a.plan_digest(), b.plan_digest()
    assert len(da) == P.capi.PLAN_DIGESTS and np.array_equal(da, db)
    # one right-hand side changed: the presolve constants and layout stay, the shapes do not
    rhs = g.rhs.copy()
    j = int(np.argmax(np.diff(g.row_ptr)))
    rhs[j] += 1
    c = P.Instance(n_vars=g.n_vars, cost=g.cost, row_ptr=g.row_ptr, col=g.col, coef=g.coef, sense=g.sense, rhs=rhs)
    c.plan()
    dc = c.plan_digest()
    assert dc[1] != da[1]
    # costs only enter the presolve constants (none here: every variable is in a row)
    d = P.Instance(n_vars=g.n_vars, cost=g.cost + 1.0, row_ptr=g.row_ptr, col=g.col, coef=g.coef, sense=g.sense,
                   rhs=g.rhs)
    d.plan()
    assert np.array_equal(d.plan_digest(), da)
    with pytest.raises(P.FdogError) as e:
        P.Instance.from_ilp(g).plan_digest()
    assert e.value.code == P.FDOG_ESTATE


def test_host_cache_reuses_and_releases_buffers(P):
    """Large host arrays that an instance frees are kept for the next instance
    of the same sizes; fdog_host_cache_release frees them and reports their
    bytes.  Instances built on reused buffers hold their own ILP exactly."""
    P.host_cache_release()
    g = ilpgen.mrf_grid(200, 200, 4, 3)
    nnz = int(g.row_ptr[-1])
    assert 4 * nnz >= 1 << 20  # the column and coefficient copies are large enough to be cached
    a = P.Instance.from_ilp(g)
    a.plan()
    da = a.plan_digest()
    a.close()
    kept = P.host_cache_release()
    assert kept >= 2 * 4 * nnz
    assert P.host_cache_release() == 0
    b = P.Instance.from_ilp(g)
    b.close()
    c = P.Instance.from_ilp(g)  # built on the buffers b left behind
    c.plan()
    assert list(c.plan_digest()) == list(da)
    c.close()
    assert P.host_cache_release() >= 2 * 4 * nnz
