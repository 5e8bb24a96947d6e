"""Ragged batching on the GPU: several instances of different sizes and
shapes solved together (one flat index space, every launch covering all of
them) give exactly the results each gets alone -- iteration counts, rounding
rounds, solutions, objectives and final multipliers, bit for bit."""
import numpy as np
import pytest

import ilpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    return P


def mixed_instances():
    rb = ilpgen._RowBuilder()
    rng = np.random.default_rng(8)
    for j in range(30):  # wide and long rows: generic kernel classes
        k = int(rng.integers(6, 24))
        cols = np.sort(rng.choice(50, k, replace=False))
        rb.add(cols, [1] * k, -1, int(rng.integers(2, 9)))
    wide = rb.finish(50, rng.standard_normal(50), "wide")
    empty = ilpgen.ILP(3, np.array([1.0, -1.0, 0.5]), np.zeros(1, np.int64), np.zeros(0, np.int32),
                       np.zeros(0, np.int32), np.zeros(0, np.int8), np.zeros(0, np.int64), name="norows")
    return [ilpgen.mrf_grid(8, 8, 3, 0), ilpgen.mrf_grid(12, 10, 4, 1, potts_max=2.0),
            ilpgen.mrf_grid(16, 16, 2, 2), ilpgen.random_ilp(40, 30, 31, max_row=8, max_coef=2),
            wide, ilpgen.fig2_example(), empty, ilpgen.mrf_grid(5, 7, 5, 3)]


def solve_alone(P, ilp, max_iters, stream, **kw):
    inst = P.Instance.from_ilp(ilp, **kw).build(0, stream)
    n, _ = inst.iterate(max_iters)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    _, _, lam = inst.multipliers()
    return n, rounds, rc, x, obj, feas, lam


@pytest.mark.parametrize("jit", [1, 0], ids=["specialised", "auto"])
@pytest.mark.parametrize("use_stream", [False, True], ids=["default-stream", "graph-stream"])
def test_batch_equals_solo(P, use_stream, jit):
    import torch

    stream = torch.cuda.Stream() if use_stream else None
    ilps = mixed_instances()
    alone = [solve_alone(P, g, 150, stream, jit=jit) for g in ilps]
    insts = [P.Instance.from_ilp(g, jit=jit).build(0, stream) for g in ilps]
    batch = P.Batch(insts, stream)
    iters, rounds, status = batch.solve(150)
    for q, (g, inst) in enumerate(zip(ilps, insts)):
        n, r, rc, x, obj, feas, lam = alone[q]
        x2, obj2, feas2 = inst.solution()
        _, _, lam2 = inst.multipliers()
        assert iters[q] == n and rounds[q] == r and status[q] == rc, (g.name, iters[q], n, rounds[q], r)
        assert np.array_equal(x, x2) and obj == obj2 and feas == feas2, g.name
        assert lam.tobytes() == lam2.tobytes(), g.name
        assert feas2 == g.feasible(x2) or status[q] != 0
    batch.close()


def test_batch_members_with_different_parameters(P):
    ilps = [ilpgen.mrf_grid(9, 9, 3, 5), ilpgen.mrf_grid(9, 9, 3, 6), ilpgen.random_ilp(30, 20, 9, max_coef=1)]
    kws = [dict(omega=0.5, rounding_dual_iters=20), dict(omega=0.3, rounding_dual_iters=7, seed=3),
           dict(omega=0.8, tol=0.0, max_rounds=40)]
    alone = [solve_alone(P, g, 120, None, **kw) for g, kw in zip(ilps, kws)]
    insts = [P.Instance.from_ilp(g, **kw).build(0) for g, kw in zip(ilps, kws)]
    iters, rounds, status = P.Batch(insts).solve(120)
    for q, inst in enumerate(insts):
        n, r, rc, x, obj, feas, lam = alone[q]
        x2, obj2, _ = inst.solution()
        _, _, lam2 = inst.multipliers()
        assert (iters[q], rounds[q], status[q]) == (n, r, rc)
        assert np.array_equal(x, x2) and obj == obj2 and lam.tobytes() == lam2.tobytes()


def test_batch_autotuner_picks_a_block_size(P):
    insts = [P.Instance.from_ilp(ilpgen.mrf_grid(32, 32, 3, s)).build(0) for s in range(4)]
    b = P.Batch(insts)
    info = b.info()
    assert info["warps_per_block"] in (2, 4, 8) and info["chunk"] >= 1


def width2_instances():
    """Instances whose BDDs all have width <= 2 (the persistent kernel's scope):
    MRF grids, cell tracking with long in-flow rows (segmented kernel), and
    matchings with products of neighbour matches."""
    return [ilpgen.mrf_grid(8, 8, 3, 0), ilpgen.mrf_grid(12, 10, 4, 1, potts_max=2.0), ilpgen.mrf_grid(16, 16, 2, 2),
            ilpgen.mrf_grid(5, 7, 5, 3), ilpgen.cell_tracking(12, 5, 20, 60), ilpgen.cell_tracking(4, 4, 20, 40),
            ilpgen.qap(3, 20, 40, 6, 3, sparse=True), ilpgen.qap(5, 30, 60, 8, 4, sparse=True)]


def batch_results(P, ilps, stream, persistent, max_iters=150):
    insts = [P.Instance.from_ilp(g, jit=-1).build(0, stream) for g in ilps]
    batch = P.Batch(insts, stream)
    if persistent:
        batch.set_persistent(True)
    iters, rounds, status = batch.solve(max_iters)
    out = []
    for q, inst in enumerate(insts):
        x, obj, feas = inst.solution()
        out.append((int(iters[q]), int(rounds[q]), int(status[q]), x.tobytes(), obj, feas,
                    inst.multipliers()[2].tobytes(), inst.lower_bound()))
    batch.close()
    return out


@pytest.mark.parametrize("use_stream", [False, True], ids=["default-stream", "own-stream"])
def test_persistent_batch_equals_graph_batch(P, use_stream):
    """The persistent kernel (one cooperative launch per chunk of iterations,
    grid barriers between the passes) gives bit for bit the results of the
    per-pass kernels: iterations, rounds, statuses, solutions, objectives,
    multipliers and bounds."""
    import torch

    stream = torch.cuda.Stream() if use_stream else None
    ilps = width2_instances()
    graph = batch_results(P, ilps, stream, False)
    persistent = batch_results(P, ilps, stream, True)
    for q, (a, b) in enumerate(zip(graph, persistent)):
        assert a == b, (q, a[:3], b[:3])


def test_persistent_barrier_wait_runs_out(P):
    """A barrier wait limit far below the time the blocks need to meet makes
    the waits run out: the solve returns FDOG_ETIMEOUT without faulting, and
    after a reset the same members solve normally on the per-pass kernels."""
    ilps = width2_instances()[:4]
    ref = batch_results(P, ilps, None, False)
    insts = [P.Instance.from_ilp(g, jit=-1).build(0) for g in ilps]
    batch = P.Batch(insts).set_persistent(True, barrier_wait_s=1e-9)
    with pytest.raises(P.FdogError) as e:
        batch.solve(150)
    assert e.value.code == P.FDOG_ETIMEOUT
    for inst in insts:
        inst.reset()
    batch.set_persistent(False)
    iters, rounds, status = batch.solve(150)
    for q, inst in enumerate(insts):
        x, obj, feas = inst.solution()
        got = (int(iters[q]), int(rounds[q]), int(status[q]), x.tobytes(), obj, feas,
               inst.multipliers()[2].tobytes(), inst.lower_bound())
        assert got == ref[q], q
    batch.close()


def test_persistent_batch_scope(P):
    """Shape-specialised kernels or BDDs wider than 2 are outside the
    persistent kernel: FDOG_EUNSUPPORTED, and the batch keeps the per-pass
    kernels."""
    insts = [P.Instance.from_ilp(ilpgen.mrf_grid(8, 8, 3, 0), jit=1).build(0)]
    batch = P.Batch(insts)
    with pytest.raises(P.FdogError) as e:
        batch.set_persistent(True)
    assert e.value.code == P.FDOG_EUNSUPPORTED
    batch.close()
    wide = mixed_instances()[4]  # cardinality rows: widths up to 9
    insts = [P.Instance.from_ilp(wide, jit=-1).build(0)]
    batch = P.Batch(insts)
    with pytest.raises(P.FdogError) as e:
        batch.set_persistent(True)
    assert e.value.code == P.FDOG_EUNSUPPORTED
    iters, _, _ = batch.solve(20)
    assert iters[0] > 0
    batch.close()
