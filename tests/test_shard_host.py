"""Host side of one instance split over several ranks (no GPU): the row
partition (fdog_shard_plan) against brute force, the per-rank ILPs, shard
planning on the host, and the exchange of per-shard sums between two gloo
ranks."""
import os
import socket
import sys

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


def cases():
    return {"mrf": ilpgen.mrf_grid(8, 8, 3, 0), "random": ilpgen.random_ilp(40, 30, 700, max_row=9, max_coef=3),
            "qap": ilpgen.qap(11, 14, 28, 6, 3), "cell": ilpgen.cell_tracking(12, 5, 20, 60)}


def brute_force_shared(g, row_shard):
    holders = [set() for _ in range(g.n_vars)]
    for j in range(len(g.row_ptr) - 1):
        for q in range(g.row_ptr[j], g.row_ptr[j + 1]):
            if g.coef[q] != 0:
                holders[g.col[q]].add(int(row_shard[j]))
    return np.array([len(h) >= 2 for h in holders], np.uint8), np.array([len(h) for h in holders])


@pytest.mark.parametrize("kind", ["mrf", "random", "qap", "cell"])
@pytest.mark.parametrize("n_shards", [1, 2, 3, 7])
def test_shard_plan_against_brute_force(P, kind, n_shards):
    g = cases()[kind]
    row_shard, copies, shared = P.capi.shard_plan(g.n_vars, g.row_ptr, g.col, g.coef, n_shards)
    n_rows = len(g.row_ptr) - 1
    assert len(row_shard) == n_rows and row_shard.min() >= 0 and row_shard.max() < n_shards
    first = np.array([g.col[g.row_ptr[j]:g.row_ptr[j + 1]].min() for j in range(n_rows)])
    order = np.lexsort((np.arange(n_rows), first))
    assert np.all(np.diff(row_shard[order]) >= 0)  # contiguous blocks in the order of each row's first variable
    nnz = np.diff(g.row_ptr)
    per = np.bincount(row_shard, weights=nnz, minlength=n_shards)
    assert np.abs(per - nnz.sum() / n_shards).max() <= nnz.max()  # balanced to within one row
    assert np.array_equal(copies, np.bincount(g.col[g.coef != 0], minlength=g.n_vars))
    want, _ = brute_force_shared(g, row_shard)
    assert np.array_equal(shared, want)
    if n_shards == 1:
        assert shared.sum() == 0


def test_shard_plan_rejects_malformed_input(P):
    g = cases()["mrf"]
    lib = P.lib()
    n_rows = len(g.row_ptr) - 1
    rs = np.zeros(n_rows, np.int32)
    cp = np.zeros(g.n_vars, np.int32)
    sh = np.zeros(g.n_vars, np.uint8)

    def call(row_ptr, col, n_shards):
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        coef = np.ascontiguousarray(g.coef, np.int32)
        return lib.fdog_shard_plan(g.n_vars, n_rows, row_ptr.ctypes.data, col.ctypes.data, coef.ctypes.data,
                                   n_shards, rs.ctypes.data, cp.ctypes.data, sh.ctypes.data)

    assert call(g.row_ptr, g.col, 2) == P.FDOG_OK
    assert call(g.row_ptr, g.col, 0) == P.FDOG_EINVAL
    bad_col = g.col.copy()
    bad_col[3] = g.n_vars
    assert call(g.row_ptr, bad_col, 2) == P.FDOG_EINVAL
    bad_ptr = g.row_ptr.copy()
    bad_ptr[2], bad_ptr[3] = bad_ptr[3], bad_ptr[2]
    assert call(bad_ptr, g.col, 2) == P.FDOG_EINVAL


@pytest.mark.parametrize("kind", ["mrf", "qap", "cell"])
def test_shard_rows_partition_the_ilp(P, kind):
    from paper_2111_10270_gb300.sharded import shard_rows

    g = cases()[kind]
    world = 3
    row_shard, copies, shared = P.capi.shard_plan(g.n_vars, g.row_ptr, g.col, g.coef, world)
    local = np.zeros((world, g.n_vars), np.int64)
    seen = []
    for r in range(world):
        n, cost, rp, col, coef, sense, rhs, rows = shard_rows(g, row_shard, copies, r)
        seen.append(rows)
        assert n == g.n_vars and len(rp) == len(rows) + 1
        for q, j in enumerate(rows):  # every row copied exactly
            a = slice(g.row_ptr[j], g.row_ptr[j + 1])
            b = slice(rp[q], rp[q + 1])
            assert np.array_equal(col[b], g.col[a]) and np.array_equal(coef[b], g.coef[a])
            assert sense[q] == g.sense[j] and rhs[q] == g.rhs[j]
        local[r] = np.bincount(col[coef != 0], minlength=g.n_vars)
        held = local[r] > 0
        assert np.array_equal(cost[held], g.cost[held])  # the target of Prop. 1 where the shard holds i
        free = copies == 0
        assert np.all(cost[~held & ~free] == 0.0)
        assert np.array_equal(cost[free], g.cost[free] if r == 0 else np.zeros(free.sum()))
    assert np.array_equal(np.sort(np.concatenate(seen)), np.arange(len(g.row_ptr) - 1))
    assert np.array_equal(local.sum(0), copies)
    assert np.array_equal((local > 0).sum(0) >= 2, shared.astype(bool))


def test_shard_planning_on_the_host(P):
    """A shard plans on the host: its shared variables are kept out of the
    tile-local and deferred-sum lists, the copy counts are checked, and
    misuse is refused."""
    from paper_2111_10270_gb300.sharded import shard_rows

    g = cases()["mrf"]
    row_shard, copies, shared = P.capi.shard_plan(g.n_vars, g.row_ptr, g.col, g.coef, 2)
    for r in range(2):
        n, cost, rp, col, coef, sense, rhs, rows = shard_rows(g, row_shard, copies, r)
        inst = P.Instance(n, cost, rp, col, coef, sense, rhs)
        inst.shard_setup(shared, copies)
        n_sh = inst.shard_info()
        assert n_sh == int(shared.sum()) > 0  # the exchange covers every shared variable, on every shard
        held = np.bincount(col, minlength=n) > 0
        kp = inst.kernel_plan()
        assert kp["local_vars"] + kp["work_vars"] + int((held & shared.astype(bool)).sum()) == int(held.sum())
        with pytest.raises(P.FdogError):
            inst.shard_setup(shared, copies)  # already planned
        inst.close()
    # copy counts that disagree with the shard's rows
    n, cost, rp, col, coef, sense, rhs, rows = shard_rows(g, row_shard, copies, 0)
    wrong = copies.copy()
    wrong[np.nonzero((np.bincount(col, minlength=n) > 0) & (shared == 0))[0][0]] += 1
    inst = P.Instance(n, cost, rp, col, coef, sense, rhs).shard_setup(shared, wrong)
    with pytest.raises(P.FdogError):
        inst.shard_info()
    inst.close()
    # the serial update and rows that need presolve are not sharded
    with pytest.raises(P.FdogError):
        P.Instance(n, cost, rp, col, coef, sense, rhs, update=1).shard_setup(shared, copies)
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], 0, 2)  # forces both variables to 1
    rb.add([1, 2], [1, 1], -1, 1)
    f = rb.finish(3, [1.0, 2.0, -1.0], "forced")
    inst = P.Instance.from_ilp(f).shard_setup(np.zeros(3, np.uint8), np.array([1, 2, 1], np.int32))
    with pytest.raises(P.FdogError) as e:
        inst.shard_info()
    assert e.value.code == P.FDOG_EUNSUPPORTED
    inst.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    import paper_2111_10270_gb300 as P
    from paper_2111_10270_gb300.sharded import allreduce_sum, shard_rows

    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = ilpgen.cell_tracking(12, 5, 20, 60)
    row_shard, copies, shared = P.capi.shard_plan(g.n_vars, g.row_ptr, g.col, g.coef, world)
    n, cost, rp, col, coef, sense, rhs, rows = shard_rows(g, row_shard, copies, rank)
    local = torch.tensor(np.bincount(col[coef != 0], minlength=n), dtype=torch.int64)
    held = (local > 0).to(torch.int64)
    part = torch.tensor(np.random.default_rng(rank).standard_normal(7), dtype=torch.float32)
    allreduce_sum(local)
    allreduce_sum(held)
    allreduce_sum(part)
    ok = (bool(np.array_equal(local.numpy(), copies)) and bool(np.array_equal(held.numpy() >= 2, shared.astype(bool)))
          and len(rows) > 0)
    want = sum(np.random.default_rng(r).standard_normal(7).astype(np.float32) for r in range(world))
    ok = ok and bool(np.allclose(part.numpy(), want, rtol=1e-6, atol=1e-6))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ok))


@pytest.mark.parametrize("world", [2, 3])
def test_shard_counts_and_sums_exchange_over_gloo(world):
    """Each rank slices its rows, and the sum of the ranks' local copy counts
    (all-reduced over gloo the way the per-pass sums are) equals the global
    counts; a variable is shared exactly when two or more ranks hold it."""
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert res == [(r, True) for r in range(world)]
