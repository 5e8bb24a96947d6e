"""GPU: one instance split over 2 or 3 ranks (fdog_shard_* through
paper_2111_10270_gb300.sharded), each rank a process with its shard on
cuda:0, the per-pass sums exchanged over gloo through host memory.  No
kernel waits on another rank: every exchange happens on the host between
launches.

Against the oracle and the unsharded GPU run on the same schedule: the bound
after every iteration (trajectory tolerance, as the other FP32 trajectory
tests), every slot's min-marginals, and the oracle's evaluation of the
gathered, finalised multipliers (bound within 1e-6 max(1, |LB|)); after the
add-back the copies of every variable sum to its cost across the shards."""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest

import ilpgen
from parity_util import MM_RTOL, lb_close, rel_err, slot_order

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def case(kind):
    """Instances whose rows need no presolve (a shard refuses presolve: it
    would fix variables that other shards' rows also hold)."""
    from test_gpu_parity import long_narrow_rows

    return {"mrf": lambda: ilpgen.mrf_grid(8, 8, 3, 0),
            "long": long_narrow_rows,  # rows of 9..1000 layers: the segmented kernels
            "qap": lambda: ilpgen.qap(11, 14, 28, 6, 3),
            "cell": lambda: ilpgen.cell_tracking(12, 5, 20, 60)}[kind]()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, kind, iters, outdir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist

    from paper_2111_10270_gb300.sharded import ShardedInstance

    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s = ShardedInstance(case(kind), rank, world, device=0, tol=0.0)
    trace = [s.iterate(1)[1] for _ in range(iters)]
    mvar, mrow, m0, m1 = s.min_marginals()
    s.finalize()
    run, fea = s.lower_bound()
    var, row, lam = s.multipliers()
    np.savez(os.path.join(outdir, f"r{rank}.npz"), trace=np.array(trace), mvar=mvar, mrow=mrow, m0=m0, m1=m1,
             run=run, fea=fea, var=var, row=row, lam=lam, n_shared=s.n_shared)
    s.close()
    dist.barrier()
    dist.destroy_process_group()


def run_sharded(kind, world, iters):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        procs = [ctx.Process(target=_rank, args=(r, world, port, kind, iters, d)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0] * world, codes
        return [dict(np.load(os.path.join(d, f"r{r}.npz"))) for r in range(world)]


@pytest.fixture(scope="module")
def P():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    return P


@pytest.mark.parametrize("kind,world", [("mrf", 2), ("mrf", 3), ("long", 2), ("qap", 2), ("cell", 3)])
def test_sharded_dual_matches_unsharded_and_oracle(P, oracle_mod, kind, world):
    iters = 30
    res = run_sharded(kind, world, iters)
    g = case(kind)
    assert sum(int(r["n_shared"]) for r in res) > 0  # the split really couples the shards
    trace = res[0]["trace"]
    for r in res[1:]:
        assert np.array_equal(r["trace"], trace)  # every rank commits the same bound
    # the same schedule unsharded on the GPU and in the oracle
    inst = P.Instance.from_ilp(g, tol=0.0).build(0)
    gl = np.array([inst.iterate(1)[1] for _ in range(iters)])
    orc = oracle_mod.Problem.from_ilp(g)
    ol, cond = [], []
    for _ in range(iters):
        ol.append(orc.iterate(1)[0])
        cond.append(np.abs(orc.energies()).sum())
    bad = [t for t in range(iters) if not (lb_close(trace[t], ol[t], scale=cond[t])
                                           and lb_close(trace[t], gl[t], scale=cond[t]))]
    assert not bad, [(t, trace[t], gl[t], ol[t]) for t in bad[:4]]
    # min-marginals of every slot, gathered over the shards, against the oracle's state
    mvar = np.concatenate([r["mvar"] for r in res])
    mrow = np.concatenate([r["mrow"] for r in res])
    m0 = np.concatenate([r["m0"] for r in res])
    m1 = np.concatenate([r["m1"] for r in res])
    om0, om1 = orc.min_marginals()
    perm = slot_order(orc, mvar, mrow)
    assert rel_err(m0[perm], om0).max() <= MM_RTOL and rel_err(m1[perm], om1).max() <= MM_RTOL
    assert rel_err(m1[perm] - m0[perm], om1 - om0).max() <= MM_RTOL
    # the oracle evaluates the gathered finalised multipliers
    var = np.concatenate([r["var"] for r in res])
    row = np.concatenate([r["row"] for r in res])
    lam = np.concatenate([r["lam"] for r in res])
    orc.set_state(lam[slot_order(orc, var, row)].astype(np.float64))
    orun, ofea = orc.lower_bounds()
    fea = float(res[0]["fea"])
    assert all(float(r["fea"]) == fea for r in res)
    assert lb_close(fea, ofea) and lb_close(float(res[0]["run"]), orun), (fea, ofea)
    # dual feasibility across the shards: sum_j lambda^j_i = c_i
    s = np.bincount(var, lam.astype(np.float64), minlength=g.n_vars)
    inb = np.bincount(var, minlength=g.n_vars) > 0
    assert np.abs(s - g.cost)[inb].max() <= 1e-5 * max(1.0, np.abs(g.cost).max())


def test_shards_refuse_single_instance_calls(P):
    from paper_2111_10270_gb300.sharded import shard_rows

    g = case("mrf")
    row_shard, copies, shared = P.capi.shard_plan(g.n_vars, g.row_ptr, g.col, g.coef, 2)
    n, cost, rp, col, coef, sense, rhs, rows = shard_rows(g, row_shard, copies, 0)
    inst = P.Instance(n, cost, rp, col, coef, sense, rhs).shard_setup(shared, copies).build(0)
    with pytest.raises(P.FdogError) as e:
        inst.iterate(3)
    assert e.value.code == P.FDOG_ESTATE
    with pytest.raises(P.FdogError) as e:
        inst.primal_round()
    assert e.value.code == P.FDOG_EUNSUPPORTED
    with pytest.raises(P.FdogError):
        P.Batch([inst])
    with pytest.raises(P.FdogError) as e:
        inst.shard_bound()  # no descending pass yet
    assert e.value.code == P.FDOG_ESTATE
    inst.close()
