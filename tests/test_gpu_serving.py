"""Continuous-batching server on the GPU: every result equals the instance's
solo result; HBM admission respects the budget; requests that arrive while
others are resident are admitted and overlap with them."""
import time

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


def solo(P, g, max_iters, jit=0):
    inst = P.Instance.from_ilp(g, jit=jit).build(0)
    n, _ = inst.iterate(max_iters)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    return rc, rounds, x, obj, feas


def mix():
    return [ilpgen.mrf_grid(10, 10, 3, 1), ilpgen.qap(3, 20, 40, 6, 3), ilpgen.cell_tracking(4, 4, 20, 40),
            ilpgen.mrf_grid(6, 14, 5, 2, potts_max=2.0), ilpgen.random_ilp(30, 25, 12, max_coef=1),
            ilpgen.fig2_example(), ilpgen.mrf_grid(20, 20, 2, 3)]


@pytest.mark.parametrize("budget,jit", [(64 << 30, 1), (1, 0)], ids=["roomy-specialised", "one-at-a-time"])
def test_server_results_equal_solo(P, budget, jit):
    ilps = mix()
    ref = [solo(P, g, 200, jit) for g in ilps]
    srv = P.Server(0, hbm_budget=budget, max_active=64, max_iters=200)
    tickets = [srv.submit(P.Instance.from_ilp(g, jit=jit)) for g in ilps]
    for t in tickets:
        assert srv.wait(t, 300)
    for g, t, (rc, rounds, x, obj, feas) in zip(ilps, tickets, ref):
        st = srv.poll(t)
        inst = srv.take(t)
        x2, obj2, feas2 = inst.solution()
        assert st["state"] == 2 and st["status"] == rc, (g.name, st, rc)
        assert np.array_equal(x, x2) and obj == obj2 and feas == feas2, g.name
    s = srv.stats()
    assert s["completed"] == len(ilps) and s["hbm_used"] == 0 and s["queued"] == 0
    srv.close()


def test_server_admits_while_busy(P):
    """A large instance is resident; small requests submitted afterwards are
    admitted into the running set and finish first."""
    big = ilpgen.mrf_grid(160, 160, 4, 7)
    small = [ilpgen.mrf_grid(6, 6, 3, s) for s in range(6)]
    srv = P.Server(0, max_iters=400)
    tb = srv.submit(P.Instance.from_ilp(big, tol=0.0))  # runs all 400 iterations
    t0 = time.time()
    while srv.poll(tb)["state"] == 0 and time.time() - t0 < 60:
        time.sleep(0.001)
    ts = [srv.submit(P.Instance.from_ilp(g)) for g in small]
    for t in ts:
        assert srv.wait(t, 300)
    st_big = srv.poll(tb)
    assert st_big["state"] in (1, 2)
    small_done = [srv.poll(t)["latency_s"] for t in ts]
    assert srv.wait(tb, 600)
    assert max(small_done) < srv.poll(tb)["latency_s"]
    for t, g in zip(ts, small):
        x, _, feas = srv.take(t).solution()
        assert feas and g.feasible(x)
    srv.close()


def test_release_and_build_again(P):
    """fdog_release frees the device memory; the solution stays readable and a
    second build (same plan) solves to the same result."""
    g = ilpgen.mrf_grid(12, 12, 3, 9)
    inst = P.Instance.from_ilp(g).build(0)
    inst.iterate(150)
    inst.primal_round()
    x, obj, feas = inst.solution()
    inst.release()
    x1, obj1, _ = inst.solution()
    assert np.array_equal(x, x1) and obj == obj1
    inst.release()  # nothing resident: still OK
    inst.build(0)
    inst.iterate(150)
    inst.primal_round()
    x2, obj2, feas2 = inst.solution()
    assert np.array_equal(x, x2) and obj == obj2 and feas == feas2
    inst.close()


def test_server_plans_requests_on_admission(P):
    """Requests submitted unplanned are planned by the worker when it admits
    them (on the device where the device builder takes them), with results
    equal to the solo ones; a request whose rows cannot be satisfied reports
    it as its status instead of failing the submission."""
    g = ilpgen.mrf_grid(24, 24, 4, 5)
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], 0, 3)  # x0 + x1 = 3: no assignment satisfies it
    bad = rb.finish(2, [1.0, -1.0], "infeasible")
    ref = solo(P, g, 200)
    srv = P.Server(0, max_iters=200)
    t = srv.submit(P.Instance.from_ilp(g))
    tb = srv.submit(P.Instance.from_ilp(bad))
    assert srv.wait(t, 300) and srv.wait(tb, 300)
    assert srv.poll(tb)["status"] == P.FDOG_EINFEASIBLE
    st = srv.poll(t)
    inst = srv.take(t)
    assert inst.plan_stats()[0]  # built by the device builder
    x, obj, feas = inst.solution()
    assert st["status"] == ref[0] and np.array_equal(x, ref[2]) and obj == ref[3] and feas == ref[4]
    assert srv.stats()["hbm_used"] == 0
    srv.close()
