"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances: min-marginals |a-b| <= 1e-4 max(1,|a|,|b|), lower bounds
|a-b| <= 1e-6 max(1,|a|); integer results (solutions, feasibility, sizes)
bit-exact.  Two kinds of parity:
  * evaluation parity: the oracle evaluates the GPU's own multipliers, so
    only the FP32 evaluation error enters;
  * trajectory parity: both run the same iteration schedule from scratch.
"""
import numpy as np
import pytest

import ilpgen
from parity_util import LB_RTOL, MM_RTOL, lb_close, rel_err, slot_order

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


def gpu_instance(P, ilp, **kw):
    kw.setdefault("tol", 0.0)
    return P.Instance.from_ilp(ilp, **kw).build(0)


# ----------------------------------------------------------------------------
# the paper's examples
# ----------------------------------------------------------------------------
def test_fig3_min_marginals_exact(P, oracle_mod):
    inst = gpu_instance(P, ilpgen.fig3_example())
    var, row, m0, m1 = inst.min_marginals()
    order = np.argsort(var)
    assert np.array_equal(m0[order], [0, 0, 0, 0])
    assert np.array_equal(m1[order], [3, 5, 3, 5])
    assert inst.lower_bound() == (0.0, 0.0)


def test_fig2_bound_stays_at_optimum_and_rounds_at_once(P):
    inst = gpu_instance(P, ilpgen.fig2_example())
    for _ in range(30):
        n, lb = inst.iterate(1)
        assert n == 1 and lb == -5.0
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    assert rc == 0 and rounds == 0 and list(x) == [1, 0, 0, 0] and obj == -5.0 and feas


def test_fig2_first_iteration_matches_oracle_exactly(P, oracle_mod):
    ilp = ilpgen.fig2_example()
    inst = gpu_instance(P, ilp)
    orc = oracle_mod.Problem.from_ilp(ilp)
    inst.iterate(1)
    orc.iterate(1)
    var, row, lam = inst.multipliers()
    hi, lo, _, _ = orc.state()
    perm = slot_order(orc, var, row)
    assert np.array_equal(lam[perm].astype(np.float64), hi - lo)  # dyadic values: exact in FP32


# ----------------------------------------------------------------------------
# trajectory and evaluation parity
# ----------------------------------------------------------------------------
def mm_parity(orc, inst):
    """Every slot's m0 and m1 and their difference against the oracle's (the
    oracle's state must be the one to compare with)."""
    var, row, m0, m1 = inst.min_marginals()
    om0, om1 = orc.min_marginals()
    perm = slot_order(orc, var, row)
    e0, e1 = rel_err(m0[perm], om0).max(), rel_err(m1[perm], om1).max()
    ed = rel_err(m1[perm] - m0[perm], om1 - om0).max()
    assert e0 <= MM_RTOL and e1 <= MM_RTOL and ed <= MM_RTOL, (e0, e1, ed)
    return max(e0, e1, ed)


def evaluation_parity(orc, inst):
    """The oracle evaluates the GPU's finalised multipliers: the feasible bound
    within 1e-6 max(1, |LB|) and every slot's min-marginals within 1e-4."""
    inst.finalize()
    var, row, lam = inst.multipliers()
    orc.set_state(lam[slot_order(orc, var, row)].astype(np.float64))
    run, fea = inst.lower_bound()
    orun, ofea = orc.lower_bounds()
    assert lb_close(fea, ofea), (fea, ofea)
    assert lb_close(run, orun), (run, orun)
    return abs(fea - ofea) / max(1.0, abs(ofea)), mm_parity(orc, inst)


def trajectory(P, oracle_mod, ilp, iters, omega=0.5, jit=1):
    """Same schedule on both sides; also returns the oracle's sum_j |E_j| after
    every iteration (the conditioning of the bound as a sum)."""
    inst = gpu_instance(P, ilp, omega=omega, jit=jit)
    orc = oracle_mod.Problem.from_ilp(ilp)
    gl = np.array([inst.iterate(1)[1] for _ in range(iters)])
    ol, cond = [], []
    for _ in range(iters):
        ol.append(orc.iterate(1, omega)[0])
        cond.append(np.abs(orc.energies()).sum())
    return inst, orc, gl, np.array(ol), np.array(cond)


@pytest.mark.parametrize("jit", [1, -1], ids=["specialised", "generic"])
@pytest.mark.parametrize("seed", range(3))
def test_tiny_mrf_trajectory_parity(P, oracle_mod, seed, jit):
    g = ilpgen.mrf_grid(8, 8, 3, seed)
    inst, orc, gl, ol, _ = trajectory(P, oracle_mod, g, 200, jit=jit)
    kp = inst.kernel_plan()
    assert (kp["static_tiles"] == 0) if jit == 1 else (kp["jit_tiles"] == 0), kp
    assert np.all(np.diff(gl) >= -1e-5 * max(1.0, abs(gl[-1])))
    bad = [t for t in range(len(gl)) if not lb_close(gl[t], ol[t])]
    assert not bad, (bad[:5], gl[bad[0]], ol[bad[0]])
    var, row, m0, m1 = inst.min_marginals()
    om0, om1 = orc.min_marginals()
    hi, lo, _, _ = orc.state()
    perm = slot_order(orc, var, row)
    # both sides report min-marginals of the plain multipliers lambda = hi - lo
    assert rel_err(m0[perm], om0).max() <= MM_RTOL
    assert rel_err(m1[perm], om1).max() <= MM_RTOL
    assert rel_err(m1[perm] - m0[perm], om1 - om0).max() <= MM_RTOL
    _, lbf = inst.lower_bound()
    _, olbf = orc.lower_bounds()
    assert lb_close(lbf, olbf)


@pytest.mark.parametrize("seed", range(3))
def test_tiny_mrf_evaluation_parity(P, oracle_mod, seed):
    """The oracle evaluates the GPU's multipliers: min-marginals and the bound
    of the finalised (dual-feasible) state."""
    g = ilpgen.mrf_grid(8, 8, 3, 10 + seed)
    inst = gpu_instance(P, g)
    inst.iterate(57)
    inst.finalize()
    var, row, lam = inst.multipliers()
    orc = oracle_mod.Problem.from_ilp(g)
    perm = slot_order(orc, var, row)
    orc.set_state(lam[perm].astype(np.float64))
    om0, om1 = orc.min_marginals()
    var2, row2, m0, m1 = inst.min_marginals()
    perm2 = slot_order(orc, var2, row2)
    assert rel_err(m0[perm2], om0).max() <= MM_RTOL
    assert rel_err(m1[perm2], om1).max() <= MM_RTOL
    run, fea = inst.lower_bound()
    orun, ofea = orc.lower_bounds()
    assert lb_close(run, orun) and lb_close(fea, ofea)
    # dual feasibility after the add-back: sum_j lambda^j_i = c_i (FP32)
    s = np.bincount(var, lam.astype(np.float64), minlength=g.n_vars)
    inb = np.bincount(var, minlength=g.n_vars) > 0
    assert np.abs(s - g.cost)[inb].max() <= 1e-5 * max(1.0, np.abs(g.cost).max())


@pytest.mark.parametrize("jit", [1, -1], ids=["specialised", "generic"])
@pytest.mark.parametrize("seed", range(8))
def test_random_ilp_trajectory_parity(P, oracle_mod, seed, jit):
    ilp = ilpgen.random_ilp(40, 30, 700 + seed, max_row=9, max_coef=3)
    omega = [0.5, 0.25, 1.0, 0.7][seed % 4]
    inst, orc, gl, ol, cond = trajectory(P, oracle_mod, ilp, 60, omega, jit=jit)
    # FP32 trajectories of a sum with cancellation: relative to sum_j |E_j|
    bad = [t for t in range(len(gl)) if not lb_close(gl[t], ol[t], scale=cond[t])]
    assert not bad, [(t, gl[t], ol[t], cond[t]) for t in bad[:4]]
    mm_parity(orc, inst)
    evaluation_parity(orc, inst)


@pytest.mark.parametrize("jit", [1, -1], ids=["specialised", "generic"])
def test_wide_and_long_rows_parity(P, oracle_mod, jit):
    """Shapes of every kernel class: widths 2 / 4 / 8 / 16 with short and long
    rows, ragged tiles; with specialised kernels on, the narrow short shapes
    take them and the rest the generic kernels in the same passes."""
    rng = np.random.default_rng(5)
    rb = ilpgen._RowBuilder()
    n = 60
    for j in range(70):
        k = int(rng.integers(2, 30))
        cols = np.sort(rng.choice(n, k, replace=False))
        kind = j % 5
        if kind == 0:
            rb.add(cols, [1] * k, -1, int(rng.integers(1, min(k, 14))))     # cardinality: width up to 15
        elif kind == 1:
            rb.add(cols, [1] * k, 0, 1)                                     # simplex
        elif kind == 2:
            a = rng.integers(1, 3, k) * rng.choice([-1, 1], k)
            rb.add(cols, a, -1, int(np.abs(a).sum() // 3))
        elif kind == 3:
            rb.add(cols[:5], [1, 1, -1, 1, -1], 0, 0)
        else:
            rb.add(cols[:3], [2, -1, -1], 1, 0)
    ilp = rb.finish(n, rng.standard_normal(n), "classes")
    inst = P.Instance.from_ilp(ilp, tol=0.0, jit=jit)
    inst.plan()
    kp = inst.kernel_plan()
    assert kp["static_tiles"] > 0 and ((kp["jit_tiles"] > 0) == (jit == 1)), kp
    inst.build(0)
    orc = oracle_mod.Problem.from_ilp(ilp)
    gl = np.array([inst.iterate(1)[1] for _ in range(40)])
    ol, cond = [], []
    for _ in range(40):
        ol.append(orc.iterate(1)[0])
        cond.append(np.abs(orc.energies()).sum())
    # FP32 trajectories of a sum with cancellation: relative to sum_j |E_j|
    bad = [t for t in range(40) if not lb_close(gl[t], ol[t], scale=cond[t])]
    assert not bad, [(t, gl[t], ol[t], cond[t]) for t in bad[:4]]
    mm_parity(orc, inst)
    evaluation_parity(orc, inst)


@pytest.mark.parametrize("jit", [1, 0], ids=["specialised", "auto"])
@pytest.mark.parametrize("kind", ["qap", "cell"])
def test_qap_and_cell_tracking_parity(P, oracle_mod, kind, jit):
    """The matching and tracking shapes at sizes the oracle runs in seconds:
    assignment variables with dozens of copies (the warp-per-variable
    deferred sums), AND rows, long in-flow rows (segmented sweeps), conflict
    sets; bound trajectory and min-marginals against the oracle."""
    ilp = ilpgen.qap(11, 14, 28, 6, 3) if kind == "qap" else ilpgen.cell_tracking(12, 5, 20, 60)
    inst, orc, gl, ol, cond = trajectory(P, oracle_mod, ilp, 40, jit=jit)
    kp = inst.kernel_plan()
    if kind == "qap":
        counts = np.bincount(orc.slot_vars(), minlength=ilp.n_vars)
        assert counts.max() > 8, counts.max()
    bad = [t for t in range(len(gl)) if not lb_close(gl[t], ol[t], scale=cond[t])]
    assert not bad, [(t, gl[t], ol[t], cond[t]) for t in bad[:4]]
    mm_parity(orc, inst)
    evaluation_parity(orc, inst)


def serial_cases():
    return {"mrf": ilpgen.mrf_grid(8, 8, 3, 2), "random": ilpgen.random_ilp(40, 30, 711, max_row=9, max_coef=3),
            "cell": ilpgen.cell_tracking(12, 5, 20, 60), "qap": ilpgen.qap(11, 14, 28, 6, 3),
            "long": long_narrow_rows()}


@pytest.mark.parametrize("kind", ["mrf", "random", "cell", "qap", "long"])
def test_serial_update_parity(P, oracle_mod, kind):
    """The level-by-level serial update (update = 1) against the oracle's
    Eq. 4, same iterations: bound after every iteration (relative to the sum
    of the subproblem energies' magnitudes) and the final min-marginals."""
    g = serial_cases()[kind]
    iters = 15
    inst = P.Instance.from_ilp(g, tol=0.0, update=1).build(0)
    gl = np.array([inst.iterate(1)[1] for _ in range(iters)])
    orc = oracle_mod.Problem.from_ilp(g)
    ol, cond = [], []
    for _ in range(iters):
        ol.append(orc.iterate_serial(1)[0])
        cond.append(np.abs(orc.energies()).sum())
    bad = [t for t in range(iters) if not lb_close(gl[t], ol[t], scale=cond[t])]
    assert not bad, [(t, gl[t], ol[t], cond[t]) for t in bad[:4]]
    mm_parity(orc, inst)
    # every copy sum still equals the cost (Eq. 4 only redistributes)
    var, _, lam = inst.multipliers()
    sums = np.bincount(var, lam.astype(np.float64), minlength=g.n_vars)
    inb = np.bincount(var, minlength=g.n_vars) > 0
    assert np.abs(sums - np.asarray(g.cost))[inb].max() <= 1e-4 * max(1.0, np.abs(g.cost).max())


def test_serial_update_runs_alone(P):
    a = P.Instance.from_ilp(ilpgen.mrf_grid(6, 6, 3, 1), update=1).build(0)
    b = P.Instance.from_ilp(ilpgen.mrf_grid(6, 6, 3, 2)).build(0)
    with pytest.raises(P.FdogError):
        P.Batch([a, b])
    srv = P.Server(0)
    with pytest.raises(P.FdogError):
        srv.submit(P.Instance.from_ilp(ilpgen.mrf_grid(6, 6, 3, 3), update=1))
    srv.close()
    n, lb = a.iterate(30)
    assert n == 30 or n > 0
    rc, rounds = a.primal_round()
    x, obj, feas = a.solution()
    assert feas and obj >= lb - 1e-6 * max(1.0, abs(lb))


def long_narrow_rows(seed=6):
    """Rows of width <= 4 and 9 .. 1000 layers: one-segment, multi-segment and
    ragged-segment shapes of the segmented kernels, some shapes filling more
    than one tile, some a tile with few BDDs."""
    rng = np.random.default_rng(seed)
    rb = ilpgen._RowBuilder()
    n = 1500
    kinds = [("le1", -1, 1), ("eq1", 0, 1), ("ge1", 1, 1), ("flow", -1, 0), ("le2", -1, 2), ("eq2", 0, 2),
             ("le3", -1, 3)]
    for k in (9, 12, 16, 17, 24, 40, 64, 65, 130, 300, 1000):
        for q, (name, sense, rhs) in enumerate(kinds):
            reps = 40 if (k == 17 and name == "le1") else (3 if k <= 65 else 1)
            for _ in range(reps):
                cols = np.sort(rng.choice(n, k, replace=False))
                coef = [1] * k
                if name == "flow":
                    coef[0] = -1
                rb.add(cols, coef, sense, rhs)
    return rb.finish(n, rng.standard_normal(n), "long-narrow")


def split_ilp(P, g, max_len):
    nv, rp, col, coef, sense, rhs, _ = P.capi.split_rows(g.n_vars, g.row_ptr, g.col, g.coef, g.sense, g.rhs,
                                                         max_len)
    return ilpgen.ILP(nv, np.concatenate([g.cost, np.zeros(nv - g.n_vars)]), rp, col, coef, sense, rhs,
                      name=g.name + "-split")


@pytest.mark.parametrize("kind", ["qap", "long"])
def test_split_rows_parity(P, oracle_mod, kind):
    """An ILP whose long at-most-one / exactly-one rows were split into chains
    (fdog_split_rows) is an ILP like any other: bound trajectory and
    min-marginals against the oracle on the split ILP; the split rows run in
    the register kernels (no segmented class left for them)."""
    g = ilpgen.qap(11, 14, 28, 6, 3) if kind == "qap" else long_narrow_rows()
    max_len = 4 if kind == "qap" else 6
    s = split_ilp(P, g, max_len)
    assert s.n_vars > g.n_vars
    inst, orc, gl, ol, cond = trajectory(P, oracle_mod, s, 40)
    bad = [t for t in range(len(gl)) if not lb_close(gl[t], ol[t], scale=cond[t])]
    assert not bad, [(t, gl[t], ol[t], cond[t]) for t in bad[:4]]
    mm_parity(orc, inst)
    evaluation_parity(orc, inst)
    if kind == "qap":
        assert np.diff(s.row_ptr).max() <= max_len


@pytest.mark.parametrize("jit", [1, -1], ids=["specialised", "generic"])
def test_long_narrow_rows_parity(P, oracle_mod, jit):
    """The segmented kernels (registers per segment of 8 layers, labels
    recomputed from shared-memory checkpoints) against the oracle: bound
    trajectory, min-marginals, and the evaluation of the finalised state."""
    ilp = long_narrow_rows()
    inst = P.Instance.from_ilp(ilp, tol=0.0, jit=jit)
    inst.plan()
    kp = inst.kernel_plan()
    assert kp["static_tiles"] > 0, kp
    inst.build(0)
    orc = oracle_mod.Problem.from_ilp(ilp)
    iters = 30
    gl = np.array([inst.iterate(1)[1] for _ in range(iters)])
    ol, cond = [], []
    for _ in range(iters):
        ol.append(orc.iterate(1)[0])
        cond.append(np.abs(orc.energies()).sum())
    bad = [t for t in range(iters) if not lb_close(gl[t], ol[t], scale=cond[t])]
    assert not bad, [(t, gl[t], ol[t], cond[t]) for t in bad[:4]]
    mm_parity(orc, inst)
    evaluation_parity(orc, inst)


# ----------------------------------------------------------------------------
# rounding
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("jit", [1, -1], ids=["specialised", "generic"])
@pytest.mark.parametrize("seed", range(3))
def test_tiny_mrf_rounding_parity(P, oracle_mod, seed, jit):
    g = ilpgen.mrf_grid(8, 8, 3, 20 + seed, potts_max=1.5)
    inst = gpu_instance(P, g, jit=jit)
    orc = oracle_mod.Problem.from_ilp(g)
    inst.iterate(200)
    orc.iterate(200)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    r = orc.round()
    assert rc == 0 and feas and g.feasible(x)
    assert abs(obj - g.objective(x)) <= 1e-9 * max(1.0, abs(obj))
    _, lbf = orc.lower_bounds()
    assert obj >= lbf - 1e-6 * max(1.0, abs(lbf))  # a feasible point is never below the bound
    scale = max(1.0, np.abs(g.cost).max())
    if r["margin"] > 1e-3 * scale:
        assert np.array_equal(x, r["x"]) and rounds == r["rounds"]


@pytest.mark.parametrize("seed", range(6))
def test_random_ilp_rounding_feasible(P, oracle_mod, seed):
    ilp = ilpgen.random_ilp(30, 25, 900 + seed, max_row=5, max_coef=1)
    inst = gpu_instance(P, ilp, max_rounds=300)
    inst.iterate(50)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    orc = oracle_mod.Problem.from_ilp(ilp)
    orc.iterate(50)
    r = orc.round(max_rounds=300)
    if rc == 0:
        assert feas == ilp.feasible(x)
        assert feas
    if r["status"] == 0 and r["margin"] > 1e-3 * max(1.0, np.abs(ilp.cost).max()):
        assert rc == 0 and np.array_equal(x, r["x"])


# ----------------------------------------------------------------------------
# edge cases, determinism, checkpoint
# ----------------------------------------------------------------------------
def test_instance_without_rows(P):
    c = np.array([1.0, -2.0, 0.5, -0.25])
    ilp = ilpgen.ILP(4, c, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32),
                     np.zeros(0, np.int8), np.zeros(0, np.int64))
    inst = gpu_instance(P, ilp)
    n, lb = inst.iterate(5)
    assert lb == -2.25
    assert inst.lower_bound() == (-2.25, -2.25)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    assert list(x) == [0, 1, 0, 1] and obj == -2.25 and feas


def test_presolve_fixed_variables_on_gpu(P, oracle_mod):
    rb = ilpgen._RowBuilder()
    rb.add([0, 1], [1, 1], 0, 2)
    rb.add([1, 2], [1, 1], -1, 1)
    rb.add([3, 4, 5], [1, -1, 1], 0, 1)
    ilp = rb.finish(7, [1.0, 2.0, -3.0, -1.0, 0.5, 0.75, -0.25], "forced")
    inst = gpu_instance(P, ilp)
    orc = oracle_mod.Problem.from_ilp(ilp)
    assert np.array_equal(inst.fixed_vars(), orc.fixed())
    gl = [inst.iterate(1)[1] for _ in range(20)]
    ol = orc.iterate(20)
    assert all(lb_close(a, b) for a, b in zip(gl, ol))
    rc, _ = inst.primal_round()
    x, obj, feas = inst.solution()
    assert rc == 0 and feas and ilp.feasible(x)


@pytest.mark.parametrize("seed", range(2))
def test_specialised_and_generic_kernels_agree(P, seed):
    """The shape-specialised code performs the same float operations as the
    generic kernels, so multipliers, bounds and min-marginals coincide."""
    g = ilpgen.mrf_grid(16, 16, 4, 40 + seed)
    out = []
    for jit in (1, -1):
        inst = gpu_instance(P, g, jit=jit)
        lbs = [inst.iterate(1)[1] for _ in range(15)]
        _, _, lam = inst.multipliers()
        _, _, m0, m1 = inst.min_marginals()
        out.append((lbs, lam, m0, m1, inst.lower_bound()))
    a, b = out
    assert a[0] == b[0] and a[4] == b[4]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


@pytest.mark.parametrize("jit", [1, -1], ids=["specialised", "generic"])
def test_tile_local_sums_match_the_separate_pass(P, jit):
    """Deferred terms formed inside the sweep for tile-local variables use the
    same operations in the same order as the deferred-sum kernel: the whole
    state stays bitwise equal with the fusion on and off."""
    g = ilpgen.mrf_grid(24, 20, 3, 51)
    out = []
    for fuse in (0, -1):
        inst = P.Instance.from_ilp(g, tol=0.0, jit=jit, fuse=fuse)
        inst.plan()
        kp = inst.kernel_plan()
        assert (kp["local_vars"] > 0) == (fuse == 0), kp
        inst.build(0)
        lbs = [inst.iterate(1)[1] for _ in range(20)]
        _, _, lam = inst.multipliers()
        rc, rounds = inst.primal_round()
        x, obj, feas = inst.solution()
        out.append((lbs, lam.tobytes(), rounds, x.tobytes(), obj))
    assert out[0] == out[1]


def test_runs_are_bitwise_deterministic(P):
    g = ilpgen.mrf_grid(16, 16, 4, 3)
    outs = []
    for _ in range(2):
        inst = gpu_instance(P, g)
        lbs = [inst.iterate(1)[1] for _ in range(30)]
        _, _, lam = inst.multipliers()
        outs.append((lbs, lam.tobytes()))
    assert outs[0] == outs[1]


def test_launch_shape_does_not_change_results(P):
    """Warps per block, grid size (one persistent wave, two waves, a block
    per tile group) and the autotuned choice: bitwise the same results."""
    g = ilpgen.mrf_grid(16, 16, 3, 4)
    res = []
    for bt, waves in ((64, 1), (128, 1), (256, 1), (128, 2), (128, -1), (64, -1), (0, 0)):
        inst = gpu_instance(P, g, block_threads=bt, grid_waves=waves)
        inst.iterate(25)
        _, _, lam = inst.multipliers()
        res.append((inst.lower_bound(), lam.tobytes()))
    assert all(r == res[0] for r in res)


def test_checkpoint_resume_is_bit_identical(P):
    g = ilpgen.mrf_grid(12, 12, 3, 5)
    a = gpu_instance(P, g)
    a.iterate(30)
    blob = a.export_state()
    a.iterate(20)
    _, _, lam_a = a.multipliers()
    lb_a = a.lower_bound()
    b = gpu_instance(P, g)
    b.import_state(blob)
    b.iterate(20)
    _, _, lam_b = b.multipliers()
    assert lam_a.tobytes() == lam_b.tobytes() and lb_a == b.lower_bound()
    c = gpu_instance(P, ilpgen.mrf_grid(12, 12, 3, 6))
    with pytest.raises(P.FdogError):
        c.import_state(blob[:-8])


def test_early_stopping_rule(P, oracle_mod):
    g = ilpgen.mrf_grid(8, 8, 3, 7)
    inst = gpu_instance(P, g, tol=1e-4, window=10, min_iters=20)
    n, lb = inst.iterate(2000)
    assert 20 <= n < 2000
    orc = oracle_mod.Problem.from_ilp(g)
    tr = orc.iterate(n + 5)
    # the oracle's bound satisfies the same rule within a couple of iterations of the stop
    stops = [t for t in range(20, len(tr)) if t + 1 > 10 and tr[t] - tr[t - 10] <= 1e-4 * max(1.0, abs(tr[t]))]
    assert stops and abs((stops[0] + 1) - n) <= 2
    # stays stopped, and further calls leave the state alone, before and after the add-back
    lam0, lb0 = inst.multipliers()[2].tobytes(), inst.lower_bound()
    assert inst.iterate(10)[0] == 0
    assert inst.multipliers()[2].tobytes() == lam0 and inst.lower_bound() == lb0
    inst.finalize()
    lam1, lb1 = inst.multipliers()[2].tobytes(), inst.lower_bound()
    assert inst.iterate(10)[0] == 0
    assert inst.multipliers()[2].tobytes() == lam1 and inst.lower_bound() == lb1


def test_stopped_instance_with_warp_per_variable_sums_stays_put(P):
    """A matching instance has variables with more than 8 copies (the
    warp-per-variable deferred sums, which share a launch with the bound and
    the commit).  Once its stopping rule fires, further iterations in the same
    graph replay and later calls change neither multipliers nor bound,
    before and after the add-back."""
    g = ilpgen.qap(5, 30, 60, 8, 4, sparse=True)
    inst = gpu_instance(P, g, tol=1e-3, window=5, min_iters=10)
    assert inst.info()["n_slots"] > 0
    n, _ = inst.iterate(3000)
    assert 10 <= n < 3000
    lam0, lb0 = inst.multipliers()[2].tobytes(), inst.lower_bound()
    assert inst.iterate(64)[0] == 0
    assert inst.multipliers()[2].tobytes() == lam0 and inst.lower_bound() == lb0
    inst.finalize()
    lam1, lb1 = inst.multipliers()[2].tobytes(), inst.lower_bound()
    assert inst.iterate(64)[0] == 0
    assert inst.multipliers()[2].tobytes() == lam1 and inst.lower_bound() == lb1


# ----------------------------------------------------------------------------
# full-size workload (512 x 512 grid, 4 labels) in the benchmark's launch configuration
# ----------------------------------------------------------------------------
def test_qap_evaluation_parity_full_size(P, oracle_mod):
    """The QAP-shaped workload at its full size (500 x 1000, 20 candidates,
    10-NN products): after 25 iterations the oracle evaluates the GPU's
    finalised multipliers (bound, every slot's min-marginals)."""
    g = ilpgen.qap(2, 500, 1000, 20)
    inst = gpu_instance(P, g)
    info = inst.info()
    assert (info["n_vars"], info["n_slots"]) == (1166481, 8115367)
    n, _ = inst.iterate(25)
    assert n == 25
    evaluation_parity(oracle_mod.Problem.from_ilp(g), inst)


def test_qap_sparse_rounding_full_size(P, oracle_mod):
    """The QAP-shaped workload with product terms between matches that are
    10-NN neighbours on both sides: the full solve (Alg. 1 to the stopping
    rule or 500 iterations, then Alg. 2) returns a feasible matching on the GPU,
    as the oracle's does, whose objective is not below the bound; the two
    rounded points are equal when the oracle's decisions have margin."""
    g = ilpgen.qap(2, 500, 1000, 20, 10, sparse=True)
    inst = P.Instance.from_ilp(g).build(0)
    n, lb = inst.iterate(500)
    rc, rounds = inst.primal_round()
    x, obj, feas = inst.solution()
    assert rc == P.FDOG_OK and feas and g.feasible(x), (rc, rounds)
    assert abs(obj - g.objective(x)) <= 1e-9 * max(1.0, abs(obj)) and obj >= lb - 1e-6 * abs(lb)
    orc = oracle_mod.Problem.from_ilp(g)
    orc.iterate(n)  # the GPU's schedule: its dual iterations, then Alg. 2
    r = orc.round()
    assert r["status"] == 0 and g.feasible(r["x"])
    if r["margin"] > 1e-3 * max(1.0, np.abs(g.cost).max()):
        assert np.array_equal(x, r["x"]) and rounds == r["rounds"]


def test_cell_batch_members_parity_full_size(P, oracle_mod):
    """The 64-instance cell-tracking batch at full size, solved as one batch
    with the autotuned launch shape (dual phase to the stopping rule, no
    rounding): three sampled members evaluated by the oracle at their final
    multipliers (bound, every slot's min-marginals)."""
    ilps = ilpgen.cell_tracking_batch(3, 64)
    insts = [P.Instance.from_ilp(g, max_rounds=0).build(0) for g in ilps]
    batch = P.Batch(insts)
    iters, _, _ = batch.solve(500)
    assert np.all(iters > 0)
    for q in (0, 31, 63):
        evaluation_parity(oracle_mod.Problem.from_ilp(ilps[q]), insts[q])
    batch.close()


def test_large_mrf_evaluation_parity_full_size(P, oracle_mod):
    g = ilpgen.mrf_grid(512, 512, 4, 1, potts_max=2.0)
    inst = gpu_instance(P, g)
    info = inst.info()
    assert (info["n_vars"], info["n_bdds"], info["n_slots"], info["n_nodes"]) == (9420800, 4448256, 21979136,
                                                                                    39510016)
    n, lb = inst.iterate(25)
    assert n == 25
    run, fea = inst.lower_bound()
    inst.finalize()
    var, row, lam = inst.multipliers()
    orc = oracle_mod.Problem.from_ilp(g)
    perm = slot_order(orc, var, row)
    orc.set_state(lam[perm].astype(np.float64))
    orun, ofea = orc.lower_bounds()
    assert lb_close(fea, ofea, LB_RTOL), (fea, ofea)
    # min-marginals of every slot at the finalised multipliers
    var2, row2, m0, m1 = inst.min_marginals()
    om0, om1 = orc.min_marginals()
    perm2 = slot_order(orc, var2, row2)
    assert rel_err(m0[perm2], om0).max() <= MM_RTOL
    assert rel_err(m1[perm2], om1).max() <= MM_RTOL
    assert run <= fea + 1e-6 * abs(fea)
