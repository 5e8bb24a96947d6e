"""GPU test of fdog_bound_reduce_noalloc, the lower-bound reduction for
callers that cannot allocate device memory (plug-ins whose host framework owns
every device allocation, real-time loops that forbid allocation after
start-up).

It must give the same bound as the library's own evaluation
(fdog_lower_bound) from the same per-subproblem energies, on two calls in a
row (the static scratch keeps the previous call's contents), and equal the
correctly rounded sum of its inputs (math.fsum) to 1e-12 relative at every
size up to its limit.  This file is collected last on purpose: a run that
stops at the first failure has run every other test by then."""
import ctypes
import math

import numpy as np
import pytest

import ilpgen
from parity_util import lb_close, slot_order

pytestmark = pytest.mark.gpu

LIMIT = 8388608  # values per call (the static scratch holds 32,768 block partials of 256 values)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    torch.cuda.set_device(0)
    return torch, P, P.lib(), torch.cuda.current_stream()


def reduce_noalloc(env, dev_in, n, constant):
    torch, P, L, stream = env
    dev_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda:0")
    ptr = ctypes.c_void_p(dev_in.data_ptr()) if dev_in is not None else ctypes.c_void_p(0)
    rc = L.fdog_bound_reduce_noalloc(ptr, n, constant, ctypes.c_void_p(dev_out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))
    assert rc == P.FDOG_OK, rc
    torch.cuda.synchronize()
    return float(dev_out.item())


def close_to_fsum(got, values, constant):
    want = math.fsum(list(values) + [constant])
    scale = max(1.0, math.fsum(abs(v) for v in values) + abs(constant))
    return abs(got - want) <= 1e-12 * scale, (got, want)


def test_noalloc_bound_reduce_matches_library_bound(env, oracle_mod):
    torch, P, L, stream = env
    g = ilpgen.mrf_grid(64, 64, 4, 11, potts_max=2.0)  # every variable lies in a row: no presolve constant
    inst = P.Instance.from_ilp(g, tol=0.0).build(0, stream)
    inst.iterate(25)
    inst.finalize()
    _, lb = inst.lower_bound()  # the existing entry point: the library's own FP64 evaluation
    # per-subproblem energies E_j of the GPU's finalised multipliers, evaluated by the oracle in FP64
    var, row, lam = inst.multipliers()
    orc = oracle_mod.Problem.from_ilp(g)
    orc.set_state(lam[slot_order(orc, var, row)].astype(np.float64))
    energies = np.asarray(orc.energies(), np.float64)
    dev_in = torch.from_numpy(energies).to("cuda:0")
    for call in range(2):
        got = reduce_noalloc(env, dev_in, len(energies), 0.0)
        assert lb_close(got, lb), (call, got, lb)
        ok, detail = close_to_fsum(got, energies, 0.0)
        assert ok, (call, detail)


@pytest.mark.parametrize("n", [0, 1, 255, 256, 257, 100003, LIMIT])
def test_noalloc_bound_reduce_sizes(env, n):
    """Empty input (the constant alone), one value, a partial block, exact and
    ragged multiples of the 256-value block, and the size limit; each twice in
    a row with a nonzero constant."""
    torch = env[0]
    rng = np.random.default_rng(1000 + n)
    values = rng.standard_normal(n) * rng.choice([1e-3, 1.0, 1e3], n)
    dev_in = torch.from_numpy(values).to("cuda:0") if n > 0 else None
    for constant in (-17.25, 3.5e4):
        for call in range(2):
            got = reduce_noalloc(env, dev_in, n, constant)
            ok, detail = close_to_fsum(got, values, constant)
            assert ok, (n, constant, call, detail)
    if n == 0:
        assert reduce_noalloc(env, None, 0, -17.25) == -17.25


def test_noalloc_bound_reduce_rejects_bad_arguments(env):
    """Sizes beyond the static scratch, negative sizes and NULL pointers are
    refused before any device work."""
    torch, P, L, stream = env
    buf = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    p = ctypes.c_void_p(buf.data_ptr())
    s = ctypes.c_void_p(stream.cuda_stream)
    assert L.fdog_bound_reduce_noalloc(p, LIMIT + 1, 0.0, p, s) == P.FDOG_EINVAL
    assert L.fdog_bound_reduce_noalloc(p, -1, 0.0, p, s) == P.FDOG_EINVAL
    assert L.fdog_bound_reduce_noalloc(ctypes.c_void_p(0), 5, 0.0, p, s) == P.FDOG_EINVAL
    assert L.fdog_bound_reduce_noalloc(p, 1, 0.0, ctypes.c_void_p(0), s) == P.FDOG_EINVAL
