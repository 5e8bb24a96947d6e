"""GPU test of fdog_bound_reduce_noalloc, the lower-bound reduction for
callers that cannot allocate device memory (plug-ins whose host framework owns
every device allocation, real-time loops that forbid allocation after
start-up).  It must give the same bound as the library's own reduction
(fdog_lower_bound) from the same per-subproblem energies, on two calls in a
row (the static scratch keeps the previous call's contents).  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest

import ilpgen
from parity_util import lb_close

pytestmark = pytest.mark.gpu


def test_noalloc_bound_reduce_matches_library_bound():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_10270_gb300 import build as b

    b.build()
    import paper_2111_10270_gb300 as P

    L = P.lib()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    g = ilpgen.mrf_grid(64, 64, 4, 11, potts_max=2.0)  # every variable lies in a row: no presolve constant
    inst = P.Instance.from_ilp(g, tol=0.0).build(0, stream)
    inst.iterate(25)
    inst.finalize()
    _, lb = inst.lower_bound()  # existing entry point: the library's own reduction
    # per-subproblem energies E_j = min(m0, m1) of any layer of row j, from the GPU's min-marginals
    var, row, m0, m1 = inst.min_marginals()
    first = np.unique(row, return_index=True)[1]
    energies = np.minimum(m0[first], m1[first]).astype(np.float64)
    dev_in = torch.from_numpy(energies).to("cuda:0")
    for call in range(2):
        dev_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda:0")
        rc = L.fdog_bound_reduce_noalloc(ctypes.c_void_p(dev_in.data_ptr()), len(energies), 0.0,
                                         ctypes.c_void_p(dev_out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == P.FDOG_OK
        torch.cuda.synchronize()
        got = float(dev_out.item())
        assert lb_close(got, lb), (call, got, lb)
    # sizes beyond the static scratch are rejected before any device work
    rc = L.fdog_bound_reduce_noalloc(ctypes.c_void_p(dev_in.data_ptr()), 8388609, 0.0,
                                     ctypes.c_void_p(dev_out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == P.FDOG_EINVAL
