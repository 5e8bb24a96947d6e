"""Helpers shared by the GPU parity tests: slot matching between the CUDA
library and the oracle, and the tolerances the comparisons use."""
import numpy as np

# min-marginals: |a - b| <= 1e-4 max(1, |a|, |b|); lower bounds: 1e-6 max(1, |a|)
MM_RTOL = 1e-4
LB_RTOL = 1e-6


def rel_err(a, b):
    """Elementwise relative error; an empty comparison yields [0.0] so that .max() works."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0 and b.size == 0:
        return np.zeros(1)
    return np.abs(a - b) / np.maximum(1.0, np.maximum(np.abs(a), np.abs(b)))


def lb_close(a, b, rtol=LB_RTOL, scale=0.0):
    """|a - b| <= rtol * max(1, |a|, |b|, scale).  `scale` is the conditioning
    of the bound as a sum, sum_j |E_j| (0 for the plain relative test)."""
    return abs(a - b) <= rtol * max(1.0, abs(a), abs(b), scale)


def slot_order(orc, gpu_var, gpu_row):
    """Permutation p with oracle slot s == GPU slot p[s] (matched by (row, var))."""
    key_gpu = gpu_row.astype(np.int64) * (1 << 32) + gpu_var.astype(np.int64)
    key_orc = orc.slot_rows().astype(np.int64) * (1 << 32) + orc.slot_vars().astype(np.int64)
    assert len(key_gpu) == len(key_orc)
    ig = np.argsort(key_gpu, kind="stable")
    io = np.argsort(key_orc, kind="stable")
    assert np.array_equal(key_gpu[ig], key_orc[io]), "GPU and oracle slot sets differ"
    perm = np.empty(len(key_orc), np.int64)
    perm[io] = ig
    return perm
