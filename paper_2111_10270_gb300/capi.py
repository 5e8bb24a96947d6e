"""ctypes binding of include/fastdog.h (argument marshalling only).

Every entry point of the C ABI is exposed under its C name on the object
returned by ``lib()``; ``Instance`` wraps an fdog_instance* and converts
numpy arrays and torch streams into plain pointers.  All arithmetic happens
inside the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

FDOG_OK = 0
FDOG_EINVAL = -1
FDOG_ENOMEM = -2
FDOG_EINFEASIBLE = -3
FDOG_ECUDA = -4
FDOG_ESTATE = -5
FDOG_ETIMEOUT = -6
FDOG_ENOCONVERGE = -7
FDOG_EUNSUPPORTED = -8
FDOG_LE, FDOG_EQ, FDOG_GE = -1, 0, 1
PLAN_DIGESTS = 9  # FDOG_PLAN_DIGESTS

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_build", "libfastdog.so")
_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("omega", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("window", ctypes.c_int32),
        ("min_iters", ctypes.c_int32),
        ("rounding_dual_iters", ctypes.c_int32),
        ("max_rounds", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("block_threads", ctypes.c_int32),
        ("jit", ctypes.c_int32),
        ("fuse", ctypes.c_int32),
        ("grid_waves", ctypes.c_int32),
        ("update", ctypes.c_int32),
        ("planner", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


# C name -> (restype, argtypes)
_P = ctypes.c_void_p
_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "fdog_host_cache_release": (ctypes.c_int, [ctypes.POINTER(_i64)]),
    "fdog_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "fdog_create": (ctypes.c_int, [_i32, _P, _i32, _P, _P, _P, _P, _P, ctypes.POINTER(Params), ctypes.POINTER(_P)]),
    "fdog_plan": (ctypes.c_int, [_P, ctypes.POINTER(_i64)]),
    "fdog_fixed_vars": (ctypes.c_int, [_P, _P]),
    "fdog_plan_stats": (ctypes.c_int, [_P, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)]),
    "fdog_plan_digest": (ctypes.c_int, [_P, _P]),
    "fdog_split_rows": (ctypes.c_int, [_i32, _i32, _P, _P, _P, _P, _P, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                       ctypes.POINTER(_i64), _P, _P, _P, _P, _P, _P]),
    "fdog_kernel_plan": (ctypes.c_int, [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                        ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                        ctypes.c_char_p, _i32]),
    "fdog_row_bdd": (ctypes.c_int, [_P, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _P, _P, _P, _P]),
    "fdog_build_bdds": (ctypes.c_int, [_P, _i32, _P]),
    "fdog_release": (ctypes.c_int, [_P]),
    "fdog_reset_dual": (ctypes.c_int, [_P]),
    "fdog_transfer_bytes": (ctypes.c_int, [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "fdog_set_profiling": (ctypes.c_int, [_P, _i32]),
    "fdog_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(_i64), ctypes.POINTER(_f64), ctypes.POINTER(_i64),
                                         ctypes.POINTER(_f64), ctypes.POINTER(_i64)]),
    "fdog_dual_iterate": (ctypes.c_int, [_P, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_f64)]),
    "fdog_finalize": (ctypes.c_int, [_P]),
    "fdog_lower_bound": (ctypes.c_int, [_P, ctypes.POINTER(_f64), ctypes.POINTER(_f64)]),
    "fdog_min_marginals": (ctypes.c_int, [_P, ctypes.POINTER(_i64), _P, _P, _P, _P]),
    "fdog_multipliers": (ctypes.c_int, [_P, ctypes.POINTER(_i64), _P, _P, _P]),
    "fdog_primal_round": (ctypes.c_int, [_P, ctypes.POINTER(_i32)]),
    "fdog_solution": (ctypes.c_int, [_P, _P, ctypes.POINTER(_f64), ctypes.POINTER(_i32)]),
    "fdog_export_state": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t)]),
    "fdog_import_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "fdog_info": (ctypes.c_int, [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                 ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "fdog_batch_create": (ctypes.c_int, [_P, _i32, _P, ctypes.POINTER(_P)]),
    "fdog_batch_solve": (ctypes.c_int, [_P, _i32, _P, _P, _P]),
    "fdog_batch_set_persistent": (ctypes.c_int, [_P, _i32, _f64]),
    "fdog_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "fdog_batch_last_error": (ctypes.c_char_p, [_P]),
    "fdog_batch_destroy": (None, [_P]),
    "fdog_server_create": (ctypes.c_int, [_i32, _i64, _i32, _i32, ctypes.POINTER(_P)]),
    "fdog_server_submit": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "fdog_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                         ctypes.POINTER(_f64), ctypes.POINTER(_f64)]),
    "fdog_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _f64]),
    "fdog_server_take": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(_P)]),
    "fdog_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                          ctypes.POINTER(_i64), ctypes.POINTER(_f64), ctypes.POINTER(_i64)]),
    "fdog_server_last_error": (ctypes.c_char_p, [_P]),
    "fdog_server_destroy": (None, [_P]),
    "fdog_shard_plan": (ctypes.c_int, [_i32, _i32, _P, _P, _P, _i32, _P, _P, _P]),
    "fdog_shard_setup": (ctypes.c_int, [_P, _P, _P]),
    "fdog_shard_info": (ctypes.c_int, [_P, ctypes.POINTER(_i32)]),
    "fdog_shard_pass": (ctypes.c_int, [_P, _i32, _P]),
    "fdog_shard_apply": (ctypes.c_int, [_P, _P]),
    "fdog_shard_bound": (ctypes.c_int, [_P, ctypes.POINTER(_f64)]),
    "fdog_shard_commit": (ctypes.c_int, [_P, _f64, ctypes.POINTER(_i32)]),
    "fdog_bound_reduce_noalloc": (ctypes.c_int, [_P, _i64, _f64, _P, _P]),
    "fdog_last_error": (ctypes.c_char_p, [_P]),
    "fdog_destroy": (None, [_P]),
    "fdog_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(
                    f"CUDA library not built: {_LIB_PATH} is missing (run __graft_entry__.build()); "
                    "there is no CPU fallback")
            L = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


class FdogError(RuntimeError):
    def __init__(self, code, where, detail=""):
        msg = lib().fdog_status_string(code).decode()
        super().__init__(f"{where}: {msg} ({code}){': ' + detail if detail else ''}")
        self.code = code


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def split_rows(n_vars, row_ptr, col, coef, sense, rhs, max_len: int):
    """fdog_split_rows: long at-most-one / exactly-one rows as chains of rows
    of at most max_len variables joined by new binaries (numbered from
    n_vars).  Returns (n_vars, row_ptr, col, coef, sense, rhs, row_origin)."""
    L = lib()
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    coef = np.ascontiguousarray(coef, np.int32)
    sense = np.ascontiguousarray(sense, np.int8)
    rhs = np.ascontiguousarray(rhs, np.int64)
    n_rows = len(row_ptr) - 1
    nv, nr, nnz = _i32(), _i32(), _i64()
    args = (int(n_vars), n_rows, _ptr(row_ptr), _ptr(col), _ptr(coef), _ptr(sense), _ptr(rhs), int(max_len))
    rc = L.fdog_split_rows(*args, ctypes.byref(nv), ctypes.byref(nr), ctypes.byref(nnz), None, None, None, None,
                           None, None)
    if rc != FDOG_OK:
        raise FdogError(rc, "fdog_split_rows")
    o_ptr = np.zeros(nr.value + 1, np.int64)
    o_col = np.zeros(max(nnz.value, 1), np.int32)
    o_coef = np.zeros(max(nnz.value, 1), np.int32)
    o_sense = np.zeros(max(nr.value, 1), np.int8)
    o_rhs = np.zeros(max(nr.value, 1), np.int64)
    o_orig = np.zeros(max(nr.value, 1), np.int32)
    rc = L.fdog_split_rows(*args, ctypes.byref(nv), ctypes.byref(nr), ctypes.byref(nnz), _ptr(o_ptr), _ptr(o_col),
                           _ptr(o_coef), _ptr(o_sense), _ptr(o_rhs), _ptr(o_orig))
    if rc != FDOG_OK:
        raise FdogError(rc, "fdog_split_rows")
    m, k = nr.value, nnz.value
    return nv.value, o_ptr, o_col[:k], o_coef[:k], o_sense[:m], o_rhs[:m], o_orig[:m]


def shard_plan(n_vars, row_ptr, col, coef, n_shards: int):
    """fdog_shard_plan: (row_shard, copies, shared) of the rows split into
    n_shards contiguous blocks with about equal numbers of non-zero entries."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    coef = np.ascontiguousarray(coef, np.int32)
    n_rows = len(row_ptr) - 1
    row_shard = np.zeros(max(n_rows, 1), np.int32)
    copies = np.zeros(max(int(n_vars), 1), np.int32)
    shared = np.zeros(max(int(n_vars), 1), np.uint8)
    rc = lib().fdog_shard_plan(int(n_vars), n_rows, _ptr(row_ptr), _ptr(col), _ptr(coef), int(n_shards),
                               _ptr(row_shard), _ptr(copies), _ptr(shared))
    if rc != FDOG_OK:
        raise FdogError(rc, "fdog_shard_plan")
    return row_shard[:n_rows], copies[:n_vars], shared[:n_vars]


def host_cache_release() -> int:
    """fdog_host_cache_release: frees the cached large host buffers, returns their bytes."""
    b = _i64()
    rc = lib().fdog_host_cache_release(ctypes.byref(b))
    if rc != FDOG_OK:
        raise FdogError(rc, "fdog_host_cache_release")
    return b.value


def default_params(**kw) -> Params:
    p = Params()
    lib().fdog_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Instance:
    """Owns one fdog_instance*: create from CSR arrays, build on a device."""

    def __init__(self, n_vars, cost, row_ptr, col, coef, sense, rhs, params: Params | None = None, **kw):
        L = lib()
        self._L = L
        self.n_vars = int(n_vars)
        cost = np.ascontiguousarray(cost, np.float64)
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        coef = np.ascontiguousarray(coef, np.int32)
        sense = np.ascontiguousarray(sense, np.int8)
        rhs = np.ascontiguousarray(rhs, np.int64)
        self.params = params if params is not None else default_params(**kw)
        h = ctypes.c_void_p()
        rc = L.fdog_create(self.n_vars, _ptr(cost), len(row_ptr) - 1, _ptr(row_ptr), _ptr(col), _ptr(coef),
                           _ptr(sense), _ptr(rhs), ctypes.byref(self.params), ctypes.byref(h))
        if rc != FDOG_OK:
            raise FdogError(rc, "fdog_create")
        self._h = h

    @classmethod
    def from_ilp(cls, ilp, params: Params | None = None, **kw):
        return cls(ilp.n_vars, ilp.cost, ilp.row_ptr, ilp.col, ilp.coef, ilp.sense, ilp.rhs, params, **kw)

    def _check(self, rc, where):
        if rc not in (FDOG_OK,):
            detail = self._L.fdog_last_error(self._h)
            raise FdogError(rc, where, detail.decode() if detail else "")
        return rc

    def close(self):
        h = getattr(self, "_h", None)
        if h and not getattr(self, "_h_owned_by_server", False):
            self._L.fdog_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def build(self, device: int = 0, stream=None):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (default stream)."""
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._check(self._L.fdog_build_bdds(self._h, device, ctypes.c_void_p(stream) if stream else None),
                    "fdog_build_bdds")
        return self

    def release(self):
        """Frees the device memory; plan and last solution stay on the host."""
        self._check(self._L.fdog_release(self._h), "fdog_release")
        return self

    def plan(self) -> int:
        b = _i64()
        self._check(self._L.fdog_plan(self._h, ctypes.byref(b)), "fdog_plan")
        return b.value

    def kernel_plan(self):
        js, jt, st, lv, wv, ws = _i32(), _i64(), _i64(), _i64(), _i64(), _i64()
        note = ctypes.create_string_buffer(2048)
        self._check(self._L.fdog_kernel_plan(self._h, ctypes.byref(js), ctypes.byref(jt), ctypes.byref(st),
                                             ctypes.byref(lv), ctypes.byref(wv), ctypes.byref(ws), note, 2048),
                    "fdog_kernel_plan")
        return {"jit_shapes": js.value, "jit_tiles": jt.value, "static_tiles": st.value, "local_vars": lv.value,
                "work_vars": wv.value, "work_slots": ws.value, "note": note.value.decode(errors="replace")}

    def plan_stats(self):
        """(built on the device?, seconds spent building the decomposition)"""
        od, sec = _i32(), ctypes.c_double()
        self._check(self._L.fdog_plan_stats(self._h, ctypes.byref(od), ctypes.byref(sec)), "fdog_plan_stats")
        return bool(od.value), sec.value

    def plan_digest(self):
        """Per-part fingerprints of the decomposition (equal digests: equal device layout)."""
        d = np.zeros(PLAN_DIGESTS, np.uint64)
        self._check(self._L.fdog_plan_digest(self._h, _ptr(d)), "fdog_plan_digest")
        return d

    def fixed_vars(self):
        f = np.zeros(self.n_vars, np.int8)
        self._check(self._L.fdog_fixed_vars(self._h, _ptr(f)), "fdog_fixed_vars")
        return f

    def row_bdd(self, row: int):
        """(vars, lstart, lo, hi) of an original row's BDD, or None if presolve removed the row."""
        k, nn = _i32(), _i32()
        self._check(self._L.fdog_row_bdd(self._h, row, ctypes.byref(k), ctypes.byref(nn), None, None, None, None),
                    "fdog_row_bdd")
        if k.value == 0:
            return None
        vars_ = np.zeros(k.value, np.int32)
        ls = np.zeros(k.value + 1, np.int32)
        lo = np.zeros(nn.value, np.int32)
        hi = np.zeros(nn.value, np.int32)
        self._check(self._L.fdog_row_bdd(self._h, row, ctypes.byref(k), ctypes.byref(nn), _ptr(vars_), _ptr(ls),
                                         _ptr(lo), _ptr(hi)), "fdog_row_bdd")
        return vars_, ls, lo, hi

    def reset(self):
        self._check(self._L.fdog_reset_dual(self._h), "fdog_reset_dual")

    def transfer_bytes(self):
        h, d = _i64(), _i64()
        self._check(self._L.fdog_transfer_bytes(self._h, ctypes.byref(h), ctypes.byref(d)), "fdog_transfer_bytes")
        return h.value, d.value

    def set_profiling(self, on: bool):
        self._check(self._L.fdog_set_profiling(self._h, 1 if on else 0), "fdog_set_profiling")

    def profile_read(self):
        ns, ms, nr, mr, nk = _i64(), _f64(), _i64(), _f64(), _i64()
        self._check(self._L.fdog_profile_read(self._h, ctypes.byref(ns), ctypes.byref(ms), ctypes.byref(nr),
                                              ctypes.byref(mr), ctypes.byref(nk)), "fdog_profile_read")
        return {"sweep_launches": ns.value, "sweep_ms": ms.value, "reduce_launches": nr.value, "reduce_ms": mr.value,
                "kernel_launches": nk.value}

    def iterate(self, k: int):
        done, lb = _i32(), _f64()
        self._check(self._L.fdog_dual_iterate(self._h, k, ctypes.byref(done), ctypes.byref(lb)), "fdog_dual_iterate")
        return done.value, lb.value

    def finalize(self):
        self._check(self._L.fdog_finalize(self._h), "fdog_finalize")

    def lower_bound(self):
        a, b = _f64(), _f64()
        self._check(self._L.fdog_lower_bound(self._h, ctypes.byref(a), ctypes.byref(b)), "fdog_lower_bound")
        return a.value, b.value

    def _slot_count(self, fn):
        n = _i64(0)
        self._check(fn(self._h, ctypes.byref(n), None, None, None, None) if fn is self._L.fdog_min_marginals
                    else fn(self._h, ctypes.byref(n), None, None, None), fn.__name__)
        return n.value

    def min_marginals(self):
        n = self._slot_count(self._L.fdog_min_marginals)
        var = np.zeros(n, np.int32)
        row = np.zeros(n, np.int32)
        m0 = np.zeros(n, np.float32)
        m1 = np.zeros(n, np.float32)
        cap = _i64(n)
        self._check(self._L.fdog_min_marginals(self._h, ctypes.byref(cap), _ptr(var), _ptr(row), _ptr(m0), _ptr(m1)),
                    "fdog_min_marginals")
        return var, row, m0, m1

    def multipliers(self):
        n = self._slot_count(self._L.fdog_multipliers)
        var = np.zeros(n, np.int32)
        row = np.zeros(n, np.int32)
        lam = np.zeros(n, np.float32)
        cap = _i64(n)
        self._check(self._L.fdog_multipliers(self._h, ctypes.byref(cap), _ptr(var), _ptr(row), _ptr(lam)),
                    "fdog_multipliers")
        return var, row, lam

    def primal_round(self):
        r = _i32()
        rc = self._L.fdog_primal_round(self._h, ctypes.byref(r))
        if rc not in (FDOG_OK, FDOG_ENOCONVERGE):
            self._check(rc, "fdog_primal_round")
        return rc, r.value

    def solution(self):
        x = np.zeros(self.n_vars, np.uint8)
        obj, feas = _f64(), _i32()
        self._check(self._L.fdog_solution(self._h, _ptr(x), ctypes.byref(obj), ctypes.byref(feas)), "fdog_solution")
        return x, obj.value, bool(feas.value)

    def export_state(self) -> bytes:
        n = ctypes.c_size_t(0)
        self._check(self._L.fdog_export_state(self._h, None, ctypes.byref(n)), "fdog_export_state")
        buf = (ctypes.c_char * n.value)()
        self._check(self._L.fdog_export_state(self._h, buf, ctypes.byref(n)), "fdog_export_state")
        return bytes(buf)

    def import_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._check(self._L.fdog_import_state(self._h, buf, len(blob)), "fdog_import_state")

    # ---- one shard of a split instance (see fastdog.h, fdog_shard_*) ----
    def shard_setup(self, shared, copies):
        shared = np.ascontiguousarray(shared, np.uint8)
        copies = np.ascontiguousarray(copies, np.int32)
        assert len(shared) == self.n_vars and len(copies) == self.n_vars
        self._check(self._L.fdog_shard_setup(self._h, _ptr(shared), _ptr(copies)), "fdog_shard_setup")
        return self

    def shard_info(self) -> int:
        n = _i32()
        self._check(self._L.fdog_shard_info(self._h, ctypes.byref(n)), "fdog_shard_info")
        return n.value

    def shard_pass(self, descending: bool, dev_sums: int):
        self._check(self._L.fdog_shard_pass(self._h, 1 if descending else 0, ctypes.c_void_p(dev_sums)),
                    "fdog_shard_pass")

    def shard_apply(self, dev_sums: int):
        self._check(self._L.fdog_shard_apply(self._h, ctypes.c_void_p(dev_sums)), "fdog_shard_apply")

    def shard_bound(self) -> float:
        v = _f64()
        self._check(self._L.fdog_shard_bound(self._h, ctypes.byref(v)), "fdog_shard_bound")
        return v.value

    def shard_commit(self, lb: float) -> bool:
        stop = _i32()
        self._check(self._L.fdog_shard_commit(self._h, float(lb), ctypes.byref(stop)), "fdog_shard_commit")
        return bool(stop.value)

    def info(self):
        v = [_i64() for _ in range(5)]
        self._check(self._L.fdog_info(self._h, *[ctypes.byref(x) for x in v]), "fdog_info")
        keys = ("n_vars", "n_bdds", "n_slots", "n_nodes", "device_bytes")
        return dict(zip(keys, (x.value for x in v)))


class Batch:
    """Owns one fdog_batch* over built Instances (which must outlive it)."""

    def __init__(self, instances, stream=None):
        L = lib()
        self._L = L
        self.instances = list(instances)
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        arr = (ctypes.c_void_p * len(self.instances))(*[i._h.value for i in self.instances])
        h = ctypes.c_void_p()
        rc = L.fdog_batch_create(arr, len(self.instances), ctypes.c_void_p(stream) if stream else None,
                                 ctypes.byref(h))
        if rc != FDOG_OK:
            raise FdogError(rc, "fdog_batch_create")
        self._h = h

    def solve(self, max_iters: int):
        n = len(self.instances)
        iters = np.zeros(n, np.int32)
        rounds = np.zeros(n, np.int32)
        status = np.zeros(n, np.int32)
        rc = self._L.fdog_batch_solve(self._h, max_iters, _ptr(iters), _ptr(rounds), _ptr(status))
        if rc != FDOG_OK:
            detail = self._L.fdog_batch_last_error(self._h)
            raise FdogError(rc, "fdog_batch_solve", detail.decode() if detail else "")
        return iters, rounds, status

    def set_persistent(self, on: bool = True, barrier_wait_s: float = 0.0):
        """fdog_batch_set_persistent: dual iterations as one persistent kernel per chunk."""
        rc = self._L.fdog_batch_set_persistent(self._h, 1 if on else 0, float(barrier_wait_s))
        if rc != FDOG_OK:
            detail = self._L.fdog_batch_last_error(self._h)
            raise FdogError(rc, "fdog_batch_set_persistent", detail.decode() if detail else "")
        return self

    def info(self):
        w, c, k = _i32(), _i32(), _i64()
        self._L.fdog_batch_info(self._h, ctypes.byref(w), ctypes.byref(c), ctypes.byref(k))
        return {"warps_per_block": w.value, "chunk": c.value, "kernel_launches": k.value}

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.fdog_batch_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


class Server:
    """Owns one fdog_server*; submit() hands Instances (created, not built) to it."""

    def __init__(self, device=0, hbm_budget=64 << 30, max_active=256, max_iters=500):
        L = lib()
        self._L = L
        h = ctypes.c_void_p()
        rc = L.fdog_server_create(device, hbm_budget, max_active, max_iters, ctypes.byref(h))
        if rc != FDOG_OK:
            raise FdogError(rc, "fdog_server_create")
        self._h = h
        self._owned = {}

    def submit(self, inst: "Instance") -> int:
        t = ctypes.c_uint64()
        rc = self._L.fdog_server_submit(self._h, inst._h, ctypes.byref(t))
        if rc != FDOG_OK:
            detail = self._L.fdog_last_error(inst._h)
            raise FdogError(rc, "fdog_server_submit", detail.decode() if detail else "")
        self._owned[t.value] = inst
        inst._h_owned_by_server = True
        return t.value

    def poll(self, ticket: int):
        st, status, lb, lat = _i32(), _i32(), _f64(), _f64()
        rc = self._L.fdog_server_poll(self._h, ticket, ctypes.byref(st), ctypes.byref(status), ctypes.byref(lb),
                                      ctypes.byref(lat))
        if rc != FDOG_OK:
            raise FdogError(rc, "fdog_server_poll")
        return {"state": st.value, "status": status.value, "lb": lb.value, "latency_s": lat.value}

    def wait(self, ticket: int, timeout_s: float = 600.0) -> bool:
        return self._L.fdog_server_wait(self._h, ticket, timeout_s) == FDOG_OK

    def take(self, ticket: int) -> "Instance":
        h = ctypes.c_void_p()
        rc = self._L.fdog_server_take(self._h, ticket, ctypes.byref(h))
        if rc != FDOG_OK:
            raise FdogError(rc, "fdog_server_take")
        inst = self._owned.pop(ticket)
        inst._h_owned_by_server = False
        return inst

    def stats(self):
        v = [_i64(), _i64(), _i64(), _i64(), _f64(), _i64()]
        self._L.fdog_server_stats(self._h, *[ctypes.byref(x) for x in v])
        keys = ("queued", "resident", "completed", "hbm_used", "busy_s", "kernel_launches")
        return dict(zip(keys, (x.value for x in v)))

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.fdog_server_destroy(h)  # destroys instances not taken
            for inst in self._owned.values():
                inst._h = None
            self._owned.clear()
            self._h = None

    def __del__(self):
        self.close()
