"""FastDOG oracle -- test infrastructure only.

A plain, slow, single-threaded FP64 CPU implementation of the paper's dual
(Alg. 1 with Eq. 5, lifted form of the Prop. 1 proof), min-marginals by
shortest paths (Eq. 6, Alg. 3/4), perturbation rounding (Alg. 2), the BDD
construction for linear rows (Def. 4, Ex. 1) and the objective.  The
arithmetic lives in ``oracle.c``; this module only compiles it with gcc and
marshals numpy arrays through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and the CUDA library never calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EINFEASIBLE, ESTATE, ENOCONVERGE = 0, -1, -2, -3, -5, -7
TOP, BOT = -1, -2


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (portable flags only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, f64, u64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        ptr = ctypes.c_void_p
        sig = {
            "orc_create": (i32, [i32, ptr, i32, ptr, ptr, ptr, ptr, ptr, ctypes.POINTER(P)]),
            "orc_destroy": (None, [P]),
            "orc_lower_bounds": (i32, [P, f64, ptr, ptr]),
            "orc_energies": (i32, [P, ptr]),
            "orc_pass": (i32, [P, i32, f64, ptr]),
            "orc_iterate": (i32, [P, i32, f64, ptr]),
            "orc_iterate_serial": (i32, [P, i32, ptr]),
            "orc_addback": (i32, [P, f64]),
            "orc_min_marginals": (i32, [P, ptr, ptr]),
            "orc_round": (i32, [P, f64, f64, f64, i32, i32, u64, ptr, ptr, ptr, ptr]),
            "orc_splitmix64": (u64, [u64]),
            "orc_uniform_pm1": (f64, [u64, i32, i32]),
            "orc_num_bdds": (i32, [P]),
            "orc_num_slots": (i64, [P]),
            "orc_num_nodes": (i64, [P]),
            "orc_const_lb": (f64, [P]),
            "orc_bdd_info": (i32, [P, i32, ptr, ptr, ptr, ptr]),
            "orc_bdd_nodes": (i32, [P, i32, ptr, ptr, ptr]),
            "orc_slot_vars": (i32, [P, ptr]),
            "orc_fixed": (i32, [P, ptr]),
            "orc_get_state": (i32, [P, ptr, ptr, ptr, ptr]),
            "orc_set_state": (i32, [P, ptr, ptr, ptr]),
            "orc_bdd_shortest_paths": (i32, [P, i32, ptr, ptr]),
            "orc_objective": (f64, [P, ptr]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


def uniform_pm1(seed: int, rnd: int, var: int) -> float:
    return float(_load().orc_uniform_pm1(seed & (2**64 - 1), rnd, var))


class Problem:
    """One 0-1 ILP  min c^T x  s.t. each row  L_j <= a_j^T x <= U_j  (Ex. 1),
    decomposed into one BDD per row after presolve, with the dual state
    initialised as in Alg. 1 (lambda^j_i = c_i / |J_i|, M-bar = 0)."""

    def __init__(self, n_vars, cost, row_ptr, col, coef, sense, rhs):
        lib = _load()
        self._lib = lib
        self.n = int(n_vars)
        self._cost = np.ascontiguousarray(cost, dtype=np.float64)
        self._row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self._col = np.ascontiguousarray(col, dtype=np.int32)
        self._coef = np.ascontiguousarray(coef, dtype=np.int32)
        self._sense = np.ascontiguousarray(sense, dtype=np.int8)
        self._rhs = np.ascontiguousarray(rhs, dtype=np.int64)
        n_rows = len(self._row_ptr) - 1
        h = ctypes.c_void_p()
        rc = lib.orc_create(self.n, _p(self._cost), n_rows, _p(self._row_ptr), _p(self._col), _p(self._coef),
                            _p(self._sense), _p(self._rhs), ctypes.byref(h))
        if rc != OK:
            raise OracleError(rc, "orc_create")
        self._h = h

    @classmethod
    def from_ilp(cls, ilp):
        return cls(ilp.n_vars, ilp.cost, ilp.row_ptr, ilp.col, ilp.coef, ilp.sense, ilp.rhs)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # ---- sizes and structure ------------------------------------------------
    @property
    def m(self) -> int:
        return int(self._lib.orc_num_bdds(self._h))

    @property
    def S(self) -> int:
        return int(self._lib.orc_num_slots(self._h))

    @property
    def N(self) -> int:
        return int(self._lib.orc_num_nodes(self._h))

    @property
    def const_lb(self) -> float:
        return float(self._lib.orc_const_lb(self._h))

    def bdd_info(self, j):
        row, k, nn, s0 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        rc = self._lib.orc_bdd_info(self._h, j, ctypes.byref(row), ctypes.byref(k), ctypes.byref(nn), ctypes.byref(s0))
        if rc != OK:
            raise OracleError(rc, "orc_bdd_info")
        return row.value, k.value, nn.value, s0.value

    def bdd_nodes(self, j):
        _, k, nn, _ = self.bdd_info(j)
        ls = np.zeros(k + 1, np.int32)
        lo = np.zeros(nn, np.int32)
        hi = np.zeros(nn, np.int32)
        self._lib.orc_bdd_nodes(self._h, j, _p(ls), _p(lo), _p(hi))
        return ls, lo, hi

    def slot_vars(self):
        v = np.zeros(self.S, np.int32)
        self._lib.orc_slot_vars(self._h, _p(v))
        return v

    def slot_rows(self):
        r = np.zeros(self.S, np.int32)
        for j in range(self.m):
            row, k, _, s0 = self.bdd_info(j)
            r[s0:s0 + k] = row
        return r

    def fixed(self):
        f = np.zeros(self.n, np.int8)
        self._lib.orc_fixed(self._h, _p(f))
        return f

    # ---- state ----------------------------------------------------------------
    def state(self):
        hi = np.zeros(self.S)
        lo = np.zeros(self.S)
        db0 = np.zeros(self.n)
        db1 = np.zeros(self.n)
        self._lib.orc_get_state(self._h, _p(hi), _p(lo), _p(db0), _p(db1))
        return hi, lo, db0, db1

    def set_state(self, lam, db0=None, db1=None):
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        assert lam.shape == (self.S,)
        db0 = None if db0 is None else np.ascontiguousarray(db0, dtype=np.float64)
        db1 = None if db1 is None else np.ascontiguousarray(db1, dtype=np.float64)
        self._lib.orc_set_state(self._h, _p(lam), _p(db0), _p(db1))

    # ---- Alg. 1 ---------------------------------------------------------------
    def run_pass(self, forward: bool, omega: float = 0.5):
        M = np.zeros(self.S)
        rc = self._lib.orc_pass(self._h, 1 if forward else 0, omega, _p(M))
        if rc != OK:
            raise OracleError(rc, "orc_pass")
        return M

    def iterate(self, k: int, omega: float = 0.5):
        tr = np.zeros(max(k, 1))
        rc = self._lib.orc_iterate(self._h, k, omega, _p(tr))
        if rc != OK:
            raise OracleError(rc, "orc_iterate")
        return tr[:k]

    def iterate_serial(self, k: int):
        """k iterations of the serial min-marginal averaging of Eq. 4 (ascending
        then descending variable order); returns the bound after each."""
        tr = np.zeros(max(k, 1))
        rc = self._lib.orc_iterate_serial(self._h, k, _p(tr))
        if rc != OK:
            raise OracleError(rc, "orc_iterate_serial")
        return tr[:k]

    def addback(self, omega: float = 0.5):
        self._lib.orc_addback(self._h, omega)

    def lower_bounds(self, omega: float = 0.5):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._lib.orc_lower_bounds(self._h, omega, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def energies(self):
        """Lifted energy E(hi^j, lo^j) of every BDD at the current state."""
        E = np.zeros(max(self.m, 1))
        self._lib.orc_energies(self._h, _p(E))
        return E[:self.m]

    def min_marginals(self):
        m0 = np.zeros(self.S)
        m1 = np.zeros(self.S)
        self._lib.orc_min_marginals(self._h, _p(m0), _p(m1))
        return m0, m1

    def shortest_paths(self, j):
        _, _, nn, _ = self.bdd_info(j)
        f = np.zeros(nn)
        g = np.zeros(nn)
        self._lib.orc_bdd_shortest_paths(self._h, j, _p(f), _p(g))
        return f, g

    # ---- Alg. 2 ---------------------------------------------------------------
    def round(self, omega=0.5, delta=1.0, alpha=1.2, kr=20, max_rounds=200, seed=0):
        x = np.zeros(self.n, np.uint8)
        rounds, obj, margin = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        rc = self._lib.orc_round(self._h, omega, delta, alpha, kr, max_rounds, seed & (2**64 - 1), _p(x),
                                 ctypes.byref(rounds), ctypes.byref(obj), ctypes.byref(margin))
        return {"status": rc, "x": x, "rounds": rounds.value, "objective": obj.value, "margin": margin.value}

    def objective(self, x):
        x = np.ascontiguousarray(x, dtype=np.uint8)
        return float(self._lib.orc_objective(self._h, _p(x)))
