"""CPU oracle for certified Katz ranking — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  The product path (the CUDA
library and its binding) never touches it, and it shares no code with them:
its arithmetic lives in ``katz_oracle.cpp`` (plain C++, FP64 and exact
128-bit walk counts, following Algorithms 1 and 2 of the paper step by step).

Every function here has at least one pin in ``tests/test_oracle_pins.py``
against something other than itself: brute-force walk enumeration, the
closed form c = alpha A (I - alpha A)^{-1} 1 solved in exact rational
arithmetic, Lemma 2 monotonicity, the complete-graph case of Lemma 3, the
star graph's closed form, the brute-force top-k criterion, and the literal
Algorithm 2 against static recomputation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "katz_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EALPHA, ENOTCONV, EOVERFLOW = 0, 1, 2, 3, 4
_NAMES = {EINVAL: "EINVAL", EALPHA: "EALPHA", ENOTCONV: "ENOTCONV", EOVERFLOW: "EOVERFLOW"}


# stopping criteria of Sec. 3.1
TOPK, RANKING, SCORE, PAIR = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {_NAMES.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (g++, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared",
                               "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            sig = {
                "oracle_max_threads": (ci, []),
                "oracle_set_threads": (None, [ci]),
                "oracle_walks_u128": (ci, [i64, P, P, ci, P]),
                "oracle_alg2_update_u128": (ci, [i64, P, P, ci, P, i64, P, P, P, P]),
                "oracle_session_create": (P, [i64, P, P, ci, i64]),
                "oracle_session_free": (None, [P]),
                "oracle_session_rank": (ci, [P, dbl, i64, dbl, ci]),
                "oracle_session_rank_criterion": (ci, [P, dbl, ci, i64, ctypes.c_int32, ctypes.c_int32, dbl, ci]),
                "oracle_session_update": (ci, [P, i64, P, P, P]),
                "oracle_session_info": (None, [P, P, P, P, P, P, P]),
                "oracle_session_ranking": (i64, [P, P, i64]),
                "oracle_session_bounds": (None, [P, P, P, P]),
                "oracle_session_omega": (ci, [P, ci, P]),
                "oracle_session_alpha_pow": (dbl, [P, ci]),
                "oracle_session_active": (i64, [P, P, i64]),
                "oracle_session_iterations": (ci, [P, dbl, i64, dbl, ci]),
                "oracle_session_run_fixed": (ci, [P, dbl, ci]),
                "oracle_converged_bounds": (ci, [i64, P, P, i64, dbl, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def walks_exact(rowptr, col, r: int) -> list[list[int]]:
    """Exact omega_1..omega_r (Eq. 5 from omega_0 = 1) as Python ints."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    n = rowptr.shape[0] - 1
    out = np.zeros((r, n, 2), np.uint64)
    st = _load().oracle_walks_u128(n, _ptr(rowptr), _ptr(col), r, _ptr(out))
    if st:
        raise OracleError(st, "walks_u128")
    return [[int(out[i, v, 1]) << 64 | int(out[i, v, 0]) for v in range(n)] for i in range(r)]


def _to_u128_array(omega: list[list[int]]) -> np.ndarray:
    r, n = len(omega), len(omega[0])
    a = np.zeros((r, n, 2), np.uint64)
    for i in range(r):
        for v in range(n):
            a[i, v, 0] = omega[i][v] & ((1 << 64) - 1)
            a[i, v, 1] = omega[i][v] >> 64
    return a


def alg2_update_exact(rowptr, col, omega: list[list[int]], src, dst, ins) -> list[list[int]]:
    """Algorithm 2 (literal, exact) applied to walk counts omega_1..omega_r of
    the graph (rowptr, col) for the arcs src->dst (ins 1 = insert, 0 = delete)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    col = np.ascontiguousarray(col, np.int32)
    n = rowptr.shape[0] - 1
    r = len(omega)
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    ins = np.ascontiguousarray(ins, np.uint8)
    a_in = _to_u128_array(omega)
    a_out = np.zeros_like(a_in)
    st = _load().oracle_alg2_update_u128(n, _ptr(rowptr), _ptr(col), r, _ptr(a_in), src.shape[0], _ptr(src),
                                         _ptr(dst), _ptr(ins), _ptr(a_out))
    if st:
        raise OracleError(st, "alg2_update")
    return [[int(a_out[i, v, 1]) << 64 | int(a_out[i, v, 0]) for v in range(n)] for i in range(r)]


def converged_bounds(lower, upper, k: int, eps: float):
    """converged() of Algorithm 1 over all nodes (M = V) on the given bounds:
    (certified, top) with top = the min(k, n) largest lower bounds in
    decreasing order, ties by smaller id."""
    lower = np.ascontiguousarray(lower, np.float64)
    upper = np.ascontiguousarray(upper, np.float64)
    n = lower.shape[0]
    top = np.empty(max(min(k, n), 1), np.int32)
    ok = _load().oracle_converged_bounds(n, _ptr(lower), _ptr(upper), int(k), float(eps), _ptr(top))
    return bool(ok), top[:min(k, n)].copy()


class Session:
    """A graph plus the state of Algorithms 1 and 2 (walk counts omega_0..omega_r,
    partial sums c_r, bounds l_r/u_r, active set M)."""

    def __init__(self, rowptr, col, undirected: bool = True, deg_bound: int = 0):
        self._rowptr = np.ascontiguousarray(rowptr, np.int64)
        self._col = np.ascontiguousarray(col, np.int32)
        self.n = int(self._rowptr.shape[0] - 1)
        self._lib = _load()
        self._h = self._lib.oracle_session_create(self.n, _ptr(self._rowptr), _ptr(self._col),
                                                  1 if undirected else 0, int(deg_bound))
        if not self._h:
            raise OracleError(EINVAL, "session_create")

    def close(self):
        if self._h:
            self._lib.oracle_session_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rank_static(self, alpha: float, k: int, eps: float, r_max: int = 200) -> int:
        """Algorithm 1 with the top-k criterion; returns the status code."""
        return int(self._lib.oracle_session_rank(self._h, alpha, k, eps, r_max))

    def rank(self, alpha: float, criterion: int, eps: float, k: int = 0, pair=(0, 1), r_max: int = 200) -> int:
        """Algorithm 1 with a stopping criterion of Sec. 3.1 (TOPK, RANKING,
        SCORE or PAIR); returns the status code."""
        return int(self._lib.oracle_session_rank_criterion(self._h, alpha, int(criterion), int(k), int(pair[0]),
                                                           int(pair[1]), eps, r_max))

    def apply_update(self, src, dst, ins) -> int:
        """Algorithm 2 semantics for an undirected batch {src[i], dst[i]}."""
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        ins = np.ascontiguousarray(ins, np.uint8)
        return int(self._lib.oracle_session_update(self._h, src.shape[0], _ptr(src), _ptr(dst), _ptr(ins)))

    def run_fixed(self, alpha: float, R: int) -> int:
        """Exactly R iterations of Algorithm 1's loop body, no convergence check."""
        return int(self._lib.oracle_session_run_fixed(self._h, alpha, R))

    def iterations(self, alpha: float, k: int, eps: float, iters: int) -> int:
        return int(self._lib.oracle_session_iterations(self._h, alpha, k, eps, iters))

    def info(self) -> dict:
        r, act, conv = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        a, g, D = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        self._lib.oracle_session_info(self._h, ctypes.byref(r), ctypes.byref(act), ctypes.byref(conv),
                                      ctypes.byref(a), ctypes.byref(g), ctypes.byref(D))
        return {"r": r.value, "active": act.value, "converged": bool(conv.value), "alpha": a.value,
                "gamma": g.value, "deg_bound": D.value}

    def ranking(self) -> np.ndarray:
        ids = np.empty(max(self.n, 1), np.int32)
        kk = self._lib.oracle_session_ranking(self._h, _ptr(ids), ids.shape[0])
        return ids[:kk].copy()

    def bounds(self):
        """(c_r, l_r, u_r) for every node."""
        c, l, u = (np.empty(self.n, np.float64) for _ in range(3))
        self._lib.oracle_session_bounds(self._h, _ptr(c), _ptr(l), _ptr(u))
        return c, l, u

    def omega(self, i: int) -> np.ndarray:
        out = np.empty(self.n, np.float64)
        st = self._lib.oracle_session_omega(self._h, i, _ptr(out))
        if st:
            raise OracleError(st, "omega")
        return out

    def alpha_pow(self, i: int) -> float:
        return float(self._lib.oracle_session_alpha_pow(self._h, i))

    def active(self) -> np.ndarray:
        buf = np.empty(max(self.n, 1), np.int32)
        m = self._lib.oracle_session_active(self._h, _ptr(buf), buf.shape[0])
        return buf[:m].copy()


def katz_static(rowptr, col, alpha: float, k: int, eps: float, undirected: bool = True, r_max: int = 200,
                deg_bound: int = 0) -> dict:
    """One static certified ranking; returns a dict with r, ranking, c, l, u,
    alpha, gamma and the session (for omega)."""
    s = Session(rowptr, col, undirected, deg_bound)
    st = s.rank_static(alpha, k, eps, r_max)
    if st:
        raise OracleError(st, "rank_static")
    info = s.info()
    c, l, u = s.bounds()
    return dict(info, ranking=s.ranking(), c=c, l=l, u=u, session=s)
