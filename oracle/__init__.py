"""CPU oracle for the least models of Sato's linear-algebraic Datalog evaluation.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
CPU-baseline leg of ``bench.py``, never by the package.  It shares no code with the CUDA
library.  The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over rows); this file
only compiles it with gcc and marshals numpy arrays.

Functions (passages they follow are cited in ``oracle.c``):
  tc_model(E)            least model of the transitive-closure program, semi-naive (Sec. 2-3)
  tc_naive(E)            the paper's "Iteration" method (Sec. 7.1, eq. series:trcl)
  tc_rtilde_lu(E, eps)   R~ = (I - eps E)^-1 eps E by FP64 LU (Proposition 1)
  tc_rtilde_col(E, eps, j)  column j of R~ by the series of Lemma 1
  sg_model(P, B)         least model of the same-generation program (Sec. 7.2), semi-naive
  tc_eps(E), sg_eps(P)   the paper's default epsilons (Sec. 4, Sec. 7.1, Sec. 7.2)
  sg_stilde_kron, sg_stilde_series   the real S~ of same generation (sg_real.py, numpy FP64)
  tail_model, tail_rtilde, tail_eps  one equation of the tail recursive class (tail.py)
  trans_model, trans_naive, trans_rtilde_kron, trans_rtilde_series, trans_eps
                         the transposed class, program prog:2 of Sec. 6.2 (transposed.py)
  tail_rtilde_real, tail_system, tail_system_stacked, tail_eps_terms
                         tail recursive equations with real lower solutions and layered systems
                         of them (tail.py)
  program.parse, program.least_model, program.naive_model
                         least models of Datalog programs over binary predicates by symbolic
                         semi-naive evaluation, with stratified negation (program.py)
Bit matrices: ceil(n/64) uint64 words per row, bit j%64 of word j//64, LSB first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .sg_real import sg_stilde_kron, sg_stilde_series  # noqa: F401  (numpy FP64, no C part)
from .tail import tail_eps, tail_model, tail_model_rows, tail_rtilde  # noqa: F401  (numpy FP64)
from .transposed import (trans_eps, trans_model, trans_naive, trans_rtilde_kron,  # noqa: F401
                         trans_rtilde_series)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            f64p = ctypes.POINTER(ctypes.c_double)
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            L.oracle_set_threads.restype = ctypes.c_int
            L.oracle_max_row_sum.argtypes = [ctypes.c_int32, u8p]
            L.oracle_max_row_sum.restype = ctypes.c_int64
            L.oracle_tc_eps.argtypes = [ctypes.c_int32, u8p]
            L.oracle_tc_eps.restype = ctypes.c_double
            L.oracle_sg_eps.argtypes = [ctypes.c_int32, u8p]
            L.oracle_sg_eps.restype = ctypes.c_double
            L.oracle_tc_seminaive.argtypes = [ctypes.c_int32, u8p, u64p, i32p]
            L.oracle_tc_naive.argtypes = [ctypes.c_int32, u8p, u8p, i32p]
            L.oracle_tc_rtilde_lu.argtypes = [ctypes.c_int32, u8p, ctypes.c_double, f64p]
            L.oracle_tc_rtilde_series_col.argtypes = [ctypes.c_int32, u8p, ctypes.c_double,
                                                      ctypes.c_int32, f64p, ctypes.c_int32,
                                                      i32p]
            L.oracle_tc_rtilde_series_row.argtypes = [ctypes.c_int32, u8p, ctypes.c_double,
                                                      ctypes.c_int32, f64p, ctypes.c_int32,
                                                      i32p]
            L.oracle_sg_seminaive.argtypes = [ctypes.c_int32, u8p, u8p, u64p, i32p]
            for f in ("oracle_tc_seminaive", "oracle_tc_naive", "oracle_tc_rtilde_lu",
                      "oracle_tc_rtilde_series_col", "oracle_tc_rtilde_series_row", "oracle_sg_seminaive"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _u8(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix")
    return a


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def words(n: int) -> int:
    return (n + 63) // 64


def set_threads(t: int) -> int:
    """Set the OpenMP thread count (t <= 0 keeps it); returns the count in use."""
    return lib().oracle_set_threads(int(t))


def tc_eps(e: np.ndarray) -> float:
    e = _u8(e)
    return lib().oracle_tc_eps(e.shape[0], _ptr(e, ctypes.c_uint8))


def sg_eps(p: np.ndarray) -> float:
    p = _u8(p)
    return lib().oracle_sg_eps(p.shape[0], _ptr(p, ctypes.c_uint8))


def max_row_sum(a: np.ndarray) -> int:
    a = _u8(a)
    return int(lib().oracle_max_row_sum(a.shape[0], _ptr(a, ctypes.c_uint8)))


def tc_model(e: np.ndarray, return_iters: bool = False):
    """Least model of the closure program as packed bits, shape (n, ceil(n/64)) uint64."""
    e = _u8(e)
    n = e.shape[0]
    out = np.zeros((n, words(n)), dtype=np.uint64)
    it = ctypes.c_int32(0)
    _check(lib().oracle_tc_seminaive(n, _ptr(e, ctypes.c_uint8), _ptr(out, ctypes.c_uint64),
                                     ctypes.byref(it)), "tc_seminaive")
    return (out, it.value) if return_iters else out


def tc_naive(e: np.ndarray, return_iters: bool = False):
    """The paper's Iteration method on 0/1 matrices; dense uint8 (n, n)."""
    e = _u8(e)
    n = e.shape[0]
    out = np.zeros((n, n), dtype=np.uint8)
    it = ctypes.c_int32(0)
    _check(lib().oracle_tc_naive(n, _ptr(e, ctypes.c_uint8), _ptr(out, ctypes.c_uint8),
                                 ctypes.byref(it)), "tc_naive")
    return (out, it.value) if return_iters else out


def tc_rtilde_lu(e: np.ndarray, eps: float | None = None) -> np.ndarray:
    """R~ = (I - eps E)^-1 eps E in FP64 (dense (n, n) float64)."""
    e = _u8(e)
    n = e.shape[0]
    if eps is None:
        eps = tc_eps(e)
    out = np.zeros((n, n), dtype=np.float64)
    _check(lib().oracle_tc_rtilde_lu(n, _ptr(e, ctypes.c_uint8), float(eps),
                                     _ptr(out, ctypes.c_double)), "tc_rtilde_lu")
    return out


def tc_rtilde_col(e: np.ndarray, eps: float, j: int, max_iter: int = 1_000_000,
                  return_iters: bool = False):
    """Column j of R~ by the monotone series of Lemma 1 (FP64)."""
    e = _u8(e)
    n = e.shape[0]
    out = np.zeros(n, dtype=np.float64)
    it = ctypes.c_int32(0)
    _check(lib().oracle_tc_rtilde_series_col(n, _ptr(e, ctypes.c_uint8), float(eps), int(j),
                                             _ptr(out, ctypes.c_double), int(max_iter),
                                             ctypes.byref(it)), "tc_rtilde_series_col")
    return (out, it.value) if return_iters else out


def tc_rtilde_row(e: np.ndarray, eps: float, i: int, max_iter: int = 1_000_000,
                  return_iters: bool = False):
    """Row i of R~ by the series of Lemma 1 read along rows, x <- eps (E_i + x E) (FP64)."""
    e = _u8(e)
    n = e.shape[0]
    out = np.zeros(n, dtype=np.float64)
    it = ctypes.c_int32(0)
    _check(lib().oracle_tc_rtilde_series_row(n, _ptr(e, ctypes.c_uint8), float(eps), int(i),
                                             _ptr(out, ctypes.c_double), int(max_iter),
                                             ctypes.byref(it)), "tc_rtilde_series_row")
    return (out, it.value) if return_iters else out


def sg_model(p: np.ndarray, b: np.ndarray | None = None, return_iters: bool = False):
    """Least model of the same-generation program as packed bits (n, ceil(n/64))."""
    p = _u8(p)
    n = p.shape[0]
    bp = None
    if b is not None:
        b = _u8(b)
        if b.shape != p.shape:
            raise ValueError("B must have the shape of P")
        bp = _ptr(b, ctypes.c_uint8)
    out = np.zeros((n, words(n)), dtype=np.uint64)
    it = ctypes.c_int32(0)
    _check(lib().oracle_sg_seminaive(n, _ptr(p, ctypes.c_uint8), bp,
                                     _ptr(out, ctypes.c_uint64), ctypes.byref(it)),
           "sg_seminaive")
    return (out, it.value) if return_iters else out


def unpack(bits: np.ndarray, n: int) -> np.ndarray:
    """Packed rows -> dense uint8 (n, n) 0/1 matrix."""
    b = np.ascontiguousarray(bits, dtype=np.uint64).reshape(n, words(n))
    by = b.view(np.uint8).reshape(n, words(n) * 8)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n].copy()


def pack(dense: np.ndarray) -> np.ndarray:
    """Dense 0/1 (n, n) -> packed rows (n, ceil(n/64)) uint64."""
    d = np.ascontiguousarray(dense != 0, dtype=np.uint8)
    n = d.shape[0]
    pad = np.zeros((n, words(n) * 64), dtype=np.uint8)
    pad[:, :n] = d
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint64).reshape(n, words(n))
