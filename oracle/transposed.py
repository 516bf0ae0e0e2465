"""Least solutions of the transposed class (Sec. 6.2), for its example program prog:2:

    r2(x,z) <- r1(x,z).      r2(x,z) <- r1(x,y), r2(z,y).

The recursive atom has its arguments interchanged, so the completion is R2 = min1(R1 + R1 R2^T)
and its linearisation (eq. matrixeq:trans:1) is

    R~2 = eps (R1 + R1 R~2^T),   0 < eps <= 1 / (1 + ||R1||_inf),

with the least (here unique) real solution whose positive entries are the least model.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  Plain numpy / scipy, FP64, no blocking.

  trans_model(R1)          least model by semi-naive evaluation of prog:2 (the T_P fixpoint of
                           Sec. 2): a round's new facts r2(x,z) come from r1(x,y) and a new fact
                           r2(z,y) of the previous round, minus what is known
  trans_naive(R1)          the series of Sec. 5 (eq. series:gen) for this program,
                           R^(k+1) = min1(R1 + R1 (R^(k))^T) from R^(0) = 0, until it stops changing
  trans_rtilde_kron(R1, eps)   R~2 by a dense solve of the vectorised equation: with the
                           commutation matrix K (K vec X = vec X^T) and vec(A X B) = (B^T kron A)
                           vec X (Sec. 6.3), vec R~2 = eps vec R1 + eps (I kron R1) K vec R~2;
                           N^2 unknowns, so for tiny N only
  trans_rtilde_series(R1, eps, tol)  R~2 as the limit of the increasing series of Lemma 3's kind,
                           X_{t+1} = eps (R1 + R1 X_t^T) from X_0 = 0, stopped when a step changes no
                           entry by more than tol (R1 sparse: a step is N * nnz multiply-adds)
  trans_eps(R1)            the default eps = 1 / (1 + ||R1||_inf) (Sec. 6.2)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def trans_eps(r1: np.ndarray) -> float:
    r1 = np.asarray(r1)
    d = float(r1.sum(axis=1).max()) if r1.size else 0.0
    return 1.0 / (1.0 + d)


def _square01(r1: np.ndarray) -> np.ndarray:
    r1 = np.asarray(r1)
    if r1.ndim != 2 or r1.shape[0] != r1.shape[1]:
        raise ValueError("R1 must be square")
    return r1 != 0


def trans_model(r1: np.ndarray) -> np.ndarray:
    """Least model of prog:2 as a dense 0/1 uint8 matrix (semi-naive evaluation)."""
    e = _square01(r1)
    n = e.shape[0]
    if n == 0:
        return np.zeros((0, 0), dtype=np.uint8)
    es = sp.csr_matrix(e.astype(np.float32))
    r = e.copy()
    delta = e.copy()
    while delta.any():
        # r2(x,z) is derived when r1(x,y) holds and r2(z,y) is a new fact: x's successors y
        # select columns y of delta, i.e. rows y of delta^T
        new = np.asarray(es @ delta.T.astype(np.float32)) > 0
        delta = new & ~r
        r |= delta
    return r.astype(np.uint8)


def trans_naive(r1: np.ndarray, return_iters: bool = False):
    """The series R^(k+1) = min1(R1 + R1 (R^(k))^T) from 0 until a fixpoint; dense uint8."""
    e = _square01(r1).astype(np.int64)
    n = e.shape[0]
    r = np.zeros((n, n), dtype=np.int64)
    k = 0
    while True:
        nxt = np.minimum(e + e @ r.T, 1)
        k += 1
        if np.array_equal(nxt, r):
            break
        r = nxt
    out = r.astype(np.uint8)
    return (out, k) if return_iters else out


def trans_rtilde_kron(r1: np.ndarray, eps: float | None = None) -> np.ndarray:
    """R~2 from the N^2 x N^2 linear system (dense; N <= about 30)."""
    e = _square01(r1).astype(np.float64)
    n = e.shape[0]
    if eps is None:
        eps = trans_eps(e)
    if n == 0:
        return np.zeros((0, 0))
    # vec stacks columns: vec(X)[i + n j] = X[i][j]; (K v)[i + n j] = v[j + n i] gives vec X^T
    kperm = np.zeros((n * n, n * n))
    for i in range(n):
        for j in range(n):
            kperm[i + n * j, j + n * i] = 1.0
    op = np.kron(np.eye(n), e) @ kperm  # vec(R1 X^T) = (I kron R1) vec(X^T)
    vec = np.linalg.solve(np.eye(n * n) - eps * op, eps * e.reshape(-1, order="F"))
    return vec.reshape((n, n), order="F")


def trans_rtilde_series(r1: np.ndarray, eps: float | None = None, tol: float = 0.0, max_steps: int = 100000,
                        return_steps: bool = False):
    """R~2 by the series X_{t+1} = eps (R1 + R1 X_t^T) from 0; stops when max |X_{t+1} - X_t| <= tol."""
    e = _square01(r1)
    n = e.shape[0]
    if eps is None:
        eps = trans_eps(e)
    es = sp.csr_matrix(e.astype(np.float64))
    ed = e.astype(np.float64)
    x = np.zeros((n, n))
    steps = 0
    while steps < max_steps:
        nxt = eps * (ed + np.asarray(es @ x.T))
        steps += 1
        change = float(np.abs(nxt - x).max()) if n else 0.0
        x = nxt
        if change <= tol:
            break
    return (x, steps) if return_steps else x
