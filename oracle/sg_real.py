"""Real-valued least solution S~ of the same-generation matrix equation (Sec. 7.2):

    S~ = eps (B + P S~ P^T),   eps = 1 / (1 + ||P||_inf^2)   (B = I: the diag facts)

whose positive entries are the least model of sg (Sec. 7.2; the two-sided class of Sec. 6.3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: imported by ``tests/`` and by the
CPU-baseline leg of ``bench.py``, never by the package.  Plain FP64 numpy/scipy, no blocking.

  sg_stilde_kron(P, B, eps)    the vectorised equation of Sec. 6.3 (eq. veceq:two-sided:1) with
                               R_1 = P, R_3 = P^T:  (I - eps (P kron P)) vec S~ = eps vec B, solved
                               as one dense linear system.  O(N^6): tiny N only.
  sg_stilde_series(P, B, eps)  the fixpoint iteration X <- eps (B + P X P^T) from X = 0, the least
                               solution as the limit of an increasing sequence (every term is
                               non-negative), run until an iteration changes nothing in FP64.
"""
from __future__ import annotations

import numpy as np


def _inputs(p, b, eps):
    p = np.ascontiguousarray(p, dtype=np.float64)
    n = p.shape[0]
    if p.ndim != 2 or p.shape[1] != n:
        raise ValueError("P must be square")
    bm = np.eye(n) if b is None else np.ascontiguousarray(b, dtype=np.float64)
    if bm.shape != p.shape:
        raise ValueError("B must have the shape of P")
    if eps is None:
        d = p.sum(axis=1).max() if n else 0.0
        eps = 1.0 / (1.0 + d * d)  # Sec. 7.2
    return p, bm, float(eps)


def sg_stilde_kron(p: np.ndarray, b: np.ndarray | None = None, eps: float | None = None) -> np.ndarray:
    """S~ from the Kronecker form of Sec. 6.3: vec(P X P^T) = (P kron P) vec X for row-major vec."""
    p, bm, eps = _inputs(p, b, eps)
    n = p.shape[0]
    if n > 40:
        raise ValueError("the Kronecker solve is for tiny N (N^2 unknowns)")
    if n == 0:
        return np.zeros((0, 0))
    k = np.kron(p, p)
    x = np.linalg.solve(np.eye(n * n) - eps * k, eps * bm.reshape(-1))
    return x.reshape(n, n)


def sg_stilde_series(p: np.ndarray, b: np.ndarray | None = None, eps: float | None = None,
                     max_iter: int = 100_000, return_iters: bool = False):
    """S~ as the limit of X_{t+1} = eps (B + P X_t P^T), X_0 = 0 (P sparse when large)."""
    p, bm, eps = _inputs(p, b, eps)
    n = p.shape[0]
    x = np.zeros((n, n))
    if n == 0:
        return (x, 0) if return_iters else x
    if n > 64:
        from scipy import sparse
        ps = sparse.csr_matrix(p)

        def step(y):
            return eps * (bm + ps @ (ps @ y.T).T)  # P (Y P^T), with Y P^T = (P Y^T)^T
    else:
        def step(y):
            return eps * (bm + p @ y @ p.T)
    it = 0
    while it < max_iter:
        nx = step(x)
        it += 1
        if np.array_equal(nx, x):
            break
        x = nx
    return (x, it) if return_iters else x
