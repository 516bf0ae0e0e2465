"""Least solutions of the tail recursive class (Sec. 6.1, eq. matrixeq:trec) for one equation:

    R~ = eps (A + B0 R~),   i.e.  R~ = (I - eps B0)^-1 eps A,

where A stands for the whole non-recursive part A_1 + B_1 R~_{j_1} + ... + B_q R~_{j_q} once the
lower equations are solved and substituted, and B0 is the coefficient of the recursive
occurrence.  The model is the least R with R = min1(A + B0 R).  Transitive closure is the case
A = B0 = E (Sec. 3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.  Plain numpy / FP64, no blocking.

  tail_model(B0, A)          the least model by semi-naive evaluation of R = A u B0 R: the new
                             facts of a round are the B0-predecessors of the previous round's
                             new facts, minus what is known (the T_P fixpoint of Sec. 2)
  tail_model_rows(B0, A, rows)  the model's rows by definition, for sampling at large N: row x is
                             the union of A's rows over the nodes reachable from x in zero or more
                             B0 steps (breadth-first search)
  tail_rtilde(B0, A, eps)    R~ by one dense FP64 solve of (I - eps B0) X = eps A
  tail_eps(B0)               the default eps = 1 / (1 + ||B0||_inf), inside the uniqueness
                             condition eps < 1 / ||B0||_inf of Sec. 6.1
"""
from __future__ import annotations

import numpy as np


def tail_eps(b0: np.ndarray) -> float:
    b0 = np.asarray(b0)
    d = float(b0.sum(axis=1).max()) if b0.size else 0.0
    return 1.0 / (1.0 + d)


def tail_model(b0: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Least R with R = A u B0 R, as a dense 0/1 uint8 matrix."""
    b0 = np.asarray(b0, dtype=np.uint8) != 0
    a = np.asarray(a, dtype=np.uint8) != 0
    if b0.shape != a.shape or b0.ndim != 2 or b0.shape[0] != b0.shape[1]:
        raise ValueError("B0 and A must be square and of one shape")
    r = a.copy()
    delta = a.copy()
    b0f = b0.astype(np.float64)  # counts of 0/1 products, exact in FP64
    while delta.any():
        # (x, z) is derived when x -> y in B0 and (y, z) is a new fact
        new = (b0f @ delta.astype(np.float64)) > 0
        delta = new & ~r
        r |= delta
    return r.astype(np.uint8)


def tail_model_rows(b0: np.ndarray, a: np.ndarray, rows) -> np.ndarray:
    """Rows of the least model (dense 0/1, len(rows) x n), each from a breadth-first search."""
    b0 = np.asarray(b0, dtype=np.uint8)
    a = np.asarray(a, dtype=np.uint8)
    n = b0.shape[0]
    succ = [np.nonzero(b0[y])[0] for y in range(n)]
    out = np.zeros((len(rows), n), dtype=np.uint8)
    for t, x in enumerate(rows):
        seen = np.zeros(n, dtype=bool)
        seen[x] = True
        frontier = [x]
        while frontier:
            nxt = []
            for y in frontier:
                for z in succ[y]:
                    if not seen[z]:
                        seen[z] = True
                        nxt.append(z)
            frontier = nxt
        out[t] = (a[seen].max(axis=0) if seen.any() else 0)
    return out


def tail_rtilde(b0: np.ndarray, a: np.ndarray, eps: float | None = None) -> np.ndarray:
    """R~ = (I - eps B0)^-1 eps A in FP64 (one dense solve)."""
    b0 = np.asarray(b0, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    n = b0.shape[0]
    if eps is None:
        eps = tail_eps(b0)
    if n == 0:
        return np.zeros((0, 0))
    return np.linalg.solve(np.eye(n) - eps * b0, eps * a)


# ---- equations with real lower solutions, and layered systems (Sec. 6.1) --------------------
#
#   R~_h = eps_h (A1_h + B0_h R~_h + sum_q B_q R~_{j_q}),   j_q < h,
#
# solved in order h = 0, 1, ... with the lower R~_{j_q} substituted (the elimination the paper
# describes after eq. matrixeq:trec).  Its model is the least R_h with
# R_h = min1(A1_h + B0_h R_h + sum_q B_q R_{j_q}).

def tail_eps_terms(b0: np.ndarray | None, bs) -> float:
    """The default eps_h = 1 / (1 + max_i (rowsum(B0)_i + sum_q rowsum(B_q)_i)): then
    eps_h F_h[1, ..., 1] <= 1 entrywise (the condition of Theorem 2), and eps_h < 1 / ||B0||_inf
    (the uniqueness condition of Sec. 6.1)."""
    mats = ([] if b0 is None else [np.asarray(b0)]) + [np.asarray(b) for b in bs]
    if not mats:
        return 1.0
    d = sum(m.astype(np.float64).sum(axis=1) for m in mats)
    return 1.0 / (1.0 + float(d.max()))


def tail_rtilde_real(b0, a1, terms, eps: float | None = None) -> np.ndarray:
    """R~ = (I - eps B0)^-1 eps (A1 + sum_q B_q R_q) in FP64; terms = [(B_q, R_q)] with R_q real
    (n x n); B0 or A1 may be None (zero)."""
    n = (b0 if b0 is not None else a1 if a1 is not None else terms[0][0]).shape[0]
    if eps is None:
        eps = tail_eps_terms(b0, [b for b, _ in terms])
    f = np.zeros((n, n)) if a1 is None else np.asarray(a1, dtype=np.float64).copy()
    for b, r in terms:
        f += np.asarray(b, dtype=np.float64) @ np.asarray(r, dtype=np.float64)
    a = np.eye(n) - (0.0 if b0 is None else eps * np.asarray(b0, dtype=np.float64))
    return np.linalg.solve(a, eps * f)


def _eq_parts(eq, n):
    z = np.zeros((n, n), dtype=np.uint8)
    a1 = z if eq.get("A1") is None else np.asarray(eq["A1"], dtype=np.uint8)
    b0 = z if eq.get("B0") is None else np.asarray(eq["B0"], dtype=np.uint8)
    return a1, b0, list(eq.get("terms", []))


def tail_system(eqs, n: int):
    """In-order solution of a layered system: eqs[h] = {"A1", "B0", "terms": [(B, j)], "eps"}
    with every j < h.  Returns (models (dense 0/1), R~ (FP64), eps per equation)."""
    models, xs, epss = [], [], []
    for h, eq in enumerate(eqs):
        a1, b0, terms = _eq_parts(eq, n)
        if any(j >= h for _, j in terms):
            raise ValueError("a term refers to an equation that is not below")
        eps = eq.get("eps") or tail_eps_terms(b0, [b for b, _ in terms])
        a = a1.astype(np.int64)
        for b, j in terms:
            a = a + np.asarray(b, dtype=np.int64) @ models[j].astype(np.int64)
        models.append(tail_model(b0, np.minimum(a, 1).astype(np.uint8)))
        xs.append(tail_rtilde_real(b0, a1, [(b, xs[j]) for b, j in terms], eps))
        epss.append(eps)
    return models, xs, epss


def tail_system_stacked(eqs, n: int, epss) -> list:
    """The same R~ from one dense solve of the whole system: unknowns stacked (m n x n), block
    (h, h) = I - eps_h B0_h, block (h, j) = -eps_h (sum of the B_q with j_q = j), right-hand side
    block h = eps_h A1_h."""
    m = len(eqs)
    big = np.eye(m * n)
    rhs = np.zeros((m * n, n))
    for h, eq in enumerate(eqs):
        a1, b0, terms = _eq_parts(eq, n)
        e = epss[h]
        big[h * n:(h + 1) * n, h * n:(h + 1) * n] -= e * b0.astype(np.float64)
        for b, j in terms:
            big[h * n:(h + 1) * n, j * n:(j + 1) * n] -= e * np.asarray(b, dtype=np.float64)
        rhs[h * n:(h + 1) * n] = e * a1.astype(np.float64)
    x = np.linalg.solve(big, rhs)
    return [x[h * n:(h + 1) * n] for h in range(m)]
