"""Brute-force references used only to pin the oracle (tiny inputs, pure Python/numpy).

Each is a textbook algorithm that shares nothing with the oracle's semi-naive evaluator or
its LU solve: breadth-first search, Warshall's algorithm (Sec. 7.1 uses it as a third
method), and naive fixpoint iteration of the same-generation equation.
"""
from collections import deque

import numpy as np


def bfs_closure(e: np.ndarray) -> np.ndarray:
    """R[i][j] = 1 iff j is reachable from i by a path of length >= 1."""
    n = e.shape[0]
    succ = [np.flatnonzero(e[i]).tolist() for i in range(n)]
    r = np.zeros((n, n), dtype=np.uint8)
    for s in range(n):
        seen = [False] * n
        q = deque(succ[s])
        for v in succ[s]:
            seen[v] = True
        while q:
            u = q.popleft()
            r[s, u] = 1
            for v in succ[u]:
                if not seen[v]:
                    seen[v] = True
                    q.append(v)
    return r


def bfs_distances(e: np.ndarray) -> np.ndarray:
    """d[i][j] = length of a shortest path of length >= 1 from i to j (0 if none)."""
    n = e.shape[0]
    succ = [np.flatnonzero(e[i]).tolist() for i in range(n)]
    d = np.zeros((n, n), dtype=np.int64)
    for s in range(n):
        dist = {}
        q = deque()
        for v in succ[s]:
            if v not in dist:
                dist[v] = 1
                q.append(v)
        while q:
            u = q.popleft()
            for v in succ[u]:
                if v not in dist:
                    dist[v] = dist[u] + 1
                    q.append(v)
        for v, dv in dist.items():
            d[s, v] = dv
    return d


def warshall(e: np.ndarray) -> np.ndarray:
    """Warshall's algorithm: for k, i: if R[i][k]: R[i] |= R[k]."""
    r = (np.asarray(e) != 0).copy()
    n = r.shape[0]
    for k in range(n):
        for i in range(n):
            if r[i, k]:
                r[i] |= r[k]
    return r.astype(np.uint8)


def sg_naive(p: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """Least S with S = min1(B + P S P^T) by naive iteration from S = 0 (integer matmuls)."""
    n = p.shape[0]
    P = (np.asarray(p) != 0).astype(np.int64)
    B = np.eye(n, dtype=np.int64) if b is None else (np.asarray(b) != 0).astype(np.int64)
    s = np.zeros((n, n), dtype=np.int64)
    while True:
        nx = np.minimum(B + P @ s @ P.T, 1)
        if np.array_equal(nx, s):
            return s.astype(np.uint8)
        s = nx
