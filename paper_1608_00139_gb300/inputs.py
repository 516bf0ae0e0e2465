"""Seeded synthetic inputs: the graphs every test, the benchmark and the oracle runs use.

This module holds no arithmetic of the method (no epsilon, no solve, no closure): it only
draws random 0/1 adjacency matrices with the shapes of the workloads the paper evaluates.

Random numbers: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator.  The c-th draw of a
stream with key k is mix64(k + (c + 1) * GAMMA), where mix64 is SplitMix64's output
function; a uniform in [0, 1) is (draw >> 11) * 2**-53.  Every draw is a pure function of
(key, counter), so matrices can be generated in row chunks, in any order, with the same
result on x86 and Arm.

Workloads (the paper's experiments, Sec. 7):
  * er_digraph      Erdos-Renyi digraph, each ordered pair an edge w.p. p (Sec. 7.1 uses
                    this generator with self-loops allowed; here ``self_loops`` is a flag
                    and off by default, i != j).
  * forest_dag      parent relation of a random forest plus a few extra DAG edges, for
                    the same-generation program (Sec. 7.2, Fig. "Tested programs").
                    Row i holds a 1 at column parent(i): P[i][parent(i)] = 1.
  * pa_dag          directed preferential attachment DAG with Zipf out-degrees, the
                    stand-in for real networks (Sec. 7.1, Table 1) in the serving mix.
  * batch_specs     the sizes and degrees of an uneven batch of closure problems.
  * poisson_stream  arrival times and kinds of a mixed query stream.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = float(2.0 ** -53)

# Stream identifiers: one per purpose so that draws never overlap.
STREAM_ER = 1
STREAM_FOREST_ROOT = 2
STREAM_FOREST_PARENT = 3
STREAM_FOREST_EXTRA = 4
STREAM_FOREST_EXTRA_PICK = 5
STREAM_PA = 6
STREAM_BATCH = 7
STREAM_POISSON = 8


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of one purpose-specific stream derived from a user seed."""
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        k = mix64(np.array([s * GAMMA + np.uint64(stream)], dtype=np.uint64))[0]
        k = mix64(np.array([k ^ np.uint64(stream * 0x632BE59BD9B4E019 & 0xFFFFFFFFFFFFFFFF)],
                           dtype=np.uint64))[0]
    return np.uint64(k)


def draws(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """Raw 64-bit draws number ``counters`` of stream ``key``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + (c + np.uint64(1)) * GAMMA)


def uniforms(key: np.uint64, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) for draws number ``counters`` of stream ``key``."""
    return (draws(key, counters) >> np.uint64(11)).astype(np.float64) * _TWO53


def er_digraph(n: int, p: float, seed: int, self_loops: bool = False,
               rows_per_chunk: int = 512) -> np.ndarray:
    """Erdos-Renyi digraph as a dense row-major uint8 0/1 matrix, E[i, j] = 1 iff i -> j.

    Pair (i, j) is an edge iff uniform number i*n + j of the ER stream is below p.  With
    ``self_loops`` false the diagonal is cleared (the generator of Sec. 7.1 draws every
    pair; the benchmark workloads take i != j).
    """
    n = int(n)
    e = np.zeros((n, n), dtype=np.uint8)
    if n == 0 or p <= 0.0:
        return e
    key = stream_key(seed, STREAM_ER)
    cols = np.arange(n, dtype=np.uint64)
    # u < p with u = (draw >> 11) * 2^-53  <=>  (draw >> 11) < ceil(p * 2^53)  (p * 2^53 is exact)
    thr = np.uint64(min(int(np.ceil(p * 2.0 ** 53)), 1 << 53))

    def fill(r0: int) -> None:
        r1 = min(n, r0 + rows_per_chunk)
        rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
        d = draws(key, rows * np.uint64(n) + cols[None, :])
        e[r0:r1] = (d >> np.uint64(11)) < thr

    starts = range(0, n, rows_per_chunk)
    if n * n >= (1 << 22) and len(starts) > 1:  # numpy releases the GIL: chunks in threads
        with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    else:
        for r0 in starts:
            fill(r0)
    if not self_loops:
        np.fill_diagonal(e, 0)
    return e


def forest_dag(n: int, seed: int, root_prob: float = 0.05, extra_prob: float = 0.005,
               extra_per_pair: bool = False) -> np.ndarray:
    """Parent relation P of a random forest plus extra DAG edges (same-generation input).

    Node 0 is a root.  Node i >= 1 is a root w.p. ``root_prob``; otherwise its parent is
    uniform in [0, i).  P[i][parent(i)] = 1, so every edge points to a smaller index and P
    is strictly lower triangular.  Extra DAG edges: by default each node i >= 1 gains, w.p.
    ``extra_prob``, one more parent j uniform in [0, i) with j != parent(i); with
    ``extra_per_pair`` each pair (i, j < i) is an extra edge independently w.p.
    ``extra_prob``.
    """
    n = int(n)
    p = np.zeros((n, n), dtype=np.uint8)
    if n <= 1:
        return p
    idx = np.arange(1, n, dtype=np.uint64)
    k_root = stream_key(seed, STREAM_FOREST_ROOT)
    k_par = stream_key(seed, STREAM_FOREST_PARENT)
    is_root = uniforms(k_root, idx) < root_prob
    i_all = np.arange(1, n, dtype=np.int64)
    par = np.floor(uniforms(k_par, idx) * i_all).astype(np.int64)
    par = np.minimum(par, i_all - 1)
    child = i_all[~is_root]
    p[child, par[~is_root]] = 1
    parent_of = np.full(n, -1, dtype=np.int64)
    parent_of[child] = par[~is_root]
    k_ex = stream_key(seed, STREAM_FOREST_EXTRA)
    if extra_per_pair:
        for r0 in range(1, n, 512):
            r1 = min(n, r0 + 512)
            rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
            cols = np.arange(n, dtype=np.uint64)[None, :]
            u = uniforms(k_ex, rows * np.uint64(n) + cols)
            mask = (u < extra_prob) & (cols < rows)
            p[r0:r1] |= mask.astype(np.uint8)
        return p
    k_pick = stream_key(seed, STREAM_FOREST_EXTRA_PICK)
    gets = uniforms(k_ex, idx) < extra_prob
    u_pick = uniforms(k_pick, idx)
    for i in i_all[gets]:
        cand = int(i) - (1 if parent_of[i] >= 0 else 0)
        if cand <= 0:
            continue
        j = min(int(u_pick[i - 1] * cand), cand - 1)
        if parent_of[i] >= 0 and j >= parent_of[i]:
            j += 1  # skip the existing parent
        p[i, j] = 1
    return p


def zipf_cutoff(a: float, mean: float) -> int:
    """Smallest K such that Zipf(a) truncated to {1..K} has mean >= ``mean`` (bisection)."""
    def m(k: int) -> float:
        ks = np.arange(1, k + 1, dtype=np.float64)
        w = ks ** (-a)
        return float((ks * w).sum() / w.sum())
    lo, hi = 1, 2
    while m(hi) < mean:
        hi *= 2
        if hi > 1 << 26:
            raise ValueError("mean not reachable for this exponent")
    while lo < hi:
        mid = (lo + hi) // 2
        if m(mid) >= mean:
            hi = mid
        else:
            lo = mid + 1
    return lo


def pa_dag(n: int, seed: int, zipf_a: float = 2.1, mean_deg: float = 5.0) -> np.ndarray:
    """Directed preferential-attachment DAG, E[i][j] = 1 for j < i.

    Node i >= 1 draws an out-degree k ~ Zipf(``zipf_a``) on {1..K} (K from
    :func:`zipf_cutoff` so that the mean is ``mean_deg``), clipped to i, and links to k
    distinct earlier nodes j chosen with probability proportional to in_degree(j) + 1.
    """
    n = int(n)
    e = np.zeros((n, n), dtype=np.uint8)
    if n <= 1:
        return e
    kmax = zipf_cutoff(zipf_a, mean_deg)
    ks = np.arange(1, kmax + 1, dtype=np.float64)
    cdf = np.cumsum(ks ** (-zipf_a))
    cdf /= cdf[-1]
    key = stream_key(seed, STREAM_PA)
    block = 1 << 16
    buf: list[float] = []
    pos = [0, 0]  # next counter, index into buf

    def nxt() -> float:  # the draws of the stream in counter order, fetched in blocks
        if pos[1] >= len(buf):
            buf[:] = uniforms(key, np.arange(pos[0], pos[0] + block, dtype=np.uint64)).tolist()
            pos[0] += block
            pos[1] = 0
        v = buf[pos[1]]
        pos[1] += 1
        return v

    urn = [0]  # node j appears in_degree(j) + 1 times
    for i in range(1, n):
        u = nxt()
        k = int(np.searchsorted(cdf, u, side="right")) + 1
        k = min(k, kmax, i)
        if k == i:
            chosen = list(range(i))
        else:
            chosen_set: set[int] = set()
            while len(chosen_set) < k:
                m = len(urn)
                chosen_set.add(urn[min(int(nxt() * m), m - 1)])
            chosen = sorted(chosen_set)
        e[i, chosen] = 1
        urn.extend(chosen)
        urn.append(i)
    return e


_ZIPF_CDF: dict = {}
_NATIVE = None
_NATIVE_LOCK = threading.Lock()
_HERE = os.path.dirname(os.path.abspath(__file__))


def _zipf_cdf(zipf_a: float, mean_deg: float) -> np.ndarray:
    """The CDF pa_dag draws out-degrees from (cached per exponent and mean)."""
    key = (float(zipf_a), float(mean_deg))
    if key not in _ZIPF_CDF:
        kmax = zipf_cutoff(zipf_a, mean_deg)
        ks = np.arange(1, kmax + 1, dtype=np.float64)
        cdf = np.cumsum(ks ** (-zipf_a))
        cdf /= cdf[-1]
        _ZIPF_CDF[key] = cdf
    return _ZIPF_CDF[key]


def _native():
    """libinputs.so (inputs_native.c, compiled with gcc next to this file when stale)."""
    global _NATIVE
    with _NATIVE_LOCK:
        if _NATIVE is None:
            src = os.path.join(_HERE, "inputs_native.c")
            lib = os.path.join(_HERE, "libinputs.so")
            if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
                tmp = f"{lib}.tmp{os.getpid()}"
                subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src], check=True)
                os.replace(tmp, lib)
            L = ctypes.CDLL(lib)
            L.inputs_pa_dag.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int64]
            L.inputs_pa_dag.restype = ctypes.c_int
            _NATIVE = L
    return _NATIVE


def pa_dag_into(out: np.ndarray, seed: int, zipf_a: float = 2.1, mean_deg: float = 5.0) -> np.ndarray:
    """The matrix of :func:`pa_dag` (n = out.shape[0], same seed) written into ``out`` by the C
    twin of the generator (the same draws in the same order); ``out`` is an n x n uint8 array
    whose rows may be strided (e.g. a view of a larger pinned buffer).  Returns ``out``."""
    n = int(out.shape[0])
    if out.dtype != np.uint8 or out.ndim != 2 or out.shape[1] != n or (n > 1 and out.strides[1] != 1):
        raise ValueError("out must be an n x n uint8 array with contiguous rows")
    cdf = _zipf_cdf(zipf_a, mean_deg)
    key = stream_key(seed, STREAM_PA)
    rc = _native().inputs_pa_dag(n, int(key), cdf.ctypes.data, len(cdf), out.ctypes.data, max(out.strides[0], n))
    if rc != 0:
        raise RuntimeError(f"inputs_pa_dag failed ({rc})")
    return out


def batch_specs(count: int = 1024, seed0: int = 1000, n_lo: int = 32, n_hi: int = 2048,
                d_lo: float = 1.0, d_hi: float = 8.0) -> list[tuple[int, float, int]]:
    """(N, p, seed) of each instance of an uneven batch of closure problems.

    Instance k uses seed ``seed0 + k``; N is uniform in {n_lo..n_hi}; the mean out-degree
    d is uniform in [d_lo, d_hi] and p = d / (N - 1).
    """
    out = []
    for k in range(count):
        key = stream_key(seed0 + k, STREAM_BATCH)
        u = uniforms(key, np.array([0, 1], dtype=np.uint64))
        nk = n_lo + min(int(u[0] * (n_hi - n_lo + 1)), n_hi - n_lo)
        d = d_lo + (d_hi - d_lo) * float(u[1])
        out.append((nk, d / max(nk - 1, 1), seed0 + k))
    return out


def poisson_stream(rate: float, duration: float, seed: int, tc_frac: float = 0.8,
                   n_lo: int = 512, n_hi: int = 16384):
    """Arrival times (s), kinds (0 = closure, 1 = same-generation), sizes and seeds.

    Inter-arrival gaps are exponential with the given rate; N is
    floor(exp(U[ln n_lo, ln n_hi])); the kind is closure w.p. ``tc_frac``.
    """
    key = stream_key(seed, STREAM_POISSON)
    t, c = 0.0, 0
    times, kinds, sizes, seeds = [], [], [], []
    while True:
        u = uniforms(key, np.array([c, c + 1, c + 2], dtype=np.uint64))
        c += 3
        t += -math.log(1.0 - float(u[0])) / rate
        if t >= duration:
            break
        times.append(t)
        kinds.append(0 if float(u[1]) < tc_frac else 1)
        nn = int(math.floor(math.exp(math.log(n_lo) + float(u[2]) *
                                     (math.log(n_hi) - math.log(n_lo)))))
        sizes.append(max(n_lo, min(n_hi, nn)))
        seeds.append(seed * 1_000_003 + len(times))
    return (np.array(times), np.array(kinds, dtype=np.int32),
            np.array(sizes, dtype=np.int64), np.array(seeds, dtype=np.int64))
