"""Pins of the CPU oracle for transitive closure (no GPU).

The oracle's least model (semi-naive) and its FP64 R~ (LU; Lemma-1 series) are checked
against things other than themselves: the paper's worked example (golden fixture), BFS and
Warshall on every small digraph, the paper's own Iteration method, closed forms of R~ on
graphs whose inverse is known, and the inequalities of Lemma 1 and Lemma 2.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1608_00139_gb300 import inputs
from tests import brute
from tests.golden.load import read


def dense_model(e):
    return oracle.unpack(oracle.tc_model(e), e.shape[0])


# --- worked example (Sec. 4, after Proposition 1) -------------------------------------

def test_worked_example_rtilde_and_model():
    g = read("worked_example_tc.txt")
    e = g["R1"].astype(np.uint8)
    eps = float(g["eps"][0, 0])
    assert oracle.tc_eps(e) == eps == 0.5
    x = oracle.tc_rtilde_lu(e, eps)
    # the paper prints four truncated decimals
    assert np.array_equal(np.floor(x * 1e4 + 1e-9) / 1e4, g["Rtilde_printed"])
    # exact values: the cycle 1->2->3->1 gives eps^d / (1 - eps^3) = {4/7, 2/7, 1/7}
    exact = np.array([[1, 4, 2, 0], [2, 1, 4, 0], [4, 2, 1, 0], [4, 2, 1, 0]]) / 7.0
    assert np.max(np.abs(x - exact)) < 1e-15
    assert np.array_equal((x > 0).astype(np.uint8), g["R2"].astype(np.uint8))
    assert np.array_equal(dense_model(e), g["R2"].astype(np.uint8))


def test_worked_example_catches_transposed_operand():
    """A transposed E (a plausible slip) must break the worked-example pin."""
    g = read("worked_example_tc.txt")
    e = g["R1"].astype(np.uint8)
    x_wrong = oracle.tc_rtilde_lu(np.ascontiguousarray(e.T), 0.5)
    assert not np.array_equal(np.floor(x_wrong * 1e4 + 1e-9) / 1e4, g["Rtilde_printed"])
    assert not np.array_equal(dense_model(np.ascontiguousarray(e.T)), g["R2"].astype(np.uint8))


# --- least model vs brute force ---------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_all_digraphs_up_to_3(n):
    for bits in range(1 << (n * n)):
        e = np.array([(bits >> k) & 1 for k in range(n * n)], dtype=np.uint8).reshape(n, n)
        ref = brute.bfs_closure(e)
        assert np.array_equal(dense_model(e), ref), e
        if n:
            assert np.array_equal(oracle.tc_naive(e), ref)


def test_all_digraphs_4():
    """All 2^16 digraphs on four constants (self-loops included)."""
    n = 4
    for bits in range(1 << 16):
        e = np.unpackbits(np.array([bits & 0xFF, bits >> 8], dtype=np.uint8),
                          bitorder="little").reshape(n, n)
        got = dense_model(e)
        ref = brute.warshall(e)
        if not np.array_equal(got, ref):
            raise AssertionError(e)


@pytest.mark.parametrize("n,p,seed", [(5, 0.3, 1), (17, 0.1, 2), (33, 0.05, 3), (64, 0.02, 4),
                                      (65, 0.03, 5), (100, 0.01, 6), (130, 0.2, 7),
                                      (200, 0.005, 8)])
def test_random_vs_bfs_and_warshall(n, p, seed):
    for loops in (False, True):
        e = inputs.er_digraph(n, p, seed, self_loops=loops)
        got = dense_model(e)
        assert np.array_equal(got, brute.bfs_closure(e))
        assert np.array_equal(got, brute.warshall(e))


@pytest.mark.parametrize("n,p,seed", [(30, 0.05, 11), (60, 0.03, 12), (90, 0.1, 13)])
def test_iteration_method_matches_and_converges_within_n(n, p, seed):
    e = inputs.er_digraph(n, p, seed)
    r, it = oracle.tc_naive(e, return_iters=True)
    assert np.array_equal(r, dense_model(e))
    assert it <= n + 1  # the naive series is constant from step n on (Sec. 3)


def test_seminaive_steps_equal_longest_shortest_path():
    e = inputs.er_digraph(80, 0.03, 21)
    _, steps = oracle.tc_model(e, return_iters=True)
    d = brute.bfs_distances(e)
    assert steps == max(int(d.max()) - 1, 0)


def test_model_is_least_fixpoint():
    """M = min1(E + E M) and no bit of M can be dropped (leastness)."""
    e = inputs.er_digraph(48, 0.05, 31)
    m = dense_model(e).astype(np.int64)
    E = e.astype(np.int64)
    assert np.array_equal(np.minimum(E + E @ m, 1), m)
    ones = np.argwhere(m)
    rng = np.random.default_rng(0)
    for i, j in ones[rng.choice(len(ones), size=min(40, len(ones)), replace=False)]:
        m2 = m.copy()
        m2[i, j] = 0
        assert not np.array_equal(np.minimum(E + E @ m2, 1), m2)


# --- R~ closed forms (Proposition 1) ---------------------------------------------------

def test_rtilde_zero_graph():
    e = np.zeros((7, 7), dtype=np.uint8)
    assert oracle.tc_eps(e) == 1.0
    assert np.all(oracle.tc_rtilde_lu(e) == 0.0)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_rtilde_all_ones_is_all_ones(n):
    """E = ones (self-loops, p_e = 1): eps = 1/(n+1) and R~ = ones (Sherman-Morrison)."""
    e = np.ones((n, n), dtype=np.uint8)
    eps = oracle.tc_eps(e)
    assert eps == 1.0 / (n + 1)
    x = oracle.tc_rtilde_lu(e, eps)
    assert np.max(np.abs(x - 1.0)) < 1e-13


@pytest.mark.parametrize("n", [2, 3, 8, 31])
def test_rtilde_complete_digraph(n):
    """E = ones - I: eps = 1/n, R~_ii = (n-1)/(n+1), R~_ij = n/(n+1)."""
    e = (1 - np.eye(n)).astype(np.uint8)
    eps = oracle.tc_eps(e)
    assert eps == 1.0 / n
    x = oracle.tc_rtilde_lu(e, eps)
    want = np.full((n, n), n / (n + 1.0))
    np.fill_diagonal(want, (n - 1) / (n + 1.0))
    assert np.max(np.abs(x - want)) < 1e-13


@pytest.mark.parametrize("n", [2, 9, 40])
def test_rtilde_directed_path(n):
    """0 -> 1 -> ... -> n-1: eps = 1/2 and R~_ij = 2^-(j-i) for j > i, else 0."""
    e = np.zeros((n, n), dtype=np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    x = oracle.tc_rtilde_lu(e)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    want = np.where(j > i, 2.0 ** (-(j - i).astype(float)), 0.0)
    assert np.array_equal(x, want)  # powers of two: exact


@pytest.mark.parametrize("L", [1, 2, 3, 7, 20])
def test_rtilde_directed_cycle(L):
    """L-cycle: R~_ij = eps^d(i,j) / (1 - eps^L) with d in [1, L]."""
    e = np.zeros((L, L), dtype=np.uint8)
    e[np.arange(L), (np.arange(L) + 1) % L] = 1
    eps = oracle.tc_eps(e)
    x = oracle.tc_rtilde_lu(e, eps)
    i, j = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    d = (j - i) % L
    d[d == 0] = L
    want = eps ** d / (1 - eps ** L)
    assert np.max(np.abs(x - want)) < 1e-15


def test_rtilde_user_eps_below_default():
    """Any 0 < eps <= 1/(1+||E||) gives the same model (Theorem 1), different R~."""
    e = inputs.er_digraph(40, 0.08, 41)
    e0 = oracle.tc_eps(e)
    xa = oracle.tc_rtilde_lu(e, e0)
    xb = oracle.tc_rtilde_lu(e, e0 / 3)
    assert np.array_equal(xa > 0, xb > 0)
    assert np.array_equal((xa > 0).astype(np.uint8), dense_model(e))
    assert np.all(xb <= xa + 1e-15)  # smaller eps, smaller least solution


# --- Theorem 1, Lemma 1, Lemma 2 on random graphs --------------------------------------

@pytest.mark.parametrize("n,p,seed", [(20, 0.1, 51), (64, 0.03, 52), (150, 0.02, 53),
                                      (257, 0.004, 54)])
def test_threshold_gives_model_and_bounds(n, p, seed):
    e = inputs.er_digraph(n, p, seed)
    eps = oracle.tc_eps(e)
    x = oracle.tc_rtilde_lu(e, eps)
    ref = brute.bfs_closure(e)
    assert np.array_equal((x > 0).astype(np.uint8), ref)          # Theorem 1
    assert x.min() >= 0.0 and x.max() <= 1.0                      # Lemma 1
    d = brute.bfs_distances(e)
    reach = ref.astype(bool)
    lb = np.where(reach, eps ** d.astype(float), 0.0)
    assert np.all(x[reach] >= lb[reach] * (1 - 1e-12))           # Lemma 2 footnote
    a = np.eye(n) - eps * e
    assert np.max(np.abs(a @ x - eps * e)) < 1e-13              # solves eq. (linear)


def test_series_column_matches_lu():
    """Two independent FP64 routes to R~: Lemma-1 series (column) and LU (Prop. 1)."""
    e = inputs.er_digraph(120, 0.03, 61)
    eps = oracle.tc_eps(e)
    x = oracle.tc_rtilde_lu(e, eps)
    for j in (0, 7, 63, 64, 119):
        col, it = oracle.tc_rtilde_col(e, eps, j, return_iters=True)
        assert it > 0
        assert np.max(np.abs(col - x[:, j])) <= 1e-14 * max(1.0, np.abs(x).max())


def test_series_column_path_closed_form():
    n = 30
    e = np.zeros((n, n), dtype=np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    col = oracle.tc_rtilde_col(e, 0.5, n - 1)
    want = 2.0 ** (-(n - 1 - np.arange(n)).astype(float))
    want[-1] = 0.0
    assert np.array_equal(col, want)


def test_series_row_matches_lu_and_columns():
    """Row i of R~ by the row-wise series against LU (Prop. 1) and against the column series at
    the crossing entries; an asymmetric graph, so a transposed operand fails."""
    e = inputs.er_digraph(150, 0.03, 62)
    eps = oracle.tc_eps(e)
    x = oracle.tc_rtilde_lu(e, eps)
    assert not np.allclose(x, x.T)
    for i in (0, 9, 63, 64, 149):
        row, it = oracle.tc_rtilde_row(e, eps, i, return_iters=True)
        assert it > 0
        assert np.max(np.abs(row - x[i, :])) <= 1e-14 * max(1.0, np.abs(x).max())
        for j in (1, 77):
            assert abs(row[j] - oracle.tc_rtilde_col(e, eps, j)[i]) <= 1e-15


def test_series_row_closed_forms():
    # directed path 0 -> 1 -> ...: eps = 1/2 and R~[0][j] = 2^-j for j >= 1
    n = 30
    e = np.zeros((n, n), dtype=np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    row = oracle.tc_rtilde_row(e, 0.5, 0)
    want = 2.0 ** (-np.arange(n).astype(float))
    want[0] = 0.0
    assert np.array_equal(row, want)
    # directed L-cycle: R~[i][j] = eps^d(i,j) / (1 - eps^L), d in [1, L]
    L = 7
    c = np.zeros((L, L), dtype=np.uint8)
    c[np.arange(L), (np.arange(L) + 1) % L] = 1
    row = oracle.tc_rtilde_row(c, 0.5, 2)
    d = (np.arange(L) - 2) % L
    d[d == 0] = L
    assert np.max(np.abs(row - 0.5 ** d / (1 - 0.5 ** L))) <= 1e-15
    with pytest.raises(RuntimeError):
        oracle.tc_rtilde_row(np.ones((4, 4), dtype=np.uint8), 0.2, 0, max_iter=3)


def test_series_column_not_converged_reports():
    e = np.ones((4, 4), dtype=np.uint8)
    with pytest.raises(RuntimeError):
        oracle.tc_rtilde_col(e, oracle.tc_eps(e), 0, max_iter=3)


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.tc_model(np.zeros((3, 4), dtype=np.uint8))
    with pytest.raises(RuntimeError):
        oracle.tc_rtilde_lu(np.zeros((3, 3), dtype=np.uint8), -1.0)


def test_pack_roundtrip():
    rng = np.random.default_rng(5)
    for n in (1, 63, 64, 65, 130):
        d = (rng.random((n, n)) < 0.3).astype(np.uint8)
        assert np.array_equal(oracle.unpack(oracle.pack(d), n), d)
