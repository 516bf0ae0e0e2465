"""Pins of the CPU oracle for same-generation (no GPU).

The semi-naive least model of S = min1(B + P S P^T) (Sec. 7.2) is checked against naive
fixpoint iteration, against the real solution of the Kronecker (vectorised) linear system
of the two-sided class (Sec. 6.3, eq. veceq:two-sided:1) thresholded at 0 (Theorem 2),
and against closed forms on chains and complete trees.
"""
import numpy as np
import pytest

import oracle
from paper_1608_00139_gb300 import inputs
from tests import brute


def dense(p, b=None):
    return oracle.unpack(oracle.sg_model(p, b), p.shape[0])


def test_empty_and_zero():
    assert oracle.sg_model(np.zeros((0, 0), dtype=np.uint8)).shape == (0, 0)
    for n in (1, 5, 64, 65):
        assert np.array_equal(dense(np.zeros((n, n), dtype=np.uint8)), np.eye(n, dtype=np.uint8))


@pytest.mark.parametrize("n", [2, 10, 100])
def test_chain_is_identity(n):
    p = np.zeros((n, n), dtype=np.uint8)
    p[np.arange(1, n), np.arange(n - 1)] = 1  # parent(i) = i-1
    assert np.array_equal(dense(p), np.eye(n, dtype=np.uint8))


@pytest.mark.parametrize("b,depth", [(2, 5), (3, 4), (4, 3)])
def test_complete_tree_is_block_diagonal_by_depth(b, depth):
    sizes = [b ** d for d in range(depth + 1)]
    n = sum(sizes)
    level = np.concatenate([np.full(s, d) for d, s in enumerate(sizes)])
    p = np.zeros((n, n), dtype=np.uint8)
    for i in range(1, n):
        p[i, (i - 1) // b] = 1  # heap numbering: parent of i is (i-1)//b
    s = dense(p)
    assert np.array_equal(s, (level[:, None] == level[None, :]).astype(np.uint8))
    assert int(s.sum()) == sum(x * x for x in sizes)


@pytest.mark.parametrize("n,seed", [(8, 1), (30, 2), (64, 3), (65, 4), (200, 5)])
def test_forest_vs_naive(n, seed):
    p = inputs.forest_dag(n, seed, extra_prob=0.05)
    assert np.array_equal(dense(p), brute.sg_naive(p))


@pytest.mark.parametrize("n,pe,seed", [(6, 0.3, 1), (20, 0.1, 2), (40, 0.05, 3), (70, 0.03, 4)])
def test_general_digraph_vs_naive(n, pe, seed):
    p = inputs.er_digraph(n, pe, seed, self_loops=True)
    assert np.array_equal(dense(p), brute.sg_naive(p))


def test_general_base_relation_vs_naive():
    p = inputs.er_digraph(40, 0.05, 9)
    b = inputs.er_digraph(40, 0.02, 10, self_loops=True)
    assert np.array_equal(dense(p, b), brute.sg_naive(p, b))


@pytest.mark.parametrize("n,pe,seed", [(4, 0.3, 1), (7, 0.2, 2), (9, 0.15, 3), (12, 0.1, 4)])
def test_kronecker_real_solution_thresholded(n, pe, seed):
    """vec S~ = eps vec B + eps (P (x) P) vec S~ with eps = 1/(1+||P||^2) (Sec. 7.2).

    Solved densely (n^2 unknowns); Theorem 2: S~ > 0 is the least model, 0 <= S~ <= 1.
    """
    p = inputs.er_digraph(n, pe, seed, self_loops=True)
    eps = oracle.sg_eps(p)
    d = oracle.max_row_sum(p)
    assert eps == 1.0 / (1.0 + d * d)
    P = p.astype(np.float64)
    K = np.kron(P, P)  # column-major vec: vec(P S P^T) = (P (x) P) vec(S)
    rhs = eps * np.eye(n).reshape(-1, order="F")
    st = np.linalg.solve(np.eye(n * n) - eps * K, rhs).reshape(n, n, order="F")
    assert st.min() > -1e-12 and st.max() <= 1.0 + 1e-12
    model = (st > 1e-300).astype(np.uint8)
    assert np.array_equal(model, dense(p))


def test_symmetric_for_identity_base():
    p = inputs.forest_dag(300, 7, extra_prob=0.02)
    s = dense(p)
    assert np.array_equal(s, s.T)


def test_catches_transposed_parent_relation():
    """Using P^T instead of P (a plausible slip) changes the model on a forest."""
    p = inputs.forest_dag(60, 3)
    assert not np.array_equal(dense(p), dense(np.ascontiguousarray(p.T)))
