"""Pins for the oracle's real same-generation solution S~ = eps (B + P S~ P^T) (Sec. 7.2, the
two-sided class of Sec. 6.3): the Kronecker solve and the fixpoint series against each other,
closed forms on chains, trees and P = 0, the least model, and the equation's residual."""
import numpy as np
import pytest

import oracle


def random_p(n, density, seed, dag=False):
    rng = np.random.default_rng(seed)
    p = (rng.random((n, n)) < density).astype(np.uint8)
    if dag:
        p = np.tril(p, -1)
    return p


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("with_b", [False, True])
def test_kron_and_series_agree(seed, with_b):
    n = 3 + seed
    p = random_p(n, 0.3, seed)  # cycles allowed: the series converges geometrically
    b = random_p(n, 0.3, 100 + seed) if with_b else None
    xk = oracle.sg_stilde_kron(p, b)
    xs = oracle.sg_stilde_series(p, b)
    assert np.abs(xk - xs).max() <= 1e-14 * max(1.0, np.abs(xk).max())


def test_zero_p_gives_eps_b():
    b = random_p(9, 0.4, 1)
    for x in (oracle.sg_stilde_kron(np.zeros((9, 9)), b), oracle.sg_stilde_series(np.zeros((9, 9)), b)):
        assert np.array_equal(x, b.astype(np.float64))  # eps = 1/(1 + 0)


@pytest.mark.parametrize("n", [12, 90])
def test_chain_closed_form(n):
    """Node i's parent is i - 1 (||P|| = 1, eps = 1/2): S~_ii = sum_{m <= i} 2^-(m+1) = 1 - 2^-(i+1)."""
    p = np.zeros((n, n), dtype=np.uint8)
    p[np.arange(1, n), np.arange(n - 1)] = 1
    want = np.diag(1.0 - 0.5 ** (np.arange(n) + 1.0))
    xs = oracle.sg_stilde_series(p)
    assert np.abs(xs - want).max() <= 1e-15
    if n <= 40:
        assert np.abs(oracle.sg_stilde_kron(p) - want).max() <= 1e-14


@pytest.mark.parametrize("depth", [3, 6])
def test_complete_binary_tree_closed_form(depth):
    """P[child][parent] = 1 on a complete binary tree (eps = 1/2).  Nodes x, y at one depth d
    whose lowest common ancestor is h levels up: S~_xy = sum_{m=h..d} 2^-(m+1) = 2^-h (1 - 2^-(d-h+1));
    nodes at different depths: 0."""
    n = 2 ** (depth + 1) - 1
    p = np.zeros((n, n), dtype=np.uint8)
    for c in range(1, n):
        p[c, (c - 1) // 2] = 1
    level = np.floor(np.log2(np.arange(n) + 1)).astype(int)
    want = np.zeros((n, n))
    for x in range(n):
        for y in range(n):
            if level[x] != level[y]:
                continue
            a, b, h = x, y, 0
            while a != b:
                a, b, h = (a - 1) // 2, (b - 1) // 2, h + 1
            d = level[x]
            want[x, y] = 2.0 ** -h * (1.0 - 2.0 ** -(d - h + 1))
    assert np.abs(oracle.sg_stilde_series(p) - want).max() <= 1e-15
    if n <= 40:
        assert np.abs(oracle.sg_stilde_kron(p) - want).max() <= 1e-14


@pytest.mark.parametrize("seed,dag,with_b", [(1, True, False), (2, False, False), (3, True, True), (4, False, True)])
def test_positive_entries_are_the_least_model(seed, dag, with_b):
    n = 120
    p = random_p(n, 0.02, seed, dag)
    b = random_p(n, 0.01, 50 + seed) if with_b else None
    x = oracle.sg_stilde_series(p, b)
    m = oracle.unpack(oracle.sg_model(p, b), n)
    assert np.array_equal((x > 0).astype(np.uint8), m)


def test_series_solves_the_equation():
    n = 200
    p = random_p(n, 0.015, 9)
    eps = oracle.sg_eps(p)
    x = oracle.sg_stilde_series(p)
    r = x - eps * (np.eye(n) + p.astype(float) @ x @ p.T.astype(float))
    assert np.abs(r).max() <= 1e-15 * max(1.0, np.abs(x).max())
    assert eps == 1.0 / (1.0 + p.sum(axis=1).max() ** 2)


def test_user_eps_below_the_default():
    p = random_p(8, 0.3, 5)
    e = oracle.sg_eps(p) / 3
    xk = oracle.sg_stilde_kron(p, None, e)
    xs = oracle.sg_stilde_series(p, None, e)
    assert np.abs(xk - xs).max() <= 1e-15


def _tree(depth):
    n = 2 ** (depth + 1) - 1
    p = np.zeros((n, n), dtype=np.uint8)
    for c in range(1, n):
        p[c, (c - 1) // 2] = 1
    return p


def test_tree_pin_catches_a_transposed_sandwich():
    """P^T X P in place of P X P^T (a plausible slip) must break the tree's closed form."""
    p = _tree(3)
    right = oracle.sg_stilde_series(p)
    wrong = oracle.sg_stilde_series(np.ascontiguousarray(p.T))
    assert np.abs(right - wrong).max() > 0.1


def test_tree_pin_catches_the_wrong_kronecker_order():
    """(P kron P^T) in place of (P kron P) for vec(P X P^T) must disagree with the series."""
    p = _tree(3).astype(np.float64)
    n = p.shape[0]
    eps = oracle.sg_eps(p)
    wrong = np.linalg.solve(np.eye(n * n) - eps * np.kron(p, p.T), eps * np.eye(n).reshape(-1)).reshape(n, n)
    assert np.abs(wrong - oracle.sg_stilde_kron(p)).max() > 0.1
