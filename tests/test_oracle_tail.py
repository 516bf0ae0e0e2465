"""Pins for the oracle's tail recursive class R~ = eps (A + B0 R~) (Sec. 6.1): the closure case
A = B0 = E against the C oracle's semi-naive model and LU, B0 = 0, a chain in closed form,
brute-force reachability on small graphs, and the equation's residual."""
import numpy as np
import pytest

import oracle


def rand01(n, p, seed):
    return (np.random.default_rng(seed).random((n, n)) < p).astype(np.uint8)


@pytest.mark.parametrize("n,p,seed", [(40, 0.05, 1), (150, 0.02, 2), (300, 0.005, 3)])
def test_closure_is_the_case_a_equals_b0(n, p, seed):
    e = rand01(n, p, seed)
    assert np.array_equal(oracle.tail_model(e, e), oracle.unpack(oracle.tc_model(e), n))
    assert oracle.tail_eps(e) == oracle.tc_eps(e)
    x = oracle.tail_rtilde(e, e)
    xr = oracle.tc_rtilde_lu(e)
    assert np.abs(x - xr).max() <= 1e-13 * max(1.0, np.abs(xr).max())


def test_zero_b0():
    a = rand01(30, 0.2, 4)
    z = np.zeros((30, 30), dtype=np.uint8)
    assert np.array_equal(oracle.tail_model(z, a), a)
    assert oracle.tail_eps(z) == 1.0
    assert np.array_equal(oracle.tail_rtilde(z, a), a.astype(np.float64))


def test_chain_closed_form():
    """B0: i -> i + 1 (eps = 1/2); A: one fact (n-1, c).  R~[i][c] = 2^-(n-i), the rest 0."""
    n, c = 60, 7
    b0 = np.zeros((n, n), dtype=np.uint8)
    b0[np.arange(n - 1), np.arange(1, n)] = 1
    a = np.zeros((n, n), dtype=np.uint8)
    a[n - 1, c] = 1
    want = np.zeros((n, n))
    want[:, c] = 2.0 ** -(n - np.arange(n, dtype=np.float64))
    assert np.abs(oracle.tail_rtilde(b0, a) - want).max() <= 1e-16
    m = oracle.tail_model(b0, a)
    assert m[:, c].all() and m.sum() == n


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_reachability(seed):
    """R[x][z] = 1 iff some y with x ->* y in B0 (zero or more steps) has A[y][z] = 1."""
    n = 12 + seed
    b0 = rand01(n, 0.15, 10 + seed)
    a = rand01(n, 0.1, 20 + seed)
    reach = np.eye(n, dtype=bool)
    for _ in range(n):
        reach = reach | ((reach.astype(int) @ b0.astype(int)) > 0)
    want = ((reach.astype(int) @ a.astype(int)) > 0).astype(np.uint8)
    assert np.array_equal(oracle.tail_model(b0, a), want)
    x = oracle.tail_rtilde(b0, a)
    assert np.array_equal((x > 0).astype(np.uint8), want)


def test_rtilde_solves_the_equation():
    n = 200
    b0 = rand01(n, 0.02, 31)
    a = rand01(n, 0.01, 32)
    eps = oracle.tail_eps(b0)
    x = oracle.tail_rtilde(b0, a, eps)
    r = x - eps * (a + b0.astype(np.float64) @ x)
    assert np.abs(r).max() <= 1e-15 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("seed", range(3))
def test_sampled_rows_match_the_whole_model(seed):
    n = 300
    b0 = rand01(n, 0.006, 40 + seed)
    a = rand01(n, 0.004, 50 + seed)
    m = oracle.tail_model(b0, a)
    rows = [0, 17, 150, n - 1]
    assert np.array_equal(oracle.tail_model_rows(b0, a, rows), m[rows])


def test_brute_force_catches_transposed_or_right_multiplied_b0():
    """B0^T (predecessors) or R B0 in place of B0 R (plausible slips) must fail the pin."""
    n = 14
    b0 = rand01(n, 0.15, 70)
    a = rand01(n, 0.1, 71)
    reach = np.eye(n, dtype=bool)
    for _ in range(n):
        reach = reach | ((reach.astype(int) @ b0.astype(int)) > 0)
    want = ((reach.astype(int) @ a.astype(int)) > 0).astype(np.uint8)
    assert not np.array_equal(oracle.tail_model(np.ascontiguousarray(b0.T), a), want)
    # R = A u R B0, the least solution computed by the same fixpoint with the product flipped
    r = a.astype(bool)
    while True:
        nxt = r | ((r.astype(int) @ b0.astype(int)) > 0)
        if np.array_equal(nxt, r):
            break
        r = nxt
    assert not np.array_equal(r.astype(np.uint8), want)
