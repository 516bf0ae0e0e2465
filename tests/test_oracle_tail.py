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


# ---- real lower solutions and layered systems ------------------------------------------------

from oracle import program as pg  # noqa: E402
from oracle import tail as tl  # noqa: E402


def path(n):
    e = np.zeros((n, n), np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    return e


def test_two_equation_chain_in_closed_form():
    """eq 0: the closure of a directed path (eps = 1/2, R~_ij = 2^-(j-i) for j > i);
    eq 1: R~1 = eps1 (I R~0), eps1 = 1/(1 + 0 + 1) = 1/2, so R~1_ij = 2^-(j-i+1)."""
    n = 9
    e = path(n)
    eqs = [{"A1": e, "B0": e}, {"terms": [(np.eye(n, dtype=np.uint8), 0)]}]
    models, xs, epss = tl.tail_system(eqs, n)
    i, j = np.indices((n, n))
    want0 = np.where(j > i, 2.0 ** -(j - i).clip(0), 0.0)
    assert epss == [0.5, 0.5]
    assert np.abs(xs[0] - want0).max() <= 1e-15
    assert np.abs(xs[1] - want0 / 2).max() <= 1e-15
    assert np.array_equal(models[0], (j > i).astype(np.uint8))
    assert np.array_equal(models[1], models[0])


def random_system(rng, n, m):
    eqs = []
    for h in range(m):
        eq = {"A1": (rng.random((n, n)) < 0.05).astype(np.uint8) if rng.random() < 0.8 else None,
              "B0": (rng.random((n, n)) < 0.08).astype(np.uint8) if rng.random() < 0.7 else None,
              "terms": [((rng.random((n, n)) < 0.06).astype(np.uint8), int(rng.integers(0, h)))
                        for _ in range(int(rng.integers(0, 3)) if h else 0)]}
        eqs.append(eq)
    return eqs


def test_in_order_solution_is_the_stacked_solve():
    rng = np.random.default_rng(21)
    for _ in range(25):
        n, m = int(rng.integers(2, 14)), int(rng.integers(1, 5))
        eqs = random_system(rng, n, m)
        models, xs, epss = tl.tail_system(eqs, n)
        stacked = tl.tail_system_stacked(eqs, n, epss)
        for h in range(m):
            assert np.abs(xs[h] - stacked[h]).max() <= 1e-13
            assert np.array_equal((xs[h] > 0).astype(np.uint8), models[h])
            assert xs[h].min() >= -1e-15 and xs[h].max() <= 1 + 1e-12  # Theorem 2's bound


def test_system_models_are_the_program_models():
    """The layered system of equations is the completion of the program
    r_h(X,Z) :- a_h(X,Z).  r_h(X,Z) :- c_h(X,Y), r_h(Y,Z).  r_h(X,Z) :- b_hq(X,Y), r_j(Y,Z)."""
    rng = np.random.default_rng(22)
    for _ in range(15):
        n, m = int(rng.integers(2, 10)), int(rng.integers(1, 4))
        eqs = random_system(rng, n, m)
        models, _, _ = tl.tail_system(eqs, n)
        lines, edb = [], {}
        for h, eq in enumerate(eqs):
            if eq["A1"] is not None:
                edb[f"a{h}"] = pg.to_pairs(eq["A1"])
                lines.append(f"r{h}(X,Z) :- a{h}(X,Z).")
            if eq["B0"] is not None:
                edb[f"c{h}"] = pg.to_pairs(eq["B0"])
                lines.append(f"r{h}(X,Z) :- c{h}(X,Y), r{h}(Y,Z).")
            for q, (b, j) in enumerate(eq["terms"]):
                edb[f"b{h}_{q}"] = pg.to_pairs(b)
                lines.append(f"r{h}(X,Z) :- b{h}_{q}(X,Y), r{j}(Y,Z).")
        if not lines:
            continue
        got = pg.least_model(pg.parse(" ".join(lines)), edb, n)
        for h in range(m):
            assert np.array_equal(pg.to_matrix(got.get(f"r{h}", set()), n), models[h])


def test_a_dropped_term_or_reordered_product_breaks_the_stacked_pin():
    rng = np.random.default_rng(23)
    n = 8
    eqs = [{"A1": (rng.random((n, n)) < 0.2).astype(np.uint8), "B0": path(n)},
           {"A1": None, "B0": path(n).T.copy(), "terms": [((rng.random((n, n)) < 0.3).astype(np.uint8), 0)]}]
    _, xs, epss = tl.tail_system(eqs, n)
    stacked = tl.tail_system_stacked(eqs, n, epss)
    b, _ = eqs[1]["terms"][0]
    wrong = tl.tail_rtilde_real(eqs[1]["B0"], None, [(b.T.copy(), xs[0])], epss[1])  # B^T R~ instead of B R~
    assert np.abs(wrong - stacked[1]).max() > 1e-6
    dropped = tl.tail_rtilde_real(eqs[1]["B0"], None, [], epss[1])
    assert np.abs(dropped - stacked[1]).max() > 1e-6
