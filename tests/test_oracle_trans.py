"""Pins of the transposed-class oracle (oracle/transposed.py, Sec. 6.2, program prog:2).

The semi-naive model is checked against hand-derived small cases, against the paper's naive
series on every digraph of up to three constants and random larger ones, and against the
same-generation oracle through the paper's reduction to a two-sided equation (eq.
matrixeq:trans:2: R2 = min1(R1 + R1 R1^T + R1 R2 R1^T)).  The real R~2 is checked against exact
rationals, the Kronecker solve of the vectorised equation, the equation's residual and the
bounds of Lemma 4's kind (0 <= R~ <= 1), and its positive entries against the model."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import transposed as tr
from paper_1608_00139_gb300 import inputs
from tests.golden.load import read


def unpack(bits, n):
    return np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :n]


@pytest.mark.parametrize("case", ["edge", "cycle2", "chain3", "instar3"])
def test_hand_derived_models(case):
    g = read("transposed_small.txt")
    r1 = g[f"{case}_R1"].astype(np.uint8)
    want = g[f"{case}_R2"].astype(np.uint8)
    assert np.array_equal(tr.trans_model(r1), want)
    assert np.array_equal(tr.trans_naive(r1), want)


@pytest.mark.parametrize("case", ["edge", "cycle2"])
def test_hand_derived_rtilde(case):
    g = read("transposed_small.txt")
    r1 = g[f"{case}_R1"].astype(np.uint8)
    want = g[f"{case}_Rtilde"]
    assert np.allclose(tr.trans_rtilde_kron(r1), want, rtol=0, atol=1e-15)
    assert np.allclose(tr.trans_rtilde_series(r1, tol=0.0), want, rtol=0, atol=1e-15)


def test_the_interchanged_arguments_matter():
    """The closure program (r2(y,z) in the body instead of r2(z,y)) gives another model on the
    chain, so an oracle that dropped the transpose fails the fixtures."""
    g = read("transposed_small.txt")
    r1 = g["chain3_R1"].astype(np.uint8)
    tc = unpack(oracle.tc_model(r1), 3)
    assert not np.array_equal(tc, tr.trans_model(r1))
    wrong = np.minimum(r1.astype(int) + r1.astype(int) @ tr.trans_model(r1).astype(int), 1)  # R1 R2, no ^T
    assert not np.array_equal(wrong.astype(np.uint8), g["chain3_R2"].astype(np.uint8))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_every_small_digraph_agrees_with_the_naive_series(n):
    for bits in itertools.product([0, 1], repeat=n * n):
        r1 = np.array(bits, dtype=np.uint8).reshape(n, n)
        assert np.array_equal(tr.trans_model(r1), tr.trans_naive(r1)), r1


def test_random_graphs_agree_with_the_naive_series():
    rng = np.random.default_rng(3)
    for _ in range(60):
        n = int(rng.integers(4, 24))
        r1 = (rng.random((n, n)) < rng.choice([0.05, 0.15, 0.3])).astype(np.uint8)
        assert np.array_equal(tr.trans_model(r1), tr.trans_naive(r1))


@pytest.mark.parametrize("n,p,seed", [(40, 0.05, 1), (97, 0.02, 2), (160, 0.01, 3), (300, 0.004, 4)])
def test_model_is_the_two_sided_reduction(n, p, seed):
    """eq. matrixeq:trans:2: the model is the least S with S = min1(B + R1 S R1^T),
    B = min1(R1 + R1 R1^T) -- the same-generation oracle with P = R1 and that B."""
    r1 = inputs.er_digraph(n, p, seed)
    b = np.minimum(r1.astype(np.int64) + r1.astype(np.int64) @ r1.T.astype(np.int64), 1).astype(np.uint8)
    s = unpack(oracle.sg_model(r1, b), n)
    assert np.array_equal(tr.trans_model(r1), s)


def test_model_on_a_forest_is_the_two_sided_reduction():
    r1 = inputs.forest_dag(300, 7)
    b = np.minimum(r1.astype(np.int64) + r1.astype(np.int64) @ r1.T.astype(np.int64), 1).astype(np.uint8)
    assert np.array_equal(tr.trans_model(r1), unpack(oracle.sg_model(r1, b), 300))


def test_kronecker_solve_thresholds_to_the_model():
    rng = np.random.default_rng(11)
    for _ in range(40):
        n = int(rng.integers(1, 9))
        r1 = (rng.random((n, n)) < 0.3).astype(np.uint8)
        x = tr.trans_rtilde_kron(r1)
        assert np.array_equal((x > 1e-14).astype(np.uint8), tr.trans_model(r1))
        assert x.min() >= -1e-15 and x.max() <= 1 + 1e-12
        e = r1.astype(np.float64)
        assert np.abs(tr.trans_eps(r1) * (e + e @ x.T) - x).max() <= 1e-14


def test_series_matches_the_kronecker_solve():
    rng = np.random.default_rng(12)
    for _ in range(20):
        n = int(rng.integers(2, 12))
        r1 = (rng.random((n, n)) < 0.25).astype(np.uint8)
        assert np.abs(tr.trans_rtilde_series(r1, tol=1e-17) - tr.trans_rtilde_kron(r1)).max() <= 1e-13


def test_series_solves_the_equation_at_moderate_size():
    r1 = inputs.er_digraph(400, 0.01, 5)
    eps = tr.trans_eps(r1)
    x, steps = tr.trans_rtilde_series(r1, eps, tol=1e-17, return_steps=True)
    e = r1.astype(np.float64)
    assert np.abs(eps * (e + e @ x.T) - x).max() <= 1e-15
    assert np.array_equal((x > 0).astype(np.uint8), tr.trans_model(r1))
    assert 0.0 <= x.min() and x.max() <= 1.0
