"""GPU parity of one equation of the tail recursive class, R~ = eps (A + B0 R~) (Sec. 6.1):
the model on every path against the oracle (semi-naive; sampled rows by breadth-first search
at N = 8192), R~ on the real paths against the oracle's FP64 solve, the closure as the case
A = B0 = E, and the underflow repair."""
import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu

ALL = ["auto", "bool_fp8", "fp64", "mixed"]


def rand01(n, p, seed):
    return (np.random.default_rng(seed).random((n, n)) < p).astype(np.uint8)


def rel_err(x, ref):
    return np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("path", ALL)
@pytest.mark.parametrize("n", [1, 63, 65, 257, 700])
def test_random_against_oracle(ctx, path, n):
    b0 = rand01(n, 3.0 / max(n, 1), 100 + n)
    a = rand01(n, 1.0 / max(n, 1), 200 + n)
    want = oracle.pack(oracle.tail_model(b0, a))
    if path in ("fp64", "mixed"):
        bits, st, x = ctx.tail_recursive(b0, a, path=path, rtilde=True)
        assert rel_err(x, oracle.tail_rtilde(b0, a, st["eps_used"])) <= 1e-10
        assert st["rows_rechecked"] == 0
    else:
        bits, st = ctx.tail_recursive(b0, a, path=path)
    assert np.array_equal(bits, want)
    assert st["eps_used"] == oracle.tail_eps(b0)
    assert st["model_ones"] == int(oracle.unpack(want, n).sum())


@pytest.mark.parametrize("path", ALL)
def test_closure_is_the_case_a_equals_b0(ctx, path):
    e = inputs.er_digraph(600, 0.004, 7)
    got, _ = ctx.tail_recursive(e, e, path=path)
    want, _ = ctx.tc_closure(e, path=path)
    assert np.array_equal(got, want)
    assert np.array_equal(got, oracle.tc_model(e))


def test_degenerate_right_hand_sides(ctx):
    n = 300
    b0 = rand01(n, 0.01, 5)
    zero = np.zeros((n, n), dtype=np.uint8)
    bits, st = ctx.tail_recursive(b0, zero)
    assert not bits.any() and st["model_ones"] == 0
    a = rand01(n, 0.02, 6)
    bits, st, x = ctx.tail_recursive(zero, a, path="fp64", rtilde=True)
    assert np.array_equal(bits, oracle.pack(a))
    assert st["eps_used"] == 1.0
    assert np.array_equal(x, a.astype(np.float64))


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_underflow_is_repaired(ctx, path):
    """B0: i -> i + 1, A: one fact (n-1, c): R~[i][c] = 2^-(n-i) underflows for n - i > 1074
    (FP64) or about 150 (the mixed path's FP32 solve); the model keeps every fact."""
    n, c = 1200, 3
    b0 = np.zeros((n, n), dtype=np.uint8)
    b0[np.arange(n - 1), np.arange(1, n)] = 1
    a = np.zeros((n, n), dtype=np.uint8)
    a[n - 1, c] = 1
    bits, st, x = ctx.tail_recursive(b0, a, path=path, rtilde=True)
    m = oracle.unpack(bits, n)
    assert m[:, c].all() and m.sum() == n
    assert st["rows_rechecked"] == n - int((x[:, c] > 0).sum()) > 0
    if path == "fp64":
        want = np.ldexp(1.0, -(n - np.arange(n)))
        assert np.abs(x[:, c] - want).max() <= 1e-300 + 1e-15 * want.max()


def test_device_memory_and_arguments(ctx):
    n = 400
    b0 = rand01(n, 0.008, 9)
    a = rand01(n, 0.003, 10)
    bits, st, x = ctx.tail_recursive(torch.from_numpy(b0).cuda(), torch.from_numpy(a).cuda(), path="mixed",
                                     rtilde=True)
    assert bits.is_cuda and x.is_cuda
    assert np.array_equal(bits.cpu().numpy().view(np.uint64), oracle.pack(oracle.tail_model(b0, a)))
    assert rel_err(x.cpu().numpy(), oracle.tail_rtilde(b0, a)) <= 1e-10
    with pytest.raises(dl.DLError) as ei:
        ctx.tail_recursive(b0, a, path="auto", rtilde=True)
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        ctx.tail_recursive(b0, a, eps=2 * oracle.tail_eps(b0))
    assert ei.value.status == dl.DL_EINVAL
    bad = a.copy()
    bad[1, 2] = 5
    with pytest.raises(dl.DLError) as ei:
        ctx.tail_recursive(b0, bad)
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(ValueError):
        ctx.tail_recursive(b0, a[:10, :10])


def test_er_8192_sampled_rows(ctx):
    n = 8192
    b0 = inputs.er_digraph(n, 1e-3, 3)
    a = inputs.er_digraph(n, 1e-4, 2)
    bits, st = ctx.tail_recursive(b0, a)
    rows = [0, 1, 977, 4096, 8000, n - 1]
    got = oracle.unpack(bits, n)[rows]
    assert np.array_equal(got, oracle.tail_model_rows(b0, a, rows))
