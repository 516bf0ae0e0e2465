"""GPU parity of the closure with a bit-packed E (the output's layout, an eighth of the bytes):
every path against the oracle's bits, host and device memory, ragged rows, heavy rows, and
the padding-bit error."""
import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 63, 64, 65, 127, 129, 257, 1000, 3000]


def graph(n, seed, deg=2.0):
    rng = np.random.default_rng(seed)
    e = (rng.random((n, n)) < min(1.0, deg / max(n, 1))).astype(np.uint8)
    # a long chain through a random order, so that the closure needs many steps
    order = rng.permutation(n)
    for a, b in zip(order[: n // 2], order[1: n // 2 + 1]):
        e[a, b] = 1
    return e


@pytest.mark.parametrize("path", ["auto", "bool_fp8"])
@pytest.mark.parametrize("n", SIZES)
def test_bits_input_matches_oracle(ctx, n, path):
    e = graph(n, 100 + n)
    want = oracle.tc_model(e)
    got, st = ctx.tc_closure_bits(oracle.pack(e), n, path=path)
    assert np.array_equal(got, want)
    assert st["eps_used"] == oracle.tc_eps(e)


@pytest.mark.parametrize("n", [65, 300])
@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_bits_input_real_paths_match_the_byte_input(ctx, n, path):
    e = graph(n, 7 + n, deg=3.0)
    want = oracle.tc_model(e)
    gb, sb, xb = ctx.tc_closure_bits(oracle.pack(e), n, path=path, rtilde=True)
    g8, s8, x8 = ctx.tc_closure(e, path=path, rtilde=True)
    assert np.array_equal(gb, want) and np.array_equal(g8, want)
    # same bytes reach the same path: the same R~ to the last bit
    assert np.array_equal(xb, x8)
    assert sb["eps_used"] == s8["eps_used"]


@pytest.mark.parametrize("path", ["auto", "bool_fp8", "fp64"])
def test_bits_input_device_memory(ctx, path):
    n = 190 if path == "fp64" else 2100
    e = graph(n, 11, deg=1.5)
    want = oracle.tc_model(e)
    eb = torch.from_numpy(oracle.pack(e).view(np.int64)).cuda()
    got, _ = ctx.tc_closure_bits(eb, n, path=path)
    assert got.is_cuda
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want)


def test_bits_input_heavy_rows_and_self_loops(ctx):
    # a row above 256 successors takes AUTO off its speculative start; self-loops count as facts
    n = 2000
    e = graph(n, 5, deg=1.0)
    e[17, :] = 1
    e[np.arange(0, n, 7), np.arange(0, n, 7)] = 1
    want = oracle.tc_model(e)
    for path in ("auto", "bool_fp8"):
        got, st = ctx.tc_closure_bits(oracle.pack(e), n, path=path)
        assert np.array_equal(got, want), path
        assert st["eps_used"] == 1.0 / (1.0 + n)


def test_bits_input_er_8192_matches_byte_input(ctx):
    n = 8192
    for p, seed in ((1e-4, 2), (1e-3, 3), (1e-2, 4)):
        e = inputs.er_digraph(n, p, seed)
        want = oracle.tc_model(e)
        got, _ = ctx.tc_closure_bits(oracle.pack(e), n)
        assert np.array_equal(got, want), p


@pytest.mark.parametrize("path", ["auto", "bool_fp8", "fp64", "mixed"])
@pytest.mark.parametrize("n", [65, 100])
def test_bits_input_padding_bit_is_rejected(ctx, n, path):
    e = graph(n, 3)
    eb = oracle.pack(e)
    eb[n // 2, -1] |= np.uint64(1) << np.uint64(63)  # column 127 >= n
    with pytest.raises(dl.DLError) as ei:
        ctx.tc_closure_bits(eb, n, path=path)
    assert ei.value.status == dl.DL_EINVAL
    assert "column" in str(ei.value)
    # the context stays usable
    got, _ = ctx.tc_closure_bits(oracle.pack(e), n, path=path)
    assert np.array_equal(got, oracle.tc_model(e))


def test_bits_input_shape_is_checked(ctx):
    with pytest.raises(ValueError):
        ctx.tc_closure_bits(np.zeros((10, 2), dtype=np.uint64), 10)
    bits, _ = ctx.tc_closure_bits(np.zeros((0, 0), dtype=np.uint64), 0)
    assert bits.shape == (0, 0)
