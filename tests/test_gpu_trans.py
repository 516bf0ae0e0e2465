"""The transposed class (dl_transposed, Sec. 6.2, program prog:2) on the GPU against the oracle.

Bits must equal the oracle's semi-naive model exactly on every path; R~2 (FP64 series) must be
within 1e-10 (max-abs error / max-abs value) of the oracle's series or Kronecker solve.  Sizes
cover the tile edges, degenerate graphs, the hand-derived cases and N = 4096."""
import numpy as np
import pytest
import torch

from oracle import transposed as tr
from paper_1608_00139_gb300 import dl, inputs
from tests.golden.load import read

pytestmark = pytest.mark.gpu


def unpack(bits, n):
    b = bits.cpu().numpy() if isinstance(bits, torch.Tensor) else bits
    return np.unpackbits(b.view(np.uint8), axis=1, bitorder="little")[:, :n]


def rel_err(x, ref):
    x = x.cpu().numpy() if isinstance(x, torch.Tensor) else x
    scale = max(float(np.abs(ref).max()), 1e-300)
    return float(np.abs(x - ref).max()) / scale


@pytest.mark.parametrize("case", ["edge", "cycle2", "chain3", "instar3"])
def test_hand_derived_cases(ctx, case):
    g = read("transposed_small.txt")
    r1 = g[f"{case}_R1"].astype(np.uint8)
    want = g[f"{case}_R2"].astype(np.uint8)
    for path in ("auto", "bool_fp8"):
        bits, _ = ctx.transposed(r1, path=path)
        assert np.array_equal(unpack(bits, r1.shape[0]), want), path
    bits, st, x = ctx.transposed(r1, path="fp64", rtilde=True)
    assert np.array_equal(unpack(bits, r1.shape[0]), want)
    if f"{case}_Rtilde" in g:
        assert np.abs(x - g[f"{case}_Rtilde"]).max() <= 1e-12  # the series stops at a change <= 1e-13 eps
    assert st["guard_flagged"] == 0


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 513])
def test_tile_edges(ctx, n):
    r1 = inputs.er_digraph(n, min(0.5, 3.0 / max(n, 1)), 100 + n)
    want = tr.trans_model(r1)
    for path in ("auto", "bool_fp8"):
        bits, _ = ctx.transposed(r1, path=path)
        assert np.array_equal(unpack(bits, n), want), (n, path)
    bits, st, x = ctx.transposed(r1, path="fp64", rtilde=True)
    assert np.array_equal(unpack(bits, n), want)
    ref = tr.trans_rtilde_kron(r1) if n <= 20 else tr.trans_rtilde_series(r1, tol=1e-18)
    assert rel_err(x, ref) <= 1e-10
    assert st["guard_flagged"] == 0
    assert abs(st["eps_used"] - tr.trans_eps(r1)) == 0.0


def degenerate(n):
    out = {"empty": np.zeros((n, n), np.uint8), "ones": np.ones((n, n), np.uint8),
           "complete": (1 - np.eye(n)).astype(np.uint8)}
    chain = np.zeros((n, n), np.uint8)
    chain[np.arange(n - 1), np.arange(1, n)] = 1
    out["chain"] = chain
    cyc = chain.copy()
    cyc[n - 1, 0] = 1
    out["cycle"] = cyc
    star = np.zeros((n, n), np.uint8)
    star[0, 1:] = 1
    out["star"] = star
    out["instar"] = star.T.copy()
    out["loops"] = np.eye(n, dtype=np.uint8)
    return out


@pytest.mark.parametrize("name", ["empty", "ones", "complete", "chain", "cycle", "star", "instar", "loops"])
def test_degenerate_graphs(ctx, name):
    n = 97
    r1 = degenerate(n)[name]
    want = tr.trans_model(r1)
    bits, _ = ctx.transposed(r1, path="auto")
    assert np.array_equal(unpack(bits, n), want)
    if name in ("ones", "complete"):
        return  # eps = 1/n: the series needs about 30 n steps (checked at small n below)
    bits, st, x = ctx.transposed(r1, path="fp64", rtilde=True)
    assert np.array_equal(unpack(bits, n), want)
    assert rel_err(x, tr.trans_rtilde_series(r1, tol=1e-18)) <= 1e-10 if want.any() else np.abs(x).max() == 0


def test_dense_graph_series_converges(ctx):
    r1 = (1 - np.eye(24)).astype(np.uint8)
    bits, st, x = ctx.transposed(r1, path="fp64", rtilde=True)
    assert np.array_equal(unpack(bits, 24), tr.trans_model(r1))
    assert rel_err(x, tr.trans_rtilde_kron(r1)) <= 1e-10


def test_device_inputs_and_outputs(ctx):
    r1 = inputs.er_digraph(300, 0.01, 41)
    dev = torch.from_numpy(r1).cuda()
    bits, st, x = ctx.transposed(dev, path="fp64", rtilde=True)
    assert bits.is_cuda and x.is_cuda
    assert np.array_equal(unpack(bits, 300), tr.trans_model(r1))
    assert rel_err(x, tr.trans_rtilde_series(r1, tol=1e-18)) <= 1e-10


def test_errors(ctx):
    r1 = inputs.er_digraph(64, 0.05, 42)
    eps = tr.trans_eps(r1)
    with pytest.raises(dl.DLError) as e:
        ctx.transposed(r1, eps=1.01 * eps, path="fp64", rtilde=True)
    assert e.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as e:
        ctx.transposed(r1, path="mixed")
    assert e.value.status == dl.DL_ENOTIMPL
    with pytest.raises(dl.DLError) as e:
        ctx.transposed(r1, path="bool_fp8", rtilde=True)
    assert e.value.status == dl.DL_EINVAL
    bad = r1.copy()
    bad[3, 4] = 2
    with pytest.raises(dl.DLError) as e:
        ctx.transposed(bad)
    assert e.value.status == dl.DL_EINVAL
    # a smaller eps than the default is allowed and gives the same model
    bits, st = ctx.transposed(r1, eps=0.5 * eps)
    assert np.array_equal(unpack(bits, 64), tr.trans_model(r1))
    assert st["eps_used"] == 0.5 * eps


@pytest.mark.parametrize("kind", ["er", "forest"])
def test_n4096(ctx, kind):
    r1 = inputs.er_digraph(4096, 1e-3, 8) if kind == "er" else inputs.forest_dag(4096, 5)
    dev = torch.from_numpy(r1).cuda()
    bits, st, x = ctx.transposed(dev, path="auto", rtilde=True)
    want = tr.trans_model(r1)
    assert np.array_equal(unpack(bits, 4096), want)
    ref = tr.trans_rtilde_series(r1, tol=1e-15 * tr.trans_eps(r1))
    assert rel_err(x, ref) <= 1e-10
    assert st["guard_flagged"] == 0
