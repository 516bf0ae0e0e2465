"""GPU parity on the benchmark's workloads at full size, bit-exact against the oracle.

Config sizes: closure on ER N=256 p=0.02 (FP64 path, R~ to 1e-10), closure on ER N=8192 with
p in {1e-4, 1e-3, 1e-2} (FP8 path: every bit; FP64 path: every bit plus sampled columns of R~
against the Lemma-1 series), same generation on the N=4096 forest + DAG edges."""
import numpy as np
import pytest

import oracle
from paper_1608_00139_gb300 import inputs

pytestmark = pytest.mark.gpu

BIG = [(1e-4, 2), (1e-3, 3), (1e-2, 4)]


@pytest.fixture(scope="module")
def big_graphs():
    return {p: inputs.er_digraph(8192, p, s) for p, s in BIG}


@pytest.fixture(scope="module")
def big_models(big_graphs):
    oracle.set_threads(0)
    return {p: oracle.tc_model(e) for p, e in big_graphs.items()}


def test_config_er256_fp64(ctx):
    e = inputs.er_digraph(256, 0.02, 1)
    bits, st, x = ctx.tc_closure(e, path="fp64", rtilde=True)
    xr = oracle.tc_rtilde_lu(e, oracle.tc_eps(e))
    assert st["eps_used"] == oracle.tc_eps(e)
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    assert np.array_equal(bits, oracle.tc_model(e))


@pytest.mark.parametrize("path", ["bool_fp8", "auto"])
@pytest.mark.parametrize("p", [p for p, _ in BIG])
def test_config_er8192_fp8(ctx, big_graphs, big_models, p, path):
    bits, st = ctx.tc_closure(big_graphs[p], path=path)
    assert np.array_equal(bits, big_models[p])
    assert st["model_ones"] == int(np.unpackbits(big_models[p].view(np.uint8)).sum())


def test_config_er8192_fp64(ctx, big_graphs, big_models):
    p = 1e-3
    e = big_graphs[p]
    bits, st, x = ctx.tc_closure(e, path="fp64", rtilde=True)
    assert np.array_equal(bits, big_models[p])
    eps = st["eps_used"]
    assert eps == oracle.tc_eps(e)
    scale = np.abs(x).max()
    for j in (0, 1, 4095, 8191):
        col = oracle.tc_rtilde_col(e, eps, j)
        assert np.abs(x[:, j] - col).max() <= 1e-10 * scale


def test_config_sg4096(ctx):
    p = inputs.forest_dag(4096, 5)
    bits, st = ctx.sg_least_model(p)
    assert np.array_equal(bits, oracle.sg_model(p))


@pytest.mark.parametrize("p", [p for p, _ in BIG])
def test_config_er8192_mixed(ctx, big_graphs, big_models, p):
    """TF32 tensor-core LU + FP64 refinement at N = 8192: every model bit, and sampled
    columns of R~ against the Lemma-1 series within 1e-10 of max |R~|."""
    e = big_graphs[p]
    bits, st, x = ctx.tc_closure(e, path="mixed", rtilde=True)
    assert np.array_equal(bits, big_models[p])
    eps = st["eps_used"]
    scale = np.abs(x).max()
    for j in (0, 4095, 8191):
        col = oracle.tc_rtilde_col(e, eps, j)
        assert np.abs(x[:, j] - col).max() <= 1e-10 * scale
