"""GPU parity of the real same-generation solution S~ = eps (B + P S~ P^T) (Sec. 7.2): the
FP64 series, the TF32 doubling with FP64 refinement and AUTO against the oracle's Kronecker
solve (tiny N) and fixpoint series; the model bits against the semi-naive oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu

PATHS = ["auto", "fp64", "mixed"]


def rel_err(x, ref):
    return np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300)


def random_p(n, density, seed, dag=False):
    rng = np.random.default_rng(seed)
    p = (rng.random((n, n)) < density).astype(np.uint8)
    return np.tril(p, -1) if dag else p


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,seed,with_b", [(1, 1, False), (5, 2, False), (12, 3, True), (30, 4, False)])
def test_tiny_against_kronecker(ctx, path, n, seed, with_b):
    p = random_p(n, 0.3, seed)  # cycles: the series converges geometrically
    b = random_p(n, 0.25, 70 + seed) if with_b else None
    x, bits, st = ctx.sg_real(p, b, path=path)
    ref = oracle.sg_stilde_kron(p, b)
    assert rel_err(x, ref) <= 1e-10
    assert st["eps_used"] == oracle.sg_eps(p)
    assert st["final_resid"] <= 1e-13
    assert np.array_equal(bits, oracle.sg_model(p, b))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n", [63, 64, 65, 257, 700])
def test_forest_dag_against_series(ctx, path, n):
    p = inputs.forest_dag(n, 5 + n)
    x, bits, st = ctx.sg_real(p, path=path)
    ref = oracle.sg_stilde_series(p)
    assert rel_err(x, ref) <= 1e-10
    assert np.array_equal(bits, oracle.sg_model(p))
    if path != "mixed":
        assert st["path_used"] == dl.PATHS["fp64"]  # nilpotent P: the series ends exactly


@pytest.mark.parametrize("path", ["auto", "mixed"])
def test_cyclic_graph_refinement(ctx, path):
    """ER digraph with cycles and ||P|| large: the series converges slowly, AUTO switches to
    the refinement; both reach the oracle's S~."""
    n = 400
    p = inputs.er_digraph(n, 0.03, 21)
    x, bits, st = ctx.sg_real(p, path=path)
    ref = oracle.sg_stilde_series(p)
    assert rel_err(x, ref) <= 1e-10
    assert st["final_resid"] <= 1e-13
    assert np.array_equal(bits, oracle.sg_model(p))


def test_chain_closed_form(ctx):
    n = 300
    p = np.zeros((n, n), dtype=np.uint8)
    p[np.arange(1, n), np.arange(n - 1)] = 1
    want = np.diag(1.0 - 0.5 ** (np.arange(n) + 1.0))
    for path in PATHS:
        x, bits, st = ctx.sg_real(p, path=path)
        assert np.abs(x - want).max() <= 1e-12, path
        assert st["eps_used"] == 0.5


def test_nonsymmetric_b_and_device_memory(ctx):
    n = 333
    p = inputs.forest_dag(n, 9)
    b = random_p(n, 0.01, 99)
    ref = oracle.sg_stilde_series(p, b)
    x, bits, st = ctx.sg_real(torch.from_numpy(p).cuda(), torch.from_numpy(b).cuda())
    assert x.is_cuda and bits.is_cuda
    assert rel_err(x.cpu().numpy(), ref) <= 1e-10
    assert np.array_equal(bits.cpu().numpy().view(np.uint64), oracle.sg_model(p, b))


def test_forest_4096_config(ctx):
    """The same-generation workload (forest + DAG edges, N = 4096, seed 5): S~ against the
    oracle's series, the bits against the semi-naive model."""
    p = inputs.forest_dag(4096, 5)
    x, bits, st = ctx.sg_real(p)
    ref = oracle.sg_stilde_series(p)
    assert rel_err(x, ref) <= 1e-12
    assert np.array_equal(bits, oracle.sg_model(p))
    assert st["path_used"] == dl.PATHS["fp64"]


def test_arguments(ctx):
    p = random_p(20, 0.2, 1)
    with pytest.raises(dl.DLError) as ei:
        ctx.sg_real(p, path="bool_fp8")
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        ctx.sg_real(p, eps=2 * oracle.sg_eps(p))
    assert ei.value.status == dl.DL_EINVAL
    bad = p.copy()
    bad[3, 4] = 2
    with pytest.raises(dl.DLError) as ei:
        ctx.sg_real(bad)
    assert ei.value.status == dl.DL_EINVAL
    x, bits, st = ctx.sg_real(p, eps=oracle.sg_eps(p) / 2, bits=False)
    assert bits is None
    assert rel_err(x, oracle.sg_stilde_series(p, None, oracle.sg_eps(p) / 2)) <= 1e-10
    x0, _, _ = ctx.sg_real(np.zeros((0, 0), dtype=np.uint8))
    assert x0.shape == (0, 0)


@pytest.mark.parametrize("path", ["auto", "fp64", "mixed"])
def test_slowly_converging_series(ctx, path):
    """A circulant P with four successors per node: eps ||P kron P|| = 16/17, so the series needs
    about 480 steps; AUTO leaves it after 64 for the refinement, FP64 runs it to the end."""
    n = 300
    p = np.zeros((n, n), dtype=np.uint8)
    for k in range(1, 5):
        p[np.arange(n), (np.arange(n) + k) % n] = 1
    x, bits, st = ctx.sg_real(p, path=path)
    ref = oracle.sg_stilde_series(p)
    assert rel_err(x, ref) <= 1e-10
    assert st["final_resid"] <= 1e-13
    assert np.array_equal(bits, oracle.sg_model(p))
    if path == "auto":
        assert st["path_used"] == dl.PATHS["mixed"] and st["iters"] > 64
    if path == "fp64":
        assert st["iters"] > 64
