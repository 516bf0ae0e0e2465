"""GPU parity at sizes the oracle finishes in well under a second: every path, tile edges,
ragged tails, degenerate inputs and argument errors.  Bits must equal the oracle's bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs
from tests.golden.load import read

pytestmark = pytest.mark.gpu

EDGE_SIZES = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 300, 511, 513]


def ref_compose(a, b):
    return oracle.pack((a.astype(np.int64) @ b.astype(np.int64)) > 0)


# --- tensor-core boolean product (the join of Sec. 2) ---------------------------------

@pytest.mark.parametrize("n", EDGE_SIZES)
def test_compose_tile_edges(ctx, n):
    rng = np.random.default_rng(n)
    a = (rng.random((n, n)) < 0.05).astype(np.uint8)
    b = (rng.random((n, n)) < 0.05).astype(np.uint8)
    bits, st = ctx.compose(a, b)
    assert np.array_equal(bits, ref_compose(a, b))


def test_compose_dense_counts_and_device_memory(ctx):
    n = 700
    rng = np.random.default_rng(3)
    a = (rng.random((n, n)) < 0.5).astype(np.uint8)
    b = (rng.random((n, n)) < 0.002).astype(np.uint8)
    ref = ref_compose(a, b)
    bits_h, st = ctx.compose(a, b)
    bits_d, _ = ctx.compose(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    assert np.array_equal(bits_h, ref)
    assert np.array_equal(bits_d.cpu().numpy().view(np.uint64), ref)
    assert st["model_ones"] == int(oracle.unpack(ref, n).sum())


# --- transitive closure ---------------------------------------------------------------

def test_worked_example_all_paths(ctx):
    g = read("worked_example_tc.txt")
    e = g["R1"].astype(np.uint8)
    want = oracle.pack(g["R2"])
    b8, st8 = ctx.tc_closure(e, path="bool_fp8")
    assert np.array_equal(b8, want)
    assert st8["eps_used"] == 0.5
    b64, st64, x = ctx.tc_closure(e, path="fp64", rtilde=True)
    assert np.array_equal(b64, want)
    exact = np.array([[1, 4, 2, 0], [2, 1, 4, 0], [4, 2, 1, 0], [4, 2, 1, 0]]) / 7.0
    assert np.max(np.abs(x - exact)) < 1e-14
    assert np.array_equal(np.floor(x * 1e4 + 1e-9) / 1e4, g["Rtilde_printed"])
    bm, stm, xm = ctx.tc_closure(e, path="mixed", rtilde=True)
    assert np.array_equal(bm, want)
    assert np.max(np.abs(xm - exact)) < 1e-10
    assert np.array_equal(np.floor(xm * 1e4 + 1e-9) / 1e4, g["Rtilde_printed"])


@pytest.mark.parametrize("n", EDGE_SIZES)
@pytest.mark.parametrize("path", ["bool_fp8", "fp64", "mixed", "auto"])
def test_closure_tile_edges(ctx, n, path):
    e = inputs.er_digraph(n, min(0.5, 3.0 / n), 100 + n)
    bits, st = ctx.tc_closure(e, path=path)
    assert np.array_equal(bits, oracle.tc_model(e))
    assert st["path_used"] == dl.PATHS[path]


@pytest.mark.parametrize("kind", ["empty", "ones_loops", "complete", "chain", "cycle",
                                  "self_loops", "star_in", "two_chains"])
def test_closure_degenerate_graphs(ctx, kind):
    n = 300
    e = np.zeros((n, n), dtype=np.uint8)
    if kind == "ones_loops":
        e[:] = 1
    elif kind == "complete":
        e[:] = 1
        np.fill_diagonal(e, 0)
    elif kind == "chain":
        e[np.arange(n - 1), np.arange(1, n)] = 1
    elif kind == "cycle":
        e[np.arange(n), (np.arange(n) + 1) % n] = 1
    elif kind == "self_loops":
        np.fill_diagonal(e, 1)
    elif kind == "star_in":
        e[1:, 0] = 1
    elif kind == "two_chains":
        e[np.arange(0, n - 2, 2), np.arange(2, n, 2)] = 1
    ref = oracle.tc_model(e)
    for path in ("bool_fp8", "fp64", "mixed", "auto"):
        bits, st = ctx.tc_closure(e, path=path)
        assert np.array_equal(bits, ref), path


@pytest.mark.parametrize("n", [64, 300])
def test_mixed_dense_complete_digraph_closed_form(ctx, n):
    """E = ones - I: R~_ii = (n-1)/(n+1), R~_ij = n/(n+1).  Dense rows put the FP64 residual
    at its rounding floor (about n u max|X|); the stated bound is kappa_inf(A) * resid."""
    e = (1 - np.eye(n)).astype(np.uint8)
    bits, st, x = ctx.tc_closure(e, path="mixed", rtilde=True)
    want = np.full((n, n), n / (n + 1.0))
    np.fill_diagonal(want, (n - 1) / (n + 1.0))
    kappa = 2.0 * n  # kappa_inf(I - eps E) <= (1 + eps ||E||) / eps
    assert np.abs(x - want).max() <= max(1e-10, 4 * kappa * st["final_resid"])
    assert np.abs(x - want).max() <= 1e-9
    assert np.array_equal(bits, oracle.pack(np.ones((n, n))))


@pytest.mark.parametrize("n,deg,seed", [(300, 0.5, 1), (700, 1.0, 2), (1000, 3.0, 3), (2049, 8.0, 4),
                                        (3000, 0.2, 5), (1500, 40.0, 6)])
def test_auto_path_sparse_and_dense(ctx, n, deg, seed):
    """DL_PATH_AUTO mixes squarings and sweeps by cost; every mix must give the oracle's model."""
    e = inputs.er_digraph(n, deg / n, seed)
    bits, st = ctx.tc_closure(e, path="auto")
    assert np.array_equal(bits, oracle.tc_model(e))
    assert st["path_used"] == dl.PATHS["auto"]
    assert st["recheck_sweeps"] >= 1


@pytest.mark.parametrize("n,seed", [(1500, 7), (3000, 8)])
def test_heavy_tailed_degrees(ctx, n, seed):
    """Preferential-attachment DAGs have rows with hundreds of successors: the sweeps split
    such rows into units combined with atomicOr; models must still equal the oracle's."""
    e = inputs.pa_dag(n, seed)
    assert oracle.max_row_sum(e) > 64
    ref = oracle.tc_model(e)
    for path in ("auto", "bool_fp8"):
        bits, st = ctx.tc_closure(e, path=path)
        assert np.array_equal(bits, ref), path
    e2 = e | e.T  # cycles everywhere, dense closure with heavy rows
    ref2 = oracle.tc_model(e2)
    for path in ("auto", "bool_fp8"):
        assert np.array_equal(ctx.tc_closure(e2, path=path)[0], ref2), path


def test_auto_path_long_chain_and_cycle(ctx):
    for n in (1000, 2500):
        e = np.zeros((n, n), dtype=np.uint8)
        e[np.arange(n - 1), np.arange(1, n)] = 1
        bits, st = ctx.tc_closure(e, path="auto")
        assert np.array_equal(bits, oracle.tc_model(e))
        e[n - 1, 0] = 1
        bits, st = ctx.tc_closure(e, path="auto")
        assert np.array_equal(bits, oracle.tc_model(e))


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_auto_permuted_chains(ctx, seed):
    """Chains under random labels (some hops go down in index, some up, so an in-place sweep
    moves a fact one hop or many), joined by a few random edges and then by a cycle, keep
    rows changing long after others have settled, and the long ones force squarings between
    sweeps; every model must equal the oracle's."""
    rng = np.random.default_rng(seed)
    n = 1800
    perm = rng.permutation(n)
    e = np.zeros((n, n), dtype=np.uint8)
    for a, b in ((0, 600), (600, 1500), (1500, n)):  # three chains of different lengths
        idx = perm[a:b]
        e[idx[:-1], idx[1:]] = 1
    extra = rng.integers(0, n, size=(40, 2))
    e[extra[:, 0], extra[:, 1]] = 1
    bits, st = ctx.tc_closure(e, path="auto")
    assert np.array_equal(bits, oracle.tc_model(e))
    e[perm[1499], perm[0]] = 1  # close the second chain into the first
    bits, st = ctx.tc_closure(e, path="auto")
    assert np.array_equal(bits, oracle.tc_model(e))


def test_chain_needs_log_squarings(ctx):
    n = 1000
    e = np.zeros((n, n), dtype=np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    bits, st = ctx.tc_closure(e, path="bool_fp8")
    assert np.array_equal(bits, oracle.tc_model(e))
    assert st["iters"] == 10  # paths up to 999 need 2^t >= 999


@pytest.mark.parametrize("path", ["fp64", "mixed"])
def test_underflow_is_repaired_by_recheck(ctx, path):
    """A chain of 1100 constants: eps = 1/2 and eps^d underflows FP64 for d > 1074 (FP32 /
    TF32 far earlier), so the threshold misses facts; the exact recheck must restore them
    (Lemma 2 footnote: reachable entries are >= eps^d, which can be below the format's range)."""
    n = 1100
    e = np.zeros((n, n), dtype=np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    bits, st = ctx.tc_closure(e, path=path)
    assert np.array_equal(bits, oracle.tc_model(e))
    assert st["rows_rechecked"] > 0


@pytest.mark.parametrize("n,p,seed", [(256, 0.02, 1), (400, 0.01, 2), (600, 0.005, 3)])
def test_fp64_rtilde_matches_oracle(ctx, n, p, seed):
    e = inputs.er_digraph(n, p, seed)
    bits, st, x = ctx.tc_closure(e, path="fp64", rtilde=True)
    xr = oracle.tc_rtilde_lu(e, st["eps_used"])
    assert st["eps_used"] == oracle.tc_eps(e)
    err = np.abs(x - xr).max() / np.abs(xr).max()
    assert err <= 1e-10
    assert np.array_equal(bits, oracle.tc_model(e))
    assert np.array_equal(oracle.pack(x > 0), bits)


@pytest.mark.parametrize("n,p,seed", [(256, 0.02, 1), (300, 0.05, 2), (640, 0.01, 3), (513, 0.002, 4)])
def test_mixed_rtilde_matches_oracle(ctx, n, p, seed):
    """TF32 LU + FP64 refinement: R~ within 1e-10 (max-abs error / max-abs value)."""
    e = inputs.er_digraph(n, p, seed)
    bits, st, x = ctx.tc_closure(e, path="mixed", rtilde=True)
    xr = oracle.tc_rtilde_lu(e, st["eps_used"])
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    assert np.array_equal(bits, oracle.tc_model(e))
    assert st["path_used"] == dl.PATHS["mixed"]
    assert st["final_resid"] <= 1e-13
    assert st["iters"] >= 1


def test_mixed_hub_and_chain_dynamic_range(ctx):
    """A hub with n-1 successors (eps = 1/n) and a long chain: R~ spans hundreds of decades and
    one row's residual sums n-1 terms (the fixed-point residual's widest sums)."""
    n = 700
    e = inputs.er_digraph(n, 0.002, 11)
    e[3, :] = 1
    e[3, 3] = 0
    for k in range(100, 399):
        e[k, k + 1] = 1
    bits, st, x = ctx.tc_closure(e, path="mixed", rtilde=True)
    xr = oracle.tc_rtilde_lu(e, st["eps_used"])
    assert st["eps_used"] == 1.0 / n
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    assert st["final_resid"] <= 1e-13
    assert np.array_equal(bits, oracle.tc_model(e))


def test_mixed_two_rows_per_residual_block(ctx):
    """n = 9800: a row of Z takes 78 KB, so the residual stages two rows per block."""
    n = 9800
    e = inputs.er_digraph(n, 5e-4, 12)
    bits, st, x = ctx.tc_closure(e, path="mixed", rtilde=True)
    assert st["final_resid"] <= 1e-13
    assert np.array_equal(bits, oracle.tc_model(e))
    for j in (0, 4321, n - 1):
        col = oracle.tc_rtilde_col(e, st["eps_used"], j)
        assert np.abs(x[:, j] - col).max() <= 1e-10 * max(np.abs(col).max(), st["eps_used"])


def test_mixed_one_row_per_residual_block(ctx):
    """n = 15000: one row of Z per residual block; the model against the oracle's."""
    n = 15000
    e = inputs.er_digraph(n, 2e-4, 13)
    bits, st, x = ctx.tc_closure(torch.from_numpy(e).cuda(), path="mixed", rtilde=True)
    assert st["final_resid"] <= 1e-13
    assert np.array_equal(bits.cpu().numpy().view(np.uint64), oracle.tc_model(e))
    # without an R~ output the path stops after the solve; the model is the same
    bits, st = ctx.tc_closure(e, path="mixed")
    assert st["iters"] == 0 and st["final_resid"] == -1.0
    assert np.array_equal(bits, oracle.tc_model(e))


def test_user_eps(ctx):
    e = inputs.er_digraph(200, 0.02, 5)
    e0 = oracle.tc_eps(e)
    bits, st, x = ctx.tc_closure(e, eps=e0 / 2, path="fp64", rtilde=True)
    assert st["eps_used"] == e0 / 2
    xr = oracle.tc_rtilde_lu(e, e0 / 2)
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
    assert np.array_equal(bits, oracle.tc_model(e))


def test_device_and_host_memory_agree(ctx):
    e = inputs.er_digraph(777, 0.004, 9)
    bh, _ = ctx.tc_closure(e)
    bd, _ = ctx.tc_closure(torch.from_numpy(e).cuda())
    assert np.array_equal(bh, bd.cpu().numpy().view(np.uint64))
    assert np.array_equal(bh, oracle.tc_model(e))


def test_argument_errors(ctx):
    e = inputs.er_digraph(50, 0.1, 1)
    bad = e.copy()
    bad[3, 4] = 2
    for path in ("bool_fp8", "fp64"):
        with pytest.raises(dl.DLError) as ei:
            ctx.tc_closure(bad, path=path)
        assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        ctx.tc_closure(e, eps=0.9)
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        ctx.tc_closure(e, thr=0.1)
    assert ei.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as ei:
        ctx.tc_closure(e, path="bool_fp8", rtilde=True)
    assert ei.value.status == dl.DL_EINVAL
    bits, st = ctx.tc_closure(np.zeros((0, 0), dtype=np.uint8))
    assert bits.shape == (0, 0)
    # the context still works after errors
    bits, _ = ctx.tc_closure(e)
    assert np.array_equal(bits, oracle.tc_model(e))


# --- same generation ------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 33, 100, 256, 257, 700])
def test_sg_forest(ctx, n):
    p = inputs.forest_dag(n, 7 + n, extra_prob=0.02)
    bits, st = ctx.sg_least_model(p)
    assert np.array_equal(bits, oracle.sg_model(p))


@pytest.mark.parametrize("n,pe", [(50, 0.05), (200, 0.01), (300, 0.004)])
def test_sg_general_digraph(ctx, n, pe):
    p = inputs.er_digraph(n, pe, n, self_loops=True)
    bits, st = ctx.sg_least_model(p)
    assert np.array_equal(bits, oracle.sg_model(p))


def test_sg_with_base_relation_and_degenerate(ctx):
    n = 150
    p = inputs.er_digraph(n, 0.02, 4)
    b = inputs.er_digraph(n, 0.01, 5, self_loops=True)
    bits, _ = ctx.sg_least_model(p, b)
    assert np.array_equal(bits, oracle.sg_model(p, b))
    z = np.zeros((n, n), dtype=np.uint8)
    bits, st = ctx.sg_least_model(z)
    assert np.array_equal(bits, oracle.pack(np.eye(n)))
    tree = np.zeros((n, n), dtype=np.uint8)
    tree[np.arange(1, n), (np.arange(1, n) - 1) // 2] = 1
    bits, st = ctx.sg_least_model(tree)
    assert np.array_equal(bits, oracle.sg_model(tree))
    with pytest.raises(dl.DLError) as ei:
        ctx.sg_least_model(p, path="fp64")
    assert ei.value.status == dl.DL_ENOTIMPL


@pytest.mark.parametrize("n,seed", [(6200, 21), (6400, 22)])
def test_sg_iteration_and_doubling_agree(ctx, n, seed):
    """At these sizes AUTO runs the Iteration on bits (S <- B | P S P^T with bit transposes
    and row gathers, heavy parent lists split into work units); bool_fp8 runs the
    tensor-core doubling.  Both must give the oracle's model, also for a base relation B that
    is not symmetric (S is then not symmetric either)."""
    oracle.set_threads(0)
    for p in (inputs.pa_dag(n, seed), inputs.forest_dag(n, seed, extra_prob=0.02)):
        ref = oracle.sg_model(p)
        a, sta = ctx.sg_least_model(p, path="auto")
        b, stb = ctx.sg_least_model(p, path="bool_fp8")
        assert np.array_equal(a, ref) and np.array_equal(b, ref)
        assert sta["path_used"] == dl.PATHS["auto"] and stb["path_used"] == dl.PATHS["bool_fp8"]
        ones = int(np.unpackbits(ref.view(np.uint8)).sum())
        assert sta["model_ones"] == ones and stb["model_ones"] == ones
    p = inputs.pa_dag(n, seed)
    bm = inputs.er_digraph(n, 2.0 / n, seed + 1, self_loops=True)
    assert not np.array_equal(bm, bm.T)
    ref = oracle.sg_model(p, bm)
    assert np.array_equal(ctx.sg_least_model(p, bm, path="auto")[0], ref)
    assert np.array_equal(ctx.sg_least_model(p, bm, path="bool_fp8")[0], ref)


def test_sg_deep_derivations_fall_back_to_doubling(ctx):
    """Two chains of 100 under one root (and isolated constants up to a size where AUTO
    iterates): the pair at depth k appears after k iterations, more than the Iteration's
    budget, so AUTO hands the problem to the doubling."""
    n = 6200
    p = np.zeros((n, n), dtype=np.uint8)
    for chain in (range(1, 101), range(101, 201)):
        prev = 0
        for v in chain:
            p[v, prev] = 1
            prev = v
    bits, st = ctx.sg_least_model(p, path="auto")
    assert np.array_equal(bits, oracle.sg_model(p))
    assert st["path_used"] == dl.PATHS["bool_fp8"]


def test_auto_speculative_start_fallbacks():
    """The AUTO closure's first steps run before the host knows the number of facts or the
    longest row.  On a fresh context: a dense graph overflows the column array (the host then
    re-plans), the same graph again fits; a graph with rows of hundreds of successors stops the
    speculative launches (heavy rows), the next graph then starts without speculating; a sparse
    graph closed by the single-row Iteration is followed by one it cannot close.  Every model
    must equal the oracle's."""
    with dl.Context(0) as c:
        graphs = [inputs.er_digraph(1500, 0.02, 31), inputs.er_digraph(1500, 0.02, 31),
                  inputs.pa_dag(1500, 32), inputs.er_digraph(1500, 0.004, 33),
                  inputs.er_digraph(1500, 0.0005, 34), inputs.er_digraph(1500, 0.003, 35),
                  inputs.pa_dag(900, 36) | inputs.pa_dag(900, 36).T]
        assert oracle.max_row_sum(graphs[2]) > 256
        for e in graphs:
            bits, st = c.tc_closure(e, path="auto")
            assert np.array_equal(bits, oracle.tc_model(e))
