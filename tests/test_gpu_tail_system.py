"""Tail recursive equations with real lower solutions and layered systems (dl_tail_recursive_real,
dl_tail_system; Sec. 6.1, eq. matrixeq:trec) on the GPU against the oracle: bits exact, R~ within
1e-10 (max-abs error / max-abs value) of the oracle's in-order FP64 solve and, for small n, of the
stacked solve of the whole system."""
import numpy as np
import pytest
import torch

from oracle import tail as tl
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def unpack(bits, n):
    b = bits.cpu().numpy() if isinstance(bits, torch.Tensor) else bits
    return np.unpackbits(b.view(np.uint8), axis=1, bitorder="little")[:, :n]


def rel_err(x, ref):
    x = x.cpu().numpy() if isinstance(x, torch.Tensor) else x
    return float(np.abs(x - ref).max()) / max(float(np.abs(ref).max()), 1e-300)


def path(n):
    e = np.zeros((n, n), np.uint8)
    e[np.arange(n - 1), np.arange(1, n)] = 1
    return e


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_two_equation_chain_in_closed_form(ctx, mode):
    n = 300
    e = path(n)
    eqs = [{"A1": e, "B0": e}, {"terms": [(np.eye(n, dtype=np.uint8), 0)]}]
    bits, st, xs = ctx.tail_system(eqs, path=mode)
    i, j = np.indices((n, n))
    want0 = np.where(j > i, np.ldexp(1.0, -(j - i).clip(0, 1074)), 0.0)
    assert rel_err(xs[0], want0) <= 1e-10
    assert rel_err(xs[1], want0 / 2) <= 1e-10
    for h in range(2):
        assert np.array_equal(unpack(bits[h], n), (j > i).astype(np.uint8))


def random_system(rng, n, m, dens=0.02):
    eqs = []
    for h in range(m):
        eqs.append({"A1": (rng.random((n, n)) < dens).astype(np.uint8) if rng.random() < 0.8 else None,
                    "B0": (rng.random((n, n)) < 1.5 / n).astype(np.uint8) if rng.random() < 0.8 else None,
                    "terms": [((rng.random((n, n)) < 1.0 / n).astype(np.uint8), int(rng.integers(0, h)))
                              for _ in range(int(rng.integers(1, 3)) if h else 0)]})
    return eqs


@pytest.mark.parametrize("n,m,seed", [(33, 3, 1), (129, 4, 2), (300, 3, 3)])
def test_random_systems(ctx, n, m, seed):
    rng = np.random.default_rng(seed)
    eqs = random_system(rng, n, m)
    models, xs_ref, epss = tl.tail_system(eqs, n)
    stacked = tl.tail_system_stacked(eqs, n, epss) if n <= 129 else None
    for mode in ("fp64", "mixed"):
        bits, st, xs = ctx.tail_system(eqs, path=mode)
        for h in range(m):
            assert np.array_equal(unpack(bits[h], n), models[h]), (mode, h)
            assert rel_err(xs[h], xs_ref[h]) <= 1e-10, (mode, h)
            if stacked is not None:
                assert rel_err(xs[h], stacked[h]) <= 1e-10
    for mode in ("auto", "bool_fp8"):
        bits, st = ctx.tail_system(eqs, path=mode, rtilde=False)
        for h in range(m):
            assert np.array_equal(unpack(bits[h], n), models[h]), (mode, h)


def test_single_equation_with_host_lower_solutions(ctx):
    rng = np.random.default_rng(9)
    n = 200
    eqs = random_system(rng, n, 3)
    models, xs_ref, epss = tl.tail_system(eqs, n)
    eq = eqs[2]
    terms = [(b, xs_ref[j]) for b, j in eq["terms"]]
    for mode in ("fp64", "mixed"):
        bits, st, x = ctx.tail_recursive_real(eq["B0"], eq["A1"], terms, path=mode)
        assert np.array_equal(unpack(bits, n), models[2])
        assert rel_err(x, xs_ref[2]) <= 1e-10
        assert st["eps_used"] == epss[2]
    # device buffers
    dterms = [(torch.from_numpy(b).cuda(), torch.from_numpy(r).cuda()) for b, r in terms]
    b0 = torch.from_numpy(eq["B0"]).cuda() if eq["B0"] is not None else None
    a1 = torch.from_numpy(eq["A1"]).cuda() if eq["A1"] is not None else None
    bits, st, x = ctx.tail_recursive_real(b0, a1, dterms, path="mixed")
    assert x.is_cuda and rel_err(x, xs_ref[2]) <= 1e-10
    assert np.array_equal(unpack(bits, n), models[2])


def test_errors(ctx):
    n = 64
    e = path(n)
    eqs = [{"A1": e, "B0": e}, {"terms": [(e, 1)]}]  # refers to itself: not below
    with pytest.raises(dl.DLError) as err:
        ctx.tail_system(eqs)
    assert err.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as err:
        ctx.tail_system([{"A1": e, "B0": e, "eps": 0.9}])  # above 1/(1 + 1)
    assert err.value.status == dl.DL_EINVAL
    with pytest.raises(dl.DLError) as err:
        ctx.tail_system([{"A1": e, "B0": e}], path="bool_fp8", rtilde=True)
    assert err.value.status == dl.DL_EINVAL


def test_n2048_layered_erdos_renyi(ctx):
    """Three layers over ER graphs at N = 2048 (B0 mean degree 3, lower terms degree 1)."""
    n = 2048
    e1 = inputs.er_digraph(n, 3.0 / n, 51)
    e2 = inputs.er_digraph(n, 3.0 / n, 52)
    e3 = inputs.er_digraph(n, 1.0 / n, 53)
    e4 = inputs.er_digraph(n, 1.0 / n, 54)
    a = inputs.er_digraph(n, 1e-3, 55)
    eqs = [{"A1": a, "B0": e1}, {"B0": e2, "terms": [(e3, 0)]}, {"A1": a, "terms": [(e4, 1), (e3, 0)]}]
    models, xs_ref, _ = tl.tail_system(eqs, n)
    dev = [{k: (torch.from_numpy(v).cuda() if isinstance(v, np.ndarray) else
                [(torch.from_numpy(b).cuda(), j) for b, j in v] if k == "terms" else v)
            for k, v in eq.items()} for eq in eqs]
    bits, st, xs = ctx.tail_system(dev, path="mixed")
    for h in range(3):
        assert np.array_equal(unpack(bits[h], n), models[h]), h
        assert rel_err(xs[h], xs_ref[h]) <= 1e-10, h
