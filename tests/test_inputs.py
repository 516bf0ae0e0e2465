"""The seeded generators: deterministic, shaped like the paper's workloads (no GPU)."""
import numpy as np

from paper_1608_00139_gb300 import inputs


def test_mix64_known_values():
    # SplitMix64 seeded with 0: first outputs of the published generator
    out = inputs.draws(np.uint64(0), np.arange(3, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_er_deterministic_and_rate():
    a = inputs.er_digraph(300, 0.05, 7)
    b = inputs.er_digraph(300, 0.05, 7, rows_per_chunk=17)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, inputs.er_digraph(300, 0.05, 8))
    assert a.dtype == np.uint8 and set(np.unique(a)) <= {0, 1}
    assert np.all(np.diag(a) == 0)
    rate = a.sum() / (300 * 299)
    assert abs(rate - 0.05) < 0.005
    c = inputs.er_digraph(50, 1.0, 1, self_loops=True)
    assert c.all()


def test_forest_is_strictly_lower_and_mostly_one_parent():
    p = inputs.forest_dag(4096, 5)
    assert not np.triu(p).any()
    deg = p.sum(1)
    roots = (deg == 0).sum()
    assert 0.02 * 4096 < roots < 0.09 * 4096
    assert (deg >= 2).sum() < 60
    assert np.array_equal(p, inputs.forest_dag(4096, 5))


def test_pa_dag_shape():
    e = inputs.pa_dag(2000, 3)
    assert not np.triu(e).any()
    assert e[1:].sum(1).min() >= 1
    assert np.array_equal(e, inputs.pa_dag(2000, 3))


def test_native_pa_dag_equals_the_python_generator():
    for n, seed in [(0, 1), (1, 1), (2, 5), (37, 2), (700, 3), (2500, 9)]:
        want = inputs.pa_dag(n, seed)
        got = inputs.pa_dag_into(np.full((n, n), 7, np.uint8), seed)
        assert np.array_equal(got, want), (n, seed)
    # into a row-strided view of a larger buffer
    buf = np.full((300, 512), 9, np.uint8)
    view = inputs.pa_dag_into(buf[:300, :300], 4)
    assert np.array_equal(view, inputs.pa_dag(300, 4)) and (buf[:, 300:] == 9).all()


def test_batch_and_stream_specs():
    specs = inputs.batch_specs(64)
    assert all(32 <= n <= 2048 and 0 < p <= 8.0 / 31 for n, p, _ in specs)
    t, k, s, _ = inputs.poisson_stream(200.0, 2.0, 6)
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    assert 250 < len(t) < 550
    assert s.min() >= 512 and s.max() <= 16384
