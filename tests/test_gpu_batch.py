"""GPU parity of dl_tc_batch: many closures of uneven size in one call (grouped tcgen05
launches per squaring round, replayed from a captured CUDA graph).  Every model must equal
the oracle's bits and the result of the same problem solved alone."""
import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def small_batch(count=40, seed0=500):
    gs = []
    for n, p, seed in inputs.batch_specs(count, seed0, n_lo=1, n_hi=700):
        gs.append(inputs.er_digraph(n, p, seed))
    gs[3] = np.zeros((0, 0), dtype=np.uint8)           # empty problem
    chain = np.zeros((300, 300), dtype=np.uint8)       # long paths: many rounds
    chain[np.arange(299), np.arange(1, 300)] = 1
    gs[5] = chain
    return gs


def test_batch_host_memory_matches_oracle(ctx):
    gs = small_batch()
    outs, st = ctx.tc_batch(gs)
    for e, b in zip(gs, outs):
        assert np.array_equal(b, oracle.tc_model(e))
    # the 300-chain outruns the first sweeps (one hop each): it needs squaring rounds
    assert st["iters"] >= 1 and st["recheck_sweeps"] >= 24
    assert st["model_ones"] == sum(int(np.unpackbits(oracle.tc_model(e).view(np.uint8)).sum())
                                   for e in gs if e.shape[0])


def test_batch_device_memory_repeat_and_alone(ctx):
    gs = small_batch(24, 900)
    dev = [torch.from_numpy(e).cuda() for e in gs]
    outs1, _ = ctx.tc_batch(dev)
    outs2, _ = ctx.tc_batch(dev)  # same buffers: the cached graph is relaunched
    for e, d, a, b in zip(gs, dev, outs1, outs2):
        ref = oracle.tc_model(e)
        assert np.array_equal(a.cpu().numpy().view(np.uint64), ref)
        assert torch.equal(a, b)
        if e.shape[0]:
            alone, _ = ctx.tc_closure(d)
            assert torch.equal(alone, a)


def test_batch_rejects_bad_input(ctx):
    gs = small_batch(6, 1200)
    bad = gs[1].copy()
    bad[0, 0] = 7
    gs[1] = bad
    with pytest.raises(dl.DLError) as ei:
        ctx.tc_batch(gs)
    assert ei.value.status == dl.DL_EINVAL
    outs, _ = ctx.tc_batch(small_batch(6, 1300))  # the context still works


def test_batch_config_1024_uneven(ctx):
    """The uneven batch workload: 1024 ER closures, N ~ U{32..2048}, mean degree ~ U[1, 8]."""
    specs = inputs.batch_specs(1024, 1000)
    gs = [torch.from_numpy(inputs.er_digraph(n, p, s)).cuda() for n, p, s in specs]
    outs, st = ctx.tc_batch(gs)
    oracle.set_threads(0)
    for k in range(1024):  # every instance
        e = gs[k].cpu().numpy()
        assert np.array_equal(outs[k].cpu().numpy().view(np.uint64), oracle.tc_model(e)), k


def test_batch_misaligned_rows_self_loops_wide_rows(ctx):
    """Inputs whose rows start at every 16-byte misalignment (device views at odd offsets),
    self-loops (E's diagonal must reach the successor lists exactly), and instances wide
    enough for rows of 2, 4 and 8 64-bit words per lane."""
    rng = np.random.default_rng(77)
    ns = [1, 5, 17, 64, 130, 700, 2100, 3000, 5000, 9000]
    gs = []
    for j, n in enumerate(ns):
        e = inputs.er_digraph(n, min(1.0, 1.5 / n), 4_000 + j)
        diag = rng.random(n) < 0.3
        e[np.arange(n), np.arange(n)] = diag.astype(np.uint8)
        gs.append(e)
    dev = []
    for j, e in enumerate(gs):
        n = e.shape[0]
        off = (3 + 5 * j) % 16
        buf = torch.zeros(off + n * n + 16, dtype=torch.uint8, device="cuda")
        view = buf[off:off + n * n].view(n, n)
        view.copy_(torch.from_numpy(e))
        dev.append(view)
    outs, _ = ctx.tc_batch(dev)
    houts, _ = ctx.tc_batch(gs)
    for e, d, h in zip(gs, outs, houts):
        ref = oracle.tc_model(e)
        assert np.array_equal(d.cpu().numpy().view(np.uint64), ref)
        assert np.array_equal(h, ref)


def test_batch_flat_buffer_matches_list_call(ctx):
    """tc_batch_flat: instances back to back in one buffer (odd offsets too), one output
    buffer; every model equals the oracle's and the per-tensor call's."""
    gs = small_batch(30, 700)
    ns = np.array([g.shape[0] for g in gs], dtype=np.int32)
    offsets, pos = [], 0
    for k, g in enumerate(gs):
        pos += k % 5  # misaligned starts
        offsets.append(pos)
        pos += g.size
    flat = np.zeros(pos + 16, dtype=np.uint8)
    for g, o in zip(gs, offsets):
        flat[o:o + g.size] = g.reshape(-1)
    for buf in (flat, torch.from_numpy(flat).cuda()):
        out, ooff, st = ctx.tc_batch_flat(buf, ns, offsets)
        out = out.cpu().numpy() if hasattr(out, "cpu") else out
        for g, n, o in zip(gs, ns, ooff):
            w = (int(n) + 63) // 64
            got = out[o:o + int(n) * w].view(np.uint64).reshape(int(n), w)
            assert np.array_equal(got, oracle.tc_model(g))
