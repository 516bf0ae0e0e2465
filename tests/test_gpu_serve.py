"""GPU tests of serving (dl_submit / dl_poll / dl_cancel): requests admitted while others
run, overlapping on the GPU; each result must equal the oracle's and the same request solved
alone."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def mix(count=24, seed=11):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(64), np.log(3000))))
        if rng.random() < 0.75:
            reqs.append((0, inputs.pa_dag(n, seed * 1000 + i) if i % 2 else
                         inputs.er_digraph(n, 3.0 / n, seed * 1000 + i)))
        else:
            reqs.append((1, inputs.forest_dag(n, seed * 1000 + i, extra_prob=0.01)))
    return reqs


def ref(kind, m):
    return oracle.tc_model(m) if kind == 0 else oracle.sg_model(m)


def test_mix_equals_oracle_and_alone():
    with dl.Context(0, max_slots=4) as c:
        reqs = mix()
        handles = [c.submit(kind, m) for kind, m in reqs]  # all submitted before any finishes
        stats = []
        for t, h in handles:
            status, st = c.poll(t, timeout_us=-1)
            assert status == dl.DL_OK
            stats.append(st)
        for (kind, m), (t, h) in zip(reqs, handles):
            assert np.array_equal(h["bits"], ref(kind, m))
            alone = c.tc_closure(m)[0] if kind == 0 else c.sg_least_model(m)[0]
            assert np.array_equal(alone, h["bits"])
        assert all(s["ms_latency"] >= s["ms_queue"] >= 0 for s in stats)
        assert max(s["ms_queue"] for s in stats) > 0  # some requests waited for a slot


def test_device_resident_requests():
    with dl.Context(0, max_slots=3) as c:
        reqs = mix(10, 12)
        dev = [(k, torch.from_numpy(m).cuda()) for k, m in reqs]
        handles = [c.submit(k, d) for k, d in dev]
        for (k, m), (t, h) in zip(reqs, handles):
            assert c.poll(t, -1)[0] == dl.DL_OK
            assert np.array_equal(h["bits"].cpu().numpy().view(np.uint64), ref(k, m))


def test_admission_budget_and_errors():
    with dl.Context(0, max_slots=1, hbm_budget_bytes=16 << 20) as c:
        big = inputs.er_digraph(4096, 1e-3, 1)  # needs about 55 MB
        with pytest.raises(dl.DLError) as ei:
            c.submit(0, big)
        assert ei.value.status == dl.DL_ENOMEM
        small = inputs.er_digraph(300, 0.01, 2)
        t, h = c.submit(0, small)
        assert c.poll(t, -1)[0] == dl.DL_OK
        assert np.array_equal(h["bits"], oracle.tc_model(small))
        with pytest.raises(dl.DLError) as ei:
            c.poll(t, 0)  # already collected
        assert ei.value.status == dl.DL_EINVAL
        bad = small.copy()
        bad[1, 1] = 3
        t, h = c.submit(0, bad)
        with pytest.raises(dl.DLError) as ei:
            c.poll(t, -1)
        assert ei.value.status == dl.DL_EINVAL


def test_cancel_queued_requests():
    with dl.Context(0, max_slots=1) as c:
        gs = [inputs.er_digraph(2048, 2e-3, 30 + i) for i in range(12)]
        handles = [c.submit(0, g) for g in gs]
        cancelled = []
        for t, _ in reversed(handles):
            rc = c.cancel(t)
            assert rc in (dl.DL_OK, dl.DL_EBUSY)
            if rc == dl.DL_OK:
                cancelled.append(t)
        assert cancelled  # with one slot, the tail of the queue was still waiting
        for (t, h), g in zip(handles, gs):
            if t in cancelled:
                with pytest.raises(dl.DLError) as ei:
                    c.poll(t, -1)
                assert ei.value.status == dl.DL_ECANCELED
            else:
                assert c.poll(t, -1)[0] == dl.DL_OK
                assert np.array_equal(h["bits"], oracle.tc_model(g))
