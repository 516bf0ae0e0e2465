"""Failure detection without a GPU fault: a bounded device-side wait on a barrier that
nothing arrives at must give up within its budget, report DL_ETIMEOUT and leave the
context usable."""
import time

import numpy as np
import pytest

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_context_survives(ctx):
    t0 = time.perf_counter()
    rc = ctx.selftest_wait_timeout(0.05)
    dt = time.perf_counter() - t0
    assert rc == dl.DL_ETIMEOUT
    assert b"expired" in dl.lib().dl_last_error()
    assert dt < 2.0
    e = inputs.er_digraph(500, 0.005, 3)
    bits, _ = ctx.tc_closure(e)
    assert np.array_equal(bits, oracle.tc_model(e))


def test_selftest_rejects_bad_budget(ctx):
    assert ctx.selftest_wait_timeout(0.0) == dl.DL_EINVAL
    assert ctx.selftest_wait_timeout(60.0) == dl.DL_EINVAL
