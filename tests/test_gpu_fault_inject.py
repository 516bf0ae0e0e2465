"""Host-side allocation-failure injection (DL_FAULT=alloc@k / alloc@k+): the call whose k-th
allocation fails returns DL_ENOMEM with a message, the context stays usable, and the next call
without the fault gives the oracle's model.  Nothing fails on the GPU: the library declines the
allocation before asking CUDA for it."""
import os

import numpy as np
import pytest

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


class fault:
    def __init__(self, spec):
        self.spec = spec

    def __enter__(self):
        os.environ["DL_FAULT"] = self.spec

    def __exit__(self, *exc):
        os.environ.pop("DL_FAULT", None)


@pytest.mark.parametrize("path", ["auto", "bool_fp8", "fp64", "mixed"])
def test_closure_alloc_failure_and_recovery(path):
    e = inputs.er_digraph(700, 0.006, 3)
    want = oracle.tc_model(e)
    failed = 0
    for k in (1, 2, 3, 4, 6, 9, 14, 20):
        with dl.Context(0) as c:  # a fresh workspace allocates every buffer again
            with fault(f"alloc@{k}"):
                try:
                    bits, _ = c.tc_closure(e, path=path, rtilde=path in ("fp64", "mixed"))[:2]
                    assert np.array_equal(bits, want), k  # k beyond this call's allocations
                except dl.DLError as err:
                    assert err.status == dl.DL_ENOMEM, (k, err)
                    assert err.message
                    failed += 1
            bits, _ = c.tc_closure(e, path=path)  # the same context, no fault
            assert np.array_equal(bits, want), k
    assert failed >= 4


def test_sticky_fault_then_recovery():
    with dl.Context(0) as ctx:  # a fresh workspace: its buffers are still to be allocated
        sticky_case(ctx)


def sticky_case(ctx):
    e = inputs.er_digraph(1500, 0.003, 4)
    with fault("alloc@1+"):
        for path in ("auto", "mixed"):
            with pytest.raises(dl.DLError) as err:
                ctx.tc_closure(e, path=path)
            assert err.value.status == dl.DL_ENOMEM
        with pytest.raises(dl.DLError) as err:
            ctx.sg_least_model(inputs.forest_dag(1500, 4))
        assert err.value.status == dl.DL_ENOMEM
    bits, _ = ctx.tc_closure(e)
    assert np.array_equal(bits, oracle.tc_model(e))
    p = inputs.forest_dag(1500, 4)
    bits, _ = ctx.sg_least_model(p)
    assert np.array_equal(bits, oracle.sg_model(p))


def test_program_alloc_failure(ctx):
    text = "r(X,Y) :- e(X,Y).  r(X,Y) :- e(X,Z), r(Z,Y)."
    e = inputs.er_digraph(600, 0.004, 5)
    prog = ctx.program(text)
    with fault("alloc@1"):
        with pytest.raises(dl.DLError) as err:
            prog.set("e", e)
        assert err.value.status == dl.DL_ENOMEM
    prog.set("e", e)
    with fault("alloc@2+"):
        with pytest.raises(dl.DLError) as err:
            prog.run()
        assert err.value.status == dl.DL_ENOMEM
    prog.run()
    assert np.array_equal(prog.get("r"), oracle.tc_model(e))


def test_serving_alloc_failure():
    e = inputs.pa_dag(2500, 7)
    with dl.Context(0, max_slots=2) as c:
        with fault("alloc@1+"):
            t, h = c.submit(0, e)
            with pytest.raises(dl.DLError) as err:
                c.poll(t, -1)
            assert err.value.status == dl.DL_ENOMEM
        t, h = c.submit(0, e)
        assert c.poll(t, -1)[0] == dl.DL_OK
        assert np.array_equal(h["bits"], oracle.tc_model(e))


def test_unknown_plan_is_ignored(ctx):
    e = inputs.er_digraph(200, 0.01, 6)
    with fault("sometimes"):
        bits, _ = ctx.tc_closure(e)
    assert np.array_equal(bits, oracle.tc_model(e))
