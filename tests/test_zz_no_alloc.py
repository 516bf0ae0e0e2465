"""dl_tc_closure_noalloc: the closure entry point that allocates no device memory.

It serves callers that cannot let a library call cudaMalloc (their device memory belongs to
another framework's pool, or an allocation's implicit synchronisation is not acceptable).
Its scratch is a fixed array inside the library, shared by every call, so this test calls it
twice in a row, on different inputs, through the C ABI, and checks each result against the
ordinary entry point dl_tc_closure (the model is exact: bits must be equal).  The file is
named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def call_noalloc(e_dev: torch.Tensor):
    n = e_dev.shape[0]
    out = torch.zeros((n, dl.words(n)), dtype=torch.int64, device=e_dev.device)
    stream = torch.cuda.current_stream(e_dev.device)
    sq = ctypes.c_int32(-1)
    rc = dl.lib().dl_tc_closure_noalloc(n, e_dev.data_ptr(), out.data_ptr(),
                                        ctypes.c_void_p(stream.cuda_stream), ctypes.byref(sq))
    return rc, out, sq.value


def test_two_calls_in_a_row_match_the_allocating_entry_point(ctx):
    cases = [inputs.er_digraph(2048, 1e-3, 71), inputs.er_digraph(1000, 4e-3, 72)]
    for e in cases:  # the second call sees the first call's leftovers in the scratch
        e_dev = torch.from_numpy(e).cuda()
        rc, out, sq = call_noalloc(e_dev)
        assert rc == dl.DL_OK, dl.lib().dl_last_error()
        assert sq >= 1
        ref, st = ctx.tc_closure(e_dev, path="bool_fp8")
        assert torch.equal(out, ref)
        assert sq == st["iters"]


def test_rejects_sizes_beyond_the_fixed_scratch():
    n = dl.NOALLOC_MAX_N + 1
    e_dev = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    rc, _, _ = call_noalloc(e_dev)
    assert rc == dl.DL_EINVAL
    assert b"2048" in dl.lib().dl_last_error()
