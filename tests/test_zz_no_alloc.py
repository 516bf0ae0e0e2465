"""dl_tc_closure_noalloc: the closure entry point that allocates no device memory.

It serves callers that cannot let a library call cudaMalloc (their device memory belongs to
another framework's pool, or an allocation's implicit synchronisation is not acceptable).
Its scratch is a fixed array inside the library, shared by every call, so this test calls it
twice in a row, on different inputs, through the C ABI, and checks each result against the
ordinary entry point dl_tc_closure and against the CPU oracle's semi-naive least model (the
model is exact: bits must be equal).  After the n = 0 warm-up call, a call must leave the
device's free memory unchanged.  The file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def call_noalloc(e_dev, out):
    n = 0 if e_dev is None else e_dev.shape[0]
    stream = torch.cuda.current_stream()
    sq = ctypes.c_int32(-1)
    rc = dl.lib().dl_tc_closure_noalloc(n, None if e_dev is None else e_dev.data_ptr(),
                                        None if out is None else out.data_ptr(),
                                        ctypes.c_void_p(stream.cuda_stream), ctypes.byref(sq))
    return rc, sq.value


def test_two_calls_in_a_row_match_the_allocating_entry_point_and_the_oracle(ctx):
    rc, _ = call_noalloc(None, None)  # warm-up: places the scratch, loads the kernels
    assert rc == dl.DL_OK, dl.lib().dl_last_error()
    cases = [inputs.er_digraph(2048, 1e-3, 71), inputs.er_digraph(1000, 4e-3, 72)]
    for e in cases:  # the second call sees the first call's leftovers in the scratch
        n = e.shape[0]
        e_dev = torch.from_numpy(e).cuda()
        out = torch.zeros((n, dl.words(n)), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        rc, sq = call_noalloc(e_dev, out)
        free_after, _ = torch.cuda.mem_get_info()
        assert rc == dl.DL_OK, dl.lib().dl_last_error()
        assert free_after == free_before  # nothing allocated on the device by the call
        assert sq >= 1
        ref, st = ctx.tc_closure(e_dev, path="bool_fp8")
        assert torch.equal(out, ref)
        assert sq == st["iters"]
        want = oracle.tc_model(e)
        assert np.array_equal(out.cpu().numpy().view(np.uint64), want)


def test_rejects_sizes_beyond_the_fixed_scratch():
    n = dl.NOALLOC_MAX_N + 1
    e_dev = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    out = torch.zeros((n, dl.words(n)), dtype=torch.int64, device="cuda")
    rc, _ = call_noalloc(e_dev, out)
    assert rc == dl.DL_EINVAL
    assert b"2048" in dl.lib().dl_last_error()
