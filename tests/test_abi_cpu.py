"""The C-ABI library builds, loads and exports every symbol include/dl.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1608_00139_gb300 import build as libbuild
from paper_1608_00139_gb300 import dl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdl():
    libbuild.build()
    return dl.lib()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^DL_API\s+[\w\s\*]+?\b(dl_\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_the_abi():
    names = declared_symbols()
    assert {"dl_create", "dl_destroy", "dl_last_error", "dl_tc_closure", "dl_sg_least_model",
            "dl_submit", "dl_poll", "dl_cancel"} <= names
    assert names == set(dl.EXPORTED)


def test_every_declared_symbol_is_exported(libdl):
    out = subprocess.run(["nm", "-D", "--defined-only", dl.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (dl_\w+)$", out, flags=re.M))
    assert declared_symbols() <= exported
    # nothing else leaks out of the library
    assert exported == declared_symbols()
    for name in declared_symbols():
        assert isinstance(getattr(libdl, name), ctypes._CFuncPtr)


def test_null_arguments_are_rejected_without_a_gpu(libdl):
    assert libdl.dl_tc_closure(None, 4, None, 0, 0.0, 0.0, 0, None, None, None) == dl.DL_EINVAL
    assert b"NULL" in libdl.dl_last_error()
    assert libdl.dl_create(None, 0, None) == dl.DL_EINVAL
    assert libdl.dl_destroy(None) == dl.DL_OK


def test_create_fails_cleanly_without_a_gpu(libdl):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dl.DLError) as ei:
        dl.Context(0)
    assert ei.value.status == dl.DL_EDEVICE
