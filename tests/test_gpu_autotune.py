"""The autotuner (dl_autotune): measured choices per size bucket, the JSON cache keyed by GPU,
driver and bucket, and models that stay bit-exact against the oracle under the tuned choices."""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1608_00139_gb300 import dl, inputs

pytestmark = pytest.mark.gpu


def test_tune_cache_and_exact_models(tmp_path):
    cache = str(tmp_path / "tune.json")
    with dl.Context(0, tune_cache=cache) as c:
        for n in (300, 2048):
            r = c.autotune(n)
            assert r["source"] == "measured"
            e = r["entry"]
            assert r["bucket"] == (512 if n == 300 else 2048)
            assert e["sq_bn"] in (128, 256) and e["t_sq_us"] > 0 and e["sweep_gbs"] > 0
            assert e["mx_reserve"] in (16, 32, 48) and e["sg_iteration"] in (-1, 0, 1)
            assert e["mx_pairs"] == -1 if n == 300 else e["mx_pairs"] in (-1, 0, 4, 8, 12, 16)
            assert e["mx_group"] in (2, 4)
            assert c.autotune(n)["source"] == "cache"  # the context's table
        data = json.load(open(cache))
        keys = list(data["entries"])
        assert len(keys) == 2 and all(k.count("|") == 2 for k in keys)
        # the models under the tuned choices
        e = inputs.er_digraph(1900, 0.002, 71)
        want = oracle.tc_model(e)
        for path in ("auto", "bool_fp8", "mixed"):
            assert np.array_equal(c.tc_closure(e, path=path)[0], want), path
        p = inputs.forest_dag(1900, 72)
        assert np.array_equal(c.sg_least_model(p)[0], oracle.sg_model(p))
    # a new context reads the cache: no measurement
    with dl.Context(0, tune_cache=cache) as c2:
        r = c2.autotune(2048)
        assert r["source"] == "cache"
        assert r["entry"] == json.load(open(cache))["entries"][r["key"]]
        assert c2.autotune(2048, force=True)["source"] == "measured"


def test_autotune_on_first_use(tmp_path):
    cache = str(tmp_path / "auto.json")
    e = inputs.er_digraph(700, 0.005, 73)
    with dl.Context(0, autotune=1, tune_cache=cache) as c:
        bits, _ = c.tc_closure(e)  # tunes the 1024 bucket first
        assert np.array_equal(bits, oracle.tc_model(e))
        assert c.autotune(700)["source"] == "cache"
    assert os.path.exists(cache)


def test_large_bucket_keeps_the_rules(ctx):
    r = ctx.autotune(20000)
    assert r["source"].startswith("defaults")


def test_env_cache(tmp_path, monkeypatch):
    cache = str(tmp_path / "env.json")
    monkeypatch.setenv("DL_TUNE_CACHE", cache)
    with dl.Context(0) as c:
        c.autotune(256)
    with dl.Context(0) as c:
        assert c.autotune(256)["source"] == "cache"


@pytest.mark.parametrize("group,grouped", [(4, 16), (4, 8), (2, 16)])
def test_grouped_lu_steps_are_exact(tmp_path, group, grouped):
    """The mixed LU with its first steps in units of 2 or 4 sharing one bulk update (forced through
    a cache entry): bits and R~ against the oracle."""
    cache = str(tmp_path / "g.json")
    with dl.Context(0) as c:
        key = c.autotune(2048)["key"]
    entry = {"sq_bn": 256, "t_sq_us": 20.0, "sweep_gbs": 600.0, "mx_reserve": 32, "mx_pairs": grouped,
             "mx_group": group, "sg_iteration": -1}
    json.dump({"version": 1, "entries": {key: entry}}, open(cache, "w"))
    e = inputs.er_digraph(2000, 0.004, 75)
    with dl.Context(0, tune_cache=cache) as c:
        assert c.autotune(2000)["entry"]["mx_group"] == group
        bits, st, x = c.tc_closure(e, path="mixed", rtilde=True)
    assert np.array_equal(bits, oracle.tc_model(e))
    xr = oracle.tc_rtilde_lu(e, st["eps_used"])
    assert np.abs(x - xr).max() <= 1e-10 * np.abs(xr).max()
