"""Benchmark: transitive-closure least models at N = 8192 on one GB300 (and N GPUs as replicas).

Workload (a step): the least models of r2 <- r1; r2 <- r1, r2 (Sec. 3) for three seeded
Erdos-Renyi digraphs with N = 8192 and p = 1e-4, 1e-3, 1e-2 (seeds 2, 3, 4; i != j), the
paper's ER workload shape (Sec. 7.1).  Metric: TFLOP/s-equivalent = (8/3) N^3 per model
(the cost of the dense direct solve of Proposition 1) / wall time, whole job.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

`value`: inputs resident in HBM (three 64 MiB matrices, 192 MiB > the 129 MB L2, each read in
every step), one C-ABI call per model on the AUTO path (single-row Iteration, bit sweeps, FP8
tensor-core squarings by cost), 3 x INFLIGHT closures in flight.  `e2e`: the same through
host buffers (H2D of E and D2H of the model bits inside the timed region).  The plain FP64
path (Proposition 1 in FP64) is timed beside it for the "vs plain FP64" comparison.
`--impl reference` times the CPU oracle (semi-naive evaluation) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 8192
INFLIGHT = 3  # contexts per model in the headline step (closures in flight = 3 x INFLIGHT)
PS = (1e-4, 1e-3, 1e-2)
SEEDS = (2, 3, 4)
METRIC = "TC least-model TFLOP/s-equiv (N=8192) vs plain FP64 path; served p50/p99 latency"
UNIT = "TFLOP/s-equiv"


# DRAM bytes per launch from the ncu captures summarised under profiles/; each is only valid
# for the kernel source it was taken on (sha256 prefixes).
TRAFFIC = {
    "gemm": {"sources": {"dl_umma.cu": "f47fffb50b28217c", "dl_ptx.cuh": "b4fd45714c88d2fc"},
             "bytes_per_launch": 177.5e6},   # ncu: DRAM read + write of one dense N = 8192 squaring
    "sweep": {"sources": {"dl_bool.cu": "4e1ad3c162a9b14b"},
              "bytes_per_launch": 8.70e6},    # ncu: one working sweep, p = 1e-3, cold L2
}


def traffic(kind: str):
    import hashlib
    csrc = os.path.join(ROOT, "paper_1608_00139_gb300", "csrc")
    for f, h in TRAFFIC[kind]["sources"].items():
        if h is None:
            continue
        with open(os.path.join(csrc, f), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != h:
                return None  # kernel changed since the counters were taken
    return TRAFFIC[kind]["bytes_per_launch"]


def flops_equiv(n: int) -> float:
    return (8.0 / 3.0) * float(n) ** 3


def peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16": float(d["bf16_tflops"]), "bf16_sustained": float(d["bf16_tflops_sustained"]),
                "hbm": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"bf16": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "fallback"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def graph_seeds(rank: int):
    """(p, seed) of each model a rank solves: every rank its own seeded replica."""
    return [(p, s + 1000 * rank) for p, s in zip(PS, SEEDS)]


def graphs(rank: int):
    from paper_1608_00139_gb300 import inputs
    return [inputs.er_digraph(N, p, s) for p, s in graph_seeds(rank)]


FRESH_K = 4  # graphs per p in the fresh-input leg (the headline's and three more seeds)


def fresh_seeds(rank: int):
    """Seeds of the fresh-input leg: for each p, the headline's seed and FRESH_K - 1 others."""
    return [[s + 10007 * r for r in range(FRESH_K)] for _, s in graph_seeds(rank)]


def max_over_ranks(values, world: int, device: str):
    """Element-wise maximum of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as tdist
    t = torch.tensor(list(values), device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running; entering
    waits (up to 5 s) for the first sample so that the sampler is live when timing starts."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return self
        deadline = time.perf_counter() + 5.0
        while time.perf_counter() < deadline and self.proc.poll() is None:
            self.tmp.flush()
            if os.path.getsize(self.tmp.name) > 0:
                break
            time.sleep(0.02)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [int(r[1]) for r in rows]
        smax = max(int(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def bench_sg(ctx, torch, reps: int = 10) -> dict:
    """Same generation on the N = 4096 forest + DAG edges (seed 5), device-resident input."""
    from paper_1608_00139_gb300 import inputs
    p = torch.from_numpy(inputs.forest_dag(4096, 5)).cuda()
    torch.cuda.synchronize()
    ctx.sg_least_model(p)
    t0 = time.perf_counter()
    for _ in range(reps):
        _, st = ctx.sg_least_model(p)
    ms = (time.perf_counter() - t0) / reps * 1e3
    return {"workload": "SG forest+DAG N=4096 seed 5", "ms": ms, "doubling_steps": st["iters"],
            "gemm_tflops": st["gemm_flops"] / (st["ms_gemm"] * 1e-3) / 1e12 if st["ms_gemm"] else None,
            "device_ms": st["ms_total"]}


SG_REAL_N = 4096


def bench_sg_real(ctx, torch, reps: int = 5) -> dict:
    """Real S~ = eps (I + P S~ P^T) of same generation on the N = 4096 forest + DAG (seed 5),
    device-resident input and outputs: the FP64 series on the GPU (exact after depth + 1 steps
    on this nilpotent P), plus the certified model bits.  Roofline of one series step (one pass
    of sg_fused_kernel here, at most two parents per node): a step must read the iterate and
    write the next one, 2 Np^2 x 8 bytes (the kernel reads X a second time for the change)."""
    from paper_1608_00139_gb300 import inputs
    p = torch.from_numpy(inputs.forest_dag(SG_REAL_N, 5)).cuda()
    torch.cuda.synchronize()
    ctx.sg_real(p)
    t0 = time.perf_counter()
    for _ in range(reps):
        _, _, st = ctx.sg_real(p)
    ms = (time.perf_counter() - t0) / reps * 1e3
    npad = (SG_REAL_N + 255) // 256 * 256
    step_bytes = 2.0 * npad * npad * 8
    pk = peaks()
    gbs = st["iters"] * step_bytes / (st["ms_solve"] * 1e-3) / 1e9 if st["ms_solve"] > 0 else None
    # the same S~ by Smith's doubling on the TF32 tensor cores with FP64 refinement
    ctx.sg_real(p, path="mixed", bits=False)
    t0 = time.perf_counter()
    _, _, sm = ctx.sg_real(p, path="mixed", bits=False)
    mixed = {"ms": (time.perf_counter() - t0) * 1e3, "refine_steps": sm["iters"], "final_resid": sm["final_resid"],
             "gemm_launches": sm["gemm_launches"],
             "gemm_tflops": sm["gemm_flops"] / (sm["ms_gemm"] * 1e-3) / 1e12 if sm["ms_gemm"] else None}
    return {"workload": "SG S~ forest+DAG N=4096 seed 5", "ms": ms, "device_ms": st["ms_total"],
            "mixed_path": mixed,
            "path_used": "fp64 series" if st["path_used"] == 1 else "mixed refinement",
            "series_steps": st["iters"], "final_resid": st["final_resid"], "ms_series": st["ms_solve"],
            "ms_model_bits": st["ms_epilogue"],
            "roofline": {"bound": "hbm", "kernel": "sg_fused_kernel (one series step)",
                         "achieved": gbs, "peak": pk["hbm"], "unit": "GB/s",
                         "frac": gbs / pk["hbm"] if gbs else None, "bytes_per_step": step_bytes,
                         "peak_source": pk["source"]}}


def bench_tail(ctx, torch, reps: int = 5) -> dict:
    """One equation of the tail recursive class, R~ = eps (A + B0 R~), at N = 8192: B0 the ER
    graph with p = 1e-3 (seed 3), A the one with p = 1e-4 (seed 2), device-resident.  The model
    (closure of B0 by AUTO, then one FP8 product) and R~ on the mixed path."""
    from paper_1608_00139_gb300 import inputs
    b0 = torch.from_numpy(inputs.er_digraph(N, 1e-3, 3)).cuda()
    a = torch.from_numpy(inputs.er_digraph(N, 1e-4, 2)).cuda()
    torch.cuda.synchronize()
    out = {"workload": "tail recursive R~ = eps (A + B0 R~), N=8192, B0 ER p=1e-3 seed 3, A ER p=1e-4 seed 2"}
    for path, reps_p in (("auto", reps), ("mixed", 2)):
        rt = path == "mixed"  # the mixed path with its R~ output (device buffer)
        ctx.tail_recursive(b0, a, path=path, rtilde=rt)
        t0 = time.perf_counter()
        for _ in range(reps_p):
            st = ctx.tail_recursive(b0, a, path=path, rtilde=rt)[1]
        out[path] = {"ms": (time.perf_counter() - t0) / reps_p * 1e3, "device_ms": st["ms_total"],
                     "model_ones": st["model_ones"], "gemm_launches": st["gemm_launches"]}
        if path == "mixed":
            out[path].update({"refine_steps": st["iters"], "final_resid": st["final_resid"],
                              "rows_rechecked": st["rows_rechecked"]})
    return out


TRANS_N = 4096


def bench_trans(ctx, torch, reps: int = 5) -> dict:
    """The transposed class, r2(x,z) <- r1(x,z); r2(x,z) <- r1(x,y), r2(z,y) (Sec. 6.2), on the
    ER graph N = 4096, p = 1e-3 (seed 8), device-resident: the model (two-sided reduction) and
    the real R~2 by the FP64 series."""
    from paper_1608_00139_gb300 import inputs
    r1 = torch.from_numpy(inputs.er_digraph(TRANS_N, 1e-3, 8)).cuda()
    torch.cuda.synchronize()
    out = {"workload": f"transposed class prog:2, ER N={TRANS_N} p=1e-3 seed 8"}
    ctx.transposed(r1)
    t0 = time.perf_counter()
    for _ in range(reps):
        _, st = ctx.transposed(r1)
    out["model"] = {"ms": (time.perf_counter() - t0) / reps * 1e3, "device_ms": st["ms_total"],
                    "model_ones": st["model_ones"], "gemm_launches": st["gemm_launches"]}
    ctx.transposed(r1, rtilde=True)
    t0 = time.perf_counter()
    _, st, _ = ctx.transposed(r1, rtilde=True)
    npad = (TRANS_N + 255) // 256 * 256
    step_bytes = 3.0 * npad * npad * 8  # a step reads X, writes X^T, writes the next X
    gbs = st["iters"] * step_bytes / (st["ms_refine"] * 1e-3) / 1e9 if st["ms_refine"] > 0 else None
    pk = peaks()
    out["rtilde"] = {"ms": (time.perf_counter() - t0) * 1e3, "series_steps": st["iters"],
                     "final_resid": st["final_resid"], "ms_series": st["ms_refine"],
                     "roofline": {"bound": "hbm", "kernel": "one series step (transpose + gather pass)",
                                  "achieved": gbs, "peak": pk["hbm"], "unit": "GB/s",
                                  "frac": gbs / pk["hbm"] if gbs else None, "bytes_per_step": step_bytes}}
    return out


def cpu_trans() -> dict:
    """The oracle on the transposed workload: semi-naive model and the FP64 series (numpy/scipy)."""
    from oracle import transposed as tr
    from paper_1608_00139_gb300 import inputs
    r1 = inputs.er_digraph(TRANS_N, 1e-3, 8)
    t0 = time.perf_counter()
    tr.trans_model(r1)
    t1 = time.perf_counter()
    tr.trans_rtilde_series(r1, tol=1e-13 * tr.trans_eps(r1))
    t2 = time.perf_counter()
    return {"model_ms": (t1 - t0) * 1e3, "rtilde_ms": (t2 - t1) * 1e3, "kind": "oracle", "cores": 1,
            "sample": "the whole N = 4096 workload"}


def cpu_tail() -> dict:
    """The oracle on the tail recursive workload: rows of the model by breadth-first search (the
    whole-model oracle needs dense products at N = 8192), a bounded sample scaled to N rows."""
    import oracle
    from paper_1608_00139_gb300 import inputs
    b0 = inputs.er_digraph(N, 1e-3, 3)
    a = inputs.er_digraph(N, 1e-4, 2)
    rows = list(range(0, N, N // 64))
    t0 = time.perf_counter()
    oracle.tail_model_rows(b0, a, rows)
    ms = (time.perf_counter() - t0) * 1e3
    return {"ms_per_row": ms / len(rows), "ms_full_estimate": ms / len(rows) * N, "kind": "oracle",
            "cores": 1, "sample": f"{len(rows)} of {N} rows by breadth-first search, scaled to {N} rows"}


def cpu_sg_real() -> dict:
    """The oracle's S~ (FP64 fixpoint series, sparse P) on the same workload, host cores."""
    import oracle
    from paper_1608_00139_gb300 import inputs
    p = inputs.forest_dag(SG_REAL_N, 5)
    t0 = time.perf_counter()
    _, it = oracle.sg_stilde_series(p, return_iters=True)
    return {"ms": (time.perf_counter() - t0) * 1e3, "kind": "oracle", "steps": it,
            "sample": "the whole N = 4096 workload"}


def bench_batch(ctx, torch, reps: int = 10) -> dict:
    """1024 uneven ER closures (N ~ U{32..2048}, mean degree ~ U[1,8], seeds 1000+k), resident
    back to back in one device buffer; each call writes every model to one device buffer."""
    from concurrent.futures import ThreadPoolExecutor

    from paper_1608_00139_gb300 import inputs
    specs = inputs.batch_specs(1024, 1000)
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        host = list(ex.map(lambda s: inputs.er_digraph(s[0], s[1], s[2]), specs))
    ns = np.array([e.shape[0] for e in host], dtype=np.int32)
    sizes = ns.astype(np.int64) ** 2
    offsets = np.concatenate(([0], np.cumsum((sizes + 255) // 256 * 256)[:-1])).astype(np.uint64)
    flat = np.zeros(int(offsets[-1]) + int(sizes[-1]), dtype=np.uint8)
    for e, o in zip(host, offsets):
        flat[int(o):int(o) + e.size] = e.reshape(-1)
    dev = torch.from_numpy(flat).cuda()
    torch.cuda.synchronize()
    ctx.tc_batch_flat(dev, ns, offsets)  # captures the graph
    t0 = time.perf_counter()
    for _ in range(reps):
        _, _, st = ctx.tc_batch_flat(dev, ns, offsets)
    ms = (time.perf_counter() - t0) / reps * 1e3
    equiv = sum(flops_equiv(n) for n, _, _ in specs)
    return {"workload": "1024 ER closures, N~U{32..2048}, degree~U[1,8]", "ms": ms,
            "tflops_equiv": equiv / (ms * 1e-3) / 1e12, "rounds": st["iters"],
            "tensor_tflops": st["gemm_flops"] / (ms * 1e-3) / 1e12, "device_ms": st["ms_total"],
            "inputs": "one resident device buffer (1.4 GB), one device output buffer"}


def bench_serving(dl, torch, device: int, seconds: float, slots: int = 4) -> dict:
    """The serving workload: a Poisson stream at 200 req/s for `seconds` (seed 6), 80% closure /
    20% same generation, each request a fresh seeded preferential-attachment DAG (N log-uniform
    in [512, 16384], the stream's own seed per request) generated ahead of its arrival into a
    ring of pinned host buffers.  Inputs go in as host memory and models come back to pinned
    host memory, so each latency holds the H2D copy of the input, the solve and the D2H copy of
    the model.  Latency: dl_submit -> completion (the library's host clock) and arrival ->
    completion (adds any lag of the submitting thread behind the arrival time)."""
    import threading
    from concurrent.futures import ThreadPoolExecutor

    from paper_1608_00139_gb300 import inputs
    times, kinds, ns, seeds = inputs.poisson_stream(200.0, seconds, 6)
    count = len(times)
    nmax, ring = 16384, 24
    wmax = (nmax + 63) // 64
    in_buf = [torch.empty(nmax * nmax, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(ring)]
    out_buf = [torch.empty(nmax * wmax, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
               for _ in range(ring)]
    free = list(range(ring))
    turn = [0]  # slots go to requests in arrival order, so the ring never holds a later request
    cv = threading.Condition()  # while an earlier one waits (no deadlock with in-order submits)
    inputs.pa_dag_into(np.empty((2, 2), np.uint8), 0)  # build / load the generator first

    def take(r):
        with cv:
            while not free or turn[0] != r:
                cv.wait()
            turn[0] += 1
            cv.notify_all()
            return free.pop()

    def give(slot):
        with cv:
            free.append(slot)
            cv.notify_all()

    def make(r):  # generate request r into a ring slot (ahead of its arrival)
        slot = take(r)
        n = int(ns[r])
        inputs.pa_dag_into(in_buf[slot][:n * n].reshape(n, n), int(seeds[r]))
        return slot

    gen = ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4))
    lat, lat_arr, queue, spans, errors, lag = [], [], [], [], 0, []
    with dl.Context(device, max_slots=slots) as c:
        # untimed warm-up at the stream's largest size, both kinds, on the default route and on the
        # tensor-core route AUTO takes for some graphs (squarings, doubling), enough requests to
        # reach every slot: the slots' workspaces (grow-only) are sized before the stream, so no
        # request in it pays for an allocation (and a cudaFree, which waits for the whole GPU)
        big = inputs.pa_dag_into(np.empty((nmax, nmax), np.uint8), 1)
        for route in ("bool_fp8", "auto"):
            warm = [c.submit(k, big, path=route) for k in (0, 1) for _ in range(slots)]
            for tk, _ in warm:
                c.poll(tk, -1)
        futs = [gen.submit(make, r) for r in range(count)]  # the ring bounds how far ahead
        outstanding = {}  # ticket -> (slot, handle, request, submit time)

        def reap(block: bool):
            nonlocal errors
            done = []
            for tk, (slot, h, r, ts) in outstanding.items():
                try:
                    rc, st = c.poll(tk, -1 if block else 0)
                except dl.DLError:
                    errors += 1
                    done.append(tk)
                    give(slot)
                    continue
                if rc != dl.DL_OK:
                    continue
                lat.append(st["ms_latency"])
                queue.append(st["ms_queue"])
                lat_arr.append(st["ms_latency"] + (ts - times[r]) * 1e3)
                spans.append((ts + st["ms_queue"] * 1e-3, ts + st["ms_latency"] * 1e-3))
                done.append(tk)
                give(slot)
            for tk in done:
                outstanding.pop(tk)

        t0 = time.perf_counter()
        for r in range(count):
            # completions free ring slots, so keep reaping while request r is generated or early
            while not futs[r].done() or time.perf_counter() - t0 < times[r]:
                reap(False)
                time.sleep(min(0.0005, max(0.0002, times[r] - (time.perf_counter() - t0))))
            slot = futs[r].result()
            n = int(ns[r])
            ts = time.perf_counter() - t0
            lag.append(ts - times[r])
            tk, h = c.submit(int(kinds[r]), in_buf[slot][:n * n].reshape(n, n),
                             out=out_buf[slot][:n * ((n + 63) // 64)].reshape(n, (n + 63) // 64))
            outstanding[tk] = (slot, h, r, ts)
        while outstanding:
            reap(True)
        wall = time.perf_counter() - t0
    gen.shutdown()
    # admitted concurrency: requests between admission and completion at the same time
    ev = sorted([(a, 1) for a, _ in spans] + [(b, -1) for _, b in spans])
    cur, peak, area = 0, 0, 0.0
    for (t_a, d), (t_b, _) in zip(ev, ev[1:] + [(ev[-1][0], 0)]):
        cur += d
        peak = max(peak, cur)
        area += cur * (t_b - t_a)
    lat_a, arr_a = np.array(lat), np.array(lat_arr)
    return {"workload": f"Poisson 200 req/s for {seconds:g} s (seed 6), 80% TC / 20% SG, a fresh seeded "
                        f"PA DAG per request, N log-uniform in [512,16384]",
            "inputs": "host (pinned) input and output per request: H2D and D2H inside each latency",
            "requests": int(count), "completed": int(len(lat)), "errors": errors,
            "p50_ms": float(np.percentile(lat_a, 50)), "p99_ms": float(np.percentile(lat_a, 99)),
            "p50_arrival_ms": float(np.percentile(arr_a, 50)), "p99_arrival_ms": float(np.percentile(arr_a, 99)),
            "p50_queue_ms": float(np.percentile(np.array(queue), 50)),
            "max_submit_lag_ms": float(max(lag) * 1e3), "solves_per_s": len(lat) / wall,
            "slots": slots, "admitted_concurrency": {"peak": peak, "mean": area / max(wall, 1e-9)},
            "mean_n": float(ns.mean()), "h2d_bytes": int((ns.astype(np.int64) ** 2).sum())}


def mixed_leg(ctx, dev) -> dict:
    """The mixed path (TF32 tensor-core LU, W = A^-1, FP64 refinement) on the three N = 8192
    graphs: with the R~ output (refined to max|R| <= 1e-13 eps, device buffer) and for the model
    alone (the solve, then threshold, certificate and recheck; no refinement)."""
    out = {}
    for name, x in zip(("p=1e-4", "p=1e-3", "p=1e-2"), dev):
        ctx.tc_closure(x, path="mixed", rtilde=True)  # warm
        _, stm, _ = ctx.tc_closure(x, path="mixed", rtilde=True)
        ctx.tc_closure(x, path="mixed")
        _, sto = ctx.tc_closure(x, path="mixed")
        out[name] = {"ms": stm["ms_total"], "tflops_equiv": stm["tflops_equiv"],
                     "refine_steps": stm["iters"], "final_resid": stm["final_resid"],
                     "ms_factor": stm["ms_factor"], "ms_solve": stm["ms_solve"],
                     "ms_refine": stm["ms_refine"], "guard_flagged": stm["guard_flagged"],
                     "rechecked_rows": stm["rows_rechecked"],
                     "tf32_tflops": stm["gemm_flops"] / (stm["ms_total"] * 1e-3) / 1e12,
                     "model_only": {"ms": sto["ms_total"], "tflops_equiv": sto["tflops_equiv"],
                                    "ms_factor": sto["ms_factor"], "ms_solve": sto["ms_solve"],
                                    "ms_refine": sto["ms_refine"], "guard_flagged": sto["guard_flagged"],
                                    "rechecked_rows": sto["rows_rechecked"]}}
    return out


def cpu_baseline(gs, budget_s: float = 30.0) -> dict:
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    done = 0
    for e in gs:
        oracle.tc_model(e)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done * flops_equiv(N) / dt / 1e12, "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": f"{done} of the 3 N=8192 graphs (one full step), semi-naive evaluation, "
                      f"{dt:.2f} s"}


def cpu_rows() -> dict:
    """The oracle timed on the other configured workloads, on this host's cores (bounded: about
    30 s in all).  Each entry states its sample, its thread count and its rate."""
    import oracle
    from paper_1608_00139_gb300 import inputs
    allc = oracle.set_threads(os.cpu_count() or 1)
    out = {"host_cores": os.cpu_count(), "cpu": _cpu_model()}

    def timed(f, *a):
        t0 = time.perf_counter()
        f(*a)
        return time.perf_counter() - t0

    # C1: the plain FP64 direct solve (Prop. 1, unpivoted LU + n right-hand sides), all cores
    e1 = inputs.er_digraph(256, 0.02, 1)
    dt = timed(oracle.tc_rtilde_lu, e1, oracle.tc_eps(e1))
    out["fp64_lu_er256"] = {"ms": dt * 1e3, "tflops_equiv": flops_equiv(256) / dt / 1e12, "threads": allc,
                            "sample": "the whole N = 256 workload (ER p = 0.02, seed 1)"}
    # C2: the FP64 solve on a bounded sample (N = 2048 at the p = 1e-3 graph's mean degree; the
    # N = 8192 solve is 64 times this work), and the semi-naive model single-threaded per graph
    e2 = inputs.er_digraph(2048, 8.2 / 2047, 3)
    dt = timed(oracle.tc_rtilde_lu, e2, oracle.tc_eps(e2))
    out["fp64_lu_er8192_sample"] = {"ms": dt * 1e3, "tflops_equiv": flops_equiv(2048) / dt / 1e12,
                                    "ms_n8192_estimate": dt * 64e3, "threads": allc,
                                    "sample": "LU solve at N = 2048, mean degree 8.2 (1/64 of the N = 8192 work)"}
    oracle.set_threads(1)
    one = {}
    for p, sd in zip(PS, SEEDS):
        one[f"p={p:g}"] = timed(oracle.tc_model, inputs.er_digraph(N, p, sd)) * 1e3
    out["seminaive_er8192_1thread"] = {"ms": one, "threads": 1,
                                       "tflops_equiv": 3 * flops_equiv(N) / (sum(one.values()) * 1e-3) / 1e12,
                                       "sample": "the three N = 8192 graphs, one thread"}
    oracle.set_threads(allc)
    # C3: same generation, semi-naive, the whole N = 4096 forest workload
    p3 = inputs.forest_dag(4096, 5)
    dt = timed(oracle.sg_model, p3)
    out["sg_seminaive_forest4096"] = {"ms": dt * 1e3, "threads": allc, "sample": "the whole workload"}
    # C4: the oracle over every instance of the uneven batch (summed)
    specs = inputs.batch_specs(1024, 1000)
    gs4 = [inputs.er_digraph(n, p, sd) for n, p, sd in specs]
    dt = timed(lambda: [oracle.tc_model(g) for g in gs4])
    out["batch_1024_summed"] = {"ms": dt * 1e3, "threads": allc,
                                "tflops_equiv": sum(flops_equiv(n) for n, _, _ in specs) / dt / 1e12,
                                "sample": "all 1024 instances, one after another"}
    # C5: the first 100 requests of the seeded serving stream, solved one after another
    _, kinds, ns, seeds = inputs.poisson_stream(200.0, 60.0, 6)
    t_tc = t_sg = 0.0
    k_tc = k_sg = 0
    for r in range(100):
        g = inputs.pa_dag_into(np.empty((int(ns[r]), int(ns[r])), np.uint8), int(seeds[r]))
        if kinds[r] == 0:
            t_tc += timed(oracle.tc_model, g)
            k_tc += 1
        else:
            t_sg += timed(oracle.sg_model, g)
            k_sg += 1
    out["serving_sample"] = {"solves_per_s": 100 / (t_tc + t_sg), "tc_ms_mean": t_tc / max(k_tc, 1) * 1e3,
                             "sg_ms_mean": t_sg / max(k_sg, 1) * 1e3, "threads": allc,
                             "sample": f"the first 100 requests of the seeded 200 req/s stream ({k_tc} TC, {k_sg} SG; "
                                       f"mean N {float(ns[:100].mean()):.0f}), generation excluded"}
    return out


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    import oracle
    gs = graphs(0)
    threads = oracle.set_threads(os.cpu_count() or 1)
    # each step solves one of the three graphs in turn (a third of the GPU arm's step), so that
    # the default number of steps ends within a few minutes; the value counts the work done
    for i in range(args.warmup):
        oracle.tc_model(gs[i % len(gs)])
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.tc_model(gs[i % len(gs)])
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = flops_equiv(N) / dt / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded Erdos-Renyi, i != j)",
            "config": {"workload": "TC ER N=8192 x p in {1e-4,1e-3,1e-2}, seeds 2/3/4"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "each step one of the 3 N=8192 graphs in turn (p = 1e-4, 1e-3, "
                                       "1e-2), semi-naive evaluation"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_part(args, device: int) -> None:
    """One secondary measurement on its own (same functions as the full run, with the same
    autotuned choices unless --no-tune)."""
    import torch

    from paper_1608_00139_gb300 import dl
    torch.cuda.set_device(device)
    if not args.no_tune:  # every context of this process reads the tuned table (DL_TUNE_CACHE)
        os.environ["DL_TUNE_CACHE"] = os.path.join(tempfile.gettempdir(), f"dl_tune_{os.getpid()}_part.json")
        with dl.Context(device) as tctx:
            for nb in (N, 4096):
                tctx.autotune(nb)
    if args.part == "serving":
        out = bench_serving(dl, torch, device, args.serve_seconds)
    elif args.part == "mixed":
        with dl.Context(device) as ctx:
            out = mixed_leg(ctx, [torch.from_numpy(e).cuda() for e in graphs(0)])
    elif args.part == "bool":
        # the squarings-only FP8 path on the three graphs (the FP8 GEMM's profiling workload)
        out = {}
        with dl.Context(device) as ctx:
            gs = [torch.from_numpy(e).cuda() for e in graphs(0)]
            for x in gs:
                ctx.tc_closure(x, path="bool_fp8")  # warm
            for name, x in zip(("p=1e-4", "p=1e-3", "p=1e-2"), gs):
                _, stb = ctx.tc_closure(x, path="bool_fp8")
                out[name] = {"ms": stb["ms_total"], "squarings": stb["iters"], "ms_gemm": stb["ms_gemm"],
                             "gemm_tflops": stb["gemm_flops"] / (stb["ms_gemm"] * 1e-3) / 1e12}
    elif args.part == "sg_real":
        with dl.Context(device) as ctx:
            out = bench_sg_real(ctx, torch)
    elif args.part == "tail":
        with dl.Context(device) as ctx:
            out = bench_tail(ctx, torch)
    elif args.part == "trans":
        with dl.Context(device) as ctx:
            out = bench_trans(ctx, torch)
    else:
        with dl.Context(device) as ctx:
            out = bench_sg(ctx, torch) if args.part == "sg" else bench_batch(ctx, torch, reps=max(1, args.steps))
    print(json.dumps({"part": args.part, args.part: out}), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="auto", choices=["auto", "bool_fp8"],
                    help="closure path of the headline (auto: squarings + sweeps by cost)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the squarings-only FP8 comparison run")
    ap.add_argument("--no-fresh", action="store_true",
                    help="skip the leg that rotates seeded graphs across solves")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the fixed rules instead of the autotuner's measured choices")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the same-generation, batch and serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the serving stream (the configured workload is 60 s)")
    ap.add_argument("--part", default="all", choices=["all", "sg", "sg_real", "tail", "trans", "batch", "serving", "mixed", "bool"],
                    help="run one secondary measurement alone and print its JSON (for profiling)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.part != "all":
        run_part(args, local)
        return

    import torch
    import torch.distributed as tdist

    from paper_1608_00139_gb300 import dl

    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl")
    from concurrent.futures import ThreadPoolExecutor
    gs = graphs(rank)
    dev = [torch.from_numpy(e).cuda() for e in gs]
    # pinned host copies for the end-to-end leg (inputs and outputs)
    host, host_bits, host_out = [], [], []
    for e in gs:
        t = torch.empty(e.shape, dtype=torch.uint8, pin_memory=True)
        t.numpy()[:] = e
        host.append(t.numpy())
        # the same E bit-packed (row-major, LSB first), for the packed-input end-to-end leg
        packed = np.packbits(e, axis=1, bitorder="little").view(np.uint64)
        tb = torch.empty(packed.shape, dtype=torch.int64, pin_memory=True)
        tb.numpy().view(np.uint64)[:] = packed
        host_bits.append(tb.numpy().view(np.uint64))
    # INFLIGHT contexts per model (one stream and host thread each): every context solves its
    # model back to back, so 3 x INFLIGHT closures are in flight; a step is still one solve of
    # each of the three models (the contexts of a model share its solves)
    nctx = len(gs) * INFLIGHT
    model_of = [i % len(gs) for i in range(nctx)]
    for _ in range(nctx):
        o = torch.empty((N, (N + 63) // 64), dtype=torch.int64, pin_memory=True)
        host_out.append(o.numpy().view(np.uint64))
    # device outputs allocated once (a step writes every word of each)
    dev_out = [torch.empty((N, (N + 63) // 64), dtype=torch.int64, device="cuda") for _ in range(nctx)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(nctx)]
    # the autotuner: measured choices for the sizes the step and the extra legs use, kept in a
    # cache file that every context of this run reads when it is created
    tuned = None
    if not args.no_tune:  # every context of this process reads the tuned table (DL_TUNE_CACHE)
        os.environ["DL_TUNE_CACHE"] = os.path.join(tempfile.gettempdir(), f"dl_tune_{os.getpid()}_{rank}.json")
        with dl.Context(local) as tctx:
            tuned = {str(nb): tctx.autotune(nb)["entry"] for nb in (N, 4096)}
    ctxs = [dl.Context(local, stream=st_) for st_ in streams]
    pool = ThreadPoolExecutor(max_workers=nctx)
    main_stream = torch.cuda.current_stream()

    def outs_for(inputs):
        return dev_out if inputs is dev else host_out

    # fresh-input leg: FRESH_K seeded graphs per p, each context moving to another graph of its
    # p on every solve, so no closure starts from a workspace that just solved the same input
    fresh = None
    fresh_count = [0] * nctx
    if not args.no_fresh:
        from paper_1608_00139_gb300 import inputs as gen
        with ThreadPoolExecutor(max_workers=8) as ex:
            fresh = [list(ex.map(lambda sd, p=p: torch.from_numpy(gen.er_digraph(N, p, sd)).cuda(), seeds))
                     for p, seeds in zip(PS, fresh_seeds(rank))]

    def solve(i, inputs, path):
        if inputs is fresh:
            m, c = model_of[i], fresh_count[i]
            fresh_count[i] += 1
            return ctxs[i].tc_closure(fresh[m][(i // len(gs) + c) % FRESH_K], path=path, out=dev_out[i])
        if inputs is host_bits:
            return ctxs[i].tc_closure_bits(inputs[model_of[i]], N, path=path, out=host_out[i])
        return ctxs[i].tc_closure(inputs[model_of[i]], path=path, out=outs_for(inputs)[i])

    def step(inputs, path=args.path):
        return list(pool.map(lambda i: solve(i, inputs, path), range(nctx)))

    def timed(inputs, path, k):
        """Device time of k steps: events fork/join the contexts' streams; each host thread
        drives its share of its model's k solves back to back."""
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ends = [torch.cuda.Event() for _ in streams]
        torch.cuda.synchronize()
        ev0.record(main_stream)
        for st_ in streams:
            st_.wait_event(ev0)

        def run(i):
            share = k // INFLIGHT + (1 if i // len(gs) < k % INFLIGHT else 0)
            return [solve(i, inputs, path)[1] for _ in range(share)]

        per_ctx = list(pool.map(run, range(nctx)))
        for e_, st_ in zip(ends, streams):
            e_.record(st_)
            main_stream.wait_event(e_)
        ev1.record(main_stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), [st for sts in per_ctx for st in sts]

    for _ in range(max(args.warmup, 3)):
        step(dev)
    with ClockSampler(local) as clk:
        if world > 1:
            tdist.barrier()
        ms_total, stats = timed(dev, args.path, args.steps)
        if world > 1:
            tdist.barrier()
        # end to end through pinned host buffers (H2D of E, D2H of bits inside the timed region)
        e2e_steps = max(1, min(args.steps, 20))
        step(host)
        e2e_ms, _ = timed(host, args.path, e2e_steps)
        e2e_s = e2e_ms * 1e-3 / e2e_steps
        # the same with E bit-packed on the host (dl_tc_closure_bits): an eighth of the H2D bytes
        step(host_bits)
        e2e_bits_ms, _ = timed(host_bits, args.path, e2e_steps)
        e2e_bits_s = e2e_bits_ms * 1e-3 / e2e_steps
        # device-resident again, but every solve on a graph its context did not just solve
        fresh_ms_step, fresh_stats = None, []
        if fresh is not None:
            step(fresh)
            fresh_steps = max(1, min(args.steps, 400))
            fresh_ms, fresh_stats = timed(fresh, args.path, fresh_steps)
            fresh_ms_step = fresh_ms / fresh_steps
    clocks = clk.summary()
    launches = sum(st["gpu_launches"] for st in stats)
    gemm_ms = sum(st["ms_gemm"] for st in stats)
    gemm_flops = sum(st["gemm_flops"] for st in stats)
    gemm_n = sum(st["gemm_launches"] for st in stats)
    headline_gemms = gemm_n
    squarings = [st["iters"] for st in stats]
    ms_step = ms_total / args.steps
    ms_step, e2e_s, e2e_bits_s = max_over_ranks([ms_step, e2e_s, e2e_bits_s], world, "cuda")
    units = world * len(gs)
    value = units * flops_equiv(N) / (ms_step * 1e-3) / 1e12
    e2e_value = units * flops_equiv(N) / e2e_s / 1e12
    gemm_share = gemm_ms / (ms_total * nctx) if ms_total > 0 else 0.0  # of the streams' time

    # the squarings-only FP8 path on the same graphs, for comparison and for the GEMM roofline
    pure = None
    if rank == 0 and args.path != "bool_fp8" and not args.no_compare:
        # one context, models in sequence: every GEMM launch runs alone (burst roofline)
        for x in dev:
            ctxs[0].tc_closure(x, path="bool_fp8")
        k2 = max(10, args.steps // 5)
        p_stats = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            for x in dev:
                p_stats.append(ctxs[0].tc_closure(x, path="bool_fp8")[1])
        torch.cuda.synchronize()
        ms2 = (time.perf_counter() - t0) / k2 * 1e3
        p_ms = sum(st["ms_gemm"] for st in p_stats)
        pure = {"path": "bool_fp8 (tensor-core squarings only), models in sequence", "ms_per_step": ms2,
                "value": len(gs) * flops_equiv(N) / (ms2 * 1e-3) / 1e12,
                "squarings_per_model": sorted(set(st["iters"] for st in p_stats)),
                "gemm_fraction_of_step": p_ms / (ms2 * k2)}
        gemm_ms = p_ms
        gemm_flops = sum(st["gemm_flops"] for st in p_stats)
        gemm_n = sum(st["gemm_launches"] for st in p_stats)

    fp64 = None
    mixed = None
    if not args.no_fp64 and rank == 0:
        ctx = ctxs[0]
        _, st64 = ctx.tc_closure(dev[1], path="fp64")  # warm
        _, st64 = ctx.tc_closure(dev[1], path="fp64")
        fp64 = {"ms": st64["ms_total"], "tflops_equiv": st64["tflops_equiv"],
                "graph": "p=1e-3 seed 3", "rechecked_rows": st64["rows_rechecked"]}
        mixed = mixed_leg(ctx, dev)

    sweep_ms = sum(st["ms_sweep"] for st in stats)
    sweep_bytes = sum(st["sweep_bytes"] for st in stats)
    sweep_n = sum(st["sweep_launches"] for st in stats)
    pk = peaks()
    fp8_peak = 2.0 * pk["bf16"]  # FP8 dense = 2 x BF16 dense (nominal ratio)
    achieved = (gemm_flops / (gemm_ms * 1e-3) / 1e12) if gemm_ms > 0 else 0.0
    roofline = {"bound": "tensor", "kernel": "umma_gemm_kernel<FP8,256,MN-major B,bool epilogue>",
                "measured_in": "squarings-only FP8 run" if pure else "headline run",
                "achieved": achieved, "peak": fp8_peak, "unit": "TFLOP/s",
                "frac": achieved / fp8_peak, "traffic": traffic("gemm"),
                "peak_source": f"2 x bf16_tflops of {pk['source']} MEASURED_PEAKS (burst)",
                "gemm_launches": gemm_n, "avg_launch_ms": gemm_ms / max(gemm_n, 1)}
    roofline_sweep = None
    if sweep_ms > 0:
        ach = sweep_bytes / (sweep_ms * 1e-3) / 1e9
        roofline_sweep = {"bound": "hbm", "kernel": "bit sweeps (sweep_rows_step / sweep_units_step + final E M)",
                          "achieved": ach, "peak": pk["hbm"], "unit": "GB/s", "frac": ach / pk["hbm"],
                          "bytes_definition": "CSR of E + one read of every bit-matrix row per sweep (minimum)",
                          "launches": sweep_n, "traffic": traffic("sweep"),
                          "share_of_busy_time": sweep_ms / (ms_total * nctx) if ms_total else None}
    # the headline's dominant kernel by device time
    dominant = roofline
    if roofline_sweep and sweep_ms > gemm_share * ms_total * nctx:
        dominant = roofline_sweep
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("bits (boolean OR, Iteration sweeps)" if headline_gemms == 0 else
                      "bits (boolean OR) + e4m3 (0/1, FP32 accumulate) squarings"),
            "data": "synthetic (seeded Erdos-Renyi, i != j)",
            "config": {"workload": "TC ER N=8192 x p in {1e-4,1e-3,1e-2}, seeds 2/3/4 (+1000*rank)",
                       "path": args.path, "l2": "inputs 3 x 64 MiB > L2, cycled each step",
                       "squarings_per_model": sorted(set(squarings)),
                       "concurrency": f"{nctx} closures in flight ({INFLIGHT} contexts per model, one stream and host thread each)",
                       "gemm_busy_fraction": gemm_share,
                       "tuned": tuned if tuned is not None else "fixed rules (--no-tune)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": len(gs) * N * N,
                    "d2h_bytes_per_step": len(gs) * N * ((N + 63) // 64) * 8},
            "e2e_bits": {"value": units * flops_equiv(N) / e2e_bits_s / 1e12, "unit": UNIT,
                         "input": "E bit-packed on the host (dl_tc_closure_bits)",
                         "h2d_bytes_per_step": len(gs) * N * ((N + 63) // 64) * 8,
                         "d2h_bytes_per_step": len(gs) * N * ((N + 63) // 64) * 8},
            "gpu_launches": launches, "roofline": dominant, "roofline_gemm": roofline,
            "roofline_sweep": roofline_sweep,
            "clocks": clocks}
    if fresh_ms_step is not None:
        fresh_ms_step = max_over_ranks([fresh_ms_step], world, "cuda")[0]
        line["fresh_inputs"] = {
            "value": units * flops_equiv(N) / (fresh_ms_step * 1e-3) / 1e12, "unit": UNIT,
            "ms_per_step": fresh_ms_step, "steps": max(1, min(args.steps, 400)),
            "inputs": f"{FRESH_K} seeded graphs per p (seeds {fresh_seeds(rank)}), device-resident; "
                      "each context solves a different graph than its previous solve",
            "gemm_launches": sum(st["gemm_launches"] for st in fresh_stats),
            "squarings_per_model": sorted(set(st["iters"] for st in fresh_stats))}
    if not args.no_extra and rank == 0:
        line["same_generation"] = bench_sg(ctxs[0], torch)
        line["sg_real"] = bench_sg_real(ctxs[0], torch)
        line["tail_recursive"] = bench_tail(ctxs[0], torch)
        line["transposed"] = bench_trans(ctxs[0], torch)
        line["batch"] = bench_batch(ctxs[0], torch)
        line["serving"] = bench_serving(dl, torch, local, args.serve_seconds)
    if pure:
        line["bool_fp8_path"] = pure
    if mixed:
        line["mixed_path"] = mixed
    if fp64:
        line["fp64_path"] = fp64
        line["speedup_vs_fp64"] = fp64["ms"] / (ms_step / len(gs))
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(gs)
        line["cpu_rows"] = cpu_rows()
        if "sg_real" in line:
            line["sg_real"]["cpu_oracle"] = cpu_sg_real()
        if "tail_recursive" in line:
            line["tail_recursive"]["cpu_oracle"] = cpu_tail()
        if "transposed" in line:
            line["transposed"]["cpu_oracle"] = cpu_trans()
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
