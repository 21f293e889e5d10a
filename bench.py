#!/usr/bin/env python
"""Benchmark of the pass-through connectivity hot path (FastCod, arXiv
2302.09247, Section 2 / Algorithm 2) on GB300.

One step = one whole pass of the hot path over one subject: zero C and C_end,
prefilter + compaction over the full vertex stream, walk + dedup + accumulate
of the survivors, and the exact overflow path.  The default workload is the
high-resolution subject (260x311x260 @ 0.7 mm, two thalami, N = 39,708,
M = 360, 5,000,000 streamlines, 9.5 GB vertex stream), inputs resident in HBM,
larger than L2.  The same JSON line carries, measured in the same run:
  dda      - the subject again with the prefilter and the walk's skip of far
             segments off, every voxel step walked: the integer DDA's own
             voxel-steps/s;
  batched  - 64 heterogeneous subjects in one graph-captured batch against one
             call per subject (subjects/s of both);
  served   - Poisson arrivals at 20/s of HCP-shaped requests: subjects/s,
             p50/p99 latency and closed-loop saturation, every request's C and
             C_end checked against the oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --config 1 --no-forms --no-dda   # the HCP-shaped subject alone

Under torchrun (N > 1) every rank processes its own subject of the same shape
(weak scaling, no data-path collective); rank 0 prints one JSON line.
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

METRIC = "DDA voxel-steps/s & subjects/s for C, bit-exact; batched vs plain; p50/p99 latency"

# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one
# prefilter launch on the high-res subject's first 1,000,000 streamlines,
# valid only while the prefilter's sources are the ones it was measured on;
# workloads scale it by their vertex count (the stream is read once, so
# traffic grows with the vertices).
PREFILTER_SOURCES = ("paper_2302_09247_gb300/csrc/k_prefilter.cu", "paper_2302_09247_gb300/csrc/fc_tma.cuh",
                     "paper_2302_09247_gb300/csrc/fc_internal.cuh", "paper_2302_09247_gb300/csrc/fc_device.cuh")
PREFILTER_TRAFFIC = {"sha256": "e3c96dd2aca3a0ce113e15ed2addcf4a8a58f6ed2eb59c1a51b564868699520b",
                     "bytes": 1911535104, "vertices": 157754709, "workload": "high-res",
                     "summary": "profiles/prefilter_kernel_highres260x311x260.md"}


def prefilter_traffic(n_vertices: int):
    """(bytes per launch, note) from the recorded capture, or (None, why)."""
    import hashlib
    h = hashlib.sha256()
    for f in PREFILTER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != PREFILTER_TRAFFIC["sha256"]:
        return None, "prefilter sources changed since the ncu capture"
    ref = PREFILTER_TRAFFIC
    if n_vertices == ref["vertices"]:
        return ref["bytes"], f"ncu capture of this workload ({ref['summary']})"
    return int(round(ref["bytes"] * n_vertices / ref["vertices"])), \
        f"ncu capture of the {ref['workload']} subject's first {ref['vertices']:,} vertices " \
        f"({ref['summary']}), scaled by vertex count"
UNIT = "voxel-steps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# nvidia-smi's sampling interval (the profiling recipe's clocks line); each
# sample queries the driver, which the served form's request loop feels
CLOCK_SAMPLE_MS = 200


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(CLOCK_SAMPLE_MS)], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons, samples = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                samples += 1
                for n, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": samples}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _allreduce(ws, x: float, op: str) -> float:
    """x reduced over the ranks (max or sum); tensors live where the process
    group's backend wants them (CUDA for NCCL, host memory for gloo)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _barrier_max(ws, x: float) -> float:
    return _allreduce(ws, x, "max")


def _barrier_sum(ws, x: float) -> float:
    return _allreduce(ws, x, "sum")


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank r's subject: same shape on every rank, different data."""
    return seed + 7919 * rank


def weak_scaling(ws, units: float, seconds: float):
    """(whole-job units/s, slowest rank's seconds): the units all ranks
    processed over the time of the slowest rank."""
    t = _barrier_max(ws, seconds)
    return _barrier_sum(ws, units) / t, t


def cpu_baseline(vols, tr, n_sample: int):
    """The oracle as it stands, single-threaded, on the first n_sample
    streamlines of the same subject (test infrastructure, timed here only)."""
    import oracle
    n = min(n_sample, tr.n_streamlines)
    off = tr.offsets[: n + 1]
    xyz = tr.xyz[: off[-1]]
    oracle.lib()  # build/load outside the timed region
    t0 = time.perf_counter()
    _, _, st = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, xyz, off)
    dt = time.perf_counter() - t0
    return {"value": st["voxel_steps"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n:,} of the subject's streamlines ({int(off[-1]):,} vertices, "
                      f"{st['voxel_steps']:,} voxel-steps) in {dt:.2f} s, one thread"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    # the workload is the full subject of this config (the same config as the
    # CUDA arm's line); each timed step is a bounded sample of it: its first
    # `sample` streamlines
    vols, tr = synth.make_subject(args.config)
    sample = min(args.ref_sample, tr.n_streamlines)
    off = tr.offsets[: sample + 1]
    xyz = tr.xyz[: int(off[-1])]
    oracle.lib()
    times, steps = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, _, st = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, xyz, off)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            steps = st["voxel_steps"]
    total = sum(times)
    value = steps * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": _config(args.config, vols, tr),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {sample:,} streamlines of the subject per step, one thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def _digest(a) -> str:
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()[:16]


def _config(cfg, vols, tr):
    names = {0: "tiny 32^3 @ 1 mm, one ROI ellipsoid, M=8",
             1: "HCP-shaped 145x174x145 @ 1.25 mm, two thalami, M=70",
             2: "high-res 260x311x260 @ 0.7 mm, two thalami, M=360"}
    c = {"workload": f"{names.get(cfg, cfg)}: N={vols.n_roi}, M={vols.n_targets}, "
                     f"{tr.n_streamlines:,} streamlines, {tr.n_vertices:,} vertices",
         "grid": list(vols.dims), "N": vols.n_roi, "M": vols.n_targets, "streamlines": tr.n_streamlines,
         "vertices": tr.n_vertices, "parallelism": "one subject per GPU",
         "l2": "inputs larger than L2 (vertex stream %.2f GB per step)" % (tr.n_vertices * 12 / 1e9)}
    return c


def batched_record(args, local) -> dict:
    """64 heterogeneous subjects in one fastcod_batch_run (a CUDA graph per batch
    shape, autotuned) against one set_volumes + add_streamlines + readback per
    subject; subjects/s of both, device-resident inputs and outputs."""
    import torch

    import synth
    from paper_2302_09247_gb300 import fastcod as fc

    dev = torch.device("cuda", local)
    subs, steps_total, nv_total, ns_total = [], 0, 0, 0
    t0 = time.perf_counter()
    for s in range(1, args.subjects + 1):
        d = synth.batched_subject_draws(s)
        n = max(1000, int(d["ns"] * args.count_scale))
        vols, tr = synth.make_subject(3, subject=s, n_streamlines=n)
        subs.append(dict(roi=torch.from_numpy(vols.roi).to(dev), lab=torch.from_numpy(vols.lab.view(np.int16)).to(dev),
                         dims=vols.dims, N=vols.n_roi, M=vols.n_targets, xyz=torch.from_numpy(tr.xyz).to(dev),
                         off=torch.from_numpy(tr.offsets).to(dev),
                         C=torch.empty((vols.n_roi, vols.n_targets), dtype=torch.int32, device=dev),
                         Ce=torch.empty((vols.n_roi, vols.n_targets), dtype=torch.int32, device=dev)))
        nv_total += tr.n_vertices
        ns_total += tr.n_streamlines
        del vols, tr
    gen_s = time.perf_counter() - t0
    objs = [fc.make_subject(x["roi"], x["lab"], x["dims"], x["N"], x["M"], x["xyz"], x["off"], x["C"], x["Ce"])
            for x in subs]
    ctx = fc.Context(local)
    for _ in range(args.warmup):
        fc.fastcod_batch_run(ctx.ctx, objs)
    for i in range(len(subs)):
        steps_total += fc.fastcod_batch_get_stats(ctx.ctx, i)["voxel_steps"]
    launches0 = ctx.profile()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    graph_ms = 0.0
    for _ in range(args.batch_steps):
        fc.fastcod_batch_run(ctx.ctx, objs)
        graph_ms += fc.fastcod_batch_get_info(ctx.ctx)["ms_graph"]
    torch.cuda.synchronize()
    batch_s = (time.perf_counter() - t0) / args.batch_steps
    clk = clocks.stop()
    info = fc.fastcod_batch_get_info(ctx.ctx)
    launches = (ctx.profile()["kernel_launches"] - launches0) / args.batch_steps
    Cb = [x["C"].clone() for x in subs]
    Ceb = [x["Ce"].clone() for x in subs]

    def plain():
        for x in subs:
            ctx.set_volumes(x["roi"], x["lab"], x["dims"], x["N"], x["M"])
            ctx.add_streamlines(x["xyz"], x["off"])
            fc.fastcod_connectivity(ctx.ctx, x["C"])
            fc.fastcod_endpoint_connectivity(ctx.ctx, x["Ce"])

    plain_s = None
    if not args.batch_only:
        plain()
        torch.cuda.synchronize()
        k = max(1, min(args.batch_steps, 3))
        t0 = time.perf_counter()
        for _ in range(k):
            plain()
        torch.cuda.synchronize()
        plain_s = (time.perf_counter() - t0) / k
        assert all(torch.equal(a, x["C"]) for a, x in zip(Cb, subs)), "batched and plain C differ"
        assert all(torch.equal(a, x["Ce"]) for a, x in zip(Ceb, subs)), "batched and plain C_end differ"
    n = len(subs)
    ctx.close()
    return {
        "workload": f"batched: {n} subjects (grids 96^3..145x174x145, M in 8/70/360, N 1,000..12,000), "
                    f"{ns_total:,} streamlines, {nv_total:,} vertices, one CUDA graph per batch shape",
        "subjects": n, "streamlines": ns_total, "vertices": nv_total, "count_scale": args.count_scale,
        "subjects_per_s": n / batch_s, "ms_per_batch": 1000 * batch_s, "steps": args.batch_steps,
        "voxel_steps_per_s": steps_total / batch_s, "graph_ms": graph_ms / args.batch_steps,
        "plain_subjects_per_s": n / plain_s if plain_s else None,
        "plain_ms_per_batch": 1000 * plain_s if plain_s else None,
        "batched_vs_plain": plain_s / batch_s if plain_s else None,
        "checked": "batched C and C_end equal the one-call-per-subject results" if plain_s else None,
        "autotuned": {"prefilter_ctas": info["prefilter_ctas"], "near_log2": info["near_log2"],
                      "task_vertices": info["task_vertices"]},
        "gpu_launches_per_batch": launches, "clocks": clk, "generation_s": gen_s,
        "timing": "wall clock around the graph replays with a device synchronisation on both sides; inputs "
                  "device-resident, larger than L2",
    }


def run_batched(args):
    """--config 3: the batched form's own JSON line."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    r = batched_record(args, local)
    line = {
        "metric": METRIC, "value": r["subjects_per_s"], "unit": "subjects/s", "n_gpus": 1,
        "steps": args.batch_steps, "warmup": args.warmup, "ms_per_step": r["ms_per_batch"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": r["workload"], "subjects": r["subjects"], "streamlines": r["streamlines"],
                   "vertices": r["vertices"], "count_scale": r["count_scale"], "l2": "inputs larger than L2"},
        "batched": r, "gpu_launches": int(round(r["gpu_launches_per_batch"] * args.batch_steps)),
        "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


def served_expected(pool_subjects, block: int, threads: int):
    """Oracle results per pool subject: prefix[k] = (C, C_end) of the first
    k * block streamlines, int32 [k_max + 1, 2, N, M], from the oracle run on
    every block (threads over blocks; integer sums are exact)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.lib()
    out = []
    for vols, tr in pool_subjects:
        nb = tr.n_streamlines // block

        def one(b, vols=vols, tr=tr):
            o = tr.offsets[b * block: (b + 1) * block + 1]
            C, Ce, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets,
                                           tr.xyz[int(o[0]): int(o[-1])], o - o[0])
            return C, Ce

        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(one, range(nb)))
        pre = np.zeros((nb + 1, 2, vols.n_roi, vols.n_targets), dtype=np.int32)
        for b, (C, Ce) in enumerate(parts):
            pre[b + 1, 0] = pre[b, 0] + C
            pre[b + 1, 1] = pre[b, 1] + Ce
        out.append(pre)
    return out


def host_link_gbs(local, nbytes: int = 1 << 30) -> float:
    """Host-to-device bandwidth of one page-locked copy right now (GB/s): the
    served latency follows this shared link."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=torch.device("cuda", local))
    d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        d.copy_(h, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) / 1000.0) / 1e9)
    del h, d
    return best


def served_record(args, local) -> dict:
    """Poisson arrivals of HCP-shaped requests (200,000..2,000,000 streamlines in
    250,000-streamline chunks from page-locked host memory) into the served
    form; subjects/s and p50/p99 end-to-end latency, then a closed-loop
    saturation run.  Every request's C and C_end is compared with the oracle's
    (sums of per-50,000-streamline oracle blocks of its pool subject)."""
    import torch

    import synth
    from paper_2302_09247_gb300 import fastcod as fc

    chunk, block = 250_000, 50_000
    pool, subjects = [], []
    t0 = time.perf_counter()
    for p in range(args.pool):
        vols, tr = synth.make_subject(4, subject=p)
        subjects.append((vols, tr))
        xyz = torch.from_numpy(tr.xyz).pin_memory()
        chunks = []
        for c in range(0, tr.n_streamlines, chunk):
            e = min(tr.n_streamlines, c + chunk)
            off = torch.from_numpy(tr.offsets[c:e + 1] - tr.offsets[c]).pin_memory()
            chunks.append((int(tr.offsets[c]), off))
        pool.append(dict(vols=vols, roi=torch.from_numpy(vols.roi).pin_memory(),
                         lab=torch.from_numpy(vols.lab.view(np.int16)).pin_memory(), xyz=xyz, chunks=chunks,
                         ns=tr.n_streamlines))
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    expect = served_expected(subjects, block, max(1, min(64, os.cpu_count() or 1))) if args.serve_check else None
    oracle_s = time.perf_counter() - t0
    del subjects
    rng = np.random.default_rng(20)

    def spec():
        return int(rng.integers(len(pool))), block * int(rng.integers(4, 41))

    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=int(args.rate * args.serve_seconds * 1.5) + 10))
    arrivals = arrivals[arrivals < args.serve_seconds]
    specs = [spec() for _ in arrivals]
    specs2 = [spec() for _ in range(4 * args.slots)]
    warm = [(p, 4 * block) for p in range(len(pool))]
    # page-locked outputs of every request, allocated before the arrivals
    N, M = pool[0]["vols"].n_roi, pool[0]["vols"].n_targets
    assert all(P["vols"].n_roi == N and P["vols"].n_targets == M for P in pool)
    n_req = len(warm) + len(specs) + len(specs2)
    outs = torch.empty((n_req, 2, N, M), dtype=torch.int32).pin_memory()
    ctx = fc.Context(local)
    srv = fc.fastcod_server_create(ctx.ctx, args.slots, 0)
    keep, issued = [], []

    def submit(sp):
        p, count = sp
        P = pool[p]
        vols = P["vols"]
        k = len(issued)
        C, Ce = outs[k, 0], outs[k, 1]
        head = fc.make_subject(P["roi"], P["lab"], vols.dims, vols.n_roi, vols.n_targets,
                               np.zeros((0, 3), np.int32), np.zeros(1, np.int64), C, Ce)
        rid = fc.fastcod_server_submit(srv, head)
        left = count
        for v0, off in P["chunks"]:
            n = min(chunk, left)
            o = off[: n + 1]
            x = P["xyz"][v0: v0 + int(o[-1])]
            left -= n
            fc.fastcod_server_push_chunk(srv, rid, x, o, last=(left == 0))
            keep.append((x, o))
            if left == 0:
                break
        keep.append(head)
        issued.append((rid, p, count, k))
        return rid

    for sp in warm:
        assert fc.fastcod_server_wait(srv, submit(sp), 120.0) == fc.FASTCOD_OK
    link_before = host_link_gbs(local)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = fc.fastcod_server_kernel_launches(srv)
    ids = []
    t_start = time.perf_counter()
    for at, sp in zip(arrivals, specs):
        d = t_start + at - time.perf_counter()
        if d > 0:
            time.sleep(d)
        ids.append(submit(sp))
    for rid in ids:
        assert fc.fastcod_server_wait(srv, rid, 300.0) == fc.FASTCOD_OK
    clk = clocks.stop()
    launches = fc.fastcod_server_kernel_launches(srv) - launches0
    infos = [fc.fastcod_server_request_info(srv, rid) for rid in ids]
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos])
    wait = np.array([i["t_admit"] - i["t_submit"] for i in infos])
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    n_streamlines = sum(c for (_, _, c, _) in issued[len(warm):len(warm) + len(ids)])
    # closed loop: everything at once
    t0 = time.perf_counter()
    ids2 = [submit(sp) for sp in specs2]
    for rid in ids2:
        assert fc.fastcod_server_wait(srv, rid, 300.0) == fc.FASTCOD_OK
    sat_s = time.perf_counter() - t0
    n2 = sum(c for (_, _, c, _) in issued[-len(ids2):])
    link_after = host_link_gbs(local)
    fc.fastcod_server_destroy(srv)
    ctx.close()
    checked, bad = 0, 0
    if expect is not None:
        for rid, p, count, k in issued:
            e = expect[p][count // block]
            ok = np.array_equal(outs[k, 0].numpy(), e[0]) and np.array_equal(outs[k, 1].numpy(), e[1])
            checked += 1
            bad += 0 if ok else 1
        assert bad == 0, f"{bad} of {checked} served results differ from the oracle"
    return {
        "workload": f"served: Poisson {args.rate}/s for {args.serve_seconds}s of HCP-shaped requests "
                    f"(200k..2M streamlines, 250k-streamline chunks from page-locked host memory, "
                    f"pool of {len(pool)} subjects), {args.slots} slots",
        "requests": len(ids), "streamlines": n_streamlines, "subjects_per_s": len(ids) / span,
        "offered_rate": args.rate, "span_s": span,
        "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)), "p99": 1000 * float(np.percentile(lat, 99)),
                       "mean": 1000 * float(lat.mean()), "max": 1000 * float(lat.max())},
        "admission_wait_ms": {"p50": 1000 * float(np.percentile(wait, 50)),
                              "p99": 1000 * float(np.percentile(wait, 99))},
        "service_ms": {"p50": 1000 * float(np.percentile(lat - wait, 50)),
                       "p99": 1000 * float(np.percentile(lat - wait, 99))},
        "host_link_gbs": {"before": link_before, "after": link_after,
                          "what": "one 1 GiB page-locked host-to-device copy, best of 3"},
        "saturation": {"requests": len(ids2), "subjects_per_s": len(ids2) / sat_s, "streamlines_per_s": n2 / sat_s},
        "bit_exact": ({"requests_checked": checked, "mismatches": bad,
                       "against": "oracle sums of 50,000-streamline blocks of each request's pool subject "
                                  "(C and C_end, every request incl. warm-up and saturation)"}
                      if expect is not None else None),
        "gpu_launches": launches, "clocks": clk, "generation_s": gen_s, "oracle_s": oracle_s,
        "latency": "request submit to completion (fastcod_server_request_info), host clock",
    }


def run_served(args):
    """--config 4: the served form's own JSON line."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    r = served_record(args, local)
    line = {
        "metric": METRIC, "value": r["subjects_per_s"], "unit": "subjects/s", "n_gpus": 1, "steps": r["requests"],
        "warmup": args.pool, "ms_per_step": 1000 * r["span_s"] / r["requests"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": r["workload"], "requests": r["requests"], "streamlines": r["streamlines"]},
        "served": r, "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_next(args):
    """Entry points beside the path, timed with CUDA events on the context's
    stream over device-resident inputs, each against its HBM roofline:
      parcellate - labels and binary32 fractions of the high-res subject's C
                   (N = 39,708, M = 360): 8 B per entry + 4 B per row;
      ingest     - fastcod_add_streamlines_mm of the HCP-shaped subject from
                   binary32 world-mm vertices (conversion, 24 B per vertex,
                   then the path, 12 B per vertex); metric voxel-steps/s;
      upsample   - fastcod_upsample of the HCP-shaped subject by --factor:
                   12 B read + 12 * factor B written per vertex."""
    import torch

    import synth
    from paper_2302_09247_gb300 import fastcod as fc

    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_kind = _peaks()
    ctx = fc.Context(local)
    stream = torch.cuda.Stream(device=dev)
    fc.fastcod_set_stream(ctx.ctx, stream)
    cfg = 2 if args.next == "parcellate" else 1
    vols, tr = synth.make_subject(cfg, n_streamlines=args.streamlines)
    xyz_d = torch.from_numpy(tr.xyz).to(dev)
    off_d = torch.from_numpy(tr.offsets).to(dev)
    extra = {}
    if args.next == "parcellate":
        ctx.set_volumes(torch.from_numpy(vols.roi).to(dev), torch.from_numpy(vols.lab.view(np.int16)).to(dev),
                        vols.dims, vols.n_roi, vols.n_targets)
        ctx.add_streamlines(xyz_d, off_d)
        N, M = vols.n_roi, vols.n_targets
        lab_out = torch.empty(N, dtype=torch.int32, device=dev)
        frac_out = torch.empty((N, M), dtype=torch.float32, device=dev)

        def step():
            fc.fastcod_parcellate(ctx.ctx, 0, lab_out, frac_out)
        units, unit, metric = float(N), "rows/s", "parcellation rows/s (label + fractions)"
        alg_bytes = 8 * N * M + 4 * N
        kernel = "parcellate_kernel"
    elif args.next == "ingest":
        ctx.set_volumes(torch.from_numpy(vols.roi).to(dev), torch.from_numpy(vols.lab.view(np.int16)).to(dev),
                        vols.dims, vols.n_roi, vols.n_targets)
        A = np.zeros((3, 4), dtype=np.float32)  # 1.25 mm voxels, origin at -90 mm
        A[:, :3] = np.eye(3, dtype=np.float32) / np.float32(1.25)
        A[:, 3] = np.float32(90.0) / np.float32(1.25)
        x_mm = torch.from_numpy(((tr.xyz.astype(np.float64) / 1024.0) * 1.25 - 90.0).astype(np.float32)).to(dev)

        def step():
            fc.fastcod_reset(ctx.ctx)
            fc.fastcod_add_streamlines_mm(ctx.ctx, x_mm, off_d, A)
        step()
        ctx.sync()
        units, unit, metric = float(ctx.stats()["voxel_steps"]), UNIT, METRIC + " (world-mm binary32 input)"
        alg_bytes = 36 * tr.n_vertices + 8 * (tr.n_streamlines + 1)
        kernel = "world_to_fixed_kernel + prefilter_kernel (the call's two streaming passes: 24 + 12 B per vertex)"
    else:
        k = args.factor
        n_out = fc.upsampled_count(tr.offsets, k)
        ux = torch.empty((n_out, 3), dtype=torch.int32, device=dev)
        uo = torch.empty(tr.n_streamlines + 1, dtype=torch.int64, device=dev)

        def step():
            fc.fastcod_upsample(ctx.ctx, xyz_d, off_d, k, ux, uo)
        units, unit, metric = float(n_out), "vertices/s", f"upsampled vertices/s (factor {k})"
        alg_bytes = 12 * tr.n_vertices + 12 * n_out + 16 * (tr.n_streamlines + 1)
        kernel = "upsample kernels (offsets scan + vertices)"
        extra["factor"] = k
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.profile()["kernel_launches"]
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = ctx.profile()["kernel_launches"] - launches0
    # the kernels' own device time: a second, profiled pass (events around
    # each call's kernels; the calls' host-side checks and synchronisations,
    # which the timed pass above includes, fall outside)
    fc.fastcod_set_option(ctx.ctx, fc.FASTCOD_OPT_PROFILE, 1)
    for _ in range(args.steps):
        step()
    prof = ctx.profile()
    fc.fastcod_set_option(ctx.ctx, fc.FASTCOD_OPT_PROFILE, 0)
    kernel_ms = (prof["ms_aux"] + (prof["ms_prefilter"] if args.next == "ingest" else 0.0)) / args.steps
    line = {
        "metric": metric, "value": units / (ms / 1000.0), "unit": unit, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32" if args.next != "parcellate" else "int32 -> f32",
        "data": "synthetic", "config": dict(_config(cfg, vols, tr), next=args.next, **extra),
        "roofline": {"bound": "hbm", "kernel": kernel, "algorithmic_bytes_per_step": alg_bytes,
                     "achieved": alg_bytes / (kernel_ms / 1000.0) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": alg_bytes / (kernel_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
                     "kernel_ms_per_step": kernel_ms,
                     "call_frac": alg_bytes / (ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
                     "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)", "traffic": None},
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


# Warp instructions the walk kernel issues per voxel step with the prefilter
# off (every streamline walked), from ncu (smsp__inst_executed.sum over the
# launch / the launch's voxel steps), valid only while the walk's sources are
# the ones it was measured on.
WALK_SOURCES = ("paper_2302_09247_gb300/csrc/k_walk.cu", "paper_2302_09247_gb300/csrc/fc_device.cuh",
                "paper_2302_09247_gb300/csrc/fc_internal.cuh")
WALK_INSTR = {"sha256": "e3345e68cfa153a017e23b6b3296bfe32931559897a46f5c444e4ff3c15bad6d",
              "warp_instr_per_voxel_step": 519023423 / 54811982,
              "summary": "profiles/walk_kernel_dda_highres260x311x260.md"}


def _sources_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def dda_record(ctx, step, stream, C_ref, Ce_ref, steps: int, local: int) -> dict:
    """The walk on the whole vertex stream: the same subject with the prefilter
    and the walk's skip of far segments off, so that every segment of every
    streamline is walked voxel by voxel and every voxel step of the metric is
    a DDA step taken; C and C_end must not change."""
    import torch

    from paper_2302_09247_gb300 import fastcod as fc

    fc.fastcod_set_option(ctx.ctx, fc.FASTCOD_OPT_PREFILTER, 0)
    fc.fastcod_set_option(ctx.ctx, fc.FASTCOD_OPT_SEGMENT_SKIP, 0)
    step()
    ctx.sync()
    st = ctx.stats()
    assert np.array_equal(ctx.connectivity(), C_ref), "C differs with the prefilter off"
    assert np.array_equal(ctx.endpoint_connectivity(), Ce_ref), "C_end differs with the prefilter off"
    ctx.set_option(fc.FASTCOD_OPT_PROFILE, 1)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    prof = ctx.profile()
    ctx.set_option(fc.FASTCOD_OPT_PROFILE, 0)
    fc.fastcod_set_option(ctx.ctx, fc.FASTCOD_OPT_PREFILTER, 1)
    fc.fastcod_set_option(ctx.ctx, fc.FASTCOD_OPT_SEGMENT_SKIP, 1)
    walk_ms = prof["ms_walk"] / max(prof["calls"], 1)
    vs = st["voxel_steps"]
    rec = {"what": "prefilter and segment skip off: every segment of every streamline walked voxel by voxel "
                   "(integer 3-D DDA, code gather, dedup, accumulate)",
           "voxel_steps_per_step": vs, "walked_streamlines": st["survivors"], "ms_per_step": ms,
           "voxel_steps_per_s": vs / (ms / 1000.0), "walk_ms_per_step": walk_ms,
           "walk_voxel_steps_per_s": vs / (walk_ms / 1000.0), "steps": steps, "clocks": clk,
           "checked": "C and C_end equal the prefiltered step's"}
    sm_mhz = clk.get("sm_mhz") or 2070.0
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * 4 * sm_mhz * 1e6  # warp instructions issued per second
    per_step = None
    if WALK_INSTR["sha256"] is not None and _sources_sha(WALK_SOURCES) == WALK_INSTR["sha256"]:
        per_step = WALK_INSTR["warp_instr_per_voxel_step"]
    rec["roofline"] = {
        "bound": "issue", "kernel": "walk_kernel",
        "peak": peak, "unit": "warp-instructions/s",
        "peak_source": f"{props.multi_processor_count} SMs x 4 schedulers x 1 warp-instruction/cycle x "
                       f"{sm_mhz:.0f} MHz (median SM clock sampled during the region)",
        "warp_instr_per_voxel_step": per_step,
        "achieved": per_step * vs / (walk_ms / 1000.0) if per_step else None,
        "frac": per_step * vs / (walk_ms / 1000.0) / peak if per_step else None,
        "instr_source": WALK_INSTR["summary"] if per_step else "walk sources changed since the ncu capture",
    }
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fastcod", choices=["fastcod", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[0, 1, 2, 3, 4],
                    help="0-2: one subject (default 2, the high-res subject, with the batched and served "
                         "forms and the DDA measured in the same line); 3: batched; 4: served")
    ap.add_argument("--no-forms", action="store_true", help="no batched / served sub-records")
    ap.add_argument("--no-dda", action="store_true", help="no DDA sub-record (prefilter off)")
    ap.add_argument("--near-log2", type=int, default=None,
                    help="near-grid cell of the plain line: (1 << n)^3 voxels, 0..3 (default: automatic)")
    ap.add_argument("--dda-steps", type=int, default=5, help="timed steps of the DDA sub-record (prefilter off)")
    ap.add_argument("--batch-steps", type=int, default=5, help="timed passes of the batched form")
    ap.add_argument("--no-serve-check", dest="serve_check", action="store_false",
                    help="skip the oracle check of the served results")
    ap.add_argument("--subjects", type=int, default=64, help="--config 3: subjects per batch")
    ap.add_argument("--batch-only", action="store_true", help="--config 3: skip the one-call-per-subject leg")
    ap.add_argument("--count-scale", type=float, default=1.0, help="--config 3: scale of the streamline counts")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="served form: length of the arrival process")
    ap.add_argument("--rate", type=float, default=20.0, help="--config 4: Poisson arrivals per second")
    ap.add_argument("--pool", type=int, default=4, help="--config 4: pre-generated subjects")
    ap.add_argument("--slots", type=int, default=16, help="--config 4: server slots")
    ap.add_argument("--next", default=None, choices=["parcellate", "ingest", "upsample"],
                    help="time an entry point beside the path instead (one JSON line of its own)")
    ap.add_argument("--factor", type=int, default=2, help="--next upsample: upsampling factor")
    ap.add_argument("--e2e-steps", type=int, default=10, help="0 skips the end-to-end leg")
    ap.add_argument("--streamlines", type=int, default=None,
                    help="use only the first N streamlines of the subject (small profiling cases)")
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--ref-sample", type=int, default=200_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.next:
        return run_next(args)
    if args.config == 3:
        return run_batched(args)
    if args.config == 4:
        return run_served(args)

    import torch

    import synth
    from paper_2302_09247_gb300 import fastcod as fc

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if dist.is_nccl_available() else "gloo")
    dev = torch.device("cuda", local)

    # one subject per rank: the preset's shape, a per-rank seed
    vs = synth.volume_spec(args.config)
    ss = synth.streamline_spec(args.config)
    ss.seed = rank_seed(ss.seed, rank)
    if args.streamlines is not None:
        ss.n_streamlines = min(ss.n_streamlines, args.streamlines)
    vols = synth.make_volumes(vs)
    tr = synth.make_tractogram(vs, ss, vols)

    stream = torch.cuda.Stream(device=dev)
    ctx = fc.Context(local)
    fc.fastcod_set_stream(ctx.ctx, stream)
    if args.near_log2 is not None:
        ctx.set_option(fc.FASTCOD_OPT_NEAR_LOG2, args.near_log2)
    roi_d = torch.from_numpy(vols.roi).to(dev)
    lab_d = torch.from_numpy(vols.lab.view(np.int16)).to(dev)
    ctx.set_volumes(roi_d, lab_d, vols.dims, vols.n_roi, vols.n_targets)
    xyz_d = torch.from_numpy(tr.xyz).to(dev)
    off_d = torch.from_numpy(tr.offsets).to(dev)
    torch.cuda.synchronize()

    def step():
        fc.fastcod_reset(ctx.ctx)
        fc.fastcod_add_streamlines(ctx.ctx, xyz_d, off_d)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    st = ctx.stats()
    C_first = ctx.connectivity()
    # the survivors' voxel steps: one more step with the count switched on
    # (an extra kernel, kept out of the timed region)
    ctx.set_option(fc.FASTCOD_OPT_WALKED_STEPS, 1)
    step()
    walked_steps = ctx.stats()["walked_steps"]
    ctx.set_option(fc.FASTCOD_OPT_WALKED_STEPS, 0)

    # ---------------------------------------------------------- timed region
    ctx.set_option(fc.FASTCOD_OPT_PROFILE, 1)
    launches0 = ctx.profile()["kernel_launches"]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    _barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = ctx.profile()
    ctx.set_option(fc.FASTCOD_OPT_PROFILE, 0)
    st_last = ctx.stats()
    C_last = ctx.connectivity()
    Ce_first = ctx.endpoint_connectivity()
    assert np.array_equal(C_first, C_last), "C changed between identical steps"
    assert st_last["voxel_steps"] == st["voxel_steps"]
    forms = not args.no_forms and ws == 1
    dda = dda_record(ctx, step, stream, C_first, Ce_first, args.dda_steps, local) \
        if not args.no_dda and ws == 1 else None

    value, t_max = weak_scaling(ws, float(st["voxel_steps"]) * args.steps, ms / 1000.0)
    ms_max = 1000.0 * t_max
    streamlines_s = _barrier_sum(ws, float(tr.n_streamlines)) * args.steps / t_max
    subjects_s = ws * args.steps / t_max

    # roofline of the dominant kernel (prefilter: the full vertex stream)
    peaks, peak_kind = _peaks()
    alg_bytes = 12 * tr.n_vertices + 8 * (tr.n_streamlines + 1)
    k2_ms = prof["ms_prefilter"] / max(prof["calls"], 1)
    achieved = alg_bytes / (k2_ms / 1000.0) / 1e9
    traffic, traffic_note = prefilter_traffic(tr.n_vertices)
    roofline = {"bound": "hbm", "kernel": "prefilter_kernel", "achieved": achieved,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)", "traffic": traffic,
                "traffic_source": traffic_note,
                "algorithmic_bytes_per_launch": alg_bytes,
                "stage_ms_per_step": {"prefilter": k2_ms, "walk": prof["ms_walk"] / max(prof["calls"], 1),
                                      "overflow": prof["ms_overflow"] / max(prof["calls"], 1)}}
    gpu_launches = prof["kernel_launches"] - launches0

    # ------------------------------------------------ end to end, host buffers
    e2e = None
    xyz_h = off_h = None
    if args.e2e_steps > 0:
        xyz_h = torch.from_numpy(tr.xyz).pin_memory()
        off_h = torch.from_numpy(tr.offsets).pin_memory()
        N, M = ctx.shape()
        C_h = torch.empty((N, M), dtype=torch.int32).pin_memory()
        Ce_h = torch.empty((N, M), dtype=torch.int32).pin_memory()
        for _ in range(2):
            fc.fastcod_reset(ctx.ctx)
            fc.fastcod_add_streamlines(ctx.ctx, xyz_h, off_h)
            fc.fastcod_connectivity(ctx.ctx, C_h)
            fc.fastcod_endpoint_connectivity(ctx.ctx, Ce_h)
        _barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fc.fastcod_reset(ctx.ctx)
            fc.fastcod_add_streamlines(ctx.ctx, xyz_h, off_h)
            fc.fastcod_connectivity(ctx.ctx, C_h)
            fc.fastcod_endpoint_connectivity(ctx.ctx, Ce_h)
        e2e_s = time.perf_counter() - t0
        assert np.array_equal(C_h.numpy(), C_first)
        e2e_value, e2e_max = weak_scaling(ws, float(st["voxel_steps"]) * args.e2e_steps, e2e_s)
        # the same calls with the page-locked xyz read in place by the kernels
        ctx.set_option(fc.FASTCOD_OPT_HOST_IN_PLACE, 1)
        for i in range(1 + args.e2e_steps):
            if i == 1:
                _barrier(ws)
                t0 = time.perf_counter()
            fc.fastcod_reset(ctx.ctx)
            fc.fastcod_add_streamlines(ctx.ctx, xyz_h, off_h)
            fc.fastcod_connectivity(ctx.ctx, C_h)
            fc.fastcod_endpoint_connectivity(ctx.ctx, Ce_h)
        in_place_max = _barrier_max(ws, time.perf_counter() - t0)
        assert np.array_equal(C_h.numpy(), C_first)
        ctx.set_option(fc.FASTCOD_OPT_HOST_IN_PLACE, 0)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": xyz_h.numel() * 4 + off_h.numel() * 8,
               "d2h_bytes_per_step": 2 * N * M * 4, "ms_per_step": 1000 * e2e_max / args.e2e_steps,
               "steps": args.e2e_steps,
               "inputs": "page-locked host memory, copied to HBM by the call",
               "read_in_place_ms_per_step": 1000 * in_place_max / args.e2e_steps}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(vols, tr, args.cpu_sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": _config(args.config, vols, tr),
            "subjects_per_s": subjects_s, "streamlines_per_s": streamlines_s,
            "voxel_steps_per_step": st["voxel_steps"], "survivors_per_step": st["survivors"],
            "overflow_per_step": st["overflow"], "pairs_per_step": st["pairs"],
            "walked_steps_per_step": walked_steps,
            "C_sum": int(C_first.sum()),
            # fingerprints of the result (int32 little-endian bytes, row-major)
            "C_sha256": _digest(C_first), "C_end_sha256": _digest(Ce_first),
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "dda": dda,
        }
    ctx.close()
    if rank == 0 and forms:
        # the batched and served forms of the metric, measured in this run
        del xyz_d, off_d, roi_d, lab_d, xyz_h, off_h, tr
        torch.cuda.empty_cache()
        line["batched"] = batched_record(args, local)
        torch.cuda.empty_cache()
        line["served"] = served_record(args, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
