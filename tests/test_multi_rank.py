"""The N > 1 host logic of bench.py on CPU: two gloo ranks (127.0.0.1)
reduce their timings and work the way the benchmark does (max of the times,
sum of the units, one JSON line from rank 0), each rank draws its own subject
of the same shape, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + rank  # rank 1 is the slow one
        units = 100.0 * (rank + 1)
        value, t = bench.weak_scaling(world, units, seconds)
        mx = bench._barrier_max(world, float(rank))
        sm = bench._barrier_sum(world, 1.0)
        bench._barrier(world)
        ss = synth.streamline_spec(0, n_streamlines=50)
        ss.seed = bench.rank_seed(ss.seed, rank)
        vs = synth.volume_spec(0)
        vols = synth.make_volumes(vs)
        tr = synth.make_tractogram(vs, ss, vols)
        q.put((rank, value, t, mx, sm, vols.dims, tr.n_streamlines, int(tr.xyz[:8].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_benchmark():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t, mx, sm, dims, ns, _ in res:
        assert t == 2.0                      # the slowest rank's time
        assert value == pytest.approx(300.0 / 2.0)  # all units over that time
        assert mx == 1.0 and sm == 2.0
        assert ns == 50
    assert res[0][5] == res[1][5]            # same shape on every rank
    assert res[0][7] != res[1][7]            # different data


def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--config", "0", "--ref-sample", "500", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the CUDA arm's config (the whole tiny subject), the sample stated beside it
    assert d["config"]["streamlines"] == 20_000 and "first 500 streamlines" in d["cpu_baseline"]["sample"]
