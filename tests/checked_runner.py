"""Parity cases run against the bounds-checked build of the library
(FASTCOD_LIBRARY names it; tests/test_gpu_checked.py starts this file in a
process of its own).  Every result must equal the oracle's and no bounds
check may fail (a failed check is reported as an error by the call)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from synth import tiny  # noqa: E402
from tests.gpu_helpers import as_device, range_end_streamlines, run_gpu  # noqa: E402
from tests.parcellation_cases import DOUBLE_ROUNDING_ROWS, as_matrix, midpoint_rows  # noqa: E402


def check(case, opts=None, flags=0, where="device"):
    roi, lab, dims, N, M, xyz, off = case
    C, Ce, st = run_gpu(roi, lab, dims, N, M, xyz, off, where, opts)
    Cr, Cer, sr = oracle.connectivity(roi, lab, dims, N, M, xyz, off, flags)
    assert np.array_equal(C, Cr) and np.array_equal(Ce, Cer), "result differs from the oracle"
    assert st["voxel_steps"] == sr["voxel_steps"]
    return st


def main():
    from paper_2302_09247_gb300 import fastcod as fc
    assert fc.LIB_PATH.endswith("libfastcod_checked.so"), fc.LIB_PATH
    # adversarial tiny cases in every mode, prefilter on and off, every segment walked
    for seed in range(4):
        rng = np.random.default_rng(3000 + seed)
        dims = tuple(int(v) for v in rng.integers(3, 10, size=3))
        roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=6, n_labels=int(rng.integers(1, 7)),
                                             many_to_one=bool(seed % 2))
        xyz, off = tiny.random_streamlines(rng, dims, 300, max_len=40)
        case = (roi, lab, dims, N, M, xyz, off)
        for pre, skip, target, sampling in ((1, 1, 0, 0), (0, 0, 0, 0), (1, 1, 1, 0), (1, 1, 0, 1)):
            opts = {fc.FASTCOD_OPT_PREFILTER: pre, fc.FASTCOD_OPT_SEGMENT_SKIP: skip,
                    fc.FASTCOD_OPT_TARGET_MODE: target, fc.FASTCOD_OPT_SAMPLING: sampling}
            flags = (oracle.TARGET_ENDPOINT if target else 0) | (oracle.VERTEX_SAMPLED if sampling else 0)
            check(case, opts, flags)
    # vertices at both ends of the coordinate range, prefilter on and off
    rng = np.random.default_rng(2024)
    dims = (20, 17, 23)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=6, n_labels=5, p_roi=0.15, p_lab=0.25)
    xyz, off = range_end_streamlines(rng, dims)
    for pre in (1, 0):
        check((roi, lab, dims, N, M, xyz, off), {fc.FASTCOD_OPT_PREFILTER: pre, fc.FASTCOD_OPT_SEGMENT_SKIP: pre})
    # sets that outgrow the per-warp tables (the overflow path) and hash-set forms
    rng = np.random.default_rng(8)
    dims = (64, 40, 24)
    nvox = dims[0] * dims[1] * dims[2]
    roi = np.arange(nvox, dtype=np.int32).reshape(dims[2], dims[1], dims[0])
    lab = rng.integers(0, 201, size=nvox).astype(np.uint16).reshape(roi.shape)
    n, T = 150, 9
    xyz = rng.integers(0, np.array(dims) * 1024, size=(n, T, 3)).reshape(-1, 3).astype(np.int32)
    off = np.arange(0, n * T + 1, T, dtype=np.int64)
    assert check((roi, lab, dims, nvox, 200, xyz, off))["overflow"] > 0
    # the HCP-shaped subject's first 100,000 streamlines, host and device inputs
    vols, tr = synth.make_subject(1, n_streamlines=100_000)
    case = (vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets)
    check(case)
    check(case, where="host")
    # a checkpoint after the first 40,000 streamlines, resumed in a new context
    o = tr.offsets
    cut = 40_000
    with fc.Context(0) as ctx:
        ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
        ctx.add_streamlines(np.ascontiguousarray(tr.xyz[:o[cut]]), np.ascontiguousarray(o[:cut + 1]))
        ck = ctx.checkpoint()
    with fc.Context(0) as ctx:
        ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
        ctx.restore(*ck)
        ctx.add_streamlines(np.ascontiguousarray(tr.xyz[o[cut]:]), np.ascontiguousarray(o[cut:] - o[cut]))
        Cr, Cer, _ = oracle.connectivity(*case)
        assert np.array_equal(ctx.connectivity(), Cr) and np.array_equal(ctx.endpoint_connectivity(), Cer)
    # a batch of three subjects
    subs = [synth.make_subject(3, subject=s, n_streamlines=20_000) for s in (1, 2, 3)]
    keep, objs, outs = [], [], []
    for vols, tr in subs:
        import torch
        C = torch.zeros((vols.n_roi, vols.n_targets), dtype=torch.int32, device="cuda:0")
        Ce = torch.zeros_like(C)
        a = [as_device(vols.roi), as_device(vols.lab), as_device(tr.xyz), as_device(tr.offsets)]
        keep.append(a)
        outs.append((C, Ce))
        objs.append(fc.make_subject(a[0], a[1], vols.dims, vols.n_roi, vols.n_targets, a[2], a[3], C, Ce))
    with fc.Context(0) as ctx:
        fc.fastcod_batch_run(ctx.ctx, objs)
    for (vols, tr), (C, Ce) in zip(subs, outs):
        Cr, Cer, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                         tr.offsets)
        assert np.array_equal(C.cpu().numpy(), Cr) and np.array_equal(Ce.cpu().numpy(), Cer)
    # parcellation of a caller's matrix
    rows, _ = midpoint_rows(5, 100, k_max=5)
    Cm = as_matrix([r for r in rows if len(r) <= 70] + DOUBLE_ROUNDING_ROWS, 70)
    lr, fr = oracle.parcellate(Cm)
    label = np.zeros(len(Cm), np.int32)
    frac = np.zeros(Cm.shape, np.float32)
    with fc.Context(0) as ctx:
        fc.fastcod_parcellate_matrix(ctx.ctx, np.ascontiguousarray(Cm.astype(np.int32)), label, frac)
    assert np.array_equal(label, lr) and np.array_equal(frac.view(np.uint32), fr.view(np.uint32))
    print("checked build: all cases equal the oracle, no bounds check failed")


if __name__ == "__main__":
    main()
