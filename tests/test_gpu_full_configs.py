"""Bit-exact parity at full size beyond the HCP-shaped subject: the high-
resolution subject (5,000,000 streamlines), the whole 64-subject batch, and
full HCP-shaped requests served concurrently in 250,000-streamline chunks.
The oracle runs on the host cores, chunked across threads (integer sums)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import as_device, run_gpu

pytestmark = pytest.mark.gpu


def _oracle(vols, tr):
    return oracle.connectivity_chunked(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets)


def test_cfg2_full_high_resolution():
    vols, tr = synth.make_subject(2)
    C, Ce, st = run_gpu(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device")
    Cr, Cer, sr = _oracle(vols, tr)
    np.testing.assert_array_equal(C, Cr)
    np.testing.assert_array_equal(Ce, Cer)
    assert st["voxel_steps"] == sr["voxel_steps"] and st["pairs"] == sr["pairs"]
    assert sr["n_contributing"] <= st["survivors"]


def test_cfg3_full_batch():
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    subs, keep, objs = [], [], []
    for s in range(1, 65):
        vols, tr = synth.make_subject(3, subject=s, n_streamlines=synth.batched_subject_draws(s)["ns"])
        N, M = vols.n_roi, vols.n_targets
        C = torch.full((N, M), -7, dtype=torch.int32, device="cuda:0")
        Ce = torch.full((N, M), -7, dtype=torch.int32, device="cuda:0")
        r, l, x, o = as_device(vols.roi), as_device(vols.lab), as_device(tr.xyz), as_device(tr.offsets)
        keep += [r, l, x, o]
        objs.append(fc.make_subject(r, l, vols.dims, N, M, x, o, C, Ce))
        subs.append((vols, tr, C, Ce))
    with fc.Context(0) as ctx:
        fc.fastcod_batch_run(ctx.ctx, objs)
        torch.cuda.synchronize()
        for i, (vols, tr, C, Ce) in enumerate(subs):
            Cr, Cer, sr = _oracle(vols, tr)
            np.testing.assert_array_equal(C.cpu().numpy(), Cr, err_msg=f"subject {i + 1}")
            np.testing.assert_array_equal(Ce.cpu().numpy(), Cer, err_msg=f"subject {i + 1}")
            st = fc.fastcod_batch_get_stats(ctx.ctx, i)
            assert st["voxel_steps"] == sr["voxel_steps"] and st["pairs"] == sr["pairs"]


def test_cfg4_served_full_requests():
    # three requests of the served workload's generator (2,000,000, 1,000,000
    # and 200,000 streamlines), every chunk pushed before any request is done,
    # so that their chunks share the device
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    chunk = 250_000
    reqs = []
    for subject, count in ((0, 2_000_000), (1, 1_000_000), (2, 200_000)):
        vols, tr = synth.make_subject(4, subject=subject, n_streamlines=count)
        reqs.append((vols, tr))
    with fc.Context(0) as ctx:
        srv = fc.fastcod_server_create(ctx.ctx, 8, 0)
        keep, ids = [], []
        try:
            for vols, tr in reqs:
                N, M = vols.n_roi, vols.n_targets
                C = torch.full((N, M), -7, dtype=torch.int32).pin_memory()
                Ce = torch.full((N, M), -7, dtype=torch.int32).pin_memory()
                roi = torch.from_numpy(vols.roi).pin_memory()
                lab = torch.from_numpy(vols.lab.view(np.int16)).pin_memory()
                head = fc.make_subject(roi, lab, vols.dims, N, M, np.zeros((0, 3), np.int32), np.zeros(1, np.int64),
                                       C, Ce)
                rid = fc.fastcod_server_submit(srv, head)
                xyz = torch.from_numpy(tr.xyz).pin_memory()
                keep += [C, Ce, roi, lab, head, xyz]
                ids.append((rid, C, Ce))
                for c in range(0, tr.n_streamlines, chunk):
                    e = min(tr.n_streamlines, c + chunk)
                    o = torch.from_numpy(tr.offsets[c:e + 1] - tr.offsets[c]).pin_memory()
                    x = xyz[int(tr.offsets[c]):int(tr.offsets[e])]
                    keep += [o, x]
                    fc.fastcod_server_push_chunk(srv, rid, x, o, last=(e == tr.n_streamlines))
            for rid, _, _ in ids:
                assert fc.fastcod_server_wait(srv, rid, 300.0) == fc.FASTCOD_OK
        finally:
            fc.fastcod_server_destroy(srv)
    for (vols, tr), (_, C, Ce) in zip(reqs, ids):
        Cr, Cer, _ = _oracle(vols, tr)
        np.testing.assert_array_equal(C.numpy(), Cr)
        np.testing.assert_array_equal(Ce.numpy(), Cer)
