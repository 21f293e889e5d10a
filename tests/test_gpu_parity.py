"""GPU parity: the CUDA path through the C ABI against the oracle, bit-exact
(integer counts, tolerance 0), on the golden worked example, adversarial tiny
grids (ties, off-grid points, T = 0/1, long segments, set overflow), the tiny
and HCP-shaped synthetic subjects, every loader / prefilter / mode option, and
host, page-locked and device inputs."""
import os

import numpy as np
import pytest

import oracle
import synth
from synth import tiny
from tests.gpu_helpers import range_end_streamlines, run_gpu

pytestmark = pytest.mark.gpu

U = 1024


def _opts(prefilter, staging, target=0, sampling=0, skip=1):
    from paper_2302_09247_gb300 import fastcod as fc
    return {fc.FASTCOD_OPT_PREFILTER: prefilter, fc.FASTCOD_OPT_STAGING: staging,
            fc.FASTCOD_OPT_TARGET_MODE: target, fc.FASTCOD_OPT_SAMPLING: sampling, fc.FASTCOD_OPT_WALKED_STEPS: 1,
            fc.FASTCOD_OPT_SEGMENT_SKIP: skip}


def _oracle_flags(target, sampling):
    return (oracle.TARGET_ENDPOINT if target else 0) | (oracle.VERTEX_SAMPLED if sampling else 0)


def _check(roi, lab, dims, N, M, xyz, off, where="device", opts=None, chunks=1, flags=0):
    C, Ce, st = run_gpu(roi, lab, dims, N, M, xyz, off, where, opts, chunks)
    Cr, Cer, sr = oracle.connectivity(roi, lab, dims, N, M, xyz, off, flags)
    np.testing.assert_array_equal(C, Cr)
    np.testing.assert_array_equal(Ce, Cer)
    assert st["voxel_steps"] == sr["voxel_steps"]
    assert st["pairs"] == sr["pairs"]
    assert st["streamlines"] == len(off) - 1
    # the walked streamlines' voxel steps (counted when asked): all of them
    # without the prefilter
    from paper_2302_09247_gb300 import fastcod as fc
    if opts is not None and opts.get(fc.FASTCOD_OPT_WALKED_STEPS):
        assert st["walked_steps"] <= st["voxel_steps"]
        if not opts.get(fc.FASTCOD_OPT_PREFILTER, 1):
            assert st["walked_steps"] == sr["voxel_steps"]
    else:
        assert st["walked_steps"] == 0
    return st, sr


def test_golden_toy():
    d, roi, lab, xyz, off = tiny.toy_fixture(os.path.join(tiny.GOLDEN, "toy_passthrough.json"))
    for where in ("device", "host"):
        for staging in (0, 1):
            C, Ce, _ = run_gpu(roi, lab, d["dims"], d["N"], d["M"], xyz, off, where, _opts(1, staging))
            assert C.tolist() == d["C_expected"]
            assert Ce.tolist() == d["C_end_expected"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("prefilter,staging", [(1, 1), (1, 0), (0, 1)])
@pytest.mark.parametrize("target,sampling", [(0, 0), (1, 0), (0, 1)])
def test_adversarial_tiny(seed, prefilter, staging, target, sampling):
    rng = np.random.default_rng(1000 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 10, size=3))
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=6, n_labels=int(rng.integers(1, 7)),
                                         many_to_one=bool(seed % 2))
    xyz, off = tiny.random_streamlines(rng, dims, 300, max_len=40)
    _check(roi, lab, dims, N, M, xyz, off, "device", _opts(prefilter, staging, target, sampling),
           flags=_oracle_flags(target, sampling))


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("prefilter", [1, 0])
@pytest.mark.parametrize("target,sampling", [(0, 0), (1, 0)])
def test_adversarial_tiny_every_segment_walked(seed, prefilter, target, sampling):
    # the walk's skip of far short segments switched off: every segment is
    # walked voxel by voxel, and the result is the same
    rng = np.random.default_rng(2000 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 10, size=3))
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=6, n_labels=int(rng.integers(1, 7)),
                                         many_to_one=bool(seed % 2))
    xyz, off = tiny.random_streamlines(rng, dims, 300, max_len=40)
    _check(roi, lab, dims, N, M, xyz, off, "device", _opts(prefilter, 1, target, sampling, skip=0),
           flags=_oracle_flags(target, sampling))


def test_long_segments_wide_walk():
    # segment extents >= 2^16 units take the 64-bit walk; coordinates near 2^23
    rng = np.random.default_rng(7)
    dims = (40, 30, 20)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=0, n_labels=5, p_roi=0.05, p_lab=0.1)
    n = 200
    pts = []
    counts = []
    for _ in range(n):
        T = int(rng.integers(2, 6))
        v = rng.integers(-(1 << 23), 1 << 23, size=(T, 3))
        v[:, :] = np.clip(v, -60 * U, 60 * U) if rng.random() < 0.7 else v
        pts.append(v)
        counts.append(T)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    xyz = np.concatenate(pts).astype(np.int32)
    for staging in (0, 1):
        _check(roi, lab, dims, N, M, xyz, off, "device", _opts(1, staging))


def test_set_overflow_path():
    # every voxel is its own ROI row and carries one of 200 labels; straight
    # streamlines across the grid meet more rows and labels than the on-chip
    # tables hold, so the exact global-memory path runs
    rng = np.random.default_rng(8)
    dims = (64, 40, 24)
    nvox = dims[0] * dims[1] * dims[2]
    roi = np.arange(nvox, dtype=np.int32).reshape(dims[2], dims[1], dims[0])
    lab = rng.integers(0, 201, size=nvox).astype(np.uint16).reshape(roi.shape)
    n, T = 150, 9
    xyz = rng.integers(0, np.array(dims) * U, size=(n, T, 3)).reshape(-1, 3).astype(np.int32)
    off = np.arange(0, T * n + 1, T, dtype=np.int64)
    st, _ = _check(roi, lab, dims, nvox, 200, xyz, off, "device", _opts(1, 1))
    assert st["overflow"] > 0
    st, _ = _check(roi, lab, dims, nvox, 200, xyz, off, "device", _opts(0, 1))  # walked steps counted in full
    assert st["overflow"] > 0


@pytest.mark.parametrize("where", ["device", "host", "pinned"])
def test_cfg0_full(where):
    vols, tr = synth.make_subject(0)
    st, sr = _check(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, where)
    assert sr["n_contributing"] <= st["survivors"] <= tr.n_streamlines


@pytest.mark.parametrize("in_place", [1, 0])
@pytest.mark.parametrize("shift", [0, 1])
def test_pinned_read_in_place_or_copied(in_place, shift):
    """Page-locked inputs read in place over the host link (aligned) or
    copied (option off, or xyz not 16-byte aligned: shift = 4 bytes)."""
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    vols, tr = synth.make_subject(0)
    buf = torch.empty(tr.xyz.size + 4, dtype=torch.int32).pin_memory()
    xp = buf[shift:shift + tr.xyz.size].view(-1, 3)
    xp.copy_(torch.from_numpy(tr.xyz))
    op = torch.from_numpy(tr.offsets).pin_memory()
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_HOST_IN_PLACE, in_place)
        ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
        for _ in range(2):
            ctx.add_streamlines(xp, op)
        C, Ce, st = ctx.connectivity(), ctx.endpoint_connectivity(), ctx.stats()
    Cr, Cer, sr = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets)
    np.testing.assert_array_equal(C, 2 * Cr)
    np.testing.assert_array_equal(Ce, 2 * Cer)
    assert st["voxel_steps"] == 2 * sr["voxel_steps"]


def test_cfg0_chunked_and_options():
    vols, tr = synth.make_subject(0)
    for prefilter, staging in ((1, 1), (0, 0), (1, 0)):
        _check(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device",
               _opts(prefilter, staging), chunks=7)


def test_cfg1_subset_all_modes():
    vols, tr = synth.make_subject(1, n_streamlines=200_000)
    for target, sampling in ((0, 0), (1, 0), (0, 1)):
        _check(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device",
               _opts(1, 1, target, sampling), flags=_oracle_flags(target, sampling))
    # the benchmark's measure of the walk itself: no prefilter, no segment skip
    _check(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device",
           _opts(0, 1, skip=0))


def test_cfg1_full_bench_configuration():
    # HCP-shaped subject, 2,000,000 streamlines, device-resident inputs and the
    # default loader: the configuration the benchmark times
    vols, tr = synth.make_subject(1)
    C, Ce, st = run_gpu(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device")
    Cr, Cer, sr = oracle.connectivity_chunked(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                              tr.offsets)
    np.testing.assert_array_equal(C, Cr)
    np.testing.assert_array_equal(Ce, Cer)
    assert st["voxel_steps"] == sr["voxel_steps"]
    assert st["pairs"] == sr["pairs"]
    assert sr["n_contributing"] <= st["survivors"]


@pytest.mark.parametrize("near_log2", [-1, 0, 1, 2, 3])
@pytest.mark.parametrize("seed", range(3))
def test_near_grid_cell_sizes(near_log2, seed):
    # every near-grid cell size must keep the prefilter conservative: the
    # result is the same exact C whatever the cell size
    from paper_2302_09247_gb300 import fastcod as fc
    rng = np.random.default_rng(3000 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 40, size=3))
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=0, n_labels=5, p_roi=0.02, p_lab=0.05)
    xyz, off = tiny.random_streamlines(rng, dims, 400, max_len=60)
    _check(roi, lab, dims, N, M, xyz, off, "device", {fc.FASTCOD_OPT_NEAR_LOG2: near_log2})
    vols, tr = synth.make_subject(0, n_streamlines=5000)
    _check(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device",
           {fc.FASTCOD_OPT_NEAR_LOG2: near_log2})


@pytest.mark.parametrize("N,M", [(20000, 5000), (20000, 8), (100, 5000), (100, 8)])
def test_walk_set_forms(N, M):
    # the walk keeps V_s / T_s as bitmaps when N <= 16384 and M < 4096, else as
    # hash sets: all four combinations against the oracle, with many distinct
    # rows and labels along each streamline
    rng = np.random.default_rng(N + M)
    dims = (24, 20, 18)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=N, n_labels=M, p_roi=0.3, p_lab=0.4, many_to_one=True)
    xyz, off = tiny.random_streamlines(rng, dims, 1500, max_len=40)
    for target in (0, 1):
        _check(roi, lab, dims, N, M, xyz, off, "device", _opts(1, 1, target, 0), flags=_oracle_flags(target, 0))


def test_batch_mixed_set_forms():
    # a batch whose subjects need the hash form (N > 16384) beside small ones
    from paper_2302_09247_gb300 import fastcod as fc
    from tests.gpu_helpers import as_device
    subs = []
    for k, (N, M) in enumerate(((20000, 8), (50, 6), (300, 4500))):
        rng = np.random.default_rng(77 + k)
        dims = (16 + k, 14, 12)
        roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=N, n_labels=M, p_roi=0.3, p_lab=0.4,
                                             many_to_one=True)
        xyz, off = tiny.random_streamlines(rng, dims, 600, max_len=30)
        subs.append((roi, lab, dims, N, M, xyz, off))
    keep, objs, outs = [], [], []
    for roi, lab, dims, N, M, xyz, off in subs:
        r, l, x, o = as_device(roi), as_device(lab), as_device(xyz), as_device(off)
        C = np.full((N, M), -7, dtype=np.int32)
        Ce = np.full((N, M), -7, dtype=np.int32)
        keep += [r, l, x, o]
        outs.append((C, Ce))
        objs.append(fc.make_subject(r, l, dims, N, M, x, o, C, Ce))
    with fc.Context(0) as ctx:
        fc.fastcod_batch_run(ctx.ctx, objs)
    for (roi, lab, dims, N, M, xyz, off), (C, Ce) in zip(subs, outs):
        Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
        np.testing.assert_array_equal(C, Cr)
        np.testing.assert_array_equal(Ce, Cer)


@pytest.mark.parametrize("dims", [(37, 11, 1), (33, 9, 2), (65, 7, 3), (20, 17, 5), (70, 13, 6)])
def test_thin_volumes_one_call_and_batched(dims):
    """Volume preparation takes four planes per thread and a brick's depth is
    four planes: grids of 1, 2, 3, 5 and 6 planes, with rows that are not a
    multiple of 32 voxels, through the single-subject call and through a
    batch (whose preparation launch also zeroes the outputs), against the
    oracle."""
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    from tests.gpu_helpers import as_device

    rng = np.random.default_rng(sum(dims))
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=5, n_labels=4, p_roi=0.15, p_lab=0.25)
    xyz, off = tiny.random_streamlines(rng, dims, 400, max_len=30)
    _check(roi, lab, dims, N, M, xyz, off, "device", _opts(1, 1))
    Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    C = torch.full((N, M), -3, dtype=torch.int32, device="cuda:0")
    Ce = torch.full((N, M), -3, dtype=torch.int32, device="cuda:0")
    keep = [as_device(roi), as_device(lab), as_device(xyz), as_device(off)]
    torch.cuda.synchronize()
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_AUTOTUNE, 0)
        fc.fastcod_batch_run(ctx.ctx, [fc.make_subject(*keep[:2], dims, N, M, keep[2], keep[3], C, Ce)])
    np.testing.assert_array_equal(C.cpu().numpy(), Cr)
    np.testing.assert_array_equal(Ce.cpu().numpy(), Cer)


def test_vertices_beside_and_far_off_the_grid():
    """The prefilter's near lookup clamps only its word index: for a voxel
    off the grown grid it may read any word, which is conservative because
    such a voxel has no ROI or labelled neighbour.  Short walks just outside
    each face, walks near the ends of the coordinate range, and streamlines
    that come in from far away in one long segment, against the oracle."""
    rng = np.random.default_rng(77)
    dims = (24, 20, 18)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=5, n_labels=4, p_roi=0.1, p_lab=0.2)
    lim = (1 << 24) - 1
    pts, counts = [], []
    for i in range(400):
        kind = i % 4
        c = rng.uniform(0, 1, size=3) * np.array(dims) * U
        if kind == 1:  # beside a face, 1 to 3 voxels out
            a = int(rng.integers(3))
            c[a] = (-rng.uniform(0.1, 3) * U) if rng.random() < 0.5 else (dims[a] + rng.uniform(0, 3)) * U
        elif kind == 2:  # near the ends of the coordinate range on some axes
            for a in range(3):
                if rng.random() < 0.6:
                    c[a] = rng.choice([-lim + 4096, lim - 4096]) + rng.uniform(-2000, 2000)
        T = int(rng.integers(2, 40))
        steps = rng.integers(-512, 513, size=(T, 3))
        v = np.clip(np.round(c) + np.cumsum(steps, axis=0), -lim, lim - 1).astype(np.int64)
        if kind == 3:  # in from far away in one long segment
            far = rng.choice([-lim + 100, lim - 100], size=3)
            v = np.vstack([far, v])
        pts.append(v)
        counts.append(len(v))
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    xyz = np.concatenate(pts).astype(np.int32)
    for staging in (0, 1):
        _check(roi, lab, dims, N, M, xyz, off, "device", _opts(1, staging))


def test_coordinates_at_the_ends_of_the_range():
    """Vertices exactly at -2^24 and 2^24 - 1, the ends of the accepted
    coordinate range: segments across the whole range on one, two and three
    axes (the walk's 64-bit cross-products at their largest), segments lying
    in an extreme plane, single vertices at the corners, and segments from
    the grid out to an extreme, against the oracle with every loader and
    with the prefilter and the segment skip on and off."""
    rng = np.random.default_rng(2024)
    dims = (20, 17, 23)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=6, n_labels=5, p_roi=0.15, p_lab=0.25)
    xyz, off = range_end_streamlines(rng, dims)
    assert xyz.min() == -(1 << 24) and xyz.max() == (1 << 24) - 1
    for prefilter in (1, 0):
        for staging in (0, 1):
            for skip in (1, 0):
                _check(roi, lab, dims, N, M, xyz, off, "device", _opts(prefilter, staging, skip=skip))


@pytest.mark.parametrize("ctas", [2, 3])
@pytest.mark.parametrize("staging", [1, 0])
def test_prefilter_launch_shapes(ctas, staging):
    """The single-subject prefilter as one CTA of 16 warps per SM (the
    default register budget) and as three CTAs of 8 at 80 registers, with the
    bulk-copy and the direct loader, on an HCP-shaped subset (near grid in
    global memory) and on the tiny subject (near grid staged in shared
    memory), against the oracle."""
    from paper_2302_09247_gb300 import fastcod as fc
    opts = dict(_opts(1, staging))
    opts[fc.FASTCOD_OPT_PREFILTER_CTAS] = ctas
    for cfg, n in ((1, 30_000), (0, 20_000)):
        vols, tr = synth.make_subject(cfg, n_streamlines=n)
        _check(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets, "device", opts)
