"""Error conventions of the C ABI on a GPU: invalid inputs found on the host
and on the device, call order, and a context that stays usable after reset."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import as_device

pytestmark = pytest.mark.gpu


@pytest.fixture
def fc():
    from paper_2302_09247_gb300 import fastcod
    return fastcod


@pytest.fixture(scope="module")
def tiny0():
    return synth.make_subject(0, n_streamlines=500)


def _ctx_with_volumes(fc, vols, where="device"):
    ctx = fc.Context(0)
    if where == "device":
        ctx.set_volumes(as_device(vols.roi), as_device(vols.lab), vols.dims, vols.n_roi, vols.n_targets)
    else:
        ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
    return ctx


def test_state_and_argument_errors(fc, tiny0):
    vols, tr = tiny0
    with fc.Context(0) as ctx:
        with pytest.raises(fc.FastCodError) as e:
            ctx.add_streamlines(tr.xyz, tr.offsets)
        assert e.value.code == fc.FASTCOD_ESTATE
        with pytest.raises(fc.FastCodError) as e:
            ctx.shape()
        assert e.value.code == fc.FASTCOD_ESTATE
        with pytest.raises(fc.FastCodError) as e:
            fc.fastcod_set_volumes(ctx.ctx, vols.roi, vols.lab, (0, 1, 1))
        assert e.value.code == fc.FASTCOD_EINVAL
        with pytest.raises(fc.FastCodError):
            fc.fastcod_set_option(ctx.ctx, 999, 1)


@pytest.mark.parametrize("where", ["device", "host"])
def test_volume_values_rejected(fc, tiny0, where):
    vols, _ = tiny0
    with fc.Context(0) as ctx:
        lab = vols.lab.copy()
        lab.reshape(-1)[123] = vols.n_targets + 1
        src = as_device(lab) if where == "device" else lab
        roi = as_device(vols.roi) if where == "device" else vols.roi
        with pytest.raises(fc.FastCodError) as e:
            ctx.set_volumes(roi, src, vols.dims, vols.n_roi, vols.n_targets)
        assert e.value.code == fc.FASTCOD_EINVAL
        bad = vols.roi.copy()
        bad.reshape(-1)[5] = vols.n_roi
        src = as_device(bad) if where == "device" else bad
        with pytest.raises(fc.FastCodError) as e:
            ctx.set_volumes(src, vols.lab if where == "host" else as_device(vols.lab), vols.dims,
                            vols.n_roi, vols.n_targets)
        assert e.value.code == fc.FASTCOD_EINVAL
        # N and M inferred from the volumes
        n, m = ctx.set_volumes(vols.roi, vols.lab, vols.dims)
        assert (n, m) == (int(vols.roi.max()) + 1, int(vols.lab.max()))


@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("staging", [0, 1])
def test_device_detected_input_errors_then_reset(fc, tiny0, where, staging):
    vols, tr = tiny0
    ctx = _ctx_with_volumes(fc, vols)
    ctx.set_option(fc.FASTCOD_OPT_STAGING, staging)
    put = as_device if where == "device" else (lambda a: np.ascontiguousarray(a))
    try:
        # non-monotone offsets
        off = tr.offsets.copy()
        off[10], off[11] = off[11], off[10]
        ctx.add_streamlines(put(tr.xyz), put(off))
        with pytest.raises(fc.FastCodError) as e:
            ctx.connectivity()
        assert e.value.code == fc.FASTCOD_EINVAL and "offsets" in str(e.value)
        ctx.reset()
        # last offset != n_vertices
        off = tr.offsets.copy()
        off[-1] -= 1
        fc.fastcod_add_streamlines(ctx.ctx, put(tr.xyz), put(off), n_vertices=tr.n_vertices)
        with pytest.raises(fc.FastCodError) as e:
            ctx.sync()
        assert e.value.code == fc.FASTCOD_EINVAL
        ctx.reset()
        # coordinate out of range
        xyz = tr.xyz.copy()
        xyz[37, 1] = 1 << 24
        ctx.add_streamlines(put(xyz), put(tr.offsets))
        with pytest.raises(fc.FastCodError) as e:
            ctx.connectivity()
        assert e.value.code == fc.FASTCOD_EINVAL and "coordinate" in str(e.value)
        ctx.reset()
        # the lower end of [-2^24, 2^24) is valid
        xyz = tr.xyz.copy()
        xyz[37, 1] = -(1 << 24)
        ctx.add_streamlines(put(xyz), put(tr.offsets))
        ctx.sync()
        # the context is usable again after reset
        ctx.reset()
        ctx.add_streamlines(put(tr.xyz), put(tr.offsets))
        C = ctx.connectivity()
        Cr, _, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                       tr.offsets)
        np.testing.assert_array_equal(C, Cr)
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def mid():
    return synth.make_subject(1, n_streamlines=60_000)


@pytest.mark.parametrize("where", ["device", "host"])
def test_offset_patterns_across_warp_ranges(fc, mid, where):
    # the prefilter gives every warp about the same number of vertices (a
    # search over the offsets): invalid offsets anywhere are still reported,
    # and valid but lopsided length mixes still count exactly
    vols, tr = mid
    put = as_device if where == "device" else (lambda a: np.ascontiguousarray(a))
    ns, nv = tr.n_streamlines, tr.n_vertices
    bad = []
    o = tr.offsets.copy()
    o[ns // 2] = nv + 1000  # a spike past the end
    bad.append(o)
    o = tr.offsets.copy()
    o[ns // 3] = -1
    bad.append(o)
    o = tr.offsets.copy()
    o[ns // 4:ns // 4 + 5000] = o[ns // 4:ns // 4 + 5000][::-1].copy()  # a decreasing block
    bad.append(o)
    o = tr.offsets.copy()
    o[1:-1] = o[1:-1][::-1].copy()  # decreasing everywhere inside
    bad.append(o)
    with _ctx_with_volumes(fc, vols) as ctx:
        for o in bad:
            ctx.add_streamlines(put(tr.xyz), put(o))
            with pytest.raises(fc.FastCodError) as e:
                ctx.connectivity()
            assert e.value.code == fc.FASTCOD_EINVAL and "offsets" in str(e.value)
            ctx.reset()
        # valid: one streamline holds every vertex among empty ones; and a
        # few very long streamlines among short ones
        T = np.diff(tr.offsets)
        lop = np.zeros(ns + 1, np.int64)
        lop[ns // 2 + 1:] = nv
        k = np.arange(ns)
        T2 = np.where(k % 997 == 0, 0, T)
        T2[7] += nv - int(T2.sum())
        for off in (lop, np.concatenate([[0], np.cumsum(T2)]).astype(np.int64)):
            assert off[-1] == nv and (np.diff(off) >= 0).all()
            ctx.reset()
            ctx.add_streamlines(put(tr.xyz), put(off))
            C, Ce, st = ctx.connectivity(), ctx.endpoint_connectivity(), ctx.stats()
            Cr, Cer, sr = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets,
                                              tr.xyz, off)
            np.testing.assert_array_equal(C, Cr)
            np.testing.assert_array_equal(Ce, Cer)
            assert st["voxel_steps"] == sr["voxel_steps"]


def test_misaligned_device_xyz_by_raw_address(fc, tiny0):
    # a raw device address 4 bytes past a 16-byte boundary is staged, not
    # rejected, and counts exactly
    import torch
    vols, tr = tiny0
    with _ctx_with_volumes(fc, vols) as ctx:
        flat = torch.from_numpy(np.concatenate([np.zeros(1, np.int32), tr.xyz.reshape(-1)])).cuda()
        off = as_device(tr.offsets)
        fc.fastcod_add_streamlines(ctx.ctx, flat.data_ptr() + 4, off, n_vertices=tr.n_vertices,
                                   n_streamlines=tr.n_streamlines)
        Cr, _, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                       tr.offsets)
        np.testing.assert_array_equal(ctx.connectivity(), Cr)


def test_user_stream_and_reset(fc, tiny0):
    import torch
    vols, tr = tiny0
    s = torch.cuda.Stream()
    with _ctx_with_volumes(fc, vols) as ctx:
        fc.fastcod_set_stream(ctx.ctx, s)
        x, o = as_device(tr.xyz), as_device(tr.offsets)
        ctx.add_streamlines(x, o)
        ctx.add_streamlines(x, o)
        C2 = ctx.connectivity()
        ctx.reset()
        assert ctx.connectivity().sum() == 0
        ctx.add_streamlines(x, o)
        C1 = ctx.connectivity()
        np.testing.assert_array_equal(C2, 2 * C1)
        st = ctx.stats()
        assert st["streamlines"] == tr.n_streamlines and st["vertices"] == tr.n_vertices


@pytest.mark.parametrize("piece", [0, 5, "last"])
def test_bounded_wait_runs_out_then_context_recovers(fc, mid, piece):
    # the bulk-copy loader withholds one vertex piece (no copy, no barrier
    # arrival): the warp that waits for it gives up after its one-second
    # limit, drains its other copies and reports the timeout; nothing is
    # faulted, and the same context then computes the right C after reset
    vols, tr = mid
    n_pieces = (tr.n_vertices + 255) // 256
    k = n_pieces - 1 if piece == "last" else piece
    ctx = _ctx_with_volumes(fc, vols)
    try:
        xyz, off = as_device(tr.xyz), as_device(tr.offsets)
        ctx.set_option(fc.FASTCOD_OPT_TEST_WITHHOLD_PIECE, k)
        ctx.add_streamlines(xyz, off)
        with pytest.raises(fc.FastCodError) as e:
            ctx.sync()
        assert e.value.code == fc.FASTCOD_ETIMEOUT and "timed out" in str(e.value)
        ctx.set_option(fc.FASTCOD_OPT_TEST_WITHHOLD_PIECE, -1)
        ctx.reset()
        ctx.add_streamlines(xyz, off)
        C, Ce = ctx.connectivity(), ctx.endpoint_connectivity()
        Cr, Cer, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                         tr.offsets)
        np.testing.assert_array_equal(C, Cr)
        np.testing.assert_array_equal(Ce, Cer)
    finally:
        ctx.close()


def test_withheld_piece_has_no_effect_on_the_direct_loader(fc, tiny0):
    vols, tr = tiny0
    ctx = _ctx_with_volumes(fc, vols)
    try:
        ctx.set_option(fc.FASTCOD_OPT_STAGING, 0)
        ctx.set_option(fc.FASTCOD_OPT_TEST_WITHHOLD_PIECE, 0)
        ctx.add_streamlines(as_device(tr.xyz), as_device(tr.offsets))
        Cr, _, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                       tr.offsets)
        np.testing.assert_array_equal(ctx.connectivity(), Cr)
        with pytest.raises(fc.FastCodError):
            ctx.set_option(fc.FASTCOD_OPT_TEST_WITHHOLD_PIECE, -2)
    finally:
        ctx.close()


def test_unaligned_device_xyz_is_staged(fc, tiny0):
    # device xyz starting 4 bytes past a 16-byte boundary: the context, the
    # batched form and the served form copy it to an aligned buffer first
    import torch
    vols, tr = tiny0
    Cr, Cer, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                     tr.offsets)
    flat = torch.zeros(tr.xyz.size + 1, dtype=torch.int32, device="cuda:0")
    flat[1:] = torch.from_numpy(tr.xyz.reshape(-1)).cuda()
    view = flat[1:].view(-1, 3)
    assert view.data_ptr() % 16 != 0
    off = as_device(tr.offsets)
    for staging in (1, 0):
        ctx = _ctx_with_volumes(fc, vols)
        try:
            ctx.set_option(fc.FASTCOD_OPT_STAGING, staging)
            ctx.add_streamlines(view, off)
            np.testing.assert_array_equal(ctx.connectivity(), Cr)
            np.testing.assert_array_equal(ctx.endpoint_connectivity(), Cer)
        finally:
            ctx.close()
    N, M = vols.n_roi, vols.n_targets
    C = torch.zeros((N, M), dtype=torch.int32, device="cuda:0")
    Ce = torch.zeros_like(C)
    with fc.Context(0) as ctx:
        s = fc.make_subject(as_device(vols.roi), as_device(vols.lab), vols.dims, N, M, view, off, C, Ce)
        fc.fastcod_batch_run(ctx.ctx, [s])
        np.testing.assert_array_equal(C.cpu().numpy(), Cr)
        np.testing.assert_array_equal(Ce.cpu().numpy(), Cer)
        srv = fc.fastcod_server_create(ctx.ctx, 2, 0)
        try:
            Ch = np.zeros((N, M), np.int32)
            Ceh = np.zeros((N, M), np.int32)
            head = fc.make_subject(vols.roi, vols.lab, vols.dims, N, M, np.zeros((0, 3), np.int32),
                                   np.zeros(1, np.int64), Ch, Ceh)
            rid = fc.fastcod_server_submit(srv, head)
            fc.fastcod_server_push_chunk(srv, rid, view, off, last=True)
            assert fc.fastcod_server_wait(srv, rid, 60.0) == fc.FASTCOD_OK
            np.testing.assert_array_equal(Ch, Cr)
            np.testing.assert_array_equal(Ceh, Cer)
        finally:
            fc.fastcod_server_destroy(srv)


@pytest.mark.parametrize("dims", [(1, 1, 70_000), (3, 70_000, 2), (2, 3, 66_000)])
def test_long_thin_grids(fc, dims):
    # Dy or Dz past the 65,535 blocks of one launch-grid dimension: bounded
    # only by the voxel count
    from synth import tiny
    rng = np.random.default_rng(sum(dims))
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=40, n_labels=6, p_roi=0.05, p_lab=0.1,
                                         many_to_one=True)
    xyz, off = tiny.random_streamlines(rng, dims, 2000, max_len=12, margin=1)
    # streamlines within 4 voxels, placed at random voxels of the grid that
    # coordinates can reach (|coordinate| < 2^24 units = 16,384 voxels)
    reach = np.minimum(np.array(dims), 16_000)
    shift = (rng.integers(0, reach, size=(len(off) - 1, 3)) * 1024).astype(np.int64)
    xyz = (xyz.astype(np.int64) % 4096 + np.repeat(shift, np.diff(off), axis=0)).astype(np.int32)
    Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    assert Cr.sum() > 0
    for where in ("device", "host"):
        ctx = fc.Context(0)
        try:
            if where == "device":
                ctx.set_volumes(as_device(roi), as_device(lab), dims, N, M)
                ctx.add_streamlines(as_device(xyz), as_device(off))
            else:
                ctx.set_volumes(roi, lab, dims, N, M)
                ctx.add_streamlines(xyz, off)
            np.testing.assert_array_equal(ctx.connectivity(), Cr)
            np.testing.assert_array_equal(ctx.endpoint_connectivity(), Cer)
        finally:
            ctx.close()
    import torch
    C = torch.zeros((N, M), dtype=torch.int32, device="cuda:0")
    Ce = torch.zeros_like(C)
    fc.fastcod_connectivity_noalloc(0, None, as_device(roi), as_device(lab), dims, N, M, as_device(xyz),
                                    as_device(off), C, Ce)
    np.testing.assert_array_equal(C.cpu().numpy(), Cr)
    np.testing.assert_array_equal(Ce.cpu().numpy(), Cer)
