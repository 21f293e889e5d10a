"""GPU parity of the entry points beside the path, through the C ABI, against
the oracle, bit-exact: parcellation outputs (labels and binary32 fractions),
world-mm ingest (and connectivity from world-mm input), upsampling (offsets,
vertices, the factor rule, and the super-resolved connectivity) and the
integer rescale; host and device buffers; invalid input rejected."""
import numpy as np
import pytest

import oracle
import synth
from synth import tiny
from tests.gpu_helpers import as_device
from tests.parcellation_cases import DOUBLE_ROUNDING_ROWS, as_matrix, midpoint_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    from paper_2302_09247_gb300 import fastcod
    return fastcod


def _subject_with_ties(seed):
    # tiny grids with few labels give rows with equal counts and rows of zeros
    rng = np.random.default_rng(seed)
    dims = (10, 9, 8)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=30, n_labels=4, p_roi=0.3, p_lab=0.3, many_to_one=True)
    xyz, off = tiny.random_streamlines(rng, dims, 300, max_len=10)
    return roi, lab, dims, N, M, xyz, off


@pytest.mark.parametrize("where", ["host", "device"])
def test_parcellate_matches_oracle(fc, where):
    import torch
    cases = [_subject_with_ties(s) for s in range(3)]
    vols, tr = synth.make_subject(1, n_streamlines=100_000)
    cases.append((vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets))
    for roi, lab, dims, N, M, xyz, off in cases:
        Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
        with fc.Context(0) as ctx:
            ctx.set_volumes(as_device(roi), as_device(lab), dims, N, M)
            ctx.add_streamlines(as_device(xyz), as_device(off))
            for which, ref in ((0, Cr), (1, Cer)):
                lr, fr = oracle.parcellate(ref)
                if where == "host":
                    label = np.full(N, -5, np.int32)
                    frac = np.full((N, M), -1, np.float32)
                    fc.fastcod_parcellate(ctx.ctx, which, label, frac)
                else:
                    lt = torch.full((N,), -5, dtype=torch.int32, device="cuda:0")
                    ft = torch.full((N, M), -1.0, dtype=torch.float32, device="cuda:0")
                    fc.fastcod_parcellate(ctx.ctx, which, lt, ft)
                    label, frac = lt.cpu().numpy(), ft.cpu().numpy()
                np.testing.assert_array_equal(label, lr)
                np.testing.assert_array_equal(frac.view(np.uint32), fr.view(np.uint32))  # bit-exact
                label2 = np.full(N, -5, np.int32)
                fc.fastcod_parcellate(ctx.ctx, which, label2, None)  # labels only
                np.testing.assert_array_equal(label2, lr)


@pytest.mark.parametrize("n_labels", [31, 50, 64, 70, 100, 200, 250, 360, 361, 512, 600])
def test_parcellate_row_widths(fc, n_labels):
    # every width class of the parcellation kernels: widths that are a
    # multiple of 4 read rows as int4 (1 to 4 per lane: 64, 100, 200, 360,
    # 512), the others hold 1, 2, 4, 8 or 16 entries per lane (31, 50, 70,
    # 250, 361), and the looping form past 512 labels; many-to-one ROI maps
    # so that rows collect large counts and ties
    rng = np.random.default_rng(n_labels)
    dims = (24, 20, 18)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=40, n_labels=n_labels, p_roi=0.3, p_lab=0.6,
                                         many_to_one=True)
    xyz, off = tiny.random_streamlines(rng, dims, 3000, max_len=14)
    Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    with fc.Context(0) as ctx:
        ctx.set_volumes(roi, lab, dims, N, M)
        ctx.add_streamlines(xyz, off)
        for which, ref in ((0, Cr), (1, Cer)):
            lr, fr = oracle.parcellate(ref)
            label = np.full(N, -5, np.int32)
            frac = np.full((N, M), -1, np.float32)
            fc.fastcod_parcellate(ctx.ctx, which, label, frac)
            np.testing.assert_array_equal(label, lr)
            np.testing.assert_array_equal(frac.view(np.uint32), fr.view(np.uint32))


@pytest.mark.parametrize("M", [2, 64, 70, 360, 600])
@pytest.mark.parametrize("where", ["host", "device", "device_unaligned"])
def test_parcellate_matrix_midpoints(fc, M, where):
    # a caller's matrix whose fractions lie on or 2^-55 beside binary32
    # midpoints (row sums 2^25..2^37), the rows where a binary64 quotient
    # rounded again to binary32 is one unit off, and small rows between them;
    # M = 2 / 70 / 600 run the one-register, four-register and looping
    # kernels, M = 64 / 360 the int4 kernels (one and three int4 per lane),
    # and with device buffers 4 bytes off a 16-byte boundary the scalar ones
    import torch
    k_max = {2: 0, 64: 5, 70: 5, 360: 6, 600: 7}[M]
    rows, _ = midpoint_rows(17 + M, 300, k_max=k_max)
    rows = [r for r in rows if len(r) <= M] + DOUBLE_ROUNDING_ROWS
    rng = np.random.default_rng(M)
    small = [list(rng.integers(0, 50, size=M)) for _ in range(40)] + [[0] * M]
    C = as_matrix(rows + small, M)
    C = C[rng.permutation(len(C))]
    assert C.max() < 2 ** 31
    lr, fr = oracle.parcellate(C)
    C32 = np.ascontiguousarray(C.astype(np.int32))
    N = len(C32)
    with fc.Context(0) as ctx:
        for rep in range(2):
            if where == "host":
                label = np.full(N, -5, np.int32)
                frac = np.full((N, M), -1, np.float32)
                fc.fastcod_parcellate_matrix(ctx.ctx, C32, label, frac)
            elif where == "device":
                lt = torch.full((N,), -5, dtype=torch.int32, device="cuda:0")
                ft = torch.full((N, M), -1.0, dtype=torch.float32, device="cuda:0")
                fc.fastcod_parcellate_matrix(ctx.ctx, torch.from_numpy(C32).cuda(), lt, ft)
                label, frac = lt.cpu().numpy(), ft.cpu().numpy()
            else:
                lt = torch.full((N,), -5, dtype=torch.int32, device="cuda:0")
                fb = torch.full((N * M + 1,), -1.0, dtype=torch.float32, device="cuda:0")
                cb = torch.zeros(N * M + 1, dtype=torch.int32, device="cuda:0")
                cb[1:] = torch.from_numpy(C32.reshape(-1)).cuda()
                ft, ct = fb[1:].view(N, M), cb[1:].view(N, M)
                assert ft.data_ptr() % 16 != 0 and ct.data_ptr() % 16 != 0
                fc.fastcod_parcellate_matrix(ctx.ctx, ct, lt, ft)
                label, frac = lt.cpu().numpy(), ft.cpu().numpy()
            np.testing.assert_array_equal(label, lr)
            np.testing.assert_array_equal(frac.view(np.uint32), fr.view(np.uint32))  # bit-exact


def test_parcellate_matrix_rejects_negative_counts(fc):
    C = np.array([[1, 2], [3, -4], [5, 6]], dtype=np.int32)
    label = np.zeros(3, np.int32)
    with fc.Context(0) as ctx:
        with pytest.raises(fc.FastCodError) as e:
            fc.fastcod_parcellate_matrix(ctx.ctx, C, label)
        assert e.value.code == fc.FASTCOD_EINVAL and "row 1" in str(e.value)
        C[1, 1] = 4
        frac = np.zeros((3, 2), np.float32)
        fc.fastcod_parcellate_matrix(ctx.ctx, C, label, frac)  # the context still works
        lr, fr = oracle.parcellate(C)
        np.testing.assert_array_equal(label, lr)
        np.testing.assert_array_equal(frac, fr)


def _affine(rng):
    A = np.zeros((3, 4), dtype=np.float32)
    A[:, :3] = (np.eye(3) / 1.25 + rng.normal(0, 0.03, (3, 3))).astype(np.float32)
    A[:, 3] = rng.uniform(-40, 60, 3).astype(np.float32)
    return A


@pytest.mark.parametrize("where", ["host", "device"])
def test_world_to_fixed_matches_oracle(fc, where):
    import torch
    rng = np.random.default_rng(11)
    A = _affine(rng)
    x = rng.uniform(-150, 150, size=(100_003, 3)).astype(np.float32)
    x[:7] = [[0, 0, 0], [1e-30, -1e-30, 0], [0.5, 0.25, 0.125], [-150, 150, -150], [3.9e-3, 7.81e-4, 1.0],
             [100.0, 100.0, 100.0], [-1e-3, -2e-3, -3e-3]]
    want = oracle.world_to_fixed(x, A)
    with fc.Context(0) as ctx:
        if where == "host":
            out = np.full(x.shape, -9, np.int32)
            fc.fastcod_world_to_fixed(ctx.ctx, x, A, out)
        else:
            ot = torch.full(x.shape, -9, dtype=torch.int32, device="cuda:0")
            fc.fastcod_world_to_fixed(ctx.ctx, as_device(x), A, ot)
            out = ot.cpu().numpy()
        np.testing.assert_array_equal(out, want)
        for bad in ([[np.nan, 0, 0]], [[np.inf, 0, 0]], [[1e9, 0, 0]]):
            with pytest.raises(fc.FastCodError) as e:
                fc.fastcod_world_to_fixed(ctx.ctx, np.array(bad, np.float32), A, np.zeros((1, 3), np.int32))
            assert e.value.code == fc.FASTCOD_EINVAL


def test_add_streamlines_mm_equals_fixed_point_path(fc):
    rng = np.random.default_rng(12)
    vols, tr = synth.make_subject(0)
    res = np.float32(1.25)
    A = np.zeros((3, 4), dtype=np.float32)  # world = 1.25 mm per voxel, origin at (-20, -20, -20) mm
    A[:, :3] = np.eye(3, dtype=np.float32) / res
    A[:, 3] = np.float32(20.0) / res
    x_mm = ((tr.xyz.astype(np.float64) / 1024.0) * 1.25 - 20.0).astype(np.float32)
    fixed = oracle.world_to_fixed(x_mm, A)
    Cr, Cer, sr = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, fixed, tr.offsets)
    with fc.Context(0) as ctx:
        ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
        fc.fastcod_add_streamlines_mm(ctx.ctx, x_mm, tr.offsets, A)
        fc.fastcod_add_streamlines_mm(ctx.ctx, as_device(x_mm), as_device(tr.offsets), A)
        C, Ce, st = ctx.connectivity(), ctx.endpoint_connectivity(), ctx.stats()
    np.testing.assert_array_equal(C, 2 * Cr)
    np.testing.assert_array_equal(Ce, 2 * Cer)
    assert st["voxel_steps"] == 2 * sr["voxel_steps"]


@pytest.mark.parametrize("factor", [1, 2, 4, 5, 8])
@pytest.mark.parametrize("where", ["host", "device"])
def test_upsample_matches_oracle(fc, factor, where):
    import torch
    rng = np.random.default_rng(20 + factor)
    xyz, off = tiny.random_streamlines(rng, (12, 12, 12), 5000, max_len=30)  # empty and one-vertex ones too
    want_xyz, want_off = oracle.upsample(xyz, off, factor)
    nv_out = fc.upsampled_count(off, factor)
    assert nv_out == len(want_xyz)
    with fc.Context(0) as ctx:
        if where == "host":
            out = np.full((nv_out, 3), -9, np.int32)
            oo = np.full(len(off), -9, np.int64)
            fc.fastcod_upsample(ctx.ctx, xyz, off, factor, out, oo)
        else:
            ot = torch.full((nv_out, 3), -9, dtype=torch.int32, device="cuda:0")
            oot = torch.full((len(off),), -9, dtype=torch.int64, device="cuda:0")
            fc.fastcod_upsample(ctx.ctx, as_device(xyz), as_device(off), factor, ot, oot)
            out, oo = ot.cpu().numpy(), oot.cpu().numpy()
        np.testing.assert_array_equal(oo, want_off)
        np.testing.assert_array_equal(out, want_xyz)
        with pytest.raises(fc.FastCodError):  # wrong output size
            fc.fastcod_upsample(ctx.ctx, xyz, off, factor, np.zeros((nv_out + 1, 3), np.int32), oo)
        bad = off.copy()
        bad[5], bad[6] = bad[6] + 1, bad[5]
        with pytest.raises(fc.FastCodError):  # invalid offsets
            fc.fastcod_upsample(ctx.ctx, xyz, bad, factor, out, oo)


@pytest.mark.parametrize("factor", [1, 2, 3, 16, 300, 1024])
def test_upsample_wide_coordinates(fc, factor):
    # vertices anywhere in int32 (differences up to 2^32 - 1, products d j
    # up to 2^42), streamline lengths 0..12 and 255..600 (one, two
    # and three chunks of the power-of-two kernel's 256 staged vertices):
    # power-of-two factors run the word-per-lane kernel, the others the
    # segment-per-lane one (300 past its staging capacity)
    import torch
    rng = np.random.default_rng(900 + factor)
    T = rng.integers(0, 13, size=200)
    T[:8] = [0, 1, 2, 0, 255, 256, 257, 600]
    off = np.concatenate([[0], np.cumsum(T)]).astype(np.int64)
    xyz = rng.integers(-2 ** 31, 2 ** 31, size=(int(off[-1]), 3), dtype=np.int64).astype(np.int32)
    xyz[:6] = [[-2 ** 31, 2 ** 31 - 1, 0], [2 ** 31 - 1, -2 ** 31, -1]] * 3
    want_xyz, want_off = oracle.upsample(xyz, off, factor)
    nv_out = fc.upsampled_count(off, factor)
    with fc.Context(0) as ctx:
        ot = torch.full((nv_out, 3), -9, dtype=torch.int32, device="cuda:0")
        oot = torch.full((len(off),), -9, dtype=torch.int64, device="cuda:0")
        fc.fastcod_upsample(ctx.ctx, as_device(xyz), as_device(off), factor, ot, oot)
        np.testing.assert_array_equal(oot.cpu().numpy(), want_off)
        np.testing.assert_array_equal(ot.cpu().numpy(), want_xyz)


def test_upsample_factor_matches_oracle(fc):
    rng = np.random.default_rng(30)
    with fc.Context(0) as ctx:
        for trial in range(6):
            xyz, off = tiny.random_streamlines(rng, (20, 20, 20), 500, max_len=20)
            for spacing in (1, 100, 512, 1023, 100000):
                assert fc.fastcod_upsample_factor(ctx.ctx, xyz, off, spacing) == \
                    oracle.upsample_factor(xyz, off, spacing)


def test_super_resolved_connectivity(fc):
    # the paper's super-resolution: upsample so that the spacing is at most
    # half a voxel, then count on the grid; GPU upsampling + GPU connectivity
    # equal the oracle's upsampling + oracle connectivity, in both voxel rules
    vols, tr = synth.make_subject(0, n_streamlines=4000)
    with fc.Context(0) as ctx:
        k = fc.fastcod_upsample_factor(ctx.ctx, tr.xyz, tr.offsets, 512)
        assert k == oracle.upsample_factor(tr.xyz, tr.offsets, 512)
        n = fc.upsampled_count(tr.offsets, k)
        ux, uo = np.empty((n, 3), np.int32), np.empty(len(tr.offsets), np.int64)
        fc.fastcod_upsample(ctx.ctx, tr.xyz, tr.offsets, k, ux, uo)
    wx, wo = oracle.upsample(tr.xyz, tr.offsets, k)
    np.testing.assert_array_equal(ux, wx)
    for sampling in (0, 1):
        with fc.Context(0) as ctx:
            ctx.set_option(fc.FASTCOD_OPT_SAMPLING, sampling)
            ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
            ctx.add_streamlines(ux, uo)
            C = ctx.connectivity()
        Cr, _, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, wx, wo,
                                       oracle.VERTEX_SAMPLED if sampling else 0)
        np.testing.assert_array_equal(C, Cr)


@pytest.mark.parametrize("where", ["host", "device"])
def test_rescale_matches_oracle(fc, where):
    import torch
    rng = np.random.default_rng(40)
    xyz = rng.integers(-300000, 300000, size=(50_001, 3)).astype(np.int32)
    num, den, add = [25, 25, 25], [14, 14, 14], [512 * 11, 512 * 11, 512 * 11]
    want = oracle.rescale(xyz, num, den, add)
    with fc.Context(0) as ctx:
        if where == "host":
            out = np.full(xyz.shape, -9, np.int32)
            fc.fastcod_rescale(ctx.ctx, xyz, num, den, add, out)
        else:
            ot = torch.full(xyz.shape, -9, dtype=torch.int32, device="cuda:0")
            fc.fastcod_rescale(ctx.ctx, as_device(xyz), num, den, add, ot)
            out = ot.cpu().numpy()
        np.testing.assert_array_equal(out, want)
        with pytest.raises(fc.FastCodError):
            fc.fastcod_rescale(ctx.ctx, np.array([[16000000, 0, 0]], np.int32), [2, 1, 1], [1, 1, 1], [0, 0, 0],
                               np.zeros((1, 3), np.int32))


def test_profile_counts_calls_beside_the_path(fc):
    # while profiling, each call beside the path adds its kernels' device time
    vols, tr = synth.make_subject(0, n_streamlines=2000)
    with fc.Context(0) as ctx:
        ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
        ctx.add_streamlines(tr.xyz, tr.offsets)
        label = np.empty(vols.n_roi, np.int32)
        fc.fastcod_parcellate(ctx.ctx, 0, label, None)
        assert ctx.profile()["aux_calls"] == 0  # profiling off
        ctx.set_option(fc.FASTCOD_OPT_PROFILE, 1)
        fc.fastcod_parcellate(ctx.ctx, 0, label, None)
        n = fc.upsampled_count(tr.offsets, 2)
        fc.fastcod_upsample(ctx.ctx, tr.xyz, tr.offsets, 2, np.empty((n, 3), np.int32),
                            np.empty(len(tr.offsets), np.int64))
        p = ctx.profile()
        assert p["aux_calls"] == 2 and p["ms_aux"] > 0.0
