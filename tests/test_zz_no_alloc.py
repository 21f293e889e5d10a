"""The allocation-free entry point, through the C ABI.

Some callers cannot allocate device memory (a host application whose own
allocator owns all of it, or a process at its memory limit); for them
fastcod_connectivity_noalloc computes C and C_end on buffers they already
hold, with its working memory in one fixed device array of the library.
Its output must equal the context API's, bit for bit (integer counts), on two
calls in a row — the second call reuses the array the first one left behind.
This file is collected last."""
import numpy as np
import pytest

import oracle
import synth
from synth import tiny
from tests.gpu_helpers import as_device, run_gpu

pytestmark = pytest.mark.gpu


def _inputs():
    cases = []
    vols, tr = synth.make_subject(0, n_streamlines=6000)
    cases.append((vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets))
    rng = np.random.default_rng(77)
    dims = (9, 7, 6)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=5, n_labels=4, many_to_one=True)
    xyz, off = tiny.random_streamlines(rng, dims, 300, max_len=25)
    cases.append((roi, lab, dims, N, M, xyz, off))
    return cases


def _noalloc(fc, case):
    import torch
    roi, lab, dims, N, M, xyz, off = case
    C = torch.full((N, M), -5, dtype=torch.int32, device="cuda:0")
    Ce = torch.full((N, M), -5, dtype=torch.int32, device="cuda:0")
    args = [as_device(roi), as_device(lab), as_device(xyz), as_device(off)]
    fc.fastcod_connectivity_noalloc(0, None, args[0], args[1], dims, N, M, args[2], args[3], C, Ce)
    return C.cpu().numpy(), Ce.cpu().numpy()


def test_noalloc_equals_context_api_on_consecutive_calls():
    from paper_2302_09247_gb300 import fastcod as fc
    cases = _inputs()
    refs = [run_gpu(*c, where="device")[:2] for c in cases]
    # two calls in a row on the same input, then the other input, then again
    for k in (0, 0, 1, 0, 1):
        C, Ce = _noalloc(fc, cases[k])
        np.testing.assert_array_equal(C, refs[k][0])
        np.testing.assert_array_equal(Ce, refs[k][1])


def test_noalloc_rejects_sizes_beyond_its_scratch_and_host_memory():
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    roi, lab, dims, N, M, xyz, off = _inputs()[1]
    C = torch.zeros((N, 1024), dtype=torch.int32, device="cuda:0")
    with pytest.raises(fc.FastCodError) as e:
        fc.fastcod_connectivity_noalloc(0, None, as_device(roi), as_device(lab), dims, N, 1024, as_device(xyz),
                                        as_device(off), C, C)
    assert e.value.code == fc.FASTCOD_EINVAL and "n_targets" in str(e.value)
    Ch = np.zeros((N, M), dtype=np.int32)
    with pytest.raises(fc.FastCodError) as e:
        fc.fastcod_connectivity_noalloc(0, None, roi, lab, dims, N, M, xyz, off, Ch, Ch)
    assert e.value.code == fc.FASTCOD_EINVAL and "device memory" in str(e.value)
    # the entry point still works afterwards
    C, _ = _noalloc(fc, _inputs()[1])
    np.testing.assert_array_equal(C, run_gpu(*_inputs()[1], where="device")[0])


def _adversarial():
    # lattice-snapped vertices on planes, edges and corners, T = 0 and T = 1
    # streamlines, points off the grid
    rng = np.random.default_rng(78)
    dims = (8, 6, 7)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=6, n_labels=5, many_to_one=True)
    xyz, off = tiny.random_streamlines(rng, dims, 400, max_len=30)
    assert (np.diff(off) == 0).any() and (np.diff(off) == 1).any()
    return roi, lab, dims, N, M, xyz, off


def test_noalloc_equals_the_oracle():
    from paper_2302_09247_gb300 import fastcod as fc
    for case in _inputs() + [_adversarial()]:
        roi, lab, dims, N, M, xyz, off = case
        Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
        for _ in range(2):
            C, Ce = _noalloc(fc, case)
            np.testing.assert_array_equal(C, Cr)
            np.testing.assert_array_equal(Ce, Cer)


def test_noalloc_rejects_invalid_input_then_recovers():
    # each invalid input is reported; the next valid call starts from a clean
    # scratch and gives the right result
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    case = _adversarial()
    roi, lab, dims, N, M, xyz, off = case
    Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    C = torch.zeros((N, M), dtype=torch.int32, device="cuda:0")
    Ce = torch.zeros((N, M), dtype=torch.int32, device="cuda:0")
    bad_off = off.copy()
    bad_off[20], bad_off[21] = bad_off[21] + 3, bad_off[20]        # decreasing
    bad_xyz = xyz.copy()
    bad_xyz[len(xyz) // 2, 2] = 1 << 24                              # coordinate at 2^24
    bad_lab = lab.copy()
    bad_lab.reshape(-1)[11] = M + 1                                  # label > M
    bad_roi = roi.copy()
    bad_roi.reshape(-1)[3] = N                                       # row >= N
    for r, l, x, o, what in ((roi, lab, xyz, bad_off, "offsets"), (roi, lab, bad_xyz, off, "coordinate"),
                             (roi, bad_lab, xyz, off, "volume"), (bad_roi, lab, xyz, off, "volume")):
        with pytest.raises(fc.FastCodError) as e:
            fc.fastcod_connectivity_noalloc(0, None, as_device(r), as_device(l), dims, N, M, as_device(x),
                                            as_device(o), C, Ce)
        assert e.value.code == fc.FASTCOD_EINVAL and what in str(e.value), str(e.value)
        Cv, Cev = _noalloc(fc, case)
        np.testing.assert_array_equal(Cv, Cr)
        np.testing.assert_array_equal(Cev, Cer)


def test_noalloc_on_a_side_stream():
    import torch
    from paper_2302_09247_gb300 import fastcod as fc
    roi, lab, dims, N, M, xyz, off = _adversarial()
    Cr, Cer, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        args = [as_device(roi), as_device(lab), as_device(xyz), as_device(off)]
        C = torch.full((N, M), -5, dtype=torch.int32, device="cuda:0")
        Ce = torch.full((N, M), -5, dtype=torch.int32, device="cuda:0")
    s.synchronize()
    fc.fastcod_connectivity_noalloc(0, s, args[0], args[1], dims, N, M, args[2], args[3], C, Ce)
    np.testing.assert_array_equal(C.cpu().numpy(), Cr)
    np.testing.assert_array_equal(Ce.cpu().numpy(), Cer)
