"""GPU parity of the batched form (fastcod_batch_run): every subject's C and
C_end equal the oracle's, bit-exact, for heterogeneous subjects (grids, N, M,
streamline counts), host and device inputs, graph replay with new input
data, and with or without the autotuner."""
import numpy as np
import pytest

import oracle
import synth
from synth import tiny
from tests.gpu_helpers import as_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    from paper_2302_09247_gb300 import fastcod
    return fastcod


def _subjects(seed_count=4, ns=4000):
    """Heterogeneous small subjects: batched-preset shapes with few streamlines,
    the tiny subject, and two adversarial tiny grids."""
    out = []
    for subj in range(1, seed_count + 1):
        vols, tr = synth.make_subject(3, subject=subj, n_streamlines=ns)
        out.append((vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets))
    vols, tr = synth.make_subject(0, n_streamlines=3000)
    out.append((vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets))
    for seed in (5, 6):
        rng = np.random.default_rng(seed)
        dims = tuple(int(v) for v in rng.integers(4, 9, size=3))
        roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=4, n_labels=3, many_to_one=True)
        xyz, off = tiny.random_streamlines(rng, dims, 200, max_len=30)
        out.append((roi, lab, dims, N, M, xyz, off))
    return out


def _run_batch(fc, ctx, subs, where):
    keep, objs, outs = [], [], []
    for roi, lab, dims, N, M, xyz, off in subs:
        if where == "device":
            r, l, x, o = as_device(roi), as_device(lab), as_device(xyz), as_device(off)
        else:
            r, l, x, o = (np.ascontiguousarray(roi), np.ascontiguousarray(lab), np.ascontiguousarray(xyz),
                          np.ascontiguousarray(off))
        C = np.full((N, M), -7, dtype=np.int32)
        Ce = np.full((N, M), -7, dtype=np.int32)
        keep += [r, l, x, o]
        outs.append((C, Ce))
        objs.append(fc.make_subject(r, l, dims, N, M, x, o, C, Ce))
    fc.fastcod_batch_run(ctx.ctx, objs)
    return outs


def _oracle(sub):
    roi, lab, dims, N, M, xyz, off = sub
    C, Ce, st = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    return C, Ce, st


@pytest.mark.parametrize("where", ["device", "host"])
def test_batch_matches_oracle(fc, where):
    subs = _subjects()
    with fc.Context(0) as ctx:
        outs = _run_batch(fc, ctx, subs, where)
        info = fc.fastcod_batch_get_info(ctx.ctx)
        assert info["n_subjects"] == len(subs)
        assert info["tasks"] >= len(subs)
        for i, (sub, (C, Ce)) in enumerate(zip(subs, outs)):
            Cr, Cer, sr = _oracle(sub)
            np.testing.assert_array_equal(C, Cr, err_msg=f"subject {i}")
            np.testing.assert_array_equal(Ce, Cer, err_msg=f"subject {i}")
            st = fc.fastcod_batch_get_stats(ctx.ctx, i)
            assert st["voxel_steps"] == sr["voxel_steps"] and st["pairs"] == sr["pairs"]
            assert st["streamlines"] == len(sub[6]) - 1
            # the same survivors as the plain path's
            with fc.Context(0) as one:
                roi, lab, dims, N, M, xyz, off = sub
                one.set_volumes(roi, lab, dims, N, M)
                one.add_streamlines(xyz, off)
                assert st["survivors"] == one.stats()["survivors"]


def test_batch_graph_replay_sees_new_data(fc):
    subs = _subjects(seed_count=2, ns=3000)
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_AUTOTUNE, 0)
        _run_batch(fc, ctx, subs, "host")
        # same shapes, different data: the vertex array reversed (every
        # streamline reversed, in reverse order) keeps C and changes C_end
        subs2 = []
        for roi, lab, dims, N, M, xyz, off in subs:
            xyz2 = np.ascontiguousarray(xyz[::-1])
            off2 = np.ascontiguousarray(off[-1] - off[::-1])
            subs2.append((roi, lab, dims, N, M, xyz2, off2))
        outs = _run_batch(fc, ctx, subs2, "host")
        assert fc.fastcod_batch_get_info(ctx.ctx)["graph_reused"] == 1
        for sub, (C, Ce) in zip(subs2, outs):
            Cr, Cer, _ = _oracle(sub)
            np.testing.assert_array_equal(C, Cr)
            np.testing.assert_array_equal(Ce, Cer)


def test_batch_autotune_identical_results(fc):
    subs = _subjects(seed_count=3, ns=2000)
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_AUTOTUNE, 1)
        a = _run_batch(fc, ctx, subs, "device")
        info = fc.fastcod_batch_get_info(ctx.ctx)
        assert info["tuned"] == 1 and info["prefilter_ctas"] in (2, 3) and -1 <= info["near_log2"] <= 3
        assert info["task_vertices"] in (1 << 14, 1 << 15, 1 << 16, 1 << 18)
        b = _run_batch(fc, ctx, subs, "device")
        assert fc.fastcod_batch_get_info(ctx.ctx)["tuned"] == 0
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_AUTOTUNE, 0)
        ctx.set_option(fc.FASTCOD_OPT_NEAR_LOG2, 3)
        c = _run_batch(fc, ctx, subs, "device")
    for (C1, E1), (C2, E2), (C3, E3) in zip(a, b, c):
        np.testing.assert_array_equal(C1, C2)
        np.testing.assert_array_equal(C1, C3)
        np.testing.assert_array_equal(E1, E3)


def test_batch_equals_plain_path(fc):
    subs = _subjects(seed_count=2, ns=5000)
    with fc.Context(0) as ctx:
        outs = _run_batch(fc, ctx, subs, "device")
        for sub, (C, Ce) in zip(subs, outs):
            roi, lab, dims, N, M, xyz, off = sub
            ctx.set_volumes(as_device(roi), as_device(lab), dims, N, M)
            ctx.add_streamlines(as_device(xyz), as_device(off))
            np.testing.assert_array_equal(ctx.connectivity(), C)
            np.testing.assert_array_equal(ctx.endpoint_connectivity(), Ce)


def test_batch_errors_name_the_subject(fc):
    subs = _subjects(seed_count=2, ns=1000)
    roi, lab, dims, N, M, xyz, off = subs[1]
    off = off.copy()
    off[3], off[4] = off[4], off[3]
    subs[1] = (roi, lab, dims, N, M, xyz, off)
    with fc.Context(0) as ctx:
        with pytest.raises(fc.FastCodError) as e:
            _run_batch(fc, ctx, subs, "host")
        assert e.value.code == fc.FASTCOD_EINVAL and "subject 1" in str(e.value)
        # the context recovers with valid input
        good = _subjects(seed_count=1, ns=500)
        outs = _run_batch(fc, ctx, good, "host")
        np.testing.assert_array_equal(outs[0][0], _oracle(good[0])[0])


@pytest.mark.parametrize("out_where", ["device", "mixed"])
def test_batch_outputs_in_device_memory(fc, out_where):
    """Outputs in device memory are zeroed and accumulated in place by the
    pass (whatever they held), on the first run and on a replay of its graph
    with the same buffers."""
    import torch
    subs = _subjects(seed_count=3, ns=3000)
    keep, objs, outs = [], [], []
    for i, (roi, lab, dims, N, M, xyz, off) in enumerate(subs):
        r, l, x, o = as_device(roi), as_device(lab), as_device(xyz), as_device(off)
        if out_where == "device" or i % 2 == 0:
            C = torch.empty((N, M), dtype=torch.int32, device="cuda:0")
            Ce = torch.empty((N, M), dtype=torch.int32, device="cuda:0")
        else:
            C, Ce = np.empty((N, M), np.int32), np.empty((N, M), np.int32)
        keep += [r, l, x, o]
        outs.append((C, Ce))
        objs.append(fc.make_subject(r, l, dims, N, M, x, o, C, Ce))
    ref = [_oracle(sub)[:2] for sub in subs]
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_AUTOTUNE, 0)
        for run, fill in enumerate((-7, 123456)):
            for C, Ce in outs:
                C.fill(fill) if isinstance(C, np.ndarray) else C.fill_(fill)
                Ce.fill(fill) if isinstance(Ce, np.ndarray) else Ce.fill_(fill)
            torch.cuda.synchronize()  # the fills run on torch's stream, the pass on the context's
            fc.fastcod_batch_run(ctx.ctx, objs)
            assert fc.fastcod_batch_get_info(ctx.ctx)["graph_reused"] == run
            for i, ((C, Ce), (Cr, Cer)) in enumerate(zip(outs, ref)):
                got = [a.cpu().numpy() if isinstance(a, torch.Tensor) else a for a in (C, Ce)]
                np.testing.assert_array_equal(got[0], Cr, err_msg=f"run {run} subject {i}")
                np.testing.assert_array_equal(got[1], Cer, err_msg=f"run {run} subject {i}")
        # new output buffers: the captured graph is updated to them (only its
        # parameters change), and the old buffers keep what they held
        old = list(outs)  # kept alive, so that the new buffers get new addresses
        for i, (C, Ce) in enumerate(outs):
            if isinstance(C, torch.Tensor):
                outs[i] = (torch.full_like(C, 99), torch.full_like(Ce, 99))
                objs[i].C_out, objs[i].Cend_out = outs[i][0].data_ptr(), outs[i][1].data_ptr()
        torch.cuda.synchronize()
        fc.fastcod_batch_run(ctx.ctx, objs)
        assert fc.fastcod_batch_get_info(ctx.ctx)["graph_reused"] == 0
        for i, ((C, Ce), (Cr, Cer), (C0, Ce0)) in enumerate(zip(outs, ref, old)):
            got = [a.cpu().numpy() if isinstance(a, torch.Tensor) else a for a in (C, Ce)]
            np.testing.assert_array_equal(got[0], Cr, err_msg=f"new buffers, subject {i}")
            np.testing.assert_array_equal(got[1], Cer, err_msg=f"new buffers, subject {i}")
            if isinstance(C0, torch.Tensor):
                np.testing.assert_array_equal(C0.cpu().numpy(), Cr)


def test_batch_task_granularity_option(fc):
    """With the autotuner off, FASTCOD_OPT_BATCH_TASK_LOG2 sets the prefilter's
    task size (here the smallest, so that subjects split into many tasks);
    a subject without vertices lies between the others.  Every subject equals
    the oracle; values outside 12..22 are refused."""
    subs = _subjects(seed_count=3, ns=3000)
    empty_off = np.zeros(6, dtype=np.int64)  # five streamlines of no vertex
    roi, lab, dims, N, M = subs[0][:5]
    subs.insert(2, (roi, lab, dims, N, M, np.zeros((0, 3), dtype=np.int32), empty_off))
    with fc.Context(0) as ctx:
        ctx.set_option(fc.FASTCOD_OPT_AUTOTUNE, 0)
        ctx.set_option(fc.FASTCOD_OPT_BATCH_TASK_LOG2, 12)
        outs = _run_batch(fc, ctx, subs, "device")
        info = fc.fastcod_batch_get_info(ctx.ctx)
        assert info["task_vertices"] == 1 << 12 and info["tasks"] > 2 * len(subs)
        for i, (sub, (C, Ce)) in enumerate(zip(subs, outs)):
            Cr, Cer, sr = _oracle(sub)
            np.testing.assert_array_equal(C, Cr, err_msg=f"subject {i}")
            np.testing.assert_array_equal(Ce, Cer, err_msg=f"subject {i}")
            assert fc.fastcod_batch_get_stats(ctx.ctx, i)["voxel_steps"] == sr["voxel_steps"]
        for bad in (0, 11, 23):
            with pytest.raises(fc.FastCodError):
                ctx.set_option(fc.FASTCOD_OPT_BATCH_TASK_LOG2, bad)
