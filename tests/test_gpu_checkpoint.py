"""GPU tests of checkpoint and resume (fastcod_restore).

A pass split at streamline boundaries, checkpointed to host or device memory
and resumed in a fresh context, ends with the oracle's C and C_end and with
the additive statistics of one uninterrupted pass (streamlines, vertices,
voxel steps, pairs).  A checkpoint that no pass can produce is refused, and
the context is then as after a reset."""

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import as_device

pytestmark = pytest.mark.gpu

# statistics that every streamline adds to on its own; survivors, overflow
# and walked steps count the work the prefilter let through, which depends
# on where a streamline sits in its call's arrays
ADDITIVE = ("streamlines", "vertices", "voxel_steps", "pairs")


@pytest.fixture(scope="module")
def fc():
    from paper_2302_09247_gb300 import fastcod
    return fastcod


@pytest.fixture(scope="module")
def subject():
    vols, tr = synth.make_subject(1, n_streamlines=60_000)
    C, Ce, st = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets)
    return vols, tr, C, Ce, st


def _part(tr, b, e):
    """Streamlines [b, e) as their own vertex and offset arrays."""
    o = tr.offsets
    return np.ascontiguousarray(tr.xyz[o[b]:o[e]]), np.ascontiguousarray(o[b:e + 1] - o[b])


def _ctx(fc, vols):
    ctx = fc.Context(0)
    ctx.set_volumes(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets)
    return ctx


@pytest.mark.parametrize("where", ["host", "device"])
def test_split_checkpoint_resume_equals_one_pass(fc, subject, where):
    vols, tr, Cr, Cer, sr = subject
    with _ctx(fc, vols) as ctx:
        ctx.add_streamlines(tr.xyz, tr.offsets)
        C1, Ce1, st1 = ctx.checkpoint()
    np.testing.assert_array_equal(C1, Cr)
    np.testing.assert_array_equal(Ce1, Cer)
    ns = tr.n_streamlines
    cuts = sorted(int(x) for x in np.random.default_rng(7).choice(np.arange(1, ns), size=3, replace=False))
    bounds = [0, *cuts, ns]
    ck = None
    for b, e in zip(bounds, bounds[1:]):
        # a fresh context for every part, as after a restart
        with _ctx(fc, vols) as ctx:
            if ck is not None:
                C, Ce, st = ck
                if where == "device":
                    C, Ce = as_device(C), as_device(Ce)
                ctx.restore(C, Ce, st)
                assert ctx.stats() == st
            ctx.add_streamlines(*_part(tr, b, e))
            ck = ctx.checkpoint()
    C, Ce, st = ck
    np.testing.assert_array_equal(C, Cr)
    np.testing.assert_array_equal(Ce, Cer)
    assert {k: st[k] for k in ADDITIVE} == {k: st1[k] for k in ADDITIVE}
    assert st["streamlines"] == ns and st["vertices"] == len(tr.xyz)
    assert st["voxel_steps"] == sr["voxel_steps"] and st["pairs"] == sr["pairs"] == int(Cr.sum())


def test_restore_in_the_same_context_and_empty_checkpoints(fc, subject):
    vols, tr, Cr, Cer, _ = subject
    with _ctx(fc, vols) as ctx:
        empty = ctx.checkpoint()
        assert not empty[0].any() and empty[2]["streamlines"] == 0
        ctx.add_streamlines(*_part(tr, 0, 1000))
        ck = ctx.checkpoint()
        ctx.add_streamlines(*_part(tr, 1000, 2000))  # discarded by the restore
        ctx.restore(*ck)
        ctx.add_streamlines(*_part(tr, 1000, tr.n_streamlines))
        np.testing.assert_array_equal(ctx.connectivity(), Cr)
        np.testing.assert_array_equal(ctx.endpoint_connectivity(), Cer)
        ctx.restore(*empty)
        assert ctx.stats() == empty[2]
        assert not ctx.connectivity().any() and not ctx.endpoint_connectivity().any()
        ctx.add_streamlines(tr.xyz, tr.offsets)
        np.testing.assert_array_equal(ctx.connectivity(), Cr)


def test_invalid_checkpoints_are_refused(fc, subject):
    vols, tr, Cr, Cer, _ = subject
    part = _part(tr, 0, 5000)
    with _ctx(fc, vols) as ctx:
        ctx.add_streamlines(*part)
        C, Ce, st = ctx.checkpoint()
        assert st["pairs"] > 0 and 0 < Ce.sum() < st["streamlines"]

        def refused(C2, Ce2, st2, msg):
            ctx.add_streamlines(*part)  # something a refusal must clear
            with pytest.raises(fc.FastCodError) as e:
                ctx.restore(C2, Ce2, st2)
            assert e.value.code == fc.FASTCOD_EINVAL and msg in str(e.value), str(e.value)
            assert all(v == 0 for v in ctx.stats().values())
            assert not ctx.connectivity().any() and not ctx.endpoint_connectivity().any()

        i = int(np.flatnonzero(C)[0])
        bad = C.copy()
        bad.flat[i] = -1
        refused(bad, Ce, st, f"checkpoint C[{i // C.shape[1]}][{i % C.shape[1]}] outside")
        bad.flat[i] = st["streamlines"] + 1
        refused(bad, Ce, st, "checkpoint C[")
        bad = Ce.copy()
        bad.flat[7] = -5
        refused(C, bad, st, f"checkpoint C_end[{7 // C.shape[1]}][{7 % C.shape[1]}] outside")
        # one increment too many or too few: C no longer sums to the pairs
        bad = C.copy()
        bad.flat[i] += 1
        refused(bad, Ce, st, "sums to")
        refused(C, Ce, {**st, "pairs": st["pairs"] - 1}, "sums to")
        # more seed/endpoint counts than streamlines (each entry still in range)
        bad = Ce.copy()
        extra = st["streamlines"] - int(Ce.sum()) + 1
        bad.flat[:extra] += 1
        refused(C, bad, st, "C_end sums to")
        # counts checked on the host
        refused(C, Ce, {**st, "streamlines": -1}, "outside [0, 2^31 - 1]")
        refused(C, Ce, {**st, "streamlines": 2 ** 31}, "outside [0, 2^31 - 1]")
        refused(C, Ce, {**st, "voxel_steps": -1}, "negative")
        refused(C, Ce, {**st, "overflow": st["survivors"] + 1}, "inconsistent")
        refused(C, Ce, {**st, "walked_steps": st["voxel_steps"] + 1}, "inconsistent")
        # the valid checkpoint is still accepted and resumes to the oracle
        ctx.restore(C, Ce, st)
        ctx.add_streamlines(*_part(tr, 5000, tr.n_streamlines))
        np.testing.assert_array_equal(ctx.connectivity(), Cr)
        np.testing.assert_array_equal(ctx.endpoint_connectivity(), Cer)


def test_restore_needs_volumes(fc):
    ctx = fc.Context(0)
    try:
        st = {k: 0 for k, _ in fc.Stats._fields_}
        with pytest.raises(fc.FastCodError) as e:
            fc.fastcod_restore(ctx.ctx, None, None, st)
        assert e.value.code == fc.FASTCOD_ESTATE
    finally:
        ctx.close()


@pytest.mark.parametrize("target,sampling", [(1, 0), (0, 1)])
def test_resume_under_the_other_rules(fc, subject, target, sampling):
    """The endpoint-target rule (Algorithm 2 taken literally) and the
    vertex-sampled rule: a two-way split resumed in a fresh context equals
    the oracle under the same rule."""
    vols, tr, _, _, _ = subject
    flags = (oracle.TARGET_ENDPOINT if target else 0) | (oracle.VERTEX_SAMPLED if sampling else 0)
    Cr, Cer, sr = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                      tr.offsets, flags)
    cut = 23_457
    ck = None
    for b, e in ((0, cut), (cut, tr.n_streamlines)):
        with _ctx(fc, vols) as ctx:
            ctx.set_option(fc.FASTCOD_OPT_TARGET_MODE, target)
            ctx.set_option(fc.FASTCOD_OPT_SAMPLING, sampling)
            if ck is not None:
                ctx.restore(*ck)
            ctx.add_streamlines(*_part(tr, b, e))
            ck = ctx.checkpoint()
    np.testing.assert_array_equal(ck[0], Cr)
    np.testing.assert_array_equal(ck[1], Cer)
    assert ck[2]["pairs"] == sr["pairs"] and ck[2]["voxel_steps"] == sr["voxel_steps"]
