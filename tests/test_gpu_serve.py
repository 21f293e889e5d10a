"""GPU tests of the served form (fastcod_server_*): continuous batching gives
each request exactly its own result (bit-exact against the oracle and
identical alone and in the mix), admission under a small HBM budget,
cancellation and per-request errors leave the other requests intact."""
import time

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import as_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    from paper_2302_09247_gb300 import fastcod
    return fastcod


@pytest.fixture(scope="module")
def subjects():
    out = {}
    vols, tr = synth.make_subject(1, n_streamlines=60_000)
    out["A"] = (vols, tr)
    vols, tr = synth.make_subject(3, subject=2, n_streamlines=30_000)
    out["B"] = (vols, tr)
    vols, tr = synth.make_subject(0)
    out["C"] = (vols, tr)
    return out


def _chunks(tr, n):
    bounds = np.linspace(0, tr.n_streamlines, n + 1).astype(np.int64)
    out = []
    for c in range(n):
        b, e = int(bounds[c]), int(bounds[c + 1])
        out.append((np.ascontiguousarray(tr.xyz[tr.offsets[b]:tr.offsets[e]]),
                    np.ascontiguousarray(tr.offsets[b:e + 1] - tr.offsets[b])))
    return out


class Req:
    def __init__(self, fc, srv, vols, where="host"):
        self.vols = vols
        self.C = np.full((vols.n_roi, vols.n_targets), -3, dtype=np.int32)
        self.Ce = np.full_like(self.C, -3)
        if where == "device":
            self.roi, self.lab = as_device(vols.roi), as_device(vols.lab)
        else:
            self.roi, self.lab = vols.roi, vols.lab
        self.head = fc.make_subject(self.roi, self.lab, vols.dims, vols.n_roi, vols.n_targets,
                                    np.zeros((0, 3), np.int32), np.zeros(1, np.int64), self.C, self.Ce)
        self.id = fc.fastcod_server_submit(srv, self.head)
        self.keep = []

    def push(self, fc, srv, xyz, off, last=False, where="host"):
        if where == "device":
            xyz, off = as_device(xyz), as_device(off)
        self.keep.append((xyz, off))
        fc.fastcod_server_push_chunk(srv, self.id, xyz, off, last)


def _oracle(vols, tr):
    C, Ce, _ = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz, tr.offsets)
    return C, Ce


def test_alone_equals_in_the_mix(fc, subjects):
    vA, tA = subjects["A"]
    ctx = fc.Context(0)
    srv = fc.fastcod_server_create(ctx.ctx, 4, 0)
    try:
        ra = Req(fc, srv, vA)
        for i, (x, o) in enumerate(_chunks(tA, 3)):
            ra.push(fc, srv, x, o, last=(i == 2))
        assert fc.fastcod_server_wait(srv, ra.id, 120.0) == fc.FASTCOD_OK
        # one request of three chunks: volume prep + near grid, then three
        # kernels per iteration, at least one iteration per chunk
        n = fc.fastcod_server_kernel_launches(srv)
        assert n >= 2 + 3 * 3 and (n - 2) % 3 == 0
        alone = ra.C.copy()
        # the same request in a mix with two others, chunks interleaved
        reqs = {k: Req(fc, srv, subjects[k][0], where=("device" if k == "B" else "host")) for k in "ABC"}
        ch = {"A": _chunks(tA, 3), "B": _chunks(subjects["B"][1], 2), "C": _chunks(subjects["C"][1], 1)}
        order = [("A", 0), ("B", 0), ("C", 0), ("A", 1), ("B", 1), ("A", 2)]
        for k, i in order:
            x, o = ch[k][i]
            reqs[k].push(fc, srv, x, o, last=(i == len(ch[k]) - 1), where=("device" if k == "B" else "host"))
        for k in "ABC":
            assert fc.fastcod_server_wait(srv, reqs[k].id, 120.0) == fc.FASTCOD_OK
            Cr, Cer = _oracle(*subjects[k])
            np.testing.assert_array_equal(reqs[k].C, Cr, err_msg=k)
            np.testing.assert_array_equal(reqs[k].Ce, Cer, err_msg=k)
            info = fc.fastcod_server_request_info(srv, reqs[k].id)
            assert info["done"] == 1 and info["streamlines"] == subjects[k][1].n_streamlines
            assert info["t_submit"] <= info["t_admit"] <= info["t_done"]
        np.testing.assert_array_equal(reqs["A"].C, alone)
    finally:
        fc.fastcod_server_destroy(srv)
        ctx.close()


def test_admission_under_small_budget(fc, subjects):
    # a 1-byte budget admits one request at a time (the loop never deadlocks)
    ctx = fc.Context(0)
    srv = fc.fastcod_server_create(ctx.ctx, 8, 1)
    try:
        reqs = []
        for k in "CBC":
            r = Req(fc, srv, subjects[k][0])
            x, o = _chunks(subjects[k][1], 1)[0]
            r.push(fc, srv, x, o, last=True)
            reqs.append((k, r))
        infos = []
        for k, r in reqs:
            assert fc.fastcod_server_wait(srv, r.id, 120.0) == fc.FASTCOD_OK
            np.testing.assert_array_equal(r.C, _oracle(*subjects[k])[0])
            infos.append(fc.fastcod_server_request_info(srv, r.id))
        for a, b in zip(infos, infos[1:]):
            assert b["t_admit"] >= a["t_done"] - 1e-3
    finally:
        fc.fastcod_server_destroy(srv)
        ctx.close()


def test_cancel_and_errors_are_isolated(fc, subjects):
    ctx = fc.Context(0)
    srv = fc.fastcod_server_create(ctx.ctx, 4, 0)
    try:
        vC, tC = subjects["C"]
        good = Req(fc, srv, vC)
        x, o = _chunks(tC, 1)[0]
        good.push(fc, srv, x, o, last=True)
        cancelled = Req(fc, srv, vC)
        cancelled.push(fc, srv, x, o)
        fc.fastcod_server_cancel(srv, cancelled.id)
        bad = Req(fc, srv, vC)
        o2 = o.copy()
        o2[5], o2[6] = o2[6], o2[5]
        bad.push(fc, srv, x, o2, last=True)
        assert fc.fastcod_server_wait(srv, good.id, 120.0) == fc.FASTCOD_OK
        assert fc.fastcod_server_wait(srv, cancelled.id, 120.0) == fc.FASTCOD_ECANCELED
        assert fc.fastcod_server_wait(srv, bad.id, 120.0) == fc.FASTCOD_EINVAL
        np.testing.assert_array_equal(good.C, _oracle(vC, tC)[0])
        assert (cancelled.C == -3).all()
        done, rc = fc.fastcod_server_poll(srv, good.id)
        assert done and rc == fc.FASTCOD_OK
    finally:
        fc.fastcod_server_destroy(srv)
        ctx.close()


def _faulty_server(fc, ctx, spec, monkeypatch):
    monkeypatch.setenv("FASTCOD_FAULT", spec)
    srv = fc.fastcod_server_create(ctx.ctx, 4, 0)
    monkeypatch.delenv("FASTCOD_FAULT")
    return srv


@pytest.mark.parametrize("spec,where,status", [("alloc:2", "device", "FASTCOD_ENOMEM"),
                                               ("h2d:2", "host", "FASTCOD_ECUDA"),
                                               ("cancel:2", "host", "FASTCOD_ECANCELED"),
                                               ("alloc:3", "host", "FASTCOD_ENOMEM")])
def test_injected_failure_hits_one_request(fc, subjects, monkeypatch, spec, where, status):
    # host-side injection (no GPU fault): exactly one request of four reports
    # the failure; the other three complete with the oracle's result
    vA, tA = subjects["A"]
    want = _oracle(vA, tA)
    ctx = fc.Context(0)
    srv = _faulty_server(fc, ctx, spec, monkeypatch)
    try:
        reqs = []
        for _ in range(4):
            r = Req(fc, srv, vA, where)
            for i, (x, o) in enumerate(_chunks(tA, 2)):
                try:
                    r.push(fc, srv, x, o, last=(i == 1), where=where)
                except fc.FastCodError as e:
                    # a request cancelled on submission may already be done
                    # when its chunks arrive: the push is refused (ESTATE)
                    assert spec.startswith("cancel") and e.code == fc.FASTCOD_ESTATE
            reqs.append(r)
        got = [fc.fastcod_server_wait(srv, r.id, 120.0) for r in reqs]
        assert sorted(got).count(getattr(fc, status)) == 1, got
        assert got.count(fc.FASTCOD_OK) == 3, got
        if spec.startswith(("alloc:2", "cancel:2")):
            assert got[1] == getattr(fc, status)  # admission and submission follow arrival order
        for r, g in zip(reqs, got):
            if g == fc.FASTCOD_OK:
                np.testing.assert_array_equal(r.C, want[0])
                np.testing.assert_array_equal(r.Ce, want[1])
        # the server keeps serving after the failure
        r = Req(fc, srv, vA, where)
        for i, (x, o) in enumerate(_chunks(tA, 2)):
            r.push(fc, srv, x, o, last=(i == 1), where=where)
        assert fc.fastcod_server_wait(srv, r.id, 120.0) == fc.FASTCOD_OK
        np.testing.assert_array_equal(r.C, want[0])
    finally:
        fc.fastcod_server_destroy(srv)
        ctx.close()


@pytest.mark.parametrize("slots", [1, 3])
def test_staging_buffers_reused_across_chunk_sizes(fc, subjects, slots):
    """Host chunks go through the server's kept staging buffers: requests
    whose chunks shrink and grow (a chunk larger than any buffer held, many
    small ones, one whole subject), from pageable and page-locked memory, one
    after another and at once, each equal to the oracle."""
    import torch
    vA, tA = subjects["A"]
    vB, tB = subjects["B"]
    Cr, Cer = _oracle(vA, tA)
    Br, Ber = _oracle(vB, tB)
    plans = [("A", 12, False), ("A", 2, True), ("B", 9, False), ("A", 1, True), ("A", 5, False)]
    ctx = fc.Context(0)
    srv = fc.fastcod_server_create(ctx.ctx, slots, 0)
    try:
        for together in (False, True):
            reqs = []
            for k, n, pinned in plans:
                vols, tr = subjects[k]
                r = Req(fc, srv, vols)
                chunks = _chunks(tr, n)
                for i, (x, o) in enumerate(chunks):
                    if pinned:
                        x, o = torch.from_numpy(x).pin_memory(), torch.from_numpy(o).pin_memory()
                    r.push(fc, srv, x, o, last=(i == n - 1))
                reqs.append((k, r))
                if not together:
                    assert fc.fastcod_server_wait(srv, r.id, 120.0) == fc.FASTCOD_OK
            for k, r in reqs:
                assert fc.fastcod_server_wait(srv, r.id, 120.0) == fc.FASTCOD_OK
                np.testing.assert_array_equal(r.C, Cr if k == "A" else Br, err_msg=f"{k} together={together}")
                np.testing.assert_array_equal(r.Ce, Cer if k == "A" else Ber, err_msg=f"{k} together={together}")
    finally:
        fc.fastcod_server_destroy(srv)
        ctx.close()


def test_request_split_at_a_chunk_boundary_sums_to_the_whole(fc, subjects):
    """A request stopped after k of its chunks and resumed as a second request
    of the remaining ones: the two results add up to the whole subject's
    (counts add per streamline), for every split point of a 5-chunk request,
    the two halves in flight together."""
    vA, tA = subjects["A"]
    Cr, Cer = _oracle(vA, tA)
    chunks = _chunks(tA, 5)
    ctx = fc.Context(0)
    srv = fc.fastcod_server_create(ctx.ctx, 4, 0)
    try:
        for k in range(1, 5):
            first, rest = Req(fc, srv, vA), Req(fc, srv, vA, where="device")
            for i, (x, o) in enumerate(chunks[:k]):
                first.push(fc, srv, x, o, last=(i == k - 1))
            for i, (x, o) in enumerate(chunks[k:]):
                rest.push(fc, srv, x, o, last=(i == len(chunks) - k - 1), where="device")
            for r in (first, rest):
                assert fc.fastcod_server_wait(srv, r.id, 120.0) == fc.FASTCOD_OK
            np.testing.assert_array_equal(first.C + rest.C, Cr, err_msg=f"split after chunk {k}")
            np.testing.assert_array_equal(first.Ce + rest.Ce, Cer, err_msg=f"split after chunk {k}")
            done = [fc.fastcod_server_request_info(srv, r.id)["streamlines"] for r in (first, rest)]
            assert sum(done) == tA.n_streamlines
    finally:
        fc.fastcod_server_destroy(srv)
        ctx.close()
