"""Pins of the oracle's connectivity matrices C and C_end.

C (Section 2, Algorithm 2: passthrough, then C(v, r) += 1 for every
pass-through v) and C_end (Algorithm 1: seed voxel row, endpoint label) are
checked against
  - a hand-derived worked example (tests/golden/toy_passthrough.json);
  - the plain definition on tiny grids: every voxel box tested against every
    segment with the exact slab test, no walk;
  - a library matrix product: C = A^T B with A[s, r] = [r in V_s] and
    B[s, t] = [t in T_s] built from brute-force voxel sets;
  - a 2-D bincount for C_end and for point-sampled streamlines;
  - invariants on the tiny synthetic subject (bounds, row/column sums,
    order, reversal, chunking, axis permutation, whole-voxel translation).
"""
import os

import numpy as np
import pytest

import oracle
import synth
from synth import tiny

U = 1024


def _lookup(roi, lab, vox):
    """row and label of integer voxels (k x 3), -1 / 0 off the grid."""
    Dz, Dy, Dx = roi.shape
    v = np.asarray(vox, dtype=np.int64).reshape(-1, 3)
    ok = (v[:, 0] >= 0) & (v[:, 0] < Dx) & (v[:, 1] >= 0) & (v[:, 1] < Dy) & (v[:, 2] >= 0) & (v[:, 2] < Dz)
    r = np.full(len(v), -1, dtype=np.int64)
    t = np.zeros(len(v), dtype=np.int64)
    r[ok] = roi[v[ok, 2], v[ok, 1], v[ok, 0]]
    t[ok] = lab[v[ok, 2], v[ok, 1], v[ok, 0]]
    return r, t


def _bf_streamline_voxels(verts, dims):
    """Brute-force voxel set of a streamline (slab test over a padded box)."""
    out = set()
    if len(verts) == 1:
        out.add(tuple(int(x) for x in np.floor_divide(verts[0].astype(np.int64), U)))
        return out
    for a, b in zip(verts[:-1], verts[1:]):
        lo = np.minimum(a, b).astype(np.int64) // U - 1
        hi = np.maximum(a, b).astype(np.int64) // U + 1
        for v in oracle.bruteforce_segment(a, b, lo, hi):
            out.add(tuple(int(x) for x in v))
    return out


def test_golden_toy():
    d, roi, lab, xyz, off = tiny.toy_fixture(os.path.join(tiny.GOLDEN, "toy_passthrough.json"))
    C, Ce, st = oracle.connectivity(roi, lab, d["dims"], d["N"], d["M"], xyz, off)
    assert C.tolist() == d["C_expected"]
    assert Ce.tolist() == d["C_end_expected"]
    for s, sl in enumerate(d["streamlines"]):
        V, T = oracle.streamline_sets(roi, lab, d["dims"], d["N"], d["M"], xyz[off[s]:off[s + 1]])
        assert V.tolist() == sl["V"], sl["name"]
        assert T.tolist() == sl["T"], sl["name"]
    Cb, Ceb = oracle.bruteforce_connectivity(roi, lab, d["dims"], d["N"], d["M"], xyz, off)
    assert Cb.tolist() == d["C_expected"] and Ceb.tolist() == d["C_end_expected"]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("flags", [0, oracle.TARGET_ENDPOINT, oracle.VERTEX_SAMPLED])
def test_walk_connectivity_equals_bruteforce(seed, flags):
    rng = np.random.default_rng(100 + seed)
    dims = tuple(int(v) for v in rng.integers(3, 9, size=3))
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=5, n_labels=int(rng.integers(1, 6)),
                                         many_to_one=bool(seed % 2))
    xyz, off = tiny.random_streamlines(rng, dims, 60)
    C, Ce, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off, flags)
    Cb, Ceb = oracle.bruteforce_connectivity(roi, lab, dims, N, M, xyz, off, flags)
    np.testing.assert_array_equal(C, Cb)
    np.testing.assert_array_equal(Ce, Ceb)


@pytest.mark.parametrize("seed", range(4))
def test_matrix_product_form(seed):
    # C = A^T B over streamlines, A and B from brute-force voxel sets; N != M
    # so a transposed operand cannot pass
    rng = np.random.default_rng(200 + seed)
    dims = (7, 5, 4)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=0, n_labels=3)
    assert N != M
    xyz, off = tiny.random_streamlines(rng, dims, 80)
    ns = len(off) - 1
    A = np.zeros((ns, N), dtype=np.int64)
    B = np.zeros((ns, M), dtype=np.int64)
    for s in range(ns):
        verts = xyz[off[s]:off[s + 1]]
        if len(verts) == 0:
            continue
        vox = np.array(sorted(_bf_streamline_voxels(verts, dims)))
        r, t = _lookup(roi, lab, vox)
        A[s, r[r >= 0]] = 1
        B[s, t[t >= 1] - 1] = 1
    C, _, st = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    np.testing.assert_array_equal(C, A.T @ B)
    assert st["pairs"] == int((A.sum(1) * B.sum(1)).sum())


def test_endpoint_matrix_is_bincount():
    # C_end is a 2-D histogram of (row of the first vertex, label of the last)
    rng = np.random.default_rng(9)
    dims = (9, 8, 7)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=0, n_labels=4, p_roi=0.5, p_lab=0.6)
    xyz, off = tiny.random_streamlines(rng, dims, 400)
    T = np.diff(off)
    keep = T >= 1
    first = np.floor_divide(xyz[off[:-1][keep]].astype(np.int64), U)
    last = np.floor_divide(xyz[off[1:][keep] - 1].astype(np.int64), U)
    r, _ = _lookup(roi, lab, first)
    _, t = _lookup(roi, lab, last)
    ok = (r >= 0) & (t >= 1)
    exp = np.bincount(r[ok] * M + (t[ok] - 1), minlength=N * M).reshape(N, M)
    _, Ce, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    np.testing.assert_array_equal(Ce, exp)


def test_point_sampled_is_bincount():
    # single-vertex streamlines: V_s and T_s come from one voxel, so C is the
    # 2-D histogram of (row, label) over voxels that are both ROI and target
    rng = np.random.default_rng(10)
    dims = (6, 7, 5)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=0, n_labels=3, p_roi=0.6, p_lab=0.6)
    n = 3000
    xyz = rng.integers(-U, np.array(dims) * U + U, size=(n, 3)).astype(np.int32)
    off = np.arange(n + 1, dtype=np.int64)
    r, t = _lookup(roi, lab, np.floor_divide(xyz.astype(np.int64), U))
    ok = (r >= 0) & (t >= 1)
    exp = np.bincount(r[ok] * M + (t[ok] - 1), minlength=N * M).reshape(N, M)
    C, Ce, st = oracle.connectivity(roi, lab, dims, N, M, xyz, off)
    np.testing.assert_array_equal(C, exp)
    np.testing.assert_array_equal(Ce, exp)  # seed = endpoint for T = 1
    assert st["voxel_steps"] == n


def test_vertex_sampled_mode_is_matrix_product():
    rng = np.random.default_rng(12)
    dims = (8, 6, 5)
    roi, lab, N, M = tiny.random_volumes(rng, dims, n_roi=0, n_labels=5)
    xyz, off = tiny.random_streamlines(rng, dims, 150)
    ns = len(off) - 1
    A = np.zeros((ns, N), dtype=np.int64)
    B = np.zeros((ns, M), dtype=np.int64)
    for s in range(ns):
        v = np.floor_divide(xyz[off[s]:off[s + 1]].astype(np.int64), U)
        r, t = _lookup(roi, lab, v)
        A[s, r[r >= 0]] = 1
        B[s, t[t >= 1] - 1] = 1
    C, _, _ = oracle.connectivity(roi, lab, dims, N, M, xyz, off, oracle.VERTEX_SAMPLED)
    np.testing.assert_array_equal(C, A.T @ B)


@pytest.fixture(scope="module")
def cfg0():
    vols, tr = synth.make_subject(0)
    C, Ce, st = oracle.connectivity(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets, tr.xyz,
                                    tr.offsets)
    return vols, tr, C, Ce, st


def _run(vols, xyz, off, flags=0, roi=None, lab=None, dims=None):
    roi = vols.roi if roi is None else roi
    lab = vols.lab if lab is None else lab
    dims = vols.dims if dims is None else dims
    return oracle.connectivity(roi, lab, dims, vols.n_roi, vols.n_targets, xyz, off, flags)


def test_invariant_bounds(cfg0):
    vols, tr, C, Ce, st = cfg0
    ns = tr.n_streamlines
    assert C.min() >= 0 and C.max() <= ns
    assert np.all(Ce <= C)  # the seed and the endpoint lie on the streamline
    assert C.sum() == st["pairs"]
    assert C.sum() > 0 and Ce.sum() > 0
    # sum of C_end = #{s : row(p^1) >= 0 and lab(p^T) >= 1}
    T = np.diff(tr.offsets)
    k = T >= 1
    r, _ = _lookup(vols.roi, vols.lab, np.floor_divide(tr.xyz[tr.offsets[:-1][k]].astype(np.int64), U))
    _, t = _lookup(vols.roi, vols.lab, np.floor_divide(tr.xyz[tr.offsets[1:][k] - 1].astype(np.int64), U))
    assert Ce.sum() == int(((r >= 0) & (t >= 1)).sum())


def test_invariant_row_and_column_sums(cfg0):
    vols, tr, C, _, _ = cfg0
    N, M = vols.n_roi, vols.n_targets
    row = np.zeros(N, dtype=np.int64)
    col = np.zeros(M, dtype=np.int64)
    for s in range(tr.n_streamlines):
        V, T = oracle.streamline_sets(vols.roi, vols.lab, vols.dims, N, M, tr.xyz[tr.offsets[s]:tr.offsets[s + 1]])
        row[V] += len(T)
        col[T - 1] += len(V)
    np.testing.assert_array_equal(C.sum(axis=1), row)
    np.testing.assert_array_equal(C.sum(axis=0), col)


def test_invariant_order_reversal_chunking(cfg0):
    vols, tr, C, Ce, _ = cfg0
    rng = np.random.default_rng(0)
    ns = tr.n_streamlines
    perm = rng.permutation(ns)
    segs = [tr.xyz[tr.offsets[s]:tr.offsets[s + 1]] for s in range(ns)]
    counts = np.array([len(segs[s]) for s in perm])
    off = np.zeros(ns + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    C2, Ce2, _ = _run(vols, np.concatenate([segs[s] for s in perm]), off)
    np.testing.assert_array_equal(C2, C)
    np.testing.assert_array_equal(Ce2, Ce)
    # reversing every streamline keeps C (P_s is the same point set)
    C3, Ce3, _ = _run(vols, np.concatenate([s[::-1] for s in segs]), tr.offsets)
    np.testing.assert_array_equal(C3, C)
    assert not np.array_equal(Ce3, Ce)  # C_end is directional
    # chunking: sum over contiguous chunks
    C4, Ce4, _ = oracle.connectivity_chunked(vols.roi, vols.lab, vols.dims, vols.n_roi, vols.n_targets,
                                             tr.xyz, tr.offsets, chunks=7)
    np.testing.assert_array_equal(C4, C)
    np.testing.assert_array_equal(Ce4, Ce)


def test_invariant_axis_permutation_and_translation(cfg0):
    vols, tr, C, Ce, _ = cfg0
    # permute the axes of the coordinates and of the volumes consistently
    perm = (2, 0, 1)  # new x = old z, new y = old x, new z = old y
    xyz = tr.xyz[:, perm]
    # volume array index order is (z, y, x); new (z, y, x) = old (y, x, z)
    roi = np.ascontiguousarray(np.transpose(vols.roi, (1, 2, 0)))
    lab = np.ascontiguousarray(np.transpose(vols.lab, (1, 2, 0)))
    dims = tuple(vols.dims[a] for a in perm)
    C2, Ce2, _ = _run(vols, xyz, tr.offsets, roi=roi, lab=lab, dims=dims)
    np.testing.assert_array_equal(C2, C)
    np.testing.assert_array_equal(Ce2, Ce)
    # translate by whole voxels: shift coordinates and pad the volumes
    k = np.array([3, 1, 2])
    roi_t = np.pad(vols.roi, ((k[2], 0), (k[1], 0), (k[0], 0)), constant_values=-1)
    lab_t = np.pad(vols.lab, ((k[2], 0), (k[1], 0), (k[0], 0)), constant_values=0)
    dims_t = tuple(int(vols.dims[a] + k[a]) for a in range(3))
    C3, Ce3, _ = _run(vols, tr.xyz + (k * U).astype(np.int32), tr.offsets, roi=roi_t, lab=lab_t, dims=dims_t)
    np.testing.assert_array_equal(C3, C)
    np.testing.assert_array_equal(Ce3, Ce)


def test_endpoint_target_mode_bounds(cfg0):
    vols, tr, C, Ce, _ = cfg0
    Cep, Ce2, _ = _run(vols, tr.xyz, tr.offsets, oracle.TARGET_ENDPOINT)
    np.testing.assert_array_equal(Ce2, Ce)
    assert np.all(Ce <= Cep) and np.all(Cep <= C)


def test_invalid_inputs_rejected():
    roi = np.full((2, 2, 2), -1, dtype=np.int32)
    lab = np.zeros((2, 2, 2), dtype=np.uint16)
    xyz = np.zeros((2, 3), dtype=np.int32)
    good = np.array([0, 2], dtype=np.int64)
    oracle.connectivity(roi, lab, (2, 2, 2), 1, 1, xyz, good)
    with pytest.raises(ValueError):
        oracle.connectivity(roi, lab, (2, 2, 2), 1, 1, xyz, np.array([1, 2], dtype=np.int64))
    bad = xyz.copy()
    bad[0, 0] = 1 << 24
    with pytest.raises(ValueError):
        oracle.connectivity(roi, lab, (2, 2, 2), 1, 1, bad, good)
    edge = xyz.copy()
    edge[0, 0] = -(1 << 24)  # the lower end of [-2^24, 2^24) is allowed
    oracle.connectivity(roi, lab, (2, 2, 2), 1, 1, edge, good)
    edge[0, 0] = -(1 << 24) - 1
    with pytest.raises(ValueError):
        oracle.connectivity(roi, lab, (2, 2, 2), 1, 1, edge, good)
    lab2 = lab.copy()
    lab2[0, 0, 0] = 2
    with pytest.raises(ValueError):
        oracle.connectivity(roi, lab2, (2, 2, 2), 1, 1, xyz, good)
