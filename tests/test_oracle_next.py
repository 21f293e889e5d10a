"""Pins of the oracle's parcellation, world-mm ingest, upsampling and rescale
functions against values fixed by the mathematics (numpy's first-occurrence
argmax, exact rationals, brute force on tiny inputs, hand-derived cases)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.parcellation_cases import DOUBLE_ROUNDING_ROWS, as_matrix, midpoint_rows


# ------------------------------------------------------------- parcellation

def _nearest_f32(q: Fraction, f: np.float32) -> bool:
    """f is the binary32 nearest to q (ties to even)."""
    up = np.nextafter(f, np.float32(np.inf))
    dn = np.nextafter(f, np.float32(-np.inf))
    e = abs(Fraction(float(f)) - q)
    if e > abs(Fraction(float(up)) - q) or e > abs(Fraction(float(dn)) - q):
        return False
    for g in (up, dn):
        if abs(Fraction(float(g)) - q) == e:  # a tie: f must have an even significand
            return (np.frombuffer(np.float32(f).tobytes(), np.uint32)[0] & 1) == 0
    return True


def test_parcellate_hand_example():
    C = np.array([[0, 3, 3], [5, 0, 1], [0, 0, 0], [0, 0, 7]])
    label, frac = oracle.parcellate(C)
    assert label.tolist() == [2, 1, 0, 3]  # ties go to the lowest label; a zero row gets 0
    assert frac[0].tolist() == [0.0, 0.5, 0.5]
    assert frac[2].tolist() == [0.0, 0.0, 0.0]
    assert frac[3].tolist() == [0.0, 0.0, 1.0]
    assert frac[1, 0] == np.float32(5 / 6) and frac[1, 2] == np.float32(1 / 6)


@pytest.mark.parametrize("seed", range(4))
def test_parcellate_against_argmax_and_exact_quotients(seed):
    rng = np.random.default_rng(seed)
    N, M = 60, 1 + seed * 9
    C = rng.integers(0, 4, size=(N, M)) * rng.integers(0, 2, size=(N, 1))  # zero rows, many ties
    C[0] = 0
    C[1, :] = 2 ** 40 + rng.integers(0, 3, size=M)  # large counts
    label, frac = oracle.parcellate(C)
    s = C.sum(axis=1)
    want = np.where(s > 0, np.argmax(C, axis=1) + 1, 0)  # numpy: first occurrence of the maximum
    np.testing.assert_array_equal(label, want)
    for r in range(N):
        for t in range(M):
            if s[r] == 0:
                assert frac[r, t] == 0.0
            else:
                assert _nearest_f32(Fraction(int(C[r, t]), int(s[r])), frac[r, t]), (r, t)


def test_parcellate_double_rounding_rows():
    # the binary64 quotient rounded again to binary32 is one unit off on these
    # rows; the fractions must be the nearest binary32 all the same
    C = np.array(DOUBLE_ROUNDING_ROWS, dtype=np.int64)
    label, frac = oracle.parcellate(C)
    assert label.tolist() == [1, 1, 1]
    for r in range(len(C)):
        s = int(C[r].sum())
        for t in range(C.shape[1]):
            assert _nearest_f32(Fraction(int(C[r, t]), s), frac[r, t]), (r, t)
        assert frac[r, 0] != np.float32(int(C[r, 0]) / s)  # not the doubly rounded value
    assert frac[0, 0] == np.float32(0.8205847)


@pytest.mark.parametrize("seed", range(3))
def test_parcellate_at_and_beside_binary32_midpoints(seed):
    # fractions exactly on a midpoint (ties to even) or 2^-55 relative beside
    # one, in eight binades, with the answer known from the construction
    rows, want = midpoint_rows(seed, 240, k_max=7)
    M = max(len(r) for r in rows)
    C = as_matrix(rows, M)
    label, frac = oracle.parcellate(C)
    for i, (pos, f) in enumerate(want):
        q = Fraction(int(C[i, pos]), int(C[i].sum()))
        assert _nearest_f32(q, f), i  # the construction itself, checked with exact rationals
        assert frac[i, pos].view(np.uint32) == f.view(np.uint32), (i, float(frac[i, pos]), float(f))
    for i in range(0, len(rows), 17):  # the row's other entries too
        s = int(C[i].sum())
        for t in range(M):
            assert _nearest_f32(Fraction(int(C[i, t]), s), frac[i, t]), (i, t)


def test_parcellate_rejects_row_sums_past_2_62():
    with pytest.raises(ValueError):
        oracle.parcellate(np.array([[2 ** 61, 2 ** 61]]))
    oracle.parcellate(np.array([[2 ** 61, 2 ** 61 - 1]]))


def test_parcellate_rejects_negative_counts():
    with pytest.raises(ValueError):
        oracle.parcellate(np.array([[1, -1]]))


# ------------------------------------------------------------------ ingest

def test_world_to_fixed_exact_cases():
    # a power-of-two scale and integer translation are exact in binary32:
    # the output is the exact product, and binary32 ties round to even
    A = np.array([[2.0, 0, 0, 3.0], [0, 0.5, 0, -1.0], [0, 0, 1.0, 0.25]], dtype=np.float32)
    x = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0], [-7.5, 9.25, -0.5]], dtype=np.float32)
    got = oracle.world_to_fixed(x, A)
    want = [[(2 * 1.0 + 3) * 1024, (0.5 * 2 - 1) * 1024, (3 + 0.25) * 1024],
            [3 * 1024, -1024, 0.25 * 1024],
            [(2 * -7.5 + 3) * 1024, (0.5 * 9.25 - 1) * 1024, (-0.5 + 0.25) * 1024]]
    np.testing.assert_array_equal(got, np.array(want, dtype=np.int64))
    # v * 1024 = k + 1/2 exactly: ties to even
    A1 = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 1.0, 0]], dtype=np.float32)
    x1 = np.array([[0.5 / 1024, 1.5 / 1024, 2.5 / 1024], [-0.5 / 1024, -1.5 / 1024, 3.5 / 1024]], dtype=np.float32)
    np.testing.assert_array_equal(oracle.world_to_fixed(x1, A1), [[0, 2, 2], [0, -2, 4]])


@pytest.mark.parametrize("seed", range(3))
def test_world_to_fixed_within_one_unit_of_exact(seed):
    # the binary32 evaluation stays within one unit (1/1024 voxel) of the
    # exactly evaluated affine for brain-sized coordinates
    rng = np.random.default_rng(seed)
    A = np.zeros((3, 4), dtype=np.float32)
    A[:, :3] = (np.eye(3) / 1.25 + rng.normal(0, 0.02, (3, 3))).astype(np.float32)
    A[:, 3] = rng.uniform(-90, 90, 3).astype(np.float32)
    x = rng.uniform(-120, 120, size=(400, 3)).astype(np.float32)
    got = oracle.world_to_fixed(x, A)
    for i in range(len(x)):
        for a in range(3):
            v = sum(Fraction(float(A[a, c])) * Fraction(float(x[i, c])) for c in range(3)) + Fraction(float(A[a, 3]))
            assert abs(Fraction(int(got[i, a])) - v * 1024) <= 1


def test_world_to_fixed_rejects_nan_and_range():
    A = np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32)
    with pytest.raises(ValueError):
        oracle.world_to_fixed(np.array([[np.nan, 0, 0]], dtype=np.float32), A)
    with pytest.raises(ValueError):
        oracle.world_to_fixed(np.array([[16384.0, 0, 0]], dtype=np.float32), A)  # 2^24 units
    oracle.world_to_fixed(np.array([[-16384.0, 0, 0]], dtype=np.float32), A)   # -2^24 is allowed


# ---------------------------------------------------------------- upsample

def _random_streamlines(rng, n=40, maxT=9):
    T = rng.integers(0, maxT, size=n)
    off = np.concatenate([[0], np.cumsum(T)]).astype(np.int64)
    xyz = rng.integers(-50000, 50000, size=(int(off[-1]), 3)).astype(np.int32)
    return xyz, off


@pytest.mark.parametrize("factor", [1, 2, 3, 7])
def test_upsample_points_on_segments(factor):
    rng = np.random.default_rng(factor)
    xyz, off = _random_streamlines(rng)
    out, oo = oracle.upsample(xyz, off, factor)
    T = np.diff(off)
    np.testing.assert_array_equal(np.diff(oo), np.where(T > 0, (T - 1) * factor + 1, 0))
    for s in range(len(T)):
        a, b, o = int(off[s]), int(off[s + 1]), int(oo[s])
        if b == a:
            continue
        np.testing.assert_array_equal(out[int(oo[s + 1]) - 1], xyz[b - 1])  # last vertex kept
        for i in range(a, b - 1):
            p, q = xyz[i].astype(np.int64), xyz[i + 1].astype(np.int64)
            for j in range(factor):
                r = out[o + (i - a) * factor + j].astype(np.int64)
                for c in range(3):
                    exact = Fraction(int(p[c])) + Fraction(int(q[c] - p[c]) * j, factor)
                    assert 0 <= exact - int(r[c]) < 1  # the point below or on the exact one
    if factor == 1:
        np.testing.assert_array_equal(out, xyz)


def test_upsample_factor_is_the_smallest_by_brute_force():
    rng = np.random.default_rng(9)
    for trial in range(30):
        xyz, off = _random_streamlines(rng, n=6, maxT=5)
        xyz //= int(rng.integers(1, 200))
        s = int(rng.integers(1, 3000))
        k = oracle.upsample_factor(xyz, off, s)
        l2 = 0
        for st in range(len(off) - 1):
            for i in range(int(off[st]), int(off[st + 1]) - 1):
                d = xyz[i + 1].astype(np.int64) - xyz[i]
                l2 = max(l2, int((d * d).sum()))
        assert (k * s) ** 2 >= l2
        assert k == 1 or ((k - 1) * s) ** 2 < l2
    # the paper's rule of thumb: a 1 mm target wants spacing <= 0.5 mm
    xyz = np.array([[0, 0, 0], [1024, 0, 0]], dtype=np.int32)
    assert oracle.upsample_factor(xyz, np.array([0, 2]), 512) == 2
    assert oracle.upsample_factor(xyz, np.array([0, 2]), 511) == 3


# ----------------------------------------------------------------- rescale

def test_rescale_floor_division():
    rng = np.random.default_rng(4)
    xyz = rng.integers(-100000, 100000, size=(300, 3)).astype(np.int32)
    num, den, add = np.array([25, 7, 1]), np.array([14, 3, 1]), np.array([512 * 11, -5, 0])
    out = oracle.rescale(xyz, num, den, add)
    want = (xyz.astype(object) * num + add) // den  # Python integers: exact floor division
    np.testing.assert_array_equal(out, want.astype(np.int64))
    np.testing.assert_array_equal(oracle.rescale(xyz, [3, 3, 3], [3, 3, 3], [0, 0, 0]), xyz)
    with pytest.raises(ValueError):
        oracle.rescale(np.array([[16000000, 0, 0]], dtype=np.int32), [2, 1, 1], [1, 1, 1], [0, 0, 0])
