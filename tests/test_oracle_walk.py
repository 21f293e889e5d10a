"""Pins of the oracle's segment walk (passthrough, Section 2 / Algorithm 2).

The walk must return exactly the voxels whose half-open boxes meet the closed
segment.  It is checked against an exact brute-force slab test (no walk),
against closed forms and against structural properties.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

U = 1024


def _set(a):
    return {tuple(int(x) for x in r) for r in a}


def _box(p0, p1, pad=1):
    v0 = np.floor_divide(np.asarray(p0, dtype=np.int64), U)
    v1 = np.floor_divide(np.asarray(p1, dtype=np.int64), U)
    return np.minimum(v0, v1) - pad, np.maximum(v0, v1) + pad


def _random_point(rng, snap):
    # coordinates in [-2, 6) voxels; snapped to a lattice so that plane, edge
    # and corner ties are frequent
    v = rng.integers(-2 * U, 6 * U, size=3)
    if snap:
        v = (v // snap) * snap
    return v.astype(np.int32)


@pytest.mark.parametrize("snap", [0, 256, 512, 1024])
def test_walk_equals_bruteforce(snap):
    rng = np.random.default_rng(1234 + snap)
    for _ in range(1500):
        p0 = _random_point(rng, snap)
        if rng.random() < 0.3:
            # short segments like the tractograms' (half a voxel)
            p1 = (p0 + rng.integers(-600, 601, size=3)).astype(np.int32)
            if snap:
                p1 = ((p1 // snap) * snap).astype(np.int32)
        else:
            p1 = _random_point(rng, snap)
        if rng.random() < 0.1:
            p1 = p0.copy()  # zero length
        if rng.random() < 0.15:
            a = rng.integers(3)
            p1[a] = p0[a]  # the segment lies in a plane of constant coordinate
        lo, hi = _box(p0, p1)
        walk = oracle.segment_voxels(p0, p1)
        bf = oracle.bruteforce_segment(p0, p1, lo, hi)
        assert _set(walk) == _set(bf), (p0, p1)
        # the walk never visits a voxel twice
        assert len(walk) == len(_set(walk))


def test_walk_in_planes_and_on_edges():
    # segments lying in grid planes / along grid edges, both directions
    cases = []
    for a in range(3):
        for s in (+1, -1):
            p0 = np.array([2 * U, 3 * U, U], dtype=np.int32)
            p1 = p0.copy()
            p1[a] += s * 3 * U
            cases.append((p0, p1))
            q1 = p0.copy()
            q1[a] += s * 3 * U
            q1[(a + 1) % 3] += s * 2 * U  # diagonal inside a plane through lattice corners
            cases.append((p0, q1))
    for p0, p1 in cases:
        lo, hi = _box(p0, p1)
        assert _set(oracle.segment_voxels(p0, p1)) == _set(oracle.bruteforce_segment(p0, p1, lo, hi))


def test_walk_structure():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        p0 = _random_point(rng, 512 if rng.random() < 0.5 else 0)
        p1 = _random_point(rng, 512 if rng.random() < 0.5 else 0)
        w = oracle.segment_voxels(p0, p1).astype(np.int64)
        assert tuple(w[0]) == tuple(np.floor_divide(p0.astype(np.int64), U))
        assert tuple(w[-1]) == tuple(np.floor_divide(p1.astype(np.int64), U))
        step = np.diff(w, axis=0)
        # each step moves every axis by at most one voxel, towards P1
        assert np.all(np.abs(step) <= 1)
        assert np.all(np.abs(step).sum(axis=1) >= 1)
        d = np.sign(p1.astype(np.int64) - p0)
        assert np.all(step * d[None, :] >= 0)


def test_reversal_invariant_set():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        snap = (0, 256, 1024)[rng.integers(3)]
        p0, p1 = _random_point(rng, snap), _random_point(rng, snap)
        assert _set(oracle.segment_voxels(p0, p1)) == _set(oracle.segment_voxels(p1, p0))


def test_closed_form_axis_aligned():
    # P0 = (x0, y, z) -> P1 = (x1, y, z): voxels floor(x0)..floor(x1) at
    # (floor y, floor z), also when y or z lie exactly on a plane
    rng = np.random.default_rng(3)
    for _ in range(500):
        a = int(rng.integers(3))
        x0, x1 = (int(v) for v in rng.integers(-3 * U, 5 * U, size=2))
        if rng.random() < 0.3:
            x0 = (x0 // U) * U
        other = [int(v) for v in rng.integers(-2 * U, 3 * U, size=2)]
        if rng.random() < 0.5:
            other[0] = (other[0] // U) * U  # on a plane
        p0 = [0, 0, 0]
        p1 = [0, 0, 0]
        p0[a], p1[a] = x0, x1
        p0[(a + 1) % 3] = p1[(a + 1) % 3] = other[0]
        p0[(a + 2) % 3] = p1[(a + 2) % 3] = other[1]
        w = oracle.segment_voxels(p0, p1)
        lo, hi = sorted((x0 // U, x1 // U))
        exp = set()
        for i in range(lo, hi + 1):
            v = [0, 0, 0]
            v[a] = i
            v[(a + 1) % 3] = other[0] // U
            v[(a + 2) % 3] = other[1] // U
            exp.add(tuple(v))
        assert _set(w) == exp
        assert len(w) == hi - lo + 1


@pytest.mark.parametrize("sign", [+1, -1])
def test_closed_form_main_diagonal(sign):
    # (a+1/2)(1,1,1) -> (b+1/2)(1,1,1), either direction: exactly the b-a+1
    # voxels (i,i,i) (all three planes are crossed at the same t)
    for a in range(-3, 3):
        for b in range(a, a + 6):
            p0 = np.full(3, a * U + U // 2, dtype=np.int32)
            p1 = np.full(3, b * U + U // 2, dtype=np.int32)
            if sign < 0:
                p0, p1 = p1, p0
            w = oracle.segment_voxels(p0, p1)
            assert _set(w) == {(i, i, i) for i in range(a, b + 1)}
            assert len(w) == b - a + 1


@pytest.mark.parametrize("dx,dy", [(1, -1), (-1, 1)])
def test_closed_form_mixed_sign_diagonal(dx, dy):
    # a 2-D diagonal with opposite signs through k lattice corners meets
    # 2k+1 voxels: at each corner the increasing axis steps at the corner and
    # the decreasing axis just after it
    for k in range(0, 7):
        p0 = np.array([U // 2, U // 2, 300], dtype=np.int32)
        p1 = p0 + np.array([dx * k * U, dy * k * U, 0], dtype=np.int32)
        w = oracle.segment_voxels(p0, p1)
        assert len(w) == 2 * k + 1
        lo, hi = _box(p0, p1)
        assert _set(w) == _set(oracle.bruteforce_segment(p0, p1, lo, hi))


def test_closed_form_generic_count():
    # a segment with no simultaneous plane crossings visits exactly
    # 1 + sum_a |floor(P1_a) - floor(P0_a)| voxels
    rng = np.random.default_rng(5)
    done = 0
    while done < 500:
        p0 = rng.integers(-4 * U, 4 * U, size=3).astype(np.int32)
        p1 = rng.integers(-4 * U, 4 * U, size=3).astype(np.int32)
        d = p1.astype(np.int64) - p0
        if np.any(d == 0):
            continue
        # plane-crossing parameters of every axis, as exact fractions
        ts = []
        for a in range(3):
            c0, c1 = p0[a] // U, p1[a] // U
            if d[a] > 0:
                ts += [((k * U - int(p0[a])), int(d[a])) for k in range(c0 + 1, c1 + 1)]
            else:
                ts += [((int(p0[a]) - k * U), int(-d[a])) for k in range(c1 + 1, c0 + 1)]
        fr = [Fraction(n, q) for n, q in ts]
        if len(set(fr)) != len(fr) or any(f in (0, 1) for f in fr):
            continue
        n = 1 + int(np.abs(np.floor_divide(p1.astype(np.int64), U) - np.floor_divide(p0.astype(np.int64), U)).sum())
        assert len(oracle.segment_voxels(p0, p1)) == n
        done += 1


def test_bruteforce_special_cases():
    # the slab test itself: a point segment hits exactly its floor voxel; a
    # segment ending exactly on a plane reaches the upper voxel when moving up
    # and does not leave the voxel when moving down
    p = np.array([1024, 2047, -1], dtype=np.int32)
    assert _set(oracle.bruteforce_segment(p, p, [-2, -2, -2], [3, 3, 3])) == {(1, 1, -1)}
    up0, up1 = [100, 100, 100], [1024, 100, 100]
    assert _set(oracle.bruteforce_segment(up0, up1, [-2, -2, -2], [3, 3, 3])) == {(0, 0, 0), (1, 0, 0)}
    dn0, dn1 = [2000, 100, 100], [1024, 100, 100]
    assert _set(oracle.bruteforce_segment(dn0, dn1, [-2, -2, -2], [3, 3, 3])) == {(1, 0, 0)}
    dn0, dn1 = [1024, 100, 100], [1000, 100, 100]
    assert _set(oracle.bruteforce_segment(dn0, dn1, [-2, -2, -2], [3, 3, 3])) == {(1, 0, 0), (0, 0, 0)}
