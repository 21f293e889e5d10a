// Device-side building blocks: error word, voxel lookup, integer segment walk
// and the per-warp shared-memory sets.
#pragma once

#include "fc_internal.cuh"

namespace fc {

constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x >> 1); }

__device__ __forceinline__ void set_error(DevState* st, int32_t code, int32_t info = 0) {
  if (atomicCAS(&st->error, 0, code) == 0) atomicExch(&st->error_info, info);
}

// Checked builds (FASTCOD_CHECKED=1) test every computed index of the
// path's gathers, scatters and list writes against its array's extent: a
// failure records kErrChecked with the site in the call's error word (st,
// when given) and the access is skipped.  In other builds the test is the
// constant true and compiles away.
#ifndef FASTCOD_CHECKED
#define FASTCOD_CHECKED 0
#endif
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, DevState* st, int32_t site) {
#if FASTCOD_CHECKED
  if (i >= 0 && i < n) return true;
  if (st) set_error(st, kErrChecked, site);
  return false;
#else
  (void)i;
  (void)n;
  (void)st;
  (void)site;
  return true;
#endif
}

__host__ __device__ inline int64_t voxel_count(const VolView& v) { return (int64_t)v.dx * v.dy * v.dz; }

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ROI row (-1 = none) and label (0 = none) of voxel (x, y, z); voxels off the
// grid have neither (loc2region outside every region).
__device__ __forceinline__ void voxel_lookup(const VolView& v, int32_t x, int32_t y, int32_t z,
                                             int32_t& row, int32_t& lab, DevState* ck = nullptr) {
  row = -1;
  lab = 0;
  if ((unsigned)x < (unsigned)v.dx && (unsigned)y < (unsigned)v.dy && (unsigned)z < (unsigned)v.dz) {
    const int32_t lin = x + v.dx * (y + v.dy * z);
    if (!in_bounds(lin, voxel_count(v), ck, kSiteCode)) return;
    const uint32_t code = __ldg(v.code + lin);
    if (code & kCodeRoi) {
      row = (int32_t)(code & kCodeRowMask);
      if (code & kCodeRoiLabelled) lab = (int32_t)__ldg(v.lab + lin);
    } else {
      lab = (int32_t)code;
    }
  }
}

// Brick bits (bit 0 ROI, bit 1 label) of brick (bx, by, bz), in range.
__device__ __forceinline__ uint32_t brick_bits(const VolView& v, int32_t bx, int32_t by, int32_t bz,
                                               DevState* ck = nullptr) {
  const int32_t b = bx + v.bx * (by + v.by * bz);
  if (!in_bounds(b, (int64_t)v.bx * v.by * v.bz, ck, kSiteBrick)) return 3u;  // conservative
  return (__ldg(v.bricks + (b >> 4)) >> ((b & 15) * 2)) & 3u;
}

// Conservative occupancy of the voxel box [lo, hi] (inclusive): the OR of the
// brick bits over every in-grid brick the box overlaps.  Boxes spanning more
// than two bricks on an axis report both bits (long segments are rare and
// walking them is always exact).
__device__ __forceinline__ uint32_t box_bits(const VolView& v, int32_t lx, int32_t ly, int32_t lz,
                                             int32_t hx, int32_t hy, int32_t hz, DevState* ck = nullptr) {
  if (hx < 0 || hy < 0 || hz < 0 || lx >= v.dx || ly >= v.dy || lz >= v.dz) return 0u;
  const int32_t bx0 = max(lx, 0) >> kBrickLog2, bx1 = min(hx, v.dx - 1) >> kBrickLog2;
  const int32_t by0 = max(ly, 0) >> kBrickLog2, by1 = min(hy, v.dy - 1) >> kBrickLog2;
  const int32_t bz0 = max(lz, 0) >> kBrickLog2, bz1 = min(hz, v.dz - 1) >> kBrickLog2;
  if (bx1 - bx0 > 1 || by1 - by0 > 1 || bz1 - bz0 > 1) return 3u;
  uint32_t bits = 0;
  for (int32_t z = bz0; z <= bz1; ++z)
    for (int32_t y = by0; y <= by1; ++y)
      for (int32_t x = bx0; x <= bx1; ++x) bits |= brick_bits(v, x, y, z, ck);
  return bits;
}

// Near bits of the cell holding voxel (vx, vy, vz) (bit 0: an ROI voxel
// within Chebyshev distance 1 of some voxel of the cell, bit 1: a labelled
// one); cells past the grown grid clamp to the zero border.  nw: the grid in
// shared memory (kSmem) or global memory.
template <bool kSmem>
__device__ __forceinline__ uint32_t near_lookup(const VolView& v, const uint32_t* nw, int32_t vx, int32_t vy,
                                                int32_t vz, DevState* ck = nullptr) {
  const uint32_t cx = min((uint32_t)((vx + 1) >> v.nsh), (uint32_t)v.cmx);
  const uint32_t cy = min((uint32_t)((vy + 1) >> v.nsh), (uint32_t)v.cmy);
  const uint32_t cz = min((uint32_t)((vz + 1) >> v.nsh), (uint32_t)v.cmz);
  const uint32_t w = (cx >> 4) + (uint32_t)v.nwx * (cy + (uint32_t)v.nny * cz);
  if (!in_bounds(w, near_words(v), ck, kSiteNear)) return 3u;  // conservative
  const uint32_t word = kSmem ? nw[w] : __ldg(nw + w);
  return (word >> ((cx & 15u) << 1)) & 3u;
}

// The same two bits at bits k and k + 1 of the result (k even), for the
// prefilter.  No per-axis clamp: for a voxel of the grown grid the index is
// the cell's, and for any other voxel the true bits are zero (no voxel within
// distance 1 lies in the grid), so whatever word the unclamped index reaches
// is conservative; only the word index itself is held inside the array.  The
// word is rotated right by twice the cell's place less k (a funnel shift
// takes the amount mod 32), which leaves the cell's bits at k and k + 1.
template <bool kSmem>
__device__ __forceinline__ uint32_t near_bits_at(const VolView& v, const uint32_t* nw, int32_t vx, int32_t vy,
                                                 int32_t vz, int k, DevState* ck = nullptr) {
  const int32_t cx = (vx + 1) >> v.nsh, cy = (vy + 1) >> v.nsh, cz = (vz + 1) >> v.nsh;
  const uint32_t nwm = (uint32_t)near_words(v) - 1u;
  const uint32_t w = min((uint32_t)(cx >> 4) + (uint32_t)v.nwx * ((uint32_t)cy + (uint32_t)v.nny * (uint32_t)cz), nwm);
  if (!in_bounds(w, near_words(v), ck, kSiteNear)) return 3u << k;  // conservative
  const uint32_t word = kSmem ? nw[w] : __ldg(nw + w);
  return __funnelshift_r(word, word, ((uint32_t)cx << 1) - (uint32_t)k) & (3u << k);
}

// ---------------------------------------------------------------------------
// Integer walk of one segment P0 -> P1 (Amanatides & Woo, exact rational
// events).  For axis a with d_a != 0 the next plane crossing is at
// t = num_a / den_a, den_a = |d_a|.  An increasing axis moves into the next
// voxel AT its crossing (allowed while t <= 1: a segment ending on a plane
// reaches the upper voxel); a decreasing axis moves JUST AFTER it (allowed
// while t < 1).  At the earliest crossing the increasing axes tied there move
// first; tied decreasing axes move on the following step, which finds the
// same t again.  Every move enters one new voxel.
//
// P is uint32_t when every den < 2^16 (compared numerators never exceed
// their den, so products stay below 2^32) and unsigned long long otherwise
// (|coordinate| < 2^24 keeps products below 2^52).
template <typename P>
struct SegWalk {
  int32_t cx, cy, cz;      // current voxel
  P nx, ny, nz;            // numerators of the next crossings
  P ex, ey, ez;            // denominators |d_a| (1 for a still axis)
  int32_t sx, sy, sz;      // direction of each axis (-1, 0, 1)

  __device__ __forceinline__ static void axis(int32_t a0, int32_t a1, int32_t& c, P& num, P& den, int32_t& sgn) {
    const int32_t d = a1 - a0;
    c = a0 >> kUnitLog2;
    if (d > 0) {
      sgn = 1;
      den = (P)d;
      num = (P)(((c + 1) << kUnitLog2) - a0);
    } else if (d < 0) {
      sgn = -1;
      den = (P)(-d);
      num = (P)(a0 - (c << kUnitLog2));
    } else {
      sgn = 0;
      den = 1;
      num = 0;
    }
  }

  __device__ __forceinline__ void init(const int32_t p0[3], const int32_t p1[3]) {
    axis(p0[0], p1[0], cx, nx, ex, sx);
    axis(p0[1], p1[1], cy, ny, ey, sy);
    axis(p0[2], p1[2], cz, nz, ez, sz);
  }

  __device__ __forceinline__ static bool pending(P num, P den, int32_t sgn) {
    return sgn > 0 ? (num <= den) : (sgn < 0 ? (num < den) : false);
  }

  // Enter the next voxel; false when the segment has no crossing left.  The
  // earliest pending crossing t* = bn / bd is found by exact cross-products;
  // the axes crossing at t* are tied.
  __device__ __forceinline__ bool step() {
    const bool q0 = pending(nx, ex, sx), q1 = pending(ny, ey, sy), q2 = pending(nz, ez, sz);
    if (!(q0 || q1 || q2)) return false;
    P bn = q0 ? nx : (q1 ? ny : nz);
    P bd = q0 ? ex : (q1 ? ey : ez);
    if (q1 && ny * bd < bn * ey) {
      bn = ny;
      bd = ey;
    }
    if (q2 && nz * bd < bn * ez) {
      bn = nz;
      bd = ez;
    }
    const bool t0 = q0 && nx * bd == bn * ex;
    const bool t1 = q1 && ny * bd == bn * ey;
    const bool t2 = q2 && nz * bd == bn * ez;
    const bool up = (t0 && sx > 0) || (t1 && sy > 0) || (t2 && sz > 0);
    const int32_t want = up ? 1 : -1;
    if (t0 && sx == want) {
      cx += want;
      nx += (P)(1 << kUnitLog2);
    }
    if (t1 && sy == want) {
      cy += want;
      ny += (P)(1 << kUnitLog2);
    }
    if (t2 && sz == want) {
      cz += want;
      nz += (P)(1 << kUnitLog2);
    }
    return true;
  }
};

// The same walk for a segment shorter than one voxel on every axis
// (|d_a| < 1024, so each axis crosses at most one plane).  The crossing
// parameters num_a / den_a are brought to the common denominator
// D = den_x den_y den_z (den = 1 for a still axis): T_a = num_a (D / den_a)
// and D stay below 2^31, so SegWalk's cross-product comparisons become plain
// unsigned comparisons of the T_a, and a crossing adds 1024 (D / den_a).  An
// axis is pending while T_a < lim_a (D + 1 for an increasing axis, D for a
// decreasing one, 0 for a still one).  Same voxels, same order, same tie
// rule as SegWalk.
struct SegShort {
  int32_t cx, cy, cz;      // current voxel
  uint32_t tx, ty, tz;     // T_a
  uint32_t lx, ly, lz;     // pending while T_a < lim_a
  uint32_t ux, uy, uz;     // 1024 D / den_a
  int32_t sx, sy, sz;      // direction of each axis (-1, 0, 1)

  __device__ __forceinline__ static void axis(int32_t a0, int32_t a1, int32_t& c, uint32_t& num, uint32_t& den,
                                              int32_t& sgn) {
    const int32_t d = a1 - a0;
    c = a0 >> kUnitLog2;
    sgn = d > 0 ? 1 : (d < 0 ? -1 : 0);
    den = d > 0 ? (uint32_t)d : (d < 0 ? (uint32_t)(-d) : 1u);
    num = d > 0 ? (uint32_t)(((c + 1) << kUnitLog2) - a0) : (d < 0 ? (uint32_t)(a0 - (c << kUnitLog2)) : 0u);
  }

  __device__ __forceinline__ void init(const int32_t p0[3], const int32_t p1[3]) {
    uint32_t nx, ny, nz, ex, ey, ez;
    axis(p0[0], p1[0], cx, nx, ex, sx);
    axis(p0[1], p1[1], cy, ny, ey, sy);
    axis(p0[2], p1[2], cz, nz, ez, sz);
    const uint32_t dyz = ey * ez, dxz = ex * ez, dxy = ex * ey, D = ex * dyz;
    tx = nx * dyz;
    ty = ny * dxz;
    tz = nz * dxy;
    ux = dyz << kUnitLog2;
    uy = dxz << kUnitLog2;
    uz = dxy << kUnitLog2;
    lx = sx > 0 ? D + 1 : (sx < 0 ? D : 0u);
    ly = sy > 0 ? D + 1 : (sy < 0 ? D : 0u);
    lz = sz > 0 ? D + 1 : (sz < 0 ? D : 0u);
  }

  __device__ __forceinline__ bool step() {
    const bool q0 = tx < lx, q1 = ty < ly, q2 = tz < lz;
    if (!(q0 || q1 || q2)) return false;
    const uint32_t m = min(min(q0 ? tx : 0xffffffffu, q1 ? ty : 0xffffffffu), q2 ? tz : 0xffffffffu);
    const bool t0 = q0 && tx == m, t1 = q1 && ty == m, t2 = q2 && tz == m;
    const int32_t want = ((t0 && sx > 0) || (t1 && sy > 0) || (t2 && sz > 0)) ? 1 : -1;
    if (t0 && sx == want) {
      cx += want;
      tx += ux;
    }
    if (t1 && sy == want) {
      cy += want;
      ty += uy;
    }
    if (t2 && sz == want) {
      cz += want;
      tz += uz;
    }
    return true;
  }
};

// ---------------------------------------------------------------------------
// Per-warp open-addressing set in shared memory (keys >= 0, empty = -1).
// Lanes holding the same key are merged with __match_any_sync first; the
// lowest lane of each group inserts with atomicCAS.  New keys are appended to
// list[n..] in lane order.  Returns the new size; sets *fail when a probe
// sequence found no slot (cannot happen while size < H).
template <int H>
__device__ __forceinline__ int set_insert(int32_t* tab, int32_t* list, int n, int32_t key, bool& fail,
                                          int32_t cap = 0x7fffffff, DevState* ck = nullptr) {
  const unsigned want = __ballot_sync(kFull, key >= 0);
  if (want == 0u) return n;
  bool fresh = false;
  if (key >= 0) {
    const unsigned peers = __match_any_sync(want, key);
    if ((peers & lanemask_lt()) == 0u) {
      uint32_t h = ((uint32_t)key * 0x9E3779B1u) >> (32 - ilog2(H));
      int probe = 0;
      for (; probe < H; ++probe) {
        const int32_t old = atomicCAS(tab + h, -1, key);
        if (old == -1) { fresh = true; break; }
        if (old == key) break;
        h = (h + 1) & (H - 1);
      }
      if (probe == H) fail = true;
    }
  }
  const unsigned fm = __ballot_sync(kFull, fresh);
  if (fresh) {
    const int at = n + __popc(fm & lanemask_lt());
    if (in_bounds(at, cap, ck, kSiteSetList)) list[at] = key;
  }
  return n + __popc(fm);
}

}  // namespace fc
