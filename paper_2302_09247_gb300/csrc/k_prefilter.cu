// K2: prefilter + compaction over the full vertex stream.
//
// Every streamline is read once.  A streamline that passes near no ROI voxel
// or near no labelled voxel can contribute neither to C nor to C_end (whose
// seed and endpoint lie on the streamline) and is dropped; the ids of the
// others are appended to a compact survivor list (one atomic per 32 survivors
// of a warp).  The test is conservative; the walk decides exactly.  On the way
// the kernel validates offsets and coordinates and counts voxel-steps.
//
// The test.  The near grid holds, per cell, whether an ROI voxel / a labelled
// voxel lies within Chebyshev distance 1 of a voxel of the cell.  A segment
// whose end voxels differ by at most one on every axis lies in the 3x3x3
// block around either end voxel, so the near bits of either end cover it.
// Every segment has an end vertex of even index, so the near bits of the
// even-indexed vertices of a streamline cover all of its short segments; a
// longer segment adds the brick occupancy of its whole voxel box (exact,
// rare); a streamline of one vertex at an odd index is kept unconditionally
// (the walk decides it).
//
// Vertex-parallel scan.  Each warp owns a contiguous range of streamlines
// holding about the same number of vertices as every other warp's, and walks
// its vertex range in 2048-vertex windows aligned to 2048, each eight
// 256-vertex pieces; in a piece, lane l takes the eight consecutive vertices
// 8l..8l+7 (six 16-byte words), so every lane is busy whatever the
// streamline lengths:
//   - the streamline boundaries (offsets) falling in the window, kept in a
//     two-group register cache of 64 offsets per warp, set the window's start
//     bits (shared-memory atomics, one word per 32 vertices);
//   - per vertex: coordinate check, voxel-step count and long-segment check of
//     the segment ending there (unless the vertex starts a streamline), and
//     at even vertices a near-grid lookup (shared memory when the grid fits);
//   - one warp scan of the per-lane hit counts of the window's pieces gives,
//     at every boundary x, the running number of ROI / target hits before x,
//     and the streamline ending at x passes when both counts grew since its
//     start boundary.
// Two loaders with identical results: TMA (default; the pieces stream through
// a ring of three 3072-byte slots per warp in shared memory, cp.async.bulk +
// mbarrier, L2 evict-first) and direct streaming loads into registers (the
// next piece in flight while the current one is processed).
#include <type_traits>

#include "fc_device.cuh"
#include "fc_tma.cuh"

#ifndef PREFILTER_PIECES
#define PREFILTER_PIECES 8
#endif

namespace fc {

namespace {

constexpr int kPieceLog2 = 8;
constexpr int kPiece = 1 << kPieceLog2;     // vertices per piece (= per TMA slot)
constexpr int kPieces = PREFILTER_PIECES;  // pieces per window
constexpr int kWinLog2 = kPieceLog2 + ilog2(kPieces);
constexpr int kWin = 1 << kWinLog2;       // vertices per window
constexpr int kCountWords = kPieces / 2;  // per-lane hit counts: two pieces (R, T bytes) per word
static_assert(kPieces == 2 || kPieces == 4 || kPieces == 8, "2, 4 or 8 pieces per window");
// a lane's hit bits of every piece of a window, 8 per piece
using HitWord = typename std::conditional<(kPieces > 4), unsigned long long, uint32_t>::type;
constexpr int kVpl = kPiece / 32;          // vertices per lane per piece
constexpr int kLaneWords = kVpl * 3;      // 24 int32 per lane per piece
constexpr int kPieceWords = kPiece * 3;     // 768 int32 = 3072 bytes
constexpr int kStages = 3;                // TMA ring depth per warp (pieces)
constexpr int kWarps = 8;                 // warps per CTA
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;  // 1 s
constexpr int32_t kInf = 0x7fffffff;
constexpr int64_t kNearSmemWords = 12288;  // direct loader: near grids up to 48 KB live in shared memory

__device__ __forceinline__ uint32_t lowmask(int32_t k) { return k >= 32 ? 0xffffffffu : ((1u << k) - 1u); }

struct WarpShared {
  int32_t sbuf[64];          // short survivors awaiting a flush
  int32_t lbuf[64];          // long survivors awaiting a flush
  uint32_t st[kWin / 32];    // start bits of the current window
};

// Per-warp scan state (registers).  Vertex positions are absolute indices
// into the subject's vertex array (< 2^31).
struct Scan {
  const int64_t* off;
  int32_t V0, V1;            // vertex range [V0, V1)
  int64_t s_lo, s_cur, s_hi; // boundaries s_lo..s_hi; s_cur = next one to decide
  int64_t cbase;             // cache: lane i holds off[cbase + i] (cA), off[cbase + 32 + i] (cB)
  int32_t cA, cB;            // kInf past s_hi
  uint32_t cumR, cumT;       // hit counts before the current window
  uint32_t lastR, lastT;     // hit counts at the last decided boundary
  int32_t last_b;            // that boundary
  uint32_t carry;            // the current window's vertex 0 starts a streamline
  int32_t qx, qy, qz;        // voxel of the last vertex processed (lane 31's)
  unsigned long long steps;  // voxel steps counted by this lane
  uint32_t singles, kept, badc;
  int nbuf, nlong;           // entries of sbuf, lbuf
  bool abort;
  int64_t id_base;           // survivor ids are id_base + streamline index
  DevState* sst;             // the subject's counters and error word
};

// Boundary base + lane (kInf past s_hi), saturated into int32 so that the
// range check below sees any out-of-range value.
__device__ __forceinline__ int32_t load_bnd(const Scan& sc, int64_t base) {
  const int64_t i = base + lane_id();
  if (i > sc.s_hi) return kInf;
  const int64_t b = __ldg(sc.off + i);
  return b < 0 ? -1 : (b >= kInf ? kInf : (int32_t)b);
}

// Offsets base .. base+31 (g, one per lane) lie in [V0, V1] and do not
// decrease, starting at or after prev.  Warp-uniform; flags the error.
__device__ __forceinline__ bool check_group(Scan& sc, int32_t g, int64_t base, int32_t prev) {
  const int32_t lane = (int32_t)lane_id();
  const int64_t i = base + lane;
  const int32_t nx = __shfl_down_sync(kFull, g, 1);
  bool ok = i > sc.s_hi || (g >= sc.V0 && g <= sc.V1);
  ok &= lane == 31 || i + 1 > sc.s_hi || g <= nx;
  ok &= lane != 0 || i > sc.s_hi || g >= prev;
  if (__all_sync(kFull, ok)) return true;
  if (lane == 0) set_error(sc.sst, kErrOffsets, (int32_t)base);
  sc.abort = true;
  return false;
}

// Position the cache so that s_cur lies in its first group.  A group is
// checked when it becomes the first one (its load was issued a group
// earlier) or when it is dropped.
__device__ __forceinline__ void cache_seek(Scan& sc) {
  while (sc.s_cur >= sc.cbase + 32 && !sc.abort) {
    const int32_t a31 = __shfl_sync(kFull, sc.cA, 31);
    if (!check_group(sc, sc.cB, sc.cbase + 32, a31)) return;
    if (sc.s_cur < sc.cbase + 64) {
      sc.cA = sc.cB;
      sc.cbase += 32;
      sc.cB = load_bnd(sc, sc.cbase + 32);
    } else {
      sc.cbase = sc.s_cur;
      sc.cA = load_bnd(sc, sc.cbase);
      sc.cB = load_bnd(sc, sc.cbase + 32);
      check_group(sc, sc.cA, sc.cbase, sc.last_b);
    }
  }
}

// Boundaries s + lane for a warp-uniform s >= cbase: from the cache when
// s < cbase + 32, else loaded and checked here (windows with more than
// 32 boundaries).
__device__ __forceinline__ int32_t fetch_bnd(Scan& sc, int64_t s, int32_t prev) {
  if (s < sc.cbase + 32) {
    const int32_t i = (int32_t)(s - sc.cbase) + (int32_t)lane_id();
    const int32_t a = __shfl_sync(kFull, sc.cA, i & 31);
    const int32_t b = __shfl_sync(kFull, sc.cB, i & 31);
    return i < 32 ? a : b;
  }
  const int32_t g = load_bnd(sc, s);
  check_group(sc, g, s, prev);
  return g;
}

// Appends the n buffered ids to the launch's survivor list (counters in gst):
// short streamlines from its front, long ones from its back, so that the walk
// can take the long ones first.
__device__ __forceinline__ void flush_ids(int& n, const int32_t* buf, bool back, const SurvList& surv,
                                          DevState* gst) {
  __syncwarp();
  uint32_t base = 0;
  if (lane_id() == 0 && n > 0) base = atomicAdd(back ? &gst->n_long : &gst->n_survivors, (uint32_t)n);
  base = __shfl_sync(kFull, base, 0);
  for (int k = (int)lane_id(); k < n; k += 32) {  // n <= 64
    const int64_t pos = (int64_t)base + k;
    const int64_t at = back ? surv.cap - 1 - pos : pos;
    if (in_bounds(at, surv.cap, gst, kSiteSurvivorWrite)) surv.ids[at] = buf[k];
  }
  __syncwarp();
  n = 0;
}

// Brick occupancy of the voxel box [lo, hi] of a long segment, out of line
// (rare).
__device__ __noinline__ uint32_t long_box(const uint32_t* bricks, int32_t dx, int32_t dy, int32_t dz, int32_t bx,
                                          int32_t by, int32_t lx, int32_t ly, int32_t lz, int32_t hx, int32_t hy,
                                          int32_t hz, DevState* ck) {
  VolView v;
  v.bricks = bricks;
  v.dx = dx;
  v.dy = dy;
  v.dz = dz;
  v.bx = bx;
  v.by = by;
  v.bz = (dz + (1 << kBrickLog2) - 1) >> kBrickLog2;
  return box_bits(v, lx, ly, lz, hx, hy, hz, ck);
}

// 1. Start of window W (first vertex, a multiple of kWin): boundaries b with
//    b - W <= kWin are decided in this window (nbw of them, from s_cur); those
//    with b - W < kWin start a streamline at a vertex of it (start bits in
//    ws.st).  b_first: the lane's boundary of the first round of 32.
__device__ __forceinline__ void window_begin(Scan& sc, WarpShared& ws, int32_t W, int32_t& nbw, int32_t& b_first) {
  const int32_t lane = (int32_t)lane_id();
  cache_seek(sc);
  for (int i = lane; i < kWin / 32; i += 32) ws.st[i] = 0u;
  __syncwarp();
  nbw = 0;
  b_first = kInf;
  int64_t s = sc.s_cur;
  int32_t prev = sc.last_b;
  for (int round = 0;; ++round) {
    const int32_t b = fetch_bnd(sc, s, prev);
    if (round == 0) b_first = b;
    const int32_t r = b - W;
    if ((uint32_t)r < (uint32_t)kWin) atomicOr(&ws.st[r >> 5], 1u << (r & 31));
    const int n = __popc(__ballot_sync(kFull, r <= kWin));
    nbw += n;
    if (n < 32 || sc.abort) break;
    prev = __shfl_sync(kFull, b, 31);
    s += 32;
  }
  __syncwarp();
}

// 2. Piece h of window W: p = the lane's 24 words, vertices
//    W + h*kPiece + 8l .. +7 (zero past the end of the array).  Returns the
//    lane's hit bits (R hits at the even bits k, T hits at bits k + 1, for
//    the lookups at the even slots k).
template <bool kSmem>
__device__ __forceinline__ uint32_t scan_piece(Scan& sc, const VolView& v, const uint32_t* nw,
                                              const int32_t (&p)[kLaneWords], int h, int32_t W, const WarpShared& ws) {
  const int32_t lane = (int32_t)lane_id();
  const uint32_t st8 = ((ws.st[h * (kPiece / 32) + (lane >> 2)] >> ((lane & 3) << 3)) & 0xffu) |
                       ((h == 0 && lane == 0) ? sc.carry : 0u);
  const int32_t base = W + h * kPiece + kVpl * lane;
  const int32_t lo = sc.V0 - base, hi = sc.V1 - base;
  const uint32_t valid8 = lowmask(min(max(hi, 0), kVpl)) & ~lowmask(min(max(lo, 0), kVpl));
  const uint32_t keep8 = valid8 & ~st8;  // slots whose incoming segment is counted

  // every lane takes part in the shuffles; lane 0 then takes the carried voxel
  int32_t q0x = __shfl_up_sync(kFull, p[kLaneWords - 3] >> kUnitLog2, 1);
  int32_t q0y = __shfl_up_sync(kFull, p[kLaneWords - 2] >> kUnitLog2, 1);
  int32_t q0z = __shfl_up_sync(kFull, p[kLaneWords - 1] >> kUnitLog2, 1);
  if (lane == 0) {
    q0x = sc.qx;
    q0y = sc.qy;
    q0z = sc.qz;
  }
  uint32_t h8 = 0u, lg = 0u, bad = 0u, stp = 0u;
  {
    int32_t qx = q0x, qy = q0y, qz = q0z;
#pragma unroll
    for (int k = 0; k < kVpl; ++k) {
      const int32_t x = p[3 * k], y = p[3 * k + 1], z = p[3 * k + 2];
      bad |= (uint32_t)(x + kCoordLimit) | (uint32_t)(y + kCoordLimit) | (uint32_t)(z + kCoordLimit);
      const int32_t vx = x >> kUnitLog2, vy = y >> kUnitLog2, vz = z >> kUnitLog2;
      const uint32_t ax = (uint32_t)abs(vx - qx), ay = (uint32_t)abs(vy - qy), az = (uint32_t)abs(vz - qz);
      const uint32_t m = 0u - ((keep8 >> k) & 1u);
      lg |= (ax | ay | az) & m;
      stp += (ax + ay + az) & m;
      if ((k & 1) == 0) h8 |= near_bits_at<kSmem>(v, nw, vx, vy, vz, k, sc.sst);
      qx = vx;
      qy = vy;
      qz = vz;
    }
  }
  sc.badc |= bad;
  sc.steps += stp + (uint32_t)__popc(keep8);
  if (lg > 1u) {
    // long segments (slots whose keep bit is set and whose end voxels differ
    // by more than one on some axis): the brick occupancy of the segment's
    // voxel box, as hits on the segment's even vertex
    int32_t qx = q0x, qy = q0y, qz = q0z;
#pragma unroll
    for (int k = 0; k < kVpl; ++k) {
      const int32_t vx = p[3 * k] >> kUnitLog2, vy = p[3 * k + 1] >> kUnitLog2, vz = p[3 * k + 2] >> kUnitLog2;
      if (((keep8 >> k) & 1u) && (uint32_t)(abs(vx - qx) | abs(vy - qy) | abs(vz - qz)) > 1u)
        h8 |= long_box(v.bricks, v.dx, v.dy, v.dz, v.bx, v.by, min(vx, qx), min(vy, qy), min(vz, qz), max(vx, qx),
                       max(vy, qy), max(vz, qz), sc.sst)
              << (k & ~1);
      qx = vx;
      qy = vy;
      qz = vz;
    }
  }
  sc.qx = __shfl_sync(kFull, p[kLaneWords - 3] >> kUnitLog2, 31);
  sc.qy = __shfl_sync(kFull, p[kLaneWords - 2] >> kUnitLog2, 31);
  sc.qz = __shfl_sync(kFull, p[kLaneWords - 1] >> kUnitLog2, 31);
  return h8;
}

// 3. End of window W: hit counts of its pieces (hh: piece h's hit bits at
//    bits 8h) and the decisions at its nbw boundaries, 32 per round.
__device__ __forceinline__ void window_end(Scan& sc, WarpShared& ws, int32_t W, int32_t nbw, int32_t b_first,
                                           HitWord hh, bool prefilter, const SurvList& surv, DevState* gst) {
  const int32_t lane = (int32_t)lane_id();
  // per-lane counts in byte fields (R and T of two pieces per word); a
  // field's prefix over the warp is at most 4 * 32 = 128, so fields never
  // carry
  uint32_t excl[kCountWords], totw[kCountWords];
#pragma unroll
  for (int w = 0; w < kCountWords; ++w) {
    const uint32_t b0 = (uint32_t)(hh >> (16 * w)) & 0xffu, b1 = (uint32_t)(hh >> (16 * w + 8)) & 0xffu;
    const uint32_t c = (uint32_t)__popc(b0 & 0x55u) | ((uint32_t)__popc(b0 & 0xaau) << 8) |
                       ((uint32_t)__popc(b1 & 0x55u) << 16) | ((uint32_t)__popc(b1 & 0xaau) << 24);
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += y;
    }
    excl[w] = inc - c;
    totw[w] = __shfl_sync(kFull, inc, 31);
  }
  // hit counts of the pieces before piece h, and of the whole window
  uint32_t baseR[kPieces + 1], baseT[kPieces + 1];
  baseR[0] = baseT[0] = 0u;
#pragma unroll
  for (int h = 0; h < kPieces; ++h) {
    const uint32_t f = totw[h >> 1] >> (16 * (h & 1));
    baseR[h + 1] = baseR[h] + (f & 0xffu);
    baseT[h + 1] = baseT[h] + ((f >> 8) & 0xffu);
  }

  int64_t s = sc.s_cur;
  int32_t prev = sc.last_b;
  for (int round = 0; nbw > 0 && !sc.abort; ++round) {
    const int32_t b = round == 0 ? b_first : fetch_bnd(sc, s, prev);
    const int n = min(nbw, 32);
    const bool in = lane < n;
    const int32_t x = min(max(b - W, 0), kWin);
    const int32_t hx = x >> kPieceLog2, xi = x & (kPiece - 1);
    const int32_t src = xi >> 3, o = xi & 7;
    uint32_t e = __shfl_sync(kFull, excl[0], src);
#pragma unroll
    for (int w = 1; w < kCountWords; ++w) {
      const uint32_t ew = __shfl_sync(kFull, excl[w], src);
      if ((hx >> 1) == w) e = ew;
    }
    const uint32_t hb = (uint32_t)(__shfl_sync(kFull, hh, src) >> (8 * (hx & (kPieces - 1)))) & 0xffu;
    uint32_t bR = baseR[kPieces], bT = baseT[kPieces];
#pragma unroll
    for (int h = kPieces - 1; h >= 0; --h)
      if (hx == h) {
        bR = baseR[h];
        bT = baseT[h];
      }
    uint32_t cR = bR, cT = bT;
    if (hx < kPieces) {
      const int sh = 16 * (hx & 1);
      cR += ((e >> sh) & 0xffu) + (uint32_t)__popc(hb & 0x55u & lowmask(o));
      cT += ((e >> (sh + 8)) & 0xffu) + (uint32_t)__popc(hb & 0xaau & lowmask(o + 1));
    }
    cR += sc.cumR;
    cT += sc.cumT;
    uint32_t pR = __shfl_up_sync(kFull, cR, 1), pT = __shfl_up_sync(kFull, cT, 1);
    int32_t pb = __shfl_up_sync(kFull, b, 1);
    if (lane == 0) {
      pR = sc.lastR;
      pT = sc.lastT;
      pb = sc.last_b;
    }
    // boundary s + lane closes streamline s + lane - 1 = [pb, b)
    const bool real = in && s + lane > sc.s_lo;
    const int32_t T = b - pb;
    const bool near_hit = (cR != pR && cT != pT) || (T == 1 && (pb & 1));
    const bool pass = real && T > 0 && (!prefilter || near_hit);
    if (real && T == 1) sc.singles += 1u;
    const bool lng = T - 1 > kLongSegments;
    const uint32_t pm = __ballot_sync(kFull, pass && !lng), pl = __ballot_sync(kFull, pass && lng);
    if (pass) {
      const int32_t id = (int32_t)(sc.id_base + s + lane - 1);
      if (lng) ws.lbuf[sc.nlong + __popc(pl & lanemask_lt())] = id;
      else ws.sbuf[sc.nbuf + __popc(pm & lanemask_lt())] = id;
    }
    sc.nbuf += __popc(pm);
    sc.nlong += __popc(pl);
    sc.kept += __popc(pm | pl);
    if (sc.nbuf >= 32) flush_ids(sc.nbuf, ws.sbuf, false, surv, gst);
    if (sc.nlong >= 32) flush_ids(sc.nlong, ws.lbuf, true, surv, gst);
    sc.lastR = __shfl_sync(kFull, cR, n - 1);
    sc.lastT = __shfl_sync(kFull, cT, n - 1);
    sc.last_b = __shfl_sync(kFull, b, n - 1);
    prev = __shfl_sync(kFull, b, 31);
    s += n;
    nbw -= n;
  }
  sc.s_cur = s;
  sc.carry = (sc.last_b - W == kWin) ? 1u : 0u;
  sc.cumR += baseR[kPieces];
  sc.cumT += baseT[kPieces];
}

// Vertex-balanced ranges.  Warp g of G scans the streamlines s with
// split(g) <= s < split(g + 1), where split(g) is the first s with
// off[s] >= nv * g / G (split(0) = 0, split(G) = ns), so that every warp
// reads about the same number of vertices whatever the length mix.  Two
// half-warp 16-ary searches (one per end of the range); the first round probes
// every 256 streamlines around the streamline-count split, which usually
// brackets the answer (three rounds in all).  On
// valid offsets split() does not decrease in g; ranges that come out reversed
// can only come from decreasing offsets and are reported by warp_init.
__device__ __forceinline__ void vertex_split(const int64_t* off, int64_t ns, int64_t nv, int64_t g, int64_t G,
                                             int64_t& s_lo, int64_t& s_hi) {
  const int32_t lane = (int32_t)lane_id(), sub = lane & 15, half = lane >> 4;
  const int64_t gg = g + half;
  const int64_t target = nv * gg / G, guess = ns * gg / G;
  int64_t lo = 0, hi = ns;  // the answer lies in [lo, hi]
  if (gg == 0 || gg == G) lo = hi = gg == 0 ? 0 : ns;
  for (int round = 0; __any_sync(kFull, lo < hi); ++round) {
    const bool act = lo < hi;
    const int64_t p = round == 0 ? min(max(guess + 256 * (sub - 7), (int64_t)0), ns)
                                 : lo + ((int64_t)(sub + 1) * (hi - lo)) / 16;  // p(15) = hi
    const bool ge = act && __ldg(off + p) >= target;
    const uint32_t m = (__ballot_sync(kFull, ge) >> (16 * half)) & 0xffffu;
    const int k = m ? __ffs(m) - 1 : 16;  // the first probe at or above the target
    const int64_t pk = __shfl_sync(kFull, p, 16 * half + min(k, 15));
    const int64_t pb = __shfl_sync(kFull, p, 16 * half + max(k - 1, 0));
    if (act) {
      if (k == 16) {  // every probe below the target: the answer lies above the last one
        lo = min(pk + 1, hi);
      } else {
        hi = pk;  // p(0) >= lo: with k = 0 the answer lies in [lo, p(0)]
        if (k > 0) lo = pb + 1;
      }
    }
  }
  s_lo = __shfl_sync(kFull, lo, 0);
  s_hi = __shfl_sync(kFull, lo, 16);
}

// Set up the scan of streamlines [s_lo, s_hi) of t; false when there is
// nothing to scan (or the offsets are invalid).
__device__ __forceinline__ bool warp_init(const Tract& t, int64_t s_lo, int64_t s_hi, Scan& sc, DevState* sst,
                                          int64_t id_base) {
  if (s_hi <= s_lo) {
    if (s_hi < s_lo && lane_id() == 0) set_error(sst, kErrOffsets, (int32_t)s_hi);
    return false;
  }
  const int64_t a = __ldg(t.off + s_lo), b = __ldg(t.off + s_hi);
  if (a < 0 || b > t.nv || a > b || (s_lo == 0 && a != 0) || (s_hi == t.ns && b != t.nv)) {
    if (lane_id() == 0) set_error(sst, kErrOffsets, (int32_t)s_lo);
    return false;
  }
  if (a == b) {
    // no vertices: every offset of the range must equal a
    bool ok = true;
    for (int64_t s = s_lo + lane_id(); s <= s_hi; s += 32) ok &= __ldg(t.off + s) == a;
    if (!__all_sync(kFull, ok) && lane_id() == 0) set_error(sst, kErrOffsets, (int32_t)s_lo);
    return false;
  }
  sc.off = t.off;
  sc.V0 = (int32_t)a;
  sc.V1 = (int32_t)b;
  sc.s_lo = s_lo;
  sc.s_cur = s_lo;
  sc.s_hi = s_hi;
  sc.cumR = sc.cumT = 0;
  sc.lastR = sc.lastT = 0;
  sc.last_b = sc.V0;
  sc.carry = 0;
  sc.qx = sc.qy = sc.qz = 0;
  sc.steps = 0;
  sc.singles = sc.kept = sc.badc = 0;
  sc.nbuf = sc.nlong = 0;
  sc.abort = false;
  sc.id_base = id_base;
  sc.sst = sst;
  sc.cbase = s_lo;
  sc.cA = load_bnd(sc, s_lo);
  sc.cB = load_bnd(sc, s_lo + 32);
  return check_group(sc, sc.cA, s_lo, sc.V0);
}

__device__ __forceinline__ void warp_finish(Scan& sc, WarpShared& ws, const SurvList& surv, DevState* gst) {
  // the last loaded group is checked here, and every boundary decided
  if (!sc.abort && sc.cbase + 32 <= sc.s_hi) check_group(sc, sc.cB, sc.cbase + 32, __shfl_sync(kFull, sc.cA, 31));
  if (!sc.abort && sc.s_cur != sc.s_hi + 1) {
    if (lane_id() == 0) set_error(sc.sst, kErrOffsets, (int32_t)sc.s_cur);
  }
  flush_ids(sc.nbuf, ws.sbuf, false, surv, gst);
  flush_ids(sc.nlong, ws.lbuf, true, surv, gst);
  unsigned long long s = sc.steps + sc.singles;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  const bool bad = __any_sync(kFull, (sc.badc >> 25) != 0u);
  if (lane_id() == 0) {
    atomicAdd(&sc.sst->voxel_steps, s);
    atomicAdd(&sc.sst->survivors, (unsigned long long)sc.kept);
    if (bad) set_error(sc.sst, kErrCoord, (int32_t)sc.s_lo);
  }
}

// ------------------------------------------------------------------ direct

// The lane's 24 words of piece hq (vertices hq * kPiece + 8l ..; zero past the
// end of the array).
__device__ __forceinline__ void load_piece(const Tract& t, int64_t hq, int32_t (&p)[kLaneWords]) {
  const int64_t g = (hq << kPieceLog2) + kVpl * lane_id();  // the lane's first vertex
  if (g + kVpl <= t.nv) {
    const int4* e = reinterpret_cast<const int4*>(t.xyz + 3 * g);  // 96-byte chunk, 16-byte aligned
#pragma unroll
    for (int i = 0; i < kLaneWords / 4; ++i) {
      const int4 a = __ldcs(e + i);
      p[4 * i] = a.x;
      p[4 * i + 1] = a.y;
      p[4 * i + 2] = a.z;
      p[4 * i + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int w = 0; w < kLaneWords; ++w) p[w] = (g + w / 3 < t.nv) ? __ldcs(t.xyz + 3 * g + w) : 0;
  }
}

// Window loop of the direct loader: the next piece is loaded while the
// current one is scanned.  Pieces wholly outside the scan's vertex range
// (at the ends of its first and last windows) are neither loaded nor scanned:
// the range's first vertex starts a streamline, so no state carries over them.
template <bool kSmem>
__device__ __forceinline__ void scan_range_direct(Scan& sc, const VolView& v, const uint32_t* nw, const Tract& t,
                                                  bool prefilter, WarpShared& ws, const SurvList& surv, DevState* gst) {
  const int64_t q0 = (int64_t)sc.V0 >> kWinLog2, q1 = (int64_t)(sc.V1 - 1) >> kWinLog2;
  const int64_t hq_lo = (int64_t)sc.V0 >> kPieceLog2, hq_hi = ((int64_t)(sc.V1 - 1) >> kPieceLog2) + 1;
  int32_t p[kLaneWords], nx[kLaneWords];
  load_piece(t, hq_lo, nx);
  for (int64_t q = q0; q <= q1 && !sc.abort; ++q) {
    const int32_t W = (int32_t)(q << kWinLog2);
    int32_t nbw, b_first;
    window_begin(sc, ws, W, nbw, b_first);
    HitWord hh = 0u;
    const int h_lo = q == q0 ? (int)(hq_lo - q * kPieces) : 0;
    const int h_hi = q == q1 ? (int)(hq_hi - q * kPieces) : kPieces;
#pragma unroll 1
    for (int h = h_lo; h < h_hi; ++h) {
      const int64_t hq = q * kPieces + h;
#pragma unroll
      for (int w = 0; w < kLaneWords; ++w) p[w] = nx[w];
      if (hq + 1 < hq_hi) load_piece(t, hq + 1, nx);
      hh |= (HitWord)scan_piece<kSmem>(sc, v, nw, p, h, W, ws) << (8 * h);
    }
    window_end(sc, ws, W, nbw, b_first, hh, prefilter, surv, gst);
  }
}

// --------------------------------------------------------------------- tma

// Per-warp ring of kStages piece slots filled by 1-D bulk copies.
// Slots are used in a fixed cyclic order for the warp's whole life (slot,
// phase), so ranges follow one another without re-initialising barriers:
// a range issues its first pieces into the slots after the last one used,
// and every piece issued is consumed (or drained) before the range ends.
// 128-byte aligned, so every warp's ring (a bulk-copy destination) starts on
// a 16-byte boundary.
struct __align__(128) TmaSmem {
  int32_t ring[kStages][kPieceWords];
  uint64_t bar[kStages];
};
static_assert(sizeof(TmaSmem) % 128 == 0 && (kPieceWords * 4) % 16 == 0, "ring slots must stay 16-byte aligned");

struct Ring {
  TmaSmem* sm;
  uint32_t slot, phase;   // next slot to consume, and the parity it completes
  uint64_t policy;
  int64_t withhold;       // test hook (kHook builds only): this piece is never copied

  __device__ __forceinline__ void init(TmaSmem* s, int64_t withhold_piece = -1) {
    sm = s;
    slot = 0;
    phase = 0;
    withhold = withhold_piece;
    policy = policy_evict_first();
    if (lane_id() == 0) {
      for (int k = 0; k < kStages; ++k) mbar_init(&sm->bar[k], 1);
      fence_mbar_init();
    }
    __syncwarp();
  }

  // lane 0 only: copy piece hq of t into slot k.  A whole piece is one bulk
  // copy; at the end of the array the part that is not a multiple of 16 bytes
  // is copied with plain loads and the rest of the slot zero-filled.
  template <bool kHook>
  __device__ __forceinline__ void issue(const Tract& t, int64_t hq, uint32_t k) {
    if (kHook && hq == withhold) return;  // neither copy nor arrival: the wait for this slot runs out
    const int64_t v0 = hq << kPieceLog2;
    int32_t* dst = sm->ring[k];
    const int32_t* src = t.xyz + 3 * v0;
    if (v0 + kPiece <= t.nv) {
      mbar_arrive_expect_tx(&sm->bar[k], (uint32_t)(kPieceWords * 4));
      bulk_g2s(dst, src, (uint32_t)(kPieceWords * 4), &sm->bar[k], policy);
      return;
    }
    const int64_t n = max((int64_t)0, t.nv - v0);
    const uint32_t bytes = (uint32_t)(n * 12);
    const uint32_t tma = bytes & ~15u;
    for (uint32_t w = tma >> 2; w < (bytes >> 2); ++w) dst[w] = __ldcs(src + w);
    for (uint32_t w = bytes >> 2; w < (uint32_t)kPieceWords; ++w) dst[w] = 0;
    if (tma) {
      mbar_arrive_expect_tx(&sm->bar[k], tma);
      bulk_g2s(dst, src, tma, &sm->bar[k], policy);
    } else {
      mbar_arrive(&sm->bar[k]);
    }
  }

  // Every lane waits on the slot to consume (acquiring its bytes); the
  // result is warp-uniform.
  __device__ __forceinline__ bool wait() {
    return __all_sync(kFull, mbar_wait_bounded(&sm->bar[slot], phase, kWaitTimeoutNs));
  }

  __device__ __forceinline__ void advance() {
    if (++slot == (uint32_t)kStages) {
      slot = 0;
      phase ^= 1u;
    }
  }
};

// Takes the next piece from the ring into p and refills its slot with piece
// `issued` when that is still part of the range (hq_end exclusive).  False
// when the wait timed out.
template <bool kHook>
__device__ __forceinline__ bool ring_take(Ring& r, const Tract& t, int64_t& issued, int64_t hq_end,
                                          int32_t (&p)[kLaneWords]) {
  if (!r.wait()) return false;
  const int4* e = reinterpret_cast<const int4*>(r.sm->ring[r.slot]) + (kLaneWords / 4) * lane_id();
#pragma unroll
  for (int i = 0; i < kLaneWords / 4; ++i) {
    const int4 a = e[i];
    p[4 * i] = a.x;
    p[4 * i + 1] = a.y;
    p[4 * i + 2] = a.z;
    p[4 * i + 3] = a.w;
  }
  // the piece is in registers: its slot takes the next one
  __syncwarp();
  if (issued < hq_end) {
    if (lane_id() == 0) {
      fence_proxy_async_smem();
      r.issue<kHook>(t, issued, r.slot);
    }
    ++issued;
  }
  r.advance();
  return true;
}

// Window loop of the TMA loader over the scan's vertex range.  Returns false
// when a wait timed out (the error is set and the ring may not be reused).
template <bool kSmem, bool kHook = false>
__device__ __forceinline__ bool scan_range_tma(Scan& sc, const VolView& v, const uint32_t* nw, const Tract& t,
                                               bool prefilter, WarpShared& ws, Ring& r, const SurvList& surv,
                                               DevState* gst) {
  // pieces wholly outside the vertex range (at the ends of the first and last
  // windows) are neither copied nor scanned
  const int64_t q0 = (int64_t)sc.V0 >> kWinLog2, q1 = (int64_t)(sc.V1 - 1) >> kWinLog2;
  const int64_t hq_lo = (int64_t)sc.V0 >> kPieceLog2, hq_end = ((int64_t)(sc.V1 - 1) >> kPieceLog2) + 1;
  int64_t taken = hq_lo;                           // pieces [hq_lo, taken) consumed
  int64_t issued = min(hq_end, hq_lo + kStages);   // pieces [taken, issued) in flight
  if (lane_id() == 0) {
    uint32_t k = r.slot;
    for (int64_t hq = hq_lo; hq < issued; ++hq) {
      r.issue<kHook>(t, hq, k);
      k = (k + 1 == (uint32_t)kStages) ? 0u : k + 1;
    }
  }
  __syncwarp();
  bool ok = true;
  for (int64_t q = q0; q <= q1 && !sc.abort && ok; ++q) {
    const int32_t W = (int32_t)(q << kWinLog2);
    int32_t nbw, b_first;
    window_begin(sc, ws, W, nbw, b_first);
    HitWord hh = 0u;
    const int h_lo = q == q0 ? (int)(hq_lo - q * kPieces) : 0;
    const int h_hi = q == q1 ? (int)(hq_end - q * kPieces) : kPieces;
#pragma unroll 1
    for (int h = h_lo; h < h_hi; ++h) {
      int32_t p[kLaneWords];
      if (!ring_take<kHook>(r, t, issued, hq_end, p)) {
        ok = false;
        break;
      }
      ++taken;
      hh |= (HitWord)scan_piece<kSmem>(sc, v, nw, p, h, W, ws) << (8 * h);
    }
    if (ok) window_end(sc, ws, W, nbw, b_first, hh, prefilter, surv, gst);
  }
  if (!ok) {
    if (lane_id() == 0) set_error(sc.sst, kErrTimeout, (int32_t)sc.s_lo);
    sc.abort = true;
    // the slot whose wait ran out is passed over (its copy, if one was ever
    // issued, is waited for no longer); the ring's phases are no longer
    // those of its slots, so the caller must not use it again
    r.advance();
    ++taken;
  }
  // no copy may be in flight when the range ends: bounded drain of the
  // pieces issued but not consumed, every one of them waited for even after
  // one wait has run out
  for (; taken < issued; ++taken) {
    if (!r.wait()) ok = false;
    r.advance();
  }
  return ok;
}

// Copy the near grid to shared memory (every thread of the CTA takes part).
__device__ __forceinline__ void stage_near(const VolView& v, uint32_t* s_near) {
  const int32_t n = (int32_t)near_words(v);
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) s_near[i] = __ldg(v.near + i);
  __syncthreads();
}

// Dynamic shared memory: [near grid (kSmem)] then, for the TMA loader, the
// warps' rings at a 128-byte aligned offset.
__host__ __device__ constexpr size_t ring_offset(size_t near_bytes) { return (near_bytes + 127) & ~(size_t)127; }

// kW warps per CTA, kMinBlocks CTAs per SM.  The default shape is one CTA of
// 16 warps per SM: with two CTAs of 8 on an SM (each warp the same share of
// the stream), the warp schedulers favoured the older CTA, which finished
// 15-18 % before the other, and the SM then ran the second one alone, on half
// its warps, for the end of the launch.
template <int kW, int kMinBlocks, bool kTma, bool kSmem, bool kHook>
__global__ void __launch_bounds__(kW * 32, kMinBlocks) prefilter_kernel(Tract t, VolView v, int prefilter,
                                                                       SurvList surv, DevState* st,
                                                                       int64_t withhold) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ WarpShared ws_all[kW];
  griddep_launch_dependents();  // the walk's CTAs may take SMs as this grid's CTAs end
  uint32_t* s_near = reinterpret_cast<uint32_t*>(smem_raw);
  if (kSmem) stage_near(v, s_near);
  const uint32_t* nw = kSmem ? s_near : v.near;
  WarpShared& ws = ws_all[threadIdx.x >> 5];
  const int64_t gw = (int64_t)blockIdx.x * kW + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * kW;
  int64_t s_lo, s_hi;
  vertex_split(t.off, t.ns, t.nv, gw, nwarps, s_lo, s_hi);
  Scan sc;
  if (!warp_init(t, s_lo, s_hi, sc, st, 0)) return;
  if (kTma) {
    const size_t off = ring_offset(kSmem ? (size_t)near_words(v) * 4 : 0);
    Ring r;
    r.init(reinterpret_cast<TmaSmem*>(smem_raw + off) + (threadIdx.x >> 5), withhold);
    scan_range_tma<kSmem, kHook>(sc, v, nw, t, prefilter != 0, ws, r, surv, st);
  } else {
    scan_range_direct<kSmem>(sc, v, nw, t, prefilter != 0, ws, surv, st);
  }
  warp_finish(sc, ws, surv, st);
}

// Batched form: warps take (subject, streamline range) tasks dynamically;
// the near grids stay in global memory (L1-cached).
template <int kMinBlocks, bool kTma>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
    prefilter_batch_kernel(const __grid_constant__ BatchTable tbl, const BatchTask* __restrict__ tasks,
                           int32_t ntasks, int prefilter, SurvList surv, DevState* gst) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ WarpShared ws_all[kWarps];
  WarpShared& ws = ws_all[threadIdx.x >> 5];
  Ring r;
  if (kTma) r.init(reinterpret_cast<TmaSmem*>(smem_raw) + (threadIdx.x >> 5));
  for (;;) {
    int32_t task = 0;
    if (lane_id() == 0) task = (int32_t)atomicAdd(&gst->work_task, 1u);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) break;
    const BatchTask tk = tasks ? tasks[task] : batch_task(tbl, task);
    const BatchSubject& S = tbl.s[tk.subject];
    Scan sc;
    if (!warp_init(S.t, tk.s_lo, tk.s_hi, sc, S.st, S.sbase)) continue;
    bool ring_ok = true;
    if (kTma)
      ring_ok = scan_range_tma<false>(sc, S.v, S.v.near, S.t, prefilter != 0, ws, r, surv, gst);
    else
      scan_range_direct<false>(sc, S.v, S.v.near, S.t, prefilter != 0, ws, surv, gst);
    warp_finish(sc, ws, surv, gst);
    if (!ring_ok) break;  // a copy may still be in flight: this warp takes no more tasks
  }
}

constexpr size_t kRingBytes = sizeof(TmaSmem) * kWarps;

// Grid = every CTA resident at once (one wave), from the occupancy the
// compiled kernel really reaches.
template <typename K>
cudaError_t resident_grid(K kernel, int threads, size_t smem, int num_sms, int* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  *grid = num_sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int kW, int kMinBlocks, bool kTma, bool kSmem>
cudaError_t launch_plain(const Tract& t, const VolView& v, bool prefilter, const SurvList& survivors, DevState* st,
                         int num_sms, cudaStream_t s, int64_t withhold) {
  // the test hook has builds of its own, so that the default one carries no
  // trace of it
  auto k = (kTma && withhold >= 0) ? prefilter_kernel<kW, kMinBlocks, kTma, kSmem, kTma>
                                   : prefilter_kernel<kW, kMinBlocks, kTma, kSmem, false>;
  const size_t near_bytes = kSmem ? (size_t)near_words(v) * 4 : 0;
  const size_t bytes = kTma ? ring_offset(near_bytes) + sizeof(TmaSmem) * kW : near_bytes;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  int grid = 0;
  if (e == cudaSuccess) e = resident_grid(k, kW * 32, bytes, num_sms, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, kW * 32, bytes, s>>>(t, v, prefilter ? 1 : 0, survivors, st, withhold);
  return cudaGetLastError();
}

// Near grids up to this many words are staged in shared memory beside the
// rings of the SM's warps.
constexpr int64_t kNearSmemWordsTma = 8192;

template <int kW, int kMinBlocks>
cudaError_t launch_one(const Tract& t, const VolView& v, bool prefilter, bool tma, const SurvList& survivors,
                       DevState* st, int num_sms, cudaStream_t s, int64_t wh) {
  const int64_t nw = near_words(v);
  if (tma) {
    if (nw <= kNearSmemWordsTma)
      return launch_plain<kW, kMinBlocks, true, true>(t, v, prefilter, survivors, st, num_sms, s, wh);
    return launch_plain<kW, kMinBlocks, true, false>(t, v, prefilter, survivors, st, num_sms, s, wh);
  }
  if (nw <= kNearSmemWords)
    return launch_plain<kW, kMinBlocks, false, true>(t, v, prefilter, survivors, st, num_sms, s, wh);
  return launch_plain<kW, kMinBlocks, false, false>(t, v, prefilter, survivors, st, num_sms, s, wh);
}

template <int kMinBlocks, bool kTma>
cudaError_t launch_batch_one(const BatchTable& tbl, const BatchTask* tasks, int32_t ntasks, bool prefilter,
                             const SurvList& survivors, DevState* gst, int num_sms, cudaStream_t s) {
  auto k = prefilter_batch_kernel<kMinBlocks, kTma>;
  const size_t bytes = kTma ? kRingBytes : 0;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  int grid = 0;
  if (e == cudaSuccess) e = resident_grid(k, kWarps * 32, bytes, num_sms, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, kWarps * 32, bytes, s>>>(tbl, tasks, ntasks, prefilter ? 1 : 0, survivors, gst);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prefilter_batch(const BatchTable& tbl, const BatchTask* tasks, int32_t ntasks, bool prefilter,
                                   bool tma, int ctas_per_sm, int32_t* survivor_ids, int64_t survivor_cap,
                                   DevState* gst, int num_sms, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const SurvList survivors{survivor_ids, survivor_cap};
  if (tma) {
    if (ctas_per_sm >= 3) return launch_batch_one<3, true>(tbl, tasks, ntasks, prefilter, survivors, gst, num_sms, s);
    return launch_batch_one<2, true>(tbl, tasks, ntasks, prefilter, survivors, gst, num_sms, s);
  }
  if (ctas_per_sm >= 3) return launch_batch_one<3, false>(tbl, tasks, ntasks, prefilter, survivors, gst, num_sms, s);
  return launch_batch_one<2, false>(tbl, tasks, ntasks, prefilter, survivors, gst, num_sms, s);
}

cudaError_t launch_prefilter(const Tract& t, const VolView& v, bool prefilter, uint32_t mode, bool tma,
                             int ctas_per_sm, int32_t* survivor_ids, int64_t survivor_cap, DevState* st, int num_sms,
                             cudaStream_t s, int64_t withhold_piece) {
  (void)mode;  // the segment and the vertex-only rules share the near test; the walk applies the rule
  if (t.ns <= 0) return cudaSuccess;
  const SurvList survivors{survivor_ids, survivor_cap};
  // the register budget of two 8-warp CTAs per SM as one CTA of 16 warps;
  // that of three (80 registers) as three CTAs of 8
  if (ctas_per_sm >= 3) return launch_one<8, 3>(t, v, prefilter, tma, survivors, st, num_sms, s, withhold_piece);
  return launch_one<16, 1>(t, v, prefilter, tma, survivors, st, num_sms, s, withhold_piece);
}

}  // namespace fc
