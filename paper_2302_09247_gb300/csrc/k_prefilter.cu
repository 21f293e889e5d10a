// K2: prefilter + compaction over the full vertex stream.
//
// Every streamline is read once.  A streamline that passes near no ROI voxel
// or near no labelled voxel can contribute neither to C nor to C_end (whose
// seed and endpoint lie on the streamline) and is dropped; the ids of the
// others are appended to a compact survivor list (one atomic per 32 survivors
// of a warp).  The test is conservative; the walk decides exactly.  On the way
// the kernel validates coordinates and counts voxel-steps.
//
// The test.  The near grid holds, for every voxel, whether an ROI voxel / a
// labelled voxel lies within Chebyshev distance 1.  A segment whose end
// voxels differ by at most one on every axis lies in the 3x3x3 block around
// its end voxel, so the near bits of that voxel cover the segment; over a
// streamline, the OR of the near bits of its vertices covers all of its
// segments (and its single point when T = 1).  A longer segment adds the
// brick occupancy of its whole voxel box (exact, rare).
//
// Vertex-parallel scan.  Each warp owns a contiguous range of streamlines and
// walks its vertex range in 128-vertex windows aligned to 128; lane l takes
// the four consecutive vertices 4l..4l+3 of the window, so every lane is busy
// regardless of streamline boundaries:
//   - boundaries (streamline starts, from the offsets) falling in the window
//     are scanned first, 32 at a time, into a start mask;
//   - per vertex: one near-grid lookup, the voxel-step count of the segment
//     ending there (unless it starts a streamline), the long-segment check;
//   - ballots turn the bits into four per-slot window masks; at every
//     boundary x, a prefix popcount of the masks gives the running count of
//     ROI / target hits, and the streamline ending at x passes when both
//     counts grew since its start boundary.
// Two loaders with identical results: direct vectorised streaming loads
// (default: 3 x 16-byte loads per lane per window) and TMA (the warp streams
// its vertex range through a 4-deep ring of 1536-byte pieces, one window each,
// in shared memory with cp.async.bulk + mbarrier, L2 evict-first).
#include "fc_device.cuh"
#include "fc_tma.cuh"

namespace fc {

namespace {

constexpr int kPieceV = 128;              // vertices per piece = per window
constexpr int kPieceLog2 = 7;
constexpr int kPieceWords = kPieceV * 3;  // 384 int32 = 1536 bytes
constexpr int kStages = 4;                // ring depth per warp
constexpr int kWarps = 8;                 // warps per CTA
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;  // 1 s
constexpr int32_t kInf = 0x7fffffff;

__device__ __forceinline__ uint32_t lowmask(int32_t k) { return k >= 32 ? 0xffffffffu : ((1u << k) - 1u); }

// Near bits of voxel (x, y, z); 0 when the voxel is more than one voxel
// outside the grid.
__device__ __forceinline__ uint32_t near_bits(const VolView& v, int32_t x, int32_t y, int32_t z) {
  const int32_t px = x + 1, py = y + 1, pz = z + 1;
  if ((unsigned)px >= (unsigned)(v.dx + 2) || (unsigned)py >= (unsigned)(v.dy + 2) || (unsigned)pz >= (unsigned)(v.dz + 2))
    return 0u;
  const int32_t cx = px >> v.nsh, cy = py >> v.nsh, cz = pz >> v.nsh;
  const int32_t w = (cx >> 4) + v.nwx * (cy + v.nny * cz);
  return (__ldg(v.near + w) >> ((cx & 15) << 1)) & 3u;
}

// Count of set bits of the four slot masks (vertex 4l+k = bit l of mask k)
// at window positions below x, x in [0, 128].
__device__ __forceinline__ uint32_t prefix4(const uint32_t m[4], int32_t x) {
  const int32_t l = x >> 2, k = x & 3;
  const uint32_t lm = lowmask(l);
  uint32_t c = __popc(m[0] & lm) + __popc(m[1] & lm) + __popc(m[2] & lm) + __popc(m[3] & lm);
  if (k > 0) c += (m[0] >> l) & 1u;
  if (k > 1) c += (m[1] >> l) & 1u;
  if (k > 2) c += (m[2] >> l) & 1u;
  return c;
}

struct WarpSmem {
  int32_t ring[kStages][kPieceWords];
  uint64_t bar[kStages];
  int32_t sbuf[64];
};

// Per-warp scan state (registers).  Vertex indices are relative to V0.
struct Scan {
  int64_t V0;
  int32_t len;              // V1 - V0
  const int64_t* off;
  int64_t s_cur, s_hi;      // next boundary to scan: off[s_cur], s_cur <= s_hi
  uint32_t cumR, cumT;      // hit counts before the current window
  uint32_t lastR, lastT;    // hit counts at the last boundary
  int32_t last_x;           // position of the last boundary
  uint32_t start_carry;     // the next window's vertex 0 starts a streamline
  int32_t qx, qy, qz;       // voxel of the previous window's last vertex
  uint32_t steps;           // voxel steps counted by this lane (flushed to steps64)
  unsigned long long steps64;
  uint32_t singles, kept;
  int nbuf;
  bool bad;
  int64_t id_base;          // survivor ids are id_base + streamline index
  DevState* sst;            // the subject's counters and error word
};

// gst holds the survivor list's counter (one list per launch).
__device__ __forceinline__ void flush_survivors(Scan& sc, int32_t* sbuf, int32_t* surv, DevState* gst) {
  __syncwarp();
  uint32_t base = 0;
  if (lane_id() == 0 && sc.nbuf > 0) base = atomicAdd(&gst->n_survivors, (uint32_t)sc.nbuf);
  base = __shfl_sync(kFull, base, 0);
  const int l = (int)lane_id();
  if (l < sc.nbuf) surv[base + l] = sbuf[l];
  if (l + 32 < sc.nbuf) surv[base + l + 32] = sbuf[l + 32];
  __syncwarp();
  sc.nbuf = 0;
}

// One window at relative position Wr (the window's first vertex minus V0).
// p: the lane's 12 words = vertices 4l..4l+3 of the window (meaningful where
// inside [0, len)).
__device__ __forceinline__ void scan_window(Scan& sc, const VolView& v, int32_t Wr, const int32_t p[12],
                                            bool prefilter, int32_t* sbuf, int32_t* surv, DevState* gst) {
  const int32_t lane = (int32_t)lane_id();

  // 1. boundaries x <= Wr + 128, 32 per round: start mask of this window
  uint32_t sm[4] = {0u, 0u, 0u, 0u};
  if (sc.start_carry) sm[0] |= 1u;
  {
    const int32_t x0 = -Wr;  // V0 starts the first streamline of the range
    if (x0 >= 0 && x0 < 128) sm[x0 & 3] |= 1u << (x0 >> 2);
  }
  int64_t s_round = sc.s_cur;
  int32_t bx;  // this lane's boundary of the current round
  int32_t nb;
  {
    const int64_t s = sc.s_cur + lane;
    bx = s <= sc.s_hi ? (int32_t)(sc.off[s] - sc.V0) : kInf;
    nb = __popc(__ballot_sync(kFull, bx <= Wr + 128));
    const int32_t r = bx - Wr;
    const bool st_in = bx <= Wr + 128 && r < 128;
#pragma unroll
    for (int k = 0; k < 4; ++k) sm[k] |= __reduce_or_sync(kFull, (st_in && (r & 3) == k) ? (1u << (r >> 2)) : 0u);
    if (nb == 32) {
      // more than 32 boundaries in one window: collect the rest of the starts
      int64_t s2 = sc.s_cur + 32;
      for (;;) {
        const int64_t t = s2 + lane;
        const int32_t b2 = t <= sc.s_hi ? (int32_t)(sc.off[t] - sc.V0) : kInf;
        const int32_t n2 = __popc(__ballot_sync(kFull, b2 <= Wr + 128));
        const int32_t r2 = b2 - Wr;
        const bool in2 = b2 <= Wr + 128 && r2 < 128;
#pragma unroll
        for (int k = 0; k < 4; ++k) sm[k] |= __reduce_or_sync(kFull, (in2 && (r2 & 3) == k) ? (1u << (r2 >> 2)) : 0u);
        if (n2 < 32) break;
        s2 += 32;
      }
    }
  }

  // 2. vertices
  uint32_t mr[4], mt[4];
  uint32_t badacc = 0;
  {
    int32_t qx = __shfl_up_sync(kFull, p[9] >> kUnitLog2, 1);
    int32_t qy = __shfl_up_sync(kFull, p[10] >> kUnitLog2, 1);
    int32_t qz = __shfl_up_sync(kFull, p[11] >> kUnitLog2, 1);
    if (lane == 0) { qx = sc.qx; qy = sc.qy; qz = sc.qz; }
    sc.qx = __shfl_sync(kFull, p[9] >> kUnitLog2, 31);
    sc.qy = __shfl_sync(kFull, p[10] >> kUnitLog2, 31);
    sc.qz = __shfl_sync(kFull, p[11] >> kUnitLog2, 31);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int32_t jr = Wr + 4 * lane + k;
      const bool act = jr >= 0 && jr < sc.len;
      const int32_t x = p[3 * k], y = p[3 * k + 1], z = p[3 * k + 2];
      const int32_t vx = x >> kUnitLog2, vy = y >> kUnitLog2, vz = z >> kUnitLog2;
      if (act) badacc |= (uint32_t)(x + kCoordLimit) | (uint32_t)(y + kCoordLimit) | (uint32_t)(z + kCoordLimit);
      uint32_t D = act ? near_bits(v, vx, vy, vz) : 0u;
      const int32_t ax = abs(vx - qx), ay = abs(vy - qy), az = abs(vz - qz);
      const bool start = (sm[k] >> lane) & 1u;
      if (act && !start) sc.steps += 1u + (uint32_t)(ax + ay + az);
      if (act && !start && (uint32_t)(ax | ay | az) > 1u)
        D |= box_bits(v, min(vx, qx), min(vy, qy), min(vz, qz), max(vx, qx), max(vy, qy), max(vz, qz));
      mr[k] = __ballot_sync(kFull, D & 1u);
      mt[k] = __ballot_sync(kFull, D & 2u);
      qx = vx;
      qy = vy;
      qz = vz;
    }
  }
  sc.bad |= __any_sync(kFull, (badacc >> 25) != 0u);

  // 3. decisions at the boundaries of this window
  while (nb > 0) {
    const bool in = lane < nb;
    uint32_t cR = 0, cT = 0;
    if (in) {
      const int32_t r = bx - Wr;
      cR = sc.cumR + prefix4(mr, r);
      cT = sc.cumT + prefix4(mt, r);
    }
    uint32_t pR = __shfl_up_sync(kFull, cR, 1), pT = __shfl_up_sync(kFull, cT, 1);
    int32_t px = __shfl_up_sync(kFull, bx, 1);
    if (lane == 0) { pR = sc.lastR; pT = sc.lastT; px = sc.last_x; }
    // boundary s closes streamline s-1 = [px, bx)
    const bool pass = in && (!prefilter || (cR > pR && cT > pT)) && (bx > px) && !sc.bad;
    if (in && bx - px == 1) sc.singles += 1u;
    const uint32_t pm = __ballot_sync(kFull, pass);
    if (pass) sbuf[sc.nbuf + __popc(pm & lanemask_lt())] = (int32_t)(sc.id_base + s_round + lane - 1);
    sc.nbuf += __popc(pm);
    sc.kept += __popc(pm);
    if (sc.nbuf >= 32) flush_survivors(sc, sbuf, surv, gst);
    sc.lastR = __shfl_sync(kFull, cR, nb - 1);
    sc.lastT = __shfl_sync(kFull, cT, nb - 1);
    sc.last_x = __shfl_sync(kFull, bx, nb - 1);
    s_round += nb;
    if (nb < 32) break;
    const int64_t s = s_round + lane;
    bx = s <= sc.s_hi ? (int32_t)(sc.off[s] - sc.V0) : kInf;
    nb = __popc(__ballot_sync(kFull, bx <= Wr + 128));
  }
  sc.s_cur = s_round;
  sc.start_carry = (sc.last_x == Wr + 128) ? 1u : 0u;
  sc.cumR += __popc(mr[0]) + __popc(mr[1]) + __popc(mr[2]) + __popc(mr[3]);
  sc.cumT += __popc(mt[0]) + __popc(mt[1]) + __popc(mt[2]) + __popc(mt[3]);
}

// Set up the scan of streamlines [s_lo, s_hi) of t after validating their
// offsets; false when there is nothing to do (or the offsets are invalid).
__device__ __forceinline__ bool warp_init(const Tract& t, int64_t s_lo, int64_t s_hi, Scan& sc, DevState* sst,
                                          int64_t id_base) {
  const unsigned lane = lane_id();
  if (s_lo == 0 && lane == 0 && (t.off[0] != 0 || t.off[t.ns] != t.nv)) set_error(sst, kErrOffsets, -1);
  bool ok = true;
  for (int64_t s = s_lo + lane; s < s_hi; s += 32) {
    const int64_t a = t.off[s], b = t.off[s + 1];
    ok &= (a >= 0) && (a <= b) && (b <= t.nv);
  }
  if (!__all_sync(kFull, ok)) {
    if (lane == 0) set_error(sst, kErrOffsets, (int32_t)s_lo);
    return false;
  }
  if (s_hi <= s_lo) return false;
  const int64_t V0 = t.off[s_lo], V1 = t.off[s_hi];
  if (V1 <= V0) return false;
  sc.V0 = V0;
  sc.len = (int32_t)(V1 - V0);
  sc.off = t.off;
  sc.s_cur = s_lo + 1;
  sc.s_hi = s_hi;
  sc.cumR = sc.cumT = 0;
  sc.lastR = sc.lastT = 0;
  sc.last_x = 0;
  sc.start_carry = 0;
  sc.qx = sc.qy = sc.qz = 0;
  sc.steps = 0;
  sc.steps64 = 0;
  sc.singles = sc.kept = 0;
  sc.nbuf = 0;
  sc.bad = false;
  sc.id_base = id_base;
  sc.sst = sst;
  return true;
}

__device__ __forceinline__ void warp_finish(Scan& sc, int32_t* sbuf, int32_t* surv, DevState* gst) {
  flush_survivors(sc, sbuf, surv, gst);
  unsigned long long s = sc.steps64 + sc.steps + sc.singles;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if (lane_id() == 0) {
    atomicAdd(&sc.sst->voxel_steps, s);
    atomicAdd(&sc.sst->survivors, (unsigned long long)sc.kept);
    if (sc.bad) set_error(sc.sst, kErrCoord, (int32_t)(sc.s_cur - 1));
  }
}

__device__ __forceinline__ void ldcs4(const int32_t* g, int32_t* d) {
  const int4 a = __ldcs(reinterpret_cast<const int4*>(g));
  d[0] = a.x;
  d[1] = a.y;
  d[2] = a.z;
  d[3] = a.w;
}

// ------------------------------------------------------------------ direct

// Window loop of the direct loader over the scan's vertex range.
__device__ __forceinline__ void scan_range_direct(Scan& sc, const VolView& v, const Tract& t, bool prefilter,
                                                  int32_t* sbuf, int32_t* surv, DevState* gst) {
  const int32_t lane = (int32_t)lane_id();
  const int64_t q0 = sc.V0 >> kPieceLog2, q1 = (sc.V0 + sc.len - 1) >> kPieceLog2;
  for (int64_t q = q0; q <= q1; ++q) {
    const int64_t g = (q << kPieceLog2) + 4 * lane;  // absolute index of the lane's first vertex
    int32_t p[12];
    if (g + 3 < t.nv) {
      const int32_t* e = t.xyz + 3 * g;  // 48-byte chunk, 16-byte aligned
      ldcs4(e, p);
      ldcs4(e + 4, p + 4);
      ldcs4(e + 8, p + 8);
    } else {
#pragma unroll
      for (int w = 0; w < 12; ++w) p[w] = (g + w / 3 < t.nv) ? __ldcs(t.xyz + 3 * g + w) : 0;
    }
    scan_window(sc, v, (int32_t)((q << kPieceLog2) - sc.V0), p, prefilter, sbuf, surv, gst);
    sc.steps64 += sc.steps;
    sc.steps = 0;
  }
}

template <int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) prefilter_direct_kernel(Tract t, VolView v, int prefilter,
                                                                                  int32_t* surv, DevState* st) {
  __shared__ int32_t sbuf_all[kWarps][64];
  int32_t* sbuf = sbuf_all[threadIdx.x >> 5];
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  Scan sc;
  if (!warp_init(t, t.ns * gw / nw, t.ns * (gw + 1) / nw, sc, st, 0)) return;
  scan_range_direct(sc, v, t, prefilter != 0, sbuf, surv, st);
  warp_finish(sc, sbuf, surv, st);
}

// Batched form: warps take (subject, streamline range) tasks dynamically.
template <int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
    prefilter_batch_kernel(const __grid_constant__ BatchTable tbl, const BatchTask* __restrict__ tasks,
                           int32_t ntasks, int prefilter, int32_t* surv, DevState* gst) {
  __shared__ int32_t sbuf_all[kWarps][64];
  int32_t* sbuf = sbuf_all[threadIdx.x >> 5];
  for (;;) {
    int32_t task = 0;
    if (lane_id() == 0) task = (int32_t)atomicAdd(&gst->work_task, 1u);
    task = __shfl_sync(kFull, task, 0);
    if (task >= ntasks) break;
    const BatchTask tk = tasks[task];
    const BatchSubject& S = tbl.s[tk.subject];
    Scan sc;
    if (!warp_init(S.t, tk.s_lo, tk.s_hi, sc, S.st, S.sbase)) continue;
    scan_range_direct(sc, S.v, S.t, prefilter != 0, sbuf, surv, gst);
    warp_finish(sc, sbuf, surv, gst);
  }
}

// --------------------------------------------------------------------- tma

struct Ring {
  WarpSmem* sm;
  const int32_t* xyz;
  int64_t nv;
  int64_t p_first, p_last, next_issue;
  uint64_t policy;

  // lane 0 only: bulk-copy piece q into its slot (the part of the array's
  // tail that is not a multiple of 16 bytes is copied with plain loads)
  __device__ __forceinline__ void issue(int64_t q) {
    const int k = (int)((q - p_first) & (kStages - 1));
    const int64_t v0 = q << kPieceLog2;
    const int64_t n = min((int64_t)kPieceV, nv - v0);
    const uint32_t bytes = (uint32_t)(n * 12);
    const uint32_t tma = bytes & ~15u;
    int32_t* dst = sm->ring[k];
    const int32_t* src = xyz + 3 * v0;
    if (tma) {
      mbar_arrive_expect_tx(&sm->bar[k], tma);
      bulk_g2s(dst, src, tma, &sm->bar[k], policy);
    } else {
      mbar_arrive(&sm->bar[k]);
    }
    for (uint32_t w = tma >> 2; w < (bytes >> 2); ++w) dst[w] = __ldcs(src + w);
  }

  // Every lane waits (acquiring the bytes); the result is warp-uniform.
  __device__ __forceinline__ bool wait(int64_t q) {
    const int k = (int)((q - p_first) & (kStages - 1));
    const uint32_t parity = (uint32_t)(((q - p_first) >> 2) & 1);
    return __all_sync(kFull, mbar_wait_bounded(&sm->bar[k], parity, kWaitTimeoutNs));
  }
};

template <int kMinBlocks>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) prefilter_tma_kernel(Tract t, VolView v, int prefilter,
                                                                               int32_t* surv, DevState* st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  WarpSmem* sm = reinterpret_cast<WarpSmem*>(smem_raw) + (threadIdx.x >> 5);
  const int32_t lane = (int32_t)lane_id();
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  Scan sc;
  if (!warp_init(t, t.ns * gw / nw, t.ns * (gw + 1) / nw, sc, st, 0)) return;

  Ring r;
  r.sm = sm;
  r.xyz = t.xyz;
  r.nv = t.nv;
  r.p_first = sc.V0 >> kPieceLog2;
  r.p_last = (sc.V0 + sc.len - 1) >> kPieceLog2;
  r.next_issue = min(r.p_last + 1, r.p_first + kStages);
  r.policy = policy_evict_first();
  if (lane == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(&sm->bar[k], 1);
    fence_mbar_init();
    for (int64_t q = r.p_first; q < r.next_issue; ++q) r.issue(q);
  }
  __syncwarp();

  bool timed_out = false;
  int64_t waited = r.p_first - 1;
  for (int64_t q = r.p_first; q <= r.p_last; ++q) {
    if (q > r.p_first) {
      // piece q-1 is consumed: refill its slot with piece q-1+kStages
      __syncwarp();
      if (lane == 0 && r.next_issue <= r.p_last) {
        fence_proxy_async_smem();
        r.issue(r.next_issue);
      }
      if (r.next_issue <= r.p_last) ++r.next_issue;
    }
    if (!r.wait(q)) {
      timed_out = true;
      break;
    }
    waited = q;
    const int4* e = reinterpret_cast<const int4*>(sm->ring[(q - r.p_first) & (kStages - 1)]) + 3 * lane;
    int32_t p[12];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int4 a = e[i];
      p[4 * i] = a.x;
      p[4 * i + 1] = a.y;
      p[4 * i + 2] = a.z;
      p[4 * i + 3] = a.w;
    }
    scan_window(sc, v, (int32_t)((q << kPieceLog2) - sc.V0), p, prefilter != 0, sm->sbuf, surv, st);
    sc.steps64 += sc.steps;
    sc.steps = 0;
  }
  if (timed_out) {
    if (lane == 0) set_error(st, kErrTimeout, (int32_t)gw);
    // no copy may be in flight when the warp leaves: bounded drain
    for (int64_t q = waited + 1; q < r.next_issue; ++q)
      if (!r.wait(q)) break;
  }
  warp_finish(sc, sm->sbuf, surv, st);
}

constexpr size_t kTmaSmemBytes = sizeof(WarpSmem) * kWarps;

// Grid = every CTA resident at once (one wave), from the occupancy the
// compiled kernel really reaches.
template <typename K>
cudaError_t resident_grid(K kernel, size_t smem, int num_sms, int* grid) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  *grid = num_sms * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int kMinBlocks>
cudaError_t launch_one(const Tract& t, const VolView& v, bool prefilter, bool tma, int32_t* survivors,
                       DevState* st, int num_sms, cudaStream_t s) {
  int grid = 0;
  if (tma) {
    auto k = prefilter_tma_kernel<kMinBlocks>;
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmemBytes);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    cudaError_t e = resident_grid(k, kTmaSmemBytes, num_sms, &grid);
    if (e != cudaSuccess) return e;
    k<<<grid, kWarps * 32, kTmaSmemBytes, s>>>(t, v, prefilter ? 1 : 0, survivors, st);
  } else {
    auto k = prefilter_direct_kernel<kMinBlocks>;
    cudaError_t e = resident_grid(k, 0, num_sms, &grid);
    if (e != cudaSuccess) return e;
    k<<<grid, kWarps * 32, 0, s>>>(t, v, prefilter ? 1 : 0, survivors, st);
  }
  return cudaGetLastError();
}

template <int kMinBlocks>
cudaError_t launch_batch_one(const BatchTable& tbl, const BatchTask* tasks, int32_t ntasks, bool prefilter,
                             int32_t* survivors, DevState* gst, int num_sms, cudaStream_t s) {
  auto k = prefilter_batch_kernel<kMinBlocks>;
  int grid = 0;
  cudaError_t e = resident_grid(k, 0, num_sms, &grid);
  if (e != cudaSuccess) return e;
  k<<<grid, kWarps * 32, 0, s>>>(tbl, tasks, ntasks, prefilter ? 1 : 0, survivors, gst);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prefilter_batch(const BatchTable& tbl, const BatchTask* tasks, int32_t ntasks, bool prefilter,
                                   int ctas_per_sm, int32_t* survivors, DevState* gst, int num_sms, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (ctas_per_sm == 4) return launch_batch_one<4>(tbl, tasks, ntasks, prefilter, survivors, gst, num_sms, s);
  return launch_batch_one<3>(tbl, tasks, ntasks, prefilter, survivors, gst, num_sms, s);
}

cudaError_t launch_prefilter(const Tract& t, const VolView& v, bool prefilter, uint32_t mode, bool tma,
                             int ctas_per_sm, int32_t* survivors, DevState* st, int num_sms, cudaStream_t s) {
  (void)mode;  // the segment and the vertex-only rules share the near test; the walk applies the rule
  if (t.ns <= 0) return cudaSuccess;
  if (ctas_per_sm == 3) return launch_one<3>(t, v, prefilter, tma, survivors, st, num_sms, s);
  return launch_one<4>(t, v, prefilter, tma, survivors, st, num_sms, s);
}

}  // namespace fc
