// K2: prefilter + compaction over the full vertex stream.
//
// Every streamline is read once.  Per segment the kernel validates the
// coordinates, adds 1 + sum_a |dfloor_a| to the voxel-step count, and ORs
// the brick occupancy bits of the segment's voxel box.  A streamline whose
// boxes touch no ROI brick or no target brick cannot contribute to C (nor to
// C_end, whose seed and endpoint lie on the streamline) and is dropped; the
// ids of the others are appended to a compact survivor list with one atomic
// per 32 survivors of a warp.  The test is conservative, never exact: the
// walk decides.
//
// Two loaders with identical results:
//   - direct: warp per streamline, coalesced streaming loads;
//   - tma (default): each warp owns a contiguous range of streamlines and
//     streams its vertex range through a 4-deep ring of 1536-byte pieces in
//     shared memory with 1-D bulk copies (cp.async.bulk) completing on
//     per-slot mbarriers, with an L2 evict-first hint.
#include "fc_device.cuh"
#include "fc_tma.cuh"

namespace fc {

// Evaluate one unit of a streamline: segment (p0, p1), or the point p0 when
// point_mode.  has_next: p1 is the next vertex of the same streamline.
__device__ __forceinline__ void eval_unit(const VolView& v, const int32_t p0[3], const int32_t p1[3],
                                          bool has_next, bool single, bool point_mode,
                                          unsigned long long& steps, uint32_t& bits, bool& bad) {
  bad |= !(coord_ok(p0[0]) && coord_ok(p0[1]) && coord_ok(p0[2]) && coord_ok(p1[0]) && coord_ok(p1[1]) &&
           coord_ok(p1[2]));
  const int32_t ax = p0[0] >> kUnitLog2, ay = p0[1] >> kUnitLog2, az = p0[2] >> kUnitLog2;
  const int32_t bx = p1[0] >> kUnitLog2, by = p1[1] >> kUnitLog2, bz = p1[2] >> kUnitLog2;
  if (single)
    steps += 1;
  else if (has_next)
    steps += 1 + (unsigned)(abs(bx - ax) + abs(by - ay) + abs(bz - az));
  if (point_mode)
    bits |= box_bits(v, ax, ay, az, ax, ay, az);
  else
    bits |= box_bits(v, min(ax, bx), min(ay, by), min(az, bz), max(ax, bx), max(ay, by), max(az, bz));
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Append the warp's buffered survivors to the global list.
__device__ __forceinline__ void flush_survivors(int32_t* sbuf, int& nbuf, int32_t* surv, DevState* st) {
  __syncwarp();
  uint32_t base = 0;
  if (lane_id() == 0 && nbuf > 0) base = atomicAdd(&st->n_survivors, (uint32_t)nbuf);
  base = __shfl_sync(kFull, base, 0);
  if ((int)lane_id() < nbuf) surv[base + lane_id()] = sbuf[lane_id()];
  __syncwarp();
  nbuf = 0;
}

// ------------------------------------------------------------------ direct

constexpr int kDirWarps = 8;

__global__ void __launch_bounds__(kDirWarps * 32) prefilter_direct_kernel(Tract t, VolView v, int prefilter,
                                                                         uint32_t mode, int32_t* surv,
                                                                         DevState* st) {
  __shared__ int32_t sbuf_all[kDirWarps][32];
  int32_t* sbuf = sbuf_all[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  const int64_t gw = (int64_t)blockIdx.x * kDirWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kDirWarps;
  if (gw == 0 && lane == 0 && (t.off[0] != 0 || t.off[t.ns] != t.nv)) set_error(st, kErrOffsets, -1);
  const bool point_mode = (mode & kModeVertexSampled) != 0;
  unsigned long long steps = 0, kept = 0;
  int nbuf = 0;
  for (int64_t s = gw; s < t.ns; s += nw) {
    const int64_t a = t.off[s], b = t.off[s + 1];
    if (a < 0 || b < a || b > t.nv) {
      if (lane == 0) set_error(st, kErrOffsets, (int32_t)s);
      continue;
    }
    const int64_t T = b - a;
    if (T == 0) continue;
    const bool single = T == 1;
    const int64_t units = (single || point_mode) ? T : T - 1;
    uint32_t bits = 0;
    bool bad = false;
    for (int64_t i0 = 0; i0 < units; i0 += 32) {
      const int64_t j = a + i0 + lane;
      const int64_t jhi = min(a + i0 + 32, b - 1);  // last vertex the window needs
      int32_t p0[3] = {0, 0, 0}, p1[3];
      if (j <= jhi) {
        p0[0] = __ldcs(t.xyz + 3 * j);
        p0[1] = __ldcs(t.xyz + 3 * j + 1);
        p0[2] = __ldcs(t.xyz + 3 * j + 2);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) p1[k] = __shfl_down_sync(kFull, p0[k], 1);
      if (lane == 31 && j + 1 <= jhi) {
        p1[0] = __ldcs(t.xyz + 3 * (j + 1));
        p1[1] = __ldcs(t.xyz + 3 * (j + 1) + 1);
        p1[2] = __ldcs(t.xyz + 3 * (j + 1) + 2);
      }
      if (i0 + lane < units) {
        const bool has_next = j + 1 < b;
        if (!has_next) { p1[0] = p0[0]; p1[1] = p0[1]; p1[2] = p0[2]; }
        eval_unit(v, p0, p1, has_next, single, single || point_mode, steps, bits, bad);
      }
    }
    bits = __reduce_or_sync(kFull, bits);
    if (__any_sync(kFull, bad)) {
      if (lane == 0) set_error(st, kErrCoord, (int32_t)s);
      continue;
    }
    if (!prefilter || bits == 3u) {
      if (lane == 0) sbuf[nbuf] = (int32_t)s;
      ++kept;
      if (++nbuf == 32) flush_survivors(sbuf, nbuf, surv, st);
    }
  }
  flush_survivors(sbuf, nbuf, surv, st);
  steps = warp_sum_u64(steps);
  if (lane == 0) {
    atomicAdd(&st->voxel_steps, steps);
    atomicAdd(&st->survivors, kept);
  }
}

// --------------------------------------------------------------------- tma

constexpr int kPieceV = 128;                 // vertices per piece
constexpr int kPieceLog2 = 7;
constexpr int kPieceWords = kPieceV * 3;     // 384 int32 = 1536 bytes
constexpr int kStages = 4;                   // ring depth per warp
constexpr int kTmaWarps = 8;
constexpr uint64_t kWaitTimeoutNs = 1000000000ull;  // 1 s

struct __align__(16) PfWarpSmem {
  int32_t ring[kStages][kPieceWords];
  uint64_t bar[kStages];
  int32_t sbuf[32];
};

constexpr size_t kTmaSmemBytes = sizeof(PfWarpSmem) * kTmaWarps;

struct Ring {
  PfWarpSmem* sm;
  const int32_t* xyz;
  int64_t nv;
  int64_t p_first, p_last;
  int64_t next_issue, next_rel, waited;
  uint64_t policy;

  // lane 0 only: bulk-copy piece q into its slot (the tail of the array that
  // is not a multiple of 16 bytes is copied with plain loads)
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

  // Every lane waits (acquiring the copied bytes); the result is made
  // warp-uniform so that a timeout cannot split the warp.
  __device__ __forceinline__ bool wait_piece(int64_t q) {
    const int k = (int)((q - p_first) & (kStages - 1));
    const uint32_t parity = (uint32_t)(((q - p_first) / kStages) & 1);
    return __all_sync(kFull, mbar_wait_bounded(&sm->bar[k], parity, kWaitTimeoutNs));
  }

  // Make vertices [jlo, jhi] resident (jlo non-decreasing across calls).
  __device__ __forceinline__ bool ensure(int64_t jlo, int64_t jhi) {
    const int64_t qlo = jlo >> kPieceLog2, qhi = jhi >> kPieceLog2;
    while (waited < qlo - 1) {
      if (!wait_piece(waited + 1)) return false;
      ++waited;
    }
    if (next_rel < qlo) {
      __syncwarp();
      if (lane_id() == 0) {
        fence_proxy_async_smem();
        for (int64_t q = next_rel; q < qlo; ++q)
          if (next_issue + (q - next_rel) <= p_last) issue(next_issue + (q - next_rel));
      }
      next_issue = min(p_last + 1, next_issue + (qlo - next_rel));
      next_rel = qlo;
    }
    while (waited < qhi) {
      if (!wait_piece(waited + 1)) return false;
      ++waited;
    }
    __syncwarp();
    return true;
  }

  __device__ __forceinline__ void load(int64_t j, int32_t p[3]) const {
    const int32_t* w = sm->ring[(int)(((j >> kPieceLog2) - p_first) & (kStages - 1))] + 3 * (j & (kPieceV - 1));
    p[0] = w[0];
    p[1] = w[1];
    p[2] = w[2];
  }

  // Wait (bounded) for every issued piece so that no copy is in flight when
  // the warp leaves.
  __device__ __forceinline__ void drain() {
    while (waited < next_issue - 1) {
      if (!wait_piece(waited + 1)) break;
      ++waited;
    }
  }
};

__global__ void __launch_bounds__(kTmaWarps * 32) prefilter_tma_kernel(Tract t, VolView v, int prefilter,
                                                                      uint32_t mode, int32_t* surv,
                                                                      DevState* st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PfWarpSmem* sm = reinterpret_cast<PfWarpSmem*>(smem_raw) + (threadIdx.x >> 5);
  const unsigned lane = lane_id();
  const int64_t gw = (int64_t)blockIdx.x * kTmaWarps + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * kTmaWarps;
  if (gw == 0 && lane == 0 && (t.off[0] != 0 || t.off[t.ns] != t.nv)) set_error(st, kErrOffsets, -1);
  const bool point_mode = (mode & kModeVertexSampled) != 0;
  const int64_t s_lo = t.ns * gw / nw, s_hi = t.ns * (gw + 1) / nw;
  unsigned long long steps = 0, kept = 0;
  int nbuf = 0;

  // validate the warp's offsets before any copy is issued
  bool ok = true;
  for (int64_t s = s_lo + lane; s < s_hi; s += 32) {
    const int64_t a = t.off[s], b = t.off[s + 1];
    ok &= (a >= 0) && (a <= b) && (b <= t.nv);
  }
  if (!__all_sync(kFull, ok)) {
    if (lane == 0) set_error(st, kErrOffsets, (int32_t)s_lo);
    return;
  }
  if (s_hi <= s_lo) return;
  const int64_t V0 = t.off[s_lo], V1 = t.off[s_hi];
  if (V1 <= V0) return;  // only empty streamlines

  Ring r;
  r.sm = sm;
  r.xyz = t.xyz;
  r.nv = t.nv;
  r.p_first = V0 >> kPieceLog2;
  r.p_last = (V1 - 1) >> kPieceLog2;
  r.next_issue = min(r.p_last + 1, r.p_first + kStages);
  r.next_rel = r.p_first;
  r.waited = r.p_first - 1;
  r.policy = policy_evict_first();
  if (lane == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(&sm->bar[k], 1);
    fence_mbar_init();
    for (int64_t q = r.p_first; q < r.next_issue; ++q) r.issue(q);
  }
  __syncwarp();

  bool abort = false;
  for (int64_t s0 = s_lo; s0 < s_hi && !abort; s0 += 32) {
    const int64_t sl = s0 + lane;
    const int64_t oa = sl < s_hi ? t.off[sl] : 0, ob = sl < s_hi ? t.off[sl + 1] : 0;
    const int cnt = (int)min((int64_t)32, s_hi - s0);
    for (int i = 0; i < cnt && !abort; ++i) {
      const int64_t a = __shfl_sync(kFull, oa, i), b = __shfl_sync(kFull, ob, i);
      const int64_t T = b - a;
      if (T == 0) continue;
      const bool single = T == 1;
      const int64_t units = (single || point_mode) ? T : T - 1;
      uint32_t bits = 0;
      bool bad = false;
      for (int64_t i0 = 0; i0 < units; i0 += 32) {
        const int64_t jhi = min(a + i0 + 32, b - 1);
        if (!r.ensure(a + i0, jhi)) { abort = true; break; }
        const int64_t j = a + i0 + lane;
        if (i0 + lane < units) {
          int32_t p0[3], p1[3];
          r.load(j, p0);
          const bool has_next = j + 1 < b;
          if (has_next) r.load(j + 1, p1);
          else { p1[0] = p0[0]; p1[1] = p0[1]; p1[2] = p0[2]; }
          eval_unit(v, p0, p1, has_next, single, single || point_mode, steps, bits, bad);
        }
      }
      if (abort) break;
      bits = __reduce_or_sync(kFull, bits);
      if (__any_sync(kFull, bad)) {
        if (lane == 0) set_error(st, kErrCoord, (int32_t)(s0 + i));
        continue;
      }
      if (!prefilter || bits == 3u) {
        if (lane == 0) sm->sbuf[nbuf] = (int32_t)(s0 + i);
        ++kept;
        if (++nbuf == 32) flush_survivors(sm->sbuf, nbuf, surv, st);
      }
    }
  }
  if (abort && lane == 0) set_error(st, kErrTimeout, (int32_t)gw);
  r.drain();
  __syncwarp();
  flush_survivors(sm->sbuf, nbuf, surv, st);
  steps = warp_sum_u64(steps);
  if (lane == 0) {
    atomicAdd(&st->voxel_steps, steps);
    atomicAdd(&st->survivors, kept);
  }
}

cudaError_t launch_prefilter(const Tract& t, const VolView& v, bool prefilter, uint32_t mode, bool tma,
                             int32_t* survivors, DevState* st, int num_sms, cudaStream_t s) {
  if (t.ns <= 0) return cudaSuccess;
  if (tma) {
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(prefilter_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kTmaSmemBytes);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
    prefilter_tma_kernel<<<num_sms * 4, kTmaWarps * 32, kTmaSmemBytes, s>>>(t, v, prefilter ? 1 : 0, mode,
                                                                             survivors, st);
  } else {
    prefilter_direct_kernel<<<num_sms * 8, kDirWarps * 32, 0, s>>>(t, v, prefilter ? 1 : 0, mode, survivors, st);
  }
  return cudaGetLastError();
}

}  // namespace fc
