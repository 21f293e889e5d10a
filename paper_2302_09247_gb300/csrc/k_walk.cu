// K3: walk, dedup and accumulate (Section 2, Algorithm 2 for each surviving
// streamline: passthrough, then C(v, r) += 1 for every pass-through v and
// target r).
//
// One warp per surviving streamline (taken dynamically, the long ones
// first), lanes over its segments.  Each lane walks its segment with the
// exact integer walk and looks up the ROI row and label of every voxel it
// enters (the per-voxel code is read through the read-only cache with an L2
// evict-last hint).  The first voxel of a segment is the last voxel of the
// previous one, so only the streamline's first segment visits its start
// voxel; short segments whose start voxel lies far from every ROI and
// labelled voxel are not walked.  Rows and labels are deduplicated per
// streamline in two per-warp shared-memory sets (V_s and T_s): bitmaps when
// the keys fit, else open-addressing hash sets after merging equal keys
// across lanes with __match_any_sync.  The outer product V_s x T_s is then
// added to C with one L2 reduction per pair, and the seed/endpoint pair to
// C_end.  A streamline whose sets outgrow the tables is handed, whole, to an
// exact CTA-per-streamline path with global-memory bitmaps.
#include "fc_device.cuh"
#include "fc_tma.cuh"

namespace fc {

constexpr int kWalkWarps = 8;
// CTAs per SM the walk kernels are compiled for (at most 64 registers a
// thread): the walk is latency-bound, and four CTAs (32 warps) per SM hide
// more of it than three.
constexpr int kWalkMinBlocks = 4;
constexpr int kHV = 512, kLimV = 256;  // V_s table slots / size limit
constexpr int kHT = 128, kLimT = 64;   // T_s table slots / size limit
constexpr int kLin = 256;              // visited voxels awaiting their code gathers

// Every insertion round adds at most 32 keys to a list, and the limits are
// checked after every round: the lists hold limit + 32 keys.
struct WalkWarpSmem {
  int32_t tabV[kHV];
  int32_t listV[kLimV + 32];
  int32_t tabT[kHT];
  int32_t listT[kLimT + 32];
  int32_t lin[kLin];
};

// The per-warp sets V_s and T_s live in tabV / tabT in one of two forms,
// chosen per launch: an open-addressing hash set (empty = -1), or, when every
// key fits (N <= 32 * kHV rows, M < 32 * kHT labels), a bitmap of the keys
// (one shared-memory atomicOr per key).  Both append new keys to listV /
// listT in lane order; a bitmap is cleared through its list.
constexpr int32_t kBitRowsMax = 32 * kHV;
constexpr int32_t kBitLabelsMax = 32 * kHT;  // labels 1 .. kBitLabelsMax - 1

template <int kWords, int kCap>
__device__ __forceinline__ int bit_insert(int32_t* tab, int32_t* list, int n, int32_t key, DevState* ck) {
  bool fresh = false;
  if (key >= 0 && in_bounds(key >> 5, kWords, ck, kSiteSetList)) {
    const uint32_t m = 1u << (key & 31);
    fresh = (atomicOr(reinterpret_cast<uint32_t*>(tab) + (key >> 5), m) & m) == 0u;
  }
  const unsigned fm = __ballot_sync(kFull, fresh);
  if (fresh) {
    const int at = n + __popc(fm & lanemask_lt());
    if (in_bounds(at, kCap, ck, kSiteSetList)) list[at] = key;
  }
  return n + __popc(fm);
}

template <bool kBitV, bool kBitT>
struct Sets {
  __device__ __forceinline__ static int insV(WalkWarpSmem& sm, int n, int32_t key, bool& fail, DevState* ck) {
    return kBitV ? bit_insert<kHV, kLimV + 32>(sm.tabV, sm.listV, n, key, ck)
                 : set_insert<kHV>(sm.tabV, sm.listV, n, key, fail, kLimV + 32, ck);
  }
  __device__ __forceinline__ static int insT(WalkWarpSmem& sm, int n, int32_t key, bool& fail, DevState* ck) {
    return kBitT ? bit_insert<kHT, kLimT + 32>(sm.tabT, sm.listT, n, key, ck)
                 : set_insert<kHT>(sm.tabT, sm.listT, n, key, fail, kLimT + 32, ck);
  }
  // empty tables at kernel start
  __device__ __forceinline__ static void init(WalkWarpSmem& sm) {
    for (int i = lane_id(); i < kHV; i += 32) sm.tabV[i] = kBitV ? 0 : -1;
    for (int i = lane_id(); i < kHT; i += 32) sm.tabT[i] = kBitT ? 0 : -1;
    __syncwarp();
  }
  // empty them again after a streamline whose sets hold nV / nT keys
  __device__ __forceinline__ static void clear(WalkWarpSmem& sm, int nV, int nT) {
    __syncwarp();
    if (kBitV) {
      for (int k = lane_id(); k < nV; k += 32) sm.tabV[sm.listV[k] >> 5] = 0;
    } else {
      for (int i = lane_id(); i < kHV; i += 32) sm.tabV[i] = -1;
    }
    if (kBitT) {
      for (int k = lane_id(); k < nT; k += 32) sm.tabT[sm.listT[k] >> 5] = 0;
    } else {
      for (int i = lane_id(); i < kHT; i += 32) sm.tabT[i] = -1;
    }
    __syncwarp();
  }
};

__device__ __forceinline__ void load_vertex(const int32_t* xyz, int64_t j, int32_t p[3]) {
  p[0] = __ldg(xyz + 3 * j);
  p[1] = __ldg(xyz + 3 * j + 1);
  p[2] = __ldg(xyz + 3 * j + 2);
}

// The 16-byte units inside the vertices [a, b) of t, prefetched into L2 by the
// bulk-copy engine: the windows after a streamline's first then load from L2
// instead of waiting on HBM one window at a time.
__device__ __forceinline__ void prefetch_vertices(const Tract& t, int64_t a, int64_t b) {
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(t.xyz + 3 * a) + 15) & ~(uintptr_t)15;
  const uintptr_t hi = reinterpret_cast<uintptr_t>(t.xyz + 3 * b) & ~(uintptr_t)15;
  if (hi > lo) bulk_prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)min(hi - lo, (uintptr_t)0x7ffffff0u));
}

// Per-voxel code of in-grid voxel (x, y, z), or ~0u off the grid (no row, no
// label).
__device__ __forceinline__ int32_t voxel_lin(const VolView& v, int32_t x, int32_t y, int32_t z) {
  if ((unsigned)x < (unsigned)v.dx && (unsigned)y < (unsigned)v.dy && (unsigned)z < (unsigned)v.dz)
    return x + v.dx * (y + v.dy * z);
  return -1;
}

__device__ __forceinline__ void decode(const VolView& v, int32_t lin, uint32_t code, int32_t& row, int32_t& lab,
                                       DevState* ck) {
  row = -1;
  lab = 0;
  if (lin < 0) return;
  if (code & kCodeRoi) {
    row = (int32_t)(code & kCodeRowMask);
    if ((code & kCodeRoiLabelled) && in_bounds(lin, voxel_count(v), ck, kSiteLabel)) lab = (int32_t)__ldg(v.lab + lin);
  } else {
    lab = (int32_t)code;
  }
}

// The listed voxels' codes, decoded and inserted into the sets, 32 keys per
// round with the size limits checked after each round.  Empties the list.
// kWide: four rounds of loads in flight at once; otherwise one
// round at a time (few registers: used inside the walk's loop, where long
// segments may fill the list).
template <typename S, bool kWide>
__device__ __forceinline__ void flush_voxels(const VolView& v, WalkWarpSmem& sm, int& nL, bool endpoint_mode,
                                             uint64_t keep, int& nV, int& nT, bool& fail, DevState* ck) {
  __syncwarp();
  constexpr int kPer = kWide ? 4 : 1;
  const int lane = (int)lane_id();
  for (int r0 = 0; r0 < nL && !fail; r0 += 32 * kPer) {  // one pass when kWide
    int32_t lin[kPer];
    uint32_t code[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) lin[k] = r0 + lane + 32 * k < nL ? sm.lin[r0 + lane + 32 * k] : -1;
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      code[k] = lin[k] >= 0 && in_bounds(lin[k], voxel_count(v), ck, kSiteCode) ? ldg_hint(v.code + lin[k], keep) : 0u;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      if (r0 + 32 * k < nL && !fail) {  // warp-uniform
        int32_t row, lab;
        decode(v, lin[k], code[k], row, lab, ck);
        if (endpoint_mode) lab = 0;
        nV = S::insV(sm, nV, row, fail, ck);
        nT = S::insT(sm, nT, lab > 0 ? lab : -1, fail, ck);
        fail = __any_sync(kFull, fail) || nV > kLimV || nT > kLimT;  // warp-uniform
      }
    }
  }
  nL = 0;
  __syncwarp();
}

// Walk the window's segments (one per lane, p0 -> p1 where has) and list
// every in-grid voxel a segment enters (and, for the streamline's first
// segment, its start voxel); the list is flushed into the sets when it
// fills.  The walk itself has no memory dependence, so a window costs no
// load latency beyond its vertices.
template <typename W, typename S>
__device__ __forceinline__ void walk_window(const VolView& v, WalkWarpSmem& sm, const int32_t p0[3],
                                            const int32_t p1[3], bool has, bool first, bool endpoint_mode,
                                            uint64_t keep, int& nL, int& nV, int& nT, bool& fail, DevState* ck) {
  W w;
  bool pend = false;
  if (has) {
    w.init(p0, p1);
    pend = first ? true : w.step();
  }
  while (__any_sync(kFull, pend)) {
    const int32_t lin = pend ? voxel_lin(v, w.cx, w.cy, w.cz) : -1;
    const unsigned m = __ballot_sync(kFull, lin >= 0);
    if (lin >= 0) {
      const int at = nL + __popc(m & lanemask_lt());
      if (in_bounds(at, kLin, ck, kSiteVoxelList)) sm.lin[at] = lin;
    }
    nL += __popc(m);
    if (pend) pend = w.step();
    if (nL > kLin - 32) {  // long segments only: windows start with room for 3 voxels a lane
      flush_voxels<S, false>(v, sm, nL, endpoint_mode, keep, nV, nT, fail, ck);
      if (fail) break;
    }
  }
}

// Walk surviving streamline s of (v, t) with the whole warp and add its
// pairs to acc.  Returns |V_s| |T_s| (warp-uniform), or -1 when its sets
// outgrew the tables: then `id` is appended to the overflow list instead.
template <typename S>
__device__ __forceinline__ int walk_one(const VolView& v, const Tract& t, const Accum& acc, uint32_t mode,
                                        WalkWarpSmem& sm, int32_t s, int32_t id, int32_t* __restrict__ ovf,
                                        int64_t ovf_cap, DevState* gst) {
  const unsigned lane = lane_id();
  const bool endpoint_mode = (mode & kModeTargetEndpoint) != 0;
  const bool point_mode = (mode & kModeVertexSampled) != 0;
  const bool walk_all = (mode & kModeWalkAll) != 0;
  const uint64_t keep = policy_evict_last();  // code gathers and C stay in L2 across the stream
  const int64_t M = v.n_lab;
  if (!in_bounds(s, t.ns, gst, kSiteSurvivorRead)) return 0;
  const int64_t a = t.off[s], b = t.off[s + 1];
  // offsets the prefilter has flagged as invalid may reach this point; such
  // a streamline is skipped (the call reports the error)
  if (a < 0 || b > t.nv || b <= a) return 0;
  const int64_t T = b - a;
  if (T > 33 && lane == 0) prefetch_vertices(t, a + 32, b);
  int nV = 0, nT = 0;
  bool fail = false;
  if (T == 1 || point_mode) {
    for (int64_t i0 = 0; i0 < T && !fail; i0 += 32) {
      const int64_t j = a + i0 + lane;
      int32_t row = -1, lab = 0;
      if (j < b) {
        int32_t p[3];
        load_vertex(t.xyz, j, p);
        voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, row, lab, gst);
      }
      if (endpoint_mode) lab = 0;
      nV = S::insV(sm, nV, row, fail, gst);
      nT = S::insT(sm, nT, lab > 0 ? lab : -1, fail, gst);
      if (nV > kLimV || nT > kLimT) fail = true;
      fail = __any_sync(kFull, fail);
    }
  } else {
    // window i0 holds segments a+i0+lane -> a+i0+lane+1, both ends loaded by
    // the lane; the next window's lines are prefetched into L1 while this one
    // is walked, so that its loads wait on L1 rather than on L2
    int nL = 0;
    for (int64_t i0 = 0; i0 < T - 1 && !fail; i0 += 32) {
      if (nL > kLin - 96) {  // room for three voxels a lane
        flush_voxels<S, true>(v, sm, nL, endpoint_mode, keep, nV, nT, fail, gst);
        if (__any_sync(kFull, fail)) break;
      }
      const int64_t j = a + i0 + lane;
      if (j + 32 < b) prefetch_l1(t.xyz + 3 * (j + 32));
      int32_t p0[3] = {0, 0, 0}, p1[3] = {0, 0, 0};
      if (j < b - 1) {
        load_vertex(t.xyz, j, p0);
        load_vertex(t.xyz, j + 1, p1);
      }
      // a segment whose end voxels differ by at most one on every axis stays
      // within Chebyshev distance 1 of its start voxel: when the near grid
      // shows no ROI and no labelled voxel there, it visits nothing that
      // counts and is not walked
      // (a segment shorter than a voxel on every axis is such a segment;
      // only longer ones need their end voxels compared)
      const bool sub = abs(p1[0] - p0[0]) < 1024 && abs(p1[1] - p0[1]) < 1024 && abs(p1[2] - p0[2]) < 1024;
      bool has = j < b - 1;
      if (has) {
        const int32_t c0x = p0[0] >> kUnitLog2, c0y = p0[1] >> kUnitLog2, c0z = p0[2] >> kUnitLog2;
        bool shortseg = sub;
        if (!sub)
          shortseg = abs((p1[0] >> kUnitLog2) - c0x) <= 1 && abs((p1[1] >> kUnitLog2) - c0y) <= 1 &&
                     abs((p1[2] >> kUnitLog2) - c0z) <= 1;
        if (shortseg && !walk_all && near_lookup<false>(v, v.near, c0x, c0y, c0z, gst) == 0u) has = false;
      }
      // windows whose segments are all shorter than a voxel on every axis
      // (the common case) take the common-denominator walk; others the
      // general one with 64-bit cross-products
      const bool tiny = !has || sub;
      if (__all_sync(kFull, tiny))
        walk_window<SegShort, S>(v, sm, p0, p1, has, j == a, endpoint_mode, keep, nL, nV, nT, fail, gst);
      else
        walk_window<SegWalk<unsigned long long>, S>(v, sm, p0, p1, has, j == a, endpoint_mode, keep, nL, nV, nT,
                                                     fail, gst);
      fail = __any_sync(kFull, fail);
    }
    if (nL > 0 && !fail) flush_voxels<S, true>(v, sm, nL, endpoint_mode, keep, nV, nT, fail, gst);
    fail = __any_sync(kFull, fail);
  }
  if (endpoint_mode && !fail) {
    // T_s = {label of the last vertex}
    int32_t row = -1, lab = 0;
    if (lane == 0) {
      int32_t p[3];
      load_vertex(t.xyz, b - 1, p);
      voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, row, lab, gst);
    }
    nT = S::insT(sm, nT, lab > 0 ? lab : -1, fail, gst);
    fail = __any_sync(kFull, fail) || nT > kLimT;
  }
  __syncwarp();
  int pairs = -1;
  if (fail) {
    if (lane == 0) {
      const uint32_t at = atomicAdd(&gst->n_overflow, 1u);
      if (in_bounds(at, ovf_cap, gst, kSiteOverflowList)) ovf[at] = id;
    }
  } else {
    pairs = nV * nT;
    const int64_t NM = (int64_t)v.n_roi * M;
    for (int p = lane; p < pairs; p += 32) {
      const int i = p / nT, k = p - i * nT;
      const int64_t e = (int64_t)sm.listV[i] * M + (sm.listT[k] - 1);
      if (in_bounds(e, NM, gst, kSiteC)) red_add_hint(acc.C + e, 1, keep);
    }
    if (lane == 0) {
      int32_t p[3], r0, l0, r1, l1;
      load_vertex(t.xyz, a, p);
      voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, r0, l0, gst);
      load_vertex(t.xyz, b - 1, p);
      voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, r1, l1, gst);
      const int64_t e = (int64_t)r0 * M + (l1 - 1);
      if (r0 >= 0 && l1 >= 1 && in_bounds(e, NM, gst, kSiteCend)) atomicAdd(acc.Cend + e, 1);
    }
  }
  S::clear(sm, nV, nT);
  return pairs;
}

__device__ __forceinline__ uint32_t next_survivor(DevState* gst) {
  uint32_t idx = 0;
  if (lane_id() == 0) idx = atomicAdd(&gst->work_next, 1u);
  return __shfl_sync(kFull, idx, 0);
}

template <bool kBitV, bool kBitT>
__global__ void __launch_bounds__(kWalkWarps * 32, kWalkMinBlocks)
    walk_kernel(Tract t, VolView v, const int32_t* __restrict__ surv, int64_t surv_cap, Accum acc, uint32_t mode,
                int32_t* __restrict__ ovf, DevState* st) {
  using S = Sets<kBitV, kBitT>;
  __shared__ WalkWarpSmem smem_all[kWalkWarps];
  WalkWarpSmem& sm = smem_all[threadIdx.x >> 5];
  S::init(sm);
  griddep_launch_dependents();
  griddep_wait();  // the prefilter's survivor list and counters
  const uint32_t nl = st->n_long, n = st->n_survivors + nl;
  if (n > 0 && !in_bounds((int64_t)n - 1, surv_cap, st, kSiteSurvivorRead)) return;
  unsigned long long pairs_acc = 0;
  for (;;) {
    const uint32_t idx = next_survivor(st);
    if (idx >= n) break;
    const int32_t s = survivor_at(surv, surv_cap, nl, idx);
    const int pairs = walk_one<S>(v, t, acc, mode, sm, s, s, ovf, surv_cap, st);
    if (pairs > 0) pairs_acc += (unsigned long long)pairs;
  }
  if (lane_id() == 0 && pairs_acc) atomicAdd(&st->pairs, pairs_acc);
}

// Voxel steps of the survivors (the metric's definition: per segment 1 + the
// sum over the axes of its ends' voxel-coordinate differences; a single
// vertex counts 1), warp per survivor, lanes over its segments.
__global__ void __launch_bounds__(256) walked_steps_kernel(Tract t, const int32_t* __restrict__ surv,
                                                           int64_t surv_cap, DevState* st) {
  const uint32_t nl = st->n_long, n = st->n_survivors + nl;
  const uint32_t lane = lane_id();
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long acc = 0;
  for (uint32_t idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < n; idx += nwarps) {
    const int32_t s = survivor_at(surv, surv_cap, nl, idx);
    const int64_t a = t.off[s], b = t.off[s + 1];
    if (a < 0 || b > t.nv || b <= a) continue;
    if (b - a == 1) {
      acc += lane == 0 ? 1ull : 0ull;
      continue;
    }
    for (int64_t j = a + lane; j + 1 < b; j += 32) {
      int32_t p0[3], p1[3];
      load_vertex(t.xyz, j, p0);
      load_vertex(t.xyz, j + 1, p1);
      acc += 1ull + (unsigned long long)(abs((p1[0] >> kUnitLog2) - (p0[0] >> kUnitLog2)) +
                                         abs((p1[1] >> kUnitLog2) - (p0[1] >> kUnitLog2)) +
                                         abs((p1[2] >> kUnitLog2) - (p0[2] >> kUnitLog2)));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane == 0 && acc) atomicAdd(&st->walked, acc);
}

// Subject of global streamline id g (subjects' sbase ascend).
__device__ __forceinline__ int subject_of(const BatchTable& tbl, int64_t g) {
  int lo = 0, hi = tbl.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tbl.s[mid].sbase <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <bool kBitV, bool kBitT>
__global__ void __launch_bounds__(kWalkWarps * 32, kWalkMinBlocks)
    walk_batch_kernel(const __grid_constant__ BatchTable tbl, const int32_t* __restrict__ surv, int64_t surv_cap,
                      uint32_t mode, int32_t* __restrict__ ovf, DevState* gst) {
  using S = Sets<kBitV, kBitT>;
  __shared__ WalkWarpSmem smem_all[kWalkWarps];
  WalkWarpSmem& sm = smem_all[threadIdx.x >> 5];
  S::init(sm);
  const uint32_t nl = gst->n_long, n = gst->n_survivors + nl;
  if (n > 0 && !in_bounds((int64_t)n - 1, surv_cap, gst, kSiteSurvivorRead)) return;
  for (;;) {
    const uint32_t idx = next_survivor(gst);
    if (idx >= n) break;
    const int32_t g = survivor_at(surv, surv_cap, nl, idx);
    const BatchSubject& B = tbl.s[subject_of(tbl, g)];
    const int pairs = walk_one<S>(B.v, B.t, B.acc, mode, sm, (int32_t)(g - B.sbase), g, ovf, surv_cap, gst);
    if (pairs > 0 && lane_id() == 0) atomicAdd(&B.st->pairs, (unsigned long long)pairs);
  }
}

// ---------------------------------------------------------------- overflow
// One CTA per overflowed streamline.  Sets are bitmaps over all N rows and
// M+1 labels in the CTA's slice of global scratch, with append lists; the
// bitmaps are cleared through the lists after each streamline, so they are
// all-zero between streamlines (the scratch is zeroed once when allocated).

int64_t overflow_scratch_words(int32_t n_roi, int32_t n_lab) {
  return ((int64_t)n_roi + 31) / 32 + ((int64_t)n_lab + 1 + 31) / 32 + n_roi + (int64_t)n_lab + 1;
}

struct OvfSets {
  uint32_t* rowbits;
  uint32_t* labbits;
  int32_t* rowlist;
  int32_t* lablist;
};

// key < n_keys (the bitmap holds n_keys bits, the list n_keys entries)
__device__ __forceinline__ void ovf_add(uint32_t* bits, int32_t* list, int* n, int32_t key, int64_t n_keys,
                                        DevState* ck) {
  if (!in_bounds(key, n_keys, ck, kSiteScratch)) return;
  const uint32_t m = 1u << (key & 31);
  if (!(atomicOr(bits + (key >> 5), m) & m)) {
    const int at = atomicAdd(n, 1);
    if (in_bounds(at, n_keys, ck, kSiteScratch)) list[at] = key;
  }
}

__device__ __forceinline__ void ovf_visit(const VolView& v, const OvfSets& z, int* nV, int* nT, bool endpoint_mode,
                                          int32_t x, int32_t y, int32_t zz, DevState* ck) {
  int32_t row, lab;
  voxel_lookup(v, x, y, zz, row, lab, ck);
  if (row >= 0) ovf_add(z.rowbits, z.rowlist, nV, row, v.n_roi, ck);
  if (!endpoint_mode && lab >= 1) ovf_add(z.labbits, z.lablist, nT, lab, (int64_t)v.n_lab + 1, ck);
}

// The whole CTA handles streamline s of (v, t): walk every segment, sets as
// bitmaps + lists in this CTA's scratch slice, then pairs and C_end.
__device__ __forceinline__ void overflow_one(const VolView& v, const Tract& t, const Accum& acc, uint32_t mode,
                                             uint32_t* slice, int32_t s, DevState* sst, int* nV, int* nT) {
  OvfSets z;
  z.rowbits = slice;
  z.labbits = z.rowbits + ((int64_t)v.n_roi + 31) / 32;
  z.rowlist = reinterpret_cast<int32_t*>(z.labbits + ((int64_t)v.n_lab + 1 + 31) / 32);
  z.lablist = z.rowlist + v.n_roi;
  const bool endpoint_mode = (mode & kModeTargetEndpoint) != 0;
  const bool point_mode = (mode & kModeVertexSampled) != 0;
  const int64_t M = v.n_lab;
  if (threadIdx.x == 0) { *nV = 0; *nT = 0; }
  __syncthreads();
  const int64_t a = t.off[s], b = t.off[s + 1];
  const int64_t T = (a >= 0 && b <= t.nv && a <= b) ? b - a : 0;  // invalid offsets: nothing (error reported)
  const bool pts = T == 1 || point_mode;
  const int64_t units = pts ? T : T - 1;
  for (int64_t u = threadIdx.x; u < units; u += blockDim.x) {
    int32_t p0[3];
    load_vertex(t.xyz, a + u, p0);
    if (pts) {
      ovf_visit(v, z, nV, nT, endpoint_mode, p0[0] >> kUnitLog2, p0[1] >> kUnitLog2, p0[2] >> kUnitLog2, sst);
    } else {
      int32_t p1[3];
      load_vertex(t.xyz, a + u + 1, p1);
      SegWalk<unsigned long long> w;
      w.init(p0, p1);
      ovf_visit(v, z, nV, nT, endpoint_mode, w.cx, w.cy, w.cz, sst);
      while (w.step()) ovf_visit(v, z, nV, nT, endpoint_mode, w.cx, w.cy, w.cz, sst);
    }
  }
  if (endpoint_mode && threadIdx.x == 0 && T >= 1) {
    int32_t p[3], row, lab;
    load_vertex(t.xyz, b - 1, p);
    voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, row, lab, sst);
    if (lab >= 1) ovf_add(z.labbits, z.lablist, nT, lab, (int64_t)v.n_lab + 1, sst);
  }
  __syncthreads();
  const int64_t pairs = (int64_t)(*nV) * (*nT);
  const int64_t NM = (int64_t)v.n_roi * M;
  for (int64_t p = threadIdx.x; p < pairs; p += blockDim.x) {
    const int64_t r = p / *nT, k = p - r * *nT;
    const int64_t e = (int64_t)z.rowlist[r] * M + (z.lablist[k] - 1);
    if (in_bounds(e, NM, sst, kSiteC)) atomicAdd(acc.C + e, 1);
  }
  if (threadIdx.x == 0) {
    if (pairs) atomicAdd(&sst->pairs, (unsigned long long)pairs);
    atomicAdd(&sst->overflow, 1ull);
    if (T >= 1) {
      int32_t p[3], r0, l0, r1, l1;
      load_vertex(t.xyz, a, p);
      voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, r0, l0, sst);
      load_vertex(t.xyz, b - 1, p);
      voxel_lookup(v, p[0] >> kUnitLog2, p[1] >> kUnitLog2, p[2] >> kUnitLog2, r1, l1, sst);
      const int64_t e = (int64_t)r0 * M + (l1 - 1);
      if (r0 >= 0 && l1 >= 1 && in_bounds(e, NM, sst, kSiteCend)) atomicAdd(acc.Cend + e, 1);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < *nV; k += blockDim.x) z.rowbits[z.rowlist[k] >> 5] = 0u;
  for (int k = threadIdx.x; k < *nT; k += blockDim.x) z.labbits[z.lablist[k] >> 5] = 0u;
  __syncthreads();
}

__global__ void __launch_bounds__(256) walk_overflow_kernel(Tract t, VolView v, const int32_t* __restrict__ ovf,
                                                            Accum acc, uint32_t mode, uint32_t* scratch,
                                                            int64_t words_per_cta, DevState* st) {
  __shared__ int nV, nT;
  griddep_wait();  // the walk's overflow list
  const uint32_t n = st->n_overflow;
  for (uint32_t i = blockIdx.x; i < n; i += gridDim.x)
    overflow_one(v, t, acc, mode, scratch + blockIdx.x * words_per_cta, ovf[i], st, &nV, &nT);
}

__global__ void __launch_bounds__(256)
    walk_overflow_batch_kernel(const __grid_constant__ BatchTable tbl, const int32_t* __restrict__ ovf, uint32_t mode,
                               uint32_t* scratch, int64_t words_per_cta, DevState* gst) {
  __shared__ int nV, nT;
  const uint32_t n = gst->n_overflow;
  for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
    const int32_t g = ovf[i];
    const BatchSubject& S = tbl.s[subject_of(tbl, g)];
    overflow_one(S.v, S.t, S.acc, mode, scratch + blockIdx.x * words_per_cta, (int32_t)(g - S.sbase), S.st, &nV,
                 &nT);
  }
}

// CTAs per SM of a walk kernel (its grid: every CTA resident at once).
template <typename K>
int walk_blocks_per_sm(K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWalkWarps * 32, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = kWalkMinBlocks;
  }
  return per_sm > 0 ? per_sm : 1;
}

// Launch in stream order with programmatic stream serialisation: the kernel
// may be scheduled while the previous one ends and waits for it in
// griddep_wait.
template <typename... Params, typename... Args>
cudaError_t launch_after_previous(void (*kernel)(Params...), int grid, int block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <bool kBitV, bool kBitT>
cudaError_t launch_walk_k(const Tract& t, const VolView& v, const int32_t* survivors, int64_t surv_cap, Accum acc,
                          uint32_t mode, int32_t* overflow_list, DevState* st, int num_sms, cudaStream_t s) {
  // CTAs per SM depend on the kernel and the architecture (one, sm_103a), so
  // they are asked once; the grid follows the context's device
  static const int per_sm = walk_blocks_per_sm(walk_kernel<kBitV, kBitT>);
  const int grid = num_sms * per_sm;
  return launch_after_previous(walk_kernel<kBitV, kBitT>, grid, kWalkWarps * 32, s, t, v, survivors, surv_cap, acc,
                               mode, overflow_list, st);
}

template <bool kBitV, bool kBitT>
cudaError_t launch_walk_batch_k(const BatchTable& tbl, const int32_t* survivors, int64_t surv_cap, uint32_t mode,
                                int32_t* overflow_list, DevState* gst, int num_sms, cudaStream_t s) {
  static const int per_sm = walk_blocks_per_sm(walk_batch_kernel<kBitV, kBitT>);
  const int grid = num_sms * per_sm;
  walk_batch_kernel<kBitV, kBitT><<<grid, kWalkWarps * 32, 0, s>>>(tbl, survivors, surv_cap, mode, overflow_list, gst);
  return cudaGetLastError();
}

cudaError_t launch_walk(const Tract& t, const VolView& v, const int32_t* survivors, int64_t surv_cap, Accum acc,
                        uint32_t mode, int32_t* overflow_list, DevState* st, int num_sms, cudaStream_t s) {
  if (t.ns <= 0) return cudaSuccess;
  const bool bv = v.n_roi <= kBitRowsMax, bt = v.n_lab < kBitLabelsMax;
  if (bv && bt) return launch_walk_k<true, true>(t, v, survivors, surv_cap, acc, mode, overflow_list, st, num_sms, s);
  if (bv) return launch_walk_k<true, false>(t, v, survivors, surv_cap, acc, mode, overflow_list, st, num_sms, s);
  if (bt) return launch_walk_k<false, true>(t, v, survivors, surv_cap, acc, mode, overflow_list, st, num_sms, s);
  return launch_walk_k<false, false>(t, v, survivors, surv_cap, acc, mode, overflow_list, st, num_sms, s);
}

cudaError_t launch_walked_steps(const Tract& t, const int32_t* survivors, int64_t survivor_cap, DevState* st,
                                int num_sms, cudaStream_t s) {
  if (t.ns <= 0) return cudaSuccess;
  walked_steps_kernel<<<num_sms * 8, 256, 0, s>>>(t, survivors, survivor_cap, st);
  return cudaGetLastError();
}

cudaError_t launch_walk_overflow(const Tract& t, const VolView& v, const int32_t* overflow_list, Accum acc,
                                 uint32_t mode, uint32_t* scratch, int32_t scratch_ctas, DevState* st,
                                 cudaStream_t s) {
  if (t.ns <= 0) return cudaSuccess;
  return launch_after_previous(walk_overflow_kernel, scratch_ctas, 256, s, t, v, overflow_list, acc, mode, scratch,
                               overflow_scratch_words(v.n_roi, v.n_lab), st);
}

cudaError_t launch_walk_batch(const BatchTable& tbl, const int32_t* survivors, int64_t surv_cap, uint32_t mode,
                              int32_t* overflow_list, DevState* gst, int num_sms, cudaStream_t s) {
  bool bv = true, bt = true;
  for (int32_t i = 0; i < tbl.n; ++i) {
    bv &= tbl.s[i].v.n_roi <= kBitRowsMax;
    bt &= tbl.s[i].v.n_lab < kBitLabelsMax;
  }
  if (bv && bt) return launch_walk_batch_k<true, true>(tbl, survivors, surv_cap, mode, overflow_list, gst, num_sms, s);
  if (bv) return launch_walk_batch_k<true, false>(tbl, survivors, surv_cap, mode, overflow_list, gst, num_sms, s);
  if (bt) return launch_walk_batch_k<false, true>(tbl, survivors, surv_cap, mode, overflow_list, gst, num_sms, s);
  return launch_walk_batch_k<false, false>(tbl, survivors, surv_cap, mode, overflow_list, gst, num_sms, s);
}

cudaError_t launch_walk_overflow_batch(const BatchTable& tbl, const int32_t* overflow_list, uint32_t mode,
                                       uint32_t* scratch, int32_t scratch_ctas, int64_t words_per_cta, DevState* gst,
                                       cudaStream_t s) {
  walk_overflow_batch_kernel<<<scratch_ctas, 256, 0, s>>>(tbl, overflow_list, mode, scratch, words_per_cta, gst);
  return cudaGetLastError();
}

}  // namespace fc
