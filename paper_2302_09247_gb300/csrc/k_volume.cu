// K1: volume preparation.  From the caller's ROI index map (int32) and target
// label volume (uint16) build the per-voxel code, a private label copy, the
// brick occupancy bits and the near grid, validating every voxel on the way
// (Section 2: the ROI voxel set V and the target regions R that loc2region
// reads).
#include "fc_device.cuh"

namespace fc {

__global__ void __launch_bounds__(256) volume_max_kernel(const int32_t* __restrict__ roi,
                                                         const uint16_t* __restrict__ lab,
                                                         int64_t nvox, DevState* st) {
  int32_t mr = -1, ml = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvox;
       i += (int64_t)gridDim.x * blockDim.x) {
    mr = max(mr, roi[i]);
    ml = max(ml, (int32_t)lab[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mr = max(mr, __shfl_xor_sync(kFull, mr, o));
    ml = max(ml, __shfl_xor_sync(kFull, ml, o));
  }
  if (lane_id() == 0) {
    atomicMax(&st->max_roi, mr);
    atomicMax(&st->max_label, ml);
  }
}

// Blocks of 8 rows x 32 voxels: a warp covers 32 consecutive voxels of a row
// (x aligned to 32) in kPrepZ consecutive planes (z aligned to kPrepZ, one
// brick deep), one thread per (x, y) column; the thread issues the loads of
// all its planes before it uses any, so that a warp has kPrepZ row pairs in
// flight.  The warp's ballots are the rows' ROI / label bit-plane words
// (planes: two planes of Dy*Dz rows of ceil(Dx/32) words).  The warp's
// voxels touch at most two brick words: their bits, ORed over the planes and
// across the warp, are set with one atomic per word.  The grid's x blocks run
// along x; its y and z blocks together number the (8-row group, plane group)
// pairs, ryb = ceil(Dy/8) row groups per plane group, so that Dy and Dz are
// bounded only by the voxel count.
constexpr int kPrepRows = 8;
constexpr int kPrepZ = 1 << kBrickLog2;

__host__ __device__ __forceinline__ int32_t plane_groups(const VolView& v) { return (v.dz + kPrepZ - 1) / kPrepZ; }

// The voxels of x block xb, 8-row group yb and plane group zq.
__device__ __forceinline__ void prep_block(const int32_t* __restrict__ roi, const uint16_t* __restrict__ lab,
                                           const VolView& v, uint32_t* __restrict__ code,
                                           uint16_t* __restrict__ lab_out, uint32_t* __restrict__ bricks,
                                           uint32_t* __restrict__ planes, DevState* st, int32_t xb, int32_t yb,
                                           int32_t zq) {
  const int32_t lane = (int32_t)threadIdx.x;
  const int32_t x = xb * 32 + lane, y = yb * kPrepRows + threadIdx.y;
  if (y >= v.dy) return;  // whole warps: y is the same for the warp's 32 lanes
  const bool in = x < v.dx;
  const int32_t z0 = zq * kPrepZ, nz = min(kPrepZ, v.dz - z0);
  const int64_t plane = (int64_t)v.dx * v.dy;
  const int64_t i0 = x + v.dx * ((int64_t)y + (int64_t)v.dy * z0);
  int32_t r[kPrepZ], l[kPrepZ];
#pragma unroll
  for (int k = 0; k < kPrepZ; ++k) {
    const bool ok = in && k < nz;
    r[k] = ok ? roi[i0 + k * plane] : -1;
    l[k] = ok ? (int32_t)lab[i0 + k * plane] : 0;
  }
  uint32_t bits = 0u;
  const int32_t wb = (v.dx + 31) >> 5;
  const int64_t rows = (int64_t)v.dy * v.dz;
#pragma unroll
  for (int k = 0; k < kPrepZ; ++k) {
    if (in && k < nz) {
      if (r[k] < -1 || r[k] >= v.n_roi || l[k] > v.n_lab) {
        set_error(st, kErrVolume, (int32_t)(i0 + k * plane));
        r[k] = -1;
        l[k] = 0;
      }
      code[i0 + k * plane] =
          r[k] >= 0 ? (kCodeRoi | (l[k] > 0 ? kCodeRoiLabelled : 0u) | (uint32_t)r[k]) : (uint32_t)l[k];
      lab_out[i0 + k * plane] = (uint16_t)l[k];
    }
    bits |= (r[k] >= 0 ? 1u : 0u) | (l[k] > 0 ? 2u : 0u);
    const uint32_t mr = __ballot_sync(kFull, r[k] >= 0);
    const uint32_t mt = __ballot_sync(kFull, l[k] > 0);
    if (lane == 0 && k < nz) {
      const int64_t row = (int64_t)y + (int64_t)v.dy * (z0 + k);
      planes[row * wb + xb] = mr;
      planes[(rows + row) * wb + xb] = mt;
    }
  }
  // brick bits: lanes of the warp's first brick word, then of its second
  const int32_t b = ((in ? x : xb * 32) >> kBrickLog2) + v.bx * ((y >> kBrickLog2) + v.by * zq);
  const int32_t wi = b >> 4;
  const uint32_t val = bits << ((b & 15) * 2);
  // the in-range lanes are a prefix of the warp and their words do not
  // decrease: lane 0 holds the first word, the last in-range lane the second
  const int32_t last = min(31, v.dx - 1 - xb * 32);
  const int32_t wA = __shfl_sync(kFull, wi, 0), wB = __shfl_sync(kFull, wi, last);
  const uint32_t oA = __reduce_or_sync(kFull, wi == wA ? val : 0u);
  const uint32_t oB = __reduce_or_sync(kFull, wi != wA ? val : 0u);
  if (lane == 0 && oA) atomicOr(bricks + wA, oA);
  if (lane == 0 && oB) atomicOr(bricks + wB, oB);
}

__host__ __device__ __forceinline__ int32_t row_groups(const VolView& v) { return (v.dy + kPrepRows - 1) / kPrepRows; }

__global__ void __launch_bounds__(32 * kPrepRows) volume_prep_kernel(const int32_t* __restrict__ roi,
                                                                     const uint16_t* __restrict__ lab, VolView v,
                                                                     uint32_t* __restrict__ code,
                                                                     uint16_t* __restrict__ lab_out,
                                                                     uint32_t* __restrict__ bricks,
                                                                     uint32_t* __restrict__ planes, DevState* st) {
  const int64_t g = (int64_t)blockIdx.z * gridDim.y + blockIdx.y;  // (row group, plane group) pair
  const int32_t ryb = row_groups(v);
  if (g >= (int64_t)ryb * plane_groups(v)) return;  // whole blocks
  const int32_t zq = (int32_t)(g / ryb);
  prep_block(roi, lab, v, code, lab_out, bricks, planes, st, (int32_t)blockIdx.x, (int32_t)(g - (int64_t)zq * ryb),
             zq);
}

// The subject of batch block b: the last one whose first block is <= b.
template <bool kNear>
__device__ __forceinline__ int32_t subject_of(const PrepTable& tbl, int64_t b) {
  int32_t lo = 0, hi = tbl.n - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if ((kNear ? tbl.s[mid].near_blk0 : tbl.s[mid].prep_blk0) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Every subject of a batch in one launch: block b of subject i's
// ceil(Dx/32) * ceil(Dy/8) * ceil(Dz/kPrepZ) blocks, x blocks fastest.
__global__ void __launch_bounds__(32 * kPrepRows) volume_prep_batch_kernel(const __grid_constant__ PrepTable tbl) {
  const int64_t b = blockIdx.x;
  const PrepSubject& S = tbl.s[subject_of<false>(tbl, b)];
  const VolView& v = S.v;
  const int64_t local = b - S.prep_blk0;
  const int32_t nxb = (v.dx + 31) / 32, ryb = row_groups(v);
  const int64_t g = local / nxb;
  const int32_t zq = (int32_t)(g / ryb);
  prep_block(S.roi, S.lab, v, const_cast<uint32_t*>(v.code), const_cast<uint16_t*>(v.lab),
             const_cast<uint32_t*>(v.bricks), S.planes, S.st, (int32_t)(local - g * nxb),
             (int32_t)(g - (int64_t)zq * ryb), zq);
  if (S.nzero > 0) {
    // the subject's blocks share the zeroing of its accumulators (coalesced
    // word stores, a slice per block)
    const int64_t nb = (int64_t)nxb * ryb * plane_groups(v);
    const int64_t per = (S.nzero + nb - 1) / nb;
    const int64_t lo = local * per, hi = min(S.nzero, lo + per);
    const int32_t t = (int32_t)(threadIdx.y * 32 + threadIdx.x);
    for (int64_t i = lo + t; i < hi; i += 32 * kPrepRows) {
      S.zero0[i] = 0;
      S.zero1[i] = 0;
    }
  }
}

// ---------------------------------------------------------------- near grid
// One thread per near word (16 cells along x).  Cell cx covers padded voxels
// [cs*cx, cs*cx + cs) per axis (padded = voxel + 1); its bits are the OR of
// the grid voxels within Chebyshev distance 1 of it, i.e. the voxels
// [cs*cx - 2, cs*cx + cs - 1] per axis.  Rows of the two bit planes are ORed
// over the y/z range, then every cell tests its (cs + 2)-bit x window.

__device__ __forceinline__ uint32_t plane_word(const uint32_t* __restrict__ rowp, int32_t w, int32_t wb) {
  return (w >= 0 && w < wb) ? __ldg(rowp + w) : 0u;
}

// Near word idx of volume v.
__device__ __forceinline__ void near_word(const uint32_t* __restrict__ planes, const VolView& v,
                                          uint32_t* __restrict__ near, int64_t idx) {
  if (idx >= (int64_t)v.nwx * v.nny * v.nnz) return;
  const int32_t wx = (int32_t)(idx % v.nwx);
  const int64_t t = idx / v.nwx;
  const int32_t cy = (int32_t)(t % v.nny), cz = (int32_t)(t / v.nny);
  const int32_t cs = 1 << v.nsh;
  const int32_t wb = (v.dx + 31) >> 5;
  const int64_t rows = (int64_t)v.dy * v.dz;
  const int32_t x_lo = cs * 16 * wx - 2;  // first voxel x of the word's window
  const int32_t w0 = x_lo >> 5;          // floor for negative x_lo too
  const int32_t sh = x_lo & 31;
  uint32_t acc[2][5] = {{0u, 0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u, 0u}};  // bits x_lo .. x_lo + 159
  const int32_t ylo = max(0, cs * cy - 2), yhi = min(v.dy - 1, cs * cy + cs - 1);
  const int32_t zlo = max(0, cs * cz - 2), zhi = min(v.dz - 1, cs * cz + cs - 1);
  for (int32_t z = zlo; z <= zhi; ++z)
    for (int32_t y = ylo; y <= yhi; ++y) {
      const int64_t row = (int64_t)y + (int64_t)v.dy * z;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const uint32_t* rowp = planes + ((int64_t)p * rows + row) * wb;
        uint32_t w[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = plane_word(rowp, w0 + k, wb);
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[p][k] |= __funnelshift_r(w[k], w[k + 1], sh);
      }
    }
  const uint32_t wmask = (1u << (cs + 2)) - 1u;
  uint32_t word = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int32_t idx = cs * k;  // window of cell 16*wx + k in acc
    const int32_t q = idx >> 5, r = idx & 31;
    uint32_t bits = 0;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const uint32_t lo = q == 0 ? acc[p][0] : (q == 1 ? acc[p][1] : (q == 2 ? acc[p][2] : acc[p][3]));
      const uint32_t hi = q == 0 ? acc[p][1] : (q == 1 ? acc[p][2] : (q == 2 ? acc[p][3] : acc[p][4]));
      if (__funnelshift_r(lo, hi, r) & wmask) bits |= 1u << p;
    }
    word |= bits << (2 * k);
  }
  near[idx] = word;
}

// One thread per near word, a flat grid over the nwx * nny * nnz words.
__global__ void __launch_bounds__(256) near_pack_kernel(const uint32_t* __restrict__ planes, VolView v,
                                                        uint32_t* __restrict__ near) {
  near_word(planes, v, near, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Every subject of a batch in one launch: subject i's words in blocks of 256
// from its first block on.
__global__ void __launch_bounds__(256) near_pack_batch_kernel(const __grid_constant__ PrepTable tbl) {
  const int64_t b = blockIdx.x;
  const PrepSubject& S = tbl.s[subject_of<true>(tbl, b)];
  near_word(S.planes, S.v, const_cast<uint32_t*>(S.v.near), (b - S.near_blk0) * 256 + threadIdx.x);
}

static int grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

cudaError_t launch_volume_max(const int32_t* roi, const uint16_t* lab, int64_t nvox, DevState* st,
                              cudaStream_t s) {
  volume_max_kernel<<<grid_for(nvox), 256, 0, s>>>(roi, lab, nvox, st);
  return cudaGetLastError();
}

cudaError_t launch_volume_prep(const int32_t* roi, const uint16_t* lab, int64_t nvox, VolView v,
                               uint32_t* code, uint16_t* lab_out, uint32_t* bricks, uint32_t* planes, DevState* st,
                               cudaStream_t s) {
  (void)nvox;
  const int64_t groups = (int64_t)row_groups(v) * plane_groups(v);  // < 2^31 / 32
  const int64_t gy = groups < 65535 ? groups : 65535;
  const int64_t gz = (groups + gy - 1) / gy;
  volume_prep_kernel<<<dim3((v.dx + 31) / 32, (unsigned)gy, (unsigned)gz), dim3(32, kPrepRows), 0, s>>>(
      roi, lab, v, code, lab_out, bricks, planes, st);
  return cudaGetLastError();
}

int64_t plane_words(int32_t dx, int32_t dy, int32_t dz) {
  return 2 * (int64_t)((dx + 31) / 32) * dy * dz;
}

cudaError_t launch_near(const VolView& v, const uint32_t* planes, uint32_t* near, cudaStream_t s) {
  const int64_t words = (int64_t)v.nwx * v.nny * v.nnz;
  near_pack_kernel<<<(unsigned)((words + 255) / 256), 256, 0, s>>>(planes, v, near);
  return cudaGetLastError();
}

void prep_table_blocks(PrepTable& tbl) {
  int64_t pb = 0, nb = 0;
  for (int32_t i = 0; i < tbl.n; ++i) {
    PrepSubject& S = tbl.s[i];
    S.prep_blk0 = pb;
    S.near_blk0 = nb;
    pb += (int64_t)((S.v.dx + 31) / 32) * row_groups(S.v) * plane_groups(S.v);
    nb += ((int64_t)S.v.nwx * S.v.nny * S.v.nnz + 255) / 256;
  }
  tbl.prep_blocks = pb;
  tbl.near_blocks = nb;
}

cudaError_t launch_volume_prep_batch(const PrepTable& tbl, cudaStream_t s) {
  if (tbl.n <= 0 || tbl.prep_blocks <= 0) return cudaSuccess;
  volume_prep_batch_kernel<<<(unsigned)tbl.prep_blocks, dim3(32, kPrepRows), 0, s>>>(tbl);
  return cudaGetLastError();
}

cudaError_t launch_near_batch(const PrepTable& tbl, cudaStream_t s) {
  if (tbl.n <= 0 || tbl.near_blocks <= 0) return cudaSuccess;
  near_pack_batch_kernel<<<(unsigned)tbl.near_blocks, 256, 0, s>>>(tbl);
  return cudaGetLastError();
}

}  // namespace fc
