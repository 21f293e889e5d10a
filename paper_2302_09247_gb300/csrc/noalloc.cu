// fastcod_connectivity_noalloc: C and C_end of one subject without any device
// allocation, for callers that cannot allocate device memory themselves or
// through the library (see fastcod.h).  Its working memory is one
// file-scope device array of fixed size; every call on a device shares it.
#include <cuda_runtime.h>

#include "fc_ctx.h"
#include "fc_device.cuh"

namespace {

constexpr int32_t kNaMaxRoi = 16384;    // largest N accepted
constexpr int32_t kNaMaxLabels = 1023;  // largest M accepted
constexpr int32_t kNaCtas = 32;         // CTAs of the walk, one scratch slice each
constexpr int64_t kNaHeaderWords = 64;  // error word, error info
constexpr int64_t kNaSliceWords =
    (kNaMaxRoi + 31) / 32 + (kNaMaxLabels + 1 + 31) / 32 + kNaMaxRoi + (kNaMaxLabels + 1);
constexpr int64_t kNaWords = kNaHeaderWords + kNaCtas * kNaSliceWords;  // 574,528 words = 2.3 MB

// The scratch.  In host code this name is a host-side stand-in, not a device
// address: the host passes the address cudaGetSymbolAddress returns.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaWords];

struct NaArgs {
  const int32_t* roi;
  const uint16_t* lab;
  int32_t dx, dy, dz, n_roi, n_lab;
  const int32_t* xyz;
  const int64_t* off;
  int64_t nv, ns;
  int32_t* C;
  int32_t* Cend;
};

__device__ __forceinline__ void na_error(uint32_t* header, int32_t code, int32_t info) {
  int32_t* h = reinterpret_cast<int32_t*>(header);
  if (atomicCAS(h, 0, code) == 0) atomicExch(h + 1, info);
}

// grid (x blocks, rows): every voxel's row and label in range; the grid's y
// and z blocks together number the Dy * Dz rows
__global__ void __launch_bounds__(128) na_validate_kernel(NaArgs a, uint32_t* scratch) {
  const int64_t row = (int64_t)blockIdx.z * gridDim.y + blockIdx.y;
  const int32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.dx || row >= (int64_t)a.dy * a.dz) return;
  const int32_t i = x + a.dx * (int32_t)row;
  const int32_t r = a.roi[i], l = (int32_t)a.lab[i];
  if (r < -1 || r >= a.n_roi || l > a.n_lab) na_error(scratch, fc::kErrVolume, i);
}

__device__ __forceinline__ void na_visit(const NaArgs& a, uint32_t* rowbits, uint32_t* labbits, int32_t* rowlist,
                                         int32_t* lablist, int* nV, int* nT, int32_t x, int32_t y, int32_t z) {
  if ((unsigned)x >= (unsigned)a.dx || (unsigned)y >= (unsigned)a.dy || (unsigned)z >= (unsigned)a.dz) return;
  const int32_t i = x + a.dx * (y + a.dy * z);
  const int32_t r = __ldg(a.roi + i), l = (int32_t)__ldg(a.lab + i);
  if (r >= 0 && r < a.n_roi) {
    const uint32_t m = 1u << (r & 31);
    if (!(atomicOr(rowbits + (r >> 5), m) & m)) rowlist[atomicAdd(nV, 1)] = r;
  }
  if (l >= 1 && l <= a.n_lab) {
    const uint32_t m = 1u << (l & 31);
    if (!(atomicOr(labbits + (l >> 5), m) & m)) lablist[atomicAdd(nT, 1)] = l;
  }
}

// One CTA per streamline (grid-stride), the sets in the CTA's scratch slice.
__global__ void __launch_bounds__(256) na_walk_kernel(NaArgs a, uint32_t* scratch) {
  __shared__ int nV, nT, bad;
  uint32_t* header = scratch;
  uint32_t* rowbits = scratch + kNaHeaderWords + blockIdx.x * kNaSliceWords;
  uint32_t* labbits = rowbits + ((int64_t)a.n_roi + 31) / 32;
  int32_t* rowlist = reinterpret_cast<int32_t*>(labbits + ((int64_t)a.n_lab + 1 + 31) / 32);
  int32_t* lablist = rowlist + a.n_roi;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (a.off[0] != 0 || a.off[a.ns] != a.nv))
    na_error(header, fc::kErrOffsets, -1);
  for (int64_t s = blockIdx.x; s < a.ns; s += gridDim.x) {
    const int64_t b0 = a.off[s], b1 = a.off[s + 1];
    if (b0 < 0 || b1 < b0 || b1 > a.nv) {
      if (threadIdx.x == 0) na_error(header, fc::kErrOffsets, (int32_t)s);
      continue;  // uniform: every thread read the same offsets
    }
    if (threadIdx.x == 0) { nV = 0; nT = 0; bad = 0; }
    __syncthreads();
    for (int64_t j = b0 + threadIdx.x; j < b1; j += blockDim.x)
      for (int k = 0; k < 3; ++k) {
        const int32_t c = a.xyz[3 * j + k];
        if (c < -fc::kCoordLimit || c >= fc::kCoordLimit) bad = 1;
      }
    __syncthreads();
    const int skip = bad;
    __syncthreads();  // every thread has read the flag before thread 0 resets it
    if (skip) {
      if (threadIdx.x == 0) na_error(header, fc::kErrCoord, (int32_t)s);
      continue;
    }
    const int64_t T = b1 - b0;
    const int64_t units = T == 1 ? 1 : T - 1;
    for (int64_t u = threadIdx.x; u < units && T >= 1; u += blockDim.x) {
      int32_t p0[3] = {a.xyz[3 * (b0 + u)], a.xyz[3 * (b0 + u) + 1], a.xyz[3 * (b0 + u) + 2]};
      if (T == 1) {
        na_visit(a, rowbits, labbits, rowlist, lablist, &nV, &nT, p0[0] >> fc::kUnitLog2, p0[1] >> fc::kUnitLog2,
                 p0[2] >> fc::kUnitLog2);
        continue;
      }
      int32_t p1[3] = {a.xyz[3 * (b0 + u + 1)], a.xyz[3 * (b0 + u + 1) + 1], a.xyz[3 * (b0 + u + 1) + 2]};
      fc::SegWalk<unsigned long long> w;
      w.init(p0, p1);
      na_visit(a, rowbits, labbits, rowlist, lablist, &nV, &nT, w.cx, w.cy, w.cz);
      while (w.step()) na_visit(a, rowbits, labbits, rowlist, lablist, &nV, &nT, w.cx, w.cy, w.cz);
    }
    __syncthreads();
    const int64_t M = a.n_lab;
    const int64_t pairs = (int64_t)nV * nT;
    for (int64_t p = threadIdx.x; p < pairs; p += blockDim.x) {
      const int64_t r = p / nT, k = p - r * nT;
      atomicAdd(a.C + (int64_t)rowlist[r] * M + (lablist[k] - 1), 1);
    }
    if (threadIdx.x == 0 && T >= 1) {
      const int32_t* q0 = a.xyz + 3 * b0;
      const int32_t* q1 = a.xyz + 3 * (b1 - 1);
      const int32_t x0 = q0[0] >> fc::kUnitLog2, y0 = q0[1] >> fc::kUnitLog2, z0 = q0[2] >> fc::kUnitLog2;
      const int32_t x1 = q1[0] >> fc::kUnitLog2, y1 = q1[1] >> fc::kUnitLog2, z1 = q1[2] >> fc::kUnitLog2;
      int32_t r0 = -1, l1 = 0;
      if ((unsigned)x0 < (unsigned)a.dx && (unsigned)y0 < (unsigned)a.dy && (unsigned)z0 < (unsigned)a.dz)
        r0 = a.roi[x0 + a.dx * (y0 + a.dy * z0)];
      if ((unsigned)x1 < (unsigned)a.dx && (unsigned)y1 < (unsigned)a.dy && (unsigned)z1 < (unsigned)a.dz)
        l1 = (int32_t)a.lab[x1 + a.dx * (y1 + a.dy * z1)];
      if (r0 >= 0 && r0 < a.n_roi && l1 >= 1 && l1 <= a.n_lab) atomicAdd(a.Cend + (int64_t)r0 * M + (l1 - 1), 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nV; k += blockDim.x) rowbits[rowlist[k] >> 5] = 0u;
    for (int k = threadIdx.x; k < nT; k += blockDim.x) labbits[lablist[k] >> 5] = 0u;
    __syncthreads();
  }
}

// The scratch's device address on the current device, looked up on every
// call: cudaGetSymbolAddress allocates nothing and is cheap, and an address
// cached across calls would go stale if the caller reset the device (the
// module, and with it the array, is loaded again afterwards).  The first
// lookup on a device loads the library's device code there (lazy module
// loading), so the first call on a device should come before any stream
// capture.
cudaError_t scratch_address(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<uint32_t*>(p);
  return cudaSuccess;
}

int na_fail(int code, const char* msg) {
  fcapi::thread_error() = msg;
  return code;
}

}  // namespace

extern "C" {

FASTCOD_API int fastcod_connectivity_noalloc(int cuda_device, void* cuda_stream, const int32_t* roi_index_map,
                                             const uint16_t* target_labels, int32_t dim_x, int32_t dim_y,
                                             int32_t dim_z, int32_t n_roi, int32_t n_targets, const int32_t* xyz,
                                             int64_t n_vertices, const int64_t* offsets, int64_t n_streamlines,
                                             int32_t* C_out, int32_t* Cend_out) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev || cuda_device >= 64) {
    (void)cudaGetLastError();
    return na_fail(FASTCOD_EINVAL, "no such CUDA device");
  }
  if (dim_x <= 0 || dim_y <= 0 || dim_z <= 0 || (int64_t)dim_x * dim_y * dim_z >= ((int64_t)1 << 31))
    return na_fail(FASTCOD_EINVAL, "invalid grid dims");
  if (n_roi < 1 || n_roi > kNaMaxRoi || n_targets < 1 || n_targets > kNaMaxLabels)
    return na_fail(FASTCOD_EINVAL,
                   "fastcod_connectivity_noalloc takes 1 <= n_roi <= 16384 and 1 <= n_targets <= 1023 "
                   "(its fixed scratch); use the context API for larger problems");
  if (n_streamlines < 0 || n_vertices < 0 || n_vertices > 0x7fffffffLL)
    return na_fail(FASTCOD_EINVAL, "invalid streamline counts");
  if (cudaSetDevice(cuda_device) != cudaSuccess) {
    (void)cudaGetLastError();
    return na_fail(FASTCOD_ECUDA, "cudaSetDevice failed");
  }
  const void* ptrs[6] = {roi_index_map, target_labels, offsets, C_out, Cend_out,
                         n_vertices ? static_cast<const void*>(xyz) : static_cast<const void*>(offsets)};
  for (const void* p : ptrs)
    if (!p || fcapi::ptr_kind(p, cuda_device) != 1)
      return na_fail(FASTCOD_EINVAL, "fastcod_connectivity_noalloc takes device memory of cuda_device only");
  uint32_t* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return na_fail(FASTCOD_ECUDA, "cudaGetSymbolAddress of the scratch failed");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t nm = (size_t)n_roi * (size_t)n_targets;
  NaArgs a{roi_index_map, target_labels, dim_x, dim_y, dim_z, n_roi, n_targets, xyz, offsets,
           n_vertices, n_streamlines, C_out, Cend_out};
  e = cudaMemsetAsync(C_out, 0, nm * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Cend_out, 0, nm * 4, s);
  // the previous call's contents: the error word and any set bits start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, (size_t)kNaWords * 4, s);
  if (e == cudaSuccess) {
    const int64_t rows = (int64_t)dim_y * dim_z, gy = rows < 65535 ? rows : 65535;
    na_validate_kernel<<<dim3((dim_x + 127) / 128, (unsigned)gy, (unsigned)((rows + gy - 1) / gy)), 128, 0, s>>>(
        a, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n_streamlines > 0) {
    na_walk_kernel<<<kNaCtas, 256, 0, s>>>(a, scratch);
    e = cudaGetLastError();
  }
  int32_t hdr[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(hdr, scratch, sizeof hdr, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return na_fail(FASTCOD_ECUDA, cudaGetErrorString(e));
  }
  switch (hdr[0]) {
    case fc::kErrNone:
      return FASTCOD_OK;
    case fc::kErrOffsets:
      return na_fail(FASTCOD_EINVAL, "offsets invalid");
    case fc::kErrCoord:
      return na_fail(FASTCOD_EINVAL, "vertex coordinate outside [-2^24, 2^24)");
    case fc::kErrVolume:
      return na_fail(FASTCOD_EINVAL, "volume value out of range");
    default:
      return na_fail(FASTCOD_ECUDA, "device error");
  }
}

}  // extern "C"
