// K1: volume preparation.  From the caller's ROI index map (int32) and target
// label volume (uint16) build the per-voxel code, a private label copy and
// the brick occupancy bits, validating every voxel on the way (Section 2:
// the ROI voxel set V and the target regions R that loc2region reads).
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

__global__ void __launch_bounds__(256) volume_prep_kernel(const int32_t* __restrict__ roi,
                                                          const uint16_t* __restrict__ lab,
                                                          int64_t nvox, VolView v,
                                                          uint32_t* __restrict__ code,
                                                          uint16_t* __restrict__ lab_out,
                                                          uint32_t* __restrict__ bricks,
                                                          DevState* st) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvox;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = roi[i];
    const int32_t l = (int32_t)lab[i];
    if (r < -1 || r >= v.n_roi || l > v.n_lab) {
      set_error(st, kErrVolume, (int32_t)min(i, (int64_t)0x7fffffff));
      continue;
    }
    uint32_t c;
    if (r >= 0)
      c = kCodeRoi | (l > 0 ? kCodeRoiLabelled : 0u) | (uint32_t)r;
    else
      c = (uint32_t)l;
    code[i] = c;
    lab_out[i] = (uint16_t)l;
    const uint32_t bits = (r >= 0 ? 1u : 0u) | (l > 0 ? 2u : 0u);
    if (bits) {
      const int32_t x = (int32_t)(i % v.dx);
      const int32_t y = (int32_t)((i / v.dx) % v.dy);
      const int32_t z = (int32_t)(i / ((int64_t)v.dx * v.dy));
      const int32_t b = (x >> kBrickLog2) + v.bx * ((y >> kBrickLog2) + v.by * (z >> kBrickLog2));
      atomicOr(bricks + (b >> 4), bits << ((b & 15) * 2));
    }
  }
}

// ---------------------------------------------------------------- near grid
// Occupancy bits of every voxel on the padded grid (zero border), then an OR
// over +-1 along x, y and z in turn (the 3x3x3 dilation), then packed.

__global__ void near_seed_kernel(const uint32_t* __restrict__ code, VolView v, uint8_t* __restrict__ pad) {
  const int64_t nvox = (int64_t)v.dx * v.dy * v.dz;
  const int32_t px = v.dx + 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvox; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = code[i];
    const uint8_t bits = (c & kCodeRoi) ? (uint8_t)(1u | ((c & kCodeRoiLabelled) ? 2u : 0u)) : (uint8_t)(c ? 2u : 0u);
    const int32_t x = (int32_t)(i % v.dx);
    const int32_t y = (int32_t)((i / v.dx) % v.dy);
    const int32_t z = (int32_t)(i / ((int64_t)v.dx * v.dy));
    pad[(x + 1) + (int64_t)px * ((y + 1) + (int64_t)(v.dy + 2) * (z + 1))] = bits;
  }
}

__global__ void near_dilate_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int32_t px,
                                   int32_t py, int32_t pz, int axis) {
  const int64_t n = (int64_t)px * py * pz;
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? px : (int64_t)px * py);
  const int32_t extent = axis == 0 ? px : (axis == 1 ? py : pz);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = (int32_t)((i / stride) % extent);
    uint8_t b = in[i];
    if (c > 0) b |= in[i - stride];
    if (c + 1 < extent) b |= in[i + stride];
    out[i] = b;
  }
}

__global__ void near_pack_kernel(const uint8_t* __restrict__ in, VolView v, uint32_t* __restrict__ near) {
  const int32_t px = v.dx + 2, py = v.dy + 2, pz = v.dz + 2;
  const int32_t cs = 1 << v.nsh;
  const int64_t nwords = (int64_t)v.nwx * v.nny * v.nnz;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
    const int32_t wx = (int32_t)(w % v.nwx);
    const int32_t cy = (int32_t)((w / v.nwx) % v.nny);
    const int32_t cz = (int32_t)(w / ((int64_t)v.nwx * v.nny));
    uint32_t word = 0;
    for (int k = 0; k < 16; ++k) {
      const int32_t cx = wx * 16 + k;
      uint32_t bits = 0;
      for (int32_t z = cz * cs; z < min(pz, (cz + 1) * cs); ++z)
        for (int32_t y = cy * cs; y < min(py, (cy + 1) * cs); ++y)
          for (int32_t x = cx * cs; x < min(px, (cx + 1) * cs); ++x)
            bits |= in[x + (int64_t)px * (y + (int64_t)py * z)];
      word |= bits << (2 * k);
    }
    near[w] = word;
  }
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
                               uint32_t* code, uint16_t* lab_out, uint32_t* bricks, DevState* st,
                               cudaStream_t s) {
  volume_prep_kernel<<<grid_for(nvox), 256, 0, s>>>(roi, lab, nvox, v, code, lab_out, bricks, st);
  return cudaGetLastError();
}

cudaError_t launch_near(const VolView& v, uint8_t* tmp, uint32_t* near, cudaStream_t s) {
  const int32_t px = v.dx + 2, py = v.dy + 2, pz = v.dz + 2;
  const int64_t n = (int64_t)px * py * pz;
  uint8_t* a = tmp;
  uint8_t* b = tmp + n;
  cudaError_t e = cudaMemsetAsync(a, 0, (size_t)n, s);
  if (e != cudaSuccess) return e;
  near_seed_kernel<<<grid_for((int64_t)v.dx * v.dy * v.dz), 256, 0, s>>>(v.code, v, a);
  near_dilate_kernel<<<grid_for(n), 256, 0, s>>>(a, b, px, py, pz, 0);
  near_dilate_kernel<<<grid_for(n), 256, 0, s>>>(b, a, px, py, pz, 1);
  near_dilate_kernel<<<grid_for(n), 256, 0, s>>>(a, b, px, py, pz, 2);
  near_pack_kernel<<<grid_for((int64_t)v.nwx * v.nny * v.nnz), 256, 0, s>>>(b, v, near);
  return cudaGetLastError();
}

}  // namespace fc
