// K1: volume preparation.  From the caller's ROI index map (int32) and target
// label volume (uint16) build the per-voxel code, a private label copy, the
// brick occupancy bits and the near grid, validating every voxel on the way
// (Section 2: the ROI voxel set V and the target regions R that loc2region
// reads).  Launch grids are (x blocks, rows, planes), so every thread knows
// its voxel without a division.
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

__global__ void __launch_bounds__(128) volume_prep_kernel(const int32_t* __restrict__ roi,
                                                          const uint16_t* __restrict__ lab, VolView v,
                                                          uint32_t* __restrict__ code,
                                                          uint16_t* __restrict__ lab_out,
                                                          uint32_t* __restrict__ bricks, DevState* st) {
  const int32_t x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= v.dx) return;
  const int32_t i = x + v.dx * (y + v.dy * z);
  const int32_t r = roi[i];
  const int32_t l = (int32_t)lab[i];
  if (r < -1 || r >= v.n_roi || l > v.n_lab) {
    set_error(st, kErrVolume, i);
    return;
  }
  code[i] = r >= 0 ? (kCodeRoi | (l > 0 ? kCodeRoiLabelled : 0u) | (uint32_t)r) : (uint32_t)l;
  lab_out[i] = (uint16_t)l;
  const uint32_t bits = (r >= 0 ? 1u : 0u) | (l > 0 ? 2u : 0u);
  if (bits) {
    const int32_t b = (x >> kBrickLog2) + v.bx * ((y >> kBrickLog2) + v.by * (z >> kBrickLog2));
    atomicOr(bricks + (b >> 4), bits << ((b & 15) * 2));
  }
}

// ---------------------------------------------------------------- near grid
// Occupancy bits of every voxel on the padded grid (zero border), then an OR
// over +-1 along x, y and z in turn (the 3x3x3 dilation), then ORed over the
// cells and packed sixteen cells per word.

__global__ void __launch_bounds__(128) near_seed_kernel(const uint32_t* __restrict__ code, VolView v,
                                                        uint8_t* __restrict__ pad) {
  const int32_t x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= v.dx) return;
  const uint32_t c = code[x + v.dx * (y + v.dy * z)];
  const uint8_t bits = (c & kCodeRoi) ? (uint8_t)(1u | ((c & kCodeRoiLabelled) ? 2u : 0u)) : (uint8_t)(c ? 2u : 0u);
  const int32_t px = v.dx + 2, py = v.dy + 2;
  pad[(x + 1) + px * ((y + 1) + py * (z + 1))] = bits;
}

// grid (x blocks, py, pz) over the padded grid
__global__ void __launch_bounds__(128) near_dilate_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                                          int32_t px, int32_t py, int32_t pz, int axis) {
  const int32_t x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= px) return;
  const int32_t i = x + px * (y + py * z);
  const int32_t c = axis == 0 ? x : (axis == 1 ? y : z);
  const int32_t extent = axis == 0 ? px : (axis == 1 ? py : pz);
  const int32_t stride = axis == 0 ? 1 : (axis == 1 ? px : px * py);
  uint8_t b = in[i];
  if (c > 0) b |= in[i - stride];
  if (c + 1 < extent) b |= in[i + stride];
  out[i] = b;
}

// grid (word blocks, nny, nnz): one thread per 16-cell word
__global__ void __launch_bounds__(128) near_pack_kernel(const uint8_t* __restrict__ in, VolView v,
                                                        uint32_t* __restrict__ near) {
  const int32_t wx = blockIdx.x * blockDim.x + threadIdx.x, cy = blockIdx.y, cz = blockIdx.z;
  if (wx >= v.nwx) return;
  const int32_t px = v.dx + 2, py = v.dy + 2, pz = v.dz + 2;
  const int32_t cs = 1 << v.nsh;
  const int32_t y1 = min(py, (cy + 1) * cs), z1 = min(pz, (cz + 1) * cs);
  uint32_t word = 0;
  for (int k = 0; k < 16; ++k) {
    const int32_t x0 = (wx * 16 + k) * cs, x1 = min(px, x0 + cs);
    uint32_t bits = 0;
    for (int32_t z = cz * cs; z < z1; ++z)
      for (int32_t y = cy * cs; y < y1; ++y)
        for (int32_t x = x0; x < x1; ++x) bits |= in[x + px * (y + py * z)];
    word |= bits << (2 * k);
  }
  near[wx + v.nwx * (cy + v.nny * cz)] = word;
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
  (void)nvox;
  volume_prep_kernel<<<dim3((v.dx + 127) / 128, v.dy, v.dz), 128, 0, s>>>(roi, lab, v, code, lab_out, bricks, st);
  return cudaGetLastError();
}

cudaError_t launch_near(const VolView& v, uint8_t* tmp, uint32_t* near, cudaStream_t s) {
  const int32_t px = v.dx + 2, py = v.dy + 2, pz = v.dz + 2;
  const int64_t n = (int64_t)px * py * pz;
  uint8_t* a = tmp;
  uint8_t* b = tmp + n;
  cudaError_t e = cudaMemsetAsync(a, 0, (size_t)n, s);
  if (e != cudaSuccess) return e;
  near_seed_kernel<<<dim3((v.dx + 127) / 128, v.dy, v.dz), 128, 0, s>>>(v.code, v, a);
  const dim3 pg((px + 127) / 128, py, pz);
  near_dilate_kernel<<<pg, 128, 0, s>>>(a, b, px, py, pz, 0);
  near_dilate_kernel<<<pg, 128, 0, s>>>(b, a, px, py, pz, 1);
  near_dilate_kernel<<<pg, 128, 0, s>>>(a, b, px, py, pz, 2);
  near_pack_kernel<<<dim3((v.nwx + 127) / 128, v.nny, v.nnz), 128, 0, s>>>(b, v, near);
  return cudaGetLastError();
}

}  // namespace fc
