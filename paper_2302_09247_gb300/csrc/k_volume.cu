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

}  // namespace fc
