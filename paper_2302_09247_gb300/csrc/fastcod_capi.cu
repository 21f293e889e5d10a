// libfastcod C ABI: context, validation, buffers, launches (see fastcod.h).
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fc_ctx.h"

namespace fcapi {

int fail(fastcod_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int ptr_kind(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == dev ? 1 : -1;
  return 0;
}

const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int grow(fastcod_ctx* c, void** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return FASTCOD_OK;
  size_t n = need < 256 ? 256 : need;
  if (*p) {
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaFree(*p));
    *p = nullptr;
    *cap = 0;
  }
  CU(cudaMalloc(p, n));
  *cap = n;
  return FASTCOD_OK;
}

std::string& thread_error() {
  static thread_local std::string msg;
  return msg;
}

}  // namespace fcapi

namespace {

using fcapi::fail;
using fcapi::grow;
using fcapi::mapped_host;
using fcapi::ptr_kind;
using fcapi::sync_check;


void free_volumes(fastcod_ctx* c) {
  cudaFree(c->d_code);
  cudaFree(c->d_lab);
  cudaFree(c->d_bricks);
  cudaFree(c->d_near);
  cudaFree(c->d_C);  // C_end shares this allocation
  cudaFree(c->d_scratch);
  c->d_code = nullptr;
  c->d_lab = nullptr;
  c->d_bricks = nullptr;
  c->d_near = nullptr;
  c->d_C = nullptr;
  c->d_Cend = nullptr;
  c->d_scratch = nullptr;
  c->has_vol = false;
}

void collect_profile(fastcod_ctx* c);

int read_state(fastcod_ctx* c, DevState* h) {
  CU(cudaMemcpyAsync(h, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  collect_profile(c);
  return FASTCOD_OK;
}

}  // namespace

// Synchronise and turn a device-detected error into a status.
int fcapi::sync_check(fastcod_ctx* c) {
  DevState h;
  int rc = read_state(c, &h);
  if (rc) return rc;
  switch (h.error) {
    case fc::kErrNone:
      return FASTCOD_OK;
    case fc::kErrOffsets:
      return fail(c, FASTCOD_EINVAL,
                  "offsets invalid near streamline %d: need offsets[0]=0, non-decreasing, offsets[n]=n_vertices",
                  h.error_info);
    case fc::kErrCoord:
      return fail(c, FASTCOD_EINVAL, "vertex coordinate outside [-2^24, 2^24) (warp range %d)", h.error_info);
    case fc::kErrVolume:
      return fail(c, FASTCOD_EINVAL, "volume value out of range at voxel %d", h.error_info);
    case fc::kErrTimeout:
      return fail(c, FASTCOD_ETIMEOUT, "device wait timed out (warp %d)", h.error_info);
    case fc::kErrChecked:
      return fail(c, FASTCOD_ECUDA, "bounds check failed (site %d)", h.error_info);
    default:
      return fail(c, FASTCOD_ECUDA, "device error %d (%d)", h.error, h.error_info);
  }
}

namespace {

fc::VolView vol_view(const fastcod_ctx* c) {
  fc::VolView v;
  v.code = c->d_code;
  v.lab = c->d_lab;
  v.bricks = c->d_bricks;
  v.near = c->d_near;
  v.dx = c->dims[0];
  v.dy = c->dims[1];
  v.dz = c->dims[2];
  v.bx = c->bdims[0];
  v.by = c->bdims[1];
  v.bz = c->bdims[2];
  fc::set_near_dims(v, c->near_shift);
  v.n_roi = c->N;
  v.n_lab = c->M;
  return v;
}

// Bytes from C to C_end in their shared allocation.
size_t accum_stride_bytes(size_t nm) { return nm ? (nm * 4 + 255) & ~(size_t)255 : 256; }

// Stream-ordered zeroing of C, C_end and every device counter (the error
// word included).
int zero_accumulators(fastcod_ctx* c) {
  const size_t nm = (size_t)c->N * (size_t)c->M;
  if (nm) CU(cudaMemsetAsync(c->d_C, 0, accum_stride_bytes(nm) + nm * 4, c->stream));
  CU(cudaMemsetAsync(c->d_state, 0, sizeof(DevState), c->stream));
  c->total_streamlines = 0;
  c->total_vertices = 0;
  return FASTCOD_OK;
}

// Fold the events of the profiled calls into the totals (the stream has been
// synchronised).
void collect_profile(fastcod_ctx* c) {
  for (size_t k = 0; k < c->ev_used; ++k) {
    float ms[4] = {0, 0, 0, 0};
    for (int i = c->ev_pool[k].no_h2d ? 1 : 0; i < 4; ++i)
      if (cudaEventElapsedTime(&ms[i], c->ev_pool[k].e[i], c->ev_pool[k].e[i + 1]) != cudaSuccess) {
        (void)cudaGetLastError();
        ms[i] = 0;
      }
    c->prof.ms_h2d += ms[0];
    c->prof.ms_prefilter += ms[1];
    c->prof.ms_walk += ms[2];
    c->prof.ms_overflow += ms[3];
    c->prof.calls += 1;
  }
  c->ev_used = 0;
}

// Pick the event set of this call: a new one while the pool is below 256
// sets, else fold the pending ones first (one synchronisation per 256 calls).
int begin_profiled_call(fastcod_ctx* c) {
  c->ev_cur = nullptr;
  if (!c->profile) return FASTCOD_OK;
  if (c->ev_used == c->ev_pool.size()) {
    if (c->ev_pool.size() < 256) {
      fastcod_ctx::EvSet set;
      for (int i = 0; i < 5; ++i) CU(cudaEventCreate(&set.e[i]));
      c->ev_pool.push_back(set);
    } else {
      CU(cudaStreamSynchronize(c->stream));
      collect_profile(c);
    }
  }
  c->ev_cur = &c->ev_pool[c->ev_used++];
  c->ev_cur->no_h2d = false;
  return FASTCOD_OK;
}

int record(fastcod_ctx* c, int i) {
  if (c->ev_cur) CU(cudaEventRecord(c->ev_cur->e[i], c->stream));
  return FASTCOD_OK;
}

int copy_out(fastcod_ctx* c, const int32_t* src, int32_t* dst) {
  if (!c->has_vol) return fail(c, FASTCOD_ESTATE, "no volumes installed");
  int rc = sync_check(c);
  if (rc) return rc;
  const size_t nm = (size_t)c->N * (size_t)c->M;
  if (!nm) return FASTCOD_OK;
  if (!dst) return fail(c, FASTCOD_EINVAL, "output pointer is NULL");
  if (ptr_kind(dst, c->device) < 0) return fail(c, FASTCOD_EINVAL, "output is device memory of another device");
  CU(cudaMemcpyAsync(dst, src, nm * 4, cudaMemcpyDefault, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return FASTCOD_OK;
}

}  // namespace

extern "C" {

FASTCOD_API int fastcod_create(fastcod_ctx** out, int cuda_device, uint32_t flags) {
  if (!out) {
    fcapi::thread_error() = "out is NULL";
    return FASTCOD_EINVAL;
  }
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
    (void)cudaGetLastError();
    fcapi::thread_error() = "no such CUDA device";
    return FASTCOD_EINVAL;
  }
  fastcod_ctx* c = new (std::nothrow) fastcod_ctx();
  if (!c) {
    fcapi::thread_error() = "host allocation failed";
    return FASTCOD_ENOMEM;
  }
  c->device = cuda_device;
  c->flags = flags;
  int rc = FASTCOD_OK;
  do {
    if (cudaSetDevice(cuda_device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
      rc = FASTCOD_ECUDA;
      break;
    }
    c->stream = c->own_stream;
    if (cudaMalloc(&c->d_state, sizeof(DevState)) != cudaSuccess) {
      rc = FASTCOD_ENOMEM;
      break;
    }
    cudaMemsetAsync(c->d_state, 0, sizeof(DevState), c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) rc = FASTCOD_ECUDA;
  } while (0);
  if (rc) {
    fcapi::thread_error() = std::string("CUDA initialisation failed: ") + cudaGetErrorString(cudaGetLastError());
    fastcod_destroy(c);
    return rc;
  }
  *out = c;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_destroy(fastcod_ctx* c) {
  if (!c) return FASTCOD_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_volumes(c);
  cudaFree(c->d_vstage);
  cudaFree(c->d_xyz);
  cudaFree(c->d_off);
  cudaFree(c->d_surv);
  cudaFree(c->d_ovf);
  for (int i = 0; i < fastcod_ctx::kAuxSlots; ++i) cudaFree(c->d_aux[i]);
  fcapi::batch_free(c);
  cudaFree(c->d_state);
  cudaFree(c->d_check);
  for (auto& set : c->ev_pool)
    for (int i = 0; i < 5; ++i) cudaEventDestroy(set.e[i]);
  for (cudaEvent_t e : c->aux_ev)
    if (e) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_set_stream(fastcod_ctx* c, void* s) {
  if (!c) return FASTCOD_EINVAL;
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  c->stream = s ? (cudaStream_t)s : c->own_stream;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_set_volumes(fastcod_ctx* c, const int32_t* roi, const uint16_t* lab, int32_t dx,
                                    int32_t dy, int32_t dz, int32_t n_roi, int32_t n_targets) {
  fcapi::Range nvtx_range("fastcod_set_volumes");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  if (dx <= 0 || dy <= 0 || dz <= 0) return fail(c, FASTCOD_EINVAL, "grid dims must be > 0");
  const int64_t nvox = (int64_t)dx * dy * dz;
  if (nvox >= ((int64_t)1 << 31)) return fail(c, FASTCOD_EINVAL, "grid has >= 2^31 voxels");
  if (!roi || !lab) return fail(c, FASTCOD_EINVAL, "volume pointer is NULL");
  if (n_roi < 0 || n_targets < 0) return fail(c, FASTCOD_EINVAL, "N and M must be >= 0");
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  const int kr = ptr_kind(roi, c->device), kl = ptr_kind(lab, c->device);
  if (kr < 0 || kl < 0) return fail(c, FASTCOD_EINVAL, "volume is device memory of another device");
  // device copies of host volumes
  const size_t rb = (size_t)nvox * 4, lb = (size_t)nvox * 2;
  const int32_t* d_roi = roi;
  const uint16_t* d_labin = lab;
  if (!kr || !kl) {
    int rc = grow(c, &c->d_vstage, &c->vstage_bytes, rb + lb);
    if (rc) return rc;
    if (!kr) {
      CU(cudaMemcpyAsync(c->d_vstage, roi, rb, cudaMemcpyHostToDevice, c->stream));
      d_roi = (const int32_t*)c->d_vstage;
    }
    if (!kl) {
      CU(cudaMemcpyAsync((char*)c->d_vstage + rb, lab, lb, cudaMemcpyHostToDevice, c->stream));
      d_labin = (const uint16_t*)((char*)c->d_vstage + rb);
    }
  }
  free_volumes(c);
  DevState h;
  memset(&h, 0, sizeof h);
  h.max_roi = -1;
  CU(cudaMemcpyAsync(c->d_state, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
  if (n_roi == 0 || n_targets == 0) {
    CU(fc::launch_volume_max(d_roi, d_labin, nvox, c->d_state, c->stream));
    int rc = read_state(c, &h);
    if (rc) return rc;
    if (n_roi == 0) n_roi = h.max_roi + 1;
    if (n_targets == 0) n_targets = h.max_label;
  }
  if (n_roi >= (1 << 30)) return fail(c, FASTCOD_EINVAL, "N must be < 2^30");
  if (n_targets > 65535) return fail(c, FASTCOD_EINVAL, "M must be < 65536");
  c->dims[0] = dx;
  c->dims[1] = dy;
  c->dims[2] = dz;
  for (int a = 0; a < 3; ++a) c->bdims[a] = (c->dims[a] + (1 << fc::kBrickLog2) - 1) >> fc::kBrickLog2;
  c->N = n_roi;
  c->M = n_targets;
  const int64_t nbricks = (int64_t)c->bdims[0] * c->bdims[1] * c->bdims[2];
  const size_t nm = (size_t)c->N * (size_t)c->M;
  CU(cudaMalloc(&c->d_code, rb));
  CU(cudaMalloc(&c->d_lab, lb));
  CU(cudaMalloc(&c->d_bricks, (size_t)((nbricks + 15) / 16) * 4));
  // C and C_end in one allocation (C_end at a 256-byte boundary), zeroed by
  // one memset
  CU(cudaMalloc(&c->d_C, 2 * accum_stride_bytes(nm)));
  c->d_Cend = c->d_C + accum_stride_bytes(nm) / 4;
  CU(cudaMemsetAsync(c->d_bricks, 0, (size_t)((nbricks + 15) / 16) * 4, c->stream));
  // exact global-memory path for streamlines whose sets outgrow shared memory
  const int64_t words = fc::overflow_scratch_words(c->N, c->M);
  int64_t ctas = 64;
  while (ctas > 1 && ctas * words * 4 > ((int64_t)256 << 20)) ctas /= 2;
  c->scratch_ctas = (int32_t)ctas;
  CU(cudaMalloc(&c->d_scratch, (size_t)(ctas * words * 4)));
  CU(cudaMemsetAsync(c->d_scratch, 0, (size_t)(ctas * words * 4), c->stream));
  // near grid (the prefilter's dilated occupancy), built from the bit planes
  c->near_shift = fc::resolve_near_log2(c->near_log2, dx, dy, dz);
  fc::VolView v = vol_view(c);
  CU(cudaMalloc(&c->d_near, (size_t)fc::near_words(v) * 4));
  v.near = c->d_near;
  uint32_t* planes = nullptr;
  CU(cudaMalloc(&planes, (size_t)fc::plane_words(dx, dy, dz) * 4));
  cudaError_t e = fc::launch_volume_prep(d_roi, d_labin, nvox, v, c->d_code, c->d_lab, c->d_bricks, planes,
                                         c->d_state, c->stream);
  if (e == cudaSuccess) e = fc::launch_near(v, planes, c->d_near, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(planes);
  CU(e);
  int rc = sync_check(c);
  if (rc) {
    free_volumes(c);
    return rc;
  }
  c->has_vol = true;
  return zero_accumulators(c);
}

FASTCOD_API int fastcod_add_streamlines(fastcod_ctx* c, const int32_t* xyz, int64_t nv, const int64_t* offsets,
                                        int64_t ns) {
  fcapi::Range nvtx_range("fastcod_add_streamlines");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  if (!c->has_vol) return fail(c, FASTCOD_ESTATE, "fastcod_set_volumes must come first");
  if (ns < 0 || nv < 0) return fail(c, FASTCOD_EINVAL, "negative count");
  if (ns == 0) return nv == 0 ? FASTCOD_OK : fail(c, FASTCOD_EINVAL, "vertices without streamlines");
  if (!offsets || (nv > 0 && !xyz)) return fail(c, FASTCOD_EINVAL, "input pointer is NULL");
  if (c->total_streamlines + ns > 0x7fffffffLL)
    return fail(c, FASTCOD_EOVERFLOW, "more than 2^31-1 streamlines since the last reset");
  if (nv > 0x7fffffffLL) return fail(c, FASTCOD_EINVAL, "more than 2^31-1 vertices in one call: split the call");
  CU(cudaSetDevice(c->device));
  const int kx = nv > 0 ? ptr_kind(xyz, c->device) : 1;
  const int ko = ptr_kind(offsets, c->device);
  if (kx < 0 || ko < 0) return fail(c, FASTCOD_EINVAL, "input is device memory of another device");
  // device xyz off a 16-byte boundary is copied to an aligned buffer first
  // (the prefilter's bulk copies and vector loads need aligned vertex rows)
  const bool unaligned = kx == 1 && nv > 0 && ((uintptr_t)xyz & 15u);
  const int32_t* d_xyz = xyz;
  const int64_t* d_off = offsets;
  if (int rc = begin_profiled_call(c)) return rc;
  // page-locked host xyz: read in place over the host link when allowed (the
  // offsets, read with dependent loads, are always copied)
  bool xyz_in_place = false;
  if (kx == 0 && c->host_in_place) {
    const void* m = mapped_host(xyz);
    if (m && !((uintptr_t)m & 15u)) {
      d_xyz = static_cast<const int32_t*>(m);
      xyz_in_place = true;
    }
  }
  // the copy stage is timed only when there is one (each recorded event costs
  // the stream a few microseconds)
  if ((kx == 0 && !xyz_in_place) || unaligned || ko == 0) {
    if (int rc = record(c, 0)) return rc;
  } else if (c->ev_cur) {
    c->ev_cur->no_h2d = true;
  }
  if ((kx == 0 && !xyz_in_place) || unaligned) {
    int rc = grow(c, (void**)&c->d_xyz, &c->xyz_bytes, (size_t)nv * 12 + 16);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->d_xyz, xyz, (size_t)nv * 12, cudaMemcpyDefault, c->stream));
    d_xyz = c->d_xyz;
  }
  if (ko == 0) {
    int rc = grow(c, (void**)&c->d_off, &c->off_bytes, (size_t)(ns + 1) * 8);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->d_off, offsets, (size_t)(ns + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    d_off = c->d_off;
  }
  {
    int rc = grow(c, (void**)&c->d_surv, &c->surv_bytes, (size_t)ns * 4);
    if (rc) return rc;
    rc = grow(c, (void**)&c->d_ovf, &c->ovf_bytes, (size_t)ns * 4);
    if (rc) return rc;
  }
  // per-call counters: n_survivors, n_overflow, work_next, work_task
  CU(cudaMemsetAsync(&c->d_state->n_survivors, 0, offsetof(DevState, voxel_steps) - offsetof(DevState, n_survivors),
                     c->stream));
  fc::Tract t;
  t.xyz = d_xyz;
  t.off = d_off;
  t.nv = nv;
  t.ns = ns;
  fc::VolView v = vol_view(c);
  fc::Accum acc;
  acc.C = c->d_C;
  acc.Cend = c->d_Cend;
  if (int rc = record(c, 1)) return rc;
  // bulk copies stage device-resident vertices; host-resident ones are read
  // with direct loads
  CU(fc::launch_prefilter(t, v, c->prefilter != 0, c->mode, c->staging_tma != 0 && !xyz_in_place, c->prefilter_ctas,
                          c->d_surv, ns, c->d_state, c->num_sms, c->stream, c->withhold_piece));
  if (int rc = record(c, 2)) return rc;
  CU(fc::launch_walk(t, v, c->d_surv, ns, acc, c->mode, c->d_ovf, c->d_state, c->num_sms, c->stream));
  if (int rc = record(c, 3)) return rc;
  CU(fc::launch_walk_overflow(t, v, c->d_ovf, acc, c->mode, c->d_scratch, c->scratch_ctas, c->d_state,
                              c->stream));
  if (int rc = record(c, 4)) return rc;
  c->prof.kernel_launches += 3;
  if (c->walked_steps) {
    CU(fc::launch_walked_steps(t, c->d_surv, ns, c->d_state, c->num_sms, c->stream));
    c->prof.kernel_launches += 1;
  }
  c->total_streamlines += ns;
  c->total_vertices += nv;
  if (c->flags & FASTCOD_SYNC) return sync_check(c);
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_connectivity(fastcod_ctx* c, int32_t* C_out) {
  fcapi::Range nvtx_range("fastcod_connectivity");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  return copy_out(c, c->d_C, C_out);
}

FASTCOD_API int fastcod_endpoint_connectivity(fastcod_ctx* c, int32_t* Cend_out) {
  fcapi::Range nvtx_range("fastcod_endpoint_connectivity");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  return copy_out(c, c->d_Cend, Cend_out);
}

FASTCOD_API int fastcod_reset(fastcod_ctx* c) {
  fcapi::Range nvtx_range("fastcod_reset");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  if (!c->has_vol) return fail(c, FASTCOD_ESTATE, "no volumes installed");
  CU(cudaSetDevice(c->device));
  return zero_accumulators(c);
}

FASTCOD_API int fastcod_get_shape(const fastcod_ctx* c, int32_t* n_roi, int32_t* n_targets) {
  if (!c) return FASTCOD_EINVAL;
  if (!c->has_vol) return FASTCOD_ESTATE;
  if (n_roi) *n_roi = c->N;
  if (n_targets) *n_targets = c->M;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_get_stats(fastcod_ctx* c, fastcod_stats* out) {
  if (!c || !out) return FASTCOD_EINVAL;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  DevState h;
  int rc = read_state(c, &h);
  if (rc) return rc;
  out->streamlines = c->total_streamlines;
  out->vertices = c->total_vertices;
  out->voxel_steps = (int64_t)h.voxel_steps;
  out->survivors = (int64_t)h.survivors;
  out->overflow = (int64_t)h.overflow;
  out->pairs = (int64_t)h.pairs;
  out->walked_steps = (int64_t)h.walked;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_restore(fastcod_ctx* c, const int32_t* C_in, const int32_t* Cend_in,
                                const fastcod_stats* stats) {
  fcapi::Range nvtx_range("fastcod_restore");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  if (!c->has_vol) return fail(c, FASTCOD_ESTATE, "no volumes installed");
  CU(cudaSetDevice(c->device));
  // a refused checkpoint leaves the context as after fastcod_reset
  auto refuse = [c](int rc) {
    const std::string msg = c->err;
    if (zero_accumulators(c) == FASTCOD_OK) (void)cudaStreamSynchronize(c->stream);
    c->err = msg;
    return rc;
  };
  if (!stats) return refuse(fail(c, FASTCOD_EINVAL, "stats is NULL"));
  const fastcod_stats& s = *stats;
  if (s.streamlines < 0 || s.streamlines > 0x7fffffffLL)
    return refuse(fail(c, FASTCOD_EINVAL, "checkpoint streamlines %lld outside [0, 2^31 - 1]",
                       (long long)s.streamlines));
  if (s.vertices < 0 || s.voxel_steps < 0 || s.survivors < 0 || s.overflow < 0 || s.pairs < 0 ||
      s.walked_steps < 0)
    return refuse(fail(c, FASTCOD_EINVAL, "checkpoint with a negative count"));
  if (s.survivors > s.streamlines || s.overflow > s.survivors || s.walked_steps > s.voxel_steps)
    return refuse(fail(c, FASTCOD_EINVAL, "checkpoint counts inconsistent (need survivors <= streamlines, "
                       "overflow <= survivors, walked_steps <= voxel_steps)"));
  const size_t nm = (size_t)c->N * (size_t)c->M;
  if (nm && (!C_in || !Cend_in)) return refuse(fail(c, FASTCOD_EINVAL, "matrix pointer is NULL"));
  if (nm && (fcapi::ptr_kind(C_in, c->device) < 0 || fcapi::ptr_kind(Cend_in, c->device) < 0))
    return refuse(fail(c, FASTCOD_EINVAL, "input is device memory of another device"));
  if (int rc = zero_accumulators(c)) return rc;
  if (int rc = grow(c, (void**)&c->d_check, &c->check_bytes, 3 * sizeof(unsigned long long))) return rc;
  CU(cudaMemsetAsync(c->d_check, 0, 2 * sizeof(unsigned long long), c->stream));
  CU(cudaMemsetAsync(c->d_check + 2, 0xff, sizeof(unsigned long long), c->stream));
  if (nm) {
    CU(cudaMemcpyAsync(c->d_C, C_in, nm * 4, cudaMemcpyDefault, c->stream));
    CU(cudaMemcpyAsync(c->d_Cend, Cend_in, nm * 4, cudaMemcpyDefault, c->stream));
    CU(fc::launch_checkpoint_check(c->d_C, c->d_Cend, (int64_t)nm, (int32_t)s.streamlines, c->d_check, c->stream));
    c->prof.kernel_launches += 1;
  }
  unsigned long long h[3];
  CU(cudaMemcpyAsync(h, c->d_check, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  int rc = FASTCOD_OK;
  if (h[2] != ~0ull) {
    const bool in_c = h[2] < nm;
    const unsigned long long k = in_c ? h[2] : h[2] - nm;
    rc = fail(c, FASTCOD_EINVAL, "checkpoint %s[%llu][%llu] outside [0, %lld streamlines]", in_c ? "C" : "C_end",
              k / (unsigned long long)c->M, k % (unsigned long long)c->M, (long long)s.streamlines);
  } else if (h[0] != (unsigned long long)s.pairs) {
    rc = fail(c, FASTCOD_EINVAL, "checkpoint C sums to %llu, its pairs count is %lld", h[0], (long long)s.pairs);
  } else if (h[1] > (unsigned long long)s.streamlines) {
    rc = fail(c, FASTCOD_EINVAL, "checkpoint C_end sums to %llu, more than its %lld streamlines", h[1],
              (long long)s.streamlines);
  }
  if (rc) return refuse(rc);
  // the running counts, in DevState order
  static_assert(offsetof(DevState, walked) - offsetof(DevState, voxel_steps) == 4 * sizeof(unsigned long long),
                "DevState counters out of order");
  const unsigned long long cnt[5] = {(unsigned long long)s.voxel_steps, (unsigned long long)s.survivors,
                                     (unsigned long long)s.overflow, (unsigned long long)s.pairs,
                                     (unsigned long long)s.walked_steps};
  CU(cudaMemcpyAsync(&c->d_state->voxel_steps, cnt, sizeof cnt, cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->total_streamlines = s.streamlines;
  c->total_vertices = s.vertices;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_get_profile(fastcod_ctx* c, fastcod_profile* out) {
  if (!c || !out) return FASTCOD_EINVAL;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  collect_profile(c);
  *out = c->prof;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_sync(fastcod_ctx* c) {
  fcapi::Range nvtx_range("fastcod_sync");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  return sync_check(c);
}

FASTCOD_API int fastcod_set_option(fastcod_ctx* c, int32_t key, int64_t value) {
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  switch (key) {
    case FASTCOD_OPT_PREFILTER:
      if (value != 0 && value != 1) break;
      c->prefilter = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_TARGET_MODE:
      if (value != 0 && value != 1) break;
      c->mode = (c->mode & ~fc::kModeTargetEndpoint) | (value ? fc::kModeTargetEndpoint : 0u);
      return FASTCOD_OK;
    case FASTCOD_OPT_SAMPLING:
      if (value != 0 && value != 1) break;
      c->mode = (c->mode & ~fc::kModeVertexSampled) | (value ? fc::kModeVertexSampled : 0u);
      return FASTCOD_OK;
    case FASTCOD_OPT_STAGING:
      if (value != 0 && value != 1) break;
      c->staging_tma = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_PREFILTER_CTAS:
      if (value != 2 && value != 3) break;
      c->prefilter_ctas = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_NEAR_LOG2:
      if (value < -1 || value > 3) break;
      c->near_log2 = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_AUTOTUNE:
      if (value != 0 && value != 1) break;
      c->autotune = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_HOST_IN_PLACE:
      if (value != 0 && value != 1) break;
      c->host_in_place = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_WALKED_STEPS:
      if (value != 0 && value != 1) break;
      c->walked_steps = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_SEGMENT_SKIP:
      if (value != 0 && value != 1) break;
      c->mode = (c->mode & ~fc::kModeWalkAll) | (value ? 0u : fc::kModeWalkAll);
      return FASTCOD_OK;
    case FASTCOD_OPT_TEST_WITHHOLD_PIECE:
      if (value < -1) break;
      c->withhold_piece = value;
      return FASTCOD_OK;
    case FASTCOD_OPT_BATCH_TASK_LOG2:
      if (value < 12 || value > 22) break;
      c->batch_task_log2 = (int)value;
      return FASTCOD_OK;
    case FASTCOD_OPT_PROFILE:
      if (value != 0 && value != 1) break;
      CU(cudaSetDevice(c->device));
      CU(cudaStreamSynchronize(c->stream));
      collect_profile(c);
      if (value && !c->profile) {
        // switching on starts a fresh profile
        const int64_t launches = c->prof.kernel_launches;
        c->prof = fastcod_profile{0, launches, 0.0, 0.0, 0.0, 0.0, 0, 0.0};
      }
      c->profile = (int)value;
      return FASTCOD_OK;
    default:
      return fail(c, FASTCOD_EINVAL, "unknown option %d", key);
  }
  return fail(c, FASTCOD_EINVAL, "invalid value %lld for option %d", (long long)value, key);
}

FASTCOD_API const char* fastcod_last_error(const fastcod_ctx* c) {
  if (!c) return fcapi::thread_error().c_str();
  return c->err.c_str();
}

}  // extern "C"
