// C ABI of the entry points beside the connectivity path (see fastcod.h):
// parcellation outputs, world-mm ingest, upsampling and rescale.  Each one
// stages host inputs into the context's scratch, runs its kernels on the
// context's stream, checks what the kernels found in a state block of its own
// (so that an error here leaves C and C_end untouched) and blocks until its
// outputs are written.
#include <cuda_runtime.h>

#include "fc_ctx.h"

namespace {

using fcapi::fail;
using fcapi::grow;
using fcapi::ptr_kind;
using fcapi::sync_check;

enum AuxSlot { kIn = 0, kOff = 1, kOut = 2, kOut2 = 3, kTmp = 4, kState = 5 };

int slot(fastcod_ctx* c, int k, size_t bytes, void** p) {
  if (int rc = grow(c, &c->d_aux[k], &c->aux_bytes[k], bytes)) return rc;
  *p = c->d_aux[k];
  return FASTCOD_OK;
}

// A device address for input p of `bytes` bytes: p itself when it is device
// memory of the context's device, else a copy in scratch slot k.
int stage_in(fastcod_ctx* c, int k, const void* p, size_t bytes, const void** d) {
  const int kind = ptr_kind(p, c->device);
  if (kind < 0) return fail(c, FASTCOD_EINVAL, "input is device memory of another device");
  if (kind == 1) {
    *d = p;
    return FASTCOD_OK;
  }
  void* s = nullptr;
  if (int rc = slot(c, k, bytes, &s)) return rc;
  if (bytes) CU(cudaMemcpyAsync(s, p, bytes, cudaMemcpyHostToDevice, c->stream));
  *d = s;
  return FASTCOD_OK;
}

// A device address to write output p of `bytes` bytes to: p itself when it is
// device memory of the context's device, else scratch slot k (copied back by
// copy_out).
int out_dst(fastcod_ctx* c, int k, void* p, size_t bytes, void** d) {
  const int kind = ptr_kind(p, c->device);
  if (kind < 0) return fail(c, FASTCOD_EINVAL, "output is device memory of another device");
  if (kind == 1) {
    *d = p;
    return FASTCOD_OK;
  }
  return slot(c, k, bytes, d);
}

int copy_out(fastcod_ctx* c, void* p, const void* d, size_t bytes) {
  if (p != d && bytes) CU(cudaMemcpyAsync(p, d, bytes, cudaMemcpyDeviceToHost, c->stream));
  return FASTCOD_OK;
}

// The aux state block, zeroed in stream order.
int state_begin(fastcod_ctx* c, DevState** st) {
  void* p = nullptr;
  if (int rc = slot(c, kState, sizeof(DevState), &p)) return rc;
  CU(cudaMemsetAsync(p, 0, sizeof(DevState), c->stream));
  *st = static_cast<DevState*>(p);
  return FASTCOD_OK;
}

// Wait for the stream and report what the kernels found.
int state_end(fastcod_ctx* c, const DevState* st, const char* what) {
  DevState h;
  CU(cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  switch (h.error) {
    case fc::kErrNone:
      return FASTCOD_OK;
    case fc::kErrOffsets:
      return fail(c, FASTCOD_EINVAL, "%s: offsets invalid near streamline %d", what, h.error_info);
    case fc::kErrCoord:
      return fail(c, FASTCOD_EINVAL, "%s: coordinate not finite or outside [-2^24, 2^24) near vertex %d", what,
                  h.error_info);
    case fc::kErrCount:
      return fail(c, FASTCOD_EINVAL, "%s: negative count in row %d", what, h.error_info);
    case fc::kErrChecked:
      return fail(c, FASTCOD_ECUDA, "%s: bounds check failed (site %d)", what, h.error_info);
    default:
      return fail(c, FASTCOD_ECUDA, "%s: device error %d (%d)", what, h.error, h.error_info);
  }
}

// Device time of a span of kernels while profiling: events before and after
// the span; span_end waits for the stream and adds the elapsed time.
int span_begin(fastcod_ctx* c) {
  if (!c->profile) return FASTCOD_OK;
  for (cudaEvent_t& e : c->aux_ev)
    if (!e) CU(cudaEventCreate(&e));
  CU(cudaEventRecord(c->aux_ev[0], c->stream));
  return FASTCOD_OK;
}

int span_end(fastcod_ctx* c, bool count_call) {
  if (!c->profile) return FASTCOD_OK;
  CU(cudaEventRecord(c->aux_ev[1], c->stream));
  CU(cudaEventSynchronize(c->aux_ev[1]));
  float ms = 0.0f;
  CU(cudaEventElapsedTime(&ms, c->aux_ev[0], c->aux_ev[1]));
  c->prof.ms_aux += ms;
  if (count_call) c->prof.aux_calls += 1;
  return FASTCOD_OK;
}

int begin(fastcod_ctx* c) {
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  CU(cudaSetDevice(c->device));
  return FASTCOD_OK;
}

int check_streamlines(fastcod_ctx* c, const void* xyz, int64_t nv, const int64_t* offsets, int64_t ns) {
  if (nv < 0 || ns < 0) return fail(c, FASTCOD_EINVAL, "negative count");
  if (!offsets || (nv > 0 && !xyz)) return fail(c, FASTCOD_EINVAL, "input pointer is NULL");
  if (nv > 0x7fffffffLL || ns > 0x7fffffffLL) return fail(c, FASTCOD_EINVAL, "more than 2^31-1 vertices or streamlines");
  return FASTCOD_OK;
}

// Validate offsets [ns + 1] (device) against nv; blocks.
int validate_offsets(fastcod_ctx* c, const int64_t* d_off, int64_t ns, int64_t nv, const char* what) {
  DevState* st = nullptr;
  if (int rc = state_begin(c, &st)) return rc;
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_check_offsets(d_off, ns, nv, st, c->stream));
  c->prof.kernel_launches += 1;
  if (int rc = span_end(c, false)) return rc;
  return state_end(c, st, what);
}

int world_to_fixed_into(fastcod_ctx* c, const float* xyz_mm, int64_t nv, const float affine[12], int32_t* d_out) {
  const void* d_in = nullptr;
  if (int rc = stage_in(c, kIn, xyz_mm, (size_t)nv * 12, &d_in)) return rc;
  DevState* st = nullptr;
  if (int rc = state_begin(c, &st)) return rc;
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_world_to_fixed(static_cast<const float*>(d_in), nv, affine, d_out, st, c->stream));
  c->prof.kernel_launches += nv > 0 ? 1 : 0;
  if (int rc = span_end(c, true)) return rc;
  return state_end(c, st, "world-mm ingest");
}

}  // namespace

extern "C" {

FASTCOD_API int fastcod_parcellate(fastcod_ctx* c, int32_t which, int32_t* label_out, float* fractions_out) {
  fcapi::Range nvtx_range("fastcod_parcellate");
  if (int rc = begin(c)) return rc;
  if (!c->has_vol) return fail(c, FASTCOD_ESTATE, "no volumes installed");
  if (which != 0 && which != 1) return fail(c, FASTCOD_EINVAL, "which must be 0 (C) or 1 (C_end)");
  if (!label_out) return fail(c, FASTCOD_EINVAL, "label_out is NULL");
  if (int rc = sync_check(c)) return rc;
  const int32_t N = c->N, M = c->M;
  void* d_label = nullptr;
  void* d_frac = nullptr;
  if (int rc = out_dst(c, kOut, label_out, (size_t)N * 4, &d_label)) return rc;
  if (fractions_out)
    if (int rc = out_dst(c, kOut2, fractions_out, (size_t)N * M * 4, &d_frac)) return rc;
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_parcellate(which ? c->d_Cend : c->d_C, N, M, static_cast<int32_t*>(d_label),
                           static_cast<float*>(d_frac), nullptr, c->stream));
  c->prof.kernel_launches += N > 0 ? 1 : 0;
  if (int rc = span_end(c, true)) return rc;
  if (int rc = copy_out(c, label_out, d_label, (size_t)N * 4)) return rc;
  if (fractions_out)
    if (int rc = copy_out(c, fractions_out, d_frac, (size_t)N * M * 4)) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_parcellate_matrix(fastcod_ctx* c, const int32_t* C, int32_t N, int32_t M,
                                          int32_t* label_out, float* fractions_out) {
  fcapi::Range nvtx_range("fastcod_parcellate_matrix");
  if (int rc = begin(c)) return rc;
  if (N < 0 || M < 1 || M > 65535) return fail(c, FASTCOD_EINVAL, "N must be >= 0 and M in [1, 65535]");
  if (N == 0) return FASTCOD_OK;
  if (!C || !label_out) return fail(c, FASTCOD_EINVAL, "pointer is NULL");
  if (int rc = sync_check(c)) return rc;
  const size_t bytes = (size_t)N * M * 4;
  const void* d_C = nullptr;
  if (int rc = stage_in(c, kIn, C, bytes, &d_C)) return rc;
  void* d_label = nullptr;
  void* d_frac = nullptr;
  if (int rc = out_dst(c, kOut, label_out, (size_t)N * 4, &d_label)) return rc;
  if (fractions_out)
    if (int rc = out_dst(c, kOut2, fractions_out, bytes, &d_frac)) return rc;
  DevState* st = nullptr;
  if (int rc = state_begin(c, &st)) return rc;
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_parcellate(static_cast<const int32_t*>(d_C), N, M, static_cast<int32_t*>(d_label),
                           static_cast<float*>(d_frac), st, c->stream));
  c->prof.kernel_launches += 1;
  if (int rc = span_end(c, true)) return rc;
  if (int rc = state_end(c, st, "parcellation")) return rc;
  if (int rc = copy_out(c, label_out, d_label, (size_t)N * 4)) return rc;
  if (fractions_out)
    if (int rc = copy_out(c, fractions_out, d_frac, bytes)) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_world_to_fixed(fastcod_ctx* c, const float* xyz_mm, int64_t n_vertices,
                                       const float affine[12], int32_t* xyz_out) {
  fcapi::Range nvtx_range("fastcod_world_to_fixed");
  if (int rc = begin(c)) return rc;
  if (n_vertices < 0 || n_vertices > 0x7fffffffLL) return fail(c, FASTCOD_EINVAL, "vertex count out of range");
  if (n_vertices == 0) return FASTCOD_OK;
  if (!xyz_mm || !affine || !xyz_out) return fail(c, FASTCOD_EINVAL, "pointer is NULL");
  void* d_out = nullptr;
  if (int rc = out_dst(c, kOut, xyz_out, (size_t)n_vertices * 12, &d_out)) return rc;
  if (int rc = world_to_fixed_into(c, xyz_mm, n_vertices, affine, static_cast<int32_t*>(d_out))) return rc;
  if (int rc = copy_out(c, xyz_out, d_out, (size_t)n_vertices * 12)) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_add_streamlines_mm(fastcod_ctx* c, const float* xyz_mm, int64_t n_vertices,
                                           const int64_t* offsets, int64_t n_streamlines, const float affine[12]) {
  fcapi::Range nvtx_range("fastcod_add_streamlines_mm");
  if (int rc = begin(c)) return rc;
  if (!c->has_vol) return fail(c, FASTCOD_ESTATE, "fastcod_set_volumes must come first");
  if (int rc = check_streamlines(c, xyz_mm, n_vertices, offsets, n_streamlines)) return rc;
  if (!affine) return fail(c, FASTCOD_EINVAL, "affine is NULL");
  if (n_vertices > 0) {
    if (int rc = grow(c, (void**)&c->d_xyz, &c->xyz_bytes, (size_t)n_vertices * 12 + 16)) return rc;
    if (int rc = world_to_fixed_into(c, xyz_mm, n_vertices, affine, c->d_xyz)) return rc;
  }
  return fastcod_add_streamlines(c, c->d_xyz, n_vertices, offsets, n_streamlines);
}

FASTCOD_API int fastcod_upsample_factor(fastcod_ctx* c, const int32_t* xyz, int64_t n_vertices,
                                        const int64_t* offsets, int64_t n_streamlines, int32_t spacing,
                                        int32_t* factor_out) {
  fcapi::Range nvtx_range("fastcod_upsample_factor");
  if (int rc = begin(c)) return rc;
  if (int rc = check_streamlines(c, xyz, n_vertices, offsets, n_streamlines)) return rc;
  if (spacing < 1 || !factor_out) return fail(c, FASTCOD_EINVAL, "spacing must be >= 1 and factor_out set");
  const void* d_xyz = nullptr;
  const void* d_off = nullptr;
  if (int rc = stage_in(c, kIn, xyz, (size_t)n_vertices * 12, &d_xyz)) return rc;
  if (int rc = stage_in(c, kOff, offsets, (size_t)(n_streamlines + 1) * 8, &d_off)) return rc;
  const int64_t* off = static_cast<const int64_t*>(d_off);
  if (int rc = validate_offsets(c, off, n_streamlines, n_vertices, "upsample factor")) return rc;
  void* d_best = nullptr;
  if (int rc = slot(c, kTmp, 8, &d_best)) return rc;
  CU(cudaMemsetAsync(d_best, 0, 8, c->stream));
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_seg_max(static_cast<const int32_t*>(d_xyz), off, n_streamlines,
                        static_cast<unsigned long long*>(d_best), c->stream));
  c->prof.kernel_launches += n_streamlines > 0 ? 1 : 0;
  if (int rc = span_end(c, true)) return rc;
  unsigned long long best = 0;
  CU(cudaMemcpyAsync(&best, d_best, 8, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  // the smallest r with r * r >= best, then the smallest k with k * spacing >= r
  int64_t lo = 0, hi = (int64_t)1 << 27;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if ((unsigned long long)(mid * mid) >= best) hi = mid; else lo = mid + 1;
  }
  int64_t k = (lo + spacing - 1) / spacing;
  if (k < 1) k = 1;
  if (k > (1 << 20)) return fail(c, FASTCOD_EINVAL, "upsampling factor above 2^20");
  *factor_out = (int32_t)k;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_upsample(fastcod_ctx* c, const int32_t* xyz, int64_t n_vertices, const int64_t* offsets,
                                 int64_t n_streamlines, int32_t factor, int32_t* xyz_out, int64_t n_vertices_out,
                                 int64_t* offsets_out) {
  fcapi::Range nvtx_range("fastcod_upsample");
  if (int rc = begin(c)) return rc;
  if (int rc = check_streamlines(c, xyz, n_vertices, offsets, n_streamlines)) return rc;
  if (factor < 1 || factor > (1 << 20)) return fail(c, FASTCOD_EINVAL, "factor must be in [1, 2^20]");
  if (!offsets_out || (n_vertices_out > 0 && !xyz_out)) return fail(c, FASTCOD_EINVAL, "output pointer is NULL");
  const void* d_xyz = nullptr;
  const void* d_off = nullptr;
  if (int rc = stage_in(c, kIn, xyz, (size_t)n_vertices * 12, &d_xyz)) return rc;
  if (int rc = stage_in(c, kOff, offsets, (size_t)(n_streamlines + 1) * 8, &d_off)) return rc;
  const int64_t* off = static_cast<const int64_t*>(d_off);
  if (int rc = validate_offsets(c, off, n_streamlines, n_vertices, "upsample")) return rc;
  void* d_oo = nullptr;
  void* d_tmp = nullptr;
  if (int rc = out_dst(c, kOut2, offsets_out, (size_t)(n_streamlines + 1) * 8, &d_oo)) return rc;
  if (int rc = slot(c, kTmp, (size_t)fc::upsample_scan_blocks(n_streamlines) * 8, &d_tmp)) return rc;
  int64_t* oo = static_cast<int64_t*>(d_oo);
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_upsample_offsets(off, n_streamlines, factor, static_cast<long long*>(d_tmp), oo, c->stream));
  c->prof.kernel_launches += 3;
  if (int rc = span_end(c, false)) return rc;
  int64_t total = 0;
  CU(cudaMemcpyAsync(&total, oo + n_streamlines, 8, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (total != n_vertices_out)
    return fail(c, FASTCOD_EINVAL, "the upsampled tractogram has %lld vertices, not %lld", (long long)total,
                (long long)n_vertices_out);
  if (total > 0x7fffffffLL) return fail(c, FASTCOD_EINVAL, "more than 2^31-1 upsampled vertices");
  void* d_out = nullptr;
  if (total > 0) {
    if (int rc = out_dst(c, kOut, xyz_out, (size_t)total * 12, &d_out)) return rc;
    if (int rc = span_begin(c)) return rc;
    CU(fc::launch_upsample_vertices(static_cast<const int32_t*>(d_xyz), off, n_streamlines, factor, oo,
                                    static_cast<int32_t*>(d_out), c->stream));
    c->prof.kernel_launches += 1;
    if (int rc = span_end(c, true)) return rc;
    if (int rc = copy_out(c, xyz_out, d_out, (size_t)total * 12)) return rc;
  } else if (c->profile) {
    c->prof.aux_calls += 1;
  }
  if (int rc = copy_out(c, offsets_out, d_oo, (size_t)(n_streamlines + 1) * 8)) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_rescale(fastcod_ctx* c, const int32_t* xyz, int64_t n_vertices, const int32_t num[3],
                                const int32_t den[3], const int64_t add[3], int32_t* xyz_out) {
  fcapi::Range nvtx_range("fastcod_rescale");
  if (int rc = begin(c)) return rc;
  if (n_vertices < 0 || n_vertices > 0x7fffffffLL) return fail(c, FASTCOD_EINVAL, "vertex count out of range");
  if (!num || !den || !add) return fail(c, FASTCOD_EINVAL, "num, den and add are required");
  for (int a = 0; a < 3; ++a)
    if (num[a] < 1 || den[a] < 1) return fail(c, FASTCOD_EINVAL, "num and den must be positive");
  if (n_vertices == 0) return FASTCOD_OK;
  if (!xyz || !xyz_out) return fail(c, FASTCOD_EINVAL, "pointer is NULL");
  const void* d_in = nullptr;
  void* d_out = nullptr;
  if (int rc = stage_in(c, kIn, xyz, (size_t)n_vertices * 12, &d_in)) return rc;
  if (int rc = out_dst(c, kOut, xyz_out, (size_t)n_vertices * 12, &d_out)) return rc;
  DevState* st = nullptr;
  if (int rc = state_begin(c, &st)) return rc;
  if (int rc = span_begin(c)) return rc;
  CU(fc::launch_rescale(static_cast<const int32_t*>(d_in), n_vertices, num, den, add, static_cast<int32_t*>(d_out), st,
                        c->stream));
  c->prof.kernel_launches += n_vertices > 0 ? 1 : 0;
  if (int rc = span_end(c, true)) return rc;
  if (int rc = state_end(c, st, "rescale")) return rc;
  if (int rc = copy_out(c, xyz_out, d_out, (size_t)n_vertices * 12)) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return FASTCOD_OK;
}

}  // extern "C"
