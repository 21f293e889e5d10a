// Batched form of the C ABI: many subjects per pass, one CUDA graph per
// batch shape, and the autotuner that picks the prefilter's configuration per
// shape (see fastcod_batch_run in fastcod.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>

#include "fc_ctx.h"

using fcapi::fail;
using fcapi::ptr_kind;

namespace {

constexpr int32_t kOverflowCtas = 64;

// What the autotuner picks per batch shape: prefilter CTAs per SM, near-grid
// cell (-1: per subject), and the work granularity of a prefilter task (about
// 2^task_log2 vertices of one subject).
struct BatchConfig {
  int ctas;
  int near_log2;
  int task_log2;
};

int64_t tasks_of(int64_t n_vertices, int task_log2) {
  const int64_t tv = (int64_t)1 << task_log2;
  return std::max<int64_t>(1, (n_vertices + tv - 1) / tv);
}

// Sub-allocation of the batch arena (byte offsets, 256-byte aligned).
struct Layout {
  size_t scratch, gstate, states, surv, ovf, staged_end;
  int64_t surv_cap;  // entries of the survivor and overflow lists
  std::vector<size_t> roi_in, lab_in, xyz_in, off_in;  // staging of host inputs (or SIZE_MAX)
  std::vector<size_t> code, lab, bricks, C, Cend, planes;
  size_t acc_lo, acc_hi;        // every subject's C and C_end in the arena (used for outputs in host memory)
  size_t bricks_lo, bricks_hi;  // every subject's brick words: one span
  std::vector<size_t> near;
  size_t total;
  int64_t scratch_words;
  int32_t ntasks;
};

}  // namespace

struct BatchState {
  void* arena = nullptr;
  size_t arena_bytes = 0;
  size_t scratch_zeroed = 0;  // bytes of the scratch region known to be zero
  uint64_t graph_key = 0;
  cudaGraphExec_t exec = nullptr;
  std::vector<DevState> states;
  std::vector<int64_t> ns, nv;  // per subject of the last batch
  std::vector<char> out_dev;    // per subject: C_out and Cend_out are device memory of this device, and the
                                // walk accumulates into them in place
  std::map<uint64_t, BatchConfig> tuned;
  bool cache_loaded = false;
  fastcod_batch_info info{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

int ilog2_64(int64_t x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

int64_t near_words(const int32_t d[3], int near_log2) {
  fc::VolView v{};
  v.dx = d[0];
  v.dy = d[1];
  v.dz = d[2];
  fc::set_near_dims(v, fc::resolve_near_log2(near_log2, d[0], d[1], d[2]));
  return fc::near_words(v);
}

Layout plan(const fastcod_subject* subs, int32_t n, const std::vector<int>& host_in, int near_log2, int task_log2,
            int64_t total_ns) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + (bytes ? bytes : 1));
    return at;
  };
  int64_t maxw = 1, maxplanes = 1;
  int32_t ntasks = 0;
  for (int32_t i = 0; i < n; ++i) {
    maxw = std::max(maxw, fc::overflow_scratch_words(subs[i].n_roi, subs[i].n_targets));
    maxplanes = std::max(maxplanes, fc::plane_words(subs[i].dims[0], subs[i].dims[1], subs[i].dims[2]));
    ntasks += (int32_t)tasks_of(subs[i].n_vertices, task_log2);
  }
  L.scratch_words = maxw;
  L.ntasks = ntasks;
  L.scratch = take((size_t)(kOverflowCtas * maxw * 4));
  L.gstate = take(sizeof(DevState));
  L.states = take(sizeof(DevState) * n);
  L.surv = take((size_t)total_ns * 4);
  L.surv_cap = total_ns;
  L.ovf = take((size_t)total_ns * 4);
  for (int32_t i = 0; i < n; ++i) {
    const fastcod_subject& S = subs[i];
    const int64_t nvox = (int64_t)S.dims[0] * S.dims[1] * S.dims[2];
    L.roi_in.push_back(host_in[4 * i] ? take((size_t)nvox * 4) : SIZE_MAX);
    L.lab_in.push_back(host_in[4 * i + 1] ? take((size_t)nvox * 2) : SIZE_MAX);
    L.xyz_in.push_back(host_in[4 * i + 2] ? take((size_t)S.n_vertices * 12 + 16) : SIZE_MAX);
    L.off_in.push_back(host_in[4 * i + 3] ? take((size_t)(S.n_streamlines + 1) * 8) : SIZE_MAX);
  }
  L.staged_end = o;
  for (int32_t i = 0; i < n; ++i) {
    const fastcod_subject& S = subs[i];
    const int64_t nvox = (int64_t)S.dims[0] * S.dims[1] * S.dims[2];
    L.code.push_back(take((size_t)nvox * 4));
    L.lab.push_back(take((size_t)nvox * 2));
    L.planes.push_back(take((size_t)fc::plane_words(S.dims[0], S.dims[1], S.dims[2]) * 4));
  }
  L.acc_lo = o;
  for (int32_t i = 0; i < n; ++i) {
    const size_t nm = (size_t)subs[i].n_roi * (size_t)subs[i].n_targets;
    L.C.push_back(take(nm * 4));
    L.Cend.push_back(take(nm * 4));
  }
  L.acc_hi = o;
  L.bricks_lo = o;
  for (int32_t i = 0; i < n; ++i) {
    const fastcod_subject& S = subs[i];
    const int64_t nb = (int64_t)((S.dims[0] + 3) / 4) * ((S.dims[1] + 3) / 4) * ((S.dims[2] + 3) / 4);
    L.bricks.push_back(take((size_t)((nb + 15) / 16) * 4));
  }
  L.bricks_hi = o;
  (void)maxplanes;
  // the configuration-dependent part last (near grids: the cell size), so
  // that the rest, staged inputs included, keeps its place from one
  // configuration to the next
  for (int32_t i = 0; i < n; ++i) L.near.push_back(take((size_t)near_words(subs[i].dims, near_log2) * 4));
  L.total = o;
  return L;
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

void fill_table(fastcod_ctx* c, const fastcod_subject* subs, int32_t n, const Layout& L, int near_log2, int task_log2,
                fc::BatchTable& tbl) {
  void* A = c->batch->arena;
  const std::vector<char>& out_dev = c->batch->out_dev;
  memset(&tbl, 0, sizeof tbl);
  tbl.n = n;
  int64_t sbase = 0, task0 = 0;
  for (int32_t i = 0; i < n; ++i) {
    const fastcod_subject& S = subs[i];
    fc::BatchSubject& B = tbl.s[i];
    fc::VolView& v = B.v;
    v.code = at<uint32_t>(A, L.code[i]);
    v.lab = at<uint16_t>(A, L.lab[i]);
    v.bricks = at<uint32_t>(A, L.bricks[i]);
    v.near = at<uint32_t>(A, L.near[i]);
    v.dx = S.dims[0];
    v.dy = S.dims[1];
    v.dz = S.dims[2];
    v.bx = (S.dims[0] + 3) / 4;
    v.by = (S.dims[1] + 3) / 4;
    v.bz = (S.dims[2] + 3) / 4;
    fc::set_near_dims(v, fc::resolve_near_log2(near_log2, S.dims[0], S.dims[1], S.dims[2]));
    v.n_roi = S.n_roi;
    v.n_lab = S.n_targets;
    B.t.xyz = L.xyz_in[i] != SIZE_MAX ? at<int32_t>(A, L.xyz_in[i]) : S.xyz;
    B.t.off = L.off_in[i] != SIZE_MAX ? at<int64_t>(A, L.off_in[i]) : S.offsets;
    B.t.nv = S.n_vertices;
    B.t.ns = S.n_streamlines;
    // device outputs are accumulated in place; host ones in the arena, copied
    // out after the graph
    B.acc.C = out_dev[i] ? S.C_out : at<int32_t>(A, L.C[i]);
    B.acc.Cend = out_dev[i] ? S.Cend_out : at<int32_t>(A, L.Cend[i]);
    B.st = at<DevState>(A, L.states) + i;
    B.sbase = sbase;
    sbase += S.n_streamlines;
    // its prefilter tasks, computed by the prefilter from these two numbers
    B.task0 = task0;
    B.ntask = tasks_of(S.n_vertices, task_log2);
    task0 += B.ntask;
  }
}

uint64_t graph_key(const fc::BatchTable& tbl, int32_t ntasks, const BatchConfig& cfg, uint32_t mode, int prefilter, int tma,
                   const void* arena, const fastcod_subject* subs, const Layout& L) {
  uint64_t h = 1469598103934665603ull;
  for (int32_t i = 0; i < tbl.n; ++i) {  // the volume inputs K1 reads
    h = mix(h, L.roi_in[i] != SIZE_MAX ? (uint64_t)L.roi_in[i] : (uint64_t)(uintptr_t)subs[i].roi_index_map);
    h = mix(h, L.lab_in[i] != SIZE_MAX ? (uint64_t)L.lab_in[i] : (uint64_t)(uintptr_t)subs[i].target_labels);
  }
  const uint64_t* w = reinterpret_cast<const uint64_t*>(&tbl);
  const size_t words = (offsetof(fc::BatchTable, s) + sizeof(fc::BatchSubject) * tbl.n) / 8;
  for (size_t i = 0; i < words; ++i) h = mix(h, w[i]);
  h = mix(h, (uint64_t)ntasks);
  h = mix(h, (uint64_t)cfg.ctas * 131 + (uint64_t)(cfg.near_log2 + 1) * 7 + (uint64_t)cfg.task_log2 * 1009);
  h = mix(h, (uint64_t)mode * 7 + (uint64_t)prefilter + 1000 * (uint64_t)(tma != 0));
  h = mix(h, (uint64_t)(uintptr_t)arena);
  return h;
}

// Capture the whole batch into a graph on the context's stream.  *exec: the
// executable graph of the last batch, updated in place when only parameters
// changed (new input or output addresses, new sizes of the same nodes), else
// replaced by a new instantiation.
int capture(fastcod_ctx* c, const fastcod_subject* subs, int32_t n, const Layout& L, const fc::BatchTable& tbl,
            const BatchConfig& cfg, cudaGraphExec_t* exec) {
  BatchState* B = c->batch;
  void* A = B->arena;
  DevState* gst = at<DevState>(A, L.gstate);
  // volume preparation of every subject: one launch for the codes, labels,
  // bricks and bit planes, one for the near grids
  fc::PrepTable* prep = new (std::nothrow) fc::PrepTable;
  if (!prep) return fail(c, FASTCOD_ENOMEM, "host allocation failed");
  memset(prep, 0, sizeof *prep);
  prep->n = n;
  for (int32_t i = 0; i < n; ++i) {
    fc::PrepSubject& P = prep->s[i];
    P.v = tbl.s[i].v;
    P.roi = L.roi_in[i] != SIZE_MAX ? at<int32_t>(A, L.roi_in[i]) : subs[i].roi_index_map;
    P.lab = L.lab_in[i] != SIZE_MAX ? at<uint16_t>(A, L.lab_in[i]) : subs[i].target_labels;
    P.planes = at<uint32_t>(A, L.planes[i]);
    P.st = tbl.s[i].st;
    P.zero0 = tbl.s[i].acc.C;  // zeroed by the prep launch, before the walk adds to them
    P.zero1 = tbl.s[i].acc.Cend;
    P.nzero = (int64_t)tbl.s[i].v.n_roi * tbl.s[i].v.n_lab;
  }
  fc::prep_table_blocks(*prep);
  const cudaError_t e0 = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e0 != cudaSuccess) {
    delete prep;
    CU(e0);
  }
  cudaError_t e = cudaMemsetAsync(gst, 0, sizeof(DevState), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<DevState>(A, L.states), 0, sizeof(DevState) * n, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<char>(A, L.bricks_lo), 0, L.bricks_hi - L.bricks_lo, c->stream);
  if (e == cudaSuccess) e = fc::launch_volume_prep_batch(*prep, c->stream);
  if (e == cudaSuccess) e = fc::launch_near_batch(*prep, c->stream);
  delete prep;
  if (e == cudaSuccess)
    e = fc::launch_prefilter_batch(tbl, nullptr, L.ntasks, c->prefilter != 0, c->staging_tma != 0, cfg.ctas,
                                   at<int32_t>(A, L.surv), L.surv_cap, gst, c->num_sms, c->stream);
  if (e == cudaSuccess)
    e = fc::launch_walk_batch(tbl, at<int32_t>(A, L.surv), L.surv_cap, c->mode, at<int32_t>(A, L.ovf), gst, c->num_sms,
                              c->stream);
  if (e == cudaSuccess)
    e = fc::launch_walk_overflow_batch(tbl, at<int32_t>(A, L.ovf), c->mode, at<uint32_t>(A, L.scratch), kOverflowCtas,
                                       L.scratch_words, gst, c->stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return fail(c, FASTCOD_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  if (*exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(*exec, g, &info) == cudaSuccess) {
      cudaGraphDestroy(g);
      return FASTCOD_OK;
    }
    (void)cudaGetLastError();
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  const cudaError_t e3 = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  CU(e3);
  return FASTCOD_OK;
}

int kernels_per_run(int32_t n) { return n > 0 ? 5 : 0; }

// Stage inputs, (re)capture when the shape changed, run the graph.
int run_config(fastcod_ctx* c, const fastcod_subject* subs, int32_t n, const std::vector<int>& host_in,
               int64_t total_ns, const BatchConfig& cfg, bool stage, float* ms) {
  BatchState* B = c->batch;
  Layout L = plan(subs, n, host_in, cfg.near_log2, cfg.task_log2, total_ns);
  if (L.total > B->arena_bytes || !B->arena) {
    if (B->exec) {
      cudaGraphExecDestroy(B->exec);
      B->exec = nullptr;
      B->graph_key = 0;
    }
    size_t cap = B->arena_bytes;
    if (int rc = fcapi::grow(c, &B->arena, &cap, L.total + L.total / 8)) return rc;
    B->arena_bytes = cap;
    B->scratch_zeroed = 0;
    stage = true;
  }
  void* A = B->arena;
  if (B->scratch_zeroed < (size_t)(kOverflowCtas * L.scratch_words * 4)) {
    CU(cudaMemsetAsync(at<uint32_t>(A, L.scratch), 0, (size_t)(kOverflowCtas * L.scratch_words * 4), c->stream));
    B->scratch_zeroed = (size_t)(kOverflowCtas * L.scratch_words * 4);
  }
  fc::BatchTable* tbl = new (std::nothrow) fc::BatchTable;
  if (!tbl) return fail(c, FASTCOD_ENOMEM, "host allocation failed");
  fill_table(c, subs, n, L, cfg.near_log2, cfg.task_log2, *tbl);
  int rc = FASTCOD_OK;
  do {
    if (stage) {
      for (int32_t i = 0; i < n && rc == FASTCOD_OK; ++i) {
        const fastcod_subject& S = subs[i];
        const int64_t nvox = (int64_t)S.dims[0] * S.dims[1] * S.dims[2];
        cudaError_t e = cudaSuccess;
        if (L.roi_in[i] != SIZE_MAX)
          e = cudaMemcpyAsync(at<void>(A, L.roi_in[i]), S.roi_index_map, (size_t)nvox * 4, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && L.lab_in[i] != SIZE_MAX)
          e = cudaMemcpyAsync(at<void>(A, L.lab_in[i]), S.target_labels, (size_t)nvox * 2, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && L.xyz_in[i] != SIZE_MAX && S.n_vertices)
          e = cudaMemcpyAsync(at<void>(A, L.xyz_in[i]), S.xyz, (size_t)S.n_vertices * 12, cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess && L.off_in[i] != SIZE_MAX)
          e = cudaMemcpyAsync(at<void>(A, L.off_in[i]), S.offsets, (size_t)(S.n_streamlines + 1) * 8,
                              cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
          (void)cudaGetLastError();
          rc = fail(c, FASTCOD_ECUDA, "batch input copy (subject %d): %s", i, cudaGetErrorString(e));
        }
      }
      if (rc) break;
    }
    const uint64_t key = graph_key(*tbl, L.ntasks, cfg, c->mode, c->prefilter, c->staging_tma, A, subs, L);
    B->info.graph_reused = (B->exec && key == B->graph_key) ? 1 : 0;
    if (!B->info.graph_reused) {
      rc = capture(c, subs, n, L, *tbl, cfg, &B->exec);
      if (rc) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
        B->graph_key = 0;
        break;
      }
      B->graph_key = key;
    }
    if (!B->e0) {
      if (cudaEventCreate(&B->e0) != cudaSuccess || cudaEventCreate(&B->e1) != cudaSuccess) {
        rc = fail(c, FASTCOD_ECUDA, "event creation failed");
        break;
      }
    }
    cudaError_t e = cudaEventRecord(B->e0, c->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(B->e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(B->e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, B->e0, B->e1);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      rc = fail(c, FASTCOD_ECUDA, "batch graph launch failed: %s", cudaGetErrorString(e));
      break;
    }
    c->prof.kernel_launches += kernels_per_run(n);
    B->info.tasks = L.ntasks;
    B->info.prefilter_ctas = cfg.ctas;
    B->info.near_log2 = cfg.near_log2;
    B->info.task_vertices = (int64_t)1 << cfg.task_log2;
    B->info.ms_graph = *ms;
  } while (0);
  delete tbl;
  return rc;
}

uint64_t shape_key(const fastcod_subject* subs, int32_t n, uint32_t mode, int prefilter) {
  int64_t nv = 0, maxvox = 0, maxnm = 0;
  for (int32_t i = 0; i < n; ++i) {
    nv += subs[i].n_vertices;
    maxvox = std::max<int64_t>(maxvox, (int64_t)subs[i].dims[0] * subs[i].dims[1] * subs[i].dims[2]);
    maxnm = std::max<int64_t>(maxnm, (int64_t)subs[i].n_roi * subs[i].n_targets);
  }
  return ((uint64_t)n << 40) ^ ((uint64_t)ilog2_64(nv + 1) << 32) ^ ((uint64_t)ilog2_64(maxvox + 1) << 24) ^
         ((uint64_t)ilog2_64(maxnm + 1) << 16) ^ ((uint64_t)mode << 8) ^ (uint64_t)prefilter;
}

void load_tune_cache(BatchState* B) {
  if (B->cache_loaded) return;
  B->cache_loaded = true;
  const char* path = getenv("FASTCOD_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  unsigned long long k;
  int ctas, nl, tl;
  char line[256];
  while (fgets(line, sizeof line, f))
    if (sscanf(line, "%llx %d %d %d", &k, &ctas, &nl, &tl) == 4 && (ctas == 2 || ctas == 3) && nl >= -1 && nl <= 3 &&
        tl >= 12 && tl <= 22)
      B->tuned[(uint64_t)k] = BatchConfig{ctas, nl, tl};
  fclose(f);
}

void save_tune_entry(uint64_t key, const BatchConfig& cfg) {
  const char* path = getenv("FASTCOD_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%llx %d %d %d\n", (unsigned long long)key, cfg.ctas, cfg.near_log2, cfg.task_log2);
  fclose(f);
}

}  // namespace

namespace fcapi {
void batch_free(fastcod_ctx* c) {
  if (!c->batch) return;
  if (c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
  if (c->batch->e0) cudaEventDestroy(c->batch->e0);
  if (c->batch->e1) cudaEventDestroy(c->batch->e1);
  cudaFree(c->batch->arena);
  delete c->batch;
  c->batch = nullptr;
}
}  // namespace fcapi

extern "C" {

FASTCOD_API int fastcod_batch_run(fastcod_ctx* c, const fastcod_subject* subs, int32_t n) {
  fcapi::Range nvtx_range("fastcod_batch_run");
  if (!c) return FASTCOD_EINVAL;
  c->err.clear();
  if (!subs || n < 1 || n > fc::kMaxBatch) return fail(c, FASTCOD_EINVAL, "n_subjects must be in 1..%d", fc::kMaxBatch);
  CU(cudaSetDevice(c->device));
  int64_t total_ns = 0;
  std::vector<int> host_in(4 * (size_t)n, 0);
  std::vector<char> out_dev((size_t)n, 0);
  for (int32_t i = 0; i < n; ++i) {
    const fastcod_subject& S = subs[i];
    if (S.dims[0] <= 0 || S.dims[1] <= 0 || S.dims[2] <= 0)
      return fail(c, FASTCOD_EINVAL, "subject %d: grid dims must be > 0", i);
    if ((int64_t)S.dims[0] * S.dims[1] * S.dims[2] >= ((int64_t)1 << 31))
      return fail(c, FASTCOD_EINVAL, "subject %d: grid has >= 2^31 voxels", i);
    if (S.n_roi <= 0 || S.n_roi >= (1 << 30) || S.n_targets <= 0 || S.n_targets > 65535)
      return fail(c, FASTCOD_EINVAL, "subject %d: need 0 < n_roi < 2^30 and 0 < n_targets < 65536", i);
    if (S.n_streamlines < 1 || S.n_vertices < 0 || S.n_vertices > 0x7fffffffLL)
      return fail(c, FASTCOD_EINVAL, "subject %d: need n_streamlines >= 1 and n_vertices < 2^31", i);
    if (!S.roi_index_map || !S.target_labels || !S.offsets || (S.n_vertices && !S.xyz) || !S.C_out || !S.Cend_out)
      return fail(c, FASTCOD_EINVAL, "subject %d: NULL pointer", i);
    const void* ptrs[4] = {S.roi_index_map, S.target_labels, S.xyz, S.offsets};
    for (int k = 0; k < 4; ++k) {
      const int kind = (k == 2 && !S.n_vertices) ? 1 : ptr_kind(ptrs[k], c->device);
      if (kind < 0) return fail(c, FASTCOD_EINVAL, "subject %d: input is device memory of another device", i);
      host_in[4 * i + k] = kind == 0;
    }
    // device xyz off a 16-byte boundary is staged like host input (the bulk
    // copies of the prefilter need 16-byte aligned sources)
    if (S.n_vertices && ((uintptr_t)S.xyz & 15u)) host_in[4 * i + 2] = true;
    const int kc = ptr_kind(S.C_out, c->device), ke = ptr_kind(S.Cend_out, c->device);
    if (kc < 0 || ke < 0) return fail(c, FASTCOD_EINVAL, "subject %d: output is device memory of another device", i);
    out_dev[i] = kc == 1 && ke == 1;
    total_ns += S.n_streamlines;
  }
  if (total_ns > 0x7fffffffLL) return fail(c, FASTCOD_EINVAL, "more than 2^31-1 streamlines in one batch");
  if (!c->batch) {
    c->batch = new (std::nothrow) BatchState;
    if (!c->batch) return fail(c, FASTCOD_ENOMEM, "host allocation failed");
  }
  BatchState* B = c->batch;
  B->out_dev = out_dev;
  B->info = fastcod_batch_info{};
  B->info.n_subjects = n;
  float ms = 0.f;
  BatchConfig cfg{c->prefilter_ctas, c->near_log2, c->batch_task_log2};
  bool staged = false;
  if (c->autotune) {
    load_tune_cache(B);
    const uint64_t skey = shape_key(subs, n, c->mode, c->prefilter);
    auto it = B->tuned.find(skey);
    if (it != B->tuned.end()) {
      cfg = it->second;
    } else {
      // timed trials: each candidate runs twice (the first run captures its graph)
      const BatchConfig cand[7] = {{2, -1, 16}, {2, -1, 14}, {2, -1, 15}, {2, -1, 18}, {3, -1, 16}, {2, 2, 16}, {2, 0, 16}};
      float best = 1e30f;
      for (const BatchConfig& k : cand) {
        float t = 0.f;
        for (int r = 0; r < 2; ++r) {
          if (int rc = run_config(c, subs, n, host_in, total_ns, k, !staged, &t)) return rc;
          staged = true;
        }
        if (t < best) {
          best = t;
          cfg = k;
        }
      }
      B->tuned[skey] = cfg;
      save_tune_entry(skey, cfg);
      B->info.tuned = 1;
    }
  }
  if (int rc = run_config(c, subs, n, host_in, total_ns, cfg, true, &ms)) return rc;
  // outputs and per-subject state
  void* A = B->arena;
  Layout L = plan(subs, n, host_in, cfg.near_log2, cfg.task_log2, total_ns);
  for (int32_t i = 0; i < n; ++i) {
    if (out_dev[i]) continue;  // accumulated in place
    const size_t nm = (size_t)subs[i].n_roi * (size_t)subs[i].n_targets;
    CU(cudaMemcpyAsync(subs[i].C_out, at<int32_t>(A, L.C[i]), nm * 4, cudaMemcpyDefault, c->stream));
    CU(cudaMemcpyAsync(subs[i].Cend_out, at<int32_t>(A, L.Cend[i]), nm * 4, cudaMemcpyDefault, c->stream));
  }
  B->states.resize(n);
  B->ns.resize(n);
  B->nv.resize(n);
  for (int32_t i = 0; i < n; ++i) {
    B->ns[i] = subs[i].n_streamlines;
    B->nv[i] = subs[i].n_vertices;
  }
  CU(cudaMemcpyAsync(B->states.data(), at<DevState>(A, L.states), sizeof(DevState) * n, cudaMemcpyDeviceToHost,
                     c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int32_t i = 0; i < n; ++i) {
    const DevState& h = B->states[i];
    if (h.error == fc::kErrNone) continue;
    const char* what = h.error == fc::kErrOffsets  ? "offsets invalid"
                       : h.error == fc::kErrCoord  ? "vertex coordinate outside [-2^24, 2^24)"
                       : h.error == fc::kErrVolume ? "volume value out of range"
                                                   : "device error";
    if (h.error == fc::kErrChecked) return fail(c, FASTCOD_ECUDA, "subject %d: bounds check failed (site %d)", i, h.error_info);
    if (h.error == fc::kErrTimeout) return fail(c, FASTCOD_ETIMEOUT, "subject %d: device wait timed out", i);
    return fail(c, FASTCOD_EINVAL, "subject %d: %s (%d)", i, what, h.error_info);
  }
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_batch_get_stats(fastcod_ctx* c, int32_t subject, fastcod_stats* out) {
  if (!c || !out) return FASTCOD_EINVAL;
  if (!c->batch || subject < 0 || subject >= (int32_t)c->batch->states.size())
    return fail(c, FASTCOD_EINVAL, "no such subject in the last batch");
  const DevState& h = c->batch->states[subject];
  out->streamlines = c->batch->ns[subject];
  out->vertices = c->batch->nv[subject];
  out->voxel_steps = (int64_t)h.voxel_steps;
  out->survivors = (int64_t)h.survivors;
  out->overflow = (int64_t)h.overflow;
  out->pairs = (int64_t)h.pairs;
  out->walked_steps = (int64_t)h.walked;
  return FASTCOD_OK;
}

FASTCOD_API int fastcod_batch_get_info(fastcod_ctx* c, fastcod_batch_info* out) {
  if (!c || !out) return FASTCOD_EINVAL;
  if (!c->batch) return fail(c, FASTCOD_ESTATE, "no batch has run");
  *out = c->batch->info;
  return FASTCOD_OK;
}

}  // extern "C"
