// Host-side internals of libfastcod shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "fastcod.h"
#include "fc_internal.cuh"

using fc::DevState;

struct BatchState;

struct fastcod_ctx {
  int device = 0;
  uint32_t flags = 0;
  int num_sms = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;

  // volumes
  bool has_vol = false;
  int32_t dims[3] = {0, 0, 0};
  int32_t bdims[3] = {0, 0, 0};
  int32_t N = 0, M = 0;
  int32_t near_shift = 1;  // cell size of the installed near grid
  uint32_t* d_code = nullptr;
  uint16_t* d_lab = nullptr;
  uint32_t* d_bricks = nullptr;
  uint32_t* d_near = nullptr;
  int32_t* d_C = nullptr;
  int32_t* d_Cend = nullptr;
  uint32_t* d_scratch = nullptr;
  int32_t scratch_ctas = 0;

  // staging of host inputs and per-call lists
  void* d_vstage = nullptr;
  size_t vstage_bytes = 0;
  int32_t* d_xyz = nullptr;
  size_t xyz_bytes = 0;
  int64_t* d_off = nullptr;
  size_t off_bytes = 0;
  int32_t* d_surv = nullptr;
  size_t surv_bytes = 0;
  int32_t* d_ovf = nullptr;
  size_t ovf_bytes = 0;

  DevState* d_state = nullptr;
  unsigned long long* d_check = nullptr;  // fastcod_restore: sums of C and C_end, first entry out of range
  size_t check_bytes = 0;

  int64_t total_streamlines = 0;
  int64_t total_vertices = 0;
  int prefilter = 1;
  uint32_t mode = 0;
  int staging_tma = 1;
  int prefilter_ctas = 2;
  int near_log2 = -1;      // near grid cell: (1 << near_log2)^3 voxels; -1 = per volume
  int autotune = 1;        // batched form: tune per batch shape
  int batch_task_log2 = 16; // batched form without the autotuner: prefilter tasks of about 2^value vertices
  int host_in_place = 0;   // read page-locked host xyz in place (option)
  int walked_steps = 0;    // count the survivors' voxel steps (option)
  int64_t withhold_piece = -1;  // test hook: vertex piece the TMA loader never copies
  int profile = 0;
  struct EvSet {
    cudaEvent_t e[5];
    bool no_h2d;  // the call copied nothing to the device: e[0] was not recorded
  };
  std::vector<EvSet> ev_pool;  // event sets of profiled calls
  size_t ev_used = 0;          // sets recorded and not yet folded into prof
  EvSet* ev_cur = nullptr;
  fastcod_profile prof = {0, 0, 0.0, 0.0, 0.0, 0.0, 0, 0.0};
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};  // kernel spans of the calls beside the path

  // device scratch of the entry points beside the path (aux_capi.cu)
  static constexpr int kAuxSlots = 6;
  void* d_aux[kAuxSlots] = {};
  size_t aux_bytes[kAuxSlots] = {};

  std::string err;
  BatchState* batch = nullptr;  // batched form (batch.cu)
};

namespace fcapi {
// An NVTX range around a call of the C ABI (shown by Nsight tools; a no-op
// when no tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
// Record a message on ctx (if any) and return code.
int fail(fastcod_ctx* c, int code, const char* fmt, ...);
// 0 = host memory, 1 = device memory of dev, -1 = device memory elsewhere.
int ptr_kind(const void* p, int dev);
// Device address of page-locked (mapped) host memory; nullptr for anything else.
const void* mapped_host(const void* p);
// Grow a device buffer to at least need bytes (synchronises before freeing).
int grow(fastcod_ctx* c, void** p, size_t* cap, size_t need);
// Synchronise the context's stream and turn a device-detected error into a
// status.
int sync_check(fastcod_ctx* c);
// Release the batched form's state (batch.cu).
void batch_free(fastcod_ctx* c);
// Message of the last failed call on this thread that has no context.
std::string& thread_error();
}  // namespace fcapi

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      (void)cudaGetLastError();                                                                    \
      return fcapi::fail(c, e_ == cudaErrorMemoryAllocation ? FASTCOD_ENOMEM : FASTCOD_ECUDA,       \
                         "%s: %s", #call, cudaGetErrorString(e_));                                  \
    }                                                                                              \
  } while (0)
