// Internal declarations shared by the CUDA translation units of libfastcod.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fc {

// 1 unit = 1/1024 voxel; the voxel of a coordinate is (c >> kUnitLog2).
constexpr int kUnitLog2 = 10;
constexpr int32_t kCoordLimit = 1 << 24;

// Brick occupancy grid: bricks of (1 << kBrickLog2)^3 voxels, two bits per
// brick (bit 0: some voxel has an ROI row, bit 1: some voxel has a label),
// sixteen bricks per 32-bit word.
constexpr int kBrickLog2 = 2;

// Per-voxel code: bit 31 set -> ROI voxel, bits 0..29 = row, bit 30 = the
// voxel also carries a label (read it from the label volume); bit 31 clear
// -> the code is the label (0 = none).
constexpr uint32_t kCodeRoi = 0x80000000u;
constexpr uint32_t kCodeRoiLabelled = 0x40000000u;
constexpr uint32_t kCodeRowMask = 0x3fffffffu;

// Device-detected error codes (first one wins).
enum DevError : int32_t {
  kErrNone = 0,
  kErrOffsets = 1,      // offsets not monotone, out of [0, n_vertices], or bad ends
  kErrCoord = 2,        // coordinate outside [-2^24, 2^24)
  kErrVolume = 3,       // roi or label value out of range
  kErrTimeout = 4,      // a bounded wait gave up
  kErrOverflowList = 5, // overflow list capacity exceeded (cannot happen by construction)
  kErrCount = 6,        // a connectivity count given to the parcellation is negative
  kErrChecked = 7       // checked builds: an index failed its bounds check (error_info: the site)
};

// Sites of the bounds checks of checked builds (FASTCOD_CHECKED=1).
enum CheckSite : int32_t {
  kSiteSurvivorRead = 1,   // survivor id read from the list, and the id itself
  kSiteSurvivorWrite = 2,  // survivor list append (prefilter)
  kSiteCode = 3,           // per-voxel code gather
  kSiteLabel = 4,          // label gather of a labelled ROI voxel
  kSiteNear = 5,           // near-grid word
  kSiteBrick = 6,          // brick-occupancy word
  kSiteVoxelList = 7,      // the walk's list of visited voxels
  kSiteSetList = 8,        // a set's key list
  kSiteC = 9,              // C entry
  kSiteCend = 10,          // C_end entry
  kSiteOverflowList = 11,  // overflow list append
  kSiteVertex = 12,        // vertex read
  kSiteScratch = 13        // overflow path's global sets
};

// Cumulative and per-call counters in device memory.
struct DevState {
  int32_t error;
  int32_t error_info;
  uint32_t n_survivors;   // this call: entries in the survivor list
  uint32_t n_overflow;    // this call: entries in the overflow list
  uint32_t work_next;     // this call: dynamic work counter of the walk kernel
  uint32_t work_task;     // this call: dynamic task counter of the batched prefilter
  uint32_t n_long;        // this call: entries at the far end of the survivor list
  uint32_t spare;
  unsigned long long voxel_steps;
  unsigned long long survivors;
  unsigned long long overflow;
  unsigned long long pairs;
  unsigned long long walked;  // voxel steps of the walked (surviving) streamlines
  int32_t max_roi;        // set_volumes: max(roi) over the volume
  int32_t max_label;      // set_volumes: max(label)
};

// Read-only view of the installed volumes.
struct VolView {
  const uint32_t* code;   // [nvox] per-voxel code
  const uint16_t* lab;    // [nvox] labels (read for labelled ROI voxels)
  const uint32_t* bricks; // brick occupancy words
  const uint32_t* near;   // dilated occupancy (see below)
  int32_t dx, dy, dz;     // grid
  int32_t bx, by, bz;     // brick grid
  int32_t nwx, nny, nnz;  // near grid: words per x-row, rows, planes (in cells)
  int32_t cmx, cmy, cmz;  // near grid: index of the all-zero border cell per axis
  int32_t nsh;            // near grid cell = (1 << nsh)^3 padded voxels
  int32_t n_roi, n_lab;   // N, M
};

// Near grid: for every voxel v of the grid grown by one voxel on each side,
// two bits (bit 0: some voxel within Chebyshev distance 1 of v has an ROI row,
// bit 1: ... has a label), ORed over cells of (1 << nsh)^3 padded voxels,
// sixteen cells along x per 32-bit word.  Voxel (x, y, z) sits at padded
// position (x+1, y+1, z+1), in cell (cx, cy, cz) = padded >> nsh:
//   word = (cx >> 4) + nwx * (cy + nny * cz),  shift = (cx & 15) * 2.
// Past the cells that cover padded positions [0, d + 2) every axis has one
// more cell, all zero (index cmx / cmy / cmz); a lookup clamps its cell
// coordinate, taken as unsigned, to that cell, so any voxel farther than one
// voxel outside the grid reads zero without a bounds test.
// A segment whose end voxels differ by at most one on every axis lies in the
// 3x3x3 block around either end, so the near bits of either end voxel (and
// of the cell holding it) cover it.
inline void set_near_dims(VolView& v, int32_t nsh) {
  const int32_t cs = 1 << nsh;
  v.nsh = nsh;
  v.cmx = (v.dx + 2 + cs - 1) / cs;
  v.cmy = (v.dy + 2 + cs - 1) / cs;
  v.cmz = (v.dz + 2 + cs - 1) / cs;
  v.nwx = (v.cmx + 1 + 15) / 16;
  v.nny = v.cmy + 1;
  v.nnz = v.cmz + 1;
}
__host__ __device__ inline int64_t near_words(const VolView& v) { return (int64_t)v.nwx * v.nny * v.nnz; }

// Cell size for a near-grid option value: 0..3 as given; -1 (automatic) the
// smallest cell whose grid stays within 40960 words (160 KB, so that it
// stays cached near the SMs), at most 3.
inline int32_t resolve_near_log2(int32_t opt, int32_t dx, int32_t dy, int32_t dz) {
  if (opt >= 0) return opt;
  for (int32_t nsh = 0; nsh < 3; ++nsh) {
    VolView v{};
    v.dx = dx;
    v.dy = dy;
    v.dz = dz;
    set_near_dims(v, nsh);
    if (near_words(v) <= 40960) return nsh;
  }
  return 3;
}

// One batch of streamlines on the device.
struct Tract {
  const int32_t* xyz;     // [nv][3]
  const int64_t* off;     // [ns + 1]
  int64_t nv, ns;
};

struct Accum {
  int32_t* C;             // [N][M]
  int32_t* Cend;          // [N][M]
};

// The survivor list of one launch, cap entries: the prefilter appends
// streamlines of at most kLongSegments segments from the front (counter
// n_survivors) and longer ones from the back (n_long); the walk takes the
// long ones first, so that no long walk is left for the end of the launch.
constexpr int32_t kLongSegments = 192;

struct SurvList {
  int32_t* ids;
  int64_t cap;
};

__device__ __forceinline__ int32_t survivor_at(const int32_t* ids, int64_t cap, uint32_t n_long, uint32_t idx) {
  return idx < n_long ? ids[cap - 1 - (int64_t)idx] : ids[idx - n_long];
}

// One subject of a batch: its volumes, streamlines, accumulators, counters,
// and the global id of its first streamline (survivor lists hold global ids).
struct BatchSubject {
  VolView v;
  Tract t;
  Accum acc;
  DevState* st;
  int64_t sbase;
  int64_t task0, ntask;  // its prefilter tasks (when no task table is given): [task0, task0 + ntask)
};

// Up to kMaxBatch subjects travel as one kernel parameter (constant bank).
constexpr int kMaxBatch = 128;
struct BatchTable {
  int32_t n;
  int32_t pad;
  BatchSubject s[kMaxBatch];
};

// Volume preparation of one subject of a batch: its inputs, its volume view
// (outputs code, lab, bricks, near), its bit planes and counters, and the
// first of its blocks in the batched prep and near-grid launches.
struct PrepSubject {
  VolView v;
  const int32_t* roi;
  const uint16_t* lab;
  uint32_t* planes;
  DevState* st;
  int64_t prep_blk0;  // first block of the prep launch
  int64_t near_blk0;  // first block of the near-grid launch
  int32_t* zero0;     // optional: [nzero] words zeroed by the prep launch (the subject's C), and
  int32_t* zero1;     // [nzero] more (its C_end); null when not wanted
  int64_t nzero;
};
struct PrepTable {
  int32_t n;
  int32_t pad;
  int64_t prep_blocks, near_blocks;  // blocks of the two launches
  PrepSubject s[kMaxBatch];
};

// A prefilter task: streamlines [s_lo, s_hi) of one subject.
struct BatchTask {
  int32_t subject;
  int32_t pad;
  int64_t s_lo, s_hi;
};

// Task `task` of a batch without a task table: subject i owns tasks
// [task0, task0 + ntask), which split its streamlines evenly by count.
__device__ __forceinline__ BatchTask batch_task(const BatchTable& tbl, int64_t task) {
  int32_t lo = 0, hi = tbl.n - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (tbl.s[mid].task0 <= task) lo = mid; else hi = mid - 1;
  }
  const BatchSubject& S = tbl.s[lo];
  const int64_t j = task - S.task0, k = S.ntask;
  BatchTask t;
  t.subject = lo;
  t.pad = 0;
  t.s_lo = S.t.ns * j / k;
  t.s_hi = S.t.ns * (j + 1) / k;
  return t;
}

// Mode bits of the walk.
constexpr uint32_t kModeTargetEndpoint = 1u;
constexpr uint32_t kModeVertexSampled = 2u;
constexpr uint32_t kModeWalkAll = 4u;  // walk every segment (no skip of far short segments)

// ---------------------------------------------------------------- launchers
// Each returns the cudaError_t of the launch.

// K1: per-voxel code, label copy and brick bits from the caller's volumes.
cudaError_t launch_volume_max(const int32_t* roi, const uint16_t* lab, int64_t nvox, DevState* st,
                              cudaStream_t s);
// planes: plane_words(dx, dy, dz) words, the ROI and label bit planes.
cudaError_t launch_volume_prep(const int32_t* roi, const uint16_t* lab, int64_t nvox, VolView v,
                               uint32_t* code, uint16_t* lab_out, uint32_t* bricks, uint32_t* planes, DevState* st,
                               cudaStream_t s);
int64_t plane_words(int32_t dx, int32_t dy, int32_t dz);
// Near grid from the bit planes written by launch_volume_prep.
cudaError_t launch_near(const VolView& v, const uint32_t* planes, uint32_t* near, cudaStream_t s);
// Both for every subject of a batch, one launch each; prep_table fills the
// table's block counts (the bricks must be zero beforehand).
void prep_table_blocks(PrepTable& tbl);
cudaError_t launch_volume_prep_batch(const PrepTable& tbl, cudaStream_t s);
cudaError_t launch_near_batch(const PrepTable& tbl, cudaStream_t s);

// K2: prefilter + compaction (+ validation and voxel-step count).
// ctas_per_sm: 2 or 3 (the register budget the kernel is compiled for).
// withhold_piece: test hook (-1 off): the TMA loader skips that piece and its
// barrier arrival, so its bounded wait runs out.
cudaError_t launch_prefilter(const Tract& t, const VolView& v, bool prefilter, uint32_t mode,
                             bool tma, int ctas_per_sm, int32_t* survivors, int64_t survivor_cap, DevState* st,
                             int num_sms, cudaStream_t s, int64_t withhold_piece = -1);

// Batched forms: every subject of the table in one launch each.  tasks:
// a table of ntasks tasks, or null for the tasks the subjects' task0 / ntask
// define.
cudaError_t launch_prefilter_batch(const BatchTable& tbl, const BatchTask* tasks, int32_t ntasks, bool prefilter,
                                   bool tma, int ctas_per_sm, int32_t* survivors, int64_t survivor_cap,
                                   DevState* gst, int num_sms, cudaStream_t s);
cudaError_t launch_walk_batch(const BatchTable& tbl, const int32_t* survivors, int64_t survivor_cap, uint32_t mode,
                              int32_t* overflow_list, DevState* gst, int num_sms, cudaStream_t s);
cudaError_t launch_walk_overflow_batch(const BatchTable& tbl, const int32_t* overflow_list, uint32_t mode,
                                       uint32_t* scratch, int32_t scratch_ctas, int64_t words_per_cta, DevState* gst,
                                       cudaStream_t s);

// K3: warp-per-streamline walk, dedup, accumulate; overflow path.
cudaError_t launch_walk(const Tract& t, const VolView& v, const int32_t* survivors, int64_t survivor_cap,
                        Accum acc, uint32_t mode, int32_t* overflow_list, DevState* st, int num_sms,
                        cudaStream_t s);
cudaError_t launch_walk_overflow(const Tract& t, const VolView& v, const int32_t* overflow_list,
                                 Accum acc, uint32_t mode, uint32_t* scratch,
                                 int32_t scratch_ctas, DevState* st, cudaStream_t s);
// Voxel steps of the survivors (warp per survivor), added to st->walked.
cudaError_t launch_walked_steps(const Tract& t, const int32_t* survivors, int64_t survivor_cap, DevState* st,
                                int num_sms, cudaStream_t s);
// words of global scratch one overflow CTA needs for N rows and M labels
int64_t overflow_scratch_words(int32_t n_roi, int32_t n_lab);

// Beside the path (k_aux.cu): parcellation of an N x M matrix (frac may be
// null; st, when given, receives kErrCount for a negative entry), world-mm ingest, offsets check, upsampling (offsets, then
// vertices; block_tmp holds upsample_scan_blocks(ns) values), rescale.
cudaError_t launch_parcellate(const int32_t* C, int32_t N, int32_t M, int32_t* label, float* frac, DevState* st,
                              cudaStream_t s);
cudaError_t launch_world_to_fixed(const float* xyz_mm, int64_t nv, const float affine[12], int32_t* out,
                                  DevState* st, cudaStream_t s);
cudaError_t launch_check_offsets(const int64_t* off, int64_t ns, int64_t nv, DevState* st, cudaStream_t s);
// Checkpoint check: out[0] += sum of C, out[1] += sum of C_end (both [nm]),
// out[2] = min(out[2], the first index over C then C_end, 2 nm entries,
// whose entry lies outside [0, max_count]).
cudaError_t launch_checkpoint_check(const int32_t* C, const int32_t* Cend, int64_t nm, int32_t max_count,
                                    unsigned long long* out, cudaStream_t s);
cudaError_t launch_seg_max(const int32_t* xyz, const int64_t* off, int64_t ns, unsigned long long* best,
                           cudaStream_t s);
int64_t upsample_scan_blocks(int64_t ns);
cudaError_t launch_upsample_offsets(const int64_t* off, int64_t ns, int32_t factor, long long* block_tmp,
                                    int64_t* out_off, cudaStream_t s);
cudaError_t launch_upsample_vertices(const int32_t* xyz, const int64_t* off, int64_t ns, int32_t factor,
                                     const int64_t* out_off, int32_t* out, cudaStream_t s);
cudaError_t launch_rescale(const int32_t* xyz, int64_t nv, const int32_t num[3], const int32_t den[3],
                           const int64_t add[3], int32_t* out, DevState* st, cudaStream_t s);

}  // namespace fc
