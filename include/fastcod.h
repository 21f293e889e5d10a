/*
 * fastcod.h - C ABI of libfastcod, a GB300 (sm_103a) implementation of the
 * pass-through brain connectivity matrix of FastCod (Bian et al., "FastCod:
 * Fast Brain Connectivity in Diffusion Imaging", arXiv 2302.09247).
 *
 * What is computed (Section 2, Algorithm 2): for ROI voxels v_1..v_N and
 * target regions R_1..R_M, a streamline l = {p^1..p^T} adds exactly 1 to
 * C[v][t] when it passes through ROI voxel v and through target region t,
 * wherever it starts or ends.  "Passes through" is the exact continuous
 * polyline: the voxels whose half-open boxes meet any of its closed segments
 * (a single-vertex streamline is its one point).  Each streamline counts
 * once per (v, t) pair.  The traditional seed-to-endpoint count of
 * Algorithm 1 (first vertex = seed, region of the last vertex) is kept beside
 * it as C_end.  All counts are exact integers.
 *
 * Units and layouts:
 *   - vertices are int32 fixed point, 1 unit = 1/1024 voxel; voxel (i,j,k)
 *     covers [1024 i, 1024 i + 1024) x [1024 j, ..) x [1024 k, ..), so the
 *     voxel of a vertex is its coordinates shifted right by 10 (floor, also
 *     for negative values); every coordinate must lie in [-2^24, 2^24);
 *   - xyz is [n_vertices][3] (x, y, z interleaved); offsets is int64
 *     [n_streamlines + 1] with offsets[0] = 0, non-decreasing,
 *     offsets[n_streamlines] = n_vertices; streamline s is vertices
 *     offsets[s] .. offsets[s+1]-1;
 *   - volumes are x-fastest: lin(i,j,k) = i + Dx*(j + Dy*k);
 *     roi_index_map[lin] is the ROI row of the voxel (-1 = not in the ROI;
 *     several voxels may share a row); target_labels[lin] is the target
 *     region 1..M (0 = none); a voxel may be both;
 *   - C and C_end are int32 [N][M] row-major; C[r][t-1] is the count for row
 *     r and label t.
 *
 * Pointers: every input and output pointer may be host memory (pageable or
 * page-locked) or device memory of the context's device; the library tells
 * them apart with cudaPointerGetAttributes.  Device xyz that does not start
 * on a 16-byte boundary (4-byte alignment, as for any int32 array, is
 * required) is first copied to an aligned buffer of the library: one more
 * pass over the vertices.  The caller owns every buffer it passes.  Work is ordered
 * on the context's stream; device inputs and page-locked host inputs must
 * stay unchanged until the next synchronising call (fastcod_connectivity,
 * fastcod_endpoint_connectivity, fastcod_get_stats, fastcod_sync) or a sync
 * of that stream; pageable host inputs may be reused when the call returns.
 *
 * Errors: every function returns FASTCOD_OK (0) or a negative FASTCOD_E*
 * code and records a message readable with fastcod_last_error.  Errors found
 * on the device (invalid offsets or coordinates in device inputs, a bounded
 * wait that ran out) are reported by the next synchronising call; after one,
 * C and C_end are undefined until fastcod_reset.  No C++ exception crosses
 * this interface.  A context is not thread-safe: one thread at a time.
 */
#ifndef FASTCOD_H
#define FASTCOD_H

#include <stdint.h>

#if defined(__GNUC__)
#define FASTCOD_API __attribute__((visibility("default")))
#else
#define FASTCOD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FASTCOD_OK = 0,
  FASTCOD_EINVAL = -1,    /* invalid argument or input data */
  FASTCOD_ENOMEM = -2,    /* device or host allocation failed */
  FASTCOD_ECUDA = -3,     /* a CUDA runtime call failed */
  FASTCOD_ESTATE = -4,    /* call out of order (e.g. streamlines before volumes) */
  FASTCOD_EOVERFLOW = -5, /* more than 2^31 - 1 streamlines since the last reset */
  FASTCOD_ETIMEOUT = -6,  /* a bounded device-side wait gave up */
  FASTCOD_ECANCELED = -7  /* request cancelled (serving) */
};

/* fastcod_create flags */
#define FASTCOD_SYNC 1u /* every call waits for its GPU work before returning */

/* fastcod_set_option keys */
enum {
  /* 1 (default): before the walk, drop the streamlines that pass near no ROI
   * voxel or near no labelled voxel (a conservative test: the near grid at
   * the even vertices, the brick occupancy of long segments' voxel boxes);
   * 0: walk every streamline.  Results are identical. */
  FASTCOD_OPT_PREFILTER = 1,
  /* target rule: 0 (default) = every label the streamline passes through;
   * 1 = only the label of the last vertex (Algorithm 2 taken literally,
   * r_j = loc2region(p^T)).  Takes effect for streamlines added afterwards. */
  FASTCOD_OPT_TARGET_MODE = 2,
  /* voxel rule: 0 (default) = continuous segments; 1 = vertices only (the
   * point-sampled reading behind the paper's upsampling rule, Section 3). */
  FASTCOD_OPT_SAMPLING = 3,
  /* vertex staging of the prefilter: 1 (default) = 1-D TMA bulk copies into
   * a per-warp shared-memory ring, 0 = direct vectorised streaming loads into
   * registers.  Results are identical. */
  FASTCOD_OPT_STAGING = 4,
  /* 1: record CUDA events around every stage on the context's stream and
   * accumulate their durations (fastcod_get_profile); 0 (default): off. */
  FASTCOD_OPT_PROFILE = 5,
  /* Register budget of the prefilter, in 8-warp CTAs per SM: 2 (default: 16
   * warps per SM at up to 128 registers a thread, run as one CTA of 16 warps
   * by the single-subject call and as two of 8 by the batched and served
   * forms) or 3 (24 warps at 80 registers, three CTAs of 8).  Results are
   * identical. */
  FASTCOD_OPT_PREFILTER_CTAS = 6,
  /* cell of the near grid (the prefilter's test, and the walk's skip of
   * segments far from every ROI and labelled voxel): (1 << value)^3 voxels,
   * 0..3, or -1 (default): per volume, the smallest cell whose grid has at
   * most 40960 words (160 KB).  Coarser cells keep the grid closer to the SMs
   * and let more streamlines through to the exact walk.  Results are
   * identical.  Applies to volumes installed afterwards. */
  FASTCOD_OPT_NEAR_LOG2 = 7,
  /* 1 (default): fastcod_batch_run picks the prefilter's CTAs per SM, the
   * near-grid cell and the work granularity of a prefilter task (vertices per
   * task) per batch shape by timed trials on the first batch of that shape
   * (cached in the context, and in the file named by the environment
   * variable FASTCOD_TUNE_CACHE when set); 0: use the options as set, with
   * the work granularity of FASTCOD_OPT_BATCH_TASK_LOG2. */
  FASTCOD_OPT_AUTOTUNE = 8,
  /* 1: fastcod_add_streamlines reads page-locked (mapped) host xyz in place,
   * the kernels streaming it over the host link while they compute (16-byte
   * aligned xyz; otherwise it is copied); 0 (default): page-locked xyz is
   * first copied to device memory (measured faster on GB300).  Host offsets
   * and pageable host inputs are always copied.  Results are identical. */
  FASTCOD_OPT_HOST_IN_PLACE = 9,
  /* 1: fastcod_add_streamlines also counts the voxel steps of the walked
   * streamlines (fastcod_stats.walked_steps), with one more kernel that reads
   * the survivors' vertices again; 0 (default): not counted (0). */
  FASTCOD_OPT_WALKED_STEPS = 10,
  /* 1 (default): the walk skips a short segment (end voxels at most one
   * apart on every axis) whose start voxel's near cell holds no ROI and no
   * labelled voxel: every voxel it visits lies within that cell's reach and
   * counts for nothing.  0: every segment is walked voxel by voxel (with
   * FASTCOD_OPT_PREFILTER = 0, every voxel step of the input is taken; the
   * benchmark's measure of the integer DDA itself).  Results are identical. */
  FASTCOD_OPT_SEGMENT_SKIP = 11,
  /* Test hook for the bounded waits: -1 (default) off; k >= 0: the
   * prefilter's bulk-copy loader neither copies the vertex piece k (vertices
   * 256 k .. 256 k + 255) nor arrives on its barrier, so the wait for that
   * piece runs out after its one-second limit.  The call then reports
   * FASTCOD_ETIMEOUT (at the next synchronising call), no copy is left in
   * flight, and the context stays usable after fastcod_reset. */
  FASTCOD_OPT_TEST_WITHHOLD_PIECE = 12,
  /* Work granularity of fastcod_batch_run's prefilter when the autotuner is
   * off: dynamic tasks of about 2^value vertices of one subject, 12..22
   * (default 16).  Results are identical. */
  FASTCOD_OPT_BATCH_TASK_LOG2 = 13
};

typedef struct fastcod_ctx fastcod_ctx;

typedef struct {
  int64_t streamlines;  /* streamlines added since the last reset */
  int64_t vertices;     /* vertices added since the last reset */
  int64_t voxel_steps;  /* sum over segments of 1 + sum_a |floor(p1_a) - floor(p0_a)|,
                           a single-vertex streamline counting 1 */
  int64_t survivors;    /* streamlines that passed the prefilter and were walked */
  int64_t overflow;     /* walked streamlines whose sets exceeded the on-chip
                           tables and took the exact global-memory path */
  int64_t pairs;        /* sum over streamlines of |V_s| * |T_s| (increments of C) */
  int64_t walked_steps; /* voxel_steps of the survivors only (the streamlines walked);
                           counted while FASTCOD_OPT_WALKED_STEPS is 1 */
} fastcod_stats;

/* Per-stage device time accumulated while FASTCOD_OPT_PROFILE is 1 (CUDA
 * events on the context's stream), and the library's kernel launches. */
typedef struct {
  int64_t calls;           /* fastcod_add_streamlines calls profiled */
  int64_t kernel_launches; /* kernels this library launched (all calls, profiled or not) */
  double ms_h2d;           /* host-to-device copies of streamline inputs */
  double ms_prefilter;     /* K2: prefilter + compaction */
  double ms_walk;          /* K3: walk + dedup + accumulate */
  double ms_overflow;      /* exact global-memory path for oversized sets */
  int64_t aux_calls;       /* calls beside the path profiled (parcellate, world-mm
                              conversion, upsample, rescale) */
  double ms_aux;           /* their kernels' device time (the host-side checks and
                              synchronisations between kernels excluded) */
} fastcod_profile;

/* Create a context on CUDA device cuda_device.  Allocates only small state;
 * volumes and streamline buffers are sized by the calls that need them.
 * *out receives the context (NULL on error). */
FASTCOD_API int fastcod_create(fastcod_ctx** out, int cuda_device, uint32_t flags);

/* Free the context and every device buffer it owns.  NULL-safe. */
FASTCOD_API int fastcod_destroy(fastcod_ctx* ctx);

/* Order the context's work on cuda_stream (a cudaStream_t of the context's
 * device; NULL = the context's own non-blocking stream). */
FASTCOD_API int fastcod_set_stream(fastcod_ctx* ctx, void* cuda_stream);

/* Install the volumes (Section 2: the ROI voxel set V = {v_1..v_N} and the
 * target regions R = {R_1..R_M}; loc2region).  dims are Dx, Dy, Dz (> 0,
 * product < 2^31).  n_roi = N (0: max(roi)+1); n_targets = M (0: max label).
 * Requires -1 <= roi < N, label <= M, N < 2^30, M < 65536.  Zeroes C,
 * C_end and the statistics.  Blocks until the volumes are validated. */
FASTCOD_API int fastcod_set_volumes(fastcod_ctx* ctx, const int32_t* roi_index_map,
                                    const uint16_t* target_labels, int32_t dim_x, int32_t dim_y,
                                    int32_t dim_z, int32_t n_roi, int32_t n_targets);

/* Accumulate streamlines into C and C_end (the passthrough count of
 * Algorithm 2 for every streamline; Algorithm 1's count for C_end).  May be
 * called many times; the result depends only on the multiset of streamlines
 * added.  At most 2^31 - 1 vertices per call. */
FASTCOD_API int fastcod_add_streamlines(fastcod_ctx* ctx, const int32_t* xyz, int64_t n_vertices,
                                        const int64_t* offsets, int64_t n_streamlines);

/* Wait for all queued work and copy C (int32 [N][M]) to C_out. */
FASTCOD_API int fastcod_connectivity(fastcod_ctx* ctx, int32_t* C_out);

/* Wait for all queued work and copy C_end (int32 [N][M]) to Cend_out. */
FASTCOD_API int fastcod_endpoint_connectivity(fastcod_ctx* ctx, int32_t* Cend_out);

/* Zero C, C_end and the statistics; keep the volumes.  Stream-ordered: it
 * does not wait for queued work. */
FASTCOD_API int fastcod_reset(fastcod_ctx* ctx);

/* N and M of the installed volumes (ESTATE before fastcod_set_volumes). */
FASTCOD_API int fastcod_get_shape(const fastcod_ctx* ctx, int32_t* n_roi, int32_t* n_targets);

/* Wait for all queued work and read the statistics. */
FASTCOD_API int fastcod_get_stats(fastcod_ctx* ctx, fastcod_stats* out);

/* Resume from a checkpoint.  A checkpoint of a context is its C
 * (fastcod_connectivity), its C_end (fastcod_endpoint_connectivity) and its
 * statistics (fastcod_get_stats), taken between fastcod_add_streamlines
 * calls.  fastcod_restore installs one in a context whose volumes give the
 * same N and M (the same context after a reset, or a new one, in another
 * process for instance): C, C_end and the statistics are replaced by the
 * checkpoint's, and later fastcod_add_streamlines calls add to them.  Each
 * streamline adds its own terms to C and C_end (Algorithm 2, Algorithm 1)
 * and to streamlines, vertices, voxel_steps and pairs, so a pass split at
 * any streamline boundary, checkpointed and resumed, ends with those of one
 * uninterrupted pass.  survivors, overflow and walked_steps count work done
 * and can differ: the prefilter's verdict on a streamline (conservative
 * either way) depends on where the streamline sits in its call's arrays.
 *   C_in, Cend_in: int32 [N][M] row-major, host or device memory of the
 *     context's device, read before the call returns (may be NULL when
 *     N * M = 0).
 *   stats: the checkpoint's statistics; streamlines in [0, 2^31 - 1], every
 *     count >= 0, survivors <= streamlines, overflow <= survivors,
 *     walked_steps <= voxel_steps.
 * The matrices are checked on the device against what every pass
 * satisfies: each entry in [0, stats->streamlines], the entries of C summing
 * to stats->pairs (one increment per (v, t) pair), those of C_end to at most
 * stats->streamlines (at most one per streamline).  A checkpoint that fails
 * a check gives FASTCOD_EINVAL and leaves C, C_end and the statistics zero,
 * as after fastcod_reset.  ESTATE before fastcod_set_volumes.  Blocking. */
FASTCOD_API int fastcod_restore(fastcod_ctx* ctx, const int32_t* C_in, const int32_t* Cend_in,
                                const fastcod_stats* stats);

/* Wait for all queued work and report any device-detected error. */
FASTCOD_API int fastcod_sync(fastcod_ctx* ctx);

/* Wait for all queued work and read the profile (zeroed when profiling is
 * switched on; fastcod_reset keeps it). */
FASTCOD_API int fastcod_get_profile(fastcod_ctx* ctx, fastcod_profile* out);

/* Set an option (FASTCOD_OPT_*). */
FASTCOD_API int fastcod_set_option(fastcod_ctx* ctx, int32_t key, int64_t value);

/* ---------------------------------------------------------------- batched
 * Many subjects in one pass: every subject's volumes are prepared, all
 * subjects' streamlines are prefiltered in one launch (dynamic tasks of one
 * subject's streamline range each), all survivors walked in one launch, the
 * whole sequence captured once per batch shape as a CUDA graph and replayed.
 * Each subject's C and C_end are computed from zero, exactly as
 * fastcod_set_volumes + fastcod_add_streamlines would, and written to its
 * caller-allocated outputs: outputs in device memory of the context's GPU
 * are zeroed and accumulated in place by the pass (so no output may overlap
 * another subject's outputs or any input of the batch), others are copied
 * out after it.  Pointers follow the same host/device rules as the
 * single-subject calls.  The context's installed volumes and accumulators
 * are not touched. */
typedef struct {
  const int32_t* roi_index_map;   /* [Dz][Dy][Dx], -1 or a row < n_roi */
  const uint16_t* target_labels;  /* [Dz][Dy][Dx], 0 or a label <= n_targets */
  int32_t dims[3];                /* Dx, Dy, Dz */
  int32_t n_roi;                  /* N (> 0, given explicitly) */
  int32_t n_targets;              /* M (> 0, given explicitly) */
  const int32_t* xyz;             /* [n_vertices][3] (device xyz off 16 bytes is staged) */
  int64_t n_vertices;
  const int64_t* offsets;         /* [n_streamlines + 1] */
  int64_t n_streamlines;
  int32_t* C_out;                 /* [N][M] */
  int32_t* Cend_out;              /* [N][M] */
} fastcod_subject;

typedef struct {
  int32_t n_subjects;
  int32_t tasks;          /* prefilter tasks of the last batch */
  int32_t prefilter_ctas; /* configuration the last batch ran with */
  int32_t near_log2;      /* -1: the per-volume automatic cell */
  int32_t graph_reused;   /* 1: the last batch replayed a captured graph */
  int32_t tuned;          /* 1: the last batch ran the autotuner's trials */
  double ms_graph;        /* device time of the last batch's graph (CUDA events) */
  int64_t task_vertices;  /* work granularity: about this many vertices per prefilter task */
} fastcod_batch_info;

/* Run a batch of 1..128 subjects (the sum of their streamlines < 2^31).
 * Blocks until every output is written; errors name the subject. */
FASTCOD_API int fastcod_batch_run(fastcod_ctx* ctx, const fastcod_subject* subjects, int32_t n_subjects);

/* Statistics of subject i of the last batch. */
FASTCOD_API int fastcod_batch_get_stats(fastcod_ctx* ctx, int32_t subject, fastcod_stats* out);

/* Shape and configuration of the last batch. */
FASTCOD_API int fastcod_batch_get_info(fastcod_ctx* ctx, fastcod_batch_info* out);

/* ---------------------------------------------------------------- served
 * A request loop with continuous batching.  A request names its volumes and
 * outputs (a fastcod_subject whose xyz / offsets fields are ignored) and then
 * receives its streamlines in chunks.  A worker thread admits waiting
 * requests in arrival order while a slot is free and the HBM reserved for
 * admitted requests (volumes, partial C and C_end, chunk staging) stays
 * within the budget; admitted requests keep their volumes and partial C on
 * the device.  Each iteration of the loop runs one batched pass over the next
 * chunk of every active request, so requests that arrive while others run
 * join the next pass and their work overlaps on the device; chunk uploads
 * run on a copy stream beside the compute stream.  When a request's last
 * chunk is done its C and C_end are written to its outputs.  The result of a
 * request does not depend on the other requests in the mix.
 *
 * Chunk buffers (host or device) must stay valid and unchanged until the
 * request is done.  Server calls are thread-safe; the context must outlive
 * the server and is only read (device, options) at creation. */
typedef struct fastcod_server fastcod_server;

typedef struct {
  int32_t status;       /* FASTCOD_OK, an error, or FASTCOD_ECANCELED (valid when done) */
  int32_t done;
  int64_t streamlines;  /* streamlines processed */
  int64_t chunks;       /* chunks processed */
  double t_submit;      /* seconds since the server was created */
  double t_admit;
  double t_done;
} fastcod_request_info;

/* max_slots: 1..128 requests on the device at once; hbm_budget_bytes: device
 * memory the server may reserve for admitted requests (0: 90% of the free
 * memory at creation).  Host chunks are copied into device staging buffers
 * that the server keeps for its life and reuses (at most 2 * max_slots + 2
 * of them, each the size of the largest chunk it held rounded up to 64 MiB;
 * more in flight at once are freed after their pass).
 *
 * Failure injection for tests, on the host only: when the environment
 * variable FASTCOD_FAULT holds comma-separated items "alloc:k", "h2d:k" or
 * "cancel:k" (k >= 1) at creation, the server's k-th per-request device
 * allocation (a request's volumes and accumulators at admission, or a host
 * chunk's staging buffer) fails as if device memory were exhausted (the
 * request ends with FASTCOD_ENOMEM), its k-th copy of a host chunk fails
 * (FASTCOD_ECUDA), or its k-th submitted request is cancelled on
 * submission (FASTCOD_ECANCELED).  The other requests are unaffected. */
FASTCOD_API int fastcod_server_create(fastcod_ctx* ctx, int32_t max_slots, int64_t hbm_budget_bytes,
                                      fastcod_server** out);

/* Queue a request; *request_id receives its id. */
FASTCOD_API int fastcod_server_submit(fastcod_server* srv, const fastcod_subject* request_head,
                                      uint64_t* request_id);

/* Append a chunk of streamlines (offsets relative to the chunk: offsets[0] =
 * 0, offsets[n_streamlines] = n_vertices); last = 1 marks the final chunk
 * (an empty last chunk is allowed). */
FASTCOD_API int fastcod_server_push_chunk(fastcod_server* srv, uint64_t request_id, const int32_t* xyz,
                                          int64_t n_vertices, const int64_t* offsets, int64_t n_streamlines,
                                          int32_t last);

/* *done = 1 once the request finished; returns its status then. */
FASTCOD_API int fastcod_server_poll(fastcod_server* srv, uint64_t request_id, int32_t* done);

/* Block until the request finished or timeout_s passed (ETIMEOUT). */
FASTCOD_API int fastcod_server_wait(fastcod_server* srv, uint64_t request_id, double timeout_s);

/* Cancel a request (its outputs are not written; status ECANCELED). */
FASTCOD_API int fastcod_server_cancel(fastcod_server* srv, uint64_t request_id);

/* Timing and counts of a request. */
FASTCOD_API int fastcod_server_request_info(fastcod_server* srv, uint64_t request_id, fastcod_request_info* out);

/* Kernels of this library the server's worker has launched so far (volume
 * prep and near grid per admitted request, three per iteration). */
FASTCOD_API int fastcod_server_kernel_launches(fastcod_server* srv, int64_t* out);

/* Finish all admitted and queued work, stop the worker, free everything. */
FASTCOD_API int fastcod_server_destroy(fastcod_server* srv);

/* ---------------------------------------------------- beside the path
 * Outputs and inputs around the connectivity matrix.  Pointers may be host
 * or device memory of the context's device; every call blocks until its
 * outputs are written.  Errors these calls find leave C and C_end as they
 * were. */

/* Parcellation outputs of C (which = 0) or C_end (which = 1) (Section 3,
 * "Pie-glyphs": the single-colour display shows, per source voxel, the region
 * with the highest connectivity; the pie-glyph shows its relative
 * connectivity strength to every region):
 *   label_out[r]      (int32 [N]) = 1 + argmax_t C[r][t], ties to the lowest
 *                     label; 0 for a row of zeros;
 *   fractions_out[r][t] (binary32 [N][M], may be NULL) = C[r][t] / sum_t
 *                     C[r][t] rounded to the nearest binary32 (ties to even);
 *                     0 for a row of zeros.
 * Waits for the queued work first (ESTATE without volumes). */
FASTCOD_API int fastcod_parcellate(fastcod_ctx* ctx, int32_t which, int32_t* label_out, float* fractions_out);

/* The same outputs for a caller's int32 matrix C [N][M] (row-major, host or
 * device memory), for instance the sum of partial matrices that several
 * contexts or GPUs accumulated over parts of one tractogram.  Needs no
 * volumes.  EINVAL when N < 0, M is outside [1, 65535] or an entry is
 * negative (the message names the row); C, C_end and the statistics of the
 * context are left as they were. */
FASTCOD_API int fastcod_parcellate_matrix(fastcod_ctx* ctx, const int32_t* C, int32_t N, int32_t M,
                                          int32_t* label_out, float* fractions_out);

/* World-mm vertices (binary32 [n][3], the form tractography writes) to this
 * library's fixed point: v_a = ((A[a][0] x + A[a][1] y) + A[a][2] z) +
 * A[a][3], every product and sum rounded to binary32 (no fused multiply-add),
 * then round(v_a * 1024) to the nearest integer, ties to even.  affine is the
 * row-major 3 x 4 world -> voxel matrix in this library's voxel units (voxel
 * i spans [i, i+1); for an image affine that maps voxel centres, add 0.5 to
 * its translation).  EINVAL when a result is not finite or falls outside
 * [-2^24, 2^24). */
FASTCOD_API int fastcod_world_to_fixed(fastcod_ctx* ctx, const float* xyz_mm, int64_t n_vertices,
                                       const float affine[12], int32_t* xyz_out);

/* fastcod_world_to_fixed into the context's buffer, then
 * fastcod_add_streamlines on it. */
FASTCOD_API int fastcod_add_streamlines_mm(fastcod_ctx* ctx, const float* xyz_mm, int64_t n_vertices,
                                           const int64_t* offsets, int64_t n_streamlines, const float affine[12]);

/* Streamline upsampling (Section 3, "Super-resolving connectivity features":
 * evenly spaced points inserted between neighbouring points, so that
 * connectivity can be computed on a finer grid than the tractography's).
 * Every segment p -> q becomes `factor` segments through the points
 * p + floor((q - p) * j / factor), j = 0 .. factor-1, followed by the
 * streamline's last vertex: a streamline of T >= 1 vertices gets
 * (T - 1) * factor + 1, an empty one none.  n_vertices_out must equal that
 * total ((n_vertices - non-empty streamlines) * factor + non-empty
 * streamlines; EINVAL otherwise); offsets_out has n_streamlines + 1 entries.
 * factor in [1, 2^20]. */
FASTCOD_API int fastcod_upsample(fastcod_ctx* ctx, const int32_t* xyz, int64_t n_vertices, const int64_t* offsets,
                                 int64_t n_streamlines, int32_t factor, int32_t* xyz_out, int64_t n_vertices_out,
                                 int64_t* offsets_out);

/* The smallest upsampling factor k >= 1 with |q - p|^2 <= (k * spacing)^2
 * on every segment (exact integers; the paper's rule of thumb takes spacing
 * at most half the target voxel, i.e. 512 units for the grid the vertices are
 * in).  EINVAL when k would exceed 2^20. */
FASTCOD_API int fastcod_upsample_factor(fastcod_ctx* ctx, const int32_t* xyz, int64_t n_vertices,
                                        const int64_t* offsets, int64_t n_streamlines, int32_t spacing,
                                        int32_t* factor_out);

/* Integer rescale of fixed-point vertices between grids (for instance from
 * the diffusion grid to a finer structural grid):
 * out_a = floor((p_a * num[a] + add[a]) / den[a]), exact in 64-bit integers,
 * num and den positive.  EINVAL when a result falls outside [-2^24, 2^24). */
FASTCOD_API int fastcod_rescale(fastcod_ctx* ctx, const int32_t* xyz, int64_t n_vertices, const int32_t num[3],
                                const int32_t den[3], const int64_t add[3], int32_t* xyz_out);

/* ------------------------------------------------------- allocation-free
 * C and C_end of one subject with no device allocation at all, neither by
 * the caller nor by the library.  It serves callers that cannot allocate
 * device memory: a host application whose own allocator owns every byte of
 * device memory, or a process already at its memory limit, can still run the
 * computation on buffers it already holds.  The paper has no counterpart;
 * this is an interface of this library.
 *
 * Every pointer must be device memory of cuda_device: the volumes, the
 * streamlines (xyz 16-byte alignment not required) and the outputs C_out and
 * Cend_out (int32 [N][M], overwritten with the result).  Work is ordered on
 * cuda_stream (NULL: the default stream) and the call returns once it is
 * done.  Limits: 1 <= n_roi <= 16384 and 1 <= n_targets <= 1023; larger
 * problems are rejected with FASTCOD_EINVAL (use the context API).  Other
 * validation and results are those of fastcod_set_volumes +
 * fastcod_add_streamlines + fastcod_connectivity /
 * fastcod_endpoint_connectivity.
 *
 * Its working memory is one fixed device array of the library (2.3 MB),
 * present on every device that loads the library until the process exits,
 * and shared by every call on that device: each call clears it first, so
 * calls that overlap on the GPU (on different streams or host threads) race
 * and must not be issued.  The first call on a device looks up the array's
 * device address with cudaGetSymbolAddress; make that first call before any
 * stream capture.  Error messages: fastcod_last_error(NULL). */
FASTCOD_API int fastcod_connectivity_noalloc(int cuda_device, void* cuda_stream, const int32_t* roi_index_map,
                                             const uint16_t* target_labels, int32_t dim_x, int32_t dim_y,
                                             int32_t dim_z, int32_t n_roi, int32_t n_targets, const int32_t* xyz,
                                             int64_t n_vertices, const int64_t* offsets, int64_t n_streamlines,
                                             int32_t* C_out, int32_t* Cend_out);

/* Message of the last error on this context ("" if none); owned by ctx,
 * valid until the next call on it.  NULL ctx: message of the last failed
 * fastcod_create or fastcod_connectivity_noalloc on this thread. */
FASTCOD_API const char* fastcod_last_error(const fastcod_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FASTCOD_H */
