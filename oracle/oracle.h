/*
 * ORACLE - TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of what FastCod's pass-through
 * connectivity computes (Bian et al., "FastCod: Fast Brain Connectivity in
 * Diffusion Imaging", arXiv 2302.09247).  Only the tests, the package smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the library never calls
 * it.
 *
 * What is computed (Section 2, Algorithm 2, passthrough / loc2region):
 *   - units: 1 = 1/1024 voxel; voxel (i,j,k) is the half-open box
 *     [1024i, 1024i+1024) x [1024j, ..) x [1024k, ..); the voxel of an integer
 *     point is floor(p / 1024) per axis;
 *   - lin(i,j,k) = i + Dx*(j + Dy*k); row(v) = roi[lin] in-grid, else -1;
 *     lab(v) = labels[lin] in-grid, else 0;
 *   - P_s = union over segments of {p^k + tau (p^{k+1} - p^k), tau in [0,1]}
 *     (T = 1: {p^1}; T = 0: empty); Vox(s) = {floor(p/1024) : p in P_s};
 *   - V_s = {row(v) >= 0 : v in Vox(s)}, T_s = {lab(v) >= 1 : v in Vox(s)};
 *   - C[r][t-1] = sum_s [r in V_s][t in T_s];
 *   - C_end[r][t-1] = sum_{s : T >= 1} [row(floor p^1) = r][lab(floor p^T) = t]
 *     (Algorithm 1, the seed read as the first vertex).
 *
 * Readings where the paper is silent: half-open voxel boxes (at a shared
 * crossing the increasing axes step at the crossing, the decreasing ones just
 * after it), the first vertex as the seed, points off the grid ignored, dedup
 * by row index and by label value.
 *
 * Options (flags):
 *   ORACLE_TARGET_ENDPOINT - T_s = {lab(floor p^T)} instead of the labels the
 *     streamline passes through (Algorithm 2 taken literally: one target, the
 *     region of the last vertex);
 *   ORACLE_VERTEX_SAMPLED  - Vox(s) = {floor(p^k / 1024)} over the vertices
 *     only (the point-sampled variant behind the paper's upsampling rule,
 *     Section 3, "Super-resolving connectivity features").
 */
#ifndef FASTCOD_ORACLE_H
#define FASTCOD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_TARGET_ENDPOINT 1u
#define ORACLE_VERTEX_SAMPLED 2u

typedef struct {
  int64_t voxel_steps;   /* sum over segments of 1 + sum_a |dfloor_a|; a T=1 streamline counts 1 */
  int64_t visits;        /* voxels visited by the walk (ties merged) */
  int64_t n_contributing;/* streamlines with V_s and T_s both non-empty */
  int64_t pairs;         /* sum_s |V_s| |T_s| */
} oracle_stats;

/* Voxels visited by the integer walk of segment p0 -> p1, in visit order.
 * Writes up to cap voxels (xyz triples) to out; returns the visit count. */
int64_t oracle_segment_voxels(const int32_t p0[3], const int32_t p1[3], int32_t* out, int64_t cap);

/* Brute force: every voxel box in [lo, hi] (inclusive, per axis) tested
 * against the segment with an exact rational slab test.  Writes the
 * intersected voxels (x fastest order of the box) to out; returns count. */
int64_t oracle_bruteforce_segment(const int32_t p0[3], const int32_t p1[3], const int32_t lo[3],
                                  const int32_t hi[3], int32_t* out, int64_t cap);

/* C and C_end (int64, row-major N x M, accumulated: the caller zeroes them).
 * Returns 0, or -1 on invalid input. */
int oracle_connectivity(const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                        int32_t N, int32_t M, const int32_t* xyz, const int64_t* offsets,
                        int64_t ns, uint32_t flags, int64_t* C, int64_t* Cend, oracle_stats* st);

/* Same result from the plain definition on a tiny grid: every in-grid voxel
 * tested against every segment with the slab test (no walk). */
int oracle_bruteforce_connectivity(const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                                   int32_t N, int32_t M, const int32_t* xyz, const int64_t* offsets,
                                   int64_t ns, uint32_t flags, int64_t* C, int64_t* Cend);

/* V_s and T_s of one streamline (sorted ascending).  Returns 0. */
int oracle_streamline_sets(const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                           int32_t N, int32_t M, const int32_t* xyz, int64_t T, uint32_t flags,
                           int32_t* V, int32_t* nV, int32_t* Tl, int32_t* nT);

/* Parcellation outputs of an N x M connectivity matrix (Section 3,
 * "Pie-glyphs": the single-colour display shows the region with the highest
 * connectivity, the pie chart each region's relative connectivity strength):
 *   label[r] = 1 + argmax_t C[r][t], ties to the lowest label; 0 when the row
 *              is all zero;
 *   frac[r][t] = C[r][t] / sum_t C[r][t] rounded to the nearest binary32
 *              (ties to even), decided by exact integer long division; 0 for
 *              an all-zero row.  frac may be NULL.
 * Returns 0, -1 when an entry is negative, or -2 when a row sum reaches
 * 2^62. */
int oracle_parcellate(const int64_t* C, int32_t N, int32_t M, int32_t* label, float* frac);

/* World-mm streamline vertices (binary32, the form tractography writes) to
 * this library's fixed point: v_a = ((A[a][0] x + A[a][1] y) + A[a][2] z)
 * + A[a][3] with every product and sum rounded to binary32 (no fused
 * multiply-add), then the coordinate is v_a * 1024 rounded to the nearest
 * integer (ties to even).  A is the row-major 3 x 4 world -> voxel affine
 * (voxel i spans [i, i+1)).  Returns 0, or -1 when a result is not finite or
 * falls outside [-2^24, 2^24). */
int oracle_world_to_fixed(const float* xyz_mm, int64_t nv, const float affine[12], int32_t* xyz);

/* Streamline upsampling (Section 3, "Super-resolving connectivity features":
 * evenly spaced points inserted between neighbouring points): every segment
 * p -> q of a streamline becomes `factor` segments through the points
 * p + floor((q - p) * j / factor), j = 0 .. factor-1, followed by the last
 * vertex.  A streamline of T >= 1 vertices gets (T - 1) * factor + 1, an
 * empty one none.  out_offsets has ns + 1 entries.  Returns the vertices
 * written, or -1 on invalid input. */
int64_t oracle_upsample(const int32_t* xyz, const int64_t* offsets, int64_t ns, int32_t factor,
                        int32_t* out_xyz, int64_t* out_offsets);

/* The smallest factor k >= 1 whose upsampled spacing is at most `spacing`
 * units on every segment: |q - p|^2 <= (k * spacing)^2 (exact integers; the
 * paper's rule of thumb takes spacing <= half the target voxel).  Returns k,
 * or -1 on invalid input or when k would exceed 2^20. */
int32_t oracle_upsample_factor(const int32_t* xyz, const int64_t* offsets, int64_t ns, int32_t spacing);

/* Integer rescale of fixed-point vertices between grids:
 * out_a = floor((p_a * num_a + add_a) / den_a), exact in 64-bit integers
 * (num_a, den_a > 0).  Returns 0, or -1 when a result falls outside
 * [-2^24, 2^24). */
int oracle_rescale(const int32_t* xyz, int64_t nv, const int32_t num[3], const int32_t den[3],
                   const int64_t add[3], int32_t* out);

#ifdef __cplusplus
}
#endif
#endif
