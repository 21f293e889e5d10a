/*
 * Seeded synthetic tractogram and volume generator.
 *
 * This module is shared input infrastructure: both the CUDA library's tests
 * and the CPU oracle's tests (and the benchmark) draw their inputs from it.
 * It holds none of the connectivity method's arithmetic: no voxel walk, no
 * region lookup, no counting.  It only rasterises geometric volumes and draws
 * random streamlines.
 *
 * Stand-ins for the paper's inputs (Section 3): the HCP thalamus segmentation
 * becomes one or more ellipsoids, the Desikan-Killiany cortical parcellation
 * becomes an M-way angular Voronoi partition of an ellipsoidal shell, and
 * MRtrix3 probabilistic tractography becomes a persistent random walk with
 * von Mises-Fisher turns.
 *
 * Conventions:
 *   - volumes are x-fastest: lin(i,j,k) = i + Dx*(j + Dy*k);
 *   - voxel (i,j,k) covers [i,i+1) x [j,j+1) x [k,k+1) in voxel units, its
 *     centre is (i+0.5, j+0.5, k+0.5);
 *   - vertices are int32 fixed point at 1/1024 voxel, quantised with llrint
 *     (round half to even) from voxel-unit coordinates.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), keyed per streamline by
 * (seed, subject, streamline index), so any chunking of the streamline range
 * reproduces the same streamlines.
 */
#ifndef SYNTH_H
#define SYNTH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYNTH_MAX_ROI_ELLIPSOIDS 4

typedef struct {
  int32_t dims[3];          /* Dx, Dy, Dz */
  double brain_c[3];        /* brain ellipsoid centre, voxel units */
  double brain_ax[3];       /* brain ellipsoid semi-axes, voxel units */
  double shell_rho_in;      /* labelled shell: normalised radius in [rho_in, 1) */
  int32_t n_labels;         /* M, >= 1 */
  uint64_t label_seed;      /* seed of the M label directions */
  int32_t n_roi;            /* number of ROI ellipsoids, 0..4 */
  double roi_c[SYNTH_MAX_ROI_ELLIPSOIDS][3];  /* centres, voxel units */
  double roi_ax[SYNTH_MAX_ROI_ELLIPSOIDS][3]; /* semi-axes, voxel units */
} synth_volume_params;

typedef struct {
  uint64_t seed;
  uint32_t subject;
  double step_vox;          /* step length in voxels (0.5) */
  double kappa;             /* von Mises-Fisher concentration per step (20) */
  int32_t len_mode;         /* 0: vertex count uniform in [len_a, len_b];
                               1: length lognormal in mm, median len_a,
                                  sigma len_sigma, clipped to [len_lo, len_hi] */
  double len_a, len_b, len_sigma, len_lo, len_hi;
  double res_mm;            /* voxel size in mm (for len_mode 1) */
  double f_roi;             /* fraction of seeds drawn inside ROI voxels */
} synth_streamline_params;

/* Rasterise the volumes.  roi[lin] = row index (assigned in lin order) for
 * voxels whose centre lies in any ROI ellipsoid, else -1; lab[lin] = 1 +
 * argmax_k <u, d_k> for voxels whose centre lies in the shell, else 0.
 * Returns N (number of ROI voxels). */
int64_t synth_volumes(const synth_volume_params* vp, int32_t* roi, uint16_t* lab,
                      int32_t n_threads);

/* Pass 1: vertex count of every streamline in [s_begin, s_end).
 * roi_lin: list of the n_roi_lin linear indices of ROI voxels (seed pool).
 * counts[s - s_begin] receives T_s. */
int synth_count(const synth_volume_params* vp, const synth_streamline_params* sp,
                const int64_t* roi_lin, int64_t n_roi_lin,
                int64_t s_begin, int64_t s_end, int32_t* counts, int32_t n_threads);

/* Pass 2: write the vertices of streamlines [s_begin, s_end).  offsets has
 * (s_end - s_begin + 1) entries relative to xyz (offsets[0] is where the
 * first streamline's first vertex goes).  xyz is int32 [n][3]. */
int synth_fill(const synth_volume_params* vp, const synth_streamline_params* sp,
               const int64_t* roi_lin, int64_t n_roi_lin,
               int64_t s_begin, int64_t s_end, const int64_t* offsets,
               int32_t* xyz, int32_t n_threads);

/* Raw SplitMix64 stream (for tests of the generator itself). */
void synth_splitmix64(uint64_t state, uint64_t* out, int64_t n);

#ifdef __cplusplus
}
#endif
#endif
