/*
 * Seeded synthetic tractogram and volume generator (see synth.h).
 * Plain C99 + pthreads; the same source builds on x86_64 and aarch64.
 */
#include "synth.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- RNG */

typedef struct { uint64_t s; } rng_t;

static inline uint64_t sm64_next(rng_t* r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* uniform in [0, 1) with 53 random bits */
static inline double u01(rng_t* r) { return (double)(sm64_next(r) >> 11) * 0x1.0p-53; }
/* uniform in (0, 1] */
static inline double u01_open0(rng_t* r) { return ((double)(sm64_next(r) >> 11) + 1.0) * 0x1.0p-53; }

static inline double gauss(rng_t* r) {
  /* Box-Muller, one output per call */
  double u1 = u01_open0(r), u2 = u01(r);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

static rng_t stream_rng(uint64_t seed, uint32_t subject, int64_t idx) {
  rng_t r;
  /* key the stream by (seed, subject, index) and decorrelate with two
   * SplitMix64 rounds */
  r.s = seed * 0xD1342543DE82EF95ull ^ ((uint64_t)subject << 40) ^ (uint64_t)idx * 0x9E3779B97F4A7C15ull;
  sm64_next(&r);
  r.s ^= (uint64_t)idx;
  sm64_next(&r);
  return r;
}

void synth_splitmix64(uint64_t state, uint64_t* out, int64_t n) {
  rng_t r = {state};
  for (int64_t i = 0; i < n; ++i) out[i] = sm64_next(&r);
}

/* ------------------------------------------------------ thread helper */

typedef void (*range_fn)(void* ctx, int64_t b, int64_t e);
typedef struct { range_fn fn; void* ctx; int64_t b, e; } job_t;

static void* job_run(void* p) {
  job_t* j = (job_t*)p;
  j->fn(j->ctx, j->b, j->e);
  return NULL;
}

static void parallel_for(int64_t n, int32_t n_threads, range_fn fn, void* ctx) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n < (int64_t)n_threads * 64) n_threads = 1;
  if (n_threads == 1) { fn(ctx, 0, n); return; }
  pthread_t th[256];
  job_t jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx;
    jobs[t].b = n * t / n_threads; jobs[t].e = n * (t + 1) / n_threads;
    pthread_create(&th[t], NULL, job_run, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* ----------------------------------------------------------- volumes */

static inline double ell_r2(const double c[3], const double ax[3], double x, double y, double z) {
  double a = (x - c[0]) / ax[0], b = (y - c[1]) / ax[1], d = (z - c[2]) / ax[2];
  return a * a + b * b + d * d;
}

typedef struct {
  const synth_volume_params* vp;
  const double* dirs;  /* M x 3 */
  int32_t* roi;
  uint16_t* lab;
} vol_ctx;

static void vol_slab(void* p, int64_t kb, int64_t ke) {
  vol_ctx* c = (vol_ctx*)p;
  const synth_volume_params* vp = c->vp;
  const int64_t Dx = vp->dims[0], Dy = vp->dims[1];
  const int M = vp->n_labels;
  for (int64_t k = kb; k < ke; ++k)
    for (int64_t j = 0; j < Dy; ++j)
      for (int64_t i = 0; i < Dx; ++i) {
        const int64_t lin = i + Dx * (j + Dy * k);
        const double x = i + 0.5, y = j + 0.5, z = k + 0.5;
        int in_roi = 0;
        for (int e = 0; e < vp->n_roi; ++e)
          if (ell_r2(vp->roi_c[e], vp->roi_ax[e], x, y, z) < 1.0) in_roi = 1;
        c->roi[lin] = in_roi ? 1 : -1; /* rows are numbered afterwards */
        uint16_t l = 0;
        const double r2 = ell_r2(vp->brain_c, vp->brain_ax, x, y, z);
        if (r2 < 1.0 && r2 >= vp->shell_rho_in * vp->shell_rho_in) {
          double ux = x - vp->brain_c[0], uy = y - vp->brain_c[1], uz = z - vp->brain_c[2];
          const double n = sqrt(ux * ux + uy * uy + uz * uz);
          if (n > 0) { ux /= n; uy /= n; uz /= n; }
          int best = 0;
          double bv = -1e300;
          for (int m = 0; m < M; ++m) {
            const double v = ux * c->dirs[3 * m] + uy * c->dirs[3 * m + 1] + uz * c->dirs[3 * m + 2];
            if (v > bv) { bv = v; best = m; } /* strict '>' : ties go to the lowest k */
          }
          l = (uint16_t)(best + 1);
        }
        c->lab[lin] = l;
      }
}

int64_t synth_volumes(const synth_volume_params* vp, int32_t* roi, uint16_t* lab, int32_t n_threads) {
  const int M = vp->n_labels;
  if (M < 1 || M > 65535) return -1;
  double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)M);
  rng_t r = stream_rng(vp->label_seed, 0xFFFFFFFFu, -1);
  for (int m = 0; m < M; ++m) {
    double a, b, d, n;
    do {
      a = gauss(&r); b = gauss(&r); d = gauss(&r);
      n = sqrt(a * a + b * b + d * d);
    } while (n < 1e-12);
    dirs[3 * m] = a / n; dirs[3 * m + 1] = b / n; dirs[3 * m + 2] = d / n;
  }
  vol_ctx c = {vp, dirs, roi, lab};
  parallel_for(vp->dims[2], n_threads, vol_slab, &c);
  free(dirs);
  /* number ROI rows in lin order */
  const int64_t nvox = (int64_t)vp->dims[0] * vp->dims[1] * vp->dims[2];
  int64_t n = 0;
  for (int64_t i = 0; i < nvox; ++i)
    if (roi[i] >= 0) roi[i] = (int32_t)(n++);
  return n;
}

/* -------------------------------------------------------- streamlines */

typedef struct {
  const synth_volume_params* vp;
  const synth_streamline_params* sp;
  const int64_t* roi_lin;
  int64_t n_roi_lin;
  int64_t s_begin;
  int32_t* counts;        /* pass 1 */
  const int64_t* offsets; /* pass 2 */
  int32_t* xyz;           /* pass 2 */
} sl_ctx;

static inline int in_brain(const synth_volume_params* vp, const double p[3]) {
  return ell_r2(vp->brain_c, vp->brain_ax, p[0], p[1], p[2]) < 1.0;
}

static int32_t max_vertices(const synth_streamline_params* sp, rng_t* r) {
  if (sp->len_mode == 0) {
    const int64_t a = (int64_t)sp->len_a, b = (int64_t)sp->len_b;
    return (int32_t)(a + (int64_t)(u01(r) * (double)(b - a + 1)));
  }
  double mm = exp(log(sp->len_a) + sp->len_sigma * gauss(r));
  if (mm < sp->len_lo) mm = sp->len_lo;
  if (mm > sp->len_hi) mm = sp->len_hi;
  const double step_mm = sp->step_vox * sp->res_mm;
  return (int32_t)(1 + llround(mm / step_mm));
}

static void seed_point(const sl_ctx* c, rng_t* r, double p[3]) {
  const synth_volume_params* vp = c->vp;
  if (c->n_roi_lin > 0 && u01(r) < c->sp->f_roi) {
    int64_t idx = (int64_t)(u01(r) * (double)c->n_roi_lin);
    if (idx >= c->n_roi_lin) idx = c->n_roi_lin - 1;
    const int64_t lin = c->roi_lin[idx];
    const int64_t Dx = vp->dims[0], Dy = vp->dims[1];
    const int64_t i = lin % Dx, j = (lin / Dx) % Dy, k = lin / (Dx * Dy);
    p[0] = (double)i + u01(r);
    p[1] = (double)j + u01(r);
    p[2] = (double)k + u01(r);
    return;
  }
  for (;;) { /* uniform in the brain ellipsoid by rejection in its box */
    for (int a = 0; a < 3; ++a) p[a] = vp->brain_c[a] + vp->brain_ax[a] * (2.0 * u01(r) - 1.0);
    if (in_brain(vp, p)) return;
  }
}

/* von Mises-Fisher turn on S^2 about mu (Wood 1994, closed form for p=3). */
static void vmf_turn(rng_t* r, double kappa, double e2k, double mu[3]) {
  const double u = u01_open0(r);
  double w = 1.0 + log(u + (1.0 - u) * e2k) / kappa;
  if (w > 1.0) w = 1.0;
  if (w < -1.0) w = -1.0;
  const double phi = 2.0 * M_PI * u01(r);
  const double s = sqrt(1.0 - w * w);
  /* orthonormal basis (b1, b2) perpendicular to mu */
  double a[3] = {1.0, 0.0, 0.0};
  if (fabs(mu[0]) > 0.9) { a[0] = 0.0; a[1] = 1.0; }
  double b1[3] = {mu[1] * a[2] - mu[2] * a[1], mu[2] * a[0] - mu[0] * a[2], mu[0] * a[1] - mu[1] * a[0]};
  double n = sqrt(b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2]);
  b1[0] /= n; b1[1] /= n; b1[2] /= n;
  const double b2[3] = {mu[1] * b1[2] - mu[2] * b1[1], mu[2] * b1[0] - mu[0] * b1[2], mu[0] * b1[1] - mu[1] * b1[0]};
  const double cp = cos(phi) * s, sp = sin(phi) * s;
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = w * mu[k] + cp * b1[k] + sp * b2[k];
  n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; ++k) mu[k] = d[k] / n;
}

static inline int32_t quant(double v) { return (int32_t)llrint(v * 1024.0); }

/* Walk streamline idx; if out != NULL write its vertices.  Returns T. */
static int32_t walk(const sl_ctx* c, int64_t idx, int32_t* out) {
  const synth_streamline_params* sp = c->sp;
  rng_t r = stream_rng(sp->seed, sp->subject, idx);
  const int32_t tmax = max_vertices(sp, &r);
  double p[3], d[3];
  seed_point(c, &r, p);
  { /* uniform initial direction */
    double n;
    do {
      d[0] = gauss(&r); d[1] = gauss(&r); d[2] = gauss(&r);
      n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    } while (n < 1e-12);
    d[0] /= n; d[1] /= n; d[2] /= n;
  }
  const double e2k = exp(-2.0 * sp->kappa);
  int32_t t = 0;
  for (;;) {
    if (out) { out[3 * t] = quant(p[0]); out[3 * t + 1] = quant(p[1]); out[3 * t + 2] = quant(p[2]); }
    ++t;
    if (t >= tmax) break;
    if (t > 1) vmf_turn(&r, sp->kappa, e2k, d);
    double q[3] = {p[0] + sp->step_vox * d[0], p[1] + sp->step_vox * d[1], p[2] + sp->step_vox * d[2]};
    if (!in_brain(c->vp, q)) break; /* stop before the first vertex outside */
    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
  }
  return t;
}

static void count_range(void* p, int64_t b, int64_t e) {
  sl_ctx* c = (sl_ctx*)p;
  for (int64_t i = b; i < e; ++i) c->counts[i] = walk(c, c->s_begin + i, NULL);
}

static void fill_range(void* p, int64_t b, int64_t e) {
  sl_ctx* c = (sl_ctx*)p;
  for (int64_t i = b; i < e; ++i) {
    const int64_t o = c->offsets[i];
    const int32_t t = walk(c, c->s_begin + i, c->xyz + 3 * o);
    (void)t;
  }
}

int synth_count(const synth_volume_params* vp, const synth_streamline_params* sp,
                const int64_t* roi_lin, int64_t n_roi_lin,
                int64_t s_begin, int64_t s_end, int32_t* counts, int32_t n_threads) {
  if (s_end < s_begin) return -1;
  sl_ctx c = {vp, sp, roi_lin, n_roi_lin, s_begin, counts, NULL, NULL};
  parallel_for(s_end - s_begin, n_threads, count_range, &c);
  return 0;
}

int synth_fill(const synth_volume_params* vp, const synth_streamline_params* sp,
               const int64_t* roi_lin, int64_t n_roi_lin,
               int64_t s_begin, int64_t s_end, const int64_t* offsets,
               int32_t* xyz, int32_t n_threads) {
  if (s_end < s_begin) return -1;
  sl_ctx c = {vp, sp, roi_lin, n_roi_lin, s_begin, NULL, offsets, xyz};
  parallel_for(s_end - s_begin, n_threads, fill_range, &c);
  return 0;
}
