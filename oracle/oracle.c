/*
 * ORACLE - TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain single-threaded C99.  Every quantity of the connectivity path is an
 * integer; rational comparisons are exact int64 cross-multiplications.  With
 * coordinates in [-2^24, 2^24) every numerator is at most 2^25 + 1024 and
 * every denominator at most 2^25, so the products stay below 2^51.  The
 * floating-point steps (parcellation fractions, world-mm ingest) state their
 * rounding and are compiled without contraction (-ffp-contract=off).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define UNIT 1024
#define COORD_LIMIT (1 << 24)

/* floor(p / 1024) for any sign: the voxel of p (Section 2 "loc2region";
 * half-open voxel boxes). */
static int64_t vox_of(int64_t p) {
  int64_t q = p / UNIT;
  if (p % UNIT != 0 && p < 0) q -= 1;
  return q;
}

/* ------------------------------------------------------------------ walk
 * Integer 3-D walk (Amanatides & Woo 1987) of the segment P0 -> P1.  The
 * parameter of the next plane crossing of axis a is num_a / den_a with
 * den_a = |d_a|:
 *   d_a > 0: num_a = 1024 (c_a + 1) - P0_a; the crossing is taken while
 *            t <= 1, and the voxel index grows AT t (the plane belongs to
 *            the upper voxel);
 *   d_a < 0: num_a = P0_a - 1024 c_a; taken while t < 1, and the index
 *            drops JUST AFTER t (the plane belongs to the voxel being left).
 * At the smallest pending t*, the increasing axes tied at t* step first
 * (that voxel holds the point P(t*)); decreasing axes tied at t* step on the
 * next round, which finds t* again.  Each step visits the new voxel. */
typedef void (*visit_fn)(void* ctx, const int64_t c[3]);

static int64_t walk_segment(const int32_t P0[3], const int32_t P1[3], visit_fn fn, void* ctx) {
  int64_t c[3], num[3], den[3];
  int sgn[3];
  for (int a = 0; a < 3; ++a) {
    const int64_t d = (int64_t)P1[a] - (int64_t)P0[a];
    c[a] = vox_of(P0[a]);
    if (d > 0) {
      sgn[a] = 1; den[a] = d; num[a] = UNIT * (c[a] + 1) - P0[a];
    } else if (d < 0) {
      sgn[a] = -1; den[a] = -d; num[a] = (int64_t)P0[a] - UNIT * c[a];
    } else {
      sgn[a] = 0; den[a] = 1; num[a] = 0;
    }
  }
  int64_t visits = 1;
  fn(ctx, c);
  for (;;) {
    int pending[3];
    int best = -1;
    for (int a = 0; a < 3; ++a) {
      pending[a] = (sgn[a] > 0 && num[a] <= den[a]) || (sgn[a] < 0 && num[a] < den[a]);
      if (!pending[a]) continue;
      if (best < 0 || num[a] * den[best] < num[best] * den[a]) best = a;
    }
    if (best < 0) break;
    int tied[3], any_pos = 0;
    for (int a = 0; a < 3; ++a) {
      tied[a] = pending[a] && num[a] * den[best] == num[best] * den[a];
      if (tied[a] && sgn[a] > 0) any_pos = 1;
    }
    for (int a = 0; a < 3; ++a) {
      if (!tied[a]) continue;
      if (any_pos && sgn[a] > 0) { c[a] += 1; num[a] += UNIT; }
      if (!any_pos && sgn[a] < 0) { c[a] -= 1; num[a] += UNIT; }
    }
    ++visits;
    fn(ctx, c);
  }
  return visits;
}

typedef struct { int32_t* out; int64_t cap, n; } list_ctx;

static void list_visit(void* p, const int64_t c[3]) {
  list_ctx* l = (list_ctx*)p;
  if (l->n < l->cap) {
    l->out[3 * l->n] = (int32_t)c[0];
    l->out[3 * l->n + 1] = (int32_t)c[1];
    l->out[3 * l->n + 2] = (int32_t)c[2];
  }
  l->n++;
}

int64_t oracle_segment_voxels(const int32_t p0[3], const int32_t p1[3], int32_t* out, int64_t cap) {
  list_ctx l = {out, cap, 0};
  walk_segment(p0, p1, list_visit, &l);
  return l.n;
}

/* ----------------------------------------------------------- brute force
 * Exact slab test.  For axis a and voxel index i the set of t where the
 * coordinate lies in [1024 i, 1024 (i+1)) is
 *   d > 0: [ (1024 i - P0)/d , (1024 (i+1) - P0)/d )
 *   d < 0: ( (P0 - 1024 (i+1))/|d| , (P0 - 1024 i)/|d| ]
 *   d = 0: all t if 1024 i <= P0 < 1024 (i+1), else none.
 * The box is hit iff the intersection of the three sets with [0, 1] is
 * non-empty.  Bounds are fractions n/q with q > 0 and an open/closed flag. */
typedef struct { int64_t n, q; int closed; } bound_t;

static int frac_cmp(bound_t x, bound_t y) {
  const int64_t l = x.n * y.q, r = y.n * x.q;
  return (l > r) - (l < r);
}

static int box_hit(const int32_t P0[3], const int32_t P1[3], const int64_t v[3]) {
  bound_t lo = {0, 1, 1}, hi = {1, 1, 1}; /* [0, 1] */
  for (int a = 0; a < 3; ++a) {
    const int64_t d = (int64_t)P1[a] - (int64_t)P0[a];
    const int64_t p = P0[a], b0 = UNIT * v[a], b1 = UNIT * (v[a] + 1);
    bound_t L, U;
    if (d == 0) {
      if (p >= b0 && p < b1) continue;
      return 0;
    } else if (d > 0) {
      L.n = b0 - p; L.q = d; L.closed = 1;
      U.n = b1 - p; U.q = d; U.closed = 0;
    } else {
      L.n = p - b1; L.q = -d; L.closed = 0;
      U.n = p - b0; U.q = -d; U.closed = 1;
    }
    /* tighten: the larger lower bound wins; on equal value, open wins */
    int c = frac_cmp(L, lo);
    if (c > 0 || (c == 0 && !L.closed)) lo = L;
    c = frac_cmp(U, hi);
    if (c < 0 || (c == 0 && !U.closed)) hi = U;
  }
  const int c = frac_cmp(lo, hi);
  return c < 0 || (c == 0 && lo.closed && hi.closed);
}

int64_t oracle_bruteforce_segment(const int32_t p0[3], const int32_t p1[3], const int32_t lo[3],
                                  const int32_t hi[3], int32_t* out, int64_t cap) {
  int64_t n = 0, v[3];
  for (v[2] = lo[2]; v[2] <= hi[2]; ++v[2])
    for (v[1] = lo[1]; v[1] <= hi[1]; ++v[1])
      for (v[0] = lo[0]; v[0] <= hi[0]; ++v[0])
        if (box_hit(p0, p1, v)) {
          if (n < cap) {
            out[3 * n] = (int32_t)v[0];
            out[3 * n + 1] = (int32_t)v[1];
            out[3 * n + 2] = (int32_t)v[2];
          }
          ++n;
        }
  return n;
}

/* ------------------------------------------------------- connectivity */

typedef struct {
  const int32_t* roi;
  const uint16_t* lab;
  int64_t Dx, Dy, Dz;
  int32_t N, M;
  uint32_t flags;
  /* sets of the current streamline, as stamp arrays + lists */
  int64_t stamp_id;
  int64_t* row_stamp;  /* [N] */
  int64_t* lab_stamp;  /* [M + 1] */
  int32_t* V; int32_t nV;
  int32_t* Tl; int32_t nT;
  int64_t visits;
} conn_ctx;

static int in_grid(const conn_ctx* k, const int64_t c[3]) {
  return c[0] >= 0 && c[0] < k->Dx && c[1] >= 0 && c[1] < k->Dy && c[2] >= 0 && c[2] < k->Dz;
}

static int64_t lin_of(const conn_ctx* k, const int64_t c[3]) { return c[0] + k->Dx * (c[1] + k->Dy * c[2]); }

static int32_t row_at(const conn_ctx* k, const int64_t c[3]) { return in_grid(k, c) ? k->roi[lin_of(k, c)] : -1; }

static int32_t lab_at(const conn_ctx* k, const int64_t c[3]) { return in_grid(k, c) ? (int32_t)k->lab[lin_of(k, c)] : 0; }

static void add_row(conn_ctx* k, int32_t r) {
  if (r >= 0 && k->row_stamp[r] != k->stamp_id) {
    k->row_stamp[r] = k->stamp_id;
    k->V[k->nV++] = r;
  }
}

static void add_lab(conn_ctx* k, int32_t t) {
  if (t >= 1 && k->lab_stamp[t] != k->stamp_id) {
    k->lab_stamp[t] = k->stamp_id;
    k->Tl[k->nT++] = t;
  }
}

static void conn_visit(void* p, const int64_t c[3]) {
  conn_ctx* k = (conn_ctx*)p;
  k->visits++;
  add_row(k, row_at(k, c));
  if (!(k->flags & ORACLE_TARGET_ENDPOINT)) add_lab(k, lab_at(k, c));
}

static void point_of(const int32_t* xyz, int64_t i, int64_t c[3]) {
  for (int a = 0; a < 3; ++a) c[a] = vox_of(xyz[3 * i + a]);
}

/* Collect V_s and T_s of the streamline with vertices xyz[0 .. T-1]. */
static int64_t streamline_sets(conn_ctx* k, const int32_t* xyz, int64_t T) {
  int64_t steps = 0;
  k->nV = 0; k->nT = 0;
  k->stamp_id++;
  if (T <= 0) return 0;
  int64_t c[3];
  if (T == 1 || (k->flags & ORACLE_VERTEX_SAMPLED)) {
    for (int64_t i = 0; i < T; ++i) {
      point_of(xyz, i, c);
      conn_visit(k, c);
    }
  } else {
    for (int64_t i = 0; i + 1 < T; ++i) walk_segment(xyz + 3 * i, xyz + 3 * (i + 1), conn_visit, k);
  }
  if (T == 1) steps = 1;
  for (int64_t i = 0; i + 1 < T; ++i) {
    int64_t s = 1;
    for (int a = 0; a < 3; ++a) {
      const int64_t d = vox_of(xyz[3 * (i + 1) + a]) - vox_of(xyz[3 * i + a]);
      s += d < 0 ? -d : d;
    }
    steps += s;
  }
  if (k->flags & ORACLE_TARGET_ENDPOINT) {
    point_of(xyz, T - 1, c);
    add_lab(k, lab_at(k, c));
  }
  return steps;
}

static int validate(const int32_t* roi, const uint16_t* lab, const int32_t dims[3], int32_t N,
                    int32_t M, const int32_t* xyz, const int64_t* offsets, int64_t ns) {
  if (dims[0] <= 0 || dims[1] <= 0 || dims[2] <= 0 || N < 0 || M < 0 || ns < 0) return -1;
  const int64_t nvox = (int64_t)dims[0] * dims[1] * dims[2];
  for (int64_t i = 0; i < nvox; ++i) {
    if (roi[i] < -1 || roi[i] >= N) return -1;
    if (lab[i] > M) return -1;
  }
  if (offsets[0] != 0) return -1;
  for (int64_t s = 0; s < ns; ++s)
    if (offsets[s + 1] < offsets[s]) return -1;
  for (int64_t i = 0; i < 3 * offsets[ns]; ++i)
    if (xyz[i] < -COORD_LIMIT || xyz[i] >= COORD_LIMIT) return -1;
  return 0;
}

static int ctx_init(conn_ctx* k, const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                    int32_t N, int32_t M, uint32_t flags) {
  memset(k, 0, sizeof(*k));
  k->roi = roi; k->lab = lab;
  k->Dx = dims[0]; k->Dy = dims[1]; k->Dz = dims[2];
  k->N = N; k->M = M; k->flags = flags;
  k->row_stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  k->lab_stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M + 1));
  k->V = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  k->Tl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M + 1));
  if (!k->row_stamp || !k->lab_stamp || !k->V || !k->Tl) return -1;
  for (int32_t i = 0; i < N; ++i) k->row_stamp[i] = -1;
  for (int32_t i = 0; i <= M; ++i) k->lab_stamp[i] = -1;
  k->stamp_id = 0;
  return 0;
}

static void ctx_free(conn_ctx* k) {
  free(k->row_stamp); free(k->lab_stamp); free(k->V); free(k->Tl);
}

static void add_endpoint(const conn_ctx* k, const int32_t* xyz, int64_t T, int64_t* Cend) {
  if (T < 1) return;
  int64_t c[3];
  point_of(xyz, 0, c);
  const int32_t r = row_at(k, c);
  point_of(xyz, T - 1, c);
  const int32_t t = lab_at(k, c);
  if (r >= 0 && t >= 1) Cend[(int64_t)r * k->M + (t - 1)] += 1;
}

int oracle_connectivity(const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                        int32_t N, int32_t M, const int32_t* xyz, const int64_t* offsets,
                        int64_t ns, uint32_t flags, int64_t* C, int64_t* Cend, oracle_stats* st) {
  if (validate(roi, lab, dims, N, M, xyz, offsets, ns) != 0) return -1;
  conn_ctx k;
  if (ctx_init(&k, roi, lab, dims, N, M, flags) != 0) { ctx_free(&k); return -1; }
  oracle_stats s = {0, 0, 0, 0};
  for (int64_t i = 0; i < ns; ++i) {
    const int64_t T = offsets[i + 1] - offsets[i];
    const int32_t* p = xyz + 3 * offsets[i];
    s.voxel_steps += streamline_sets(&k, p, T);
    /* C(v, r) += 1 for every pass-through v and every target r (Alg. 2) */
    for (int32_t a = 0; a < k.nV; ++a)
      for (int32_t b = 0; b < k.nT; ++b) C[(int64_t)k.V[a] * M + (k.Tl[b] - 1)] += 1;
    if (k.nV > 0 && k.nT > 0) s.n_contributing++;
    s.pairs += (int64_t)k.nV * k.nT;
    if (Cend) add_endpoint(&k, p, T, Cend);
  }
  s.visits = k.visits;
  if (st) *st = s;
  ctx_free(&k);
  return 0;
}

int oracle_bruteforce_connectivity(const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                                   int32_t N, int32_t M, const int32_t* xyz, const int64_t* offsets,
                                   int64_t ns, uint32_t flags, int64_t* C, int64_t* Cend) {
  if (validate(roi, lab, dims, N, M, xyz, offsets, ns) != 0) return -1;
  conn_ctx k;
  if (ctx_init(&k, roi, lab, dims, N, M, flags) != 0) { ctx_free(&k); return -1; }
  /* per-voxel hit flags of the current streamline over the whole grid */
  const int64_t nvox = k.Dx * k.Dy * k.Dz;
  unsigned char* hit = (unsigned char*)malloc((size_t)nvox);
  for (int64_t i = 0; i < ns; ++i) {
    const int64_t T = offsets[i + 1] - offsets[i];
    const int32_t* p = xyz + 3 * offsets[i];
    memset(hit, 0, (size_t)nvox);
    int64_t v[3];
    for (v[2] = 0; v[2] < k.Dz; ++v[2])
      for (v[1] = 0; v[1] < k.Dy; ++v[1])
        for (v[0] = 0; v[0] < k.Dx; ++v[0]) {
          int h = 0;
          if (T == 1 || (flags & ORACLE_VERTEX_SAMPLED)) {
            for (int64_t j = 0; j < T && !h; ++j) {
              int64_t c[3];
              point_of(p, j, c);
              h = c[0] == v[0] && c[1] == v[1] && c[2] == v[2];
            }
          } else {
            for (int64_t j = 0; j + 1 < T && !h; ++j) h = box_hit(p + 3 * j, p + 3 * (j + 1), v);
          }
          hit[lin_of(&k, v)] = (unsigned char)h;
        }
    /* sets as membership flags over rows and labels */
    k.stamp_id++;
    k.nV = 0; k.nT = 0;
    for (int64_t l = 0; l < nvox; ++l) {
      if (!hit[l]) continue;
      add_row(&k, roi[l]);
      if (!(flags & ORACLE_TARGET_ENDPOINT)) add_lab(&k, (int32_t)lab[l]);
    }
    if ((flags & ORACLE_TARGET_ENDPOINT) && T >= 1) {
      int64_t c[3];
      point_of(p, T - 1, c);
      add_lab(&k, lab_at(&k, c));
    }
    for (int32_t a = 0; a < k.nV; ++a)
      for (int32_t b = 0; b < k.nT; ++b) C[(int64_t)k.V[a] * M + (k.Tl[b] - 1)] += 1;
    if (Cend) add_endpoint(&k, p, T, Cend);
  }
  free(hit);
  ctx_free(&k);
  return 0;
}

static int cmp_i32(const void* a, const void* b) {
  const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

int oracle_streamline_sets(const int32_t* roi, const uint16_t* lab, const int32_t dims[3],
                           int32_t N, int32_t M, const int32_t* xyz, int64_t T, uint32_t flags,
                           int32_t* V, int32_t* nV, int32_t* Tl, int32_t* nT) {
  conn_ctx k;
  if (ctx_init(&k, roi, lab, dims, N, M, flags) != 0) { ctx_free(&k); return -1; }
  streamline_sets(&k, xyz, T);
  qsort(k.V, (size_t)k.nV, sizeof(int32_t), cmp_i32);
  qsort(k.Tl, (size_t)k.nT, sizeof(int32_t), cmp_i32);
  memcpy(V, k.V, sizeof(int32_t) * (size_t)k.nV);
  memcpy(Tl, k.Tl, sizeof(int32_t) * (size_t)k.nT);
  *nV = k.nV; *nT = k.nT;
  ctx_free(&k);
  return 0;
}

/* ------------------------------------------------------------ parcellation */

__extension__ typedef unsigned __int128 u128;

static int bit_length(uint64_t x) {
  int n = 0;
  while (x) {
    ++n;
    x >>= 1;
  }
  return n;
}

/* The binary32 nearest to a / b (0 <= a <= b, 0 < b < 2^63), ties to even,
 * by exact integer long division: with s chosen so that 2^23 <= a 2^s / b <
 * 2^24, the quotient q = floor(a 2^s / b) is the significand truncated and
 * the remainder decides the rounding (above half: up; exactly half: up when
 * q is odd).  A carry to 2^24 moves to the next binade.  The result
 * q 2^-s is a normal binary32 (a / b >= 2^-63), so the scaling is exact. */
static float nearest_f32_quotient(uint64_t a, uint64_t b) {
  if (a == 0) return 0.0f;
  int s = 24 + bit_length(b) - bit_length(a); /* a 2^s / b lies in (2^23, 2^25) */
  u128 num = (u128)a << s;
  u128 q = num / b;
  if (q >= ((u128)1 << 24)) { /* one binade too high */
    s -= 1;
    num = (u128)a << s;
    q = num / b;
  }
  const u128 r = num - q * b;
  if (2 * r > b || (2 * r == b && (q & 1))) q += 1;
  if (q == ((u128)1 << 24)) {
    q >>= 1;
    s -= 1;
  }
  return ldexpf((float)(uint32_t)q, -s);
}

int oracle_parcellate(const int64_t* C, int32_t N, int32_t M, int32_t* label, float* frac) {
  for (int32_t r = 0; r < N; ++r) {
    const int64_t* row = C + (int64_t)r * M;
    int64_t sum = 0, best = 0;
    int32_t arg = 0;
    for (int32_t t = 0; t < M; ++t) {
      if (row[t] < 0) return -1;
      if (row[t] >= ((int64_t)1 << 62) - sum) return -2; /* the row sum must stay below 2^62 */
      sum += row[t];
      if (row[t] > best) {
        best = row[t];
        arg = t + 1;
      }
    }
    label[r] = arg;
    if (frac) {
      for (int32_t t = 0; t < M; ++t)
        frac[(int64_t)r * M + t] = sum > 0 ? nearest_f32_quotient((uint64_t)row[t], (uint64_t)sum) : 0.0f;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ ingest */

int oracle_world_to_fixed(const float* xyz_mm, int64_t nv, const float affine[12], int32_t* xyz) {
  for (int64_t i = 0; i < nv; ++i) {
    const float x = xyz_mm[3 * i], y = xyz_mm[3 * i + 1], z = xyz_mm[3 * i + 2];
    for (int a = 0; a < 3; ++a) {
      const float* A = affine + 4 * a;
      volatile float t0 = A[0] * x; /* volatile: every product and sum rounded on its own */
      volatile float t1 = A[1] * y;
      volatile float s0 = t0 + t1;
      volatile float t2 = A[2] * z;
      volatile float s1 = s0 + t2;
      volatile float v = s1 + A[3];
      const float u = v * 1024.0f;
      if (!(u >= -16777216.0f && u < 16777216.0f)) return -1;
      const long r = lrintf(u);
      if (r < -16777216L || r >= 16777216L) return -1;
      xyz[3 * i + a] = (int32_t)r;
    }
  }
  return 0;
}

/* --------------------------------------------------------------- upsample */

static int64_t floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

int64_t oracle_upsample(const int32_t* xyz, const int64_t* offsets, int64_t ns, int32_t factor,
                        int32_t* out_xyz, int64_t* out_offsets) {
  if (factor < 1 || offsets[0] != 0) return -1;
  int64_t o = 0;
  out_offsets[0] = 0;
  for (int64_t s = 0; s < ns; ++s) {
    const int64_t a = offsets[s], b = offsets[s + 1];
    if (b < a) return -1;
    for (int64_t i = a; i + 1 < b; ++i) {
      for (int32_t j = 0; j < factor; ++j) {
        for (int c = 0; c < 3; ++c) {
          const int64_t p = xyz[3 * i + c], q = xyz[3 * (i + 1) + c];
          out_xyz[3 * o + c] = (int32_t)(p + floor_div((q - p) * j, factor));
        }
        ++o;
      }
    }
    if (b > a) {
      for (int c = 0; c < 3; ++c) out_xyz[3 * o + c] = xyz[3 * (b - 1) + c];
      ++o;
    }
    out_offsets[s + 1] = o;
  }
  return o;
}

int32_t oracle_upsample_factor(const int32_t* xyz, const int64_t* offsets, int64_t ns, int32_t spacing) {
  if (spacing < 1) return -1;
  int64_t best = 0; /* largest squared segment length */
  for (int64_t s = 0; s < ns; ++s) {
    for (int64_t i = offsets[s]; i + 1 < offsets[s + 1]; ++i) {
      int64_t l2 = 0;
      for (int c = 0; c < 3; ++c) {
        const int64_t d = (int64_t)xyz[3 * (i + 1) + c] - xyz[3 * i + c];
        l2 += d * d;
      }
      if (l2 > best) best = l2;
    }
  }
  /* r = the smallest integer with r * r >= best (binary search; best < 2^53),
     then the smallest k with k * spacing >= r */
  int64_t lo = 0, hi = (int64_t)1 << 27;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (mid * mid >= best) hi = mid; else lo = mid + 1;
  }
  int64_t k = (lo + spacing - 1) / spacing;
  if (k < 1) k = 1;
  return k > (1 << 20) ? -1 : (int32_t)k;
}

int oracle_rescale(const int32_t* xyz, int64_t nv, const int32_t num[3], const int32_t den[3],
                   const int64_t add[3], int32_t* out) {
  for (int c = 0; c < 3; ++c)
    if (num[c] < 1 || den[c] < 1) return -1;
  for (int64_t i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) {
      const int64_t v = floor_div((int64_t)xyz[3 * i + c] * num[c] + add[c], den[c]);
      if (v < -16777216LL || v >= 16777216LL) return -1;
      out[3 * i + c] = (int32_t)v;
    }
  return 0;
}
