// Kernels beside the connectivity path: the parcellation outputs of a
// connectivity matrix (Section 3, "Pie-glyphs"), world-mm ingest through an
// affine, streamline upsampling and the integer rescale between grids
// (Section 3, "Super-resolving connectivity features").  All are single
// streaming passes (HBM-bound); every result is exact or rounds as stated.
#include "fc_device.cuh"
#include "fc_tma.cuh"

namespace fc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {  // b > 0
  const int64_t q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

int grid_for(int64_t items, int per_thread = 1) {
  const int64_t b = (items + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  return (int)(b < 1 ? 1 : (b > (1 << 20) ? (1 << 20) : b));
}

// ------------------------------------------------------------ parcellation
// sign(a 2^s - K b) over 128-bit integers (a, b < 2^63, K < 2^27, 0 <= s,
// a 2^s < 2^128).
__device__ __forceinline__ int cmp_shifted(uint64_t a, int s, uint64_t K, uint64_t b) {
  const uint64_t lh = s >= 64 ? a << (s - 64) : (s == 0 ? 0ull : a >> (64 - s));
  const uint64_t ll = s >= 64 ? 0ull : a << s;
  const uint64_t rh = __umul64hi(K, b), rl = K * b;
  if (lh != rh) return lh < rh ? -1 : 1;
  if (ll != rl) return ll < rl ? -1 : 1;
  return 0;
}

// sign(a / b - (x + y) / 2) for neighbouring positive binary32 values x < y:
// their midpoint is exact in binary64 (26 significant bits); written as
// K 2^-s with K odd, the comparison is a 2^s against K b.
__device__ __forceinline__ int cmp_midpoint(uint64_t a, uint64_t b, float x, float y) {
  const double mid = ((double)x + (double)y) * 0.5;
  const uint64_t bits = (uint64_t)__double_as_longlong(mid);
  uint64_t K = (bits & 0xfffffffffffffull) | (1ull << 52);  // mid = K 2^(e - 1075)
  int s = 1075 - (int)((bits >> 52) & 0x7ff);
  const int tz = __ffsll((long long)K) - 1;
  K >>= tz;
  s -= tz;
  return cmp_shifted(a, s, K, b);
}

// The binary32 nearest to a / b (0 <= a <= b, 0 < b < 2^47), ties to even.
// The binary64 quotient rounded to binary32 is within one unit of it (a
// second rounding can cross a midpoint); the exact comparisons with the two
// midpoints around that candidate settle it.
__device__ __forceinline__ float quotient_rn(uint64_t a, uint64_t b) {
  if (a == 0) return 0.0f;
  const float f = __double2float_rn(__ddiv_rn((double)a, (double)b));
  const uint32_t u = __float_as_uint(f);
  const float up = __uint_as_float(u + 1), dn = __uint_as_float(u - 1);
  const int cu = cmp_midpoint(a, b, f, up);
  if (cu > 0 || (cu == 0 && (u & 1))) return up;
  const int cd = cmp_midpoint(a, b, dn, f);
  if (cd < 0 || (cd == 0 && (u & 1))) return dn;
  return f;
}

// One entry's fraction: one binary32 division when the row sum is below 2^24
// (both integers exact in binary32, and IEEE division rounds to nearest),
// else the exact rule above.
__device__ __forceinline__ float row_fraction(int32_t v, long long sum) {
  if (sum <= 0) return 0.0f;
  if (sum < (1ll << 24)) return __fdiv_rn((float)v, (float)sum);
  return quotient_rn((uint64_t)v, (uint64_t)sum);
}

// One warp per row: the maximum with the lowest label on ties, the row sum
// (64-bit), then the fractions: the binary32 nearest to count / sum.  With
// st given, a negative entry is an error (kErrCount, the row).
__global__ void __launch_bounds__(kThreads) parcellate_kernel(const int32_t* __restrict__ C, int32_t N, int32_t M,
                                                              int32_t* __restrict__ label, float* __restrict__ frac,
                                                              DevState* st) {
  const int32_t lane = (int32_t)lane_id();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += nwarps) {
    const int32_t* row = C + r * M;
    long long sum = 0;
    int32_t best = 0, arg = 0x7fffffff, lo = 0;
    for (int32_t t = lane; t < M; t += 32) {
      const int32_t v = __ldg(row + t);
      sum += v;
      lo = min(lo, v);
      if (v > best) {  // ascending t per lane: the first maximum stays
        best = v;
        arg = t;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int32_t ob = __shfl_xor_sync(kFull, best, o), oa = __shfl_xor_sync(kFull, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
      sum += __shfl_xor_sync(kFull, sum, o);
    }
    if (st && __any_sync(kFull, lo < 0) && lane == 0) set_error(st, kErrCount, (int32_t)r);
    if (lane == 0) label[r] = best > 0 ? arg + 1 : 0;
    if (frac)
      for (int32_t t = lane; t < M; t += 32) frac[r * M + t] = row_fraction(__ldg(row + t), sum);
  }
}

// The same for rows of at most 32 * kPer entries, each lane's entries held in
// registers: one load per entry, all issued at once, and the fractions
// computed from the registers (the generic kernel reads the row twice).
template <int kPer>
__global__ void __launch_bounds__(kThreads) parcellate_rows_kernel(const int32_t* __restrict__ C, int32_t N,
                                                                   int32_t M, int32_t* __restrict__ label,
                                                                   float* __restrict__ frac, DevState* st) {
  const int32_t lane = (int32_t)lane_id();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += nwarps) {
    const int32_t* row = C + r * M;
    int32_t v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) v[k] = lane + 32 * k < M ? __ldg(row + lane + 32 * k) : 0;
    long long sum = 0;
    int32_t best = 0, arg = 0x7fffffff, lo = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      sum += v[k];
      lo = min(lo, v[k]);
      if (v[k] > best) {  // ascending t per lane: the first maximum stays
        best = v[k];
        arg = lane + 32 * k;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int32_t ob = __shfl_xor_sync(kFull, best, o), oa = __shfl_xor_sync(kFull, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
      sum += __shfl_xor_sync(kFull, sum, o);
    }
    if (st && __any_sync(kFull, lo < 0) && lane == 0) set_error(st, kErrCount, (int32_t)r);
    if (lane == 0) label[r] = best > 0 ? arg + 1 : 0;
    if (frac) {
      float* out = frac + r * M;
#pragma unroll
      for (int k = 0; k < kPer; ++k)
        if (lane + 32 * k < M) out[lane + 32 * k] = row_fraction(v[k], sum);
    }
  }
}

// The same for rows whose width M is a multiple of 4 with 16-byte aligned C
// and fractions: each lane holds kV int4 (entries 128 k + 4 lane + j), one
// 16-byte load each, and writes its fractions as float4.  The row sum is
// warp-uniform, so the exact-quotient branch (sum at or above 2^24) is taken
// once per row instead of once per entry; that branch re-reads the row.
template <int kV>
__global__ void __launch_bounds__(kThreads) parcellate_rows_vec_kernel(const int32_t* __restrict__ C, int32_t N,
                                                                       int32_t M, int32_t* __restrict__ label,
                                                                       float* __restrict__ frac, DevState* st) {
  const int32_t lane = (int32_t)lane_id();
  const int32_t M4 = M >> 2;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < N; r += nwarps) {
    const int4* row = reinterpret_cast<const int4*>(C + r * M);
    int4 v[kV];
#pragma unroll
    for (int k = 0; k < kV; ++k) v[k] = lane + 32 * k < M4 ? __ldcs(row + lane + 32 * k) : make_int4(0, 0, 0, 0);
    long long sum = 0;
    int32_t best = 0, arg = 0x7fffffff, lo = 0;
#pragma unroll
    for (int k = 0; k < kV; ++k) {
      const int32_t e[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sum += e[j];
        lo = min(lo, e[j]);
        if (e[j] > best) {  // ascending t per lane: the first maximum stays
          best = e[j];
          arg = 128 * k + 4 * lane + j;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int32_t ob = __shfl_xor_sync(kFull, best, o), oa = __shfl_xor_sync(kFull, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
      sum += __shfl_xor_sync(kFull, sum, o);
    }
    if (st && __any_sync(kFull, lo < 0) && lane == 0) set_error(st, kErrCount, (int32_t)r);
    if (lane == 0) label[r] = best > 0 ? arg + 1 : 0;
    if (!frac) continue;
    float4* out = reinterpret_cast<float4*>(frac + r * M);
    if (sum < (1ll << 24)) {  // both integers exact in binary32: one IEEE division each
      const float fs = (float)sum;
#pragma unroll
      for (int k = 0; k < kV; ++k)
        if (lane + 32 * k < M4) {
          float4 f;
          f.x = sum > 0 ? __fdiv_rn((float)v[k].x, fs) : 0.0f;
          f.y = sum > 0 ? __fdiv_rn((float)v[k].y, fs) : 0.0f;
          f.z = sum > 0 ? __fdiv_rn((float)v[k].z, fs) : 0.0f;
          f.w = sum > 0 ? __fdiv_rn((float)v[k].w, fs) : 0.0f;
          __stcs(out + lane + 32 * k, f);
        }
    } else {  // rare: read the row again rather than hold the exact rule's registers across it
      const int32_t* row32 = C + r * M;
      for (int32_t t = lane; t < M; t += 32) frac[r * M + t] = row_fraction(__ldg(row32 + t), sum);
    }
  }
}

// ------------------------------------------------------------------ ingest
// v_a = ((A[a][0] x + A[a][1] y) + A[a][2] z) + A[a][3], every operation a
// round-to-nearest binary32 intrinsic (no contraction), then v_a * 1024
// rounded to the nearest integer (ties to even).
struct Affine {
  float a[12];
};

__global__ void __launch_bounds__(kThreads) world_to_fixed_kernel(const float* __restrict__ in, int64_t nv,
                                                                  Affine A, int32_t* __restrict__ out,
                                                                  DevState* st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const float x = __ldcs(in + 3 * i), y = __ldcs(in + 3 * i + 1), z = __ldcs(in + 3 * i + 2);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(A.a[4 * a], x), __fmul_rn(A.a[4 * a + 1], y)),
                                          __fmul_rn(A.a[4 * a + 2], z)),
                                A.a[4 * a + 3]);
      const float u = __fmul_rn(v, 1024.0f);
      const bool in_range = u >= -16777216.0f && u < 16777216.0f;  // false for NaN
      const int32_t r = in_range ? __float2int_rn(u) : 0;
      ok &= in_range && r >= -16777216 && r < 16777216;
      out[3 * i + a] = r;
    }
    if (!ok) set_error(st, kErrCoord, (int32_t)min(i, (int64_t)0x7fffffff));
  }
}

// ---------------------------------------------------------------- upsample

// Largest squared segment length (warp per streamline, lanes over segments).
__global__ void __launch_bounds__(kThreads) seg_max_kernel(const int32_t* __restrict__ xyz,
                                                           const int64_t* __restrict__ off, int64_t ns,
                                                           unsigned long long* best) {
  const int32_t lane = (int32_t)lane_id();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long m = 0;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < ns; s += nwarps) {
    const int64_t a = off[s], b = off[s + 1];
    for (int64_t i = a + lane; i + 1 < b; i += 32) {
      long long l2 = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const long long d = (long long)__ldg(xyz + 3 * (i + 1) + c) - __ldg(xyz + 3 * i + c);
        l2 += d * d;
      }
      m = max(m, (unsigned long long)l2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if (lane == 0 && m) atomicMax(best, m);
}

// Offsets of the upsampled streamlines: out[s] = factor * off[s] - (factor - 1)
// * (non-empty streamlines before s).  Three passes: per-block counts of
// non-empty streamlines, their exclusive scan in one block, then each block's
// own scan.
constexpr int kScanItems = 8;  // streamlines per thread

__global__ void __launch_bounds__(kThreads) nonempty_counts_kernel(const int64_t* __restrict__ off, int64_t ns,
                                                                   long long* __restrict__ block_sum) {
  const int64_t base = (int64_t)blockIdx.x * kThreads * kScanItems;
  long long c = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t s = base + (int64_t)k * kThreads + threadIdx.x;
    if (s < ns) c += off[s + 1] > off[s] ? 1 : 0;
  }
  __shared__ long long red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if (lane_id() == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    block_sum[blockIdx.x] = t;
  }
}

// Exclusive scan of n block sums in place (one block of kThreads threads).
__global__ void __launch_bounds__(kThreads) scan_blocks_kernel(long long* __restrict__ v, int32_t n) {
  __shared__ long long part[kThreads];
  const int32_t per = (n + kThreads - 1) / kThreads;
  const int32_t lo = min(n, (int32_t)threadIdx.x * per), hi = min(n, lo + per);
  long long t = 0;
  for (int32_t i = lo; i < hi; ++i) t += v[i];
  part[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int k = 0; k < kThreads; ++k) {
      const long long x = part[k];
      part[k] = run;
      run += x;
    }
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (int32_t i = lo; i < hi; ++i) {
    const long long x = v[i];
    v[i] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(kThreads) upsample_offsets_kernel(const int64_t* __restrict__ off, int64_t ns,
                                                                    int32_t factor,
                                                                    const long long* __restrict__ block_base,
                                                                    int64_t* __restrict__ out) {
  // each thread takes kScanItems consecutive streamlines; a block scan of
  // the per-thread counts gives each thread its first index
  const int64_t base = (int64_t)blockIdx.x * kThreads * kScanItems + (int64_t)threadIdx.x * kScanItems;
  long long c = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t s = base + k;
    if (s < ns) c += off[s + 1] > off[s] ? 1 : 0;
  }
  __shared__ long long warp_tot[kThreads / 32];
  const int32_t lane = (int32_t)lane_id();
  long long inc = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long y = __shfl_up_sync(kFull, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) warp_tot[threadIdx.x >> 5] = inc;
  __syncthreads();
  long long before = block_base[blockIdx.x];
  for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += warp_tot[w];
  long long e = before + inc - c;  // non-empty streamlines before `base`
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t s = base + k;
    if (s > ns) break;
    out[s] = (int64_t)factor * off[s] - (int64_t)(factor - 1) * e;
    if (s < ns && off[s + 1] > off[s]) ++e;
  }
}

// Upsampled vertices: warp per streamline, lanes over its segments.  With
// d = q - p = q0 * factor + r0 (0 <= r0 < factor), floor(d * j / factor) =
// q0 * j + floor(r0 * j / factor): one division per segment and axis (a shift
// for a power-of-two factor, 32-bit when d fits), then the points follow with
// one carry test each.  The running sums are kept modulo 2^32: every point
// lies between p and q, so its int32 value is exact.  A round computes the
// points of up to 32 segments into a per-warp shared buffer; the warp then
// writes the round's contiguous output with coalesced stores.  The next
// round's vertices and the next streamline's offsets load while a round is
// computed and written, so that a streamline costs about one memory round
// trip instead of one per round.
constexpr int kUpCap = 256;  // points staged per warp (3 KB)

__device__ __forceinline__ void seg_split(int64_t d, int32_t factor, int32_t flog2, uint32_t& q0, uint32_t& r0) {
  if (flog2 >= 0) {  // arithmetic shift: floor division by 2^flog2
    q0 = (uint32_t)(d >> flog2);
    r0 = (uint32_t)d & (uint32_t)(factor - 1);
  } else if (d == (int64_t)(int32_t)d) {
    const int32_t dd = (int32_t)d;
    int32_t q = dd / factor, r = dd - q * factor;
    if (r < 0) {
      q -= 1;
      r += factor;
    }
    q0 = (uint32_t)q;
    r0 = (uint32_t)r;
  } else {
    const int64_t q = floor_div(d, factor);
    q0 = (uint32_t)q;
    r0 = (uint32_t)(d - q * factor);
  }
}

// Vertices i and i + 1 (the segment's ends).
__device__ __forceinline__ void load_segment(const int32_t* __restrict__ xyz, int64_t i, int32_t (&pa)[3],
                                             int32_t (&pb)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    pa[c] = __ldg(xyz + 3 * i + c);
    pb[c] = __ldg(xyz + 3 * (i + 1) + c);
  }
}

struct SegPoints {
  uint32_t p[3], q0[3], r0[3], acc_q[3], acc_r[3];

  __device__ __forceinline__ void init(const int32_t (&pa)[3], const int32_t (&pb)[3], int32_t factor,
                                       int32_t flog2) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      p[c] = (uint32_t)pa[c];
      seg_split((int64_t)pb[c] - pa[c], factor, flog2, q0[c], r0[c]);
      acc_q[c] = 0;
      acc_r[c] = 0;
    }
  }
  // writes point j (in order j = 0, 1, ...) and advances
  __device__ __forceinline__ void emit(int32_t* w, int32_t factor) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w[c] = (int32_t)(p[c] + acc_q[c]);
      acc_q[c] += q0[c];
      acc_r[c] += r0[c];
      if (acc_r[c] >= (uint32_t)factor) {
        acc_r[c] -= (uint32_t)factor;
        acc_q[c] += 1u;
      }
    }
  }
};

__global__ void __launch_bounds__(kThreads) upsample_kernel(const int32_t* __restrict__ xyz,
                                                            const int64_t* __restrict__ off, int64_t ns,
                                                            int32_t factor, int32_t flog2,
                                                            const int64_t* __restrict__ out_off,
                                                            int32_t* __restrict__ out) {
  __shared__ int32_t stage[kThreads / 32][3 * kUpCap];
  int32_t* sb = stage[threadIdx.x >> 5];
  const int32_t lane = (int32_t)lane_id();
  const int32_t per = factor <= kUpCap ? min(32, kUpCap / factor) : 0;  // segments per round
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t s0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t a = 0, b = 0, o = 0;
  if (s0 < ns) {
    a = off[s0];
    b = off[s0 + 1];
    o = out_off[s0];
  }
  for (int64_t s = s0; s < ns; s += nwarps) {
    int64_t an = 0, bn = 0, on = 0;  // the next streamline's offsets, in flight
    if (s + nwarps < ns) {
      an = off[s + nwarps];
      bn = off[s + nwarps + 1];
      on = out_off[s + nwarps];
    }
    if (b > a) {
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) out[3 * (o + (b - 1 - a) * factor) + c] = __ldg(xyz + 3 * (b - 1) + c);
      }
      if (per == 0) {  // factors above the staging capacity: each lane writes its own segments
        for (int64_t i = a + lane; i + 1 < b; i += 32) {
          int32_t pa[3], pb[3];
          load_segment(xyz, i, pa, pb);
          SegPoints g;
          g.init(pa, pb, factor, flog2);
          int32_t* dst = out + 3 * (o + (i - a) * factor);
          for (int32_t j = 0; j < factor; ++j) g.emit(dst + 3 * j, factor);
        }
      } else {
        int32_t cp[3] = {0, 0, 0}, cq[3] = {0, 0, 0};  // this round's segment of the lane
        if (a + lane + 1 < b && lane < per) load_segment(xyz, a + lane, cp, cq);
        for (int64_t i0 = a; i0 + 1 < b; i0 += per) {
          const int32_t nseg = (int32_t)min((int64_t)per, b - 1 - i0);
          int32_t np[3] = {0, 0, 0}, nq[3] = {0, 0, 0};  // the next round's, in flight
          if (i0 + per + lane + 1 < b && lane < per) load_segment(xyz, i0 + per + lane, np, nq);
          if (lane < nseg) {
            SegPoints g;
            g.init(cp, cq, factor, flog2);
            int32_t* w = sb + 3 * lane * factor;
            for (int32_t j = 0; j < factor; ++j) g.emit(w + 3 * j, factor);
          }
          __syncwarp();
          const int32_t nw = 3 * nseg * factor;
          int32_t* dst = out + 3 * (o + (i0 - a) * factor);
          for (int32_t k = lane; k < nw; k += 32) __stcs(dst + k, sb[k]);
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cp[c] = np[c];
            cq[c] = nq[c];
          }
        }
      }
    }
    a = an;
    b = bn;
    o = on;
  }
}

// Upsampled vertices for a power-of-two factor 2^L: warp per streamline.
// The warp stages up to kStageV of the streamline's vertices in shared
// memory (coalesced loads, all in flight at once), then each lane computes
// output words: word k of the chunk's output is axis c = k mod 3 of point
// P = k / 3, on the chunk's segment i = P >> L at j = P & (2^L - 1):
// x_i[c] + floor((x_{i+1}[c] - x_i[c]) j / 2^L), an arithmetic shift of a
// 64-bit product.  Chunks overlap by one vertex (the end of their last
// segment); the streamline's last chunk adds its last point, P = n << L for
// n + 1 staged vertices, which is j = 0 at the last vertex.  Stores are one
// coalesced word per lane.  While a streamline is written, the next one's
// vertices are requested into L2 with one bulk prefetch, so that its staging
// loads hit L2.
constexpr int kStageV = 256;  // vertices staged per warp (3 KB)

__global__ void __launch_bounds__(kThreads) upsample_pow2_kernel(const int32_t* __restrict__ xyz,
                                                                 const int64_t* __restrict__ off, int64_t ns,
                                                                 int32_t flog2, const int64_t* __restrict__ out_off,
                                                                 int32_t* __restrict__ out) {
  __shared__ int32_t stage[kThreads / 32][3 * kStageV];
  int32_t* sv = stage[threadIdx.x >> 5];
  const int32_t lane = (int32_t)lane_id();
  const uint32_t jmask = (1u << flog2) - 1u;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t s0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t a = 0, b = 0, o = 0;
  if (s0 < ns) {
    a = off[s0];
    b = off[s0 + 1];
    o = out_off[s0];
  }
  for (int64_t s = s0; s < ns; s += nwarps) {
    int64_t an = 0, bn = 0, on = 0;  // the next streamline's offsets, in flight
    if (s + nwarps < ns) {
      an = off[s + nwarps];
      bn = off[s + nwarps + 1];
      on = out_off[s + nwarps];
    }
    if (lane == 0 && bn > an) {  // the next streamline's vertices, 16-byte aligned inside
      const uintptr_t lo = (reinterpret_cast<uintptr_t>(xyz + 3 * an) + 15) & ~(uintptr_t)15;
      const uintptr_t hi = reinterpret_cast<uintptr_t>(xyz + 3 * bn) & ~(uintptr_t)15;
      if (hi > lo) bulk_prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)min(hi - lo, (uintptr_t)0x7ffffff0u));
    }
    const int64_t T = b - a;
    for (int64_t c0 = 0; c0 < T; c0 += kStageV - 1) {
      const int32_t nvc = (int32_t)min((int64_t)kStageV, T - c0);  // staged vertices
      const bool last = c0 + nvc == T;
      const int32_t* src = xyz + 3 * (a + c0);
      __syncwarp();
      const int32_t nwd = 3 * nvc;
#pragma unroll 4
      for (int32_t w = lane; w < nwd; w += 32) sv[w] = __ldg(src + w);
      __syncwarp();
      const uint32_t nout = 3u * (((uint32_t)(nvc - 1) << flog2) + (last ? 1u : 0u));  // words
      int32_t* dst = out + 3 * (o + (c0 << flog2));
      for (uint32_t k = (uint32_t)lane; k < nout; k += 32) {
        const uint32_t P = k / 3u, c = k - 3u * P, i = P >> flog2, jj = P & jmask;
        const int32_t x0 = sv[3 * i + c];
        const int32_t x1 = jj ? sv[3 * i + 3 + c] : x0;
        const long long dv = (long long)x1 - x0;
        __stcs(dst + k, (int32_t)((uint32_t)x0 + (uint32_t)((dv * jj) >> flog2)));
      }
      if (last) break;
    }
    a = an;
    b = bn;
    o = on;
  }
}

// Offsets [ns + 1] start at 0, do not decrease and end at nv.
__global__ void __launch_bounds__(kThreads) check_offsets_kernel(const int64_t* __restrict__ off, int64_t ns,
                                                                 int64_t nv, DevState* st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= ns; s += stride) {
    const int64_t a = off[s];
    bool ok = a >= 0 && a <= nv;
    if (s == 0) ok &= a == 0;
    if (s == ns) ok &= a == nv;
    if (s < ns) ok &= off[s + 1] >= a;
    if (!ok) set_error(st, kErrOffsets, (int32_t)min(s, (int64_t)0x7fffffff));
  }
}

// ------------------------------------------------------ checkpoint check
__global__ void __launch_bounds__(kThreads) checkpoint_check_kernel(const int32_t* __restrict__ C,
                                                                    const int32_t* __restrict__ Cend, int64_t nm,
                                                                    int32_t max_count,
                                                                    unsigned long long* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long sc = 0, se = 0, bad = ~0ull;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nm; k += stride) {
    const int32_t x = __ldcs(C + k), y = __ldcs(Cend + k);
    if (x < 0 || x > max_count) bad = min(bad, (unsigned long long)k);
    if (y < 0 || y > max_count) bad = min(bad, (unsigned long long)(nm + k));
    sc += (unsigned long long)max(x, 0);
    se += (unsigned long long)max(y, 0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sc += __shfl_xor_sync(kFull, sc, o);
    se += __shfl_xor_sync(kFull, se, o);
    bad = min(bad, __shfl_xor_sync(kFull, bad, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (sc) atomicAdd(out, sc);
    if (se) atomicAdd(out + 1, se);
    if (bad != ~0ull) atomicMin(out + 2, bad);
  }
}

// ----------------------------------------------------------------- rescale
struct Rescale {
  int64_t num[3], den[3], add[3];
};

__global__ void __launch_bounds__(kThreads) rescale_kernel(const int32_t* __restrict__ xyz, int64_t n_coords,
                                                           Rescale R, int32_t* __restrict__ out, DevState* st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_coords; k += stride) {
    const int c = (int)(k % 3);
    const int64_t v = floor_div((int64_t)__ldcs(xyz + k) * R.num[c] + R.add[c], R.den[c]);
    const bool ok = v >= -16777216 && v < 16777216;
    out[k] = ok ? (int32_t)v : 0;
    if (!ok) set_error(st, kErrCoord, (int32_t)min(k / 3, (int64_t)0x7fffffff));
  }
}

}  // namespace

cudaError_t launch_parcellate(const int32_t* C, int32_t N, int32_t M, int32_t* label, float* frac, DevState* st,
                              cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int g = grid_for((int64_t)N * 32);
  const bool vec = M % 4 == 0 && ((uintptr_t)C % 16 == 0) && (!frac || (uintptr_t)frac % 16 == 0);
  if (vec && M <= 512) {
    const auto k = M <= 128 ? parcellate_rows_vec_kernel<1>
                   : M <= 256 ? parcellate_rows_vec_kernel<2>
                   : M <= 384 ? parcellate_rows_vec_kernel<3> : parcellate_rows_vec_kernel<4>;
    k<<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  } else if (M <= 32) parcellate_rows_kernel<1><<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  else if (M <= 64) parcellate_rows_kernel<2><<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  else if (M <= 128) parcellate_rows_kernel<4><<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  else if (M <= 256) parcellate_rows_kernel<8><<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  else if (M <= 512) parcellate_rows_kernel<16><<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  else parcellate_kernel<<<g, kThreads, 0, s>>>(C, N, M, label, frac, st);
  return cudaGetLastError();
}

cudaError_t launch_world_to_fixed(const float* xyz_mm, int64_t nv, const float affine[12], int32_t* out,
                                  DevState* st, cudaStream_t s) {
  if (nv <= 0) return cudaSuccess;
  Affine A;
  for (int k = 0; k < 12; ++k) A.a[k] = affine[k];
  world_to_fixed_kernel<<<grid_for(nv, 4), kThreads, 0, s>>>(xyz_mm, nv, A, out, st);
  return cudaGetLastError();
}

cudaError_t launch_seg_max(const int32_t* xyz, const int64_t* off, int64_t ns, unsigned long long* best,
                           cudaStream_t s) {
  if (ns <= 0) return cudaSuccess;
  seg_max_kernel<<<grid_for(ns * 32, 8), kThreads, 0, s>>>(xyz, off, ns, best);
  return cudaGetLastError();
}

int64_t upsample_scan_blocks(int64_t ns) { return (ns + 1 + (int64_t)kThreads * kScanItems - 1) / ((int64_t)kThreads * kScanItems); }

cudaError_t launch_checkpoint_check(const int32_t* C, const int32_t* Cend, int64_t nm, int32_t max_count,
                                    unsigned long long* out, cudaStream_t s) {
  if (nm <= 0) return cudaSuccess;
  checkpoint_check_kernel<<<grid_for(nm, 8), kThreads, 0, s>>>(C, Cend, nm, max_count, out);
  return cudaGetLastError();
}

cudaError_t launch_check_offsets(const int64_t* off, int64_t ns, int64_t nv, DevState* st, cudaStream_t s) {
  check_offsets_kernel<<<grid_for(ns + 1, 4), kThreads, 0, s>>>(off, ns, nv, st);
  return cudaGetLastError();
}

cudaError_t launch_upsample_offsets(const int64_t* off, int64_t ns, int32_t factor, long long* block_tmp,
                                    int64_t* out_off, cudaStream_t s) {
  const int64_t nb = upsample_scan_blocks(ns);
  nonempty_counts_kernel<<<(unsigned)nb, kThreads, 0, s>>>(off, ns, block_tmp);
  scan_blocks_kernel<<<1, kThreads, 0, s>>>(block_tmp, (int32_t)nb);
  upsample_offsets_kernel<<<(unsigned)nb, kThreads, 0, s>>>(off, ns, factor, block_tmp, out_off);
  return cudaGetLastError();
}

cudaError_t launch_upsample_vertices(const int32_t* xyz, const int64_t* off, int64_t ns, int32_t factor,
                                     const int64_t* out_off, int32_t* out, cudaStream_t s) {
  if (ns <= 0) return cudaSuccess;
  const int32_t flog2 = (factor & (factor - 1)) == 0 ? __builtin_ctz((unsigned)factor) : -1;
  if (flog2 >= 0 && flog2 <= 20) upsample_pow2_kernel<<<grid_for(ns * 32, 8), kThreads, 0, s>>>(xyz, off, ns, flog2, out_off, out);
  else upsample_kernel<<<grid_for(ns * 32, 8), kThreads, 0, s>>>(xyz, off, ns, factor, flog2, out_off, out);
  return cudaGetLastError();
}

cudaError_t launch_rescale(const int32_t* xyz, int64_t nv, const int32_t num[3], const int32_t den[3],
                           const int64_t add[3], int32_t* out, DevState* st, cudaStream_t s) {
  if (nv <= 0) return cudaSuccess;
  Rescale R;
  for (int c = 0; c < 3; ++c) {
    R.num[c] = num[c];
    R.den[c] = den[c];
    R.add[c] = add[c];
  }
  rescale_kernel<<<grid_for(nv * 3, 4), kThreads, 0, s>>>(xyz, nv * 3, R, out, st);
  return cudaGetLastError();
}

}  // namespace fc
