// Device helpers of the samplers of Alg. 2's sampling step (an exponential race),
// shared by the single-problem samplers (k_sample.cu, k_common.cu) and the batched
// kernel (k_batched.cu): the FP32 log-domain key of a row, the constants of the
// cut, the exact FP64 key, the (key, row) sort and the gather of the drawn rows.
#pragma once

#include <math.h>

#include "rbrp_internal.cuh"

namespace rbrp {

constexpr int kMargin = 32;          // extra candidates kept by the FP32 cut
constexpr int kBins = 2048;          // 11-bit digits
constexpr int kSampThreads = 256;
constexpr int kSampPerThread = 2;
constexpr float kCutGuard = 2e-4f;   // absolute slack in log space (FP32 key error bound)

// ln(d) from the FP64 bit pattern with FP32 arithmetic: exponent * ln2 + ln(mantissa).
__device__ __forceinline__ float log_d_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return (float)log(d);  // subnormal d (rare): FP64 logarithm
  const double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL));
  return (float)(e - 1023) * 0.69314718055994531f + logf((float)m);
}

// FP32 log-domain key of row i (smaller = drawn earlier); 0xFFFFFFFF for ineligible rows.
__device__ __forceinline__ unsigned int approx_key(double di, long long i, unsigned long long block_no,
                                                   unsigned long long seed, unsigned long long problem, int greedy) {
  if (!(di > 0.0)) return 0xFFFFFFFFu;
  float key;
  if (greedy) {
    key = -log_d_f32(di);
  } else {
    unsigned long long c[4] = {(unsigned long long)i, block_no, 0ULL, 0ULL};
    philox4x64_10(c, seed, problem);
    // E = -log(u) > 0 with u = ((w0 >> 11) + 1/2) 2^-53: logf(u) for u < 1/2, and
    // -log1pf(-(1 - u)) above, where 1 - u is exact in FP64 (keeps E accurate near u = 1)
    const double u = ((double)(c[0] >> 11) + 0.5) * 0x1.0p-53;
    const float e = (u < 0.5) ? -logf((float)u) : -log1pf(-(float)(1.0 - u));
    key = logf(e) - log_d_f32(di);
  }
  const unsigned int bits = __float_as_uint(key);
  return (bits >> 31) ? ~bits : (bits | 0x80000000u);
}

__device__ __forceinline__ float key_to_float(unsigned int k) {
  return __uint_as_float((k >> 31) ? (k & 0x7FFFFFFFu) : ~k);
}


// ---------------------------------------------------------------- exact FP64 selection
// (key, row) pairs ordered by exact FP64 key, then row: the order of S_t.
struct Pair {
  unsigned long long key;
  long long idx;
};

__device__ __forceinline__ bool pair_less(const Pair& a, const Pair& b) {
  return (a.key < b.key) || (a.key == b.key && a.idx < b.idx);
}

// Ascending bitonic sort of sh[0, kSortChunk) by one CTA of kSortChunk / 2 threads
// (one compare-exchange per thread and stage).  Begins and ends with a barrier.
__device__ __forceinline__ void sort_chunk(Pair* sh) {
  __syncthreads();
  for (int k = 2; k <= kSortChunk; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int t = threadIdx.x;
      const int i = (t / j) * 2 * j + (t % j);
      const int l = i + j;
      const bool up = ((i & k) == 0);
      const Pair a = sh[i], c = sh[l];
      if (up ? pair_less(c, a) : pair_less(a, c)) {
        sh[i] = c;
        sh[l] = a;
      }
      __syncthreads();
    }
  }
}

// Exact FP64 key of row i (the oracle's): -log(u_i) / d_i, or -d_i for the greedy
// sampler, as an orderable integer; kIneligible for d_i <= 0.
__device__ __forceinline__ unsigned long long exact_key(double di, long long i, unsigned long long block_no,
                                                        unsigned long long seed, unsigned long long problem,
                                                        int greedy) {
  if (!(di > 0.0)) return kIneligible;
  if (greedy) return orderable(-di);
  const double u = philox_uniform((unsigned long long)i, block_no, seed, problem);
  return orderable(-log(u) / di);
}

// Inverse of orderable().
__device__ __forceinline__ double from_orderable(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k));
}

// V(r, :) = src(rows[r], :) for r < bt, split into (row, column segment) units over
// `units_of` CTAs starting at unit `first`; rows outside [0, n) are skipped.
template <typename TS, typename TV>
__device__ __forceinline__ void gather_units(const TS* __restrict__ src, long long lds, TV* __restrict__ V,
                                             long long ldv, long long d, long long n, const long long* rows, int bt,
                                             int first, int stride) {
  const int seg = 2 * blockDim.x;
  const int nseg = (int)((d + seg - 1) / seg);
  for (int u = first; u < bt * nseg; u += stride) {
    const int r = u / nseg;
    const long long i = rows[r];
    if (i < 0 || i >= n) continue;
    const long long c0 = (long long)(u % nseg) * seg;
    const TS* s = src + i * lds;
    TV* v = V + (long long)r * ldv;
    for (long long j = c0 + threadIdx.x; j < c0 + seg && j < d; j += blockDim.x) v[j] = (TV)s[j];
  }
}

// first_block: the block that reads g.src0 (when given) in place of g.src.
__device__ __forceinline__ void gather_rows(const GatherSpec& g, long long n, const long long* rows, int bt, int first,
                                            int stride, bool first_block) {
  if (!g.V) return;
  const void* src = (first_block && g.src0) ? g.src0 : g.src;
  const long long lds = (first_block && g.src0) ? g.lds0 : g.lds;
  if (g.src64 && g.v64)
    gather_units((const double*)src, lds, (double*)g.V, g.ldv, g.d, n, rows, bt, first, stride);
  else if (g.src64)
    gather_units((const double*)src, lds, (float*)g.V, g.ldv, g.d, n, rows, bt, first, stride);
  else if (g.v64)
    gather_units((const float*)src, lds, (double*)g.V, g.ldv, g.d, n, rows, bt, first, stride);
  else
    gather_units((const float*)src, lds, (float*)g.V, g.ldv, g.d, n, rows, bt, first, stride);
}

}  // namespace rbrp
