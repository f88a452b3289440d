// Device helpers of the exact two-stage sampler (Alg. 2's sampling step as an
// exponential race), shared by the single-problem sampler (k_sample.cu) and
// the batched kernel (k_batched.cu): the FP32 log-domain key of a row and the
// constants of the cut.
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

}  // namespace rbrp
