// Alg. 2's sampling step on the GPU: S_t ~ d / ||d||_1 without replacement (reading of
// the sampling step as an exponential race: keys kappa_i = -log(u_i) / d_i over
// eligible rows, the b_t smallest in ascending (kappa, i) order; the greedy
// variant of the blockwise greedy remark uses -d_i).
//
// Two stages, exact:
//  1. a log-domain FP32 key log(-log u_i) - log d_i per row (Philox and FP32
//     logarithms only; FP64 arithmetic is slow on GB300) and an 11 + 11-bit
//     radix histogram over those keys choose a cut that keeps at least
//     b + kMargin candidates;
//  2. the compaction pass computes the FP64 keys of the candidates exactly as
//     the oracle does; one CTA ranks them and checks that the cut lies more
//     than the FP32 error bound above the b_t-th exact key, so no row outside
//     the cut can belong to S_t.  If the check fails (or the candidate list overflows) it raises
//     State::sample_fallback and the exact FP64 tree sampler in k_common.cu
//     runs instead.
// The histogram buffers are cleared by the final kernel for the next block.
// Where the device supports cooperative launches the four passes run as one
// launch (k_sample_coop) with grid barriers between them.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <atomic>

#include "rbrp_internal.cuh"
#include "sample_common.cuh"

namespace rbrp {

// Pass 1: keys and the histogram of their top 11 bits (eligible rows only).
__global__ void __launch_bounds__(kSampThreads) k_samp_keys(const double* __restrict__ dvec, long long n,
                                                            unsigned int* __restrict__ K32,
                                                            unsigned int* __restrict__ hist1, int greedy,
                                                            unsigned long long seed, unsigned long long problem,
                                                            const State* st) {
  if (st->done) return;
  __shared__ unsigned int h[kBins];
  for (int j = threadIdx.x; j < kBins; j += kSampThreads) h[j] = 0;
  __syncthreads();
  const unsigned long long block_no = (unsigned long long)st->t + 1ULL;
  const long long base = (long long)blockIdx.x * kSampThreads * kSampPerThread;
#pragma unroll
  for (int q = 0; q < kSampPerThread; ++q) {
    const long long i = base + q * kSampThreads + threadIdx.x;
    if (i >= n) break;
    const unsigned int k = approx_key(dvec[i], i, block_no, seed, problem, greedy);
    K32[i] = k;
    if (k != 0xFFFFFFFFu) atomicAdd(&h[k >> 21], 1u);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kBins; j += kSampThreads)
    if (h[j]) atomicAdd(&hist1[j], h[j]);
}

// Block-wide search over a 2048-bin histogram: the first bin where the running
// count reaches `want`; returns the count below that bin in *below (or bin
// kBins and the total when the histogram holds fewer than `want`).  The first
// kSampThreads threads each sum eight bins and take an exclusive scan of those
// sums; the one thread whose range contains the want-th count walks its bins.
// Callable from any block size >= kSampThreads (the other threads only take
// part in the barriers).  The bins are read through L2 (__ldcg): in the
// cooperative sampler they were filled by other CTAs' atomics earlier in the
// same launch, and every CTA must see the same counts to take the same branch
// at the next grid barrier (a non-coherent or L1-cached read could be stale).
__device__ int find_bin(const unsigned int* hist, unsigned int want, unsigned int* below, unsigned int* total) {
  __shared__ unsigned int wsum[kSampThreads / 32];
  __shared__ int s_bin;
  __shared__ unsigned int s_below, s_total;
  constexpr int per = kBins / kSampThreads;  // 8 bins per thread
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned int c[per], sum = 0, incl = 0;
  if (t < kSampThreads) {
#pragma unroll
    for (int q = 0; q < per; ++q) {
      c[q] = __ldcg(hist + t * per + q);
      sum += c[q];
    }
    incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    if (t == 0) {
      s_bin = kBins;
      s_below = 0;
    }
  }
  __syncthreads();
  if (t < kSampThreads) {
    unsigned int before = 0, all = 0;
#pragma unroll
    for (int q = 0; q < kSampThreads / 32; ++q) {
      if (q < w) before += wsum[q];
      all += wsum[q];
    }
    incl += before;
    const unsigned int excl = incl - sum;
    if (excl < want && incl >= want) {
      unsigned int r2 = excl;
#pragma unroll
      for (int q = 0; q < per; ++q) {
        if (r2 + c[q] >= want) {
          s_bin = t * per + q;
          s_below = r2;
          break;
        }
        r2 += c[q];
      }
    }
    if (t == 0) s_total = all;
  }
  __syncthreads();
  const int bin = s_bin;
  *total = s_total;
  *below = (bin == kBins) ? s_total : s_below;
  __syncthreads();  // the shared results may be overwritten by the next call
  return bin;
}

// Pass 2: histogram of the next 11 bits inside the bin where the b + kMargin-th key falls.
__global__ void __launch_bounds__(kSampThreads) k_samp_hist2(const unsigned int* __restrict__ K32, long long n,
                                                             const unsigned int* __restrict__ hist1,
                                                             unsigned int* __restrict__ hist2, int want,
                                                             const State* st) {
  if (st->done) return;
  unsigned int below, total;
  const int b1 = find_bin(hist1, (unsigned int)want, &below, &total);
  if (b1 >= kBins) return;  // fewer eligible rows than wanted: every eligible row is a candidate
  __shared__ unsigned int h[kBins];
  for (int j = threadIdx.x; j < kBins; j += kSampThreads) h[j] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSampThreads * kSampPerThread;
#pragma unroll
  for (int q = 0; q < kSampPerThread; ++q) {
    const long long i = base + q * kSampThreads + threadIdx.x;
    if (i >= n) break;
    const unsigned int k = K32[i];
    if ((int)(k >> 21) == b1 && k != 0xFFFFFFFFu) atomicAdd(&h[(k >> 10) & 0x7FF], 1u);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kBins; j += kSampThreads)
    if (h[j]) atomicAdd(&hist2[j], h[j]);
}

// The 22-bit cut: rows whose key's top 22 bits are <= cut22 are candidates
// (0x3FFFFF when every eligible row is).
__device__ unsigned int cut22(const unsigned int* hist1, const unsigned int* hist2, int want) {
  unsigned int below1, total1, below2, total2;
  const int b1 = find_bin(hist1, (unsigned int)want, &below1, &total1);
  if (b1 >= kBins) return 0x3FFFFFu;
  const int b2 = find_bin(hist2, (unsigned int)(want - (int)below1), &below2, &total2);
  return ((unsigned int)b1 << 11) | (unsigned int)(b2 >= kBins ? kBins - 1 : b2);
}

// Pass 3: compact the candidate rows with their exact FP64 keys (computed
// here, spread over the grid, exactly as the oracle does).
__global__ void __launch_bounds__(kSampThreads) k_samp_compact(const unsigned int* __restrict__ K32,
                                                               const double* __restrict__ dvec, long long n,
                                                               const unsigned int* __restrict__ hist1,
                                                               const unsigned int* __restrict__ hist2, int want,
                                                               int* __restrict__ cand,
                                                               unsigned long long* __restrict__ cand_key,
                                                               double* __restrict__ cand_log,
                                                               unsigned int* __restrict__ ncand, int cap, int greedy,
                                                               unsigned long long seed, unsigned long long problem,
                                                               const State* st) {
  if (st->done) return;
  const unsigned int c22 = cut22(hist1, hist2, want);
  const unsigned long long block_no = (unsigned long long)st->t + 1ULL;
  const long long base = (long long)blockIdx.x * kSampThreads * kSampPerThread;
#pragma unroll
  for (int q = 0; q < kSampPerThread; ++q) {
    const long long i = base + q * kSampThreads + threadIdx.x;
    if (i >= n) break;
    const unsigned int k = K32[i];
    if (k != 0xFFFFFFFFu && (k >> 10) <= c22) {
      const unsigned int pos = atomicAdd(ncand, 1u);
      if ((int)pos < cap) {
        const double di = dvec[i];
        double key, lg;
        if (greedy) {
          key = -di;
          lg = -log(di);
        } else {
          const double u = philox_uniform((unsigned long long)i, block_no, seed, problem);
          key = -log(u) / di;
          lg = log(key);
        }
        cand[pos] = (int)i;
        cand_key[pos] = orderable(key);
        cand_log[pos] = lg;
      }
    }
  }
}

// Pass 4 (one CTA): exact FP64 keys of the candidates, ranking, the margin
// check, S_t and b_t; clears the histograms for the next block.
__global__ void __launch_bounds__(1024) k_samp_final(long long n, unsigned int* __restrict__ hist1,
                                                     unsigned int* __restrict__ hist2, int want,
                                                     const int* __restrict__ cand,
                                                     const unsigned long long* __restrict__ cand_key,
                                                     const double* __restrict__ cand_log,
                                                     unsigned int* __restrict__ ncand, int cap, int b,
                                                     long long* __restrict__ S_t, State* st) {
  if (st->done) return;
  __shared__ unsigned long long ek[kSampCap];
  __shared__ long long eidx[kSampCap];
  __shared__ double elog[kSampCap];
  __shared__ long long sorted_idx[kMaxBlock];
  __shared__ double sorted_log[kMaxBlock];
  unsigned int below1, total1;
  find_bin(hist1, (unsigned int)want, &below1, &total1);  // total1 = number of eligible rows
  const unsigned int c22 = cut22(hist1, hist2, want);
  const int nc = (int)__ldcg(ncand);  // counted by every CTA's atomics
  const bool overflow = nc > cap;
  const int m = overflow ? 0 : nc;
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    ek[e] = cand_key[e];
    eidx[e] = cand[e];
    elog[e] = cand_log[e];
  }
  __syncthreads();
  long long bt = (long long)total1;
  if (bt > b) bt = b;
  const long long room = st->k_cap - st->k;
  if (bt > room) bt = room;
  if (bt < 0) bt = 0;
  // rank of each candidate among the candidates by (exact key, row); the b_t smallest are kept
  for (int e = threadIdx.x; e < m; e += blockDim.x) {
    int rank = 0;
    const unsigned long long ke = ek[e];
    const long long ie = eidx[e];
    for (int f = 0; f < m; ++f) rank += (ek[f] < ke || (ek[f] == ke && eidx[f] < ie)) ? 1 : 0;
    if (rank < bt) {
      sorted_idx[rank] = ie;
      sorted_log[rank] = elog[e];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool exact = !overflow && m >= bt;
    if (exact && bt > 0 && (long long)m < (long long)total1 && c22 != 0x3FFFFFu) {
      // every row outside the cut has an FP32 key >= the smallest key above the cut
      const float outside = key_to_float(((c22 + 1u) << 10));
      exact = sorted_log[bt - 1] < (double)outside - (double)kCutGuard - 1e-6 * fabs((double)outside);
    }
    if (!exact) {
      st->sample_fallback = 1;
    } else {
      st->sample_fallback = 0;
      st->b_t = bt;
      if (bt == 0) st->done = 1;
    }
  }
  __syncthreads();
  if (!st->sample_fallback)
    for (int e = threadIdx.x; e < bt; e += blockDim.x) S_t[e] = sorted_idx[e];
  // clear the pass buffers for the next block
  for (int j = threadIdx.x; j < kBins; j += blockDim.x) {
    hist1[j] = 0;
    hist2[j] = 0;
  }
  if (threadIdx.x == 0) *ncand = 0;
}

__global__ void k_samp_clear(unsigned int* __restrict__ hist1, unsigned int* __restrict__ hist2,
                             unsigned int* __restrict__ ncand) {
  for (int j = threadIdx.x; j < kBins; j += blockDim.x) {
    hist1[j] = 0;
    hist2[j] = 0;
  }
  if (threadIdx.x < 16) ncand[threadIdx.x] = 0;  // the count, and the grid barrier words
}

// ---------------------------------------------------------------- one cooperative launch
// The same four passes in one launch of one CTA per SM (cooperative, so all
// CTAs are resident), separated by grid barriers instead of kernel
// boundaries: keys + first histogram | second histogram | compaction with
// exact keys | ranking, margin check and S_t by CTA 0.  Results are those of
// the four kernels above (same keys, cut, candidates and ranking).
constexpr int kCoopThreads = 512;
// Grid barrier over gridDim.x CTAs: arrival counter bar[0] (reset by the last
// arriver) and generation bar[1].  The wait is bounded (`limit` polls, by
// default ~1-2 s): on timeout the CTA records RBRP_ETIMEOUT in the State and
// carries on (every CTA still passes every barrier, so no CTA is left
// waiting; the results of that block are then void, every later kernel of the
// call sees the State's done flag, and the next call clears the barrier
// words before its first launch of this kernel).
__device__ __forceinline__ void grid_barrier(unsigned int* bar, State* st, unsigned limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen0 = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned int spins = 0;
      while (*vgen == gen0) {
        if (++spins > limit) {
          st->status = RBRP_ETIMEOUT;
          st->done = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kCoopThreads) k_sample_coop(const double* __restrict__ dvec, long long n,
                                                              unsigned int* __restrict__ K32,
                                                              unsigned int* __restrict__ hist1,
                                                              unsigned int* __restrict__ hist2, int want,
                                                              int* __restrict__ cand,
                                                              unsigned long long* __restrict__ cand_key,
                                                              double* __restrict__ cand_log,
                                                              unsigned int* __restrict__ ncand, int cap, int b,
                                                              int greedy, unsigned long long seed,
                                                              unsigned long long problem, long long* __restrict__ S_t,
                                                              State* st) {
  pdl_wait();
  if (st->done) return;  // read before any CTA writes the State: the same for every CTA
  __shared__ unsigned int h[kBins];
  unsigned int* bar = ncand + 2;
  const unsigned glim = st->spin_grid;
  const unsigned long long block_no = (unsigned long long)st->t + 1ULL;
  const long long gstride = (long long)gridDim.x * kCoopThreads;
  const long long g0 = (long long)blockIdx.x * kCoopThreads + threadIdx.x;
  // pass 1: keys and the histogram of their top 11 bits
  for (int j = threadIdx.x; j < kBins; j += kCoopThreads) h[j] = 0;
  __syncthreads();
  for (long long i = g0; i < n; i += gstride) {
    const unsigned int k = approx_key(dvec[i], i, block_no, seed, problem, greedy);
    K32[i] = k;
    if (k != 0xFFFFFFFFu) atomicAdd(&h[k >> 21], 1u);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kBins; j += kCoopThreads)
    if (h[j]) atomicAdd(&hist1[j], h[j]);
  grid_barrier(bar, st, glim);
  // pass 2: histogram of the next 11 bits inside the cut bin -- skipped (with
  // its barrier) when the whole cut bin adds few candidates (the final ranking
  // is quadratic in their number), which every CTA decides alike from the
  // same first histogram
  unsigned int below1, total1;
  const int b1 = find_bin(hist1, (unsigned int)want, &below1, &total1);
  const bool one_level = b1 < kBins && below1 + __ldcg(hist1 + b1) <= (unsigned int)(2 * want);
  if (b1 < kBins && !one_level) {
    for (int j = threadIdx.x; j < kBins; j += kCoopThreads) h[j] = 0;
    __syncthreads();
    for (long long i = g0; i < n; i += gstride) {
      const unsigned int k = K32[i];
      if ((int)(k >> 21) == b1 && k != 0xFFFFFFFFu) atomicAdd(&h[(k >> 10) & 0x7FF], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kBins; j += kCoopThreads)
      if (h[j]) atomicAdd(&hist2[j], h[j]);
  }
  if (!one_level) grid_barrier(bar, st, glim);
  // pass 3: candidates with their exact FP64 keys
  unsigned int c22 = 0x3FFFFFu;
  if (one_level) {
    c22 = ((unsigned int)b1 << 11) | 0x7FFu;  // every row of the cut bin
  } else if (b1 < kBins) {
    unsigned int below2, total2;
    const int b2 = find_bin(hist2, (unsigned int)(want - (int)below1), &below2, &total2);
    c22 = ((unsigned int)b1 << 11) | (unsigned int)(b2 >= kBins ? kBins - 1 : b2);
  }
  for (long long i = g0; i < n; i += gstride) {
    const unsigned int k = K32[i];
    if (k != 0xFFFFFFFFu && (k >> 10) <= c22) {
      const unsigned int pos = atomicAdd(ncand, 1u);
      if ((int)pos < cap) {
        const double di = dvec[i];
        double key, lg;
        if (greedy) {
          key = -di;
          lg = -log(di);
        } else {
          const double u = philox_uniform((unsigned long long)i, block_no, seed, problem);
          key = -log(u) / di;
          lg = log(key);
        }
        cand[pos] = (int)i;
        cand_key[pos] = orderable(key);
        cand_log[pos] = lg;
      }
    }
  }
  grid_barrier(bar, st, glim);
  if (blockIdx.x != 0) return;
  // pass 4 (CTA 0): rank the candidates, check the margin, write S_t and b_t
  __shared__ unsigned long long ek[kSampCap];
  __shared__ int eidx[kSampCap];
  __shared__ double elog[kSampCap];
  __shared__ long long sorted_idx[kMaxBlock];
  __shared__ double sorted_log[kMaxBlock];
  const int nc = (int)__ldcg(ncand);  // counted by every CTA's atomics
  const bool overflow = nc > cap;
  const int m = overflow ? 0 : nc;
  for (int e = threadIdx.x; e < m; e += kCoopThreads) {  // written by other CTAs: read from L2
    ek[e] = __ldcg(cand_key + e);
    eidx[e] = __ldcg(cand + e);
    elog[e] = __ldcg(cand_log + e);
  }
  __syncthreads();
  long long bt = (long long)total1;
  if (bt > b) bt = b;
  const long long room = st->k_cap - st->k;
  if (bt > room) bt = room;
  if (bt < 0) bt = 0;
  for (int e = threadIdx.x; e < m; e += kCoopThreads) {
    int rank = 0;
    const unsigned long long ke = ek[e];
    const int ie = eidx[e];
    for (int f = 0; f < m; ++f) rank += (ek[f] < ke || (ek[f] == ke && eidx[f] < ie)) ? 1 : 0;
    if (rank < bt) {
      sorted_idx[rank] = ie;
      sorted_log[rank] = elog[e];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !st->done) {
    bool exact = !overflow && m >= bt;
    if (exact && bt > 0 && (long long)m < (long long)total1 && c22 != 0x3FFFFFu) {
      // every row outside the cut has an FP32 key >= the smallest key above the cut
      const float outside = key_to_float(((c22 + 1u) << 10));
      exact = sorted_log[bt - 1] < (double)outside - (double)kCutGuard - 1e-6 * fabs((double)outside);
    }
    if (!exact) {
      st->sample_fallback = 1;
    } else {
      st->sample_fallback = 0;
      st->b_t = bt;
      if (bt == 0) st->done = 1;
    }
  }
  __syncthreads();
  if (!st->sample_fallback)
    for (int e = threadIdx.x; e < bt; e += kCoopThreads) S_t[e] = sorted_idx[e];
  // clear the pass buffers for the next block (every other CTA is past its last read)
  for (int j = threadIdx.x; j < kBins; j += kCoopThreads) {
    hist1[j] = 0;
    hist2[j] = 0;
  }
  if (threadIdx.x == 0) *ncand = 0;
}

size_t sample2_scratch_bytes(long long n) {
  return (size_t)n * 4 + 2 * kBins * 4 + 64 + (size_t)kSampCap * (4 + 8 + 8) + 16;
}

cudaError_t launch_sample_clear(void* scratch, long long n, cudaStream_t s) {
  unsigned int* K32 = (unsigned int*)scratch;
  unsigned int* hist1 = K32 + n;
  unsigned int* hist2 = hist1 + kBins;
  unsigned int* ncand = hist2 + kBins;
  k_samp_clear<<<1, 256, 0, s>>>(hist1, hist2, ncand);
  return counted(cudaGetLastError());
}

cudaError_t launch_sample2(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                           unsigned long long problem, void* scratch, long long* S_t, State* st, cudaStream_t s) {
  unsigned int* K32 = (unsigned int*)scratch;
  unsigned int* hist1 = K32 + n;
  unsigned int* hist2 = hist1 + kBins;
  unsigned int* ncand = hist2 + kBins;
  int* cand = (int*)(ncand + 16);
  // 8-byte aligned arrays after the candidate rows
  unsigned long long* cand_key = (unsigned long long*)(((uintptr_t)(cand + kSampCap) + 15) & ~(uintptr_t)15);
  double* cand_log = (double*)(cand_key + kSampCap);
  const int want = b + kMargin;
  {
    // one cooperative launch, one CTA per SM, when the device allows it (asked once per device)
    static std::atomic<int> coop_sms[64];  // 0: not asked, -1: not available, else the SM count
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (coop_sms[dev] == 0) {
      int sms = 0, per_sm = 0, coop = 0;
      const bool ok = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
                      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_coop, kCoopThreads, 0) ==
                          cudaSuccess &&
                      per_sm >= 1;
      (void)cudaGetLastError();
      coop_sms[dev] = ok ? sms : -1;
    }
    if (coop_sms[dev] > 0) {
      const int sms = coop_sms[dev];
      int cap = kSampCap;
      // cooperative, and allowed to be scheduled as the previous kernel drains
      // (programmatic dependent launch; the kernel starts with pdl_wait())
      static std::atomic<int> pdl_ok{1};
      if (pdl_ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)sms);
        cfg.blockDim = dim3(kCoopThreads);
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, k_sample_coop, dvec, n, K32, hist1, hist2, want, cand,
                                                 cand_key, cand_log, ncand, cap, b, greedy, seed, problem, S_t, st);
        if (e == cudaSuccess) return counted(e);
        (void)cudaGetLastError();  // the combination is not supported: plain cooperative launches from now on
        pdl_ok = 0;
      }
      void* args[] = {(void*)&dvec, (void*)&n, (void*)&K32, (void*)&hist1, (void*)&hist2, (void*)&want,
                      (void*)&cand, (void*)&cand_key, (void*)&cand_log, (void*)&ncand, (void*)&cap, (void*)&b,
                      (void*)&greedy, (void*)&seed, (void*)&problem, (void*)&S_t, (void*)&st};
      return counted(cudaLaunchCooperativeKernel((const void*)k_sample_coop, dim3((unsigned)sms), dim3(kCoopThreads),
                                                 args, 0, s));
    }
  }
  const unsigned grid = (unsigned)((n + kSampThreads * kSampPerThread - 1) / (kSampThreads * kSampPerThread));
  k_samp_keys<<<grid, kSampThreads, 0, s>>>(dvec, n, K32, hist1, greedy, seed, problem, st);
  cudaError_t e = counted(cudaGetLastError());
  if (e != cudaSuccess) return e;
  k_samp_hist2<<<grid, kSampThreads, 0, s>>>(K32, n, hist1, hist2, want, st);
  if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
  k_samp_compact<<<grid, kSampThreads, 0, s>>>(K32, dvec, n, hist1, hist2, want, cand, cand_key, cand_log, ncand,
                                                kSampCap, greedy, seed, problem, st);
  if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
  k_samp_final<<<1, 1024, 0, s>>>(n, hist1, hist2, want, cand, cand_key, cand_log, ncand, kSampCap, b, S_t, st);
  return counted(cudaGetLastError());
}

}  // namespace rbrp
