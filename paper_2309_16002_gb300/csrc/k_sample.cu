// Alg. 2's sampling step on the GPU: S_t ~ d / ||d||_1 without replacement (reading of
// the sampling step as an exponential race: keys kappa_i = -log(u_i) / d_i over
// eligible rows, the b_t smallest in ascending (kappa, i) order; the greedy
// variant of the blockwise greedy remark uses -d_i).  The drawn rows are then
// gathered into V (the projection step's V = R(S_t, :), or X(S_t, :) in the
// downdate form), so the block's next kernel starts from V.
//
// Two stages, exact, in one cooperative launch (one CTA per SM, grid barriers
// between the passes):
//  1. a log-domain FP32 key log(-log u_i) - log d_i per row (Philox and FP32
//     logarithms only; FP64 arithmetic is slow on GB300) and an 11 + 11-bit
//     radix histogram over those keys choose a cut that keeps at least
//     b + kMargin candidates;
//  2. each CTA lists its candidates and computes their FP64 keys exactly as the
//     oracle does; every CTA then ranks all candidates by (key, row), checks
//     that the cut lies more than the FP32 error bound above the b_t-th exact key
//     (so no row outside the cut can belong to S_t) and, all CTAs having reached
//     the same decision from the same data, gathers its share of the rows of V.
// Three grid barriers per block (two when the first histogram already places the
// cut), each ~2-3 us on GB300.
// If the check fails, or the candidate list overflows, State::sample_fallback is
// raised and the exact FP64 sampler (k_sample_exact, launched after this kernel
// and returning at once otherwise) draws the block and gathers V instead.
//
// The pass buffers (histograms, candidate count) come in two sets: block t uses
// set t mod 2 and clears the other one, which the previous block's launch used
// and the next block's will use, so no pass of a block waits to clear its own.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <atomic>

#include "rbrp_internal.cuh"
#include "sample_common.cuh"

namespace rbrp {

namespace {

constexpr int kCoopThreads = 1024;
// Error allowance, relative to 1 + |log kappa|, of the FP32 logarithm that the
// margin check takes of the b_t-th exact key (log_d_f32: an FP32 product for the
// exponent term plus an FP32 logarithm of the mantissa, each good to an FP32 ulp or
// two of 1 + |log kappa|, i.e. below ~2e-7 of it).
constexpr double kLogCheckSlack = 1e-6;

// Layout of the sampler's scratch (sample2_scratch_bytes): per-row FP32 keys, two
// sets of histograms, control words, the candidates' rows and exact keys.
struct SampLayout {
  unsigned int* K32;   // n
  unsigned int* H1;    // 2 x kBins (set-major)
  unsigned int* H2;    // 2 x kBins
  unsigned int* ctl;   // 16 words: [0], [1] candidate count per set; [2], [3] grid barrier;
                       // [4] finished level-0 CTAs of the exact sampler
  int* cand;           // kSampCap
  unsigned long long* cand_key;  // kSampCap
};

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

SampLayout samp_layout(void* scratch, long long n) {
  SampLayout L;
  uint8_t* p = (uint8_t*)scratch;
  L.K32 = (unsigned int*)p;
  p += align16((size_t)n * 4);
  L.H1 = (unsigned int*)p;
  p += 2 * kBins * 4;
  L.H2 = (unsigned int*)p;
  p += 2 * kBins * 4;
  L.ctl = (unsigned int*)p;
  p += 64;
  L.cand = (int*)p;
  p += align16((size_t)kSampCap * 4);
  L.cand_key = (unsigned long long*)p;
  return L;
}

}  // namespace

size_t sample2_scratch_bytes(long long n) {
  return align16((size_t)n * 4) + 4 * kBins * 4 + 64 + align16((size_t)kSampCap * 4) + (size_t)kSampCap * 8 + 256;
}

// Block-wide search over a 2048-bin histogram: the first bin where the running
// count reaches `want`; returns the count below that bin in *below (or bin
// kBins and the total when the histogram holds fewer than `want`).  The first
// 256 threads each sum eight bins and take an exclusive scan of those sums; the
// one thread whose range contains the want-th count walks its bins.  The bins
// are read through L2 (__ldcg): they were filled by other CTAs' atomics earlier
// in the same launch, and every CTA must see the same counts to take the same
// branch at the next grid barrier (a non-coherent or L1-cached read could be
// stale).
__device__ int find_bin(const unsigned int* hist, unsigned int want, unsigned int* below, unsigned int* total) {
  constexpr int kScan = 256;
  __shared__ unsigned int wsum[kScan / 32];
  __shared__ int s_bin;
  __shared__ unsigned int s_below, s_total;
  constexpr int per = kBins / kScan;  // 8 bins per thread
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned int c[per], sum = 0, incl = 0;
  if (t < kScan) {
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
  if (t < kScan) {
    unsigned int before = 0, all = 0;
#pragma unroll
    for (int q = 0; q < kScan / 32; ++q) {
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

struct CoopArgs {
  const double* dvec;
  long long n;
  unsigned int* K32;
  unsigned int* H1;
  unsigned int* H2;
  unsigned int* ctl;
  int* cand;
  unsigned long long* cand_key;
  int want, cap, b, greedy;
  unsigned long long seed, problem;
  long long* S_t;
  State* st;
  GatherSpec g;
};

__global__ void __launch_bounds__(kCoopThreads) k_sample_coop(const __grid_constant__ CoopArgs a) {
  pdl_wait();
  State* st = a.st;
  if (st->done) return;  // read before any CTA writes the State: the same for every CTA
  __shared__ unsigned int h[kBins];
  __shared__ unsigned long long ek[kSampCap];
  __shared__ int eidx[kSampCap];
  __shared__ int rnk[kSampCap];
  __shared__ long long sorted_idx[kMaxBlock];
  __shared__ unsigned long long s_kth;
  __shared__ int s_exact, s_cnt;
  __shared__ unsigned int s_base;
  const long long n = a.n;
  const unsigned long long tblk = st->t;
  const long long room = st->k_cap - st->k;
  const unsigned glim = st->spin_grid;
  const unsigned long long block_no = tblk + 1ULL;  // the paper's t
  const int set = (int)(tblk & 1ULL), other = set ^ 1;
  unsigned int* hist1 = a.H1 + set * kBins;
  unsigned int* hist2 = a.H2 + set * kBins;
  unsigned int* ncand = a.ctl + set;
  unsigned int* bar = a.ctl + 2;
  const int tid = threadIdx.x, lane = tid & 31;
  const long long gstride = (long long)gridDim.x * kCoopThreads;
  const long long g0 = (long long)blockIdx.x * kCoopThreads + tid;
  // the other set: last used by the previous block's launch (complete), next by the next block's
  if (blockIdx.x == gridDim.x - 1) {
    for (int j = tid; j < kBins; j += kCoopThreads) {
      a.H1[other * kBins + j] = 0;
      a.H2[other * kBins + j] = 0;
    }
    if (tid == 0) a.ctl[other] = 0;
  }
  // pass 1: keys and the histogram of their top 11 bits
  for (int j = tid; j < kBins; j += kCoopThreads) h[j] = 0;
  __syncthreads();
  for (long long i = g0; i < n; i += gstride) {
    const unsigned int k = approx_key(a.dvec[i], i, block_no, a.seed, a.problem, a.greedy);
    a.K32[i] = k;
    if (k != 0xFFFFFFFFu) atomicAdd(&h[k >> 21], 1u);
  }
  __syncthreads();
  for (int j = tid; j < kBins; j += kCoopThreads)
    if (h[j]) atomicAdd(&hist1[j], h[j]);
  grid_barrier(bar, st, glim);
  // pass 2: histogram of the next 11 bits inside the cut bin -- skipped (with
  // its barrier) when the whole cut bin adds few candidates, which every CTA
  // decides alike from the same first histogram
  unsigned int below1, total1;
  const int b1 = find_bin(hist1, (unsigned int)a.want, &below1, &total1);
  const bool one_level = b1 < kBins && below1 + __ldcg(hist1 + b1) <= (unsigned int)(2 * a.want);
  if (b1 < kBins && !one_level) {
    for (int j = tid; j < kBins; j += kCoopThreads) h[j] = 0;
    __syncthreads();
    for (long long i = g0; i < n; i += gstride) {
      const unsigned int k = a.K32[i];
      if ((int)(k >> 21) == b1 && k != 0xFFFFFFFFu) atomicAdd(&h[(k >> 10) & 0x7FF], 1u);
    }
    __syncthreads();
    for (int j = tid; j < kBins; j += kCoopThreads)
      if (h[j]) atomicAdd(&hist2[j], h[j]);
    grid_barrier(bar, st, glim);
  }
  unsigned int c22 = 0x3FFFFFu;  // rows whose key's top 22 bits are <= c22 are candidates
  if (one_level) {
    c22 = ((unsigned int)b1 << 11) | 0x7FFu;  // every row of the cut bin
  } else if (b1 < kBins) {
    unsigned int below2, total2;
    const int b2 = find_bin(hist2, (unsigned int)(a.want - (int)below1), &below2, &total2);
    c22 = ((unsigned int)b1 << 11) | (unsigned int)(b2 >= kBins ? kBins - 1 : b2);
  }
  // pass 3: the CTA's candidates into a shared list (one shared atomic per warp), one
  // reservation in the global list per CTA, then their exact FP64 keys, packed into
  // the CTA's first warps (a CTA holds a few dozen candidates at most on the usual
  // inputs, and GB300's FP64 pipe retires about two FMAs per clock per SM)
  int* lrow = eidx;  // (eidx is free until pass 4)
  if (tid == 0) s_cnt = 0;
  __syncthreads();
  for (long long i0 = g0 - lane; i0 < n; i0 += gstride) {
    const long long i = i0 + lane;
    bool pick = false;
    if (i < n) {
      const unsigned int k = a.K32[i];
      pick = k != 0xFFFFFFFFu && (k >> 10) <= c22;
    }
    const unsigned int mk = __ballot_sync(0xffffffffu, pick);
    if (mk == 0u) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(&s_cnt, __popc(mk));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int pos = base + __popc(mk & ((1u << lane) - 1u));
    if (pick && pos < kSampCap) lrow[pos] = (int)i;
  }
  __syncthreads();
  const int lc = min(s_cnt, kSampCap);
  if (tid == 0) s_base = s_cnt ? atomicAdd(ncand, (unsigned int)s_cnt) : 0u;
  __syncthreads();
  for (int e = tid; e < lc; e += kCoopThreads) {
    const unsigned int pos = s_base + (unsigned int)e;
    if ((int)pos < a.cap) {
      const long long i = lrow[e];
      a.cand[pos] = (int)i;
      a.cand_key[pos] = exact_key(a.dvec[i], i, block_no, a.seed, a.problem, a.greedy);
    }
  }
  grid_barrier(bar, st, glim);
  // pass 4 (every CTA, the same result): rank the candidates by (exact key, row),
  // check the margin, then CTA 0 writes S_t, b_t and the State, and every CTA
  // gathers its share of V
  const int nc = (int)__ldcg(ncand);  // counted by every CTA's atomics
  const bool overflow = nc > a.cap;
  const int m = overflow ? 0 : nc;
  for (int e = tid; e < m; e += kCoopThreads) {
    ek[e] = __ldcg(a.cand_key + e);  // written by other CTAs: read from L2
    eidx[e] = __ldcg(a.cand + e);
    rnk[e] = 0;
  }
  long long bt = (long long)total1;
  if (bt > a.b) bt = a.b;
  if (bt > room) bt = room;
  if (bt < 0) bt = 0;
  __syncthreads();
  // rank of candidate e = the number of candidates before it; the m x m comparisons
  // are split into m x S (candidate, segment) units over all threads
  if (m > 0) {
    const int S = max(1, kCoopThreads / m), L = (m + S - 1) / S;
    for (int u = tid; u < m * S; u += kCoopThreads) {
      const int e = u % m, f0 = (u / m) * L, f1 = min(m, f0 + L);
      const unsigned long long ke = ek[e];
      const int ie = eidx[e];
      int cnt = 0, f = f0;
      for (; f + 4 <= f1; f += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const unsigned long long kf = ek[f + q];
          const int jf = eidx[f + q];
          cnt += (int)((kf < ke) | ((kf == ke) & (jf < ie)));
        }
      }
      for (; f < f1; ++f) {
        const unsigned long long kf = ek[f];
        const int jf = eidx[f];
        cnt += (int)((kf < ke) | ((kf == ke) & (jf < ie)));
      }
      if (cnt) atomicAdd(&rnk[e], cnt);
    }
  }
  __syncthreads();
  for (int e = tid; e < m; e += kCoopThreads) {
    const int r = rnk[e];
    if (r < bt) sorted_idx[r] = eidx[e];
    if (r == bt - 1) s_kth = ek[e];
  }
  __syncthreads();
  if (tid == 0) {
    bool exact = !overflow && m >= bt;
    if (exact && bt > 0 && (long long)m < (long long)total1 && c22 != 0x3FFFFFu) {
      // every row outside the cut has an FP32 log-domain key >= the smallest key above
      // the cut; the b_t-th exact key's logarithm (greedy: -log d), taken in FP32 with
      // its own error allowance, must lie below that by more than the FP32 key bound
      const float outside = key_to_float(((c22 + 1u) << 10));
      const double kb = from_orderable(s_kth);
      const float lk = a.greedy ? -log_d_f32(-kb) : log_d_f32(kb);
      const double T = (double)outside - (double)kCutGuard - 1e-6 * fabs((double)outside);
      exact = (double)lk + kLogCheckSlack * (1.0 + fabs((double)lk)) < T;
    }
    s_exact = exact ? 1 : 0;
    if (blockIdx.x == 0 && !st->done) {
      if (!exact) {
        st->sample_fallback = 1;
      } else {
        st->sample_fallback = 0;
        st->b_t = bt;
        if (bt == 0) st->done = 1;
      }
    }
  }
  __syncthreads();
  if (!s_exact) return;
  if (blockIdx.x == 0)
    for (int e = tid; e < bt; e += kCoopThreads) a.S_t[e] = sorted_idx[e];
  gather_rows(a.g, n, sorted_idx, (int)bt, blockIdx.x, gridDim.x, tblk == 0);
}

// ---------------------------------------------------------------- the exact FP64 sampler
// Alg. 2's sampling step with exact FP64 keys for every row: each CTA sorts
// kSortChunk rows by (key, row) and keeps its b smallest; the last CTA to finish
// (a counter, no waiting) merges those lists in chunks of kSortChunk until one
// chunk is left, writes S_t and b_t and gathers V.  Runs when `force` is set or the
// two-stage sampler raised State::sample_fallback; otherwise returns at once.
__device__ void exact_finish(Pair* sh, long long n, int b, long long* S_t, State* st, const GatherSpec& g,
                             bool first_block) {
  __shared__ int nfin;
  __shared__ long long rows[kMaxBlock];
  if (threadIdx.x == 0) nfin = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < b; e += blockDim.x)
    if (sh[e].key != kIneligible) atomicAdd(&nfin, 1);
  __syncthreads();
  long long bt = nfin;
  if (bt > b) bt = b;
  const long long room = st->k_cap - st->k;
  if (bt > room) bt = room;
  if (bt < 0) bt = 0;
  for (int e = threadIdx.x; e < bt; e += blockDim.x) {
    S_t[e] = sh[e].idx;
    rows[e] = sh[e].idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->b_t = bt;
    st->sample_fallback = 0;
    if (bt == 0) st->done = 1;
  }
  gather_rows(g, n, rows, (int)bt, 0, 1, first_block);
}

__global__ void __launch_bounds__(kSortChunk / 2) k_sample_exact(const double* __restrict__ dvec, long long n,
                                                                 Pair* __restrict__ bufA, Pair* __restrict__ bufB,
                                                                 unsigned int* __restrict__ counter, int b, int greedy,
                                                                 unsigned long long seed, unsigned long long problem,
                                                                 long long* __restrict__ S_t, State* st, int force,
                                                                 const __grid_constant__ GatherSpec g) {
  pdl_wait();
  if (st->done || (!force && !st->sample_fallback)) return;
  __shared__ Pair sh[kSortChunk];
  __shared__ int s_last;
  const unsigned long long block_no = (unsigned long long)st->t + 1ULL;  // the paper's t
  const long long base = (long long)blockIdx.x * kSortChunk;
  for (int e = threadIdx.x; e < kSortChunk; e += blockDim.x) {
    const long long i = base + e;
    Pair p{kIneligible, LLONG_MAX};
    if (i < n) {
      p.key = exact_key(dvec[i], i, block_no, seed, problem, greedy);
      p.idx = i;
    }
    sh[e] = p;
  }
  sort_chunk(sh);
  if (gridDim.x == 1) {
    exact_finish(sh, n, b, S_t, st, g, block_no == 1ULL);
    return;
  }
  for (int e = threadIdx.x; e < b; e += blockDim.x) bufA[(long long)blockIdx.x * b + e] = sh[e];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;  // for the next block
  // the last CTA: merge the lists, kSortChunk pairs at a time
  long long n_in = (long long)gridDim.x * b;
  Pair* in = bufA;
  Pair* out = bufB;
  for (;;) {
    const long long chunks = (n_in + kSortChunk - 1) / kSortChunk;
    for (long long c = 0; c < chunks; ++c) {
      for (int e = threadIdx.x; e < kSortChunk; e += blockDim.x) {
        const long long j = c * kSortChunk + e;
        Pair p{kIneligible, LLONG_MAX};
        if (j < n_in) {
          p.key = __ldcg(&in[j].key);  // written by other CTAs: read from L2
          p.idx = __ldcg(&in[j].idx);
        }
        sh[e] = p;
      }
      sort_chunk(sh);
      if (chunks == 1) {
        exact_finish(sh, n, b, S_t, st, g, block_no == 1ULL);
        return;
      }
      for (int e = threadIdx.x; e < b; e += blockDim.x) out[c * b + e] = sh[e];
      __syncthreads();
    }
    __threadfence();
    __syncthreads();
    n_in = chunks * b;
    Pair* tmp = in;
    in = out;
    out = tmp;
  }
}

__global__ void k_samp_clear(unsigned int* __restrict__ H1, unsigned int* __restrict__ H2,
                             unsigned int* __restrict__ ctl) {
  for (int j = threadIdx.x; j < 2 * kBins; j += blockDim.x) {
    H1[j] = 0;
    H2[j] = 0;
  }
  if (threadIdx.x < 16) ctl[threadIdx.x] = 0;  // counts, barrier words, merge counter
}

cudaError_t launch_sample_clear(void* scratch, long long n, cudaStream_t s) {
  const SampLayout L = samp_layout(scratch, n);
  k_samp_clear<<<1, 256, 0, s>>>(L.H1, L.H2, L.ctl);
  return counted(cudaGetLastError());
}

cudaError_t launch_sample2(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                           unsigned long long problem, void* scratch, long long* S_t, State* st,
                           const GatherSpec& g, int* exact_always, cudaStream_t s) {
  *exact_always = 0;
  const SampLayout L = samp_layout(scratch, n);
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
  if (coop_sms[dev] < 0) {  // no cooperative launches: the exact sampler draws every block
    *exact_always = 1;
    return cudaSuccess;
  }
  CoopArgs a;
  a.dvec = dvec;
  a.n = n;
  a.K32 = L.K32;
  a.H1 = L.H1;
  a.H2 = L.H2;
  a.ctl = L.ctl;
  a.cand = L.cand;
  a.cand_key = L.cand_key;
  a.want = b + kMargin;
  a.cap = kSampCap;
  a.b = b;
  a.greedy = greedy;
  a.seed = seed;
  a.problem = problem;
  a.S_t = S_t;
  a.st = st;
  a.g = g;
  // cooperative, and allowed to be scheduled as the previous kernel drains
  // (programmatic dependent launch; the kernel starts with pdl_wait())
  static std::atomic<int> pdl_ok{1};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)coop_sms[dev]);
  cfg.blockDim = dim3(kCoopThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_ok ? 2 : 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_sample_coop, a);
  if (e != cudaSuccess && cfg.numAttrs == 2) {
    (void)cudaGetLastError();  // the combination is not supported: plain cooperative launches from now on
    pdl_ok = 0;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_sample_coop, a);
  }
  return counted(e);
}

cudaError_t launch_sample_exact(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                                unsigned long long problem, void* cand_a, void* cand_b, void* scratch, long long* S_t,
                                State* st, int force, const GatherSpec& g, cudaStream_t s) {
  const SampLayout L = samp_layout(scratch, n);
  const long long groups = (n + kSortChunk - 1) / kSortChunk;
  return counted(launch_pdl(k_sample_exact, dim3((unsigned)(groups > 0 ? groups : 1)), dim3(kSortChunk / 2), 0, s,
                            dvec, n, (Pair*)cand_a, (Pair*)cand_b, L.ctl + 4, b, greedy, seed, problem, S_t, st,
                            force, g));
}

}  // namespace rbrp
