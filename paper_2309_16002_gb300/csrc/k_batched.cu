// Batched RBRP: many small independent row IDs (Alg. 2 + Alg. 3) in one
// persistent launch.
//
// Each CTA takes whole problems from a work queue (largest first) and runs the
// complete method for one problem at a time on CUDA cores: initial norms,
// the block loop (exact exponential-race sampling, gather, CGS2 against Q,
// the pivoted-Cholesky form of the robust blockwise filter with tau_b = 1/b_t,
// CholQR of the accepted rows with one CGS pass and a second CholQR, the
// residual update with row-norm recomputation, the stopping test) and the W
// solve.  Problems are small (m <= 4096 rows, n <= 256 columns, blocks of
// b <= 32), so a problem's residual, L and Q live in the CTA's workspace slot
// (L2-resident) and the small b x b steps run in shared memory; no step needs
// more than one SM, and the only inter-CTA traffic is the work counter.
//
// The passes over rows (initial norms, CGS, FP64 residual update) share one
// routine: a warp holds a group of rows in registers (n <= 256: eight values
// a lane), issues all their loads at once, and for each basis row forms the
// coefficients (a butterfly all-reduce over the warp) and subtracts.  The FP32
// residual update, the largest pass, spreads a row over eight lanes instead
// (four rows a warp, float4 columns), which cuts the shuffle levels per
// coefficient from five per row to three for four rows.  Loads of a group are
// in flight together; a problem's residual sits in L2 and each pass is a few
// hundred kilobytes.
//
// T is the storage and arithmetic type (float or double); NT (256 or 512) the
// CTA size, a schedule parameter chosen by the host (autotuned per batch).
// Results do not depend on NT: sums over rows use a fixed 256-way partition
// and every other reduction is per warp.  Sampling keys are the exact FP64
// keys of Alg. 2's sampling step as in the single-problem sampler: FP32 log-domain
// keys choose >= b_t + 32 candidates, their FP64 keys are ranked, and a margin
// check against the FP32 error bound proves that no other row could be drawn
// (else every eligible row is keyed in FP64).  Problem p uses Philox problem
// id pbase + p.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "rbrp_internal.cuh"
#include "sample_common.cuh"

namespace rbrp {
namespace bt {

constexpr int kMaxWarps = kBatchMaxThreads / 32;
constexpr int kSumLanes = 256;   // fixed partition of sums over rows
constexpr int kCand = 1024;      // candidates the sampler ranks exactly

// Offsets of one slot (bytes), for the batch maxima.
struct Slot {
  size_t R, L, Q, d, mark, V, Y, K64, Wt, total;
};
__host__ __device__ inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline Slot slot_layout(long long m, long long n, long long kc, int b, size_t sT) {
  Slot s;
  size_t o = 0;
  s.R = o;
  o = al256(o + (size_t)m * ((n + 3) / 4 * 4) * sT);  // leading dimension n rounded up to 4
  s.L = o;
  o = al256(o + (size_t)m * kc * sT);
  s.Q = o;
  o = al256(o + (size_t)kc * n * sT);
  s.d = o;
  o = al256(o + (size_t)m * 8);
  s.mark = o;
  o = al256(o + (size_t)m * 4);
  s.V = o;
  o = al256(o + (size_t)b * n * sT);
  s.Y = o;
  o = al256(o + (size_t)b * n * sT);
  s.K64 = o;  // fallback sampler keys
  o = al256(o + (size_t)m * 8);
  s.Wt = o;   // W solve scratch, column-major
  o = al256(o + (size_t)m * kc * sT);
  s.total = o;
  return s;
}

struct Smem {
  unsigned int keys[kBatchMaxRows];
  unsigned int hist[kBins];
  unsigned long long ek[kCand];
  double elg[kCand];  // log of each candidate's exact key
  int cand[kCand];
  int St[32];
  int perm[32];
  double G[32][33];   // Gram / Schur complement
  double Lw[32][33];  // factor, candidate-indexed then pivot-indexed
  double red[kMaxWarps];
  unsigned int cnt;
  int bin, bp;
  unsigned int below, total;
  int flag;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread, warps in order; every thread gets the result.
// Callers fill only threads < kSumLanes, so the value does not depend on NT.
template <int NT>
__device__ double block_sum(double v, Smem& sm) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) s += sm.red[q];
  return s;
}

// First bin of sm.hist where the running count reaches want (kBins if never),
// with the count below it; every thread gets both.
template <int NT>
__device__ int find_bin_cta(Smem& sm, unsigned int want, unsigned int* below) {
  constexpr int per = kBins / NT;
  constexpr int NW = NT / 32;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  unsigned int c[per], sum = 0;
#pragma unroll
  for (int q = 0; q < per; ++q) {
    c[q] = sm.hist[t * per + q];
    sum += c[q];
  }
  unsigned int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) sm.red[w] = (double)incl;
  if (t == 0) sm.bin = kBins;
  __syncthreads();
  unsigned int before = 0, all = 0;
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const unsigned int x = (unsigned int)sm.red[q];
    if (q < w) before += x;
    all += x;
  }
  incl += before;
  const unsigned int excl = incl - sum;
  if (excl < want && incl >= want) {
    unsigned int r2 = excl;
#pragma unroll
    for (int q = 0; q < per; ++q) {
      if (r2 + c[q] >= want) {
        sm.bin = t * per + q;
        sm.below = r2;
        break;
      }
      r2 += c[q];
    }
  }
  if (t == 0) sm.total = all;
  __syncthreads();
  const int bin = sm.bin;
  *below = (bin == kBins) ? sm.total : sm.below;
  __syncthreads();
  return bin;
}

// Exact FP64 key of row i (as ordered bits) and its logarithm (Alg. 2, sampling step).
__device__ __forceinline__ void exact_key(double di, long long i, unsigned long long t, unsigned long long seed,
                                          unsigned long long p, int greedy, unsigned long long* key, double* lg) {
  if (greedy) {
    *key = orderable(-di);
    *lg = -log(di);
  } else {
    const double u = philox_uniform((unsigned long long)i, t, seed, p);
    const double k = -log(u) / di;
    *key = orderable(k);
    *lg = log(k);
  }
}

template <int NT>
__device__ void sample_cut(const double* d, const int* mark, long long m, int bt, long long ne, unsigned long long t,
                           const BatchedArgs& a, unsigned long long p, Smem& sm);

// S_t (bt rows, in draw order) into sm.St.  ne = number of eligible rows.
// The two-stage draw, or (a.exact, or when its check fails) the full ranking.
template <int NT>
__device__ void sample_cta(const double* d, const int* mark, long long m, int bt, long long ne, unsigned long long t,
                           const BatchedArgs& a, unsigned long long p, unsigned long long* K64, Smem& sm) {
  const int tid = threadIdx.x;
  if (a.exact) {
    if (tid == 0) sm.flag = 1;
    __syncthreads();
  } else {
    sample_cut<NT>(d, mark, m, bt, ne, t, a, p, sm);
  }
  if (!sm.flag) return;
  // full ranking: FP64 keys of every eligible row, ranked by counting
  for (long long i = tid; i < m; i += NT) {
    unsigned long long k = kIneligible;
    if (mark[i] == 0 && d[i] > 0.0) {
      double lg;
      exact_key(d[i], i, t, a.seed, p, a.greedy, &k, &lg);
    }
    K64[i] = k;
  }
  __syncthreads();
  for (long long i = tid; i < m; i += NT) {
    const unsigned long long ki = K64[i];
    if (ki == kIneligible) continue;
    long long rank = 0;
    for (long long j = 0; j < m && rank < bt; ++j) {
      const unsigned long long kj = K64[j];
      rank += (kj < ki || (kj == ki && j < i)) ? 1 : 0;
    }
    if (rank < bt) sm.St[rank] = (int)i;
  }
  __syncthreads();
}

// The two-stage draw: FP32 keys, a 2 x 11-bit radix cut keeping >= bt + kMargin
// candidates, their exact keys ranked; sm.flag = 1 when the margin check
// fails or the candidates overflow (the caller then ranks every row).
template <int NT>
__device__ void sample_cut(const double* d, const int* mark, long long m, int bt, long long ne, unsigned long long t,
                           const BatchedArgs& a, unsigned long long p, Smem& sm) {
  const int tid = threadIdx.x;
  for (long long i = tid; i < m; i += NT) {
    const bool elig = mark[i] == 0 && d[i] > 0.0;
    sm.keys[i] = elig ? approx_key(d[i], i, t, a.seed, p, a.greedy) : 0xFFFFFFFFu;
  }
  const unsigned int want = (unsigned int)(bt + kMargin < ne ? bt + kMargin : ne);
  for (int j = tid; j < kBins; j += NT) sm.hist[j] = 0;
  __syncthreads();
  for (long long i = tid; i < m; i += NT)
    if (sm.keys[i] != 0xFFFFFFFFu) atomicAdd(&sm.hist[sm.keys[i] >> 21], 1u);
  __syncthreads();
  unsigned int below1 = 0, below2 = 0;
  const int b1 = find_bin_cta<NT>(sm, want, &below1);
  for (int j = tid; j < kBins; j += NT) sm.hist[j] = 0;
  __syncthreads();
  for (long long i = tid; i < m; i += NT) {
    const unsigned int k = sm.keys[i];
    if (k != 0xFFFFFFFFu && (int)(k >> 21) == b1) atomicAdd(&sm.hist[(k >> 10) & 0x7FF], 1u);
  }
  __syncthreads();
  int b2 = find_bin_cta<NT>(sm, want - below1, &below2);
  if (b2 >= kBins) b2 = kBins - 1;
  const unsigned int c22 = ((unsigned int)b1 << 11) | (unsigned int)b2;
  if (tid == 0) sm.cnt = 0;
  __syncthreads();
  for (long long i = tid; i < m; i += NT) {
    const unsigned int k = sm.keys[i];
    if (k != 0xFFFFFFFFu && (k >> 10) <= c22) {
      const unsigned int pos = atomicAdd(&sm.cnt, 1u);
      if (pos < (unsigned int)kCand) sm.cand[pos] = (int)i;
    }
  }
  __syncthreads();
  const int nc = (int)sm.cnt;
  const bool overflow = nc > kCand;
  const int mc = overflow ? 0 : nc;
  for (int e = tid; e < mc; e += NT) {
    double lg;
    exact_key(d[sm.cand[e]], sm.cand[e], t, a.seed, p, a.greedy, &sm.ek[e], &lg);
    sm.elg[e] = lg;
  }
  if (tid == 0) sm.flag = (!overflow && mc >= bt) ? 0 : 1;
  __syncthreads();
  const float outside = key_to_float(((c22 + 1u) << 10));
  for (int e = tid; e < mc; e += NT) {
    int rank = 0;
    const unsigned long long ke = sm.ek[e];
    const int ie = sm.cand[e];
    for (int f = 0; f < mc; ++f) rank += (sm.ek[f] < ke || (sm.ek[f] == ke && sm.cand[f] < ie)) ? 1 : 0;
    if (rank < bt) sm.St[rank] = ie;
    // every row outside the cut has an FP32 key >= the smallest key above the
    // cut; the bt-th exact key must lie below that by more than the FP32 error bound
    if (rank == bt - 1 && (long long)mc < ne &&
        !(sm.elg[e] < (double)outside - (double)kCutGuard - 1e-6 * fabs((double)outside)))
      sm.flag = 1;
  }
  __syncthreads();
}

// Rows i < nrows of src (row-major, leading dimension ls, n <= 256 columns;
// row i read from src row rowmap[i] when rowmap is given; B has leading
// dimension n): c_ij = <src_i, B_j> for
// j < nb, every c_ij from the original row (classical Gram-Schmidt), and
// y_i = src_i - sum_j c_ij B_j with the terms subtracted in ascending j
// (BASIS = false: no basis, y_i = src_i).  COEF: coef[j * ldc + i] = c_ij.
// y_i goes to dst row i (leading dimension ldd >= n, columns n .. ldd - 1
// written as zeros), zeroed when mark && mark[i] != 0; NORM:
// dn[i] = ||y_i||^2 (0 for zeroed rows), the per-lane partial sums and their
// warp reduction in T.  One warp per group of RPW rows, whose loads are all
// issued before any arithmetic.  dst may alias src (each group is read
// completely before it is written).  STREAM: src is read once (the input X),
// with evict-first loads so that it does not push the residuals of the
// resident problems out of L2.  No barrier inside; the caller synchronises.
template <int NT, int RPW, int VEC, bool BASIS, bool COEF, bool NORM, typename T, typename TS, bool STREAM = false>
__device__ void project_rows(const TS* src, long long ls, const int* rowmap, T* dst, long long ldd, long long nrows,
                             long long n, const T* B, int nb, T* coef, long long ldc, double* dn, const int* mark) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long i0 = (long long)w * RPW; i0 < nrows; i0 += (long long)NW * RPW) {
    T x[RPW][VEC], y[RPW][VEC];
    bool zero[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const long long i = i0 + r;
      const long long si = (i < nrows) ? (rowmap ? (long long)rowmap[i] : i) : 0;
      zero[r] = mark && i < nrows && mark[i] != 0;  // read with the row, before any store of the group
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const long long c = lane + 32 * u;
        if (i < nrows && c < n) x[r][u] = STREAM ? (T)__ldcs(src + si * ls + c) : (T)src[si * ls + c];
        else x[r][u] = (T)0;
        y[r][u] = x[r][u];
      }
    }
    if (BASIS) {
      for (int j = 0; j < nb; ++j) {
        T q[VEC];
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const long long c = lane + 32 * u;
          q[u] = c < n ? B[(long long)j * n + c] : (T)0;
        }
        T s[RPW];
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          T acc = 0;
#pragma unroll
          for (int u = 0; u < VEC; ++u) acc += x[r][u] * q[u];
          s[r] = acc;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int r = 0; r < RPW; ++r) s[r] += __shfl_xor_sync(0xffffffffu, s[r], o);
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
#pragma unroll
          for (int u = 0; u < VEC; ++u) y[r][u] -= s[r] * q[u];
          if (COEF && lane == 0 && i0 + r < nrows) coef[(long long)j * ldc + i0 + r] = s[r];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const long long i = i0 + r;
      if (i >= nrows) break;
      T nr = 0;
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const long long c = lane + 32 * u;
        if (c >= ldd) continue;
        const T v = (zero[r] || c >= n) ? (T)0 : y[r][u];  // columns n .. ldd - 1: zero padding
        dst[i * ldd + c] = v;
        nr += v * v;
      }
      if (NORM) {
        // the warp reduction in T: on GB300 every FP64 warp instruction costs
        // about 64 issue cycles, which made FP64 shuffles and adds the largest
        // part of this pass
        const T s = warp_sum(nr);
        if (lane == 0) dn[i] = zero[r] ? 0.0 : (double)s;
      }
    }
  }
}

// The residual update of the FP32 form (Alg. 2, update step), with a row
// spread over eight lanes instead of 32: lanes 8g .. 8g + 7 of a warp hold row
// i0 + g (four rows a warp), lane q of the octet the float4 at columns
// 4q + 32u .. 4q + 32u + 3 for u < 8, so that the octet reads 128 contiguous
// bytes of a row per load (R and Q' with leading dimension ldr, a multiple of
// 4, padding columns zero).  A coefficient then takes three shuffle levels, each serving
// the warp's four rows at once, where the 32-lane layout takes five per row.
// c_ij = <R_i, Q'_j> from the original row, R_i -= sum_j c_ij Q'_j in
// ascending j, coef[j * ldc + i] = c_ij, dn[i] = ||R_i||^2; rows with
// mark[i] != 0 are zeroed (dn = 0).
template <int NT, int VEC>
__device__ void update_rows_oct(float* R, long long ldr, long long m, const float* Qs, int bp, float* coef,
                                long long ldc, double* dn, const int* mark) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 3, q = lane & 7;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i0 = (long long)w * 4; i0 < m; i0 += (long long)NW * 4) {
    const long long i = i0 + g;
    const bool valid = i < m;
    const bool zero = valid && mark[i] != 0;
    float4 x[VEC], y[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      const long long c = 4 * q + 32 * u;
      x[u] = (valid && c < ldr) ? *(const float4*)(R + i * ldr + c) : z4;
      y[u] = x[u];
    }
    const int nu = (int)((ldr - 4 * q + 31) / 32);  // float4 groups this lane holds
    for (int j = 0; j < bp; ++j) {
      const float* qj = Qs + (long long)j * ldr + 4 * q;
      // Q'_j is read from shared memory twice (dot, then subtraction) to keep
      // the registers for the row
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int u = 0; u < VEC; u += 2) {
        const float4 q0 = (u < nu) ? *(const float4*)(qj + 32 * u) : z4;
        const float4 q1 = (u + 1 < nu) ? *(const float4*)(qj + 32 * u + 32) : z4;
        a0 = fmaf(x[u].x, q0.x, a0);
        a0 = fmaf(x[u].y, q0.y, a0);
        a0 = fmaf(x[u].z, q0.z, a0);
        a0 = fmaf(x[u].w, q0.w, a0);
        a1 = fmaf(x[u + 1].x, q1.x, a1);
        a1 = fmaf(x[u + 1].y, q1.y, a1);
        a1 = fmaf(x[u + 1].z, q1.z, a1);
        a1 = fmaf(x[u + 1].w, q1.w, a1);
      }
      float acc = a0 + a1;
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const float4 qv = (u < nu) ? *(const float4*)(qj + 32 * u) : z4;
        y[u].x = fmaf(-acc, qv.x, y[u].x);
        y[u].y = fmaf(-acc, qv.y, y[u].y);
        y[u].z = fmaf(-acc, qv.z, y[u].z);
        y[u].w = fmaf(-acc, qv.w, y[u].w);
      }
      if (q == 0 && valid) coef[(long long)j * ldc + i] = acc;
    }
    float nr = 0.f;
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      const long long c = 4 * q + 32 * u;
      if (zero) y[u] = z4;
      if (valid && c < ldr) *(float4*)(R + i * ldr + c) = y[u];
      nr = fmaf(y[u].x, y[u].x, nr);
      nr = fmaf(y[u].y, y[u].y, nr);
      nr = fmaf(y[u].z, y[u].z, nr);
      nr = fmaf(y[u].w, y[u].w, nr);
    }
    nr += __shfl_xor_sync(0xffffffffu, nr, 4);
    nr += __shfl_xor_sync(0xffffffffu, nr, 2);
    nr += __shfl_xor_sync(0xffffffffu, nr, 1);
    if (q == 0 && valid) dn[i] = zero ? 0.0 : (double)nr;
  }
}

// sm.G[i][j] = <V_i, V_j> for i, j < rows (V row-major, leading dimension n);
// row i's values stay in registers while its warp walks j <= i.
template <int NT, typename T, int VEC>
__device__ void gram_rows(const T* V, int rows, long long n, Smem& sm) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = w; i < rows; i += NW) {
    T x[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      const long long c = lane + 32 * u;
      x[u] = c < n ? V[(long long)i * n + c] : (T)0;
    }
    for (int j = 0; j <= i; ++j) {
      T acc = 0;
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        const long long c = lane + 32 * u;
        acc += x[u] * (c < n ? V[(long long)j * n + c] : (T)0);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        sm.G[i][j] = (double)acc;
        sm.G[j][i] = (double)acc;
      }
    }
  }
}

// Pivoted (piv = 1) or plain Cholesky of sm.G (m x m, in T precision) by warp 0;
// pivoted: truncated at the tail-mass test with tau_b.  Fills sm.perm, sm.Lw
// (pivot order, lower), sm.bp.
template <typename T>
__device__ void chol_warp(Smem& sm, int m, double tau_b, int piv) {
  if (threadIdx.x >= 32) {
    __syncthreads();
    return;
  }
  const int j = threadIdx.x;
  bool alive = j < m;
  T dj = alive ? (T)sm.G[j][j] : (T)0;
  const T total = warp_sum<T>(alive ? dj : (T)0);
  int bp = 0;
  for (int i = 0; i < m; ++i) {
    const T msum = warp_sum<T>(alive ? dj : (T)0);
    T best = alive ? dj : (T)-1;
    int vi = alive ? j : INT_MAX;
    if (!piv) {
      best = (j == i) ? dj : (T)-1;
      vi = (j == i) ? j : INT_MAX;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
      if (ob > best || (ob == best && oi < vi)) {
        best = ob;
        vi = oi;
      }
    }
    if (piv && !(msum >= (T)tau_b * total && msum > (T)0)) break;
    if (vi == INT_MAX || !(best > (T)0)) break;
    const int p = vi;
    const T pv = sqrt(best);
    const T gjp = alive ? (T)sm.G[j][p] : (T)0;
    const T l = (j == p) ? pv : gjp / pv;
    if (alive) sm.Lw[j][i] = (double)l;
    if (j == p) alive = false;
    // rank-1 downdate of the remaining Schur complement rows
    for (int r = 0; r < m; ++r) {
      const T lr = __shfl_sync(0xffffffffu, l, r);
      if (alive) sm.G[j][r] = (double)((T)sm.G[j][r] - l * lr);
    }
    if (alive) dj = (T)sm.G[j][j];
    if (j == 0) sm.perm[i] = p;
    __syncwarp();
    bp = i + 1;
  }
  __syncwarp();
  // pivot-order factor into the G array: G[i][l] = Lw[perm[i]][l]
  for (int i = 0; i < bp; ++i)
    if (j <= i) sm.G[i][j] = sm.Lw[sm.perm[i]][j];
  if (j == 0) sm.bp = bp;
  __syncthreads();
}

// Y (bp x n) = Lc^{-1} V(perm) with Lc = sm.G (lower), one thread per column.
template <int NT, typename T>
__device__ void trsm_cols(Smem& sm, const T* V, const int* perm, T* Y, int bp, long long n) {
  for (long long c = threadIdx.x; c < n; c += NT) {
    for (int i = 0; i < bp; ++i) {
      T y = V[(perm ? perm[i] : i) * n + c];
      for (int l = 0; l < i; ++l) y -= (T)sm.G[i][l] * Y[l * n + c];
      Y[i * n + c] = y / (T)sm.G[i][i];
    }
  }
  __syncthreads();
}

// Triangle of Alg. 3 inside one chunk of columns off .. off + kk - 1 (kk <= K):
// w_j = (w_j - sum_{j < a < kk} w_a L1(off + a, off + j)) / L1(off + j, off + j),
// from the last column; L1(a, b) = L1s[a * 32 + b].  Fully unrolled, so w
// stays in registers.
template <int K, typename T>
__device__ __forceinline__ void tri_solve(T (&w)[K], int kk, const T* L1s, int off) {
#pragma unroll
  for (int j = K - 1; j >= 0; --j) {
    if (j < kk) {
      T acc = w[j];
#pragma unroll
      for (int a2 = j + 1; a2 < K; ++a2)
        if (a2 < kk) acc -= w[a2] * L1s[(off + a2) * 32 + off + j];
      w[j] = acc / L1s[(off + j) * 32 + off + j];
    }
  }
}

// wl_j -= sum_{a < kh} wh_a L1(offh + a, j) for j < K (the solved later chunk
// applied to the earlier one).
template <int K, typename T>
__device__ __forceinline__ void chunk_sub(T (&wl)[K], const T (&wh)[K], int kh, const T* L1s, int offh) {
#pragma unroll
  for (int a2 = 0; a2 < K; ++a2) {
    if (a2 < kh) {
#pragma unroll
      for (int j = 0; j < K; ++j) wl[j] -= wh[a2] * L1s[(offh + a2) * 32 + j];
    }
  }
}

// Alg. 3 for k <= 32: w L1 = L(i, :) for every row i, with L1(a, b) =
// L1s[a * 32 + b] lower triangular, solved from the last column,
// w_j = (L(i, j) - sum_{a > j} w_a L1(a, j)) / L1(j, j); one thread per row, w
// in registers (columns 16 .. k - 1 first when k > 16).  Rows of S get zeros
// here (their unit entries are set afterwards).  W is written with streaming
// stores (it is output only).
template <int NT, typename T>
__device__ void wsolve_rows(const T* L, long long m, int k, const T* L1s, const int* mark, double* Wp, long long kc) {
  for (long long i = threadIdx.x; i < m; i += NT) {
    const bool sk = mark[i] != 0;
    if (k <= 8) {
      T w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = (j < k) ? L[(long long)j * m + i] : (T)0;
      tri_solve<8, T>(w, k, L1s, 0);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j < k) __stcs(Wp + i * kc + j, sk ? 0.0 : (double)w[j]);
    } else {
      const int kh = k > 16 ? k - 16 : 0;
      T lo[16], hi[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        lo[j] = (j < k) ? L[(long long)j * m + i] : (T)0;
        hi[j] = (j < kh) ? L[(long long)(16 + j) * m + i] : (T)0;
      }
      if (kh > 0) {
        tri_solve<16, T>(hi, kh, L1s, 16);
        chunk_sub<16, T>(lo, hi, kh, L1s, 16);
      }
      tri_solve<16, T>(lo, k < 16 ? k : 16, L1s, 0);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < k) __stcs(Wp + i * kc + j, sk ? 0.0 : (double)lo[j]);
        if (j < kh) __stcs(Wp + i * kc + 16 + j, sk ? 0.0 : (double)hi[j]);
      }
    }
  }
}

// Sum over rows of a per-row value, in the fixed kSumLanes partition.
template <int NT, typename F>
__device__ double rows_sum(long long m, Smem& sm, F f) {
  double part = 0.0;
  if (threadIdx.x < kSumLanes)
    for (long long i = threadIdx.x; i < m; i += kSumLanes) part += f(i);
  return block_sum<NT>(part, sm);
}

template <int NT, typename T, int VEC>
__device__ void solve_problem(const BatchedArgs& a, int p, uint8_t* slotp, Smem& sm, T* sQp) {
  constexpr int RPW = sizeof(T) == 4 ? 4 : 2;   // rows per warp group in the row passes
  constexpr int RPW0 = sizeof(T) == 4 ? 8 : 4;  // the same for the pass over X (no basis)
  const int tid = threadIdx.x;
  const long long m = a.rows[p], n = a.cols[p];
  long long kc = m < n ? m : n;
  if (a.k_max > 0 && a.k_max < kc) kc = a.k_max;
  const Slot so = slot_layout(a.m_max, a.n_max, a.kc_max, a.b, sizeof(T));
  const long long ldr = (n + 3) / 4 * 4;  // leading dimension of R (and of Q' in shared memory on the FP32 form)
  T* R = (T*)(slotp + so.R);
  T* L = (T*)(slotp + so.L);   // column-major: L[j * m + i]
  T* Q = (T*)(slotp + so.Q);   // rows of Q^T, ld = n
  double* d = (double*)(slotp + so.d);
  int* mark = (int*)(slotp + so.mark);
  T* V = (T*)(slotp + so.V);
  T* Y = (T*)(slotp + so.Y);
  unsigned long long* K64 = (unsigned long long*)(slotp + so.K64);
  T* Wt = (T*)(slotp + so.Wt);  // column-major
  long long* skel = a.skel[p];

  // Alg. 2, start and initial norms: R = X and d_i = ||X_i||^2 in one pass over X
  if (a.x_is_fp64)
    project_rows<NT, RPW0, VEC, false, false, true, T, double, true>((const double*)a.X[p], n, nullptr, R, ldr, m, n,
                                                                (const T*)nullptr, 0, nullptr, 0, d, nullptr);
  else
    project_rows<NT, RPW0, VEC, false, false, true, T, float, true>((const float*)a.X[p], n, nullptr, R, ldr, m, n,
                                                               (const T*)nullptr, 0, nullptr, 0, d, nullptr);
  for (long long i = tid; i < m; i += NT) mark[i] = 0;
  __syncthreads();
  const double D0 = rows_sum<NT>(m, sm, [&](long long i) { return d[i]; });
  double D = D0;
  long long k = 0;
  unsigned long long t = 0;
  int status = isfinite(D0) ? RBRP_OK : RBRP_ENONFINITE;

  while (status == RBRP_OK) {
    // Alg. 2, stopping test
    if (a.tau >= 0.0 && !(D > a.tau * D0)) break;
    if (k >= kc) {
      if (a.tau >= 0.0) status = RBRP_ENOTCONVERGED;
      break;
    }
    const long long ne =
        (long long)rows_sum<NT>(m, sm, [&](long long i) { return (mark[i] == 0 && d[i] > 0.0) ? 1.0 : 0.0; });
    if (ne == 0) break;
    long long btl = (long long)a.b < ne ? (long long)a.b : ne;
    if (kc - k < btl) btl = kc - k;
    const int bt = (int)btl;
    ++t;
    // sampling step
    sample_cta<NT>(d, mark, m, bt, ne, t, a, a.pbase + (unsigned long long)p, K64, sm);
    // projection step: V = R(S_t, :) projected against Q twice (CGS2)
    project_rows<NT, RPW, VEC, true, false, false, T, T>(R, ldr, sm.St, V, n, bt, n, Q, (int)k, nullptr, 0, nullptr,
                                                    nullptr);
    __syncthreads();
    if (k > 0) {
      project_rows<NT, RPW, VEC, true, false, false, T, T>(V, n, nullptr, V, n, bt, n, Q, (int)k, nullptr, 0, nullptr,
                                                      nullptr);
      __syncthreads();
    }
    // local CPQR and truncation: G = V V^T, pivoted Cholesky with the tail-mass truncation
    gram_rows<NT, T, VEC>(V, bt, n, sm);
    __syncthreads();
    const double tau_b = a.tau_b >= 0.0 ? a.tau_b : 1.0 / (double)bt;
    chol_warp<T>(sm, bt, tau_b, 1);
    const int bp = sm.bp;
    if (bp == 0) break;
    // acceptance: Q'_V by CholQR of V(perm), a CGS pass against Q, a second CholQR
    trsm_cols<NT, T>(sm, V, sm.perm, Y, bp, n);
    for (int i = tid; i < bp; i += NT) {
      const long long row = sm.St[sm.perm[i]];
      skel[k + i] = row;
      mark[row] = (int)t;
    }
    if (k > 0)
      project_rows<NT, RPW, VEC, true, false, false, T, T>(Y, n, nullptr, Y, n, bp, n, Q, (int)k, nullptr, 0, nullptr,
                                                      nullptr);
    __syncthreads();
    gram_rows<NT, T, VEC>(Y, bp, n, sm);
    __syncthreads();
    chol_warp<T>(sm, bp, 0.0, 0);
    if (sm.bp < bp) {
      status = RBRP_ENONFINITE;
      break;
    }
    trsm_cols<NT, T>(sm, Y, nullptr, Q + k * n, bp, n);
    if constexpr (sizeof(T) == 4) {
      for (long long e = tid; e < bp * ldr; e += NT) {
        const long long r = e / ldr, c = e % ldr;
        sQp[e] = c < n ? Q[(k + r) * n + c] : (T)0;
      }
    } else {
      for (long long e = tid; e < bp * n; e += NT) sQp[e] = Q[k * n + e];
    }
    __syncthreads();
    // update step (residual form): Lhat = R Q'^T into L(:, k : k + b'), R -= Lhat Q',
    // d_i = ||R_i||^2, rows accepted so far zeroed
    if constexpr (sizeof(T) == 4)
      update_rows_oct<NT, VEC>(R, ldr, m, sQp, bp, L + k * m, m, d, mark);
    else
      project_rows<NT, RPW, VEC, true, true, true, T, T>(R, ldr, nullptr, R, ldr, m, n, sQp, bp, L + k * m, m, d, mark);
    __syncthreads();
    D = rows_sum<NT>(m, sm, [&](long long i) { return d[i]; });
    k += bp;
    if (!isfinite(D)) {
      status = RBRP_ENONFINITE;
      break;
    }
  }

  // Alg. 3: W L1 = L with L1 = L(S, :); W(S, :) = I.
  if (status != RBRP_ENONFINITE && k <= 32) {
    T* L1s = (T*)&sm.Lw[0][0];  // L1 as a 32 x 32 array of T
    for (long long e = tid; e < k * k; e += NT) {
      const long long a2 = e / k, b2 = e % k;
      L1s[a2 * 32 + b2] = L[b2 * m + skel[a2]];
    }
    __syncthreads();
    double* Wp = a.W[p];
    wsolve_rows<NT, T>(L, m, (int)k, L1s, mark, Wp, kc);
    __syncthreads();
    for (long long j = tid; j < k; j += NT) Wp[skel[j] * kc + j] = 1.0;
  } else if (status != RBRP_ENONFINITE) {
    // k > 32: row i of W by back substitution over the columns from the last,
    // one thread per row, through a column-major scratch copy of L
    for (long long e = tid; e < k * m; e += NT) Wt[e] = L[e];
    __syncthreads();
    for (long long i = tid; i < m; i += NT) {
      for (long long jj = k - 1; jj >= 0; --jj) {
        const long long sj = skel[jj];
        const T wj = Wt[jj * m + i] / L[jj * m + sj];
        Wt[jj * m + i] = wj;
        for (long long l = 0; l < jj; ++l) Wt[l * m + i] -= wj * L[l * m + sj];
      }
    }
    __syncthreads();
    double* Wp = a.W[p];
    for (long long e = tid; e < m * k; e += NT) {
      const long long i = e / k, j = e % k;
      Wp[i * kc + j] = mark[i] ? 0.0 : (double)Wt[j * m + i];
    }
    __syncthreads();
    for (long long j = tid; j < k; j += NT) Wp[skel[j] * kc + j] = 1.0;
  }
  if (tid == 0) {
    a.k_out[p] = k;
    a.err[p] = D0 > 0.0 ? D / D0 : 0.0;
    a.status[p] = status;
  }
  __syncthreads();
}

template <int NT, typename T, int VEC>
__global__ void __launch_bounds__(NT, kBatchMaxThreads / NT) k_batched(BatchedArgs a) {
  extern __shared__ __align__(16) uint8_t dyn[];
  Smem& sm = *(Smem*)dyn;
  T* sQp = (T*)(dyn + (sizeof(Smem) + 15) / 16 * 16);  // Q' (b' x n)
  __shared__ int s_p;
  uint8_t* slotp = a.slots + (size_t)blockIdx.x * a.slot_bytes;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int q = atomicAdd(a.next, 1u);
      s_p = (q < (unsigned int)a.P) ? a.order[q] : -1;
    }
    __syncthreads();
    const int p = s_p;
    __syncthreads();
    if (p < 0) break;
    solve_problem<NT, T, VEC>(a, p, slotp, sm, sQp);
  }
}

// The kernel for a schedule: CTA size, precision, and the row width of the row
// passes (values a lane holds: 8 for n <= 256, 4 for n <= 128).
const void* pick(int threads, int fp64, int vec) {
  if (vec == 8) {
    if (threads == 256) return fp64 ? (const void*)k_batched<256, double, 8> : (const void*)k_batched<256, float, 8>;
    if (threads == 512) return fp64 ? (const void*)k_batched<512, double, 8> : (const void*)k_batched<512, float, 8>;
  } else if (vec == 4) {
    if (threads == 256) return fp64 ? (const void*)k_batched<256, double, 4> : (const void*)k_batched<256, float, 4>;
    if (threads == 512) return fp64 ? (const void*)k_batched<512, double, 4> : (const void*)k_batched<512, float, 4>;
  }
  return nullptr;
}

}  // namespace bt

// ---------------------------------------------------------------------------- host

size_t batched_slot_bytes(long long m_max, long long n_max, long long kc_max, int b, int fp64) {
  return bt::slot_layout(m_max, n_max, kc_max, b, fp64 ? 8 : 4).total;
}

int batched_sms() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

size_t batched_dyn_smem(long long n_max, int fp64) {
  return (sizeof(bt::Smem) + 15) / 16 * 16 + (size_t)kBatchMaxBlock * ((n_max + 3) / 4 * 4) * (fp64 ? 8 : 4);
}

cudaError_t batched_configure(int threads, int fp64, long long n_max, int vec, int* per_sm) {
  *per_sm = 0;
  const void* f = bt::pick(threads, fp64, vec);
  if (!f) return cudaErrorInvalidValue;
  if (n_max > 32LL * vec) return cudaSuccess;  // a row does not fit the row width: 0 CTAs
  // the kernel's limit is a property of the function, shared by every bucket that
  // launches it: set it for the widest rows the row width admits
  const long long n_cap = std::min<long long>(kBatchMaxCols, 32LL * vec);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)batched_dyn_smem(n_cap, fp64));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, f, threads, batched_dyn_smem(n_max, fp64));
}

cudaError_t launch_batched(const BatchedArgs& a, int threads, int vec, int ctas, cudaStream_t s) {
  const void* f = bt::pick(threads, a.fp64, vec);
  if (!f || ctas < 1 || a.n_max > 32LL * vec) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.next, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const size_t dyn = batched_dyn_smem(a.n_max, a.fp64);
  BatchedArgs arg = a;
  void* params[] = {&arg};
  e = cudaLaunchKernel(f, dim3((unsigned)ctas), dim3((unsigned)threads), params, dyn, s);
  return counted(e);
}

}  // namespace rbrp
