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
// T is the storage and arithmetic type (float or double).  Sampling keys are
// exact FP64 keys of Alg. 2 line 5 as in the single-problem sampler: FP32
// log-domain keys choose >= b_t + 32 candidates, their FP64 keys are ranked,
// and a margin check against the FP32 error bound proves that no other row
// could be drawn (else every eligible row is keyed in FP64).  Problem p uses
// Philox problem id pbase + p.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "rbrp_internal.cuh"
#include "sample_common.cuh"

namespace rbrp {
namespace bt {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCand = 1024;  // candidates the sampler ranks exactly

struct Args {
  int P;
  const void* const* X;      // device array: problem p is m_p x n_p, row-major, ld = n_p
  const long long* rows;     // m_p
  const long long* cols;     // n_p
  const int* order;          // processing order
  long long* const* skel;    // device array: k_cap_p entries each
  double* const* W;          // device array: m_p x k_cap_p FP64 each, ld = k_cap_p
  long long* k_out;          // P
  double* err;               // P: ||d||_1 / ||d0||_1
  int* status;               // P: rbrp_status
  double tau, tau_b;
  int b, greedy, x_is_fp64;
  long long k_max;
  unsigned long long seed;
  unsigned long long pbase;  // Philox problem id of problem 0
  uint8_t* slots;            // per-CTA workspace slots
  size_t slot_bytes;
  long long m_max, n_max, kc_max;
  unsigned int* next;        // work counter, zero before the launch
};

// Offsets of one slot (bytes), for the batch maxima.
struct Slot {
  size_t R, L, Q, d, mark, V, Y, C, K64, Wt, total;
};
__host__ __device__ inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline Slot slot_layout(long long m, long long n, long long kc, int b, size_t sT) {
  Slot s;
  size_t o = 0;
  s.R = o;
  o = al256(o + (size_t)m * n * sT);
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
  s.C = o;
  o = al256(o + (size_t)b * kc * sT);
  s.K64 = o;  // fallback sampler keys
  o = al256(o + (size_t)m * 8);
  s.Wt = o;   // W solve scratch, column-major
  o = al256(o + (size_t)m * kc * sT);
  s.total = o;
  return s;
}

struct Smem {
  unsigned int keys[4096];
  unsigned int hist[kBins];
  unsigned long long ek[kCand];
  int cand[kCand];
  int St[32];
  int perm[32];
  double G[32][33];   // Gram / Schur complement
  double Lw[32][33];  // factor, candidate-indexed then pivot-indexed
  double red[kWarps];
  unsigned int cnt;
  int bin, bp;
  unsigned int below, total;
  int flag;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread in a fixed order; every thread gets the result.
__device__ double block_sum(double v, Smem& sm) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) s += sm.red[q];
  return s;
}

// First bin of sm.hist where the running count reaches want (kBins if never),
// with the count below it; every thread gets both.
__device__ int find_bin_cta(Smem& sm, unsigned int want, unsigned int* below) {
  constexpr int per = kBins / kThreads;
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
  for (int q = 0; q < kWarps; ++q) {
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

// Exact FP64 key of row i (as ordered bits) and its logarithm (Alg. 2 line 5).
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

// S_t (bt rows, in draw order) into sm.St.  ne = number of eligible rows.
__device__ void sample_cta(const double* d, const int* mark, long long m, int bt, long long ne, unsigned long long t,
                           const Args& a, unsigned long long p, unsigned long long* K64, Smem& sm) {
  const int tid = threadIdx.x;
  for (long long i = tid; i < m; i += kThreads) {
    const bool elig = mark[i] == 0 && d[i] > 0.0;
    sm.keys[i] = elig ? approx_key(d[i], i, t, a.seed, p, a.greedy) : 0xFFFFFFFFu;
  }
  const unsigned int want = (unsigned int)(bt + kMargin < ne ? bt + kMargin : ne);
  for (int j = tid; j < kBins; j += kThreads) sm.hist[j] = 0;
  __syncthreads();
  for (long long i = tid; i < m; i += kThreads)
    if (sm.keys[i] != 0xFFFFFFFFu) atomicAdd(&sm.hist[sm.keys[i] >> 21], 1u);
  __syncthreads();
  unsigned int below1 = 0, below2 = 0;
  const int b1 = find_bin_cta(sm, want, &below1);
  for (int j = tid; j < kBins; j += kThreads) sm.hist[j] = 0;
  __syncthreads();
  for (long long i = tid; i < m; i += kThreads) {
    const unsigned int k = sm.keys[i];
    if (k != 0xFFFFFFFFu && (int)(k >> 21) == b1) atomicAdd(&sm.hist[(k >> 10) & 0x7FF], 1u);
  }
  __syncthreads();
  int b2 = find_bin_cta(sm, want - below1, &below2);
  if (b2 >= kBins) b2 = kBins - 1;
  const unsigned int c22 = ((unsigned int)b1 << 11) | (unsigned int)b2;
  if (tid == 0) sm.cnt = 0;
  __syncthreads();
  for (long long i = tid; i < m; i += kThreads) {
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
  for (int e = tid; e < mc; e += kThreads) {
    double lg;
    exact_key(d[sm.cand[e]], sm.cand[e], t, a.seed, p, a.greedy, &sm.ek[e], &lg);
  }
  __syncthreads();
  for (int e = tid; e < mc; e += kThreads) {
    int rank = 0;
    const unsigned long long ke = sm.ek[e];
    const int ie = sm.cand[e];
    for (int f = 0; f < mc; ++f) rank += (sm.ek[f] < ke || (sm.ek[f] == ke && sm.cand[f] < ie)) ? 1 : 0;
    if (rank < bt) sm.St[rank] = ie;
  }
  __syncthreads();
  if (tid == 0) {
    bool exact = !overflow && mc >= bt;
    if (exact && (long long)mc < ne) {
      // every row outside the cut has an FP32 key >= the smallest key above the cut;
      // the bt-th exact key must lie below that by more than the FP32 error bound
      double lg;
      unsigned long long kk;
      exact_key(d[sm.St[bt - 1]], sm.St[bt - 1], t, a.seed, p, a.greedy, &kk, &lg);
      const float outside = key_to_float(((c22 + 1u) << 10));
      exact = lg < (double)outside - (double)kCutGuard - 1e-6 * fabs((double)outside);
    }
    sm.flag = exact ? 0 : 1;
  }
  __syncthreads();
  if (!sm.flag) return;
  // fallback: FP64 keys of every eligible row, ranked by counting
  for (long long i = tid; i < m; i += kThreads) {
    unsigned long long k = kIneligible;
    if (mark[i] == 0 && d[i] > 0.0) {
      double lg;
      exact_key(d[i], i, t, a.seed, p, a.greedy, &k, &lg);
    }
    K64[i] = k;
  }
  __syncthreads();
  for (long long i = tid; i < m; i += kThreads) {
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

// Dot products of rows of A (ra rows) with rows of B (rb rows), length n, into
// Cm (ra x ldc); one warp per pair.
template <typename T>
__device__ void rows_dot(const T* A, const T* B, int ra, int rb, long long n, T* Cm, long long ldc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int pr = w; pr < ra * rb; pr += kWarps) {
    const int i = pr / rb, j = pr % rb;
    T s = 0;
    for (long long c = lane; c < n; c += 32) s += A[i * n + c] * B[j * n + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) Cm[i * ldc + j] = s;
  }
}

// V (rows x n) <- V - (V Q^T) Q over the first k rows of Q (CGS).
template <typename T>
__device__ void cgs(T* V, int rows, const T* Q, long long k, long long n, T* C, long long ldc) {
  if (k <= 0) return;
  rows_dot<T>(V, Q, rows, (int)k, n, C, ldc);
  __syncthreads();
  for (long long e = threadIdx.x; e < rows * n; e += kThreads) {
    const long long i = e / n, c = e % n;
    T s = 0;
    for (long long j = 0; j < k; ++j) s += C[i * ldc + j] * Q[j * n + c];
    V[e] -= s;
  }
  __syncthreads();
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
  const T total = (T)warp_sum(alive ? (double)dj : 0.0);
  int bp = 0;
  for (int i = 0; i < m; ++i) {
    const T msum = (T)warp_sum(alive ? (double)dj : 0.0);
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
template <typename T>
__device__ void trsm_cols(Smem& sm, const T* V, const int* perm, T* Y, int bp, long long n) {
  for (long long c = threadIdx.x; c < n; c += kThreads) {
    for (int i = 0; i < bp; ++i) {
      T y = V[(perm ? perm[i] : i) * n + c];
      for (int l = 0; l < i; ++l) y -= (T)sm.G[i][l] * Y[l * n + c];
      Y[i * n + c] = y / (T)sm.G[i][i];
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void solve_problem(const Args& a, int p, uint8_t* slotp, Smem& sm, T* sQp) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long m = a.rows[p], n = a.cols[p];
  long long kc = m < n ? m : n;
  if (a.k_max > 0 && a.k_max < kc) kc = a.k_max;
  const Slot so = slot_layout(a.m_max, a.n_max, a.kc_max, a.b, sizeof(T));
  T* R = (T*)(slotp + so.R);
  T* L = (T*)(slotp + so.L);   // column-major: L[j * m + i]
  T* Q = (T*)(slotp + so.Q);   // rows of Q^T, ld = n
  double* d = (double*)(slotp + so.d);
  int* mark = (int*)(slotp + so.mark);
  T* V = (T*)(slotp + so.V);
  T* Y = (T*)(slotp + so.Y);
  T* C = (T*)(slotp + so.C);
  unsigned long long* K64 = (unsigned long long*)(slotp + so.K64);
  T* Wt = (T*)(slotp + so.Wt);  // column-major
  long long* skel = a.skel[p];

  // Alg. 2 lines 1-2
  for (long long e = tid; e < m * n; e += kThreads)
    R[e] = a.x_is_fp64 ? (T)((const double*)a.X[p])[e] : (T)((const float*)a.X[p])[e];
  __syncthreads();
  for (long long i = w; i < m; i += kWarps) {
    T sl = 0;  // per lane in T (FP64 arithmetic costs ~64 cycles per warp instruction on GB300)
    for (long long c = lane; c < n; c += 32) {
      const T x = R[i * n + c];
      sl += x * x;
    }
    const double s = warp_sum((double)sl);
    if (lane == 0) {
      d[i] = s;
      mark[i] = 0;
    }
  }
  __syncthreads();
  double part = 0.0;
  for (long long i = tid; i < m; i += kThreads) part += d[i];
  const double D0 = block_sum(part, sm);
  double D = D0;
  long long k = 0;
  unsigned long long t = 0;
  int status = isfinite(D0) ? RBRP_OK : RBRP_ENONFINITE;

  while (status == RBRP_OK) {
    // Alg. 2 line 3
    if (a.tau >= 0.0 && !(D > a.tau * D0)) break;
    if (k >= kc) {
      if (a.tau >= 0.0) status = RBRP_ENOTCONVERGED;
      break;
    }
    double ecount = 0.0;
    for (long long i = tid; i < m; i += kThreads) ecount += (mark[i] == 0 && d[i] > 0.0) ? 1.0 : 0.0;
    const long long ne = (long long)block_sum(ecount, sm);
    if (ne == 0) break;
    long long btl = (long long)a.b < ne ? (long long)a.b : ne;
    if (kc - k < btl) btl = kc - k;
    const int bt = (int)btl;
    ++t;
    // line 5
    sample_cta(d, mark, m, bt, ne, t, a, a.pbase + (unsigned long long)p, K64, sm);
    // line 6: V = R(S_t, :), CGS2
    for (long long e = tid; e < bt * n; e += kThreads) V[e] = R[(long long)sm.St[e / n] * n + e % n];
    __syncthreads();
    cgs<T>(V, bt, Q, k, n, C, kc);
    cgs<T>(V, bt, Q, k, n, C, kc);
    // lines 7-8: G = V V^T, pivoted Cholesky with the tail-mass truncation
    {
      T* Gt = Y;  // bt x bt scratch
      rows_dot<T>(V, V, bt, bt, n, Gt, bt);
      __syncthreads();
      for (int e = tid; e < bt * bt; e += kThreads) sm.G[e / bt][e % bt] = (double)Gt[e];
      __syncthreads();
    }
    const double tau_b = a.tau_b >= 0.0 ? a.tau_b : 1.0 / (double)bt;
    chol_warp<T>(sm, bt, tau_b, 1);
    const int bp = sm.bp;
    if (bp == 0) break;
    // lines 9-10, 13: Q'_V by CholQR of V(perm), a CGS pass against Q, a second CholQR
    trsm_cols<T>(sm, V, sm.perm, Y, bp, n);
    for (int i = tid; i < bp; i += kThreads) {
      const long long row = sm.St[sm.perm[i]];
      skel[k + i] = row;
      mark[row] = (int)t;
    }
    cgs<T>(Y, bp, Q, k, n, C, kc);
    {
      T* Gt = V;
      rows_dot<T>(Y, Y, bp, bp, n, Gt, bp);
      __syncthreads();
      for (int e = tid; e < bp * bp; e += kThreads) sm.G[e / bp][e % bp] = (double)Gt[e];
      __syncthreads();
    }
    chol_warp<T>(sm, bp, 0.0, 0);
    if (sm.bp < bp) {
      status = RBRP_ENONFINITE;
      break;
    }
    trsm_cols<T>(sm, Y, nullptr, Q + k * n, bp, n);
    for (long long e = tid; e < bp * n; e += kThreads) sQp[e] = Q[k * n + e];
    __syncthreads();
    // lines 12, 16 (residual form): Lhat = R Q'^T, R -= Lhat Q', d_i = ||R_i||^2; accepted rows zeroed
    for (long long i = w; i < m; i += kWarps) {
      T x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long c = lane + 32 * u;
        x[u] = c < n ? R[i * n + c] : (T)0;
      }
      const bool acc = mark[i] != 0;
      T lh[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j >= bp) break;
        T s = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const long long c = lane + 32 * u;
          if (c < n) s += x[u] * sQp[j * n + c];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        lh[j] = s;
      }
      if (lane < bp) {
        T mine = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j == lane) mine = lh[j];
        L[(k + lane) * m + i] = mine;
      }
      T nr = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long c = lane + 32 * u;
        if (c >= n) continue;
        T v = x[u];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j >= bp) break;
          v -= lh[j] * sQp[j * n + c];
        }
        if (acc) v = (T)0;
        R[i * n + c] = v;
        nr += v * v;
      }
      const double nrd = warp_sum((double)nr);
      if (lane == 0) d[i] = acc ? 0.0 : nrd;
    }
    __syncthreads();
    double dp = 0.0;
    for (long long i = tid; i < m; i += kThreads) dp += d[i];
    D = block_sum(dp, sm);
    k += bp;
    if (!isfinite(D)) {
      status = RBRP_ENONFINITE;
      break;
    }
  }

  // Alg. 3: W L1 = L with L1 = L(S, :); W(S, :) = I.  Row i of W by back
  // substitution over the columns from the last, one thread per row.
  if (status != RBRP_ENONFINITE) {
    for (long long e = tid; e < k * m; e += kThreads) Wt[e] = L[e];
    __syncthreads();
    for (long long i = tid; i < m; i += kThreads) {
      for (long long jj = k - 1; jj >= 0; --jj) {
        const long long sj = skel[jj];
        const T wj = Wt[jj * m + i] / L[jj * m + sj];
        Wt[jj * m + i] = wj;
        for (long long l = 0; l < jj; ++l) Wt[l * m + i] -= wj * L[l * m + sj];
      }
    }
    __syncthreads();
    double* Wp = a.W[p];
    for (long long e = tid; e < m * k; e += kThreads) {
      const long long i = e / k, j = e % k;
      Wp[i * kc + j] = mark[i] ? 0.0 : (double)Wt[j * m + i];
    }
    __syncthreads();
    for (long long j = tid; j < k; j += kThreads) Wp[skel[j] * kc + j] = 1.0;
  }
  if (tid == 0) {
    a.k_out[p] = k;
    a.err[p] = D0 > 0.0 ? D / D0 : 0.0;
    a.status[p] = status;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_batched(Args a) {
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
    solve_problem<T>(a, p, slotp, sm, sQp);
  }
}

}  // namespace bt

// ---------------------------------------------------------------------------- host

size_t batched_slot_bytes(long long m_max, long long n_max, long long kc_max, int b, int fp64) {
  return bt::slot_layout(m_max, n_max, kc_max, b, fp64 ? 8 : 4).total;
}

int batched_ctas() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t launch_batched(int P, const void* const* X_dev, const long long* rows_dev, const long long* cols_dev,
                           const int* order_dev, long long* const* skel_dev, double* const* W_dev, long long* k_out,
                           double* err, int* status, double tau, double tau_b, int b, int greedy, int x_is_fp64,
                           long long k_max, unsigned long long seed, unsigned long long pbase, int fp64, void* slots, size_t slot_bytes,
                           long long m_max, long long n_max, long long kc_max, unsigned int* next, int ctas,
                           cudaStream_t s) {
  bt::Args a;
  a.P = P;
  a.X = X_dev;
  a.rows = rows_dev;
  a.cols = cols_dev;
  a.order = order_dev;
  a.skel = skel_dev;
  a.W = W_dev;
  a.k_out = k_out;
  a.err = err;
  a.status = status;
  a.tau = tau;
  a.tau_b = tau_b;
  a.b = b;
  a.greedy = greedy;
  a.x_is_fp64 = x_is_fp64;
  a.k_max = k_max;
  a.seed = seed;
  a.pbase = pbase;
  a.slots = (uint8_t*)slots;
  a.slot_bytes = slot_bytes;
  a.m_max = m_max;
  a.n_max = n_max;
  a.kc_max = kc_max;
  a.next = next;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  const size_t dyn = (sizeof(bt::Smem) + 15) / 16 * 16 + (size_t)32 * n_max * (fp64 ? 8 : 4);
  if (fp64) {
    e = cudaFuncSetAttribute(bt::k_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    bt::k_batched<double><<<ctas, bt::kThreads, dyn, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(bt::k_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    bt::k_batched<float><<<ctas, bt::kThreads, dyn, s>>>(a);
  }
  return counted(cudaGetLastError());
}

}  // namespace rbrp
