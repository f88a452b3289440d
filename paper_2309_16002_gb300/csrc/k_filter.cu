// The robust blockwise filter and the new basis Q' of one RBRP block.
//
// Alg. 2's local CPQR, truncation and acceptance with the robust blockwise filtering remark (Sec. 4): the
// candidates V (b_t rows) are pivoted like a column-pivoted QR of V^T and the
// factorisation is truncated at the first step i where the trailing mass
// ||R_V(i:, i:)||_F^2 drops below tau_b ||R_V||_F^2.  On the GPU this is the
// pivoted Cholesky factorisation of the FP64 Gram matrix G = V V^T: the same
// pivots and the same trailing masses in exact arithmetic (the Schur-complement
// diagonal is each remaining candidate's residual norm^2 and its sum is the
// trailing mass).  Q'_V then comes from V_perm = Lc Y by forward substitution
// (CholQR), which keeps Y_i in the span of the first i pivots and therefore
// L1 lower triangular (Sec. 5.1).
//
// GB300 retires about two FP64 FMAs per clock per SM, spread over its four
// sub-partitions, so the b x b factorisation keeps the Schur complement in
// registers of 256 threads (eight warps) and spends its per-step budget on
// three barriers and independent register FMAs.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "rbrp_internal.cuh"

namespace rbrp {

constexpr int kRegCholThreads = 256;
constexpr int kRegCholMax = 128;

// Packed lower-triangle index e -> (r, c), r >= c, row-major (e = r (r + 1) / 2 + c).
__device__ __forceinline__ void tri_rc(int e, int& r, int& c) {
  int rr = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
  while ((rr + 1) * (rr + 2) / 2 <= e) ++rr;
  while (rr * (rr + 1) / 2 > e) --rr;
  r = rr;
  c = e - rr * (rr + 1) / 2;
}

// Right-looking pivoted (or plain) Cholesky with the lower triangle of the
// Schur complement in registers: thread t owns packed elements t, t + 256, ...
// Candidates keep their original index; `alive` marks the unpivoted ones.
template <int SLOTS>
__global__ void __launch_bounds__(kRegCholThreads) k_pchol_reg(const double* __restrict__ G, long long ldg,
                                                               double* __restrict__ Lc, long long ldl,
                                                               double* __restrict__ Lw, int* __restrict__ perm,
                                                               const long long* __restrict__ S_t,
                                                               long long* __restrict__ skel, int* __restrict__ mark,
                                                               State* st, int pivoted, long long mark_base,
                                                               long long mark_n) {
  if (st->done) return;
  __shared__ double diag[kRegCholMax];
  __shared__ double lcol[kRegCholMax];
  __shared__ int alive[kRegCholMax];
  __shared__ int s_perm[kRegCholMax];
  __shared__ int s_piv, s_stop;
  __shared__ double s_pv, s_rinv;
  const int m = pivoted ? (int)st->b_t : (int)st->bp;
  const int tid = threadIdx.x;
  const int ne = m * (m + 1) / 2;
  double a[SLOTS];
  short rr[SLOTS], cc[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int e = tid + kRegCholThreads * s;
    int r = -1, c = -1;
    double v = 0.0;
    if (e < ne) {
      tri_rc(e, r, c);
      v = G[(long long)r * ldg + c];
      if (r == c) diag[r] = v;
    }
    a[s] = v;
    rr[s] = (short)r;
    cc[s] = (short)c;
  }
  for (int j = tid; j < m; j += kRegCholThreads) alive[j] = 1;
  __syncthreads();
  double total = 0.0;
  if (tid < 32) {
    for (int j = tid; j < m; j += 32) total += diag[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  }
  double tau_b = st->tau_b;
  if (tau_b < 0.0) tau_b = (m > 0) ? 1.0 / (double)m : 1.0;
  int bp = 0;
  for (int i = 0; i < m; ++i) {
    // (a) trailing mass and pivot (largest residual norm^2, ties to the smaller candidate index).
    // The comparison runs on order-preserving integer keys (FP64 compares and
    // shuffles sit on GB300's slow FP64 path); only the mass is summed in FP64.
    if (tid < 32) {
      double msum = 0.0;
      unsigned long long key = 0ULL;  // below every orderable double
      int vi = INT_MAX;
      for (int j = tid; j < m; j += 32) {
        if (!alive[j]) continue;
        const double dj = diag[j];
        msum += dj;
        const unsigned long long kj = (pivoted == 1) ? orderable(dj) : (j == i ? ~0ULL : 0ULL);
        if (kj > key || (kj == key && j < vi)) {
          key = kj;
          vi = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        msum += __shfl_xor_sync(0xffffffffu, msum, o);
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
        const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
        if (ok > key || (ok == key && oi < vi)) {
          key = ok;
          vi = oi;
        }
      }
      if (tid == 0) {
        const double v = (vi == INT_MAX) ? 0.0 : diag[vi];
        int stop = 0;
        if (pivoted == 1 && !(msum >= tau_b * total && msum > 0.0)) stop = 1;
        if (vi == INT_MAX || !(v > 0.0)) stop = 1;
        s_stop = stop;
        s_piv = vi;
        if (!stop) {
          const double r = rsqrt(v);  // one FP64 reciprocal square root per step
          s_rinv = r;
          s_pv = v * r;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_piv;
    const double rinv = s_rinv;
    // (b) column p of the factor: owners of row/column p publish l_j = S(j, p) / sqrt(S(p, p))
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int r = rr[s], c = cc[s];
      if (r < 0) continue;
      int j = -1;
      if (c == p && r != p) j = r;
      else if (r == p && c != p) j = c;
      if (j >= 0 && alive[j]) {
        const double l = a[s] * rinv;
        lcol[j] = l;
        Lw[(long long)j * kMaxBlock + i] = l;
      }
    }
    if (tid == 0) {
      Lw[(long long)p * kMaxBlock + i] = s_pv;
      alive[p] = 0;
      s_perm[i] = p;
      if (perm) perm[i] = p;
    }
    __syncthreads();
    // (c) rank-1 downdate of the remaining lower triangle
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      const int r = rr[s], c = cc[s];
      if (r < 0 || !alive[r] || !alive[c]) continue;
      a[s] -= lcol[r] * lcol[c];
      if (r == c) diag[r] = a[s];
    }
    __syncthreads();
    bp = i + 1;
  }
  for (int e = tid; e < bp * bp; e += kRegCholThreads) {
    const int i = e / bp, l = e % bp;
    Lc[(long long)i * ldl + l] = (l <= i) ? Lw[(long long)s_perm[i] * kMaxBlock + l] : 0.0;
  }
  if (pivoted) {
    const long long k = st->k;
    const int tno = (int)(st->t + 1);
    for (int i = tid; i < bp; i += kRegCholThreads) {
      const long long row = S_t[s_perm[i]];
      skel[k + i] = row;
      if (row - mark_base >= 0 && row - mark_base < mark_n) mark[row - mark_base] = tno;  // rows of this shard
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (pivoted) {
      st->bp = bp;
      st->bp_pad = (bp + 15) / 16 * 16;
      if (bp == 0) st->done = 1;
    } else if (bp < m) {
      st->status = RBRP_ENONFINITE;  // the Gram matrix of Q' lost positive definiteness
      st->done = 1;
    }
  }
}

// Left-looking form for m > 128 candidates (FP64 / FP32 paths with b up to 256):
// the factor is kept candidate-indexed in global memory.
__global__ void __launch_bounds__(256) k_pchol_global(const double* __restrict__ G, long long ldg,
                                               double* __restrict__ Lc, long long ldl, double* __restrict__ Lw,
                                               int* __restrict__ perm, const long long* __restrict__ S_t,
                                               long long* __restrict__ skel, int* __restrict__ mark, State* st,
                                               int pivoted, long long mark_base, long long mark_n) {
  if (st->done) return;
  __shared__ double diag[kMaxBlock];
  __shared__ int alive[kMaxBlock];
  __shared__ int s_piv;
  __shared__ double s_total, s_pv;
  __shared__ int s_stop;
  __shared__ int s_perm[kMaxBlock];
  const int m = pivoted ? (int)st->b_t : (int)st->bp;
  const int tid = threadIdx.x;
  for (int j = tid; j < m; j += blockDim.x) {
    diag[j] = G[(long long)j * ldg + j];
    alive[j] = 1;
  }
  __syncthreads();
  // total = ||V||_F^2 (fixed-order sum)
  if (tid < 32) {
    double s = 0.0;
    for (int j = tid; j < m; j += 32) s += diag[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) s_total = s;
  }
  __syncthreads();
  double tau_b = st->tau_b;
  if (tau_b < 0.0) tau_b = (m > 0) ? 1.0 / (double)m : 1.0;
  int bp = 0;
  for (int i = 0; i < m; ++i) {
    // trailing mass and argmax (ties to the smallest candidate position)
    double v = -DBL_MAX;
    int vi = INT_MAX;
    double msum = 0.0;
    if (tid < 32) {
      for (int j = tid; j < m; j += 32) {
        if (!alive[j]) continue;
        msum += diag[j];
        const bool better = (pivoted == 1) ? (diag[j] > v || (diag[j] == v && j < vi)) : (j == i);
        if (better) { v = diag[j]; vi = j; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        msum += __shfl_xor_sync(0xffffffffu, msum, o);
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
        if (ov > v || (ov == v && oi < vi)) { v = ov; vi = oi; }
      }
      if (tid == 0) {
        s_piv = vi;
        s_pv = v;
        int stop = 0;
        if (pivoted == 1 && !(msum >= tau_b * s_total && msum > 0.0)) stop = 1;
        if (vi == INT_MAX || !(v > 0.0)) stop = 1;
        s_stop = stop;
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_piv;
    const double pivval = sqrt(s_pv), rinv = 1.0 / pivval;
    // column i of the factor for every remaining candidate j (Lw is candidate-indexed)
    for (int j = tid; j < m; j += blockDim.x) {
      if (!alive[j]) continue;
      if (j == p) {
        Lw[(long long)j * kMaxBlock + i] = pivval;
        continue;
      }
      double sacc = G[(long long)j * ldg + p];
      for (int l = 0; l < i; ++l) sacc -= Lw[(long long)j * kMaxBlock + l] * Lw[(long long)p * kMaxBlock + l];
      const double lji = sacc * rinv;
      Lw[(long long)j * kMaxBlock + i] = lji;
      diag[j] -= lji * lji;
    }
    __syncthreads();
    if (tid == 0) {
      alive[p] = 0;
      s_perm[i] = p;
      if (perm) perm[i] = p;
    }
    __syncthreads();
    bp = i + 1;
  }
  __syncthreads();
  // pivot-order factor Lc (bp x bp, lower triangular)
  for (int e = tid; e < bp * bp; e += blockDim.x) {
    const int i = e / bp, l = e % bp;
    Lc[(long long)i * ldl + l] = (l <= i) ? Lw[(long long)s_perm[i] * kMaxBlock + l] : 0.0;
  }
  if (pivoted) {
    const long long k = st->k;
    const int tno = (int)(st->t + 1);
    for (int i = tid; i < bp; i += blockDim.x) {
      const long long row = S_t[s_perm[i]];
      skel[k + i] = row;
      if (row - mark_base >= 0 && row - mark_base < mark_n) mark[row - mark_base] = tno;  // rows of this shard
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (pivoted) {
      st->bp = bp;
      st->bp_pad = (bp + 15) / 16 * 16;
      if (bp == 0) st->done = 1;
    } else if (bp < m) {
      st->status = RBRP_ENONFINITE;  // Gram of Q' lost positive definiteness
      st->done = 1;
    }
  }
}


// FP32 form of the filter for the plain TF32 path, whose residual already
// carries TF32 rounding (~2^-11 relative), far coarser than FP32: the same
// pivoting, truncation and outputs as k_pchol_reg, followed in the same CTA by
// Linv = Lc^{-1} (bp x bp, lower triangular), so that Q'_V = Linv V_perm is one
// product instead of a serial substitution.
//
// The factorisation is left-looking: at step i the new factor column for
// every remaining candidate j is (G(j, p) - sum_{t<i} L(j, t) L(p, t)) /
// sqrt(d_p), and the residual norms d_j drop by its square.  Thread j owns
// candidate j (its factor row in shared memory, its d_j in a register); a step
// is a warp-shuffle argmax, one block barrier to combine the four warps, and a
// short dot product with four independent accumulators.  Then the same
// threads form the inverse, four lanes per column.
constexpr int kPcholF32Threads = 128;

__global__ void __launch_bounds__(kPcholF32Threads) k_pchol_f32(const float* __restrict__ G, long long ldg,
                                                                float* __restrict__ Linv, long long ldl,
                                                                int* __restrict__ perm,
                                                                const long long* __restrict__ S_t,
                                                                long long* __restrict__ skel, int* __restrict__ mark,
                                                                State* st, int mmax) {
  if (st->done) return;
  extern __shared__ __align__(16) float fsm[];
  const int LDF = (mmax + 4) & ~3;  // factor rows: float4 steps over t
  const int LDG = mmax + 1;         // G rows: odd stride, conflict-free column reads
  float* Lw = fsm;                  // Lw[j * LDF + t]: factor entry of candidate j at step t
  float* Gs = fsm + mmax * LDF;     // G, later the pivot-order factor Ls (stride LDF)
  float* Ls = Gs;
  float* X = Lw;                    // the inverse, once Ls is built
  __shared__ float rdg[kRegCholMax];
  __shared__ int s_perm[kRegCholMax];
  __shared__ float s_ms[2][4], s_bv[2][4];
  __shared__ int s_bi[2][4];
  __shared__ float s_tot[4];
  const int m = (int)st->b_t;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // thread c stages column c; sixteen loads in flight per thread
  for (int r0 = 0; r0 < m; r0 += 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = (r0 + u < m && tid < m) ? G[(long long)(r0 + u) * ldg + tid] : 0.f;
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (r0 + u < m && tid < m) Gs[(r0 + u) * LDG + tid] = v[u];
  }
  for (int e = tid; e < m * LDF; e += kPcholF32Threads) Lw[e] = 0.f;
  __syncthreads();
  double tau_b = st->tau_b;
  if (tau_b < 0.0) tau_b = (m > 0) ? 1.0 / (double)m : 1.0;
  const float tb = (float)tau_b;
  const int j = tid;
  bool alive = j < m;
  float dj = alive ? Gs[j * LDG + j] : 0.f;
  {
    float t = dj;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_tot[warp] = t;
  }
  __syncthreads();
  const float total = (s_tot[0] + s_tot[1]) + (s_tot[2] + s_tot[3]);
  const float* lj = Lw + j * LDF;
  int bp = 0;
  for (int i = 0; i < m; ++i) {
    // trailing mass and pivot (largest residual norm^2, ties to the smaller index)
    float msum = alive ? dj : 0.f, best = alive ? dj : -1.f;
    int vi = alive ? j : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      msum += __shfl_xor_sync(0xffffffffu, msum, o);
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
      if (ob > best || (ob == best && oi < vi)) {
        best = ob;
        vi = oi;
      }
    }
    const int sl = i & 1;
    if (lane == 0) {
      s_ms[sl][warp] = msum;
      s_bv[sl][warp] = best;
      s_bi[sl][warp] = vi;
    }
    __syncthreads();
    msum = (s_ms[sl][0] + s_ms[sl][1]) + (s_ms[sl][2] + s_ms[sl][3]);
    best = s_bv[sl][0];
    vi = s_bi[sl][0];
#pragma unroll
    for (int w = 1; w < 4; ++w) {
      const float ob = s_bv[sl][w];
      const int oi = s_bi[sl][w];
      if (ob > best || (ob == best && oi < vi)) {
        best = ob;
        vi = oi;
      }
    }
    if (!(msum >= tb * total && msum > 0.f) || vi == INT_MAX || !(best > 0.f)) break;
    const int p = vi;
    const float rinv = rsqrtf(best);
    if (alive) {
      if (j == p) {
        Lw[j * LDF + i] = best * rinv;
        alive = false;
      } else {
        const float* lp = Lw + p * LDF;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int t = 0; t < i; t += 4) {  // entries past step i - 1 are still zero
          const float4 x = *(const float4*)(lj + t);
          const float4 y = *(const float4*)(lp + t);
          a0 = fmaf(x.x, y.x, a0);
          a1 = fmaf(x.y, y.y, a1);
          a2 = fmaf(x.z, y.z, a2);
          a3 = fmaf(x.w, y.w, a3);
        }
        const float l = (Gs[j * LDG + p] - ((a0 + a1) + (a2 + a3))) * rinv;
        Lw[j * LDF + i] = l;
        dj -= l * l;
      }
    }
    if (tid == 0) {
      rdg[i] = rinv;
      s_perm[i] = p;
      if (perm) perm[i] = p;
    }
    bp = i + 1;
  }
  __syncthreads();
  // pivot-order factor (over G, which is no longer needed)
  for (int e = tid; e < bp * bp; e += kPcholF32Threads) {
    const int i = e / bp, l = e % bp;
    Ls[i * LDF + l] = (l <= i) ? Lw[s_perm[i] * LDF + l] : 0.f;
  }
  __syncthreads();
  // Linv = Ls^{-1} by forward substitution, column c by the four lanes of a quad
  {
    const int part = tid & 3;
    const unsigned qmask = 0xFu << (lane & 28);
    for (int c = tid >> 2; c < bp; c += kPcholF32Threads / 4) {
      for (int i = c; i < bp; ++i) {
        float acc = 0.f;
        for (int l = c + part; l < i; l += 4) acc = fmaf(Ls[i * LDF + l], X[l * LDF + c], acc);
        acc += __shfl_xor_sync(qmask, acc, 1);
        acc += __shfl_xor_sync(qmask, acc, 2);
        if (part == 0) X[i * LDF + c] = ((i == c ? 1.f : 0.f) - acc) * rdg[i];
        __syncwarp(qmask);
      }
    }
  }
  __syncthreads();
  for (int i = 0; i < bp; ++i)
    for (int c = tid; c < bp; c += kPcholF32Threads) Linv[(long long)i * ldl + c] = (c <= i) ? X[i * LDF + c] : 0.f;
  {
    const long long k = st->k;
    const int tno = (int)(st->t + 1);
    for (int i = tid; i < bp; i += kPcholF32Threads) {
      const long long row = S_t[s_perm[i]];
      skel[k + i] = row;
      mark[row] = tno;
    }
  }
  __syncthreads();
  if (tid == 0) {
    st->bp = bp;
    st->bp_pad = (bp + 15) / 16 * 16;
    if (bp == 0) st->done = 1;
  }
}

// The same filter for blocks of at most 64 candidates, built around latency: the
// factorisation runs in one warp with no block-wide barrier.  Right-looking: lane l
// holds columns l and l + 32 of the Schur complement (the Gram matrix minus the factor
// so far) in registers.  Each step takes the trailing mass (a warp sum) and the pivot
// (the largest remaining d_r > 0, ties to the smaller index: a warp max over the FP32
// bit patterns, which order like the values for d_r >= 0, then a warp min over the
// indices holding it), and stops at the first step whose trailing mass fails the
// truncation test of Alg. 2; every lane reads c_r = S(r, p) for its two candidates
// from its own columns (the matrix is symmetric up to rounding) and the lanes publish
// the column c through shared memory together; each forms l_r = c_r / sqrt(d_p) and
// applies the rank-1 update S(j, r) -= c_j c_r / d_p to its two columns.  The next step's reductions depend only on the downdated diagonal, so
// they are issued before the 128 multiply-adds of the update and their latency
// overlaps it.  The kernel writes the pivot-order factor Lc; Q'_V = Lc^{-1} V_perm
// follows as a column-parallel substitution (k_trsm_rows_f32).
constexpr int kPchol64 = 64;
constexpr int kPchol64Threads = 32;   // the factorisation: one warp
constexpr int kPchol64Sum = 256;      // the Gram partial sums: the whole CTA
constexpr int kPchol64LDF = 68;       // factor rows: float4 steps over t

__global__ void __launch_bounds__(kPchol64Sum) k_pchol_f32_64(const float* __restrict__ G, long long ldg,
                                                              const float* __restrict__ gram, int ntn,
                                                              float* __restrict__ Lc_out, long long ldl,
                                                              int* __restrict__ perm,
                                                              const long long* __restrict__ S_t,
                                                              long long* __restrict__ skel,
                                                              int* __restrict__ mark, State* st) {
  pdl_wait();
  if (st->done) return;
  // Gs: the Gram matrix (rows = columns, by symmetry), then the factor L (row j =
  // candidate j, column t = step t) once the columns are in registers
  __shared__ __align__(16) float Gs[kPchol64 * kPchol64LDF];
  __shared__ int s_perm[kPchol64];
  __shared__ __align__(16) float lv[kPchol64];  // the pivot's Schur column, published each step
  const int m = (int)st->b_t;
  // the Gram matrix: the sum of the column-tile partials (in tile order) that the CGS
  // product left, or G itself; every thread of the CTA takes part, sixteen entries
  // each, with the loads of four partials of all sixteen in flight together (the
  // partials come from L2, and a chain of dependent round trips would dominate)
  {
    constexpr int E = kPchol64 * kPchol64 / kPchol64Sum;  // entries per thread
    constexpr int T = 4;                                   // partials per round
    float v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = 0.f;
    if (gram) {
      for (int t0 = 0; t0 < ntn; t0 += T) {
        float x[T][E];
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
          for (int q = 0; q < E; ++q)
            x[t][q] = (t0 + t < ntn) ? gram[(size_t)(t0 + t) * (kPchol64 * kPchol64) + threadIdx.x + q * kPchol64Sum]
                                     : 0.f;
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
          for (int q = 0; q < E; ++q) v[q] += x[t][q];
      }
    }
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int e = threadIdx.x + q * kPchol64Sum, r = e >> 6, c = e & 63;
      if (!gram) v[q] = (r < m && c < m) ? G[(long long)r * ldg + c] : 0.f;
      Gs[r * kPchol64LDF + c] = (r < m && c < m) ? v[q] : 0.f;
    }
  }
  __syncthreads();
  if (threadIdx.x >= kPchol64Threads) return;
  const int lane = threadIdx.x;
  const int c0 = lane, c1 = lane + 32;
  float col0[kPchol64], col1[kPchol64];  // S(:, c0), S(:, c1) = rows c0, c1 of the symmetric Gram matrix
#pragma unroll
  for (int j = 0; j < kPchol64; j += 4) {
    const float4 x = *(const float4*)(Gs + c0 * kPchol64LDF + j);
    const float4 y = *(const float4*)(Gs + c1 * kPchol64LDF + j);
    col0[j] = x.x;
    col0[j + 1] = x.y;
    col0[j + 2] = x.z;
    col0[j + 3] = x.w;
    col1[j] = y.x;
    col1[j + 1] = y.y;
    col1[j + 2] = y.z;
    col1[j + 3] = y.w;
  }
  float d0 = Gs[c0 * kPchol64LDF + c0], d1 = Gs[c1 * kPchol64LDF + c1];
  __syncwarp();
  float* Lw = Gs;  // reused for the factor
  for (int e = lane; e < kPchol64 * kPchol64LDF; e += kPchol64Threads) Lw[e] = 0.f;
  double tau_b = st->tau_b;
  if (tau_b < 0.0) tau_b = (m > 0) ? 1.0 / (double)m : 1.0;
  const float tb = (float)tau_b;
  bool a0 = c0 < m, a1 = c1 < m;
  float total = (a0 ? d0 : 0.f) + (a1 ? d1 : 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  // the trailing mass and the pivot of the coming step, from the diagonal alone
  float ms;
  unsigned mx, p;
  auto reduce = [&]() {
    ms = (a0 ? d0 : 0.f) + (a1 ? d1 : 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ms += __shfl_xor_sync(0xffffffffu, ms, o);
    // the FP32 bit pattern orders like the value for d_r >= 0: the largest pattern over the
    // warp, then the smallest index that holds it (two warp reductions)
    const unsigned b0 = (a0 && d0 > 0.f) ? __float_as_uint(d0) : 0u;
    const unsigned b1 = (a1 && d1 > 0.f) ? __float_as_uint(d1) : 0u;
    mx = __reduce_max_sync(0xffffffffu, b0 > b1 ? b0 : b1);
    const unsigned cand = (mx != 0u && b0 == mx) ? (unsigned)c0 : ((mx != 0u && b1 == mx) ? (unsigned)c1 : 64u);
    const unsigned pm = __reduce_min_sync(0xffffffffu, cand);
    p = mx ? pm : 0xffffffffu;
  };
  __syncwarp();
  reduce();
  int steps = 0;
  for (int i = 0; i < m; ++i) {
    if (mx == 0u || !(ms >= tb * total && ms > 0.f)) break;  // the same on every lane; b' = i
    const float rinv = rsqrtf(__uint_as_float(mx));
    const float rdp = rinv * rinv;
    // c_j = S(j, p): every lane reads its own two entries S(c0, p), S(c1, p) (the Schur
    // complement is symmetric up to rounding) with a warp-uniform switch, and the lanes
    // publish the column together for the rank-1 update
    float cr0 = 0.f, cr1 = 0.f;
    switch (p) {
#define RBRP_PICK(k) \
  case k:            \
    cr0 = col0[k];   \
    cr1 = col1[k];   \
    break;
#define RBRP_PICK8(k) RBRP_PICK(k) RBRP_PICK(k + 1) RBRP_PICK(k + 2) RBRP_PICK(k + 3) \
                      RBRP_PICK(k + 4) RBRP_PICK(k + 5) RBRP_PICK(k + 6) RBRP_PICK(k + 7)
      RBRP_PICK8(0) RBRP_PICK8(8) RBRP_PICK8(16) RBRP_PICK8(24)
      RBRP_PICK8(32) RBRP_PICK8(40) RBRP_PICK8(48) RBRP_PICK8(56)
#undef RBRP_PICK8
#undef RBRP_PICK
      default:
        break;
    }
    lv[c0] = cr0;
    lv[c1] = cr1;
    __syncwarp();
    const float l0 = cr0 * rinv, l1 = cr1 * rinv;
    if (a0) Lw[c0 * kPchol64LDF + i] = l0;
    if (a1) Lw[c1 * kPchol64LDF + i] = l1;
    if ((unsigned)c0 == p) a0 = false;
    if ((unsigned)c1 == p) a1 = false;
    d0 -= l0 * l0;
    d1 -= l1 * l1;
    if (lane == 0) s_perm[i] = (int)p;
    steps = i + 1;
    reduce();  // the next step's, overlapping the update below
    // rank-1 update of both columns: S(j, r) -= c_j c_r / d_p
    const float f0 = cr0 * rdp, f1 = cr1 * rdp;
#pragma unroll
    for (int j = 0; j < kPchol64; j += 4) {
      const float4 l4 = *(const float4*)(lv + j);
      col0[j] = fmaf(-l4.x, f0, col0[j]);
      col0[j + 1] = fmaf(-l4.y, f0, col0[j + 1]);
      col0[j + 2] = fmaf(-l4.z, f0, col0[j + 2]);
      col0[j + 3] = fmaf(-l4.w, f0, col0[j + 3]);
      col1[j] = fmaf(-l4.x, f1, col1[j]);
      col1[j + 1] = fmaf(-l4.y, f1, col1[j + 1]);
      col1[j + 2] = fmaf(-l4.z, f1, col1[j + 2]);
      col1[j + 3] = fmaf(-l4.w, f1, col1[j + 3]);
    }
    __syncwarp();  // every lane has read lv before the lanes write the next pivot's column
  }
  const int bp = steps;
  __syncwarp();
  // the pivot-order factor Lc(i, l) = Lw[perm[i]][l] for l <= i < b' (zero
  // elsewhere) to Lc_out, two columns per lane (coalesced across lanes);
  // Q'_V = Lc^{-1} V_perm is then a column-parallel substitution (k_trsm_rows_f32)
#pragma unroll 4
  for (int i = 0; i < kPchol64; ++i) {
    const int pi = i < bp ? s_perm[i] : 0;
    Lc_out[(long long)i * ldl + c0] = (c0 <= i && i < bp) ? Lw[pi * kPchol64LDF + c0] : 0.f;
    Lc_out[(long long)i * ldl + c1] = (c1 <= i && i < bp) ? Lw[pi * kPchol64LDF + c1] : 0.f;
  }
  {
    const long long k = st->k;
    const int tno = (int)(st->t + 1);
    for (int i = lane; i < bp; i += kPchol64Threads) {
      const int pi = s_perm[i];
      if (perm) perm[i] = pi;
      const long long row = S_t[pi];
      skel[k + i] = row;
      mark[row] = tno;
    }
  }
  __syncwarp();
  if (lane == 0) {
    st->bp = bp;
    st->bp_pad = (bp + 15) / 16 * 16;
    if (bp == 0) st->done = 1;
  }
}

// Q'_V = Lc^{-1} V(perm, :) on the plain TF32 path (Alg. 2, acceptance): rows by
// forward substitution, Y(i, :) = (V(perm[i], :) - sum_{l<i} Lc(i, l) Y(l, :)) / Lc(i, i)
// for i < b' <= 64, FP32.  32 columns per CTA, one octet of lanes per column;
// lane q of the octet holds rows q, q + 8, ... of its column in registers and,
// right-looking, subtracts Lc(r, i) y_i from its remaining rows as soon as
// y_i is known (one shuffle from the lane that owns row i), so a row costs a
// multiply, a shuffle and a fused multiply-add on the critical path.
// With Qp set, the kernel also writes the update's operand copies of Q'
// (rows of Qp, ld ldp, and the transpose QpT, ld ldpt, rows >= b' and columns
// >= d zero; Qp covers qrows rows), which k_qp_lowp makes otherwise.
__global__ void __launch_bounds__(256) k_trsm_rows_f32(const float* __restrict__ Lc, long long ldl,
                                                       const int* __restrict__ perm, const float* __restrict__ V,
                                                       long long ldv, float* __restrict__ Ybase, DimRef y_off,
                                                       long long ldy, long long d, float* __restrict__ Qp,
                                                       long long ldp, float* __restrict__ QpT, long long ldpt,
                                                       int qrows, const State* st) {
  pdl_wait();
  if (st->done) return;
  __shared__ float Ls[kPchol64][kPchol64 + 1];
  __shared__ float rdiag[kPchol64];
  const int bp = (int)st->bp;
  const int lane = threadIdx.x & 31, cl = threadIdx.x >> 3, part = threadIdx.x & 7;
  const long long c = (long long)blockIdx.x * 32 + cl;
  for (int e = threadIdx.x; e < kPchol64 * kPchol64; e += blockDim.x) {
    const int r = e >> 6, l = e & 63;
    Ls[r][l] = (r < bp && l < bp) ? Lc[(long long)r * ldl + l] : 0.f;
  }
  for (int r = threadIdx.x; r < kPchol64; r += blockDim.x) rdiag[r] = (r < bp) ? 1.f / Lc[(long long)r * ldl + r] : 0.f;
  float b[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int r = part + 8 * q;
    b[q] = (r < bp && c < d) ? V[(long long)perm[r] * ldv + c] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int qi = 0; qi < 8; ++qi) {
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int i = 8 * qi + o;
      if (i < bp) {
        float yi = b[qi] * rdiag[i];                           // right on the lane that owns row i
        yi = __shfl_sync(0xffffffffu, yi, (lane & ~7) | o);
        if (part == o) b[qi] = yi;
#pragma unroll
        for (int q = qi; q < 8; ++q) {
          const int r = part + 8 * q;
          if (r > i) b[q] = fmaf(-Ls[r][i], yi, b[q]);
        }
      }
    }
  }
  if (c < d) {
    float* Y = Ybase + dim_val(y_off);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = part + 8 * q;
      if (r < bp) Y[(long long)r * ldy + c] = b[q];
    }
  }
  if (Qp && c < ldp) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = part + 8 * q;
      const float v = (r < bp && c < d) ? tf32_rn(b[q]) : 0.f;  // the nearest TF32 value
      if (r < qrows) Qp[(long long)r * ldp + c] = v;
      if (r < qrows && c < d) QpT[c * ldpt + r] = v;
    }
  }
}

cudaError_t launch_trsm_rows_f32(const float* Lc, long long ldl, const int* perm, const float* V, long long ldv,
                                 float* Y, DimRef y_off, long long ldy, long long d, float* Qp, long long ldp,
                                 float* QpT, long long ldpt, int qrows, const State* st, cudaStream_t s) {
  const long long cols = Qp ? std::max(d, ldp) : d;
  return counted(launch_pdl(k_trsm_rows_f32, dim3((unsigned)((cols + 31) / 32)), dim3(256), 0, s, Lc, ldl, perm, V,
                            ldv, Y, y_off, ldy, d, Qp, ldp, QpT, ldpt, qrows, st));
}

int filter_f32_writes_factor(int b) { return b <= kPchol64; }

cudaError_t launch_filter_f32(const float* G, long long ldg, const float* gram, int ntn, const long long* S_t,
                              float* Lout, long long ldl, int* perm, long long* skel, int* mark, int b, State* st,
                              cudaStream_t s) {
  float* Linv = Lout;  // the factor for b <= 64, its inverse above
  if (b > kRegCholMax) return cudaErrorInvalidValue;
  if (b <= kPchol64) {
    return counted(launch_pdl(k_pchol_f32_64, dim3(1), dim3(kPchol64Sum), 0, s, G, ldg, gram, ntn, Linv, ldl, perm,
                              S_t, skel, mark, st));
  }
  if (gram) return cudaErrorInvalidValue;  // (Gram partials only for b <= 64)
  const int ldf = (b + 4) & ~3;
  const size_t smem = (size_t)2 * b * ldf * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_pchol_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_pchol_f32<<<1, kPcholF32Threads, smem, s>>>(G, ldg, Linv, ldl, perm, S_t, skel, mark, st, b);
  return counted(cudaGetLastError());
}

static cudaError_t launch_pchol_any(const double* G, long long ldg, double* Lc, long long ldl, int* perm,
                                    const long long* S_t, long long* skel, int* mark, int b, State* st, int pivoted,
                                    cudaStream_t s, long long mark_base = 0, long long mark_n = LLONG_MAX) {
  // Lw (candidate-indexed factor, kMaxBlock x kMaxBlock) lives right after Lc in the workspace
  double* Lw = Lc + (long long)kMaxBlock * ldl;
  const int ne = b * (b + 1) / 2;
  if (ne <= 9 * kRegCholThreads)
    k_pchol_reg<9><<<1, kRegCholThreads, 0, s>>>(G, ldg, Lc, ldl, Lw, perm, S_t, skel, mark, st, pivoted, mark_base,
                                                 mark_n);
  else if (b <= kRegCholMax)
    k_pchol_reg<33><<<1, kRegCholThreads, 0, s>>>(G, ldg, Lc, ldl, Lw, perm, S_t, skel, mark, st, pivoted, mark_base,
                                                  mark_n);
  else
    k_pchol_global<<<1, 256, 0, s>>>(G, ldg, Lc, ldl, Lw, perm, S_t, skel, mark, st, pivoted, mark_base, mark_n);
  return counted(cudaGetLastError());
}

// mark_base / mark_n: the rows of S_t are global row indices; only those in
// [mark_base, mark_base + mark_n) belong to this residual and are marked (a row
// shard of one ID; the whole problem passes 0 and n).
cudaError_t launch_filter(const double* G, long long ldg, const long long* S_t, double* Lc, long long ldl,
                          int* perm, long long* skel, int* mark, int b, State* st, cudaStream_t s, long long mark_base,
                          long long mark_n) {
  return launch_pchol_any(G, ldg, Lc, ldl, perm, S_t, skel, mark, b, st, 1, s, mark_base, mark_n);
}

// Forced acceptance (sketchy pivoting's OSID on the sketch): the b_t candidates are
// taken in the order given, with no pivoting and no truncation; only a candidate
// that has no residual left (Gram matrix not positive definite) ends the block.
cudaError_t launch_filter_forced(const double* G, long long ldg, const long long* S_t, double* Lc, long long ldl,
                                 int* perm, long long* skel, int* mark, int b, State* st, cudaStream_t s) {
  return launch_pchol_any(G, ldg, Lc, ldl, perm, S_t, skel, mark, b, st, 2, s);
}

cudaError_t launch_chol(const double* G, long long ldg, double* Lc, long long ldl, int b, State* st,
                        cudaStream_t s) {
  return launch_pchol_any(G, ldg, Lc, ldl, nullptr, nullptr, nullptr, nullptr, b, st, 0, s);
}

// ============================================================================
// Q' rows by forward substitution: Y(i,:) = (V(perm[i],:) - sum_{l<i} Lc(i,l) Y(l,:)) / Lc(i,i),
// i < b'.  With V_perm = Lc Y and Lc lower triangular, Y has orthonormal rows
// spanning the accepted candidates in pivot order.
// ============================================================================
// Same substitution with 16 columns per CTA: the right-hand sides sit in shared
// memory and each dot product sum_{l<i} Lc(i,l) Y(l,c) is split over 16 threads
// (a quarter-warp per column pair) and combined with shuffles.
__global__ void __launch_bounds__(256) k_trsm_rows16(const double* __restrict__ Lc, long long ldl,
                                                     const int* __restrict__ perm, const double* __restrict__ V,
                                                     long long ldv, double* __restrict__ Ybase, DimRef y_off,
                                                     long long ldy, long long d, const State* st) {
  if (st->done) return;
  __shared__ double Ys[kMaxBlock][16];
  __shared__ double rdiag[kMaxBlock];
  const int bp = (int)st->bp;
  const int cl = threadIdx.x >> 4, part = threadIdx.x & 15;  // column within the chunk, summation lane
  const long long c = (long long)blockIdx.x * 16 + cl;
  for (int i = part; i < bp; i += 16) {
    const int src = perm ? perm[i] : i;
    Ys[i][cl] = (c < d) ? V[(long long)src * ldv + c] : 0.0;
  }
  // reciprocals of the diagonal once (FP64 division is costly on GB300)
  for (int i = threadIdx.x; i < bp; i += blockDim.x) rdiag[i] = 1.0 / Lc[(long long)i * ldl + i];
  __syncthreads();
  for (int i = 0; i < bp; ++i) {
    double acc = 0.0;
    for (int l = part; l < i; l += 16) acc = fma(Lc[(long long)i * ldl + l], Ys[l][cl], acc);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (part == 0) Ys[i][cl] = (Ys[i][cl] - acc) * rdiag[i];
    __syncthreads();
  }
  if (c < d) {
    double* Y = Ybase + dim_val(y_off);
    for (int i = part; i < bp; i += 16) Y[(long long)i * ldy + c] = Ys[i][cl];
  }
}

cudaError_t launch_trsm_rows(const double* Lc, long long ldl, const int* perm, const double* V, long long ldv,
                             double* Y, DimRef y_off, long long ldy, long long d, int b, const State* st,
                             cudaStream_t s) {
  (void)b;
  k_trsm_rows16<<<(unsigned)((d + 15) / 16), 256, 0, s>>>(Lc, ldl, perm, V, ldv, Y, y_off, ldy, d, st);
  return counted(cudaGetLastError());
}

}  // namespace rbrp
