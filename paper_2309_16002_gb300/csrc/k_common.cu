// SIMT kernels of the RBRP block loop (Alg. 2) and of the interpolation matrix
// (Alg. 3): initial norms, the Philox exponential-race sampler, the gather of
// candidate rows, a split-K GEMM used for CGS2 / Gram / FP64 update products,
// the pivoted-Cholesky form of the robust blockwise filter, row triangular
// solves that build Q', the norm pass and the block finalisation.
//
// All per-block kernels take their sizes from the device State and return at
// once when State::done is set, so a block is a fixed launch sequence.
#include <float.h>
#include <limits.h>
#include <math.h>

#include "rbrp_internal.cuh"
#include "sample_common.cuh"

namespace rbrp {

// ============================================================================
// Alg. 2, initial norms: d0(i) = ||x_i||^2, copy of X into the residual R.
// One warp per row; per-CTA partial sums in a fixed order (deterministic).
// ============================================================================
template <typename TX, typename TR>
__global__ void __launch_bounds__(256) k_init_norms(const TX* __restrict__ X, long long n, long long d,
                                                    long long ldx, TR* __restrict__ R, long long ldr,
                                                    double* __restrict__ dvec, int* __restrict__ mark,
                                                    double* __restrict__ partials) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double wsum[8];
  double mine = 0.0;
  const long long lim = R ? ldr : d;  // no residual copy (downdate form): norms only
  for (long long i = (long long)blockIdx.x * 8 + warp; i < n; i += (long long)gridDim.x * 8) {
    const TX* x = X + i * ldx;
    TR* r = R ? R + i * ldr : nullptr;
    double s = 0.0;
    if (sizeof(TR) == 8) {
      for (long long j = lane; j < lim; j += 32) {
        TR v = (j < d) ? (TR)x[j] : (TR)0;
        if (r) r[j] = v;
        const double dv = (double)v;
        s = fma(dv, dv, s);
      }
    } else {
      // FP32 residual: per-lane FP32 partial sums (FP64 FMAs run at ~2/clock/SM on GB300)
      float sf = 0.f;
      for (long long j = lane; j < lim; j += 32) {
        TR v = (j < d) ? (TR)x[j] : (TR)0;
        if (r) r[j] = v;
        const float fv = (float)v;
        sf = fmaf(fv, fv, sf);
      }
      s = (double)sf;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      dvec[i] = s;
      mark[i] = 0;
    }
    mine += s;
  }
  if (lane == 0) wsum[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    partials[blockIdx.x] = t;
  }
}

// FP32 input and FP32 residual (the tensor-core paths), 16-byte rows: the same sums
// from float4 loads, eight in flight per lane, so the pass over X runs near the HBM
// rate (one 4-byte load per lane and step leaves too few bytes in flight).
__global__ void __launch_bounds__(256) k_init_norms_f32v(const float* __restrict__ X, long long n, long long d,
                                                         long long ldx, float* __restrict__ R, long long ldr,
                                                         double* __restrict__ dvec, int* __restrict__ mark,
                                                         double* __restrict__ partials) {
  constexpr int U = 8;  // float4 loads in flight per lane
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double wsum[8];
  double mine = 0.0;
  const long long nv = d / 4;
  for (long long i = (long long)blockIdx.x * 8 + warp; i < n; i += (long long)gridDim.x * 8) {
    const float4* x4 = (const float4*)(X + i * ldx);
    float4* r4 = R ? (float4*)(R + i * ldr) : nullptr;
    float sf = 0.f;
    for (long long v0 = lane; v0 < nv; v0 += 32 * U) {
      float4 q[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long v = v0 + 32 * u;
        q[u] = (v < nv) ? x4[v] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long v = v0 + 32 * u;
        if (r4 && v < nv) r4[v] = q[u];
        sf = fmaf(q[u].x, q[u].x, sf);
        sf = fmaf(q[u].y, q[u].y, sf);
        sf = fmaf(q[u].z, q[u].z, sf);
        sf = fmaf(q[u].w, q[u].w, sf);
      }
    }
    for (long long j = 4 * nv + lane; j < d; j += 32) {
      const float v = X[i * ldx + j];
      if (R) R[i * ldr + j] = v;
      sf = fmaf(v, v, sf);
    }
    if (R)
      for (long long j = d + lane; j < ldr; j += 32) R[i * ldr + j] = 0.f;
    double sum = (double)sf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
      dvec[i] = sum;
      mark[i] = 0;
    }
    mine += sum;
  }
  if (lane == 0) wsum[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    partials[blockIdx.x] = t;
  }
}

cudaError_t launch_init_norms(const void* X, int x_is_fp64, long long n, long long d, long long ldx,
                              void* R, int r_is_fp64, long long ldr, double* dvec, int* mark,
                              double* partials, int nparts, State* st, cudaStream_t s) {
  (void)st;
  dim3 grid(nparts), block(256);
  const bool vec = !x_is_fp64 && !r_is_fp64 && (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0 &&
                   (!R || ((ldr & 3) == 0 && ((uintptr_t)R & 15) == 0));
  if (vec)
    k_init_norms_f32v<<<grid, block, 0, s>>>((const float*)X, n, d, ldx, (float*)R, ldr, dvec, mark, partials);
  else if (x_is_fp64 && r_is_fp64)
    k_init_norms<double, double><<<grid, block, 0, s>>>((const double*)X, n, d, ldx, (double*)R, ldr, dvec, mark, partials);
  else if (x_is_fp64)
    k_init_norms<double, float><<<grid, block, 0, s>>>((const double*)X, n, d, ldx, (float*)R, ldr, dvec, mark, partials);
  else if (r_is_fp64)
    k_init_norms<float, double><<<grid, block, 0, s>>>((const float*)X, n, d, ldx, (double*)R, ldr, dvec, mark, partials);
  else
    k_init_norms<float, float><<<grid, block, 0, s>>>((const float*)X, n, d, ldx, (float*)R, ldr, dvec, mark, partials);
  return counted(cudaGetLastError());
}

__device__ __forceinline__ void stop_test(State* st) {
  const bool cap = st->k >= st->k_cap;
  const bool tol_met = (st->tau >= 0.0) && !(st->D > st->tau * st->D0);
  st->done = (cap || tol_met) ? 1 : 0;
}

__global__ void k_finish_init(const double* __restrict__ partials, int np, State* st, double tau, double tau_b,
                              long long k_cap, unsigned spin_mbar, unsigned spin_grid) {
  const double D0 = fixed_sum_partials<kFixedSumThreads>(partials, np);
  if (threadIdx.x == 0) {
    st->spin_mbar = spin_mbar;
    st->spin_grid = spin_grid;
    st->tau = tau;
    st->tau_b = tau_b;
    st->k_cap = k_cap;
    st->D0 = D0;
    st->D = D0;
    st->k = 0;
    st->t = 0;
    st->b_t = 0;
    st->bp = 0;
    st->bp_pad = 0;
    st->sample_fallback = 0;
    st->status = 0;
    st->iters = 0;
    if (!isfinite(D0)) {
      st->status = RBRP_ENONFINITE;
      st->done = 1;
    } else {
      stop_test(st);
    }
  }
}

cudaError_t launch_finish_init(const double* partials, int nparts, State* st, double tau, double tau_b,
                               long long k_cap, cudaStream_t s) {
  unsigned spin_mbar = kDefaultSpinMbar, spin_grid = kDefaultSpinGrid;
  wait_limits(&spin_mbar, &spin_grid);
  k_finish_init<<<1, kFixedSumThreads, 0, s>>>(partials, nparts, st, tau, tau_b, k_cap, spin_mbar, spin_grid);
  return counted(cudaGetLastError());
}

// ============================================================================
// Alg. 2, sampling step: S_t ~ d / ||d||_1 without replacement, as an exponential race:
// key kappa_i = -log(u_i) / d_i over eligible rows (d_i > 0; accepted rows
// have d_i = 0), the b_t smallest in ascending (kappa, i) order.  The greedy
// sampler (blockwise greedy remark) uses key -d_i.  Selection is a tree of
// CTA-wide bitonic sorts: every CTA sorts 2048 (key, row) pairs and keeps its
// b smallest, until one CTA is left.
// ============================================================================

__global__ void __launch_bounds__(1024) k_sample_level(const double* __restrict__ dvec, long long n,
                                                       const Pair* __restrict__ in, long long n_in,
                                                       Pair* __restrict__ out, int b, int greedy,
                                                       unsigned long long seed, unsigned long long problem,
                                                       long long* __restrict__ S_t, State* st, int first,
                                                       int last, int force, long long row_base,
                                                       unsigned long long* __restrict__ keys_out) {
  pdl_wait();
  // exact FP64 sampler: runs when the two-stage sampler asked for it, or always
  // (force, on the first level, which then raises the flag for the later levels)
  if (st->done || (!force && !st->sample_fallback)) return;
  if (force && blockIdx.x == 0 && threadIdx.x == 0 && !last) st->sample_fallback = 1;
  __shared__ Pair sh[kSortChunk];
  const unsigned long long block_no = (unsigned long long)st->t + 1ULL;  // the paper's t
  const long long base = (long long)blockIdx.x * kSortChunk;
  for (int e = threadIdx.x; e < kSortChunk; e += blockDim.x) {
    const long long gidx = base + e;
    Pair p{kIneligible, LLONG_MAX};
    if (first) {
      if (gidx < n) {
        // a row shard draws with its rows' global indices (row_base + local index)
        p.key = exact_key(dvec[gidx], gidx + row_base, block_no, seed, problem, greedy);
        p.idx = gidx;
      }
    } else if (gidx < n_in) {
      p = in[gidx];
    }
    sh[e] = p;
  }
  sort_chunk(sh);  // ascending by (key, idx)
  if (!last) {
    for (int e = threadIdx.x; e < b; e += blockDim.x) out[(long long)blockIdx.x * b + e] = sh[e];
    return;
  }
  __shared__ int nfin;
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
    if (keys_out) keys_out[e] = sh[e].key;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->b_t = bt;
    st->sample_fallback = 0;
    if (bt == 0 && !keys_out) st->done = 1;  // a row shard without candidates is not finished
  }
}

size_t sample_scratch_pairs(long long n, int b) {
  const long long g0 = (n + kSortChunk - 1) / kSortChunk;
  return (size_t)(g0 * b + 1);
}

cudaError_t launch_sample(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                          unsigned long long problem, void* cand_a, void* cand_b, long long* S_t,
                          State* st, int force, cudaStream_t s, long long row_base,
                          unsigned long long* keys_out) {
  long long groups = (n + kSortChunk - 1) / kSortChunk;
  Pair* bufs[2] = {(Pair*)cand_a, (Pair*)cand_b};
  int cur = 0;
  cudaError_t e = counted(launch_pdl(k_sample_level, dim3((unsigned)groups), dim3(1024), 0, s, dvec, n,
                                     (const Pair*)nullptr, 0LL, bufs[cur], b, greedy, seed, problem, S_t, st, 1,
                                     groups == 1 ? 1 : 0, force, row_base, keys_out));
  if (e != cudaSuccess) return e;
  while (groups > 1) {
    const long long n_in = groups * b;
    groups = (n_in + kSortChunk - 1) / kSortChunk;
    e = counted(launch_pdl(k_sample_level, dim3((unsigned)groups), dim3(1024), 0, s, dvec, n, (const Pair*)bufs[cur],
                           n_in, bufs[cur ^ 1], b, greedy, seed, problem, S_t, st, 0, groups == 1 ? 1 : 0, 0,
                           row_base, keys_out));
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  return cudaSuccess;
}

// ============================================================================
// Alg. 2, projection step (first half): V = R(S_t, :) (FP64, or FP32 on the plain TF32 path).
// ============================================================================
template <typename TR, typename TV>
__global__ void k_gather(const TR* __restrict__ R, long long ldr, const long long* __restrict__ S_t,
                         TV* __restrict__ V, long long ldv, long long d, const State* st) {
  pdl_wait();
  if (st->done) return;
  const long long i = blockIdx.y;
  if (i >= st->b_t) return;
  const TR* r = R + S_t[i] * ldr;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < d; j += (long long)gridDim.x * blockDim.x)
    V[i * ldv + j] = (TV)r[j];
}

cudaError_t launch_gather(const void* R, int r_is_fp64, long long ldr, const long long* S_t, void* V, int v_is_fp64,
                          long long ldv, long long d, int b, const State* st, cudaStream_t s) {
  dim3 grid((unsigned)((d + 255) / 256), (unsigned)b);
  if (r_is_fp64)
    return counted(launch_pdl(k_gather<double, double>, grid, dim3(256), 0, s, (const double*)R, ldr, S_t, (double*)V,
                              ldv, d, st));
  if (v_is_fp64)
    return counted(launch_pdl(k_gather<float, double>, grid, dim3(256), 0, s, (const float*)R, ldr, S_t, (double*)V,
                              ldv, d, st));
  return counted(launch_pdl(k_gather<float, float>, grid, dim3(256), 0, s, (const float*)R, ldr, S_t, (float*)V, ldv,
                            d, st));
}

// ============================================================================
// Split-K SIMT GEMM: C = alpha A B + beta C on strided views, sizes from the
// device.  TILE x TILE output tile (64 or 32), 256 threads, (TILE/16)^2 outputs
// per thread, K step 16.  TACC is the product/accumulation type (the operands
// are converted to it when staged); the epilogue combines in double.  Small
// FP64 products use the 32-wide tile with a fine K split so that every SM gets
// work (GB300 retires ~2 FP64 FMA per clock per SM).
// ============================================================================
template <typename TA, typename TB, typename TC, typename TACC, int TILE>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs g, int splits) {
  constexpr int R = TILE / 16;          // outputs per thread along each axis
  constexpr int LOADS = TILE * 16 / 256;  // staged elements per thread per operand
  if (g.st && g.st->done) return;
  const long long M = dim_val(g.M), N = dim_val(g.N), K = dim_val(g.K);
  const long long m0 = (long long)blockIdx.y * TILE, n0 = (long long)blockIdx.x * TILE;
  if (m0 >= M || n0 >= N) return;
  const TA* A = (const TA*)g.A.base + dim_val(g.A.off);
  const TB* B = (const TB*)g.B.base + dim_val(g.B.off);
  TC* C = (TC*)g.C.base + dim_val(g.C.off);
  long long kc = (K + splits - 1) / splits;
  kc = (kc + 15) / 16 * 16;
  const long long kb = (long long)blockIdx.z * kc;
  const long long ke = (kb + kc < K) ? kb + kc : K;

  __shared__ TACC As[16][TILE];
  __shared__ TACC Bs[16][TILE];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  TACC acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = (TACC)0;

  const bool a_kmajor = (g.A.cs == 1);
  const bool b_nmajor = (g.B.cs == 1);
  for (long long k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int q = 0; q < LOADS; ++q) {
      const int e = tid + 256 * q;
      int r, c;
      if (a_kmajor) { r = e >> 4; c = e & 15; } else { r = e % TILE; c = e / TILE; }
      const long long gm = m0 + r, gk = k0 + c;
      As[c][r] = (gm < M && gk < ke) ? (TACC)A[gm * g.A.rs + gk * g.A.cs] : (TACC)0;
      int rb, cb;
      if (b_nmajor) { rb = e / TILE; cb = e % TILE; } else { rb = e & 15; cb = e >> 4; }
      const long long hk = k0 + rb, hn = n0 + cb;
      Bs[rb][cb] = (hk < ke && hn < N) ? (TACC)B[hk * g.B.rs + hn * g.B.cs] : (TACC)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      TACC a[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (splits == 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const long long gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const long long gn = n0 + tx + 16 * j;
        if (gn >= N) continue;
        TC* cp = C + gm * g.C.rs + gn * g.C.cs;
        double v = g.alpha * (double)acc[i][j];
        if (g.beta != 0.0) v += g.beta * (double)(*cp);
        *cp = (TC)v;
      }
    }
  } else {
    TACC* P = (TACC*)g.partial + (long long)blockIdx.z * g.pm * g.pn;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const long long gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const long long gn = n0 + tx + 16 * j;
        if (gn < N) P[gm * g.pn + gn] = acc[i][j];
      }
    }
  }
}

template <typename TC, typename TACC>
__global__ void k_gemm_reduce(GemmArgs g, int splits) {
  if (g.st && g.st->done) return;
  const long long M = dim_val(g.M), N = dim_val(g.N);
  TC* C = (TC*)g.C.base + dim_val(g.C.off);
  const TACC* P = (const TACC*)g.partial;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / N, j = e % N;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += (double)P[(long long)z * g.pm * g.pn + i * g.pn + j];
    TC* cp = C + i * g.C.rs + j * g.C.cs;
    double v = g.alpha * s;
    if (g.beta != 0.0) v += g.beta * (double)(*cp);
    *cp = (TC)v;
  }
}

template <typename TA, typename TB, typename TC, typename TACC>
cudaError_t launch_gemm(const GemmArgs& g, long long Mmax, long long Nmax, int splits, int tile, cudaStream_t s) {
  if (Mmax <= 0 || Nmax <= 0) return cudaSuccess;
  if (splits < 1) splits = 1;
  if (tile == 32) {
    dim3 grid((unsigned)((Nmax + 31) / 32), (unsigned)((Mmax + 31) / 32), (unsigned)splits);
    k_gemm<TA, TB, TC, TACC, 32><<<grid, 256, 0, s>>>(g, splits);
  } else {
    dim3 grid((unsigned)((Nmax + 63) / 64), (unsigned)((Mmax + 63) / 64), (unsigned)splits);
    k_gemm<TA, TB, TC, TACC, 64><<<grid, 256, 0, s>>>(g, splits);
  }
  cudaError_t e = counted(cudaGetLastError());
  if (e != cudaSuccess || splits == 1) return e;
  long long tot = Mmax * Nmax;
  unsigned rb = (unsigned)((tot + 255) / 256);
  if (rb > 4096) rb = 4096;
  k_gemm_reduce<TC, TACC><<<rb, 256, 0, s>>>(g, splits);
  return counted(cudaGetLastError());
}

template cudaError_t launch_gemm<double, double, double, double>(const GemmArgs&, long long, long long, int, int, cudaStream_t);
template cudaError_t launch_gemm<float, float, float, float>(const GemmArgs&, long long, long long, int, int, cudaStream_t);
template cudaError_t launch_gemm<double, double, double, float>(const GemmArgs&, long long, long long, int, int, cudaStream_t);
template cudaError_t launch_gemm<float, double, float, float>(const GemmArgs&, long long, long long, int, int, cudaStream_t);
template cudaError_t launch_gemm<float, double, double, double>(const GemmArgs&, long long, long long, int, int, cudaStream_t);

// ============================================================================
// FP32 copies of the new basis rows for the low-precision update:
// Qp (b'_pad x ldp, rows = basis vectors) and QpT (d x ldpt, transposed).
// Rows >= b' and columns >= d are zero so padded MMA tiles add nothing.
// ============================================================================
// With the lo buffers set (3xTF32), hi is the FP32 value with the 13 low
// mantissa bits cleared (exact in TF32) and lo = fp32(q - hi) is the rest.
template <typename TQ>
__global__ void k_qp_lowp(const TQ* __restrict__ Qt, long long ldq, float* __restrict__ Qp,
                          float* __restrict__ Qp_lo, long long ldp, float* __restrict__ QpT, float* __restrict__ QpT_lo,
                          long long ldpt, long long d, int bmax, const State* st) {
  pdl_wait();
  if (st->done) return;
  const long long k = st->k;
  const int bp = (int)st->bp;
  const long long tot = (long long)bmax * ldp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ldp);
    const long long j = e % ldp;
    const TQ q = (i < bp && j < d) ? Qt[(k + i) * ldq + j] : (TQ)0;
    // nearest TF32 values (the MMA would truncate an FP32 operand): hi, and lo = q - hi
    const float hi = tf32_rn((float)q);
    float lo = 0.0f;
    if (Qp_lo) {
      lo = tf32_rn((float)(q - (TQ)hi));
      Qp_lo[(long long)i * ldp + j] = lo;
    }
    Qp[(long long)i * ldp + j] = hi;
    if (j < d && QpT) {
      QpT[j * ldpt + i] = hi;
      if (QpT_lo) QpT_lo[j * ldpt + i] = lo;
    }
  }
}

cudaError_t launch_qp_lowp(const void* Qt, int q_is_fp64, long long ldq, float* Qp, float* Qp_lo, long long ldp,
                           float* QpT, float* QpT_lo, long long ldpt, long long d, int b, const State* st,
                           cudaStream_t s) {
  long long tot = (long long)b * ldp;
  unsigned g = (unsigned)((tot + 255) / 256);
  if (g > 2048) g = 2048;
  if (q_is_fp64)
    return counted(launch_pdl(k_qp_lowp<double>, dim3(g), dim3(256), 0, s, (const double*)Qt, ldq, Qp, Qp_lo, ldp, QpT,
                              QpT_lo, ldpt, d, b, st));
  return counted(launch_pdl(k_qp_lowp<float>, dim3(g), dim3(256), 0, s, (const float*)Qt, ldq, Qp, Qp_lo, ldp, QpT,
                            QpT_lo, ldpt, d, b, st));
}

// ============================================================================
// Alg. 2, new residual norms (residual form): d_i = ||R_i||^2; rows accepted in this block
// are zeroed (R_i = 0, d_i = 0).  One warp per row, fixed-order partials.
// ============================================================================
template <typename TR>
__global__ void __launch_bounds__(256) k_norms_zero(TR* __restrict__ R, long long ldr, long long n, long long d,
                                                    const int* __restrict__ mark, double* __restrict__ dvec,
                                                    double* __restrict__ partials, const State* st) {
  if (st->done) return;
  const int tno = (int)(st->t + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double wsum[8];
  double mine = 0.0;
  for (long long i = (long long)blockIdx.x * 8 + warp; i < n; i += (long long)gridDim.x * 8) {
    TR* r = R + i * ldr;
    double s = 0.0;
    if (mark[i] == tno) {
      for (long long j = lane; j < d; j += 32) r[j] = (TR)0;
    } else {
      for (long long j = lane; j < d; j += 32) {
        const double v = (double)r[j];
        s = fma(v, v, s);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0) dvec[i] = s;
    mine += s;
  }
  if (lane == 0) wsum[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    partials[blockIdx.x] = t;
  }
}

cudaError_t launch_norms_zero(void* R, int r_is_fp64, long long ldr, long long n, long long d, const int* mark,
                              double* dvec, double* partials, int nparts, const State* st, cudaStream_t s) {
  if (r_is_fp64)
    k_norms_zero<double><<<nparts, 256, 0, s>>>((double*)R, ldr, n, d, mark, dvec, partials, st);
  else
    k_norms_zero<float><<<nparts, 256, 0, s>>>((float*)R, ldr, n, d, mark, dvec, partials, st);
  return counted(cudaGetLastError());
}

// Alg. 2, new residual norms as printed (downdate form): with Lhat = X Q'^T in columns
// k .. k + b' - 1 of L, d_i -= ||Lhat_i||^2 for the rows not yet in S, d_i = 0
// for the rows accepted in this block (their Lhat row is kept), and Lhat_i = 0
// for rows accepted in earlier blocks (their residual is zero, so their Lhat
// row is, and L(S, :) stays lower triangular).  FP64; one warp per row.
template <typename TL>
__global__ void __launch_bounds__(256) k_downdate(TL* __restrict__ L, long long ldl, long long n,
                                                  const int* __restrict__ mark, double* __restrict__ dvec,
                                                  double* __restrict__ partials, const State* st) {
  if (st->done) return;
  const int tno = (int)(st->t + 1);
  const long long k = st->k;
  const int bp = (int)st->bp;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double wsum[8];
  double mine = 0.0;
  for (long long i = (long long)blockIdx.x * 8 + warp; i < n; i += (long long)gridDim.x * 8) {
    TL* l = L + i * ldl + k;
    const int mk = mark[i];
    double di = 0.0;
    if (mk != 0 && mk != tno) {
      for (int j = lane; j < bp; j += 32) l[j] = (TL)0;
    } else if (mk == 0) {
      double s = 0.0;
      for (int j = lane; j < bp; j += 32) s = fma((double)l[j], (double)l[j], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      di = dvec[i] - s;  // may round below zero for an exhausted row: d_i <= 0 is not eligible
    }
    if (lane == 0) dvec[i] = di;
    mine += di;
  }
  if (lane == 0) wsum[warp] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    partials[blockIdx.x] = t;
  }
}

cudaError_t launch_downdate(double* L, long long ldl, long long n, const int* mark, double* dvec, double* partials,
                            int nparts, const State* st, cudaStream_t s) {
  k_downdate<double><<<nparts, 256, 0, s>>>(L, ldl, n, mark, dvec, partials, st);
  return counted(cudaGetLastError());
}

cudaError_t launch_downdate_f32(float* L, long long ldl, long long n, const int* mark, double* dvec, double* partials,
                                int nparts, const State* st, cudaStream_t s) {
  k_downdate<float><<<nparts, 256, 0, s>>>(L, ldl, n, mark, dvec, partials, st);
  return counted(cudaGetLastError());
}

// Alg. 2, stopping test after a block: D = ||d||_1, k += b', t += 1.  Inside the
// device-side loop (loop != 0) it also sets the while node's condition from the
// State, whether or not the block ran, with a guard on the number of iterations.
__global__ void k_finalize_block(const double* __restrict__ partials, int np, State* st, cudaGraphConditionalHandle h,
                                 int loop) {
  pdl_wait();
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = st->done;
  __syncthreads();
  if (!s_done) {
    const double D = fixed_sum_partials<kFixedSumThreads>(partials, np);
    if (threadIdx.x == 0) finish_block(st, D);
  }
  if (loop && threadIdx.x == 0) {
    const long long it = ++st->iters;
    if (!st->done && it > st->k_cap + 2) {  // cannot happen: every block accepts a row or stops
      st->status = RBRP_ETIMEOUT;
      st->done = 1;
    }
    cudaGraphSetConditional(h, st->done ? 0u : 1u);
  }
}

cudaError_t launch_finalize_block(const double* partials, int nparts, State* st, cudaStream_t s,
                                  cudaGraphConditionalHandle h, int loop) {
  return counted(
      launch_pdl(k_finalize_block, dim3(1), dim3(kFixedSumThreads), 0, s, partials, nparts, st, h, loop));
}

// ============================================================================
// Alg. 3 pieces: column copies, L1 = L(S, :), per-row triangular solve on a
// column block, and W(S, :) = I.
// ============================================================================
template <typename TL, typename TW>
__global__ void k_copy_cols(const TL* __restrict__ L, long long ldl, long long n, long long c0, long long c1,
                            TW* __restrict__ W, long long ldw) {
  const long long w = c1 - c0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * w; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / w, j = c0 + e % w;
    W[i * ldw + j] = (TW)L[i * ldl + j];
  }
}

static unsigned grid_for(long long tot) {
  long long g = (tot + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (unsigned)g;
}

cudaError_t launch_copy_cols_to_f64(const void* L, int l_is_fp64, long long ldl, long long n, long long c0,
                                    long long c1, double* W, long long ldw, cudaStream_t s) {
  if (c1 <= c0 || n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n * (c1 - c0));
  if (l_is_fp64)
    k_copy_cols<double, double><<<g, 256, 0, s>>>((const double*)L, ldl, n, c0, c1, W, ldw);
  else
    k_copy_cols<float, double><<<g, 256, 0, s>>>((const float*)L, ldl, n, c0, c1, W, ldw);
  return counted(cudaGetLastError());
}

cudaError_t launch_copy_cols_to_f32(const void* L, int l_is_fp64, long long ldl, long long n, long long c0,
                                    long long c1, float* W, long long ldw, cudaStream_t s) {
  if (c1 <= c0 || n <= 0) return cudaSuccess;
  const unsigned g = grid_for(n * (c1 - c0));
  if (l_is_fp64)
    k_copy_cols<double, float><<<g, 256, 0, s>>>((const double*)L, ldl, n, c0, c1, W, ldw);
  else
    k_copy_cols<float, float><<<g, 256, 0, s>>>((const float*)L, ldl, n, c0, c1, W, ldw);
  return counted(cudaGetLastError());
}

template <typename TL>
__global__ void k_gather_rows(const TL* __restrict__ L, long long ldl, const long long* __restrict__ rows,
                              long long count, long long width, double* __restrict__ out, long long ldo) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count * width;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / width, j = e % width;
    out[i * ldo + j] = (double)L[rows[i] * ldl + j];
  }
}

cudaError_t launch_gather_rows_f64(const void* L, int l_is_fp64, long long ldl, const long long* rows, long long k,
                                   double* out, long long ldo, cudaStream_t s) {
  return launch_gather_rows_rect(L, l_is_fp64, ldl, rows, k, k, out, ldo, s);
}

cudaError_t launch_gather_rows_rect(const void* L, int l_is_fp64, long long ldl, const long long* rows,
                                    long long count, long long width, double* out, long long ldo, cudaStream_t s) {
  if (count <= 0 || width <= 0) return cudaSuccess;
  const unsigned g = grid_for(count * width);
  if (l_is_fp64)
    k_gather_rows<double><<<g, 256, 0, s>>>((const double*)L, ldl, rows, count, width, out, ldo);
  else
    k_gather_rows<float><<<g, 256, 0, s>>>((const float*)L, ldl, rows, count, width, out, ldo);
  return counted(cudaGetLastError());
}

// W(i, J) <- W(i, J) L1(J, J)^{-1} for a column block J = [j0, j0 + nb) (L1 lower
// triangular): w_j = (rhs_j - sum_{m > j} w_m L1(m, j)) / L1(j, j), j descending.
template <typename T>
__global__ void __launch_bounds__(128) k_trsm_cols(T* __restrict__ W, long long ldw, long long n, long long j0, int nb,
                                                   const double* __restrict__ L1, long long ld1) {
  __shared__ T Ls[64][65];
  __shared__ T rinv[64];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int a = e / nb, c = e % nb;
    Ls[a][c] = (T)L1[(j0 + a) * ld1 + j0 + c];
  }
  // reciprocals of the diagonal once per CTA instead of one division per element
  for (int j = threadIdx.x; j < nb; j += blockDim.x) rinv[j] = (T)(1.0 / L1[(j0 + j) * ld1 + j0 + j]);
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T w[64];
  T* row = W + i * ldw + j0;
#pragma unroll
  for (int j = 0; j < 64; ++j) w[j] = (j < nb) ? row[j] : (T)0;
#pragma unroll
  for (int j = 63; j >= 0; --j) {
    if (j >= nb) continue;
    T s = w[j];
#pragma unroll
    for (int m = j + 1; m < 64; ++m)
      if (m < nb) s -= w[m] * Ls[m][j];
    w[j] = s * rinv[j];
  }
#pragma unroll
  for (int j = 0; j < 64; ++j)
    if (j < nb) row[j] = w[j];
}

template <typename T>
cudaError_t launch_trsm_cols(T* W, long long ldw, long long n, long long j0, int nb, const double* L1, long long ld1,
                             cudaStream_t s) {
  if (n <= 0 || nb <= 0) return cudaSuccess;
  k_trsm_cols<T><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(W, ldw, n, j0, nb, L1, ld1);
  return counted(cudaGetLastError());
}
template cudaError_t launch_trsm_cols<double>(double*, long long, long long, long long, int, const double*, long long,
                                              cudaStream_t);
template cudaError_t launch_trsm_cols<float>(float*, long long, long long, long long, int, const double*, long long,
                                             cudaStream_t);

// W(S, :) = I_k exactly; with W32 set, the FP32 solve result is first widened into W.
__global__ void k_w_identity(double* __restrict__ W, long long ldw, long long k, const long long* __restrict__ skel,
                             long long r0, long long r1) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / k, j = e % k;
    const long long r = skel[i];
    if (r >= r0 && r < r1) W[r * ldw + j] = (i == j) ? 1.0 : 0.0;
  }
}

cudaError_t launch_w_identity_rows(double* W, long long ldw, long long k, const long long* skel, long long r0,
                                   long long r1, cudaStream_t s) {
  if (k <= 0 || r1 <= r0) return cudaSuccess;
  k_w_identity<<<grid_for(k * k), 256, 0, s>>>(W, ldw, k, skel, r0, r1);
  return counted(cudaGetLastError());
}

}  // namespace rbrp

namespace rbrp {


}  // namespace rbrp
