// Sketchy pivoting on the GPU (Sec. 3.2): LU with partial (row) pivoting of the
// first k columns of the sketch Y = X Omega selects the skeletons, and the
// forced-acceptance pass of the block loop then builds the oversampled sketchy
// interpolation matrix of Alg. 4 on all l columns of Y.
//
// LUPP is blocked right-looking Gaussian elimination without row exchanges:
// pivoted rows are only marked.  The k columns are stored column-major (A,
// n x k, ld n) so that a column is contiguous.  Per panel of up to 32 columns:
//  1. k_lupp_panel (one cooperative launch, one CTA per SM, each CTA a fixed
//     slice of rows): for every column of the panel each CTA finds its largest
//     |entry| among unmarked rows and publishes it with the row's panel entries;
//     after one grid barrier every CTA picks the same winner (largest |entry|,
//     ties to the smaller row), reads the winner's panel row from the published
//     copy and eliminates the column from its own rows (multipliers stored in
//     place).  The published copies are double-buffered by column parity, so
//     one barrier per column suffices (no CTA can overwrite a buffer another CTA
//     still reads: it would first have to pass the next barrier).
//  2. k_lupp_u12: U12 = L11^{-1} A(piv, trailing) for the panel's pivot rows.
//  3. the trailing update A(:, trailing) -= A(:, panel) U12 as one SIMT GEMM
//     (rows already pivoted receive garbage there; they are never read again).
// A zero pivot (Y(:, 1:k) of rank below k) ends the selection: *rank is the
// number of pivots found.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "rbrp_internal.cuh"

namespace rbrp {

constexpr int kLuThreads = 512;
constexpr int kLuPanel = 32;

// Y (n x k of a row-major n x l array, leading dimension ldy) -> A column-major (ld n).
template <typename T>
__global__ void __launch_bounds__(256) k_lupp_load(const T* __restrict__ Y, long long ldy, long long n, int k,
                                                   T* __restrict__ A) {
  __shared__ T tile[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int q = ty; q < 32; q += 8) {
    const long long r = r0 + q;
    const int c = c0 + tx;
    tile[q][tx] = (r < n && c < k) ? Y[r * ldy + c] : (T)0;
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int c = c0 + q;
    const long long r = r0 + tx;
    if (r < n && c < k) A[(long long)c * n + r] = tile[tx][q];
  }
}

// Grid barrier over gridDim.x co-resident CTAs (cooperative launch): arrival
// counter bar[0] (reset by the last arriver) and generation bar[1].  Bounded:
// after `limit` polls the CTA records the timeout in *status and carries on.
__device__ __forceinline__ void lu_grid_barrier(unsigned int* bar, int* status, unsigned limit) {
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
          atomicExch(status, (int)RBRP_ETIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Larger of two (|value|, row) candidates: larger value, ties to the smaller row.
__device__ __forceinline__ void lu_better(double& v, long long& i, double v2, long long i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

template <typename T>
__global__ void __launch_bounds__(kLuThreads) k_lupp_panel(T* __restrict__ A, long long n, int j0, int w,
                                                           int* __restrict__ mark, long long* __restrict__ piv,
                                                           int* __restrict__ rank, double* cval, long long* cidx,
                                                           T* crow, unsigned int* bar, int* status, unsigned limit) {
  __shared__ double s_v[kLuThreads / 32];
  __shared__ long long s_i[kLuThreads / 32];
  __shared__ T prow[kLuPanel];
  __shared__ long long s_best;
  __shared__ int s_win, s_stop;
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const long long chunk = (n + G - 1) / G;
  const long long r0 = (long long)c * chunk, r1 = min(n, r0 + chunk);
  if (tid == 0) s_stop = (__ldcg(rank) < j0) ? 1 : 0;  // an earlier panel ended the selection
  __syncthreads();
  if (s_stop) return;  // the same for every CTA
  for (int jj = 0; jj < w; ++jj) {
    const int j = j0 + jj, buf = jj & 1;
    const T* colj = A + (long long)j * n;
    // (a) this CTA's candidate: the largest |A(i, j)| over its unmarked rows
    double v = -1.0;
    long long bi = LLONG_MAX;
    for (long long i = r0 + tid; i < r1; i += kLuThreads)
      if (!mark[i]) lu_better(v, bi, fabs((double)colj[i]), i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const long long i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      lu_better(v, bi, v2, i2);
    }
    if (lane == 0) {
      s_v[wp] = v;
      s_i[wp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      for (int q = 1; q < kLuThreads / 32; ++q) lu_better(v, bi, s_v[q], s_i[q]);
      s_best = (v > 0.0) ? bi : -1;
      cval[buf * G + c] = (v > 0.0) ? v : 0.0;
      cidx[buf * G + c] = s_best;
    }
    __syncthreads();
    if (tid < w) {
      const long long b = s_best;
      crow[((long long)buf * G + c) * kLuPanel + tid] = (b >= 0) ? A[(long long)(j0 + tid) * n + b] : (T)0;
    }
    __threadfence();
    lu_grid_barrier(bar, status, limit);
    // (b) the winner, the same in every CTA (published copies read through L2)
    if (wp == 0) {
      double bv = -1.0;
      long long bw = LLONG_MAX;
      int bc = -1;
      for (int q = lane; q < G; q += 32) {
        const double vq = __ldcg(cval + buf * G + q);
        const long long iq = __ldcg(cidx + buf * G + q);
        if (iq >= 0 && (vq > bv || (vq == bv && iq < bw))) {
          bv = vq;
          bw = iq;
          bc = q;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const long long i2 = __shfl_xor_sync(0xffffffffu, bw, o);
        const int c2 = __shfl_xor_sync(0xffffffffu, bc, o);
        if (c2 >= 0 && (bc < 0 || v2 > bv || (v2 == bv && i2 < bw))) {
          bv = v2;
          bw = i2;
          bc = c2;
        }
      }
      if (lane == 0) {
        s_win = bc;
        s_best = bw;
        s_stop = (bc < 0 || !(bv > 0.0)) ? 1 : 0;
      }
    }
    __syncthreads();
    if (s_stop) break;  // no nonzero pivot left: the same decision in every CTA
    const long long p = s_best;
    if (tid < w) prow[tid] = __ldcg(crow + ((long long)buf * G + s_win) * kLuPanel + tid);
    if (tid == 0) {
      if (c == 0) {
        piv[j] = p;
        *rank = j + 1;
      }
      if (p >= r0 && p < r1) mark[p] = 1;
    }
    __syncthreads();
    // (c) eliminate column j from this CTA's unmarked rows
    const T pv = prow[jj];
    for (long long i = r0 + tid; i < r1; i += kLuThreads) {
      if (i == p || mark[i]) continue;
      const T m = colj[i] / pv;
      A[(long long)j * n + i] = m;
      for (int t = jj + 1; t < w; ++t) A[(long long)(j0 + t) * n + i] -= m * prow[t];
    }
    __syncthreads();
  }
}

// U12 (w x ncols, row-major) = L11^{-1} A(piv(j0 : j0 + w), j0 + w : k) with L11 the
// unit lower-triangular multipliers among the panel's pivot rows.
// Returns at once when the panel ended the selection early (its pivot list is then
// incomplete; the trailing update that follows only moves garbage no later step reads).
template <typename T>
__global__ void __launch_bounds__(128) k_lupp_u12(const T* __restrict__ A, long long n, int j0, int w, int k,
                                                  const long long* __restrict__ piv, const int* __restrict__ rank,
                                                  T* __restrict__ U12) {
  __shared__ T L11[kLuPanel][kLuPanel];
  __shared__ long long pr[kLuPanel];
  if (*rank < j0 + w) return;
  const int ncols = k - j0 - w;
  for (int e = threadIdx.x; e < w; e += blockDim.x) pr[e] = piv[j0 + e];
  __syncthreads();
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int a = e / w, b = e % w;
    L11[a][b] = (b < a) ? A[(long long)(j0 + b) * n + pr[a]] : (T)0;
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncols) return;
  T u[kLuPanel];
#pragma unroll
  for (int a = 0; a < kLuPanel; ++a) {
    if (a >= w) break;
    T x = A[(long long)(j0 + w + col) * n + pr[a]];
    for (int b = 0; b < a; ++b) x -= L11[a][b] * u[b];
    u[a] = x;
    U12[(long long)a * ncols + col] = x;
  }
}

// Forced sampling step (OSID): S_t = the next b_t entries of the skeleton list.
__global__ void k_forced_take(const long long* __restrict__ list, const int* __restrict__ count,
                              long long* __restrict__ S_t, State* st, int b) {
  pdl_wait();
  if (st->done) return;
  const long long k = st->k;
  long long bt = (long long)(*count) - k;
  if (bt > b) bt = b;
  if (bt > st->k_cap - k) bt = st->k_cap - k;
  if (bt < 0) bt = 0;
  for (long long e = threadIdx.x; e < bt; e += blockDim.x) S_t[e] = list[k + e];
  if (threadIdx.x == 0) {
    st->b_t = bt;
    st->sample_fallback = 0;
    if (bt == 0) st->done = 1;
  }
}

cudaError_t launch_forced_take(const long long* list, const int* count, long long* S_t, State* st, int b,
                               cudaStream_t s) {
  return counted(launch_pdl(k_forced_take, dim3(1), dim3(256), 0, s, list, count, S_t, st, b));
}

size_t lupp_scratch_bytes(int sms) {
  return (size_t)2 * sms * (8 + 8 + 8 * kLuPanel) + 64;
}

template <typename T>
cudaError_t launch_lupp(const T* Y, long long ldy, long long n, int k, T* A, T* U12, int* mark, long long* piv,
                        int* rank_status, void* scratch, int sms, unsigned limit, cudaStream_t s) {
  // scratch: bar (2 words) | cval (2 G doubles) | cidx (2 G) | crow (2 G x 32 T)
  unsigned int* bar = (unsigned int*)scratch;
  double* cval = (double*)((char*)scratch + 64);
  long long* cidx = (long long*)(cval + 2 * sms);
  T* crow = (T*)(cidx + 2 * sms);
  int* rank = rank_status;
  int* status = rank_status + 1;
  cudaError_t e;
  if ((e = cudaMemsetAsync(bar, 0, 8, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(mark, 0, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(rank_status, 0, 8, s)) != cudaSuccess) return e;
  k_lupp_load<T><<<dim3((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32)), 256, 0, s>>>(Y, ldy, n, k, A);
  if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
  for (int j0 = 0; j0 < k; j0 += kLuPanel) {
    const int w = std::min(kLuPanel, k - j0);
    {
      int jj0 = j0, ww = w;
      long long nn = n;
      T* AA = A;
      void* args[] = {(void*)&AA, (void*)&nn, (void*)&jj0, (void*)&ww, (void*)&mark, (void*)&piv, (void*)&rank,
                      (void*)&cval, (void*)&cidx, (void*)&crow, (void*)&bar, (void*)&status, (void*)&limit};
      e = cudaLaunchCooperativeKernel((const void*)k_lupp_panel<T>, dim3((unsigned)sms), dim3(kLuThreads), args, 0,
                                      s);
      if ((e = counted(e)) != cudaSuccess) return e;
    }
    const int ncols = k - j0 - w;
    if (ncols <= 0) break;
    k_lupp_u12<T><<<(ncols + 127) / 128, 128, 0, s>>>(A, n, j0, w, k, piv, rank, U12);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    // trailing update, transposed so that both operands and the result are read and
    // written along rows of A's columns: A(:, j0+w:)^T -= U12^T A(:, j0:j0+w)^T
    GemmArgs g;
    g.A = MatRef{U12, dim_const(0), 1, ncols};           // (c, a) -> U12[a * ncols + c]
    g.B = MatRef{A, dim_const((long long)j0 * n), n, 1};  // (a, i) -> A[(j0 + a) n + i]
    g.C = MatRef{A, dim_const((long long)(j0 + w) * n), n, 1};
    g.M = dim_const(ncols);
    g.N = dim_const(n);
    g.K = dim_const(w);
    g.alpha = -1.0;
    g.beta = 1.0;
    g.partial = nullptr;
    g.pm = ncols;
    g.pn = n;
    g.st = nullptr;
    if ((e = launch_gemm<T, T, T, T>(g, ncols, n, 1, kGemmTile, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_lupp<double>(const double*, long long, long long, int, double*, double*, int*, long long*,
                                         int*, void*, int, unsigned, cudaStream_t);
template cudaError_t launch_lupp<float>(const float*, long long, long long, int, float*, float*, int*, long long*,
                                        int*, void*, int, unsigned, cudaStream_t);

int lupp_panel_width() { return kLuPanel; }

// Largest number of k_lupp_panel CTAs that are co-resident (one per SM if that fits).
cudaError_t lupp_grid(int* sms) {
  int dev = 0, n_sm = 0, per = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lupp_panel<double>, kLuThreads, 0)) != cudaSuccess)
    return e;
  if (per < 1) return cudaErrorNotSupported;
  *sms = n_sm;
  return cudaSuccess;
}

}  // namespace rbrp
