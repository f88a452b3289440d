// Small dense products of the per-block chain (Alg. 2, projection to acceptance): the CGS2
// coefficients V Q^T, the corrections V -= C Q, and the Gram matrix V V^T.
// M is a block of b <= 256 rows, N and K are up to k_cap or d; too small for
// tensor-core tiles to pay, so these run on CUDA cores.
//
// Operands are stored as TS (FP32 on the plain TF32 path, FP64 otherwise);
// products, per-CTA sums and split partials are in TACC (FP32 on the mixed
// paths, FP64 on the FP64 path).  GB300 retires about two FP64 operations per
// clock per SM, so nothing on the FP32 paths touches FP64.  K is split over
// grid.z so that every SM gets work; each CTA writes its partial tile, and the
// last CTA of a tile to arrive (atomic counter) sums the partials in split
// order and applies C = alpha * sum + beta * C.  The sum
// order is fixed, so results do not depend on CTA scheduling, and no separate
// reduction launch is needed.  Counters are reset by the CTA that used them.
#include <cooperative_groups.h>
#include <limits.h>

#include <algorithm>

#include <atomic>

#include "rbrp_internal.cuh"

namespace rbrp {

namespace {

constexpr int KS = 32;  // K per shared-memory step

// 16 bytes of TS: two doubles or four floats.
template <typename TS>
struct alignas(16) Vec16 {
  static constexpr int N = 16 / (int)sizeof(TS);
  TS v[N];
};

// Row r, columns c .. c + N - 1 of a row-major array (zeros outside rlim x clim).
template <typename TS>
__device__ __forceinline__ Vec16<TS> ld16(const TS* P, long long r, long long c, long long rlim, long long clim,
                                          long long ld) {
  Vec16<TS> x;
  constexpr int N = Vec16<TS>::N;
  if (r >= rlim || c >= clim) {
#pragma unroll
    for (int t = 0; t < N; ++t) x.v[t] = (TS)0;
    return x;
  }
  const TS* p = P + r * ld + c;
  if (c + N <= clim) return *(const Vec16<TS>*)p;
#pragma unroll
  for (int t = 0; t < N; ++t) x.v[t] = (c + t < clim) ? p[t] : (TS)0;
  return x;
}

template <typename T, int R>
__device__ __forceinline__ void ld_vec(const T* p, T (&v)[R]) {
  if constexpr (sizeof(T) * R == 16) {
    const float4 x = *(const float4*)p;
    const T* t = (const T*)&x;
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
  } else if constexpr (sizeof(T) * R == 32) {
    const float4 x = *(const float4*)p, y = *(const float4*)(p + R / 2);
    const T* t0 = (const T*)&x;
    const T* t1 = (const T*)&y;
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      v[i] = t0[i];
      v[R / 2 + i] = t1[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = p[i];
  }
}

// The product of one TILE x TILE output tile over K range [kb, ke): thread
// (tx, ty) accumulates rows m0 + ty R + i, columns n0 + tx R + j in acc.
// TS: storage type of A, B; TACC: products and sums.  BKC: B is N x K with K
// contiguous (C = A B^T); otherwise K x N with N contiguous (C = A B,
// optionally with gathered rows).
template <typename TS, typename TACC, bool BKC, int TILE>
__device__ __forceinline__ void tile_product(const SgemmArgs& g, const TS* A, const TS* B, long long M, long long N,
                                             long long m0, long long n0, long long kb, long long ke,
                                             TACC (*As)[TILE + 4], TACC (*Bs)[TILE + 4],
                                             TACC (&acc)[TILE / 16][TILE / 16]) {
  constexpr int R = TILE / 16;              // outputs per thread along each axis
  constexpr int VN = Vec16<TS>::N;          // elements per 16-byte load
  constexpr int VPR = KS / VN;              // loads per K-row of a K-contiguous tile
  constexpr int NL = TILE * VPR / 256;      // loads per thread per operand and step
  static_assert(NL >= 1 && TILE * VPR % 256 == 0, "tile");
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = (TACC)0;

  Vec16<TS> ra[NL], rb[NL];
  auto load = [&](long long k0) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q;
      ra[q] = ld16<TS>(A, m0 + e / VPR, k0 + VN * (e % VPR), M, ke, g.lda);
      if (BKC) {
        rb[q] = ld16<TS>(B, n0 + e / VPR, k0 + VN * (e % VPR), N, ke, g.ldb);
      } else {
        long long kr = k0 + e / (TILE / VN);
        if (kr >= ke) kr = LLONG_MAX;
        else if (g.b_rows) kr = g.b_rows[kr];
        rb[q] = ld16<TS>(B, kr, n0 + VN * (e % (TILE / VN)), LLONG_MAX, N, g.ldb);
      }
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = tid + 256 * q;
      const int r = e / VPR, kv = e % VPR;
#pragma unroll
      for (int t = 0; t < VN; ++t) As[VN * kv + t][r] = (TACC)ra[q].v[t];
      if (BKC) {
#pragma unroll
        for (int t = 0; t < VN; ++t) Bs[VN * kv + t][r] = (TACC)rb[q].v[t];
      } else {
        const int kr = e / (TILE / VN), nv = e % (TILE / VN);
#pragma unroll
        for (int t = 0; t < VN; ++t) Bs[kr][VN * nv + t] = (TACC)rb[q].v[t];
      }
    }
  };

  if (kb < ke) load(kb);
  for (long long k0 = kb; k0 < ke; k0 += KS) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + KS < ke) load(k0 + KS);  // next step's loads overlap this step's products
#pragma unroll 8
    for (int kk = 0; kk < KS; ++kk) {
      TACC a[R], bv[R];
      ld_vec<TACC, R>(&As[kk][ty * R], a);
      ld_vec<TACC, R>(&Bs[kk][tx * R], bv);
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
  }
}

template <typename TS, typename TACC, bool BKC, int TILE>
__global__ void __launch_bounds__(256) k_sgemm(SgemmArgs g) {
  constexpr int R = TILE / 16;
  constexpr int LD = TILE + 4;
  if (g.st && g.st->done) return;
  const long long M = dim_val(g.M), N = dim_val(g.N), K = dim_val(g.K);
  const long long m0 = (long long)blockIdx.y * TILE, n0 = (long long)blockIdx.x * TILE;
  if (m0 >= M || n0 >= N) return;
  const TS* A = (const TS*)g.A + dim_val(g.a_off);
  const TS* B = (const TS*)g.B + dim_val(g.b_off);
  TS* C = (TS*)g.C + dim_val(g.c_off);
  const long long kb = (long long)blockIdx.z * g.kc;
  const long long ke = (kb + g.kc < K) ? kb + g.kc : K;
  __shared__ __align__(16) TACC As[KS][LD];
  __shared__ __align__(16) TACC Bs[KS][LD];
  __shared__ int s_last;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  TACC acc[R][R];
  tile_product<TS, TACC, BKC, TILE>(g, A, B, M, N, m0, n0, kb, ke, As, Bs, acc);

  const TS alpha = (TS)g.alpha, beta = (TS)g.beta;
  const int splits = (int)gridDim.z;
  if (splits == 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const long long gm = m0 + ty * R + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const long long gn = n0 + tx * R + j;
        if (gn >= N) continue;
        TS* cp = C + gm * g.ldc + gn;
        TS v = alpha * (TS)acc[i][j];
        if (g.beta != 0.0) v += beta * *cp;
        *cp = v;
      }
    }
    return;
  }
  const long long t = (long long)blockIdx.y * gridDim.x + blockIdx.x;
  TACC* Pall = (TACC*)g.partial;
  TACC* P = Pall + ((size_t)t * splits + blockIdx.z) * (TILE * TILE);
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) P[(ty * R + i) * TILE + tx * R + j] = acc[i][j];
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&g.cnt[t], 1u) == (unsigned)(splits - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // sum the partials in split order; the loads of four splits are issued
  // together so that their L2 latencies overlap
  const TACC* P0 = Pall + (size_t)t * splits * (TILE * TILE);
  TACC v[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) v[i][j] = (TACC)0;
  for (int z0 = 0; z0 < splits; z0 += 4) {
    TACC x[4][R][R];
#pragma unroll
    for (int zz = 0; zz < 4; ++zz) {
      const TACC* Pz = P0 + (size_t)(z0 + zz) * (TILE * TILE);
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j)
          x[zz][i][j] = (z0 + zz < splits) ? __ldcg(Pz + (ty * R + i) * TILE + tx * R + j) : (TACC)0;
    }
#pragma unroll
    for (int zz = 0; zz < 4; ++zz)
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) v[i][j] += x[zz][i][j];
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const long long gm = m0 + ty * R + i;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const long long gn = n0 + tx * R + j;
      if (gm < M && gn < N) {
        TS* cp = C + gm * g.ldc + gn;
        TS w = alpha * (TS)v[i][j];
        if (g.beta != 0.0) w += beta * *cp;
        *cp = w;
      }
    }
  }
  if (tid == 0) g.cnt[t] = 0u;
}

// FP32 accumulation with the K splits of a tile as one thread-block cluster
// (cluster rank = split index, gridDim.z = cluster size CS in {2, 4, 8, 16}):
// each CTA leaves its partial tile in shared memory; after a cluster barrier
// CTA r sums rows [r 64 / CS, (r + 1) 64 / CS) of the tile over the cluster's
// CTAs in rank order through distributed shared memory and writes them, and a
// second barrier keeps every CTA's shared memory alive until all have read
// it.  The sum order is fixed, and nothing goes through global memory but the
// operands and the result.
template <typename TS, bool BKC>
__global__ void __launch_bounds__(256) k_sgemm_cl(SgemmArgs g) {
  constexpr int TILE = 64, R = TILE / 16, LD = TILE + 4, LP = TILE + 1;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  pdl_wait();
  // every early exit below is taken by all CTAs of a cluster (same tile, same State)
  if (g.st && g.st->done) return;
  const long long M = dim_val(g.M), N = dim_val(g.N), K = dim_val(g.K);
  const long long m0 = (long long)blockIdx.y * TILE, n0 = (long long)blockIdx.x * TILE;
  if (m0 >= M || n0 >= N) return;
  const TS* A = (const TS*)g.A + dim_val(g.a_off);
  const TS* B = (const TS*)g.B + dim_val(g.b_off);
  TS* C = (TS*)g.C + dim_val(g.c_off);
  const long long kb = (long long)blockIdx.z * g.kc;
  const long long ke = (kb + g.kc < K) ? kb + g.kc : K;
  __shared__ __align__(16) float AB[2][KS][LD];  // operand stages; then this CTA's rows of the result
  __shared__ float P[TILE * LP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[R][R];
  tile_product<TS, float, BKC, TILE>(g, A, B, M, N, m0, n0, kb, ke, AB[0], AB[1], acc);
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) P[(ty * R + i) * LP + tx * R + j] = acc[i][j];
  cluster.sync();
  const int cs = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int rows = TILE / cs;
  const TS alpha = (TS)g.alpha, beta = (TS)g.beta;
  float* Vred = &AB[0][0][0];  // rows [rank rows, (rank + 1) rows) of the result tile (Gram form)
  for (int e = tid; e < rows * TILE; e += 256) {
    const int r = rank * rows + e / TILE, c = e % TILE;
    float v = 0.f;
    for (int z = 0; z < cs; ++z) v += cluster.map_shared_rank(P, z)[r * LP + c];
    const long long gm = m0 + r, gn = n0 + c;
    float out = 0.f;
    if (gm < M && gn < N) {
      TS* cp = C + gm * g.ldc + gn;
      TS w = alpha * (TS)v;
      if (g.beta != 0.0) w += beta * *cp;
      *cp = w;
      out = (float)w;
    }
    if (g.gram) Vred[e] = out;
  }
  cluster.sync();
  if (!g.gram) return;
  // Gram partial of this column tile: the whole 64 x 64 result tile into P (read from
  // the cluster's CTAs), then this CTA's rows of T T^T; every row pair is summed over
  // c in the same order, so the partial is exactly symmetric
  for (int e = tid; e < TILE * TILE; e += 256) {
    const int r = e / TILE, c = e % TILE, z = r / rows;
    P[r * LP + c] = cluster.map_shared_rank(Vred, z)[(r - z * rows) * TILE + c];
  }
  cluster.sync();  // every CTA has copied the others' rows
  float* gt = g.gram + (size_t)blockIdx.x * (TILE * TILE);
  for (int e = tid; e < rows * TILE; e += 256) {
    const int i = rank * rows + e / TILE, j = e % TILE;
    const float* pi = P + i * LP;
    const float* pj = P + j * LP;
    float sum = 0.f;
#pragma unroll 8
    for (int c = 0; c < TILE; ++c) sum = fmaf(pi[c], pj[c], sum);
    gt[i * TILE + j] = sum;
  }
}

}  // namespace

int sgemm_tile(int acc_fp64) { return acc_fp64 ? 32 : 64; }

// Cluster size (power of two, <= 16) for FP32 split-K products: about
// `target` CTAs over the (Mmax x Nmax) tiles of 64, and K per split a
// multiple of KS.
void sgemm_cluster(long long Mmax, long long Nmax, long long Kmax, long long target, int* cs, int* kc) {
  const long long tiles = ((Mmax + 63) / 64) * ((Nmax + 63) / 64);
  int c = 1;
  while (c < 16 && tiles * c < target && (long long)(c * 2) * KS <= std::max<long long>(Kmax, KS)) c *= 2;
  long long k = (Kmax + c - 1) / c;
  k = std::max<long long>(KS, (k + KS - 1) / KS * KS);
  *cs = c;
  *kc = (int)k;
}

template <typename TS, bool BKC>
cudaError_t launch_sgemm_cluster(const SgemmArgs& g, long long Mmax, long long Nmax, int cs, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_sgemm_cl<TS, BKC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((Nmax + 63) / 64), (unsigned)((Mmax + 63) / 64), (unsigned)cs);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = (unsigned)cs;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // the kernel starts with pdl_wait()
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  if (cs > 8) {
    // 16 CTAs per cluster is beyond the portable size: use it only where the
    // device can hold such a cluster (asked once per process), else two
    // splits per CTA
    static std::atomic<int> ok16{-1};
    if (ok16 < 0) {
      int nclusters = 0;
      ok16 = (cudaOccupancyMaxActiveClusters(&nclusters, k_sgemm_cl<TS, BKC>, &cfg) == cudaSuccess && nclusters >= 1);
      (void)cudaGetLastError();
    }
    if (!ok16) {
      SgemmArgs g2 = g;
      g2.kc = g.kc * 2;
      at[0].val.clusterDim.z = 8;
      cfg.gridDim.z = 8;
      return counted(cudaLaunchKernelEx(&cfg, k_sgemm_cl<TS, BKC>, g2));
    }
  }
  return counted(cudaLaunchKernelEx(&cfg, k_sgemm_cl<TS, BKC>, g));
}

template cudaError_t launch_sgemm_cluster<float, true>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm_cluster<float, false>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm_cluster<double, true>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm_cluster<double, false>(const SgemmArgs&, long long, long long, int, cudaStream_t);

// K per split (multiple of KS) and the resulting number of splits for about
// `target` CTAs over the (Mmax x Nmax) tiles.
void sgemm_splits(long long Mmax, long long Nmax, long long Kmax, int tile, long long target, int* splits,
                  int* kc) {
  const long long tiles = ((Mmax + tile - 1) / tile) * ((Nmax + tile - 1) / tile);
  long long s = std::max(1LL, (target + tiles - 1) / std::max(1LL, tiles));
  long long k = (Kmax + s - 1) / s;
  k = std::max<long long>(KS, (k + KS - 1) / KS * KS);
  *kc = (int)k;
  *splits = (int)std::max(1LL, (Kmax + k - 1) / k);
}

template <typename TS, typename TACC, bool BKC>
cudaError_t launch_sgemm(const SgemmArgs& g, long long Mmax, long long Nmax, int splits, cudaStream_t s) {
  constexpr int TILE = sizeof(TACC) == 8 ? 32 : 64;
  dim3 grid((unsigned)((Nmax + TILE - 1) / TILE), (unsigned)((Mmax + TILE - 1) / TILE), (unsigned)splits);
  k_sgemm<TS, TACC, BKC, TILE><<<grid, 256, 0, s>>>(g);
  return counted(cudaGetLastError());
}

template cudaError_t launch_sgemm<float, float, true>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm<float, float, false>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm<double, float, true>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm<double, float, false>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm<double, double, true>(const SgemmArgs&, long long, long long, int, cudaStream_t);
template cudaError_t launch_sgemm<double, double, false>(const SgemmArgs&, long long, long long, int, cudaStream_t);

}  // namespace rbrp
