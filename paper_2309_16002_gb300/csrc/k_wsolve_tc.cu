// Interpolation matrix of Alg. 3 on Blackwell tensor cores (sm_103a).
//
// W L1 = L with L1 = L(S, :) lower triangular (Sec. 5.1) is solved by blocks of
// 64 columns from the right: for J = [j0, j0 + nb) and J+ = [j0 + nb, k),
//   W(:, J) = (L(:, J) - W(:, J+) L1(J+, J)) L1(J, J)^{-1}.
// One launch per block J; each CTA owns 128 rows.  The product W(:, J+) L1(J+, J)
// runs on tcgen05 (kind::tf32, FP32 accumulators in TMEM) in the 3xTF32 form
// (hi*hi + hi*lo + lo*hi, ~FP32 accuracy), with W(:, J+) staged by TMA and
// split into hi/lo in shared memory and L1^T precomputed as hi/lo.  The
// epilogue (one thread per row) subtracts the product from L(:, J) and solves
// with the 64 x 64 triangle L1(J, J) held in shared memory, writing W(:, J).
// The result is an FP32 W (the RBRP_W_FP32 solve).  Every mbarrier wait is
// bounded (RBRP_ETIMEOUT, as in the update kernel).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rbrp_internal.cuh"
#include "tc_common.cuh"

namespace rbrp {
namespace tc {

constexpr int WM = 128;   // rows per tile (MMA M)
constexpr int WN = 64;    // column block (MMA N)
constexpr int WK = 32;    // K chunk: 128 bytes of FP32
constexpr int WS = 3;     // pipeline stages
constexpr int kWThreads = 320;  // producer, MMA, 4 epilogue warps, 4 converter warps
constexpr int kDiagLd = WN + 1;  // padded row of a staged diagonal block

struct WCfg {
  static constexpr int A = WM * WK * 4;             // W(:, J+) chunk (16 KB), hi; lo follows
  static constexpr int B = WN * WK * 4;             // L1^T chunk (8 KB), hi; lo follows
  static constexpr int ST = 2 * A + 2 * B;          // [A hi][A lo][B hi][B lo]
  static constexpr int P = WS * ST;
  static constexpr int LS_OFF = P;                  // L1(J, J) as FP32 (64 x 65) and 64 reciprocals
  static constexpr int LS_BYTES = (WN * kDiagLd + WN) * 4;
  static constexpr int WR_OFF = LS_OFF + ((LS_BYTES + 1023) / 1024) * 1024;  // per-thread rows of W(:, J)
  static constexpr int WR_BYTES = WM * kDiagLd * 4;
  static constexpr int BAR_OFF = WR_OFF + ((WR_BYTES + 1023) / 1024) * 1024;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;
};

template <typename TL>
__global__ void __launch_bounds__(kWThreads, 1)
    k_wsolve_tc(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmBlo, const TL* __restrict__ L, long long ldl,
                float* __restrict__ W, long long ldw, double* __restrict__ W64, long long ldw64,
                const float* __restrict__ Ldiag, long long n, long long k, int j0, int nb, State* st) {
  using C = WCfg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(smem);
  const uint32_t sBar = sb + C::BAR_OFF;
  auto full = [&](int s) { return sBar + 8u * s; };
  auto empty = [&](int s) { return sBar + 8u * (WS + s); };
  auto conv = [&](int s) { return sBar + 8u * (2 * WS + s); };
  auto d_full = [&](int b) { return sBar + 8u * (3 * WS + b); };
  auto d_empty = [&](int b) { return sBar + 8u * (3 * WS + 2 + b); };
  uint32_t* tmem_slot = (uint32_t*)(smem + C::BAR_OFF + 8 * (3 * WS + 4));
  float* Ls = (float*)(smem + C::LS_OFF);           // Ls[a * 65 + c] = L1(j0 + a, j0 + c)
  float* rinv = Ls + WN * kDiagLd;

  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j1 = j0 + nb;
  const int K = (int)(k - j1);
  const int nK = (K + WK - 1) / WK;
  const long long ntiles = (n + WM - 1) / WM;

  // the diagonal triangle L1(J, J) and its reciprocals (FP32, prepared once per solve)
  {
    const float* src = Ldiag + (long long)(j0 / WN) * (WN * kDiagLd + WN);
    for (int e = threadIdx.x; e < WN * kDiagLd + WN; e += kWThreads) Ls[e] = src[e];
  }
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < WS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
      mbar_init(conv(s), 128);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(d_full(b), 1);
      mbar_init(d_empty(b), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *(volatile uint32_t*)tmem_slot;
  volatile int* abort = &s_abort;

  if (warp == 0) {
    // ---------------- TMA producer: the chunk ring runs on across this CTA's tiles
    if (lane == 0 && nK > 0) {
      long long g = 0;
      for (long long tile = blockIdx.x; tile < ntiles && !*abort; tile += gridDim.x) {
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int s = (int)(g % WS);
          const uint32_t ph = (uint32_t)(g / WS) & 1u;
          if (!mbar_wait(empty(s), ph ^ 1u, abort)) break;
          mbar_expect_tx(full(s), (uint32_t)(C::A + 2 * C::B));
          const uint32_t base = sb + s * C::ST;
          const int x = j1 + kc * WK;
          tma_load_2d(base, &tmW, full(s), x, (int)(tile * WM));
          tma_load_2d(base + 2 * C::A, &tmB, full(s), x, j0);
          tma_load_2d(base + 2 * C::A + C::B, &tmBlo, full(s), x, j0);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: tile `it` accumulates into TMEM buffer it & 1
    if (lane == 0) {
      const uint32_t id = idesc_tf32(WM, WN);
      long long g = 0;
      int it = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        if (!mbar_wait(d_empty(buf), (uint32_t)((it >> 1) & 1) ^ 1u, abort)) break;
        tc_after();
        const uint32_t dt = tmem + (uint32_t)(buf * WN);
        bool ok = true;
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int s = (int)(g % WS);
          const uint32_t ph = (uint32_t)(g / WS) & 1u;
          if (!mbar_wait(full(s), ph, abort) || !mbar_wait(conv(s), ph, abort)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t a = sb + s * C::ST, alo = a + C::A, b = a + 2 * C::A, blo = b + C::B;
#pragma unroll
          for (int kk = 0; kk < WK / 8; ++kk) {
            mma_tf32(dt, sdesc(a + kk * 32), sdesc(b + kk * 32), id, (kc | kk) != 0 ? 1u : 0u);
            mma_tf32(dt, sdesc(a + kk * 32), sdesc(blo + kk * 32), id, 1u);
            mma_tf32(dt, sdesc(alo + kk * 32), sdesc(b + kk * 32), id, 1u);
          }
          mma_commit(empty(s));
        }
        if (!ok) break;
        if (nK > 0)
          mma_commit(d_full(buf));
        else
          mbar_arrive(d_full(buf));
      }
    }
  } else if (warp >= 6) {
    // ---------------- warps 6-9: split every A chunk into TF32 hi (in place) and lo
    const int r = threadIdx.x - 192;  // 0..127, one tile row each
    long long g = 0;
    for (long long tile = blockIdx.x; tile < ntiles && nK > 0; tile += gridDim.x) {
      bool ok = true;
      for (int kc = 0; kc < nK; ++kc, ++g) {
        const int s = (int)(g % WS);
        const uint32_t ph = (uint32_t)(g / WS) & 1u;
        if (!mbar_wait(full(s), ph, abort)) {
          ok = false;
          break;
        }
        uint8_t* a = smem + s * C::ST + (r >> 3) * 1024 + (r & 7) * 128;
        uint8_t* alo = a + C::A;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const float4 x = *(float4*)(a + ch * 16);
          const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
          *(float4*)(a + ch * 16) = h;
          *(float4*)(alo + ch * 16) = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
        fence_async_smem();
        mbar_arrive(conv(s));
      }
      if (!ok) break;
    }
  } else {
    // ---------------- warps 2-5: per-row epilogue and triangular solve, one tile at a time
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    // this thread's row of the right-hand side, in shared memory (stride 65: conflict-free)
    float* wr = (float*)(smem + C::WR_OFF) + r * kDiagLd;
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int buf = it & 1;
      const long long row = tile * WM + r;
      if (!mbar_wait(d_full(buf), (uint32_t)(it >> 1) & 1u, abort)) break;
      tc_after();
      if (nK > 0) {
        uint32_t v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(buf * WN), v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) wr[j] = -__uint_as_float(v[j]);
        tmem_ld32(tmem + lane_base + (uint32_t)(buf * WN) + 32u, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) wr[32 + j] = -__uint_as_float(v[j]);
      } else {
        for (int j = 0; j < WN; ++j) wr[j] = 0.f;
      }
      tc_before();
      mbar_arrive(d_empty(buf));  // the TMEM buffer may take the tile after next
      if (row < n) {
        const TL* lrow = L + row * ldl + j0;
        for (int j = 0; j < nb; ++j) wr[j] += (float)lrow[j];
        // w L1(J, J) = rhs with L1(J, J) lower triangular: columns from the last to the first
#pragma unroll 1
        for (int j = nb - 1; j >= 0; --j) {
          float s0 = wr[j], s1 = 0.f;
          int m = j + 1;
#pragma unroll 2
          for (; m + 1 < nb; m += 2) {
            s0 -= wr[m] * Ls[m * kDiagLd + j];
            s1 -= wr[m + 1] * Ls[(m + 1) * kDiagLd + j];
          }
          if (m < nb) s0 -= wr[m] * Ls[m * kDiagLd + j];
          wr[j] = (s0 + s1) * rinv[j];
        }
        float* wrow = W + row * ldw + j0;
        double* w64 = W64 + row * ldw64 + j0;
        for (int j = 0; j < nb; ++j) {
          wrow[j] = wr[j];
          w64[j] = (double)wr[j];
        }
      }
    }
  }

  tc_before();
  __syncthreads();
  if (s_abort) {
    for (int i = 0; i < 64; ++i) __nanosleep(1000);
    if (threadIdx.x == 0) {
      st->status = RBRP_ETIMEOUT;
      st->done = 1;
    }
  }
  if (warp == 1) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
  }
}

// L1T_hi / L1T_lo (k x ld FP32): hi/lo split of L1^T, L1T(c, r) = L1(r, c).
__global__ void k_l1t_split(const double* __restrict__ L1, long long ld1, long long k, float* __restrict__ hi,
                            float* __restrict__ lo, long long ld) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < k * ld; e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / ld, r = e % ld;
    const double v = (r < k) ? L1[r * ld1 + c] : 0.0;
    const float h = tf32_hi((float)v);
    hi[e] = h;
    lo[e] = (float)(v - (double)h);
  }
}

// FP32 copies of the 64 x 64 diagonal blocks of L1 (row stride 65) followed by
// the 64 reciprocals of their diagonals, one record per column block.
__global__ void k_l1_diag(const double* __restrict__ L1, long long ld1, long long k, float* __restrict__ Ldiag,
                          long long nblk) {
  const long long per = WN * kDiagLd + WN;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nblk * per; e += (long long)gridDim.x * blockDim.x) {
    const long long J = e / per, off = e % per, j0 = J * WN;
    float v = 0.f;
    if (off < WN * kDiagLd) {
      const long long a = off / kDiagLd, c = off % kDiagLd;
      if (c < WN && j0 + a < k && j0 + c < k) v = (float)L1[(j0 + a) * ld1 + j0 + c];
    } else {
      const long long j = off - WN * kDiagLd;
      if (j0 + j < k) v = (float)(1.0 / L1[(j0 + j) * ld1 + j0 + j]);
    }
    Ldiag[e] = v;
  }
}

template <typename TL>
cudaError_t wsolve_all(const TL* L, long long ldl, float* W, long long ldw, double* W64, long long ldw64,
                       const double* L1, long long ld1, float* L1T_hi, float* L1T_lo, long long ldt, float* Ldiag,
                       long long n, long long k, State* st, cudaStream_t s) {
  using C = WCfg;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_wsolve_tc<TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  {
    long long tot = k * ldt;
    unsigned g = (unsigned)((tot + 255) / 256);
    if (g > 8192) g = 8192;
    k_l1t_split<<<g, 256, 0, s>>>(L1, ld1, k, L1T_hi, L1T_lo, ldt);
    cudaError_t e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
    const long long nb_all = (k + WN - 1) / WN;
    k_l1_diag<<<(unsigned)((nb_all * (WN * kDiagLd + WN) + 255) / 256), 256, 0, s>>>(L1, ld1, k, Ldiag, nb_all);
    e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
  }
  CUtensorMap mW, mB, mBlo;
  if (!make_map(&mW, W, k, n, ldw * 4, WK, WM)) return cudaErrorInvalidValue;
  if (!make_map(&mB, L1T_hi, k, k, ldt * 4, WK, WN)) return cudaErrorInvalidValue;
  if (!make_map(&mBlo, L1T_lo, k, k, ldt * 4, WK, WN)) return cudaErrorInvalidValue;
  int sms = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const long long ntiles = (n + WM - 1) / WM;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);  // persistent: one CTA per SM
  const long long nblk = (k + WN - 1) / WN;
  for (long long J = nblk - 1; J >= 0; --J) {
    const int j0 = (int)(J * WN);
    const int nb = (int)((k - j0 < WN) ? (k - j0) : WN);
    k_wsolve_tc<TL><<<grid, kWThreads, C::SMEM, s>>>(mW, mB, mBlo, L, ldl, W, ldw, W64, ldw64, Ldiag, n, k, j0, nb,
                                                     st);
    cudaError_t e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace tc

size_t wsolve_diag_floats(long long k) { return (size_t)((k + tc::WN - 1) / tc::WN) * (tc::WN * tc::kDiagLd + tc::WN); }

cudaError_t launch_wsolve_tc(const void* L, int l_is_fp64, long long ldl, float* W, long long ldw, double* W64,
                             long long ldw64, const double* L1, long long ld1, float* L1T_hi, float* L1T_lo,
                             long long ldt, float* Ldiag, long long n, long long k, State* st, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  if (l_is_fp64)
    return tc::wsolve_all<double>((const double*)L, ldl, W, ldw, W64, ldw64, L1, ld1, L1T_hi, L1T_lo, ldt, Ldiag, n,
                                  k, st, s);
  return tc::wsolve_all<float>((const float*)L, ldl, W, ldw, W64, ldw64, L1, ld1, L1T_hi, L1T_lo, ldt, Ldiag, n, k,
                               st, s);
}

}  // namespace rbrp
