// Interpolation matrix of Alg. 3 on Blackwell tensor cores (sm_103a).
//
// W L1 = L with L1 = L(S, :) lower triangular (Sec. 5.1) is solved by blocks
// of 64 columns from the right.  With J = [j0, j0 + 64), J+ = [j0 + 64, k) and
// T_J = L1(J, J):
//   W(:, J) = (L(:, J) - W(:, J+) L1(J+, J)) T_J^{-1}
//           = [L(:, J) | W(:, J+)] G(J u J+, J),
//   G(J, J) = T_J^{-1},  G(J+, J) = -L1(J+, J) T_J^{-1}.
// k_wsolve_g forms G once (FP32; one 64-wide row solve with T_J per row of G),
// so each block of W is a single product and no substitution runs on the n
// rows of W.
//
// k_wsolve_rows is persistent: a CTA owns 128-row tiles of W and runs every
// block J of a tile from the right, so W(tile, J+) -- written by the same CTA
// shortly before, split into TF32 hi/lo -- is re-read from L2 rather than HBM.
// The products run on tcgen05 (kind::tf32) in the 3xTF32 form (hi*hi + hi*lo +
// lo*hi, about FP32 accuracy) with FP32 accumulators in TMEM, double-buffered:
// the MMAs of block J start on L(tile, J) and W(tile, J+2 ...) while the
// epilogue drains block J+1.  The newest block W(tile, J+1) does not go through
// global memory before block J uses it: the epilogue writes it, split, into
// shared memory in the MMA operand layout; the MMA reads it last; the producer
// then stores it (TMA) for the blocks further left.  The epilogue also writes
// the FP64 result rows.
//
// Roles (320 threads): warp 0 lane 0 issues TMA loads and stores, warp 1 owns
// TMEM and lane 0 issues the MMAs, warps 2-5 (one row each) are the epilogue,
// warps 6-9 split the L chunks into hi/lo in place.  Every mbarrier wait is
// bounded: after the limit the CTA records RBRP_ETIMEOUT in the State, stops,
// drains the TMA fills and MMAs it issued (each with a bounded wait), frees its
// TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "rbrp_internal.cuh"
#include "tc_common.cuh"

namespace rbrp {
namespace tc {

constexpr int WM = 128;         // rows per tile (MMA M)
constexpr int WN = 64;          // column block (MMA N)
constexpr int WK = 32;          // K chunk: 128 bytes of FP32
constexpr int WS = 3;           // pipeline stages
constexpr int kWThreads = 320;  // producer, MMA, 4 epilogue warps, 4 converter warps

struct WCfg {
  static constexpr int A = WM * WK * 4;     // A chunk (16 KB), hi; lo follows
  static constexpr int B = WN * WK * 4;     // G^T chunk (8 KB), hi; lo follows
  static constexpr int ST = 2 * A + 2 * B;  // [A hi][A lo][B hi][B lo]
  static constexpr int P = WS * ST;
  static constexpr int F_OFF = P;           // newest block: [c0 hi][c0 lo][c1 hi][c1 lo]
  static constexpr int BAR_OFF = F_OFF + 4 * A;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;
};
static_assert(WCfg::SMEM <= 227 * 1024, "shared memory");

// The K chunks of block J in MMA order: L(:, J); W(:, J+) beyond block J+1
// (from global memory); W(:, J+1) (from shared memory).
struct WSeq {
  int j0, nL, nW, nF, wx;
  __device__ __forceinline__ WSeq(int J, int k) {
    j0 = J * WN;
    const int nb = min(WN, k - j0);
    nL = (nb + WK - 1) / WK;
    wx = j0 + 2 * WN;
    nW = wx < k ? (k - wx + WK - 1) / WK : 0;
    nF = (j0 + WN < k) ? (min(WN, k - j0 - WN) + WK - 1) / WK : 0;
  }
  __device__ __forceinline__ int n() const { return nL + nW + nF; }
  // 0: L(:, J), 1: W from global memory, 2: W(:, J+1) from shared memory
  __device__ __forceinline__ int kind(int i) const { return i < nL ? 0 : (i < nL + nW ? 1 : 2); }
  __device__ __forceinline__ int x(int i) const {
    return i < nL ? j0 + WK * i : (i < nL + nW ? wx + WK * (i - nL) : j0 + WN + WK * (i - nL - nW));
  }
};

template <bool L64>
__global__ void __launch_bounds__(kWThreads, 1)
    k_wsolve_rows(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmWh,
                  const __grid_constant__ CUtensorMap tmWl, const __grid_constant__ CUtensorMap tmGh,
                  const __grid_constant__ CUtensorMap tmGl, double* __restrict__ W64, long long ldw64, int w64_vec,
                  int n, int k, State* st) {
  using C = WCfg;
  pdl_wait();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(smem);
  const uint32_t sBar = sb + C::BAR_OFF;
  auto full = [&](int s) { return sBar + 8u * s; };
  auto empty = [&](int s) { return sBar + 8u * (WS + s); };
  auto conv = [&](int s) { return sBar + 8u * (2 * WS + s); };
  auto d_full = [&](int b) { return sBar + 8u * (3 * WS + b); };
  auto d_empty = [&](int b) { return sBar + 8u * (3 * WS + 2 + b); };
  const uint32_t f_full = sBar + 8u * (3 * WS + 4);  // epilogue -> MMA, producer: newest block written
  const uint32_t f_free = sBar + 8u * (3 * WS + 5);  // producer -> epilogue: its TMA store has read it
  uint32_t* tmem_slot = (uint32_t*)(smem + C::BAR_OFF + 8 * (3 * WS + 6));
  const uint32_t drain = sBar + 8u * (3 * WS + 7);  // abort path: MMA drain

  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblk = (k + WN - 1) / WN;
  const int ntiles = (n + WM - 1) / WM;

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
    mbar_init(f_full, 128);
    mbar_init(f_free, 1);
    mbar_init(drain, 1);
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
  const uint32_t lim = st->spin_mbar;
  uint32_t fills = 0;  // TMA fills issued by the producer (for the abort drain)

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      const uint64_t keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
      uint32_t g = 0, f = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int y = tile * WM;
        for (int J = nblk - 1; J >= 0 && ok; --J) {
          const WSeq q(J, k);
          for (int i = 0; i < q.n(); ++i, ++g) {
            const int kind = q.kind(i), x = q.x(i);
            if (kind == 1 && i == q.nL) tma_wait_all0();  // the stores of W(tile, J+2 ...) are complete
            const int s = (int)(g % WS);
            const uint32_t ph = (g / WS) & 1u;
            if (!mbar_wait(empty(s), ph ^ 1u, abort, lim)) {
              ok = false;
              break;
            }
            const uint32_t base = sb + s * C::ST;
            const uint32_t abytes = kind == 2 ? 0u : ((kind == 0 && !L64) ? (uint32_t)C::A : 2u * C::A);
            mbar_expect_tx(full(s), abytes + 2u * C::B);
            if (kind == 0) {
              tma_load_2d_hint(base, &tmL, full(s), x, y, stream);
              if (L64) tma_load_2d_hint(base + C::A, &tmL, full(s), x + 16, y, stream);
            } else if (kind == 1) {
              tma_load_2d_hint(base, &tmWh, full(s), x, y, keep);
              tma_load_2d_hint(base + C::A, &tmWl, full(s), x, y, keep);
            }
            tma_load_2d_hint(base + 2 * C::A, &tmGh, full(s), x, q.j0, keep);
            tma_load_2d_hint(base + 2 * C::A + C::B, &tmGl, full(s), x, q.j0, keep);
          }
          if (!ok || q.nF == 0) continue;
          // W(tile, J+1) for the blocks left of J (none after J = 0)
          if (!mbar_wait(f_full, f & 1u, abort, lim)) {
            ok = false;
            break;
          }
          if (J > 0) {
            for (int c = 0; c < q.nF; ++c) {
              const uint32_t fb = sb + C::F_OFF + c * 2 * C::A;
              tma_store_2d_hint(&tmWh, fb, q.j0 + WN + c * WK, y, keep);
              tma_store_2d_hint(&tmWl, fb + C::A, q.j0 + WN + c * WK, y, keep);
            }
            tma_commit();
            tma_wait_read0();
          }
          mbar_arrive(f_free);
          ++f;
        }
      }
      fills = g;
      tma_wait_all0();
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer; block `it` of this CTA accumulates in TMEM buffer it & 1
    if (lane == 0) {
      const uint32_t id = idesc_tf32(WM, WN);
      uint32_t g = 0, f = 0, it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int J = nblk - 1; J >= 0; --J, ++it) {
          const WSeq q(J, k);
          const int buf = it & 1;
          if (!mbar_wait(d_empty(buf), ((it >> 1) & 1u) ^ 1u, abort, lim)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t dt = tmem + (uint32_t)(buf * WN);
          for (int i = 0; i < q.n(); ++i, ++g) {
            const int kind = q.kind(i);
            const int s = (int)(g % WS);
            const uint32_t ph = (g / WS) & 1u;
            if (!mbar_wait(full(s), ph, abort, lim)) {
              ok = false;
              break;
            }
            // every chunk passes the converters (which split the L chunks), so
            // none of them can fall a whole ring behind
            if (!mbar_wait(conv(s), ph, abort, lim)) {
              ok = false;
              break;
            }
            if (kind == 2 && i == q.nL + q.nW) {
              if (!mbar_wait(f_full, f & 1u, abort, lim)) {
                ok = false;
                break;
              }
            }
            tc_after();
            const uint32_t sbase = sb + s * C::ST;
            const uint32_t a = kind == 2 ? sb + C::F_OFF + (uint32_t)((i - q.nL - q.nW) * 2 * C::A) : sbase;
            const uint32_t alo = a + C::A, b = sbase + 2 * C::A, blo = b + C::B;
#pragma unroll
            for (int kk = 0; kk < WK / 8; ++kk) {
              mma_tf32(dt, sdesc(a + kk * 32), sdesc(b + kk * 32), id, (i | kk) != 0 ? 1u : 0u);
              mma_tf32(dt, sdesc(a + kk * 32), sdesc(blo + kk * 32), id, 1u);
              mma_tf32(dt, sdesc(alo + kk * 32), sdesc(b + kk * 32), id, 1u);
            }
            mma_commit(empty(s));
          }
          if (!ok) break;
          if (q.nF > 0) ++f;
          mma_commit(d_full(buf));
        }
      }
    }
  } else if (warp >= 6) {
    // ---------------- warps 6-9: split each L chunk into TF32 hi (in place) and lo;
    // pass the other chunks on
    const int r = threadIdx.x - 192;  // 0..127, one tile row each
    const int r7 = r & 7;
    uint32_t g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int J = nblk - 1; J >= 0 && ok; --J) {
        const WSeq q(J, k);
        for (int i = 0; i < q.n(); ++i, ++g) {
          const int s = (int)(g % WS);
          if (!mbar_wait(full(s), (g / WS) & 1u, abort, lim)) {
            ok = false;
            break;
          }
          if (q.kind(i) != 0) {
            mbar_arrive(conv(s));
            continue;
          }
          uint8_t* a = smem + s * C::ST + (r >> 3) * 1024 + r7 * 128;  // this row, 128-byte swizzled
          uint8_t* alo = a + C::A;
          if (L64) {
            // FP64 columns 0-15 sit in the hi region, 16-31 in the lo region
            double v[32];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const double2 u0 = *(const double2*)(a + ((c ^ r7) << 4));
              const double2 u1 = *(const double2*)(alo + ((c ^ r7) << 4));
              v[2 * c] = u0.x;
              v[2 * c + 1] = u0.y;
              v[16 + 2 * c] = u1.x;
              v[16 + 2 * c + 1] = u1.y;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              float h[4], l[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                h[e] = tf32_rn((float)v[4 * c + e]);
                l[e] = tf32_rn((float)(v[4 * c + e] - (double)h[e]));
              }
              *(float4*)(a + ((c ^ r7) << 4)) = make_float4(h[0], h[1], h[2], h[3]);
              *(float4*)(alo + ((c ^ r7) << 4)) = make_float4(l[0], l[1], l[2], l[3]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const uint32_t o = (uint32_t)((c ^ r7) << 4);  // distinct banks across 8 consecutive rows
              const float4 x = *(const float4*)(a + o);
              const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
              *(float4*)(a + o) = h;
              *(float4*)(alo + o) = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
            }
          }
          fence_async_smem();
          mbar_arrive(conv(s));
        }
      }
    }
  } else {
    // ---------------- warps 2-5: epilogue, one row of the tile per thread
    const int q4 = warp & 3;
    const int r = 32 * q4 + lane;
    const int r7 = r & 7;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    uint32_t it = 0, f = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const long long row = (long long)tile * WM + r;
      for (int J = nblk - 1; J >= 0; --J, ++it) {
        const int buf = it & 1;
        if (!mbar_wait(d_full(buf), (it >> 1) & 1u, abort, lim)) {
          ok = false;
          break;
        }
        tc_after();
        uint32_t v0[32], v1[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(buf * WN), v0);
        tmem_ld32(tmem + lane_base + (uint32_t)(buf * WN) + 32u, v1);
        tmem_wait_ld();
        tc_before();
        mbar_arrive(d_empty(buf));
        if (J > 0) {
          // W(tile, J) as the MMA operand of block J-1 (hi/lo, 128-byte swizzle)
          if (f > 0 && !mbar_wait(f_free, (f - 1) & 1u, abort, lim)) {
            ok = false;
            break;
          }
          uint8_t* fr = smem + C::F_OFF + (r >> 3) * 1024 + r7 * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint32_t o = (uint32_t)((c ^ r7) << 4);
            const float4 x0 = make_float4(__uint_as_float(v0[4 * c]), __uint_as_float(v0[4 * c + 1]),
                                          __uint_as_float(v0[4 * c + 2]), __uint_as_float(v0[4 * c + 3]));
            const float4 x1 = make_float4(__uint_as_float(v1[4 * c]), __uint_as_float(v1[4 * c + 1]),
                                          __uint_as_float(v1[4 * c + 2]), __uint_as_float(v1[4 * c + 3]));
            const float4 h0 = make_float4(tf32_rn(x0.x), tf32_rn(x0.y), tf32_rn(x0.z), tf32_rn(x0.w));
            const float4 h1 = make_float4(tf32_rn(x1.x), tf32_rn(x1.y), tf32_rn(x1.z), tf32_rn(x1.w));
            *(float4*)(fr + o) = h0;
            *(float4*)(fr + C::A + o) =
                make_float4(tf32_rn(x0.x - h0.x), tf32_rn(x0.y - h0.y), tf32_rn(x0.z - h0.z), tf32_rn(x0.w - h0.w));
            *(float4*)(fr + 2 * C::A + o) = h1;
            *(float4*)(fr + 3 * C::A + o) =
                make_float4(tf32_rn(x1.x - h1.x), tf32_rn(x1.y - h1.y), tf32_rn(x1.z - h1.z), tf32_rn(x1.w - h1.w));
          }
          fence_async_smem();
          mbar_arrive(f_full);
          ++f;
        }
        if (row < n) {
          const int j0 = J * WN;
          const int nb = min(WN, k - j0);
          double* w = W64 + row * ldw64 + j0;
          if (w64_vec && nb == WN) {
#pragma unroll
            for (int c = 0; c < 16; ++c)
              __stcs((double2*)w + c,
                     make_double2((double)__uint_as_float(v0[2 * c]), (double)__uint_as_float(v0[2 * c + 1])));
#pragma unroll
            for (int c = 0; c < 16; ++c)
              __stcs((double2*)w + 16 + c,
                     make_double2((double)__uint_as_float(v1[2 * c]), (double)__uint_as_float(v1[2 * c + 1])));
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c < nb) w[c] = (double)__uint_as_float(v0[c]);
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (32 + c < nb) w[32 + c] = (double)__uint_as_float(v1[c]);
          }
        }
      }
    }
  }

  tc_before();
  __syncthreads();
  if (s_abort) {
    // every role has left its loop: the producer waits for the fills it issued
    // and the MMA issuer for its MMAs before the memory is released (the
    // producer's stores were waited for above)
    if (lane == 0 && warp == 0) drain_ring(full(0), WS, fills);
    if (lane == 0 && warp == 1) drain_mma(drain);
    tc_before();
    __syncthreads();
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

// Rows r0 .. r0 + 127 of G(:, J), one CTA per (row block, J).  Row r solves
// y T_J = rhs with rhs = e_(r - j0) for r in J (then G(r, J) = y) and
// rhs = L1(r, J) for r past J (then G(r, J) = -y), by back substitution over
// the columns of y from the last, each finished y_c updating the earlier
// right-hand sides.  FP32; the result is stored transposed and split for the
// MMA B operand: Gh/Gl[(j0 + c) * ldt + r].
__global__ void __launch_bounds__(128) k_wsolve_g(const double* __restrict__ L1, long long ld1, int k,
                                                  float* __restrict__ Gh, float* __restrict__ Gl, long long ldt) {
  pdl_wait();
  const int J = blockIdx.y, j0 = J * WN;
  const int r0 = blockIdx.x * 128;
  if (r0 + 128 <= j0 || r0 >= k) return;
  const int nb = min(WN, k - j0);
  __shared__ __align__(16) float Ts[WN][WN];  // Ts[c][a] = L1(j0 + c, j0 + a) for a < c < nb, else 0
  __shared__ float rinv[WN];
  for (int e = threadIdx.x; e < WN * WN; e += 128) {
    const int c = e / WN, a = e % WN;
    Ts[c][a] = (a < c && c < nb) ? (float)L1[(long long)(j0 + c) * ld1 + j0 + a] : 0.f;
  }
  if (threadIdx.x < WN) {
    const int c = threadIdx.x;
    rinv[c] = c < nb ? (float)(1.0 / L1[(long long)(j0 + c) * ld1 + j0 + c]) : 0.f;
  }
  __syncthreads();
  const int r = r0 + threadIdx.x;
  if (r < j0 || r >= k) return;
  const bool in_J = r < j0 + nb;
  float y[WN];
#pragma unroll
  for (int c = 0; c < WN; ++c)
    y[c] = in_J ? (c == r - j0 ? 1.f : 0.f) : (c < nb ? (float)L1[(long long)r * ld1 + j0 + c] : 0.f);
#pragma unroll
  for (int c = WN - 1; c >= 0; --c) {
    const float yc = y[c] * rinv[c];
    y[c] = yc;
#pragma unroll
    for (int a = 0; a + 4 <= c; a += 4) {
      const float4 t = *(const float4*)&Ts[c][a];
      y[a] -= yc * t.x;
      y[a + 1] -= yc * t.y;
      y[a + 2] -= yc * t.z;
      y[a + 3] -= yc * t.w;
    }
#pragma unroll
    for (int a = c & ~3; a < c; ++a) y[a] -= yc * Ts[c][a];
  }
  const float sg = in_J ? 1.f : -1.f;
#pragma unroll
  for (int c = 0; c < WN; ++c) {
    if (c < nb) {
      const float v = sg * y[c];
      const float h = tf32_rn(v);
      Gh[(long long)(j0 + c) * ldt + r] = h;
      Gl[(long long)(j0 + c) * ldt + r] = tf32_rn(v - h);
    }
  }
}

template <bool L64>
cudaError_t wsolve_all(const void* L, long long ldl, float* Wh, float* Wl, long long ldw32, double* W64,
                       long long ldw64, const double* L1, long long ld1, float* Gh, float* Gl, long long ldt,
                       long long r0, long long r1, bool form_g, long long k, State* st, cudaStream_t s) {
  using C = WCfg;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  if (dev >= 64 || !(attr_set.load() >> dev & 1ULL)) {
    e = cudaFuncSetAttribute(k_wsolve_rows<L64>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set.fetch_or(1ULL << dev);
  }
  if (form_g) {
    const int nblk = (int)((k + WN - 1) / WN);
    cudaError_t eg = launch_pdl(k_wsolve_g, dim3((unsigned)((k + 127) / 128), (unsigned)nblk), dim3(128), 0, s, L1,
                                ld1, (int)k, Gh, Gl, ldt);
    if (eg != cudaSuccess) return eg;
    e = counted(cudaGetLastError());
    if (e != cudaSuccess) return e;
  }
  if (r1 <= r0) return cudaSuccess;
  // Rows [r0, r1) only: the maps and W64 start at row r0 (r0 is a multiple of
  // the tile height, so every base stays 16-byte aligned and tiles line up).
  const long long n = r1 - r0;
  L = (const char*)L + r0 * ldl * (L64 ? 8 : 4);
  Wh += r0 * ldw32;
  Wl += r0 * ldw32;
  W64 += r0 * ldw64;

  CUtensorMap mL, mWh, mWl, mGh, mGl;
  if (L64) {
    if (!make_map(&mL, L, k, n, ldl * 8, 16, WM, true)) return cudaErrorInvalidValue;
  } else {
    if (!make_map(&mL, L, k, n, ldl * 4, WK, WM)) return cudaErrorInvalidValue;
  }
  if (!make_map(&mWh, Wh, k, n, ldw32 * 4, WK, WM)) return cudaErrorInvalidValue;
  if (!make_map(&mWl, Wl, k, n, ldw32 * 4, WK, WM)) return cudaErrorInvalidValue;
  if (!make_map(&mGh, Gh, k, k, ldt * 4, WK, WN)) return cudaErrorInvalidValue;
  if (!make_map(&mGl, Gl, k, k, ldt * 4, WK, WN)) return cudaErrorInvalidValue;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (n + WM - 1) / WM;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);  // persistent: one CTA per SM
  const int vec = (((uintptr_t)W64 & 15) == 0 && (ldw64 & 1) == 0) ? 1 : 0;
  cudaError_t er = launch_pdl(k_wsolve_rows<L64>, dim3(grid), dim3(kWThreads), (size_t)C::SMEM, s, mL, mWh, mWl, mGh,
                              mGl, W64, ldw64, vec, (int)n, (int)k, st);
  if (er != cudaSuccess) return er;
  return counted(cudaGetLastError());
}

}  // namespace tc

cudaError_t launch_wsolve_tc(const void* L, int l_is_fp64, long long ldl, float* Wh, float* Wl, long long ldw32,
                             double* W64, long long ldw64, const double* L1, long long ld1, float* Gh, float* Gl,
                             long long ldt, long long n, long long r0, long long r1, bool form_g, long long k,
                             State* st, cudaStream_t s) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  if (r0 < 0 || r1 > n || r0 % tc::WM != 0) return cudaErrorInvalidValue;
  if (l_is_fp64)
    return tc::wsolve_all<true>(L, ldl, Wh, Wl, ldw32, W64, ldw64, L1, ld1, Gh, Gl, ldt, r0, r1, form_g, k, st, s);
  return tc::wsolve_all<false>(L, ldl, Wh, Wl, ldw32, W64, ldw64, L1, ld1, Gh, Gl, ldt, r0, r1, form_g, k, st, s);
}

int wsolve_tc_rows_per_tile() { return tc::WM; }

}  // namespace rbrp
