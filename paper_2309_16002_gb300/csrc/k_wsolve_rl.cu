// Interpolation matrix of Alg. 3 on Blackwell tensor cores (sm_103a), right-looking.
//
// W L1 = L with L1 = L(S, :) lower triangular (Sec. 5.1) is solved by column blocks
// of 64 from the right.  With the block-inverse factors of k_wsolve_g,
//   G(J, J) = T_J^{-1},  G(J', J) = -L1(J', J) T_J^{-1}  (J' > J),
// each block of W is
//   W(:, J) = L(:, J) G(J, J) + sum_{J' > J} W(:, J') G(J', J),
// a sum whose terms all go through the tensor cores.  A CTA owns 128-row tiles
// and keeps the accumulators D(:, J) of a whole panel of up to 512 columns in
// tensor memory: it first adds L(:, J) G(J, J) for every block of the panel
// (and, for a panel left of others, the contributions of the W columns to its
// right, read back once from an exact FP32 copy), then walks the blocks from the right: once D(:, J)
// is complete it is W(:, J); the epilogue writes it out and stages it, split
// into TF32 hi/lo, as the A operand of one product
//   D(:, panel start .. j0) += W(:, J) G(J, panel start .. j0)
// whose first 64 columns (the next block) are issued first.  Each W block is
// thus read by the tensor cores straight from shared memory once, instead of
// being re-read for every block to its left; the B operand (rows of the
// factors, K-major) streams from L2 in slices of up to 256 columns, hi and lo
// halves in separate stages.  The products run
// in the 3xTF32 form (hi*hi + hi*lo + lo*hi, about FP32 accuracy) with FP32
// accumulators.  Panels right of the first one are separate launches, so the
// W columns a panel reads back were written by an earlier launch.
//
// Roles (320 threads): warp 0 lane 0 issues the TMA loads, warp 1 owns the
// tensor memory and lane 0 issues the MMAs, warps 2-5 (one row each) are the
// epilogue, warps 6-9 split the A chunks (L, or W read back) into hi/lo in place.  Every mbarrier wait is bounded: after the limit the CTA records
// RBRP_ETIMEOUT in the State, stops, drains the TMA fills and MMAs it issued
// (each with a bounded wait), frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "rbrp_internal.cuh"
#include "tc_common.cuh"

namespace rbrp {
namespace tc {

constexpr int RM = 128;           // rows per tile (MMA M)
constexpr int RB = 64;            // column block
constexpr int RK = 32;            // K chunk: 128 bytes of FP32
constexpr int RNS = 256;          // widest N slice of the products into the panel
constexpr int RPW = 512;          // panel width = tensor-memory columns
constexpr int RAS = 2;            // A-ring stages (in the space of the staged W block, see RCfg)
constexpr int RBS = 5;            // B-ring stages
constexpr int kRThreads = 320;

struct RCfg {
  static constexpr int A = RM * RK * 4;              // one half (hi or lo) of an A chunk: 16 KB
  static constexpr int B = RNS * RK * 4;             // one B stage: the hi or lo half of a chunk of <= 256 rows
  // The A ring (L chunks, W read back) is only used before the first W block of a
  // tile is staged, and the staged block only after the A chunks of the tile have
  // been consumed, so the two share 64 KB and the B ring gets five stages (160 KB
  // in flight covers the ~2 us a load from L2 takes under this traffic).
  static constexpr int F_OFF = 0;                    // the newest W block: [c0 hi][c0 lo][c1 hi][c1 lo]
  static constexpr int A_OFF = 0;                    // A ring: RAS x [hi][lo], aliasing F
  static constexpr int B_OFF = 4 * A;                // B ring: RBS stages, each a hi or a lo half
  static constexpr int BAR_OFF = B_OFF + RBS * B;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;
};
static_assert(RCfg::SMEM <= 227 * 1024, "shared memory");
static_assert(RAS * 2 * RCfg::A <= 4 * RCfg::A, "the A ring fits in the staged block's space");

// Width of the next N slice of a product into [n0, n0 + rem) (rem a multiple of 64):
// one tcgen05.mma of kind::tf32 holds the MMA issue for about the same time up to
// N = 128 and N = 256 doubles the work per instruction, so slices are as wide as the
// range allows.
__host__ __device__ inline int slice_w(int rem) { return rem >= 256 ? 256 : (rem >= 128 ? 128 : 64); }

// The panel [ps, pe) of a launch: blocks Jlo .. Jhi; wback: a later launch (a panel
// to the left) reads this panel's W back, from the exact FP32 copy Wb.
struct RPanel {
  int ps, pe, Jlo, Jhi, wback;
};

template <bool L64>
__global__ void __launch_bounds__(kRThreads, 1)
    k_wsolve_rl(const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmW,
                const __grid_constant__ CUtensorMap tmG256h, const __grid_constant__ CUtensorMap tmG256l,
                const __grid_constant__ CUtensorMap tmG128h, const __grid_constant__ CUtensorMap tmG128l,
                const __grid_constant__ CUtensorMap tmG64h, const __grid_constant__ CUtensorMap tmG64l,
                double* __restrict__ W64, long long ldw64, int w64_vec, float* __restrict__ Wb, long long ldwb,
                int n, int k, RPanel pn, State* st) {
  using C = RCfg;
  pdl_wait();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(smem);
  const uint32_t sBar = sb + C::BAR_OFF;
  auto a_full = [&](int s) { return sBar + 8u * s; };
  auto a_conv = [&](int s) { return sBar + 8u * (RAS + s); };
  auto a_empty = [&](int s) { return sBar + 8u * (2 * RAS + s); };
  auto b_full = [&](int s) { return sBar + 8u * (3 * RAS + s); };
  auto b_empty = [&](int s) { return sBar + 8u * (3 * RAS + RBS + s); };
  const uint32_t d_ready = sBar + 8u * (3 * RAS + 2 * RBS);      // MMA -> epilogue: D(:, J) complete
  const uint32_t d_empty = d_ready + 8u;                          // epilogue -> MMA: the tile's D read out
  const uint32_t f_full = d_ready + 16u;                          // epilogue -> MMA: W(:, J) staged
  const uint32_t f_free = d_ready + 24u;                          // MMA -> epilogue: the stage is read
  const uint32_t drain = d_ready + 32u;                           // abort path: MMA drain
  const uint32_t tile_done = d_ready + 40u;                       // MMA -> producer: a tile's MMAs issued and done
  uint32_t* tmem_slot = (uint32_t*)(smem + C::BAR_OFF + 8 * (3 * RAS + 2 * RBS + 6));
  static_assert(8 * (3 * RAS + 2 * RBS + 7) <= 256, "barrier area");

  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (n + RM - 1) / RM;
  const int ps = pn.ps, pe = pn.pe, Jlo = pn.Jlo, Jhi = pn.Jhi;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < RAS; ++s) {
      mbar_init(a_full(s), 1);
      mbar_init(a_conv(s), 128);
      mbar_init(a_empty(s), 1);
    }
    for (int s = 0; s < RBS; ++s) {
      mbar_init(b_full(s), 1);
      mbar_init(b_empty(s), 1);
    }
    mbar_init(d_ready, 1);
    mbar_init(d_empty, 128);
    mbar_init(f_full, 128);
    mbar_init(f_free, 1);
    mbar_init(drain, 1);
    mbar_init(tile_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)RPW)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *(volatile uint32_t*)tmem_slot;
  volatile int* abort = &s_abort;
  const uint32_t lim = st->spin_mbar;
  uint32_t fa = 0, fb = 0;  // TMA fills issued into the A / B ring (for the abort drain)

  if (warp == 0) {
    // ---------------- TMA producer: the A and B chunks in the order the MMAs take them
    if (lane == 0) {
      const uint64_t keep = l2_policy_evict_last(), stream = l2_policy_evict_first();
      uint32_t ga = 0, gb = 0;
      bool ok = true;
      // A chunk: L (FP32: one box; FP64: two boxes of 16 columns) or W read back (FP32)
      auto load_a = [&](const CUtensorMap* map, bool f64, int x, int y) {
        const int s = (int)(ga % RAS);
        if (!mbar_wait(a_empty(s), ((ga / RAS) & 1u) ^ 1u, abort, lim)) return false;
        const uint32_t base = sb + C::A_OFF + s * 2 * C::A;
        mbar_expect_tx(a_full(s), f64 ? 2u * C::A : (uint32_t)C::A);
        tma_load_2d_hint(base, map, a_full(s), x, y, stream);
        if (f64) tma_load_2d_hint(base + C::A, map, a_full(s), x + 16, y, stream);
        ++ga;
        ++fa;
        return true;
      };
      // B chunk: rows n0 .. n0 + w - 1 of the factors (K-major), its hi half into one
      // stage and its lo half into the next
      auto load_b = [&](int w, int x, int n0) {
        for (int half = 0; half < 2; ++half) {
          const int s = (int)(gb % RBS);
          if (!mbar_wait(b_empty(s), ((gb / RBS) & 1u) ^ 1u, abort, lim)) return false;
          const uint32_t base = sb + C::B_OFF + s * C::B;
          const CUtensorMap* m = w == 256 ? (half ? &tmG256l : &tmG256h)
                                          : (w == 128 ? (half ? &tmG128l : &tmG128h) : (half ? &tmG64l : &tmG64h));
          mbar_expect_tx(b_full(s), (uint32_t)(w * RK * 4));
          tma_load_2d_hint(base, m, b_full(s), x, n0, keep);
          ++gb;
          ++fb;
        }
        return true;
      };
      uint32_t tp = 0;  // tiles of this CTA so far
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tp) {
        const int y = tile * RM;
        // the A ring shares its space with the staged W block: wait until every MMA of
        // the previous tile (the last ones read the staged block) has completed.  One
        // completion per tile, and this wait comes before the loads the next one needs,
        // so the barrier is never two phases behind it.
        if (tp > 0 && !mbar_wait(tile_done, (tp - 1) & 1u, abort, lim)) break;
        // 1. D(:, J) = L(:, J) G(J, J) for every block of the panel
        for (int J = Jhi; J >= Jlo && ok; --J)
          for (int kc = 0; kc < 2 && ok; ++kc) {
            const int x = J * RB + RK * kc;
            if (x >= k) break;
            ok = load_a(&tmL, L64, x, y) && load_b(RB, x, J * RB);
          }
        // 2. D(:, panel) += W(:, pe ..) G(pe .., panel)
        for (int x = pe; x < k && ok; x += RK) {
          ok = load_a(&tmW, false, x, y);
          for (int n0 = ps, w = 0; n0 < pe && ok; n0 += w) {
            w = slice_w(pe - n0);
            ok = load_b(w, x, n0);
          }
        }
        // 3. after W(:, J): the next block's 64 columns, then the rest of the panel
        for (int J = Jhi; J > Jlo && ok; --J) {
          const int j0 = J * RB;
          for (int kc = 0; kc < 2 && ok; ++kc) {
            const int x = j0 + RK * kc;
            if (x >= k) break;
            ok = load_b(RB, x, j0 - RB);
          }
          for (int n0 = ps, w = 0; n0 < j0 - RB && ok; n0 += w) {
            w = slice_w(j0 - RB - n0);
            for (int kc = 0; kc < 2 && ok; ++kc) {
              const int x = j0 + RK * kc;
              if (x >= k) break;
              ok = load_b(w, x, n0);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      uint32_t ga = 0, gb = 0, nf = 0, it = 0;
      bool ok = true;
      auto wait_a = [&](int& s) {
        s = (int)(ga % RAS);
        const uint32_t ph = (ga / RAS) & 1u;
        return mbar_wait(a_full(s), ph, abort, lim) && mbar_wait(a_conv(s), ph, abort, lim);
      };
      // 3xTF32 product of one K chunk (4 steps of 8) into D columns d .. d + w - 1:
      // A_hi B_hi + A_lo B_hi from the B stage holding the hi half, then A_hi B_lo
      // from the next stage (first: the first product into D, which overwrites it)
      auto mma_chunk = [&](uint32_t d, uint32_t a, uint32_t alo, int w, bool first) {
        const uint32_t id = idesc_tf32(RM, w);
        for (int half = 0; half < 2; ++half) {
          const int s = (int)(gb % RBS);
          if (!mbar_wait(b_full(s), (gb / RBS) & 1u, abort, lim)) return false;
          tc_after();
          const uint32_t b = sb + C::B_OFF + s * C::B;
#pragma unroll
          for (int kk = 0; kk < RK / 8; ++kk) {
            if (half == 0) {
              mma_tf32(d, sdesc(a + kk * 32), sdesc(b + kk * 32), id, (first && kk == 0) ? 0u : 1u);
              mma_tf32(d, sdesc(alo + kk * 32), sdesc(b + kk * 32), id, 1u);
            } else {
              mma_tf32(d, sdesc(a + kk * 32), sdesc(b + kk * 32), id, 1u);
            }
          }
          mma_commit(b_empty(s));
          ++gb;
        }
        return true;
      };
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        // the previous tile's accumulators have been read out
        if (it > 0 && !mbar_wait(d_empty, (it - 1) & 1u, abort, lim)) break;
        tc_after();
        // 1. D(:, J) = L(:, J) G(J, J)
        for (int J = Jhi; J >= Jlo && ok; --J)
          for (int kc = 0; kc < 2; ++kc) {
            const int x = J * RB + RK * kc;
            if (x >= k) break;
            int sa;
            if (!wait_a(sa)) {
              ok = false;
              break;
            }
            tc_after();
            const uint32_t a = sb + C::A_OFF + sa * 2 * C::A;
            if (!mma_chunk(tmem + (uint32_t)(J * RB - ps), a, a + C::A, RB, kc == 0)) {
              ok = false;
              break;
            }
            mma_commit(a_empty(sa));
            ++ga;
          }
        // 2. the W columns right of the panel
        for (int x = pe; x < k && ok; x += RK) {
          int sa;
          if (!wait_a(sa)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t a = sb + C::A_OFF + sa * 2 * C::A;
          for (int n0 = ps, w = 0; n0 < pe && ok; n0 += w) {
            w = slice_w(pe - n0);
            ok = mma_chunk(tmem + (uint32_t)(n0 - ps), a, a + C::A, w, false);
          }
          mma_commit(a_empty(sa));
          ++ga;
        }
        if (!ok) break;
        mma_commit(d_ready);  // D(:, Jhi) is complete
        // 3. the blocks from the right
        for (int J = Jhi; J > Jlo && ok; --J) {
          const int j0 = J * RB;
          if (!mbar_wait(f_full, nf & 1u, abort, lim)) {
            ok = false;
            break;
          }
          ++nf;
          tc_after();
          const uint32_t f = sb + C::F_OFF;
          for (int kc = 0; kc < 2 && ok; ++kc) {
            const int x = j0 + RK * kc;
            if (x >= k) break;
            const uint32_t a = f + kc * 2 * C::A;
            ok = mma_chunk(tmem + (uint32_t)(j0 - RB - ps), a, a + C::A, RB, false);
          }
          if (!ok) break;
          mma_commit(d_ready);  // D(:, J - 1) is complete
          for (int n0 = ps, w = 0; n0 < j0 - RB && ok; n0 += w) {
            w = slice_w(j0 - RB - n0);
            for (int kc = 0; kc < 2 && ok; ++kc) {
              const int x = j0 + RK * kc;
              if (x >= k) break;
              const uint32_t a = f + kc * 2 * C::A;
              ok = mma_chunk(tmem + (uint32_t)(n0 - ps), a, a + C::A, w, false);
            }
          }
          mma_commit(f_free);  // the staged W(:, J) is no longer read
        }
        if (!ok) break;
        mma_commit(tile_done);  // every MMA of this tile
      }
    }
  } else if (warp >= 6) {
    // ---------------- warps 6-9: split each A chunk into TF32 hi (in place) and lo
    const int r = threadIdx.x - 192;  // 0..127, one tile row each
    const int r7 = r & 7;
    uint32_t ga = 0;
    bool ok = true;
    auto convert = [&](bool f64) {
      const int s = (int)(ga % RAS);
      if (!mbar_wait(a_full(s), (ga / RAS) & 1u, abort, lim)) return false;
      uint8_t* a = smem + C::A_OFF + s * 2 * C::A + (r >> 3) * 1024 + r7 * 128;  // this row, 128-byte swizzled
      uint8_t* alo = a + C::A;
      if (f64) {
        // FP64 columns 0-15 sit in the hi half, 16-31 in the lo half
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
          const uint32_t o = (uint32_t)((c ^ r7) << 4);
          const float4 x = *(const float4*)(a + o);
          const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
          *(float4*)(a + o) = h;
          *(float4*)(alo + o) =
              make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
        }
      }
      fence_async_smem();
      mbar_arrive(a_conv(s));
      ++ga;
      return true;
    };
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int J = Jhi; J >= Jlo && ok; --J)
        for (int kc = 0; kc < 2 && ok; ++kc) {
          if (J * RB + RK * kc >= k) break;
          ok = convert(L64);
        }
      for (int x = pe; x < k && ok; x += RK) ok = convert(false);
    }
  } else {
    // ---------------- warps 2-5: epilogue, one row of the tile per thread
    const int q4 = warp & 3;
    const int r = 32 * q4 + lane;
    const int r7 = r & 7;
    const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
    uint32_t nd = 0, nf = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const long long row = (long long)tile * RM + r;
      for (int J = Jhi; J >= Jlo; --J) {
        const int j0 = J * RB;
        if (!mbar_wait(d_ready, nd & 1u, abort, lim)) {
          ok = false;
          break;
        }
        ++nd;
        tc_after();
        uint32_t v0[32], v1[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(j0 - ps), v0);
        tmem_ld32(tmem + lane_base + (uint32_t)(j0 - ps) + 32u, v1);
        tmem_wait_ld();
        tc_before();
        if (J > Jlo) {
          // W(:, J) as the A operand of the product into the blocks left of it (hi/lo, 128-byte swizzle)
          if (nf > 0 && !mbar_wait(f_free, (nf - 1) & 1u, abort, lim)) {
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
          ++nf;
        }
        if (row < n && pn.wback) {
          // the exact FP32 value of W(:, J) (the accumulator), for the panels to the left
          float4* wb = (float4*)(Wb + row * ldwb + j0);
#pragma unroll
          for (int c = 0; c < 8; ++c)
            wb[c] = make_float4(__uint_as_float(v0[4 * c]), __uint_as_float(v0[4 * c + 1]),
                                __uint_as_float(v0[4 * c + 2]), __uint_as_float(v0[4 * c + 3]));
#pragma unroll
          for (int c = 0; c < 8; ++c)
            wb[8 + c] = make_float4(__uint_as_float(v1[4 * c]), __uint_as_float(v1[4 * c + 1]),
                                    __uint_as_float(v1[4 * c + 2]), __uint_as_float(v1[4 * c + 3]));
        }
        if (row < n) {
          const int nb = min(RB, k - j0);
          double* w = W64 + row * ldw64 + j0;
          if (w64_vec && nb == RB) {
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
      if (!ok) break;
      mbar_arrive(d_empty);  // every accumulator of this tile has been read
    }
  }

  tc_before();
  __syncthreads();
  if (s_abort) {
    // every role has left its loop: the producer waits for the fills it issued and
    // the MMA issuer for its MMAs before the memory is released
    if (lane == 0 && warp == 0) {
      drain_ring(a_full(0), RAS, fa);
      drain_ring(b_full(0), RBS, fb);
    }
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)RPW) : "memory");
  }
}

// Rows [r0, r1) of W (r0 a multiple of 128) by panels of up to eight blocks, the
// rightmost first, one launch each.  Wb (FP32, ldwb a multiple of 4, 16-byte
// aligned): the scratch for the W columns that later panels read back.
template <bool L64>
cudaError_t wsolve_rl(const void* L, long long ldl, double* W64, long long ldw64, float* Wb, long long ldwb,
                      const float* Gh, const float* Gl, long long ldt, long long r0, long long r1, long long k,
                      State* st, cudaStream_t s) {
  using C = RCfg;
  const long long n = r1 - r0;
  if (n <= 0 || k <= 0) return cudaSuccess;
  if ((ldwb & 3) != 0 || ldwb < (k + RB - 1) / RB * RB || ((uintptr_t)Wb & 15) != 0) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  if (dev >= 64 || !(attr_set.load() >> dev & 1ULL)) {
    e = cudaFuncSetAttribute(k_wsolve_rl<L64>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set.fetch_or(1ULL << dev);
  }
  L = (const char*)L + r0 * ldl * (L64 ? 8 : 4);
  W64 += r0 * ldw64;
  Wb += r0 * ldwb;
  CUtensorMap mL, mW, mG256h, mG256l, mG128h, mG128l, mG64h, mG64l;
  if (L64) {
    if (!make_map(&mL, L, k, n, ldl * 8, 16, RM, true)) return cudaErrorInvalidValue;
  } else {
    if (!make_map(&mL, L, k, n, ldl * 4, RK, RM)) return cudaErrorInvalidValue;
  }
  if (!make_map(&mW, Wb, k, n, ldwb * 4, RK, RM)) return cudaErrorInvalidValue;
  if (!make_map(&mG256h, Gh, k, k, ldt * 4, RK, 256)) return cudaErrorInvalidValue;
  if (!make_map(&mG256l, Gl, k, k, ldt * 4, RK, 256)) return cudaErrorInvalidValue;
  if (!make_map(&mG128h, Gh, k, k, ldt * 4, RK, 128)) return cudaErrorInvalidValue;
  if (!make_map(&mG128l, Gl, k, k, ldt * 4, RK, 128)) return cudaErrorInvalidValue;
  if (!make_map(&mG64h, Gh, k, k, ldt * 4, RK, RB)) return cudaErrorInvalidValue;
  if (!make_map(&mG64l, Gl, k, k, ldt * 4, RK, RB)) return cudaErrorInvalidValue;
  const long long ntiles = (n + RM - 1) / RM;
  const int sms = device_sms();
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);  // persistent: one CTA per SM
  const int vec = (((uintptr_t)W64 & 15) == 0 && (ldw64 & 1) == 0) ? 1 : 0;
  const int nblk = (int)((k + RB - 1) / RB);
  for (int Jhi = nblk - 1; Jhi >= 0;) {
    RPanel pn;
    pn.Jhi = Jhi;
    pn.Jlo = Jhi - (RPW / RB - 1) > 0 ? Jhi - (RPW / RB - 1) : 0;
    pn.ps = pn.Jlo * RB;
    pn.pe = (int)((long long)(Jhi + 1) * RB < k ? (Jhi + 1) * RB : k);
    pn.wback = pn.Jlo > 0;
    e = launch_pdl(k_wsolve_rl<L64>, dim3(grid), dim3(kRThreads), (size_t)C::SMEM, s, mL, mW, mG256h, mG256l,
                   mG128h, mG128l, mG64h, mG64l, W64, ldw64, vec, Wb, ldwb, (int)n, (int)k, pn, st);
    if (e != cudaSuccess) return e;
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    Jhi = pn.Jlo - 1;
  }
  return cudaSuccess;
}

template cudaError_t wsolve_rl<true>(const void*, long long, double*, long long, float*, long long, const float*,
                                     const float*, long long, long long, long long, long long, State*, cudaStream_t);
template cudaError_t wsolve_rl<false>(const void*, long long, double*, long long, float*, long long, const float*,
                                      const float*, long long, long long, long long, long long, State*, cudaStream_t);

}  // namespace tc
}  // namespace rbrp
