// Fused residual update of RBRP on Blackwell tensor cores (sm_103a).
//
// Alg. 2's update step in the residual form: for every tile of rows of R,
//   Lhat = R_tile Q'^T            (GEMM 1, K = d, N = b'_pad)
//   R_tile <- R_tile - Lhat Q'    (GEMM 2, K = b'_pad, N = d in column chunks)
//   d_i = ||R_i||^2, rows accepted in this block set to 0,
//   Lhat written to L(:, k : k + b').
// Operands are staged by TMA (128-byte swizzle) and multiplied by tcgen05.mma
// kind::tf32 with FP32 accumulators in tensor memory.  The R tile is read twice
// (GEMM 1 and the subtraction); the second read is mostly served by L2.
//
// Two kernels:
//  - k_update_tf32p, the update itself: persistent (one CTA per SM walking tiles
//    of up to 128 rows), b'_pad <= 64 columns of Q' a launch (wider blocks run as
//    successive 64-column chunks), plain TF32 or the 3xTF32 split (SPLIT), with
//    Lhat kept in tensor memory as GEMM 2's A operand.  Its roles and rings are
//    described where it is defined.
//  - k_update_tf32, non-persistent 64-row tiles: with G1 it computes only Lhat =
//    X Q'^T for the downdate form of the update step (3xTF32), and it serves a
//    direct plain-TF32 call with up to 128 columns.
//
// The 3xTF32 split: every operand x is taken as hi + lo with hi a TF32 value and
// lo = x - hi rounded to TF32, and each product is hi*hi + hi*lo + lo*hi; that
// brings the contraction to ~FP32 accuracy, so the residual does not pick up the
// per-block floor that plain TF32 leaves (relative energy ~u^2 with u = 2^-11).
// Q' and Lhat are split with hi rounded to nearest; in the persistent kernel the
// R chunk as loaded is its own hi half (the MMA reads FP32 as TF32 by dropping the
// low 13 mantissa bits) and lo is taken against that truncation.
//
// k_update_tf32's roles (192 threads): warp 0 lane 0 issues TMA loads, warp 1
// owns TMEM and lane 0 issues the MMAs, warps 2-5 (128 threads, one row each)
// split the GEMM-1 A operand (SPLIT), run the epilogues and issue the TMA stores.
// Row norms are summed in FP32 over each 32-column piece and the piece sums in
// FP64 (per-element FP64 arithmetic would cost ~2 FMA/clock/SM on GB300).
// Every mbarrier wait of both kernels is bounded: after the limit the CTA records
// RBRP_ETIMEOUT in the State, stops issuing work, waits for the TMA copies and
// MMAs it has issued (drain_ring / drain_mma), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "rbrp_internal.cuh"
#include "tc_common.cuh"

namespace rbrp {
namespace tc {

constexpr int BM = 128;           // MMA M (TMEM lanes)
constexpr int ROWS = 64;          // rows of R per CTA; MMA rows ROWS..BM-1 are don't-care
constexpr int BK1 = 32;           // FP32 elements per 128-byte swizzle row
constexpr int NB2 = 32;           // d-columns per GEMM-2 chunk (MMA N)
constexpr int kThreads = 192;

// A tile holds ROWS rows of R, half the MMA's M: every CTA's share of R is
// read twice (GEMM 1, then the subtraction), and with 64-row tiles the data
// between the two reads of all resident CTAs stays well inside L2, so the
// second read does not go back to HBM.  An MMA reads BM rows of A; rows
// ROWS..BM-1 come from whatever shared memory follows the chunk (the next
// buffer of the ring) and only feed accumulator rows nobody reads.
template <int BMAX, bool SPLIT>
struct Cfg {
  static constexpr int S1 = (BMAX <= 64 && !SPLIT) ? 4 : 3;  // GEMM-1 stages
  static constexpr int S3 = S1;                              // GEMM-2 / epilogue stages
  static constexpr int NOP = SPLIT ? 2 : 1;            // hi (and lo) copies of an operand
  static constexpr int A1 = ROWS * BK1 * 4;            // one R chunk (8 KB)
  static constexpr int B1 = BMAX * BK1 * 4;            // one Q' chunk
  static constexpr int ST1 = NOP * (A1 + B1);          // [A hi][B hi]([A lo][B lo])
  static constexpr int R3 = ROWS * NB2 * 4;            // one R chunk for the subtraction (8 KB)
  static constexpr int B2A = NB2 * 128;                // one 32-wide K atom of the GEMM-2 B tile
  static constexpr int B2 = (BMAX / 32) * B2A;
  static constexpr int ST3 = R3 + NOP * B2;
  static constexpr int P = (S1 * ST1 > S3 * ST3) ? S1 * ST1 : S3 * ST3;
  static constexpr int A2A = BM * 128;                 // one 32-wide K atom of Lhat
  static constexpr int A2 = (BMAX / 32) * A2A;
  static constexpr int BAR_OFF = P + NOP * A2;
  // the BM-row A reads of GEMM 1 (last stage, lo copy) end inside the Lhat buffers
  static_assert((S1 - 1) * ST1 + (NOP - 1) * (A1 + B1) + BM * BK1 * 4 <= P + NOP * A2, "A over-read");
  static constexpr int BAR_BYTES = 320;
  static constexpr int SMEM = BAR_OFF + BAR_BYTES + 1024;
  static constexpr uint32_t D2COL = BMAX;              // D2 double buffer after D1
  static constexpr uint32_t TMEM_COLS = (BMAX + 2 * NB2 <= 128) ? 128 : 256;
  static constexpr int MIN_BLOCKS = (SMEM <= 110 * 1024) ? 2 : 1;
};

// ------------------------------------------------------------------ kernel
// G1 = true runs GEMM 1 only: Lhat = A Q'^T into L(:, k + c0 ...) for every row of
// A (the downdate form of the update step: A = X, read only; d is downdated by
// launch_downdate afterwards), with no subtraction, no norms and no stores of A.
template <int BMAX, bool SPLIT, bool G1 = false>
__global__ void __launch_bounds__(kThreads, Cfg<BMAX, SPLIT>::MIN_BLOCKS)
    k_update_tf32(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmX,
                  const __grid_constant__ CUtensorMap tmQ,
                  const __grid_constant__ CUtensorMap tmQlo, const __grid_constant__ CUtensorMap tmQT,
                  const __grid_constant__ CUtensorMap tmQTlo, float* __restrict__ L, long long ldl, long long n,
                  long long d, const int* __restrict__ mark, double* __restrict__ dvec,
                  double* __restrict__ partials, State* st, int c0) {
  using C = Cfg<BMAX, SPLIT>;
  constexpr int S1 = C::S1, S3 = C::S3;
  if (st->done) return;
  // this launch applies columns c0 .. c0 + BMAX - 1 of Q' (a chunk of a wider block);
  // rows accepted in this block keep their residual until the last chunk (the later
  // chunks' coefficients of those rows are part of L1), which then zeroes it
  const int bp = min((int)st->bp - c0, BMAX);
  if (bp <= 0) return;
  const bool last_chunk = c0 + BMAX >= (int)st->bp;
  // the residual starts as X and is never copied: the first block's first launch
  // reads X (tmX) and stores R, every later launch reads and stores R
  const CUtensorMap* tmSrc = (!G1 && st->t == 0 && c0 == 0) ? &tmX : &tmR;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(smem);
  const uint32_t sA2 = sb + C::P;             // Lhat hi; Lhat lo follows at + A2 (SPLIT)
  const uint32_t sBar = sb + C::BAR_OFF;
  // barrier map (8 bytes each)
  auto full1 = [&](int s) { return sBar + 8u * s; };
  auto empty1 = [&](int s) { return sBar + 8u * (S1 + s); };
  auto conv1 = [&](int s) { return sBar + 8u * (2 * S1 + s); };            // SPLIT: A lo written
  auto full3 = [&](int s) { return sBar + 8u * (3 * S1 + s); };
  auto empty3 = [&](int s) { return sBar + 8u * (3 * S1 + S3 + s); };
  auto epi_done = [&](int s) { return sBar + 8u * (3 * S1 + 2 * S3 + s); };
  const uint32_t d1_full = sBar + 8u * (3 * S1 + 3 * S3);
  const uint32_t a2_ready = d1_full + 8u;
  auto d2_full = [&](int b) { return a2_ready + 8u + 8u * b; };
  auto d2_empty = [&](int b) { return a2_ready + 24u + 8u * b; };
  const uint32_t red_bar = a2_ready + 40u;
  uint32_t* tmem_slot = (uint32_t*)(smem + C::BAR_OFF + 8 * (3 * S1 + 3 * S3 + 7));
  const uint32_t drain = sBar + 8u * (3 * S1 + 3 * S3 + 8);  // abort path: MMA drain
  static_assert(8 * (3 * S1 + 3 * S3 + 9) <= C::BAR_BYTES, "barrier area");

  __shared__ int s_abort;
  __shared__ double s_red[4];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long row0 = (long long)blockIdx.x * ROWS;
  const long long kcol = st->k + c0;
  const int N1 = (bp + 15) / 16 * 16;
  const int tno = (int)(st->t + 1);
  const int nK1 = (int)((d + BK1 - 1) / BK1);
  const int nC = (int)((d + NB2 - 1) / NB2);

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < S1; ++s) {
      mbar_init(full1(s), 1);
      mbar_init(empty1(s), 1);
      mbar_init(conv1(s), 128);
    }
    for (int s = 0; s < S3; ++s) {
      mbar_init(full3(s), 1);
      mbar_init(empty3(s), 2);
      mbar_init(epi_done(s), 128);
    }
    mbar_init(d1_full, 1);
    mbar_init(a2_ready, 128);
    for (int b = 0; b < 2; ++b) {
      mbar_init(d2_full(b), 1);
      mbar_init(d2_empty(b), 128);
    }
    mbar_init(red_bar, 128);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *(volatile uint32_t*)tmem_slot;
  volatile int* abort = &s_abort;
  const uint32_t lim = st->spin_mbar;
  uint32_t fills1 = 0, fills3 = 0;  // TMA fills issued into ring 1 / ring 3 (for the abort drain)

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      // The first read of the R tile asks L2 to keep it (it is read again for the
      // subtraction); the second read and the stores ask for early eviction.
      const uint64_t keep = l2_policy_evict_last(), drop = l2_policy_evict_first();
      for (int kc = 0; kc < nK1; ++kc) {
        const int s = kc % S1;
        const uint32_t ph = (uint32_t)(kc / S1) & 1u;
        if (!mbar_wait(empty1(s), ph ^ 1u, abort, lim)) break;
        mbar_expect_tx(full1(s), (uint32_t)((C::A1 + C::B1) + (SPLIT ? C::B1 : 0)));
        const uint32_t base = sb + s * C::ST1;
        tma_load_2d_hint(base, tmSrc, full1(s), kc * BK1, (int)row0, keep);
        tma_load_2d(base + C::A1, &tmQ, full1(s), kc * BK1, 0);
        if (SPLIT) tma_load_2d(base + 2 * C::A1 + C::B1, &tmQlo, full1(s), kc * BK1, 0);
        ++fills1;
      }
      // phase-3 buffers alias the phase-1 ring: reuse only after GEMM 1 has drained it.
      // Chunks are taken last-to-first so the most recently loaded columns are re-read first.
      if (!G1 && mbar_wait(d1_full, 0, abort, lim)) {
        for (int c = 0; c < nC; ++c) {
          const int s = c % S3;
          const uint32_t ph = (uint32_t)(c / S3) & 1u;
          const int col = (nC - 1 - c) * NB2;
          if (!mbar_wait(empty3(s), ph ^ 1u, abort, lim)) break;
          mbar_expect_tx(full3(s), (uint32_t)C::ST3);
          const uint32_t base = sb + s * C::ST3;
          tma_load_2d_hint(base, tmSrc, full3(s), col, (int)row0, drop);
#pragma unroll
          for (int a = 0; a < BMAX / 32; ++a) {
            tma_load_2d(base + C::R3 + a * C::B2A, &tmQT, full3(s), a * 32, col);
            if (SPLIT) tma_load_2d(base + C::R3 + C::B2 + a * C::B2A, &tmQTlo, full3(s), a * 32, col);
          }
          ++fills3;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      const uint32_t id1 = idesc_tf32(BM, N1);
      for (int kc = 0; kc < nK1; ++kc) {
        const int s = kc % S1;
        const uint32_t ph = (uint32_t)(kc / S1) & 1u;
        if (!mbar_wait(full1(s), ph, abort, lim)) break;
        if (SPLIT && !mbar_wait(conv1(s), ph, abort, lim)) break;
        tc_after();
        const uint32_t a = sb + s * C::ST1, b = a + C::A1;
        const uint32_t alo = a + C::A1 + C::B1, blo = alo + C::A1;
#pragma unroll
        for (int kk = 0; kk < BK1 / 8; ++kk) {
          mma_tf32(tmem, sdesc(a + kk * 32), sdesc(b + kk * 32), id1, (kc | kk) != 0 ? 1u : 0u);
          if (SPLIT) {
            mma_tf32(tmem, sdesc(a + kk * 32), sdesc(blo + kk * 32), id1, 1u);
            mma_tf32(tmem, sdesc(alo + kk * 32), sdesc(b + kk * 32), id1, 1u);
          }
        }
        mma_commit(empty1(s));
      }
      mma_commit(d1_full);
      if (!G1 && mbar_wait(a2_ready, 0, abort, lim)) {
        tc_after();
        const uint32_t id2 = idesc_tf32(BM, NB2);
        const int nk2 = N1 / 8;
        for (int c = 0; c < nC; ++c) {
          const int s = c % S3;
          const uint32_t ph = (uint32_t)(c / S3) & 1u;
          const int buf = c & 1;
          const uint32_t bph = (uint32_t)(c >> 1) & 1u;
          if (!mbar_wait(full3(s), ph, abort, lim)) break;
          if (!mbar_wait(d2_empty(buf), bph ^ 1u, abort, lim)) break;
          tc_after();
          const uint32_t dt = tmem + C::D2COL + (uint32_t)(buf * NB2);
          const uint32_t b2 = sb + s * C::ST3 + C::R3;
          for (int q = 0; q < nk2; ++q) {
            const int a = q >> 2, kk = q & 3;
            const uint32_t ao = a * C::A2A + kk * 32, bo = a * C::B2A + kk * 32;
            mma_tf32(dt, sdesc(sA2 + ao), sdesc(b2 + bo), id2, q != 0 ? 1u : 0u);
            if (SPLIT) {
              mma_tf32(dt, sdesc(sA2 + ao), sdesc(b2 + C::B2 + bo), id2, 1u);
              mma_tf32(dt, sdesc(sA2 + C::A2 + ao), sdesc(b2 + bo), id2, 1u);
            }
          }
          mma_commit(empty3(s));
          mma_commit(d2_full(buf));
        }
      }
    }
  } else {
    // ---------------- warps 2-5: 128 threads, thread <-> row
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const int et = threadIdx.x - 64;
    const long long row = row0 + r;
    const bool own = r < ROWS;  // warps with q >= 2 own no row of R
    const bool in = own && row < n;
    const bool marked = !G1 && last_chunk && in && (mark[row] == tno);
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint64_t drop = l2_policy_evict_first();
    if (SPLIT) {
      // split each GEMM-1 A chunk in place: hi stays, lo goes to its own buffer
      for (int kc = 0; kc < nK1; ++kc) {
        const int s = kc % S1;
        const uint32_t ph = (uint32_t)(kc / S1) & 1u;
        if (!mbar_wait(full1(s), ph, abort, lim)) break;
        if (!own) {
          mbar_arrive(conv1(s));
          continue;
        }
        uint8_t* a = smem + s * C::ST1 + (r >> 3) * 1024 + (r & 7) * 128;
        uint8_t* alo = smem + s * C::ST1 + C::A1 + C::B1 + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          float4 x = *(float4*)(a + ch * 16);
          float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
          *(float4*)(a + ch * 16) = h;
          *(float4*)(alo + ch * 16) = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
        }
        fence_async_smem();
        mbar_arrive(conv1(s));
      }
    }
    double nrm = 0.0;
    if (mbar_wait(d1_full, 0, abort, lim)) {
      tc_after();
      for (int cb = 0; own && cb * 32 < N1; ++cb) {
        uint32_t v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(cb * 32), v);
        tmem_wait_ld();
        if (in) {
          float* lrow = L + row * ldl + kcol + cb * 32;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (cb * 32 + j < bp) lrow[j] = __uint_as_float(v[j]);
        }
        if (G1) continue;
        uint8_t* a2 = smem + C::P + cb * C::A2A;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const float4 x = make_float4(__uint_as_float(v[4 * ch]), __uint_as_float(v[4 * ch + 1]),
                                       __uint_as_float(v[4 * ch + 2]), __uint_as_float(v[4 * ch + 3]));
          if (SPLIT) {
            const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
            *(float4*)(a2 + swz(r, ch)) = h;
            *(float4*)(a2 + C::A2 + swz(r, ch)) =
                make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
          } else {
            *(float4*)(a2 + swz(r, ch)) = x;
          }
        }
      }
    }
    fence_async_smem();
    tc_before();
    mbar_arrive(a2_ready);
    for (int c = 0; c < nC && !G1; ++c) {
      const int s = c % S3;
      const uint32_t ph = (uint32_t)(c / S3) & 1u;
      const int buf = c & 1;
      const uint32_t bph = (uint32_t)(c >> 1) & 1u;
      if (!mbar_wait(full3(s), ph, abort, lim)) break;
      if (!mbar_wait(d2_full(buf), bph, abort, lim)) break;
      tc_after();
      uint32_t u[32];
      if (own) {
        tmem_ld32(tmem + lane_base + C::D2COL + (uint32_t)(buf * NB2), u);
        tmem_wait_ld();
      }
      uint8_t* rrow = smem + s * C::ST3;
      float part = 0.f;
#pragma unroll
      for (int ch = 0; ch < 8 && own; ++ch) {
        float4* p = (float4*)(rrow + swz(r, ch));
        float4 x = *p;
        x.x -= __uint_as_float(u[4 * ch]);
        x.y -= __uint_as_float(u[4 * ch + 1]);
        x.z -= __uint_as_float(u[4 * ch + 2]);
        x.w -= __uint_as_float(u[4 * ch + 3]);
        if (marked) x = make_float4(0.f, 0.f, 0.f, 0.f);
        part = fmaf(x.x, x.x, part);
        part = fmaf(x.y, x.y, part);
        part = fmaf(x.z, x.z, part);
        part = fmaf(x.w, x.w, part);
        *p = x;
      }
      nrm += (double)part;
      tc_before();
      mbar_arrive(d2_empty(buf));
      fence_async_smem();
      mbar_arrive(epi_done(s));
      if (et == 0) {
        // every epilogue thread has written its row of this chunk (bounded wait)
        if (!mbar_wait(epi_done(s), ph, abort, lim)) break;
        tma_store_2d_hint(&tmR, sb + s * C::ST3, (nC - 1 - c) * NB2, (int)row0, drop);
        tma_commit();
        // with at most this store pending, the previous chunk's stage has been read out
        if (c > 0) {
          tma_wait_read1();
          mbar_arrive(empty3((c - 1) % S3));
        }
      }
    }
    if (in && !G1) dvec[row] = marked ? 0.0 : nrm;
    double t = in ? nrm : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) s_red[q] = t;
    mbar_arrive(red_bar);
    if (et == 0) {
      if (mbar_wait(red_bar, 0, abort, lim) && !G1) {
        partials[2 * blockIdx.x] = (s_red[0] + s_red[1]) + (s_red[2] + s_red[3]);
        partials[2 * blockIdx.x + 1] = 0.0;
      }
      tma_wait_all0();
    }
  }

  tc_before();
  __syncthreads();
  if (s_abort) {
    // every role has left its loop: the producer waits for the fills it issued
    // into both rings and the MMA issuer for its MMAs before the memory is
    // released (the epilogue's stores were waited for above)
    if (threadIdx.x == 0) {
      drain_ring(full1(0), S1, fills1);
      drain_ring(full3(0), S3, fills3);
    }
    if (warp == 1 && lane == 0) drain_mma(drain);
    tc_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      st->status = RBRP_ETIMEOUT;
      st->done = 1;
    }
  }
  if (warp == 1) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ persistent form
// Plain TF32, b'_pad <= 64.  One CTA per SM walks tiles of prows <= 128 rows,
// t = blockIdx.x, blockIdx.x + gridDim.x, ...; GEMM 1 of tile t+1 streams R from
// HBM through ring 1 while GEMM 2 of tile t re-reads R (mostly from L2) through
// ring 3.  The host picks prows (a multiple of 8) so that every CTA walks the same
// number of tiles, up to one: with 128-row tiles, 10^5 rows on 152 SMs leave 22 CTAs
// a sixth tile that the other 130 wait for (rows prows..127 of the MMA are unused).
//
// On sm_103a one tcgen05.mma of kind::tf32 (K = 8) occupies the SM's tensor
// pipe for ~100 cycles up to N = 128 and reaches the full rate only at large N,
// so the kernel is built to issue few, wide MMAs: all 128 rows of M are real
// rows; GEMM 2 runs as 128-column chunks (N = 128) with its A operand (Lhat)
// read straight from the GEMM-1 accumulator in tensor memory; the epilogue
// then walks each chunk in 32-column pieces through its own shared-memory ring.
// Loads take 1.5-2.5 us under this traffic; the rings are sized for that.
// Roles: warp 0 loads ring 1, warp 1 owns TMEM and issues GEMM 1, warp 2 loads
// the R pieces of ring 3, warp 3 issues GEMM 2, warps 4-7 (one TMEM lane
// quarter each, thread <-> row) are the epilogue, warp 8 stores finished R
// pieces, warp 9 loads the Q'^T chunks.  D1 (Lhat) and D2 are double-buffered.
constexpr int PROWS = 128;        // the MMA's M: rows prows .. 127 of a tile are don't-care
constexpr int PNB = 128;          // columns per GEMM-2 chunk (MMA N)
constexpr int PPC = PNB / NB2;    // 32-column epilogue pieces per chunk
constexpr int PSB = 1;            // Q'^T chunk stages: load, MMA (a chunk lasts ~8 kcycles)
constexpr int kPTileRows = 128;   // TR of the form the dispatch launches

// TR: the largest tile height (rows per stage); shorter stages give deeper rings in
// the same shared memory.  Ring 1 holds R and Q' chunks, ring 3 the re-read R pieces.
// SPLIT: the 3xTF32 form (hi*hi + hi*lo + lo*hi): ring 1 holds [R][Q' hi][R lo][Q' lo]
// (R as loaded serves as its hi half; four converter warps write R lo), the Q'^T stage
// its hi and lo halves, and tensor memory Lhat's hi and lo halves (the epilogue writes
// them back as GEMM 2's A).
template <int BMAX, int TR, bool SPLIT = false>
struct PCfg {
  static_assert(TR == 128 || TR == 96 || TR == 64, "tile height");
  static_assert(!SPLIT || TR == 128, "the split form uses 128-row stages");
  static_assert(TR <= PROWS, "the MMA's M bounds the tile height");
  static constexpr int NOP = SPLIT ? 2 : 1;           // hi (and lo) copies of an operand
  static constexpr int PS1 = SPLIT ? 3 : (TR == 128 ? 4 : (TR == 96 ? 5 : 6));   // ring-1 stages
  static constexpr int PS3 = SPLIT ? 3 : (TR == 128 ? 6 : (TR == 96 ? 7 : 12));  // ring-3 stages
  // GEMM-2 chunk width (MMA N): the split form's 64 leaves room for a third ring-1 stage
  static constexpr int NB = SPLIT ? 64 : PNB;
  static constexpr int PC = NB / NB2;                 // 32-column epilogue pieces per chunk
  static constexpr int THREADS = SPLIT ? 448 : 320;
  static constexpr int A1 = TR * BK1 * 4;             // one R chunk (prows * 128 bytes filled)
  static constexpr int B1 = BMAX * BK1 * 4;           // Q' chunk
  static constexpr int ST1 = NOP * (A1 + B1);
  static constexpr int R3 = TR * NB2 * 4;             // one R piece
  static constexpr int B2A = NB * 128;                // one 32-wide K atom of a Q'^T chunk
  static constexpr int B2 = (BMAX / 32) * B2A;        // one half (hi or lo) of a Q'^T chunk
  static constexpr int OFF3 = PS1 * ST1;
  static constexpr int OFFB = OFF3 + PS3 * R3;
  static constexpr int BAR_OFF = OFFB + PSB * NOP * B2;
  static constexpr int BAR_BYTES = (8 * (2 * PS1 + 3 * PS3 + 2 * PSB) + 104 + 8 * PS1 + 127) / 128 * 128;
  static constexpr int SMEM = BAR_OFF + BAR_BYTES + 1024;
  static_assert(ST1 % 1024 == 0 && A1 % 1024 == 0 && R3 % 1024 == 0, "swizzle atoms");
  static constexpr uint32_t D1LO = 2 * BMAX;           // SPLIT: Lhat lo x2 after Lhat (hi) x2
  static constexpr uint32_t D2COL = NOP * 2 * BMAX;    // then D2 x2 (NB columns each)
  static constexpr uint32_t TMEM_COLS = (D2COL + 2 * NB <= 256) ? 256 : 512;
  static_assert(D2COL + 2 * NB <= 512, "tensor memory");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

template <int BMAX, int TR, bool SPLIT>
__global__ void __launch_bounds__(PCfg<BMAX, TR, SPLIT>::THREADS, 1)
    k_update_tf32p(const __grid_constant__ CUtensorMap tmR, const __grid_constant__ CUtensorMap tmX,
                   const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmQlo,
                   const __grid_constant__ CUtensorMap tmQT, const __grid_constant__ CUtensorMap tmQTlo,
                   float* __restrict__ L, long long ldl, long long n,
                   long long d, int prows, const int* __restrict__ mark, double* __restrict__ dvec,
                   double* __restrict__ partials, State* st, int c0) {
  using C = PCfg<BMAX, TR, SPLIT>;
  constexpr int PS1 = C::PS1, PS3 = C::PS3;
  pdl_wait();
  if (st->done) return;
  // this launch applies columns c0 .. c0 + BMAX - 1 of Q' (a chunk of a wider block);
  // rows accepted in this block keep their residual until the last chunk (the later
  // chunks' coefficients of those rows are part of L1), which then zeroes it
  const int bp = min((int)st->bp - c0, BMAX);
  if (bp <= 0) return;
  const bool last_chunk = c0 + BMAX >= (int)st->bp;
  // the residual starts as X and is never copied: the first block's first launch
  // reads X (tmX) and stores R, every later launch reads and stores R
  const CUtensorMap* tmSrc = (st->t == 0 && c0 == 0) ? &tmX : &tmR;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sb = smem_u32(smem);
  const uint32_t sBar = sb + C::BAR_OFF;
  auto full1 = [&](int s) { return sBar + 8u * s; };
  auto empty1 = [&](int s) { return sBar + 8u * (PS1 + s); };
  auto full3 = [&](int s) { return sBar + 8u * (2 * PS1 + s); };
  auto empty3 = [&](int s) { return sBar + 8u * (2 * PS1 + PS3 + s); };
  auto epi_done = [&](int s) { return sBar + 8u * (2 * PS1 + 2 * PS3 + s); };
  auto fullb = [&](int s) { return sBar + 8u * (2 * PS1 + 3 * PS3 + s); };
  auto emptyb = [&](int s) { return sBar + 8u * (2 * PS1 + 3 * PS3 + PSB + s); };
  const uint32_t x0 = sBar + 8u * (2 * PS1 + 3 * PS3 + 2 * PSB);
  auto d1_full = [&](int b) { return x0 + 8u * b; };
  auto d1_empty = [&](int b) { return x0 + 16u + 8u * b; };
  auto d2_full = [&](int b) { return x0 + 32u + 8u * b; };
  auto d2_empty = [&](int b) { return x0 + 48u + 8u * b; };
  uint32_t* tmem_slot = (uint32_t*)(smem + (x0 + 64u - sb));
  const uint32_t drain1 = x0 + 72u, drain3 = x0 + 80u;  // abort path: MMA drains of GEMM 1 / GEMM 2
  auto lhat_ready = [&](int b) { return x0 + 88u + 8u * b; };  // SPLIT: Lhat hi/lo written back
  auto conv1 = [&](int s) { return x0 + 104u + 8u * s; };     // SPLIT: R lo of stage s written
  static_assert(8 * (2 * PS1 + 3 * PS3 + 2 * PSB) + 104 + 8 * PS1 <= C::BAR_BYTES, "barrier area");

  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long kcol = st->k + c0;
  const int N1 = (bp + 15) / 16 * 16;
  const int tno = (int)(st->t + 1);
  const int nK1 = (int)((d + BK1 - 1) / BK1);  // 32-column chunks of GEMM 1 (and epilogue pieces)
  constexpr int PNB = C::NB, PPC = C::PC;      // this form's GEMM-2 chunk width and pieces
  const int nJ = (int)((d + PNB - 1) / PNB);   // GEMM-2 chunks
  const long long ntiles = (n + prows - 1) / prows;
  const uint32_t a1_bytes = (uint32_t)(prows * BK1 * 4), r3_bytes = (uint32_t)(prows * NB2 * 4);
  // Odd blocks walk the tiles from the last: a block then starts on the tiles the
  // previous block wrote last, which are still in L2 (the residual is larger
  // than L2, so a fixed order would always start on the least recent tiles).
  // Partial sums stay indexed by the tile's position, so their order is fixed.
  const bool rev = ((st->t + c0 / BMAX) & 1) != 0;  // successive chunks of a block alternate too
  auto ptile = [&](long long tl) { return rev ? ntiles - 1 - tl : tl; };
  // GEMM 2 walks its chunks from the last (the most recently read columns
  // first); a chunk j covers pieces 4j .. min(4j + 4, nK1) - 1.
  auto npieces = [&](int j) { const int r = nK1 - PPC * j; return r < PPC ? r : PPC; };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < PS1; ++s) {
      mbar_init(full1(s), 1);
      mbar_init(empty1(s), 1);
    }
    for (int s = 0; s < PS3; ++s) {
      mbar_init(full3(s), 1);
      mbar_init(empty3(s), 1);
      mbar_init(epi_done(s), 128);
    }
    for (int s = 0; s < PSB; ++s) {
      mbar_init(fullb(s), 1);
      mbar_init(emptyb(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(d1_full(b), 1);
      mbar_init(d1_empty(b), 129);  // the epilogue (128) and the last GEMM-2 commit of the tile
      mbar_init(d2_full(b), 1);
      mbar_init(d2_empty(b), 128);
    }
    mbar_init(drain1, 1);
    mbar_init(drain3, 1);
    for (int b = 0; b < 2; ++b) mbar_init(lhat_ready(b), 128);
    for (int s = 0; s < PS1; ++s) mbar_init(conv1(s), 128);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *(volatile uint32_t*)tmem_slot;
  volatile int* abort = &s_abort;
  const uint32_t lim = st->spin_mbar;
  uint32_t fills = 0;  // TMA fills issued by this thread's ring (for the abort drain)

  if (warp == 0) {
    // ---------------- ring 1: R and Q' chunks for GEMM 1 (R asked to stay in L2)
    if (lane == 0) {
      const uint64_t keep = l2_policy_evict_last();
      uint32_t g = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int kc = 0; kc < nK1; ++kc, ++g) {
          const int s = (int)(g % PS1);
          if (!mbar_wait(empty1(s), ((g / PS1) & 1u) ^ 1u, abort, lim)) {
            ok = false;
            break;
          }
          mbar_expect_tx(full1(s), a1_bytes + (uint32_t)(C::NOP * C::B1));
          const uint32_t base = sb + s * C::ST1;
          tma_load_2d_hint(base, tmSrc, full1(s), kc * BK1, (int)(ptile(tile) * prows), keep);
          tma_load_2d(base + C::A1, &tmQ, full1(s), kc * BK1, 0);
          if (SPLIT) tma_load_2d(base + 2 * C::A1 + C::B1, &tmQlo, full1(s), kc * BK1, 0);
        }
      }
      fills = g;
    }
  } else if (warp == 1) {
    // ---------------- GEMM 1: D1[it & 1] = R_tile Q'^T
    if (lane == 0) {
      const uint32_t id1 = idesc_tf32(BM, N1);
      uint32_t g = 0, it = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        if (!mbar_wait(d1_empty(buf), ((it >> 1) & 1u) ^ 1u, abort, lim)) break;
        tc_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BMAX);
        for (int kc = 0; kc < nK1; ++kc, ++g) {
          const int s = (int)(g % PS1);
          if (!mbar_wait(full1(s), (g / PS1) & 1u, abort, lim)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t a = sb + s * C::ST1, b = a + C::A1;
          const uint32_t alo = b + C::B1, blo = alo + C::A1;
          // R hi is the chunk as loaded (the MMA reads FP32 as TF32, dropping the low 13 bits):
          // hi*hi and hi*lo start at once, lo*hi once the converters have written R lo
#pragma unroll
          for (int kk = 0; kk < BK1 / 8; ++kk) {
            mma_tf32(dt, sdesc(a + kk * 32), sdesc(b + kk * 32), id1, (kc | kk) != 0 ? 1u : 0u);
            if (SPLIT) mma_tf32(dt, sdesc(a + kk * 32), sdesc(blo + kk * 32), id1, 1u);
          }
          if (SPLIT) {
            if (!mbar_wait(conv1(s), (g / PS1) & 1u, abort, lim)) {
              ok = false;
              break;
            }
            tc_after();
#pragma unroll
            for (int kk = 0; kk < BK1 / 8; ++kk) mma_tf32(dt, sdesc(alo + kk * 32), sdesc(b + kk * 32), id1, 1u);
          }
          mma_commit(empty1(s));
        }
        if (!ok) break;
        mma_commit(d1_full(buf));
      }
    }
  } else if (warp == 2) {
    // ---------------- ring 3: R pieces of GEMM 2 (second read), for the epilogue; no cache
    // hint (marking the re-read lines evict-first measured ~2 % slower)
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int jj = 0; jj < nJ && ok; ++jj) {
          const int j = nJ - 1 - jj;
          for (int pc = 0; pc < npieces(j); ++pc, ++g) {
            const int s = (int)(g % PS3);
            if (!mbar_wait(empty3(s), ((g / PS3) & 1u) ^ 1u, abort, lim)) {
              ok = false;
              break;
            }
            mbar_expect_tx(full3(s), r3_bytes);
            tma_load_2d(sb + C::OFF3 + s * C::R3, tmSrc, full3(s), (PPC * j + pc) * NB2, (int)(ptile(tile) * prows));
          }
        }
      }
      fills = g;
    }
  } else if (warp == 9) {
    // ---------------- Q'^T chunks of GEMM 2, for the MMA
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int jj = 0; jj < nJ; ++jj, ++g) {
          const int j = nJ - 1 - jj;
          const int s = (int)(g % PSB);
          if (!mbar_wait(emptyb(s), ((g / PSB) & 1u) ^ 1u, abort, lim)) {
            ok = false;
            break;
          }
          mbar_expect_tx(fullb(s), (uint32_t)(C::NOP * C::B2));
          const uint32_t base = sb + C::OFFB + s * C::NOP * C::B2;
#pragma unroll
          for (int a = 0; a < BMAX / 32; ++a) {
            tma_load_2d(base + a * C::B2A, &tmQT, fullb(s), a * 32, j * PNB);
            if (SPLIT) tma_load_2d(base + C::B2 + a * C::B2A, &tmQTlo, fullb(s), a * 32, j * PNB);
          }
        }
      }
      fills = g;
    }
  } else if (warp == 3) {
    // ---------------- GEMM 2: D2[g & 1] = Lhat Q'(:, chunk), Lhat = D1[it & 1] in TMEM
    if (lane == 0) {
      const uint32_t id2 = idesc_tf32(BM, PNB);
      const int nk2 = N1 / 8;
      uint32_t g = 0, it = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        const int dbuf = it & 1;
        // the plain form reads Lhat from the GEMM-1 accumulator; the split form waits for
        // the epilogue's hi and lo halves
        if (!mbar_wait(SPLIT ? lhat_ready(dbuf) : d1_full(dbuf), (it >> 1) & 1u, abort, lim)) break;
        tc_after();
        const uint32_t a1 = tmem + (uint32_t)(dbuf * BMAX);
        const uint32_t a1lo = tmem + C::D1LO + (uint32_t)(dbuf * BMAX);
        for (int jj = 0; jj < nJ; ++jj, ++g) {
          const int s = (int)(g % PSB);
          const int buf = g & 1;
          if (!mbar_wait(fullb(s), (g / PSB) & 1u, abort, lim) || !mbar_wait(d2_empty(buf), ((g >> 1) & 1u) ^ 1u, abort, lim)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t dt = tmem + C::D2COL + (uint32_t)(buf * PNB);
          const uint32_t b2 = sb + C::OFFB + s * C::NOP * C::B2;
          for (int q = 0; q < nk2; ++q) {
            const int a = q >> 2, kk = q & 3;
            mma_tf32_ta(dt, a1 + (uint32_t)(q * 8), sdesc(b2 + a * C::B2A + kk * 32), id2, q != 0 ? 1u : 0u);
            if (SPLIT) {
              mma_tf32_ta(dt, a1 + (uint32_t)(q * 8), sdesc(b2 + C::B2 + a * C::B2A + kk * 32), id2, 1u);
              mma_tf32_ta(dt, a1lo + (uint32_t)(q * 8), sdesc(b2 + a * C::B2A + kk * 32), id2, 1u);
            }
          }
          mma_commit(emptyb(s));
          mma_commit(d2_full(buf));
        }
        if (!ok) break;
        mma_commit(d1_empty(dbuf));  // Lhat of this tile is no longer read
      }
    }
  } else if (warp >= 4 && warp <= 7) {
    // ---------------- epilogue: TMEM lane quarter q = warp & 3, thread <-> row
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    uint32_t g = 0, gj = 0, it = 0;
    bool ok = true;
    double part = 0.0;  // this warp's rows over the CTA's tiles, in its tile order
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
      const long long row = ptile(tile) * prows + r;
      const bool in = r < prows && row < n;  // MMA rows prows..127 are don't-care
      const bool marked = last_chunk && in && (mark[row] == tno);
      // Lhat: TMEM -> registers -> L (GEMM 2 reads it from TMEM itself)
      const int dbuf = it & 1;
      if (!mbar_wait(d1_full(dbuf), (it >> 1) & 1u, abort, lim)) break;
      tc_after();
      uint32_t v[BMAX];
      tmem_ld32(tmem + lane_base + (uint32_t)(dbuf * BMAX), *(uint32_t(*)[32])&v[0]);
      if (BMAX > 32) tmem_ld32(tmem + lane_base + (uint32_t)(dbuf * BMAX) + 32u, *(uint32_t(*)[32])&v[32 % BMAX]);
      tmem_wait_ld();
      tc_before();
      if (!SPLIT) mbar_arrive(d1_empty(dbuf));
      if (in) {
        float* lrow = L + row * ldl + kcol;
#pragma unroll
        for (int jx = 0; jx < BMAX; ++jx)
          if (jx < bp) lrow[jx] = __uint_as_float(v[jx]);
      }
      if (SPLIT) {
        // Lhat's TF32 hi (over the accumulator) and lo halves, GEMM 2's A operand
#pragma unroll
        for (int cb = 0; cb < BMAX / 32; ++cb) {
          uint32_t h[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float x = __uint_as_float(v[32 * cb + j]);
            const float hi = tf32_rn(x);
            h[j] = __float_as_uint(hi);
            v[32 * cb + j] = __float_as_uint(tf32_rn(x - hi));
          }
          tmem_st32(tmem + lane_base + (uint32_t)(dbuf * BMAX + 32 * cb), h);
          tmem_st32(tmem + lane_base + C::D1LO + (uint32_t)(dbuf * BMAX + 32 * cb), *(uint32_t(*)[32])&v[32 * cb]);
        }
        tmem_wait_st();
        tc_before();
        mbar_arrive(lhat_ready(dbuf));
        mbar_arrive(d1_empty(dbuf));
      }
      // GEMM 2 chunks, 32-column pieces: R -= Lhat Q', row norms, accepted rows zeroed
      float nrm = 0.f;  // FP32: the residual itself carries TF32 rounding
      for (int jj = 0; jj < nJ && ok; ++jj, ++gj) {
        const int j = nJ - 1 - jj;
        const int b2 = gj & 1;
        if (!mbar_wait(d2_full(b2), (gj >> 1) & 1u, abort, lim)) {
          ok = false;
          break;
        }
        tc_after();
        for (int pc = 0; pc < npieces(j); ++pc, ++g) {
          const int s = (int)(g % PS3);
          if (!mbar_wait(full3(s), (g / PS3) & 1u, abort, lim)) {
            ok = false;
            break;
          }
          uint32_t u[32];
          tmem_ld32(tmem + lane_base + C::D2COL + (uint32_t)(b2 * PNB + pc * NB2), u);
          tmem_wait_ld();
          uint8_t* rrow = smem + C::OFF3 + s * C::R3;
          // all loads first, then the arithmetic, then all stores; rows prows .. 127 lie
          // past the piece (in the next stage when the stages hold fewer than 128 rows)
          float4 x[8];
#pragma unroll
          for (int ch = 0; ch < 8; ++ch)
            x[ch] = r < prows ? *(const float4*)(rrow + swz(r, ch)) : make_float4(0.f, 0.f, 0.f, 0.f);
          float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            x[ch].x -= __uint_as_float(u[4 * ch]);
            x[ch].y -= __uint_as_float(u[4 * ch + 1]);
            x[ch].z -= __uint_as_float(u[4 * ch + 2]);
            x[ch].w -= __uint_as_float(u[4 * ch + 3]);
            if (marked) x[ch] = make_float4(0.f, 0.f, 0.f, 0.f);
            p0 = fmaf(x[ch].x, x[ch].x, p0);
            p1 = fmaf(x[ch].y, x[ch].y, p1);
            p2 = fmaf(x[ch].z, x[ch].z, p2);
            p3 = fmaf(x[ch].w, x[ch].w, p3);
          }
          if (r < prows) {
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) *(float4*)(rrow + swz(r, ch)) = x[ch];
          }
          nrm += (p0 + p1) + (p2 + p3);
          fence_async_smem();
          mbar_arrive(epi_done(s));
        }
        tc_before();
        mbar_arrive(d2_empty(b2));
      }
      if (!ok) break;
      if (in) dvec[row] = marked ? 0.0 : (double)nrm;
      double t = in ? (double)nrm : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      part += t;
    }
    // one partial per (CTA, lane quarter): the block's finalisation sums 4 x grid values
    if (lane == 0) partials[4 * blockIdx.x + q] = part;
  } else if (warp == 8) {
    // ---------------- stores of finished R pieces; one bulk store is kept reading while the
    // next is issued, and a stage is released once the store after it has been issued
    if (lane == 0) {
      const uint64_t drop = l2_policy_evict_first();
      uint32_t g = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int jj = 0; jj < nJ && ok; ++jj) {
          const int j = nJ - 1 - jj;
          for (int pc = 0; pc < npieces(j); ++pc, ++g) {
            const int s = (int)(g % PS3);
            if (!mbar_wait(epi_done(s), (g / PS3) & 1u, abort, lim)) {
              ok = false;
              break;
            }
            tma_store_2d_hint(&tmR, sb + C::OFF3 + s * C::R3, (PPC * j + pc) * NB2, (int)(ptile(tile) * prows), drop);
            tma_commit();
            if (g > 0) {
              tma_wait_read<1>();  // the previous piece's store has read its stage
              mbar_arrive(empty3((int)((g - 1) % PS3)));
            }
          }
        }
      }
      tma_wait_read<0>();
      if (g > 0) mbar_arrive(empty3((int)((g - 1) % PS3)));
      tma_wait_all0();
    }
  } else if (SPLIT && warp >= 10) {
    // ---------------- converters (split form): R lo = R - hi of each ring-1 R chunk, hi
    // being R with its low 13 mantissa bits dropped (what the MMA reads from the FP32 chunk),
    // rounded to TF32; thread <-> row, 16-byte pieces in a bank-spread order
    const int r = 32 * (warp - 10) + lane;
    uint32_t g = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      for (int kc = 0; kc < nK1; ++kc, ++g) {
        const int s = (int)(g % PS1);
        if (!mbar_wait(full1(s), (g / PS1) & 1u, abort, lim)) {
          ok = false;
          break;
        }
        uint8_t* a = smem + s * C::ST1 + (r >> 3) * 1024 + (r & 7) * 128;
        uint8_t* alo = a + C::A1 + C::B1;
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const int cc = (ch ^ (r & 7)) * 16;
          const float4 x = *(const float4*)(a + cc);
          auto tr = [](float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); };
          *(float4*)(alo + cc) = make_float4(tf32_rn(x.x - tr(x.x)), tf32_rn(x.y - tr(x.y)), tf32_rn(x.z - tr(x.z)),
                                             tf32_rn(x.w - tr(x.w)));
        }
        fence_async_smem();
        mbar_arrive(conv1(s));
      }
    }
  }

  tc_before();
  __syncthreads();
  if (s_abort) {
    // Every role has left its loop.  Before the shared and tensor memory are
    // released, each producer waits for the fills it issued and each MMA issuer
    // for the MMAs it issued (the R stores were waited for by warp 8 above).
    if (lane == 0) {
      if (warp == 0) drain_ring(full1(0), PS1, fills);
      else if (warp == 2) drain_ring(full3(0), PS3, fills);
      else if (warp == 9) drain_ring(fullb(0), PSB, fills);
      else if (warp == 1) drain_mma(drain1);
      else if (warp == 3) drain_mma(drain3);
    }
    tc_before();
    __syncthreads();
    if (threadIdx.x == 0) {
      st->status = RBRP_ETIMEOUT;
      st->done = 1;
    }
  }
  if (warp == 1) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

// Tile height and grid of the persistent form: for the fewest rounds of tr-row tiles
// over the SMs and the next two round counts, the smallest height (a multiple of 8, at
// least 32, at most tr) that covers n rows in that many rounds; of these, the one
// whose busiest CTA walks the fewest rows.
struct PTiles {
  int prows;
  long long ntiles;
  unsigned grid;
};
static PTiles ptiles(long long n, int sms, int tr) {
  const long long r0 = std::max<long long>(1, ((n + tr - 1) / tr + sms - 1) / sms);
  PTiles best{tr, (n + tr - 1) / tr, 0};
  long long best_rows = -1;
  for (long long rounds = r0; rounds < r0 + 3; ++rounds) {
    long long h = (n + sms * rounds - 1) / (sms * rounds);
    h = std::min<long long>(tr, std::max<long long>(32, (h + 7) / 8 * 8));
    const long long nt = (n + h - 1) / h;
    const long long rows = (nt + sms - 1) / sms * h;  // rows of the busiest CTA
    if (best_rows < 0 || rows < best_rows) {
      best_rows = rows;
      best.prows = (int)h;
      best.ntiles = nt;
    }
  }
  best.grid = (unsigned)std::min<long long>(best.ntiles, sms);
  return best;
}

// SM count of the current device (asked once per device): the persistent grid, and
// with it the number of partial sums the update leaves.
int device_sms() {
  static std::atomic<int> sms[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 152;
    sms[dev] = v;
  }
  return sms[dev];
}

template <int BMAX, int TR, bool SPLIT>
cudaError_t launch_pcfg(float* R, long long ldr, long long n, long long d, const float* Qp, const float* Qp_lo,
                        long long qrows, long long ldp, const float* QpT, const float* QpT_lo, long long qtcols,
                        long long ldpt, float* L, long long ldl, const int* mark, double* dvec, double* partials,
                        const State* st, int c0, cudaStream_t s, const float* X0, long long ldx0) {
  using C = PCfg<BMAX, TR, SPLIT>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  if (dev >= 64 || !(attr_set.load() >> dev & 1ULL)) {
    e = cudaFuncSetAttribute(k_update_tf32p<BMAX, TR, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set.fetch_or(1ULL << dev);
  }
  CUtensorMap mR, mX, mQ, mQT, mQlo, mQTlo;
  const PTiles pt = ptiles(n, device_sms(), TR);
  if (!make_map(&mR, R, d, n, ldr * 4, 32, pt.prows)) return cudaErrorInvalidValue;
  if (X0 ? !make_map(&mX, X0, d, n, ldx0 * 4, 32, pt.prows) : false) return cudaErrorInvalidValue;
  if (!X0) mX = mR;
  if (!make_map(&mQ, Qp, d, qrows, ldp * 4, 32, BMAX)) return cudaErrorInvalidValue;
  if (!make_map(&mQT, QpT, qtcols, d, ldpt * 4, 32, C::NB)) return cudaErrorInvalidValue;
  if (SPLIT) {
    if (!Qp_lo || !QpT_lo) return cudaErrorInvalidValue;
    if (!make_map(&mQlo, Qp_lo, d, qrows, ldp * 4, 32, BMAX)) return cudaErrorInvalidValue;
    if (!make_map(&mQTlo, QpT_lo, qtcols, d, ldpt * 4, 32, C::NB)) return cudaErrorInvalidValue;
  } else {
    mQlo = mQ;
    mQTlo = mQT;
  }
  return counted(launch_pdl(k_update_tf32p<BMAX, TR, SPLIT>, dim3(pt.grid), dim3(C::THREADS), (size_t)C::SMEM, s, mR,
                            mX, mQ, mQlo, mQT, mQTlo, L, ldl, n, d, pt.prows, mark, dvec, partials,
                            const_cast<State*>(st), c0));
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // looked up once (a function-local static is initialised exactly once, also
  // under concurrent first calls)
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

bool make_map(CUtensorMap* m, const void* ptr, long long inner, long long outer, long long row_bytes, int box_inner,
              int box_outer, bool f64) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BMAX, bool SPLIT, bool G1 = false>
cudaError_t launch_cfg(float* R, long long ldr, long long n, long long d, const float* Qp, const float* Qp_lo,
                       long long qrows, long long ldp, const float* QpT, const float* QpT_lo, long long qtcols,
                       long long ldpt, float* L, long long ldl, const int* mark, double* dvec, double* partials,
                       const State* st, int c0, cudaStream_t s, const float* X0 = nullptr, long long ldx0 = 0) {
  using C = Cfg<BMAX, SPLIT>;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(attr_set.load() >> dev & 1ULL)) {
      e = cudaFuncSetAttribute(k_update_tf32<BMAX, SPLIT, G1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
      if (e != cudaSuccess) return e;
      if (dev < 64) attr_set.fetch_or(1ULL << dev);
    }
  }
  CUtensorMap mR, mX, mQ, mQlo, mQT, mQTlo;
  if (!make_map(&mR, R, d, n, ldr * 4, 32, ROWS)) return cudaErrorInvalidValue;
  if (X0 ? !make_map(&mX, X0, d, n, ldx0 * 4, 32, ROWS) : false) return cudaErrorInvalidValue;
  if (!X0) mX = mR;
  if (!make_map(&mQ, Qp, d, qrows, ldp * 4, 32, BMAX)) return cudaErrorInvalidValue;
  if (!make_map(&mQT, QpT, qtcols, d, ldpt * 4, 32, NB2)) return cudaErrorInvalidValue;
  if (SPLIT) {
    if (!make_map(&mQlo, Qp_lo, d, qrows, ldp * 4, 32, BMAX)) return cudaErrorInvalidValue;
    if (!make_map(&mQTlo, QpT_lo, qtcols, d, ldpt * 4, 32, NB2)) return cudaErrorInvalidValue;
  } else {
    mQlo = mQ;
    mQTlo = mQT;
  }
  const unsigned grid = (unsigned)((n + ROWS - 1) / ROWS);
  k_update_tf32<BMAX, SPLIT, G1><<<grid, kThreads, C::SMEM, s>>>(mR, mX, mQ, mQlo, mQT, mQTlo, L, ldl, n, d, mark,
                                                                 dvec, partials, const_cast<State*>(st), c0);
  return counted(cudaGetLastError());
}

}  // namespace tc

// Partial sums the update leaves for launch_finalize_block: 4 per CTA of the
// persistent form (one CTA per SM, at most one per tile), or 2 per 64-row tile.
int update_tf32_parts(long long n, int bmax, int split) {
  if (bmax <= 64) return 4 * (int)tc::ptiles(n, tc::device_sms(), split ? 128 : tc::kPTileRows).grid;
  return 2 * (int)((n + tc::ROWS - 1) / tc::ROWS);
}

int update_tf32_chunk(int ldpt, int split) {
  // both forms run on the persistent kernel in chunks of up to 64 columns (a plain TF32
  // launch of 128 columns on the 64-row kernel measured slower than two persistent passes)
  (void)split;
  return ldpt < 64 ? ldpt : 64;
}

cudaError_t launch_update_tf32(float* R, long long ldr, long long n, long long d, const float* Qp, const float* Qp_lo,
                               long long ldp, const float* QpT, const float* QpT_lo, long long ldpt, float* L,
                               long long ldl, const int* mark, double* dvec, double* partials, const State* st,
                               int bmax, int split, int c0, cudaStream_t s, const float* X0, long long ldx0) {
  // columns c0 .. of Q': rows c0.. of the Qp copies, columns c0.. of the QpT copies (c0 is a
  // multiple of 64, so the bases stay 256-byte aligned for the tensor maps)
  if (c0 < 0 || c0 % 64 != 0 || c0 >= ldpt) return cudaErrorInvalidValue;
  if (X0 && ((ldx0 & 3) != 0 || ((uintptr_t)X0 & 15) != 0)) return cudaErrorInvalidValue;
  const float* Qc = Qp + (long long)c0 * ldp;
  const float* Qlc = Qp_lo ? Qp_lo + (long long)c0 * ldp : nullptr;
  const float* QTc = QpT + c0;
  const float* QTlc = QpT_lo ? QpT_lo + c0 : nullptr;
  const long long qrows = ldpt - c0, qtcols = ldpt - c0;
#define RBRP_TC_ARGS \
  R, ldr, n, d, Qc, Qlc, qrows, ldp, QTc, QTlc, qtcols, ldpt, L, ldl, mark, dvec, partials, st, c0, s, X0, ldx0
#define RBRP_TCP_ARGS \
  R, ldr, n, d, Qc, Qlc, qrows, ldp, QTc, QTlc, qtcols, ldpt, L, ldl, mark, dvec, partials, st, c0, s, X0, ldx0
  if (split) {
    if (bmax <= 32) return tc::launch_pcfg<32, 128, true>(RBRP_TCP_ARGS);
    if (bmax <= 64) return tc::launch_pcfg<64, 128, true>(RBRP_TCP_ARGS);
    return cudaErrorInvalidValue;
  }
  if (bmax <= 32) return tc::launch_pcfg<32, tc::kPTileRows, false>(RBRP_TCP_ARGS);
  if (bmax <= 64) return tc::launch_pcfg<64, tc::kPTileRows, false>(RBRP_TCP_ARGS);
#undef RBRP_TCP_ARGS
  if (bmax <= 128) return tc::launch_cfg<128, false>(RBRP_TC_ARGS);
#undef RBRP_TC_ARGS
  return cudaErrorInvalidValue;
}

// Downdate form in 3xTF32: Lhat = X Q'^T (columns c0 .. of Q') into L for every row
// of X (FP32, read only; ldx a multiple of 4 and X 16-byte aligned for the tensor map).
cudaError_t launch_lhat_tf32x3(const float* X, long long ldx, long long n, long long d, const float* Qp,
                               const float* Qp_lo, long long ldp, const float* QpT, const float* QpT_lo,
                               long long ldpt, float* L, long long ldl, const State* st, int bmax, int c0,
                               cudaStream_t s) {
  if (c0 < 0 || c0 % 64 != 0 || c0 >= ldpt) return cudaErrorInvalidValue;
  if ((ldx & 3) != 0 || ((uintptr_t)X & 15) != 0) return cudaErrorInvalidValue;
  const float* Qc = Qp + (long long)c0 * ldp;
  const float* Qlc = Qp_lo + (long long)c0 * ldp;
  const long long qrows = ldpt - c0;
  float* Xw = const_cast<float*>(X);  // GEMM 1 only reads it
  // (the Q'^T maps are encoded but not read by GEMM 1)
#define RBRP_G1_ARGS Xw, ldx, n, d, Qc, Qlc, qrows, ldp, QpT + c0, QpT_lo + c0, qrows, ldpt, L, ldl, nullptr, nullptr, \
                     nullptr, st, c0, s
  if (bmax <= 32) return tc::launch_cfg<32, true, true>(RBRP_G1_ARGS);
  if (bmax <= 64) return tc::launch_cfg<64, true, true>(RBRP_G1_ARGS);
#undef RBRP_G1_ARGS
  return cudaErrorInvalidValue;
}

}  // namespace rbrp
