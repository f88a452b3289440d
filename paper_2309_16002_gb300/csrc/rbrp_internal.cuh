// Internal declarations shared by the CUDA translation units of the RBRP library.
//
// Every per-block kernel reads the sizes it works on (b_t, b', k) from a State
// record in device memory, so that one block of Alg. 2 is a fixed sequence of
// launches whose grids depend only on the problem's maxima (n, d, b, k_cap).
// The host never needs to read a size back between blocks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/rbrp.h"

namespace rbrp {

// ---------------------------------------------------------------- device state
struct State {
  long long k;       // |S| accepted so far
  long long t;       // blocks completed (the paper's t after the block ends)
  long long b_t;     // rows drawn in the current block
  long long bp;      // rows accepted in the current block (b')
  long long k_cap;   // min(n, d, k_max)
  long long done;    // 1 once the stopping test of Alg. 2 ends the loop
  long long status;  // rbrp_status raised on the device (0 = ok)
  long long bp_pad;  // b' rounded up to a multiple of 16 (tensor-core N)
  long long sample_fallback;  // 1: the exact FP64 tree sampler must draw this block
  unsigned int spin_mbar;     // polls of one bounded mbarrier wait (tensor-core kernels)
  unsigned int spin_grid;     // polls of one bounded grid barrier (cooperative sampler)
  long long iters;            // blocks run by the device-side loop (its iteration bound)
  double D0;         // ||d0||_1
  double D;          // ||d||_1 after the last block
  double tau;        // tolerance (< 0: fixed-rank mode)
  double tau_b;      // filter tolerance (< 0: 1/b_t)
};

// A size or offset resolved on the device: c + mul * (*p)  (p may be null).
struct DimRef {
  const long long* p;
  long long c;
  long long mul;
};
__host__ __device__ inline DimRef dim_const(long long c) { return DimRef{nullptr, c, 0}; }
__host__ __device__ inline DimRef dim_dev(const long long* p, long long mul = 1, long long c = 0) {
  return DimRef{p, c, mul};
}
__device__ __forceinline__ long long dim_val(const DimRef& r) { return r.c + (r.p ? r.mul * (*r.p) : 0); }

// A strided matrix view: element (i, j) at base[off + i * rs + j * cs].
struct MatRef {
  void* base;
  DimRef off;
  long long rs, cs;
};

// C[M x N] = alpha * A[M x K] * B[K x N] + beta * C  (beta == 0 never reads C).
struct GemmArgs {
  MatRef A, B, C;
  DimRef M, N, K;
  double alpha, beta;
  void* partial;        // split-K partial sums: splits x pm x pn (TACC)
  long long pm, pn;     // partial buffer extents (maxima of M, N)
  const State* st;      // kernels return at once when st->done (if non-null)
};

// C[M x N] = alpha * A B^T (or A B) + beta * C for the small products of the
// per-block chain (k_sgemm.cu).  A is M x K with K contiguous; B is N x K with
// K contiguous (C = A B^T) or K x N with N contiguous (C = A B).  Element type
// per launch (FP32 or FP64); leading dimensions multiples of 4 and bases
// 16-byte aligned.
struct SgemmArgs {
  const void* A;
  DimRef a_off;
  long long lda;
  const void* B;
  DimRef b_off;
  long long ldb;
  void* C;
  DimRef c_off;
  long long ldc;
  DimRef M, N, K;
  double alpha, beta;
  void* partial;      // split-K partial tiles (accumulation type)
  unsigned* cnt;      // one arrival counter per output tile, zero between launches
  const int* b_rows;  // C = A B only: row r of B is row b_rows[r] of the array (null: r)
  int kc;             // K per split, a multiple of 32
  const State* st;    // kernels return at once when st->done (if non-null)
  // (FP32 cluster form with one M tile of 64 rows, optional) the Gram partial of every
  // 64-column tile tn of the result: gram[tn * 4096 + i * 64 + j] = sum over the tile's
  // columns c of C(i, c) C(j, c), rows past M and columns past N as zeros
  float* gram = nullptr;
};

// ---------------------------------------------------------------- Philox4x64-10
// Salmon et al. (SC'11): two 64x64->128 multiplies per round, Weyl key bump.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const unsigned long long n0 = hi1 ^ c[1] ^ k0;
    const unsigned long long n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// Uniform in (0, 1) for (row, block): ((w0 >> 11) + 1/2) * 2^-53.
__device__ __forceinline__ double philox_uniform(unsigned long long row, unsigned long long block,
                                                 unsigned long long seed, unsigned long long problem) {
  unsigned long long c[4] = {row, block, 0ULL, 0ULL};
  philox4x64_10(c, seed, problem);
  return ((double)(c[0] >> 11) + 0.5) * 0x1.0p-53;
}

// Order-preserving map of a double to an unsigned 64-bit key.
// The TF32 value nearest x (ties away from zero), returned as an FP32 value that
// the MMA reads exactly.  The 3xTF32 splits take hi = tf32_rn(x) and
// lo = tf32_rn(x - hi): with rounding, lo is signed and centred on zero, so the
// terms the split drops (lo*lo and the rounding of lo) carry no bias.  A
// truncating split (low bits cleared) leaves lo with the sign of x and shrinks
// every product by ~1e-6 relative; the downdate d_i - ||Lhat_i||^2 (Alg. 2,
// update step as printed) turns that into a one-sided error in d.
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ unsigned long long orderable(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
constexpr unsigned long long kIneligible = 0xFFFFFFFFFFFFFFFFULL;

// ---------------------------------------------------------------- end of a block
// Sum of np partials in a fixed order (independent of timing and of NT >= 256):
// thread t < 256 adds partials t, t + 256, ... in order (eight loads in
// flight), then the warps' sums are combined in warp order (warps past the
// eighth add exact zeros).  Every thread of the CTA calls it and gets the sum.
constexpr int kFixedSumThreads = 256;
template <int NT>
__device__ __forceinline__ double fixed_sum_partials(const double* partials, int np) {
  static_assert(NT >= kFixedSumThreads && NT % 32 == 0, "CTA size");
  __shared__ double red[NT / 32];
  const int tid = threadIdx.x, lane = tid & 31;
  double s = 0.0;
  if (tid < kFixedSumThreads) {
    for (int i0 = tid; i0 < np; i0 += 8 * kFixedSumThreads) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (i0 + u * kFixedSumThreads < np) ? partials[i0 + u * kFixedSumThreads] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[tid >> 5] = s;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) t += red[w];
  return t;
}

// Alg. 2, stopping test after a block: D = ||d||_1, k += b', t += 1.
__device__ __forceinline__ void finish_block(State* st, double D) {
  st->D = D;
  st->k += st->bp;
  st->t += 1;
  if (!isfinite(D)) {
    st->status = RBRP_ENONFINITE;
    st->done = 1;
  } else {
    const bool cap = st->k >= st->k_cap;
    const bool tol_met = (st->tau >= 0.0) && !(st->D > st->tau * st->D0);
    st->done = (cap || tol_met) ? 1 : 0;
  }
}

// ---------------------------------------------------------------- programmatic dependent launch
// The kernels of the per-block chain are launched with launch_pdl: the next
// kernel in the stream may then be scheduled as the one before it drains, and
// its first statement, pdl_wait(), returns once that kernel has completed and
// its writes are visible (at once after an ordinary launch).  Nothing calls
// the early trigger, so a kernel's CTAs are only scheduled after every CTA of
// the kernel before it has exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---------------------------------------------------------------- instrumentation
// Number of kernels the library has launched (read by rbrp_profile_end).
extern std::atomic<long long> g_kernel_launches;
inline cudaError_t counted(cudaError_t e) {
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

// ---------------------------------------------------------------- constants
constexpr int kMaxBlock = 256;      // largest b
constexpr int kSortChunk = 2048;    // sampler: elements sorted per CTA
constexpr int kGemmTile = 64;       // SIMT GEMM tile (M and N)
constexpr int kSampCap = 1024;      // candidates the two-stage sampler can rank exactly

// ---------------------------------------------------------------- launch wrappers
// (defined in k_common.cu / k_update_tc.cu; all enqueue on `s` and return the
//  launch error, never synchronise)
cudaError_t launch_init_norms(const void* X, int x_is_fp64, long long n, long long d, long long ldx,
                              void* R, int r_is_fp64, long long ldr, double* dvec, int* mark,
                              double* partials, int nparts, State* st, cudaStream_t s);
cudaError_t launch_finish_init(const double* partials, int nparts, State* st, double tau, double tau_b,
                               long long k_cap, cudaStream_t s);
// Poll limits of the bounded device waits, copied into the State of every call
// (rbrp_set_wait_limits; the defaults are far above any wait a healthy run needs).
constexpr unsigned kDefaultSpinMbar = 1u << 24;
constexpr unsigned kDefaultSpinGrid = 1u << 25;
void wait_limits(unsigned* mbar, unsigned* grid);
// row_base: the Philox counter of local row i is row_base + i (a row shard of one
// ID); keys_out (optional, b entries): the ordered keys of S_t, and then a shard
// without candidates is not marked done.
cudaError_t launch_sample(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                          unsigned long long problem, void* cand_a, void* cand_b, long long* S_t,
                          State* st, int force, cudaStream_t s, long long row_base = 0,
                          unsigned long long* keys_out = nullptr);
size_t sample_scratch_pairs(long long n, int b);
// Rows gathered into V once S_t is known (the projection step's V = R(S_t, :), or
// X(S_t, :) in the downdate form).
struct GatherSpec {
  const void* src;  // FP32 or FP64 rows, leading dimension lds
  long long lds;
  const void* src0;  // (optional) the rows read by the first block instead (same type), ld lds0
  long long lds0;
  void* V;          // FP32 or FP64 rows, leading dimension ldv (nullptr: no gather)
  long long ldv;
  long long d;
  int src64, v64;
};
// Two-stage sampler (k_sample.cu): FP32 log-domain cut + exact FP64 ranking of
// the candidates, then the gather of V; sets State::sample_fallback when the
// exact sampler (launch_sample_exact, always enqueued after it) must draw the
// block instead.  *exact_always = 1 (and nothing enqueued) when the device has no
// cooperative launches: the exact sampler then draws every block.
cudaError_t launch_sample2(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                           unsigned long long problem, void* scratch, long long* S_t, State* st,
                           const GatherSpec& g, int* exact_always, cudaStream_t s);
// Exact FP64 sampler in one launch (k_sample.cu) with the gather of V; draws the
// block when force or State::sample_fallback is set, else returns at once.
// cand_a, cand_b: sample_scratch_pairs(n, b) pairs each; scratch: the two-stage
// sampler's (its merge counter).
cudaError_t launch_sample_exact(const double* dvec, long long n, int b, int greedy, unsigned long long seed,
                                unsigned long long problem, void* cand_a, void* cand_b, void* scratch, long long* S_t,
                                State* st, int force, const GatherSpec& g, cudaStream_t s);
cudaError_t launch_sample_clear(void* scratch, long long n, cudaStream_t s);
size_t sample2_scratch_bytes(long long n);
cudaError_t launch_gather(const void* R, int r_is_fp64, long long ldr, const long long* S_t, void* V, int v_is_fp64,
                          long long ldv, long long d, int b, const State* st, cudaStream_t s);
template <typename TA, typename TB, typename TC, typename TACC>
cudaError_t launch_gemm(const GemmArgs& g, long long Mmax, long long Nmax, int splits, int tile, cudaStream_t s);
cudaError_t launch_filter(const double* G, long long ldg, const long long* S_t, double* Lc, long long ldl,
                          int* perm, long long* skel, int* mark, int b, State* st, cudaStream_t s,
                          long long mark_base = 0, long long mark_n = (1LL << 62));
// FP32 filter (plain TF32 path): as launch_filter on an FP32 Gram matrix.  Into
// Lout (b' x b', FP32, lower triangular, leading dimension ldl) it writes, for
// b <= 64 (filter_f32_writes_factor), the pivot-order factor Lc, after which
// launch_trsm_rows_f32 forms Q'_V = Lc^{-1} V_perm (and the update's copies of
// Q' when Qp is given); for larger b the explicit inverse Lc^{-1}, which a
// product with V_perm turns into Q'_V.
int filter_f32_writes_factor(int b);
cudaError_t launch_trsm_rows_f32(const float* Lc, long long ldl, const int* perm, const float* V, long long ldv,
                                 float* Y, DimRef y_off, long long ldy, long long d, float* Qp, long long ldp,
                                 float* QpT, long long ldpt, int qrows, const State* st, cudaStream_t s);
// gram (b <= 64, optional): the Gram matrix as ntn partials of 64 x 64 (SgemmArgs::gram),
// summed in order, in place of G.
cudaError_t launch_filter_f32(const float* G, long long ldg, const float* gram, int ntn, const long long* S_t,
                              float* Lout, long long ldl, int* perm, long long* skel, int* mark, int b, State* st,
                              cudaStream_t s);
cudaError_t launch_chol(const double* G, long long ldg, double* Lc, long long ldl, int b,
                        State* st, cudaStream_t s);
// Forced acceptance: the b_t candidates in the given order, no pivoting, no truncation.
cudaError_t launch_filter_forced(const double* G, long long ldg, const long long* S_t, double* Lc, long long ldl,
                                 int* perm, long long* skel, int* mark, int b, State* st, cudaStream_t s);

// Sketchy pivoting (k_lupp.cu): LU with partial pivoting of Y(:, 0:k) (row-major n x
// ldy) into the column-major scratch A (n x k); pivots to piv, their number to
// rank_status[0], a timed-out grid barrier to rank_status[1].  U12: 32 x k scratch;
// mark: n ints; scratch: lupp_scratch_bytes(sms).  sms from lupp_grid.
template <typename T>
cudaError_t launch_lupp(const T* Y, long long ldy, long long n, int k, T* A, T* U12, int* mark, long long* piv,
                        int* rank_status, void* scratch, int sms, unsigned limit, cudaStream_t s);
size_t lupp_scratch_bytes(int sms);
cudaError_t lupp_grid(int* sms);
int lupp_panel_width();
// Forced sampling step: S_t = list[k .. k + b_t), b_t = min(b, *count - k, k_cap - k).
cudaError_t launch_forced_take(const long long* list, const int* count, long long* S_t, State* st, int b,
                               cudaStream_t s);
cudaError_t launch_trsm_rows(const double* Lc, long long ldl, const int* perm, const double* V,
                             long long ldv, double* Y, DimRef y_off, long long ldy, long long d, int b,
                             const State* st, cudaStream_t s);
// FP32 copies of the new basis rows Q' from Qt (FP64 or FP32; with Qp_lo set, the TF32 hi/lo split).
cudaError_t launch_qp_lowp(const void* Qt, int q_is_fp64, long long ldq, float* Qp, float* Qp_lo, long long ldp,
                           float* QpT, float* QpT_lo, long long ldpt, long long d, int b, const State* st,
                           cudaStream_t s);
cudaError_t launch_downdate(double* L, long long ldl, long long n, const int* mark, double* dvec, double* partials,
                            int nparts, const State* st, cudaStream_t s);
// The same with FP32 coefficients (the 3xTF32 downdate form); the sums stay FP64.
cudaError_t launch_downdate_f32(float* L, long long ldl, long long n, const int* mark, double* dvec, double* partials,
                                int nparts, const State* st, cudaStream_t s);
cudaError_t launch_norms_zero(void* R, int r_is_fp64, long long ldr, long long n, long long d,
                              const int* mark, double* dvec, double* partials, int nparts,
                              const State* st, cudaStream_t s);
// loop != 0: inside the device-side block loop (the last kernel of the captured
// block), also sets the while node's condition h to "another block" unless the
// stopping test ended the loop, and ends it after k_cap + 2 iterations in any case
// (no block can run more often).
cudaError_t launch_finalize_block(const double* partials, int nparts, State* st, cudaStream_t s,
                                  cudaGraphConditionalHandle h = 0, int loop = 0);
cudaError_t launch_copy_cols_to_f64(const void* L, int l_is_fp64, long long ldl, long long n,
                                    long long c0, long long c1, double* W, long long ldw,
                                    cudaStream_t s);
cudaError_t launch_copy_cols_to_f32(const void* L, int l_is_fp64, long long ldl, long long n,
                                    long long c0, long long c1, float* W, long long ldw,
                                    cudaStream_t s);
cudaError_t launch_gather_rows_f64(const void* L, int l_is_fp64, long long ldl, const long long* rows,
                                   long long k, double* out, long long ldo, cudaStream_t s);
// count rows (indices in rows, device) of width columns each, as FP64.
cudaError_t launch_gather_rows_rect(const void* L, int l_is_fp64, long long ldl, const long long* rows,
                                    long long count, long long width, double* out, long long ldo, cudaStream_t s);
template <typename T>
cudaError_t launch_trsm_cols(T* W, long long ldw, long long n, long long j0, int nb, const double* L1,
                             long long ld1, cudaStream_t s);
// W(S, :) = I restricted to the skeleton rows that fall in [r0, r1).
cudaError_t launch_w_identity_rows(double* W, long long ldw, long long k, const long long* skel, long long r0,
                                   long long r1, cudaStream_t s);

// Small products (k_sgemm.cu).  TS: element type in memory.  TACC = float:
// FP32 products, 64 x 64 tiles; double: FP64 products, 32 x 32 tiles.  BKC
// selects C = A B^T.
template <typename TS, typename TACC, bool BKC>
cudaError_t launch_sgemm(const SgemmArgs& g, long long Mmax, long long Nmax, int splits, cudaStream_t s);
int sgemm_tile(int acc_fp64);
// FP32-accumulating products with the K splits of a tile as one thread-block
// cluster (cs in {2, 4, 8, 16}) reduced through distributed shared memory.
void sgemm_cluster(long long Mmax, long long Nmax, long long Kmax, long long target, int* cs, int* kc);
template <typename TS, bool BKC>
cudaError_t launch_sgemm_cluster(const SgemmArgs& g, long long Mmax, long long Nmax, int cs, cudaStream_t s);
void sgemm_splits(long long Mmax, long long Nmax, long long Kmax, int tile, long long target, int* splits,
                  int* kc);
constexpr int kSgemmCounters = 4096;

// tcgen05 fused residual update (k_update_tc.cu): per 128-row tile,
// Lhat = R Q'^T (TF32 in, FP32 accumulate in TMEM), R -= Lhat Q', d_i = ||R_i||^2,
// rows accepted in this block zeroed; Lhat stored to L(:, k : k + b').
// split = 1: 3xTF32 (Qp_lo / QpT_lo hold the low parts of Q').  One launch applies
// the columns c0 .. c0 + bmax - 1 of Q' (c0 a multiple of 64): the rows of Q' are
// orthonormal, so R - (R Q'^T) Q' is the same as applying its column chunks one
// after the other, and a block wider than one launch takes several (the last
// launch's norms and partial sums are the block's; launches past b' return at once).
// X0 (optional; FP32, ldx0 a multiple of 4, 16-byte aligned): the input, read in
// place of R by the first block's first launch, so R = X is never copied.
cudaError_t launch_update_tf32(float* R, long long ldr, long long n, long long d, const float* Qp,
                               const float* Qp_lo, long long ldp, const float* QpT, const float* QpT_lo,
                               long long ldpt, float* L, long long ldl, const int* mark, double* dvec,
                               double* partials, const State* st, int bmax, int split, int c0, cudaStream_t s,
                               const float* X0 = nullptr, long long ldx0 = 0);
int update_tf32_parts(long long n, int bmax, int split);
// The downdate form in 3xTF32 (update step as printed): Lhat = X Q'^T for every row
// of the FP32 input X (read only) into L(:, k + c0 ...), columns c0 .. c0 + bmax - 1
// of Q'; launch_downdate_f32 then zeroes the rows accepted earlier and downdates d.
cudaError_t launch_lhat_tf32x3(const float* X, long long ldx, long long n, long long d, const float* Qp,
                               const float* Qp_lo, long long ldp, const float* QpT, const float* QpT_lo,
                               long long ldpt, float* L, long long ldl, const State* st, int bmax, int c0,
                               cudaStream_t s);
// Columns of Q' per launch for a block of b'_pad <= ldpt columns.
int update_tf32_chunk(int ldpt, int split);

// Alg. 3 with an FP32 result on tensor cores (k_wsolve_tc.cu, k_wsolve_rl.cu): W
// (n x k) from L (FP32 or FP64, leading dimension ldl) and L1 = L(S, :) (FP64,
// k x k, ld1).  Wb (n x ldwb FP32 scratch, ldwb a multiple of 4 and >= k rounded
// up to 64, 16-byte aligned) receives the exact FP32 W columns that a later panel
// reads back (k > 512); Gh/Gl (k x ldt FP32 scratch) the transposed block-inverse
// factor G split into TF32 hi/lo.  W64 (n x k FP64, leading dimension ldw64)
// receives the result; rows of S are not set.  form_g launches the G factor
// first; rows [r0, r1) of W are then solved (r0 a multiple of
// wsolve_tc_rows_per_tile(); r1 <= r0 solves none), so the rows can be produced
// in several launches after one G.
cudaError_t launch_wsolve_tc(const void* L, int l_is_fp64, long long ldl, float* Wb, long long ldwb, double* W64,
                             long long ldw64, const double* L1, long long ld1, float* Gh, float* Gl, long long ldt,
                             long long n, long long r0, long long r1, bool form_g, long long k, State* st,
                             cudaStream_t s);
int wsolve_tc_rows_per_tile();

// Batched form (k_batched.cu): one persistent launch over P small problems.
constexpr long long kBatchMaxRows = 4096;
constexpr long long kBatchMaxCols = 256;
constexpr int kBatchMaxBlock = 32;
constexpr int kBatchMaxThreads = 512;
constexpr int kBatchMaxCtasPerSm = 2;
struct BatchedArgs {
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
  int b, greedy, exact, x_is_fp64, fp64;  // exact: always the full FP64 ranking
  long long k_max;
  unsigned long long seed;
  unsigned long long pbase;  // Philox problem id of problem 0
  uint8_t* slots;            // per-CTA workspace slots
  size_t slot_bytes;
  long long m_max, n_max, kc_max;
  unsigned int* next;        // work counter, zeroed by launch_batched
};
size_t batched_slot_bytes(long long m_max, long long n_max, long long kc_max, int b, int fp64);
int batched_sms();
size_t batched_dyn_smem(long long n_max, int fp64);
// Row widths of the batched kernel's row passes (values of a row a lane holds):
// 8 (n <= 256) or 4 (n <= 128, half the registers and multiply-adds a row).
constexpr int kBatchVecs[] = {8, 4};
// Sets the kernel's shared-memory limit for (threads, precision, n_max, row width)
// and reports how many such CTAs fit on one SM (0: the shape cannot run).
cudaError_t batched_configure(int threads, int fp64, long long n_max, int vec, int* per_sm);
// Zeroes the work counter and launches ctas CTAs of `threads` threads: two
// stream operations and nothing else, so the call can be captured in a graph
// (batched_configure must have run for this shape).
cudaError_t launch_batched(const BatchedArgs& a, int threads, int vec, int ctas, cudaStream_t s);

}  // namespace rbrp
