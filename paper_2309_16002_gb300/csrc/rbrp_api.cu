// Host orchestration of RBRP (Alg. 2) and the ID (Alg. 3) behind the C ABI of
// include/rbrp.h.  No device memory is allocated here: the caller's workspace
// is carved into the buffers below.  One block of Alg. 2 is a fixed sequence of
// launches whose sizes live in the device State; the host reads the State back
// once per group of blocks to see whether the stopping test has fired (blocks
// queued after that return at once).
#include <stdio.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "rbrp_internal.cuh"

namespace rbrp {

std::atomic<long long> g_kernel_launches{0};
constexpr int kMaxDevicesLoop = 64;

// Poll limits of the bounded device waits (rbrp_set_wait_limits).
std::atomic<unsigned> g_spin_mbar{kDefaultSpinMbar};
std::atomic<unsigned> g_spin_grid{kDefaultSpinGrid};
void wait_limits(unsigned* mbar, unsigned* grid) {
  *mbar = g_spin_mbar.load();
  *grid = g_spin_grid.load();
}

namespace {

thread_local int g_last_cuda = 0;

// ---------------------------------------------------------------- profiling (rbrp_profile_*)
struct EventPool {
  std::vector<cudaEvent_t> ev;
  size_t used = 0;
  cudaError_t next_pair(cudaEvent_t* a, cudaEvent_t* b) {
    while (ev.size() < used + 2) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev.push_back(e);
    }
    *a = ev[used];
    *b = ev[used + 1];
    used += 2;
    return cudaSuccess;
  }
};

struct Profile {
  bool on = false;
  long long launches0 = 0;
  EventPool upd, wsv;
  long long blocks = 0, skel = 0;
};
Profile g_prof;

// Records an event pair around `body` on stream s when profiling is on.
template <typename F>
cudaError_t timed(EventPool& pool, cudaStream_t s, F&& body) {
  if (!g_prof.on) return body();
  cudaEvent_t a, b;
  cudaError_t e = pool.next_pair(&a, &b);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventRecord(a, s)) != cudaSuccess) return e;
  if ((e = body()) != cudaSuccess) return e;
  return cudaEventRecord(b, s);
}

struct Plan {
  long long n, d, k_cap;
  int b, prec, r64, l64, w32, greedy, f32, exact_sampler, downdate;
  int chain64;  // FP64 storage and FP64 products for every step of the per-block chain
  int forced;   // skeletons taken from a given list (the OSID pass of sketchy pivoting)
  long long ldr, ldl, ldq, ldp, ldpt, ldc, ldg, ldlc, ldw32, ldt;
  int nparts;
  int s_upd1, s_upd2;
  size_t pm, pn;  // split-K partial buffer extents (elements per split)
  size_t partial_elems;
  size_t off_R, off_L, off_Q, off_d, off_mark, off_part, off_state, off_St, off_ca, off_cb, off_V, off_Y, off_C,
      off_G, off_Lc, off_perm, off_gp, off_Qp, off_QpT, off_Qplo, off_QpTlo, off_L1, off_Wh, off_Gh, off_Gl,
      off_samp2, off_cnt, off_gram, total;
};

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// K-splits so that about `target` CTAs get work, each at least one 16-deep K step.
// FP64 products want every SM busy (~4 CTAs per SM); FP32 products are cheap
// enough that fewer splits (less partial-sum traffic) win.
int splits_for(long long M, long long N, long long K, int tile = kGemmTile, long long target = 608) {
  const long long tiles = ((M + tile - 1) / tile) * ((N + tile - 1) / tile);
  long long s = (target + tiles - 1) / std::max(1LL, tiles);
  const long long kmax = std::max(1LL, (K + 15) / 16);
  s = std::min(s, kmax);
  s = std::max(1LL, std::min(s, 256LL));
  return (int)s;
}

rbrp_status make_plan(long long n, long long d, const rbrp_opts* o, Plan* p, int forced = 0,
                      long long kc_force = 0) {
  if (!o || n <= 0 || d <= 0) return RBRP_EINVAL;
  if (o->block < 1 || o->block > kMaxBlock) return RBRP_EINVAL;
  if (o->precision < RBRP_FP64 || o->precision > RBRP_TF32X3) return RBRP_EINVAL;
  if (o->sampler < RBRP_SAMPLER_RANDOM || o->sampler > RBRP_SAMPLER_GREEDY_EXACT) return RBRP_EINVAL;
  if (o->w_precision != RBRP_W_FP64 && o->w_precision != RBRP_W_FP32) return RBRP_EINVAL;
  if (o->tau_b > 1.0) return RBRP_EINVAL;
  if (o->form != RBRP_FORM_RESIDUAL && o->form != RBRP_FORM_DOWNDATE) return RBRP_EINVAL;
  // the downdate cancels: FP64, or the 3xTF32 split (FP32-accurate coefficients, FP64 d)
  if (o->form == RBRP_FORM_DOWNDATE && o->precision != RBRP_FP64 && o->precision != RBRP_TF32X3) return RBRP_EINVAL;
  if (o->chain != RBRP_CHAIN_DEFAULT && o->chain != RBRP_CHAIN_FP64) return RBRP_EINVAL;
  if (n >= (1LL << 31) || d >= (1LL << 31)) return RBRP_EINVAL;
  if (n > (1LL << 48) / d) return RBRP_EINVAL;  // n d elements: every byte count below stays far from overflow
  // the FP32 filter of the plain TF32 chain takes b <= 128 candidates (the tensor-core
  // update itself takes any b <= 256, in column chunks of Q')
  if (o->precision == RBRP_TF32 && o->chain != RBRP_CHAIN_FP64 && !forced && o->block > 128) return RBRP_EINVAL;
  memset(p, 0, sizeof(*p));
  p->n = n;
  p->d = d;
  long long kc = std::min(n, d);
  if (o->k_max > 0) kc = std::min(kc, (long long)o->k_max);
  if (kc_force > 0) kc = std::min(d, kc_force);  // a row shard: the whole ID's rank cap
  p->k_cap = kc;
  p->b = o->block;
  p->prec = o->precision;
  p->r64 = (o->precision == RBRP_FP64);
  p->l64 = p->r64;
  p->w32 = (o->w_precision == RBRP_W_FP32);
  p->forced = forced;
  // the forced pass runs the FP64 chain: its filter is the FP64 Cholesky in the given order
  p->chain64 = (o->precision == RBRP_FP64 || o->chain == RBRP_CHAIN_FP64 || forced);
  p->f32 = (o->precision == RBRP_TF32 && !p->chain64);  // FP32 storage for the per-block chain
  p->greedy = (o->sampler == RBRP_SAMPLER_GREEDY || o->sampler == RBRP_SAMPLER_GREEDY_EXACT);
  p->exact_sampler = (o->sampler == RBRP_SAMPLER_RANDOM_EXACT || o->sampler == RBRP_SAMPLER_GREEDY_EXACT);
  p->downdate = (o->form == RBRP_FORM_DOWNDATE);
  p->ldr = round_up(d, 32);
  p->ldq = round_up(d, 32);
  p->ldl = round_up(kc, 8);
  p->ldp = p->ldq;
  p->ldpt = round_up(p->b, 32);
  p->ldc = round_up(kc, 8);
  p->ldg = p->b;
  p->ldlc = kMaxBlock;
  p->ldw32 = round_up(kc, 64);  // whole 64-column blocks of the read-back copy
  p->ldt = round_up(kc, 32);
  {
    long long np = (n + 7) / 8;
    p->nparts = (int)std::min(np, 4LL * 152);
  }
  const long long b = p->b;
  p->s_upd1 = splits_for(n, b, d);
  p->s_upd2 = splits_for(n, d, b);
  size_t need = 0;
  if (p->prec == RBRP_FP64 || p->prec == RBRP_FP32) {
    need = std::max<size_t>(need, (size_t)p->s_upd1 * n * b);
    need = std::max<size_t>(need, (size_t)p->s_upd2 * n * d);
  }
  need = std::max<size_t>(need, (size_t)splits_for(n, 64, kc) * n * 64);
  {
    // small products (k_sgemm.cu): splits x tiles x tile^2 FP64 partials
    const int cgs64 = p->chain64, gram64 = !p->f32;
    auto sg_need = [&](long long M, long long N, long long K, int acc64) {
      const int tile = sgemm_tile(acc64);
      int sp = 1, kcs = 0;
      sgemm_splits(M, N, K, tile, acc64 ? 608 : 160, &sp, &kcs);
      const long long tiles = ((M + tile - 1) / tile) * ((N + tile - 1) / tile);
      return (size_t)sp * tiles * tile * tile;
    };
    need = std::max<size_t>(need, sg_need(b, kc, d, cgs64));
    need = std::max<size_t>(need, sg_need(b, d, kc, cgs64));
    need = std::max<size_t>(need, sg_need(b, b, d, gram64));
  }
  p->partial_elems = need;

  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off = (size_t)round_up((long long)(off + bytes), 256);
    return o2;
  };
  const size_t sR = p->r64 ? 8 : 4, sL = p->l64 ? 8 : 4;
  p->off_R = take(p->downdate ? 0 : (size_t)n * p->ldr * sR);  // the downdate form keeps no residual
  p->off_L = take((size_t)n * p->ldl * sL);
  p->off_Q = take((size_t)kc * p->ldq * 8 + (size_t)kMaxBlock * p->ldq * 8);
  p->off_d = take((size_t)n * 8);
  p->off_mark = take((size_t)n * 4);
  p->off_part = take((size_t)std::max<long long>(std::max(p->nparts, 1024),
                                                  std::max(update_tf32_parts(n, 64, 0), update_tf32_parts(n, 128, 0))) *
                     8);
  p->off_state = take(sizeof(State));
  p->off_St = take((size_t)kMaxBlock * 8);
  p->off_ca = take(sample_scratch_pairs(n, p->b) * 16);
  p->off_cb = take(sample_scratch_pairs(n, p->b) * 16);
  p->off_V = take((size_t)b * p->ldq * 8);
  p->off_Y = take((size_t)b * p->ldq * 8);
  p->off_C = take((size_t)b * p->ldc * 8);
  p->off_G = take((size_t)b * b * 8);
  p->off_Lc = take((size_t)(kMaxBlock * p->ldlc + kMaxBlock * kMaxBlock) * 8);
  p->off_perm = take((size_t)kMaxBlock * 4);
  p->off_gp = take(p->partial_elems * 8);
  p->off_Qp = take((size_t)p->ldpt * p->ldp * 4);
  p->off_QpT = take((size_t)p->ldq * p->ldpt * 4);
  p->off_Qplo = take(p->prec == RBRP_TF32X3 ? (size_t)p->ldpt * p->ldp * 4 : 0);
  p->off_QpTlo = take(p->prec == RBRP_TF32X3 ? (size_t)p->ldq * p->ldpt * 4 : 0);
  p->off_L1 = take((size_t)kc * kc * 8);
  p->off_Wh = take(p->w32 ? (size_t)n * p->ldw32 * 4 : 0);
  p->off_Gh = take(p->w32 ? (size_t)kc * p->ldt * 4 : 0);
  p->off_Gl = take(p->w32 ? (size_t)kc * p->ldt * 4 : 0);
  p->off_samp2 = take(sample2_scratch_bytes(n));
  p->off_cnt = take((size_t)kSgemmCounters * 4);
  p->off_gram = take((p->f32 && filter_f32_writes_factor(p->b)) ? (size_t)((d + 63) / 64) * 4096 * 4 : 0);
  p->total = off;
  return RBRP_OK;
}

#define CK(call)                        \
  do {                                  \
    cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) {            \
      g_last_cuda = (int)e_;            \
      return RBRP_ECUDA;                \
    }                                   \
  } while (0)

struct Bufs {
  const void* X;  // the input (read by the downdate form)
  int x64;
  long long ldx;
  void* R;
  void* L;
  double* Qt;
  double* dvec;
  int* mark;
  double* part;
  State* st;
  long long* S_t;
  void* ca;
  void* cb;
  double* V;
  double* Y;
  double* C;
  double* G;
  double* Lc;
  int* perm;
  void* gp;
  float* Qp;
  float* QpT;
  float* Qp_lo;
  float* QpT_lo;
  double* L1;
  float* Wh;
  float* Gh;
  float* Gl;
  void* samp2;
  float* gram32;  // FP32 path, b <= 64: Gram partials of the CGS product's column tiles
  unsigned* cnt;
  long long* skel;
  const long long* forced_list;  // forced pass: the skeletons in order
  const int* forced_count;       // forced pass: their number (device)
  long long mark_base, mark_n;   // rows [mark_base, mark_base + mark_n) of the ID are this residual's
  int r_from_x = 0;  // R = X is not copied: the first block reads X (FP32 tensor-core update paths)
  cudaGraphConditionalHandle loop_h = 0;  // the while node's condition, while the loop body is captured
  int loop = 0;                           // 1 while the loop body is captured
};

Bufs carve(const Plan& p, void* ws) {
  char* b = (char*)ws;
  Bufs u;
  u.R = b + p.off_R;
  u.L = b + p.off_L;
  u.Qt = (double*)(b + p.off_Q);
  u.dvec = (double*)(b + p.off_d);
  u.mark = (int*)(b + p.off_mark);
  u.part = (double*)(b + p.off_part);
  u.st = (State*)(b + p.off_state);
  u.S_t = (long long*)(b + p.off_St);
  u.ca = b + p.off_ca;
  u.cb = b + p.off_cb;
  u.V = (double*)(b + p.off_V);
  u.Y = (double*)(b + p.off_Y);
  u.C = (double*)(b + p.off_C);
  u.G = (double*)(b + p.off_G);
  u.Lc = (double*)(b + p.off_Lc);
  u.perm = (int*)(b + p.off_perm);
  u.gp = b + p.off_gp;
  u.Qp = (float*)(b + p.off_Qp);
  u.QpT = (float*)(b + p.off_QpT);
  u.Qp_lo = (p.prec == RBRP_TF32X3) ? (float*)(b + p.off_Qplo) : nullptr;
  u.QpT_lo = (p.prec == RBRP_TF32X3) ? (float*)(b + p.off_QpTlo) : nullptr;
  u.L1 = (double*)(b + p.off_L1);
  u.Wh = p.w32 ? (float*)(b + p.off_Wh) : nullptr;
  u.Gh = p.w32 ? (float*)(b + p.off_Gh) : nullptr;
  u.Gl = p.w32 ? (float*)(b + p.off_Gl) : nullptr;
  u.samp2 = b + p.off_samp2;
  u.gram32 = (float*)(b + p.off_gram);
  u.cnt = (unsigned*)(b + p.off_cnt);
  u.skel = nullptr;
  u.forced_list = nullptr;
  u.forced_count = nullptr;
  u.mark_base = 0;
  u.mark_n = p.n;
  return u;
}

MatRef mat(void* base, DimRef off, long long rs, long long cs) { return MatRef{base, off, rs, cs}; }

template <typename TA, typename TB, typename TC, typename TACC>
cudaError_t gemm(const Plan& p, const Bufs& u, MatRef A, MatRef B, MatRef C, DimRef M, DimRef N, DimRef K,
                 double alpha, double beta, long long Mmax, long long Nmax, int splits, const State* st,
                 cudaStream_t s, int tile = kGemmTile) {
  GemmArgs g;
  g.A = A;
  g.B = B;
  g.C = C;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.partial = u.gp;
  g.pm = Mmax;
  g.pn = Nmax;
  g.st = st;
  if ((size_t)splits * Mmax * Nmax > p.partial_elems) splits = 1;
  return launch_gemm<TA, TB, TC, TACC>(g, Mmax, Nmax, splits, tile, s);
}

// Small product of the per-block chain (k_sgemm.cu); BKC: C = A B^T, else C = A B.
template <typename TS, typename TACC, bool BKC>
cudaError_t sgemm(const Plan& p, const Bufs& u, const void* A, DimRef a_off, long long lda, const void* B,
                  DimRef b_off, long long ldb, void* C, DimRef c_off, long long ldc, DimRef M, DimRef N, DimRef K,
                  long long Mmax, long long Nmax, long long Kmax, double alpha, double beta, cudaStream_t s,
                  const int* b_rows = nullptr, float* gram = nullptr) {
  SgemmArgs g;
  g.b_rows = b_rows;
  g.gram = gram;
  g.A = A;
  g.a_off = a_off;
  g.lda = lda;
  g.B = B;
  g.b_off = b_off;
  g.ldb = ldb;
  g.C = C;
  g.c_off = c_off;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.alpha = alpha;
  g.beta = beta;
  g.partial = u.gp;
  g.cnt = u.cnt;
  g.st = u.st;
  const int acc64 = sizeof(TACC) == 8;
  if (!acc64) {
    // FP32 accumulation: split-K reduced inside a thread-block cluster
    int cs = 1, kcl = 32;
    sgemm_cluster(Mmax, Nmax, Kmax, 160, &cs, &kcl);
    if (cs > 1 || gram) {  // (the Gram partials come from the cluster form only)
      g.kc = kcl;
      return launch_sgemm_cluster<TS, BKC>(g, Mmax, Nmax, cs, s);
    }
  }
  const int tile = sgemm_tile(acc64);
  int splits = 1, kc = 32;
  sgemm_splits(Mmax, Nmax, Kmax, tile, acc64 ? 608 : 160, &splits, &kc);
  const long long tiles = ((Mmax + tile - 1) / tile) * ((Nmax + tile - 1) / tile);
  if ((size_t)splits * tiles * tile * tile > p.partial_elems || tiles > kSgemmCounters) {
    splits = 1;
    kc = (int)((Kmax + 31) / 32 * 32);
  }
  g.kc = kc;
  return launch_sgemm<TS, TACC, BKC>(g, Mmax, Nmax, splits, s);
}

// V <- V - (V Qt^T) Qt on rows [0, rows) of V (rows from the device), in FP64.
//
// V and Q stay FP64 and the correction is subtracted in FP64.  On the mixed
// paths (TF32 / FP32 residual) the correction products use FP32 (TACC = float):
// the rows of V come from a residual that is already orthogonal to Q up to the
// update's rounding, so the coefficients are small and each pass shrinks the
// component in span(Q) by the FP32 product accuracy (~1e-7); two passes leave
// it at FP64 level.  The FP64 path, and any path with the FP64 chain
// (RBRP_CHAIN_FP64), keeps FP64 products throughout.
template <typename TS, typename TACC>
cudaError_t cgs_pass_t(const Plan& p, const Bufs& u, void* V, DimRef voff, DimRef rows, cudaStream_t s,
                       float* gram = nullptr) {
  const State* st = u.st;
  const long long kc = p.k_cap, b = p.b;
  // C = V Qt^T  (rows x k)
  cudaError_t e = sgemm<TS, TACC, true>(p, u, V, voff, p.ldq, u.Qt, dim_const(0), p.ldq, u.C, dim_const(0), p.ldc,
                                        rows, dim_dev(&st->k), dim_const(p.d), b, kc, p.d, 1.0, 0.0, s);
  if (e != cudaSuccess) return e;
  // V -= C Qt
  return sgemm<TS, TACC, false>(p, u, u.C, dim_const(0), p.ldc, u.Qt, dim_const(0), p.ldq, V, voff, p.ldq, rows,
                                dim_const(p.d), dim_dev(&st->k), b, p.d, kc, -1.0, 1.0, s, nullptr, gram);
}

// V (rows [0, rows) at V + voff, leading dimension ldq) <- V - (V Qt^T) Qt over Qt rows [0, k).
// FP32 storage and products on the plain TF32 path; FP64 storage with FP32
// products on the other mixed paths; FP64 throughout on the FP64 path.
// gram (FP32 path, b <= 64): also the Gram partials of the result's column tiles.
cudaError_t cgs_pass(const Plan& p, const Bufs& u, void* V, DimRef rows, cudaStream_t s,
                     DimRef voff = dim_const(0), float* gram = nullptr) {
  if (p.f32) return cgs_pass_t<float, float>(p, u, V, voff, rows, s, gram);
  if (p.chain64) return cgs_pass_t<double, double>(p, u, V, voff, rows, s);
  return cgs_pass_t<double, float>(p, u, V, voff, rows, s);
}

cudaError_t enqueue_update_simt(const Plan& p, const Bufs& u, cudaStream_t s);

cudaError_t enqueue_chain(const Plan& p, const Bufs& u, const rbrp_opts* o, cudaStream_t s);

// One block of Alg. 2 (sampling through the new residual norms), all sizes on the device.
cudaError_t enqueue_block(const Plan& p, const Bufs& u, const rbrp_opts* o, cudaStream_t s) {
  State* st = u.st;
  const long long n = p.n, d = p.d;
  cudaError_t e;
#define LK(call)                     \
  do {                               \
    e = (call);                      \
    if (e != cudaSuccess) return e;  \
  } while (0)
  // projection step, first half, done by the sampler: V = R(S_t, :), or X(S_t, :) in the
  // downdate form (the update step as printed; projected in the chain)
  GatherSpec g;
  if (p.downdate) {
    g.src = u.X;
    g.src64 = u.x64;
    g.lds = u.ldx;
    g.v64 = 1;
  } else {
    g.src = u.R;
    g.src64 = p.r64;
    g.lds = p.ldr;
    g.v64 = !p.f32;
  }
  g.src0 = u.r_from_x ? u.X : nullptr;  // the first block reads X in place of R
  g.lds0 = u.ldx;
  g.V = u.V;
  g.ldv = p.ldq;
  g.d = d;
  // sampling step: S_t (two-stage sampler; the exact sampler runs only if it asks for it),
  // or, in the forced pass, the next rows of the given skeleton list
  if (p.forced) {
    LK(launch_forced_take(u.forced_list, u.forced_count, u.S_t, st, p.b, s));
    if (p.downdate)
      LK(launch_gather(const_cast<void*>(u.X), u.x64, u.ldx, u.S_t, u.V, 1, p.ldq, d, p.b, st, s));
    else
      LK(launch_gather(u.R, p.r64, p.ldr, u.S_t, u.V, !p.f32, p.ldq, d, p.b, st, s));
  } else {
    int exact_always = p.exact_sampler;
    if (!exact_always)
      LK(launch_sample2(u.dvec, n, p.b, p.greedy, o->seed, o->problem, u.samp2, u.S_t, st, g, &exact_always, s));
    LK(launch_sample_exact(u.dvec, n, p.b, p.greedy, o->seed, o->problem, u.ca, u.cb, u.samp2, u.S_t, st,
                           exact_always, g, s));
  }
  return enqueue_chain(p, u, o, s);
}

// The rest of a block once V = the candidates' rows (b_t of them, in S_t order) is in
// place: projection against Q, the robust filter, acceptance, update, stopping test.
cudaError_t enqueue_chain(const Plan& p, const Bufs& u, const rbrp_opts* o, cudaStream_t s) {
  State* st = u.st;
  const long long n = p.n, d = p.d, b = p.b;
  cudaError_t e;
  (void)o;
  // (one pass on the plain TF32 path: the sampled residual rows are orthogonal
  // to Q up to the TF32 rounding of the update, and one FP32 pass already takes
  // that to the FP32 floor, which a second FP32 pass cannot lower)
  // local CPQR and truncation: G = V V^T, pivoted Cholesky with the tail-mass truncation
  // (on the FP32 path with b <= 64 the CGS product leaves the Gram partials of its
  // column tiles, which the filter sums)
  const bool gram_fused = p.f32 && filter_f32_writes_factor((int)p.b);
  LK(cgs_pass(p, u, u.V, dim_dev(&st->b_t), s, dim_const(0), gram_fused ? u.gram32 : nullptr));
  if (!p.f32) LK(cgs_pass(p, u, u.V, dim_dev(&st->b_t), s));
  if (p.f32) {
    // FP32 chain: Gram, filter with Lc^{-1}, Q'_V = Lc^{-1} V_perm as one
    // product.  Q'_V is a combination of rows already projected off Q, so its
    // component in span(Q) stays ~cond(Lc) times the FP32 floor, far below the
    // TF32 rounding of the update; it is not projected again.
    if (!gram_fused)
      LK((sgemm<float, float, true>(p, u, u.V, dim_const(0), p.ldq, u.V, dim_const(0), p.ldq, u.G, dim_const(0),
                                    p.ldg, dim_dev(&st->b_t), dim_dev(&st->b_t), dim_const(d), b, b, d, 1.0, 0.0, s)));
    LK(launch_filter_f32((const float*)u.G, p.ldg, gram_fused ? u.gram32 : nullptr, (int)((d + 63) / 64), u.S_t,
                         (float*)u.Lc, p.ldlc, u.perm, u.skel, u.mark, p.b, st, s));
    if (filter_f32_writes_factor((int)p.b))  // also writes the update's copies of Q' (no k_qp_lowp)
      LK(launch_trsm_rows_f32((const float*)u.Lc, p.ldlc, u.perm, (const float*)u.V, p.ldq, (float*)u.Qt,
                              dim_dev(&st->k, p.ldq), p.ldq, d, u.Qp, p.ldp, u.QpT, p.ldpt, (int)p.ldpt, st, s));
    else
      LK((sgemm<float, float, false>(p, u, u.Lc, dim_const(0), p.ldlc, u.V, dim_const(0), p.ldq, u.Qt,
                                     dim_dev(&st->k, p.ldq), p.ldq, dim_dev(&st->bp), dim_const(d), dim_dev(&st->bp),
                                     b, d, b, 1.0, 0.0, s, u.perm)));
  } else {
    LK((sgemm<double, double, true>(p, u, u.V, dim_const(0), p.ldq, u.V, dim_const(0), p.ldq, u.G, dim_const(0),
                                    p.ldg, dim_dev(&st->b_t), dim_dev(&st->b_t), dim_const(d), b, b, d, 1.0, 0.0, s)));
    if (p.forced)
      LK(launch_filter_forced(u.G, p.ldg, u.S_t, u.Lc, p.ldlc, u.perm, u.skel, u.mark, p.b, st, s));
    else
      LK(launch_filter(u.G, p.ldg, u.S_t, u.Lc, p.ldlc, u.perm, u.skel, u.mark, p.b, st, s, u.mark_base, u.mark_n));
    // Q'_V: Y = Lc^{-1} V(perm) (CholQR), then CGS against Q.  The FP64 chain
    // adds a second CholQR pass (orthogonality to FP64 rounding); with the
    // default chain of the mixed paths one FP64 CholQR already leaves
    // ~u64 * cond^2 <= ~1e-8, far below
    // the rounding of their residual update, so Q' is written in place and only
    // re-projected.
    if (p.chain64) {
      LK(launch_trsm_rows(u.Lc, p.ldlc, u.perm, u.V, p.ldq, u.Y, dim_const(0), p.ldq, d, p.b, st, s));
      LK(cgs_pass(p, u, u.Y, dim_dev(&st->bp), s));
      LK((sgemm<double, double, true>(p, u, u.Y, dim_const(0), p.ldq, u.Y, dim_const(0), p.ldq, u.G, dim_const(0),
                                      p.ldg, dim_dev(&st->bp), dim_dev(&st->bp), dim_const(d), b, b, d, 1.0, 0.0, s)));
      LK(launch_chol(u.G, p.ldg, u.Lc, p.ldlc, p.b, st, s));
      LK(launch_trsm_rows(u.Lc, p.ldlc, nullptr, u.Y, p.ldq, u.Qt, dim_dev(&st->k, p.ldq), p.ldq, d, p.b, st, s));
    } else {
      LK(launch_trsm_rows(u.Lc, p.ldlc, u.perm, u.V, p.ldq, u.Qt, dim_dev(&st->k, p.ldq), p.ldq, d, p.b, st, s));
      LK(cgs_pass(p, u, u.Qt, dim_dev(&st->bp), s, dim_dev(&st->k, p.ldq)));
    }
  }
  // update step as printed, in 3xTF32: Lhat = X Q'^T on tensor cores, d_i -= ||Lhat_i||^2 in FP64
  if (p.downdate && p.prec == RBRP_TF32X3) {
    LK(launch_qp_lowp(u.Qt, 1, p.ldq, u.Qp, u.Qp_lo, p.ldp, u.QpT, u.QpT_lo, p.ldpt, d, (int)p.ldpt, st, s));
    const int cw = update_tf32_chunk((int)p.ldpt, 1);
    LK(timed(g_prof.upd, s, [&] {
      cudaError_t ce = cudaSuccess;
      for (int c0 = 0; c0 < (int)p.ldpt && ce == cudaSuccess; c0 += cw)
        ce = launch_lhat_tf32x3((const float*)u.X, u.ldx, n, d, u.Qp, u.Qp_lo, p.ldp, u.QpT, u.QpT_lo, p.ldpt,
                                (float*)u.L, p.ldl, st, cw, c0, s);
      if (ce == cudaSuccess)
        ce = launch_downdate_f32((float*)u.L, p.ldl, n, u.mark, u.dvec, u.part, p.nparts, st, s);
      return ce;
    }));
    LK(launch_finalize_block(u.part, p.nparts, st, s, u.loop_h, u.loop));
    return cudaSuccess;
  }
  // update step (residual form): Lhat = R Q'^T, R -= Lhat Q', d_i = ||R_i||^2
  if (p.prec == RBRP_TF32 || p.prec == RBRP_TF32X3) {
    const int split = (p.prec == RBRP_TF32X3);
    if (!(p.f32 && filter_f32_writes_factor((int)p.b)))  // else the Q' substitution wrote them
      LK(launch_qp_lowp(u.Qt, !p.f32, p.ldq, u.Qp, u.Qp_lo, p.ldp, u.QpT, u.QpT_lo, p.ldpt, d, (int)p.ldpt, st, s));
    // blocks wider than one launch (above 64 columns) run as successive column chunks of Q'
    const int cw = update_tf32_chunk((int)p.ldpt, split);
    LK(timed(g_prof.upd, s, [&] {
      cudaError_t ce = cudaSuccess;
      for (int c0 = 0; c0 < (int)p.ldpt && ce == cudaSuccess; c0 += cw)
        ce = launch_update_tf32((float*)u.R, p.ldr, n, d, u.Qp, u.Qp_lo, p.ldp, u.QpT, u.QpT_lo, p.ldpt,
                                (float*)u.L, p.ldl, u.mark, u.dvec, u.part, st, cw, split, c0, s,
                                u.r_from_x ? (const float*)u.X : nullptr, u.ldx);
      return ce;
    }));
    LK(launch_finalize_block(u.part, update_tf32_parts(n, cw, split), st, s, u.loop_h, u.loop));
    return cudaSuccess;
  }
  LK(timed(g_prof.upd, s, [&] { return enqueue_update_simt(p, u, s); }));
  LK(launch_finalize_block(u.part, p.nparts, st, s, u.loop_h, u.loop));
#undef LK
  return cudaSuccess;
}

// Residual update on CUDA cores (FP64 or FP32): Lhat = R Q'^T, R -= Lhat Q', norms.
cudaError_t enqueue_update_simt(const Plan& p, const Bufs& u, cudaStream_t s) {
  State* st = u.st;
  const long long n = p.n, d = p.d, b = p.b;
  cudaError_t e;
#define LK(call)                     \
  do {                               \
    e = (call);                      \
    if (e != cudaSuccess) return e;  \
  } while (0)
  if (p.downdate) {
    // update step as printed: Lhat = X Q'^T into L(:, k : k + b'), d_i -= ||Lhat_i||^2
    if (u.x64)
      LK((gemm<double, double, double, double>(
          p, u, mat(const_cast<void*>(u.X), dim_const(0), u.ldx, 1), mat(u.Qt, dim_dev(&st->k, p.ldq), 1, p.ldq),
          mat(u.L, dim_dev(&st->k), p.ldl, 1), dim_const(n), dim_dev(&st->bp), dim_const(d), 1.0, 0.0, n, b,
          p.s_upd1, st, s)));
    else
      LK((gemm<float, double, double, double>(
          p, u, mat(const_cast<void*>(u.X), dim_const(0), u.ldx, 1), mat(u.Qt, dim_dev(&st->k, p.ldq), 1, p.ldq),
          mat(u.L, dim_dev(&st->k), p.ldl, 1), dim_const(n), dim_dev(&st->bp), dim_const(d), 1.0, 0.0, n, b,
          p.s_upd1, st, s)));
    LK(launch_downdate((double*)u.L, p.ldl, n, u.mark, u.dvec, u.part, p.nparts, st, s));
    return cudaSuccess;
  }
  if (p.prec == RBRP_FP64) {
    LK((gemm<double, double, double, double>(
        p, u, mat(u.R, dim_const(0), p.ldr, 1), mat(u.Qt, dim_dev(&st->k, p.ldq), 1, p.ldq),
        mat(u.L, dim_dev(&st->k), p.ldl, 1), dim_const(n), dim_dev(&st->bp), dim_const(d), 1.0, 0.0, n, b, p.s_upd1,
        st, s)));
    LK((gemm<double, double, double, double>(
        p, u, mat(u.L, dim_dev(&st->k), p.ldl, 1), mat(u.Qt, dim_dev(&st->k, p.ldq), p.ldq, 1),
        mat(u.R, dim_const(0), p.ldr, 1), dim_const(n), dim_const(d), dim_dev(&st->bp), -1.0, 1.0, n, d, p.s_upd2,
        st, s)));
  } else {
    LK((gemm<float, double, float, float>(
        p, u, mat(u.R, dim_const(0), p.ldr, 1), mat(u.Qt, dim_dev(&st->k, p.ldq), 1, p.ldq),
        mat(u.L, dim_dev(&st->k), p.ldl, 1), dim_const(n), dim_dev(&st->bp), dim_const(d), 1.0, 0.0, n, b, p.s_upd1,
        st, s)));
    LK((gemm<float, double, float, float>(
        p, u, mat(u.L, dim_dev(&st->k), p.ldl, 1), mat(u.Qt, dim_dev(&st->k, p.ldq), p.ldq, 1),
        mat(u.R, dim_const(0), p.ldr, 1), dim_const(n), dim_const(d), dim_dev(&st->bp), -1.0, 1.0, n, d, p.s_upd2,
        st, s)));
  }
  LK(launch_norms_zero(u.R, p.r64, p.ldr, n, d, u.mark, u.dvec, u.part, p.nparts, st, s));
#undef LK
  return cudaSuccess;
}

// Receiver of finished row ranges of W: after done(r0, r1) is called, rows
// [r0, r1) of W are final once the work queued on the stream so far completes,
// so a caller can start copying them while later rows are still being solved.
struct WSink {
  long long chunk_rows = 0;  // rows per range (rounded to whole tiles)
  cudaError_t (*done)(void* ctx, long long r0, long long r1, long long k, cudaStream_t s) = nullptr;
  void* ctx = nullptr;
};

// Alg. 3: W(S,:) = I, W(rest,:) = L2 L1^{-1}, blocked right-to-left substitution.
// l1_given: L1 is already in u.L1 (a row shard receives it from the other shards);
// skel then holds this residual's row of each skeleton (negative: not here).
rbrp_status solve_w(const Plan& p, const Bufs& u, long long k, const long long* skel, double* W, long long ldw,
                    cudaStream_t s, const WSink* sink = nullptr, bool l1_given = false) {
  if (k <= 0) return RBRP_OK;
  const long long n = p.n;
  if (!l1_given) CK(launch_gather_rows_f64(u.L, p.l64, p.ldl, skel, k, u.L1, k, s));
  const long long nblk = (k + 63) / 64;
  if (!p.w32) {
    CK(launch_copy_cols_to_f64(u.L, p.l64, p.ldl, n, 0, k, W, ldw, s));
    for (long long J = nblk - 1; J >= 0; --J) {
      const long long j0 = J * 64, nb = std::min(64LL, k - j0), rest = k - j0 - nb;
      if (rest > 0) {
        CK((gemm<double, double, double, double>(
            p, u, mat(W, dim_const(j0 + nb), ldw, 1), mat(u.L1, dim_const((j0 + nb) * k + j0), k, 1),
            mat(W, dim_const(j0), ldw, 1), dim_const(n), dim_const(nb), dim_const(rest), -1.0, 1.0, n, 64,
            splits_for(n, 64, rest), nullptr, s)));
      }
      CK(launch_trsm_cols<double>(W, ldw, n, j0, (int)nb, u.L1, k, s));
    }
    CK(launch_w_identity_rows(W, ldw, k, skel, 0, n, s));  // W(S, :) = I exactly
    if (sink) CK(sink->done(sink->ctx, 0, n, k, s));
  } else if (!sink) {
    // FP32 solve on tensor cores (3xTF32): every 64-column block of W is one
    // product with the precomputed block-inverse factor, then W(S, :) = I.
    CK(launch_wsolve_tc(u.L, p.l64, p.ldl, u.Wh, p.ldw32, W, ldw, u.L1, k, u.Gh, u.Gl, p.ldt, n, 0, n, true,
                        k, u.st, s));
    CK(launch_w_identity_rows(W, ldw, k, skel, 0, n, s));  // W(S, :) = I exactly
  } else {
    // The same solve in row ranges (rows are independent once G is formed),
    // each finished with its skeleton rows set to I and handed to the sink.
    const long long tile = wsolve_tc_rows_per_tile();
    const long long chunk = std::max(tile, (sink->chunk_rows + tile - 1) / tile * tile);
    CK(launch_wsolve_tc(u.L, p.l64, p.ldl, u.Wh, p.ldw32, W, ldw, u.L1, k, u.Gh, u.Gl, p.ldt, n, 0, 0, true,
                        k, u.st, s));
    for (long long r0 = 0; r0 < n; r0 += chunk) {
      const long long r1 = std::min(n, r0 + chunk);
      CK(launch_wsolve_tc(u.L, p.l64, p.ldl, u.Wh, p.ldw32, W, ldw, u.L1, k, u.Gh, u.Gl, p.ldt, n, r0, r1,
                          false, k, u.st, s));
      CK(launch_w_identity_rows(W, ldw, k, skel, r0, r1, s));
      CK(sink->done(sink->ctx, r0, r1, k, s));
    }
  }
  return RBRP_OK;
}

// ---------------------------------------------------------------- device-side block loop
// The blocks of Alg. 2 run as one CUDA graph: a while node whose body is one block
// (captured from enqueue_block), whose last kernel (the block's finalisation) sets
// the node's condition from the State's stopping test.  The host launches the graph once and
// reads the State once after the loop; nothing of the loop comes back to the host.
// Graphs are cached per (device, buffers, sizes, options): the captured kernels hold
// the workspace and output pointers and the plan's sizes (the tolerance lives in the
// State, so one graph serves any tol).
struct LoopKey {
  int dev, x64, pad_;
  const void* ws;
  const void* X;
  const long long* skel;
  const long long* flist;
  const int* fcount;
  long long n, d, ldx, total;
  rbrp_opts o;
};
struct LoopEntry {
  LoopKey key;
  cudaGraph_t g;
  cudaGraphExec_t x;
};
std::mutex g_loop_mu;
std::vector<LoopEntry> g_loops;
std::atomic<int> g_loop_mode{0};  // 0: device-side loop where it can be built, 1: host-side groups
int g_loop_broken[kMaxDevicesLoop] = {0};
cudaStream_t g_capture_stream[kMaxDevicesLoop] = {nullptr};
constexpr size_t kLoopCache = 8;

// Builds (or finds) the executable loop graph; cudaErrorNotSupported if this device
// cannot capture the block (the caller then queues blocks from the host).
cudaError_t loop_graph(const Plan& p, const Bufs& u, const rbrp_opts* o, const LoopKey& key, cudaGraphExec_t* out) {
  std::lock_guard<std::mutex> lock(g_loop_mu);
  for (auto& e : g_loops)
    if (memcmp(&e.key, &key, sizeof(LoopKey)) == 0) {
      *out = e.x;
      return cudaSuccess;
    }
  if (g_loop_broken[key.dev]) return cudaErrorNotSupported;
  cudaError_t e;
  if (!g_capture_stream[key.dev]) {
    e = cudaStreamCreateWithFlags(&g_capture_stream[key.dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaStream_t cs = g_capture_stream[key.dev];
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    Bufs ul = u;  // the block's last kernel sets the condition
    ul.loop_h = h;
    ul.loop = 1;
    cudaError_t be = enqueue_block(p, ul, o, cs);
    cudaGraph_t got = nullptr;
    e = cudaStreamEndCapture(cs, &got);
    if (be != cudaSuccess) e = be;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (x) cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    g_loop_broken[key.dev] = 1;  // fall back to host-side groups on this device from now on
    return cudaErrorNotSupported;
  }
  if (g_loops.size() >= kLoopCache) {
    cudaGraphExecDestroy(g_loops.front().x);
    cudaGraphDestroy(g_loops.front().g);
    g_loops.erase(g_loops.begin());
  }
  g_loops.push_back(LoopEntry{key, g, x});
  *out = x;
  return cudaSuccess;
}

// Forced skeletons for run(): the list (device, in acceptance order) and its length (device).
struct Forced {
  const long long* list;
  const int* count;
};

rbrp_status run(const void* X, int x_is_fp64, long long n, long long d, long long ldx, double tol,
                const rbrp_opts* o, void* ws, size_t ws_bytes, long long* skel, double* W, long long ldw,
                rbrp_result* res, cudaStream_t s, const WSink* sink = nullptr, const Forced* forced = nullptr) {
  Plan p;
  rbrp_status rs = make_plan(n, d, o, &p, forced ? 1 : 0);
  if (rs != RBRP_OK) return rs;
  if (!X || !skel || !W || !res || !ws) return RBRP_EINVAL;
  if (ldx < d || ldw < p.k_cap) return RBRP_EINVAL;
  // the 3xTF32 downdate reads X itself with a tensor map: FP32, 16-byte rows and base
  if (p.downdate && p.prec == RBRP_TF32X3 && (x_is_fp64 || (ldx & 3) != 0 || ((uintptr_t)X & 15) != 0))
    return RBRP_EINVAL;
  if (((uintptr_t)ws & 255) != 0 || ws_bytes < p.total) return RBRP_EWORKSPACE;
  if (!(tol < 1.0)) return RBRP_EINVAL;
  memset(res, 0, sizeof(*res));
  Bufs u = carve(p, ws);
  u.skel = skel;
  if (forced) {
    u.forced_list = forced->list;
    u.forced_count = forced->count;
  }
  u.X = X;
  u.x64 = x_is_fp64 ? 1 : 0;
  u.ldx = ldx;
  // Alg. 2's start R = X: on the FP32 tensor-core update paths the first block reads X
  // itself (sampler gather and update), so no copy of X is made; elsewhere R is a copy
  u.r_from_x = (!p.downdate && !forced && !p.r64 && !x_is_fp64 && (p.prec == RBRP_TF32 || p.prec == RBRP_TF32X3) &&
                (ldx & 3) == 0 && ((uintptr_t)X & 15) == 0)
                   ? 1
                   : 0;
  State* st = u.st;
  // Alg. 2, start and initial norms (with the copy of X into R where one is made)
  CK(launch_init_norms(X, x_is_fp64, n, d, ldx, (p.downdate || u.r_from_x) ? nullptr : u.R, p.r64, p.ldr, u.dvec,
                       u.mark, u.part, p.nparts, st, s));
  CK(launch_finish_init(u.part, p.nparts, st, tol, o->tau_b, p.k_cap, s));
  CK(launch_sample_clear(u.samp2, n, s));
  CK(cudaMemsetAsync(u.cnt, 0, (size_t)kSgemmCounters * 4, s));
  // Alg. 2's loop, on the device where the block can be captured into a graph
  // (not while the profiling counters time each update launch with events).
  State h;
  bool looped = false;
  int dev = 0;
  if (g_loop_mode.load() == 0 && !g_prof.on && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 &&
      dev < kMaxDevicesLoop) {
    LoopKey key;
    memset(&key, 0, sizeof(key));
    key.dev = dev;
    key.x64 = u.x64;
    key.ws = ws;
    key.X = X;
    key.skel = skel;
    key.flist = u.forced_list;
    key.fcount = u.forced_count;
    key.n = n;
    key.d = d;
    key.ldx = ldx;
    key.total = (long long)p.total;
    key.o = *o;
    cudaGraphExec_t gx = nullptr;
    const cudaError_t ge = loop_graph(p, u, o, key, &gx);
    if (ge == cudaSuccess) {
      CK(cudaGraphLaunch(gx, s));
      CK(cudaMemcpyAsync(&h, st, sizeof(State), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      looped = true;
    } else if (ge != cudaErrorNotSupported) {
      g_last_cuda = (int)ge;
      return RBRP_ECUDA;
    }
  }
  // Otherwise blocks are queued from the host in groups and the State is read
  // back after each group.  The group size is the number of blocks still
  // expected, extrapolated from the observed per-block decay of ||d||_1 (or of
  // the rank gap in fixed-rank mode), so that few blocks are queued past the
  // stop (those return at once) and few host round trips are needed.
  long long queued = 0;
  long long group = 2;
  for (; !looped;) {
    for (long long g = 0; g < group && queued < p.k_cap; ++g, ++queued) {
      cudaError_t e = enqueue_block(p, u, o, s);
      if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        return RBRP_ECUDA;
      }
    }
    CK(cudaMemcpyAsync(&h, st, sizeof(State), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h.done || queued >= p.k_cap) break;
    double est = 2.0;
    if (h.t > 0 && h.k > 0) {
      const double per_block_k = (double)h.k / (double)h.t;
      est = (double)(h.k_cap - h.k) / per_block_k;  // blocks to the rank cap
      if (tol >= 0.0 && h.D > 0.0 && h.D0 > 0.0 && h.D < h.D0) {
        const double rate = log(h.D0 / h.D) / (double)h.t;  // mean log-decay per block
        const double need = log(h.D / (tol * h.D0)) / rate;
        if (need < est) est = need;
      }
    }
    group = std::max<long long>(1, std::min<long long>(16, (long long)ceil(est)));
  }
  if (h.status != 0) return (rbrp_status)h.status;
  res->k = h.k;
  res->blocks = h.t;
  res->d0 = h.D0;
  res->d_final = h.D;
  res->rel_err_sq = (h.D0 > 0.0) ? h.D / h.D0 : 0.0;
  // Alg. 3
  {
    rbrp_status wrs = RBRP_OK;
    cudaError_t te = timed(g_prof.wsv, s, [&] {
      wrs = solve_w(p, u, h.k, skel, W, ldw, s, sink);
      return cudaSuccess;
    });
    if (te != cudaSuccess) {
      g_last_cuda = (int)te;
      return RBRP_ECUDA;
    }
    if (wrs != RBRP_OK) return wrs;
  }
  if (g_prof.on) {
    g_prof.blocks += h.t;
    g_prof.skel += h.k;
  }
  CK(cudaStreamSynchronize(s));
  if (tol >= 0.0 && h.D > tol * h.D0) return RBRP_ENOTCONVERGED;
  return RBRP_OK;
}

}  // namespace
// ---------------------------------------------------------------- fixed scratch for rbrp_id_noalloc
// Some callers cannot allocate device memory at all: code running inside an
// allocator-free runtime (a plugin or an embedded engine that owns every byte
// of device memory and forbids cudaMalloc once it has started), or code that
// must not add to a memory pool it does not control.  For them the workspace of
// rbrp_id_noalloc is this fixed array, which the CUDA runtime places in device
// memory when the library's module is loaded on a device; every GPU that loads
// the library keeps these RBRP_NOALLOC_SCRATCH_BYTES bytes until the process
// exits.  In host code `g_noalloc_scratch` only names a host-side stand-in, so
// the device address is looked up with cudaGetSymbolAddress (once per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[RBRP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

// Device address of the fixed scratch on the current device (looked up on first use).
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace rbrp

using namespace rbrp;

extern "C" {

void rbrp_default_opts(rbrp_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = RBRP_TF32;
  o->block = 64;
  o->tau_b = -1.0;
  o->k_max = 0;
  o->seed = 0;
  o->problem = 0;
  o->sampler = RBRP_SAMPLER_RANDOM;
  o->w_precision = RBRP_W_FP64;
}

rbrp_status rbrp_workspace_size(int64_t n, int64_t d, const rbrp_opts* o, size_t* bytes) {
  if (!bytes) return RBRP_EINVAL;
  Plan p;
  rbrp_status rs = make_plan(n, d, o, &p);
  if (rs != RBRP_OK) return rs;
  *bytes = p.total;
  return RBRP_OK;
}

rbrp_status rbrp_id(const void* X, int x_is_fp64, int64_t n, int64_t d, int64_t ldx, double tol, const rbrp_opts* o,
                    void* workspace, size_t ws_bytes, int64_t* skel, double* W, int64_t ldw, rbrp_result* res,
                    rbrp_stream_t stream) {
  return run(X, x_is_fp64, n, d, ldx, tol, o, workspace, ws_bytes, (long long*)skel, W, ldw, res,
             (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// Per-shape buckets of a batch: problems with n > kBatchNarrow columns, then those with
// n <= kBatchNarrow (the ones a row width of 4 values a lane can hold); each bucket is
// its own persistent launch with its own schedule (CTA size, CTAs per SM, row width)
// and slot size, the launches one after the other on the stream.
constexpr long long kBatchNarrow = 128;
constexpr int kBatchBuckets = 2;
struct BatchPlan {
  long long m_max, n_max, kc_max, elems;
  int slots, fp64;
  size_t off_X, off_rows, off_cols, off_order, off_skel, off_W, off_next, slot, off_slots, total;
  int nb;                                      // non-empty buckets
  int bclass[kBatchBuckets];                   // their classes: 0 wide, 1 narrow
  int bstart[kBatchBuckets], bcount[kBatchBuckets];  // their ranges in the processing order
  long long bm[kBatchBuckets], bn[kBatchBuckets], bkc[kBatchBuckets], belems[kBatchBuckets];
  size_t bslot[kBatchBuckets];
};

int batch_class(long long n) { return n > kBatchNarrow ? 0 : 1; }

rbrp_status batch_plan(int32_t P, const int64_t* m, const int64_t* n, const rbrp_opts* o, BatchPlan* bp) {
  if (P < 0 || !o || !bp || (P > 0 && (!m || !n))) return RBRP_EINVAL;
  if (o->block < 1 || o->block > kBatchMaxBlock || o->tau_b > 1.0) return RBRP_EINVAL;
  if (o->precision < RBRP_FP64 || o->precision > RBRP_TF32X3) return RBRP_EINVAL;
  if (o->sampler < RBRP_SAMPLER_RANDOM || o->sampler > RBRP_SAMPLER_GREEDY_EXACT) return RBRP_EINVAL;
  memset(bp, 0, sizeof(*bp));
  bp->m_max = bp->n_max = bp->kc_max = 1;
  for (int32_t p = 0; p < P; ++p) {
    if (m[p] < 1 || m[p] > kBatchMaxRows || n[p] < 1 || n[p] > kBatchMaxCols) return RBRP_EINVAL;
    long long kc = std::min<long long>(m[p], n[p]);
    if (o->k_max > 0) kc = std::min<long long>(kc, o->k_max);
    bp->m_max = std::max<long long>(bp->m_max, m[p]);
    bp->n_max = std::max<long long>(bp->n_max, n[p]);
    bp->kc_max = std::max<long long>(bp->kc_max, kc);
    bp->elems += (long long)m[p] * n[p];
  }
  bp->fp64 = (o->precision == RBRP_FP64);
  // the buckets, wide first
  {
    long long cm[kBatchBuckets] = {0, 0}, cn[kBatchBuckets] = {0, 0}, ckc[kBatchBuckets] = {0, 0},
              ce[kBatchBuckets] = {0, 0};
    int cnt[kBatchBuckets] = {0, 0};
    for (int32_t p = 0; p < P; ++p) {
      const int c = batch_class(n[p]);
      long long kc = std::min<long long>(m[p], n[p]);
      if (o->k_max > 0) kc = std::min<long long>(kc, o->k_max);
      cm[c] = std::max<long long>(cm[c], m[p]);
      cn[c] = std::max<long long>(cn[c], n[p]);
      ckc[c] = std::max<long long>(ckc[c], kc);
      ce[c] += (long long)m[p] * n[p];
      ++cnt[c];
    }
    int start = 0;
    for (int c = 0; c < kBatchBuckets; ++c) {
      if (cnt[c] == 0) continue;
      const int b = bp->nb++;
      bp->bclass[b] = c;
      bp->bstart[b] = start;
      bp->bcount[b] = cnt[c];
      bp->bm[b] = cm[c];
      bp->bn[b] = cn[c];
      bp->bkc[b] = ckc[c];
      bp->belems[b] = ce[c];
      bp->bslot[b] = batched_slot_bytes(cm[c], cn[c], ckc[c], o->block, bp->fp64);
      start += cnt[c];
    }
  }
  // one slot per CTA of the largest schedule (kBatchMaxCtasPerSm CTAs on every SM);
  // a bucket of smaller problems fits more of its own slots in the same space
  bp->slots = std::max(1, std::min<int>(P, batched_sms() * kBatchMaxCtasPerSm));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off = (size_t)round_up((long long)(off + bytes), 256);
    return o2;
  };
  bp->off_X = take((size_t)P * 8);
  bp->off_rows = take((size_t)P * 8);
  bp->off_cols = take((size_t)P * 8);
  bp->off_order = take((size_t)P * 4);
  bp->off_skel = take((size_t)P * 8);
  bp->off_W = take((size_t)P * 8);
  bp->off_next = take(16);
  bp->slot = batched_slot_bytes(bp->m_max, bp->n_max, bp->kc_max, o->block, bp->fp64);
  bp->off_slots = take((size_t)bp->slots * bp->slot);
  bp->total = off;
  return RBRP_OK;
}

// Autotuner memory: the fastest schedule measured for a batch of this shape.
struct TuneKey {
  int fp64, block;
  long long P, m_max, n_max, elems;
  bool operator<(const TuneKey& o) const {
    if (fp64 != o.fp64) return fp64 < o.fp64;
    if (block != o.block) return block < o.block;
    if (P != o.P) return P < o.P;
    if (m_max != o.m_max) return m_max < o.m_max;
    if (n_max != o.n_max) return n_max < o.n_max;
    return elems < o.elems;
  }
};
struct Sched {
  int threads, per_sm, vec;
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, Sched>> g_tune_cache;

bool tune_lookup(const TuneKey& k, Sched* sc) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : g_tune_cache)
    if (!(e.first < k) && !(k < e.first)) {
      *sc = e.second;
      return true;
    }
  return false;
}

void tune_store(const TuneKey& k, const Sched& sc) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& e : g_tune_cache)
    if (!(e.first < k) && !(k < e.first)) {
      e.second = sc;
      return;
    }
  g_tune_cache.push_back({k, sc});
}

constexpr int kSchedThreads[] = {256, 512};

}  // namespace

struct BatchBucket {
  BatchedArgs args;  // this bucket's queue (P, order, counter) and slot shape; tau set per run
  TuneKey key;
  int threads, per_sm, vec, ctas;
  long long slots;   // slots of this bucket's size in the slot space
};

struct rbrp_batch_s {
  BatchPlan plan;
  int nb;
  BatchBucket bk[kBatchBuckets];
};

namespace {

// The narrowest row width that holds a row of the bucket.
int default_vec(const BatchBucket& b) { return b.args.n_max <= 32LL * 4 ? 4 : 8; }

// Makes (threads, per_sm, vec) bucket b's schedule if the kernel shape fits.
rbrp_status apply_schedule(rbrp_batch_s* h, int b, int threads, int per_sm, int vec) {
  if (b < 0 || b >= h->nb) return RBRP_EINVAL;
  if (per_sm < 1 || per_sm > kBatchMaxCtasPerSm) return RBRP_EINVAL;
  BatchBucket& k = h->bk[b];
  int fit = 0;
  CK(batched_configure(threads, h->plan.fp64, k.args.n_max, vec, &fit));
  if (fit < per_sm) return RBRP_EINVAL;
  k.threads = threads;
  k.per_sm = per_sm;
  k.vec = vec;
  k.ctas = (int)std::max<long long>(1, std::min<long long>(k.slots, (long long)batched_sms() * per_sm));
  return RBRP_OK;
}

rbrp_status run_bucket(rbrp_batch_s* h, int b, double tol, cudaStream_t s) {
  BatchedArgs a = h->bk[b].args;
  a.tau = tol;
  CK(launch_batched(a, h->bk[b].threads, h->bk[b].vec, h->bk[b].ctas, s));
  return RBRP_OK;
}

}  // namespace

extern "C" {

rbrp_status rbrp_batched_workspace_size(int32_t P, const int64_t* m, const int64_t* n, const rbrp_opts* o,
                                        size_t* bytes) {
  if (!bytes) return RBRP_EINVAL;
  BatchPlan bp;
  rbrp_status rs = batch_plan(P, m, n, o, &bp);
  if (rs != RBRP_OK) return rs;
  *bytes = bp.total;
  return RBRP_OK;
}

rbrp_status rbrp_batch_create(int32_t P, const void* const* X, const int64_t* m, const int64_t* n, int x_is_fp64,
                              const rbrp_opts* o, void* workspace, size_t ws_bytes, int64_t* const* skel,
                              double* const* W, int64_t* k_out, double* rel_err_sq, int32_t* status,
                              rbrp_stream_t stream, rbrp_batch* out) {
  if (!out) return RBRP_EINVAL;
  *out = nullptr;
  BatchPlan bp;
  rbrp_status rs = batch_plan(P, m, n, o, &bp);
  if (rs != RBRP_OK) return rs;
  if (P < 1) return RBRP_EINVAL;
  if (!X || !skel || !W || !k_out || !rel_err_sq || !status || !workspace) return RBRP_EINVAL;
  for (int32_t p = 0; p < P; ++p)
    if (!X[p] || !skel[p] || !W[p]) return RBRP_EINVAL;
  if (((uintptr_t)workspace & 255) != 0 || ws_bytes < bp.total) return RBRP_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* ws = (uint8_t*)workspace;
  std::vector<long long> rows(P), cols(P);
  std::vector<int> order(P);
  for (int32_t p = 0; p < P; ++p) {
    rows[p] = m[p];
    cols[p] = n[p];
    order[p] = p;
  }
  // by bucket (wide, then narrow), largest problems first inside a bucket, so the
  // last problems of a launch to start are short ones
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ca = batch_class(cols[a]), cb = batch_class(cols[b]);
    if (ca != cb) return ca < cb;
    return rows[a] * cols[a] > rows[b] * cols[b];
  });
  CK(cudaMemcpyAsync(ws + bp.off_X, X, (size_t)P * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ws + bp.off_rows, rows.data(), (size_t)P * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ws + bp.off_cols, cols.data(), (size_t)P * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ws + bp.off_order, order.data(), (size_t)P * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ws + bp.off_skel, skel, (size_t)P * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ws + bp.off_W, W, (size_t)P * 8, cudaMemcpyHostToDevice, s));
  // (copies from pageable host memory return once the source has been read, so
  // the vectors above may be released on return)
  rbrp_batch_s* h = new (std::nothrow) rbrp_batch_s();
  if (!h) return RBRP_ENOMEM;
  h->plan = bp;
  BatchedArgs a;
  a.P = P;
  a.X = (const void* const*)(ws + bp.off_X);
  a.rows = (const long long*)(ws + bp.off_rows);
  a.cols = (const long long*)(ws + bp.off_cols);
  a.order = (const int*)(ws + bp.off_order);
  a.skel = (long long* const*)(ws + bp.off_skel);
  a.W = (double* const*)(ws + bp.off_W);
  a.k_out = (long long*)k_out;
  a.err = rel_err_sq;
  a.status = (int*)status;
  a.tau = 0.0;
  a.tau_b = o->tau_b;
  a.b = o->block;
  a.greedy = (o->sampler == RBRP_SAMPLER_GREEDY || o->sampler == RBRP_SAMPLER_GREEDY_EXACT);
  a.exact = (o->sampler == RBRP_SAMPLER_RANDOM_EXACT || o->sampler == RBRP_SAMPLER_GREEDY_EXACT);
  a.x_is_fp64 = x_is_fp64 ? 1 : 0;
  a.fp64 = bp.fp64;
  a.k_max = o->k_max;
  a.seed = o->seed;
  a.pbase = o->problem;
  a.slots = ws + bp.off_slots;
  a.slot_bytes = bp.slot;
  a.m_max = bp.m_max;
  a.n_max = bp.n_max;
  a.kc_max = bp.kc_max;
  a.next = (unsigned int*)(ws + bp.off_next);
  h->nb = bp.nb;
  for (int b = 0; b < bp.nb; ++b) {
    BatchBucket& k = h->bk[b];
    k.args = a;
    k.args.P = bp.bcount[b];
    k.args.order = a.order + bp.bstart[b];
    k.args.next = a.next + b;  // one work counter per bucket
    k.args.m_max = bp.bm[b];
    k.args.n_max = bp.bn[b];
    k.args.kc_max = bp.bkc[b];
    k.args.slot_bytes = bp.bslot[b];
    k.slots = std::min<long long>(bp.bcount[b], (long long)((size_t)bp.slots * bp.slot / bp.bslot[b]));
    k.key = TuneKey{bp.fp64, o->block, (long long)bp.bcount[b], bp.bm[b], bp.bn[b], bp.belems[b]};
    // schedule: the tuned one for this bucket's shape if any, else 256 threads, one
    // CTA per SM, the narrowest row width
    Sched sc{256, 1, default_vec(k)};
    tune_lookup(k.key, &sc);
    rs = apply_schedule(h, b, sc.threads, sc.per_sm, sc.vec);
    if (rs != RBRP_OK) rs = apply_schedule(h, b, 256, 1, default_vec(k));
    if (rs != RBRP_OK) {
      delete h;
      return rs;
    }
  }
  *out = h;
  return RBRP_OK;
}

rbrp_status rbrp_batch_set_schedule(rbrp_batch h, int32_t threads, int32_t ctas_per_sm) {
  if (!h) return RBRP_EINVAL;
  for (int b = 0; b < h->nb; ++b) {
    const rbrp_status rs = apply_schedule(h, b, threads, ctas_per_sm, default_vec(h->bk[b]));
    if (rs != RBRP_OK) return rs;
  }
  return RBRP_OK;
}

rbrp_status rbrp_batch_get_schedule(rbrp_batch h, int32_t* threads, int32_t* ctas_per_sm, int32_t* ctas) {
  if (!h) return RBRP_EINVAL;
  if (threads) *threads = h->bk[0].threads;
  if (ctas_per_sm) *ctas_per_sm = h->bk[0].per_sm;
  if (ctas) *ctas = h->bk[0].ctas;
  return RBRP_OK;
}

int32_t rbrp_batch_buckets(rbrp_batch h) { return h ? h->nb : 0; }

rbrp_status rbrp_batch_get_bucket(rbrp_batch h, int32_t i, int32_t* problems, int64_t* n_max, int32_t* threads,
                                  int32_t* ctas_per_sm, int32_t* vec, int32_t* ctas) {
  if (!h || i < 0 || i >= h->nb) return RBRP_EINVAL;
  const BatchBucket& k = h->bk[i];
  if (problems) *problems = k.args.P;
  if (n_max) *n_max = k.args.n_max;
  if (threads) *threads = k.threads;
  if (ctas_per_sm) *ctas_per_sm = k.per_sm;
  if (vec) *vec = k.vec;
  if (ctas) *ctas = k.ctas;
  return RBRP_OK;
}

rbrp_status rbrp_batch_set_bucket_schedule(rbrp_batch h, int32_t i, int32_t threads, int32_t ctas_per_sm,
                                           int32_t vec) {
  if (!h) return RBRP_EINVAL;
  return apply_schedule(h, i, threads, ctas_per_sm, vec);
}

rbrp_status rbrp_batch_run(rbrp_batch h, double tol, rbrp_stream_t stream) {
  if (!h) return RBRP_EINVAL;
  if (!(tol < 1.0)) return RBRP_EINVAL;
  for (int b = 0; b < h->nb; ++b) {
    const rbrp_status rs = run_bucket(h, b, tol, (cudaStream_t)stream);
    if (rs != RBRP_OK) return rs;
  }
  return RBRP_OK;
}

rbrp_status rbrp_batch_autotune(rbrp_batch h, double tol, int32_t reps, rbrp_stream_t stream, float* best_ms) {
  if (!h || reps < 1) return RBRP_EINVAL;
  if (!(tol < 1.0)) return RBRP_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  {
    const cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
      cudaEventDestroy(e0);
      g_last_cuda = (int)ce;
      return RBRP_ECUDA;
    }
  }
  rbrp_status rs = RBRP_OK;
  float total = 0.f;
  // each bucket alone: every (CTA size, CTAs per SM, row width) that fits
  for (int b = 0; b < h->nb && rs == RBRP_OK; ++b) {
    BatchBucket& k = h->bk[b];
    Sched best{k.threads, k.per_sm, k.vec};
    float best_t = -1.f;
    for (int th : kSchedThreads) {
      for (int per = 1; per <= kBatchMaxCtasPerSm && rs == RBRP_OK; ++per) {
        for (int vec : kBatchVecs) {
          if (rs != RBRP_OK) break;
          if (apply_schedule(h, b, th, per, vec) != RBRP_OK) continue;  // shape does not fit
          rs = run_bucket(h, b, tol, s);                                 // warm-up
          cudaError_t e = cudaSuccess;
          if (rs == RBRP_OK) e = cudaEventRecord(e0, s);
          for (int r = 0; r < reps && rs == RBRP_OK && e == cudaSuccess; ++r) rs = run_bucket(h, b, tol, s);
          if (rs == RBRP_OK && e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (rs == RBRP_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (rs == RBRP_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            g_last_cuda = (int)e;
            rs = RBRP_ECUDA;
          }
          if (rs == RBRP_OK && (best_t < 0.f || ms < best_t)) {
            best_t = ms;
            best = Sched{th, per, vec};
          }
        }
      }
    }
    if (rs != RBRP_OK) break;
    rs = apply_schedule(h, b, best.threads, best.per_sm, best.vec);
    if (rs == RBRP_OK) tune_store(k.key, best);
    total += best_t / (float)reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != RBRP_OK) return rs;
  if (best_ms) *best_ms = total;
  return RBRP_OK;
}

void rbrp_batch_destroy(rbrp_batch h) { delete h; }

rbrp_status rbrp_id_batched(int32_t P, const void* const* X, const int64_t* m, const int64_t* n, int x_is_fp64,
                            double tol, const rbrp_opts* o, void* workspace, size_t ws_bytes, int64_t* const* skel,
                            double* const* W, int64_t* k_out, double* rel_err_sq, int32_t* status,
                            rbrp_stream_t stream) {
  if (P == 0) {
    BatchPlan bp;
    return batch_plan(P, m, n, o, &bp);
  }
  if (!(tol < 1.0)) return RBRP_EINVAL;
  rbrp_batch h = nullptr;
  rbrp_status rs = rbrp_batch_create(P, X, m, n, x_is_fp64, o, workspace, ws_bytes, skel, W, k_out, rel_err_sq,
                                     status, stream, &h);
  if (rs != RBRP_OK) return rs;
  rs = rbrp_batch_run(h, tol, stream);
  rbrp_batch_destroy(h);
  return rs;
}

rbrp_status rbrp_host_workspace_size(int64_t n, int64_t d, int x_is_fp64, const rbrp_opts* o, size_t* bytes) {
  if (!bytes) return RBRP_EINVAL;
  Plan p;
  rbrp_status rs = make_plan(n, d, o, &p);
  if (rs != RBRP_OK) return rs;
  size_t off = (size_t)round_up((long long)p.total, 256);
  off += (size_t)round_up((long long)n * d * (x_is_fp64 ? 8 : 4), 256);
  off += (size_t)round_up((long long)n * p.k_cap * 8, 256);
  off += (size_t)round_up((long long)p.k_cap * 8, 256);
  *bytes = off;
  return RBRP_OK;
}

namespace {
// Device-to-host copy of W by row ranges on its own stream (rbrp_id_host).
struct HostCopy {
  const double* Wd = nullptr;
  double* W_host = nullptr;
  long long ldw = 0;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaError_t err = cudaSuccess;

  // Rows [r0, r1) are final once the work queued on s so far completes: the
  // copy stream waits for that point, then copies the k used columns.
  static cudaError_t done(void* ctx, long long r0, long long r1, long long k, cudaStream_t s) {
    HostCopy* h = (HostCopy*)ctx;
    cudaError_t e = cudaEventRecord(h->ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cs, h->ev, 0);
    if (e == cudaSuccess && k > 0)
      e = cudaMemcpy2DAsync(h->W_host + r0 * h->ldw, (size_t)h->ldw * 8, h->Wd + r0 * h->ldw, (size_t)h->ldw * 8,
                            (size_t)k * 8, (size_t)(r1 - r0), cudaMemcpyDeviceToHost, h->cs);
    if (e != cudaSuccess && h->err == cudaSuccess) h->err = e;
    return e;
  }
  // Waits for every queued copy, then frees the stream and the event.
  cudaError_t release() {
    cudaError_t e = cudaSuccess;
    if (cs) {
      e = cudaStreamSynchronize(cs);
      cudaStreamDestroy(cs);
      cs = nullptr;
    }
    if (ev) {
      cudaEventDestroy(ev);
      ev = nullptr;
    }
    return e;
  }
};
}  // namespace

rbrp_status rbrp_id_host(const void* X_host, int x_is_fp64, int64_t n, int64_t d, double tol, const rbrp_opts* o,
                         void* workspace, size_t ws_bytes, int64_t* skel_host, double* W_host, rbrp_result* res,
                         rbrp_stream_t stream) {
  if (!X_host || !skel_host || !W_host || !res || !workspace) return RBRP_EINVAL;
  Plan p;
  rbrp_status rs = make_plan(n, d, o, &p);
  if (rs != RBRP_OK) return rs;
  size_t need = 0;
  rs = rbrp_host_workspace_size(n, d, x_is_fp64, o, &need);
  if (rs != RBRP_OK) return rs;
  if (((uintptr_t)workspace & 255) != 0 || ws_bytes < need) return RBRP_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)workspace;
  size_t off = (size_t)round_up((long long)p.total, 256);
  void* Xd = base + off;
  off += (size_t)round_up((long long)n * d * (x_is_fp64 ? 8 : 4), 256);
  double* Wd = (double*)(base + off);
  off += (size_t)round_up((long long)n * p.k_cap * 8, 256);
  long long* Sd = (long long*)(base + off);
  const size_t xb = (size_t)n * d * (x_is_fp64 ? 8 : 4);
  CK(cudaMemcpyAsync(Xd, X_host, xb, cudaMemcpyHostToDevice, s));
  // W leaves the device in row ranges on a second stream while the solve of
  // the later ranges runs (the host link, not the solve, bounds this tail).
  HostCopy hc;
  hc.Wd = Wd;
  hc.W_host = W_host;
  hc.ldw = p.k_cap;
  CK(cudaStreamCreateWithFlags(&hc.cs, cudaStreamNonBlocking));
  cudaError_t ce = cudaEventCreateWithFlags(&hc.ev, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    hc.release();
    g_last_cuda = (int)ce;
    return RBRP_ECUDA;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  WSink sink;
  sink.chunk_rows = (long long)sms * wsolve_tc_rows_per_tile();  // one tile per SM per range
  sink.done = &HostCopy::done;
  sink.ctx = &hc;
  rs = run(Xd, x_is_fp64, n, d, d, tol, o, workspace, p.total, Sd, Wd, p.k_cap, res, s, &sink);
  if (rs == RBRP_OK || rs == RBRP_ENOTCONVERGED) {
    if (res->k > 0) {
      ce = cudaMemcpyAsync(skel_host, Sd, (size_t)res->k * 8, cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        g_last_cuda = (int)ce;
        rs = RBRP_ECUDA;
      }
    }
  }
  if (hc.err != cudaSuccess && (rs == RBRP_OK || rs == RBRP_ENOTCONVERGED)) {
    g_last_cuda = (int)hc.err;
    rs = RBRP_ECUDA;
  }
  const cudaError_t re = hc.release();
  if (re != cudaSuccess && (rs == RBRP_OK || rs == RBRP_ENOTCONVERGED)) {
    g_last_cuda = (int)re;
    rs = RBRP_ECUDA;
  }
  return rs;
}

const char* rbrp_status_string(rbrp_status s) {
  switch (s) {
    case RBRP_OK: return "ok";
    case RBRP_EINVAL: return "invalid argument";
    case RBRP_ENOMEM: return "out of memory";
    case RBRP_ECUDA: return "CUDA error";
    case RBRP_ENONFINITE: return "non-finite value in X or in the residual";
    case RBRP_ENOTCONVERGED: return "k_max reached before the tolerance";
    case RBRP_ETIMEOUT: return "bounded device wait timed out";
    case RBRP_EWORKSPACE: return "workspace misaligned or too small";
  }
  return "unknown status";
}

int rbrp_last_cuda_error(void) { return g_last_cuda; }

rbrp_status rbrp_set_loop_mode(int32_t mode) {
  if (mode != RBRP_LOOP_DEVICE && mode != RBRP_LOOP_HOST) return RBRP_EINVAL;
  g_loop_mode = mode;
  return RBRP_OK;
}

void rbrp_set_wait_limits(uint32_t mbarrier_polls, uint32_t barrier_polls) {
  g_spin_mbar = mbarrier_polls ? mbarrier_polls : kDefaultSpinMbar;
  g_spin_grid = barrier_polls ? barrier_polls : kDefaultSpinGrid;
}

// rbrp_id with the workspace taken from the fixed device array above: no
// cudaMalloc, no cudaFree, no allocating library call.  The run writes every
// scratch word it reads before reading it (norms, residual copy, State, sampler
// candidates, Gram and factor buffers are all produced inside the call), so
// the contents left by the previous call need no clearing.
rbrp_status rbrp_id_noalloc(const void* X, int x_is_fp64, int64_t n, int64_t d, int64_t ldx, double tol,
                            const rbrp_opts* o, int64_t* skel, double* W, int64_t ldw, rbrp_result* res,
                            rbrp_stream_t stream) {
  size_t need = 0;
  rbrp_status rs = rbrp_workspace_size(n, d, o, &need);
  if (rs != RBRP_OK) return rs;
  if (need > (size_t)RBRP_NOALLOC_SCRATCH_BYTES) return RBRP_EWORKSPACE;
  void* ws = nullptr;
  CK(noalloc_scratch(&ws));
  return run(X, x_is_fp64, n, d, ldx, tol, o, ws, (size_t)RBRP_NOALLOC_SCRATCH_BYTES, (long long*)skel, W, ldw, res,
             (cudaStream_t)stream);
}

// ---------------------------------------------------------------- sketchy pivoting + OSID
}  // extern "C"

namespace {

struct SketchPlan {
  Plan rp;                 // the forced block loop on Y(:, 0:ocols)
  long long l, k, ocols;
  int sk64, sms;
  size_t off_Y, off_A, off_U, off_lu, off_piv, off_rs, off_mark, total;
};

rbrp_status sketch_plan(long long n, long long d, long long l, long long k, const rbrp_sketch_opts* so,
                        rbrp_opts* ro, SketchPlan* sp, bool need_grid) {
  if (!so || !ro || !sp) return RBRP_EINVAL;
  if (n < 1 || d < 1 || l < 1 || k < 1 || k > l || k > n || l >= (1LL << 31)) return RBRP_EINVAL;
  if (so->precision < RBRP_FP64 || so->precision > RBRP_TF32X3) return RBRP_EINVAL;
  const long long ocols = so->osid_cols == 0 ? l : (long long)so->osid_cols;
  if (ocols < k || ocols > l) return RBRP_EINVAL;
  memset(sp, 0, sizeof(*sp));
  rbrp_default_opts(ro);
  ro->precision = so->precision;
  ro->block = so->block;
  ro->w_precision = so->w_precision;
  ro->k_max = k;
  ro->chain = RBRP_CHAIN_FP64;
  rbrp_status rs = make_plan(n, ocols, ro, &sp->rp, 1);
  if (rs != RBRP_OK) return rs;
  if (n > (1LL << 48) / l) return RBRP_EINVAL;
  sp->l = l;
  sp->k = k;
  sp->ocols = ocols;
  sp->sk64 = (so->precision == RBRP_FP64);
  sp->sms = 152;
  if (need_grid) {
    cudaError_t e = lupp_grid(&sp->sms);
    if (e != cudaSuccess) {
      g_last_cuda = (int)e;
      return RBRP_ECUDA;
    }
  }
  const size_t ts = sp->sk64 ? 8 : 4;
  size_t off = (size_t)round_up((long long)sp->rp.total, 256);
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off = (size_t)round_up((long long)(off + bytes), 256);
    return o2;
  };
  sp->off_Y = take((size_t)n * l * ts);
  sp->off_A = take((size_t)n * k * ts);
  sp->off_U = take((size_t)lupp_panel_width() * k * ts);
  sp->off_lu = take(lupp_scratch_bytes(std::max(sp->sms, 152)));
  sp->off_piv = take((size_t)k * 8);
  sp->off_rs = take(8);
  sp->off_mark = take((size_t)n * 4);
  sp->total = off;
  return RBRP_OK;
}

}  // namespace

extern "C" {

rbrp_status rbrp_sketch_workspace_size(int64_t n, int64_t d, int64_t l, int64_t k, const rbrp_sketch_opts* o,
                                       size_t* bytes) {
  if (!bytes) return RBRP_EINVAL;
  rbrp_opts ro;
  SketchPlan sp;
  rbrp_status rs = sketch_plan(n, d, l, k, o, &ro, &sp, false);
  if (rs != RBRP_OK) return rs;
  *bytes = sp.total;
  return RBRP_OK;
}

rbrp_status rbrp_sketch_id(const void* X, int x_is_fp64, int64_t n, int64_t d, int64_t ldx, const void* Omega,
                           int64_t l, int64_t k, const rbrp_sketch_opts* o, void* workspace, size_t ws_bytes,
                           int64_t* skel, double* W, int64_t ldw, rbrp_result* res, rbrp_stream_t stream) {
  rbrp_opts ro;
  SketchPlan sp;
  rbrp_status rs = sketch_plan(n, d, l, k, o, &ro, &sp, true);
  if (rs != RBRP_OK) return rs;
  if (!X || !Omega || !workspace || !skel || !W || !res) return RBRP_EINVAL;
  if (ldx < d || ldw < k) return RBRP_EINVAL;
  if (x_is_fp64 && !sp.sk64) return RBRP_EINVAL;  // the FP32 sketch takes FP32 input
  if (((uintptr_t)workspace & 255) != 0 || ws_bytes < sp.total) return RBRP_EWORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  memset(res, 0, sizeof(*res));
  char* base = (char*)workspace;
  void* Y = base + sp.off_Y;
  void* A = base + sp.off_A;
  void* U = base + sp.off_U;
  long long* piv = (long long*)(base + sp.off_piv);
  int* rstat = (int*)(base + sp.off_rs);
  int* mark = (int*)(base + sp.off_mark);
  // sketching step (Sec. 3.2): Y = X Omega, n x l row-major
  GemmArgs g;
  g.A = MatRef{const_cast<void*>(X), dim_const(0), ldx, 1};
  g.B = MatRef{const_cast<void*>(Omega), dim_const(0), l, 1};
  g.C = MatRef{Y, dim_const(0), l, 1};
  g.M = dim_const(n);
  g.N = dim_const(l);
  g.K = dim_const(d);
  g.alpha = 1.0;
  g.beta = 0.0;
  g.partial = nullptr;
  g.pm = n;
  g.pn = l;
  g.st = nullptr;
  if (sp.sk64 && x_is_fp64)
    CK((launch_gemm<double, double, double, double>(g, n, l, 1, kGemmTile, s)));
  else if (sp.sk64)
    CK((launch_gemm<float, double, double, double>(g, n, l, 1, kGemmTile, s)));
  else
    CK((launch_gemm<float, float, float, float>(g, n, l, 1, kGemmTile, s)));
  // skeleton selection: LU with partial pivoting of Y(:, 0:k)
  unsigned mlim = kDefaultSpinMbar, glim = kDefaultSpinGrid;
  wait_limits(&mlim, &glim);
  if (sp.sk64)
    CK(launch_lupp<double>((const double*)Y, l, n, (int)k, (double*)A, (double*)U, mark, piv, rstat,
                           base + sp.off_lu, sp.sms, glim, s));
  else
    CK(launch_lupp<float>((const float*)Y, l, n, (int)k, (float*)A, (float*)U, mark, piv, rstat, base + sp.off_lu,
                          sp.sms, glim, s));
  int h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, rstat, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h[1] != 0) return RBRP_ETIMEOUT;
  const long long r = h[0];
  if (r == 0) return RBRP_OK;  // Y(:, 0:k) is zero: no skeleton
  // interpolation matrix (Alg. 4): the block loop on Y(:, 0:ocols) with the
  // pivots as forced skeletons gives W = Y Y_S^+ (W(S,:) = I, W(rest,:) = L2 L1^{-1})
  ro.k_max = r;
  Forced f{piv, rstat};
  rs = run(Y, sp.sk64, n, sp.ocols, l, -1.0, &ro, workspace, sp.rp.total, (long long*)skel, W, ldw, res, s,
           nullptr, &f);
  if (rs == RBRP_OK && res->k < r) return RBRP_ENOTCONVERGED;
  return rs;
}

// ---------------------------------------------------------------- row shards of one ID
}  // extern "C"

struct rbrp_shard_s {
  Plan p;
  Bufs u;
  rbrp_opts o;
  long long n, d, row_base, k_cap;
  long long* skel;            // device: k_cap global rows, acceptance order
  unsigned long long* keys;   // device: the draw's ordered keys
  long long* idx;             // device: local row indices of a request
  double* buf;                // device: FP64 staging of requested rows
  cudaStream_t s;
};

namespace {

struct ShardLayout {
  Plan p;
  size_t off_skel, off_keys, off_idx, off_buf, total;
};

rbrp_status shard_layout(long long n, long long d, long long k_cap, const rbrp_opts* o, ShardLayout* L) {
  if (!o || !L || n < 1 || d < 1 || k_cap < 1 || k_cap > d) return RBRP_EINVAL;
  if (o->form != RBRP_FORM_RESIDUAL) return RBRP_EINVAL;
  rbrp_status rs = make_plan(n, d, o, &L->p, 0, k_cap);
  if (rs != RBRP_OK) return rs;
  if (L->p.f32) return RBRP_EINVAL;  // the shard steps run the FP64 filter: not the FP32 chain of RBRP_TF32
  size_t off = (size_t)round_up((long long)L->p.total, 256);
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off = (size_t)round_up((long long)(off + bytes), 256);
    return o2;
  };
  const long long kc = L->p.k_cap;
  L->off_skel = take((size_t)kc * 8);
  L->off_keys = take((size_t)kMaxBlock * 8);
  L->off_idx = take((size_t)std::max<long long>(kMaxBlock, kc) * 8);
  L->off_buf = take((size_t)std::max<long long>((long long)kMaxBlock * d, kc * kc) * 8);
  L->total = off;
  return RBRP_OK;
}

double decode_key(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
  double x;
  memcpy(&x, &b, 8);
  return x;
}

// Local positions of the requested global rows that this shard holds.
void shard_local(const rbrp_shard_s* h, const int64_t* rows, int64_t count, std::vector<long long>* loc,
                 std::vector<int64_t>* pos, int32_t* owned) {
  for (int64_t i = 0; i < count; ++i) {
    const long long g = rows[i];
    const bool mine = g >= h->row_base && g < h->row_base + h->n;
    if (owned) owned[i] = mine ? 1 : 0;
    if (mine) {
      loc->push_back(g - h->row_base);
      pos->push_back(i);
    }
  }
}

}  // namespace

extern "C" {

rbrp_status rbrp_shard_workspace_size(int64_t n_local, int64_t d, int64_t k_cap, const rbrp_opts* o, size_t* bytes) {
  if (!bytes) return RBRP_EINVAL;
  ShardLayout L;
  rbrp_status rs = shard_layout(n_local, d, k_cap, o, &L);
  if (rs != RBRP_OK) return rs;
  *bytes = L.total;
  return RBRP_OK;
}

rbrp_status rbrp_shard_create(const void* X, int x_is_fp64, int64_t n_local, int64_t d, int64_t ldx, int64_t row_base,
                              int64_t k_cap, const rbrp_opts* o, void* workspace, size_t ws_bytes,
                              rbrp_stream_t stream, rbrp_shard* out, double* sum_sq) {
  if (!out || !sum_sq) return RBRP_EINVAL;
  *out = nullptr;
  ShardLayout L;
  rbrp_status rs = shard_layout(n_local, d, k_cap, o, &L);
  if (rs != RBRP_OK) return rs;
  if (!X || !workspace || ldx < d || row_base < 0) return RBRP_EINVAL;
  if (((uintptr_t)workspace & 255) != 0 || ws_bytes < L.total) return RBRP_EWORKSPACE;
  rbrp_shard_s* h = new (std::nothrow) rbrp_shard_s();
  if (!h) return RBRP_ENOMEM;
  char* base = (char*)workspace;
  h->p = L.p;
  h->u = carve(h->p, workspace);
  h->o = *o;
  h->n = n_local;
  h->d = d;
  h->row_base = row_base;
  h->k_cap = h->p.k_cap;
  h->skel = (long long*)(base + L.off_skel);
  h->keys = (unsigned long long*)(base + L.off_keys);
  h->idx = (long long*)(base + L.off_idx);
  h->buf = (double*)(base + L.off_buf);
  h->s = (cudaStream_t)stream;
  Bufs& u = h->u;
  u.skel = h->skel;
  u.X = X;
  u.x64 = x_is_fp64 ? 1 : 0;
  u.ldx = ldx;
  u.mark_base = row_base;
  u.mark_n = n_local;
  const Plan& p = h->p;
  cudaStream_t s = h->s;
  State st;
  cudaError_t e = launch_init_norms(X, x_is_fp64, n_local, d, ldx, u.R, p.r64, p.ldr, u.dvec, u.mark, u.part,
                                    p.nparts, u.st, s);
  if (e == cudaSuccess) e = launch_finish_init(u.part, p.nparts, u.st, -1.0, o->tau_b, h->k_cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(u.cnt, 0, (size_t)kSgemmCounters * 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, u.st, sizeof(State), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete h;
    g_last_cuda = (int)e;
    return RBRP_ECUDA;
  }
  if (st.status != 0) {
    delete h;
    return (rbrp_status)st.status;
  }
  *sum_sq = st.D0;
  *out = h;
  return RBRP_OK;
}

rbrp_status rbrp_shard_draw(rbrp_shard h, int64_t* rows, double* keys, int64_t* count) {
  if (!h || !rows || !keys || !count) return RBRP_EINVAL;
  *count = 0;
  Bufs& u = h->u;
  const Plan& p = h->p;
  cudaStream_t s = h->s;
  State st;
  CK(launch_sample(u.dvec, h->n, p.b, p.greedy, h->o.seed, h->o.problem, u.ca, u.cb, u.S_t, u.st, 1, s,
                   h->row_base, h->keys));
  CK(cudaMemcpyAsync(&st, u.st, sizeof(State), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st.status != 0) return (rbrp_status)st.status;
  if (st.done || st.b_t <= 0) return RBRP_OK;
  std::vector<long long> loc((size_t)st.b_t);
  std::vector<unsigned long long> kk((size_t)st.b_t);
  CK(cudaMemcpyAsync(loc.data(), u.S_t, (size_t)st.b_t * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(kk.data(), h->keys, (size_t)st.b_t * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (long long i = 0; i < st.b_t; ++i) {
    rows[i] = loc[(size_t)i] + h->row_base;
    keys[i] = decode_key(kk[(size_t)i]);
  }
  *count = st.b_t;
  return RBRP_OK;
}

rbrp_status rbrp_shard_rows(rbrp_shard h, const int64_t* rows, int64_t count, double* V, int32_t* owned) {
  if (!h || count < 0 || count > kMaxBlock || (count > 0 && (!rows || !V || !owned))) return RBRP_EINVAL;
  std::vector<long long> loc;
  std::vector<int64_t> pos;
  shard_local(h, rows, count, &loc, &pos, owned);
  if (loc.empty()) return RBRP_OK;
  const long long m = (long long)loc.size(), d = h->d;
  std::vector<double> tmp((size_t)(m * d));
  cudaStream_t s = h->s;
  CK(cudaMemcpyAsync(h->idx, loc.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s));
  CK(launch_gather_rows_rect(h->u.R, h->p.r64, h->p.ldr, h->idx, m, d, h->buf, d, s));
  CK(cudaMemcpyAsync(tmp.data(), h->buf, (size_t)(m * d) * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (long long i = 0; i < m; ++i) memcpy(V + pos[(size_t)i] * d, tmp.data() + i * d, (size_t)d * 8);
  return RBRP_OK;
}

rbrp_status rbrp_shard_block(rbrp_shard h, const double* V, const int64_t* S_t, int64_t b_t, int64_t* accepted,
                             int64_t* bp, double* d_sum) {
  if (!h || !V || !S_t || !accepted || !bp || !d_sum) return RBRP_EINVAL;
  const Plan& p = h->p;
  if (b_t < 1 || b_t > p.b) return RBRP_EINVAL;
  Bufs& u = h->u;
  cudaStream_t s = h->s;
  const long long bt = b_t;
  State st;
  CK(cudaMemcpy2DAsync(u.V, (size_t)p.ldq * 8, V, (size_t)h->d * 8, (size_t)h->d * 8, (size_t)bt,
                       cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(u.S_t, S_t, (size_t)bt * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(&u.st->b_t, &bt, 8, cudaMemcpyHostToDevice, s));
  {
    const cudaError_t e = enqueue_chain(p, u, &h->o, s);
    if (e != cudaSuccess) {
      g_last_cuda = (int)e;
      return RBRP_ECUDA;
    }
  }
  CK(cudaMemcpyAsync(&st, u.st, sizeof(State), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st.status != 0) return (rbrp_status)st.status;
  const long long k0 = st.k - st.bp;
  *bp = st.bp;
  *d_sum = st.D;
  if (st.bp > 0) {
    CK(cudaMemcpyAsync(accepted, h->skel + k0, (size_t)st.bp * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return RBRP_OK;
}

rbrp_status rbrp_shard_l_rows(rbrp_shard h, const int64_t* rows, int64_t count, int64_t k, double* Lrows,
                              int32_t* owned) {
  if (!h || count < 0 || count > h->k_cap || k < 0 || k > h->k_cap || (count > 0 && (!rows || !Lrows || !owned)))
    return RBRP_EINVAL;
  std::vector<long long> loc;
  std::vector<int64_t> pos;
  shard_local(h, rows, count, &loc, &pos, owned);
  if (loc.empty() || k == 0) return RBRP_OK;
  const long long m = (long long)loc.size();
  std::vector<double> tmp((size_t)(m * k));
  cudaStream_t s = h->s;
  CK(cudaMemcpyAsync(h->idx, loc.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s));
  CK(launch_gather_rows_rect(h->u.L, h->p.l64, h->p.ldl, h->idx, m, k, h->buf, k, s));
  CK(cudaMemcpyAsync(tmp.data(), h->buf, (size_t)(m * k) * 8, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (long long i = 0; i < m; ++i) memcpy(Lrows + pos[(size_t)i] * k, tmp.data() + i * k, (size_t)k * 8);
  return RBRP_OK;
}

rbrp_status rbrp_shard_w(rbrp_shard h, const double* L1, const int64_t* skel, int64_t k, double* W, int64_t ldw) {
  if (!h || k < 0 || k > h->k_cap || (k > 0 && (!L1 || !skel || !W)) || ldw < k) return RBRP_EINVAL;
  if (k == 0) return RBRP_OK;
  cudaStream_t s = h->s;
  std::vector<long long> loc((size_t)k);
  for (int64_t j = 0; j < k; ++j) {
    const long long g = skel[j];
    loc[(size_t)j] = (g >= h->row_base && g < h->row_base + h->n) ? g - h->row_base : -1;
  }
  CK(cudaMemcpyAsync(h->u.L1, L1, (size_t)(k * k) * 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->idx, loc.data(), (size_t)k * 8, cudaMemcpyHostToDevice, s));
  rbrp_status rs = solve_w(h->p, h->u, k, h->idx, W, ldw, s, nullptr, true);
  if (rs != RBRP_OK) return rs;
  CK(cudaStreamSynchronize(s));
  return RBRP_OK;
}

void rbrp_shard_destroy(rbrp_shard h) { delete h; }

void rbrp_profile_begin(void) {
  g_prof.on = true;
  g_prof.launches0 = g_kernel_launches.load();
  g_prof.upd.used = 0;
  g_prof.wsv.used = 0;
  g_prof.blocks = 0;
  g_prof.skel = 0;
}

rbrp_status rbrp_profile_end(rbrp_profile* out) {
  if (!out) return RBRP_EINVAL;
  memset(out, 0, sizeof(*out));
  out->launches = g_kernel_launches.load() - g_prof.launches0;
  out->blocks = g_prof.blocks;
  out->skeletons = g_prof.skel;
  EventPool* pools[2] = {&g_prof.upd, &g_prof.wsv};
  double* ms[2] = {&out->update_ms, &out->wsolve_ms};
  int64_t* cnt[2] = {&out->update_launches, &out->wsolve_calls};
  for (int q = 0; q < 2; ++q) {
    for (size_t i = 0; i + 1 < pools[q]->used; i += 2) {
      cudaError_t e = cudaEventSynchronize(pools[q]->ev[i + 1]);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pools[q]->ev[i], pools[q]->ev[i + 1]);
      if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        g_prof.on = false;
        return RBRP_ECUDA;
      }
      *ms[q] += t;
      *cnt[q] += 1;
    }
  }
  g_prof.on = false;
  return RBRP_OK;
}

}  // extern "C"
