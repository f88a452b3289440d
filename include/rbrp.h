/*
 * rbrp.h -- C ABI of the GB300 (sm_103a) implementation of Robust Blockwise
 * Random Pivoting (RBRP) for the row interpolative decomposition X ~ W X_S.
 *
 * Method: Dong, Chen, Martinsson, Pearce, "Robust Blockwise Random Pivoting:
 * Fast and Accurate Adaptive Interpolative Decomposition", arXiv 2309.16002.
 *   - problem statement (row ID, skeleton indices S, interpolation matrix W):
 *     Eq. (1.1); skeletonization error E_X(S): Eq. (1.2)
 *   - skeleton selection: Alg. 2 (RBRP) with the robust blockwise filtering
 *     remark of Sec. 4 (truncated local CPQR, tau_b = 1/b) and the blockwise
 *     greedy remark (RBGP) for the greedy sampler
 *   - interpolation matrix: Alg. 3, W(S,:) = I, W(rest,:) = L2 L1^{-1}
 *
 * All functions are plain C: pointers, sizes and a CUDA stream handle.  No
 * function allocates device memory: the caller owns X, every output buffer
 * and the workspace (size from rbrp_workspace_size).  The library keeps no
 * state between calls.
 *
 * Errors: every function returns an rbrp_status.  On RBRP_EINVAL /
 * RBRP_EWORKSPACE nothing was launched.  On RBRP_ECUDA the CUDA error is
 * available from rbrp_last_cuda_error().  On RBRP_ENONFINITE (a NaN or Inf in
 * X, or a non-finite residual) and RBRP_ETIMEOUT the outputs are unspecified.
 * RBRP_ENOTCONVERGED means k reached k_max (or min(n, d)) before the
 * tolerance: S and W are valid for that k.
 */
#ifndef RBRP_H
#define RBRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st *rbrp_stream_t;

typedef enum {
  RBRP_OK = 0,
  RBRP_EINVAL = 1,          /* bad argument (sizes, pointers, options)            */
  RBRP_ENOMEM = 2,          /* reserved: the library never allocates              */
  RBRP_ECUDA = 3,           /* a CUDA runtime call or launch failed               */
  RBRP_ENONFINITE = 4,      /* NaN/Inf in X or in the residual                    */
  RBRP_ENOTCONVERGED = 5,   /* |S| hit k_max or min(n, d) before the tolerance    */
  RBRP_ETIMEOUT = 6,        /* a bounded device wait gave up                      */
  RBRP_EWORKSPACE = 7       /* workspace pointer misaligned or too small          */
} rbrp_status;

/* Arithmetic of the residual-update contraction (the O(n d b') step).  The
 * per-block chain around it (the rows drawn, the projection against Q, the
 * Gram matrix, the pivoted filter and Q') runs in the precision's default
 * chain unless rbrp_opts.chain asks for the FP64 chain (rbrp_chain).  The
 * sampling keys and the sums of the row norms are FP64 in every form. */
typedef enum {
  RBRP_FP64 = 0,   /* residual R and every step in FP64 (CUDA-core DFMA)          */
  RBRP_TF32 = 1,   /* R in FP32, update on tcgen05 tensor cores (TF32 in, FP32    */
                   /* accumulate).  Default chain: FP32 throughout -- FP32 copies */
                   /* of the drawn rows and of Q, ONE projection pass against Q   */
                   /* with FP32 products, FP32 Gram matrix and FP32 pivoted       */
                   /* Cholesky filter, Q' = Lc^{-1} V_perm in FP32 (b <= 128; the */
                   /* FP64 chain takes b <= 256, in 64-column chunks of Q').      */
  RBRP_FP32 = 2,   /* R in FP32, update on CUDA cores in FP32.  Default chain:    */
                   /* FP64 storage of V and Q, two projection passes (CGS2) with  */
                   /* FP32 products, FP64 Gram and filter, one FP64 CholQR pass   */
  RBRP_TF32X3 = 3  /* as RBRP_TF32 with every operand split into TF32 hi + lo and */
                   /* three products per step (~FP32-accurate update); blocks     */
                   /* wider than 64 run as 64-column chunks of Q' (each chunk one */
                   /* pass over R); default chain as RBRP_FP32                    */
} rbrp_precision;

/* Precision of the per-block chain (rbrp_opts.chain). */
typedef enum {
  RBRP_CHAIN_DEFAULT = 0,   /* the chain listed with each rbrp_precision            */
  RBRP_CHAIN_FP64 = 1       /* FP64 storage and FP64 products for every small step:
                               CGS2 against Q (two passes), the Gram matrix and the
                               pivoted filter, Q' by two CholQR passes; combined with
                               RBRP_TF32 this keeps tensor cores for the update only
                               (RBRP_FP64 always runs this chain)                   */
} rbrp_chain;

typedef enum {
  RBRP_SAMPLER_RANDOM = 0,  /* Alg. 2 sampling step: ~ d/||d||_1 without replacement */
  RBRP_SAMPLER_GREEDY = 1,  /* blockwise greedy remark (Sec. 4): top-b of d          */
  /* The same draws as RANDOM / GREEDY (identical S_t), always computed by the
   * single-stage exact sampler (FP64 keys of every eligible row, ranked in full)
   * instead of the FP32 cut with its exact check: a slower reference form, also
   * the path the fast sampler falls back to when its check fails.              */
  RBRP_SAMPLER_RANDOM_EXACT = 2,
  RBRP_SAMPLER_GREEDY_EXACT = 3
} rbrp_sampler;

/* How the update step of Alg. 2 (coefficients and new residual norms) is carried out. */
typedef enum {
  RBRP_FORM_RESIDUAL = 0,   /* R <- R - (R Q'^T) Q' in a residual copy of X, d_i =
                               ||R_i||^2 recomputed (robust at any precision)       */
  RBRP_FORM_DOWNDATE = 1    /* as printed: X read-only, Lhat = X Q'^T, d_i -=
                               ||Lhat_i||^2; half the memory traffic of the residual
                               form and no residual copy.  The downdate cancels, so
                               it runs in RBRP_FP64 or in RBRP_TF32X3 (Lhat from the
                               3xTF32 split, ~FP32-accurate, d in FP64; X must then
                               be FP32 with ldx a multiple of 4 and a 16-byte base) */
} rbrp_form;

typedef enum {
  RBRP_W_FP64 = 0,          /* Alg. 3 triangular solve in FP64                      */
  RBRP_W_FP32 = 1           /* same solve in FP32 (for the TF32 path)               */
} rbrp_w_precision;

typedef struct {
  int32_t precision;    /* rbrp_precision                                        */
  int32_t block;        /* b, 1 <= b <= 256 (Alg. 2 input (c))                    */
  double tau_b;         /* < 0: 1/b_t (the paper's choice); 0: plain BRP; else
                           a fixed filter tolerance in [0, 1] (Alg. 2 input (d))  */
  int64_t k_max;        /* <= 0: min(n, d); else caps |S|.  With tol < 0 the call
                           runs in fixed-rank mode and stops at |S| = k_max.      */
  uint64_t seed;        /* Philox4x64-10 key word 0                               */
  uint64_t problem;     /* Philox4x64-10 key word 1 (problem id)                  */
  int32_t sampler;      /* rbrp_sampler                                           */
  int32_t w_precision;  /* rbrp_w_precision                                       */
  int32_t form;         /* rbrp_form (rbrp_id only; the batched call ignores it)  */
  int32_t chain;        /* rbrp_chain (rbrp_id only; the batched call ignores it) */
} rbrp_opts;

typedef struct {
  int64_t k;            /* number of skeletons |S|                                */
  int64_t blocks;       /* number of blocks t run by Alg. 2                       */
  double d0;            /* ||d0||_1 = ||X||_F^2                                  */
  double d_final;       /* ||d||_1 at exit = ||X - L Q^T||_F^2 (Sec. 5.1 proof)   */
  double rel_err_sq;    /* d_final / d0, the quantity tested against tol          */
} rbrp_result;

/* Fill *o with the defaults: TF32, b = 64, tau_b = 1/b_t, k_max = min(n, d),
 * seed 0, problem 0, random sampler, W in FP64, residual form, default chain. */
void rbrp_default_opts(rbrp_opts *o);

/* Bytes of device workspace rbrp_id needs for an n x d problem with options o
 * (residual copy of X, L, Q, the norms d and the per-block buffers).
 * RBRP_EINVAL for n < 1, d < 1, n or d >= 2^31, n d > 2^48 (no byte count can
 * then overflow), a null o or bytes, or an option out of range. */
rbrp_status rbrp_workspace_size(int64_t n, int64_t d, const rbrp_opts *o, size_t *bytes);

/*
 * rbrp_id -- rank-adaptive row ID of X by Alg. 2 followed by Alg. 3.
 *
 * X          device, row-major n x d, leading dimension ldx >= d (elements),
 *            FP64 if x_is_fp64 else FP32.  Read only.
 * tol        tau of Alg. 2: stop once ||d||_1 <= tol * ||d0||_1, i.e. the
 *            squared relative residual ||X - L Q^T||_F^2 / ||X||_F^2 <= tol.
 *            tol < 0 selects fixed-rank mode (stop at |S| = k_max).
 * workspace  device, >= rbrp_workspace_size bytes, 256-byte aligned; scratch
 *            only, contents undefined on return.
 * skel       device int64[k_cap] (k_cap = k_max or min(n, d)): S in
 *            acceptance order (block order, pivot order within a block).
 * W          device FP64, row-major n x k_cap with leading dimension ldw >=
 *            k_cap; column j belongs to skel[j]; only columns < k are written.
 * res        host; filled on return.
 * stream     all device work is ordered on this stream; the call returns after
 *            the stream has finished the work it queued (res is host data).
 */
rbrp_status rbrp_id(const void *X, int x_is_fp64, int64_t n, int64_t d, int64_t ldx,
                    double tol, const rbrp_opts *o, void *workspace, size_t ws_bytes,
                    int64_t *skel, double *W, int64_t ldw, rbrp_result *res,
                    rbrp_stream_t stream);

/* Bytes of device workspace rbrp_id_host needs: rbrp_workspace_size plus room
 * for X and W on the device. */
rbrp_status rbrp_host_workspace_size(int64_t n, int64_t d, int x_is_fp64, const rbrp_opts *o,
                                     size_t *bytes);

/*
 * rbrp_id_host -- rbrp_id on HOST buffers: copies X (host, row-major n x d,
 * leading dimension d) to the device, runs rbrp_id, copies S and W back.
 * skel_host: int64[k_cap]; W_host: FP64 n x k_cap row-major (ldw = k_cap),
 * columns >= k left untouched.  Pinned host memory makes the copies
 * asynchronous; pageable memory works but is slower.  W is copied out in row
 * ranges on a second stream (created and destroyed inside the call) while the
 * W solve (Alg. 3) of the later ranges still runs on `stream`.  The call is
 * synchronous: every copy has completed when it returns, on success or error.
 */
rbrp_status rbrp_id_host(const void *X_host, int x_is_fp64, int64_t n, int64_t d, double tol,
                         const rbrp_opts *o, void *workspace, size_t ws_bytes,
                         int64_t *skel_host, double *W_host, rbrp_result *res,
                         rbrp_stream_t stream);

/*
 * Profiling counters (instrumentation; no counterpart in the paper).  Between
 * rbrp_profile_begin() and rbrp_profile_end() the library counts every kernel
 * it launches and brackets each residual-update launch (Alg. 2, update step)
 * and each W solve (Alg. 3) with CUDA events recorded on the caller's stream.
 * rbrp_profile_end synchronises those events, fills *out and stops counting.
 * Process-wide; not thread-safe; calls outside a begin/end pair cost nothing.
 */
typedef struct {
  int64_t launches;         /* kernels launched by the library                   */
  int64_t update_launches;  /* residual-update launches timed                    */
  double update_ms;         /* summed event time of those launches               */
  int64_t wsolve_calls;     /* W solves timed                                    */
  double wsolve_ms;         /* summed event time of the W solves                 */
  int64_t blocks;           /* Alg. 2 blocks run (sum over calls)                */
  int64_t skeletons;        /* skeletons accepted (sum over calls)               */
} rbrp_profile;

void rbrp_profile_begin(void);
rbrp_status rbrp_profile_end(rbrp_profile *out);

/*
 * rbrp_id_noalloc -- rbrp_id for callers that cannot allocate device memory.
 * (An addition of this library; the paper has no counterpart.)
 *
 * Some callers run where cudaMalloc is not an option: inside an engine or
 * plugin host that owns all device memory and forbids further allocation, or
 * in code that must not grow a memory pool it does not control.  This entry
 * point takes the same inputs and caller-owned outputs as rbrp_id (X, skel, W
 * and res exactly as documented there) but uses, instead of a caller
 * workspace, one fixed array of RBRP_NOALLOC_SCRATCH_BYTES bytes that lives in
 * the library's device image: it calls no cudaMalloc, no cudaFree and no
 * allocating library routine.  Every GPU on which the library's module is
 * loaded holds that array until the process exits.
 *
 * Limits and behaviour:
 *  - a problem whose rbrp_workspace_size exceeds RBRP_NOALLOC_SCRATCH_BYTES is
 *    rejected with RBRP_EWORKSPACE before anything is launched;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  Under CUDA's lazy module loading (the
 *    default) this lookup is also what loads the module and commits the
 *    array's memory on that device, so the first call can fail with
 *    RBRP_ECUDA if the device is short of memory then: callers that must not
 *    fail later should make one small call at start-up (or load modules
 *    eagerly, CUDA_MODULE_LOADING=EAGER);
 *  - the address is remembered per device index for the primary context (the
 *    one the CUDA runtime uses); after cudaDeviceReset, or from a thread
 *    bound to another context of the same device, it is not valid;
 *  - all calls on a device share the one array and it keeps the previous
 *    call's contents (each call rewrites what it reads), so calls whose work
 *    overlaps on the GPU (different streams, different host threads) race and
 *    must be serialised by the caller.
 */
#define RBRP_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
rbrp_status rbrp_id_noalloc(const void *X, int x_is_fp64, int64_t n, int64_t d, int64_t ldx,
                            double tol, const rbrp_opts *o, int64_t *skel, double *W, int64_t ldw,
                            rbrp_result *res, rbrp_stream_t stream);

/*
 * rbrp_id_batched -- P independent row IDs (Alg. 2 then Alg. 3 for each) in one
 * persistent launch: each CTA takes whole problems from a work queue, largest
 * first, and runs the method for one problem at a time.
 *
 * Problem p is X[p] (device, row-major m[p] x n[p] with leading dimension n[p],
 * FP32, or FP64 when x_is_fp64), solved to tol with the options o (block b,
 * tau_b, k_max, seed, sampler); its Philox problem id is o->problem + p, so
 * its skeletons are drawn exactly as rbrp_id would draw them with that problem
 * id, and a caller that splits one list of problems into contiguous shards
 * (one call per shard, o->problem = index of the shard's first problem) gets
 * the same results as one call over the whole list.
 * Precision: o->precision == RBRP_FP64 keeps the residual and every step in
 * FP64; any other value keeps the residual, the products and the W solve in
 * FP32 (row norms and their sums in FP64, sampling keys exact FP64);
 * o->w_precision is not used.
 * Limits: 1 <= m[p] <= 4096, 1 <= n[p] <= 256, 1 <= o->block <= 32; otherwise
 * RBRP_EINVAL before anything is launched.
 * Arguments: X, m, n, skel and W are HOST arrays of P entries (X, skel and W
 * hold device pointers); they may be released when the call returns.
 * Outputs (caller-owned, device): skel[p] receives k_p <= k_cap_p =
 * min(m[p], n[p], k_max) row indices in acceptance order; W[p] (m[p] x k_cap_p
 * FP64, leading dimension k_cap_p) receives columns 0..k_p-1 of W with the rows
 * of S set to unit rows; k_out[p] = k_p, rel_err_sq[p] = ||d||_1 / ||d0||_1 and
 * status[p] (RBRP_OK, RBRP_ENOTCONVERGED or RBRP_ENONFINITE) are written to the
 * device arrays k_out, rel_err_sq and status (P entries each), valid once the
 * stream has reached the end of the call.
 * Workspace: device, 256-byte aligned, at least rbrp_batched_workspace_size
 * bytes; its contents need not be initialised.
 * Errors: RBRP_EINVAL, RBRP_EWORKSPACE, RBRP_ECUDA as for rbrp_id.
 */
rbrp_status rbrp_batched_workspace_size(int32_t P, const int64_t *m, const int64_t *n, const rbrp_opts *o,
                                        size_t *bytes);
rbrp_status rbrp_id_batched(int32_t P, const void *const *X, const int64_t *m, const int64_t *n, int x_is_fp64,
                            double tol, const rbrp_opts *o, void *workspace, size_t ws_bytes,
                            int64_t *const *skel, double *const *W, int64_t *k_out, double *rel_err_sq,
                            int32_t *status, rbrp_stream_t stream);

/*
 * Batch handle: the same computation as rbrp_id_batched, split so that the
 * device work can be replayed and captured in a CUDA graph.
 *
 * rbrp_batch_create validates the problems exactly as rbrp_id_batched does,
 * writes the problem table (pointers, sizes, processing order) into the
 * workspace with copies queued on `stream`, and returns a host handle that
 * remembers the workspace, the output arrays and the options (the caller
 * keeps all of them alive and unchanged until rbrp_batch_destroy).  The
 * handle allocates only host memory.
 *
 * Buckets: the problems are split by shape into at most two buckets, those
 * with n > 128 columns and those with n <= 128 (empty buckets are dropped,
 * wide first); each bucket is one persistent launch over its own work queue,
 * with its own schedule and per-CTA slot size.
 *
 * rbrp_batch_run queues one solve of every problem to tolerance tol on
 * `stream`: per bucket a 4-byte memset of its work counter and one kernel
 * launch, no host synchronisation and no host-to-device copy, so it may be
 * captured in a CUDA graph (the graph then replays the solve with that tol;
 * outputs are rewritten in full on every run).  Runs on one handle must not
 * overlap on the GPU (they share the workspace).
 *
 * Schedule of a bucket: `threads` (256 or 512) threads per CTA, `ctas_per_sm`
 * (1 or 2) CTAs resident on every SM, and the row width `vec` of the row
 * passes (the values of a row one lane holds: 8, for n <= 256, or 4, for n <=
 * 128, half the registers and multiply-adds a row).  Results do not depend on
 * the schedule.  A new handle takes, per bucket, the schedule that
 * rbrp_batch_autotune last chose for a bucket of the same shape in this
 * process (same precision, block, problem count, largest m and n, total
 * elements), else 256 threads, one CTA per SM and the narrowest row width
 * that holds the bucket's rows.  rbrp_batch_autotune times, bucket by bucket,
 * every schedule that fits on the device (one warm-up and `reps` timed
 * launches each, CUDA events on `stream`, synchronising the stream), keeps
 * the fastest on the handle and in the process-wide table, and returns the
 * sum over buckets of their times per run in *best_ms (may be NULL); it must
 * not be called while `stream` is being captured, and it overwrites the
 * outputs (with the same values any run produces).
 * rbrp_batch_set_schedule sets (threads, ctas_per_sm) on every bucket, each
 * with its narrowest row width; rbrp_batch_set_bucket_schedule sets bucket
 * i's three values; both return RBRP_EINVAL for a schedule the device cannot
 * hold (shared memory or registers) or a row width narrower than the
 * bucket's rows.  rbrp_batch_get_schedule reports bucket 0's schedule and
 * CTAs launched; rbrp_batch_buckets the number of buckets (0 for NULL);
 * rbrp_batch_get_bucket bucket i's problem count, largest n, schedule and
 * CTAs launched (any pointer may be NULL).
 *
 * Errors: as rbrp_id_batched; RBRP_EINVAL for a NULL handle, RBRP_ENOMEM if
 * the host handle cannot be allocated.
 */
typedef struct rbrp_batch_s *rbrp_batch;
rbrp_status rbrp_batch_create(int32_t P, const void *const *X, const int64_t *m, const int64_t *n, int x_is_fp64,
                              const rbrp_opts *o, void *workspace, size_t ws_bytes, int64_t *const *skel,
                              double *const *W, int64_t *k_out, double *rel_err_sq, int32_t *status,
                              rbrp_stream_t stream, rbrp_batch *out);
rbrp_status rbrp_batch_run(rbrp_batch h, double tol, rbrp_stream_t stream);
rbrp_status rbrp_batch_autotune(rbrp_batch h, double tol, int32_t reps, rbrp_stream_t stream, float *best_ms);
rbrp_status rbrp_batch_set_schedule(rbrp_batch h, int32_t threads, int32_t ctas_per_sm);
rbrp_status rbrp_batch_get_schedule(rbrp_batch h, int32_t *threads, int32_t *ctas_per_sm, int32_t *ctas);
int32_t rbrp_batch_buckets(rbrp_batch h);
rbrp_status rbrp_batch_get_bucket(rbrp_batch h, int32_t i, int32_t *problems, int64_t *n_max, int32_t *threads,
                                  int32_t *ctas_per_sm, int32_t *vec, int32_t *ctas);
rbrp_status rbrp_batch_set_bucket_schedule(rbrp_batch h, int32_t i, int32_t threads, int32_t ctas_per_sm,
                                           int32_t vec);
void rbrp_batch_destroy(rbrp_batch h);

/*
 * Sketchy pivoting with LU partial pivoting and the oversampled sketchy ID
 * (SkLUPP-OSID): the comparison method of Sec. 3.2 and Alg. 4, not rank-adaptive.
 *
 *   Y = X Omega (n x l): the sketching step of Sec. 3.2;
 *   S = the k pivot rows of LU with partial (row) pivoting of Y(:, 0:k), in pivot
 *       order (largest |Schur complement entry|, ties to the smaller row; a zero
 *       pivot ends the selection, so |S| < k when Y(:, 0:k) has rank below k);
 *   W = Y_c Y_{S,c}^+ with Y_c = Y(:, 0:c), c = osid_cols: Alg. 4 (OSID, c = l,
 *       the paper uses l = 3k) or Eq. (5.2) (c = k).  W(S,:) = I.
 *
 * W is built by the block loop of rbrp_id run on Y_c with S forced in order (no
 * sampling, no pivoting, no truncation: Sec. 5.1's identity L2 L1^{-1} = Y_c Y_{S,c}^+
 * for the accepted rows), so its update, chain and W solve are those of rbrp_id.
 *
 * X          device, row-major n x d, leading dimension ldx >= d; FP64 or FP32
 *            (x_is_fp64).  Read only.
 * Omega      device, row-major d x l: the embedding, drawn by the caller (the paper:
 *            i.i.d. N(0, 1/l) entries); FP64 when o->precision == RBRP_FP64, else FP32
 *            (then X must be FP32 too).  Read only.
 * k          skeletons wanted, 1 <= k <= min(n, l); osid_cols in [k, l] (0 = l).
 * o          precision: RBRP_FP64 runs the sketch, LUPP and the W pass in FP64; any
 *            other value runs the sketch and LUPP in FP32 and the W pass's update in
 *            that precision (its per-block chain always FP64); block: rows accepted
 *            per block of the W pass (as rbrp_opts.block); w_precision: the final solve.
 * skel       device int64[k]: S in pivot order.
 * W          device FP64 n x k, leading dimension ldw >= k; columns < |S| written.
 * res        host: k = |S|, blocks of the W pass, d0 and d_final of the W pass on Y_c
 *            (so rel_err_sq = ||Y_c - W Y_{S,c}||_F^2 / ||Y_c||_F^2, the sketched error).
 * workspace  device, 256-byte aligned, >= rbrp_sketch_workspace_size bytes.
 * Returns RBRP_ENOTCONVERGED when the W pass accepted fewer rows than LUPP chose (a
 * chosen row without residual left in Y_c); RBRP_ETIMEOUT when a bounded grid
 * barrier of the LUPP kernel gave up; otherwise as rbrp_id.  The call synchronises
 * the stream once after LUPP (to size the W pass) and returns after the work ends.
 */
typedef struct {
  int32_t precision;    /* rbrp_precision (see above)                              */
  int32_t block;        /* rows per block of the W pass, as rbrp_opts.block          */
  int32_t w_precision;  /* rbrp_w_precision                                         */
  int32_t osid_cols;    /* 0: all l columns (OSID, Alg. 4); k: Eq. (5.2)             */
} rbrp_sketch_opts;
rbrp_status rbrp_sketch_workspace_size(int64_t n, int64_t d, int64_t l, int64_t k, const rbrp_sketch_opts *o,
                                       size_t *bytes);
rbrp_status rbrp_sketch_id(const void *X, int x_is_fp64, int64_t n, int64_t d, int64_t ldx, const void *Omega,
                           int64_t l, int64_t k, const rbrp_sketch_opts *o, void *workspace, size_t ws_bytes,
                           int64_t *skel, double *W, int64_t ldw, rbrp_result *res, rbrp_stream_t stream);

/*
 * Row shards of one ID (the row-sharded block loop of Alg. 2 across processes;
 * SURVEY's multi-GPU design; no counterpart in the paper beyond Alg. 2 itself).
 *
 * The rows of X are split into contiguous shards, one per process (or several per
 * process); rows [row_base, row_base + n_local) of X live on this shard.  Every step of
 * a block runs on the shard's GPU through these calls; the caller exchanges the small
 * per-block data between shards (host arrays here; an all-gather / all-reduce between
 * processes):
 *   1. rbrp_shard_draw: this shard's candidates of the sampling step -- its b_t rows with
 *      the smallest race keys (Philox counters use the GLOBAL row index, so the keys are
 *      those one unsharded call draws), in ascending (key, row) order; rows are global
 *      indices, keys the race keys kappa (or -d_i for the greedy sampler).  b_t here is
 *      min(b, eligible rows of this shard, k_cap - k).  The caller merges all shards'
 *      lists and keeps the b_t globally smallest pairs (b_t = min(b, sum of the counts,
 *      k_cap - k)), in (key, row) order: that is S_t of one unsharded call.
 *   2. rbrp_shard_rows: the current residual rows (FP64) of the requested global rows
 *      this shard holds (owned[i] = 1), for the caller to assemble V = R(S_t, :).
 *   3. rbrp_shard_block: with V (b_t x d, FP64, row-major) and S_t identical on every
 *      shard, runs the rest of the block -- projection against Q (CGS2), the robust
 *      filter, acceptance, the update of this shard's rows, its ||d||_1 -- and returns the
 *      accepted global rows (b' of them) and this shard's ||d||_1.  Every shard computes
 *      the same Q', so the shards stay in step; the caller sums ||d||_1 over shards and
 *      runs the stopping test (||d||_1 <= tol ||d0||_1, ||d0||_1 = the sum of the sum_sq
 *      values rbrp_shard_create returned).
 *   4. after the loop: rbrp_shard_l_rows gives the rows of L held here for the requested
 *      skeleton rows; the caller assembles L1 = L(S, :) (k x k) and passes it to
 *      rbrp_shard_w, which solves Alg. 3 for this shard's rows of W (W(S,:) = I on the
 *      skeleton rows held here).
 * k_cap is the whole ID's min(n, d, k_max) (not this shard's).  The shard runs the FP64
 * filter, so o->precision may be RBRP_FP64, RBRP_FP32 or RBRP_TF32X3, or RBRP_TF32 with
 * o->chain = RBRP_CHAIN_FP64; residual form only.  The handle holds pointers into the
 * caller's workspace and X (both kept alive until rbrp_shard_destroy); every call is
 * synchronous on `stream` and returns RBRP_EINVAL for bad arguments, RBRP_ECUDA for CUDA
 * errors.
 */
typedef struct rbrp_shard_s *rbrp_shard;
rbrp_status rbrp_shard_workspace_size(int64_t n_local, int64_t d, int64_t k_cap, const rbrp_opts *o, size_t *bytes);
rbrp_status rbrp_shard_create(const void *X, int x_is_fp64, int64_t n_local, int64_t d, int64_t ldx, int64_t row_base,
                              int64_t k_cap, const rbrp_opts *o, void *workspace, size_t ws_bytes,
                              rbrp_stream_t stream, rbrp_shard *out, double *sum_sq);
rbrp_status rbrp_shard_draw(rbrp_shard h, int64_t *rows, double *keys, int64_t *count);
rbrp_status rbrp_shard_rows(rbrp_shard h, const int64_t *rows, int64_t count, double *V, int32_t *owned);
rbrp_status rbrp_shard_block(rbrp_shard h, const double *V, const int64_t *S_t, int64_t b_t, int64_t *accepted,
                             int64_t *bp, double *d_sum);
rbrp_status rbrp_shard_l_rows(rbrp_shard h, const int64_t *rows, int64_t count, int64_t k, double *Lrows,
                              int32_t *owned);
rbrp_status rbrp_shard_w(rbrp_shard h, const double *L1, const int64_t *skel, int64_t k, double *W, int64_t ldw);
void rbrp_shard_destroy(rbrp_shard h);

/* Human-readable name of a status code (static string). */
const char *rbrp_status_string(rbrp_status s);

/* The cudaError_t value behind the last RBRP_ECUDA returned on this thread. */
int rbrp_last_cuda_error(void);

/*
 * How the blocks of Alg. 2 are driven (process-wide; default RBRP_LOOP_DEVICE).
 * RBRP_LOOP_DEVICE: one CUDA graph per call whose conditional while node repeats
 * one block, the stopping test setting the node's condition on the device; the host
 * launches the graph and reads the result once.  The graph is built at the first call
 * with a given set of buffers, sizes and options and reused by later such calls
 * (rbrp_id is then not itself capturable into a caller's graph: it synchronises its
 * stream once to size the W solve).  RBRP_LOOP_HOST: the host queues blocks in groups
 * and reads the device state after each group.  Both run the same kernels and give
 * identical results; the device loop is used unless capture is unavailable, or while
 * profiling counters are on (they time each update launch with events).
 */
#define RBRP_LOOP_DEVICE 0
#define RBRP_LOOP_HOST 1
rbrp_status rbrp_set_loop_mode(int32_t mode);

/*
 * Bounded device waits (failure detection; no counterpart in the paper).  Every
 * wait of the library's kernels on another part of the same launch -- the
 * mbarrier waits between the roles of the tensor-core kernels (fused update,
 * W solve) and the grid barriers of the cooperative sampler -- gives up after
 * a number of polls.  The kernel then records RBRP_ETIMEOUT in the call's
 * device state, stops issuing work, waits for the copies and tensor-core
 * operations it has already issued, releases its tensor memory and returns;
 * every later kernel of the call returns at once and the call returns
 * RBRP_ETIMEOUT with its outputs unspecified.  The workspace stays usable: the
 * next call starts from a fresh state.
 * rbrp_set_wait_limits sets the poll limits of the calls started after it
 * (process-wide; 0 restores the default of 2^24 mbarrier polls and 2^25 grid
 * barrier polls, about a second each, far above any wait of a healthy run).  A
 * small limit makes the waits of a healthy run give up: that is how the
 * failure path is tested without hanging or faulting a GPU.
 */
void rbrp_set_wait_limits(uint32_t mbarrier_polls, uint32_t barrier_polls);

#ifdef __cplusplus
}
#endif

#endif /* RBRP_H */
