/*
 * tor.h -- C ABI of libtor: exact Torontonians on NVIDIA GB300 (sm_103a).
 *
 * The Torontonian of a 2n x 2n Hermitian matrix O (paper Sec. 1, Eq. tor) is
 *
 *     Tor(O) = sum_{Z subset of {1..n}} (-1)^{n-|Z|} / sqrt(det(I - O_Z)),
 *
 * where O_Z keeps, for each mode j in Z, both its a_j and a_j^dag rows and
 * columns.  For a Gaussian state with complex Husimi covariance Sigma the
 * input is the sampling matrix O = I - Sigma^{-1} (Sec. 1, Eq. A).
 *
 * The library evaluates the sum on the GPU by the paper's recursive subset
 * tree (Sec. 2, Algorithm 2 and Figs. 1-2): subsets share the Cholesky data of
 * their common prefix, so adding one mode costs one rank-2 Schur update of the
 * parent's trailing block instead of a new factorisation.
 *
 * Conventions for every call:
 *   - Every function returns a tor_status; nothing aborts or throws across this
 *     ABI (a host allocation that fails inside a call gives TOR_ENOMEM).
 *     Per-matrix failures are reported in tor_result.status.
 *   - Matrices are row-major complex128 (tor_c128 == numpy complex128 ==
 *     torch.cdouble) with leading dimension `ld` >= 2n, in complex elements.
 *   - Row order is TOR_LAYOUT_BLOCK (a_1..a_n, a_1^dag..a_n^dag) unless the
 *     context was created with TOR_LAYOUT_PAIRS (a_1, a_1^dag, a_2, ...), the
 *     order the paper uses (Sec. 2).  Tor is the same in both (rows and columns
 *     are permuted together).
 *   - Host inputs are copied before the call returns; the caller keeps
 *     ownership of every buffer it passes.  With TOR_IN_DEVICE the O pointers
 *     are device pointers on the context's device; they are read on the
 *     context's stream and must stay valid until the call returns (tor_eval*)
 *     or until the ticket has been polled (tor_submit).
 *   - n = 0 gives Tor = 1 (0 x 0 determinant).  n > 64 gives TOR_ETOOBIG.
 *   - Input checks (skipped with TOR_NO_CHECK): O Hermitian within
 *     1e-12 * max|O| (else TOR_ENOTHERM), finite entries (else TOR_EINVAL).
 *     I - O must be positive definite; a non-positive pivot anywhere in the
 *     tree gives TOR_ENOTPD for that matrix.
 */
#ifndef LIBTOR_TOR_H
#define LIBTOR_TOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TOR_OK = 0,
  TOR_EINVAL = 1,     /* bad argument or non-finite input */
  TOR_ENOTHERM = 2,   /* O is not Hermitian within tolerance */
  TOR_ENOTPD = 3,     /* I - O (or one of its principal blocks) is not positive definite */
  TOR_ENOMEM = 4,     /* device or pinned-host allocation failed, or over the memory budget */
  TOR_EAGAIN = 5,     /* result not ready yet (tor_poll) / queue full (tor_submit) */
  TOR_ETIMEOUT = 6,   /* the evaluation ran past tor_config.timeout_s and was stopped */
  TOR_ECANCELED = 7,  /* the evaluation was cancelled with tor_cancel */
  TOR_ECUDA = 8,      /* a CUDA runtime call failed; see tor_last_error */
  TOR_ETOOBIG = 9     /* n > 64 (or above the limit of the call) */
} tor_status;

typedef struct { double re, im; } tor_c128;

enum { TOR_LAYOUT_BLOCK = 0, TOR_LAYOUT_PAIRS = 1 };
/* tor_config.flags:
 *   TOR_IN_DEVICE  O pointers of tor_eval* are device pointers (e.g. torch CUDA tensors)
 *   TOR_NO_CHECK   skip the Hermitian / finiteness check of the input
 *   TOR_GRAPHS     capture each evaluation pass into a CUDA graph and replay it for
 *                  later calls of the same shape (same sizes in the same order)
 *   TOR_COMPLEX_PATH  evaluate every matrix in complex arithmetic.  By default a
 *                  matrix of the form [[P, Q], [conj(Q), conj(P)]] in block layout
 *                  (within 1e-12 max|O|; every physical Gaussian state has it) is
 *                  evaluated in real arithmetic on V = U^H (I - O) U, U the per-mode
 *                  map from (a, a^dag) to the quadratures (x, p): every principal
 *                  block of V has the determinant of the matching block of I - O,
 *                  and the update costs a quarter of the complex multiply-adds.
 *   TOR_EXTENDED   extended-precision factor (paper Sec. 5, "X = extended"): B = I - O,
 *                  every pivot, Schur-complement entry, determinant factor and term
 *                  in double-double arithmetic (about 106-bit significands; the FP64
 *                  path carries only the sum in double-double).  For weakly squeezed
 *                  states, whose terms cancel almost completely, the error falls from
 *                  ~1e-16 sum|term| to ~1e-30 sum|term|, at about 12x (real basis) to
 *                  19x (complex) the time per term.  The real basis is taken only for
 *                  exactly structured O here (the FP64 path accepts 1e-12 max|O|). */
enum { TOR_IN_DEVICE = 1u, TOR_NO_CHECK = 2u, TOR_GRAPHS = 4u, TOR_COMPLEX_PATH = 8u, TOR_EXTENDED = 16u };

/* tor_session_create kinds */
enum { TOR_SESSION_SIGMA = 0, TOR_SESSION_O = 1 };

typedef struct tor_ctx tor_ctx;
typedef struct tor_session tor_session;

typedef struct {
  int device;          /* CUDA device ordinal */
  void* stream;        /* cudaStream_t to run on; NULL = the library creates its own */
  size_t mem_budget;   /* cap on the device memory the context holds (slots and sessions), bytes; 0 = no cap */
  int prefix_depth;    /* unit prefix depth p for every n; -1 = built-in plan / autotune table */
  int layout;          /* TOR_LAYOUT_BLOCK or TOR_LAYOUT_PAIRS */
  unsigned flags;      /* TOR_IN_DEVICE | TOR_NO_CHECK */
  double timeout_s;    /* per call; 0 = none.  Past it the kernels stop and return TOR_ETIMEOUT */
} tor_config;

typedef struct {
  double hi, lo;       /* Tor as an unevaluated double-double sum hi + lo */
  double abs_sum;      /* sum over all subsets of |term|: the scale of the rounding error */
  double err_est;      /* a-priori error estimate 8 n u abs_sum, u = 2^-53 (2^-104 extended) */
  int n;               /* modes of this matrix */
  tor_status status;   /* per-matrix status */
  int path;            /* arithmetic used: bit 0 real (x, p) basis (else complex, see
                          TOR_COMPLEX_PATH), bit 1 double-double factor (TOR_EXTENDED) */
  int reserved;
} tor_result;

/* Fills *cfg with defaults: device 0, own stream, no budget, planned prefix
 * depth, block layout, no flags, no timeout. */
void tor_config_default(tor_config* cfg);

/* Creates a context on cfg->device (cfg may be NULL for defaults).  Allocates
 * nothing large until the first evaluation.  *out is NULL on failure. */
tor_status tor_create(const tor_config* cfg, tor_ctx** out);

/* Frees the context and all its device and pinned memory.  Requests still
 * queued for the serving loop are dropped, running kernels are asked to stop
 * (as tor_cancel), and the call blocks until the GPU work has ended.  Tickets
 * of the context are invalid afterwards.  NULL is ignored. */
void tor_destroy(tor_ctx* ctx);

/* Tor of one 2n x 2n matrix (Eq. tor).  Blocking.  The call's return value is
 * the first error of the call; *out carries the per-matrix status too. */
tor_status tor_eval(tor_ctx* ctx, int n, const tor_c128* O, int ld, tor_result* out);

/* Tor of `count` matrices of mixed sizes in one persistent-kernel launch.
 * n[i], O[i], ld[i] describe matrix i; out[i] receives its result.  Each
 * result is bitwise identical to tor_eval of the same matrix on the same
 * context (the unit decomposition depends on n only).  Blocking. */
tor_status tor_eval_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O,
                          const int* ld, tor_result* out);

/* The plain one-call-per-matrix path, looped in C: evaluates the `count`
 * matrices one after the other, each exactly as its own tor_eval call (its
 * own intake, units and reduce launches and one synchronisation), with no
 * interpreter between the calls.  Arguments as for tor_eval_batch; ms (may be
 * NULL) receives count host-measured wall times in milliseconds, one per
 * matrix (call entry to return).  Results equal tor_eval_batch's bitwise.
 * The paper has no counterpart: this is the plain path that a batched launch
 * of many matrices is compared with.  Returns the first error. */
tor_status tor_eval_seq(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                        tor_result* out, double* ms);

/* Queues one matrix for evaluation and returns at once with a ticket.  The
 * context's serving thread batches queued requests continuously: a request
 * that arrives while others run is admitted as soon as a slot and the device
 * memory budget allow.  Large requests (more than 2^25 subset terms) run FIFO
 * in two low-priority lanes, one request each, so the next large request's
 * blocks take the SMs that the current one's last tasks leave idle; small
 * requests are batched FIFO into two high-priority lanes, whose blocks take
 * SMs as soon as any block of a large request ends, and may pass large
 * requests that wait.  The serving thread polls running jobs without sleeping,
 * and when it goes idle it spins for up to 50 ms before it sleeps, so that a
 * request arriving soon starts without a thread wake-up (it occupies one host
 * core meanwhile).  (Environment: TOR_SERVE_IDLE_SPIN_MS sets that spin, 0 =
 * sleep at once; for experiments TOR_SERVE_SLICE_MS = t makes large requests
 * yield the SMs every t ms, and TOR_SERVE_LARGE_LANES = 1..3.)  Each result is bitwise the same as
 * tor_eval of the same matrix on the same context.  TOR_EAGAIN if the queue
 * is full. */
tor_status tor_submit(tor_ctx* ctx, int n, const tor_c128* O, int ld, uint64_t* ticket);

/* Waits up to timeout_s (0 = do not wait, < 0 = forever) for a ticket.
 * Returns TOR_EAGAIN if it is still pending, TOR_EINVAL for an unknown or
 * already collected ticket, else the request's status with *out filled. */
tor_status tor_poll(tor_ctx* ctx, uint64_t ticket, tor_result* out, double timeout_s);

/* Waits up to timeout_s (0 = do not wait, < 0 = forever) until any of the
 * `count` tickets has completed, collects that one request (as tor_poll does)
 * and writes its position in tickets[] to *index.  The others stay pending.
 * Returns TOR_EAGAIN if none completed in time, TOR_EINVAL if a ticket is
 * unknown or already collected, else the collected request's status.  For a
 * client with many requests in flight, which then sees each completion when
 * it happens rather than in submission order.  Serving machinery; the paper
 * has no counterpart. */
tor_status tor_poll_any(tor_ctx* ctx, const uint64_t* tickets, int count, double timeout_s, int* index,
                        tor_result* out);

/* Device bytes the context holds now -- every slot's buffers and the
 * resident matrices of its sessions -- and its budget (tor_config.mem_budget,
 * 0 = none); either pointer may be NULL.  Under a budget the serving loop
 * admits a batch only if the bytes held stay within it: idle slots give their
 * buffers back first, then the batch shrinks, and a request that cannot fit
 * with nothing else running fails with TOR_ENOMEM.  A blocking call over the
 * budget fails with TOR_ENOMEM (it does not take memory from serving slots).
 * Serving machinery; the paper has no counterpart. */
tor_status tor_memory(tor_ctx* ctx, size_t* held, size_t* budget);

/* Served requests, completed batches and requests still queued (any may be NULL). */
tor_status tor_serving_stats(tor_ctx* ctx, long long* served, long long* batches, long long* queued);

/* ---- chain-rule marginals (threshold GBS sampling, paper Sec. 1) ----
 *
 * Sampling click patterns mode by mode needs Tor of the sampling matrix of
 * every prefix of the modes: O^(j) = I - (Sigma_[j])^{-1}, where Sigma_[j] is
 * the covariance of modes 0..j-1 (Eq. A applied to the marginal state), and
 * the click probability of a pattern S on those modes is
 * Tor(O^(j)_S) / sqrt(det Sigma_[j]).
 *
 * tor_session_create takes the full n_total-mode covariance Sigma
 * (kind TOR_SESSION_SIGMA) or sampling matrix O (kind TOR_SESSION_O), 2n x 2n
 * with leading dimension ld in the context's layout, computes every O^(j)
 * on the host (extended precision, one rank-2 downdate of Sigma^{-1} per
 * mode) and keeps them all resident on the device (16 * sum_j 4 j^2 bytes,
 * ~64 MB for 144 modes).  The caller's buffer may be freed afterwards. */
tor_status tor_session_create(tor_ctx* ctx, int n_total, const tor_c128* M, int ld, int kind,
                              tor_session** out);

/* Frees a session's device matrices.  Requests of this session still queued
 * are completed with TOR_ECANCELED, and the call blocks until every request
 * of the session that is already running on the GPU has finished, so no
 * kernel reads the matrices after they are freed.  A session may outlive its
 * context (destroying the context detaches it).  NULL is ignored. */
void tor_session_destroy(tor_session* s);

/* Copies the session's resident O^(j) (2j x 2j, the exact matrix every
 * marginal of prefix j reads) to the host buffer out, row-major with leading
 * dimension ld >= 2j, in the layout of the context the session was made on
 * (block if that context is gone): the sampling matrix of the first j modes'
 * marginal state (Eq. A applied to Sigma_[j], Sec. 1).  For checking marginals
 * against another evaluator on identical inputs.  TOR_EINVAL for j outside
 * [1, n_total] or ld < 2j; TOR_ECUDA if the copy fails.  Blocking. */
tor_status tor_session_marginal_matrix(tor_session* s, int j, tor_c128* out, int ld);

/* Tor(O^(j)_S) for S = modes[0..k-1] (distinct, each < j, any order), blocking. */
tor_status tor_eval_marginal(tor_ctx* ctx, tor_session* s, int j, int k, const int* modes,
                             tor_result* out);

/* Queues the same evaluation for the serving loop (see tor_submit); poll the
 * ticket with tor_poll.  The mode list is copied. */
tor_status tor_submit_marginal(tor_ctx* ctx, tor_session* s, int j, int k, const int* modes,
                               uint64_t* ticket);

/* Draws click patterns of threshold detectors on the first n_modes modes of
 * the session's state by the chain rule -- the use of the Torontonian as the
 * probability of a threshold-detection outcome (Sec. 1).  For each sample,
 * modes j = 0, 1, ... are decided in order: with S the clicks so far,
 *   t0 = Tor(O^(j+1)_S),  t1 = Tor(O^(j+1)_{S u {j}}),
 *   P(click at j | S) = t1 / (t0 + t1),
 * and mode j clicks iff uniforms[i * n_modes + j] < P(click at j | S).
 *   uniforms  count x n_modes doubles in [0, 1), sample-major: the random
 *             numbers, drawn by the caller (the call itself draws none).
 *   patterns  out: count x n_modes bytes, 1 = click.
 *   prob      out (may be NULL): P(pattern) = Tor(O^(n_modes)_S) / sqrt(det
 *             Sigma_[n_modes]), the probability of each drawn pattern.
 *   max_dev   out (may be NULL): the largest |(t0 + t1) / sqrt(det Sigma_[j+1])
 *             - P(S on the first j modes)| / P(...) over samples and steps --
 *             the chain rule's consistency, a rounding-level number.
 * One step evaluates the distinct marginals of all samples (samples with the
 * same clicks so far share theirs; at most 2 count per step) in batched
 * blocking launches of the context, as tor_eval_batch would, so each t equals
 * tor_eval_marginal's bitwise.  Each evaluation is exact and costs 2^|S|; patterns with more
 * than 64 clicks return TOR_ETOOBIG.  Under TOR_EXTENDED the t's carry ~106
 * bits, for weakly squeezed states whose Torontonians cancel (Sec. 5).
 * Returns TOR_EINVAL for bad arguments (n_modes > the session's modes, a
 * uniform outside [0, 1)), else the first failing status of an evaluation;
 * blocking; patterns and prob are valid only on TOR_OK. */
tor_status tor_sample(tor_ctx* ctx, tor_session* s, int count, int n_modes, const double* uniforms,
                      unsigned char* patterns, double* prob, double* max_dev);

/* Asks the kernels running for this context to stop at their next unit
 * boundary; the affected results get TOR_ECANCELED.  Thread-safe. */
tor_status tor_cancel(tor_ctx* ctx);

/* Human-readable name of a status.  Never NULL. */
const char* tor_strerror(tor_status s);

/* Last CUDA error string seen by this context ("" if none); with ctx == NULL,
 * the last error of a failed tor_create on this thread.  Never NULL. */
const char* tor_last_error(tor_ctx* ctx);

/* ---- inspection and measurement (same kernels, more output) ---- */

/* Prefix depth p the context uses for n modes (2^p equal units, each a subtree
 * over the last n - p modes).  -1 if n is out of range. */
int tor_plan_prefix_depth(tor_ctx* ctx, int n);

/* Sets the prefix depth used for n modes from now on (the autotuner's entry
 * point).  p in [0, min(n-1, 30)] (2^30 unit partials take 32 GB), or -1 for
 * the built-in plan.  Changing it changes the summation order, so results
 * before and after differ in rounding. */
tor_status tor_set_prefix_depth(tor_ctx* ctx, int n, int p);

/* Like tor_eval, but also copies the 2^p per-unit partial sums to the host:
 * unit u (bit j of u set <=> mode j is in Z, for j < p) sums the terms of all
 * Z whose first p decisions are u.  partials must hold 3 * 2^p doubles:
 * (hi, lo, abs_sum) per unit, in u order.  p = tor_plan_prefix_depth(ctx, n). */
tor_status tor_eval_units(tor_ctx* ctx, int n, const tor_c128* O, int ld, double* partials,
                          size_t partials_len, tor_result* out);

/* ---- sharding one matrix across processes or GPUs ----
 *
 * The final reduction of tor_eval is a fixed binary tree whose leaves are the
 * matrix's warp tasks: 2^(p-5) of them for prefix depth p >= 5, each the sum
 * of 32 units.  tor_plan_leaves gives that count (2^p units for p < 5).
 * tor_eval_range evaluates the leaves [leaf_lo, leaf_lo + leaf_count) only and
 * returns their binary-tree sum in out (hi, lo, abs_sum, status).  leaf_count
 * must be a power of two and leaf_lo a multiple of it, and p >= 5.  Combining
 * the results of the 2^s equal aligned ranges with the same tree (double-double
 * addition, left operand first) reproduces tor_eval's result bitwise. */
long long tor_plan_leaves(tor_ctx* ctx, int n);
tor_status tor_eval_range(tor_ctx* ctx, int n, const tor_c128* O, int ld, long long leaf_lo, long long leaf_count,
                          tor_result* out);

/* A shard of each of several matrices in one launch (one process's share of a
 * strong-scaled batch, paper Sec. 4): matrix i (n[i], O[i], ld[i] as for
 * tor_eval_batch; ld may be NULL for 2 n[i]) evaluates the leaves
 * [leaf_lo[i], leaf_lo[i] + leaf_count[i]) under the rules of tor_eval_range,
 * or, with leaf_count[i] < 0, all of them (any p).  The warp tasks of all the
 * ranges share one persistent launch, largest subtrees first, so the tail of
 * one matrix's range is filled by the others'.  Each out[i] equals the
 * tor_eval_range (or tor_eval) result of its matrix alone bitwise.  An invalid
 * range (leaf_count 0, not a power of two, misaligned, beyond the leaves, or
 * p < 5) sets out[i].status = TOR_EINVAL and the others still run; returns the
 * first error. */
tor_status tor_eval_range_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                                const long long* leaf_lo, const long long* leaf_count, tor_result* out);

/* Device time of the last tor_eval / tor_eval_batch, split by kernel, from CUDA
 * events on the context's stream: [0] intake, [1] units, [2] reduce, [3] total
 * (ms).  With TOR_GRAPHS only the total is measured; [0..2] are -1.  times
 * must hold 4 doubles. */
tor_status tor_last_times(tor_ctx* ctx, double* times);

/* Autotuner: for every n in [n_lo, n_hi], times tor_eval at prefix depths
 * around the built-in plan (control flow depends on n and p only, so a fixed
 * synthetic matrix serves) and keeps the fastest for this context.  Spends
 * about budget_s seconds in total.  chosen (may be NULL) receives
 * n_hi - n_lo + 1 depths.  Not for contexts created with TOR_IN_DEVICE. */
tor_status tor_autotune(tor_ctx* ctx, int n_lo, int n_hi, double budget_s, int* chosen);

/* Autotuner for a batch shape: tunes the prefix depths of the sizes in the
 * batch (n[i], O[i], ld[i] as for tor_eval_batch, in the context's input kind)
 * for the throughput of the whole batch, which may want other depths than
 * single matrices of those sizes (larger units cost less per term once many
 * matrices fill the GPU).  Coordinate descent in steps of one level over: the
 * depths of all sizes together, then each size holding at least a tenth of
 * the batch's subset terms, then the remaining sizes together; each trial
 * times the whole batch (best of two after a warm-up), and a coordinate moves
 * while the batch gets faster by more than 0.5 %.  Spends
 * about budget_s seconds (at least one trial).  chosen (may be NULL) receives
 * count depths, one per matrix.  The depths stay in the context's plan (save
 * them with tor_plan_save); results change in rounding with the depth.  The
 * paper has no counterpart (its decomposition is the uneven first loop of
 * Algorithm 2, Sec. 4). */
tor_status tor_autotune_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                              double budget_s, int* chosen);

/* Writes / reads the context's prefix-depth table (text: "n p" per line,
 * plus the resident warp count it was tuned for).  tor_plan_load rejects a
 * table tuned for a different number of resident warps with TOR_EINVAL.
 * tor_create loads the table named by the environment variable
 * TOR_AUTOTUNE_CACHE, if set, unless cfg->prefix_depth >= 0. */
tor_status tor_plan_save(tor_ctx* ctx, const char* path);
tor_status tor_plan_load(tor_ctx* ctx, const char* path);

/* Measures the device's FP64 FMA throughput with a saturating kernel (all SMs,
 * 8 warps each, independent chains) for about `seconds`.  Writes DFMA per
 * second and FP64 TFLOP/s (2 flops per DFMA). */
tor_status tor_probe_fp64(int device, double seconds, double* dfma_per_s, double* fp64_tflops);

/* The FP64 reciprocal and reciprocal square root of every include step's 2x2
 * pivot (the rsqrt and rcp of Algorithm 1's diagonal and of the Schur
 * complement's pivot, Sec. 2): the hardware estimate (rcp/rsqrt.approx.ftz.f64)
 * refined by one cubic series step.  For each of the `count` host doubles x[i]
 * writes four host doubles out[4i..4i+3] computed on `device`: the library's
 * reciprocal, CUDA's IEEE division 1.0 / x (round to nearest), the library's
 * reciprocal square root and CUDA's rsqrt(x) -- so a test can state the error
 * of the library's versions.  Valid for normal x with a normal reciprocal
 * (2^-1022 <= |x| < 2^1022; positive x for the square root): the estimates
 * flush subnormals to zero.  Allocates and frees device memory; blocking.
 * TOR_EINVAL for bad arguments (count above 2^26). */
tor_status tor_check_recip(int device, int count, const double* x, double* out);

/* ---- evaluation without allocation ---- */

/* Largest n tor_eval_noalloc accepts. */
#define TOR_NOALLOC_MAX_N 16

/* Tor of one matrix with no memory allocation of any kind, for callers that
 * must not allocate while they run (a process whose device memory is owned by
 * a pre-reserved pool, a latency-critical loop in which cudaMalloc/cudaFree
 * would synchronise the device, a plugin allowed to allocate only at start-up).
 * The paper has no counterpart; it is a deployment variant of tor_eval.
 *
 *   device  CUDA device ordinal; the call makes it current and restores the
 *           caller's current device before returning.
 *   n, O, ld, layout
 *           as for tor_eval, but O is a DEVICE pointer on `device`
 *           (row-major complex128, leading dimension ld >= 2n).
 *   stream  cudaStream_t on `device` (NULL = the legacy default stream).
 *   out     DEVICE pointer to one tor_result, written by the GPU.
 *
 * The call only enqueues work on `stream` and returns; synchronise the stream
 * before reading *out.  Per-matrix failures (not Hermitian, not positive
 * definite, non-finite input) appear in out->status.  The return value covers
 * the call itself: TOR_ETOOBIG for n > TOR_NOALLOC_MAX_N, TOR_EINVAL for bad
 * arguments (n < 1, NULL pointers, ld < 2n, unknown layout or device),
 * TOR_ECUDA if a launch fails.
 *
 * All intermediate data lives in one static device array of 12 MiB compiled
 * into the library, which every device that loads the library keeps until
 * the process exits.  Calls share it: calls whose GPU work overlaps (other
 * streams or threads on the same device) race and must be ordered by the
 * caller.  The first call on each device looks up the array's device address
 * (and may load the library's GPU module), so make that first call before
 * any stream capture starts. */
tor_status tor_eval_noalloc(int device, int n, const tor_c128* O, int ld, int layout, void* stream,
                            tor_result* out);

#ifdef __cplusplus
}
#endif

#endif /* LIBTOR_TOR_H */
