/*
 * tor_oracle.c -- TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct CPU
 * reference for the Torontonian.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never does.
 *
 * What it computes (paper Sec. 1, Eq. tor):
 *     Tor(O) = sum_{Z subset of [n]} (-1)^{n-|Z|} / sqrt(|det(I - O_Z)|)
 * where O_Z keeps, for every mode j in Z, both of its rows/columns (a_j and
 * a_j^dag).  n = number of modes; O is 2n x 2n.
 *
 * Two independent formulations, both in binary128 ("quad"):
 *   tor_oracle_brute      -- the definition written out: every subset, its own
 *                            LU determinant with partial pivoting, terms summed in
 *                            mask order with Neumaier compensation.
 *   tor_oracle_recursive  -- the paper's Algorithm 2 (Sec. 2): start from the
 *                            Cholesky factor (Algorithm 1) of I - A, remove one
 *                            mode per recursion step with strictly increasing mode
 *                            index, reuse the blocks L11 and L21 of the parent factor
 *                            and recompute only L22 (Fig. 2), one addend per step.
 *
 * Quad type: __float128 on x86_64 (libquadmath), long double on aarch64 (IEEE
 * binary128 there).  Inputs are complex128, converted exactly to quad.
 *
 * Readings of the paper taken here:
 *   - |det| in Eq. tor: the determinant of I - O_Z is real and positive for valid
 *     input; the code uses |Re det| and reports max |Im det|/|det|.
 *   - The empty subset contributes (-1)^n (determinant of a 0x0 matrix is 1).
 *   - Mask bit j set <=> mode j is in Z.  Block layout: mode j owns rows {j, j+n};
 *     pairs layout: rows {2j, 2j+1}.
 *
 * Parity pins for this file live in tests/test_oracle_pins.py (closed forms,
 * physics identities, brute force vs Algorithm 2).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <stdio.h>

#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 quad;
static quad q_sqrt(quad x) { return sqrtq(x); }
static quad q_fabs(quad x) { return fabsq(x); }
#else
#include <math.h>
typedef long double quad;
static quad q_sqrt(quad x) { return sqrtl(x); }
static quad q_fabs(quad x) { return fabsl(x); }
#endif

typedef struct { quad re, im; } cq;

static cq c_sub(cq a, cq b) { cq r = {a.re - b.re, a.im - b.im}; return r; }
static cq c_mul(cq a, cq b) { cq r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return r; }
static cq c_conj(cq a) { cq r = {a.re, -a.im}; return r; }
static quad c_abs2(cq a) { return a.re * a.re + a.im * a.im; }
static cq c_div(cq a, cq b) {
  quad d = c_abs2(b);
  cq r = {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
  return r;
}

/* Mutations planted on purpose by tests (0 = none).  They show that the pins
 * catch a plausible mistake; production callers always pass 0. */
enum { MUT_NONE = 0, MUT_SIGN = 1, MUT_PAIRING = 2, MUT_DROP_EMPTY = 3, MUT_NO_IDENTITY = 4,
       MUT_TRANSPOSE_HALF = 5 };

typedef struct {
  int n, layout, ld, mutate;
  const double* O; /* interleaved (re, im), row-major, leading dimension ld (complex elements) */
} problem;

/* Row index of component c (0 = a, 1 = a^dag) of mode j. */
static int row_of(const problem* P, int j, int c) {
  if (P->mutate == MUT_PAIRING) return P->layout == 0 ? 2 * j + c : j + c * P->n;
  return P->layout == 0 ? j + c * P->n : 2 * j + c;
}

static cq O_at(const problem* P, int r, int s) {
  const double* p = P->O + 2 * ((size_t)r * P->ld + s);
  cq v = {(quad)p[0], (quad)p[1]};
  return v;
}

/* det(I - O_Z) by LU with partial pivoting; returns det, sets im_ratio. */
static cq det_IminusOZ(const problem* P, uint64_t mask, cq* W, int* idx) {
  int k = 0;
  for (int j = 0; j < P->n; ++j) if ((mask >> j) & 1ull) { idx[k++] = j; }
  int m = 2 * k;
  if (m == 0) { cq one = {1, 0}; return one; }
  /* gather rows in the order (a of each selected mode, then a^dag of each) */
  int* rows = idx + P->n;
  for (int t = 0; t < k; ++t) { rows[t] = row_of(P, idx[t], 0); rows[t + k] = row_of(P, idx[t], 1); }
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      cq o = (P->mutate == MUT_TRANSPOSE_HALF && a < k && b >= k) ? O_at(P, rows[b], rows[a])
                                                                 : O_at(P, rows[a], rows[b]);
      cq v = {-o.re, -o.im};
      if (a == b && P->mutate != MUT_NO_IDENTITY) v.re += 1;
      W[a * m + b] = v;
    }
  cq det = {1, 0};
  for (int c = 0; c < m; ++c) {
    int piv = c; quad best = c_abs2(W[c * m + c]);
    for (int r = c + 1; r < m; ++r) { quad v = c_abs2(W[r * m + c]); if (v > best) { best = v; piv = r; } }
    if (best == 0) { cq z = {0, 0}; return z; }
    if (piv != c) {
      for (int b = 0; b < m; ++b) { cq t = W[c * m + b]; W[c * m + b] = W[piv * m + b]; W[piv * m + b] = t; }
      det.re = -det.re; det.im = -det.im;
    }
    cq d = W[c * m + c];
    det = c_mul(det, d);
    for (int r = c + 1; r < m; ++r) {
      cq f = c_div(W[r * m + c], d);
      for (int b = c + 1; b < m; ++b) W[r * m + b] = c_sub(W[r * m + b], c_mul(f, W[c * m + b]));
    }
  }
  return det;
}

typedef struct {
  const problem* P;
  uint64_t base, stride, k0, k1;
  quad* terms; double* im_ratio;
} job;

static void* brute_worker(void* arg) {
  job* J = (job*)arg;
  const problem* P = J->P;
  int mm = 2 * P->n;
  cq* W = (cq*)malloc(sizeof(cq) * (size_t)(mm > 0 ? mm * mm : 1));
  int* idx = (int*)malloc(sizeof(int) * (size_t)(3 * P->n + 2));
  double worst = 0;
  for (uint64_t k = J->k0; k < J->k1; ++k) {
    uint64_t mask = J->base + k * J->stride;
    cq det = det_IminusOZ(P, mask, W, idx);
    int z = __builtin_popcountll(mask);
    quad mag2 = c_abs2(det);
    if (mag2 > 0) { double ir = (double)(q_fabs(det.im) / q_sqrt(mag2)); if (ir > worst) worst = ir; }
    quad t = 1 / q_sqrt(q_fabs(det.re));
    int neg = (P->n - z) & 1;
    if (P->mutate == MUT_SIGN) neg = z & 1;   /* (-1)^{|Z|}: wrong whenever n is odd */
    if (P->mutate == MUT_DROP_EMPTY && mask == 0) t = 0;
    J->terms[k - J->k0] = neg ? -t : t;
  }
  *J->im_ratio = worst;
  free(W); free(idx);
  return 0;
}

/* Neumaier compensated summation (Neumaier, ZAMM 54 (1974)) in quad. */
typedef struct { quad s, c; } neumaier;
static void nm_add(neumaier* a, quad x) {
  quad t = a->s + x;
  if (q_fabs(a->s) >= q_fabs(x)) a->c += (a->s - t) + x; else a->c += (x - t) + a->s;
  a->s = t;
}

static void quad_to_dd(quad v, double* hi, double* lo) {
  double h = (double)v;
  *hi = h;
  *lo = (double)(v - (quad)h);
}

/*
 * Sum of the terms of the masks base + k*stride, k in [0, count), in k order.
 * out[0..1] = Tor as double-double (hi, lo), out[2] = sum |term|,
 * out[3] = max |Im det| / |det| seen, out[4] = count summed.
 * Returns 0 on success, -1 on bad arguments.
 */
int tor_oracle_brute(int n, const double* O, int ld, int layout, uint64_t base, uint64_t stride,
                     uint64_t count, int nthreads, int mutate, double* out) {
  if (n < 0 || n > 40 || (n > 0 && !O) || !out || ld < 2 * n || nthreads < 1 || stride == 0) return -1;
  problem P = {n, layout, ld, mutate, O};
  neumaier acc = {0, 0}, abs_acc = {0, 0};
  double worst = 0;
  const uint64_t CH = 1ull << 16;
  quad* terms = (quad*)malloc(sizeof(quad) * CH);
  if (!terms) return -1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256]; job J[256]; double ir[256];
  for (uint64_t k0 = 0; k0 < count; k0 += CH) {
    uint64_t k1 = k0 + CH < count ? k0 + CH : count;
    uint64_t span = k1 - k0;
    int T = (int)((uint64_t)nthreads < span ? (uint64_t)nthreads : span);
    for (int t = 0; t < T; ++t) {
      uint64_t a = k0 + span * t / T, b = k0 + span * (t + 1) / T;
      J[t].P = &P; J[t].base = base; J[t].stride = stride; J[t].k0 = a; J[t].k1 = b;
      J[t].terms = terms + (a - k0); J[t].im_ratio = &ir[t];
      if (T == 1) brute_worker(&J[t]); else pthread_create(&th[t], 0, brute_worker, &J[t]);
    }
    for (int t = 0; t < T; ++t) {
      if (T > 1) pthread_join(th[t], 0);
      if (ir[t] > worst) worst = ir[t];
    }
    for (uint64_t i = 0; i < span; ++i) { nm_add(&acc, terms[i]); nm_add(&abs_acc, q_fabs(terms[i])); }
  }
  free(terms);
  quad tor = acc.s + acc.c;
  quad_to_dd(tor, &out[0], &out[1]);
  out[2] = (double)(abs_acc.s + abs_acc.c);
  out[3] = worst;
  out[4] = (double)count;
  return 0;
}

/* Tor as a decimal string with 34 significant digits (x86: quadmath_snprintf). */
int tor_oracle_brute_string(int n, const double* O, int ld, int layout, int nthreads, char* buf, int len) {
  double out[5];
  int rc = tor_oracle_brute(n, O, ld, layout, 0, 1, n >= 0 && n < 64 ? (1ull << n) : 0, nthreads, 0, out);
  if (rc) return rc;
  /* hi + lo carries ~106 bits; print both parts, the caller adds them exactly. */
#if defined(__x86_64__)
  quadmath_snprintf(buf, (size_t)len, "%.34Qe", (__float128)out[0] + (__float128)out[1]);
#else
  snprintf(buf, (size_t)len, "%.34Le", (long double)out[0] + (long double)out[1]);
#endif
  return 0;
}

/* ---------------- Algorithm 2 of the paper (remove-mode recursion) ---------------- */

typedef struct {
  int n, N;            /* modes, matrix size 2n (pairs order inside) */
  cq* A;               /* I - O in pairs order, full N x N */
  neumaier tor, abs;
  int mutate;
} rec_state;

/* Cholesky (Algorithm 1), rows r0..m-1 of L given rows < r0 already in place.
 * M is the m x m matrix (full), L is m x m lower triangular (row-major). */
static int chol_rows(const cq* M, cq* L, int m, int r0) {
  /* rows < r0 and columns < r0 are already in place (L11, L21); compute L22 */
  for (int i = r0; i < m; ++i) {
    for (int j = r0; j < i; ++j) {
      cq s = M[i * m + j];
      for (int k = 0; k < j; ++k) s = c_sub(s, c_mul(L[i * m + k], c_conj(L[j * m + k])));
      L[i * m + j] = c_div(s, L[j * m + j]);
    }
    quad d = M[i * m + i].re;
    for (int k = 0; k < i; ++k) d -= c_abs2(L[i * m + k]);
    if (!(d > 0)) return -1;
    cq v = {q_sqrt(d), 0};
    L[i * m + i] = v;
  }
  return 0;
}

/* One step of Algorithm 2: remove mode i (at position q of kept) from the kept set.
 * createAZ builds I - A_Z for the reduced set; the rows and columns before the
 * removed mode keep L11 and L21 of the parent factor (Fig. 2) and only the block
 * 22 is refactored (Algorithm 1).  Returns the new kept list and factor
 * (caller frees), or 0 if I - A_Z is not positive definite. */
static cq* remove_mode(const rec_state* S, const int* kept, int nk, const cq* L, int q, int** kept_out) {
  int m = 2 * nk;
  int nk2 = nk - 1, m2 = 2 * nk2;
  int* kept2 = (int*)malloc(sizeof(int) * (size_t)(nk2 > 0 ? nk2 : 1));
  for (int t = 0, u = 0; t < nk; ++t) if (t != q) kept2[u++] = kept[t];
  /* Only lower triangles are written and read: M2 and L2 are Hermitian and
   * lower triangular respectively, and Algorithm 1 reads M2 on and below the
   * diagonal. */
  cq* M2 = (cq*)malloc(sizeof(cq) * (size_t)(m2 > 0 ? m2 * m2 : 1));
  cq* L2 = (cq*)malloc(sizeof(cq) * (size_t)(m2 > 0 ? m2 * m2 : 1));
  int r0 = 2 * q;
  /* createAZ: the entries of I - A_Z for the reduced mode set (A is global)
   * that the refactorisation of block 22 reads: rows r0.., columns r0..row */
  for (int a = r0; a < m2; ++a)
    for (int b = r0; b <= a; ++b) {
      int ra = 2 * kept2[a / 2] + (a & 1), rb = 2 * kept2[b / 2] + (b & 1);
      M2[a * m2 + b] = S->A[ra * S->N + rb];
    }
  /* reuse L11 (rows/cols before mode i) and L21 (rows after, cols before) */
  for (int a = 0; a < m2; ++a)
    for (int b = 0; b < r0 && b <= a; ++b) {
      int pa = a < r0 ? a : a + 2;   /* row index in the parent factor */
      L2[a * m2 + b] = L[pa * m + b];
    }
  int rc = chol_rows(M2, L2, m2, r0);   /* recompute block 22 */
  free(M2);
  if (rc) { free(kept2); free(L2); return 0; }
  *kept_out = kept2;
  return L2;
}

/* The addend of one node: (-1)^{#removed} / sqrt(prod |L_aa|^2), into the node's sums. */
static void add_term(rec_state* S, const cq* L, int m, int removed_count) {
  quad det = 1;
  for (int a = 0; a < m; ++a) det *= c_abs2(L[a * m + a]);
  quad t = 1 / q_sqrt(det);
  quad term = (removed_count & 1) ? -t : t;
  nm_add(&S->tor, term);
  nm_add(&S->abs, t);
}

/* kept: list of kept modes (ascending), L: factor of I - A restricted to them.
 * Removes, one per step, every kept mode i >= start (the loop of Algorithm 2),
 * adds that node's addend and recurses with start = i + 1. */
static int recursive_tor(rec_state* S, const int* kept, int nk, const cq* L, int removed_count, int start) {
  for (int i = start; i < S->n; ++i) {
    /* position of mode i in kept */
    int q = -1;
    for (int t = 0; t < nk; ++t) if (kept[t] == i) { q = t; break; }
    if (q < 0) continue;
    int* kept2 = 0;
    cq* L2 = remove_mode(S, kept, nk, L, q, &kept2);
    if (!L2) return -1;
    add_term(S, L2, 2 * (nk - 1), removed_count + 1);
    int rc = recursive_tor(S, kept2, nk - 1, L2, removed_count + 1, i + 1);
    free(kept2); free(L2);
    if (rc) return rc;
  }
  return 0;
}

/* Task u of a split at depth d (the paper distributes the first loop of
 * Algorithm 2 over workers, Sec. 4; here the tasks are the 2^d patterns of
 * removals among modes 0..d-1, which have equal subtrees).  The task reaches
 * the node that removed exactly the modes of u (removals in increasing mode
 * order, as the recursion makes them), adds its addend, then runs the
 * recursion over the modes d..n-1 only.  Every subset of removed modes
 * belongs to exactly one task. */
typedef struct {
  const rec_state* S0;
  int d;
  const cq* L0;
  uint64_t next, ntasks;
  pthread_mutex_t* lock;
  neumaier* tor; neumaier* abs; int* rc;
} alg2_pool;

static int alg2_task(const rec_state* S0, int d, const cq* L0, uint64_t u, neumaier* tor, neumaier* abs) {
  rec_state S = *S0;
  S.tor.s = S.tor.c = 0; S.abs.s = S.abs.c = 0;
  int n = S.n;
  int* kept = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j) kept[j] = j;
  int nk = n, removed = 0;
  cq* L = (cq*)malloc(sizeof(cq) * (size_t)(n > 0 ? 4 * n * n : 1));
  memcpy(L, L0, sizeof(cq) * (size_t)(4 * n * n));
  int rc = 0;
  for (int i = 0; i < d && !rc; ++i) {
    if (!((u >> i) & 1ull)) continue;
    int q = -1;
    for (int t = 0; t < nk; ++t) if (kept[t] == i) { q = t; break; }
    int* kept2 = 0;
    cq* L2 = remove_mode(&S, kept, nk, L, q, &kept2);
    if (!L2) { rc = -1; break; }
    free(kept); free(L);
    kept = kept2; L = L2; --nk; ++removed;
  }
  if (!rc) {
    add_term(&S, L, 2 * nk, removed);
    rc = recursive_tor(&S, kept, nk, L, removed, d);
  }
  free(kept); free(L);
  *tor = S.tor; *abs = S.abs;
  return rc;
}

static void* alg2_worker(void* arg) {
  alg2_pool* P = (alg2_pool*)arg;
  for (;;) {
    pthread_mutex_lock(P->lock);
    uint64_t u = P->next++;
    pthread_mutex_unlock(P->lock);
    if (u >= P->ntasks) break;
    P->rc[u] = alg2_task(P->S0, P->d, P->L0, u, &P->tor[u], &P->abs[u]);
  }
  return 0;
}

/* Algorithm 2 of the paper in binary128, split into the 2^split tasks above and
 * run on nthreads threads.  Each task sums its addends with Neumaier
 * compensation; the task sums are then added in task order, so the value
 * depends on split but not on nthreads.  split = 0 is the plain recursion from
 * the root.  out[0..1] = Tor (dd), out[2] = sum |term|.  Returns 0, -1 (args)
 * or -2 (not PD). */
int tor_oracle_recursive_split(int n, const double* O, int ld, int layout, int split, int nthreads, double* out) {
  if (n < 0 || n > 40 || (n > 0 && !O) || !out || ld < 2 * n || split < 0 || split > n || split > 20 ||
      nthreads < 1)
    return -1;
  problem P = {n, layout, ld, 0, O};
  rec_state S;
  S.n = n; S.N = 2 * n; S.mutate = 0;
  S.tor.s = S.tor.c = 0; S.abs.s = S.abs.c = 0;
  int N = 2 * n;
  S.A = (cq*)calloc((size_t)(N > 0 ? N * N : 1), sizeof(cq));
  /* pairs order (a_1, a_1^dag, a_2, ...): Sec. 2 */
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      cq o = O_at(&P, row_of(&P, a / 2, a & 1), row_of(&P, b / 2, b & 1));
      cq v = {-o.re, -o.im};
      if (a == b) v.re += 1;
      S.A[a * N + b] = v;
    }
  cq* L = (cq*)calloc((size_t)(N > 0 ? N * N : 1), sizeof(cq));
  int rc = chol_rows(S.A, L, N, 0);   /* Algorithm 1 on I - A */
  if (rc) { free(S.A); free(L); return -2; }
  uint64_t ntasks = 1ull << split;
  neumaier* tt = (neumaier*)calloc((size_t)ntasks, sizeof(neumaier));
  neumaier* ta = (neumaier*)calloc((size_t)ntasks, sizeof(neumaier));
  int* trc = (int*)calloc((size_t)ntasks, sizeof(int));
  pthread_mutex_t lock = PTHREAD_MUTEX_INITIALIZER;
  alg2_pool pool = {&S, split, L, 0, ntasks, &lock, tt, ta, trc};
  if (nthreads > 256) nthreads = 256;
  if ((uint64_t)nthreads > ntasks) nthreads = (int)ntasks;
  if (nthreads == 1) {
    alg2_worker(&pool);
  } else {
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], 0, alg2_worker, &pool);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], 0);
  }
  neumaier acc = {0, 0}, abs_acc = {0, 0};
  for (uint64_t u = 0; u < ntasks; ++u) {
    if (trc[u]) rc = -2;
    nm_add(&acc, tt[u].s); nm_add(&acc, tt[u].c);
    nm_add(&abs_acc, ta[u].s); nm_add(&abs_acc, ta[u].c);
  }
  free(tt); free(ta); free(trc); free(L); free(S.A);
  if (rc) return -2;
  quad_to_dd(acc.s + acc.c, &out[0], &out[1]);
  out[2] = (double)(abs_acc.s + abs_acc.c);
  return 0;
}

/* The plain recursion from the root on one thread (split 0). */
int tor_oracle_recursive(int n, const double* O, int ld, int layout, double* out) {
  return tor_oracle_recursive_split(n, O, ld, layout, 0, 1, out);
}

/* Quad determinant of I - O_Z for one mask (for tests of the determinant step). */
int tor_oracle_det(int n, const double* O, int ld, int layout, uint64_t mask, double* out) {
  if (n < 0 || n > 40 || (n > 0 && !O) || !out) return -1;
  problem P = {n, layout, ld, 0, O};
  int mm = 2 * n;
  cq* W = (cq*)malloc(sizeof(cq) * (size_t)(mm > 0 ? mm * mm : 1));
  int* idx = (int*)malloc(sizeof(int) * (size_t)(3 * n + 2));
  cq d = det_IminusOZ(&P, mask, W, idx);
  out[0] = (double)d.re; out[1] = (double)d.im;
  free(W); free(idx);
  return 0;
}

int tor_oracle_quad_bits(void) {
  /* 113 for IEEE binary128 */
  quad one = 1, eps = 1; int b = 0;
  while ((quad)(one + eps) != one && b < 200) { eps /= 2; ++b; }
  return b;
}
