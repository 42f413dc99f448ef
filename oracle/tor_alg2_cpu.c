/*
 * tor_alg2_cpu.c -- CPU BASELINE; TEST AND BENCHMARK INFRASTRUCTURE ONLY.
 * Not the oracle (that is tor_oracle.c, in binary128) and not the product: only
 * the test suite and the benchmark's CPU-baseline leg load this library.
 *
 * The paper's recursive Torontonian (Sec. 2, Algorithm 2, with the Cholesky
 * factor of Algorithm 1 and the reuse of the factor blocks of Fig. 2) in FP64
 * complex arithmetic, multithreaded over subtrees.  It stands in for the
 * paper's own CPU implementation (TBB tasks, Sec. 4) when the GPU's throughput
 * is quoted against a CPU running the same method.
 *
 * Remove direction, as in Algorithm 2: a node is the set K of kept modes with
 * the Cholesky factor L of (I - O) restricted to K (pairs order, rows 2t and
 * 2t+1 for the t-th kept mode).  Its children remove one kept mode i >= start;
 * removed indices strictly increase, so every subset is visited once.  A child
 * keeps the factor rows and columns before mode i and recomputes the trailing
 * rows (Algorithm 1 from row 2q on).  Every node adds
 *     (-1)^{#removed} / sqrt(det(I - O_K)) = (-1)^{#removed} / prod_a L_aa.
 *
 * Parallel split: a node whose largest removed mode is r has 2^(n-1-r) nodes
 * below and including it.  Nodes with more than 2^n / (32 threads) are split
 * (the caller's thread adds their own terms), the others are the tasks,
 * ordered largest subtree first; threads take them from an atomic counter and
 * rebuild each task's factor from the root along its removals.  Sums: Neumaier in FP64,
 * per task in visiting order, then over tasks in task order, so the result does
 * not depend on the thread count or the schedule.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double re, im;
} cd;

typedef struct {
  double s, c;
} nsum; /* Neumaier sum */

static void ns_add(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

typedef struct {
  int n, N;
  cd* A;            /* I - O, pairs order, full N x N */
  int ntasks;       /* tasks to evaluate (a prefix of the ordered list) */
  const int* pool;  /* removed modes of the task nodes, ascending, back to back */
  const int* task_off, *task_len;  /* task t: pool[task_off[t] .. task_off[t] + task_len[t]) */
  nsum* task_tor;   /* per task */
  nsum* task_abs;
  int* task_rc;
  int next;         /* atomic task counter */
} alg2;

/* Factor rows r0..m-1 of the m x m matrix of the kept modes (row-major L),
 * rows and columns below r0 already in place.  0, or -1 if not positive definite. */
static int chol_from(const alg2* S, const int* kept, int m, cd* L, int r0) {
  for (int i = r0; i < m; ++i) {
    const int ri = 2 * kept[i >> 1] + (i & 1);
    for (int j = r0; j < i; ++j) {
      const int rj = 2 * kept[j >> 1] + (j & 1);
      cd s = S->A[ri * S->N + rj];
      for (int k = 0; k < j; ++k) { /* s -= L_ik conj(L_jk) */
        const cd a = L[i * m + k], b = L[j * m + k];
        s.re -= a.re * b.re + a.im * b.im;
        s.im -= a.im * b.re - a.re * b.im;
      }
      const double djj = L[j * m + j].re;
      L[i * m + j].re = s.re / djj;
      L[i * m + j].im = s.im / djj;
    }
    double d = S->A[ri * S->N + ri].re;
    for (int k = 0; k < i; ++k) d -= L[i * m + k].re * L[i * m + k].re + L[i * m + k].im * L[i * m + k].im;
    if (!(d > 0)) return -1;
    L[i * m + i].re = sqrt(d);
    L[i * m + i].im = 0.0;
  }
  return 0;
}

/* Child of (kept, nk, L): remove kept position q.  Writes kept2 and L2. */
static int child(const alg2* S, const int* kept, int nk, const cd* L, int q, int* kept2, cd* L2) {
  const int m = 2 * nk, m2 = m - 2, r0 = 2 * q;
  for (int t = 0, u = 0; t < nk; ++t)
    if (t != q) kept2[u++] = kept[t];
  for (int a = 0; a < m2; ++a) {
    const int pa = a < r0 ? a : a + 2; /* the row in the parent factor */
    const int lim = a < r0 ? a + 1 : r0;
    for (int b = 0; b < lim; ++b) L2[a * m2 + b] = L[pa * m + b];
  }
  return chol_from(S, kept2, m2, L2, r0);
}

static double inv_sqrt_det(const cd* L, int m) {
  double p = 1.0;
  for (int a = 0; a < m; ++a) p *= L[a * m + a].re;
  return 1.0 / p;
}

/* All nodes below (kept, nk, L) with removals from mode `start` on (the node's own term not included). */
static int subtree(const alg2* S, const int* kept, int nk, const cd* L, int removed, int start, int* kbuf, cd* lbuf,
                   nsum* tor, nsum* ab) {
  const int n = S->n, N = S->N;
  int* kept2 = kbuf;
  cd* L2 = lbuf;
  for (int q = 0; q < nk; ++q) {
    if (kept[q] < start) continue;
    int rc = child(S, kept, nk, L, q, kept2, L2);
    if (rc) return rc;
    const double t = inv_sqrt_det(L2, 2 * (nk - 1));
    ns_add(tor, ((removed + 1) & 1) ? -t : t);
    ns_add(ab, t);
    rc = subtree(S, kept2, nk - 1, L2, removed + 1, kept[q] + 1, kbuf + n, lbuf + (size_t)N * N, tor, ab);
    if (rc) return rc;
  }
  return 0;
}

/* Factor of the node with removed modes rm[0..d) (ascending), built from the root. */
static int node_factor(const alg2* S, const int* rm, int d, int* kept, cd* L, int* kt, cd* Lt) {
  const int n = S->n, N = S->N;
  for (int j = 0; j < n; ++j) kept[j] = j;
  memset(L, 0, sizeof(cd) * (size_t)N * N);
  if (chol_from(S, kept, N, L, 0)) return -1;
  int nk = n;
  for (int e = 0; e < d; ++e) {
    int q = 0;
    while (kept[q] != rm[e]) ++q;
    if (child(S, kept, nk, L, q, kt, Lt)) return -1;
    --nk;
    memcpy(kept, kt, sizeof(int) * (size_t)nk);
    memcpy(L, Lt, sizeof(cd) * (size_t)(2 * nk) * (2 * nk));
  }
  return 0;
}

static void* worker(void* arg) {
  alg2* S = (alg2*)arg;
  const int n = S->n, N = S->N;
  int* kept = (int*)malloc(sizeof(int) * (size_t)n * (n + 3));
  cd* L = (cd*)calloc((size_t)N * N * (n + 3), sizeof(cd));
  if (!kept || !L) {
    free(kept);
    free(L);
    return (void*)1;
  }
  for (;;) {
    const int t = __atomic_fetch_add(&S->next, 1, __ATOMIC_RELAXED);
    if (t >= S->ntasks) break;
    const int* rm = S->pool + S->task_off[t];
    const int d = S->task_len[t];
    nsum tor = {0, 0}, ab = {0, 0};
    int rc = node_factor(S, rm, d, kept, L, kept + n, L + (size_t)N * N);
    const int nk = n - d;
    if (!rc) {
      const double v = inv_sqrt_det(L, 2 * nk);
      ns_add(&tor, (d & 1) ? -v : v);
      ns_add(&ab, v);
      rc = subtree(S, kept, nk, L, d, rm[d - 1] + 1, kept + 2 * n, L + (size_t)2 * N * N, &tor, &ab);
    }
    S->task_tor[t] = tor;
    S->task_abs[t] = ab;
    S->task_rc[t] = rc;
  }
  free(kept);
  free(L);
  return 0;
}

/* Growable list of removed-mode sets. */
typedef struct {
  int *pool, *off, *len;
  long long used, cap;
  int cnt, capn;
} setlist;

static int sl_push(setlist* L, const int* R, int d) {
  if (L->used + d > L->cap) {
    long long c = L->cap ? 2 * L->cap : 1024;
    while (c < L->used + d) c *= 2;
    int* p = (int*)realloc(L->pool, sizeof(int) * (size_t)c);
    if (!p) return -1;
    L->pool = p;
    L->cap = c;
  }
  if (L->cnt == L->capn) {
    int c = L->capn ? 2 * L->capn : 256;
    int* o = (int*)realloc(L->off, sizeof(int) * (size_t)c);
    if (!o) return -1;
    L->off = o;
    int* l = (int*)realloc(L->len, sizeof(int) * (size_t)c);
    if (!l) return -1;
    L->len = l;
    L->capn = c;
  }
  L->off[L->cnt] = (int)L->used;
  L->len[L->cnt] = d;
  memcpy(L->pool + L->used, R, sizeof(int) * (size_t)d);
  L->used += d;
  ++L->cnt;
  return 0;
}

static void sl_free(setlist* L) {
  free(L->pool);
  free(L->off);
  free(L->len);
}

/* Node R (d removed modes, ascending): a task if its subtree has at most T
 * nodes, else split (R goes to `top`, its children are visited in order). */
static int gen(int n, double T, int* R, int d, setlist* top, setlist* tasks) {
  const double size = d == 0 ? ldexp(1.0, n) : ldexp(1.0, n - 1 - R[d - 1]);
  if (d > 0 && size <= T) return sl_push(tasks, R, d);
  if (sl_push(top, R, d)) return -1;
  for (int i = d ? R[d - 1] + 1 : 0; i < n; ++i) {
    R[d] = i;
    if (gen(n, T, R, d + 1, top, tasks)) return -1;
  }
  return 0;
}

/*
 * Tor of the 2n x 2n matrix O (complex128 interleaved, row stride ld complex
 * entries; layout 0: mode j owns rows {j, j+n}; 1: rows {2j, 2j+1}).
 * threads >= 1.  max_tasks < 0: every node (the full sum); otherwise only the
 * split nodes and the first max_tasks tasks (largest first), a bounded sample
 * for timing.  out[0] = the (partial) Tor, out[1] = its sum of |term|,
 * out[2] = the number of terms evaluated.  Returns 0, -1 (arguments, memory)
 * or -2 (not positive definite).
 */
int tor_alg2_fp64(int n, const double* O, int ld, int layout, int threads, long long max_tasks, double* out) {
  if (n < 1 || n > 60 || !O || !out || ld < 2 * n || threads < 1) return -1;
  alg2 S;
  memset(&S, 0, sizeof S);
  S.n = n;
  S.N = 2 * n;
  const int N = S.N;
  S.A = (cd*)malloc(sizeof(cd) * (size_t)N * N);
  if (!S.A) return -1;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const int ja = a >> 1, ca = a & 1, jb = b >> 1, cb = b & 1;
      const int ra = layout ? 2 * ja + ca : ja + ca * n, rb = layout ? 2 * jb + cb : jb + cb * n;
      const double* o = O + 2 * ((size_t)ra * ld + rb);
      S.A[a * N + b].re = (a == b ? 1.0 : 0.0) - o[0];
      S.A[a * N + b].im = -o[1];
    }
  setlist top, gtasks;
  memset(&top, 0, sizeof top);
  memset(&gtasks, 0, sizeof gtasks);
  int R[64];
  double T = ldexp(1.0, n) / (32.0 * threads);
  if (T < 1.0) T = 1.0;
  int rc = gen(n, T, R, 0, &top, &gtasks) ? -1 : 0;
  /* tasks ordered largest subtree first (largest removed mode ascending), in generation order within a size */
  const int total = gtasks.cnt;
  int* off = (int*)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
  int* len = (int*)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
  S.task_tor = (nsum*)calloc((size_t)(total > 0 ? total : 1), sizeof(nsum));
  S.task_abs = (nsum*)calloc((size_t)(total > 0 ? total : 1), sizeof(nsum));
  S.task_rc = (int*)calloc((size_t)(total > 0 ? total : 1), sizeof(int));
  int* kept = (int*)malloc(sizeof(int) * (size_t)n * 2);
  cd* L = (cd*)calloc((size_t)N * N * 2, sizeof(cd));
  if (!off || !len || !S.task_tor || !S.task_abs || !S.task_rc || !kept || !L) rc = -1;
  if (!rc) {
    int k = 0;
    for (int r = 0; r < n; ++r)
      for (int t = 0; t < total; ++t)
        if (gtasks.pool[gtasks.off[t] + gtasks.len[t] - 1] == r) {
          off[k] = gtasks.off[t];
          len[k] = gtasks.len[t];
          ++k;
        }
    S.pool = gtasks.pool;
    S.task_off = off;
    S.task_len = len;
    S.ntasks = max_tasks < 0 || max_tasks > total ? total : (int)max_tasks;
  }
  nsum tor = {0, 0}, ab = {0, 0};
  double terms = 0;
  /* the split nodes' own terms, in generation order */
  for (int s = 0; !rc && s < top.cnt; ++s) {
    const int d = top.len[s];
    if (node_factor(&S, top.pool + top.off[s], d, kept, L, kept + n, L + (size_t)N * N)) {
      rc = -2;
      break;
    }
    const double v = inv_sqrt_det(L, 2 * (n - d));
    ns_add(&tor, (d & 1) ? -v : v);
    ns_add(&ab, v);
    terms += 1;
  }
  if (!rc) {
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    int started = 0;
    if (!th) rc = -1;
    for (int t = 0; !rc && t < threads; ++t)
      if (pthread_create(&th[t], NULL, worker, &S) == 0) ++started;
    if (!rc && started == 0 && worker(&S)) rc = -1;
    for (int t = 0; t < started; ++t) {
      void* r = 0;
      pthread_join(th[t], &r);
      if (r) rc = -1;
    }
    free(th);
    for (int t = 0; !rc && t < S.ntasks; ++t) {
      if (S.task_rc[t]) {
        rc = -2;
        break;
      }
      ns_add(&tor, S.task_tor[t].s);
      ns_add(&tor, S.task_tor[t].c);
      ns_add(&ab, S.task_abs[t].s);
      ns_add(&ab, S.task_abs[t].c);
      terms += ldexp(1.0, n - 1 - S.pool[S.task_off[t] + S.task_len[t] - 1]);
    }
  }
  if (!rc) {
    out[0] = tor.s + tor.c;
    out[1] = ab.s + ab.c;
    out[2] = terms;
  }
  free(kept);
  free(L);
  free(off);
  free(len);
  free(S.task_tor);
  free(S.task_abs);
  free(S.task_rc);
  sl_free(&top);
  sl_free(&gtasks);
  free(S.A);
  return rc;
}
