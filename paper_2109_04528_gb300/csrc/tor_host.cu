// tor_host.cu -- host runtime and C ABI of libtor (declared in include/tor.h).
//
// A job is a list of matrices evaluated by one pass of the GPU pipeline
//   H2D (inputs, descriptors) -> k_intake -> k_units (persistent) -> k_reduce -> D2H
// on one "slot": a stream plus its own device and pinned buffers.  The
// blocking calls (tor_eval, tor_eval_batch, ...) use the context's main slot.
// tor_submit / tor_submit_marginal feed a serving thread that keeps several
// slots in flight on separate streams: requests that arrive while jobs run are
// admitted into the next free slot as soon as the device-memory budget allows,
// so a new job starts on SMs that the previous job's tail leaves idle.
// With TOR_GRAPHS a slot captures its whole pass into a CUDA graph and
// replays it for every later job of the same shape.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tor.h"
#include "tor_internal.h"

using namespace tor;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  std::atomic<long long>* acct = nullptr;  // the context's count of device bytes held, or null
  bool exact = false;                      // allocate exactly what is asked (under a memory budget)
  cudaStream_t astream = nullptr;          // stream-ordered allocation on this stream (serving slots)
  // grows (never shrinks); bumps *gen when the address changes
  cudaError_t ensure(size_t bytes, uint64_t* gen) {
    if (bytes <= cap && p) return cudaSuccess;
    bytes = std::max<size_t>(bytes, 256);
    size_t want = exact ? bytes : std::max(bytes, cap + cap / 2);
    release();
    ++*gen;
    cudaError_t e = alloc(want);
    if (e != cudaSuccess && want > bytes) {
      cudaGetLastError();
      want = bytes;
      e = alloc(want);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return e;
    }
    cap = want;
    if (acct) *acct += (long long)cap;
    return cudaSuccess;
  }
  cudaError_t alloc(size_t bytes) {
    // a serving slot allocates in its own stream's order: unlike cudaMalloc /
    // cudaFree this does not wait for the kernels of the other slots
    return astream ? cudaMallocAsync(&p, bytes, astream) : cudaMalloc(&p, bytes);
  }
  void release() {
    if (p) {
      if (astream) cudaFreeAsync(p, astream);
      else cudaFree(p);
      if (acct) *acct -= (long long)cap;
    }
    p = nullptr;
    cap = 0;
  }
};

struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes, uint64_t* gen) {
    if (bytes <= cap && p) return cudaSuccess;
    bytes = std::max<size_t>(bytes, 256);
    size_t want = std::max(bytes, cap + cap / 2);
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    ++*gen;
    cudaError_t e = cudaMallocHost(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
  }
};

inline int tri(int n) { return n * (2 * n + 1); }
inline double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// One matrix of a job, as the caller described it.
struct MatIn {
  int n = 0;                    // modes of the matrix to evaluate
  const tor_c128* O = nullptr;  // source matrix (host, or device if dev)
  int ld = 0;                   // leading dimension of O (complex elements)
  int n_src = 0;                // modes of the source matrix
  int layout = TOR_LAYOUT_BLOCK;
  bool dev = false;             // O is a device pointer
  const int* modes = nullptr;   // host list of n source modes (session marginals), or null
  long long leaf_lo = 0;        // tor_eval_range: first reduction leaf (warp task) to evaluate
  long long leaf_count = -1;    // tor_eval_range: number of leaves; -1 = all
  bool bad_range = false;       // the caller asked for an empty range (TOR_EINVAL)
  int real_hint = -1;           // 1/0: structured or not, already known (sessions); -1 = detect
};

struct Slot {
  Slot() = default;
  Slot(const Slot&) = delete;
  Slot& operator=(const Slot&) = delete;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevBuf d_O, d_B, d_front, d_partials, d_flags, d_results, d_lane, d_warp, d_modes;
  HostBuf h_O, h_front, h_results, h_ctl, h_modes;
  // d_front holds the control words (64 bytes, zero at the start of a pass), the
  // matrix descriptors and the task list, uploaded from h_front in one copy
  void *p_ctl = nullptr, *p_mats = nullptr, *p_tasks = nullptr;
  size_t off_mats = 0, off_tasks = 0, front_bytes = 0;
  cudaEvent_t ev[5] = {};
  cudaEvent_t done = nullptr;
  uint64_t gen = 0;
  struct Graph {
    uint64_t key, gen;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  // the prepared job
  std::vector<int> act;  // index into the caller's list, job order
  std::vector<MatDesc> mats;
  std::vector<TaskDesc> tasks;
  std::vector<long long> task_shape;  // the job shape `tasks` was built for
  uint64_t tasks_staged_gen = ~0ull;  // buffer generation when `tasks` was copied into h_front
  int J = 0;
  long long o_elems = 0, b_elems = 0, parts = 0, reds = 0, red_chunks = 0, mode_elems = 0, lane_e = 0, warp_e = 0;
  bool want_parts = false;
  size_t bytes = 0;
  int cancel_epoch = 0;
  bool busy = false;
  bool graphed = false;  // the last pass was a graph replay
  // scratch-slot pool of non-persistent k_units launches (one bit per resident block)
  unsigned* d_pool = nullptr;
  int pool_words = 0;
  // serving state
  cudaEvent_t units_done = nullptr;  // end of a time slice of k_units
  int phase = 0;                     // 0 idle, 1 k_units slice in flight, 2 reduce and copies in flight
  bool large = false;                // a large lane: one large request at a time, low priority
  double t_start = 0;

  static constexpr int kBufs = 9;
  DevBuf* bufs[kBufs] = {&d_O, &d_B, &d_front, &d_partials, &d_flags, &d_results, &d_lane, &d_warp, &d_modes};
  size_t dev_bytes() const {
    size_t t = 0;
    for (const DevBuf* b : bufs) t += b->cap;
    return t;
  }
  void release_dev() {
    for (DevBuf* b : bufs) b->release();
  }
  void release() {
    for (DevBuf* b : bufs) b->release();
    for (HostBuf* b : {&h_O, &h_front, &h_results, &h_ctl, &h_modes}) b->release();
    if (d_pool) cudaFree(d_pool);
    d_pool = nullptr;
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
    for (int i = 0; i < 5; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    if (done) cudaEventDestroy(done);
    if (units_done) cudaEventDestroy(units_done);
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

}  // namespace

struct tor_session {
  tor_ctx* ctx = nullptr;  // null once the context has been destroyed
  int device = 0;
  int real = 0;            // Sigma is structured: every O^(j) takes the real (x, p) path
  int N = 0;
  int inflight = 0;        // requests taken by the serving loop and not completed (guarded by ctx->q_mu)
  int blocking = 0;        // tor_eval_marginal calls in progress (guarded by ctx->q_mu)
  bool closing = false;
  DevBuf d_O;                  // O^(j) for j = 1..N, pairs layout, 2j x 2j row-major each
  std::vector<long long> off;  // element offset of O^(j)
  std::vector<long double> logdet_sigma;  // log det Sigma_[j], j = 0..N (0 for j = 0)
  uint64_t gen = 0;
};

struct Request {
  uint64_t ticket = 0;
  tor_session* sess = nullptr;  // the session a marginal request reads, or null
  MatIn in;
  std::vector<tor_c128> O;  // owned copy of a host matrix
  std::vector<int> modes;   // owned copy of a marginal's mode list
  tor_result res{};
  bool done = false;
};

struct tor_ctx {
  tor_config cfg{};
  int sms = 0, blocks_per_sm = 0, grid = 0, nwarps = 0;
  int plan[65];
  Slot main;
  int* h_cancel = nullptr;  // host-mapped cancel counter
  int* d_cancel = nullptr;
  double last_times[4] = {0, 0, 0, 0};
  std::string last_error;
  std::mutex run_mu;  // serialises use of the main slot and the plan table
  // serving
  std::mutex q_mu;
  std::condition_variable q_cv, done_cv;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  std::thread server;
  bool server_started = false, stopping = false;
  // bumped (under q_mu) by every enqueue and by tor_destroy: an idle serving
  // thread that spins instead of sleeping watches it without taking the lock
  std::atomic<unsigned long long> q_events{0};
  double idle_spin_s = 0.05;  // idle serving thread spins this long before it sleeps (TOR_SERVE_IDLE_SPIN_MS)
  size_t queue_limit = 1 << 20;
  int n_serve_slots = 4;   // large lanes first, then small lanes
  int n_large_slots = 2;   // two large requests in flight: the next one's blocks fill the tail of the current one
  long long large_slice_ns = 0;  // > 0: large jobs yield the SMs every slice (TOR_SERVE_SLICE_MS); 0 = run through
  int max_batch = 4096;
  double max_batch_terms = 268435456.0;  // ~45 ms of GPU work per served batch (2^28 subset terms)
  std::vector<std::unique_ptr<Slot>> serve;
  std::atomic<long long> served{0}, batches{0};
  std::vector<tor_session*> sessions;  // live sessions of this context (guarded by q_mu)
  // device bytes held by the slots' buffers and the sessions' matrices: what
  // tor_config.mem_budget caps
  std::atomic<long long> dev_held{0};
};

// Bytes of one matrix entry the kernels may use: complex128, or a complex
// double-double in extended precision (TOR_EXTENDED); and of one lane-scratch
// element (a real and a complex area side by side).
static size_t entry_bytes(const tor_ctx* ctx) {
  return (ctx->cfg.flags & TOR_EXTENDED) ? kWarpEntryBytesExt : kWarpEntryBytes;
}
static size_t lane_entry_bytes(const tor_ctx* ctx) {
  return (ctx->cfg.flags & TOR_EXTENDED) ? kLaneEntryBytesExt : kLaneEntryBytes;
}

// Last error of a call that had no context to record it in (tor_create).
static thread_local std::string g_create_error;

static tor_status cuda_fail(tor_ctx* ctx, cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  if (ctx) ctx->last_error = buf;
  g_create_error = buf;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TOR_ENOMEM : TOR_ECUDA;
}

#define CK(call, what)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

// Built-in plan, the shape the autotuner finds on GB300 (2432 resident warps
// of k_units, 1216 of k_units_ext), scaled by lw = floor(log2(resident warps)):
//   small n: units over M = 4 modes (as much parallelism as the tree offers);
//   then p = lw + 5, about one wave of 2^lw warp tasks;
//   from n = lw + 16 on, p = lw + 8, about eight waves (room for the tail);
//   units of at most kMaxPlanM modes (2^20 subsets, already far more work per
//   unit than its root build), so the lane stacks, which grow as M^3, stay
//   bounded for n > 40 as well.
constexpr int kMaxPlanM = 20;
static int default_prefix_depth(int n, int nwarps) {
  int lw = 0;
  while ((2ll << lw) <= std::max(nwarps, 1)) ++lw;
  int p;
  if (n <= lw + 9) p = n - 4;
  else if (n <= lw + 13) p = lw + 5;
  else if (n <= lw + 15) p = lw + 6;
  else if (n <= lw + 20) p = lw + 8;
  else p = lw + 9;
  p = std::max(p, n - kMaxPlanM);
  return std::max(0, std::min(p, n - 1));
}

// Largest prefix depth: 2^30 unit partials (32 GB) and 2^25 warp tasks.
constexpr int kMaxPrefixDepth = 30;

static int plan_p(tor_ctx* ctx, int n) {
  int p;
  if (ctx->plan[n] >= 0) p = ctx->plan[n];
  else if (ctx->cfg.prefix_depth >= 0) p = ctx->cfg.prefix_depth;
  else p = default_prefix_depth(n, ctx->nwarps);
  return std::max(0, std::min(std::min(p, n - 1), kMaxPrefixDepth));
}

// priority: 0 = default; < 0 = the device's highest; > 0 = its lowest
static cudaError_t slot_init(Slot& s, cudaStream_t stream, int priority = 0) {
  cudaError_t e;
  if (stream) {
    s.stream = stream;
    s.own_stream = false;
  } else {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);  // numerically lower = higher priority
    const int prio = priority < 0 ? hi : priority > 0 ? lo : 0;
    if ((e = cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio)) != cudaSuccess) return e;
    s.own_stream = true;
  }
  for (int i = 0; i < 5; ++i)
    if ((e = cudaEventCreate(&s.ev[i])) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&s.units_done, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
}

// A slot's device buffers count toward the context's held bytes; under a
// memory budget they are allocated exactly; serving slots allocate in their
// own stream's order.
static void slot_account(tor_ctx* ctx, Slot& S, bool stream_ordered) {
  for (DevBuf* b : S.bufs) {
    b->acct = &ctx->dev_held;
    b->exact = ctx->cfg.mem_budget != 0;
    b->astream = stream_ordered ? S.stream : nullptr;
  }
}

// A shard of a matrix with prefix depth p: leaf_count a power of two, leaf_lo a
// multiple of it, inside the 2^(p-5) reduction leaves, and p >= 5.
static bool range_ok(int p, long long leaf_lo, long long leaf_count) {
  if (p < 5 || leaf_count < 1 || (leaf_count & (leaf_count - 1)) || leaf_lo < 0 || leaf_lo % leaf_count) return false;
  return leaf_lo + leaf_count <= (1ll << (p - 5));
}

// Device bytes of each of a slot's buffers (in Slot::bufs order) that a job of
// these matrices needs: the sizes slot_prepare allocates.
struct Needs {
  size_t b[Slot::kBufs] = {};
  size_t total() const {
    size_t t = 0;
    for (size_t v : b) t += v;
    return t;
  }
};

static Needs job_needs(tor_ctx* ctx, const std::vector<MatIn>& ins, size_t count) {
  long long o = 0, bt = 0, parts = 0, reds = 0, md = 0, lane_e = 0, warp_e = 0, ntask = 0;
  long long small_units[65] = {};  // n -> units of the matrices with p < 5 (one lane each)
  long long J = 0;
  for (size_t i = 0; i < count; ++i) {
    const MatIn& m = ins[i];
    if (m.n < 1 || m.n > 64 || m.bad_range) continue;
    const int p = plan_p(ctx, m.n);
    if (m.leaf_count > 0 && !range_ok(p, m.leaf_lo, m.leaf_count)) continue;
    ++J;
    if (!m.dev && !m.modes) o += 4ll * m.n * m.n;
    if (m.modes) md += m.n;
    bt += tri(m.n);
    parts += 1ll << p;
    if (m.leaf_count > 0) {
      long long r = 1;
      while (r < m.leaf_count) r <<= 1;
      reds += r;
    } else {
      reds += 1ll << (p >= 5 ? p - 5 : p);
    }
    if (p >= 5) ntask += m.leaf_count > 0 ? m.leaf_count : (1ll << (p - 5));
    else small_units[m.n] += 1ll << p;
    lane_e = std::max(lane_e, lane_elems_for(m.n, p));
    warp_e = std::max(warp_e, warp_elems_for(m.n, p));
  }
  for (long long u : small_units) ntask += (u + 31) / 32;
  const size_t eb = entry_bytes(ctx);
  const size_t off_tasks = (256 + (size_t)J * sizeof(MatDesc) + 255) / 256 * 256;
  Needs N;
  N.b[0] = (size_t)o * 16;                                                  // d_O
  N.b[1] = (size_t)bt * eb;                                                 // d_B
  N.b[2] = off_tasks + (size_t)ntask * sizeof(TaskDesc);                    // d_front
  N.b[3] = (size_t)(parts + reds) * 32;                                     // d_partials
  N.b[4] = (size_t)J * sizeof(int);                                         // d_flags
  N.b[5] = (size_t)J * sizeof(ResultRec);                                   // d_results
  N.b[6] = (size_t)ctx->nwarps * 32 * (size_t)lane_e * lane_entry_bytes(ctx);  // d_lane
  N.b[7] = (size_t)ctx->nwarps * (size_t)warp_e * eb;                       // d_warp
  N.b[8] = (size_t)md * sizeof(int);                                        // d_modes
  for (size_t& v : N.b) v = std::max<size_t>(v, 256);  // DevBuf's smallest allocation
  return N;
}

// Bytes slot S would add to what the context holds to run a job with these
// needs: each buffer too small is replaced by one of exactly the needed size
// (the slots of a budgeted context allocate exactly).
static size_t slot_growth(const Slot& S, const Needs& N) {
  size_t g = 0;
  for (int i = 0; i < Slot::kBufs; ++i)
    if (N.b[i] > S.bufs[i]->cap || !S.bufs[i]->p) g += N.b[i] - std::min(N.b[i], S.bufs[i]->cap);
  return g;
}

static bool over_budget(tor_ctx* ctx, const Slot& S, const Needs& N) {
  if (!ctx->cfg.mem_budget) return false;
  const long long held = ctx->dev_held.load();
  return (size_t)std::max(0ll, held) + slot_growth(S, N) > ctx->cfg.mem_budget;
}

// Copies host matrices into the pinned staging buffer: one copy per matrix when
// its rows are contiguous, row by row otherwise; a job staging more than 32 MB
// is split over up to 8 threads by matrix (memory bandwidth, not the copy
// loop, then limits it).
template <class Copy>
static void stage_host_matrices(const std::vector<Copy>& copies, size_t bytes) {
  auto run = [&](size_t a, size_t b) {
    for (size_t i = a; i < b; ++i) {
      const Copy& c = copies[i];
      if (c.ld == c.m) {
        memcpy(c.dst, c.src, sizeof(tor_c128) * (size_t)c.m * c.m);
      } else {
        for (int r = 0; r < c.m; ++r)
          memcpy(c.dst + (size_t)r * c.m, c.src + (size_t)r * c.ld, sizeof(tor_c128) * c.m);
      }
    }
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t T = bytes >= ((size_t)32 << 20) ? std::min<size_t>({8, hw, copies.size()}) : 1;
  if (T <= 1) {
    run(0, copies.size());
    return;
  }
  std::vector<std::thread> th;
  const size_t per = (copies.size() + T - 1) / T;
  for (size_t t = 1; t < T; ++t) {
    const size_t a = std::min(copies.size(), t * per), b = std::min(copies.size(), a + per);
    if (a < b) th.emplace_back(run, a, b);
  }
  run(0, std::min(copies.size(), per));
  for (std::thread& x : th) x.join();
}

// Validates the inputs, fills trivial results, plans the job and fills the
// slot's pinned staging buffers.  Returns the first error; *any = job has work.
static tor_status slot_prepare(tor_ctx* ctx, Slot& S, const std::vector<MatIn>& ins, tor_result* out,
                               bool want_parts, bool* any) {
  *any = false;
  tor_status first = TOR_OK;
  auto note = [&](tor_status s) {
    if (first == TOR_OK && s != TOR_OK) first = s;
  };
  const int count = (int)ins.size();
  S.act.clear();
  S.J = 0;
  for (int i = 0; i < count; ++i) {
    const MatIn& m = ins[i];
    tor_result& r = out[i];
    memset(&r, 0, sizeof r);
    r.n = m.n;
    if (m.n < 0) r.status = TOR_EINVAL;
    else if (m.n > 64) r.status = TOR_ETOOBIG;
    else if (m.n == 0) {
      r.hi = 1.0;
      r.abs_sum = 1.0;
      r.status = TOR_OK;
    } else if (!m.O || (!m.modes && m.ld < 2 * m.n) || (m.modes && m.ld < 2 * m.n_src)) r.status = TOR_EINVAL;
    else if (m.bad_range || (m.leaf_count > 0 && !range_ok(plan_p(ctx, m.n), m.leaf_lo, m.leaf_count)))
      r.status = TOR_EINVAL;
    else {
      S.act.push_back(i);
      continue;
    }
    note(r.status);
  }
  if (S.act.empty()) return first;
  // job order: by n descending so equal sizes are adjacent (stable: same n keeps caller order)
  auto by_n = [&](int a, int b) { return ins[a].n > ins[b].n; };
  if (!std::is_sorted(S.act.begin(), S.act.end(), by_n)) std::stable_sort(S.act.begin(), S.act.end(), by_n);
  const int J = (int)S.act.size();
  S.mats.assign(J, MatDesc{});
  S.o_elems = S.b_elems = S.parts = S.reds = S.red_chunks = S.mode_elems = S.lane_e = S.warp_e = 0;
  for (int j = 0; j < J; ++j) {
    const MatIn& m = ins[S.act[j]];
    const int p = plan_p(ctx, m.n);
    MatDesc& D = S.mats[j];
    D.n = m.n;
    D.p = p;
    // the arithmetic: forced complex, known (sessions), or detected by k_intake
    D.real = (ctx->cfg.flags & TOR_COMPLEX_PATH) ? 0 : m.real_hint;
    D.ext = (ctx->cfg.flags & TOR_EXTENDED) ? 1 : 0;
    D.layout = m.layout;
    D.n_src = m.modes ? m.n_src : m.n;
    // unit u's partial at part_off + u.  A shard needs all 2^p places too: the 32
    // units of warp task t are t + l 2^(p-5), spread over the whole range of u.
    D.part_off = S.parts;
    S.parts += 1ll << p;
    D.red_log2 = p >= 5 ? p - 5 : p;
    D.red_lo = 0;
    if (m.leaf_count > 0) {  // a shard: leaves [leaf_lo, leaf_lo + leaf_count) only (p >= 5)
      int lg = 0;
      while ((1ll << lg) < m.leaf_count) ++lg;
      D.red_log2 = lg;
      D.red_lo = m.leaf_lo;
    }
    D.red_off = S.reds;
    S.reds += 1ll << D.red_log2;
    D.red_chunk0 = (int)S.red_chunks;
    S.red_chunks += red_chunks(D.red_log2);
    S.b_elems += tri(m.n);
    if (!m.dev && !m.modes) S.o_elems += 4ll * m.n * m.n;
    if (m.modes) S.mode_elems += m.n;
    S.lane_e = std::max(S.lane_e, lane_elems_for(m.n, p));
    S.warp_e = std::max(S.warp_e, warp_elems_for(m.n, p));
  }
  // warp tasks, largest subtrees first.  All tasks of one size group (equal n,
  // adjacent after the sort above) share M, so ordering the groups stably by M
  // and emitting their tasks in order is a stable sort of the tasks by M.
  // The list depends only on the job's shape (sizes, prefix depths and leaf
  // ranges in job order); a slot keeps the list of its last job and reuses it
  // when the shape repeats (a batch of thousands of matrices has millions of
  // tasks, whose ordering is host time with the GPU idle).
  std::vector<long long> shape;
  shape.reserve(3 * (size_t)J);
  for (int j = 0; j < J; ++j) {
    const MatIn& m = ins[S.act[j]];
    shape.push_back((long long)S.mats[j].n | (long long)S.mats[j].p << 8);
    shape.push_back(m.leaf_lo);
    shape.push_back(m.leaf_count);
  }
  const bool reuse_tasks = !S.tasks.empty() && shape == S.task_shape;
  struct Group {
    int j, k, M;
  };
  std::vector<Group> groups;
  long long ntasks = 0;
  for (int j = 0; j < J;) {
    int k = j;
    while (k < J && S.mats[k].n == S.mats[j].n) ++k;
    const int p = S.mats[j].p;
    groups.push_back({j, k, S.mats[j].n - p});
    for (int a = j; a < k && p >= 5; ++a) {
      const MatIn& m = ins[S.act[a]];
      ntasks += m.leaf_count > 0 ? m.leaf_count : (1ll << (p - 5));
    }
    if (p < 5) ntasks += ((((long long)(k - j)) << p) + 31) / 32;
    j = k;
  }
  std::stable_sort(groups.begin(), groups.end(), [](const Group& a, const Group& b) { return a.M > b.M; });
  if (!reuse_tasks) {
    S.tasks.clear();
    S.task_shape.swap(shape);
    S.tasks_staged_gen = ~0ull;
  }
  if (!reuse_tasks) S.tasks.reserve((size_t)ntasks);
  for (const Group& g : groups) {
    if (reuse_tasks) break;
    const int j = g.j, k = g.k, p = S.mats[j].p, M = g.M;
    if (p >= 5) {
      for (int a = j; a < k; ++a) {
        const MatIn& m = ins[S.act[a]];
        const long long t0 = m.leaf_count > 0 ? m.leaf_lo : 0;
        const long long t1 = m.leaf_count > 0 ? m.leaf_lo + m.leaf_count : (1ll << (p - 5));
        for (long long t = t0; t < t1; ++t) S.tasks.push_back({a, (int)t, 1, M});
      }
    } else {
      const long long units = (long long)(k - j) << p;
      for (long long t = 0; t * 32 < units; ++t) S.tasks.push_back({j, (int)t, k - j, M});
    }
  }
  S.want_parts = want_parts;
  // buffers
  const size_t eb = entry_bytes(ctx);
  const size_t lane_bytes = (size_t)ctx->nwarps * 32 * S.lane_e * lane_entry_bytes(ctx);
  const size_t warp_bytes = (size_t)ctx->nwarps * S.warp_e * eb;
  const Needs needs = job_needs(ctx, ins, ins.size());
  S.bytes = needs.total();
  if (over_budget(ctx, S, needs)) {
    for (int j = 0; j < J; ++j) out[S.act[j]].status = TOR_ENOMEM;
    S.act.clear();
    S.J = 0;
    return TOR_ENOMEM;
  }
  uint64_t* g = &S.gen;
  CK(S.d_O.ensure(S.o_elems * 16, g), "alloc O");
  CK(S.d_B.ensure(S.b_elems * eb, g), "alloc B");
  CK(S.d_partials.ensure((S.parts + S.reds) * 32, g), "alloc partials");
  S.off_mats = 256;
  S.off_tasks = (S.off_mats + J * sizeof(MatDesc) + 255) / 256 * 256;
  S.front_bytes = S.off_tasks + S.tasks.size() * sizeof(TaskDesc);
  CK(S.d_front.ensure(S.front_bytes, g), "alloc descriptors");
  CK(S.d_flags.ensure(J * sizeof(int), g), "alloc flags");
  CK(S.d_results.ensure(J * sizeof(ResultRec), g), "alloc results");
  CK(S.d_lane.ensure(lane_bytes, g), "alloc lane scratch");
  CK(S.d_warp.ensure(warp_bytes, g), "alloc warp scratch");
  CK(S.d_modes.ensure(S.mode_elems * sizeof(int), g), "alloc modes");
  CK(S.h_O.ensure(S.o_elems * 16, g), "pinned O");
  CK(S.h_front.ensure(S.front_bytes, g), "pinned descriptors");
  CK(S.h_results.ensure(J * sizeof(ResultRec) + (want_parts ? S.parts * 32 : 0), g), "pinned results");
  CK(S.h_ctl.ensure(64, g), "pinned control");
  CK(S.h_modes.ensure(S.mode_elems * sizeof(int), g), "pinned modes");
  S.p_ctl = S.d_front.p;
  S.p_mats = (char*)S.d_front.p + S.off_mats;
  S.p_tasks = (char*)S.d_front.p + S.off_tasks;
  // staging
  long long oo = 0, bo = 0, mo = 0;
  double2* dO = (double2*)S.d_O.p;
  double2* dB = (double2*)S.d_B.p;
  tor_c128* hO = (tor_c128*)S.h_O.p;
  int* hm = (int*)S.h_modes.p;
  struct HostCopy {
    const tor_c128* src;
    tor_c128* dst;
    int m, ld;  // m x m entries from rows ld apart
  };
  std::vector<HostCopy> copies;
  for (int j = 0; j < J; ++j) {
    const MatIn& m = ins[S.act[j]];
    MatDesc& D = S.mats[j];
    const int mm = 2 * m.n;
    if (m.modes) {
      D.O = (const double2*)m.O;  // resident session matrix
      D.ld = m.ld;
      memcpy(hm + mo, m.modes, sizeof(int) * m.n);
      D.modes = (const int*)S.d_modes.p + mo;
      mo += m.n;
    } else if (m.dev) {
      D.O = (const double2*)m.O;
      D.ld = m.ld;
      D.modes = nullptr;
    } else {
      copies.push_back({m.O, hO + oo, mm, m.ld});
      D.O = dO + oo;
      D.ld = mm;
      D.modes = nullptr;
      oo += (long long)mm * mm;
    }
    D.B = dB + bo;
    bo += tri(m.n) * (long long)(eb / sizeof(double2));
  }
  stage_host_matrices(copies, (size_t)oo * sizeof(tor_c128));
  memset(S.h_front.p, 0, 64);  // the control words
  memcpy((char*)S.h_front.p + S.off_mats, S.mats.data(), J * sizeof(MatDesc));
  if (S.tasks_staged_gen != S.gen) {  // not already in the pinned staging buffer
    memcpy((char*)S.h_front.p + S.off_tasks, S.tasks.data(), S.tasks.size() * sizeof(TaskDesc));
    S.tasks_staged_gen = S.gen;
  }
  S.J = J;
  *any = true;
  return first;
}

static uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

// The stream operations of one pass, in three phases: front (inputs,
// descriptors, k_intake), units (k_units, possibly one time slice of it),
// back (k_reduce, results).  The timing events stay outside graphs.
static tor_status rec_front(tor_ctx* ctx, Slot& S, bool timed) {
  cudaStream_t s = S.stream;
  const int J = S.J;
  if (timed) CK(cudaEventRecord(S.ev[0], s), "event");
  if (S.o_elems) CK(cudaMemcpyAsync(S.d_O.p, S.h_O.p, S.o_elems * 16, cudaMemcpyHostToDevice, s), "H2D O");
  if (S.mode_elems)
    CK(cudaMemcpyAsync(S.d_modes.p, S.h_modes.p, S.mode_elems * sizeof(int), cudaMemcpyHostToDevice, s), "H2D modes");
  CK(cudaMemcpyAsync(S.p_ctl, S.h_front.p, S.front_bytes, cudaMemcpyHostToDevice, s), "H2D descriptors");
  if (timed) CK(cudaEventRecord(S.ev[1], s), "event");
  const bool check = !(ctx->cfg.flags & TOR_NO_CHECK);
  CK(launch_intake((const MatDesc*)S.p_mats, J, check ? 1 : 0, (int*)S.d_flags.p, s), "k_intake");
  if (timed) CK(cudaEventRecord(S.ev[2], s), "event");
  return TOR_OK;
}

// One launch of k_units; with slice_ns > 0 it stops taking tasks after that
// long and copies (ticket, abort word) to h_ctl so the host can relaunch it.
static tor_status rec_units(tor_ctx* ctx, Slot& S, long long slice_ns, bool one_task = false) {
  UnitsParams prm{};
  prm.mats = (const MatDesc*)S.p_mats;
  prm.tasks = (const TaskDesc*)S.p_tasks;
  prm.ntasks = (int)S.tasks.size();
  prm.ticket = (unsigned*)S.p_ctl;
  prm.abort_word = (int*)S.p_ctl + 1;
  prm.partials = (Part*)S.d_partials.p;
  prm.red_leaves = (Part*)S.d_partials.p + S.parts;
  prm.mat_flags = (int*)S.d_flags.p;
  prm.lane_scratch = (double2*)S.d_lane.p;
  prm.lane_elems = S.lane_e;
  prm.warp_scratch = (double2*)S.d_warp.p;
  prm.warp_elems = S.warp_e;
  prm.cancel = ctx->d_cancel;
  prm.cancel_epoch = S.cancel_epoch;
  prm.budget_ns = ctx->cfg.timeout_s > 0 ? (long long)(ctx->cfg.timeout_s * 1e9) : 0;
  prm.job_t0 = (unsigned long long*)((char*)S.p_ctl + 8);  // control words 2..3, zeroed with the pass
  prm.slice_ns = slice_ns;
  prm.ext = (ctx->cfg.flags & TOR_EXTENDED) ? 1 : 0;
  int grid = ctx->grid;
  if (one_task && S.d_pool) {  // a warp per task, blocks end throughout the job (see UnitsParams)
    prm.one_task = 1;
    prm.slot_pool = S.d_pool;
    prm.slot_words = S.pool_words;
    const int wpb = units_block_threads() / 32;
    grid = (int)std::min<long long>(((long long)S.tasks.size() + wpb - 1) / wpb, 0x7fffffffll);
  }
  CK(launch_units(prm, grid, S.stream), "k_units");
  if (slice_ns > 0) {
    CK(cudaMemcpyAsync(S.h_ctl.p, S.p_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, S.stream), "D2H ticket");
    CK(cudaEventRecord(S.units_done, S.stream), "event");
  }
  return TOR_OK;
}

static tor_status rec_back(tor_ctx* ctx, Slot& S, bool timed) {
  cudaStream_t s = S.stream;
  const int J = S.J;
  if (timed) CK(cudaEventRecord(S.ev[3], s), "event");
  CK(launch_reduce((const MatDesc*)S.p_mats, J, S.red_chunks, (Part*)S.d_partials.p + S.parts, (const int*)S.d_flags.p,
                   (ResultRec*)S.d_results.p, s),
     "k_reduce");
  if (timed) CK(cudaEventRecord(S.ev[4], s), "event");
  CK(cudaMemcpyAsync(S.h_results.p, S.d_results.p, J * sizeof(ResultRec), cudaMemcpyDeviceToHost, s), "D2H results");
  if (S.want_parts)
    CK(cudaMemcpyAsync((char*)S.h_results.p + J * sizeof(ResultRec), S.d_partials.p, S.parts * 32,
                       cudaMemcpyDeviceToHost, s),
       "D2H partials");
  CK(cudaMemcpyAsync(S.h_ctl.p, S.p_ctl, 2 * sizeof(int), cudaMemcpyDeviceToHost, s), "D2H control");
  return TOR_OK;
}

static tor_status slot_record(tor_ctx* ctx, Slot& S, bool timed) {
  tor_status st = rec_front(ctx, S, timed);
  if (st == TOR_OK) st = rec_units(ctx, S, 0);
  if (st == TOR_OK) st = rec_back(ctx, S, timed);
  return st;
}

// Enqueues the prepared job (graph replay when enabled and the shape repeats).
static tor_status slot_launch(tor_ctx* ctx, Slot& S, bool graphs) {
  S.cancel_epoch = __atomic_load_n(ctx->h_cancel, __ATOMIC_SEQ_CST);
  S.graphed = graphs;
  if (!S.graphed) {
    tor_status st = slot_record(ctx, S, true);
    if (st != TOR_OK) return st;
    CK(cudaEventRecord(S.done, S.stream), "event");
    return TOR_OK;
  }
  // The key holds what the captured pass depends on: launch shapes, copy sizes
  // and the values passed by value to the kernels.  What the kernels read from
  // the descriptors (source matrix, its size and layout, mode lists, the
  // arithmetic) is copied in by the pass itself, so it may differ between replays.
  uint64_t key = mix(0, (uint64_t)S.J);
  for (const MatDesc& D : S.mats)
    key = mix(key, (uint64_t)D.n | (uint64_t)D.p << 8 | (uint64_t)(D.modes != nullptr) << 29 | (uint64_t)D.ext << 33);
  for (const MatDesc& D : S.mats) key = mix(key, (uint64_t)D.red_lo << 8 ^ (uint64_t)D.red_log2);
  key = mix(key, (uint64_t)S.o_elems);
  key = mix(key, (uint64_t)S.mode_elems);
  key = mix(key, (uint64_t)S.tasks.size());
  key = mix(key, (uint64_t)S.want_parts);
  key = mix(key, (uint64_t)S.lane_e << 1 ^ (uint64_t)S.warp_e << 33);
  key = mix(key, (uint64_t)(uint32_t)S.cancel_epoch);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : S.graphs)
    if (g.key == key && g.gen == S.gen) exec = g.exec;
  if (!exec) {
    CK(cudaStreamBeginCapture(S.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    tor_status st = slot_record(ctx, S, false);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(S.stream, &graph);
    if (st != TOR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
    // keep a small cache; entries of older buffer generations can never match again
    std::vector<Slot::Graph> keep;
    for (auto& g : S.graphs) {
      if (g.gen != S.gen) cudaGraphExecDestroy(g.exec);
      else keep.push_back(g);
    }
    S.graphs.swap(keep);
    if (S.graphs.size() >= 64) {
      cudaGraphExecDestroy(S.graphs.front().exec);
      S.graphs.erase(S.graphs.begin());
    }
    S.graphs.push_back({key, S.gen, exec});
  }
  CK(cudaEventRecord(S.ev[0], S.stream), "event");
  CK(cudaGraphLaunch(exec, S.stream), "graph launch");
  CK(cudaEventRecord(S.ev[4], S.stream), "event");
  CK(cudaEventRecord(S.done, S.stream), "event");
  return TOR_OK;
}

// Reads back a finished job into out[] (indexed like the prepared inputs).
static tor_status slot_finish(Slot& S, tor_result* out, double* unit_partials, double* times) {
  tor_status first = TOR_OK;
  const ResultRec* hr = (const ResultRec*)S.h_results.p;
  const int abort_word = ((const int*)S.h_ctl.p)[1];
  for (int j = 0; j < S.J; ++j) {
    tor_result& r = out[S.act[j]];
    const ResultRec& q = hr[j];
    r.hi = q.hi;
    r.lo = q.lo;
    r.abs_sum = q.abs_sum;
    r.err_est = 8.0 * r.n * std::ldexp(1.0, S.mats[j].ext ? -104 : -53) * q.abs_sum;
    r.path = ((q.flags & FLAG_REAL) ? 1 : 0) | (S.mats[j].ext ? 2 : 0);
    if (q.flags & FLAG_NONFINITE) r.status = TOR_EINVAL;
    else if (q.flags & FLAG_NOTHERM) r.status = TOR_ENOTHERM;
    else if (abort_word & ABORT_NOSLOT) r.status = TOR_ECUDA;
    else if (abort_word & ABORT_CANCEL) r.status = TOR_ECANCELED;
    else if (abort_word & ABORT_TIMEOUT) r.status = TOR_ETIMEOUT;
    else if (q.flags & FLAG_NOTPD) r.status = TOR_ENOTPD;
    else r.status = TOR_OK;
    if (first == TOR_OK && r.status != TOR_OK) first = r.status;
  }
  if (unit_partials && S.J == 1) {
    const Part* hp = (const Part*)((const char*)S.h_results.p + S.J * sizeof(ResultRec));
    const long long U = 1ll << S.mats[0].p;
    for (long long u = 0; u < U; ++u) {
      unit_partials[3 * u] = hp[u].hi;
      unit_partials[3 * u + 1] = hp[u].lo;
      unit_partials[3 * u + 2] = hp[u].abs_sum;
    }
  }
  if (times) {
    float ms[4] = {-1, -1, -1, -1};
    if (!S.graphed) {
      cudaEventElapsedTime(&ms[0], S.ev[1], S.ev[2]);
      cudaEventElapsedTime(&ms[1], S.ev[2], S.ev[3]);
      cudaEventElapsedTime(&ms[2], S.ev[3], S.ev[4]);
    }
    cudaEventElapsedTime(&ms[3], S.ev[0], S.ev[4]);
    cudaGetLastError();
    for (int i = 0; i < 4; ++i) times[i] = ms[i];
  }
  return first;
}

// Blocking evaluation on the main slot (caller holds run_mu).
static tor_status run_blocking(tor_ctx* ctx, const std::vector<MatIn>& ins, tor_result* out, double* unit_partials,
                               size_t unit_len, bool allow_graphs = true) {
  CK(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
  for (int i = 0; i < 4; ++i) ctx->last_times[i] = 0;
  Slot& S = ctx->main;
  bool any = false;
  tor_status first = slot_prepare(ctx, S, ins, out, unit_partials != nullptr, &any);
  if (!any) return first;
  if (unit_partials && (S.J != 1 || unit_len < 3ull * (1ull << S.mats[0].p))) return TOR_EINVAL;
  tor_status st = slot_launch(ctx, S, allow_graphs && (ctx->cfg.flags & TOR_GRAPHS) != 0);
  if (st != TOR_OK) return st;
  CK(cudaStreamSynchronize(S.stream), "kernel execution");
  tor_status fin = slot_finish(S, out, unit_partials, ctx->last_times);
  return first != TOR_OK ? first : fin;
}

// ---------------------------------------------------------------------------
// Serving thread: continuous batching over several slots.
// ---------------------------------------------------------------------------
// Marks requests taken from the queue as finished; releases their session.
static void complete(tor_ctx* ctx, std::vector<Request*>& reqs) {  // caller holds q_mu
  for (Request* r : reqs) {
    r->done = true;
    if (r->sess) --r->sess->inflight;
  }
  ctx->done_cv.notify_all();
}

// Work of one request in subset terms (2^n).
static double request_terms(const Request* r) { return std::ldexp(1.0, std::max(0, std::min(r->in.n, 64))); }

// Serving slots: serve[0 .. n_large_slots) are the large lanes (one large
// request each, low stream priority, k_units as non-persistent one-task-per-warp
// launches, so a high-priority small batch's blocks take SMs as the large
// request's warps finish their tasks); the others are small lanes (FIFO batches
// of small requests, high priority).  With large_slice_ns > 0 a large request
// runs as persistent launches in time slices instead, continuing from its task
// ticket after each, so it is never restarted and its result does not depend
// on the interruptions.
static void server_loop(tor_ctx* ctx) {
  cudaSetDevice(ctx->cfg.device);
  struct InFlight {
    std::vector<Request*> reqs;
    std::vector<tor_result> res;
    bool failed = false;
  };
  std::vector<InFlight> fl(ctx->serve.size());
  const long long slice_ns = ctx->large_slice_ns;
  auto fail_slot = [&](size_t i, tor_status st) {
    Slot& S = *ctx->serve[i];
    for (int a : S.act) fl[i].res[a].status = st;
    fl[i].failed = true;
  };
  for (;;) {
    bool progressed = false;
    // 1. advance slots in flight
    for (size_t i = 0; i < ctx->serve.size(); ++i) {
      Slot& S = *ctx->serve[i];
      if (!S.busy) continue;
      if (S.phase == 1) {  // a k_units slice has ended?
        const cudaError_t q = cudaEventQuery(S.units_done);
        if (q == cudaErrorNotReady) continue;
        tor_status st = TOR_OK;
        if (q != cudaSuccess) {
          cudaGetLastError();
          st = TOR_ECUDA;
        } else {
          const unsigned ticket = ((const unsigned*)S.h_ctl.p)[0];
          const int abort_word = ((const int*)S.h_ctl.p)[1];
          const bool timed_out = ctx->cfg.timeout_s > 0 && now_s() - S.t_start > ctx->cfg.timeout_s;
          if (ticket < S.tasks.size() && !abort_word && !timed_out) {
            st = rec_units(ctx, S, slice_ns);  // continue from the ticket
            if (st == TOR_OK) {
              progressed = true;
              continue;
            }
          } else if (timed_out && ticket < S.tasks.size()) {
            int* w = (int*)S.h_ctl.p + 8;  // pinned; the results of this job become TOR_ETIMEOUT
            *w = ABORT_TIMEOUT;
            cudaMemcpyAsync((int*)S.p_ctl + 1, w, sizeof(int), cudaMemcpyHostToDevice, S.stream);
          }
        }
        if (st == TOR_OK) st = rec_back(ctx, S, false);
        if (st == TOR_OK && cudaEventRecord(S.done, S.stream) != cudaSuccess) st = TOR_ECUDA;
        if (st != TOR_OK) fail_slot(i, st);
        S.phase = 2;
        progressed = true;
        if (st == TOR_OK) continue;
      }
      // phase 2: reduce and copies
      if (!fl[i].failed) {
        const cudaError_t q = cudaEventQuery(S.done);
        if (q == cudaErrorNotReady) continue;
        if (q == cudaSuccess) slot_finish(S, fl[i].res.data(), nullptr, nullptr);
        else {
          cudaGetLastError();
          fail_slot(i, TOR_ECUDA);
        }
      }
      {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        for (size_t k = 0; k < fl[i].reqs.size(); ++k) fl[i].reqs[k]->res = fl[i].res[k];
        complete(ctx, fl[i].reqs);
      }
      ctx->served += (long long)fl[i].reqs.size();
      ctx->batches += 1;
      S.busy = false;
      S.phase = 0;
      fl[i] = InFlight();
      progressed = true;
    }
    // 2. admission: large requests FIFO into the large lane, small requests
    //    FIFO into the small lanes (they may pass a large request that waits)
    for (size_t i = 0; i < ctx->serve.size(); ++i) {
      Slot& S = *ctx->serve[i];
      if (S.busy) continue;
      const bool large_lane = (int)i < ctx->n_large_slots;
      const double big = ctx->max_batch_terms / 8;
      std::vector<Request*> batch;
      {
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        double terms = 0;
        for (auto it = ctx->queue.begin(); it != ctx->queue.end() && (int)batch.size() < ctx->max_batch;) {
          Request* r = *it;
          const double t = request_terms(r);
          const bool is_big = t > big;
          if (is_big != large_lane) {
            ++it;
            continue;
          }
          if (!batch.empty() && (large_lane || terms + t > ctx->max_batch_terms)) break;
          terms += t;
          if (r->sess) ++r->sess->inflight;  // the session's matrices stay alive until complete()
          batch.push_back(r);
          it = ctx->queue.erase(it);
        }
      }
      if (batch.empty()) continue;
      std::vector<MatIn> ins;
      for (Request* r : batch) ins.push_back(r->in);
      // device-memory budget: everything the context holds (every slot's
      // buffers, the sessions' matrices) stays within mem_budget.  Idle slots
      // give their buffers back first; then the batch shrinks; a request that
      // cannot fit even with nothing else running fails with TOR_ENOMEM, else
      // it waits for a running job to finish.
      if (ctx->cfg.mem_budget) {
        Needs need = job_needs(ctx, ins, ins.size());
        if (over_budget(ctx, S, need)) {
          for (size_t k = 0; k < ctx->serve.size(); ++k)
            if (k != i && !ctx->serve[k]->busy) ctx->serve[k]->release_dev();
          std::unique_lock<std::mutex> ml(ctx->run_mu, std::try_to_lock);
          if (ml) ctx->main.release_dev();
        }
        while (batch.size() > 1 && over_budget(ctx, S, need)) {
          std::lock_guard<std::mutex> lk(ctx->q_mu);
          if (batch.back()->sess) --batch.back()->sess->inflight;
          ctx->queue.push_front(batch.back());
          batch.pop_back();
          ins.pop_back();
          need = job_needs(ctx, ins, ins.size());
        }
        if (over_budget(ctx, S, need)) {
          bool others = false;  // another slot (or a blocking call on the main slot) holds memory in use
          for (size_t k = 0; k < ctx->serve.size(); ++k) others |= k != i && ctx->serve[k]->busy;
          {
            std::unique_lock<std::mutex> ml(ctx->run_mu, std::try_to_lock);
            others |= !ml;
          }
          const long long alone = ctx->dev_held.load() - (long long)S.dev_bytes() + (long long)need.total();
          if (!others && alone > (long long)ctx->cfg.mem_budget) {  // cannot fit even alone
            std::lock_guard<std::mutex> lk(ctx->q_mu);
            batch[0]->res = tor_result{};
            batch[0]->res.n = batch[0]->in.n;
            batch[0]->res.status = TOR_ENOMEM;
            complete(ctx, batch);
            continue;
          }
          if (!others) {
            S.release_dev();  // fits once this slot's own smaller buffers are gone
          } else {            // wait for a job in flight to finish
            std::lock_guard<std::mutex> lk(ctx->q_mu);
            if (batch[0]->sess) --batch[0]->sess->inflight;
            ctx->queue.push_front(batch[0]);
            continue;
          }
        }
      }
      std::vector<tor_result> res(ins.size());
      bool any = false;
      tor_status st;
      try {
        st = slot_prepare(ctx, S, ins, res.data(), false, &any);
      } catch (const std::bad_alloc&) {
        any = false;
        st = TOR_ENOMEM;
        for (size_t k = 0; k < res.size(); ++k) {
          res[k] = tor_result{};
          res[k].n = ins[k].n;
          res[k].status = TOR_ENOMEM;
        }
      }
      if (any && !large_lane && S.J == 1) {
        // a lone small request: its pass is replayed from a CUDA graph of its shape
        // (one launch instead of four copies and three to four kernels)
        S.t_start = now_s();
        st = slot_launch(ctx, S, true);
      } else if (any) {
        S.cancel_epoch = __atomic_load_n(ctx->h_cancel, __ATOMIC_SEQ_CST);
        S.graphed = false;
        S.t_start = now_s();
        st = rec_front(ctx, S, false);
        if (st == TOR_OK) st = rec_units(ctx, S, large_lane ? slice_ns : 0, large_lane && slice_ns == 0);
        if (st == TOR_OK && !(large_lane && slice_ns > 0)) {
          st = rec_back(ctx, S, false);
          if (st == TOR_OK && cudaEventRecord(S.done, S.stream) != cudaSuccess) st = TOR_ECUDA;
        }
      }
      if (!any || st == TOR_ECUDA || st == TOR_ENOMEM) {
        // nothing to run, or the launch failed: complete now
        std::lock_guard<std::mutex> lk(ctx->q_mu);
        for (size_t k = 0; k < batch.size(); ++k) {
          batch[k]->res = res[k];
          if (any && std::find(S.act.begin(), S.act.end(), (int)k) != S.act.end()) batch[k]->res.status = st;
        }
        complete(ctx, batch);
        continue;
      }
      S.busy = true;
      S.large = large_lane;
      S.phase = (large_lane && slice_ns > 0) ? 1 : 2;
      fl[i].reqs = std::move(batch);
      fl[i].res = std::move(res);
      progressed = true;
    }
    // 3. idle / stop
    bool busy = false;
    for (auto& sl : ctx->serve) busy |= sl->busy;
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    if (ctx->stopping && !busy && ctx->queue.empty()) return;
    if (!progressed) {
      if (!busy && ctx->queue.empty()) {
        // idle: spin a while before sleeping, so that a request arriving soon is
        // taken without the wake-up latency of a sleeping thread
        if (ctx->idle_spin_s > 0) {
          const unsigned long long seen = ctx->q_events.load(std::memory_order_acquire);
          lk.unlock();
          const double t_end = now_s() + ctx->idle_spin_s;
          while (ctx->q_events.load(std::memory_order_acquire) == seen && now_s() < t_end) std::this_thread::yield();
          lk.lock();
        }
        ctx->q_cv.wait(lk, [&] { return ctx->stopping || !ctx->queue.empty(); });
      } else {
        // jobs in flight: poll their events again at once (a timed wait would
        // sleep for the kernel's timer slack, ~50 us, on every completion)
        lk.unlock();
        std::this_thread::yield();
      }
    }
  }
}

static tor_status start_server(tor_ctx* ctx) {  // caller holds q_mu
  if (ctx->server_started) return TOR_OK;
  cudaSetDevice(ctx->cfg.device);
  for (int i = 0; i < ctx->n_serve_slots; ++i) {
    std::unique_ptr<Slot> s(new Slot());
    // large lanes low priority, small lanes high
    cudaError_t e = slot_init(*s, nullptr, i < ctx->n_large_slots ? 1 : -1);
    if (e != cudaSuccess) {
      s->release();
      return cuda_fail(ctx, e, "serving slot");
    }
    slot_account(ctx, *s, true);
    if (i < ctx->n_large_slots) {  // the scratch-slot pool of its non-persistent launches
      s->pool_words = (ctx->grid + 31) / 32;
      std::vector<unsigned> init((size_t)s->pool_words, 0u);
      if (ctx->grid % 32) init.back() = ~0u << (ctx->grid % 32);  // no slots past the resident blocks
      e = cudaMalloc((void**)&s->d_pool, sizeof(unsigned) * init.size());
      if (e == cudaSuccess) e = cudaMemcpy(s->d_pool, init.data(), sizeof(unsigned) * init.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        s->release();
        return cuda_fail(ctx, e, "serving slot pool");
      }
    }
    // pinned staging sized up front: growing it later (cudaFreeHost) would wait for the device
    uint64_t* g = &s->gen;
    for (HostBuf* b : {&s->h_O, &s->h_front}) e = e == cudaSuccess ? b->ensure(1 << 20, g) : e;
    for (HostBuf* b : {&s->h_results, &s->h_ctl, &s->h_modes}) e = e == cudaSuccess ? b->ensure(1 << 16, g) : e;
    if (e != cudaSuccess) {
      s->release();
      return cuda_fail(ctx, e, "serving slot staging");
    }
    ctx->serve.push_back(std::move(s));
  }
  ctx->server = std::thread(server_loop, ctx);
  ctx->server_started = true;
  return TOR_OK;
}

static tor_status enqueue_request(tor_ctx* ctx, Request* r, uint64_t* ticket) {
  {
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    if (ctx->queue.size() >= ctx->queue_limit) {
      delete r;
      return TOR_EAGAIN;
    }
    tor_status st = start_server(ctx);
    if (st != TOR_OK) {
      delete r;
      return st;
    }
    r->ticket = ctx->next_ticket++;
    ctx->reqs[r->ticket] = r;
    ctx->queue.push_back(r);
    *ticket = r->ticket;
    ctx->q_events.fetch_add(1, std::memory_order_release);
  }
  ctx->q_cv.notify_one();
  return TOR_OK;
}

// ---------------------------------------------------------------------------
// Sessions: resident chain-rule prefix matrices O^(j) = I - (Sigma_[j])^{-1}.
// Computed on the host in long double: K = Sigma^{-1} (or I - O), then one
// rank-2 downdate per removed mode, K_[j-1] = K_aa - K_ab K_bb^{-1} K_ba,
// which is the inverse of the leading block Sigma_[j-1].
// ---------------------------------------------------------------------------
namespace {
struct CL {
  long double re, im;
};
inline CL cadd(CL a, CL b) { return {a.re + b.re, a.im + b.im}; }
inline CL csub(CL a, CL b) { return {a.re - b.re, a.im - b.im}; }
inline CL cmul(CL a, CL b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline CL cconj(CL a) { return {a.re, -a.im}; }

// In-place inverse of an HPD matrix (m x m, row-major) via A = L L^H; false if not PD.
bool hpd_inverse(std::vector<CL>& A, int m) {
  std::vector<CL> L((size_t)m * m, CL{0, 0});
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      CL s = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) s = csub(s, cmul(L[(size_t)i * m + k], cconj(L[(size_t)j * m + k])));
      if (i == j) {
        if (!(s.re > 0)) return false;
        L[(size_t)i * m + i] = {sqrtl(s.re), 0};
      } else {
        const long double d = L[(size_t)j * m + j].re;
        L[(size_t)i * m + j] = {s.re / d, s.im / d};
      }
    }
  }
  // W = L^{-1} (lower triangular), A^{-1} = W^H W
  std::vector<CL> W((size_t)m * m, CL{0, 0});
  for (int i = 0; i < m; ++i) {
    W[(size_t)i * m + i] = {1.0L / L[(size_t)i * m + i].re, 0};
    for (int j = 0; j < i; ++j) {
      CL s{0, 0};
      for (int k = j; k < i; ++k) s = csub(s, cmul(L[(size_t)i * m + k], W[(size_t)k * m + j]));
      const long double d = L[(size_t)i * m + i].re;
      W[(size_t)i * m + j] = {s.re / d, s.im / d};
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      CL s{0, 0};
      for (int k = std::max(i, j); k < m; ++k) s = cadd(s, cmul(cconj(W[(size_t)k * m + i]), W[(size_t)k * m + j]));
      A[(size_t)i * m + j] = s;
    }
  return true;
}
}  // namespace

// Nothing throws across the C ABI: an allocation failure inside an entry point
// becomes TOR_ENOMEM (locks are scoped, so they are released on the way out).
template <class F>
static tor_status guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return TOR_ENOMEM;
  } catch (...) {
    return TOR_EINVAL;
  }
}

extern "C" {

void tor_config_default(tor_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof *cfg);
  cfg->device = 0;
  cfg->stream = nullptr;
  cfg->mem_budget = 0;
  cfg->prefix_depth = -1;
  cfg->layout = TOR_LAYOUT_BLOCK;
  cfg->flags = 0;
  cfg->timeout_s = 0.0;
}

const char* tor_strerror(tor_status s) {
  switch (s) {
    case TOR_OK: return "ok";
    case TOR_EINVAL: return "invalid argument or non-finite input";
    case TOR_ENOTHERM: return "input matrix is not Hermitian";
    case TOR_ENOTPD: return "I - O is not positive definite";
    case TOR_ENOMEM: return "out of memory or over the memory budget";
    case TOR_EAGAIN: return "not ready / queue full";
    case TOR_ETIMEOUT: return "timed out";
    case TOR_ECANCELED: return "cancelled";
    case TOR_ECUDA: return "CUDA error";
    case TOR_ETOOBIG: return "too many modes for this call";
  }
  return "unknown status";
}

const char* tor_last_error(tor_ctx* ctx) { return ctx ? ctx->last_error.c_str() : g_create_error.c_str(); }

tor_status tor_plan_load(tor_ctx* ctx, const char* path);

static tor_status tor_create_impl(const tor_config* cfg, tor_ctx** out) {
  if (!out) return TOR_EINVAL;
  *out = nullptr;
  tor_config c;
  tor_config_default(&c);
  if (cfg) c = *cfg;
  if (c.layout != TOR_LAYOUT_BLOCK && c.layout != TOR_LAYOUT_PAIRS) return TOR_EINVAL;
  if (c.timeout_s < 0) return TOR_EINVAL;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
  if (c.device < 0 || c.device >= ndev) return TOR_EINVAL;
  tor_ctx* ctx = new tor_ctx();
  ctx->cfg = c;
  for (int i = 0; i < 65; ++i) ctx->plan[i] = -1;
  auto fail = [&](cudaError_t err, const char* what) {
    tor_status s = cuda_fail(ctx, err, what);
    tor_destroy(ctx);
    return s;
  };
  if ((e = cudaSetDevice(c.device)) != cudaSuccess) return fail(e, "cudaSetDevice");
  if ((e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, c.device)) != cudaSuccess)
    return fail(e, "attribute");
  if ((e = units_blocks_per_sm(&ctx->blocks_per_sm, (c.flags & TOR_EXTENDED) ? 1 : 0)) != cudaSuccess)
    return fail(e, "occupancy");
  ctx->blocks_per_sm = std::max(1, ctx->blocks_per_sm);
  ctx->grid = ctx->sms * ctx->blocks_per_sm;
  ctx->nwarps = ctx->grid * (units_block_threads() / 32);
  if ((e = slot_init(ctx->main, (cudaStream_t)c.stream)) != cudaSuccess) return fail(e, "stream/events");
  slot_account(ctx, ctx->main, false);
  if (const char* v = getenv("TOR_SERVE_SLICE_MS")) ctx->large_slice_ns = (long long)(atof(v) * 1e6);
  if (const char* v = getenv("TOR_SERVE_IDLE_SPIN_MS")) ctx->idle_spin_s = std::max(0.0, atof(v) * 1e-3);
  if (const char* v = getenv("TOR_SERVE_LARGE_LANES")) ctx->n_large_slots = std::max(1, std::min(3, atoi(v)));
  if ((e = cudaHostAlloc((void**)&ctx->h_cancel, sizeof(int), cudaHostAllocMapped)) != cudaSuccess)
    return fail(e, "cancel flag");
  *ctx->h_cancel = 0;
  if ((e = cudaHostGetDevicePointer((void**)&ctx->d_cancel, ctx->h_cancel, 0)) != cudaSuccess)
    return fail(e, "cancel flag map");
  if (c.prefix_depth < 0) {
    const char* cache = getenv("TOR_AUTOTUNE_CACHE");
    if (cache && *cache) tor_plan_load(ctx, cache);  // a missing or foreign table is ignored
  }
  *out = ctx;
  return TOR_OK;
}

tor_status tor_create(const tor_config* cfg, tor_ctx** out) {
  return guarded([&] { return tor_create_impl(cfg, out); });
}

void tor_destroy(tor_ctx* ctx) {
  if (!ctx) return;
  {
    // requests still queued are dropped (TOR_ECANCELED); jobs on the GPU are asked to stop
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    ctx->stopping = true;
    ctx->q_events.fetch_add(1, std::memory_order_release);
    for (Request* r : ctx->queue) {
      r->res = tor_result{};
      r->res.n = r->in.n;
      r->res.status = TOR_ECANCELED;
      r->done = true;
    }
    ctx->queue.clear();
    if (ctx->h_cancel) __atomic_add_fetch(ctx->h_cancel, 1, __ATOMIC_SEQ_CST);
  }
  ctx->done_cv.notify_all();
  ctx->q_cv.notify_all();
  if (ctx->server.joinable()) ctx->server.join();
  for (auto& kv : ctx->reqs) delete kv.second;
  ctx->reqs.clear();
  for (tor_session* s : ctx->sessions) {  // sessions outlive the context, detached
    s->ctx = nullptr;
    s->d_O.acct = nullptr;
  }
  ctx->sessions.clear();
  cudaSetDevice(ctx->cfg.device);
  if (ctx->main.stream) {
    const cudaError_t e = cudaStreamSynchronize(ctx->main.stream);
    if (e != cudaSuccess && getenv("TOR_DEBUG"))
      fprintf(stderr, "libtor: tor_destroy: stream synchronize failed: %s\n", cudaGetErrorString(e));
  }
  ctx->main.release();
  for (auto& s : ctx->serve) s->release();
  ctx->serve.clear();
  if (ctx->h_cancel) cudaFreeHost(ctx->h_cancel);
  cudaGetLastError();
  delete ctx;
}

int tor_plan_prefix_depth(tor_ctx* ctx, int n) {
  if (!ctx || n < 0 || n > 64) return -1;
  if (n == 0) return 0;
  return plan_p(ctx, n);
}

tor_status tor_set_prefix_depth(tor_ctx* ctx, int n, int p) {
  if (!ctx || n < 1 || n > 64 || p < -1 || p > n - 1 || p > kMaxPrefixDepth) return TOR_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  ctx->plan[n] = p;
  return TOR_OK;
}

tor_status tor_cancel(tor_ctx* ctx) {
  if (!ctx) return TOR_EINVAL;
  __atomic_add_fetch(ctx->h_cancel, 1, __ATOMIC_SEQ_CST);
  return TOR_OK;
}

tor_status tor_last_times(tor_ctx* ctx, double* times) {
  if (!ctx || !times) return TOR_EINVAL;
  for (int i = 0; i < 4; ++i) times[i] = ctx->last_times[i];
  return TOR_OK;
}

tor_status tor_probe_fp64(int device, double seconds, double* dfma_per_s, double* fp64_tflops) {
  if (!dfma_per_s || !fp64_tflops || seconds <= 0) return TOR_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return TOR_ECUDA;
  }
  double r = 0;
  cudaError_t e = run_probe_fp64(seconds, &r);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TOR_ECUDA;
  }
  *dfma_per_s = r;
  *fp64_tflops = 2.0 * r / 1e12;
  return TOR_OK;
}

static tor_status tor_eval_batch_impl(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                          tor_result* out) {
  if (!ctx || count < 0 || (count > 0 && (!n || !O || !out))) return TOR_EINVAL;
  std::vector<MatIn> ins(count);
  const bool dev = (ctx->cfg.flags & TOR_IN_DEVICE) != 0;
  for (int i = 0; i < count; ++i) {
    ins[i].n = n[i];
    ins[i].O = O[i];
    ins[i].ld = ld ? ld[i] : 2 * n[i];
    ins[i].n_src = n[i];
    ins[i].layout = ctx->cfg.layout;
    ins[i].dev = dev;
  }
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  return run_blocking(ctx, ins, out, nullptr, 0);
}

tor_status tor_eval_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                          tor_result* out) {
  return guarded([&] { return tor_eval_batch_impl(ctx, count, n, O, ld, out); });
}

static tor_status tor_eval_impl(tor_ctx* ctx, int n, const tor_c128* O, int ld, tor_result* out) {
  if (!ctx || !out) return TOR_EINVAL;
  const tor_c128* Op[1] = {O};
  int lds[1] = {ld};
  return tor_eval_batch(ctx, 1, &n, Op, lds, out);
}

tor_status tor_eval(tor_ctx* ctx, int n, const tor_c128* O, int ld, tor_result* out) {
  return guarded([&] { return tor_eval_impl(ctx, n, O, ld, out); });
}

static tor_status tor_eval_seq_impl(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                                    tor_result* out, double* ms) {
  if (!ctx || count < 0 || (count > 0 && (!n || !O || !ld || !out))) return TOR_EINVAL;
  tor_status first = TOR_OK;
  for (int i = 0; i < count; ++i) {
    const auto t0 = std::chrono::steady_clock::now();
    const tor_status st = tor_eval_impl(ctx, n[i], O[i], ld[i], &out[i]);
    if (ms) ms[i] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (first == TOR_OK && st != TOR_OK) first = st;
  }
  return first;
}

tor_status tor_eval_seq(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                        tor_result* out, double* ms) {
  return guarded([&] { return tor_eval_seq_impl(ctx, count, n, O, ld, out, ms); });
}

static tor_status tor_eval_units_impl(tor_ctx* ctx, int n, const tor_c128* O, int ld, double* partials, size_t partials_len,
                          tor_result* out) {
  if (!ctx || !out || !partials || n < 1 || n > 64) return TOR_EINVAL;
  std::vector<MatIn> ins(1);
  ins[0].n = n;
  ins[0].O = O;
  ins[0].ld = ld;
  ins[0].n_src = n;
  ins[0].layout = ctx->cfg.layout;
  ins[0].dev = (ctx->cfg.flags & TOR_IN_DEVICE) != 0;
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  return run_blocking(ctx, ins, out, partials, partials_len);
}

tor_status tor_eval_units(tor_ctx* ctx, int n, const tor_c128* O, int ld, double* partials, size_t partials_len,
                          tor_result* out) {
  return guarded([&] { return tor_eval_units_impl(ctx, n, O, ld, partials, partials_len, out); });
}

long long tor_plan_leaves(tor_ctx* ctx, int n) {
  if (!ctx || n < 1 || n > 64) return -1;
  const int p = plan_p(ctx, n);
  return 1ll << (p >= 5 ? p - 5 : p);
}

static tor_status tor_eval_range_impl(tor_ctx* ctx, int n, const tor_c128* O, int ld, long long leaf_lo, long long leaf_count,
                          tor_result* out) {
  if (!ctx || !out || n < 1 || n > 64) return TOR_EINVAL;
  if (!range_ok(plan_p(ctx, n), leaf_lo, leaf_count)) return TOR_EINVAL;
  std::vector<MatIn> ins(1);
  ins[0].n = n;
  ins[0].O = O;
  ins[0].ld = ld;
  ins[0].n_src = n;
  ins[0].layout = ctx->cfg.layout;
  ins[0].dev = (ctx->cfg.flags & TOR_IN_DEVICE) != 0;
  ins[0].leaf_lo = leaf_lo;
  ins[0].leaf_count = leaf_count;
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  return run_blocking(ctx, ins, out, nullptr, 0);
}

tor_status tor_eval_range(tor_ctx* ctx, int n, const tor_c128* O, int ld, long long leaf_lo, long long leaf_count,
                          tor_result* out) {
  return guarded([&] { return tor_eval_range_impl(ctx, n, O, ld, leaf_lo, leaf_count, out); });
}

static tor_status tor_eval_range_batch_impl(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O,
                                            const int* ld, const long long* leaf_lo, const long long* leaf_count,
                                            tor_result* out) {
  if (!ctx || count < 0 || (count > 0 && (!n || !O || !leaf_lo || !leaf_count || !out))) return TOR_EINVAL;
  std::vector<MatIn> ins(count);
  const bool dev = (ctx->cfg.flags & TOR_IN_DEVICE) != 0;
  for (int i = 0; i < count; ++i) {
    ins[i].n = n[i];
    ins[i].O = O[i];
    ins[i].ld = ld ? ld[i] : 2 * n[i];
    ins[i].n_src = n[i];
    ins[i].layout = ctx->cfg.layout;
    ins[i].dev = dev;
    if (leaf_count[i] >= 0) {  // a shard; slot_prepare flags an invalid range TOR_EINVAL
      ins[i].leaf_lo = leaf_lo[i];
      ins[i].leaf_count = leaf_count[i];
      ins[i].bad_range = leaf_count[i] == 0;
    }
  }
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  return run_blocking(ctx, ins, out, nullptr, 0);
}

tor_status tor_eval_range_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                                const long long* leaf_lo, const long long* leaf_count, tor_result* out) {
  return guarded([&] { return tor_eval_range_batch_impl(ctx, count, n, O, ld, leaf_lo, leaf_count, out); });
}

static tor_status tor_submit_impl(tor_ctx* ctx, int n, const tor_c128* O, int ld, uint64_t* ticket) {
  if (!ctx || !ticket || n < 0 || (n > 0 && !O) || ld < 2 * n) return TOR_EINVAL;
  if (n > 64) return TOR_ETOOBIG;
  if (ctx->cfg.flags & TOR_IN_DEVICE) return TOR_EINVAL;  // the queue copies host inputs only
  Request* r = new Request();
  r->O.resize((size_t)4 * n * n);
  for (int i = 0; i < 2 * n; ++i)
    memcpy(r->O.data() + (size_t)i * 2 * n, O + (size_t)i * ld, sizeof(tor_c128) * 2 * n);
  r->in.n = n;
  r->in.O = r->O.data();
  r->in.ld = 2 * n;
  r->in.n_src = n;
  r->in.layout = ctx->cfg.layout;
  return enqueue_request(ctx, r, ticket);
}

tor_status tor_submit(tor_ctx* ctx, int n, const tor_c128* O, int ld, uint64_t* ticket) {
  return guarded([&] { return tor_submit_impl(ctx, n, O, ld, ticket); });
}

tor_status tor_poll(tor_ctx* ctx, uint64_t ticket, tor_result* out, double timeout_s) {
  if (!ctx || !out) return TOR_EINVAL;
  std::unique_lock<std::mutex> lk(ctx->q_mu);
  auto it = ctx->reqs.find(ticket);
  if (it == ctx->reqs.end()) return TOR_EINVAL;
  Request* r = it->second;
  if (!r->done) {
    if (timeout_s == 0) return TOR_EAGAIN;
    if (timeout_s < 0) ctx->done_cv.wait(lk, [&] { return r->done; });
    else if (!ctx->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; }))
      return TOR_EAGAIN;
  }
  *out = r->res;
  ctx->reqs.erase(it);
  delete r;
  return out->status;
}

tor_status tor_poll_any(tor_ctx* ctx, const uint64_t* tickets, int count, double timeout_s, int* index,
                        tor_result* out) {
  if (!ctx || !out || !index || count < 1 || !tickets) return TOR_EINVAL;
  std::unique_lock<std::mutex> lk(ctx->q_mu);
  std::vector<Request*> rs((size_t)count);
  for (int i = 0; i < count; ++i) {
    auto it = ctx->reqs.find(tickets[i]);
    if (it == ctx->reqs.end()) return TOR_EINVAL;
    rs[i] = it->second;
  }
  int hit = -1;
  auto any_done = [&] {
    for (int i = 0; i < count; ++i)
      if (rs[i]->done) {
        hit = i;
        return true;
      }
    return false;
  };
  if (!any_done()) {
    if (timeout_s == 0) return TOR_EAGAIN;
    if (timeout_s < 0) ctx->done_cv.wait(lk, any_done);
    else if (!ctx->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), any_done)) return TOR_EAGAIN;
  }
  *index = hit;
  *out = rs[hit]->res;
  ctx->reqs.erase(tickets[hit]);
  delete rs[hit];
  return out->status;
}

tor_status tor_memory(tor_ctx* ctx, size_t* held, size_t* budget) {
  if (!ctx) return TOR_EINVAL;
  if (held) *held = (size_t)std::max(0ll, ctx->dev_held.load());
  if (budget) *budget = ctx->cfg.mem_budget;
  return TOR_OK;
}

tor_status tor_serving_stats(tor_ctx* ctx, long long* served, long long* batches, long long* queued) {
  if (!ctx) return TOR_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->q_mu);
  if (served) *served = ctx->served.load();
  if (batches) *batches = ctx->batches.load();
  if (queued) *queued = (long long)ctx->queue.size();
  return TOR_OK;
}

static tor_status tor_session_create_impl(tor_ctx* ctx, int n_total, const tor_c128* M, int ld, int kind,
                              tor_session** out) {
  if (!ctx || !out || !M || n_total < 1 || n_total > 1024 || ld < 2 * n_total) return TOR_EINVAL;
  if (kind != TOR_SESSION_SIGMA && kind != TOR_SESSION_O) return TOR_EINVAL;
  *out = nullptr;
  const int N = n_total, m = 2 * N;
  const bool block = ctx->cfg.layout == TOR_LAYOUT_BLOCK;
  auto src = [&](int r) { return block ? (r >> 1) + (r & 1) * N : r; };  // pairs row -> input row
  // K = (Sigma_[N])^{-1} in pairs order
  std::vector<CL> K((size_t)m * m);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      const tor_c128 v = M[(size_t)src(a) * ld + src(b)];
      K[(size_t)a * m + b] = kind == TOR_SESSION_O ? CL{(a == b ? 1.0L : 0.0L) - v.re, -(long double)v.im}
                                                   : CL{(long double)v.re, (long double)v.im};
    }
  // structure of K = Sigma^{-1} in pairs order: K(a_j^dag, a_k^dag) = conj K(a_j, a_k),
  // K(a_j^dag, a_k) = conj K(a_j, a_k^dag)
  long double kmax = 0, kdev = 0;
  for (int j = 0; j < N; ++j)
    for (int k = 0; k < N; ++k) {
      const CL aa = K[(size_t)(2 * j) * m + 2 * k], dd = K[(size_t)(2 * j + 1) * m + 2 * k + 1];
      const CL ac = K[(size_t)(2 * j) * m + 2 * k + 1], ca = K[(size_t)(2 * j + 1) * m + 2 * k];
      for (long double v : {aa.re, aa.im, dd.re, dd.im, ac.re, ac.im, ca.re, ca.im}) kmax = std::max(kmax, fabsl(v));
      kdev = std::max({kdev, fabsl(dd.re - aa.re), fabsl(dd.im + aa.im), fabsl(ca.re - ac.re), fabsl(ca.im + ac.im)});
    }
  if (kind == TOR_SESSION_SIGMA && !hpd_inverse(K, m)) return TOR_ENOTPD;
  tor_session* s = new tor_session();
  s->real = kdev <= 1e-12L * kmax && !(ctx->cfg.flags & TOR_COMPLEX_PATH);
  s->ctx = ctx;
  s->device = ctx->cfg.device;
  s->N = N;
  s->off.assign(N + 1, 0);
  long long tot = 0;
  for (int j = 1; j <= N; ++j) {
    s->off[j] = tot;
    tot += 4ll * j * j;
  }
  std::vector<tor_c128> host((size_t)tot);
  // det K^(j) = det(K_bb) det K^(j-1) (Schur complement of mode j-1's 2x2 block K_bb), so
  // log det Sigma_[j] = -sum_{i <= j} log det(K_bb at step i)
  std::vector<long double> logd(N + 1, 0.0L);
  for (int j = N; j >= 1; --j) {
    const int mj = 2 * j;
    tor_c128* Oj = host.data() + s->off[j];
    if (!s->real) {
      for (int a = 0; a < mj; ++a)
        for (int b = 0; b < mj; ++b) {
          const CL k = K[(size_t)a * m + b];
          Oj[(size_t)a * mj + b] = tor_c128{(double)((a == b ? 1.0L : 0.0L) - k.re), (double)(-k.im)};
        }
    } else {
      // A physical state: write O^(j) exactly Hermitian and exactly of the form
      // O(a_u^dag, a_v^dag) = conj O(a_u, a_v), O(a_u^dag, a_v) = conj O(a_u, a_v^dag),
      // from the average of the (rounding-level different) entries that the
      // structure identifies, each rounded once.
      auto o = [&](int a, int b) {
        const CL k = K[(size_t)a * m + b];
        return CL{(a == b ? 1.0L : 0.0L) - k.re, -k.im};
      };
      for (int u = 0; u < j; ++u)
        for (int v = 0; v <= u; ++v) {
          const CL x1 = o(2 * u, 2 * v), y1 = o(2 * u + 1, 2 * v + 1), x2 = o(2 * v, 2 * u), y2 = o(2 * v + 1, 2 * u + 1);
          const CL z1 = o(2 * u, 2 * v + 1), w1 = o(2 * u + 1, 2 * v), z2 = o(2 * v, 2 * u + 1), w2 = o(2 * v + 1, 2 * u);
          // P(u, v) ~ x1 ~ conj y1 ~ conj x2 ~ y2;  Q(u, v) = Q(v, u) ~ z1 ~ conj w1 ~ z2 ~ conj w2
          const tor_c128 P{(double)((x1.re + y1.re + x2.re + y2.re) / 4), (double)((x1.im - y1.im - x2.im + y2.im) / 4)};
          const tor_c128 Q{(double)((z1.re + w1.re + z2.re + w2.re) / 4), (double)((z1.im - w1.im + z2.im - w2.im) / 4)};
          const tor_c128 Pc{P.re, -P.im}, Qc{Q.re, -Q.im};
          Oj[(size_t)(2 * u) * mj + 2 * v] = P;
          Oj[(size_t)(2 * u + 1) * mj + 2 * v + 1] = Pc;
          Oj[(size_t)(2 * v) * mj + 2 * u] = Pc;
          Oj[(size_t)(2 * v + 1) * mj + 2 * u + 1] = P;
          Oj[(size_t)(2 * u) * mj + 2 * v + 1] = Q;
          Oj[(size_t)(2 * u + 1) * mj + 2 * v] = Qc;
          Oj[(size_t)(2 * v) * mj + 2 * u + 1] = Q;
          Oj[(size_t)(2 * v + 1) * mj + 2 * u] = Qc;
        }
    }
    if (j == 1) {
      const long double d1 = K[0].re * K[(size_t)m + 1].re - (K[1].re * K[1].re + K[1].im * K[1].im);
      if (!(d1 > 0)) {
        delete s;
        return TOR_ENOTPD;
      }
      logd[1] = logl(d1);
      break;
    }
    // remove mode j-1 (rows/cols b0, b0+1): K <- K_aa - K_ab K_bb^{-1} K_ba
    const int b0 = mj - 2;
    const CL p = K[(size_t)b0 * m + b0], q = K[(size_t)b0 * m + b0 + 1], r = K[(size_t)(b0 + 1) * m + b0],
             t = K[(size_t)(b0 + 1) * m + b0 + 1];
    const CL det = csub(cmul(p, t), cmul(q, r));
    const long double dd = det.re * det.re + det.im * det.im;
    if (!(dd > 0) || !(det.re > 0)) {
      delete s;
      return TOR_ENOTPD;
    }
    logd[j] = logl(det.re);
    const CL idet{det.re / dd, -det.im / dd};
    const CL i00 = cmul(t, idet), i01 = cmul(CL{-q.re, -q.im}, idet), i10 = cmul(CL{-r.re, -r.im}, idet),
             i11 = cmul(p, idet);
    for (int a = 0; a < b0; ++a) {
      const CL ka0 = K[(size_t)a * m + b0], ka1 = K[(size_t)a * m + b0 + 1];
      const CL u0 = cadd(cmul(ka0, i00), cmul(ka1, i10)), u1 = cadd(cmul(ka0, i01), cmul(ka1, i11));
      for (int b = 0; b < b0; ++b) {
        const CL d = cadd(cmul(u0, K[(size_t)b0 * m + b]), cmul(u1, K[(size_t)(b0 + 1) * m + b]));
        K[(size_t)a * m + b] = csub(K[(size_t)a * m + b], d);
      }
    }
  }
  s->logdet_sigma.assign(N + 1, 0.0L);
  for (int j = 1; j <= N; ++j) s->logdet_sigma[j] = s->logdet_sigma[j - 1] - logd[j];
  cudaSetDevice(ctx->cfg.device);
  if (ctx->cfg.mem_budget && (size_t)std::max(0ll, ctx->dev_held.load()) + (size_t)tot * 16 > ctx->cfg.mem_budget) {
    delete s;
    return TOR_ENOMEM;
  }
  s->d_O.acct = &ctx->dev_held;
  cudaError_t e = s->d_O.ensure((size_t)tot * 16, &s->gen);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_O.p, host.data(), (size_t)tot * 16, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tor_status st = cuda_fail(ctx, e, "session upload");
    s->d_O.release();
    delete s;
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    ctx->sessions.push_back(s);
  }
  *out = s;
  return TOR_OK;
}

tor_status tor_session_create(tor_ctx* ctx, int n_total, const tor_c128* M, int ld, int kind,
                              tor_session** out) {
  return guarded([&] { return tor_session_create_impl(ctx, n_total, M, ld, kind, out); });
}

void tor_session_destroy(tor_session* s) {
  if (!s) return;
  if (tor_ctx* ctx = s->ctx) {
    // Drop the session's queued requests, then wait until no job in flight
    // reads its matrices any more; only then free them.
    std::unique_lock<std::mutex> lk(ctx->q_mu);
    s->closing = true;
    std::deque<Request*> keep;
    for (Request* r : ctx->queue) {
      if (r->sess == s) {
        r->res = tor_result{};
        r->res.n = r->in.n;
        r->res.status = TOR_ECANCELED;
        r->done = true;
      } else {
        keep.push_back(r);
      }
    }
    ctx->queue.swap(keep);
    ctx->done_cv.notify_all();
    ctx->done_cv.wait(lk, [&] { return s->inflight == 0 && s->blocking == 0; });
    ctx->sessions.erase(std::remove(ctx->sessions.begin(), ctx->sessions.end(), s), ctx->sessions.end());
  }
  cudaSetDevice(s->device);
  s->d_O.release();
  delete s;
}

tor_status tor_session_marginal_matrix(tor_session* s, int j, tor_c128* out, int ld) {
  if (!s || !out || j < 1 || j > s->N || ld < 2 * j) return TOR_EINVAL;
  return guarded([&] {
    const int mj = 2 * j;
    std::vector<tor_c128> pairs((size_t)mj * mj);
    cudaSetDevice(s->device);
    cudaError_t e = cudaMemcpy(pairs.data(), (const double2*)s->d_O.p + s->off[j], pairs.size() * 16,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s->ctx, e, "session matrix copy");
    // resident copies are in pairs order; hand the caller its context's layout
    const bool block = !s->ctx || s->ctx->cfg.layout == TOR_LAYOUT_BLOCK;
    auto dst = [&](int r) { return block ? (r >> 1) + (r & 1) * j : r; };
    for (int a = 0; a < mj; ++a)
      for (int b = 0; b < mj; ++b) out[(size_t)dst(a) * ld + dst(b)] = pairs[(size_t)a * mj + b];
    return TOR_OK;
  });
}

}  // extern "C"

static tor_status marginal_in(tor_session* s, int j, int k, const int* modes, MatIn& in, std::vector<int>& own) {
  if (!s || j < 1 || j > s->N || k < 0 || k > j || (k > 0 && !modes)) return TOR_EINVAL;
  if (k > 64) return TOR_ETOOBIG;
  own.assign(modes, modes + k);
  std::sort(own.begin(), own.end());
  for (int i = 0; i < k; ++i)
    if (own[i] < 0 || own[i] >= j || (i && own[i] == own[i - 1])) return TOR_EINVAL;
  in.n = k;
  in.O = (const tor_c128*)((const double2*)s->d_O.p + s->off[j]);
  in.ld = 2 * j;
  in.n_src = j;
  in.layout = TOR_LAYOUT_PAIRS;
  in.dev = true;
  in.modes = k ? own.data() : nullptr;
  in.real_hint = s->real;
  return TOR_OK;
}

extern "C" {

tor_status tor_eval_marginal(tor_ctx* ctx, tor_session* s, int j, int k, const int* modes, tor_result* out) {
  if (!ctx || !out || !s || s->ctx != ctx) return TOR_EINVAL;
  std::vector<MatIn> ins(1);
  std::vector<int> own;
  tor_status st = marginal_in(s, j, k, modes, ins[0], own);
  if (st != TOR_OK) return st;
  {
    std::lock_guard<std::mutex> lq(ctx->q_mu);
    if (s->closing) return TOR_EINVAL;
    ++s->blocking;
  }
  try {
    std::lock_guard<std::mutex> lk(ctx->run_mu);
    st = run_blocking(ctx, ins, out, nullptr, 0);
  } catch (const std::bad_alloc&) {
    st = TOR_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lq(ctx->q_mu);
    --s->blocking;
  }
  ctx->done_cv.notify_all();
  return st;
}

static tor_status tor_submit_marginal_impl(tor_ctx* ctx, tor_session* s, int j, int k, const int* modes, uint64_t* ticket) {
  if (!ctx || !ticket || !s || s->ctx != ctx) return TOR_EINVAL;
  Request* r = new Request();
  tor_status st = marginal_in(s, j, k, modes, r->in, r->modes);
  if (st != TOR_OK) {
    delete r;
    return st;
  }
  r->in.modes = k ? r->modes.data() : nullptr;
  r->sess = s;
  {
    std::lock_guard<std::mutex> lq(ctx->q_mu);
    if (s->closing) {
      delete r;
      return TOR_EINVAL;
    }
  }
  return enqueue_request(ctx, r, ticket);
}

tor_status tor_submit_marginal(tor_ctx* ctx, tor_session* s, int j, int k, const int* modes, uint64_t* ticket) {
  return guarded([&] { return tor_submit_marginal_impl(ctx, s, j, k, modes, ticket); });
}

// Threshold-detector sampling by the chain rule: for every sample, mode j is
// decided from the two continuations of its clicks S so far on the first
// j + 1 modes, t0 = Tor(O^(j+1)_S) and t1 = Tor(O^(j+1)_{S u {j}}).  One step
// evaluates the distinct marginals of all samples (samples that share their
// clicks so far share them) in batched blocking launches of the context.
constexpr size_t kSampleBatch = 8192;  // marginals per launch
static tor_status tor_sample_impl(tor_ctx* ctx, tor_session* s, int count, int n_modes, const double* uniforms,
                      unsigned char* patterns, double* prob, double* max_dev) {
  if (!ctx || !s || s->ctx != ctx || count < 0 || n_modes < 1 || n_modes > s->N) return TOR_EINVAL;
  if (count > 0 && (!uniforms || !patterns)) return TOR_EINVAL;
  for (long long i = 0; i < (long long)count * n_modes; ++i)
    if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) return TOR_EINVAL;
  {
    std::lock_guard<std::mutex> lq(ctx->q_mu);
    if (s->closing) return TOR_EINVAL;
    ++s->blocking;  // the session's matrices stay until the call returns
  }
  std::vector<std::vector<int>> S(count);       // clicks so far, ascending
  std::vector<long double> pprev(count, 1.0L);  // P(clicks S on the modes decided so far)
  std::vector<int> id0(count), id1(count);
  long double dev = 0.0L;
  tor_status first = TOR_OK;
  try {
    for (int j = 0; j < n_modes && first == TOR_OK; ++j) {
      // the step's distinct marginals: S and S u {j} of every sample
      std::map<std::vector<int>, int> index;
      std::vector<const std::vector<int>*> keys;
      auto add = [&](const std::vector<int>& key) {
        auto it = index.emplace(key, (int)keys.size()).first;
        if (it->second == (int)keys.size()) keys.push_back(&it->first);
        return it->second;
      };
      for (int i = 0; i < count; ++i) {
        id0[i] = add(S[i]);
        S[i].push_back(j);
        id1[i] = add(S[i]);
        S[i].pop_back();
      }
      const size_t U = keys.size();
      std::vector<MatIn> ins(U);
      std::vector<std::vector<int>> own(U);
      for (size_t u = 0; u < U && first == TOR_OK; ++u) {
        const tor_status st = marginal_in(s, j + 1, (int)keys[u]->size(), keys[u]->data(), ins[u], own[u]);
        if (st != TOR_OK) first = st;
        ins[u].modes = own[u].empty() ? nullptr : own[u].data();
      }
      std::vector<tor_result> res(U);
      size_t chunk = kSampleBatch;  // halved while a chunk does not fit the memory budget
      for (size_t b = 0; b < U && first == TOR_OK;) {
        const size_t e = std::min(U, b + chunk);
        std::vector<MatIn> part(ins.begin() + b, ins.begin() + e);
        tor_status st;
        {
          std::lock_guard<std::mutex> lk(ctx->run_mu);
          st = run_blocking(ctx, part, res.data() + b, nullptr, 0, false);  // every step has a new shape: no graphs
        }
        if (st == TOR_ENOMEM && chunk > 1) {
          chunk /= 2;
          continue;
        }
        if (st != TOR_OK) first = st;
        b = e;
      }
      if (first != TOR_OK) break;
      const long double norm = expl(-0.5L * s->logdet_sigma[j + 1]);  // 1 / sqrt(det Sigma_[j+1])
      for (int i = 0; i < count; ++i) {
        const tor_result& r0 = res[id0[i]];
        const tor_result& r1 = res[id1[i]];
        const long double a = ((long double)r0.hi + (long double)r0.lo) * norm;
        const long double b = ((long double)r1.hi + (long double)r1.lo) * norm;
        if (pprev[i] > 0) dev = std::max(dev, fabsl(a + b - pprev[i]) / pprev[i]);
        const long double p1 = b / (a + b);
        const bool click = (long double)uniforms[(size_t)i * n_modes + j] < p1;
        patterns[(size_t)i * n_modes + j] = click ? 1 : 0;
        if (click) S[i].push_back(j);
        pprev[i] = click ? b : a;
      }
    }
  } catch (const std::bad_alloc&) {
    first = TOR_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lq(ctx->q_mu);
    --s->blocking;
  }
  ctx->done_cv.notify_all();
  if (first != TOR_OK) return first;
  if (prob)
    for (int i = 0; i < count; ++i) prob[i] = (double)pprev[i];
  if (max_dev) *max_dev = (double)dev;
  return TOR_OK;
}

tor_status tor_sample(tor_ctx* ctx, tor_session* s, int count, int n_modes, const double* uniforms,
                      unsigned char* patterns, double* prob, double* max_dev) {
  return guarded([&] { return tor_sample_impl(ctx, s, count, n_modes, uniforms, patterns, prob, max_dev); });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuner: for each n, time tor_eval at prefix depths around the built-in
// plan and keep the fastest.  The kernels' control flow depends on n and p
// only, so a fixed synthetic matrix (0.3 I plus a small seeded Hermitian
// perturbation, I - O positive definite) times every input of that size.
// ---------------------------------------------------------------------------
static void synthetic_matrix(int n, std::vector<tor_c128>& O, bool structured, int layout) {
  const int m = 2 * n;
  O.assign((size_t)m * m, tor_c128{0.0, 0.0});
  uint64_t x = 0x9E3779B97F4A7C15ull ^ (uint64_t)n;
  auto next = [&]() {  // splitmix64 -> uniform in [-1, 1)
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-52 - 1.0;
  };
  const double eps = 0.2 / m;
  for (int r = 0; r < m; ++r) {
    O[(size_t)r * m + r] = tor_c128{0.3, 0.0};
    for (int c = 0; c < r; ++c) {
      const double a = eps * next(), b = eps * next();
      O[(size_t)r * m + c] = tor_c128{a, b};
      O[(size_t)c * m + r] = tor_c128{a, -b};
    }
  }
  if (!structured) return;
  // impose [[P, Q], [conj(Q), conj(P)]] (block layout), the form of a physical state
  auto row = [&](int mode, int c) { return layout == TOR_LAYOUT_BLOCK ? mode + c * n : 2 * mode + c; };
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      const tor_c128 aa = O[(size_t)row(j, 0) * m + row(k, 0)];
      O[(size_t)row(j, 1) * m + row(k, 1)] = tor_c128{aa.re, -aa.im};
    }
  for (int j = 0; j < n; ++j)
    for (int k = 0; k <= j; ++k) {  // Q symmetric
      const tor_c128 q = O[(size_t)row(j, 0) * m + row(k, 1)];
      O[(size_t)row(k, 0) * m + row(j, 1)] = q;
      O[(size_t)row(j, 1) * m + row(k, 0)] = tor_c128{q.re, -q.im};
      O[(size_t)row(k, 1) * m + row(j, 0)] = tor_c128{q.re, -q.im};
    }
}

extern "C" {

static tor_status tor_autotune_impl(tor_ctx* ctx, int n_lo, int n_hi, double budget_s, int* chosen) {
  if (!ctx || n_lo < 1 || n_hi > 64 || n_lo > n_hi || budget_s <= 0) return TOR_EINVAL;
  if (ctx->cfg.flags & TOR_IN_DEVICE) return TOR_EINVAL;  // times host inputs
  const double per_n = budget_s / (n_hi - n_lo + 1);
  std::vector<tor_c128> O;
  for (int n = n_lo; n <= n_hi; ++n) {
    synthetic_matrix(n, O, !(ctx->cfg.flags & TOR_COMPLEX_PATH), ctx->cfg.layout);
    int base;
    {
      std::lock_guard<std::mutex> lk(ctx->run_mu);
      ctx->plan[n] = -1;
      base = plan_p(ctx, n);
    }
    std::vector<int> cands;
    for (int d = -4; d <= 4; ++d) {
      const int p = base + d, M = n - p;
      if (p < 0 || M < 1 || M > 22) continue;
      cands.push_back(p);
    }
    double best_t = 1e300;
    int best_p = base;
    const double t_start = now_s();
    for (int p : cands) {
      {
        std::lock_guard<std::mutex> lk(ctx->run_mu);
        ctx->plan[n] = p;
      }
      tor_result r;
      tor_status st = tor_eval(ctx, n, O.data(), 2 * n, &r);  // warm-up (and buffer growth)
      if (st != TOR_OK) return st;
      double tmin = 1e300;
      for (int rep = 0; rep < 3; ++rep) {
        st = tor_eval(ctx, n, O.data(), 2 * n, &r);
        if (st != TOR_OK) return st;
        tmin = std::min(tmin, ctx->last_times[3]);
        if (now_s() - t_start > per_n) break;
      }
      if (tmin < best_t) {
        best_t = tmin;
        best_p = p;
      }
      if (now_s() - t_start > per_n) break;
    }
    {
      std::lock_guard<std::mutex> lk(ctx->run_mu);
      ctx->plan[n] = best_p;
    }
    if (chosen) chosen[n - n_lo] = best_p;
  }
  return TOR_OK;
}

tor_status tor_autotune(tor_ctx* ctx, int n_lo, int n_hi, double budget_s, int* chosen) {
  return guarded([&] { return tor_autotune_impl(ctx, n_lo, n_hi, budget_s, chosen); });
}

// Batch autotuner: coordinate descent over the prefix depths of the batch's
// sizes, largest total work first, timing the whole batch (one tor_eval_batch
// per trial, best of two after a warm-up).  A depth moves while the batch gets
// faster by more than 0.5 %; the search ends when no size improves or the
// budget is spent.
static tor_status tor_autotune_batch_impl(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O,
                                          const int* ld, double budget_s, int* chosen) {
  if (!ctx || count < 1 || !n || !O || budget_s <= 0) return TOR_EINVAL;
  std::map<int, double> work;  // size -> subset terms in the batch
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > 64) return TOR_EINVAL;
    work[n[i]] += std::ldexp(1.0, n[i]);
  }
  std::vector<int> sizes;
  for (const auto& kv : work) sizes.push_back(kv.first);
  std::stable_sort(sizes.begin(), sizes.end(), [&](int a, int b) { return work[a] > work[b]; });
  std::vector<tor_result> res((size_t)count);
  auto time_batch = [&](double* ms) -> tor_status {
    double best = 1e300;
    for (int rep = 0; rep < 3; ++rep) {  // the first pass warms up (and grows buffers)
      tor_status st = tor_eval_batch_impl(ctx, count, n, O, ld, res.data());
      if (st != TOR_OK) return st;
      if (rep) best = std::min(best, ctx->last_times[3]);
    }
    *ms = best;
    return TOR_OK;
  };
  auto set_p = [&](int nn, int p) {
    std::lock_guard<std::mutex> lk(ctx->run_mu);
    ctx->plan[nn] = p;
  };
  auto get_p = [&](int nn) {
    std::lock_guard<std::mutex> lk(ctx->run_mu);
    return plan_p(ctx, nn);
  };
  // Coordinates of the descent, each a set of sizes whose depths move together by
  // one level per step: all sizes at once (a batch often wants every unit larger
  // or smaller, and one size alone moves the batch time less than the threshold),
  // then each size that holds at least a tenth of the work, then the remaining
  // sizes as one group.
  double total = 0;
  for (const auto& kv : work) total += kv.second;
  std::vector<std::vector<int>> coords;
  coords.push_back(sizes);
  std::vector<int> rest;
  for (int nn : sizes) {
    if (work[nn] >= 0.1 * total) coords.push_back({nn});
    else rest.push_back(nn);
  }
  if (!rest.empty() && rest.size() < sizes.size()) coords.push_back(rest);
  auto valid = [&](int nn, int q) { return q >= 0 && q <= std::min(nn - 1, kMaxPrefixDepth) && nn - q <= 22; };
  // moves every size of c by dir (sizes already at a limit stay); false if none moved
  auto shift = [&](const std::vector<int>& c, int dir, std::vector<int>& old) {
    bool any = false;
    old.clear();
    for (int nn : c) {
      const int p = get_p(nn);
      old.push_back(p);
      if (valid(nn, p + dir)) {
        set_p(nn, p + dir);
        any = true;
      }
    }
    return any;
  };
  auto restore = [&](const std::vector<int>& c, const std::vector<int>& old) {
    for (size_t k = 0; k < c.size(); ++k) set_p(c[k], old[k]);
  };
  const double t_end = now_s() + budget_s;
  double best;
  tor_status st = time_batch(&best);
  if (st != TOR_OK) return st;
  std::vector<int> old;
  for (int pass = 0; pass < 3 && now_s() < t_end; ++pass) {
    bool moved = false;
    for (const std::vector<int>& c : coords) {
      if (now_s() >= t_end) break;
      bool improved = false;
      for (int dir : {-1, +1}) {
        while (now_s() < t_end && shift(c, dir, old)) {
          double t;
          st = time_batch(&t);
          if (st != TOR_OK) {
            restore(c, old);
            return st;
          }
          if (t < best * 0.995) {
            best = t;
            improved = moved = true;
          } else {
            restore(c, old);
            break;
          }
        }
        if (improved) break;  // improved in this direction: the other one starts from worse
      }
    }
    if (!moved) break;
  }
  if (chosen)
    for (int i = 0; i < count; ++i) chosen[i] = get_p(n[i]);
  return TOR_OK;
}

tor_status tor_autotune_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                              double budget_s, int* chosen) {
  return guarded([&] { return tor_autotune_batch_impl(ctx, count, n, O, ld, budget_s, chosen); });
}

static tor_status tor_plan_save_impl(tor_ctx* ctx, const char* path) {
  if (!ctx || !path) return TOR_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) return TOR_EINVAL;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->cfg.device) != cudaSuccess) {
    cudaGetLastError();
    snprintf(prop.name, sizeof prop.name, "unknown");
  }
  fprintf(f, "# libtor prefix-depth plan: device %s, %d SMs, %d resident warps\n", prop.name, ctx->sms, ctx->nwarps);
  fprintf(f, "warps %d\n", ctx->nwarps);
  {
    std::lock_guard<std::mutex> lk(ctx->run_mu);
    for (int n = 1; n <= 64; ++n)
      if (ctx->plan[n] >= 0) fprintf(f, "%d %d\n", n, ctx->plan[n]);
  }
  fclose(f);
  return TOR_OK;
}

tor_status tor_plan_save(tor_ctx* ctx, const char* path) {
  return guarded([&] { return tor_plan_save_impl(ctx, path); });
}

static tor_status tor_plan_load_impl(tor_ctx* ctx, const char* path) {
  if (!ctx || !path) return TOR_EINVAL;
  FILE* f = fopen(path, "r");
  if (!f) return TOR_EINVAL;
  char line[256];
  int warps = -1;
  std::vector<std::pair<int, int>> rows;
  while (fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    int a, b;
    if (sscanf(line, "warps %d", &a) == 1) {
      warps = a;
      continue;
    }
    if (sscanf(line, "%d %d", &a, &b) == 2 && a >= 1 && a <= 64 && b >= 0 && b < a) rows.push_back({a, b});
  }
  fclose(f);
  if (warps != ctx->nwarps) return TOR_EINVAL;  // tuned for another device shape
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  for (auto& r : rows) ctx->plan[r.first] = r.second;
  return TOR_OK;
}

tor_status tor_plan_load(tor_ctx* ctx, const char* path) {
  return guarded([&] { return tor_plan_load_impl(ctx, path); });
}

}  // extern "C"
