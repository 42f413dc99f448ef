// tor_host.cu -- host runtime and C ABI of libtor (declared in include/tor.h).
//
// A call to tor_eval / tor_eval_batch runs, on the context's stream:
//   H2D copy of the inputs -> k_intake -> k_units (persistent) -> k_reduce -> D2H
// and then waits for the stream.  tor_submit / tor_poll feed a serving thread
// that batches queued requests into the same pipeline.
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
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max(bytes, cap * 3 / 2);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) { cudaGetLastError(); p = nullptr; return e; }
      want = bytes;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max(bytes, cap * 3 / 2);
    cudaError_t e = cudaMallocHost(&p, want);
    if (e != cudaSuccess) { cudaGetLastError(); p = nullptr; return e; }
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

}  // namespace

struct Request {
  uint64_t ticket;
  int n;
  std::vector<tor_c128> O;  // 2n x 2n, ld = 2n
  tor_result res;
  bool done = false;
};

struct tor_ctx {
  tor_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 0, blocks_per_sm = 0, grid = 0, nwarps = 0;
  int plan[65];
  DevBuf d_O, d_B, d_mats, d_tasks, d_partials, d_flags, d_results, d_lane, d_warp, d_ctl;
  HostBuf h_O, h_mats, h_tasks, h_results, h_ctl;
  int* h_cancel = nullptr;  // host-mapped
  int* d_cancel = nullptr;
  cudaEvent_t ev[5] = {};
  double last_times[4] = {0, 0, 0, 0};
  std::string last_error;
  std::mutex run_mu;
  // serving
  std::mutex q_mu;
  std::condition_variable q_cv, done_cv;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> reqs;
  uint64_t next_ticket = 1;
  std::thread server;
  bool server_started = false, stopping = false;
  size_t queue_limit = 1 << 16;
};

static tor_status cuda_fail(tor_ctx* ctx, cudaError_t e, const char* what) {
  if (ctx) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    ctx->last_error = buf;
  }
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TOR_ENOMEM : TOR_ECUDA;
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

static int default_prefix_depth(int n, int nwarps) {
  if (n <= 8) return 0;
  // aim for >= 8 warp tasks per resident warp (2^(p-5) tasks for p >= 5),
  // with every unit a subtree over M in [8, 20] modes
  int need = 0;
  while ((1ll << need) < 8ll * std::max(nwarps, 1)) ++need;
  int M = n - 5 - need;
  M = std::max(8, std::min(20, M));
  M = std::min(M, n - 1);
  return n - M;
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
    case TOR_ETOOBIG: return "too many modes (n > 64)";
  }
  return "unknown status";
}

const char* tor_last_error(tor_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

tor_status tor_create(const tor_config* cfg, tor_ctx** out) {
  if (!out) return TOR_EINVAL;
  *out = nullptr;
  tor_config c;
  tor_config_default(&c);
  if (cfg) c = *cfg;
  if (c.layout != TOR_LAYOUT_BLOCK && c.layout != TOR_LAYOUT_PAIRS) return TOR_EINVAL;
  if (c.timeout_s < 0) return TOR_EINVAL;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) { cudaGetLastError(); return TOR_ECUDA; }
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
  if ((e = units_blocks_per_sm(&ctx->blocks_per_sm)) != cudaSuccess) return fail(e, "occupancy");
  ctx->blocks_per_sm = std::max(1, ctx->blocks_per_sm);
  ctx->grid = ctx->sms * ctx->blocks_per_sm;
  ctx->nwarps = ctx->grid * (units_block_threads() / 32);
  if (c.stream) {
    ctx->stream = (cudaStream_t)c.stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return fail(e, "stream");
    ctx->own_stream = true;
  }
  for (int i = 0; i < 5; ++i)
    if ((e = cudaEventCreate(&ctx->ev[i])) != cudaSuccess) return fail(e, "event");
  if ((e = cudaHostAlloc((void**)&ctx->h_cancel, sizeof(int), cudaHostAllocMapped)) != cudaSuccess)
    return fail(e, "cancel flag");
  *ctx->h_cancel = 0;
  if ((e = cudaHostGetDevicePointer((void**)&ctx->d_cancel, ctx->h_cancel, 0)) != cudaSuccess)
    return fail(e, "cancel flag map");
  *out = ctx;
  return TOR_OK;
}

void tor_destroy(tor_ctx* ctx) {
  if (!ctx) return;
  {
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    ctx->stopping = true;
  }
  ctx->q_cv.notify_all();
  if (ctx->server.joinable()) ctx->server.join();
  for (auto& kv : ctx->reqs) delete kv.second;
  ctx->reqs.clear();
  cudaSetDevice(ctx->cfg.device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (DevBuf* b : {&ctx->d_O, &ctx->d_B, &ctx->d_mats, &ctx->d_tasks, &ctx->d_partials, &ctx->d_flags,
                    &ctx->d_results, &ctx->d_lane, &ctx->d_warp, &ctx->d_ctl})
    b->release();
  for (HostBuf* b : {&ctx->h_O, &ctx->h_mats, &ctx->h_tasks, &ctx->h_results, &ctx->h_ctl}) b->release();
  if (ctx->h_cancel) cudaFreeHost(ctx->h_cancel);
  for (int i = 0; i < 5; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaGetLastError();
  delete ctx;
}

int tor_plan_prefix_depth(tor_ctx* ctx, int n) {
  if (!ctx || n < 0 || n > 64) return -1;
  if (n == 0) return 0;
  int p;
  if (ctx->plan[n] >= 0) p = ctx->plan[n];
  else if (ctx->cfg.prefix_depth >= 0) p = ctx->cfg.prefix_depth;
  else p = default_prefix_depth(n, ctx->nwarps);
  return std::max(0, std::min(p, n - 1));
}

tor_status tor_set_prefix_depth(tor_ctx* ctx, int n, int p) {
  if (!ctx || n < 1 || n > 64 || p < -1 || p > n - 1) return TOR_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  ctx->plan[n] = p;
  return TOR_OK;
}

tor_status tor_cancel(tor_ctx* ctx) {
  if (!ctx) return TOR_EINVAL;
  __atomic_store_n(ctx->h_cancel, 1, __ATOMIC_SEQ_CST);
  return TOR_OK;
}

tor_status tor_last_times(tor_ctx* ctx, double* times) {
  if (!ctx || !times) return TOR_EINVAL;
  for (int i = 0; i < 4; ++i) times[i] = ctx->last_times[i];
  return TOR_OK;
}

tor_status tor_probe_fp64(int device, double seconds, double* dfma_per_s, double* fp64_tflops) {
  if (!dfma_per_s || !fp64_tflops || seconds <= 0) return TOR_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return TOR_ECUDA; }
  double r = 0;
  cudaError_t e = run_probe_fp64(seconds, &r);
  if (e != cudaSuccess) { cudaGetLastError(); return TOR_ECUDA; }
  *dfma_per_s = r;
  *fp64_tflops = 2.0 * r / 1e12;
  return TOR_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// The evaluation pipeline for a set of matrices.
// ----------------------------------------------------------------------------
static tor_status run_job(tor_ctx* ctx, int count, const int* ns, const tor_c128* const* Os, const int* lds,
                          tor_result* out, bool device_inputs, double* unit_partials, size_t unit_len) {
  CK(cudaSetDevice(ctx->cfg.device), "cudaSetDevice");
  const int layout = ctx->cfg.layout;
  const bool check = !(ctx->cfg.flags & TOR_NO_CHECK);
  tor_status first = TOR_OK;
  auto note = [&](tor_status s) {
    if (first == TOR_OK && s != TOR_OK) first = s;
  };
  // argument checks and trivial cases
  std::vector<int> act;
  act.reserve(count);
  for (int i = 0; i < count; ++i) {
    tor_result& r = out[i];
    memset(&r, 0, sizeof r);
    r.n = ns[i];
    if (ns[i] < 0) r.status = TOR_EINVAL;
    else if (ns[i] > 64) r.status = TOR_ETOOBIG;
    else if (ns[i] == 0) { r.hi = 1.0; r.abs_sum = 1.0; r.status = TOR_OK; }
    else if (!Os[i] || (lds && lds[i] < 2 * ns[i])) r.status = TOR_EINVAL;
    else { act.push_back(i); continue; }
    note(r.status);
  }
  for (int i = 0; i < 4; ++i) ctx->last_times[i] = 0;
  if (act.empty()) return first;
  // job order: by n descending so equal sizes are adjacent
  std::stable_sort(act.begin(), act.end(), [&](int a, int b) { return ns[a] > ns[b]; });
  const int J = (int)act.size();
  std::vector<MatDesc> mats(J);
  std::vector<TaskDesc> tasks;
  long long o_elems = 0, b_elems = 0, parts = 0, lane_e = 0, warp_e = 0;
  for (int j = 0; j < J; ++j) {
    const int n = ns[act[j]];
    const int p = tor_plan_prefix_depth(ctx, n);
    mats[j].n = n;
    mats[j].p = p;
    mats[j].layout = layout;
    mats[j].part_off = parts;
    parts += 1ll << p;
    b_elems += tri(n);
    if (!device_inputs) o_elems += 4ll * n * n;
    lane_e = std::max(lane_e, lane_elems_for(n, p));
    warp_e = std::max(warp_e, warp_elems_for(n, p));
  }
  // tasks, largest subtrees first
  for (int j = 0; j < J;) {
    int k = j;
    while (k < J && mats[k].n == mats[j].n) ++k;
    const int p = mats[j].p, M = mats[j].n - p;
    if (p >= 5) {
      for (int a = j; a < k; ++a)
        for (int t = 0; t < (1 << (p - 5)); ++t) tasks.push_back({a, t, 1, M});
    } else {
      const long long units = (long long)(k - j) << p;
      for (long long t = 0; t * 32 < units; ++t) tasks.push_back({j, (int)t, k - j, M});
    }
    j = k;
  }
  std::stable_sort(tasks.begin(), tasks.end(), [](const TaskDesc& a, const TaskDesc& b) { return a.M > b.M; });
  if (unit_partials && (J != 1 || unit_len < 3ull * (1ull << mats[0].p))) return TOR_EINVAL;
  // device memory
  const size_t lane_bytes = (size_t)ctx->nwarps * 32 * lane_e * sizeof(double2);
  const size_t warp_bytes = (size_t)ctx->nwarps * warp_e * sizeof(double2);
  const size_t need = o_elems * 16 + b_elems * 16 + parts * 32 + J * sizeof(MatDesc) +
                      tasks.size() * sizeof(TaskDesc) + J * (4 + sizeof(ResultRec)) + lane_bytes + warp_bytes + 64;
  if (ctx->cfg.mem_budget && need > ctx->cfg.mem_budget) {
    for (int j = 0; j < J; ++j) out[act[j]].status = TOR_ENOMEM;
    return TOR_ENOMEM;
  }
  CK(ctx->d_O.ensure(std::max<long long>(o_elems, 1) * 16), "alloc O");
  CK(ctx->d_B.ensure(b_elems * 16), "alloc B");
  CK(ctx->d_partials.ensure(parts * 32), "alloc partials");
  CK(ctx->d_mats.ensure(J * sizeof(MatDesc)), "alloc mats");
  CK(ctx->d_tasks.ensure(std::max<size_t>(tasks.size(), 1) * sizeof(TaskDesc)), "alloc tasks");
  CK(ctx->d_flags.ensure(J * sizeof(int)), "alloc flags");
  CK(ctx->d_results.ensure(J * sizeof(ResultRec)), "alloc results");
  CK(ctx->d_lane.ensure(std::max<size_t>(lane_bytes, 16)), "alloc lane scratch");
  CK(ctx->d_warp.ensure(std::max<size_t>(warp_bytes, 16)), "alloc warp scratch");
  CK(ctx->d_ctl.ensure(64), "alloc control");
  CK(ctx->h_O.ensure(std::max<long long>(o_elems, 1) * 16), "pinned O");
  CK(ctx->h_mats.ensure(J * sizeof(MatDesc)), "pinned mats");
  CK(ctx->h_tasks.ensure(std::max<size_t>(tasks.size(), 1) * sizeof(TaskDesc)), "pinned tasks");
  CK(ctx->h_results.ensure(J * sizeof(ResultRec) + (unit_partials ? parts * 32 : 0)), "pinned results");
  // inputs
  long long oo = 0, bo = 0;
  double2* dO = (double2*)ctx->d_O.p;
  double2* dB = (double2*)ctx->d_B.p;
  tor_c128* hO = (tor_c128*)ctx->h_O.p;
  for (int j = 0; j < J; ++j) {
    const int i = act[j], n = ns[i], m = 2 * n;
    const int ld = lds ? lds[i] : m;
    if (device_inputs) {
      mats[j].O = (const double2*)Os[i];
      mats[j].ld = ld;
    } else {
      for (int r = 0; r < m; ++r) memcpy(hO + oo + (long long)r * m, Os[i] + (long long)r * ld, sizeof(tor_c128) * m);
      mats[j].O = dO + oo;
      mats[j].ld = m;
      oo += (long long)m * m;
    }
    mats[j].B = dB + bo;
    bo += tri(n);
  }
  memcpy(ctx->h_mats.p, mats.data(), J * sizeof(MatDesc));
  memcpy(ctx->h_tasks.p, tasks.data(), tasks.size() * sizeof(TaskDesc));
  cudaStream_t s = ctx->stream;
  __atomic_store_n(ctx->h_cancel, 0, __ATOMIC_SEQ_CST);
  CK(cudaEventRecord(ctx->ev[0], s), "event");
  if (!device_inputs) CK(cudaMemcpyAsync(dO, hO, o_elems * 16, cudaMemcpyHostToDevice, s), "H2D O");
  CK(cudaMemcpyAsync(ctx->d_mats.p, ctx->h_mats.p, J * sizeof(MatDesc), cudaMemcpyHostToDevice, s), "H2D mats");
  CK(cudaMemcpyAsync(ctx->d_tasks.p, ctx->h_tasks.p, tasks.size() * sizeof(TaskDesc), cudaMemcpyHostToDevice, s),
     "H2D tasks");
  CK(cudaMemsetAsync(ctx->d_ctl.p, 0, 64, s), "memset control");
  CK(cudaEventRecord(ctx->ev[1], s), "event");
  CK(launch_intake((const MatDesc*)ctx->d_mats.p, J, check ? 1 : 0, (int*)ctx->d_flags.p, s), "k_intake");
  CK(cudaEventRecord(ctx->ev[2], s), "event");
  UnitsParams prm;
  prm.mats = (const MatDesc*)ctx->d_mats.p;
  prm.tasks = (const TaskDesc*)ctx->d_tasks.p;
  prm.ntasks = (int)tasks.size();
  prm.ticket = (unsigned*)ctx->d_ctl.p;
  prm.abort_word = (int*)ctx->d_ctl.p + 1;
  prm.partials = (Part*)ctx->d_partials.p;
  prm.mat_flags = (int*)ctx->d_flags.p;
  prm.lane_scratch = (double2*)ctx->d_lane.p;
  prm.lane_elems = lane_e;
  prm.warp_scratch = (double2*)ctx->d_warp.p;
  prm.warp_elems = warp_e;
  prm.cancel = ctx->d_cancel;
  prm.budget_ns = ctx->cfg.timeout_s > 0 ? (long long)(ctx->cfg.timeout_s * 1e9) : 0;
  CK(launch_units(prm, ctx->grid, s), "k_units");
  CK(cudaEventRecord(ctx->ev[3], s), "event");
  CK(launch_reduce((const MatDesc*)ctx->d_mats.p, J, (const Part*)ctx->d_partials.p, (const int*)ctx->d_flags.p,
                   (ResultRec*)ctx->d_results.p, s),
     "k_reduce");
  CK(cudaEventRecord(ctx->ev[4], s), "event");
  ResultRec* hr = (ResultRec*)ctx->h_results.p;
  CK(cudaMemcpyAsync(hr, ctx->d_results.p, J * sizeof(ResultRec), cudaMemcpyDeviceToHost, s), "D2H results");
  Part* hparts = (Part*)((char*)ctx->h_results.p + J * sizeof(ResultRec));
  if (unit_partials)
    CK(cudaMemcpyAsync(hparts, ctx->d_partials.p, parts * 32, cudaMemcpyDeviceToHost, s), "D2H partials");
  int abort_word = 0;
  CK(cudaMemcpyAsync(&abort_word, (int*)ctx->d_ctl.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H abort");
  CK(cudaStreamSynchronize(s), "kernel execution");
  float ms[4];
  cudaEventElapsedTime(&ms[0], ctx->ev[1], ctx->ev[2]);
  cudaEventElapsedTime(&ms[1], ctx->ev[2], ctx->ev[3]);
  cudaEventElapsedTime(&ms[2], ctx->ev[3], ctx->ev[4]);
  cudaEventElapsedTime(&ms[3], ctx->ev[0], ctx->ev[4]);
  for (int i = 0; i < 4; ++i) ctx->last_times[i] = ms[i];
  for (int j = 0; j < J; ++j) {
    tor_result& r = out[act[j]];
    const ResultRec& q = hr[j];
    r.hi = q.hi;
    r.lo = q.lo;
    r.abs_sum = q.abs_sum;
    r.err_est = 8.0 * r.n * std::ldexp(1.0, -53) * q.abs_sum;
    if (q.flags & FLAG_NONFINITE) r.status = TOR_EINVAL;
    else if (q.flags & FLAG_NOTHERM) r.status = TOR_ENOTHERM;
    else if (abort_word & ABORT_CANCEL) r.status = TOR_ECANCELED;
    else if (abort_word & ABORT_TIMEOUT) r.status = TOR_ETIMEOUT;
    else if (q.flags & FLAG_NOTPD) r.status = TOR_ENOTPD;
    else r.status = TOR_OK;
    note(r.status);
  }
  if (unit_partials) {
    const long long U = 1ll << mats[0].p;
    for (long long u = 0; u < U; ++u) {
      unit_partials[3 * u] = hparts[u].hi;
      unit_partials[3 * u + 1] = hparts[u].lo;
      unit_partials[3 * u + 2] = hparts[u].abs_sum;
    }
  }
  return first;
}

// ----------------------------------------------------------------------------
// Serving thread: drains the submit queue in batches.
// ----------------------------------------------------------------------------
static void server_loop(tor_ctx* ctx) {
  for (;;) {
    std::vector<Request*> batch;
    {
      std::unique_lock<std::mutex> lk(ctx->q_mu);
      ctx->q_cv.wait(lk, [&] { return ctx->stopping || !ctx->queue.empty(); });
      if (ctx->stopping && ctx->queue.empty()) return;
      while (!ctx->queue.empty()) {
        batch.push_back(ctx->queue.front());
        ctx->queue.pop_front();
      }
    }
    std::vector<int> ns(batch.size()), lds(batch.size());
    std::vector<const tor_c128*> Os(batch.size());
    std::vector<tor_result> res(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
      ns[i] = batch[i]->n;
      lds[i] = 2 * batch[i]->n;
      Os[i] = batch[i]->O.data();
    }
    {
      std::lock_guard<std::mutex> lk(ctx->run_mu);
      run_job(ctx, (int)batch.size(), ns.data(), Os.data(), lds.data(), res.data(), false, nullptr, 0);
    }
    {
      std::lock_guard<std::mutex> lk(ctx->q_mu);
      for (size_t i = 0; i < batch.size(); ++i) {
        batch[i]->res = res[i];
        batch[i]->done = true;
      }
    }
    ctx->done_cv.notify_all();
  }
}

extern "C" {

tor_status tor_eval_batch(tor_ctx* ctx, int count, const int* n, const tor_c128* const* O, const int* ld,
                          tor_result* out) {
  if (!ctx || count < 0 || (count > 0 && (!n || !O || !out))) return TOR_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  return run_job(ctx, count, n, O, ld, out, (ctx->cfg.flags & TOR_IN_DEVICE) != 0, nullptr, 0);
}

tor_status tor_eval(tor_ctx* ctx, int n, const tor_c128* O, int ld, tor_result* out) {
  if (!ctx || !out) return TOR_EINVAL;
  const tor_c128* Op[1] = {O};
  int lds[1] = {ld};
  return tor_eval_batch(ctx, 1, &n, Op, lds, out);
}

tor_status tor_eval_units(tor_ctx* ctx, int n, const tor_c128* O, int ld, double* partials, size_t partials_len,
                          tor_result* out) {
  if (!ctx || !out || !partials || n < 1 || n > 64) return TOR_EINVAL;
  const tor_c128* Op[1] = {O};
  int lds[1] = {ld};
  std::lock_guard<std::mutex> lk(ctx->run_mu);
  return run_job(ctx, 1, &n, Op, lds, out, (ctx->cfg.flags & TOR_IN_DEVICE) != 0, partials, partials_len);
}

tor_status tor_submit(tor_ctx* ctx, int n, const tor_c128* O, int ld, uint64_t* ticket) {
  if (!ctx || !ticket || n < 0 || (n > 0 && !O) || ld < 2 * n) return TOR_EINVAL;
  if (n > 64) return TOR_ETOOBIG;
  if (ctx->cfg.flags & TOR_IN_DEVICE) return TOR_EINVAL;  // the queue copies host inputs only
  Request* r = new Request();
  r->n = n;
  r->O.resize((size_t)4 * n * n);
  for (int i = 0; i < 2 * n; ++i) memcpy(r->O.data() + (size_t)i * 2 * n, O + (size_t)i * ld, sizeof(tor_c128) * 2 * n);
  {
    std::lock_guard<std::mutex> lk(ctx->q_mu);
    if (ctx->queue.size() >= ctx->queue_limit) {
      delete r;
      return TOR_EAGAIN;
    }
    r->ticket = ctx->next_ticket++;
    ctx->reqs[r->ticket] = r;
    ctx->queue.push_back(r);
    if (!ctx->server_started) {
      ctx->server = std::thread(server_loop, ctx);
      ctx->server_started = true;
    }
    *ticket = r->ticket;
  }
  ctx->q_cv.notify_one();
  return TOR_OK;
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

}  // extern "C"
