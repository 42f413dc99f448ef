// tor_noalloc.cu -- tor_eval_noalloc: one Torontonian without any allocation.
//
// Some callers cannot allocate GPU memory while they run: a serving process
// whose device memory is entirely pre-reserved by its own pool (a cudaMalloc
// would fail or fragment that pool), a latency-critical loop where cudaMalloc
// and cudaFree would synchronise the device and stall other streams, or a
// plugin that is only allowed to allocate at start-up.  This entry point needs
// nothing from the allocator: the caller brings the input and the output in
// device memory, and every intermediate buffer (the matrix B, the task list,
// the unit partials, the lane and warp stacks, the control words) lives in one
// file-scope device array that the library image carries.
//
// The array is g_noalloc_scratch below (12 MiB).  Every device that loads the
// library keeps it until the process exits.  All calls share it and it keeps
// whatever the last call left there; the set-up kernel clears the words that
// must start at zero (task ticket, abort word, cancel word, status flags) at the
// start of every call, and every other region is fully overwritten before it is
// read.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads on the same device) race on the array: order them on
// one stream, or wait for one before issuing the next.
//
// Host code cannot use the array's name as a device address (on the host it
// names a shadow variable).  The first call on each device therefore looks up
// the device address with cudaGetSymbolAddress, with that device current, and
// caches it; that first call may load the library's GPU module, so make it
// before any stream capture begins.
#include <mutex>

#include "../../include/tor.h"
#include "tor_internal.h"

namespace tor {
namespace {

constexpr size_t kNoallocBytes = 12u << 20;
constexpr int kNoallocMaxN = TOR_NOALLOC_MAX_N;
constexpr int kNoallocMmax = 6;       // unit subtrees over at most 6 modes
constexpr int kNoallocBlocks = 8;     // 8 blocks x 4 warps = 32 persistent warps
constexpr int kMaxDevices = 64;
constexpr int kLanes = 32;           // lanes per warp (lane stacks are interleaved by lane)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
__host__ __device__ constexpr int plan_p(int n) { return n > kNoallocMmax ? n - kNoallocMmax : 0; }
constexpr long long max_lane_elems() {
  long long m = 0;
  for (int n = 1; n <= kNoallocMaxN; ++n) m = lane_elems_c(n, plan_p(n)) > m ? lane_elems_c(n, plan_p(n)) : m;
  return m;
}
constexpr long long max_warp_elems() {
  long long m = 0;
  for (int n = 1; n <= kNoallocMaxN; ++n) m = warp_elems_c(n, plan_p(n)) > m ? warp_elems_c(n, plan_p(n)) : m;
  return m;
}
constexpr int kWarps = kNoallocBlocks * 4;
constexpr long long kMaxUnits = 1LL << plan_p(kNoallocMaxN);

// byte offsets of the regions inside g_noalloc_scratch
constexpr size_t OFF_CTL = 0;                                            // ticket, abort, cancel (64 B)
constexpr size_t OFF_FLAGS = align256(OFF_CTL + 64);                     // one int
constexpr size_t OFF_MATS = align256(OFF_FLAGS + sizeof(int));           // one MatDesc
constexpr size_t OFF_TASKS = align256(OFF_MATS + sizeof(MatDesc));      // <= 32 TaskDesc
constexpr size_t OFF_RES = align256(OFF_TASKS + 64 * sizeof(TaskDesc));  // one ResultRec
constexpr size_t OFF_B = align256(OFF_RES + sizeof(ResultRec));
constexpr size_t OFF_PARTS = align256(OFF_B + sizeof(double2) * tri_size(kNoallocMaxN));
constexpr size_t OFF_REDS = align256(OFF_PARTS + sizeof(Part) * kMaxUnits);
constexpr size_t OFF_LANE = align256(OFF_REDS + sizeof(Part) * kMaxUnits);
constexpr size_t OFF_WARP = align256(OFF_LANE + (size_t)kLaneEntryBytes * kLanes * max_lane_elems() * kWarps);
constexpr size_t END = align256(OFF_WARP + (size_t)kWarpEntryBytes * max_warp_elems() * kWarps);
static_assert(END <= kNoallocBytes, "no-alloc scratch layout does not fit the static array");

// Fills the job descriptors and clears the control words, writing the array directly.
__global__ void k_noalloc_setup(const double2* O, int n, int ld, int layout) {
  unsigned char* base = g_noalloc_scratch;
  const int p = plan_p(n), M = n - p;
  if (threadIdx.x == 0) {
    int* ctl = (int*)(base + OFF_CTL);
    for (int i = 0; i < 16; ++i) ctl[i] = 0;
    *(int*)(base + OFF_FLAGS) = 0;
    MatDesc* D = (MatDesc*)(base + OFF_MATS);
    D->O = O;
    D->modes = nullptr;
    D->n_src = n;
    D->real = 0;
    D->ext = 0;
    D->B = (double2*)(base + OFF_B);
    D->part_off = 0;
    D->red_off = 0;
    D->red_lo = 0;
    D->red_log2 = p >= 5 ? p - 5 : p;
    D->red_chunk0 = 0;
    D->n = n;
    D->p = p;
    D->ld = ld;
    D->layout = layout;
  }
  TaskDesc* T = (TaskDesc*)(base + OFF_TASKS);
  const int ntasks = p >= 5 ? (1 << (p - 5)) : 1;
  for (int t = threadIdx.x; t < ntasks; t += blockDim.x) {
    if (p >= 5) T[t] = TaskDesc{0, t, 1, M};
    else T[t] = TaskDesc{0, 0, 1, M};
  }
}

// ResultRec + abort word -> the caller's tor_result (same status rules as tor_eval).
__global__ void k_noalloc_finish(tor_result* out, int n) {
  const unsigned char* base = g_noalloc_scratch;
  const ResultRec q = *(const ResultRec*)(base + OFF_RES);
  const int abort_word = ((const int*)(base + OFF_CTL))[1];
  tor_result r;
  r.hi = q.hi;
  r.lo = q.lo;
  r.abs_sum = q.abs_sum;
  r.err_est = 8.0 * n * 1.1102230246251565e-16 * q.abs_sum;
  r.n = n;
  r.path = 0;
  r.reserved = 0;
  if (q.flags & FLAG_NONFINITE) r.status = TOR_EINVAL;
  else if (q.flags & FLAG_NOTHERM) r.status = TOR_ENOTHERM;
  else if (abort_word & ABORT_CANCEL) r.status = TOR_ECANCELED;
  else if (abort_word & ABORT_TIMEOUT) r.status = TOR_ETIMEOUT;
  else if (q.flags & FLAG_NOTPD) r.status = TOR_ENOTPD;
  else r.status = TOR_OK;
  *out = r;
}

std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};

}  // namespace
}  // namespace tor

using namespace tor;

extern "C" tor_status tor_eval_noalloc(int device, int n, const tor_c128* O, int ld, int layout, void* stream,
                                       tor_result* out) {
  if (n < 1 || !O || !out || ld < 2 * n) return n > kNoallocMaxN ? TOR_ETOOBIG : TOR_EINVAL;
  if (n > kNoallocMaxN) return TOR_ETOOBIG;
  if (layout != TOR_LAYOUT_BLOCK && layout != TOR_LAYOUT_PAIRS) return TOR_EINVAL;
  if (device < 0 || device >= kMaxDevices) return TOR_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return TOR_ECUDA; }
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return TOR_EINVAL; }
  tor_status st = TOR_OK;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) { cudaGetLastError(); st = TOR_ECUDA; }
      else g_addr[device] = (unsigned char*)p;
    }
    base = g_addr[device];
  }
  if (st == TOR_OK) {
    cudaStream_t s = (cudaStream_t)stream;
    const int p = plan_p(n);
    k_noalloc_setup<<<1, 32, 0, s>>>((const double2*)O, n, ld, layout);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_intake((const MatDesc*)(base + OFF_MATS), 1, 1, (int*)(base + OFF_FLAGS), s);
    if (e == cudaSuccess) {
      UnitsParams prm{};
      prm.mats = (const MatDesc*)(base + OFF_MATS);
      prm.tasks = (const TaskDesc*)(base + OFF_TASKS);
      prm.ntasks = p >= 5 ? (1 << (p - 5)) : 1;
      prm.ticket = (unsigned*)(base + OFF_CTL);
      prm.abort_word = (int*)(base + OFF_CTL) + 1;
      prm.cancel = (const volatile int*)(base + OFF_CTL) + 2;
      prm.cancel_epoch = 0;
      prm.budget_ns = 0;
      prm.slice_ns = 0;
      prm.partials = (Part*)(base + OFF_PARTS);
      prm.red_leaves = (Part*)(base + OFF_REDS);
      prm.mat_flags = (int*)(base + OFF_FLAGS);
      prm.lane_scratch = (double2*)(base + OFF_LANE);
      prm.lane_elems = max_lane_elems();
      prm.warp_scratch = (double2*)(base + OFF_WARP);
      prm.warp_elems = max_warp_elems();
      e = launch_units(prm, kNoallocBlocks, s);
    }
    if (e == cudaSuccess)
      e = launch_reduce((const MatDesc*)(base + OFF_MATS), 1, red_chunks(p >= 5 ? p - 5 : p), (Part*)(base + OFF_REDS),
                        (const int*)(base + OFF_FLAGS), (ResultRec*)(base + OFF_RES), s);
    if (e == cudaSuccess) {
      k_noalloc_finish<<<1, 1, 0, s>>>(out, n);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) { cudaGetLastError(); st = TOR_ECUDA; }
  }
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
