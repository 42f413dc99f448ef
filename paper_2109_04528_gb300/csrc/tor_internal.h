// tor_internal.h -- structures shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tor {

// Partial sum of one unit: Tor contribution as double-double, and sum |term|.
struct __align__(32) Part {
  double hi, lo, abs_sum, pad;
};

// One matrix of a job.
struct MatDesc {
  const double2* O;     // source matrix on the device (row-major, leading dimension ld)
  const int* modes;     // device list of the n source modes to keep, or null (modes 0..n-1)
  double2* B;           // packed lower triangle of B = I - O in pairs order, n(2n+1) entries
                        // (twice as many double2 when ext)
  long long part_off;   // first of this matrix's 2^p unit partials
  long long red_off;    // first of this matrix's reduction leaves (task partials if p >= 5, else unit partials)
  int red_log2;         // log2 of the number of reduction leaves: p - 5 if p >= 5, else p
  int red_chunk0;       // first block of this matrix in the first reduction stage (red_chunk_log2 > 0)
  int n, p, ld, layout;
  int n_src;            // modes of the source matrix (n unless `modes` selects a submatrix)
  int real;             // -1: let k_intake detect the structure; 0: complex; 1: real (x, p) path
  int ext;              // 1: double-double arithmetic (B holds ddc_t / dd_t entries), k_units_ext
  long long red_lo;     // first reduction leaf this job evaluates (tor_eval_range); 0 otherwise
};

// One warp task.  p >= 5: 32 units of matrix `mat` sharing the decisions on
// modes 0..p-6 (= bits of `sub`); lane l takes the decisions on modes
// p-5..p-1 from its 5 bits.  p < 5: units q = 32 sub + lane of the nmat
// consecutive matrices starting at `mat` (same n and p), q < nmat 2^p.
struct TaskDesc {
  int mat, sub, nmat, M;
};

enum { FLAG_NOTPD = 1, FLAG_NOTHERM = 2, FLAG_NONFINITE = 4, FLAG_REAL = 8 };

// Scratch bytes per counted element.  Lane scratch: a warp's region holds a
// real-entry area and a complex-entry area (float64 + complex128, or their
// double-double forms), since the lanes of one task may take either; warp
// (task-node) scratch: one complex entry.
constexpr int kLaneEntryBytes = 8 + 16, kLaneEntryBytesExt = 16 + 32;
constexpr int kWarpEntryBytes = 16, kWarpEntryBytesExt = 32;
enum { ABORT_TIMEOUT = 1, ABORT_CANCEL = 2, ABORT_NOSLOT = 4 };

struct UnitsParams {
  const MatDesc* mats;
  const TaskDesc* tasks;
  int ntasks;
  unsigned* ticket;            // zeroed before the launch
  Part* partials;              // (hi, lo, abs_sum, 0) per unit
  Part* red_leaves;            // per warp task (p >= 5: its 32 units summed by a fixed lane tree) or per unit
  int* mat_flags;              // FLAG_* per matrix
  double2* lane_scratch;       // per warp: 32 * lane_elems * kLaneEntryBytes(Ext) bytes, lane-interleaved
  long long lane_elems;
  double2* warp_scratch;       // per warp: warp_elems * kWarpEntryBytes(Ext) bytes, contiguous
  long long warp_elems;
  const volatile int* cancel;  // host-mapped cancel counter
  int cancel_epoch;            // its value when the job started; a change = stop
  long long budget_ns;         // 0 = no time limit, else counted from the job's start (job_t0)
  unsigned long long* job_t0;  // zeroed before the job; its first warp stores %globaltimer there, so a
                               // launch whose warps start late (one task each) or a relaunch keeps the
                               // job's clock.  Null: each warp counts from its own start
  long long slice_ns;          // > 0: warps stop taking tasks after this long (no abort); the host
                               // relaunches the kernel, which continues from the ticket
  int* abort_word;             // ABORT_* bits set by the kernel
  int ext;                     // 1: launch k_units_ext (double-double entries)
  // Non-persistent launch (one_task = 1): the grid has a warp per task and every
  // warp takes one task, so blocks end all through the job and the block slots
  // they free go to whichever kernel waits -- a higher-priority stream's first.
  // A block then takes its warps' scratch from the slot it claims in slot_pool
  // (one bit per resident block, slot_words words; bits past the resident count
  // are preset) and gives the slot back when it ends.
  int one_task;
  unsigned* slot_pool;
  int slot_words;
};

struct ResultRec {
  double hi, lo, abs_sum;
  int flags, pad;
};

// Two-stage reduction: with more than 256 leaves, the first stage sums aligned
// chunks of 2^red_chunk_log2 leaves (one thread block each, at most 256 chunks
// per matrix), the second the chunk sums; one binary tree over leaf index.
__host__ __device__ constexpr int red_chunk_log2(int red_log2) {
  return red_log2 <= 8 ? 0 : (red_log2 - 8 > 8 ? red_log2 - 8 : 8);
}
__host__ __device__ constexpr long long red_chunks(int red_log2) {
  return red_chunk_log2(red_log2) ? 1ll << (red_log2 - red_chunk_log2(red_log2)) : 0;
}

// ---- scratch sizes, in entries of the arithmetic's own type (one definition
// for the kernels, the host runtime and the allocation-free entry point) ----
__host__ __device__ constexpr int tri_size(int m) { return m * (2 * m + 1); }  // packed entries, m modes
// sum_{k=3}^{m-1} k(2k+1): offset of the lane stack buffer for m modes past the
// root (levels from 3 modes up: a walk with 2-mode register subtrees stores
// 3-mode nodes)
__host__ __device__ constexpr int stack_off(int m) {
  int s = 0;
  for (int k = 3; k < m; ++k) s += tri_size(k);
  return s;
}
// breadth-first fan-out arena of a task: level d's include children (2^d nodes of m0 - d - 1 modes)
__host__ __device__ constexpr int arena_off(int m0, int d) {
  int s = 0;
  for (int e = 0; e < d; ++e) s += (1 << e) * tri_size(m0 - e - 1);
  return s;
}
// pivot-column scratch (one of the two arrays) of a task-node build: 2R entries
// per node being included, R = 2(m - 1) rows; the prefix includes take one node
// of up to n modes, fan-out level d takes its 2^d nodes of m0 - d modes at once
__host__ __device__ constexpr int pivot_cols(int n, int m0) {
  int c = 4 * n;
  for (int d = 0; d < 5; ++d) {
    const int v = (1 << d) * 4 * (m0 - d - 1);
    c = v > c ? v : c;
  }
  return c;
}
// per lane (interleaved by lane): unit root, stack buffers, pivot columns
__host__ __device__ constexpr long long lane_elems_c(int n, int p) {
  return (long long)(p >= 5 ? tri_size(n - p) : tri_size(n)) + stack_off(n - p) + 4LL * n;
}
// per warp (p >= 5 only): task node, fan-out arena, two pivot-column arrays
__host__ __device__ constexpr long long warp_elems_c(int n, int p) {
  return p < 5 ? 0 : (long long)tri_size(n) + arena_off(n - p + 5, 5) + 2LL * pivot_cols(n, n - p + 5);
}
inline long long lane_elems_for(int n, int p) { return lane_elems_c(n, p); }
inline long long warp_elems_for(int n, int p) { return warp_elems_c(n, p); }

cudaError_t launch_intake(const MatDesc* d_mats, int nmats, int check, int* d_flags, cudaStream_t s);
cudaError_t launch_units(const UnitsParams& prm, int grid, cudaStream_t s);
cudaError_t launch_reduce(const MatDesc* d_mats, int nmats, long long nchunks, Part* partials, const int* flags,
                          ResultRec* out, cudaStream_t s);
int units_block_threads();
cudaError_t units_blocks_per_sm(int* blocks, int ext);
cudaError_t run_probe_fp64(double seconds, double* dfma_per_s);

}  // namespace tor
