// tor_kernels.cu -- the GPU path of the subset-tree Torontonian.
//
//   k_intake  : B = I - O in pairs order, packed lower triangle (paper Sec. 1
//               Eq. A and the row order of Sec. 2), or its real (x, p) form V
//               for structured O; Hermitian / finite checks.
//   k_units   : persistent warps; each warp task evaluates 32 units (prefix
//               subtrees) of the tree of Algorithm 2, one unit per lane.
//   k_units_ext : the same in double-double arithmetic (extended precision).
//   k_reduce_chunks, k_reduce : fixed-shape binary tree over each matrix's
//               task partials (each already a fixed lane tree over 32 units), in
//               double-double; large matrices in two stages.
//   k_probe   : FP64 FMA throughput probe (the roofline's denominator).
#include "tor_dd.cuh"
#include "tor_device.cuh"
#include "tor_internal.h"

namespace tor {

// ------------------------------------------------------------------ helpers
// (scratch sizes: tri_size, stack_off, arena_off, pivot_cols in tor_internal.h)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ includes

// Include the first mode of node (src, o rows offset) with m modes; write the
// child (m-1 modes) to (dst, dst_o).  In place when dst == src and
// dst_o == o + 2.  xs/ys: scratch of 2(m-1) elements each.  Returns rho.
template <class S>
__device__ __noinline__ typename S::Re lane_include_mem(const LaneMem<S> L, int src, int o, int m, int dst,
                                                        int dst_o, int xs, int ys, bool& bad) {
  using T = typename S::T;
  const Pivot<S> pv = make_pivot<S>(L.ldd(src + P(o, o)), L.ld(src + P(o + 1, o)), L.ldd(src + P(o + 1, o + 1)));
  bad |= !pv.ok;
  const int R = 2 * (m - 1);
  for (int r = 0; r < R; ++r) {
    const T x = L.ld(src + P(o + 2 + r, o));
    L.st(xs + r, x);
    L.st(ys + r, S::reduce_col(x, L.ld(src + P(o + 2 + r, o + 1)), pv.cl));
  }
  for (int i = 0; i < R; ++i) {
    const T xi = L.ld(xs + i), yi = L.ld(ys + i);
    const T xt = S::scale(xi, pv.ia), yt = S::scale(yi, pv.id2);
    const int srow = src + P(o + 2 + i, o + 2);
    const int drow = dst + P(dst_o + i, dst_o);
#pragma unroll(S::kUnrollK)
    for (int k = 0; k < i; ++k) L.st(drow + k, S::rank2_off(L.ld(srow + k), xt, L.ld(xs + k), yt, L.ld(ys + k)));
    L.st(drow + i, S::diag(S::rank2_diag(L.ldd(srow + i), xt, xi, yt, yi)));
  }
  return pv.rho;
}

// Copies the node (src, o) with m modes (packed, not interleaved) into the
// lane's stack at element 0, 8 entries per pass: their loads are issued before
// their stores, so they overlap.  Used for entries wider than 8 bytes (complex
// and double-double), where it measured faster; the FP64 real path keeps the
// plain loop, which needs fewer registers in the caller.
template <class S>
__device__ __noinline__ void lane_copy_node(const LaneMem<S> L, const typename S::T* src, int o, int m) {
  using T = typename S::T;
  const int tot = tri_size(m);
  int i = 0, k = 0;
  for (int e0 = 0; e0 < tot; e0 += 8) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (e0 + u < tot) v[u] = src[P(i + o, k + o)];
      if (++k > i) {
        k = 0;
        ++i;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (e0 + u < tot) L.st(e0 + u, v[u]);
  }
}

// Cooperative include: the lanes of a warp split the entries of nodes stored
// contiguously (packed, not interleaved).  Used for the shared upper part of
// the tree, where nodes are large.  The warp is divided into groups of gs
// lanes (gs = 32 >> d, li = lane within its group); every group includes the
// first mode of its own node (src, o) with m modes -- all nodes of one
// breadth-first level at once, so the pivot costs one pass per level, not one
// per node.  All lanes of a group compute its pivot; xs / ys are the group's
// pivot-column scratch (2R entries each); the call ends with __syncwarp so the
// children are visible to every lane.  In place when dst == src and
// dst_o == o + 2.  Each entry gets the same arithmetic whatever the grouping.
template <class S>
__device__ __noinline__ typename S::Re coop_include(const typename S::T* src, int o, int m, typename S::T* dst,
                                                    int dst_o, typename S::T* xs, typename S::T* ys, int gs, int li,
                                                    bool& bad) {
  using T = typename S::T;
  const Pivot<S> pv = make_pivot<S>(S::re(src[P(o, o)]), src[P(o + 1, o)], S::re(src[P(o + 1, o + 1)]));
  bad |= !pv.ok;
  const int R = 2 * (m - 1);
  // xs[0..R) = x, xs[R..2R) = x / d1; ys[0..R) = y', ys[R..2R) = y' / d2
  for (int r = li; r < R; r += gs) {
    const T x = src[P(o + 2 + r, o)];
    const T y = S::reduce_col(x, src[P(o + 2 + r, o + 1)], pv.cl);
    xs[r] = x;
    xs[R + r] = S::scale(x, pv.ia);
    ys[r] = y;
    ys[R + r] = S::scale(y, pv.id2);
  }
  __syncwarp();
  const int tot = (R * (R + 1)) / 2;
  int i = 0, k = li;
  while (k > i) {
    k -= i + 1;
    ++i;
  }
  for (int e = li; e < tot; e += gs) {
    const T xt = xs[R + i], yt = ys[R + i];
    const T sv = src[P(o + 2 + i, o + 2 + k)];
    T out;
    if (k < i) out = S::rank2_off(sv, xt, xs[k], yt, ys[k]);
    else out = S::diag(S::rank2_diag(S::re(sv), xt, xs[i], yt, ys[i]));
    dst[P(dst_o + i, dst_o + k)] = out;
    k += gs;
    while (k > i) {
      k -= i + 1;
      ++i;
    }
  }
  __syncwarp();
  return pv.rho;
}

// ------------------------------------------------------------------ lane DFS

// Walks the subtree below a lane's unit root (a view (root, root_o) with M
// modes, phi_root, incl_root modes included so far out of n - M decided) and
// adds its 2^M signed terms to acc, their magnitudes to ab.
//
// Levels are indexed by the number of modes m of the node.  With K =
// S::kRegModes, the binary counter c enumerates the K-mode nodes in
// depth-first order: bit t of c is the decision (1 = include) taken at the
// level with K + 1 + t modes.  Going from c-1 to c flips bit t = ctz(c) from
// 0 to 1 and every lower bit back to 0: one include at level K + 1 + t, then
// excludes.  Included children are
// written to the buffer of their own size (buffer m holds an m-mode matrix),
// excluded children are views of their parent, so a node is never
// overwritten while a pending include still needs it.  The nodes of
// K = S::kRegModes modes (3, or 4 for the FP64 real type) and everything
// below them live in registers.
template <class S>
__device__ __noinline__ void lane_dfs(const LaneMem<S> L, int root, int root_o, int M, int n,
                                      typename S::Re phi_root, int incl_root, int buf4, int xs, int ys,
                                      typename S::Acc& acc, double& ab, bool& bad) {
  using Re = typename S::Re;
  constexpr int K = S::kRegModes;  // register-resident subtree: K modes, 2K x 2K
  if (M <= K) {
    const int excl_above = (n - M) - incl_root;
    Re v{};
    double a = 0.0;
    if (M == 1) {
      HM<S, 2> R2;
      lane_load_node<S, 2>(L, root, root_o, R2);
      Subtree<S, 2>::run(R2, phi_root, v, a, bad);
    } else if (M == 2) {
      HM<S, 4> R4;
      lane_load_node<S, 4>(L, root, root_o, R4);
      Subtree<S, 4>::run(R4, phi_root, v, a, bad);
    } else if (M == 3) {
      HM<S, 6> R6;
      lane_load_node<S, 6>(L, root, root_o, R6);
      Subtree<S, 6>::run(R6, phi_root, v, a, bad);
    } else {
      if constexpr (K >= 4) {
        HM<S, 8> R8;
        lane_load_node<S, 8>(L, root, root_o, R8);
        Subtree<S, 8>::run(R8, phi_root, v, a, bad);
      }
    }
    if (excl_above & 1) v = S::neg(v);
    acc.add(v);
    ab += a;
    return;
  }
  int nb[65], nof[65];
  Re ph[65];
  nb[M] = root;
  nof[M] = root_o;
  ph[M] = phi_root;
  for (int m = M - 1; m > K; --m) {
    nb[m] = nb[m + 1];
    nof[m] = nof[m + 1] + 2;
    ph[m] = ph[m + 1];
  }
  const unsigned long long count = 1ull << (M - K);
  for (unsigned long long c = 0; c < count; ++c) {
    if (c != 0 && (c & 1ull) == 0) {
      const int mi = K + 1 + __ffsll((long long)c) - 1;
      const int dst = buf4 + stack_off(mi - 1);
      const Re rho = lane_include_mem<S>(L, nb[mi], nof[mi], mi, dst, 0, xs, ys, bad);
      nb[mi - 1] = dst;
      nof[mi - 1] = 0;
      ph[mi - 1] = S::mul(ph[mi], rho);
      for (int m = mi - 2; m > K; --m) {
        nb[m] = nb[m + 1];
        nof[m] = nof[m + 1] + 2;
        ph[m] = ph[m + 1];
      }
    }
    HM<S, 2 * K> RK;
    Re phiK;
    if (c & 1ull) {
      phiK = S::mul(ph[K + 1], lane_include_reg<S, 2 * K>(L, nb[K + 1], nof[K + 1], RK, bad));
    } else {
      lane_load_trail<S, 2 * K>(L, nb[K + 1], nof[K + 1], RK);
      phiK = ph[K + 1];
    }
    Re v;
    double a;
    Subtree<S, 2 * K>::run(RK, phiK, v, a, bad);
    const int excl_above = (n - K) - (incl_root + __popcll(c));
    if (excl_above & 1) v = S::neg(v);
    acc.add(v);
    ab += a;
  }
}

// ------------------------------------------------------------------ kernels

// Source row of component c (0 = a, 1 = a^dag) of job mode t of matrix D.
__device__ __forceinline__ int src_row(const MatDesc& D, int t, int c) {
  const int m = D.modes ? D.modes[t] : t;
  return D.layout == 0 ? m + c * D.n_src : 2 * m + c;
}

// One block per matrix.  Pass 1 checks every entry: finite; Hermitian,
// max |O_rs - conj(O_sr)| <= 1e-12 max |O|; and structured,
// O(a_j^dag, a_k^dag) = conj O(a_j, a_k), O(a_j^dag, a_k) = conj O(a_j, a_k^dag)
// within the same tolerance (the form of every physical Gaussian state), all
// in the max(|Re|, |Im|) norm of each entry (exactly, with D.ext).  Pass 2 writes, in packed lower
// triangle, either the complex B = I - O in pairs order or, for a structured
// O (unless D.real == 0), the real V = U^H B U in (x_1, p_1, x_2, p_2, ...)
// order:
//   V(x_j, x_k) = Re A + Re C,  V(x_j, p_k) = Im C - Im A,
//   V(p_j, x_k) = Im A + Im C,  V(p_j, p_k) = Re A - Re C,
// with A = B(a_j, a_k) and C = B(a_j, a_k^dag).  flags gets FLAG_REAL when V
// was written.  With D.ext the entries are written as double-doubles (ddc_t or
// dd_t): 1 - O_ii exactly, and each entry of V to within 3 u^2.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;  // |v| patterns >= this: inf or NaN
// max of two |v| patterns that ignores NaN (patterns above infinity), as fmax does
__device__ __forceinline__ unsigned long long umax(unsigned long long a, unsigned long long b) {
  if (a > kInfBits) return b;
  if (b > kInfBits) return a;
  return a > b ? a : b;
}

__global__ void __launch_bounds__(256) k_intake(const MatDesc* __restrict__ mats, int check, int* __restrict__ flags) {
  const MatDesc D = mats[blockIdx.x];
  const int n = D.n, tot = n * (2 * n + 1);
  __shared__ unsigned long long s_max, s_dev, s_sdev;
  __shared__ int s_bad, s_real;
  if (threadIdx.x == 0) {
    s_max = 0;
    s_dev = 0;
    s_sdev = 0;
    s_bad = 0;
  }
  __syncthreads();
  // Maxima of |.| kept as bit patterns: with the sign bit cleared, doubles
  // order like their patterns, so the comparisons run on the integer pipe, not
  // the FP64 one; NaNs are skipped like fmax skips them (a non-finite entry is
  // flagged on its own).  Four entries per pass, their loads issued together.
  unsigned long long mx = 0, dev = 0, sdev = 0;
  int bad = 0;
  const int full = 4 * n * n;
  constexpr int kI = 4;
  for (int e0 = threadIdx.x; e0 < full; e0 += kI * blockDim.x) {
    double2 a[kI], b[kI], c[kI];
#pragma unroll
    for (int u = 0; u < kI; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < full) {
        const int r = e / (2 * n), s = e % (2 * n);  // full matrix, pairs order
        a[u] = D.O[(size_t)src_row(D, r >> 1, r & 1) * D.ld + src_row(D, s >> 1, s & 1)];
        b[u] = D.O[(size_t)src_row(D, s >> 1, s & 1) * D.ld + src_row(D, r >> 1, r & 1)];
        // structure: the entry of the opposite components of the same modes
        c[u] = D.O[(size_t)src_row(D, r >> 1, 1 - (r & 1)) * D.ld + src_row(D, s >> 1, 1 - (s & 1))];
      }
    }
#pragma unroll
    for (int u = 0; u < kI; ++u) {
      if (e0 + u * blockDim.x < full) {
        const unsigned long long ax = abs_bits(a[u].x), ay = abs_bits(a[u].y);
        if (ax >= kInfBits || ay >= kInfBits) bad = 1;
        mx = umax(mx, umax(ax, ay));
        dev = umax(dev, umax(abs_bits(a[u].x - b[u].x), abs_bits(a[u].y + b[u].y)));
        sdev = umax(sdev, umax(abs_bits(a[u].x - c[u].x), abs_bits(a[u].y + c[u].y)));
      }
    }
  }
  atomicMax(&s_max, mx);
  atomicMax(&s_dev, dev);
  atomicMax(&s_sdev, sdev);
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double gmax = __longlong_as_double((long long)s_max);
    const double gdev = __longlong_as_double((long long)s_dev), gsdev = __longlong_as_double((long long)s_sdev);
    int f = 0;
    if (s_bad) f |= FLAG_NONFINITE;
    if (check && !(gdev <= 1e-12 * gmax)) f |= FLAG_NOTHERM;
    // FP64 arithmetic takes structure within 1e-12 max|O| (the real form uses
    // one half of the blocks, a change far below its rounding); double-double
    // arithmetic only exact structure, and ignores a caller's hint.
    int real;
    if (D.real == 0) real = 0;
    else if (D.ext) real = !s_bad && gsdev == 0.0;
    else real = D.real == 1 ? 1 : (!s_bad && gsdev <= 1e-12 * gmax);
    if (real) f |= FLAG_REAL;
    s_real = real;
    flags[blockIdx.x] = f;
  }
  __syncthreads();
  const int real = s_real;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (P(r, 0) > e) --r;
    while (P(r + 1, 0) <= e) ++r;
    const int s = e - P(r, 0);
    if (!real) {
      const double2 a = D.O[(size_t)src_row(D, r >> 1, r & 1) * D.ld + src_row(D, s >> 1, s & 1)];
      if (!D.ext) {
        D.B[e] = r == s ? make_double2(1.0 - a.x, 0.0) : make_double2(-a.x, -a.y);
      } else {
        ddc_t v{dd_t{-a.x, 0.0}, dd_t{-a.y, 0.0}};
        if (r == s) {
          two_sum(1.0, -a.x, v.x.h, v.x.l);
          v.y = dd_t{0.0, 0.0};
        }
        ((ddc_t*)D.B)[e] = v;
      }
    } else {
      const int j = r >> 1, k = s >> 1;
      const double2 oa = D.O[(size_t)src_row(D, j, 0) * D.ld + src_row(D, k, 0)];
      const double2 oc = D.O[(size_t)src_row(D, j, 0) * D.ld + src_row(D, k, 1)];
      if (!D.ext) {
        const double Are = (j == k ? 1.0 : 0.0) - oa.x, Aim = -oa.y, Cre = -oc.x, Cim = -oc.y;
        double v;
        if ((r & 1) == 0) v = (s & 1) == 0 ? Are + Cre : Cim - Aim;
        else v = (s & 1) == 0 ? Aim + Cim : Are - Cre;
        ((double*)D.B)[e] = v;
      } else {
        dd_t Are{-oa.x, 0.0};
        if (j == k) two_sum(1.0, -oa.x, Are.h, Are.l);
        const dd_t Aim{-oa.y, 0.0}, Cre{-oc.x, 0.0}, Cim{-oc.y, 0.0};
        dd_t v;
        if ((r & 1) == 0) v = (s & 1) == 0 ? dd_add(Are, Cre) : dd_add(Cim, dd_neg(Aim));
        else v = (s & 1) == 0 ? dd_add(Aim, Cim) : dd_add(Are, dd_neg(Cre));
        ((dd_t*)D.B)[e] = v;
      }
    }
  }
}

// Unit partial (hi, lo, abs).  For p < 5 the unit partials are the reduction leaves.
template <class S>
__device__ __forceinline__ Part write_partial(const UnitsParams& prm, const MatDesc& D, int mat, long long u,
                                              const typename S::Acc& acc, double ab, bool bad) {
  double hi, lo;
  S::acc_out(acc, hi, lo);
  const Part v{hi, lo, ab, 0.0};
  prm.partials[D.part_off + u] = v;
  if (D.p < 5) prm.red_leaves[D.red_off + u] = v;
  if (bad) atomicOr(&prm.mat_flags[mat], FLAG_NOTPD);
  return v;
}

// Sum of the 32 lanes' unit partials of a task by a fixed binary tree over lane
// index.  Each level adds the high parts exactly (two_sum) and the low parts
// with the rounding error in FP64, left unnormalised; one two_sum at the end
// normalises.  8 FP64 instructions per level instead of the 20 of a normalised
// double-word sum, and each level costs a full warp instruction however few
// lanes add.  Error: the low parts stay below ~5u sum|hi|, so their roundings
// add below ~25u^2 sum|partial| (u = 2^-53), far inside both tolerances.
__device__ __forceinline__ void write_task_partial(const UnitsParams& prm, const MatDesc& D, int sub, Part v,
                                                   int lane) {
  double h = v.hi, l = v.lo, a = v.abs_sum;
#pragma unroll
  for (int off = 1; off < kWarp; off <<= 1) {
    const double h2 = __shfl_down_sync(0xffffffffu, h, off);
    const double l2 = __shfl_down_sync(0xffffffffu, l, off);
    const double a2 = __shfl_down_sync(0xffffffffu, a, off);
    if ((lane & (2 * off - 1)) == 0) {
      double s, e;
      two_sum(h, h2, s, e);
      h = s;
      l = __dadd_rn(__dadd_rn(l, l2), e);
      a = a + a2;
    }
  }
  if (lane == 0) {
    double hh, ll;
    two_sum(h, l, hh, ll);
    prm.red_leaves[D.red_off + (sub - D.red_lo)] = Part{hh, ll, a, 0.0};
  }
}

// p >= 5: the warp builds the task node (depth p - 5) cooperatively, fans it
// out breadth-first over 5 more levels into 32 unit roots, one per lane, and
// each lane walks its own subtree.
template <class S>
__device__ void run_task_shared(const UnitsParams& prm, const TaskDesc T, int lane, char* lreg, char* wreg) {
  using E = typename S::T;
  using Re = typename S::Re;
  const LaneMem<S> L{(E*)lreg + lane};
  E* WS = (E*)wreg;
  const MatDesc D = prm.mats[T.mat];
  const int n = D.n, p = D.p, M = n - p, m0 = M + 5;
  E* SB = WS;
  E* arena = WS + tri_size(n);
  E* xsw = arena + arena_off(m0, 5);
  E* ysw = xsw + pivot_cols(n, m0);
  bool bad = false;
  // 1. task node: decisions on modes 0..p-6 are the bits of T.sub (same for all lanes)
  const E* src = (const E*)D.B;
  int o = 0, incl = 0;
  Re phi = S::one();
  bool own = false;
  for (int j = 0; j < p - 5; ++j) {
    if ((T.sub >> j) & 1) {
      Re rho;
      if (!own) {
        rho = coop_include<S>(src, o, n - j, SB, 0, xsw, ysw, kWarp, lane, bad);
        src = SB;
        o = 0;
        own = true;
      } else {
        rho = coop_include<S>(SB, o, n - j, SB, o + 2, xsw, ysw, kWarp, lane, bad);
        o += 2;
      }
      phi = S::mul(phi, rho);
      ++incl;
    } else {
      o += 2;
    }
  }
  // 2. breadth-first fan-out: lane q holds level-d node q (bit e of q = decision on mode p-5+e).
  //    Level d includes all its 2^d nodes at once: lane group g (gs = 32 >> d lanes) takes node g,
  //    writes its include child to the arena, and lane nodes + g takes that child.
  const E* nptr = src;
  int no = o, nincl = incl;
  Re nphi = phi;
  for (int d = 0; d < 5; ++d) {
    const int nodes = 1 << d, m = m0 - d, gs = kWarp >> d, R = 2 * (m - 1);
    const int g = lane / gs, li = lane % gs;
    const E* gp = (const E*)__shfl_sync(0xffffffffu, (unsigned long long)nptr, g);
    const int go = __shfl_sync(0xffffffffu, no, g);
    const Re rho = coop_include<S>(gp, go, m, arena + arena_off(m0, d) + g * tri_size(m - 1), 0, xsw + g * 2 * R,
                                   ysw + g * 2 * R, gs, li, bad);
    // the lane taking node q's include child reads q's phi, its count and rho (held by group q)
    const int q = lane >= nodes && lane < 2 * nodes ? lane - nodes : 0;
    const Re qphi = S::shfl(nphi, q);
    const int qincl = __shfl_sync(0xffffffffu, nincl, q);
    const Re qrho = S::shfl(rho, q * gs);
    if (lane >= nodes && lane < 2 * nodes) {
      nptr = arena + arena_off(m0, d) + q * tri_size(m - 1);
      no = 0;
      nphi = S::mul(qphi, qrho);
      nincl = qincl + 1;
    }
    if (lane < nodes) no += 2;
  }
  // 3. copy the lane's unit root into its private stack
  const int root_sz = tri_size(M);
  if constexpr (sizeof(E) > 8) {
    lane_copy_node<S>(L, nptr, no, M);
  } else {
    const int RR = 2 * M;
    for (int i = 0; i < RR; ++i)
      for (int k = 0; k <= i; ++k) L.st(P(i, k), nptr[P(i + no, k + no)]);
  }
  const int xs = root_sz + stack_off(M), ys = xs + 2 * n;
  typename S::Acc acc = S::acc0();
  double ab = 0.0;
  lane_dfs<S>(L, 0, 0, M, n, nphi, nincl, root_sz, xs, ys, acc, ab, bad);
  const long long u = (long long)T.sub | ((long long)lane << (p - 5));
  const Part v = write_partial<S>(prm, D, T.mat, u, acc, ab, bad);
  write_task_partial(prm, D, T.sub, v, lane);
}

// p < 5: lanes take units of up to 32 small matrices of one size and type;
// each lane builds its own root from B by in-place includes.
template <class S>
__device__ void run_task_lanes(const UnitsParams& prm, const TaskDesc T, int lane, char* lreg) {
  using E = typename S::T;
  const LaneMem<S> L{(E*)lreg + lane};
  const int p = prm.mats[T.mat].p;
  const long long q = (long long)T.sub * kWarp + lane;
  if (q >= ((long long)T.nmat << p)) return;
  const int mat = T.mat + (int)(q >> p);
  const MatDesc D = prm.mats[mat];
  const int n = D.n, M = n - p;
  const long long u = q & ((1ll << p) - 1);
  const int root_sz = tri_size(n);
  const E* B = (const E*)D.B;
  if constexpr (sizeof(E) > 8) {
    lane_copy_node<S>(L, B, 0, n);
  } else {
    for (int e = 0; e < root_sz; ++e) L.st(e, B[e]);
  }
  const int xs = root_sz + stack_off(M), ys = xs + 2 * n;
  bool bad = false;
  int o = 0, incl = 0;
  typename S::Re phi = S::one();
  for (int j = 0; j < p; ++j) {
    if ((u >> j) & 1) {
      phi = S::mul(phi, lane_include_mem<S>(L, 0, o, n - j, 0, o + 2, xs, ys, bad));
      ++incl;
    }
    o += 2;
  }
  typename S::Acc acc = S::acc0();
  double ab = 0.0;
  lane_dfs<S>(L, 0, o, M, n, phi, incl, root_sz, xs, ys, acc, ab, bad);
  write_partial<S>(prm, D, mat, u, acc, ab, bad);
}

// p < 5: each lane takes the arithmetic of its own matrix (the lanes of a task
// share n and p; they diverge only if the batch mixes structured and general inputs).
template <class SR, class SC>
__device__ __forceinline__ void run_task_lanes_any(const UnitsParams& prm, const TaskDesc T, int lane, char* lreg_r,
                                                   char* lreg_c) {
  const int p = prm.mats[T.mat].p;
  const long long q = (long long)T.sub * kWarp + lane;
  if (q >= ((long long)T.nmat << p)) return;
  const int mat = T.mat + (int)(q >> p);
  if (prm.mat_flags[mat] & FLAG_REAL) run_task_lanes<SR>(prm, T, lane, lreg_r);
  else run_task_lanes<SC>(prm, T, lane, lreg_c);
}

constexpr int kUnitsThreads = 128;

// The persistent task loop, in the arithmetic of SR (structured inputs, real
// (x, p) basis) and SC (general inputs).  A warp's lane scratch holds an SR
// area and an SC area side by side, each lane-interleaved in its own entry
// size, because the lanes of one task (p < 5) may take different arithmetic;
// its task-node scratch (p >= 5: one matrix, one arithmetic) is sized for SC.
// Claims a free bit of the slot pool (one bit per resident block of a
// non-persistent launch): the slot whose scratch the block's warps use.  At most
// that many blocks of the launch are resident at once, so a free bit exists;
// the search is bounded all the same (-1 if it finds none).
__device__ __noinline__ int claim_slot(unsigned* pool, int words, int start) {
  // a slot released by a block that has just ended may not be visible yet:
  // pass over the pool up to 4096 times, pausing between passes (~ms in all)
  for (int it = 0; it < 4096 * words; ++it) {
    if (it && it % words == 0) __nanosleep(256);
    const int w = (start + it) % words;
    unsigned cur = atomicOr(&pool[w], 0u);
    for (int tries = 0; tries < 33 && cur != 0xffffffffu; ++tries) {
      const int b = __ffs(~cur) - 1;
      const unsigned old = atomicOr(&pool[w], 1u << b);
      if (!(old & (1u << b))) return w * 32 + b;
      cur = old | (1u << b);
    }
  }
  return -1;
}

template <class SR, class SC>
__device__ __forceinline__ void units_loop(const UnitsParams& prm) {
  using TR = typename SR::T;
  using TC = typename SC::T;
  const int lane = threadIdx.x & (kWarp - 1);
  __shared__ int s_slot;
  long long blk = blockIdx.x;
  if (prm.one_task) {
    if (threadIdx.x == 0) {
      s_slot = claim_slot(prm.slot_pool, prm.slot_words, (int)(blockIdx.x % prm.slot_words));
      __threadfence();  // the previous holder's stores (fenced before its release) precede ours
    }
    __syncthreads();
    if (s_slot < 0) {  // no slot (cannot happen within the occupancy bound): the job reports a failure
      if (threadIdx.x == 0) atomicOr(prm.abort_word, ABORT_NOSLOT);
      return;
    }
    blk = s_slot;
  }
  const long long gw = blk * (blockDim.x / kWarp) + threadIdx.x / kWarp;
  char* lreg_r = (char*)prm.lane_scratch + gw * kWarp * prm.lane_elems * (long long)(sizeof(TR) + sizeof(TC));
  char* lreg_c = lreg_r + (long long)kWarp * prm.lane_elems * (long long)sizeof(TR);
  char* wreg = (char*)prm.warp_scratch + gw * prm.warp_elems * (long long)sizeof(TC);
  const unsigned long long t0 = global_ns();  // this launch's start (time slices)
  unsigned long long t_job = t0;               // the job's start (time budget)
  if (lane == 0 && prm.job_t0 && prm.budget_ns > 0) {
    const unsigned long long first = atomicCAS(prm.job_t0, 0ull, t0);
    if (first) t_job = first;
  }
  for (;;) {
    unsigned t = 0xffffffffu;
    if (lane == 0) {
      int ab = 0;
      const unsigned long long now = global_ns();
      if (*prm.cancel != prm.cancel_epoch) ab = ABORT_CANCEL;
      else if (prm.budget_ns > 0 && (long long)(now - t_job) > prm.budget_ns) ab = ABORT_TIMEOUT;
      if (ab) atomicOr(prm.abort_word, ab);
      else if (*(volatile int*)prm.abort_word == 0 && !(prm.slice_ns > 0 && (long long)(now - t0) > prm.slice_ns))
        t = atomicAdd(prm.ticket, 1u);
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= (unsigned)prm.ntasks) break;
    const TaskDesc T = prm.tasks[t];
    if (prm.mats[T.mat].p >= 5) {  // one matrix per task: the whole warp takes its arithmetic
      if (prm.mat_flags[T.mat] & FLAG_REAL) run_task_shared<SR>(prm, T, lane, lreg_r, wreg);
      else run_task_shared<SC>(prm, T, lane, lreg_c, wreg);
    } else {
      run_task_lanes_any<SR, SC>(prm, T, lane, lreg_r, lreg_c);
    }
    __syncwarp();
    if (prm.one_task) break;
  }
  if (prm.one_task) {  // every warp of the block is done with the slot's scratch: give it back
    __threadfence();  // this thread's scratch stores are performed before the slot can be reused
    __syncthreads();
    if (threadIdx.x == 0) atomicAnd(&prm.slot_pool[s_slot >> 5], ~(1u << (s_slot & 31)));
  }
}

static_assert(sizeof(Real::T) + sizeof(Cplx::T) == kLaneEntryBytes, "lane scratch layout");
static_assert(sizeof(Cplx::T) == kWarpEntryBytes, "warp scratch layout");
static_assert(sizeof(RealX::T) + sizeof(CplxX::T) == kLaneEntryBytesExt, "lane scratch layout (ext)");
static_assert(sizeof(CplxX::T) == kWarpEntryBytesExt, "warp scratch layout (ext)");

__global__ void __launch_bounds__(kUnitsThreads, 4) k_units(const UnitsParams prm) { units_loop<Real, Cplx>(prm); }

// Extended precision: double-double entries need about twice the registers,
// so two blocks of 128 threads per SM.
constexpr int kExtBlocksPerSm = 2;
__global__ void __launch_bounds__(kUnitsThreads, kExtBlocksPerSm) k_units_ext(const UnitsParams prm) {
  units_loop<RealX, CplxX>(prm);
}

// Reduction of each matrix's 2^red_log2 leaves (task partials, or unit
// partials for p < 5): one perfect binary tree over leaf index, left operand
// first, in accurate double-word sums.  The tree is cut into aligned blocks
// that separate thread blocks evaluate (k_reduce_chunks, then k_reduce); every
// internal node gets the same operands whatever the cut, so the result does not
// depend on it.
constexpr int kReduceThreads = 256;

// Sum of k leaves x[0], x[stride], ... (k a power of two) as a perfect binary tree.
__device__ __forceinline__ void chunk_tree(const Part* x, long long stride, long long k, double& h, double& l,
                                           double& a) {
  double h_st[40], l_st[40], a_st[40];
  int top = 0;
  for (long long i = 0; i < k; ++i) {
    const Part v = x[i * stride];
    double vh = v.hi, vl = v.lo, va = v.abs_sum;
    for (long long q = i; q & 1; q >>= 1) {
      --top;
      dd_add(h_st[top], l_st[top], vh, vl, vh, vl);
      va = a_st[top] + va;
    }
    h_st[top] = vh;
    l_st[top] = vl;
    a_st[top] = va;
    ++top;
  }
  h = h_st[0];
  l = l_st[0];
  a = a_st[0];
}

// Perfect binary tree over the values of threads 0..T-1 (T a power of two, at
// most kReduceThreads), pairs (2i, 2i+1) at each level, the active threads
// packed into the lowest warps.  Called by every thread; thread 0 gets the sum.
__device__ __forceinline__ void block_tree(double& h, double& l, double& a, int T) {
  __shared__ double sh[2][kReduceThreads], sl[2][kReduceThreads], sa[2][kReduceThreads];
  const int t = threadIdx.x;
  int cur = 0;
  if (t < T) {
    sh[0][t] = h;
    sl[0][t] = l;
    sa[0][t] = a;
  }
  __syncthreads();
  for (int cnt = T >> 1; cnt >= 1; cnt >>= 1) {
    if (t < cnt) {
      double hh, ll;
      dd_add(sh[cur][2 * t], sl[cur][2 * t], sh[cur][2 * t + 1], sl[cur][2 * t + 1], hh, ll);
      sh[cur ^ 1][t] = hh;
      sl[cur ^ 1][t] = ll;
      sa[cur ^ 1][t] = sa[cur][2 * t] + sa[cur][2 * t + 1];
    }
    cur ^= 1;
    __syncthreads();
  }
  h = sh[cur][0];
  l = sl[cur][0];
  a = sa[cur][0];
}

// First stage: block b sums one aligned chunk of 2^red_chunk_log2 leaves of
// its matrix (the last matrix with red_chunk0 <= b) and writes the sum over the
// chunk's first leaf.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_chunks(const MatDesc* __restrict__ mats, int nmats,
                                                                  Part* partials) {
  const int b = blockIdx.x;
  int lo = 0, hi = nmats - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mats[mid].red_chunk0 <= b) lo = mid;
    else hi = mid - 1;
  }
  const MatDesc D = mats[lo];
  const long long C = 1ll << red_chunk_log2(D.red_log2);
  Part* x = partials + D.red_off + (long long)(b - D.red_chunk0) * C;
  const long long k = C / kReduceThreads;
  double h, l, a;
  chunk_tree(x + threadIdx.x * k, 1, k, h, l, a);
  block_tree(h, l, a, kReduceThreads);
  if (threadIdx.x == 0) x[0] = Part{h, l, a, 0.0};
}

// Second stage, one block per matrix: the 2^(red_log2 - red_chunk_log2) chunk
// sums (or all the leaves, when there was no first stage).
__global__ void __launch_bounds__(kReduceThreads) k_reduce(const MatDesc* __restrict__ mats,
                                                           const Part* __restrict__ partials,
                                                           const int* __restrict__ flags, ResultRec* out) {
  const MatDesc D = mats[blockIdx.x];
  const int clog = red_chunk_log2(D.red_log2);
  const long long stride = 1ll << clog;
  const long long U = 1ll << (D.red_log2 - clog);
  const int T = (int)(U < kReduceThreads ? U : kReduceThreads);
  const long long k = U / T;
  const Part* x = partials + D.red_off;
  double h = 0.0, l = 0.0, a = 0.0;
  if ((int)threadIdx.x < T) chunk_tree(x + (long long)threadIdx.x * k * stride, stride, k, h, l, a);
  block_tree(h, l, a, T);
  if (threadIdx.x == 0) {
    ResultRec r;
    r.hi = h;
    r.lo = l;
    r.abs_sum = a;
    r.flags = flags[blockIdx.x];
    r.pad = 0;
    out[blockIdx.x] = r;
  }
}

// FP64 throughput probe: independent FMA chains, 8 warps per SM.
__global__ void __launch_bounds__(256) k_probe(double* out, int iters) {
  double a0 = 1e-3, a1 = 2e-3, a2 = 3e-3, a3 = 4e-3;
  const double b = 0.9999999, c = 1e-9 * (threadIdx.x + 1);
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_intake(const MatDesc* d_mats, int nmats, int check, int* d_flags, cudaStream_t s) {
  if (nmats <= 0) return cudaSuccess;
  k_intake<<<nmats, 256, 0, s>>>(d_mats, check, d_flags);
  return cudaGetLastError();
}
cudaError_t launch_units(const UnitsParams& prm, int grid, cudaStream_t s) {
  if (prm.ntasks <= 0) return cudaSuccess;
  if (prm.ext) k_units_ext<<<grid, kUnitsThreads, 0, s>>>(prm);
  else k_units<<<grid, kUnitsThreads, 0, s>>>(prm);
  return cudaGetLastError();
}
cudaError_t launch_reduce(const MatDesc* d_mats, int nmats, long long nchunks, Part* partials, const int* flags,
                          ResultRec* out, cudaStream_t s) {
  if (nmats <= 0) return cudaSuccess;
  if (nchunks > 0) {
    if (nchunks > 0x7fffffffll) return cudaErrorInvalidValue;
    k_reduce_chunks<<<(unsigned)nchunks, kReduceThreads, 0, s>>>(d_mats, nmats, partials);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_reduce<<<nmats, kReduceThreads, 0, s>>>(d_mats, partials, flags, out);
  return cudaGetLastError();
}
int units_block_threads() { return kUnitsThreads; }
cudaError_t units_blocks_per_sm(int* blocks, int ext) {
  return ext ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_units_ext, kUnitsThreads, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_units, kUnitsThreads, 0);
}

cudaError_t run_probe_fp64(double seconds, double* dfma_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blocks = sms, threads = 256;
  double* d = nullptr;
  if ((e = cudaMalloc(&d, sizeof(double) * blocks * threads)) != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int iters = 20000;
  float ms = 0.f;
  for (int rep = 0; rep < 6; ++rep) {  // grow until the run is long enough
    cudaEventRecord(e0);
    k_probe<<<blocks, threads>>>(d, iters);
    cudaEventRecord(e1);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms > 1000.0 * seconds || rep == 5) break;
    double scale = (1000.0 * seconds) / (ms > 0.01f ? ms : 0.01f);
    if (scale > 100) scale = 100;
    iters = (int)(iters * scale * 1.05) + 1;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  *dfma_per_s = (double)blocks * threads * iters * 4.0 / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  return e;
}

}  // namespace tor
