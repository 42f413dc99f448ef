// tor_device.cuh -- device building blocks of the subset-tree Torontonian.
//
// Notation (paper Sec. 2): B = I - O in pairs order (a_1, a_1^dag, a_2, ...),
// so mode j owns rows {2j, 2j+1}.  A node of the subset tree at depth j is the
// set K of included modes among 0..j-1; it carries
//   S   = B_TT - B_TK B_KK^{-1} B_KT   (Schur complement over the undecided
//         modes T = j..n-1; the trailing block of the partial Cholesky factor
//         of B restricted to K u T, Fig. 1 / Fig. 2),
//   phi = det(B_KK)^{-1/2}.
// Excluding mode j keeps S minus mode j's rows (no arithmetic).  Including it
// extends the factor by mode j's two rows (Algorithm 1 on the 2x2 pivot block)
// and updates the trailing block by the rank-2 Schur term -- the reuse of
// L11/L21 that Fig. 2 describes, run in the add-a-mode direction.  A leaf
// (all n modes decided, included set Z) contributes (-1)^{n-|Z|} phi_Z
// (Eq. tor).
//
// Storage of a Hermitian matrix: packed lower triangle, element (r, s), r >= s,
// at index P(r, s) = r (r + 1) / 2 + s, complex128 (double2).  Diagonal
// entries are real (imaginary part 0).  A node is a "view": a buffer plus a
// row offset o; its element (i, k) lives at P(i + o, k + o).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tor {

constexpr int kWarp = 32;

__host__ __device__ __forceinline__ int P(int r, int s) { return (r * (r + 1)) / 2 + s; }

// ---------------------------------------------------------------------------
// FP64 reciprocal and reciprocal square root.
// The hardware estimates (rcp/rsqrt.approx.ftz.f64) have relative error below
// 2^-19.9 on GB300.  One step of the cubic series refinement brings them to
// double precision:
//   1/x      : y' = y (1 + e + e^2),          e = 1 - x y      (series of 1/(1-e))
//   x^{-1/2} : y' = y (1 + e/2 + 3 e^2 / 8),  e = 1 - x y^2    (series of (1-e)^{-1/2})
// The dropped terms are O(e^3) < 2^-59; rounding adds about one ulp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp_est(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rsqrt_est(double x) {
  double r;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rcp64(double x) {
  double y = rcp_est(x);
  double e = fma(-x, y, 1.0);
  double s = fma(e, e, e);
  return fma(y, s, y);
}
__device__ __forceinline__ double rsqrt64(double x) {
  double y = rsqrt_est(x);
  double t = x * y;
  double e = fma(-t, y, 1.0);
  double p = fma(0.375, e, 0.5);
  double q = y * e;
  return fma(q, p, y);
}

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum, Dekker FastTwoSum) and the
// double-double accumulator (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), algorithm Sum2).  The _rn
// intrinsics keep the compiler from contracting or reordering them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}
struct DD {
  double s, c;  // running sum and accumulated rounding errors (Sum2)
  __device__ __forceinline__ void add(double x) {
    double e;
    two_sum(s, x, s, e);
    c = __dadd_rn(c, e);
  }
};
// (ah, al) + (bh, bl) -> normalised double-double
__device__ __forceinline__ void dd_add(double ah, double al, double bh, double bl, double& h, double& l) {
  double s, e;
  two_sum(ah, bh, s, e);
  e = __dadd_rn(e, __dadd_rn(al, bl));
  fast_two_sum(s, e, h, l);
}

// ---------------------------------------------------------------------------
// The 2x2 pivot of an include step (Algorithm 1 on mode j's two rows).
// Pivot block [[a, conj(b)], [b, e]], a = S(0,0), b = S(1,0), e = S(1,1).
// LDL^H: d1 = a, l = b / a, d2 = e - |b|^2 / a.  With x = S(:,0), y = S(:,1)
// over the trailing rows, the Schur complement is
//   S' = S_22 - x x^H / d1 - y' y'^H / d2,   y' = y - x conj(l),
// and the determinant factor of the step is rho = (d1 d2)^{-1/2}.
// ---------------------------------------------------------------------------
struct Pivot {
  double ia;   // 1 / d1
  double id2;  // 1 / d2 = a rho^2
  double rho;  // (a e - |b|^2)^{-1/2}
  double2 cl;  // conj(l) = conj(b) / a
  bool ok;     // d1 > 0 and d1 d2 > 0: the block is positive definite
};
__device__ __forceinline__ Pivot make_pivot(double a, double2 b, double e) {
  Pivot P;
  double bb = fma(b.x, b.x, b.y * b.y);
  double det2 = fma(a, e, -bb);
  P.ok = (a > 0.0) && (det2 > 0.0);
  P.rho = rsqrt64(det2);
  P.ia = rcp64(a);
  P.cl = make_double2(b.x * P.ia, -b.y * P.ia);
  P.id2 = a * (P.rho * P.rho);
  return P;
}

// y' = y - x * cl
__device__ __forceinline__ double2 reduce_col(double2 x, double2 y, double2 cl) {
  double2 r;
  r.x = fma(-x.x, cl.x, y.x);
  r.x = fma(x.y, cl.y, r.x);
  r.y = fma(-x.x, cl.y, y.y);
  r.y = fma(-x.y, cl.x, r.y);
  return r;
}
// s - xt conj(xk) - yt conj(yk)   (8 DFMA)
__device__ __forceinline__ double2 rank2_off(double2 s, double2 xt, double2 xk, double2 yt, double2 yk) {
  s.x = fma(-xt.x, xk.x, s.x);
  s.x = fma(-xt.y, xk.y, s.x);
  s.x = fma(-yt.x, yk.x, s.x);
  s.x = fma(-yt.y, yk.y, s.x);
  s.y = fma(-xt.y, xk.x, s.y);
  s.y = fma(xt.x, xk.y, s.y);
  s.y = fma(-yt.y, yk.x, s.y);
  s.y = fma(yt.x, yk.y, s.y);
  return s;
}
// d - Re(xt conj(x)) - Re(yt conj(y))   (4 DFMA)
__device__ __forceinline__ double rank2_diag(double d, double2 xt, double2 x, double2 yt, double2 y) {
  d = fma(-xt.x, x.x, d);
  d = fma(-xt.y, x.y, d);
  d = fma(-yt.x, y.x, d);
  d = fma(-yt.y, y.y, d);
  return d;
}
__device__ __forceinline__ double2 cscale(double2 v, double s) { return make_double2(v.x * s, v.y * s); }

// ---------------------------------------------------------------------------
// Register-resident nodes: HM<R> is an R x R Hermitian matrix (R = 2m rows)
// with real diagonal d[] and strictly lower entries o[TI(i,k)], i > k.
// Everything below is fully unrolled, so the arrays live in registers.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int TI(int i, int k) { return (i * (i - 1)) / 2 + k; }

template <int R>
struct HM {
  double d[R];
  double2 o[(R * (R - 1)) / 2];
};

// Exclude the first mode: the trailing (R-2) x (R-2) block.
template <int R>
__device__ __forceinline__ void hm_trail(const HM<R>& A, HM<R - 2>& C) {
#pragma unroll
  for (int i = 0; i < R - 2; ++i) {
    C.d[i] = A.d[i + 2];
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = A.o[TI(i + 2, k + 2)];
  }
}

// Include the first mode: C = Schur complement, returns rho.
template <int R>
__device__ __forceinline__ double hm_include(const HM<R>& A, HM<R - 2>& C, bool& bad) {
  Pivot pv = make_pivot(A.d[0], A.o[TI(1, 0)], A.d[1]);
  bad |= !pv.ok;
  double2 x[R - 2], yp[R - 2];
#pragma unroll
  for (int r = 0; r < R - 2; ++r) {
    x[r] = A.o[TI(r + 2, 0)];
    yp[r] = reduce_col(x[r], A.o[TI(r + 2, 1)], pv.cl);
  }
#pragma unroll
  for (int i = 0; i < R - 2; ++i) {
    double2 xt = cscale(x[i], pv.ia), yt = cscale(yp[i], pv.id2);
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = rank2_off(A.o[TI(i + 2, k + 2)], xt, x[k], yt, yp[k]);
    C.d[i] = rank2_diag(A.d[i + 2], xt, x[i], yt, yp[i]);
  }
  return pv.rho;
}

// One mode left (2 x 2 node): its two leaves, exclude (-phi) and include
// (+phi rho).  v = signed sum, ab = sum of magnitudes.
__device__ __forceinline__ void leaf_pair(double a, double2 b, double e, double phi, double& v, double& ab,
                                          bool& bad) {
  double bb = fma(b.x, b.x, b.y * b.y);
  double det2 = fma(a, e, -bb);
  bad |= !((a > 0.0) && (det2 > 0.0));
  double pr = phi * rsqrt64(det2);
  v = pr - phi;
  ab = pr + phi;
}

// Sum over the 2^(R/2) leaves below a register node:
//   v = sum (-1)^{#modes excluded below this node} phi_leaf,  ab = sum phi_leaf.
template <int R>
struct Subtree {
  static __device__ __forceinline__ void run(const HM<R>& A, double phi, double& v, double& ab, bool& bad) {
    HM<R - 2> E;
    hm_trail<R>(A, E);
    double v1, a1;
    Subtree<R - 2>::run(E, phi, v1, a1, bad);
    HM<R - 2> I;
    double rho = hm_include<R>(A, I, bad);
    double v2, a2;
    Subtree<R - 2>::run(I, phi * rho, v2, a2, bad);
    v = v2 - v1;
    ab = a1 + a2;
  }
};
template <>
struct Subtree<2> {
  static __device__ __forceinline__ void run(const HM<2>& A, double phi, double& v, double& ab, bool& bad) {
    leaf_pair(A.d[0], A.o[0], A.d[1], phi, v, ab, bad);
  }
};

// ---------------------------------------------------------------------------
// Lane-private memory.  Each lane of a warp owns a private stack of packed
// matrices; the 32 lanes' copies are interleaved element by element, so when
// all lanes touch element e of their own matrices (they run the same control
// flow) the warp reads 32 consecutive double2 (512 contiguous bytes).
// ---------------------------------------------------------------------------
struct LaneMem {
  double2* p;  // lane's element 0 (= warp region + lane)
  __device__ __forceinline__ double2 ld(int e) const { return p[(size_t)e * kWarp]; }
  __device__ __forceinline__ void st(int e, double2 v) const { p[(size_t)e * kWarp] = v; }
};

// Include the first mode of node (src, o rows offset) with m modes; write the
// child (m-1 modes) to (dst, dst_o).  In place when dst == src and
// dst_o == o + 2.  xs/ys: scratch of 2(m-1) elements each.  Returns rho.
__device__ __noinline__ double lane_include_mem(const LaneMem L, int src, int o, int m, int dst, int dst_o,
                                                int xs, int ys, bool& bad);

// Load the trailing 6 x 6 block of a node with 4 modes (exclude its first mode).
__device__ __forceinline__ void lane_load_trail4(const LaneMem L, int src, int o, HM<6>& C) {
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    C.d[i] = L.ld(src + P(o + 2 + i, o + 2 + i)).x;
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = L.ld(src + P(o + 2 + i, o + 2 + k));
  }
}
// Include the first mode of a 4-mode node in memory; child (3 modes) in registers.
__device__ __forceinline__ double lane_include4(const LaneMem L, int src, int o, HM<6>& C, bool& bad) {
  Pivot pv = make_pivot(L.ld(src + P(o, o)).x, L.ld(src + P(o + 1, o)), L.ld(src + P(o + 1, o + 1)).x);
  bad |= !pv.ok;
  double2 x[6], yp[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    x[r] = L.ld(src + P(o + 2 + r, o));
    yp[r] = reduce_col(x[r], L.ld(src + P(o + 2 + r, o + 1)), pv.cl);
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double2 xt = cscale(x[i], pv.ia), yt = cscale(yp[i], pv.id2);
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = rank2_off(L.ld(src + P(o + 2 + i, o + 2 + k)), xt, x[k], yt, yp[k]);
    C.d[i] = rank2_diag(L.ld(src + P(o + 2 + i, o + 2 + i)).x, xt, x[i], yt, yp[i]);
  }
  return pv.rho;
}
// Load a whole node with R/2 modes (R <= 6) from memory into registers.
template <int R>
__device__ __forceinline__ void lane_load_node(const LaneMem L, int src, int o, HM<R>& C) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    C.d[i] = L.ld(src + P(o + i, o + i)).x;
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = L.ld(src + P(o + i, o + k));
  }
}

// ---------------------------------------------------------------------------
// Cooperative include: the 32 lanes of a warp split the entries of one node
// stored contiguously (packed, not interleaved).  Used for the shared upper
// part of the tree, where nodes are large.  All lanes compute the pivot; the
// call ends with __syncwarp so the child is visible to every lane.
// ---------------------------------------------------------------------------
__device__ __noinline__ double coop_include(const double2* src, int o, int m, double2* dst, int dst_o, double2* xs,
                                            double2* ys, bool& bad);

}  // namespace tor
