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
// Four scalar types run the same tree:
//   Cplx  complex128 entries: any Hermitian O with I - O positive definite.
//   Real  float64 entries: O of a physical Gaussian state, which has the form
//         [[P, Q], [conj(Q), conj(P)]] in block layout.  The per-mode unitary
//         U = (1/sqrt 2) [[1, i], [1, -i]] from (a, a^dag) to the quadratures
//         (x, p) maps such a B to the real symmetric V = U^H B U, and every
//         principal block of V has the determinant of the matching block of B
//         (|det U| = 1), so the whole tree can run in real arithmetic at a
//         quarter of the multiply-adds.
//   CplxX, RealX  the same two in double-double arithmetic (about 106-bit
//         significands): the extended-precision factor of Sec. 5, where the
//         pivots, the Schur updates, phi and every term are carried in
//         double-double (tor_dd.cuh).
// Each type names its real scalar Re (double or dd_t) and its accumulator Acc.
//
// Storage of a symmetric / Hermitian matrix: packed lower triangle, element
// (r, s), r >= s, at index P(r, s) = r (r + 1) / 2 + s.  Diagonal entries are
// real (complex: imaginary part 0).  A node is a "view": a buffer plus a row
// offset o; its element (i, k) lives at P(i + o, k + o).
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
// (ah, al) + (bh, bl) -> normalised double-double, relative error <= 3 u^2
// also under cancellation (Joldes, Muller, Popescu, "Tight and rigorous error
// bounds for basic building blocks of double-word arithmetic", ACM TOMS 44
// (2017), AccurateDWPlusDW).
__device__ __forceinline__ void dd_add(double ah, double al, double bh, double bl, double& h, double& l) {
  double s, e, t, f;
  two_sum(ah, bh, s, e);
  two_sum(al, bl, t, f);
  e = __dadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __dadd_rn(e, f);
  fast_two_sum(s, e, h, l);
}

// ---------------------------------------------------------------------------
// Scalar types.  Each provides the operations of the include step:
//   det2(a, b, e)        a e - |b|^2 (determinant of the 2x2 pivot block)
//   cl(b, ia)            conj(l) = conj(b) / a          (l = b / a)
//   reduce_col(x, y, cl) y' = y - x conj(l)
//   scale(v, s)          v s
//   rank2_off(s, xt, xk, yt, yk)   s - xt conj(xk) - yt conj(yk)
//   rank2_diag(d, xt, x, yt, y)    d - Re(xt conj(x)) - Re(yt conj(y))
//   re(v), diag(d)       real part; the stored form of a real diagonal entry
// and, on its real scalar Re: mul, sub, neg, pos (> 0), rcp, rsqrt, hi (the
// leading double), one, shfl (warp broadcast from a lane).
// Positive and finite, decided on the bit pattern with integer operations: on
// GB300 an FP64 comparison takes an issue slot of the FP64 pipe, like an FMA,
// while integer operations run on another pipe.  The bit patterns of the
// positive finite doubles are exactly 1 .. 0x7FEFFFFFFFFFFFFF; +-0, negative
// values, infinities and NaNs fall outside.
__device__ __forceinline__ bool pos_finite(double a) {
  return (unsigned long long)__double_as_longlong(a) - 1ull < 0x7FEFFFFFFFFFFFFFull;
}

// ---------------------------------------------------------------------------
struct Fp64Re {  // real scalar operations of the two FP64 types
  using Re = double;
  using Acc = DD;
  static constexpr int kUnrollK = 2;  // unroll of the entry loop of an include from memory
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double neg(double a) { return -a; }
  static __device__ __forceinline__ bool pos(double a) { return pos_finite(a); }
  static __device__ __forceinline__ double rcp(double a) { return rcp64(a); }
  static __device__ __forceinline__ double rsqrt(double a) { return rsqrt64(a); }
  static __device__ __forceinline__ double hi(double a) { return a; }
  // a leaf pair phi (exclude) and phi r (include): signed sum phi r - phi and
  // magnitude sum phi r + phi, one FMA each
  static __device__ __forceinline__ void pair_sums(double phi, double r, double& v, double& ab) {
    v = fma(phi, r, -phi);
    ab = fma(phi, r, phi);
  }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double shfl(double a, int q) { return __shfl_sync(0xffffffffu, a, q); }
  static __device__ __forceinline__ Acc acc0() { return DD{0.0, 0.0}; }
  static __device__ __forceinline__ void acc_out(const Acc& a, double& h, double& l) { fast_two_sum(a.s, a.c, h, l); }
};
struct Cplx : Fp64Re {
  using T = double2;
  static constexpr int kRegModes = 3;
  static __device__ __forceinline__ double re(T v) { return v.x; }
  static __device__ __forceinline__ T diag(double d) { return make_double2(d, 0.0); }
  static __device__ __forceinline__ double abs2(T b) { return fma(b.x, b.x, b.y * b.y); }
  static __device__ __forceinline__ double det2(double a, T b, double e) { return fma(a, e, -abs2(b)); }
  static __device__ __forceinline__ T cl(T b, double ia) { return make_double2(b.x * ia, -b.y * ia); }
  static __device__ __forceinline__ T reduce_col(T x, T y, T c) {
    T r;
    r.x = fma(-x.x, c.x, y.x);
    r.x = fma(x.y, c.y, r.x);
    r.y = fma(-x.x, c.y, y.y);
    r.y = fma(-x.y, c.x, r.y);
    return r;
  }
  static __device__ __forceinline__ T scale(T v, double s) { return make_double2(v.x * s, v.y * s); }
  static __device__ __forceinline__ T rank2_off(T s, T xt, T xk, T yt, T yk) {  // 8 DFMA
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
  static __device__ __forceinline__ double rank2_diag(double d, T xt, T x, T yt, T y) {  // 4 DFMA
    d = fma(-xt.x, x.x, d);
    d = fma(-xt.y, x.y, d);
    d = fma(-yt.x, y.x, d);
    d = fma(-yt.y, y.y, d);
    return d;
  }
};
struct Real : Fp64Re {
  using T = double;
  static constexpr int kRegModes = 4;  // modes of the register-resident subtrees of the lane walk
  static __device__ __forceinline__ double re(T v) { return v; }
  static __device__ __forceinline__ T diag(double d) { return d; }
  static __device__ __forceinline__ double abs2(T b) { return b * b; }
  static __device__ __forceinline__ double det2(double a, T b, double e) { return fma(a, e, -abs2(b)); }
  static __device__ __forceinline__ T cl(T b, double ia) { return b * ia; }
  static __device__ __forceinline__ T reduce_col(T x, T y, T c) { return fma(-x, c, y); }
  static __device__ __forceinline__ T scale(T v, double s) { return v * s; }
  static __device__ __forceinline__ T rank2_off(T s, T xt, T xk, T yt, T yk) {  // 2 DFMA
    return fma(-yt, yk, fma(-xt, xk, s));
  }
  static __device__ __forceinline__ double rank2_diag(double d, T xt, T x, T yt, T y) {
    return fma(-yt, y, fma(-xt, x, d));
  }
};

// ---------------------------------------------------------------------------
// The 2x2 pivot of an include step (Algorithm 1 on mode j's two rows).
// Pivot block [[a, conj(b)], [b, e]], a = S(0,0), b = S(1,0), e = S(1,1).
// LDL^H: d1 = a, l = b / a, d2 = e - |b|^2 / a.  With x = S(:,0), y = S(:,1)
// over the trailing rows, the Schur complement is
//   S' = S_22 - x x^H / d1 - y' y'^H / d2,   y' = y - x conj(l),
// and the determinant factor of the step is rho = (d1 d2)^{-1/2}.
// ---------------------------------------------------------------------------
template <class S>
struct Pivot {
  using Re = typename S::Re;
  Re ia;             // 1 / d1
  Re id2;            // 1 / d2 = a rho^2
  Re rho;            // (a e - |b|^2)^{-1/2}
  typename S::T cl;  // conj(l) = conj(b) / a
  bool ok;           // d1 > 0 and d1 d2 > 0, both finite: the block is positive definite
};
template <class S>
__device__ __forceinline__ Pivot<S> make_pivot(typename S::Re a, typename S::T b, typename S::Re e) {
  using Re = typename S::Re;
  Pivot<S> pv;
  const Re det2 = S::det2(a, b, e);
  pv.ok = S::pos(a) & S::pos(det2);
  pv.rho = S::rsqrt(det2);
  pv.ia = S::rcp(a);
  pv.cl = S::cl(b, pv.ia);
  pv.id2 = S::mul(a, S::mul(pv.rho, pv.rho));
  return pv;
}

// ---------------------------------------------------------------------------
// Register-resident nodes: HM<S, R> is an R x R matrix (R = 2m rows) with real
// diagonal d[] and strictly lower entries o[TI(i,k)], i > k.  Everything below
// is fully unrolled, so the arrays live in registers.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int TI(int i, int k) { return (i * (i - 1)) / 2 + k; }

template <class S, int R>
struct HM {
  typename S::Re d[R];
  typename S::T o[(R * (R - 1)) / 2];
};

// Exclude the first mode: the trailing (R-2) x (R-2) block.
template <class S, int R>
__device__ __forceinline__ void hm_trail(const HM<S, R>& A, HM<S, R - 2>& C) {
#pragma unroll
  for (int i = 0; i < R - 2; ++i) {
    C.d[i] = A.d[i + 2];
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = A.o[TI(i + 2, k + 2)];
  }
}

// Include the first mode: C = Schur complement, returns rho.
template <class S, int R>
__device__ __forceinline__ typename S::Re hm_include(const HM<S, R>& A, HM<S, R - 2>& C, bool& bad) {
  using T = typename S::T;
  const Pivot<S> pv = make_pivot<S>(A.d[0], A.o[TI(1, 0)], A.d[1]);
  bad |= !pv.ok;
  T x[R - 2], yp[R - 2];
#pragma unroll
  for (int r = 0; r < R - 2; ++r) {
    x[r] = A.o[TI(r + 2, 0)];
    yp[r] = S::reduce_col(x[r], A.o[TI(r + 2, 1)], pv.cl);
  }
#pragma unroll
  for (int i = 0; i < R - 2; ++i) {
    const T xt = S::scale(x[i], pv.ia), yt = S::scale(yp[i], pv.id2);
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = S::rank2_off(A.o[TI(i + 2, k + 2)], xt, x[k], yt, yp[k]);
    C.d[i] = S::rank2_diag(A.d[i + 2], xt, x[i], yt, yp[i]);
  }
  return pv.rho;
}

// One mode left (2 x 2 node): its two leaves, exclude (-phi) and include
// (+phi rho).  v = signed sum, ab = sum of magnitudes.
template <class S>
__device__ __forceinline__ void leaf_pair(typename S::Re a, typename S::T b, typename S::Re e, typename S::Re phi,
                                          typename S::Re& v, double& ab, bool& bad) {
  using Re = typename S::Re;
  const Re det2 = S::det2(a, b, e);
  bad |= !(S::pos(a) & S::pos(det2));
  S::pair_sums(phi, S::rsqrt(det2), v, ab);
}

// Sum over the 2^(R/2) leaves below a register node:
//   v = sum (-1)^{#modes excluded below this node} phi_leaf,  ab = sum phi_leaf.
template <class S, int R>
struct Subtree {
  using Re = typename S::Re;
  static __device__ __forceinline__ void run(const HM<S, R>& A, Re phi, Re& v, double& ab, bool& bad) {
    HM<S, R - 2> E;
    hm_trail<S, R>(A, E);
    Re v1;
    double a1;
    Subtree<S, R - 2>::run(E, phi, v1, a1, bad);
    HM<S, R - 2> I;
    const Re rho = hm_include<S, R>(A, I, bad);
    Re v2;
    double a2;
    Subtree<S, R - 2>::run(I, S::mul(phi, rho), v2, a2, bad);
    v = S::sub(v2, v1);
    ab = a1 + a2;
  }
};
template <class S>
struct Subtree<S, 2> {
  using Re = typename S::Re;
  static __device__ __forceinline__ void run(const HM<S, 2>& A, Re phi, Re& v, double& ab, bool& bad) {
    leaf_pair<S>(A.d[0], A.o[0], A.d[1], phi, v, ab, bad);
  }
};

// ---------------------------------------------------------------------------
// Lane-private memory.  Each lane of a warp owns a private stack of packed
// matrices; the 32 lanes' copies are interleaved element by element, so when
// all lanes touch element e of their own matrices (they run the same control
// flow) the warp reads 32 consecutive elements.
// ---------------------------------------------------------------------------
template <class S>
struct LaneMem {
  typename S::T* p;  // lane's element 0 (= warp region + lane)
  __device__ __forceinline__ typename S::T ld(int e) const { return p[(size_t)e * kWarp]; }
  __device__ __forceinline__ void st(int e, typename S::T v) const { p[(size_t)e * kWarp] = v; }
  __device__ __forceinline__ typename S::Re ldd(int e) const { return S::re(ld(e)); }
};

// Load the trailing R x R block of a node with R/2 + 1 modes (exclude its first mode).
template <class S, int R>
__device__ __forceinline__ void lane_load_trail(const LaneMem<S> L, int src, int o, HM<S, R>& C) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    C.d[i] = L.ldd(src + P(o + 2 + i, o + 2 + i));
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = L.ld(src + P(o + 2 + i, o + 2 + k));
  }
}
// Include the first mode of a node with R/2 + 1 modes in memory; the child (R/2 modes) in registers.
template <class S, int R>
__device__ __forceinline__ typename S::Re lane_include_reg(const LaneMem<S> L, int src, int o, HM<S, R>& C, bool& bad) {
  using T = typename S::T;
  const Pivot<S> pv = make_pivot<S>(L.ldd(src + P(o, o)), L.ld(src + P(o + 1, o)), L.ldd(src + P(o + 1, o + 1)));
  bad |= !pv.ok;
  T x[R], yp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    x[r] = L.ld(src + P(o + 2 + r, o));
    yp[r] = S::reduce_col(x[r], L.ld(src + P(o + 2 + r, o + 1)), pv.cl);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const T xt = S::scale(x[i], pv.ia), yt = S::scale(yp[i], pv.id2);
#pragma unroll
    for (int k = 0; k < i; ++k)
      C.o[TI(i, k)] = S::rank2_off(L.ld(src + P(o + 2 + i, o + 2 + k)), xt, x[k], yt, yp[k]);
    C.d[i] = S::rank2_diag(L.ldd(src + P(o + 2 + i, o + 2 + i)), xt, x[i], yt, yp[i]);
  }
  return pv.rho;
}
// Load a whole node with R/2 modes from memory into registers.
template <class S, int R>
__device__ __forceinline__ void lane_load_node(const LaneMem<S> L, int src, int o, HM<S, R>& C) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    C.d[i] = L.ldd(src + P(o + i, o + i));
#pragma unroll
    for (int k = 0; k < i; ++k) C.o[TI(i, k)] = L.ld(src + P(o + i, o + k));
  }
}

}  // namespace tor
