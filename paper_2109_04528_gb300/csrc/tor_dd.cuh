// tor_dd.cuh -- double-double arithmetic and the extended-precision scalar
// types RealX and CplxX.
//
// Sec. 5 shows the Torontonian of weakly squeezed states to be a sum of 2^n
// terms close to +-1 that cancel almost completely, so the error of each term
// (relative to the term) decides the accuracy of the result; there the factor
// arithmetic has to run in more than double precision.  These types carry
// every quantity of the include step -- pivots, Schur-complement entries, the
// running product phi and the terms -- as a double-double h + l (|l| <=
// ulp(h) / 2, about 106 significant bits).
//
// Building blocks, error-free under round-to-nearest: two_sum (Knuth),
// fast_two_sum (Dekker), two_prod by FMA.  Operations and their FP64
// instruction counts:
//   dd_add    20  accurate double-word sum (Joldes, Muller, Popescu, ACM TOMS
//                 44 (2017), AccurateDWPlusDW): relative error <= 3 u^2, also
//                 under cancellation
//   dd_sum    11  sloppy double-word sum (the same paper's SloppyDWPlusDW): its
//                 relative error is unbounded under cancellation, its absolute
//                 error stays below ~2 u^2 (|a| + |b|); used for the sums of
//                 terms, whose accuracy is measured against sum |term|
//   dd_mul     4  double-word product (the same paper's DWTimesDW with the
//                 lo * lo term dropped and without its final renormalisation:
//                 the low part, the product's rounding error plus the cross
//                 terms, stays below ~2.5 u of the high part, so the pair is a
//                 double word as it stands): relative error <= ~5 u^2
//   ProdAcc       s + sum_i (+-) b_i c_i with one normalisation at the end:
//                 12 per product + 3 (a sum that starts from a product: 5 for
//                 it); absolute error ~ u^2 (|s| + sum |b_i c_i|).  The final
//                 fast_two_sum is exact when |h| >= |t|; when h has cancelled
//                 below t it adds at most u |t|, inside the same bound
//   dd_rcp    13  Newton step for 1/a from the FP64 reciprocal, evaluated in
//                 double-double: 1/a = y (1 + e + e^2 + ...), e = 1 - a y
//   dd_rsqrt  19  the same for a^{-1/2}: y (1 + e/2 + 3e^2/8 + ...), e = 1 - a y^2
// (u = 2^-53.)  The Newton terms dropped are O(e^2) <= 2^-104.
#pragma once
#include "tor_device.cuh"

namespace tor {

struct __align__(16) dd_t {
  double h, l;
};

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

__device__ __forceinline__ dd_t dd_add(dd_t a, dd_t b) {
  dd_t r;
  dd_add(a.h, a.l, b.h, b.l, r.h, r.l);
  return r;
}
__device__ __forceinline__ dd_t dd_neg(dd_t a) { return dd_t{-a.h, -a.l}; }
__device__ __forceinline__ dd_t dd_sum(dd_t a, dd_t b) {
  double s, e;
  two_sum(a.h, b.h, s, e);
  e = __dadd_rn(e, __dadd_rn(a.l, b.l));
  dd_t r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ dd_t dd_mul(dd_t a, dd_t b) {
  double p, e;
  two_prod(a.h, b.h, p, e);
  e = __fma_rn(a.h, b.l, e);
  e = __fma_rn(a.l, b.h, e);
  return dd_t{p, e};
}

// Sum of products, normalised once: h + t holds the running value.
struct ProdAcc {
  double h, t;
  __device__ __forceinline__ explicit ProdAcc(dd_t s) : h(s.h), t(s.l) {}
  // start from the product b c (7 operations): h + t = b c to ~u^2
  __device__ __forceinline__ ProdAcc(dd_t b, dd_t c) {
    two_prod(b.h, c.h, h, t);
    t = __fma_rn(b.h, c.l, t);
    t = __fma_rn(b.l, c.h, t);
  }
  __device__ __forceinline__ void add(dd_t b, dd_t c) {  // += b c
    double p, e, s, r;
    two_prod(b.h, c.h, p, e);
    e = __fma_rn(b.h, c.l, e);
    e = __fma_rn(b.l, c.h, e);
    two_sum(h, p, s, r);
    h = s;
    t = __dadd_rn(t, __dadd_rn(r, e));
  }
  __device__ __forceinline__ void sub(dd_t b, dd_t c) { add(dd_neg(b), c); }  // -= b c
  __device__ __forceinline__ dd_t out() const {
    dd_t r;
    fast_two_sum(h, t, r.h, r.l);
    return r;
  }
};

__device__ __forceinline__ dd_t dd_rcp(dd_t a) {
  const double y = rcp64(a.h);
  double p, q;
  two_prod(a.h, y, p, q);                                         // a.h y = p + q exactly
  const double e = __fma_rn(-a.l, y, __dsub_rn(__dsub_rn(1.0, p), q));  // 1 - a y; 1 - p is exact
  dd_t r;
  fast_two_sum(y, __dmul_rn(y, e), r.h, r.l);
  return r;
}

__device__ __forceinline__ dd_t dd_rsqrt(dd_t a) {
  const double y = rsqrt64(a.h);
  double s, t, p, q;
  two_prod(y, y, s, t);    // y^2 = s + t exactly
  two_prod(a.h, s, p, q);  // a.h s = p + q exactly
  double e = __dsub_rn(__dsub_rn(1.0, p), q);  // 1 - a y^2, to ~u^2
  e = __fma_rn(-a.h, t, e);
  e = __fma_rn(-a.l, s, e);
  dd_t r;
  fast_two_sum(y, __dmul_rn(__dmul_rn(0.5, y), e), r.h, r.l);
  return r;
}

// ---------------------------------------------------------------------------
// Scalar types (same interface as Cplx / Real in tor_device.cuh).
// ---------------------------------------------------------------------------
struct XRe {
  using Re = dd_t;
  // entry loop of an include from memory not unrolled: measured against 2x, the
  // same bits, +3.1 % on the complex path (n = 26), +1.0 % on the real path at
  // n = 16..24, neutral on the n = 30 + 34 step
  static constexpr int kUnrollK = 1;
  // modes of the register-resident subtrees of the lane walk: 2 (a 3-mode node
  // of double words is 42 doubles, of complex ones 84, which crowds the 255
  // registers; measured with 2 modes: real +6.6 %, complex +22 %)
  static constexpr int kRegModes = 2;
  struct Acc {
    dd_t s;
    __device__ __forceinline__ void add(dd_t v) { s = dd_sum(s, v); }
  };
  static __device__ __forceinline__ dd_t mul(dd_t a, dd_t b) { return dd_mul(a, b); }
  static __device__ __forceinline__ dd_t sub(dd_t a, dd_t b) { return dd_sum(a, dd_neg(b)); }  // sums of terms only
  static __device__ __forceinline__ dd_t neg(dd_t a) { return dd_neg(a); }
  static __device__ __forceinline__ bool pos(dd_t a) { return pos_finite(a.h); }  // h + l > 0 iff h > 0
  static __device__ __forceinline__ dd_t rcp(dd_t a) { return dd_rcp(a); }
  static __device__ __forceinline__ dd_t rsqrt(dd_t a) { return dd_rsqrt(a); }
  static __device__ __forceinline__ double hi(dd_t a) { return a.h; }
  static __device__ __forceinline__ dd_t one() { return dd_t{1.0, 0.0}; }
  static __device__ __forceinline__ void pair_sums(dd_t phi, dd_t r, dd_t& v, double& ab) {
    const dd_t pr = dd_mul(phi, r);
    v = dd_sum(pr, dd_neg(phi));
    ab = pr.h + phi.h;
  }
  static __device__ __forceinline__ dd_t shfl(dd_t a, int q) {
    return dd_t{__shfl_sync(0xffffffffu, a.h, q), __shfl_sync(0xffffffffu, a.l, q)};
  }
  static __device__ __forceinline__ Acc acc0() { return Acc{dd_t{0.0, 0.0}}; }
  static __device__ __forceinline__ void acc_out(const Acc& a, double& h, double& l) {
    h = a.s.h;
    l = a.s.l;
  }
};

struct RealX : XRe {
  using T = dd_t;
  static __device__ __forceinline__ dd_t re(T v) { return v; }
  static __device__ __forceinline__ T diag(dd_t d) { return d; }
  static __device__ __forceinline__ dd_t det2(dd_t a, T b, dd_t e) {
    ProdAcc s(a, e);
    s.sub(b, b);
    return s.out();
  }
  static __device__ __forceinline__ T cl(T b, dd_t ia) { return dd_mul(b, ia); }
  static __device__ __forceinline__ T reduce_col(T x, T y, T c) {
    ProdAcc s(y);
    s.sub(x, c);
    return s.out();
  }
  static __device__ __forceinline__ T scale(T v, dd_t s) { return dd_mul(v, s); }
  static __device__ __forceinline__ T rank2_off(T s, T xt, T xk, T yt, T yk) {
    ProdAcc a(s);
    a.sub(xt, xk);
    a.sub(yt, yk);
    return a.out();
  }
  static __device__ __forceinline__ dd_t rank2_diag(dd_t d, T xt, T x, T yt, T y) { return rank2_off(d, xt, x, yt, y); }
};

struct __align__(16) ddc_t {
  dd_t x, y;  // real and imaginary parts
};

struct CplxX : XRe {
  using T = ddc_t;
  static __device__ __forceinline__ dd_t re(T v) { return v.x; }
  static __device__ __forceinline__ T diag(dd_t d) { return ddc_t{d, dd_t{0.0, 0.0}}; }
  static __device__ __forceinline__ dd_t det2(dd_t a, T b, dd_t e) {  // a e - |b|^2
    ProdAcc s(a, e);
    s.sub(b.x, b.x);
    s.sub(b.y, b.y);
    return s.out();
  }
  static __device__ __forceinline__ T cl(T b, dd_t ia) { return ddc_t{dd_mul(b.x, ia), dd_neg(dd_mul(b.y, ia))}; }
  static __device__ __forceinline__ T reduce_col(T x, T y, T c) {  // y - x c
    ProdAcc r(y.x), i(y.y);
    r.sub(x.x, c.x);
    r.add(x.y, c.y);
    i.sub(x.x, c.y);
    i.sub(x.y, c.x);
    return ddc_t{r.out(), i.out()};
  }
  static __device__ __forceinline__ T scale(T v, dd_t s) { return ddc_t{dd_mul(v.x, s), dd_mul(v.y, s)}; }
  static __device__ __forceinline__ T rank2_off(T s, T xt, T xk, T yt, T yk) {  // s - xt conj(xk) - yt conj(yk)
    ProdAcc r(s.x), i(s.y);
    r.sub(xt.x, xk.x);
    r.sub(xt.y, xk.y);
    r.sub(yt.x, yk.x);
    r.sub(yt.y, yk.y);
    i.sub(xt.y, xk.x);
    i.add(xt.x, xk.y);
    i.sub(yt.y, yk.x);
    i.add(yt.x, yk.y);
    return ddc_t{r.out(), i.out()};
  }
  static __device__ __forceinline__ dd_t rank2_diag(dd_t d, T xt, T x, T yt, T y) {
    ProdAcc r(d);
    r.sub(xt.x, x.x);
    r.sub(xt.y, x.y);
    r.sub(yt.x, y.x);
    r.sub(yt.y, y.y);
    return r.out();
  }
};

}  // namespace tor
