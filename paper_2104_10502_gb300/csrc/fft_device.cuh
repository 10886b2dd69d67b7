// Device-side building blocks of the shared-memory 3D FFT.
//
// All transforms are in place, on lines held in shared memory, with every
// thread of the block cooperating on every stage:
//   * inverse transforms (G -> r, e^{+i}) run mixed-radix decimation in
//     frequency (DIF): natural order in, digit-reversed order out;
//   * forward transforms (r -> G, e^{-i}) run decimation in time (DIT):
//     digit-reversed order in, natural order out.
// A pointwise multiply placed between the two therefore needs no permutation
// pass: it only indexes its operand through the digit-reversal table.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "common.h"
#include "ff.cuh"

namespace qe {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

// A complex float-float value is kept packed: hi = (re.hi, im.hi) and lo =
// (re.lo, im.lo), each pair one f32x2 operand, so that the operations on real
// and imaginary parts run as one instruction for both (ff.cuh).  Same 16 bytes
// as complex<double> in shared memory and in the stick workspace.
template <>
struct alignas(16) cx<ff> {
  f2 hi, lo;
};
__device__ __forceinline__ ff2 as2(cx<ff> a) { return {a.hi, a.lo}; }
__device__ __forceinline__ cx<ff> of2(ff2 a) { return {a.hi, a.lo}; }

// Element construction and access that the tiles use for every element type.
template <typename T>
__device__ __forceinline__ cx<T> cx_zero() {
  if constexpr (std::is_same<T, ff>::value) return {f2_of(0.f, 0.f), f2_of(0.f, 0.f)};
  else return {T(0), T(0)};
}
template <typename T>
__device__ __forceinline__ cx<T> cx_from(double re, double im) {
  if constexpr (std::is_same<T, ff>::value) {
    const ff a(re), b(im);
    return {f2_of(a.hi, b.hi), f2_of(a.lo, b.lo)};
  } else {
    return {T(re), T(im)};
  }
}
template <typename T>
__device__ __forceinline__ void cx_to(cx<T> a, double& re, double& im) {
  if constexpr (std::is_same<T, ff>::value) {
    float rh, ih, rl, il;
    f2_split(a.hi, rh, ih);
    f2_split(a.lo, rl, il);
    re = (double)rh + (double)rl;
    im = (double)ih + (double)il;
  } else {
    re = (double)a.x;
    im = (double)a.y;
  }
}

__device__ __forceinline__ cx<ff> cadd(cx<ff> a, cx<ff> b) { return of2(as2(a) + as2(b)); }
__device__ __forceinline__ cx<ff> csub(cx<ff> a, cx<ff> b) { return of2(as2(a) - as2(b)); }
__device__ __forceinline__ cx<ff> cscale(cx<ff> a, ff s) { return of2(as2(a) * ff2_bcast(s)); }

template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.x * s, a.y * s}; }
// i * s * a
template <typename T>
__device__ __forceinline__ cx<T> cimul(cx<T> a, T s) { return {-s * a.y, s * a.x}; }
// SIGN i a (negations only, no products; packed: a lane swap and a sign)
template <int SIGN, typename T>
__device__ __forceinline__ cx<T> rot_i(cx<T> a) {
  if constexpr (std::is_same<T, ff>::value) {
    if constexpr (SIGN > 0) return {neg2_0(swap2(a.hi)), neg2_0(swap2(a.lo))};
    else return {neg2_1(swap2(a.hi)), neg2_1(swap2(a.lo))};
  } else {
    if constexpr (SIGN > 0) return {-a.y, a.x};
    else return {a.y, -a.x};
  }
}
// A value about to be stored by the last stage of a transform: float-float
// operations leave their results unnormalised (ff.cuh), these stores renormalise.
template <typename T>
__device__ __forceinline__ cx<T> settle(cx<T> a) {
  if constexpr (std::is_same<T, ff>::value) return of2(ff2_settle(as2(a)));
  else return a;
}

// ---- small DFTs: X_q = sum_r v_r exp(SIGN 2 pi i r q / R) --------------------
template <typename T, int SIGN>
__device__ __forceinline__ void dft2(cx<T>* v) {
  const cx<T> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft3(cx<T>* v) {
  const T h = T(0.5);
  const T s3 = T(SIGN * 0.866025403784438646763723170752936183);  // SIGN sin(2 pi / 3)
  const cx<T> t1 = cadd(v[1], v[2]);
  const cx<T> t2 = {v[0].x - h * t1.x, v[0].y - h * t1.y};
  const cx<T> d = cimul(csub(v[1], v[2]), s3);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(t2, d);
  v[2] = csub(t2, d);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft4(cx<T>* v) {
  const cx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  const cx<T> c = cadd(v[1], v[3]), d = rot_i<SIGN>(csub(v[1], v[3]));
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft5(cx<T>* v) {
  // cos(2pi/5) = (sqrt5 - 1)/4, cos(4pi/5) = -(sqrt5 + 1)/4,
  // sin(2pi/5) = sqrt((5 + sqrt5)/8), sin(4pi/5) = sqrt((5 - sqrt5)/8)
  const T c1 = T(0.309016994374947424102293417182819059);
  const T c2 = T(-0.809016994374947424102293417182819059);
  const T s1 = T(SIGN * 0.951056516295153572116439333379382143);
  const T s2 = T(SIGN * 0.587785252292473129168705954639072769);
  const cx<T> a = v[0];
  const cx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const cx<T> t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const cx<T> r1 = {a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
  const cx<T> r2 = {a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
  // i (s1 t3 + s2 t4) and i (s2 t3 - s1 t4)
  const cx<T> i1 = {-(s1 * t3.y + s2 * t4.y), s1 * t3.x + s2 * t4.x};
  const cx<T> i2 = {-(s2 * t3.y - s1 * t4.y), s2 * t3.x - s1 * t4.x};
  v[0] = cadd(a, cadd(t1, t2));
  v[1] = cadd(r1, i1);
  v[4] = csub(r1, i1);
  v[2] = cadd(r2, i2);
  v[3] = csub(r2, i2);
}

// Radix 3 and 5 on packed float-float values: the constants as broadcast pairs,
// the products by +-i as lane swaps (rot_i); same operations as dft3 / dft5.
template <int SIGN>
__device__ __forceinline__ void dft3_ff(cx<ff>* v) {
  const ff2 half = {f2_of(0.5f, 0.5f), f2_of(0.5f, 0.5f)};   // exact scaling of both parts
  const ff2 s3 = ff2_bcast(ff(0.866025403784438646763723170752936183));   // sin(2 pi / 3)
  const ff2 a = as2(v[0]), t1 = as2(v[1]) + as2(v[2]);
  const ff2 t2 = a - ff2{mul2(t1.hi, half.hi), mul2(t1.lo, half.lo)};
  const cx<ff> d = rot_i<SIGN>(of2((as2(v[1]) - as2(v[2])) * s3));
  v[0] = of2(a + t1);
  v[1] = of2(t2 + as2(d));
  v[2] = of2(t2 - as2(d));
}

template <int SIGN>
__device__ __forceinline__ void dft5_ff(cx<ff>* v) {
  const ff2 c1 = ff2_bcast(ff(0.309016994374947424102293417182819059));
  const ff2 c2 = ff2_bcast(ff(-0.809016994374947424102293417182819059));
  const ff2 s1 = ff2_bcast(ff(0.951056516295153572116439333379382143));
  const ff2 s2 = ff2_bcast(ff(0.587785252292473129168705954639072769));
  const ff2 a = as2(v[0]);
  const ff2 t1 = as2(v[1]) + as2(v[4]), t2 = as2(v[2]) + as2(v[3]);
  const ff2 t3 = as2(v[1]) - as2(v[4]), t4 = as2(v[2]) - as2(v[3]);
  const ff2 r1 = (a + c1 * t1) + c2 * t2;
  const ff2 r2 = (a + c2 * t1) + c1 * t2;
  // SIGN i (|s1| t3 + |s2| t4) and SIGN i (|s2| t3 - |s1| t4)
  const ff2 i1 = as2(rot_i<SIGN>(of2(s1 * t3 + s2 * t4)));
  const ff2 i2 = as2(rot_i<SIGN>(of2(s2 * t3 - s1 * t4)));
  v[0] = of2(a + (t1 + t2));
  v[1] = of2(r1 + i1);
  v[4] = of2(r1 - i1);
  v[2] = of2(r2 + i2);
  v[3] = of2(r2 - i2);
}

template <typename T, int SIGN, int R>
__device__ __forceinline__ void dftR(cx<T>* v) {
  constexpr bool kFF = std::is_same<T, ff>::value;
  if constexpr (R == 2) {
    dft2<T, SIGN>(v);
  } else if constexpr (R == 3) {
    if constexpr (kFF) dft3_ff<SIGN>(v);
    else dft3<T, SIGN>(v);
  } else if constexpr (R == 4) {
    dft4<T, SIGN>(v);
  } else {
    if constexpr (kFF) dft5_ff<SIGN>(v);
    else dft5<T, SIGN>(v);
  }
}

// Twiddle exp(SIGN 2 pi i t / n) from the table tw[t] = exp(-2 pi i t / n).
template <typename T, int SIGN>
__device__ __forceinline__ cx<T> twid(const cx<T>* tw, int t) {
  const cx<T> w = tw[t];
  return SIGN < 0 ? w : cx<T>{w.x, -w.y};
}

// ---- (c, t) twiddles: w = c (1 + i t), c = cos a, t = tan a -----------------------
// FP64 transforms keep their tables in this form, so that a twiddle applied before
// a butterfly costs two FMAs and its factor c folds into the butterfly's own
// additions (the FMA formulation of twiddled butterflies, Goedecker 1993): a
// radix-2 butterfly takes 6 instead of 8 FP64 instructions, a radix-4 one 24
// instead of 28.  The rounding error stays ~eps |v| for any t: c (v.x - t v.y)
// rounds at |t v.y| and is then scaled by c, |c t| = |sin a| <= 1.  Quarter
// turns (c = 0) are stored as c = 2^-60, t = +-2^60 (the product then equals
// -+v.y to within 2^-60 |v.x| + eps |v.y|).
template <typename T>
__host__ __device__ constexpr bool ct_twiddles() { return sizeof(T) == 8; }

// v (1 + i t)
template <typename T>
__device__ __forceinline__ cx<T> rot1(cx<T> v, T t) { return {fma(-t, v.y, v.x), fma(t, v.x, v.y)}; }
// a + s u
template <typename T>
__device__ __forceinline__ cx<T> caxpy(cx<T> a, T s, cx<T> u) { return {fma(s, u.x, a.x), fma(s, u.y, a.y)}; }

// Division by a divisor fixed for a whole stage: q = hi32(x * ceil(2^32 / d)),
// exact for x, d < 2^16 (x d < 2^32 bounds the rounding of the multiplier
// below the gap 1/d between x/d and the next integer).  Replaces the runtime
// integer divisions in the butterfly index arithmetic.  Every index it divides
// counts elements of one shared-memory tile (at most 227 KB / 8 B < 2^15), and
// every divisor is a line count or length within that tile.
struct FastDiv {
  unsigned d, m;
  __device__ __forceinline__ explicit FastDiv(int dv) : d((unsigned)dv) {
    m = d <= 1 ? 0u : (unsigned)(0xFFFFFFFFu / d) + 1u;
  }
  __device__ __forceinline__ int div(int x) const {
    return d <= 1 ? x : (int)__umulhi((unsigned)x, m);
  }
};

// x = a + s u, y = a - s u (two FMAs each part)
template <typename T>
__device__ __forceinline__ void axpm(cx<T> a, T s, cx<T> u, cx<T>& x, cx<T>& y) {
  x = caxpy(a, s, u);
  y = caxpy(a, -s, u);
}

// ---- the same butterflies on packed float-float values ---------------------------
// Table entry t is two values: C = (c, c) and T = (-t, t) as pairs (c and t of
// exp(-2 pi i t / n)), so that v (1 + i t) = v + T * (v.im, v.re) is one fused
// pair operation on the lane-swapped v, and a scale by c one pair product.  The
// conjugate twiddle (SIGN > 0) negates T.  a +- c u share the product c u (the
// same results as two fused operations: their two-sums are exact).
template <int SIGN>
__device__ __forceinline__ ff2 tw_t(const cx<ff>* tw, int t) {
  const ff2 x = as2(tw[2 * t + 1]);
  if constexpr (SIGN < 0) return x;
  else return {neg2(x.hi), neg2(x.lo)};
}
__device__ __forceinline__ ff2 tw_c(const cx<ff>* tw, int t) { return as2(tw[2 * t]); }
// v (1 + i t) with tt = (-t, t)
__device__ __forceinline__ ff2 rot1_ff(ff2 v, ff2 tt) {
  return tt * ff2{swap2(v.hi), swap2(v.lo)} + v;
}
__device__ __forceinline__ void axpm_ff(ff2 a, ff2 c, ff2 u, ff2& x, ff2& y) {
  const ff2 p = c * u;
  x = a + p;
  y = a - p;
}
template <int SIGN>
__device__ __forceinline__ ff2 rot_i_ff(ff2 a) { return as2(rot_i<SIGN>(of2(a))); }

template <int SIGN, int R>
__device__ __forceinline__ void bfly_ct_ff(cx<ff>* v, const cx<ff>* tw, int i1) {
  if constexpr (R == 2) {
    const ff2 u = rot1_ff(as2(v[1]), tw_t<SIGN>(tw, i1));
    ff2 x, y;
    axpm_ff(as2(v[0]), tw_c(tw, i1), u, x, y);
    v[0] = of2(x);
    v[1] = of2(y);
  } else if constexpr (R == 4) {
    const ff2 t1 = tw_t<SIGN>(tw, i1), t2 = tw_t<SIGN>(tw, 2 * i1);
    const ff2 c1 = tw_c(tw, i1), c2 = tw_c(tw, 2 * i1);
    const ff2 u2 = rot1_ff(as2(v[2]), t2), u3 = rot1_ff(as2(v[3]), t2);
    ff2 a, b, e, f, x0, x1, x2, x3;
    axpm_ff(as2(v[0]), c2, u2, a, b);
    axpm_ff(as2(v[1]), c2, u3, e, f);
    e = rot1_ff(e, t1);
    f = rot1_ff(f, t1);
    axpm_ff(a, c1, e, x0, x2);
    axpm_ff(b, c1, rot_i_ff<SIGN>(f), x1, x3);
    v[0] = of2(x0);
    v[1] = of2(x1);
    v[2] = of2(x2);
    v[3] = of2(x3);
  } else {
#pragma unroll
    for (int q = 1; q < R; ++q)
      v[q] = of2(tw_c(tw, q * i1) * rot1_ff(as2(v[q]), tw_t<SIGN>(tw, q * i1)));
    dftR<ff, SIGN, R>(v);
  }
}

template <int SIGN>
__device__ __forceinline__ void bfly_ct_ends_ff(const cx<ff>* v, const cx<ff>* tw, int i1,
                                                cx<ff>& x0, cx<ff>& x3) {
  const ff2 t1 = tw_t<SIGN>(tw, i1), t2 = tw_t<SIGN>(tw, 2 * i1);
  const ff2 c1 = tw_c(tw, i1), c2 = tw_c(tw, 2 * i1);
  const ff2 u2 = rot1_ff(as2(v[2]), t2), u3 = rot1_ff(as2(v[3]), t2);
  ff2 a, b, e, f;
  axpm_ff(as2(v[0]), c2, u2, a, b);
  axpm_ff(as2(v[1]), c2, u3, e, f);
  e = rot1_ff(e, t1);
  f = rot1_ff(f, t1);
  x0 = of2(c1 * e + a);
  x3 = of2(b - c1 * rot_i_ff<SIGN>(f));
}

// Twiddled butterfly on (c, t) tables: y_0 = v_0, y_q = w^q v_q (w^q = tw[q i1],
// conjugated for SIGN > 0), then the R-point DFT of y.  Radix 4 uses w^3 = w w^2:
// y_1 + y_3 = w (v_1 + w^2 v_3) and y_1 - y_3 = w (v_1 - w^2 v_3), so only w and
// w^2 are read, each scale c multiplying into an FMA of the butterfly.
template <typename T, int SIGN, int R>
__device__ __forceinline__ void bfly_ct(cx<T>* v, const cx<T>* tw, int i1) {
  if constexpr (std::is_same<T, ff>::value) {
    bfly_ct_ff<SIGN, R>(v, tw, i1);
  } else if constexpr (R == 2) {
    const cx<T> w1 = twid<T, SIGN>(tw, i1);
    const cx<T> u = rot1(v[1], w1.y), a = v[0];
    axpm(a, w1.x, u, v[0], v[1]);
  } else if constexpr (R == 4) {
    const cx<T> w1 = twid<T, SIGN>(tw, i1), w2 = twid<T, SIGN>(tw, 2 * i1);
    const cx<T> u2 = rot1(v[2], w2.y), u3 = rot1(v[3], w2.y);
    cx<T> a, b, e, f;
    axpm(v[0], w2.x, u2, a, b);
    axpm(v[1], w2.x, u3, e, f);
    e = rot1(e, w1.y);   // (y_1 + y_3) / c_1
    f = rot1(f, w1.y);   // (y_1 - y_3) / c_1
    // X_0,2 = a +- (y_1 + y_3), X_1,3 = b +- SIGN i (y_1 - y_3)
    axpm(a, w1.x, e, v[0], v[2]);
    axpm(b, w1.x, rot_i<SIGN>(f), v[1], v[3]);
  } else {
#pragma unroll
    for (int q = 1; q < R; ++q) {
      const cx<T> w = twid<T, SIGN>(tw, q * i1);
      const cx<T> u = rot1(v[q], w.y);
      v[q] = {w.x * u.x, w.x * u.y};
    }
    dftR<T, SIGN, R>(v);
  }
}

// Outputs 0 and 3 of the twiddled radix-4 butterfly bfly_ct (the forward stage
// whose outputs 1 and 2 are never read): 20 instead of 24 FP64 instructions.
template <typename T, int SIGN>
__device__ __forceinline__ void bfly_ct_ends(const cx<T>* v, const cx<T>* tw, int i1, cx<T>& x0,
                                             cx<T>& x3) {
  if constexpr (std::is_same<T, ff>::value) {
    bfly_ct_ends_ff<SIGN>(v, tw, i1, x0, x3);
    return;
  } else {
  const cx<T> w1 = twid<T, SIGN>(tw, i1), w2 = twid<T, SIGN>(tw, 2 * i1);
  const cx<T> u2 = rot1(v[2], w2.y), u3 = rot1(v[3], w2.y);
  cx<T> a, b, e, f;
  axpm(v[0], w2.x, u2, a, b);
  axpm(v[1], w2.x, u3, e, f);
  e = rot1(e, w1.y);
  f = rot1(f, w1.y);
  x0 = caxpy(a, w1.x, e);
  x3 = caxpy(b, -w1.x, rot_i<SIGN>(f));
  }
}

// One radix-R stage over `nlines` lines of length n.  Element e of line l sits
// at base[lofs(l) + e * es], lofs(l) = lofs_tab ? lofs_tab[l] : l * ls.
// line_fast selects which index varies fastest across consecutive threads
// (pick the one that makes consecutive threads touch consecutive addresses).
//
// Without CT (tables of w itself): DIF applies the R-point DFT and then the
// twiddles w_L^{jq} to its outputs; DIT applies w_L^{jq} to its inputs and then
// the DFT.  With CT ((c, t) tables) both directions twiddle the inputs:
//   * DIT as above (digit-reversed in, natural out);
//   * the DIF traversal (natural in, digit-reversed out) becomes decimation in
//     time with natural-order input: the butterfly of block blk and offset j
//     combines the same elements blk L + j + q M, but first multiplies element q
//     by w^{q k M}, k = perm[blk L] the frequency held at the block's first
//     position (perm = the digit reversal of the stages), and leaves the same
//     digit-reversed order.  Block 0 (the whole first stage) needs no twiddles.
// prune (CT, radix 4, the stage of span n): the data vanish (inverse input) or
// are not needed (forward output) outside [0, K] + [n - K, n), K < n / 4 (a
// sphere padded by at least 2x), which excludes positions q = 1, 2 of every
// butterfly: the first inverse stage neither reads nor adds its inputs 1 and 2,
// the last forward stage computes only its outputs 0 and 3.
template <typename T, int SIGN, bool DIT, int R, bool CT>
__device__ __forceinline__ void fft_stage(cx<T>* base, int es, int ls, const int* lofs_tab,
                                          int nlines, bool line_fast, int n, int L,
                                          const cx<T>* tw, const int* perm, bool prune,
                                          bool fin) {
  const int M = L / R;
  const int per_line = n / R;
  const int nit = nlines * per_line;
  const int tstep = n / L;
  const FastDiv fd_lines(nlines), fd_per(per_line), fd_m(M);
  for (int it = threadIdx.x; it < nit; it += blockDim.x) {
    int line, rest;
    if (line_fast) { rest = fd_lines.div(it); line = it - rest * nlines; }
    else { line = fd_per.div(it); rest = it - line * per_line; }
    const int blk = fd_m.div(rest);
    const int j = rest - blk * M;
    const int off = lofs_tab ? lofs_tab[line] : line * ls;
    cx<T>* p = base + off + (blk * L + j) * es;
    const int step = M * es;
    cx<T> v[R];
    if constexpr (CT && !DIT && R == 4) {
      if (prune) {
        const cx<T> a = p[0], d = p[3 * step], id = rot_i<SIGN>(d);
        p[0] = cadd(a, d);
        p[2 * step] = csub(a, d);
        p[step] = csub(a, id);
        p[3 * step] = cadd(a, id);
        continue;
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = p[q * step];
    if constexpr (CT && DIT && R == 4) {
      if (prune) {
        // last forward stage of a padded transform: outputs q = 1, 2 fall
        // outside [0, K] + [n - K, n) and are never read, so only X_0 and X_3
        cx<T> x0, x3;
        if (j != 0) {
          bfly_ct_ends<T, SIGN>(v, tw, j * tstep, x0, x3);
        } else {
          const cx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
          const cx<T> c = cadd(v[1], v[3]), d = rot_i<SIGN>(csub(v[1], v[3]));
          x0 = cadd(a, c);
          x3 = csub(b, d);
        }
        p[0] = settle(x0);
        p[3 * step] = settle(x3);
        continue;
      }
    }
    if constexpr (CT) {
      // twiddle index of input 1 (0: every twiddle is 1); consecutive threads
      // share blk and j in the line-fast passes, so the branch is warp-uniform
      const int i1 = DIT ? j * tstep : (blk == 0 ? 0 : __ldg(perm + blk * L) * M);
      if (i1 != 0) bfly_ct<T, SIGN, R>(v, tw, i1);
      else dftR<T, SIGN, R>(v);
    } else if constexpr (DIT) {
      // j == 0 (every butterfly when M == 1): every twiddle is 1, skip the
      // products; consecutive threads share j in the line-fast passes, so the
      // branch is uniform across most warps
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(v[q], twid<T, SIGN>(tw, j * q * tstep));
      }
      dftR<T, SIGN, R>(v);
    } else {
      dftR<T, SIGN, R>(v);
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmul(v[q], twid<T, SIGN>(tw, j * q * tstep));
      }
    }
    if (fin) {   // uniform across the block: one branch per stage, no per-value select
#pragma unroll
      for (int q = 0; q < R; ++q) p[q * step] = settle(v[q]);
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) p[q * step] = v[q];
    }
  }
}

template <typename T, int SIGN, bool DIT, bool CT>
__device__ __forceinline__ void fft_stage_any(cx<T>* base, int es, int ls, const int* lofs,
                                              int nlines, bool line_fast, int n, int R, int L,
                                              const cx<T>* tw, const int* perm, bool prune,
                                              bool fin) {
  switch (R) {
    case 2: fft_stage<T, SIGN, DIT, 2, CT>(base, es, ls, lofs, nlines, line_fast, n, L, tw, perm, false, fin); break;
    case 3: fft_stage<T, SIGN, DIT, 3, CT>(base, es, ls, lofs, nlines, line_fast, n, L, tw, perm, false, fin); break;
    case 4: fft_stage<T, SIGN, DIT, 4, CT>(base, es, ls, lofs, nlines, line_fast, n, L, tw, perm, prune, fin); break;
    default: fft_stage<T, SIGN, DIT, 5, CT>(base, es, ls, lofs, nlines, line_fast, n, L, tw, perm, false, fin); break;
  }
}

// Two consecutive stages fused in registers: stage a (radix RA over spans of
// length L) and stage b (radix RB over the spans of length L / RA it leaves).
// A work item holds the RA x RB elements blk L + jb + qb Mb + qa Ma (Ma = L/RA,
// Mb = Ma/RB, qa < RA, qb < RB): exactly the elements that the RB stage-a
// butterflies j = jb + qb Mb produce and the RA stage-b butterflies j = jb
// consume.  Every element sees the same operations in the same order as in
// two separate stages (bit-identical results), with one shared-memory round
// trip and one barrier instead of two.  DIF applies a then b, DIT b then a.
template <typename T, int SIGN, bool DIT, int RA, int RB>
__device__ __forceinline__ void fft_stage2(cx<T>* base, int es, int ls, const int* lofs_tab,
                                           int nlines, bool line_fast, int n, int L,
                                           const cx<T>* tw) {
  const int Ma = L / RA, Mb = Ma / RB;
  const int per_line = n / (RA * RB);
  const int nit = nlines * per_line;
  const int tsa = n / L, tsb = n / Ma;
  const FastDiv fd_lines(nlines), fd_per(per_line), fd_mb(Mb);
  for (int it = threadIdx.x; it < nit; it += blockDim.x) {
    int line, rest;
    if (line_fast) { rest = fd_lines.div(it); line = it - rest * nlines; }
    else { line = fd_per.div(it); rest = it - line * per_line; }
    const int blk = fd_mb.div(rest);
    const int jb = rest - blk * Mb;
    const int off = lofs_tab ? lofs_tab[line] : line * ls;
    cx<T>* p = base + off + (blk * L + jb) * es;
    const int sa = Ma * es, sb = Mb * es;
    cx<T> v[RA][RB];
#pragma unroll
    for (int qa = 0; qa < RA; ++qa)
#pragma unroll
      for (int qb = 0; qb < RB; ++qb) v[qa][qb] = p[qa * sa + qb * sb];
    if (!DIT) {
#pragma unroll
      for (int qb = 0; qb < RB; ++qb) {
        cx<T> u[RA];
#pragma unroll
        for (int qa = 0; qa < RA; ++qa) u[qa] = v[qa][qb];
        dftR<T, SIGN, RA>(u);
        const int ja = jb + qb * Mb;
#pragma unroll
        for (int qa = 1; qa < RA; ++qa) u[qa] = cmul(u[qa], twid<T, SIGN>(tw, ja * qa * tsa));
#pragma unroll
        for (int qa = 0; qa < RA; ++qa) v[qa][qb] = u[qa];
      }
#pragma unroll
      for (int qa = 0; qa < RA; ++qa) {
        dftR<T, SIGN, RB>(v[qa]);
        if (Mb > 1) {
#pragma unroll
          for (int qb = 1; qb < RB; ++qb) v[qa][qb] = cmul(v[qa][qb], twid<T, SIGN>(tw, jb * qb * tsb));
        }
      }
    } else {
#pragma unroll
      for (int qa = 0; qa < RA; ++qa) {
        if (Mb > 1) {
#pragma unroll
          for (int qb = 1; qb < RB; ++qb) v[qa][qb] = cmul(v[qa][qb], twid<T, SIGN>(tw, jb * qb * tsb));
        }
        dftR<T, SIGN, RB>(v[qa]);
      }
#pragma unroll
      for (int qb = 0; qb < RB; ++qb) {
        cx<T> u[RA];
#pragma unroll
        for (int qa = 0; qa < RA; ++qa) u[qa] = v[qa][qb];
        const int ja = jb + qb * Mb;
#pragma unroll
        for (int qa = 1; qa < RA; ++qa) u[qa] = cmul(u[qa], twid<T, SIGN>(tw, ja * qa * tsa));
        dftR<T, SIGN, RA>(u);
#pragma unroll
        for (int qa = 0; qa < RA; ++qa) v[qa][qb] = u[qa];
      }
    }
#pragma unroll
    for (int qa = 0; qa < RA; ++qa)
#pragma unroll
      for (int qb = 0; qb < RB; ++qb) p[qa * sa + qb * sb] = v[qa][qb];
  }
}

// Largest register tile of a fused pair (complex elements per work item).
template <typename T>
__host__ __device__ constexpr int fuse_limit() { return sizeof(T) == 8 ? 16 : 20; }

template <typename T, int SIGN, bool DIT, int RA>
__device__ __forceinline__ void fft_stage2_b(cx<T>* base, int es, int ls, const int* lofs,
                                             int nlines, bool line_fast, int n, int RB, int L,
                                             const cx<T>* tw) {
  switch (RB) {
    case 2: fft_stage2<T, SIGN, DIT, RA, 2>(base, es, ls, lofs, nlines, line_fast, n, L, tw); break;
    case 3: fft_stage2<T, SIGN, DIT, RA, 3>(base, es, ls, lofs, nlines, line_fast, n, L, tw); break;
    case 4: fft_stage2<T, SIGN, DIT, RA, 4>(base, es, ls, lofs, nlines, line_fast, n, L, tw); break;
    default:
      if constexpr (RA * 5 <= fuse_limit<T>())
        fft_stage2<T, SIGN, DIT, RA, 5>(base, es, ls, lofs, nlines, line_fast, n, L, tw);
      break;
  }
}

template <typename T, int SIGN, bool DIT>
__device__ __forceinline__ void fft_stage2_any(cx<T>* base, int es, int ls, const int* lofs,
                                               int nlines, bool line_fast, int n, int RA, int RB,
                                               int L, const cx<T>* tw) {
  switch (RA) {
    case 2: fft_stage2_b<T, SIGN, DIT, 2>(base, es, ls, lofs, nlines, line_fast, n, RB, L, tw); break;
    case 3: fft_stage2_b<T, SIGN, DIT, 3>(base, es, ls, lofs, nlines, line_fast, n, RB, L, tw); break;
    case 4: fft_stage2_b<T, SIGN, DIT, 4>(base, es, ls, lofs, nlines, line_fast, n, RB, L, tw); break;
    default: fft_stage2_b<T, SIGN, DIT, 5>(base, es, ls, lofs, nlines, line_fast, n, RB, L, tw); break;
  }
}

// Whole in-place transform of every line; ends with __syncthreads().
// Must be called by every thread of the block.  With FUSE, consecutive stages
// are fused in pairs while the pair's register tile stays within fuse_limit
// (same results; fewer shared-memory passes for more registers per thread).
// FP64 (ct_twiddles) runs unfused on a (c, t) table; its DIF traversal needs
// perm (the digit reversal of rp); prune drops the padding in the stage of span
// n (the first inverse, the last forward stage; fft_stage).
template <typename T, int SIGN, bool DIT, bool FUSE = false>
__device__ void fft_lines(cx<T>* base, int es, int ls, const int* lofs, int nlines,
                          bool line_fast, const Radix& rp, const cx<T>* tw,
                          const int* perm = nullptr, bool prune = false) {
  constexpr bool CT = ct_twiddles<T>();
  static_assert(!(CT && FUSE), "fused stage pairs take tables of w");
  if (!DIT) {
    int s = 0;
    while (s < rp.nst) {
      bool fused = false;
      if constexpr (FUSE) {
        if (s + 1 < rp.nst && rp.r[s] * rp.r[s + 1] <= fuse_limit<T>()) {
          fft_stage2_any<T, SIGN, false>(base, es, ls, lofs, nlines, line_fast, rp.n, rp.r[s],
                                         rp.r[s + 1], rp.L[s], tw);
          s += 2;
          fused = true;
        }
      }
      if (!fused) {
        fft_stage_any<T, SIGN, false, CT>(base, es, ls, lofs, nlines, line_fast, rp.n, rp.r[s],
                                          rp.L[s], tw, perm, prune && s == 0, s == rp.nst - 1);
        s += 1;
      }
      __syncthreads();
    }
  } else {
    int s = rp.nst - 1;
    while (s >= 0) {
      bool fused = false;
      if constexpr (FUSE) {
        if (s >= 1 && rp.r[s - 1] * rp.r[s] <= fuse_limit<T>()) {
          fft_stage2_any<T, SIGN, true>(base, es, ls, lofs, nlines, line_fast, rp.n, rp.r[s - 1],
                                        rp.r[s], rp.L[s - 1], tw);
          s -= 2;
          fused = true;
        }
      }
      if (!fused) {
        fft_stage_any<T, SIGN, true, CT>(base, es, ls, lofs, nlines, line_fast, rp.n, rp.r[s],
                                         rp.L[s], tw, perm, prune && s == 0, s == 0);
        s -= 1;
      }
      __syncthreads();
    }
  }
}

}  // namespace qe
