// Plane transforms with register-resident sub-transforms (square planes of a
// compile-time size N = A * B).
//
// A length-N line transform runs in two passes over shared memory (the
// "four-step" split of Cooley and Tukey):
//   inverse (G -> r, natural input):
//     pass 1, for each n2 < B: the A-point DFT over n1 of x[B n1 + n2], times
//             w_N^{+n2 k1}, stored back at B k1 + n2;
//     pass 2, for each k1 < A: the B-point DFT over n2 of the B contiguous
//             values at B k1 + n2, stored at B k1 + k2;
//     so that position B k1 + k2 holds the value of index r = k1 + A k2;
//   forward (r -> G, input in that order, natural output):
//     pass 1, for each k1 < A: the B-point DFT over k2 of the contiguous
//             values at B k1 + k2, times w_N^{-k1 m2}, stored at B k1 + m2;
//     pass 2, for each m2 < B: the A-point DFT over k1 of the values at
//             B k1 + m2, stored at B m1 + m2 = m.
// Each A- or B-point DFT is one thread's work on values held in registers: a
// compile-time mixed-radix transform (radices 4 first, then 2, 3, 5), so that
// every index and every twiddle index inside it is a constant (trivial
// twiddles 1, -1, +-i are folded away).  The inverse pass 2 and the forward
// pass 1 of the x lines touch the same B values of a row, so the V multiply
// sits between them in registers: one plane pair takes 7 barriers.
//
// Sphere padding (K < N/4, the half-width of the sticks' range on an axis):
// the inverse input is zero for n1 in [A/4, 3A/4), which drops two inputs of
// every butterfly of the first radix-4 stage; the forward output is read only
// for m1 outside [A/4, 3A/4), which drops two outputs of the last one.
#pragma once

#include <type_traits>

#include "fft_device.cuh"

namespace qe {

// ---- compile-time radix plan of a register transform of length R -------------------
__host__ __device__ constexpr int rr_count(int R) {
  int n = 0;
  while (R % 4 == 0) { R /= 4; ++n; }
  while (R % 2 == 0) { R /= 2; ++n; }
  while (R % 3 == 0) { R /= 3; ++n; }
  while (R % 5 == 0) { R /= 5; ++n; }
  return n;
}
__host__ __device__ constexpr int rr_radix(int R, int s) {
  int n = 0;
  while (R % 4 == 0) { if (n == s) return 4; R /= 4; ++n; }
  while (R % 2 == 0) { if (n == s) return 2; R /= 2; ++n; }
  while (R % 3 == 0) { if (n == s) return 3; R /= 3; ++n; }
  while (R % 5 == 0) { if (n == s) return 5; R /= 5; ++n; }
  return 1;
}
// span of stage s (the sub-transform length it splits)
__host__ __device__ constexpr int rr_span(int R, int s) {
  int L = R;
  for (int i = 0; i < s; ++i) L /= rr_radix(R, i);
  return L;
}
// frequency held at register p after the in-place DIF stages (natural input)
__host__ __device__ constexpr int rr_rev(int R, int p) {
  int k = 0, w = 1, rest = p;
  for (int s = 0; s < rr_count(R); ++s) {
    const int r = rr_radix(R, s), M = rr_span(R, s) / r;
    const int q = rest / M;
    rest -= q * M;
    k += q * w;
    w *= r;
  }
  return k;
}
// line position of index r (0 <= r < A B) in the two-pass order: B (r mod A) + r div A
__host__ __device__ constexpr int sq_pos(int A, int B, int r) { return B * (r % A) + r / A; }

// ---- twiddle tables ---------------------------------------------------------------------
// Table of w_t = exp(-2 pi i t / NT), t < NT.  float / double: w itself.  Float-float:
// two entries per t, (c, c) and (-s, s) with w = c - i s... written as ff pairs, so that
// v w = v (c, c) + swap(v) (-s, s) is one pair product and one fused pair operation.
template <typename T>
__host__ __device__ constexpr int sq_tw_slots() { return std::is_same<T, ff>::value ? 2 : 1; }

template <typename T>
__device__ __forceinline__ void sq_tw_put(cx<T>* tab, int t, double re, double im) {
  if constexpr (std::is_same<T, ff>::value) {
    const ff c(re), s(im);
    tab[2 * t] = {f2_of(c.hi, c.hi), f2_of(c.lo, c.lo)};
    tab[2 * t + 1] = {f2_of(-s.hi, s.hi), f2_of(-s.lo, s.lo)};
  } else {
    tab[t] = {T(re), T(im)};
  }
}

// v exp(SIGN 2 pi i t / NT) from the table (t < NT)
template <typename T, int SIGN>
__device__ __forceinline__ cx<T> sq_twmul(cx<T> v, const cx<T>* tab, int t) {
  if constexpr (std::is_same<T, ff>::value) {
    const ff2 a = as2(v);
    const ff2 p = a * as2(tab[2 * t]);
    const ff2 sw = {swap2(a.hi), swap2(a.lo)};
    ff2 s = as2(tab[2 * t + 1]);
    if constexpr (SIGN > 0) s = {neg2(s.hi), neg2(s.lo)};
    return of2(s * sw + p);
  } else {
    const cx<T> w = tab[t];
    const T wi = SIGN < 0 ? w.y : -w.y;
    return {v.x * w.x - v.y * wi, v.x * wi + v.y * w.x};
  }
}

template <typename T>
__device__ __forceinline__ cx<T> sq_neg(cx<T> a) {
  if constexpr (std::is_same<T, ff>::value) return {neg2(a.hi), neg2(a.lo)};
  else return {-a.x, -a.y};
}

// v exp(SIGN 2 pi i TI / NT) for a compile-time index: 1, -1, +-i folded away
template <typename T, int SIGN, int NT, int TI>
__device__ __forceinline__ cx<T> sq_twc(cx<T> v, const cx<T>* tab) {
  constexpr int t = TI % NT;
  if constexpr (t == 0) return v;
  else if constexpr (4 * t == NT) return rot_i<SIGN>(v);
  else if constexpr (2 * t == NT) return sq_neg<T>(v);
  else if constexpr (4 * t == 3 * NT) return rot_i<-SIGN>(v);
  else return sq_twmul<T, SIGN>(v, tab, t);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1.
template <int I, int N, typename F>
__device__ __forceinline__ void sfor_from(F& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    sfor_from<I + 1, N>(f);
  }
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_from<0, N>(f);
}

// ---- register transforms ---------------------------------------------------------------
// DIF stage S of a length-R transform on v[0..R): butterflies over q of
// v[blk L + j + q M], then v[.. + q M] *= w_L^{SIGN j q} (w_L^x = w_NT^{x NT / L}).
// PRUNE (stage 0, radix 4): inputs q = 1, 2 are zero.
template <typename T, int SIGN, int R, int NT, int S, bool PRUNE>
__device__ __forceinline__ void rr_dif_stage(cx<T>* v, const cx<T>* tab) {
  constexpr int r = rr_radix(R, S), L = rr_span(R, S), M = L / r;
  sfor<R / L>([&](auto BLK) {
    sfor<M>([&](auto J) {
      constexpr int o = decltype(BLK)::value * L + decltype(J)::value;
      constexpr int tj = decltype(J)::value * (NT / L);
      cx<T> u[r];
      if constexpr (PRUNE && S == 0 && r == 4) {
        const cx<T> a = v[o], d = v[o + 3 * M], id = rot_i<SIGN>(d);
        u[0] = cadd(a, d);
        u[2] = csub(a, d);
        u[1] = csub(a, id);
        u[3] = cadd(a, id);
      } else {
#pragma unroll
        for (int q = 0; q < r; ++q) u[q] = v[o + q * M];
        dftR<T, SIGN, r>(u);
      }
      v[o] = u[0];
      sfor<r - 1>([&](auto Q) {
        constexpr int q = decltype(Q)::value + 1;
        v[o + q * M] = sq_twc<T, SIGN, NT, tj * q>(u[q], tab);
      });
    });
  });
}

template <typename T, int SIGN, int R, int NT, int S, bool PRUNE>
__device__ __forceinline__ void rr_dif_from(cx<T>* v, const cx<T>* tab) {
  if constexpr (S < rr_count(R)) {
    rr_dif_stage<T, SIGN, R, NT, S, PRUNE>(v, tab);
    rr_dif_from<T, SIGN, R, NT, S + 1, PRUNE>(v, tab);
  }
}

// Natural input, v[p] = X[rr_rev(R, p)] out.
template <typename T, int SIGN, int R, int NT, bool PRUNE>
__device__ __forceinline__ void rr_dif(cx<T>* v, const cx<T>* tab) {
  rr_dif_from<T, SIGN, R, NT, 0, PRUNE>(v, tab);
}

// DIT stage S (the transpose of the DIF stage): twiddles first, then the
// butterflies.  PRUNE (stage 0, radix 4): only outputs q = 0 and 3 are formed
// (the others are left as they are and must not be read).
template <typename T, int SIGN, int R, int NT, int S, bool PRUNE>
__device__ __forceinline__ void rr_dit_stage(cx<T>* v, const cx<T>* tab) {
  constexpr int r = rr_radix(R, S), L = rr_span(R, S), M = L / r;
  sfor<R / L>([&](auto BLK) {
    sfor<M>([&](auto J) {
      constexpr int o = decltype(BLK)::value * L + decltype(J)::value;
      constexpr int tj = decltype(J)::value * (NT / L);
      cx<T> u[r];
      u[0] = v[o];
      sfor<r - 1>([&](auto Q) {
        constexpr int q = decltype(Q)::value + 1;
        u[q] = sq_twc<T, SIGN, NT, tj * q>(v[o + q * M], tab);
      });
      if constexpr (PRUNE && S == 0 && r == 4) {
        const cx<T> a = cadd(u[0], u[2]), b = csub(u[0], u[2]);
        const cx<T> c = cadd(u[1], u[3]), d = rot_i<SIGN>(csub(u[1], u[3]));
        v[o] = cadd(a, c);
        v[o + 3 * M] = csub(b, d);
      } else {
        dftR<T, SIGN, r>(u);
#pragma unroll
        for (int q = 0; q < r; ++q) v[o + q * M] = u[q];
      }
    });
  });
}

template <typename T, int SIGN, int R, int NT, int S, bool PRUNE>
__device__ __forceinline__ void rr_dit_from(cx<T>* v, const cx<T>* tab) {
  if constexpr (S >= 0) {
    rr_dit_stage<T, SIGN, R, NT, S, PRUNE>(v, tab);
    rr_dit_from<T, SIGN, R, NT, S - 1, PRUNE>(v, tab);
  }
}

// v[p] = x[rr_rev(R, p)] in, natural order out.
template <typename T, int SIGN, int R, int NT, bool PRUNE>
__device__ __forceinline__ void rr_dit(cx<T>* v, const cx<T>* tab) {
  rr_dit_from<T, SIGN, R, NT, rr_count(R) - 1, PRUNE>(v, tab);
}

// ---- the passes of one line --------------------------------------------------------------
// Every pass is called for one (line, sub) work item; `p` points at the line's
// element 0 and `es` is the element stride.  Values are settled (float-float
// renormalised) where a transform ends.
template <int N>
struct SqSplit;
template <> struct SqSplit<96> { static constexpr int A = 12, B = 8; };
template <> struct SqSplit<48> { static constexpr int A = 12, B = 4; };
template <> struct SqSplit<32> { static constexpr int A = 8, B = 4; };

// inverse pass 1: n2 = sub
template <typename T, int N, bool PRUNE>
__device__ __forceinline__ void sq_inv1(cx<T>* p, int es, int n2, const cx<T>* tab) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B;
  cx<T> v[A];
#pragma unroll
  for (int n1 = 0; n1 < A; ++n1) {
    if (!PRUNE || n1 < A / 4 || n1 >= 3 * A / 4) v[n1] = p[(B * n1 + n2) * es];
    else v[n1] = cx_zero<T>();
  }
  rr_dif<T, +1, A, N, PRUNE>(v, tab);
  sfor<A>([&](auto I) {
    constexpr int i = decltype(I)::value, k1 = rr_rev(A, i);
    const cx<T> w = (k1 == 0 || n2 == 0) ? v[i] : sq_twmul<T, +1>(v[i], tab, n2 * k1);
    p[(B * k1 + n2) * es] = w;
  });
}

// inverse pass 2: k1 = sub; results settled (end of the inverse transform)
template <typename T, int N>
__device__ __forceinline__ void sq_inv2_regs(const cx<T>* p, int es, int k1, const cx<T>* tab,
                                            cx<T>* out) {
  constexpr int B = SqSplit<N>::B;
  cx<T> v[B];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) v[n2] = p[(B * k1 + n2) * es];
  rr_dif<T, +1, B, N, false>(v, tab);
  sfor<B>([&](auto I) {
    constexpr int i = decltype(I)::value;
    out[rr_rev(B, i)] = settle(v[i]);   // out[k2]
  });
}

// forward pass 1 on registers in[k2] (position B k1 + k2): out[m2], twiddled by w_N^{-k1 m2}
template <typename T, int N>
__device__ __forceinline__ void sq_fwd1_regs(const cx<T>* in, int k1, const cx<T>* tab, cx<T>* out) {
  constexpr int B = SqSplit<N>::B;
  cx<T> v[B];
  sfor<B>([&](auto I) {
    constexpr int i = decltype(I)::value;
    v[i] = in[rr_rev(B, i)];
  });
  rr_dit<T, -1, B, N, false>(v, tab);
  out[0] = v[0];
#pragma unroll
  for (int m2 = 1; m2 < B; ++m2) out[m2] = k1 == 0 ? v[m2] : sq_twmul<T, -1>(v[m2], tab, k1 * m2);
}

// forward pass 2: m2 = sub; results settled; PRUNE stores only m1 outside [A/4, 3A/4)
template <typename T, int N, bool PRUNE>
__device__ __forceinline__ void sq_fwd2(cx<T>* p, int es, int m2, const cx<T>* tab) {
  constexpr int A = SqSplit<N>::A, B = SqSplit<N>::B;
  cx<T> v[A];
  sfor<A>([&](auto I) {
    constexpr int i = decltype(I)::value;
    v[i] = p[(B * rr_rev(A, i) + m2) * es];
  });
  rr_dit<T, -1, A, N, PRUNE>(v, tab);
#pragma unroll
  for (int m1 = 0; m1 < A; ++m1)
    if (!PRUNE || m1 < A / 4 || m1 >= 3 * A / 4) p[(B * m1 + m2) * es] = settle(v[m1]);
}

}  // namespace qe
