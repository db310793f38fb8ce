// Shared-memory FFT engine for batches of short lines (one CTA, several lines).
//
// Stockham autosort (ping-pong between two shared-memory buffers, no bit
// reversal): stage s with radix R combines sub-transforms of size Ns into
// Ns*R.  Butterfly j (< n/R) reads x[j + r n/R], r < R, twiddles input r by
// w^{r k n/(Ns R)} (k = j mod Ns, w = exp(-2 pi i/n)), does an R-point DFT in
// registers and writes y[(j/Ns) Ns R + k + q Ns], q < R.  The divisions by
// the per-stage constants n/R and Ns use precomputed multiply-shift
// reciprocals.  Radices 2, 3, 4, 5, 7, 8, 9, 11, 13 and 17 have dedicated butterflies
// built from the constant roots of unity; other primes up to kMaxDirectPrime
// use one thread per output.  A prime length p whose p - 1 factors that way
// uses Rader's algorithm (the DFT as a cyclic convolution of length p - 1 in
// primitive-root order); other lengths with a larger prime factor use
// Bluestein: X = conj(c) . IFFT_m( FFT_m(x conj(c)) . FFT_m(b) / m ),
// c_j = exp(i pi j^2 / n), m smooth >= 2n - 1.
#pragma once

#include <cuda_runtime.h>

#include "fcsph_ff.cuh"
#include "fcsph_internal.h"

namespace fcsph {

template <typename T> struct CT;
template <> struct CT<double> { typedef double2 t; };
template <> struct CT<float> { typedef float2 t; };
template <> struct CT<ff> { typedef ff2 t; };

template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {  // a * conj(b)
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) {
  V r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename V> __device__ __forceinline__ V csub(V a, V b) {
  V r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
// Sums inside one butterfly: plain sums here; FP32-pair values skip the
// renormalisation (fcsph_ff.cuh) and cnorm restores it at the store.
template <typename V> __device__ __forceinline__ V cadd_nr(V a, V b) { return cadd(a, b); }
template <typename V> __device__ __forceinline__ V csub_nr(V a, V b) { return csub(a, b); }
template <typename V> __device__ __forceinline__ V cnorm(V a) { return a; }
template <typename V> __device__ __forceinline__ V cmul_nr(V a, V b) { return cmul(a, b); }
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) {
  V r;
  r.x = a.x * s;
  r.y = a.y * s;
  return r;
}
template <typename V, typename A, typename B> __device__ __forceinline__ V mk(A x, B y) {
  V r;
  r.x = x;
  r.y = y;
  return r;
}
// -i * a (forward sign) or +i * a (inverse)
template <typename V, bool INV> __device__ __forceinline__ V rot(V a) {
  return INV ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

// Root e of the length-n table, conjugated for the inverse transform.
template <typename V, bool INV> __device__ __forceinline__ V root(const V* __restrict__ tw, int e) {
  V w = tw[e];
  if (INV) w.y = -w.y;
  return w;
}

__device__ __forceinline__ int fdiv(int x, const FastDiv d) {
  return (int)((__umulhi((unsigned)x, d.m) + (unsigned)x) >> d.l);
}

// cos(2 pi j / R) and sin(2 pi j / R), j = 1..(R-1)/2, for the odd radices;
// cosk/sink extend them to any k by symmetry.  With unrolled loops k is a
// compile-time constant and the switch folds to an immediate.
template <int R> __device__ __forceinline__ double cos_tab(int j);
template <int R> __device__ __forceinline__ double sin_tab(int j);
template <> __device__ __forceinline__ double cos_tab<3>(int j) {
  switch (j) {
      case 1: return -0.4999999999999998;
    default: return 1.0;
  }
}
template <> __device__ __forceinline__ double sin_tab<3>(int j) {
  switch (j) {
      case 1: return 0.8660254037844387;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double cos_tab<5>(int j) {
  switch (j) {
      case 1: return 0.30901699437494745;
      case 2: return -0.8090169943749473;
    default: return 1.0;
  }
}
template <> __device__ __forceinline__ double sin_tab<5>(int j) {
  switch (j) {
      case 1: return 0.9510565162951535;
      case 2: return 0.5877852522924732;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double cos_tab<7>(int j) {
  switch (j) {
      case 1: return 0.6234898018587336;
      case 2: return -0.22252093395631434;
      case 3: return -0.900968867902419;
    default: return 1.0;
  }
}
template <> __device__ __forceinline__ double sin_tab<7>(int j) {
  switch (j) {
      case 1: return 0.7818314824680298;
      case 2: return 0.9749279121818236;
      case 3: return 0.43388373911755823;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double cos_tab<11>(int j) {
  switch (j) {
      case 1: return 0.8412535328311812;
      case 2: return 0.41541501300188644;
      case 3: return -0.142314838273285;
      case 4: return -0.654860733945285;
      case 5: return -0.9594929736144974;
    default: return 1.0;
  }
}
template <> __device__ __forceinline__ double sin_tab<11>(int j) {
  switch (j) {
      case 1: return 0.5406408174555976;
      case 2: return 0.9096319953545183;
      case 3: return 0.9898214418809328;
      case 4: return 0.7557495743542583;
      case 5: return 0.28173255684142967;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double cos_tab<13>(int j) {
  switch (j) {
      case 1: return 0.8854560256532099;
      case 2: return 0.5680647467311559;
      case 3: return 0.120536680255323;
      case 4: return -0.35460488704253545;
      case 5: return -0.7485107481711012;
      case 6: return -0.970941817426052;
    default: return 1.0;
  }
}
template <> __device__ __forceinline__ double sin_tab<13>(int j) {
  switch (j) {
      case 1: return 0.4647231720437685;
      case 2: return 0.8229838658936564;
      case 3: return 0.992708874098054;
      case 4: return 0.9350162426854148;
      case 5: return 0.6631226582407952;
      case 6: return 0.23931566428755768;
    default: return 0.0;
  }
}
template <> __device__ __forceinline__ double cos_tab<17>(int j) {
  switch (j) {
      case 1: return 0.9324722294043558;
      case 2: return 0.7390089172206591;
      case 3: return 0.4457383557765383;
      case 4: return 0.09226835946330202;
      case 5: return -0.2736629900720829;
      case 6: return -0.6026346363792563;
      case 7: return -0.850217135729614;
      case 8: return -0.9829730996839018;
    default: return 1.0;
  }
}
template <> __device__ __forceinline__ double sin_tab<17>(int j) {
  switch (j) {
      case 1: return 0.3612416661871529;
      case 2: return 0.6736956436465572;
      case 3: return 0.8951632913550623;
      case 4: return 0.9957341762950345;
      case 5: return 0.961825643172819;
      case 6: return 0.7980172272802396;
      case 7: return 0.5264321628773561;
      case 8: return 0.18374951781657037;
    default: return 0.0;
  }
}
template <int R> __device__ __forceinline__ double cosk(int k) {
  k %= R;
  return k == 0 ? 1.0 : cos_tab<R>(2 * k <= R ? k : R - k);
}
template <int R> __device__ __forceinline__ double sink(int k) {
  k %= R;
  return k == 0 ? 0.0 : (2 * k <= R ? sin_tab<R>(k) : -sin_tab<R>(R - k));
}

// Odd prime R: y_q = x0 + sum_{r<=h} [ (x_r + x_{R-r}) cos(2 pi r q/R)
//                                    -/+ i (x_r - x_{R-r}) sin(2 pi r q/R) ].
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_odd(typename CT<T>::t* v) {
  typedef typename CT<T>::t V;
  constexpr int h = (R - 1) / 2;
  V A[h], B[h];
#pragma unroll
  for (int r = 1; r <= h; ++r) {
    A[r - 1] = cadd_nr(v[r], v[R - r]);
    B[r - 1] = csub_nr(v[r], v[R - r]);
  }
  V o[R];
  V y0 = v[0];
#pragma unroll
  for (int r = 0; r < h; ++r) y0 = cadd_nr(y0, A[r]);
  o[0] = y0;
#pragma unroll
  for (int q = 1; q <= h; ++q) {
    V re = v[0];
    V im = mk<V>(0.0, 0.0);
#pragma unroll
    for (int r = 1; r <= h; ++r) {
      const T c = (T)cosk<R>((r * q) % R);
      const T s = (T)sink<R>((r * q) % R);
      re.x = madd_nr(re.x, A[r - 1].x, c);
      re.y = madd_nr(re.y, A[r - 1].y, c);
      im.x = madd_nr(im.x, B[r - 1].x, s);
      im.y = madd_nr(im.y, B[r - 1].y, s);
    }
    const V ri = rot<V, INV>(im);  // -i * im (forward)
    o[q] = cadd_nr(re, ri);
    o[R - q] = csub_nr(re, ri);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = o[q];
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(typename CT<T>::t& a0, typename CT<T>::t& a1, typename CT<T>::t& a2,
                                     typename CT<T>::t& a3) {
  typedef typename CT<T>::t V;
  const V t0 = cadd_nr(a0, a2), t1 = csub_nr(a0, a2);
  const V t2 = cadd_nr(a1, a3), t3 = rot<V, INV>(csub_nr(a1, a3));
  a0 = cadd_nr(t0, t2);
  a2 = csub_nr(t0, t2);
  a1 = cadd_nr(t1, t3);
  a3 = csub_nr(t1, t3);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft3(typename CT<T>::t& a0, typename CT<T>::t& a1, typename CT<T>::t& a2) {
  typename CT<T>::t v[3] = {a0, a1, a2};
  dft_odd<T, 3, INV>(v);
  a0 = v[0];
  a1 = v[1];
  a2 = v[2];
}

// In-register R-point DFT, v[q] <- sum_r v[r] w_R^{r q}.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(typename CT<T>::t* v) {
  typedef typename CT<T>::t V;
  if constexpr (R == 2) {
    const V a = v[0], b = v[1];
    v[0] = cadd_nr(a, b);
    v[1] = csub_nr(a, b);
  } else if constexpr (R == 4) {
    dft4<T, INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    // even/odd split: E = DFT4(x0,x2,x4,x6), O = DFT4(x1,x3,x5,x7); y_q = E_q + w8^q O_q
    V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    V o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T, INV>(e0, e1, e2, e3);
    dft4<T, INV>(o0, o1, o2, o3);
    const T h = (T)0.70710678118654752440;
    // w8^1 = h(1 -/+ i), w8^2 = -/+ i, w8^3 = h(-1 -/+ i)
    const V p1 = INV ? mk<V>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : mk<V>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    const V p2 = rot<V, INV>(o2);
    const V p3 = INV ? mk<V>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : mk<V>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    v[0] = cadd_nr(e0, o0);
    v[4] = csub_nr(e0, o0);
    v[1] = cadd_nr(e1, p1);
    v[5] = csub_nr(e1, p1);
    v[2] = cadd_nr(e2, p2);
    v[6] = csub_nr(e2, p2);
    v[3] = cadd_nr(e3, p3);
    v[7] = csub_nr(e3, p3);
  } else if constexpr (R == 9) {
    // r = 3a + b: Z_b = DFT3_a(x_{3a+b}); T_b(q1) = w9^{b q1} Z_b(q1); y_{q1+3 q2} = DFT3_b(T)(q2)
    V z[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      V a0 = v[b], a1 = v[b + 3], a2 = v[b + 6];
      dft3<T, INV>(a0, a1, a2);
      z[b] = a0;
      z[3 + b] = a1;
      z[6 + b] = a2;  // z[3 q1 + b]
    }
    const T c1 = (T)0.76604444311897803520, s1 = (T)0.64278760968653932632;  // 2 pi / 9
    const T c2 = (T)0.17364817766693034885, s2 = (T)0.98480775301220805936;  // 4 pi / 9
    const T c4 = (T)-0.93969262078590838405, s4 = (T)0.34202014332566873304; // 8 pi / 9
    const T sg = INV ? (T)1 : (T)-1;
    const V w1 = mk<V>(c1, sg * s1), w2 = mk<V>(c2, sg * s2), w4 = mk<V>(c4, sg * s4);
    z[4] = cmul(z[4], w1);  // q1 = 1, b = 1
    z[5] = cmul(z[5], w2);  // q1 = 1, b = 2
    z[7] = cmul(z[7], w2);  // q1 = 2, b = 1
    z[8] = cmul(z[8], w4);  // q1 = 2, b = 2
#pragma unroll
    for (int q1 = 0; q1 < 3; ++q1) {
      V a0 = z[3 * q1], a1 = z[3 * q1 + 1], a2 = z[3 * q1 + 2];
      dft3<T, INV>(a0, a1, a2);
      v[q1] = a0;
      v[q1 + 3] = a1;
      v[q1 + 6] = a2;
    }
  } else {
    dft_odd<T, R, INV>(v);
  }
}

// Work a Rader transform folds into the first and last register stage of its
// two length-(p-1) passes (null pointers: none).  ldmap (first stage of the
// first pass): input element e is loaded from position ldmap[e] (primitive-
// root order g^e; real parts of pool entries).  mul (last stage of the first
// pass): output e is stored as conj(y_e * mul[e]), and y_0 (= sum_{j>0} x_j)
// goes to slot rn + 1 first.  stmap (last stage of the second pass): output e
// is stored at position stmap[e] (g^-e) as x_0 + conj(y_e), x_0 from slot rn
// of the line; position 0 gets x_0 + A_0, A_0 from slot rn + 1 of aux.
// Folded only into the FP64 and FP32 engines: in the FP32-pair engine the
// extra branches of the stage loop cost more registers (spills) than the
// passes they save.
template <typename T> struct RaderFold { static constexpr bool on = true; };
template <> struct RaderFold<ff> { static constexpr bool on = false; };

template <typename V> struct StageFx {
  const V* ldmap = nullptr;
  const V* mul = nullptr;
  const V* stmap = nullptr;
  const V* aux = nullptr;
  int rn = 0;
};

// cin / cout: conjugate the values as they are loaded / stored (the first and
// last stage of an inverse transform computed as conj(DFT(conj x))).
template <typename T, int R, bool INV>
__device__ void stage_reg(const typename CT<T>::t* __restrict__ src, typename CT<T>::t* __restrict__ dst, int nl,
                          int ls, int n, int Ns, const FastDiv dnb, const FastDiv dns,
                          const typename CT<T>::t* __restrict__ tw, bool cin, bool cout,
                          const StageFx<typename CT<T>::t>& fx) {
  typedef typename CT<T>::t V;
  const int nb = n / R;
  const int s = n / (Ns * R);
  for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
    const int line = fdiv(t, dnb);
    const int j = t - line * nb;
    const int g = fdiv(j, dns);
    const int k = j - g * Ns;
    const V* in = src + (size_t)line * ls;
    V v[R];
    if (RaderFold<T>::on && fx.ldmap) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = in[pool_index(fx.ldmap[j + r * nb].x)];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = in[j + r * nb];
    }
    if (cin) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
    }
    if (k > 0) {
      const int ks = k * s;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul_nr(v[r], root<V, INV>(tw, r * ks));
    }
    dft_reg<T, R, INV>(v);
    V* ol = dst + (size_t)line * ls;
    const int p0 = g * Ns * R + k;
    if (RaderFold<T>::on && fx.mul) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int pos = p0 + r * Ns;
        V w = cnorm(v[r]);
        if (pos == 0) ol[fx.rn + 1] = w;
        w = cmul(w, fx.mul[pos]);
        w.y = -w.y;
        ol[pos] = w;
      }
    } else if (RaderFold<T>::on && fx.stmap) {
      const V x0 = in[fx.rn];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int pos = p0 + r * Ns;
        const V y = cnorm(v[r]);
        V o;
        o.x = x0.x + y.x;
        o.y = x0.y - y.y;
        if (cout) o.y = -o.y;
        ol[pool_index(fx.stmap[pos].x)] = o;
        if (pos == 0) {
          V z = cadd(x0, fx.aux[(size_t)line * ls + fx.rn + 1]);
          if (cout) z.y = -z.y;
          ol[0] = z;
        }
      }
    } else {
      if (cout) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) ol[p0 + r * Ns] = cnorm(v[r]);
    }
  }
}

// Large prime radix: one thread per output element.
template <typename T, bool INV>
__device__ void stage_big(const typename CT<T>::t* __restrict__ src, typename CT<T>::t* __restrict__ dst, int nl,
                          int ls, int n, int Ns, int R, const FastDiv dn, const typename CT<T>::t* __restrict__ tw,
                          bool cin, bool cout) {
  typedef typename CT<T>::t V;
  const int nb = n / R;
  const int NsR = Ns * R;
  const int s = n / NsR;
  for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
    const int line = fdiv(t, dn);
    const int o = t - line * n;
    const int g = o / NsR;
    const int mm = o - g * NsR;
    const int k = mm % Ns;
    const int j = g * Ns + k;
    const V* in = src + (size_t)line * ls;
    V acc = in[j];
    if (cin) acc.y = -acc.y;
    const int estep = (mm * s) % n;  // exponent increment per r
    int e = 0;
    for (int r = 1; r < R; ++r) {
      e += estep;
      if (e >= n) e -= n;
      V x = in[j + r * nb];
      if (cin) x.y = -x.y;
      acc = cadd(acc, cmul(x, root<V, INV>(tw, e)));
    }
    if (cout) acc.y = -acc.y;
    dst[(size_t)line * ls + o] = acc;
  }
}

// Radices with a register butterfly (stage_reg); others run stage_big.
__device__ __forceinline__ bool reg_radix(int R) {
  return R == 2 || R == 3 || R == 4 || R == 5 || R == 7 || R == 8 || R == 9 || R == 11 || R == 13 || R == 17;
}

// Runs the forward stages of p on nl lines held in a (stride ls), b is
// scratch of the same shape.  All threads of the block must call it.
// Returns the buffer holding the result (a or b).
// conj_in / conj_out: conjugate the input as the first stage loads it and
// the output as the last stage stores it (the inverse as conj(DFT(conj x)));
// no-op if the plan has no stage.  fx: Rader work folded into the first
// (ldmap) and last (mul, stmap) stage, which must then be register stages.
template <typename T>
__device__ __forceinline__ typename CT<T>::t* fft_run(typename CT<T>::t* a, typename CT<T>::t* b, int nl, int ls,
                                                      const Plan1& p, const typename CT<T>::t* __restrict__ tw,
                                                      bool conj_in, bool conj_out,
                                                      const StageFx<typename CT<T>::t>& fx) {
  typedef typename CT<T>::t V;
  int Ns = 1;
  const int n = p.n;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    const bool ci = conj_in && s == 0, co = conj_out && s == p.nst - 1;
    StageFx<V> f;
    if (s == 0) f.ldmap = fx.ldmap;
    if (s == p.nst - 1) {
      f.mul = fx.mul;
      f.stmap = fx.stmap;
      f.aux = fx.aux;
      f.rn = fx.rn;
    }
    switch (R) {
      case 2: stage_reg<T, 2, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 3: stage_reg<T, 3, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 4: stage_reg<T, 4, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 5: stage_reg<T, 5, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 7: stage_reg<T, 7, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 8: stage_reg<T, 8, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 9: stage_reg<T, 9, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 11: stage_reg<T, 11, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 13: stage_reg<T, 13, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      case 17: stage_reg<T, 17, false>(a, b, nl, ls, n, Ns, p.dnb[s], p.dns[s], tw, ci, co, f); break;
      default: stage_big<T, false>(a, b, nl, ls, n, Ns, R, p.dn, tw, ci, co); break;
    }
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Length-n DFT of nl lines (data in a[0..n) of each line; ls >= P.line_len()),
// forward or (inv) unnormalised inverse; b is scratch.  Returns the buffer
// holding the result.  Every transform runs the forward stages only, through
// one call site, so a kernel holds a single copy of the butterflies:
//  - inverse: IDFT(x) = conj(DFT(conj(x)));
//  - Rader (prime n = P.base.n, P.rd): slots n and n + 1 of every line hold x_0
//    and A_0 = sum_{j>0} x_j; x is gathered in primitive-root order g^q,
//    transformed (length m = n - 1), multiplied by the transformed kernel and
//    conjugated, transformed again (= conj of the inverse), and
//    X_{g^-q} = x_0 + conj(y_q), X_0 = x_0 + A_0;
//  - Bluestein (P.bs): X = conj(c) . IDFT_m( DFT_m(x conj(c)) . DFT_m(b) / m ),
//    c_j = exp(i pi j^2 / n), with the IDFT again as conj(DFT(conj)).
template <typename T>
__device__ __noinline__ typename CT<T>::t* fft_any_rt(typename CT<T>::t* a, typename CT<T>::t* b, int nl, int ls, const FftPlan& P,
                                         const typename CT<T>::t* __restrict__ pool, bool inv) {
  typedef typename CT<T>::t V;
  const int n = P.base.n;
  const bool two = P.rd || P.bs;
  const Plan1& sp = two ? P.sub : P.base;
  const int m = sp.n;
  // plan fields read inside loops, held in registers (the plan may live in
  // global memory, where the loops' stores could alias it)
  const FastDiv sdn = sp.dn, bdn = P.base.dn;
  const V* bh = pool + P.bhat;
  V* src = a;
  V* dst = b;
  // Rader whose length-(n-1) plan starts and ends with register stages: the
  // gather, the kernel multiply and the scatter run inside those stages
  const bool rfuse = RaderFold<T>::on && P.rd && reg_radix(sp.radix[0]) && reg_radix(sp.radix[sp.nst - 1]);
  // ---- input stage
  if (rfuse) {
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
      V x0 = a[(size_t)line * ls];
      if (inv) x0.y = -x0.y;
      a[(size_t)line * ls + n] = x0;
      b[(size_t)line * ls + n] = x0;
    }
  } else if (P.rd) {
    const V* gi = pool + P.gidx;
    for (int t = threadIdx.x; t < nl * m; t += blockDim.x) {
      const int line = fdiv(t, sdn);
      const int q = t - line * m;
      V v = a[(size_t)line * ls + pool_index(gi[q].x)];
      if (inv) v.y = -v.y;
      b[(size_t)line * ls + q] = v;
    }
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
      V x0 = a[(size_t)line * ls];
      if (inv) x0.y = -x0.y;
      a[(size_t)line * ls + n] = x0;
      b[(size_t)line * ls + n] = x0;
    }
    src = b;
    dst = a;
  } else if (P.bs) {
    const V* ch = pool + P.chirp;
    for (int t = threadIdx.x; t < nl * m; t += blockDim.x) {
      const int line = fdiv(t, sdn);
      const int j = t - line * m;
      V* x = a + (size_t)line * ls + j;
      if (j < n) {
        V v = *x;
        if (inv) v.y = -v.y;
        *x = cmulc(v, ch[j]);
      } else {
        *x = mk<V>(0.0, 0.0);
      }
    }
  }
  __syncthreads();
  // ---- one or two forward passes through a single call site (a direct
  // inverse conjugates in its first and last stage)
  V* r = src;
#pragma unroll 1
  for (int pass = 0; pass < (two ? 2 : 1); ++pass) {
    StageFx<V> fx;
    bool ci = !two && inv, co = !two && inv;
    if (rfuse) {
      fx.rn = n;
      if (pass == 0) {
        fx.ldmap = pool + P.gidx;
        fx.mul = bh;
        ci = inv;
      } else {
        fx.stmap = pool + P.sidx;
        fx.aux = src;  // the first pass's result: A_0 in slot n + 1
        co = inv;
      }
    }
    r = fft_run<T>(src, dst, nl, ls, sp, pool + sp.tw, ci, co, fx);
    V* o = (r == src) ? dst : src;
    if (pass == 0 && two && !rfuse) {
      for (int t = threadIdx.x; t < nl * m; t += blockDim.x) {
        const int line = fdiv(t, sdn);
        const int k = t - line * m;
        V* x = r + (size_t)line * ls + k;
        if (P.rd && k == 0) {  // A_0 = sum_{j>0} x_j, kept before the multiply overwrites it
          r[(size_t)line * ls + n + 1] = *x;
          o[(size_t)line * ls + n + 1] = *x;
        }
        V w = cmul(*x, bh[k]);
        w.y = -w.y;
        *x = w;
      }
      __syncthreads();
    }
    src = r;
    dst = o;
  }
  // ---- output stage (r holds the result of the last pass)
  if (rfuse) return r;
  if (P.rd) {
    const V* si = pool + P.sidx;
    V* out = dst;
    for (int t = threadIdx.x; t < nl * m; t += blockDim.x) {
      const int line = fdiv(t, sdn);
      const int q = t - line * m;
      const V* yl = r + (size_t)line * ls;
      V v;
      v.x = yl[n].x + yl[q].x;
      v.y = yl[n].y - yl[q].y;
      if (inv) v.y = -v.y;
      out[(size_t)line * ls + pool_index(si[q].x)] = v;
    }
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
      const V* yl = r + (size_t)line * ls;
      V v = cadd(yl[n], yl[n + 1]);
      if (inv) v.y = -v.y;
      out[(size_t)line * ls] = v;
    }
    __syncthreads();
    return out;
  }
  if (P.bs) {
    const V* ch = pool + P.chirp;
    for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
      const int line = fdiv(t, bdn);
      const int j = t - line * n;
      V* x = r + (size_t)line * ls + j;
      V z = *x;
      z.y = -z.y;
      V v = cmulc(z, ch[j]);
      if (inv) v.y = -v.y;
      *x = v;
    }
    __syncthreads();
    return r;
  }
  return r;
}

template <typename T, bool INV>
__device__ __forceinline__ typename CT<T>::t* fft_any(typename CT<T>::t* a, typename CT<T>::t* b, int nl, int ls,
                                                      const FftPlan& P, const typename CT<T>::t* __restrict__ pool) {
  return fft_any_rt<T>(a, b, nl, ls, P, pool, INV);
}

}  // namespace fcsph
