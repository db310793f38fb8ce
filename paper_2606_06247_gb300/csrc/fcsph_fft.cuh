// Shared-memory FFT engine for batches of short lines (one CTA, several lines).
//
// Stockham autosort (ping-pong between two shared-memory buffers, no bit
// reversal): stage s with radix R combines sub-transforms of size Ns into
// Ns*R.  Butterfly j (< n/R) reads x[j + r n/R], r < R, twiddles input r by
// w^{r k n/(Ns R)} (k = j mod Ns, w = exp(-2 pi i/n)), does an R-point DFT in
// registers and writes y[(j/Ns) Ns R + k + q Ns], q < R.  Radices 2 and 4 are
// multiplication-free; 3, 5, 7 use table roots; larger primes (up to
// kMaxDirectPrime) use one thread per output.  Lengths with a larger prime
// factor use Bluestein: X = conj(c) . IFFT_m( FFT_m(x conj(c)) . FFT_m(b) / m ),
// c_j = exp(i pi j^2 / n), m smooth >= 2n - 1.
#pragma once

#include <cuda_runtime.h>

#include "fcsph_internal.h"

namespace fcsph {

template <typename T> struct CT;
template <> struct CT<double> { typedef double2 t; };
template <> struct CT<float> { typedef float2 t; };

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
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) {
  V r;
  r.x = a.x * s;
  r.y = a.y * s;
  return r;
}
template <typename V> __device__ __forceinline__ V mk(double x, double y) {
  V r;
  r.x = x;
  r.y = y;
  return r;
}

// Root e of the length-n table, conjugated for the inverse transform.
template <typename V, bool INV> __device__ __forceinline__ V root(const V* __restrict__ tw, int e) {
  V w = tw[e];
  if (INV) w.y = -w.y;
  return w;
}

// In-register R-point DFT, v[q] <- sum_r v[r] w_R^{r q}, w_R = root(n/R).
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(typename CT<T>::t* v, const typename CT<T>::t* __restrict__ tw, int n) {
  typedef typename CT<T>::t V;
  if (R == 2) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 4) {
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    V t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    // forward: -i * d ; inverse: +i * d
    V t3 = INV ? mk<V>(-d.y, d.x) : mk<V>(d.y, -d.x);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else {
    V o[R];
    const int step = n / R;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      V acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], root<V, INV>(tw, ((r * q) % R) * step)));
      o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = o[q];
  }
}

template <typename T, int R, bool INV>
__device__ void stage_reg(const typename CT<T>::t* __restrict__ src, typename CT<T>::t* __restrict__ dst, int nl,
                          int ls, int n, int Ns, const typename CT<T>::t* __restrict__ tw) {
  typedef typename CT<T>::t V;
  const int nb = n / R;
  const int s = n / (Ns * R);
  for (int t = threadIdx.x; t < nl * nb; t += blockDim.x) {
    const int line = t / nb;
    const int j = t - line * nb;
    const int k = j % Ns;
    const V* in = src + (size_t)line * ls;
    V v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      V x = in[j + r * nb];
      if (r > 0 && k > 0) x = cmul(x, root<V, INV>(tw, r * k * s));
      v[r] = x;
    }
    dft_reg<T, R, INV>(v, tw, n);
    const int base = (j / Ns) * Ns * R + k;
    V* out = dst + (size_t)line * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
  }
}

// Large prime radix: one thread per output element.
template <typename T, bool INV>
__device__ void stage_big(const typename CT<T>::t* __restrict__ src, typename CT<T>::t* __restrict__ dst, int nl,
                          int ls, int n, int Ns, int R, const typename CT<T>::t* __restrict__ tw) {
  typedef typename CT<T>::t V;
  const int nb = n / R;
  const int NsR = Ns * R;
  const int s = n / NsR;
  for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
    const int line = t / n;
    const int o = t - line * n;
    const int g = o / NsR;
    const int mm = o - g * NsR;
    const int k = mm % Ns;
    const int j = g * Ns + k;
    const V* in = src + (size_t)line * ls;
    V acc = in[j];
    const int estep = (mm * s) % n;  // exponent increment per r
    int e = 0;
    for (int r = 1; r < R; ++r) {
      e += estep;
      if (e >= n) e -= n;
      acc = cadd(acc, cmul(in[j + r * nb], root<V, INV>(tw, e)));
    }
    dst[(size_t)line * ls + o] = acc;
  }
}

// Runs the stages of p on nl lines held in a (stride ls), b is scratch of the
// same shape.  All threads of the block must call it.  Returns the buffer
// holding the result (a or b).
template <typename T, bool INV>
__device__ typename CT<T>::t* fft_run(typename CT<T>::t* a, typename CT<T>::t* b, int nl, int ls, const Plan1& p,
                                      const typename CT<T>::t* __restrict__ tw) {
  typedef typename CT<T>::t V;
  int Ns = 1;
  const int n = p.n;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    switch (R) {
      case 2: stage_reg<T, 2, INV>(a, b, nl, ls, n, Ns, tw); break;
      case 3: stage_reg<T, 3, INV>(a, b, nl, ls, n, Ns, tw); break;
      case 4: stage_reg<T, 4, INV>(a, b, nl, ls, n, Ns, tw); break;
      case 5: stage_reg<T, 5, INV>(a, b, nl, ls, n, Ns, tw); break;
      case 7: stage_reg<T, 7, INV>(a, b, nl, ls, n, Ns, tw); break;
      default: stage_big<T, INV>(a, b, nl, ls, n, Ns, R, tw); break;
    }
    __syncthreads();
    V* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Length-n DFT of nl lines (data in a[0..n) of each line; ls >= P.line_len()).
template <typename T, bool INV>
__device__ typename CT<T>::t* fft_any(typename CT<T>::t* a, typename CT<T>::t* b, int nl, int ls, const FftPlan& P,
                                      const typename CT<T>::t* __restrict__ pool) {
  typedef typename CT<T>::t V;
  if (!P.bs) return fft_run<T, INV>(a, b, nl, ls, P.base, pool + P.base.tw);
  const int n = P.base.n;
  const int m = P.sub.n;
  const V* ch = pool + P.chirp;
  const V* bh = pool + P.bhat;
  // a_j = x_j conj(c_j) (x conjugated first for the inverse), zero-padded to m
  for (int t = threadIdx.x; t < nl * m; t += blockDim.x) {
    const int line = t / m;
    const int j = t - line * m;
    V* x = a + (size_t)line * ls + j;
    if (j < n) {
      V v = *x;
      if (INV) v.y = -v.y;
      *x = cmulc(v, ch[j]);
    } else {
      *x = mk<V>(0.0, 0.0);
    }
  }
  __syncthreads();
  V* r = fft_run<T, false>(a, b, nl, ls, P.sub, pool + P.sub.tw);
  V* o = (r == a) ? b : a;
  for (int t = threadIdx.x; t < nl * m; t += blockDim.x) {
    const int line = t / m;
    const int j = t - line * m;
    V* x = r + (size_t)line * ls + j;
    *x = cmul(*x, bh[j]);
  }
  __syncthreads();
  r = fft_run<T, true>(r, o, nl, ls, P.sub, pool + P.sub.tw);
  for (int t = threadIdx.x; t < nl * n; t += blockDim.x) {
    const int line = t / n;
    const int j = t - line * n;
    V* x = r + (size_t)line * ls + j;
    V v = cmulc(*x, ch[j]);
    if (INV) v.y = -v.y;
    *x = v;
  }
  __syncthreads();
  return r;
}

}  // namespace fcsph
