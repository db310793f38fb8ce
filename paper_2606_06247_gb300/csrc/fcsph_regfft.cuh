// Register-resident FP32 FFT of one line of n = N1 N2 points by a team of
// threads (the CTA), for the wall-normal passes of FP32 contexts whose
// extended length factors that way (e.g. 540 = 20 x 27, 1050 = 30 x 35).
//
// Four-step split with t < N2, j, k1 < N1, k2 < N2:
//   X[k1 + N1 k2] = sum_t w_N2^{t k2} w_n^{t k1} sum_j x[t + N2 j] w_N1^{j k1}.
// Thread t < N2 holds x[t + N2 j] and runs the N1-point DFT in registers,
// multiplies by w_n^{t k1} (the context's pool roots) and writes its column of
// the N1 x N2 block to shared memory (rows of odd stride: no bank conflicts);
// after one barrier thread k1 < N1 reads its row and runs the N2-point DFT in
// registers, ending with X[k1 + N1 k2], k2 < N2.  The inverse runs the same
// steps backwards with conjugate roots.  Composite sizes are split into two
// register DFTs with constant roots (fcsph_roots.cuh) down to the radices of
// dft_reg.
#pragma once

#include <cuda_runtime.h>

#include "fcsph_fft.cuh"
#include "fcsph_roots.cuh"

namespace fcsph {

// Designated split N = A x B of a composite register-DFT size (0: a base radix).
template <int N> struct RegSplit { static constexpr int a = 0; };
template <> struct RegSplit<10> { static constexpr int a = 2; };
template <> struct RegSplit<14> { static constexpr int a = 2; };
template <> struct RegSplit<15> { static constexpr int a = 3; };
template <> struct RegSplit<20> { static constexpr int a = 4; };
template <> struct RegSplit<21> { static constexpr int a = 3; };
template <> struct RegSplit<25> { static constexpr int a = 5; };
template <> struct RegSplit<27> { static constexpr int a = 3; };
template <> struct RegSplit<28> { static constexpr int a = 4; };
template <> struct RegSplit<30> { static constexpr int a = 3; };
template <> struct RegSplit<35> { static constexpr int a = 5; };
template <> struct RegSplit<6> { static constexpr int a = 2; };
template <> struct RegSplit<36> { static constexpr int a = 4; };
template <> struct RegSplit<42> { static constexpr int a = 6; };
template <> struct RegSplit<50> { static constexpr int a = 5; };

// exp(-/+ 2 pi i e / N) (forward / inverse) for a composite N.
template <int N, bool INV> __device__ __forceinline__ float2 rroot(int e) {
  const float s = rsin<N>(e);
  return make_float2(rcos<N>(e), INV ? s : -s);
}

// In-register N-point DFT, natural order in and out:
// v[a B + b]: B DFTs of size A over a, times w_N^{b k1}, then A DFTs of size B.
template <int N, bool INV> __device__ __forceinline__ void dft_c(float2* v) {
  constexpr int A = RegSplit<N>::a;
  if constexpr (A == 0) {
    dft_reg<float, N, INV>(v);
  } else {
    constexpr int B = N / A;
    float2 t[N];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      float2 g[A];
#pragma unroll
      for (int a = 0; a < A; ++a) g[a] = v[a * B + b];
      dft_c<A, INV>(g);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) t[b * A + k1] = (b * k1 == 0) ? g[k1] : cmul(g[k1], rroot<N, INV>(b * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      float2 h[B];
#pragma unroll
      for (int b = 0; b < B; ++b) h[b] = t[b * A + k1];
      dft_c<B, INV>(h);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = h[k2];
    }
  }
}

template <int N1, int N2> struct TeamFFT {
  static constexpr int NV = N1 > N2 ? N1 : N2;       // complex registers per thread
  static constexpr int S = (N2 % 2) ? N2 : N2 + 1;    // odd row stride of the exchange block
  static constexpr int XCHG = N1 * S;                 // float2 elements of the exchange block
  static constexpr int THREADS = (NV + 31) / 32 * 32;
  // <= 128 registers per thread; teams of more than 35 points per thread
  // (the Bluestein lengths 1080 = 30 x 36 and 2100 = 42 x 50) get up to 255
  static constexpr int MIN_CTAS = NV > 35 ? 256 / THREADS : 512 / THREADS;

  // Forward: v[j] = x[t + N2 j] (t < N2) on entry; v[k2] = X[t + N1 k2]
  // (t < N1) on return.  Every thread of the CTA calls it.
  static __device__ __forceinline__ void fwd(float2* v, float2* xs, const float2* __restrict__ roots, int t) {
    if (t < N2) {
      dft_c<N1, false>(v);
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], roots[t * k1]);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) xs[k1 * S + t] = v[k1];
    }
    __syncthreads();
    if (t < N1) {
#pragma unroll
      for (int b = 0; b < N2; ++b) v[b] = xs[t * S + b];
      dft_c<N2, false>(v);
    }
    __syncthreads();
  }

  // Inverse (unnormalised): v[k2] = X[t + N1 k2] (t < N1) on entry;
  // v[j] = x[t + N2 j] (t < N2) on return.
  static __device__ __forceinline__ void inv(float2* v, float2* xs, const float2* __restrict__ roots, int t) {
    if (t < N1) {
      dft_c<N2, true>(v);
#pragma unroll
      for (int b = 0; b < N2; ++b) xs[t * S + b] = v[b];
    }
    __syncthreads();
    if (t < N2) {
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) v[k1] = xs[k1 * S + t];
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmulc(v[k1], roots[t * k1]);
      dft_c<N1, true>(v);
    }
    __syncthreads();
  }
};

// Length-n DFT (forward, or INV: the unnormalised inverse) of the line L by
// Bluestein's chirp-z convolution on the team FFT of length m = N1 N2 >= 2n - 1:
// a_j = x_j conj(c_j) for j < n, zero up to m; y = IDFT_m(DFT_m(a) . bhat), the
// inverse unnormalised, bhat = DFT_m(b) / m of the chirp filter b; then
// X_k = conj(c_k) y_k, with c_j = exp(i pi j^2 / n); the inverse as
// conj(DFT(conj x)).  In: L[j], j < n (L holds m values).  Out: L[k], k < n.
// chirp: c_j, j < n; roots: w_m^e, e < m.  Every thread of the CTA calls it.
template <int N1, int N2, bool INV>
__device__ __forceinline__ void bluestein_team(float2* L, float2* xs, int n, const float2* __restrict__ chirp,
                                               const float2* __restrict__ bhat, const float2* __restrict__ roots,
                                               int t) {
  typedef TeamFFT<N1, N2> TF;
  constexpr int m = N1 * N2;
  for (int j = t; j < m; j += blockDim.x) {
    float2 a = make_float2(0.f, 0.f);
    if (j < n) {
      float2 x = L[j];
      if (INV) x.y = -x.y;
      a = cmulc(x, chirp[j]);
    }
    L[j] = a;
  }
  __syncthreads();
  float2 v[TF::NV];
  if (t < N2) {
#pragma unroll
    for (int j = 0; j < N1; ++j) v[j] = L[t + N2 * j];
  }
  TF::fwd(v, xs, roots, t);
  if (t < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) v[k2] = cmul(v[k2], bhat[t + N1 * k2]);
  }
  TF::inv(v, xs, roots, t);
  if (t < N2) {
#pragma unroll
    for (int j = 0; j < N1; ++j) {
      const int idx = t + N2 * j;
      if (idx < n) {
        float2 z = cmulc(v[j], chirp[idx]);
        if (INV) z.y = -z.y;
        L[idx] = z;
      }
    }
  }
  __syncthreads();
}

}  // namespace fcsph
