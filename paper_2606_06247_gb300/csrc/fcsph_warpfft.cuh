// Register-resident FP32 FFT of lines of n = 32 M points (M = 2 .. 32), one
// warp per 32 / M lines, for the x (periodic) pass of FP32 contexts.
//
// Four-step split n = M x 32 with lane t < 32 and j, k1 < M, k2 < 32:
//   X[k1 + M k2] = sum_t w_32^{t k2} w_n^{t k1} sum_j x[t + 32 j] w_M^{j k1}.
// Lane t holds x[t + 32 j] of each of its warp's lines (coalesced loads),
// runs the M-point DFTs in registers, applies w_n^{t k1} (roots of the
// context's pool), exchanges the M x 32 blocks through shared memory (one
// write and one read per value, padded rows: no bank conflicts), and runs a
// 32-point DFT in registers.  Afterwards lane L = l M + k1 holds
// X_l[k1 + M k2] for k2 < 32.  The inverse runs the same steps backwards
// with conjugate roots, from that layout back to x[t + 32 j] in lane t, so a
// forward transform, a pointwise multiply and an inverse transform need no
// reordering between them.  Every lane carries 32 complex values.
#pragma once

#include <cuda_runtime.h>

#include "fcsph_fft.cuh"

namespace fcsph {

// exp(-/+ 2 pi i e / 32) for the forward / inverse transform; e is a
// compile-time constant in the unrolled loops, so the switch folds.
__device__ __forceinline__ float c32(int e) {
  e &= 31;
  const int q = e >> 3, r = e & 7;
  float v;
  switch (r) {  // cos(2 pi r / 32)
    case 0: v = 1.0f; break;
    case 1: v = 0.98078528040323044913f; break;
    case 2: v = 0.92387953251128675613f; break;
    case 3: v = 0.83146961230254523708f; break;
    case 4: v = 0.70710678118654752440f; break;
    case 5: v = 0.55557023301960222474f; break;
    case 6: v = 0.38268343236508977173f; break;
    default: v = 0.19509032201612826785f; break;
  }
  // cos of the angle (q * 8 + r) * 2 pi / 32 = q * pi / 2 + theta
  const float s = r == 0 ? 0.0f : (r == 1 ? 0.19509032201612826785f : r == 2 ? 0.38268343236508977173f
                                   : r == 3 ? 0.55557023301960222474f : r == 4 ? 0.70710678118654752440f
                                   : r == 5 ? 0.83146961230254523708f : r == 6 ? 0.92387953251128675613f
                                                                             : 0.98078528040323044913f);
  switch (q) {
    case 0: return v;
    case 1: return -s;
    case 2: return -v;
    default: return s;
  }
}
__device__ __forceinline__ float s32(int e) { return c32(e + 24); }  // sin(x) = cos(x - pi/2) = cos(x + 3 pi/2)

template <bool INV> __device__ __forceinline__ float2 w32(int e) {
  return make_float2(c32(e), INV ? s32(e) : -s32(e));
}

// In-register 16- and 32-point DFTs (natural order in and out):
// a[n1 R2 + n2]: B[n2][k1] = DFT_R1 over n1, times w_{R1 R2}^{n2 k1}, then
// A[k1 + R1 k2] = DFT_R2 over n2.
template <bool INV> __device__ __forceinline__ void dft32r(float2* a) {
  float2 b[32];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 t[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) t[n1] = a[4 * n1 + n2];
    dft_reg<float, 8, INV>(t);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) b[n2 * 8 + k1] = (n2 * k1 == 0) ? t[k1] : cmul(t[k1], w32<INV>(n2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) {
    float2 u0 = b[k1], u1 = b[8 + k1], u2 = b[16 + k1], u3 = b[24 + k1];
    dft4<float, INV>(u0, u1, u2, u3);
    a[k1] = u0;
    a[k1 + 8] = u1;
    a[k1 + 16] = u2;
    a[k1 + 24] = u3;
  }
}

template <bool INV> __device__ __forceinline__ void dft16r(float2* a) {
  float2 b[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 t0 = a[n2], t1 = a[4 + n2], t2 = a[8 + n2], t3 = a[12 + n2];
    dft4<float, INV>(t0, t1, t2, t3);
    const float2 t[4] = {t0, t1, t2, t3};
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) b[n2 * 4 + k1] = (n2 * k1 == 0) ? t[k1] : cmul(t[k1], w32<INV>(2 * n2 * k1));
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 u0 = b[k1], u1 = b[4 + k1], u2 = b[8 + k1], u3 = b[12 + k1];
    dft4<float, INV>(u0, u1, u2, u3);
    a[k1] = u0;
    a[k1 + 4] = u1;
    a[k1 + 8] = u2;
    a[k1 + 12] = u3;
  }
}

template <int M, bool INV> __device__ __forceinline__ void dft_m(float2* a) {
  if constexpr (M == 32) dft32r<INV>(a);
  else if constexpr (M == 16) dft16r<INV>(a);
  else dft_reg<float, M, INV>(a);
}

// v[l M + k1] *= w_n^{lane k1} (conjugate for the inverse), n = 32 M.  For
// M > 8 the root is formed as w^{lane (k1 mod 8)} w^{8 lane (k1 / 8)} from
// 8 + M/8 - 1 loads (one extra rounding), which keeps the per-lane roots
// from occupying M registers pairs at once.
template <int M, bool INV>
__device__ __forceinline__ void twiddle(float2* v, const float2* __restrict__ roots, int lane) {
  constexpr int LPW = 32 / M;
  if constexpr (M <= 8) {
#pragma unroll
    for (int k1 = 1; k1 < M; ++k1) {
      const float2 w = roots[lane * k1];
#pragma unroll
      for (int l = 0; l < LPW; ++l) v[l * M + k1] = INV ? cmulc(v[l * M + k1], w) : cmul(v[l * M + k1], w);
    }
  } else {
    float2 lo[8];
#pragma unroll
    for (int r = 1; r < 8; ++r) lo[r] = roots[lane * r];
#pragma unroll
    for (int hi = 0; hi < M / 8; ++hi) {
      const float2 wh = hi ? roots[lane * 8 * hi] : make_float2(1.f, 0.f);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int k1 = 8 * hi + r;
        if (k1 == 0) continue;
        const float2 w = r == 0 ? wh : (hi == 0 ? lo[r] : cmul(wh, lo[r]));
#pragma unroll
        for (int l = 0; l < LPW; ++l) v[l * M + k1] = INV ? cmulc(v[l * M + k1], w) : cmul(v[l * M + k1], w);
      }
    }
  }
}

// Shared memory per warp for the block exchange: 32 rows of 33 floats for the
// real and the imaginary parts.
constexpr int kWarpXchgFloats = 2 * 32 * 33;

// Forward transform of the warp's 32 / M lines; v[l M + j] = x_l[lane + 32 j]
// on entry, v[k2] = X_l[k1 + M k2] (l M + k1 = lane) on return.  roots: the
// n roots exp(-2 pi i e / n), e < n.  xs: kWarpXchgFloats floats of this warp.
template <int M>
__device__ __forceinline__ void warp_fft_fwd(float2* v, float* xs, const float2* __restrict__ roots, int lane) {
  constexpr int LPW = 32 / M;
#pragma unroll
  for (int l = 0; l < LPW; ++l) dft_m<M, false>(v + l * M);
  twiddle<M, false>(v, roots, lane);
  float* re = xs;
  float* im = xs + 32 * 33;
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 32; ++s) {
    re[s * 33 + lane] = v[s].x;
    im[s * 33 + lane] = v[s].y;
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = make_float2(re[lane * 33 + t], im[lane * 33 + t]);
  __syncwarp();
  dft32r<false>(v);
}

// Inverse (unnormalised) of warp_fft_fwd: from v[k2] = X_l[k1 + M k2] to
// v[l M + j] = x_l[lane + 32 j].
template <int M>
__device__ __forceinline__ void warp_fft_inv(float2* v, float* xs, const float2* __restrict__ roots, int lane) {
  constexpr int LPW = 32 / M;
  dft32r<true>(v);
  float* re = xs;
  float* im = xs + 32 * 33;
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    re[lane * 33 + t] = v[t].x;
    im[lane * 33 + t] = v[t].y;
  }
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 32; ++s) v[s] = make_float2(re[s * 33 + lane], im[s * 33 + lane]);
  __syncwarp();
  twiddle<M, true>(v, roots, lane);
#pragma unroll
  for (int l = 0; l < LPW; ++l) dft_m<M, true>(v + l * M);
}

}  // namespace fcsph
