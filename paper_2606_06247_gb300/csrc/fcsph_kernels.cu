// CUDA kernels of the FC spectral ISPH hot path (sm_103a).
//
// Data layout (HBM).  Real fields f[b][c][j] (j = y, contiguous; c = x index,
// or x * nz + z on a 3D grid).  Spectra after the y transform are stored
// transposed, S[b][field][ky][c] (c contiguous), so that the x pass reads
// whole rows (3D: x lines at stride nz, after a z pass over contiguous runs).
// The FC-extended grid is never materialised in HBM on the hot path: the
// continuation is computed in shared memory inside the transform kernels.
//
// Transform kernels run 32, 64 or 128 threads per CTA (one warp, whose
// barriers are warp barriers, for full batches; more where a pass has few
// lines or long ones), the threads of a CTA sharing its lines.  Column
// kernels (y direction) handle
// 2*Pp adjacent columns of one instance: two real columns are packed into
// one complex line (a + i b), transformed together, and separated with the
// Hermitian split
//   A_k = (Z_k + conj Z_{-k}) / 2,  B_k = (Z_k - conj Z_{-k}) / (2i).
// Row kernels (x direction) handle Rr x lines of one instance; outputs are
// formed and inverted one at a time.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "fcsph_fft.cuh"
#include "fcsph_warpfft.cuh"
#include "fcsph_regfft.cuh"
#include "fcsph_tma.cuh"
#include "fcsph_internal.h"

using namespace fcsph;

namespace {

constexpr int kThreads = 256;
// FFT kernels are templated on their CTA width NT = 32, 64 or 128 threads;
// the threads of a CTA share its lines.  One warp per CTA keeps every barrier
// of the shared-memory FFT a warp barrier, and is fastest when the pass has
// CTAs enough to fill the GPU.  Wider CTAs carry each line with more threads:
// they cut the latency of passes with few lines (small grids and batches),
// and for long FP32 lines (~1000 points) they hold less shared memory per
// warp, so more warps fit on an SM.
// Minimum resident CTAs per SM asked of the register allocator: FP32-pair
// code would otherwise take all 255 registers (8 one-warp CTAs per SM).
// FP64 and FP32x2: <= 168 registers at every width; FP32: <= 128 at 32 and
// 64 threads, <= 64 at 128 (more resident warps beat the few spills this
// costs in the column and row passes).
template <typename T, int NT> struct MinCtas { static constexpr int v = 384 / NT; };
template <> struct MinCtas<float, 32> { static constexpr int v = 16; };
template <> struct MinCtas<float, 64> { static constexpr int v = 8; };
template <> struct MinCtas<float, 128> { static constexpr int v = 8; };
// The line operator keeps three lines and its outputs live across the
// transforms: at 128 threads it gets <= 128 registers (4 CTAs per SM) rather
// than spilling at 64.
template <typename T, int NT> struct LineMinCtas { static constexpr int v = MinCtas<T, NT>::v; };
template <> struct LineMinCtas<float, 128> { static constexpr int v = 4; };

// Calls f(std::integral_constant<int, NT>) for the CTA width nt (32, 64, 128).
template <typename F> cudaError_t with_width(int nt, F&& f) {
  if (nt == 64) return f(std::integral_constant<int, 64>{});
  if (nt == 128) return f(std::integral_constant<int, 128>{});
  if (nt != 32) return cudaErrorInvalidValue;
  return f(std::integral_constant<int, 32>{});
}

template <typename T> struct PoolOf;
template <> struct PoolOf<double> { static const double2* get(const fcsph_ctx* c) { return c->pool64; } };
template <> struct PoolOf<float> { static const float2* get(const fcsph_ctx* c) { return c->pool32; } };
template <> struct PoolOf<ff> { static const ff2* get(const fcsph_ctx* c) { return static_cast<const ff2*>(c->poolff); } };

__device__ __forceinline__ size_t fidx(const GridDev& g, int b, int i, int j) {
  return ((size_t)b * g.ncol + i) * g.ny + j;
}

// ---------------------------------------------------------------------------
// Compensated dot product for the FC continuation sum_m E[m] b[m]: the table
// entries reach ~1e4 while the result is O(|b|), so each product is split
// exactly (p + e = a*b via fma) and the terms are added with TwoSum; the
// result is accurate to a few ulps of the result instead of ulps of the terms.
struct Dot2 {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double a, double b) {
    const double p = a * b;
    const double e = fma(a, b, -p);
    const double t = s + p;
    const double bp = t - s;
    c += (s - (t - bp)) + (p - bp) + e;
    s = t;
  }
  __device__ __forceinline__ double value() const { return s + c; }
};

// FC continuation sum of one line component: compensated FP64 (Dot2, table
// in double) for FP64 transforms; FP32-pair arithmetic (table in FP32 pairs)
// for FP32x2 and FP32 transforms.  For FP32 the pair sum (error ~2^-48 of
// sum |E b|) rounds to the same FP32 value an FP64 sum would, on the FP32
// units: the sum needs more than FP32 because the terms reach ~1e3-1e4 |b|.
template <typename T> struct FcTab { typedef double t; };
template <> struct FcTab<ff> { typedef ff t; };
template <> struct FcTab<float> { typedef ff t; };

template <typename T> struct FcAcc {
  Dot2 a;
  __device__ __forceinline__ void add(double e, T x) { a.add(e, (double)x); }
  __device__ __forceinline__ T value() const { return (T)a.value(); }
};
template <> struct FcAcc<ff> {
  ff a;
  __device__ __forceinline__ void add(ff e, ff x) { a += e * x; }
  __device__ __forceinline__ ff value() const { return a; }
};
template <> struct FcAcc<float> {
  ff a;
  __device__ __forceinline__ void add(ff e, float x) { a = ff_fma(a, e, ff_make(x, 0.f)); }
  __device__ __forceinline__ float value() const { return __fadd_rn(a.h, a.l); }
};

// Appends the C continuation values of nl lines (stride ls, data in [0, n)):
// line[n + c] = sum_m E[c][m] line[n - d + m] + E[c][d + m] line[m].
template <typename T>
__device__ __forceinline__ void fc_append(typename CT<T>::t* lines, int nl, int ls, int n, int C, int d,
                                          const typename FcTab<T>::t* __restrict__ E) {
  typedef typename CT<T>::t V;
  for (int p = 0; p < nl; ++p) {
    V* L = lines + (size_t)p * ls;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
      const typename FcTab<T>::t* Er = E + c * 2 * d;
      FcAcc<T> ax, ay;
      for (int m = 0; m < d; ++m) {
        const V vr = L[n - d + m];
        const V vl = L[m];
        ax.add(Er[m], vr.x);
        ax.add(Er[d + m], vl.x);
        ay.add(Er[m], vr.y);
        ay.add(Er[d + m], vl.y);
      }
      L[n + c] = mk<V>(ax.value(), ay.value());
    }
  }
}

template <typename T>
__device__ void col_store_spectrum(const typename CT<T>::t* R, int Pp, int ls, const GridDev& g, int i0, int n,
                                   int dct, typename CT<T>::t* __restrict__ spec);

// ---------------------------------------------------------------------------
// Forward transform of packed column pairs held in shared memory.
// lines: Pp lines of stride ls, line p has column i0+2p in .x and i0+2p+1 in
// .y for j < ny.  dct = 0: FC-extend to my with table E ([C][2d], FP64
// accumulation, FP32 pairs for FP32x2) and FFT (length my); dct = 1: even extension to 2(ny-1) and
// FFT (DCT-I, Eq. 31).  Stores the half spectrum (or the ny real DCT
// coefficients as (c, 0)) into spec[ky][i] for this instance/field.
template <typename T>
__device__ void col_forward_store(typename CT<T>::t* lines, typename CT<T>::t* scratch, int Pp, int ls,
                                  const GridDev& g, int i0, const typename FcTab<T>::t* __restrict__ E,
                                  const FftPlan& P,
                                  const typename CT<T>::t* __restrict__ pool, int dct,
                                  typename CT<T>::t* __restrict__ spec) {
  typedef typename CT<T>::t V;
  const int ny = g.ny;
  if (!dct) {
    fc_append<T>(lines, Pp, ls, ny, g.n_cont, g.n_match, E);
  } else {
    const int M = 2 * (ny - 1);
    for (int p = 0; p < Pp; ++p)
      for (int jj = 1 + threadIdx.x; jj <= ny - 2; jj += blockDim.x)
        lines[(size_t)p * ls + M - jj] = lines[(size_t)p * ls + jj];
  }
  __syncthreads();
  V* R = fft_any<T, false>(lines, scratch, Pp, ls, P, pool);
  col_store_spectrum<T>(R, Pp, ls, g, i0, P.base.n, dct, spec);
}

// Half spectrum (or, dct = 1, the ny real DCT-I coefficients as (c, 0)) of
// the Pp transformed packed column pairs in R (stride ls, length n) into
// spec[ky][i] of columns i0 + 2p, i0 + 2p + 1.
template <typename T>
__device__ void col_store_spectrum(const typename CT<T>::t* R, int Pp, int ls, const GridDev& g, int i0, int n,
                                   int dct, typename CT<T>::t* __restrict__ spec) {
  typedef typename CT<T>::t V;
  const int ny = g.ny;
  const int nk = dct ? ny : g.hy;
  const T h = (T)0.5;
  for (int p = 0; p < Pp; ++p) {
    const int i = i0 + 2 * p;
    const V* L = R + (size_t)p * ls;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
      const V z = L[k];
      const V zm = L[k == 0 ? 0 : n - k];
      V a, b;  // columns i and i + 1
      if (dct) {
        a = mk<V>(h * (z.x + zm.x), 0);
        b = mk<V>(h * (z.y + zm.y), 0);
      } else {
        a = mk<V>(h * (z.x + zm.x), h * (z.y - zm.y));
        b = mk<V>(h * (z.y + zm.y), h * (zm.x - z.x));
      }
      V* S = spec + (size_t)k * g.ncol + i;
      if (i < g.ncol) S[0] = a;
      if (i + 1 < g.ncol) S[1] = b;
    }
  }
}

// Gathers nout half spectra (spec + o*fstride, rows ky < hy) of the column
// pairs into full-length packed lines Z_k = A_k + i B_k and Z_{n-k} =
// conj(A_k) + i conj(B_k); DC and Nyquist keep only the real parts.
template <typename T>
__device__ void col_gather_hermitian(typename CT<T>::t* lines, int Pp, int ls, const GridDev& g, int i0,
                                     const typename CT<T>::t* spec, size_t fstride, int nout, int n) {
  typedef typename CT<T>::t V;
  const int hy = g.hy;
  for (int o = 0; o < nout; ++o)
    for (int p = 0; p < Pp; ++p) {
      const int ia = i0 + 2 * p, ib = ia + 1;
      V* L = lines + ((size_t)o * Pp + p) * ls;
      for (int k = threadIdx.x; k < hy; k += blockDim.x) {
        const V* S = spec + o * fstride + (size_t)k * g.ncol;
        V A = mk<V>(0.0, 0.0), B = mk<V>(0.0, 0.0);
        if (ia < g.ncol) A = S[ia];
        if (ib < g.ncol) B = S[ib];
        const bool self = (k == 0) || (2 * k == n);
        V z0, z1;
        if (self) {
          z0.x = A.x;
          z0.y = B.x;
          L[k] = z0;
        } else {
          z0.x = A.x - B.y;
          z0.y = A.y + B.x;
          z1.x = A.x + B.y;
          z1.y = B.x - A.y;
          L[k] = z0;
          L[n - k] = z1;
        }
      }
    }
}

// Packed DCT-I coefficient pairs (real parts of spec rows l < ny) into lines.
template <typename T>
__device__ void col_gather_dct(typename CT<T>::t* lines, int Pp, int ls, const GridDev& g, int i0,
                               const typename CT<T>::t* spec) {
  typedef typename CT<T>::t V;
  const int ny = g.ny, M = 2 * (ny - 1);
  for (int p = 0; p < Pp; ++p) {
    const int ia = i0 + 2 * p, ib = ia + 1;
    V* L = lines + (size_t)p * ls;
    for (int l = threadIdx.x; l < ny; l += blockDim.x) {
      const V* S = spec + (size_t)l * g.ncol;
      V z = mk<V>(0.0, 0.0);
      if (ia < g.ncol) z.x = S[ia].x;
      if (ib < g.ncol) z.y = S[ib].x;
      L[l] = z;
      if (l >= 1 && l <= ny - 2) L[M - l] = z;
    }
  }
}

// ---------------------------------------------------------------------------
// Column forward: load nf real fields, FC (or DCT) + FFT, store spectra.
template <typename T, typename U>
__device__ __forceinline__ void col_fwd_body(const GridDev& g, const U* f0, const U* f1, const U* f2,
                                             const typename FcTab<T>::t* E, const FftPlan& P,
                                             const typename CT<T>::t* pool, int dct, typename CT<T>::t* spec,
                                             size_t fstride, size_t bstride, int Pp, int ls, int bx, int by, int bz) {
  typedef typename CT<T>::t V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* lines = reinterpret_cast<V*>(smem_raw);
  V* scratch = lines + (size_t)Pp * ls;
  const int b = bz + g.b0, f = by;
  if (inactive(g, b)) return;
  const int i0 = bx * 2 * Pp;
  const U* src = f == 0 ? f0 : (f == 1 ? f1 : f2);
  const int W = 2 * Pp;
  const int ny = g.ny;
  const size_t base = ((size_t)b * g.ncol + i0) * ny;
  for (int col = 0; col < W; ++col) {
    T* L = reinterpret_cast<T*>(lines + (size_t)(col >> 1) * ls) + (col & 1);
    const bool in = i0 + col < g.ncol;
    for (int j = threadIdx.x; j < ny; j += blockDim.x)
      L[2 * j] = in ? (T)src[base + (size_t)col * ny + j] : (T)0;
  }
  __syncthreads();
  col_forward_store<T>(lines, scratch, Pp, ls, g, i0, E, P, pool, dct, spec + b * bstride + f * fstride);
}

template <typename T, typename U, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T, NT>::v) k_col_fwd(GridDev g, const U* __restrict__ f0, const U* __restrict__ f1, const U* __restrict__ f2,
                                                         const typename FcTab<T>::t* __restrict__ E, const __grid_constant__ FftPlan P,
                                                      const typename CT<T>::t* __restrict__ pool, int dct,
                                                      typename CT<T>::t* __restrict__ spec, size_t fstride,
                                                      size_t bstride, int Pp, int ls) {
  col_fwd_body<T, U>(g, f0, f1, f2, E, P, pool, dct, spec, fstride, bstride, Pp, ls, blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------------------
// Symbols (Eq. 16 reading): W_hat(s) = e^{-s} sum_{m<n} s^m/m!, s = |k|^2 h^2/4;
// DX = i kx W_hat, DY = i ky W_hat, DZ = i kz W_hat (each zero on its own
// axis' Nyquist plane), LAP = -|k|^2 W_hat, W = W_hat (kz = 0 in 2D).
// Returned as (re, im) in the compute type.  Products and sums of the
// wavenumbers use round-to-nearest intrinsics, which the compiler never
// contracts into FMAs: every CTA width then evaluates the same expression.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ ff mul_rn(ff a, ff b) { return a * b; }
__device__ __forceinline__ ff add_rn(ff a, ff b) { return a + b; }
__device__ __forceinline__ ff div_rn(ff a, ff b) { return a / b; }

template <typename T>
__device__ __forceinline__ typename CT<T>::t symbol(int op, T kx, T ky, T kz, bool nyq_x, bool nyq_y, bool nyq_z,
                                                    T What) {
  typedef typename CT<T>::t V;
  switch (op) {
    case SYM_W: return mk<V>(What, 0.0);
    case SYM_DX: return mk<V>(0.0, nyq_x ? (T)0 : mul_rn(kx, What));
    case SYM_DY: return mk<V>(0.0, nyq_y ? (T)0 : mul_rn(ky, What));
    case SYM_DZ: return mk<V>(0.0, nyq_z ? (T)0 : mul_rn(kz, What));
    case SYM_LAP: {
      const T k2 = add_rn(add_rn(mul_rn(kx, kx), mul_rn(ky, ky)), mul_rn(kz, kz));
      return mk<V>(-mul_rn(k2, What), 0.0);
    }
    case SYM_ONE: return mk<V>((T)1.0, 0.0);
    default: {  // projection terms: g = (i kx W_hat, i ky W_hat) up to the common factor i W_hat
      const T gx = nyq_x ? (T)0 : kx, gy = nyq_y ? (T)0 : ky;
      const T g2 = add_rn(mul_rn(gx, gx), mul_rn(gy, gy));
      if (!(static_cast<float>(g2) > 0.f)) return mk<V>(0.0, 0.0);
      const T num = op == SYM_NPXX ? mul_rn(gx, gx) : op == SYM_NPXY ? mul_rn(gx, gy) : mul_rn(gy, gy);
      return mk<V>(-div_rn(num, g2), 0.0);
    }
  }
}

// sum_{m<n} s^m / m! (n = family) in Horner form with constant coefficients:
// W_hat = e^{-s} times this.
template <typename T> __device__ __forceinline__ T kernel_poly(int family, T s) {
  const T one = (T)1.0;
  switch (family) {
    case 1: return one;
    case 2: return one + s;
    case 3: return one + s * (one + s * (T)0.5);
    case 4: return one + s * (one + s * ((T)0.5 + s * (T)(1.0 / 6.0)));
    default: return one + s * (one + s * ((T)0.5 + s * ((T)(1.0 / 6.0) + s * (T)(1.0 / 24.0))));
  }
}

// Row (x) pass over the x lines of the y half-spectra: line q of an instance
// is the ky = q / nz row at z index kq = q % nz (3D: the spectra are already
// transformed in z; 2D: nz = 1, line q = row ky), its nx elements at stride
// nz.  For Rr lines of one instance: load nin input lines, FC-extend in x
// (walled x), FFT (length mx); then for each output in turn form
// sum_t S_t * F_t times `scale`, inverse FFT, truncate to nx and store.
// The symbols S_t are W_hat (Wt: the context's [hy nz][mx] table of Eq. 16 in
// the transform type) times 1, i kx, i ky, i kz or -|k|^2.
// Shared memory: the nin input lines and their scratch (2 nin Rr lines; one
// half holds the spectra, the other serves the outputs), plus Rr lines when
// nin = 1.
template <typename T>
__device__ __forceinline__ void row_sym_body(const GridDev& g, const typename CT<T>::t* sp_in, typename CT<T>::t* sp_out,
                                             size_t fstride_in, size_t bstride_in, size_t fstride_out,
                                             size_t bstride_out, const RowOps& ops, const typename FcTab<T>::t* E,
                                             const FftPlan& P, const typename CT<T>::t* pool, const T* Wt,
                                             double scale, int Rr, int ls, int bx, int by) {
  typedef typename CT<T>::t V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nin = ops.nin, nout = ops.nout;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + (size_t)nin * Rr * ls;
  const int b = by + g.b0;
  if (inactive(g, b)) return;
  const int q0 = bx * Rr;
  const int nx = g.nx, mx = g.mx, nz = g.nz;
  const int nq = g.hy * nz;
  for (int f = 0; f < nin; ++f)
    for (int r = 0; r < Rr; ++r) {
      const int q = q0 + r;
      V* L = A + ((size_t)f * Rr + r) * ls;
      const V* S = sp_in + b * bstride_in + f * fstride_in + (size_t)(q / nz) * g.ncol + (q % nz);
      for (int i = threadIdx.x; i < nx; i += blockDim.x) L[i] = q < nq ? S[(size_t)i * nz] : mk<V>(0.0, 0.0);
    }
  __syncthreads();
  if (g.x_walls) {
    fc_append<T>(A, nin * Rr, ls, nx, g.n_cont, g.n_match, E);
    __syncthreads();
  }
  V* X = fft_any<T, false>(A, B, nin * Rr, ls, P, pool);
  V* Cq = (X == A) ? B : A;
  V* D = nin >= 2 ? Cq + (size_t)Rr * ls : B + (size_t)Rr * ls;
  const T ckx = (T)g.ckx_d, cky = (T)g.cky_d, ckz = (T)g.ckz_d;  // 2 pi / (mx dx), 2 pi / (my dy), 2 pi / (nz dz)
  const T tscale = (T)scale;
  for (int o = 0; o < nout; ++o) {
    for (int r = 0; r < Rr; ++r) {
      const int q = q0 + r < nq ? q0 + r : 0;
      const int ky = q / nz, kq = q - (q / nz) * nz;
      const int kzeta = (2 * kq <= nz) ? kq : kq - nz;
      const T kyw = cky * (T)ky, kz = ckz * (T)kzeta;
      const bool nyq_y = (g.my % 2 == 0) && (2 * ky == g.my);
      const bool nyq_z = (nz % 2 == 0) && (2 * kq == nz);
      // W_hat of row q from the context's table (Eq. 16, built once on the host)
      const T* Wq = Wt + (size_t)q * mx;
      for (int kxi = threadIdx.x; kxi < mx; kxi += blockDim.x) {
        const int kappa = (2 * kxi <= mx) ? kxi : kxi - mx;
        const T kx = ckx * (T)kappa;
        const bool nyq_x = (mx % 2 == 0) && (2 * kxi == mx);
        const T What = Wq[kxi];
        V acc = mk<V>(0.0, 0.0);
        for (int t = 0; t < ops.nterm[o]; ++t) {
          const V s = symbol<T>(ops.op[o][t], kx, kyw, kz, nyq_x, nyq_y, nyq_z, What);
          const V x = X[((size_t)ops.field[o][t] * Rr + r) * ls + kxi];
          // acc += s x, rounded step by step (no contraction: the same result at every CTA width)
          acc.x = add_rn(acc.x, add_rn(mul_rn(s.x, x.x), -mul_rn(s.y, x.y)));
          acc.y = add_rn(acc.y, add_rn(mul_rn(s.x, x.y), mul_rn(s.y, x.x)));
        }
        Cq[(size_t)r * ls + kxi] = cscale(acc, tscale);
      }
    }
    __syncthreads();
    V* Y = fft_any<T, true>(Cq, D, Rr, ls, P, pool);
    for (int r = 0; r < Rr; ++r) {
      const int q = q0 + r;
      if (q >= nq) break;
      V* S = sp_out + b * bstride_out + o * fstride_out + (size_t)(q / nz) * g.ncol + (q % nz);
      const V* Yl = Y + (size_t)r * ls;
      for (int i = threadIdx.x; i < nx; i += blockDim.x) S[(size_t)i * nz] = Yl[i];
    }
    __syncthreads();
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T, NT>::v) k_row_sym(GridDev g, const typename CT<T>::t* __restrict__ sp_in,
                                                         typename CT<T>::t* __restrict__ sp_out, size_t fstride_in,
                                                         size_t bstride_in, size_t fstride_out, size_t bstride_out,
                                                         const __grid_constant__ RowOps ops,
                                                         const typename FcTab<T>::t* __restrict__ E,
                                                         const __grid_constant__ FftPlan P, const typename CT<T>::t* __restrict__ pool,
                                                         const T* __restrict__ Wt, double scale, int Rr, int ls) {
  row_sym_body<T>(g, sp_in, sp_out, fstride_in, bstride_in, fstride_out, bstride_out, ops, E, P, pool, Wt, scale, Rr, ls,
                  blockIdx.x, blockIdx.y);
}

// Per-lane constants of the register row pass for one row: lane k1 owns the
// frequencies kxi = k1 + M k2 (k2 < 32) of row q (Wq: its W_hat row).
struct WRowSym {
  float ckx, kyw, kz;
  bool nyq_y, nyq_z;
  int mx, k1;
  const float* Wq;
  float kx0, wrap;  // ckx k1 and ckx mx: kx = kx0 + ckx M k2 (- wrap past mx/2), no int-to-float per element
};

// v[k2] += symbol OP (kx of k1 + M k2) x spectrum value ([k2][lane] at xr, xi).
template <int OP, int M>
__device__ __forceinline__ void w_accumulate(float2* v, const float* xr, const float* xi, const WRowSym& r) {
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) {
    const int kxi = r.k1 + M * k2;
    const float kxu = fmaf(r.ckx, (float)(M * k2), r.kx0);  // M k2 is a compile-time constant
    const float kx = (2 * kxi <= r.mx) ? kxu : kxu - r.wrap;
    const bool nyq_x = (r.mx % 2 == 0) && (2 * kxi == r.mx);
    const float What = (OP == SYM_ONE || OP == SYM_NPXX || OP == SYM_NPXY || OP == SYM_NPYY) ? 1.f : r.Wq[kxi];
    const float2 sy = symbol<float>(OP, kx, r.kyw, r.kz, nyq_x, r.nyq_y, r.nyq_z, What);
    const float2 x = make_float2(xr[k2 * 32], xi[k2 * 32]);
    if (OP == SYM_DX || OP == SYM_DY || OP == SYM_DZ) {  // purely imaginary symbol i sy.y
      v[k2].x = add_rn(v[k2].x, -mul_rn(sy.y, x.y));
      v[k2].y = add_rn(v[k2].y, mul_rn(sy.y, x.x));
    } else {  // real symbol sy.x
      v[k2].x = add_rn(v[k2].x, mul_rn(sy.x, x.x));
      v[k2].y = add_rn(v[k2].y, mul_rn(sy.x, x.y));
    }
  }
}

// Row pass of FP32 contexts with periodic x lines of mx = nx = 32 M points
// (M = 2 .. 32): the same operation as k_row_sym, with the register FFT of
// fcsph_warpfft.cuh.  One warp carries 32 / M rows through every transform;
// a CTA holds 4 warps.  The forward spectra of the nin inputs wait in shared
// memory ([field][k2][lane] of this warp, conflict-free) while the outputs are
// formed one at a time, each in the registers of the lane that owns its
// frequencies kx = k1 + M k2 (lane = l M + k1).
template <int M>
__global__ void __launch_bounds__(128, 3) k_row_sym_w(GridDev g, const float2* __restrict__ sp_in,
                                                      float2* __restrict__ sp_out, size_t fstride_in,
                                                      size_t bstride_in, size_t fstride_out, size_t bstride_out,
                                                      const __grid_constant__ RowOps ops,
                                                      const float2* __restrict__ roots,
                                                      const float* __restrict__ Wt, double scale) {
  constexpr int LPW = 32 / M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nin = ops.nin, nout = ops.nout;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* xs = reinterpret_cast<float*>(smem_raw) + (size_t)warp * (kWarpXchgFloats + nin * 2 * 32 * 32);
  float* spre = xs + kWarpXchgFloats;
  float* spim = spre + nin * 32 * 32;
  const int b = blockIdx.y + g.b0;
  if (inactive(g, b)) return;
  const int mx = g.mx, nz = g.nz;
  const int nq = g.hy * nz;
  const int q0 = (blockIdx.x * 4 + warp) * LPW;
  if (q0 >= nq) return;  // whole warp beyond the last row (uniform)
  for (int f = 0; f < nin; ++f) {
    float2 v[32];
#pragma unroll
    for (int l = 0; l < LPW; ++l) {
      const int q = q0 + l;
      const float2* S = sp_in + b * bstride_in + f * fstride_in + (size_t)(q / nz) * g.ncol + (q % nz);
#pragma unroll
      for (int j = 0; j < M; ++j) v[l * M + j] = q < nq ? S[(size_t)(lane + 32 * j) * nz] : make_float2(0.f, 0.f);
    }
    warp_fft_fwd<M>(v, xs, roots, lane);
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
      spre[(f * 32 + k2) * 32 + lane] = v[k2].x;
      spim[(f * 32 + k2) * 32 + lane] = v[k2].y;
    }
  }
  __syncwarp();
  const int l = lane / M, k1 = lane - (lane / M) * M;
  const int q = q0 + l < nq ? q0 + l : q0;
  const float ckx = g.ckx_f, cky = g.cky_f, ckz = g.ckz_f;
  const int ky = q / nz, kq = q - (q / nz) * nz;
  const int kzeta = (2 * kq <= nz) ? kq : kq - nz;
  const float kyw = cky * (float)ky, kz = ckz * (float)kzeta;
  const bool nyq_y = (g.my % 2 == 0) && (2 * ky == g.my);
  const bool nyq_z = (nz % 2 == 0) && (2 * kq == nz);
  const float* Wq = Wt + (size_t)q * mx;
  const float tscale = (float)scale;
  const WRowSym rs{ckx, kyw, kz, nyq_y, nyq_z, mx, k1, Wq, ckx * (float)k1, ckx * (float)mx};
  for (int o = 0; o < nout; ++o) {
    float2 v[32];
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = make_float2(0.f, 0.f);
    for (int t = 0; t < ops.nterm[o]; ++t) {
      const float* xr = spre + ops.field[o][t] * 32 * 32 + lane;
      const float* xi = spim + ops.field[o][t] * 32 * 32 + lane;
      switch (ops.op[o][t]) {  // uniform over the warp: one unrolled loop per symbol
        case SYM_W: w_accumulate<SYM_W, M>(v, xr, xi, rs); break;
        case SYM_DX: w_accumulate<SYM_DX, M>(v, xr, xi, rs); break;
        case SYM_DY: w_accumulate<SYM_DY, M>(v, xr, xi, rs); break;
        case SYM_LAP: w_accumulate<SYM_LAP, M>(v, xr, xi, rs); break;
        case SYM_DZ: w_accumulate<SYM_DZ, M>(v, xr, xi, rs); break;
        case SYM_ONE: w_accumulate<SYM_ONE, M>(v, xr, xi, rs); break;
        case SYM_NPXX: w_accumulate<SYM_NPXX, M>(v, xr, xi, rs); break;
        case SYM_NPXY: w_accumulate<SYM_NPXY, M>(v, xr, xi, rs); break;
        default: w_accumulate<SYM_NPYY, M>(v, xr, xi, rs); break;
      }
    }
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = cscale(v[k2], tscale);
    warp_fft_inv<M>(v, xs, roots, lane);
#pragma unroll
    for (int l2 = 0; l2 < LPW; ++l2) {
      const int qq = q0 + l2;
      if (qq < nq) {
        float2* S = sp_out + b * bstride_out + o * fstride_out + (size_t)(qq / nz) * g.ncol + (qq % nz);
#pragma unroll
        for (int j = 0; j < M; ++j) S[(size_t)(lane + 32 * j) * nz] = v[l2 * M + j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Line operator: every column of [batch][nx][ny] is an independent
// wall-normal line.  Per column pair (packed as one complex line): FC-extend
// (table E), FFT (length my); then for each output the symbol at kx = 0 --
// W_hat(ky), i ky W_hat (zero on the Nyquist mode), -ky^2 W_hat, and 0 for
// d/dx -- times the spectrum, inverse FFT, truncation to ny, scale 1/my.  The
// symbols are Hermitian in ky, so the real and imaginary parts of the packed
// result are the two columns' outputs.  One kernel per call.
struct LineOuts {
  int nout;
  int op[4];
  void* out[4];
};

template <typename T, typename U, int NT>
__global__ void __launch_bounds__(NT, LineMinCtas<T, NT>::v) k_line_op(GridDev g, const U* __restrict__ f,
                                                                      long long ncols,
                                                                      const typename FcTab<T>::t* __restrict__ E,
                                                                      const __grid_constant__ FftPlan P,
                                                                      const typename CT<T>::t* __restrict__ pool,
                                                                      const __grid_constant__ LineOuts lo, int Pp,
                                                                      int ls) {
  typedef typename CT<T>::t V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* X = reinterpret_cast<V*>(smem_raw);
  V* Cq = X + (size_t)Pp * ls;
  V* D = Cq + (size_t)Pp * ls;
  const long long c0 = (long long)blockIdx.x * 2 * Pp;
  const int ny = g.ny, my = g.my;
  for (int col = 0; col < 2 * Pp; ++col) {
    const long long cc = c0 + col;
    T* L = reinterpret_cast<T*>(X + (size_t)(col >> 1) * ls) + (col & 1);
    for (int j = threadIdx.x; j < ny; j += blockDim.x) L[2 * j] = cc < ncols ? (T)f[cc * ny + j] : (T)0;
  }
  __syncthreads();
  fc_append<T>(X, Pp, ls, ny, g.n_cont, g.n_match, E);
  __syncthreads();
  V* R = fft_any<T, false>(X, Cq, Pp, ls, P, pool);
  V* W1 = (R == X) ? Cq : X;
  const T hh = (T)g.hh_d, cky = (T)g.cky_d;  // h^2 / 4, 2 pi / (my dy)
  const T tscale = (T)(1.0 / my);
  for (int o = 0; o < lo.nout; ++o) {
    const int op = lo.op[o];
    for (int p = 0; p < Pp; ++p)
    for (int k = threadIdx.x; k < my; k += blockDim.x) {
      const int kappa = (2 * k <= my) ? k : k - my;
      const T ky = cky * (T)kappa;
      const T What = pool[g.ey_off + (kappa < 0 ? -kappa : kappa)].x * kernel_poly<T>(g.family, ky * ky * hh);
      const bool nyq = (my % 2 == 0) && (2 * k == my);
      V s;
      if (op == SYM_W)
        s = mk<V>(What, 0);
      else if (op == SYM_DY)
        s = mk<V>(0, nyq ? (T)0 : ky * What);
      else if (op == SYM_LAP)
        s = mk<V>(-(ky * ky) * What, 0);
      else
        s = mk<V>(0, 0);
      W1[(size_t)p * ls + k] = cscale(cmul(s, R[(size_t)p * ls + k]), tscale);
    }
    __syncthreads();
    V* Y = fft_any<T, true>(W1, D, Pp, ls, P, pool);
    U* out = reinterpret_cast<U*>(lo.out[o]);
    for (int col = 0; col < 2 * Pp; ++col) {
      const long long cc = c0 + col;
      if (cc >= ncols) break;
      const V* Yl = Y + (size_t)(col >> 1) * ls;
      for (int j = threadIdx.x; j < ny; j += blockDim.x) out[cc * ny + j] = (U)((col & 1) ? Yl[j].y : Yl[j].x);
    }
    __syncthreads();
  }
}

// Two adjacent FP32 columns (c0 = src[0..ny), c1 = src[ny..2 ny); c1 absent:
// zeros) packed into the complex line L[j] = (c0[j], c1[j]).  With ny a
// multiple of 4 and a 16-byte aligned start every thread issues its float4
// loads of both columns back to back; otherwise plain loads.
__device__ __forceinline__ void load_pair_f32(float2* L, const float* __restrict__ src, bool has1, int ny) {
  const int t = threadIdx.x, nt = blockDim.x;
  if ((ny & 3) == 0 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
    const float4* c0 = reinterpret_cast<const float4*>(src);
    const float4* c1 = reinterpret_cast<const float4*>(src + ny);
    for (int m = t; m < ny / 4; m += nt) {
      const float4 a = c0[m];
      const float4 b = has1 ? c1[m] : make_float4(0.f, 0.f, 0.f, 0.f);
      float4* d = reinterpret_cast<float4*>(L + 4 * m);
      d[0] = make_float4(a.x, b.x, a.y, b.y);
      d[1] = make_float4(a.z, b.z, a.w, b.w);
    }
  } else {
    for (int j = t; j < ny; j += nt) L[j] = make_float2(src[j], has1 ? src[ny + j] : 0.f);
  }
}

// The line operator of FP32 contexts with the register team FFT
// (fcsph_regfft.cuh) for extended lengths n = N1 N2: one column pair per CTA;
// the forward spectrum waits in shared memory, each value where the thread
// that owns its frequency (k = t + N1 k2) reads it back, while the outputs are
// formed one at a time.
template <int N1, int N2>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_line_op_r(
    GridDev g, const float* __restrict__ f, long long ncols, const typename FcTab<float>::t* __restrict__ E,
    const float2* __restrict__ pool, const float2* __restrict__ roots, const __grid_constant__ LineOuts lo) {
  typedef TeamFFT<N1, N2> TF;
  constexpr int n = N1 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* L = reinterpret_cast<float2*>(smem_raw);
  float2* xs = L + n;
  const long long c0 = (long long)blockIdx.x * 2;
  const int ny = g.ny, t = threadIdx.x;
  load_pair_f32(L, f + c0 * ny, c0 + 1 < ncols, ny);
  __syncthreads();
  fc_append<float>(L, 1, n, ny, g.n_cont, g.n_match, E);
  __syncthreads();
  float2 x[TF::NV];
  if (t < N2) {
#pragma unroll
    for (int j = 0; j < N1; ++j) x[j] = L[t + N2 * j];
  }
  TF::fwd(x, xs, roots, t);
  if (t < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) L[t + N1 * k2] = x[k2];
  }
  const float hh = g.hh_f, cky = g.cky_f, tscale = g.inv_my_f;  // n = my
  const float ky0 = cky * (float)t;
  for (int o = 0; o < lo.nout; ++o) {
    const int op = lo.op[o];
    float2 y[TF::NV];
    if (t < N1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int k = t + N1 * k2;
        const int kappa = (2 * k <= n) ? k : k - n;
        const float kyu = fmaf(cky, (float)(N1 * k2), ky0);  // N1 k2 is a compile-time constant
        const float ky = (2 * k <= n) ? kyu : kyu - cky * (float)n;
        const float What = pool[g.ey_off + (kappa < 0 ? -kappa : kappa)].x * kernel_poly<float>(g.family, ky * ky * hh);
        const bool nyq = (n % 2 == 0) && (2 * k == n);
        float2 sy;
        if (op == SYM_W)
          sy = make_float2(What, 0.f);
        else if (op == SYM_DY)
          sy = make_float2(0.f, nyq ? 0.f : ky * What);
        else if (op == SYM_LAP)
          sy = make_float2(-(ky * ky) * What, 0.f);
        else
          sy = make_float2(0.f, 0.f);
        y[k2] = cscale(cmul(sy, L[k]), tscale);
      }
    }
    TF::inv(y, xs, roots, t);
    if (t < N2) {
      float* out = reinterpret_cast<float*>(lo.out[o]);
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const int row = t + N2 * j;
        if (row < ny) {
          if (c0 < ncols) out[c0 * ny + row] = y[j].x;
          if (c0 + 1 < ncols) out[(c0 + 1) * ny + row] = y[j].y;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// z pass of the 3D channel: in the spectra [b][field][row][x][z] every run of
// nz values (fixed b, field, row, x) is one periodic z line; L lines per CTA
// are transformed in place, forward or (inv) unnormalised inverse.  Instances
// with active[b] == 0 (isph_step's mask, when given) are left alone.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T, NT>::v) k_zlines(typename CT<T>::t* __restrict__ spec,
                                                                      int lines_per_field, size_t fstride,
                                                                      size_t bstride, const __grid_constant__ FftPlan P,
                                                                      const typename CT<T>::t* __restrict__ pool, int L,
                                                                      int ls, int inv, const unsigned char* active,
                                                                      int b0) {
  typedef typename CT<T>::t V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.z + b0;
  if (active && !active[b]) return;
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + (size_t)L * ls;
  const int n = P.base.n;
  V* base = spec + b * bstride + blockIdx.y * fstride;
  const int l0 = blockIdx.x * L;
  for (int r = 0; r < L; ++r) {
    const bool in = l0 + r < lines_per_field;
    const V* S = base + (size_t)(l0 + r) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) A[(size_t)r * ls + j] = in ? S[j] : mk<V>(0.0, 0.0);
  }
  __syncthreads();
  V* Y = fft_any_rt<T>(A, B, L, ls, P, pool, inv != 0);
  for (int r = 0; r < L; ++r) {
    if (l0 + r >= lines_per_field) break;
    V* S = base + (size_t)(l0 + r) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) S[j] = Y[(size_t)r * ls + j];
  }
}

// ---------------------------------------------------------------------------
// PPE row pass (Eqs. 31-33): rows l < ny hold DCT-I-in-y coefficients.  x
// periodic: FFT (length nx); walled x: DCT-I via FFT of the even extension
// (length 2(nx-1)).  Multiply by -1/(lam_k^2 + lam_l^2) (apply = 0, (0,0) -> 0),
// by -(lam_k^2 + lam_l^2) (apply = 1), or by 1 except 0 on the (0,0) mode
// (apply = 2, removes the constant mode), times the inverse-transform scales,
// transform back, store.  3D: line q is the l = q / nz row at z index
// kq = q % nz of the DFT-z-transformed coefficients, elements at stride nz,
// and lam_z^2 joins the denominator.
template <typename T>
__device__ __forceinline__ void row_ppe_body(const GridDev& g, typename CT<T>::t* spec, size_t bstride, const FftPlan& P,
                                             const typename CT<T>::t* pool, int apply, int Rr, int ls, int bx, int by) {
  typedef typename CT<T>::t V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + (size_t)Rr * ls;
  const int b = by + g.b0;
  if (inactive(g, b)) return;
  const int q0 = bx * Rr;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nq = ny * nz;
  const int n = P.base.n;  // nx or 2(nx-1)
  for (int r = 0; r < Rr; ++r) {
    const int q = q0 + r;
    V* L = A + (size_t)r * ls;
    const V* S = spec + b * bstride + (size_t)(q / nz) * g.ncol + (q % nz);
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const V v = q < nq ? S[(size_t)i * nz] : mk<V>(0.0, 0.0);
      L[i] = v;
      if (g.x_walls && i >= 1 && i <= nx - 2) L[n - i] = v;
    }
  }
  __syncthreads();
  V* X = fft_any<T, false>(A, B, Rr, ls, P, pool);
  V* O = (X == A) ? B : A;
  const T norm = (T)(1.0 / ((double)n * 2.0 * (ny - 1) * nz));
  const int nk = g.x_walls ? nx : n;
  for (int r = 0; r < Rr; ++r) {
    const int q = q0 + r < nq ? q0 + r : 0;
    const int l = q / nz, kq = q - (q / nz) * nz;
    // lam_l^2 (+ lam_z^2) from the per-axis tables (Eq. 33 eigenvalues)
    const T dyz = pool[g.ly2_off + l].x + pool[g.lz2_off + kq].x;
    const bool zero_yz = l == 0 && kq == 0;
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    const T den = pool[g.lx2_off + k].x + dyz;
    T f;
    if (apply == 1)
      f = -(den * norm);
    else if (apply == 2)
      f = (k == 0 && zero_yz) ? (T)0.0 : norm;
    else
      f = (k == 0 && zero_yz) ? (T)0.0 : -(norm / den);
    const V x = X[(size_t)r * ls + k];
    const V y = cscale(x, f);
    if (g.x_walls) {
      O[(size_t)r * ls + k] = y;
      if (k >= 1 && k <= nx - 2) O[(size_t)r * ls + n - k] = y;
    } else {
      X[(size_t)r * ls + k] = y;
    }
  }
  }
  __syncthreads();
  V* Y;
  if (g.x_walls)
    Y = fft_any<T, false>(O, X, Rr, ls, P, pool);  // DCT-I is its own inverse up to the folded scale
  else
    Y = fft_any<T, true>(X, O, Rr, ls, P, pool);
  for (int r = 0; r < Rr; ++r) {
    const int q = q0 + r;
    if (q >= nq) break;
    V* S = spec + b * bstride + (size_t)(q / nz) * g.ncol + (q % nz);
    const V* Yl = Y + (size_t)r * ls;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) S[(size_t)i * nz] = Yl[i];
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T, NT>::v) k_row_ppe(GridDev g, typename CT<T>::t* __restrict__ spec,
                                                      size_t bstride, const __grid_constant__ FftPlan P,
                                                      const typename CT<T>::t* __restrict__ pool, int apply, int Rr,
                                                      int ls) {
  row_ppe_body<T>(g, spec, bstride, P, pool, apply, Rr, ls, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Column inverse with epilogues.
enum { EPI_OUT = 0, EPI_MOM = 1, EPI_DIV = 2, EPI_CORR = 3, EPI_PPE_SOLVE = 4, EPI_PPE_RESID = 5, EPI_PPE_ADD = 6 };

struct EpiArgs {
  // EPI_OUT
  void* outs[6];
  int out_double;
  // step state (double), per velocity component (2D: u, v; 3D: u, v, w)
  const double* vel[3];   // MOM: velocity at the start of the substep
  double* Fp[3];          // MOM: F^{k-1} in, F^k out
  double* vs[3];          // MOM: u* out; CORR: u* in
  double* vo[3];          // CORR: corrected velocity out
  int mom_terms;          // MOM: outputs per component (d/dx, d/dy, [d/dz], lap)
  double* bvec;       // DIV: out b; PPE_RESID: in b
  double* phi;        // PPE_*: out phi / residual / accumulate
  void* phi_any;      // PPE_SOLVE in the context's I/O type when not double
  int phi_double;
  StepDev s;
  // fused forward: nf fields, table, plan, output spectra, dct
  int fwd_nf;
  int fwd_dct;
  const void* fwdE;   // FC table in the transform's FcTab type
  FftPlan fwdP;
  void* fwd_spec;
  size_t fwd_fstride, fwd_bstride;
  int* status;
};

// L2 prefetch hints for the column pass.  Only addresses the kernel reads
// later are named, so every one lies inside its buffer.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Rows k < hy of one field's half-spectrum at the CTA's column pairs.
template <typename V>
__device__ void prefetch_spec_pairs(const GridDev& g, int i0, int Pp, const V* spec) {
  for (int t = threadIdx.x; t < g.hy * Pp; t += blockDim.x) {
    const int k = t / Pp, p = t - k * Pp;
    if (i0 + 2 * p < g.ncol) prefetch_l2(spec + (size_t)k * g.ncol + i0 + 2 * p);
  }
}

// The CTA's columns of one FP64 field of instance b, 128-byte lines.
__device__ void prefetch_field_cols(const GridDev& g, int b, int i0, int Pp, const double* f) {
  const int per = (g.ny + 15) / 16 + 1;  // lines of one column, one more for an unaligned start
  const int nc = min(2 * Pp, g.ncol - i0);
  for (int t = threadIdx.x; t < nc * per; t += blockDim.x) {
    const int c = t / per, l = t - c * per;
    prefetch_l2(f + fidx(g, b, i0 + c, min(16 * l, g.ny - 1)));
  }
}

// The FP64 field the fused forward of a column pass transforms: its f-th new
// field, which the epilogue has written to global memory.
__device__ __forceinline__ const double* fwd_field(const EpiArgs& ea, int EPI, int f) {
  if (EPI == EPI_MOM) return ea.vs[f];
  if (EPI == EPI_CORR) return ea.vo[f];
  if (EPI == EPI_DIV) return ea.bvec;
  return ea.phi;  // PPE_SOLVE, PPE_ADD
}

// The epilogue kind is a runtime argument (uniform across the grid): one
// instantiation per precision keeps the build small.
//
// Column pairs i0 + 2p, i0 + 2p + 1 (p < Pp) of one instance.  The nout
// inverse transforms run one at a time: gather the half spectrum of output o
// into packed lines Z, inverse FFT (scratch S), then the epilogue consumes
// output o.  Per-point FP64 values that later outputs or the fused forward
// need stay in global memory, in the arrays the epilogue writes anyway (and
// in L2 between the passes over one CTA's columns): the momentum terms
// accumulate u.grad + nu lap of each component in its u* array (overwritten
// by u* at the last term), and the fused forward transforms fwd_field(f)
// (f < fwd_nf), the new fields of this pass, with Z and S as its lines.
// Shared memory then holds only the lines: 2 Pp ls values.
template <typename T>
__device__ __forceinline__ void col_inv_body(const GridDev& g, const typename CT<T>::t* spec, size_t fstride,
                                             size_t bstride, int nout, const FftPlan& P,
                                             const typename CT<T>::t* pool, const EpiArgs& ea, int Pp, int ls,
                                             const int EPI, int bx, int by) {
  typedef typename CT<T>::t V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Z = reinterpret_cast<V*>(smem_raw);
  V* S = Z + (size_t)Pp * ls;
  const int b = by + g.b0;
  if (inactive(g, b)) return;
  const int i0 = bx * 2 * Pp;
  const int ny = g.ny;
  const bool ppe = (EPI == EPI_PPE_SOLVE || EPI == EPI_PPE_RESID || EPI == EPI_PPE_ADD);
  // the instance's step parameters and the epilogue factors, once per CTA:
  // inside the point loops the compiler would reload them after every store
  // and repeat the FP64 divisions per point
  const double nu_b = ea.s.nu_inst ? ea.s.nu_inst[b] : ea.s.nu;
  const double fx_b = ea.s.fx_inst ? ea.s.fx_inst[b] : ea.s.fx;
  const double dt_b = ea.s.dt_inst ? ea.s.dt_inst[b] : ea.s.dt;
  const double div_c = EPI == EPI_DIV ? ea.s.rho / (ea.s.a * dt_b) : 0.0;   // rho / (a dt)
  const double corr_c = EPI == EPI_CORR ? ea.s.a * dt_b / ea.s.rho : 0.0;  // a dt / rho
  for (int o = 0; o < nout; ++o) {
    V* R;
    if (ppe) {
      col_gather_dct<T>(Z, Pp, ls, g, i0, spec + b * bstride);
      __syncthreads();
      R = fft_any<T, false>(Z, S, Pp, ls, P, pool);
    } else {
      col_gather_hermitian<T>(Z, Pp, ls, g, i0, spec + b * bstride + o * fstride, fstride, 1, P.base.n);
      // while this output is transformed, bring the next one's spectrum and
      // this output's FP64 epilogue operands (state columns) into L2
      if (o + 1 < nout) prefetch_spec_pairs(g, i0, Pp, spec + b * bstride + (o + 1) * fstride);
      if (EPI == EPI_MOM) {
        const int nt = ea.mom_terms, comp = o / nt, term = o - comp * nt;
        prefetch_field_cols(g, b, i0, Pp, ea.vel[term < nt - 1 ? term : comp]);
        if (term == nt - 1) prefetch_field_cols(g, b, i0, Pp, ea.Fp[comp]);
      } else if (EPI == EPI_CORR) {
        prefetch_field_cols(g, b, i0, Pp, ea.vs[o]);
      }
      __syncthreads();
      R = fft_any<T, true>(Z, S, Pp, ls, P, pool);
    }
    for (int p = 0; p < Pp; ++p)
    for (int j = threadIdx.x; j < ny; j += blockDim.x) {
      const V z = R[(size_t)p * ls + j];
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int i = i0 + 2 * p + w;
        if (i >= g.ncol) continue;
        const size_t id = fidx(g, b, i, j);
        const T zv = w ? z.y : z.x;
        if (EPI == EPI_OUT) {
          // straight from the compute type to the output type
          if (ea.out_double)
            reinterpret_cast<double*>(ea.outs[o])[id] = (double)zv;
          else
            reinterpret_cast<float*>(ea.outs[o])[id] = (float)zv;
          continue;
        }
        const double val = (double)zv;
        if (EPI == EPI_MOM) {
          // output comp * nt + term: d/dx, d/dy, (d/dz,) lap of component comp;
          // F_comp = u . grad(comp) - nu lap(comp) accumulates in u*_comp
          const int nt = ea.mom_terms;
          const int comp = o / nt, term = o - comp * nt;
          double* a = ea.vs[comp] + id;
          if (term == 0) {
            *a = ea.vel[0][id] * val;
          } else if (term < nt - 1) {
            *a += ea.vel[term][id] * val;
          } else {
            const double nu = nu_b;
            const double F = *a - nu * val;
            const double f = comp == 0 ? fx_b : (comp == 1 ? ea.s.fy : ea.s.fz);
            const double dt = dt_b;
            double cs = ea.vel[comp][id] + dt * (-ea.s.g * F - ea.s.z * ea.Fp[comp][id] + ea.s.a * f);
            // y walls: the tangential x velocity takes the wall speeds, the others 0
            if (j == 0) cs = comp == 0 ? ea.s.u_bottom : 0.0;
            if (j == ny - 1) cs = comp == 0 ? ea.s.u_top : 0.0;
            if (g.x_walls && (i == 0 || i == g.nx - 1)) cs = 0.0;
            ea.Fp[comp][id] = F;
            *a = cs;
            if (!isfinite(cs)) atomicOr(ea.status, 1);
          }
        } else if (EPI == EPI_DIV) {
          ea.bvec[id] = div_c * val;
        } else if (EPI == EPI_CORR) {
          // output o: d phi / d(axis o) -> component o
          const double c = corr_c;
          double cn = ea.vs[o][id] - c * val;
          if (j == 0) cn = o == 0 ? ea.s.u_bottom : 0.0;
          if (j == ny - 1) cn = o == 0 ? ea.s.u_top : 0.0;
          if (g.x_walls && (i == 0 || i == g.nx - 1)) cn = 0.0;
          ea.vo[o][id] = cn;
          if (!isfinite(cn)) atomicOr(ea.status, 1);
        } else if (EPI == EPI_PPE_SOLVE) {
          if (ea.phi_double)
            reinterpret_cast<double*>(ea.phi_any)[id] = val;
          else
            reinterpret_cast<float*>(ea.phi_any)[id] = (float)val;
          if (ea.phi) ea.phi[id] = val;
        } else if (EPI == EPI_PPE_RESID) {
          ea.phi[id] = ea.bvec[id] - val;  // r = b - L phi
        } else if (EPI == EPI_PPE_ADD) {
          ea.phi[id] = ea.phi[id] + val;
        }
      }
    }
    __syncthreads();
  }
  for (int f = 0; f < ea.fwd_nf; ++f) {
    // the new field f as this CTA's threads stored it above (a thread reads
    // back its own points; columns beyond nx, a ragged last pair, are zero)
    const double* a = fwd_field(ea, EPI, f);
    for (int p = 0; p < Pp; ++p) {
      const int i = i0 + 2 * p;
      V* L = Z + (size_t)p * ls;
      for (int j = threadIdx.x; j < ny; j += blockDim.x)
        L[j] = mk<V>(i < g.ncol ? a[fidx(g, b, i, j)] : 0.0, i + 1 < g.ncol ? a[fidx(g, b, i + 1, j)] : 0.0);
    }
    __syncthreads();
    col_forward_store<T>(Z, S, Pp, ls, g, i0, reinterpret_cast<const typename FcTab<T>::t*>(ea.fwdE), ea.fwdP, pool,
                         ea.fwd_dct, reinterpret_cast<V*>(ea.fwd_spec) + b * ea.fwd_bstride + f * ea.fwd_fstride);
    __syncthreads();
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, MinCtas<T, NT>::v) k_col_inv(GridDev g, const typename CT<T>::t* __restrict__ spec,
                                                         size_t fstride, size_t bstride, int nout,
                                                         const __grid_constant__ FftPlan P,
                                                         const typename CT<T>::t* __restrict__ pool,
                                                         const __grid_constant__ EpiArgs ea, int Pp, int ls,
                                                         const int EPI) {
  col_inv_body<T>(g, spec, fstride, bstride, nout, P, pool, ea, Pp, ls, EPI, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Persistent step of several size classes in one launch.  Every pass of one
// RK3 step of every class is recorded as a descriptor (the arguments its
// launch would get); a work item is one CTA's share of one pass for one
// instance: (descriptor, tile x, tile y, instance).  Items are listed pass by
// pass (pass index p of every class, then p + 1, ...), and the CTAs of one
// launch take them in that order from an atomic counter.  Item (c, b, p)
// waits until every tile of pass p - 1 of the same instance has finished
// (a per-(class, instance, pass) counter), so the classes' passes and their
// instances interleave freely.  No deadlock is possible: an item only waits
// for items taken before it, and the oldest unfinished item waits for nothing.
// Waits are bounded (time and spin count); one that runs out sets bit 1 of
// the plan's status word, and from then on every item is skipped (and
// counted) so the launch drains at once.
enum { PK_COL_FWD = 1, PK_ROW_SYM = 2, PK_COL_INV = 3, PK_ROW_PPE = 4 };

struct PassDesc {
  int kind;
  int gx, gy, gz;  // the grid the pass's own launch would have
  size_t smem;
  int Pp, Rr, ls;
  GridDev g;
  FftPlan P;
  const void* pool;
  const void* E;
  // column forward / column inverse
  const void* f[3];
  int dct;
  void* spec;
  size_t fstride, bstride;
  // row passes
  const void* sp_in;
  void* sp_out;
  size_t fs_in, bs_in, fs_out, bs_out;
  RowOps ops;
  const void* W;
  double scale;
  int apply;
  // column inverse
  int nout, epi;
  EpiArgs ea;
};

struct WorkItem {
  int desc, bx, by, b;
  int dep;   // counter the item waits on (-1: none)
  int need;  // value that counter must reach
  int self;  // counter the item increments when done
};

constexpr int kPersistTimeout = 2;          // status bit: a dependency wait ran out
constexpr long long kPersistMaxSpins = 1ll << 26;

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One function per pass kind, each compiled (and register-allocated) on its
// own rather than all four inlined into the persistent loop.  The descriptor
// is read-only for the whole launch and aliases nothing the pass writes
// (__restrict__): its fields are loaded once, not again after every store.
template <typename T> __device__ __noinline__ void item_col_fwd(const PassDesc& __restrict__ d, int bx, int by, int b) {
  typedef typename CT<T>::t V;
  col_fwd_body<T, double>(d.g, (const double*)d.f[0], (const double*)d.f[1], (const double*)d.f[2],
                          (const typename FcTab<T>::t*)d.E, d.P, (const V*)d.pool, d.dct, (V*)d.spec, d.fstride,
                          d.bstride, d.Pp, d.ls, bx, by, b);
}
template <typename T> __device__ __noinline__ void item_row_sym(const PassDesc& __restrict__ d, int bx, int b) {
  typedef typename CT<T>::t V;
  row_sym_body<T>(d.g, (const V*)d.sp_in, (V*)d.sp_out, d.fs_in, d.bs_in, d.fs_out, d.bs_out, d.ops,
                  (const typename FcTab<T>::t*)d.E, d.P, (const V*)d.pool, (const T*)d.W, d.scale, d.Rr, d.ls, bx, b);
}
template <typename T> __device__ __noinline__ void item_col_inv(const PassDesc& __restrict__ d, int bx, int b) {
  typedef typename CT<T>::t V;
  col_inv_body<T>(d.g, (const V*)d.spec, d.fstride, d.bstride, d.nout, d.P, (const V*)d.pool, d.ea, d.Pp, d.ls,
                  d.epi, bx, b);
}
template <typename T> __device__ __noinline__ void item_row_ppe(const PassDesc& __restrict__ d, int bx, int b) {
  typedef typename CT<T>::t V;
  row_ppe_body<T>(d.g, (V*)d.spec, d.bstride, d.P, (const V*)d.pool, d.apply, d.Rr, d.ls, bx, b);
}

__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__device__ __forceinline__ void run_item(const PassDesc& d, int bx, int by, int b) {
  switch (d.kind) {
    case PK_COL_FWD: item_col_fwd<T>(d, bx, by, b); break;
    case PK_ROW_SYM: item_row_sym<T>(d, bx, b); break;
    case PK_COL_INV: item_col_inv<T>(d, bx, b); break;
    case PK_ROW_PPE: item_row_ppe<T>(d, bx, b); break;
    default: break;
  }
}

// stall >= 0: item `stall` waits for a count that never comes (a test of the
// bounded wait).
// Register budget of the persistent kernel: its pass bodies read the grid,
// plan and epilogue fields from the descriptor in global memory, where the
// per-pass kernels take them as constant-bank operands, so the same code needs
// more registers; the FP32-pair kernel gets up to 255 (8 warps per SM) rather
// than spilling at 168.
template <typename T, int NT> struct PersistMinCtas { static constexpr int v = MinCtas<T, NT>::v; };
template <> struct PersistMinCtas<ff, 32> { static constexpr int v = 8; };
template <> struct PersistMinCtas<ff, 64> { static constexpr int v = 4; };
template <> struct PersistMinCtas<ff, 128> { static constexpr int v = 2; };

template <typename T, int NT>
__global__ void __launch_bounds__(NT, PersistMinCtas<T, NT>::v) k_persist(const PassDesc* descs, const WorkItem* items,
                                                                  int n_items, unsigned* counters, unsigned* next,
                                                                  int* status, long long wait_ns, int stall) {
  __shared__ int s_idx, s_run;
  for (;;) {
    if (threadIdx.x == 0) {
      const int idx = (int)atomicAdd(next, 1u);
      int run = 1;
      if (idx < n_items) {
        const WorkItem it = items[idx];
        if (it.dep >= 0) {
          const unsigned need = idx == stall ? 0xffffffffu : (unsigned)it.need;
          const unsigned* cnt = counters + it.dep;
          const long long t0 = global_ns();
          for (long long spin = 0;; ++spin) {
            if (ld_acquire_gpu(cnt) >= need) break;
            if ((*(volatile int*)status & kPersistTimeout) || spin > kPersistMaxSpins || global_ns() - t0 > wait_ns) {
              atomicOr(status, kPersistTimeout);
              run = 0;
              break;
            }
            __nanosleep(100);
          }
        }
        if (*(volatile int*)status & kPersistTimeout) run = 0;
      }
      s_idx = idx;
      s_run = run;
    }
    // thread 0's acquire of the dependency count, then the CTA barrier, orders
    // the dependency's writes before every load of this item
    __syncthreads();
    const int idx = s_idx, run = s_run;
    if (idx >= n_items) return;
    const WorkItem& it = items[idx];
    if (run) run_item<T>(descs[it.desc], it.bx, it.by, it.b);
    // the barrier, then thread 0's release increment, orders every write of
    // this item before its count
    __syncthreads();
    if (threadIdx.x == 0 && it.self >= 0) red_release_gpu_add(counters + it.self, 1u);
  }
}

// ---------------------------------------------------------------------------
// Wall-normal passes of FP32 contexts with the register team FFT of
// fcsph_regfft.cuh, for extended lengths n = N1 N2 with a direct plan: one
// column pair per CTA of TeamFFT<N1, N2>::THREADS threads.  k_col_fwd_r does
// what k_col_fwd does for FP32 fields (load, FC, forward transform, half
// spectrum); k_col_out_r what k_col_inv does with EPI_OUT into FP32 outputs
// (Hermitian gather, inverse transform, store), for every output.
template <int N1, int N2>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_col_fwd_r(
    GridDev g, const float* __restrict__ f0, const float* __restrict__ f1, const float* __restrict__ f2,
    const typename FcTab<float>::t* __restrict__ E, const float2* __restrict__ roots, float2* __restrict__ spec,
    size_t fstride, size_t bstride) {
  typedef TeamFFT<N1, N2> TF;
  constexpr int n = N1 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* L = reinterpret_cast<float2*>(smem_raw);
  float2* xs = L + n;
  const int b = blockIdx.z + g.b0, f = blockIdx.y;
  if (inactive(g, b)) return;
  const int i0 = blockIdx.x * 2;
  const float* src = f == 0 ? f0 : (f == 1 ? f1 : f2);
  const int ny = g.ny, t = threadIdx.x;
  load_pair_f32(L, src + ((size_t)b * g.ncol + i0) * ny, i0 + 1 < g.ncol, ny);
  __syncthreads();
  fc_append<float>(L, 1, n, ny, g.n_cont, g.n_match, E);
  __syncthreads();
  float2 v[TF::NV];
  if (t < N2) {
#pragma unroll
    for (int j = 0; j < N1; ++j) v[j] = L[t + N2 * j];
  }
  TF::fwd(v, xs, roots, t);
  if (t < N1) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) L[t + N1 * k2] = v[k2];
  }
  __syncthreads();
  col_store_spectrum<float>(L, 1, n, g, i0, n, 0, spec + b * bstride + f * fstride);
}

template <int N1, int N2>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_col_out_r(
    GridDev g, const float2* __restrict__ spec, size_t fstride, size_t bstride, int nout, const EpiArgs ea,
    const float2* __restrict__ roots) {
  typedef TeamFFT<N1, N2> TF;
  constexpr int n = N1 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* L = reinterpret_cast<float2*>(smem_raw);
  float2* xs = L + n;
  const int b = blockIdx.y + g.b0;
  if (inactive(g, b)) return;
  const int i0 = blockIdx.x * 2;
  const int ny = g.ny, t = threadIdx.x;
  for (int o = 0; o < nout; ++o) {
    col_gather_hermitian<float>(L, 1, n, g, i0, spec + b * bstride + o * fstride, fstride, 1, n);
    // the next output's half spectrum into L2 while this one is transformed
    if (o + 1 < nout) prefetch_spec_pairs(g, i0, 1, spec + b * bstride + (o + 1) * fstride);
    __syncthreads();
    float2 v[TF::NV];
    if (t < N1) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) v[k2] = L[t + N1 * k2];
    }
    TF::inv(v, xs, roots, t);
    if (t < N2) {
      float* out = reinterpret_cast<float*>(ea.outs[o]);
#pragma unroll
      for (int j = 0; j < N1; ++j) {
        const int row = t + N2 * j;
        if (row < ny) {
          out[fidx(g, b, i0, row)] = v[j].x;
          if (i0 + 1 < g.ncol) out[fidx(g, b, i0 + 1, row)] = v[j].y;
        }
      }
    }
  }
}

// Wall-normal passes of FP32 contexts whose extended length n has a large
// prime factor (n = 537 and 1049 with n_cont = 25 at 512 and 1024 nodes):
// Bluestein's convolution on the register team FFT of length m = 1080 =
// 30 x 36 or 2100 = 42 x 50 (bluestein_team), one column pair per CTA.  The
// chirp, the transformed filter and the m roots come from the context's plan
// (P.chirp, P.bhat, P.sub.tw) in the FP32 pool.
template <int N1, int N2>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_col_fwd_rb(
    GridDev g, const float* __restrict__ f0, const float* __restrict__ f1, const float* __restrict__ f2,
    const typename FcTab<float>::t* __restrict__ E, const float2* __restrict__ chirp,
    const float2* __restrict__ bhat, const float2* __restrict__ roots, float2* __restrict__ spec, size_t fstride,
    size_t bstride) {
  constexpr int m = N1 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* L = reinterpret_cast<float2*>(smem_raw);
  float2* xs = L + m;
  const int b = blockIdx.z + g.b0, f = blockIdx.y;
  if (inactive(g, b)) return;
  const int i0 = blockIdx.x * 2;
  const float* src = f == 0 ? f0 : (f == 1 ? f1 : f2);
  const int ny = g.ny, n = g.my, t = threadIdx.x;
  load_pair_f32(L, src + ((size_t)b * g.ncol + i0) * ny, i0 + 1 < g.ncol, ny);
  __syncthreads();
  fc_append<float>(L, 1, m, ny, g.n_cont, g.n_match, E);
  __syncthreads();
  bluestein_team<N1, N2, false>(L, xs, n, chirp, bhat, roots, t);
  col_store_spectrum<float>(L, 1, m, g, i0, n, 0, spec + b * bstride + f * fstride);
}

template <int N1, int N2>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_col_out_rb(
    GridDev g, const float2* __restrict__ spec, size_t fstride, size_t bstride, int nout, const EpiArgs ea,
    const float2* __restrict__ chirp, const float2* __restrict__ bhat, const float2* __restrict__ roots) {
  constexpr int m = N1 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* L = reinterpret_cast<float2*>(smem_raw);
  float2* xs = L + m;
  const int b = blockIdx.y + g.b0;
  if (inactive(g, b)) return;
  const int i0 = blockIdx.x * 2;
  const int ny = g.ny, n = g.my, t = threadIdx.x;
  for (int o = 0; o < nout; ++o) {
    col_gather_hermitian<float>(L, 1, m, g, i0, spec + b * bstride + o * fstride, fstride, 1, n);
    if (o + 1 < nout) prefetch_spec_pairs(g, i0, 1, spec + b * bstride + (o + 1) * fstride);
    __syncthreads();
    bluestein_team<N1, N2, true>(L, xs, n, chirp, bhat, roots, t);
    float* out = reinterpret_cast<float*>(ea.outs[o]);
    for (int j = t; j < ny; j += blockDim.x) {
      out[fidx(g, b, i0, j)] = L[j].x;
      if (i0 + 1 < g.ncol) out[fidx(g, b, i0 + 1, j)] = L[j].y;
    }
    __syncthreads();
  }
}

// line_op on the Bluestein team transform: the forward spectrum stays in L,
// each output is formed in W (symbol times spectrum over n) and inverted there.
template <int N1, int N2>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_line_op_rb(
    GridDev g, const float* __restrict__ f, long long ncols, const typename FcTab<float>::t* __restrict__ E,
    const float2* __restrict__ pool, const float2* __restrict__ chirp, const float2* __restrict__ bhat,
    const float2* __restrict__ roots, const __grid_constant__ LineOuts lo) {
  constexpr int m = N1 * N2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* L = reinterpret_cast<float2*>(smem_raw);
  float2* W = L + m;
  float2* xs = W + m;
  const long long c0 = (long long)blockIdx.x * 2;
  const int ny = g.ny, n = g.my, t = threadIdx.x;
  load_pair_f32(L, f + c0 * ny, c0 + 1 < ncols, ny);
  __syncthreads();
  fc_append<float>(L, 1, m, ny, g.n_cont, g.n_match, E);
  __syncthreads();
  bluestein_team<N1, N2, false>(L, xs, n, chirp, bhat, roots, t);
  const float hh = g.hh_f, cky = g.cky_f, tscale = g.inv_my_f;  // n = my
  for (int o = 0; o < lo.nout; ++o) {
    const int op = lo.op[o];
    for (int k = t; k < n; k += blockDim.x) {
      const int kappa = (2 * k <= n) ? k : k - n;
      const float ky = cky * (float)kappa;
      const float What = pool[g.ey_off + (kappa < 0 ? -kappa : kappa)].x * kernel_poly<float>(g.family, ky * ky * hh);
      const bool nyq = (n % 2 == 0) && (2 * k == n);
      float2 sy;
      if (op == SYM_W)
        sy = make_float2(What, 0.f);
      else if (op == SYM_DY)
        sy = make_float2(0.f, nyq ? 0.f : ky * What);
      else if (op == SYM_LAP)
        sy = make_float2(-(ky * ky) * What, 0.f);
      else
        sy = make_float2(0.f, 0.f);
      W[k] = cscale(cmul(sy, L[k]), tscale);
    }
    __syncthreads();
    bluestein_team<N1, N2, true>(W, xs, n, chirp, bhat, roots, t);
    float* out = reinterpret_cast<float*>(lo.out[o]);
    for (int j = t; j < ny; j += blockDim.x) {
      if (c0 < ncols) out[c0 * ny + j] = W[j].x;
      if (c0 + 1 < ncols) out[(c0 + 1) * ny + j] = W[j].y;
    }
    __syncthreads();
  }
}

// k_col_out_r (BS: k_col_out_rb) with TMA staging, persistent over (column pair, output) units:
// while one unit's inverse transform runs, the next unit's half-spectrum rows
// (the pair's two complex values of rows ky < hy, 16 bytes a row) arrive in
// a staging buffer by 2D tiled bulk copies (nbox boxes of rows_box rows) on
// one mbarrier, so the column pass no longer waits on its strided gather.
// The wait for a copy is bounded: on a timeout the CTA sets bit 1 of the
// status word, waits once more (bounded) for its copy in flight and returns.
template <int N1, int N2, bool BS>
__global__ void __launch_bounds__(TeamFFT<N1, N2>::THREADS, TeamFFT<N1, N2>::MIN_CTAS) k_col_out_rt(
    GridDev g, const __grid_constant__ CUtensorMap tmap, int rows_box, int nbox, int nfo, int nout,
    const EpiArgs ea, const float2* __restrict__ roots, int npairs, const float2* __restrict__ chirp,
    const float2* __restrict__ bhat) {
  typedef TeamFFT<N1, N2> TF;
  constexpr int m = N1 * N2;
  const int n = BS ? g.my : m;  // the line's length (BS: transformed by Bluestein on length m)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // bulk tensor copies land on 128-byte boundaries (the launch adds 128 bytes)
  float4* stage = reinterpret_cast<float4*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  float2* L = reinterpret_cast<float2*>(stage + (size_t)nbox * rows_box);
  float2* xs = L + m;
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_ok;
  const int t = threadIdx.x;
  const int ny = g.ny, hy = g.hy;
  const long long W = (long long)g.nb * npairs;
  const uint32_t bytes = (uint32_t)(nbox * rows_box * 16);
  auto pair_of = [&](long long k) { return (long long)blockIdx.x + (k / nout) * gridDim.x; };
  auto issue = [&](long long k) {  // thread 0: copies of unit k into the stage
    const long long w = pair_of(k);
    const int o = (int)(k % nout);
    const int b = g.b0 + (int)(w / npairs), i0 = (int)(w % npairs) * 2;
    const int row0 = (b * nfo + o) * g.rows;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar, bytes);
    for (int q = 0; q < nbox; ++q) tma_load_2d(stage + (size_t)q * rows_box, &tmap, 2 * i0, row0 + q * rows_box, &bar);
  };
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (pair_of(0) >= W) return;
  if (t == 0) issue(0);
  for (long long k = 0; pair_of(k) < W; ++k) {
    const long long w = pair_of(k);
    const int o = (int)(k % nout);
    const int b = g.b0 + (int)(w / npairs), i0 = (int)(w % npairs) * 2;
    const uint32_t par = (uint32_t)(k & 1);
    if (t == 0) s_ok = mbar_wait_bounded(&bar, par) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {
      if (t == 0) {
        atomicOr(ea.status, 2);
        mbar_wait_bounded(&bar, par);
      }
      return;
    }
    mbar_try_wait(&bar, par);  // every thread observes the completed phase
    // Hermitian unpack: Z_k = A_k + i B_k, Z_{n-k} = conj(A_k) + i conj(B_k)
    for (int kk = t; kk < hy; kk += blockDim.x) {
      const float4 r = stage[kk];
      if (kk == 0 || 2 * kk == n) {
        L[kk] = make_float2(r.x, r.z);
      } else {
        L[kk] = make_float2(r.x - r.w, r.y + r.z);
        L[n - kk] = make_float2(r.x + r.w, r.z - r.y);
      }
    }
    __syncthreads();
    if (t == 0 && pair_of(k + 1) < W) issue(k + 1);  // the stage is free again
    float* out = reinterpret_cast<float*>(ea.outs[o]);
    if constexpr (BS) {
      bluestein_team<N1, N2, true>(L, xs, n, chirp, bhat, roots, t);
      for (int j = t; j < ny; j += blockDim.x) {
        out[fidx(g, b, i0, j)] = L[j].x;
        if (i0 + 1 < g.ncol) out[fidx(g, b, i0 + 1, j)] = L[j].y;
      }
      __syncthreads();  // L is rewritten by the next unit
    } else {
      float2 v[TF::NV];
      if (t < N1) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) v[k2] = L[t + N1 * k2];
      }
      TF::inv(v, xs, roots, t);
      if (t < N2) {
#pragma unroll
        for (int j = 0; j < N1; ++j) {
          const int row = t + N2 * j;
          if (row < ny) {
            out[fidx(g, b, i0, row)] = v[j].x;
            if (i0 + 1 < g.ncol) out[fidx(g, b, i0 + 1, row)] = v[j].y;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// fc_extend (Eq. 30) as a standalone kernel: y continuation of every column,
// then x continuation of every extended row (walled x).
template <typename U>
__global__ void k_fc_extend_y(GridDev g, const U* __restrict__ f, U* __restrict__ fe, const double* __restrict__ E) {
  const size_t total = (size_t)g.batch * g.ncol * g.my;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % g.my);
    const size_t bi = t / g.my;
    const int i = (int)(bi % g.ncol);
    const int b = (int)(bi / g.ncol);
    const U* col = f + ((size_t)b * g.ncol + i) * g.ny;
    double v;
    if (j < g.ny) {
      v = (double)col[j];
    } else {
      const int c = j - g.ny, d = g.n_match;
      Dot2 acc;
      for (int m = 0; m < d; ++m) {
        acc.add(E[c * 2 * d + m], (double)col[g.ny - d + m]);
        acc.add(E[c * 2 * d + d + m], (double)col[m]);
      }
      v = acc.value();
    }
    fe[((size_t)b * (g.x_walls ? g.mx : g.ncol) + i) * g.my + j] = (U)v;
  }
}

template <typename U>
__global__ void k_fc_extend_x(GridDev g, U* __restrict__ fe, const double* __restrict__ E) {
  const int C = g.n_cont, d = g.n_match;
  const size_t total = (size_t)g.batch * C * g.my;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % g.my);
    const size_t bc = t / g.my;
    const int c = (int)(bc % C);
    const int b = (int)(bc / C);
    U* base = fe + (size_t)b * g.mx * g.my;
    Dot2 acc;
    for (int m = 0; m < d; ++m) {
      acc.add(E[c * 2 * d + m], (double)base[(size_t)(g.nx - d + m) * g.my + j]);
      acc.add(E[c * 2 * d + d + m], (double)base[(size_t)m * g.my + j]);
    }
    base[(size_t)(g.nx + c) * g.my + j] = (U)acc.value();
  }
}

// Batched DFT of contiguous lines (engine test entry); IO is the element type
// in memory (double2 for the double-float engine, else the engine's own).
template <typename T, bool INV, typename IO = typename CT<T>::t>
__global__ void __launch_bounds__(kThreads) k_dft_lines(int n, int nlines, const IO* __restrict__ in,
                                                        IO* __restrict__ out, const __grid_constant__ FftPlan P,
                                                        const typename CT<T>::t* __restrict__ pool, int L, int ls) {
  typedef typename CT<T>::t V;
  typedef decltype(IO().x) E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + (size_t)L * ls;
  const int l0 = blockIdx.x * L;
  for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
    const int r = e / n, j = e - (e / n) * n;
    if (l0 + r < nlines) {
      const IO x = in[(size_t)(l0 + r) * n + j];
      A[(size_t)r * ls + j] = mk<V>(x.x, x.y);
    } else {
      A[(size_t)r * ls + j] = mk<V>(0.0, 0.0);
    }
  }
  __syncthreads();
  V* Y = fft_any<T, INV>(A, B, L, ls, P, pool);
  for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
    const int r = e / n, j = e - (e / n) * n;
    if (l0 + r < nlines) {
      const V y = Y[(size_t)r * ls + j];
      out[(size_t)(l0 + r) * n + j] = mk<IO>(static_cast<E>(y.x), static_cast<E>(y.y));
    }
  }
}

// Residual diagnostics, one block per instance: out[0] += sum_b (r - mean_b(r))^2,
// out[1] += sum_b b^2 (two passes over the instance: mean, then deviations).
__global__ void k_resid_inst(const double* __restrict__ r, const double* __restrict__ b, size_t n_inst, double* out) {
  __shared__ double sh[2][kThreads];
  const double* ri = r + blockIdx.x * n_inst;
  const double* bi = b + blockIdx.x * n_inst;
  double s0 = 0.0;
  for (size_t t = threadIdx.x; t < n_inst; t += blockDim.x) s0 += ri[t];
  sh[0][threadIdx.x] = s0;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
    __syncthreads();
  }
  const double mean = sh[0][0] / (double)n_inst;
  __syncthreads();
  double d2 = 0.0, b2 = 0.0;
  for (size_t t = threadIdx.x; t < n_inst; t += blockDim.x) {
    const double d = ri[t] - mean;
    d2 += d * d;
    b2 += bi[t] * bi[t];
  }
  sh[0][threadIdx.x] = d2;
  sh[1][threadIdx.x] = b2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(out + 0, sh[0][0]);
    atomicAdd(out + 1, sh[1][0]);
  }
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, const float* __restrict__ xf, size_t n,
                       double a) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] += a * (x ? x[t] : (double)xf[t]);
}

__global__ void k_narrow(float* __restrict__ y, const double* __restrict__ x, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}

__global__ void k_sub(double* __restrict__ r, const double* __restrict__ b, const double* __restrict__ lb, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    r[t] = b[t] - lb[t];
}

// ---------------------------------------------------------------------------
// Host-side launch helpers.

// Largest count (>= 1, <= cap) of units fitting in `budget` bytes.
int fit_units(size_t per_unit, size_t budget, int cap) {
  int u = (int)(budget / per_unit);
  if (u < 1) u = 1;
  if (u > cap) u = cap;
  return u;
}

constexpr size_t kSmemBudget = 96 * 1024;  // per CTA of the multi-line engine test kernel
constexpr size_t kSmemMax = 227 * 1024;

// Every kernel's dynamic shared-memory limit is raised once, at the first
// context creation (init_kernel_attributes), so that no attribute call ever
// happens while a stream is being captured; launches only check the size.
cudaError_t check_smem(size_t bytes) {
  return bytes > kSmemMax ? cudaErrorInvalidValue : cudaSuccess;
}

template <typename K> cudaError_t raise_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
}

// FC table (bc) in the FcTab type of precision prec.
const void* fc_table(const fcsph_ctx* c, int prec, int bc) {
  const size_t off = (bc == FCSPH_NEUMANN ? 1 : 0) * (size_t)c->gd.n_cont * 2 * c->gd.n_match;
  if (prec == FCSPH_F32X2 || prec == FCSPH_F32) return static_cast<const ff*>(c->dEff) + off;
  return c->dE + off;
}

// Fields per instance of the spectrum buffers: spec_in holds the forward
// transforms of the velocity components (2D: 2, 3D: 3), spec_out the row
// pass outputs (2D: 6, 3D: 12).
size_t spec_in_fields(const fcsph_ctx* c) { return c->gd.nz > 1 ? 3 : 2; }
size_t spec_out_fields(const fcsph_ctx* c) { return c->gd.nz > 1 ? 12 : 6; }

int col_ls(const fcsph_ctx* c) {
  int ls = c->plan_y.line_len();
  if (c->plan_py.line_len() > ls) ls = c->plan_py.line_len();
  return ls;
}

}  // namespace

// ===========================================================================
// Launchers

// Recording (fcsph_ctx::rec set): a pass of isph_step is appended to the
// recording as a descriptor instead of being launched.  FP64 and FP32x2 only
// (the persistent kernel's types).
struct PersistRec {
  std::vector<PassDesc> descs;
};

template <typename T> cudaError_t rec_push(fcsph_ctx* c, PassDesc& d) {
  if (!std::is_same<T, double>::value && !std::is_same<T, ff>::value) return cudaErrorNotSupported;
  d.pool = PoolOf<T>::get(c);
  c->rec->descs.push_back(d);
  return cudaSuccess;
}

static PassDesc new_desc(const fcsph_ctx* c, int kind, dim3 grid, size_t smem) {
  PassDesc d;
  memset(&d, 0, sizeof(d));
  d.kind = kind;
  d.gx = (int)grid.x;
  d.gy = (int)grid.y;
  d.gz = (int)grid.z;
  d.smem = smem;
  d.g = c->gd;
  return d;
}

cudaError_t init_kernel_attributes() {
  cudaError_t e = cudaSuccess;
#define FCSPH_RAISE(K)                           \
  if ((e = raise_smem(K)) != cudaSuccess) return e;
  FCSPH_RAISE((k_dft_lines<double, false>))
  FCSPH_RAISE((k_dft_lines<double, true>))
  FCSPH_RAISE((k_dft_lines<float, false>))
  FCSPH_RAISE((k_dft_lines<float, true>))
  FCSPH_RAISE((k_dft_lines<ff, false, double2>))
  FCSPH_RAISE((k_dft_lines<ff, true, double2>))
  FCSPH_RAISE((k_line_op_r<20, 27>))
  FCSPH_RAISE((k_line_op_r<30, 35>))
  FCSPH_RAISE((k_col_fwd_r<20, 27>))
  FCSPH_RAISE((k_col_fwd_r<30, 35>))
  FCSPH_RAISE((k_col_out_r<20, 27>))
  FCSPH_RAISE((k_col_out_r<30, 35>))
  FCSPH_RAISE((k_col_fwd_rb<30, 36>))
  FCSPH_RAISE((k_col_fwd_rb<42, 50>))
  FCSPH_RAISE((k_col_out_rb<30, 36>))
  FCSPH_RAISE((k_col_out_rb<42, 50>))
  FCSPH_RAISE((k_line_op_rb<30, 36>))
  FCSPH_RAISE((k_line_op_rb<42, 50>))
  {
    const int lim = (int)kSmemMax - 64;
    if ((e = cudaFuncSetAttribute(k_col_out_rt<20, 27, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_col_out_rt<30, 35, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_col_out_rt<30, 36, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_col_out_rt<42, 50, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) !=
            cudaSuccess)
      return e;
  }
  FCSPH_RAISE((k_row_sym_w<2>))
  FCSPH_RAISE((k_row_sym_w<4>))
  FCSPH_RAISE((k_row_sym_w<8>))
  FCSPH_RAISE((k_row_sym_w<16>))
  FCSPH_RAISE((k_row_sym_w<32>))
  // the persistent kernel holds two static shared words besides its dynamic
  // shared memory
  for (int nt : {32, 64, 128}) {
    e = with_width(nt, [](auto w) {
      constexpr int NT = decltype(w)::value;
      const int lim = (int)kSmemMax - 64;
      cudaError_t r = cudaFuncSetAttribute(k_persist<double, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
      if (r != cudaSuccess) return r;
      return cudaFuncSetAttribute(k_persist<ff, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    });
    if (e != cudaSuccess) return e;
  }
  for (int nt : {32, 64, 128}) {
    e = with_width(nt, [](auto w) {
      constexpr int NT = decltype(w)::value;
      cudaError_t r = cudaSuccess;
      if ((r = raise_smem(k_col_fwd<double, double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_col_fwd<ff, double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_col_fwd<float, double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_col_fwd<float, float, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_line_op<double, double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_line_op<ff, double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_line_op<float, float, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_row_sym<double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_row_sym<ff, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_row_sym<float, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_row_ppe<double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_row_ppe<ff, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_row_ppe<float, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_col_inv<double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_col_inv<ff, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_col_inv<float, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_zlines<double, NT>)) != cudaSuccess) return r;
      if ((r = raise_smem(k_zlines<ff, NT>)) != cudaSuccess) return r;
      return raise_smem(k_zlines<float, NT>);
    });
    if (e != cudaSuccess) return e;
  }
#undef FCSPH_RAISE
  return cudaSuccess;
}

// Largest dynamic shared memory any FFT kernel of context c needs with
// row_lines rows per row-pass CTA and col_pairs column pairs per column CTA.
size_t tiling_smem(const fcsph_ctx* c, int row_lines, int col_pairs) {
  const size_t cb = c->prec.fft_prec == FCSPH_F32 ? sizeof(float2) : sizeof(double2);
  const size_t row = (c->gd.nz > 1 ? 6 : 4) * (size_t)row_lines * c->plan_x.line_len() * cb;
  const size_t ppe = 2 * (size_t)row_lines * c->plan_px.line_len() * cb;
  const size_t col = (size_t)col_pairs * 2 * (size_t)col_ls(c) * cb;
  size_t m = row > ppe ? row : ppe;
  return m > col ? m : col;
}

size_t tiling_smem_limit() { return kSmemMax; }

cudaError_t launch_fc_extend(fcsph_ctx* c, const void* f, void* fext, int bc) {
  ProfScope ps(c, FCSPH_PROF_OTHER);
  const double* E = c->dE + (bc == FCSPH_NEUMANN ? 1 : 0) * c->gd.n_cont * 2 * c->gd.n_match;
  const int blocks = 152 * 8;
  if (c->prec.fft_prec != FCSPH_F32) {  // double fields (F64, F32X2)
    k_fc_extend_y<double><<<blocks, kThreads, 0, c->stream>>>(c->gd, (const double*)f, (double*)fext, E);
    c->launches++;
    if (c->gd.x_walls) {
      k_fc_extend_x<double><<<blocks, kThreads, 0, c->stream>>>(c->gd, (double*)fext, E);
      c->launches++;
    }
  } else {
    k_fc_extend_y<float><<<blocks, kThreads, 0, c->stream>>>(c->gd, (const float*)f, (float*)fext, E);
    c->launches++;
    if (c->gd.x_walls) {
      k_fc_extend_x<float><<<blocks, kThreads, 0, c->stream>>>(c->gd, (float*)fext, E);
      c->launches++;
    }
  }
  return cudaGetLastError();
}


// Register column FFT for FP32 contexts: the split n = N1 N2 of the extended
// wall-normal length when the plan is direct and the length is one of the
// supported ones, else 0.
int col_r_split(const fcsph_ctx* c) {
  const FftPlan& P = c->plan_y;
  if (c->prec.fft_prec != FCSPH_F32 || P.bs || P.rd) return 0;
  switch (P.base.n) {
    case 540: return 20;
    case 1050: return 30;
    default: return 0;
  }
}

template <int N1, int N2>
static cudaError_t col_fwd_r(fcsph_ctx* c, int nf, const void* const* fields, int bc, void* spec) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  const size_t smem = ((size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const auto* E = static_cast<const typename FcTab<float>::t*>(fc_table(c, FCSPH_F32, bc));
  dim3 grid((g.ncol + 1) / 2, nf, g.nb);
  const size_t fstride = (size_t)g.rows * g.ncol;
  const size_t bstride = spec_in_fields(c) * fstride;
  ProfScope ps(c, FCSPH_PROF_COL_FWD);
  const float* f0 = (const float*)fields[0];
  k_col_fwd_r<N1, N2><<<grid, TF::THREADS, smem, c->stream>>>(
      g, f0, (const float*)(nf > 1 ? fields[1] : fields[0]), (const float*)(nf > 2 ? fields[2] : fields[0]), E,
      c->pool32 + c->plan_y.base.tw, (float2*)spec, fstride, bstride);
  c->launches++;
  return cudaGetLastError();
}

// Register Bluestein column FFT for FP32 contexts: the split N1 of the
// Bluestein length m (1080 = 30 x 36, 2100 = 42 x 50) of the extended
// wall-normal length, else 0.
int col_rb_split(const fcsph_ctx* c) {
  const FftPlan& P = c->plan_y;
  if (c->prec.fft_prec != FCSPH_F32 || !P.bs) return 0;
  switch (P.sub.n) {
    case 1080: return 30;
    case 2100: return 42;
    default: return 0;
  }
}

template <int N1, int N2>
static cudaError_t col_fwd_rb(fcsph_ctx* c, int nf, const void* const* fields, int bc, void* spec) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  const FftPlan& P = c->plan_y;
  const size_t smem = ((size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const auto* E = static_cast<const typename FcTab<float>::t*>(fc_table(c, FCSPH_F32, bc));
  dim3 grid((g.ncol + 1) / 2, nf, g.nb);
  const size_t fstride = (size_t)g.rows * g.ncol;
  const size_t bstride = spec_in_fields(c) * fstride;
  ProfScope ps(c, FCSPH_PROF_COL_FWD);
  const float* f0 = (const float*)fields[0];
  k_col_fwd_rb<N1, N2><<<grid, TF::THREADS, smem, c->stream>>>(
      g, f0, (const float*)(nf > 1 ? fields[1] : fields[0]), (const float*)(nf > 2 ? fields[2] : fields[0]), E,
      c->pool32 + P.chirp, c->pool32 + P.bhat, c->pool32 + P.sub.tw, (float2*)spec, fstride, bstride);
  c->launches++;
  return cudaGetLastError();
}

template <int N1, int N2>
static cudaError_t col_out_rb(fcsph_ctx* c, const void* spec, int nout, EpiArgs& ea) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  const FftPlan& P = c->plan_y;
  const size_t smem = ((size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const size_t fs = (size_t)g.rows * g.ncol;
  dim3 grid((g.ncol + 1) / 2, g.nb);
  ProfScope ps(c, FCSPH_PROF_COL_OUT);
  k_col_out_rb<N1, N2><<<grid, TF::THREADS, smem, c->stream>>>(g, (const float2*)spec, fs, spec_out_fields(c) * fs,
                                                              nout, ea, c->pool32 + P.chirp, c->pool32 + P.bhat,
                                                              c->pool32 + P.sub.tw);
  c->launches++;
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// The TMA column-output pass: needs an even number of columns (16-byte rows
// of the tensor map and 16-byte aligned pair coordinates), a 16-byte aligned
// spectrum buffer and no instance mask; returns cudaErrorNotSupported
// otherwise (the caller then runs k_col_out_r).
template <int N1, int N2, bool BS>
static cudaError_t col_out_rt(fcsph_ctx* c, const void* spec, int nout, EpiArgs& ea) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  EncodeTiledFn enc = encode_tiled();
  if (!enc || g.ncol % 2 || ((uintptr_t)spec & 15) || g.active) return cudaErrorNotSupported;
  const int nfo = spec_out_fields(c);
  const int nbox = (g.hy + 255) / 256;
  const int rows_box = ((g.hy + nbox - 1) / nbox + 7) / 8 * 8;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * g.ncol, (cuuint64_t)g.batch * nfo * g.rows};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * g.ncol * sizeof(float)};
  const cuuint32_t box[2] = {4, (cuuint32_t)rows_box};
  const cuuint32_t es[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(spec), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorNotSupported;
  const size_t smem = 128 + (size_t)nbox * rows_box * 16 + ((size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem + 64);
  if (e != cudaSuccess) return cudaErrorNotSupported;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_col_out_rt<N1, N2, BS>, TF::THREADS, smem)) !=
          cudaSuccess)
    return e;
  const int npairs = (g.ncol + 1) / 2;
  const long long W = (long long)g.nb * npairs;
  const long long grid = std::min<long long>(W, (long long)sms * (occ > 0 ? occ : 1));
  ea.status = c->dstatus;
  ProfScope ps(c, FCSPH_PROF_COL_OUT);
  const FftPlan& P = c->plan_y;
  const float2* roots = c->pool32 + (BS ? P.sub.tw : P.base.tw);
  k_col_out_rt<N1, N2, BS><<<(unsigned)grid, TF::THREADS, smem, c->stream>>>(
      g, map, rows_box, nbox, nfo, nout, ea, roots, npairs, BS ? c->pool32 + P.chirp : nullptr,
      BS ? c->pool32 + P.bhat : nullptr);
  c->launches++;
  return cudaGetLastError();
}

template <int N1, int N2>
static cudaError_t col_out_r(fcsph_ctx* c, const void* spec, int nout, EpiArgs& ea) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  const size_t smem = ((size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const size_t fs = (size_t)g.rows * g.ncol;
  dim3 grid((g.ncol + 1) / 2, g.nb);
  ProfScope ps(c, FCSPH_PROF_COL_OUT);
  k_col_out_r<N1, N2><<<grid, TF::THREADS, smem, c->stream>>>(g, (const float2*)spec, fs, spec_out_fields(c) * fs,
                                                             nout, ea, c->pool32 + c->plan_y.base.tw);
  c->launches++;
  return cudaGetLastError();
}

template <typename T, typename U>
static cudaError_t col_fwd_t(fcsph_ctx* c, int prec, int nf, const void* const* fields, int bc, void* spec, int dct) {
  const GridDev& g = c->gd;
  if constexpr (sizeof(T) == sizeof(float) && sizeof(U) == sizeof(float)) {
    if (!dct) {
      switch (col_r_split(c)) {
        case 20: return col_fwd_r<20, 27>(c, nf, fields, bc, spec);
        case 30: return col_fwd_r<30, 35>(c, nf, fields, bc, spec);
        default: break;
      }
      switch (col_rb_split(c)) {
        case 30: return col_fwd_rb<30, 36>(c, nf, fields, bc, spec);
        case 42: return col_fwd_rb<42, 50>(c, nf, fields, bc, spec);
        default: break;
      }
    }
  }
  const FftPlan& P = dct ? c->plan_py : c->plan_y;
  const int ls = P.line_len();
  const int Pp = c->col_pairs;
  const size_t smem = 2 * (size_t)ls * sizeof(typename CT<T>::t) * Pp;
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const auto* E = static_cast<const typename FcTab<T>::t*>(fc_table(c, prec, bc));
  dim3 grid((g.ncol + 2 * Pp - 1) / (2 * Pp), nf, g.nb);
  const size_t fstride = (size_t)g.rows * g.ncol;
  const size_t bstride = (dct ? 1 : spec_in_fields(c)) * fstride;
  if (c->rec) {
    if (!std::is_same<U, double>::value) return cudaErrorNotSupported;
    PassDesc d = new_desc(c, PK_COL_FWD, grid, smem);
    d.Pp = Pp;
    d.ls = ls;
    d.P = P;
    d.E = E;
    for (int k = 0; k < 3; ++k) d.f[k] = fields[k < nf ? k : 0];
    d.dct = dct;
    d.spec = spec;
    d.fstride = fstride;
    d.bstride = bstride;
    return rec_push<T>(c, d);
  }
  ProfScope ps(c, FCSPH_PROF_COL_FWD);
  return with_width(c->col_threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    k_col_fwd<T, U, NT><<<grid, NT, smem, c->stream>>>(g, (const U*)fields[0],
                                                       (const U*)(nf > 1 ? fields[1] : fields[0]),
                                                       (const U*)(nf > 2 ? fields[2] : fields[0]), E, P,
                                                       PoolOf<T>::get(c), dct, (typename CT<T>::t*)spec, fstride,
                                                       bstride, Pp, ls);
    c->launches++;
    return cudaGetLastError();
  });
}

cudaError_t launch_col_fwd(fcsph_ctx* c, int prec, int nf, const void* const* fields, int fields_double, int bc,
                           void* spec, int dct) {
  if (prec == FCSPH_F64) {
    if (!fields_double) return cudaErrorInvalidValue;
    return col_fwd_t<double, double>(c, prec, nf, fields, bc, spec, dct);
  }
  if (prec == FCSPH_F32X2) {
    if (!fields_double) return cudaErrorInvalidValue;
    return col_fwd_t<ff, double>(c, prec, nf, fields, bc, spec, dct);
  }
  if (fields_double) return col_fwd_t<float, double>(c, prec, nf, fields, bc, spec, dct);
  return col_fwd_t<float, float>(c, prec, nf, fields, bc, spec, dct);
}

// Shared memory of k_row_sym_w: per warp the exchange block and nin spectra.
size_t row_w_smem(int nin) { return 4 * ((size_t)kWarpXchgFloats + (size_t)nin * 2 * 32 * 32) * sizeof(float); }

// M = mx / 32 when the FP32 row pass can take the register FFT (periodic x,
// direct plan, mx = 32 M with M a power of two in 2 .. 32), else 0.
int row_w_m(const fcsph_ctx* c) {
  const GridDev& g = c->gd;
  if (c->prec.fft_prec != FCSPH_F32 || g.x_walls || g.mx != g.nx || c->plan_x.bs || c->plan_x.rd) return 0;
  for (int m = 2; m <= 32; m *= 2)
    if (g.mx == 32 * m) return m;
  return 0;
}

template <int M>
static cudaError_t row_sym_w(fcsph_ctx* c, const void* sp_in, void* sp_out, const RowOps& ops, double scale, int kind) {
  const GridDev& g = c->gd;
  const size_t smem = row_w_smem(ops.nin);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  constexpr int rows_per_cta = 4 * (32 / M);
  dim3 grid((g.hy * g.nz + rows_per_cta - 1) / rows_per_cta, g.nb);
  const size_t fs = (size_t)g.rows * g.ncol;
  ProfScope ps(c, kind);
  k_row_sym_w<M><<<grid, 128, smem, c->stream>>>(g, (const float2*)sp_in, (float2*)sp_out, fs, spec_in_fields(c) * fs,
                                                 fs, spec_out_fields(c) * fs, ops, c->pool32 + c->plan_x.base.tw,
                                                 static_cast<const float*>(c->dW), scale);
  c->launches++;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t row_sym_t(fcsph_ctx* c, int prec, const void* sp_in, void* sp_out, const RowOps& ops, double scale,
                             int bc, int kind) {
  const GridDev& g = c->gd;
  if (prec == FCSPH_F32) {
    switch (row_w_m(c)) {
      case 2: return row_sym_w<2>(c, sp_in, sp_out, ops, scale, kind);
      case 4: return row_sym_w<4>(c, sp_in, sp_out, ops, scale, kind);
      case 8: return row_sym_w<8>(c, sp_in, sp_out, ops, scale, kind);
      case 16: return row_sym_w<16>(c, sp_in, sp_out, ops, scale, kind);
      case 32: return row_sym_w<32>(c, sp_in, sp_out, ops, scale, kind);
      default: break;
    }
  }
  const int ls = c->plan_x.line_len();
  const int Rr = c->row_lines;
  const int nlines = 2 * ops.nin + (ops.nin == 1 ? 1 : 0);
  const size_t smem = (size_t)nlines * Rr * ls * sizeof(typename CT<T>::t);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const auto* E = static_cast<const typename FcTab<T>::t*>(fc_table(c, prec, bc));
  const size_t fs = (size_t)g.rows * g.ncol;
  dim3 grid((g.hy * g.nz + Rr - 1) / Rr, g.nb);
  if (c->rec) {
    PassDesc d = new_desc(c, PK_ROW_SYM, grid, smem);
    d.Rr = Rr;
    d.ls = ls;
    d.P = c->plan_x;
    d.E = E;
    d.sp_in = sp_in;
    d.sp_out = sp_out;
    d.fs_in = fs;
    d.bs_in = spec_in_fields(c) * fs;
    d.fs_out = fs;
    d.bs_out = spec_out_fields(c) * fs;
    d.ops = ops;
    d.W = c->dW;
    d.scale = scale;
    return rec_push<T>(c, d);
  }
  ProfScope ps(c, kind);
  return with_width(c->row_threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    k_row_sym<T, NT><<<grid, NT, smem, c->stream>>>(g, (const typename CT<T>::t*)sp_in, (typename CT<T>::t*)sp_out,
                                                    fs, spec_in_fields(c) * fs, fs, spec_out_fields(c) * fs, ops, E,
                                                    c->plan_x, PoolOf<T>::get(c), static_cast<const T*>(c->dW),
                                                    scale, Rr, ls);
    c->launches++;
    return cudaGetLastError();
  });
}

// One launch for any number of outputs: the outputs are formed and inverted
// one at a time, so shared memory does not grow with them.
cudaError_t launch_row_sym(fcsph_ctx* c, int prec, const void* sp_in, void* sp_out, const RowOps& ops, double scale,
                           int bc, int kind) {
  if (prec == FCSPH_F64) return row_sym_t<double>(c, prec, sp_in, sp_out, ops, scale, bc, kind);
  if (prec == FCSPH_F32X2) return row_sym_t<ff>(c, prec, sp_in, sp_out, ops, scale, bc, kind);
  return row_sym_t<float>(c, prec, sp_in, sp_out, ops, scale, bc, kind);
}

template <int N1, int N2>
static cudaError_t line_op_r(fcsph_ctx* c, const void* f, const LineOuts& lo, int bc) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  const size_t smem = ((size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const long long ncols = (long long)g.batch * g.ncol;
  const auto* E = static_cast<const typename FcTab<float>::t*>(fc_table(c, FCSPH_F32, bc));
  ProfScope ps(c, FCSPH_PROF_COL_OUT);
  k_line_op_r<N1, N2><<<(unsigned)((ncols + 1) / 2), TF::THREADS, smem, c->stream>>>(
      g, (const float*)f, ncols, E, c->pool32, c->pool32 + c->plan_y.base.tw, lo);
  c->launches++;
  return cudaGetLastError();
}

template <int N1, int N2>
static cudaError_t line_op_rb(fcsph_ctx* c, const void* f, const LineOuts& lo, int bc) {
  typedef TeamFFT<N1, N2> TF;
  const GridDev& g = c->gd;
  const FftPlan& P = c->plan_y;
  const size_t smem = (2 * (size_t)N1 * N2 + TF::XCHG) * sizeof(float2);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const long long ncols = (long long)g.batch * g.ncol;
  const auto* E = static_cast<const typename FcTab<float>::t*>(fc_table(c, FCSPH_F32, bc));
  ProfScope ps(c, FCSPH_PROF_COL_OUT);
  k_line_op_rb<N1, N2><<<(unsigned)((ncols + 1) / 2), TF::THREADS, smem, c->stream>>>(
      g, (const float*)f, ncols, E, c->pool32, c->pool32 + P.chirp, c->pool32 + P.bhat, c->pool32 + P.sub.tw, lo);
  c->launches++;
  return cudaGetLastError();
}

template <typename T, typename U>
static cudaError_t line_op_t(fcsph_ctx* c, int prec, const void* f, const int* ops, int nout, int bc, void* const* outs) {
  const GridDev& g = c->gd;
  if constexpr (sizeof(T) == sizeof(float) && sizeof(U) == sizeof(float)) {
    const int split = col_r_split(c);
    if (split) {
      LineOuts lo;
      memset(&lo, 0, sizeof(lo));
      lo.nout = nout;
      for (int o = 0; o < nout; ++o) {
        lo.op[o] = ops[o];
        lo.out[o] = outs[o];
      }
      if (split == 20) return line_op_r<20, 27>(c, f, lo, bc);
      if (split == 30) return line_op_r<30, 35>(c, f, lo, bc);
    }
    const int bsplit = col_rb_split(c);
    if (bsplit) {
      LineOuts lo;
      memset(&lo, 0, sizeof(lo));
      lo.nout = nout;
      for (int o = 0; o < nout; ++o) {
        lo.op[o] = ops[o];
        lo.out[o] = outs[o];
      }
      if (bsplit == 30) return line_op_rb<30, 36>(c, f, lo, bc);
      if (bsplit == 42) return line_op_rb<42, 50>(c, f, lo, bc);
    }
  }
  const FftPlan& P = c->plan_y;
  const int ls = P.line_len();
  const int Pp = c->col_pairs;
  const size_t smem = 3 * (size_t)Pp * ls * sizeof(typename CT<T>::t);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  LineOuts lo;
  memset(&lo, 0, sizeof(lo));
  lo.nout = nout;
  for (int o = 0; o < nout; ++o) {
    lo.op[o] = ops[o];
    lo.out[o] = outs[o];
  }
  const long long ncols = (long long)g.batch * g.ncol;
  const long long blocks = (ncols + 2 * Pp - 1) / (2 * Pp);
  const auto* E = static_cast<const typename FcTab<T>::t*>(fc_table(c, prec, bc));
  ProfScope ps(c, FCSPH_PROF_COL_OUT);
  return with_width(c->col_threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    k_line_op<T, U, NT><<<(unsigned)blocks, NT, smem, c->stream>>>(g, (const U*)f, ncols, E, P, PoolOf<T>::get(c),
                                                                   lo, Pp, ls);
    c->launches++;
    return cudaGetLastError();
  });
}

cudaError_t launch_line_op(fcsph_ctx* c, const void* f, const int* ops, int nout, int bc, void* const* outs) {
  const int prec = c->prec.fft_prec;
  if (prec == FCSPH_F64) return line_op_t<double, double>(c, prec, f, ops, nout, bc, outs);
  if (prec == FCSPH_F32X2) return line_op_t<ff, double>(c, prec, f, ops, nout, bc, outs);
  return line_op_t<float, float>(c, prec, f, ops, nout, bc, outs);
}

template <typename T>
static cudaError_t zpass_t(fcsph_ctx* c, void* spec, int nf, size_t bstride, int rows_used, int inv) {
  const GridDev& g = c->gd;
  const FftPlan& P = c->plan_z;
  const int ls = P.line_len();
  int L = 256 / g.nz;
  if (L < 1) L = 1;
  if (L > 8) L = 8;
  const size_t smem = 2 * (size_t)L * ls * sizeof(typename CT<T>::t);
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  const int lines = rows_used * g.nx;
  dim3 grid((lines + L - 1) / L, nf, g.nb);
  ProfScope ps(c, FCSPH_PROF_OTHER);
  return with_width(c->row_threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    k_zlines<T, NT><<<grid, NT, smem, c->stream>>>((typename CT<T>::t*)spec, lines, (size_t)g.rows * g.ncol, bstride,
                                                   P, PoolOf<T>::get(c), L, ls, inv, g.active, g.b0);
    c->launches++;
    return cudaGetLastError();
  });
}

// 3D: z transforms of nf fields of every instance (fields 0..nf-1 of the
// buffer, instance stride bstride, rows_used spectrum rows each); no-op in 2D.
cudaError_t launch_zpass(fcsph_ctx* c, int prec, void* spec, int nf, size_t bstride, int rows_used, int inv) {
  if (c->gd.nz <= 1 || nf <= 0) return cudaSuccess;
  if (prec == FCSPH_F64) return zpass_t<double>(c, spec, nf, bstride, rows_used, inv);
  if (prec == FCSPH_F32X2) return zpass_t<ff>(c, spec, nf, bstride, rows_used, inv);
  return zpass_t<float>(c, spec, nf, bstride, rows_used, inv);
}

template <typename T>
static cudaError_t col_inv_common(fcsph_ctx* c, int epi, const void* spec, int nout, EpiArgs& ea) {
  const GridDev& g = c->gd;
  const FftPlan& P = epi >= EPI_PPE_SOLVE ? c->plan_py : c->plan_y;
  // lines sized for the inverse plan and the fused forward's plan
  int ls = P.line_len();
  if (ea.fwd_nf > 0 && ea.fwdP.line_len() > ls) ls = ea.fwdP.line_len();
  const int Pp = c->col_pairs;
  // the lines only: FP64 values kept across outputs stay in global memory
  const size_t smem = (size_t)2 * ls * sizeof(typename CT<T>::t) * Pp;
  const size_t fs = (size_t)g.rows * g.ncol;
  const size_t bs = (epi >= EPI_PPE_SOLVE ? 1 : spec_out_fields(c)) * fs;  // spec_ppe or spec_out
  dim3 grid((g.ncol + 2 * Pp - 1) / (2 * Pp), g.nb);
  const typename CT<T>::t* pool = PoolOf<T>::get(c);
  if (epi < EPI_OUT || epi > EPI_PPE_ADD) return cudaErrorInvalidValue;
  if (ea.fwd_nf > 3 || (epi == EPI_MOM && nout != ea.fwd_nf * ea.mom_terms)) return cudaErrorInvalidValue;
  // the fused forward of a PPE pass reads the FP64 potential
  if (ea.fwd_nf > 0 && (epi == EPI_PPE_SOLVE || epi == EPI_PPE_ADD) && ea.phi == nullptr) return cudaErrorInvalidValue;
  if (ea.fwd_nf > 0 && (epi == EPI_OUT || epi == EPI_PPE_RESID)) return cudaErrorInvalidValue;
  ea.status = c->dstatus;
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  if (c->rec) {
    PassDesc d = new_desc(c, PK_COL_INV, grid, smem);
    d.Pp = Pp;
    d.ls = ls;
    d.P = P;
    d.spec = const_cast<void*>(spec);
    d.fstride = fs;
    d.bstride = bs;
    d.nout = nout;
    d.epi = epi;
    d.ea = ea;
    return rec_push<T>(c, d);
  }
  static const int kinds[7] = {FCSPH_PROF_COL_OUT, FCSPH_PROF_COL_MOM, FCSPH_PROF_COL_DIV, FCSPH_PROF_COL_CORR,
                               FCSPH_PROF_COL_PPE, FCSPH_PROF_COL_PPE, FCSPH_PROF_COL_PPE};
  ProfScope ps(c, kinds[epi]);
  return with_width(c->col_threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    k_col_inv<T, NT><<<grid, NT, smem, c->stream>>>(g, (const typename CT<T>::t*)spec, fs, bs, nout, P, pool,
                                                    ea, Pp, ls, epi);
    c->launches++;
    return cudaGetLastError();
  });
}

static cudaError_t col_inv(fcsph_ctx* c, int prec, int epi, const void* spec, int nout, EpiArgs& ea) {
  if (prec == FCSPH_F64) return col_inv_common<double>(c, epi, spec, nout, ea);
  if (prec == FCSPH_F32X2) return col_inv_common<ff>(c, epi, spec, nout, ea);
  return col_inv_common<float>(c, epi, spec, nout, ea);
}

static EpiArgs epi_defaults() {
  EpiArgs ea;
  memset(&ea, 0, sizeof(ea));
  return ea;
}

cudaError_t launch_col_out(fcsph_ctx* c, const void* spec, int nout, void* const* outs) {
  EpiArgs ea = epi_defaults();
  for (int o = 0; o < nout; ++o) ea.outs[o] = outs[o];
  ea.out_double = c->prec.fft_prec != FCSPH_F32;
  if (!ea.out_double) {
    cudaError_t e = cudaErrorNotSupported;
    switch (col_r_split(c)) {
      case 20:
        if (c->tma) e = col_out_rt<20, 27, false>(c, spec, nout, ea);
        return e == cudaErrorNotSupported ? col_out_r<20, 27>(c, spec, nout, ea) : e;
      case 30:
        if (c->tma) e = col_out_rt<30, 35, false>(c, spec, nout, ea);
        return e == cudaErrorNotSupported ? col_out_r<30, 35>(c, spec, nout, ea) : e;
      default: break;
    }
    switch (col_rb_split(c)) {
      case 30:
        if (c->tma) e = col_out_rt<30, 36, true>(c, spec, nout, ea);
        return e == cudaErrorNotSupported ? col_out_rb<30, 36>(c, spec, nout, ea) : e;
      case 42:
        if (c->tma) e = col_out_rt<42, 50, true>(c, spec, nout, ea);
        return e == cudaErrorNotSupported ? col_out_rb<42, 50>(c, spec, nout, ea) : e;
      default: break;
    }
  }
  return col_inv(c, c->prec.fft_prec, EPI_OUT, spec, nout, ea);
}

template <typename T>
static cudaError_t row_ppe_t(fcsph_ctx* c, void* spec, int apply) {
  const GridDev& g = c->gd;
  const int ls = c->plan_px.line_len();
  const int Rr = c->row_lines;
  const size_t smem = 2 * (size_t)ls * sizeof(typename CT<T>::t) * Rr;
  cudaError_t e = check_smem(smem);
  if (e != cudaSuccess) return e;
  dim3 grid((g.ny * g.nz + Rr - 1) / Rr, g.nb);
  if (c->rec) {
    PassDesc d = new_desc(c, PK_ROW_PPE, grid, smem);
    d.Rr = Rr;
    d.ls = ls;
    d.P = c->plan_px;
    d.spec = spec;
    d.bstride = (size_t)g.rows * g.ncol;
    d.apply = apply;
    return rec_push<T>(c, d);
  }
  ProfScope ps(c, FCSPH_PROF_ROW_PPE);
  return with_width(c->row_threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    k_row_ppe<T, NT><<<grid, NT, smem, c->stream>>>(g, (typename CT<T>::t*)spec, (size_t)g.rows * g.ncol, c->plan_px,
                                                    PoolOf<T>::get(c), apply, Rr, ls);
    c->launches++;
    return cudaGetLastError();
  });
}

cudaError_t launch_row_ppe(fcsph_ctx* c, int prec, void* spec, int apply) {
  if (prec == FCSPH_F64) return row_ppe_t<double>(c, spec, apply);
  if (prec == FCSPH_F32X2) return row_ppe_t<ff>(c, spec, apply);
  return row_ppe_t<float>(c, spec, apply);
}

// mode: 0 solve (phi out, optional Neumann-FC forward), 1 residual r = rhs - L phi into `phi`
// (double), 2 accumulate phi += value (double).
cudaError_t launch_col_ppe_inv(fcsph_ctx* c, int prec, const void* spec, void* phi, int phi_double, double* phi64,
                               int mode, const double* rhs, int neumann_fwd, void* spec_fwd) {
  EpiArgs ea = epi_defaults();
  int epi = EPI_PPE_SOLVE;
  if (mode == 0) {
    ea.phi_any = phi;
    ea.phi_double = phi_double;
    ea.phi = phi64;
  } else if (mode == 1) {
    epi = EPI_PPE_RESID;
    ea.phi = (double*)phi;
    ea.bvec = (double*)rhs;
  } else {
    epi = EPI_PPE_ADD;
    ea.phi = (double*)phi;
  }
  if (neumann_fwd) {
    ea.fwd_nf = 1;
    ea.fwd_dct = 0;
    ea.fwdE = fc_table(c, prec, FCSPH_NEUMANN);
    ea.fwdP = c->plan_y;
    ea.fwd_spec = spec_fwd;
    ea.fwd_fstride = (size_t)c->gd.rows * c->gd.ncol;
    ea.fwd_bstride = spec_in_fields(c) * ea.fwd_fstride;
  }
  return col_inv(c, prec, epi, spec, 1, ea);
}

cudaError_t launch_step_mom(fcsph_ctx* c, const StepDev& s, const void* spec_mom, const double* const* vel,
                            double* const* Fp, double* const* vs, void* spec_next) {
  const int nc = c->gd.nz > 1 ? 3 : 2;
  EpiArgs ea = epi_defaults();
  for (int q = 0; q < nc; ++q) {
    ea.vel[q] = vel[q];
    ea.Fp[q] = Fp[q];
    ea.vs[q] = vs[q];
  }
  ea.mom_terms = nc + 1;
  ea.s = s;
  ea.fwd_nf = nc;
  ea.fwd_dct = 0;
  ea.fwdE = fc_table(c, c->prec.fft_prec, FCSPH_DIRICHLET);
  ea.fwdP = c->plan_y;
  ea.fwd_spec = spec_next;
  ea.fwd_fstride = (size_t)c->gd.rows * c->gd.ncol;
  ea.fwd_bstride = nc * ea.fwd_fstride;
  return col_inv(c, c->prec.fft_prec, EPI_MOM, spec_mom, nc * (nc + 1), ea);
}

cudaError_t launch_step_div(fcsph_ctx* c, const StepDev& s, const void* spec1, double* b, void* spec_dct) {
  EpiArgs ea = epi_defaults();
  ea.bvec = b;
  ea.s = s;
  ea.fwd_nf = 1;
  ea.fwd_dct = 1;
  ea.fwdE = fc_table(c, c->prec.fft_prec, FCSPH_DIRICHLET);
  ea.fwdP = c->plan_py;
  ea.fwd_spec = spec_dct;
  ea.fwd_fstride = (size_t)c->gd.rows * c->gd.ncol;
  ea.fwd_bstride = ea.fwd_fstride;
  return col_inv(c, c->prec.fft_prec, EPI_DIV, spec1, 1, ea);
}

cudaError_t launch_step_corr(fcsph_ctx* c, const StepDev& s, const void* spec_grad, double* const* vs,
                             double* const* vo, void* spec_next) {
  const int nc = c->gd.nz > 1 ? 3 : 2;
  EpiArgs ea = epi_defaults();
  for (int q = 0; q < nc; ++q) {
    ea.vs[q] = vs[q];
    ea.vo[q] = vo[q];
  }
  ea.s = s;
  if (spec_next) {
    ea.fwd_nf = nc;
    ea.fwd_dct = 0;
    ea.fwdE = fc_table(c, c->prec.fft_prec, FCSPH_DIRICHLET);
    ea.fwdP = c->plan_y;
    ea.fwd_spec = spec_next;
    ea.fwd_fstride = (size_t)c->gd.rows * c->gd.ncol;
    ea.fwd_bstride = nc * ea.fwd_fstride;
  }
  return col_inv(c, c->prec.fft_prec, EPI_CORR, spec_grad, nc, ea);
}

template <typename T, typename IO>
cudaError_t dft_lines_t(int n, int nlines, int dir, const void* in, void* out, cudaStream_t st, const FftPlan& plan,
                        const void* pool) {
  typedef typename CT<T>::t V;
  const int ls = plan.line_len();
  const size_t per = 2 * (size_t)ls * sizeof(V);
  const int L = fit_units(per, kSmemBudget, 16);
  const size_t smem = per * L;
  const int blocks = (nlines + L - 1) / L;
  cudaError_t e;
  if (dir < 0) {
    if ((e = check_smem(smem)) != cudaSuccess) return e;
    k_dft_lines<T, false, IO><<<blocks, kThreads, smem, st>>>(n, nlines, (const IO*)in, (IO*)out, plan,
                                                              (const V*)pool, L, ls);
  } else {
    if ((e = check_smem(smem)) != cudaSuccess) return e;
    k_dft_lines<T, true, IO><<<blocks, kThreads, smem, st>>>(n, nlines, (const IO*)in, (IO*)out, plan,
                                                             (const V*)pool, L, ls);
  }
  return cudaGetLastError();
}

size_t dft_lines_smem(int prec, const FftPlan& plan) {
  const size_t cb = prec == FCSPH_F32 ? sizeof(CT<float>::t) : prec == FCSPH_F32X2 ? sizeof(CT<ff>::t)
                                                                                 : sizeof(CT<double>::t);
  const size_t per = 2 * (size_t)plan.line_len() * cb;
  return per * fit_units(per, kSmemBudget, 16);
}

size_t dft_smem_max() { return kSmemMax; }

cudaError_t launch_dft_lines(int n, int nlines, int dir, int prec, const void* in, void* out, cudaStream_t st,
                             const FftPlan& plan, const void* pool) {
  if (prec == FCSPH_F64) return dft_lines_t<double, double2>(n, nlines, dir, in, out, st, plan, pool);
  if (prec == FCSPH_F32X2) return dft_lines_t<ff, double2>(n, nlines, dir, in, out, st, plan, pool);
  return dft_lines_t<float, float2>(n, nlines, dir, in, out, st, plan, pool);
}

cudaError_t launch_resid_norm(fcsph_ctx* c, const double* r, const double* b, double* out2) {
  cudaMemsetAsync(out2, 0, 2 * sizeof(double), c->stream);
  ProfScope ps(c, FCSPH_PROF_OTHER);
  k_resid_inst<<<c->gd.batch, kThreads, 0, c->stream>>>(r, b, (size_t)c->gd.ncol * c->gd.ny, out2);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_axpy(fcsph_ctx* c, double* y, const double* x, const float* xf, int n, double a) {
  ProfScope ps(c, FCSPH_PROF_OTHER);
  k_axpy<<<152 * 4, kThreads, 0, c->stream>>>(y, x, xf, (size_t)n, a);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_sub(fcsph_ctx* c, double* r, const double* b, const double* lb, int n) {
  ProfScope ps(c, FCSPH_PROF_OTHER);
  k_sub<<<152 * 4, kThreads, 0, c->stream>>>(r, b, lb, (size_t)n);
  c->launches++;
  return cudaGetLastError();
}

cudaError_t launch_narrow(fcsph_ctx* c, float* y, const double* x, int n) {
  ProfScope ps(c, FCSPH_PROF_OTHER);
  k_narrow<<<152 * 4, kThreads, 0, c->stream>>>(y, x, (size_t)n);
  c->launches++;
  return cudaGetLastError();
}

// ===========================================================================
// Persistent multi-class step (see k_persist)

struct PersistPlan {
  int prec = FCSPH_F32X2;
  std::vector<PersistRec*> recs;     // one recording per class
  std::vector<int> inst;             // instances per class
  PassDesc* d_descs = nullptr;
  WorkItem* d_items = nullptr;
  unsigned* d_counters = nullptr;    // counters, then the item dispenser
  int* d_status = nullptr;
  int n_items = 0, n_counters = 0, grid = 0, threads = 32;
  size_t smem = 0;
  cudaGraphExec_t gexec = nullptr;
  long long graph_wait_ns = -1;
};

PersistPlan* persist_create(int prec) {
  PersistPlan* p = new PersistPlan();
  p->prec = prec;
  return p;
}

void persist_destroy(PersistPlan* p) {
  if (!p) return;
  for (PersistRec* r : p->recs) delete r;
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  cudaFree(p->d_descs);
  cudaFree(p->d_items);
  cudaFree(p->d_counters);
  cudaFree(p->d_status);
  delete p;
}

PersistRec* persist_add_class(PersistPlan* p, int instances) {
  PersistRec* r = new PersistRec();
  p->recs.push_back(r);
  p->inst.push_back(instances);
  return r;
}

// Tiles of descriptor d per instance, and the instance count of its grid.
static int desc_tiles(const PassDesc& d) { return d.kind == PK_COL_FWD ? d.gx * d.gy : d.gx; }
static int desc_insts(const PassDesc& d) { return d.kind == PK_COL_FWD ? d.gz : d.gy; }

cudaError_t persist_finalize(PersistPlan* p, std::string* err) {
  std::vector<PassDesc> descs;
  std::vector<int> first(p->recs.size()), npass(p->recs.size()), cbase(p->recs.size());
  int maxp = 0, nc = 0;
  for (size_t c = 0; c < p->recs.size(); ++c) {
    first[c] = (int)descs.size();
    npass[c] = (int)p->recs[c]->descs.size();
    cbase[c] = nc;
    for (const PassDesc& d : p->recs[c]->descs) {
      if (desc_insts(d) != p->inst[c]) {
        *err = "persistent plan: a pass does not cover the class's instances";
        return cudaErrorInvalidValue;
      }
      descs.push_back(d);
      if (d.smem > p->smem) p->smem = d.smem;
    }
    nc += p->inst[c] * npass[c];
    if (npass[c] > maxp) maxp = npass[c];
  }
  // within a pass, the classes with the longest lines (most work per item)
  // come first, so that the short items of small classes fill the end of it
  std::vector<size_t> order(p->recs.size());
  for (size_t c = 0; c < order.size(); ++c) order[c] = c;
  auto weight = [&](size_t c) { return npass[c] ? descs[first[c]].g.my + descs[first[c]].g.mx : 0; };
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b2) { return weight(a) > weight(b2); });
  std::vector<WorkItem> items;
  for (int ps = 0; ps < maxp; ++ps)
    for (size_t c : order) {
      if (ps >= npass[c]) continue;
      const int di = first[c] + ps;
      const PassDesc& d = descs[di];
      const int prev_tiles = ps > 0 ? desc_tiles(descs[di - 1]) : 0;
      for (int b = 0; b < p->inst[c]; ++b) {
        const int self = cbase[c] + b * npass[c] + ps;
        const int ny = d.kind == PK_COL_FWD ? d.gy : 1;
        for (int by = 0; by < ny; ++by)
          for (int bx = 0; bx < d.gx; ++bx) {
            WorkItem it;
            it.desc = di;
            it.bx = bx;
            it.by = by;
            it.b = b;
            it.dep = ps > 0 ? self - 1 : -1;
            it.need = prev_tiles;
            it.self = self;
            items.push_back(it);
          }
      }
    }
  if (items.empty() || p->smem + 64 > kSmemMax) {  // 64: the kernel's own static shared words
    *err = items.empty() ? "persistent plan: nothing to run" : "persistent plan: a pass exceeds shared memory";
    return cudaErrorInvalidValue;
  }
  p->n_items = (int)items.size();
  p->n_counters = nc;
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_descs, descs.size() * sizeof(PassDesc))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_items, items.size() * sizeof(WorkItem))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_counters, (size_t)(nc + 1) * sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_status, sizeof(int))) != cudaSuccess) {
    *err = "persistent plan: device memory";
    return e;
  }
  if ((e = cudaMemcpy(p->d_descs, descs.data(), descs.size() * sizeof(PassDesc), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) {
    *err = "persistent plan: upload";
    return e;
  }
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  // CTA width: the one with the most resident warps per SM (the narrowest on
  // a tie): one warp per CTA unless shared memory (the largest pass of any
  // class) caps the CTAs an SM holds
  int best_warps = 0;
  for (int nt : {32, 64, 128}) {
    int occ = 0;
    e = with_width(nt, [&](auto w) {
      constexpr int NT = decltype(w)::value;
      return p->prec == FCSPH_F64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<double, NT>, NT, p->smem)
                                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist<ff, NT>, NT, p->smem);
    });
    if (e != cudaSuccess) return e;
    if (occ * nt / 32 > best_warps) {
      best_warps = occ * nt / 32;
      p->threads = nt;
      p->grid = sms * occ;
    }
  }
  if (best_warps == 0) {
    *err = "persistent plan: no CTA fits an SM";
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

static cudaError_t persist_enqueue(PersistPlan* p, cudaStream_t st, long long wait_ns, int stall) {
  cudaError_t e = cudaMemsetAsync(p->d_counters, 0, (size_t)(p->n_counters + 1) * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  unsigned* next = p->d_counters + p->n_counters;
  return with_width(p->threads, [&](auto w) {
    constexpr int NT = decltype(w)::value;
    if (p->prec == FCSPH_F64)
      k_persist<double, NT><<<p->grid, NT, p->smem, st>>>(p->d_descs, p->d_items, p->n_items, p->d_counters, next,
                                                          p->d_status, wait_ns, stall);
    else
      k_persist<ff, NT><<<p->grid, NT, p->smem, st>>>(p->d_descs, p->d_items, p->n_items, p->d_counters, next,
                                                      p->d_status, wait_ns, stall);
    return cudaGetLastError();
  });
}

// One persistent launch (counter reset + kernel).  Without a stall it replays
// a CUDA graph of the two, captured on first use.
cudaError_t persist_launch(PersistPlan* p, cudaStream_t st, cudaStream_t cap, long long wait_ns, int stall) {
  if (stall >= 0) return persist_enqueue(p, st, wait_ns, stall);
  if (!p->gexec || p->graph_wait_ns != wait_ns) {
    if (p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t le = persist_enqueue(p, cap, wait_ns, -1);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return le != cudaSuccess ? le : e;
    }
    e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    p->graph_wait_ns = wait_ns;
  }
  return cudaGraphLaunch(p->gexec, st);
}

// Reads and clears the plan's status word (synchronises st).
cudaError_t persist_status(PersistPlan* p, cudaStream_t st, int* status) {
  *status = 0;
  cudaError_t e = cudaMemcpyAsync(status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && *status) e = cudaMemsetAsync(p->d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

long long persist_items(const PersistPlan* p) { return p ? p->n_items : 0; }
int persist_grid(const PersistPlan* p) { return p ? p->grid : 0; }
int persist_threads(const PersistPlan* p) { return p ? p->threads : 0; }
