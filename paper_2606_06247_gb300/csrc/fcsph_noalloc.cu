// fcsph_dft_noalloc: the batched DFT of fcsph_dft for callers that may not
// allocate device memory, e.g. code running inside a CUDA graph capture, a
// memory pool that forbids outside allocations, or a host process that must
// not touch the CUDA allocator at all.  Its scratch (roots of unity, the
// Bluestein chirp and filter) lives in one file-scope device array instead of
// a cudaMalloc'd buffer.
//
// Sharing and lifetime: every call, on every stream, uses the same array, and
// the array keeps the last call's contents; each call rewrites all of the
// scratch it reads (including the zero padding of the Bluestein filter)
// before using it.  Two calls whose work overlaps on the GPU therefore race
// on the array: serialise them (same stream, or events).  Each GPU that loads
// the library holds the array (kNoallocScratchBytes) until the process exits.
#include <mutex>

#include <cuda_runtime.h>

#include "fcsph_internal.h"

using namespace fcsph;

namespace {

constexpr size_t kNoallocScratchBytes = 1u << 20;  // 1 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in and must not be passed
// to a kernel).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// Allocation-free plan: the Stockham factorisation of make_plan (radices 8,
// then 4 or 2; 9, then 3; 5; 7; primes <= kMaxDirectPrime), else Bluestein with the smallest
// 2^a 3^b 5^c 7^d >= 2n - 1.  Offsets are into a pool laid out as
// [twiddles of the direct length | (Bluestein) chirp n | filter m].
bool factor_fixed(int n, Plan1* p) {
  int cnt[8] = {0};
  int big[kMaxStages];
  int nbig = 0;
  int r = n;
  for (int q = 2; q <= 7; ++q)
    while (r % q == 0) {
      ++cnt[q];
      r /= q;
    }
  for (int q = 11; r > 1; q += 2) {
    while (r % q == 0) {
      if (q > kMaxDirectPrime || nbig == kMaxStages) return false;
      big[nbig++] = q;
      r /= q;
    }
  }
  int rad[kMaxStages];
  int nr = 0;
  auto push = [&](int q) {
    if (nr == kMaxStages) return false;
    rad[nr++] = q;
    return true;
  };
  while (cnt[2] >= 3) {
    if (!push(8)) return false;
    cnt[2] -= 3;
  }
  if (cnt[2] == 2 && !push(4)) return false;
  if (cnt[2] == 1 && !push(2)) return false;
  while (cnt[3] >= 2) {
    if (!push(9)) return false;
    cnt[3] -= 2;
  }
  if (cnt[3] == 1 && !push(3)) return false;
  for (int i = 0; i < cnt[5]; ++i)
    if (!push(5)) return false;
  for (int i = 0; i < cnt[7]; ++i)
    if (!push(7)) return false;
  for (int i = 0; i < nbig; ++i)
    if (!push(big[i])) return false;
  plan_set_radices(p, n, rad, nr);
  return true;
}

bool plan_fixed(int n, FftPlan* P, int* pool_len) {
  P->bs = 0;
  P->base.tw = 0;
  if (factor_fixed(n, &P->base)) {
    *pool_len = n;
    return true;
  }
  int m = 2 * n - 1;
  for (;; ++m) {
    int r = m;
    for (int q = 2; q <= 7; ++q)
      while (r % q == 0) r /= q;
    if (r == 1) break;
  }
  if (!factor_fixed(m, &P->sub)) return false;
  P->bs = 1;
  plan_set_radices(&P->base, n, nullptr, 0);
  P->sub.tw = 0;
  P->chirp = m;
  P->bhat = m + n;
  *pool_len = m + n + m;
  return true;
}

// Writes the pool for plan P into the FP64 scratch: roots exp(-2 pi i e/L)
// (L = direct length), and for Bluestein the chirp exp(i pi j^2/n) and the
// zero-padded filter b (to be transformed in place afterwards).
__global__ void k_fill_pool(double2* pool, int L, int bs, int n, int m, int chirp, int bhat) {
  const int total = bs ? m + n + m : L;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    double s, c;
    if (t < L) {
      sincospi(-2.0 * (double)t / (double)L, &s, &c);
      pool[t] = make_double2(c, s);
    } else if (t < chirp + n) {
      const long long j = t - chirp;
      sincospi((double)((j * j) % (2LL * n)) / (double)n, &s, &c);
      pool[t] = make_double2(c, s);
    } else {
      const int j = t - bhat;  // filter index 0..m-1: b_j = c_j (j < n), b_{m-j} = c_j, else 0
      long long k = -1;
      if (j < n)
        k = j;
      else if (m - j < n)
        k = m - j;
      if (k >= 0) {
        sincospi((double)((k * k) % (2LL * n)) / (double)n, &s, &c);
        pool[t] = make_double2(c, s);
      } else {
        pool[t] = make_double2(0.0, 0.0);
      }
    }
  }
}

// Scales the transformed filter by 1/m and writes the FP32 copy of the pool.
__global__ void k_finish_pool(double2* pool, float2* pool32, int total, int bs, int bhat, int m) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    double2 v = pool[t];
    if (bs && t >= bhat) {
      v.x /= m;
      v.y /= m;
      pool[t] = v;
    }
    pool32[t] = make_float2((float)v.x, (float)v.y);
  }
}

}  // namespace

extern "C" fcsph_status fcsph_dft_noalloc(int n, int nlines, int dir, int prec, const void* in, void* out,
                                          void* stream) {
  if (n < 1 || nlines < 0 || (dir != -1 && dir != 1) || (prec != FCSPH_F64 && prec != FCSPH_F32) || !in || !out)
    return FCSPH_EINVAL;
  FftPlan P;
  int pool_len = 0;
  if (!plan_fixed(n, &P, &pool_len)) return FCSPH_EINVAL;
  const size_t need = (size_t)pool_len * (sizeof(double2) + sizeof(float2));
  if (need > kNoallocScratchBytes) return FCSPH_EINVAL;  // n too large for the fixed scratch
  if (nlines == 0) return FCSPH_OK;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return FCSPH_ECUDA;
  double2* pool64 = reinterpret_cast<double2*>(base);
  float2* pool32 = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(base) + (size_t)pool_len * sizeof(double2));
  cudaStream_t st = (cudaStream_t)stream;
  const int L = P.bs ? P.sub.n : n;
  k_fill_pool<<<64, 256, 0, st>>>(pool64, L, P.bs, n, P.bs ? P.sub.n : 0, P.chirp, P.bhat);
  if (cudaGetLastError() != cudaSuccess) return FCSPH_ECUDA;
  if (P.bs) {
    FftPlan direct;
    direct.base = P.sub;
    direct.bs = 0;
    if (launch_dft_lines(P.sub.n, 1, -1, FCSPH_F64, pool64 + P.bhat, pool64 + P.bhat, st, direct, pool64) !=
        cudaSuccess)
      return FCSPH_ECUDA;
  }
  k_finish_pool<<<64, 256, 0, st>>>(pool64, pool32, pool_len, P.bs, P.bhat, P.bs ? P.sub.n : 1);
  if (cudaGetLastError() != cudaSuccess) return FCSPH_ECUDA;
  if (launch_dft_lines(n, nlines, dir, prec, in, out, st, P,
                       prec == FCSPH_F64 ? (const void*)pool64 : (const void*)pool32) != cudaSuccess)
    return FCSPH_ECUDA;
  return FCSPH_OK;
}
