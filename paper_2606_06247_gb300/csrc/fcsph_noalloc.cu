// fcsph_dft_noalloc: the batched DFT of fcsph_dft for callers that may not
// allocate device memory, e.g. an application whose memory pool owns all
// device memory, or a host thread that must not call into the CUDA allocator
// at all.  Its scratch (roots of unity, the Bluestein chirp and filter) lives
// in one file-scope device array instead of a cudaMalloc'd buffer.
//
// Sharing and lifetime: every call, on every stream, uses the same array, and
// the array keeps the last call's contents; each call rewrites all of the
// scratch it reads (including the zero padding of the Bluestein filter)
// before using it.  Two calls whose work overlaps on the GPU therefore race
// on the array: serialise them (same stream, or events).  Each GPU that loads
// the library holds the array (kNoallocScratchBytes) until the process exits.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address and raises the kernels' shared-memory limits; both
// allocate nothing.
#include <mutex>
#include <string>

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
// to a kernel).  The same first call raises the dynamic shared-memory limit
// of every kernel on that device, which the transform launches need.
cudaError_t scratch_address(void** out, const char** where) {
  int dev = 0;
  *where = "cudaGetDevice";
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    *where = "kernel attributes";
    e = init_kernel_attributes();
    if (e != cudaSuccess) return e;
    void* p = nullptr;
    *where = "cudaGetSymbolAddress";
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
  for (int q = 11; r > 1 && q * q <= r; q += 2) {
    while (r % q == 0) {
      if (q > kMaxDirectPrime || nbig == kMaxStages) return false;
      big[nbig++] = q;
      r /= q;
    }
  }
  if (r > 1) {  // the prime left over once q^2 > r
    if (r > kMaxDirectPrime || nbig == kMaxStages) return false;
    big[nbig++] = r;
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

namespace {

fcsph_status reject(fcsph_status st, const std::string& msg) {
  set_global_error("fcsph_dft_noalloc: " + msg);
  return st;
}

fcsph_status cuda_reject(cudaError_t e, const char* where) {
  return reject(FCSPH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" fcsph_status fcsph_dft_noalloc(int n, int nlines, int dir, int prec, const void* in, void* out,
                                          void* stream) {
  if (n < 1 || nlines < 0 || (dir != -1 && dir != 1) || !in || !out) return reject(FCSPH_EINVAL, "bad argument");
  if (prec != FCSPH_F64 && prec != FCSPH_F32)
    return reject(FCSPH_EINVAL, "precision must be FCSPH_F64 or FCSPH_F32 (FCSPH_F32X2 is not supported)");
  constexpr size_t kEntry = sizeof(double2) + sizeof(float2);
  if ((size_t)n > kNoallocScratchBytes / kEntry)  // the pool holds at least n entries
    return reject(FCSPH_EINVAL, "length " + std::to_string(n) + " needs more than the fixed scratch");
  FftPlan P;
  int pool_len = 0;
  if (!plan_fixed(n, &P, &pool_len)) return reject(FCSPH_EINVAL, "no plan for length " + std::to_string(n));
  if ((size_t)pool_len * kEntry > kNoallocScratchBytes)
    return reject(FCSPH_EINVAL, "length " + std::to_string(n) + " needs more than the fixed scratch");
  // Every transform line must fit in one CTA's shared memory: the main
  // transform (length n, or m for Bluestein) and, for Bluestein, the FP64
  // transform of the length-m filter.
  FftPlan filt;
  filt.base = P.sub;
  filt.bs = 0;
  if (dft_lines_smem(prec, P) > dft_smem_max() || (P.bs && dft_lines_smem(FCSPH_F64, filt) > dft_smem_max()))
    return reject(FCSPH_EINVAL, "length " + std::to_string(n) + ": a transform line exceeds one CTA's shared memory");
  if (nlines == 0) return FCSPH_OK;
  // An error pending from earlier work on this thread is not this call's; it
  // is reported and left in place for its owner.
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return cuda_reject(e, "CUDA error pending before the call");
  void* base = nullptr;
  const char* where = "";
  if ((e = scratch_address(&base, &where)) != cudaSuccess) return cuda_reject(e, where);
  double2* pool64 = reinterpret_cast<double2*>(base);
  float2* pool32 = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(base) + (size_t)pool_len * sizeof(double2));
  cudaStream_t st = (cudaStream_t)stream;
  const int L = P.bs ? P.sub.n : n;
  k_fill_pool<<<64, 256, 0, st>>>(pool64, L, P.bs, n, P.bs ? P.sub.n : 0, P.chirp, P.bhat);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_reject(e, "fill pool");
  if (P.bs && (e = launch_dft_lines(P.sub.n, 1, -1, FCSPH_F64, pool64 + P.bhat, pool64 + P.bhat, st, filt, pool64)) !=
                  cudaSuccess)
    return cuda_reject(e, "Bluestein filter");
  k_finish_pool<<<64, 256, 0, st>>>(pool64, pool32, pool_len, P.bs, P.bhat, P.bs ? P.sub.n : 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_reject(e, "finish pool");
  if ((e = launch_dft_lines(n, nlines, dir, prec, in, out, st, P,
                            prec == FCSPH_F64 ? (const void*)pool64 : (const void*)pool32)) != cudaSuccess)
    return cuda_reject(e, "transform");
  return FCSPH_OK;
}
