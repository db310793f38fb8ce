// C ABI of the FC spectral ISPH hot path: contexts, tables, plans, workspace
// and the call sequences of fc_extend / spectral_op / spectral_div /
// ppe_solve / isph_step (Sec. 5.2).  All arithmetic runs in the kernels of
// fcsph_kernels.cu; this file only validates, allocates and sequences.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fcsph_internal.h"

#include <nvtx3/nvToolsExt.h>

using namespace fcsph;

namespace {

std::mutex g_err_mu;
std::string g_err;  // context-free calls

void set_global_err(const std::string& s) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = s;
}

fcsph_status fail(fcsph_ctx* c, fcsph_status st, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    set_global_err(msg);
  return st;
}

fcsph_status cuda_fail(fcsph_ctx* c, cudaError_t e, const char* where) {
  return fail(c, FCSPH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FCSPH_CK(call, where)                      \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

size_t cplx_bytes(int prec) { return prec == FCSPH_F32 ? 8 : 16; }

// Upload a host pool, fill Bluestein filters with the FP64 engine, then make
// the FP32 copy.  `fill` lists (plan, filter) pairs.
struct Fill {
  FftPlan P;
  std::vector<double> re, im;
};

// FP32x2 copy of an FP64 pool already on the device (and synchronised): each
// component split into hi = fl(x), lo = fl(x - hi).
cudaError_t pool_ff_copy(const double2* d64, size_t n, void** out) {
  std::vector<double2> h(n);
  cudaError_t e = cudaMemcpy(h.data(), d64, n * sizeof(double2), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  std::vector<float4> hf(n);
  for (size_t i = 0; i < n; ++i) {
    const float rh = (float)h[i].x, ih = (float)h[i].y;
    hf[i] = make_float4(rh, (float)(h[i].x - (double)rh), ih, (float)(h[i].y - (double)ih));
  }
  if ((e = cudaMalloc(out, n * sizeof(float4))) != cudaSuccess) return e;
  return cudaMemcpy(*out, hf.data(), n * sizeof(float4), cudaMemcpyHostToDevice);
}

fcsph_status upload_pool(fcsph_ctx* c, Pool& pool, std::vector<Fill>& fills, double2** d64, float2** d32,
                         cudaStream_t st) {
  const size_t n = pool.re.size();
  std::vector<double2> h(n);
  for (size_t i = 0; i < n; ++i) h[i] = make_double2(pool.re[i], pool.im[i]);
  FCSPH_CK(cudaMalloc((void**)d64, n * sizeof(double2)), "cudaMalloc(pool64)");
  FCSPH_CK(cudaMalloc((void**)d32, n * sizeof(float2)), "cudaMalloc(pool32)");
  FCSPH_CK(cudaMemcpyAsync(*d64, h.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st), "pool upload");
  for (Fill& f : fills) {
    const int m = f.P.sub.n;
    std::vector<double2> hb(m);
    for (int j = 0; j < m; ++j) hb[j] = make_double2(f.re[j], f.im[j]);
    double2* tmp = nullptr;
    FCSPH_CK(cudaMalloc((void**)&tmp, m * sizeof(double2)), "cudaMalloc(bluestein)");
    FCSPH_CK(cudaMemcpyAsync(tmp, hb.data(), m * sizeof(double2), cudaMemcpyHostToDevice, st), "bluestein upload");
    FftPlan direct;
    direct.base = f.P.sub;
    direct.bs = 0;
    cudaError_t e = launch_dft_lines(m, 1, -1, FCSPH_F64, tmp, tmp, st, direct, *d64);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(c, e, "bluestein filter");
    }
    FCSPH_CK(cudaMemcpyAsync(hb.data(), tmp, m * sizeof(double2), cudaMemcpyDeviceToHost, st), "bluestein download");
    FCSPH_CK(cudaStreamSynchronize(st), "bluestein sync");
    cudaFree(tmp);
    for (int j = 0; j < m; ++j) h[f.P.bhat + j] = make_double2(hb[j].x / m, hb[j].y / m);
  }
  FCSPH_CK(cudaMemcpyAsync(*d64, h.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st), "pool upload 2");
  std::vector<float2> hf(n);
  for (size_t i = 0; i < n; ++i) hf[i] = make_float2((float)h[i].x, (float)h[i].y);
  FCSPH_CK(cudaMemcpyAsync(*d32, hf.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st), "pool32 upload");
  FCSPH_CK(cudaStreamSynchronize(st), "pool sync");
  return FCSPH_OK;
}

FftPlan plan_for(int n, Pool* pool, std::vector<Fill>* fills) {
  Fill f;
  FftPlan P = make_plan(n, pool, &f.re, &f.im);
  if (P.bs || P.rd) {
    f.P = P;
    fills->push_back(f);
  }
  return P;
}

// Default CTA width of a pass of `ctas` one-warp CTAs: 12 such CTAs fit on
// each of the 152 SMs; a pass that fills a quarter of that or less gets
// 4-warp CTAs, half or less 2-warp CTAs.
int default_width(long long ctas) {
  const long long full = 152LL * 12;
  if (4 * ctas <= full) return 128;
  if (2 * ctas <= full) return 64;
  return 32;
}

// FP64 / FP32x2 CTA width for a pass whose CTAs hold smem_cta bytes of shared
// memory: registers (<= 168 a thread) allow 12 resident warps per SM at any
// width; when shared memory fits fewer one-warp CTAs than that (long lines),
// the narrowest width that reaches 12 warps.
int smem_width(size_t smem_cta) {
  const size_t per_sm = 228 * 1024, reserved = 1024;
  const long long fit = (long long)(per_sm / (smem_cta + reserved));
  for (int w : {32, 64, 128})
    if (fit * (w / 32) >= 12) return w;
  return 128;
}

RowOps ops_none() {
  RowOps o;
  memset(&o, 0, sizeof(o));
  return o;
}

size_t field_elems(const fcsph_ctx* c) { return (size_t)c->gd.batch * c->gd.ncol * c->gd.ny; }

// Spectrum buffer geometry (fields per instance) and z passes of the 3D grid.
static size_t spec_fs(const fcsph_ctx* c) { return (size_t)c->gd.rows * c->gd.ncol; }
static size_t in_bstride(const fcsph_ctx* c) { return (c->gd.nz > 1 ? 3 : 2) * spec_fs(c); }
static size_t out_bstride(const fcsph_ctx* c) { return (c->gd.nz > 1 ? 12 : 6) * spec_fs(c); }

}  // namespace

void set_global_error(const std::string& msg) { set_global_err(msg); }

// NVTX range names of the pass kinds (FCSPH_PROF_*), for fcsph_set_tracing.
static const char* const kPassNames[FCSPH_PROF_KINDS] = {
    "fcsph col_fwd", "fcsph row_mom", "fcsph row_div", "fcsph row_grad", "fcsph row_op",  "fcsph col_mom",
    "fcsph col_div", "fcsph col_corr", "fcsph col_out", "fcsph row_ppe", "fcsph col_ppe", "fcsph other"};

ProfScope::ProfScope(fcsph_ctx* ctx, int k) : c(ctx), kind(k) {
  if (c && c->trace_on && k >= 0 && k < FCSPH_PROF_KINDS) {
    nvtxRangePushA(kPassNames[k]);
    traced = true;
  }
  if (!c || !c->prof_on) return;
  cudaEvent_t a;
  if (!c->ev_free.empty()) {
    a = c->ev_free.back();
    c->ev_free.pop_back();
  } else if (cudaEventCreate(&a) != cudaSuccess) {
    return;
  }
  if (!c->ev_free.empty()) {
    b = c->ev_free.back();
    c->ev_free.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    c->ev_free.push_back(a);
    b = nullptr;
    return;
  }
  cudaEventRecord(a, c->stream);
  c->pending.push_back({kind, a, b});
}

ProfScope::~ProfScope() {
  if (b) cudaEventRecord(b, c->stream);
  if (traced) nvtxRangePop();
}

// An NVTX range around one call of the C ABI when tracing is on.
struct TraceRange {
  bool on;
  TraceRange(const fcsph_ctx* c, const char* name) : on(c && c->trace_on) {
    if (on) nvtxRangePushA(name);
  }
  ~TraceRange() {
    if (on) nvtxRangePop();
  }
};

extern "C" {

fcsph_status fcsph_fc_table(const fcsph_fc* fc, int bc, double* out_host, size_t n_out) {
  if (!fc || !out_host) return fail(nullptr, FCSPH_EINVAL, "fcsph_fc_table: null argument");
  std::vector<double> E;
  std::string err;
  int st = fc_table_build(fc, bc, &E, &err);
  if (st != FCSPH_OK) return fail(nullptr, (fcsph_status)st, err);
  if (n_out < E.size()) return fail(nullptr, FCSPH_EINVAL, "fcsph_fc_table: output too small");
  memcpy(out_host, E.data(), E.size() * sizeof(double));
  return FCSPH_OK;
}

fcsph_status fcsph_create(const fcsph_grid* grid, const fcsph_fc* fc, const fcsph_kernel* kernel,
                          const fcsph_precision* prec, const double* fc_table_dir, const double* fc_table_neu,
                          void* stream, fcsph_ctx** out) {
  if (!grid || !fc || !kernel || !prec || !out) return fail(nullptr, FCSPH_EINVAL, "fcsph_create: null argument");
  *out = nullptr;
  if (grid->nx < 4 || grid->ny < 2 * fc->n_match || grid->batch < 1 || !(grid->lx > 0) || !(grid->ly > 0))
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: need nx >= 4, ny >= 2*n_match, batch >= 1, lx, ly > 0");
  if (grid->nx > 8192 || grid->ny > 8192)
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: nx, ny > 8192 not supported");
  if (grid->batch > 65535)  // instances index the y (or z) dimension of every launch grid
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: batch > 65535 not supported");
  if (kernel->family < FCSPH_G2 || kernel->family > FCSPH_G10 || !(kernel->h_over_dx >= 0))
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: bad kernel");
  if (prec->fft_prec != FCSPH_F64 && prec->fft_prec != FCSPH_F32 && prec->fft_prec != FCSPH_F32X2)
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: bad precision");
  if (grid->x_walls && grid->nx < 2 * fc->n_match)
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: walled x needs nx >= 2*n_match");
  const int nz = grid->nz > 1 ? grid->nz : 1;
  if (nz > 1 && (grid->x_walls || !(grid->lz > 0) || nz > 8192))
    return fail(nullptr, FCSPH_EINVAL, "fcsph_create: a 3D grid (nz > 1) needs periodic x, lz > 0, nz <= 8192");
  if (nz > 1 && prec->ppe_refine_iters > 0)
    return fail(nullptr, FCSPH_EUNSUPPORTED, "fcsph_create: PPE refinement is 2D only");
  fcsph_ctx* c = new fcsph_ctx();
  c->grid = *grid;
  c->fc = *fc;
  c->kern = *kernel;
  c->prec = *prec;
  c->stream = (cudaStream_t)stream;
  for (int bc = 0; bc < 2; ++bc) {
    const double* given = bc == 0 ? fc_table_dir : fc_table_neu;
    if (given) {
      c->hE[bc].assign(given, given + (size_t)fc->n_cont * 2 * fc->n_match);
    } else {
      std::string err;
      int st = fc_table_build(fc, bc, &c->hE[bc], &err);
      if (st != FCSPH_OK) {
        delete c;
        return fail(nullptr, (fcsph_status)st, err);
      }
    }
  }
  GridDev& g = c->gd;
  g.nx = grid->nx;
  g.ny = grid->ny;
  g.nz = nz;
  g.ncol = g.nx * nz;
  g.dz = nz > 1 ? grid->lz / nz : 1.0;
  g.batch = grid->batch;
  g.nb = grid->batch;
  g.x_walls = grid->x_walls ? 1 : 0;
  g.n_match = fc->n_match;
  g.n_cont = fc->n_cont;
  g.my = g.ny + g.n_cont;
  g.mx = g.x_walls ? g.nx + g.n_cont : g.nx;
  g.hy = g.my / 2 + 1;
  g.rows = g.hy > g.ny ? g.hy : g.ny;
  g.lx = grid->lx;
  g.ly = grid->ly;
  g.dx = g.x_walls ? grid->lx / (g.nx - 1) : grid->lx / g.nx;
  g.dy = grid->ly / (g.ny - 1);
  g.h = kernel->h_over_dx * g.dx;
  g.ckx_d = 2.0 * 3.14159265358979323846 / (g.mx * g.dx);
  g.cky_d = 2.0 * 3.14159265358979323846 / (g.my * g.dy);
  g.ckz_d = 2.0 * 3.14159265358979323846 / (g.nz * g.dz);
  g.hh_d = g.h * g.h * 0.25;
  g.ckx_f = (float)g.ckx_d;
  g.cky_f = (float)g.cky_d;
  g.ckz_f = (float)g.ckz_d;
  g.hh_f = (float)g.hh_d;
  g.inv_my_f = (float)(1.0 / g.my);
  g.family = kernel->family;

  Pool pool;
  std::vector<Fill> fills;
  c->plan_y = plan_for(g.my, &pool, &fills);
  c->plan_x = plan_for(g.mx, &pool, &fills);
  c->plan_py = plan_for(2 * (g.ny - 1), &pool, &fills);
  c->plan_px = plan_for(g.x_walls ? 2 * (g.nx - 1) : g.nx, &pool, &fills);
  const std::vector<double> gx = gauss_axis(g.mx, g.dx, g.h, g.mx), gy = gauss_axis(g.my, g.dy, g.h, g.hy),
                            gz = gauss_axis(nz, g.dz, g.h, nz);
  g.ex_off = pool.add(gx, std::vector<double>(g.mx, 0.0));
  g.ey_off = pool.add(gy, std::vector<double>(g.hy, 0.0));
  g.ez_off = pool.add(gz, std::vector<double>(nz, 0.0));
  if (nz > 1) c->plan_z = plan_for(nz, &pool, &fills);
  {
    // Passes with fewer one-warp CTAs than the GPU holds leave SMs idle: give
    // each CTA 2 or 4 warps instead.  Long lines: one warp per CTA leaves too
    // few warps per SM (shared memory bound), so those passes share each
    // CTA's lines among more warps (FP32 lines of >= 768 points: 2 (row) or 4
    // (column); FP64 / FP32x2: the narrowest width that reaches 12 warps).
    const long long col_ctas = (long long)((g.ncol + 1) / 2) * g.batch;
    const long long row_ctas = (long long)g.hy * g.nz * g.batch;
    c->row_threads = default_width(row_ctas);
    c->col_threads = default_width(col_ctas);
    if (prec->fft_prec == FCSPH_F32) {
      if (c->plan_x.line_len() >= kWideLine) c->row_threads = std::max(c->row_threads, 64);
      if (c->plan_y.line_len() >= kWideLine) c->col_threads = 128;
    } else {
      // shared memory of the momentum passes, the largest of each kind: one
      // row CTA (2 nc lines) and one column-pair CTA (2 lines; its FP64
      // values stay in global memory)
      const size_t cb = 16, nc = g.nz > 1 ? 3 : 2;
      c->row_threads = std::max(c->row_threads, smem_width(2 * nc * c->plan_x.line_len() * cb));
      c->col_threads = std::max(c->col_threads, smem_width(2 * (size_t)c->plan_y.line_len() * cb));
    }
  }
  {
    // Eq. 33 eigenvalues: DFT lam_k = 2 pi kappa / Lx (kappa signed, Nyquist positive), DCT-I lam = pi k / L
    const double pi = 3.14159265358979323846;
    std::vector<double> lx2(g.nx), ly2(g.ny);
    for (int k = 0; k < g.nx; ++k) {
      double lk;
      if (g.x_walls) {
        lk = pi * k / g.lx;
      } else {
        const int kappa = (2 * k <= g.nx) ? k : k - g.nx;
        lk = 2.0 * pi * kappa / g.lx;
      }
      lx2[k] = lk * lk;
    }
    for (int l = 0; l < g.ny; ++l) {
      const double ll = pi * l / g.ly;
      ly2[l] = ll * ll;
    }
    g.lx2_off = pool.add(lx2, std::vector<double>(g.nx, 0.0));
    g.ly2_off = pool.add(ly2, std::vector<double>(g.ny, 0.0));
    std::vector<double> lz2(nz, 0.0);
    for (int k = 0; k < nz && nz > 1; ++k) {
      const int kappa = (2 * k <= nz) ? k : k - nz;
      const double lk = 2.0 * pi * kappa / grid->lz;
      lz2[k] = lk * lk;
    }
    g.lz2_off = pool.add(lz2, std::vector<double>(nz, 0.0));
  }

  fcsph_status st = FCSPH_OK;
  cudaError_t e;
#define CREATE_CK(call, where)             \
  if ((e = (call)) != cudaSuccess) {       \
    st = cuda_fail(c, e, where);           \
    goto fail_out;                         \
  }
  {
    CREATE_CK(init_kernel_attributes(), "kernel attributes");
    st = upload_pool(c, pool, fills, &c->pool64, &c->pool32, c->stream);
    if (st != FCSPH_OK) goto fail_out;
    CREATE_CK(pool_ff_copy(c->pool64, pool.re.size(), &c->poolff), "FP32x2 pool");
    const size_t ne = (size_t)g.n_cont * 2 * g.n_match;
    CREATE_CK(cudaMalloc((void**)&c->dE, 2 * ne * sizeof(double)), "cudaMalloc(E)");
    CREATE_CK(cudaMemcpy(c->dE, c->hE[0].data(), ne * sizeof(double), cudaMemcpyHostToDevice), "E upload");
    CREATE_CK(cudaMemcpy(c->dE + ne, c->hE[1].data(), ne * sizeof(double), cudaMemcpyHostToDevice), "E upload");
    if (prec->fft_prec != FCSPH_F64) {  // FP32-pair tables for the FP32 and FP32x2 FC sums
      std::vector<float2> hf(2 * ne);
      for (size_t i = 0; i < 2 * ne; ++i) {
        const double x = c->hE[i / ne][i % ne];
        const float h = (float)x;
        hf[i] = make_float2(h, (float)(x - (double)h));
      }
      CREATE_CK(cudaMalloc(&c->dEff, 2 * ne * sizeof(float2)), "cudaMalloc(Eff)");
      CREATE_CK(cudaMemcpy(c->dEff, hf.data(), 2 * ne * sizeof(float2), cudaMemcpyHostToDevice), "Eff upload");
    }
    {  // W_hat on the extended grid (Eq. 16), rounded once to the transform type
      const std::vector<double> W = what_table(gx, gy, gz, g.mx, g.my, g.nz, g.hy, g.dx, g.dy, g.dz, g.h, g.family);
      std::vector<float2> wf;
      std::vector<float> w32;
      const void* src = W.data();
      size_t bytes = W.size() * sizeof(double);
      if (prec->fft_prec == FCSPH_F32X2) {
        wf.resize(W.size());
        for (size_t i = 0; i < W.size(); ++i) {
          const float h = (float)W[i];
          wf[i] = make_float2(h, (float)(W[i] - (double)h));
        }
        src = wf.data();
        bytes = wf.size() * sizeof(float2);
      } else if (prec->fft_prec == FCSPH_F32) {
        w32.assign(W.begin(), W.end());
        src = w32.data();
        bytes = w32.size() * sizeof(float);
      }
      CREATE_CK(cudaMalloc(&c->dW, bytes), "cudaMalloc(W)");
      CREATE_CK(cudaMemcpy(c->dW, src, bytes, cudaMemcpyHostToDevice), "W upload");
    }
    const size_t fs = (size_t)g.rows * g.ncol * g.batch;
    const size_t cb = cplx_bytes(prec->fft_prec);
    const bool d3 = g.nz > 1;
    CREATE_CK(cudaMalloc(&c->spec_in, (d3 ? 3 : 2) * fs * cb), "cudaMalloc(spec_in)");
    CREATE_CK(cudaMalloc(&c->spec_out, (d3 ? 12 : 6) * fs * cb), "cudaMalloc(spec_out)");
    CREATE_CK(cudaMalloc(&c->spec_ppe, fs * 16), "cudaMalloc(spec_ppe)");  // FP64-sized: refinement
    CREATE_CK(cudaMalloc((void**)&c->work, (d3 ? 7 : 6) * field_elems(c) * sizeof(double)), "cudaMalloc(work)");
    CREATE_CK(cudaMalloc((void**)&c->dred, 8 * sizeof(double)), "cudaMalloc(red)");
    CREATE_CK(cudaMalloc((void**)&c->dstatus, sizeof(int)), "cudaMalloc(status)");
    CREATE_CK(cudaMemset(c->dstatus, 0, sizeof(int)), "status clear");
    CREATE_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
  }
  *out = c;
  return FCSPH_OK;
fail_out:
  set_global_err(c->err);
  fcsph_destroy(c);
  return st;
#undef CREATE_CK
}

fcsph_status fcsph_destroy(fcsph_ctx* c) {
  if (!c) return FCSPH_OK;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (auto& p : c->pending) {
    c->ev_free.push_back(p.a);
    c->ev_free.push_back(p.b);
  }
  for (cudaEvent_t ev : c->ev_free) cudaEventDestroy(ev);
  cudaFree(c->pool64);
  cudaFree(c->pool32);
  cudaFree(c->poolff);
  cudaFree(c->dE);
  cudaFree(c->dEff);
  cudaFree(c->dW);
  cudaFree(c->spec_in);
  cudaFree(c->spec_out);
  cudaFree(c->spec_ppe);
  cudaFree(c->work);
  cudaFree(c->dred);
  cudaFree(c->dstatus);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  persist_destroy(c->pplan);
  for (cudaStream_t gs : c->grp_streams) cudaStreamDestroy(gs);
  for (cudaEvent_t ge : c->grp_events) cudaEventDestroy(ge);
  delete c;
  return FCSPH_OK;
}

fcsph_status fcsph_get_fc_table(const fcsph_ctx* c, int bc, double* out_host, size_t n_out) {
  if (!c || !out_host || (bc != 0 && bc != 1)) return fail(nullptr, FCSPH_EINVAL, "fcsph_get_fc_table: bad argument");
  if (n_out < c->hE[bc].size()) return fail(nullptr, FCSPH_EINVAL, "fcsph_get_fc_table: output too small");
  memcpy(out_host, c->hE[bc].data(), c->hE[bc].size() * sizeof(double));
  return FCSPH_OK;
}

fcsph_status fc_extend(fcsph_ctx* c, const void* f, void* f_ext, int bc) {
  TraceRange tr(c, "fcsph fc_extend");
  if (!c || !f || !f_ext || (bc != 0 && bc != 1)) return fail(c, FCSPH_EINVAL, "fc_extend: bad argument");
  FCSPH_CK(launch_fc_extend(c, f, f_ext, bc), "fc_extend");
  return FCSPH_OK;
}

fcsph_status spectral_op(fcsph_ctx* c, const void* f, unsigned op_mask, int bc, void* const* outs) {
  TraceRange tr(c, "fcsph spectral_op");
  if (!c || !f || !outs || (bc != 0 && bc != 1)) return fail(c, FCSPH_EINVAL, "spectral_op: bad argument");
  const unsigned all = c->gd.nz > 1 ? 31u : 15u;
  if (op_mask == 0 || (op_mask & ~all))
    return fail(c, FCSPH_EINVAL, "spectral_op: op_mask must be a nonempty subset of W|DX|DY|LAP (|DZ on 3D grids)");
  RowOps ops = ops_none();
  ops.nin = 1;
  const int sym[5] = {SYM_W, SYM_DX, SYM_DY, SYM_LAP, SYM_DZ};
  for (int b = 0; b < 5; ++b)
    if (op_mask & (1u << b)) {
      if (!outs[ops.nout]) return fail(c, FCSPH_EINVAL, "spectral_op: null output pointer");
      ops.nterm[ops.nout] = 1;
      ops.field[ops.nout][0] = 0;
      ops.op[ops.nout][0] = sym[b];
      ops.nout++;
    }
  const int p = c->prec.fft_prec;
  const void* fl[1] = {f};
  FCSPH_CK(launch_col_fwd(c, p, 1, fl, p != FCSPH_F32, bc, c->spec_in, 0), "spectral_op fwd");
  FCSPH_CK(launch_zpass(c, p, c->spec_in, 1, in_bstride(c), c->gd.hy, 0), "spectral_op z fwd");
  FCSPH_CK(launch_row_sym(c, p, c->spec_in, c->spec_out, ops, 1.0 / ((double)c->gd.mx * c->gd.my * c->gd.nz), bc,
                          FCSPH_PROF_ROW_OP),
           "spectral_op row");
  FCSPH_CK(launch_zpass(c, p, c->spec_out, ops.nout, out_bstride(c), c->gd.hy, 1), "spectral_op z inv");
  FCSPH_CK(launch_col_out(c, c->spec_out, ops.nout, outs), "spectral_op inv");
  return FCSPH_OK;
}

fcsph_status line_op(fcsph_ctx* c, const void* f, unsigned op_mask, int bc, void* const* outs) {
  TraceRange tr(c, "fcsph line_op");
  if (!c || !f || !outs || (bc != 0 && bc != 1)) return fail(c, FCSPH_EINVAL, "line_op: bad argument");
  if (op_mask == 0 || op_mask > 15u) return fail(c, FCSPH_EINVAL, "line_op: op_mask must be a nonempty subset of W|DX|DY|LAP");
  const int sym[4] = {SYM_W, SYM_DX, SYM_DY, SYM_LAP};
  int ops[4], n = 0;
  for (int b = 0; b < 4; ++b)
    if (op_mask & (1u << b)) {
      if (!outs[n]) return fail(c, FCSPH_EINVAL, "line_op: null output pointer");
      ops[n++] = sym[b];
    }
  FCSPH_CK(launch_line_op(c, f, ops, n, bc, outs), "line_op");
  return FCSPH_OK;
}

fcsph_status spectral_div(fcsph_ctx* c, const void* fx, const void* fy, void* out) {
  TraceRange tr(c, "fcsph spectral_div");
  if (!c || !fx || !fy || !out) return fail(c, FCSPH_EINVAL, "spectral_div: bad argument");
  if (c->gd.nz > 1) return fail(c, FCSPH_EUNSUPPORTED, "spectral_div: 2D grids only");
  RowOps ops = ops_none();
  ops.nin = 2;
  ops.nout = 1;
  ops.nterm[0] = 2;
  ops.field[0][0] = 0;
  ops.op[0][0] = SYM_DX;
  ops.field[0][1] = 1;
  ops.op[0][1] = SYM_DY;
  const int p = c->prec.fft_prec;
  const void* fl[2] = {fx, fy};
  void* outs[1] = {out};
  FCSPH_CK(launch_col_fwd(c, p, 2, fl, p != FCSPH_F32, FCSPH_DIRICHLET, c->spec_in, 0), "spectral_div fwd");
  FCSPH_CK(launch_row_sym(c, p, c->spec_in, c->spec_out, ops, 1.0 / ((double)c->gd.mx * c->gd.my), FCSPH_DIRICHLET,
                          FCSPH_PROF_ROW_OP),
           "spectral_div row");
  FCSPH_CK(launch_col_out(c, c->spec_out, 1, outs), "spectral_div inv");
  return FCSPH_OK;
}

fcsph_status spectral_project(fcsph_ctx* c, const void* fx, const void* fy, void* out_x, void* out_y) {
  TraceRange tr(c, "fcsph spectral_project");
  if (!c || !fx || !fy || !out_x || !out_y) return fail(c, FCSPH_EINVAL, "spectral_project: bad argument");
  if (c->gd.nz > 1) return fail(c, FCSPH_EUNSUPPORTED, "spectral_project: 2D grids only");
  // out_x = U - (gx^2 U + gx gy V)/|g|^2, out_y = V - (gx gy U + gy^2 V)/|g|^2
  RowOps ops = ops_none();
  ops.nin = 2;
  ops.nout = 2;
  const int terms[2][3][2] = {{{0, SYM_ONE}, {0, SYM_NPXX}, {1, SYM_NPXY}}, {{1, SYM_ONE}, {0, SYM_NPXY}, {1, SYM_NPYY}}};
  for (int o = 0; o < 2; ++o) {
    ops.nterm[o] = 3;
    for (int t = 0; t < 3; ++t) {
      ops.field[o][t] = terms[o][t][0];
      ops.op[o][t] = terms[o][t][1];
    }
  }
  const int p = c->prec.fft_prec;
  const void* fl[2] = {fx, fy};
  void* outs[2] = {out_x, out_y};
  FCSPH_CK(launch_col_fwd(c, p, 2, fl, p != FCSPH_F32, FCSPH_DIRICHLET, c->spec_in, 0), "spectral_project fwd");
  FCSPH_CK(launch_row_sym(c, p, c->spec_in, c->spec_out, ops, 1.0 / ((double)c->gd.mx * c->gd.my), FCSPH_DIRICHLET,
                          FCSPH_PROF_ROW_OP),
           "spectral_project row");
  FCSPH_CK(launch_col_out(c, c->spec_out, 2, outs), "spectral_project inv");
  return FCSPH_OK;
}

// Iterative refinement of the PPE solution phi64 (double, device) for the
// right-hand side b64: b0 = b64 without its (0,0) transform mode (FP64), then
// `iters` sweeps of r = b0 - L phi (FP64) and phi += solve(r) (context
// precision).  Removing the constant mode first keeps it out of the FP32
// corrections, whose rounding it would otherwise dominate.  The last sweep
// optionally ends with the Neumann-FC forward transform of phi (spec_in).
static fcsph_status ppe_refine(fcsph_ctx* c, const double* b64, double* phi64, int iters, int neumann_fwd) {
  const int p = c->prec.fft_prec;
  const size_t n = field_elems(c);
  double* r = c->work + 4 * n;
  double* b0 = c->work + 5 * n;
  const void* bl[1] = {b64};
  FCSPH_CK(launch_col_fwd(c, FCSPH_F64, 1, bl, 1, FCSPH_DIRICHLET, c->spec_ppe, 1), "refine project fwd");
  FCSPH_CK(launch_row_ppe(c, FCSPH_F64, c->spec_ppe, 2), "refine project row");
  FCSPH_CK(launch_col_ppe_inv(c, FCSPH_F64, c->spec_ppe, b0, 1, nullptr, 0, nullptr, 0, nullptr), "refine project inv");
  for (int it = 0; it < iters; ++it) {
    const void* pl[1] = {phi64};
    FCSPH_CK(launch_col_fwd(c, FCSPH_F64, 1, pl, 1, FCSPH_DIRICHLET, c->spec_ppe, 1), "refine L fwd");
    FCSPH_CK(launch_row_ppe(c, FCSPH_F64, c->spec_ppe, 1), "refine L row");
    FCSPH_CK(launch_col_ppe_inv(c, FCSPH_F64, c->spec_ppe, r, 1, nullptr, 1, b0, 0, nullptr), "refine resid");
    const void* rl[1] = {r};
    FCSPH_CK(launch_col_fwd(c, p, 1, rl, 1, FCSPH_DIRICHLET, c->spec_ppe, 1), "refine fwd");
    FCSPH_CK(launch_row_ppe(c, p, c->spec_ppe, 0), "refine row");
    const bool last = it + 1 == iters;
    FCSPH_CK(launch_col_ppe_inv(c, p, c->spec_ppe, phi64, 1, phi64, 2, nullptr, (neumann_fwd && last) ? 1 : 0,
                                c->spec_in),
             "refine add");
  }
  return FCSPH_OK;
}

fcsph_status ppe_solve(fcsph_ctx* c, const void* rhs, void* phi, double* resid_out) {
  TraceRange tr(c, "fcsph ppe_solve");
  if (!c || !rhs || !phi) return fail(c, FCSPH_EINVAL, "ppe_solve: bad argument");
  const int p = c->prec.fft_prec;
  const size_t n = field_elems(c);
  double* b64 = c->work + 2 * n;
  double* phi64 = c->work + 3 * n;
  if (p != FCSPH_F32) {
    FCSPH_CK(cudaMemcpyAsync(b64, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "ppe rhs copy");
  } else {
    FCSPH_CK(cudaMemsetAsync(b64, 0, n * sizeof(double), c->stream), "ppe rhs clear");
    FCSPH_CK(launch_axpy(c, b64, nullptr, (const float*)rhs, (int)n, 1.0), "ppe rhs widen");
  }
  const int iters = p == FCSPH_F32 ? c->prec.ppe_refine_iters : 0;
  const void* bl[1] = {b64};
  FCSPH_CK(launch_col_fwd(c, p, 1, bl, 1, FCSPH_DIRICHLET, c->spec_ppe, 1), "ppe fwd");
  FCSPH_CK(launch_zpass(c, p, c->spec_ppe, 1, spec_fs(c), c->gd.ny, 0), "ppe z fwd");
  FCSPH_CK(launch_row_ppe(c, p, c->spec_ppe, 0), "ppe row");
  FCSPH_CK(launch_zpass(c, p, c->spec_ppe, 1, spec_fs(c), c->gd.ny, 1), "ppe z inv");
  FCSPH_CK(launch_col_ppe_inv(c, p, c->spec_ppe, iters > 0 ? (void*)phi64 : phi, iters > 0 ? 1 : (p != FCSPH_F32),
                              phi64, 0, nullptr, 0, nullptr),
           "ppe inv");
  if (iters > 0) {
    fcsph_status st = ppe_refine(c, b64, phi64, iters, 0);
    if (st != FCSPH_OK) return st;
    FCSPH_CK(launch_narrow(c, (float*)phi, phi64, (int)n), "ppe phi narrow");
  }
  if (resid_out) {
    // r = b - L phi in FP64; its constant (0,0) part per instance is removed
    double* r = c->work + 4 * n;
    const void* pl[1] = {phi64};
    FCSPH_CK(launch_col_fwd(c, FCSPH_F64, 1, pl, 1, FCSPH_DIRICHLET, c->spec_ppe, 1), "resid fwd");
    FCSPH_CK(launch_zpass(c, FCSPH_F64, c->spec_ppe, 1, spec_fs(c), c->gd.ny, 0), "resid z fwd");
    FCSPH_CK(launch_row_ppe(c, FCSPH_F64, c->spec_ppe, 1), "resid row");
    FCSPH_CK(launch_zpass(c, FCSPH_F64, c->spec_ppe, 1, spec_fs(c), c->gd.ny, 1), "resid z inv");
    FCSPH_CK(launch_col_ppe_inv(c, FCSPH_F64, c->spec_ppe, r, 1, nullptr, 1, b64, 0, nullptr), "resid inv");
    FCSPH_CK(launch_resid_norm(c, r, b64, c->dred), "resid norm");
    double h2[2];
    FCSPH_CK(cudaMemcpyAsync(h2, c->dred, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "resid read");
    FCSPH_CK(cudaStreamSynchronize(c->stream), "resid sync");
    *resid_out = h2[1] > 0 ? std::sqrt(h2[0] / h2[1]) : std::sqrt(h2[0]);
  }
  return FCSPH_OK;
}

// One substep (Eqs. 5-9).  Precondition: spec_in holds the Dirichlet-FC
// y transforms of the velocity components.  Postcondition (fwd_next): the
// same for the new velocity.  3D grids transform every x pass's inputs in z
// first and its outputs back in z after.
static fcsph_status substep(fcsph_ctx* c, const fcsph_state* s, const StepDev& sd, int fwd_next) {
  const int p = c->prec.fft_prec;
  const size_t n = field_elems(c);
  const bool d3 = c->gd.nz > 1;
  const int nc = d3 ? 3 : 2;
  const int hy = c->gd.hy, ny = c->gd.ny;
  double* vs[3] = {c->work, c->work + n, c->work + 3 * n};  // u*, v*, w*
  double* b = c->work + 2 * n;
  const double scale = 1.0 / ((double)c->gd.mx * c->gd.my * c->gd.nz);
  const double* vel[3] = {s->u, s->v, s->w};
  double* Fp[3] = {s->fu, s->fv, s->fw};
  double* vo[3] = {s->u, s->v, s->w};
  // momentum: d/dx, d/dy, (d/dz,) lap of every component
  RowOps mom = ops_none();
  mom.nin = nc;
  mom.nout = nc * (nc + 1);
  const int opl2[3] = {SYM_DX, SYM_DY, SYM_LAP};
  const int opl3[4] = {SYM_DX, SYM_DY, SYM_DZ, SYM_LAP};
  for (int o = 0; o < mom.nout; ++o) {
    mom.nterm[o] = 1;
    mom.field[o][0] = o / (nc + 1);
    mom.op[o][0] = d3 ? opl3[o % 4] : opl2[o % 3];
  }
  FCSPH_CK(launch_zpass(c, p, c->spec_in, nc, in_bstride(c), hy, 0), "step mom z fwd");
  FCSPH_CK(launch_row_sym(c, p, c->spec_in, c->spec_out, mom, scale, FCSPH_DIRICHLET, FCSPH_PROF_ROW_MOM), "step mom row");
  FCSPH_CK(launch_zpass(c, p, c->spec_out, mom.nout, out_bstride(c), hy, 1), "step mom z inv");
  FCSPH_CK(launch_step_mom(c, sd, c->spec_out, vel, Fp, vs, c->spec_in), "step mom col");
  // divergence of u*
  RowOps dv = ops_none();
  dv.nin = nc;
  dv.nout = 1;
  dv.nterm[0] = nc;
  const int dops[3] = {SYM_DX, SYM_DY, SYM_DZ};
  for (int t = 0; t < nc; ++t) {
    dv.field[0][t] = t;
    dv.op[0][t] = dops[t];
  }
  FCSPH_CK(launch_zpass(c, p, c->spec_in, nc, in_bstride(c), hy, 0), "step div z fwd");
  FCSPH_CK(launch_row_sym(c, p, c->spec_in, c->spec_out, dv, scale, FCSPH_DIRICHLET, FCSPH_PROF_ROW_DIV), "step div row");
  FCSPH_CK(launch_zpass(c, p, c->spec_out, 1, out_bstride(c), hy, 1), "step div z inv");
  FCSPH_CK(launch_step_div(c, sd, c->spec_out, b, c->spec_ppe), "step div col");
  // PPE: the DCT-y forward of b is already in spec_ppe (fused above)
  const int iters = p == FCSPH_F32 ? c->prec.ppe_refine_iters : 0;
  FCSPH_CK(launch_zpass(c, p, c->spec_ppe, 1, spec_fs(c), ny, 0), "step ppe z fwd");
  FCSPH_CK(launch_row_ppe(c, p, c->spec_ppe, 0), "step ppe row");
  FCSPH_CK(launch_zpass(c, p, c->spec_ppe, 1, spec_fs(c), ny, 1), "step ppe z inv");
  FCSPH_CK(launch_col_ppe_inv(c, p, c->spec_ppe, s->p, 1, s->p, 0, nullptr, iters == 0 ? 1 : 0, c->spec_in),
           "step ppe col");
  if (iters > 0) {
    fcsph_status st = ppe_refine(c, b, s->p, iters, 1);
    if (st != FCSPH_OK) return st;
  }
  // gradient of phi and the correction
  RowOps gr = ops_none();
  gr.nin = 1;
  gr.nout = nc;
  for (int o = 0; o < nc; ++o) {
    gr.nterm[o] = 1;
    gr.op[o][0] = dops[o];
  }
  FCSPH_CK(launch_zpass(c, p, c->spec_in, 1, in_bstride(c), hy, 0), "step grad z fwd");
  FCSPH_CK(launch_row_sym(c, p, c->spec_in, c->spec_out, gr, scale, FCSPH_NEUMANN, FCSPH_PROF_ROW_GRAD), "step grad row");
  FCSPH_CK(launch_zpass(c, p, c->spec_out, nc, out_bstride(c), hy, 1), "step grad z inv");
  FCSPH_CK(launch_step_corr(c, sd, c->spec_out, vs, vo, fwd_next ? c->spec_in : nullptr), "step corr col");
  return FCSPH_OK;
}

static fcsph_status one_step(fcsph_ctx* c, const fcsph_state* s, const fcsph_step_params* prm) {
  static const double A3[3] = {8.0 / 15.0, 2.0 / 15.0, 1.0 / 3.0};
  static const double G3[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
  static const double Z3[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
  const int nsub = prm->scheme == FCSPH_SCHEME_RK3 ? 3 : 1;
  for (int k = 0; k < nsub; ++k) {
    StepDev sd;
    sd.nu = prm->nu;
    sd.rho = prm->rho;
    sd.dt = prm->dt;
    sd.fx = prm->force_x;
    sd.fy = prm->force_y;
    sd.fz = prm->force_z;
    sd.u_bottom = prm->u_bottom;
    sd.u_top = prm->u_top;
    sd.nu_inst = prm->nu_inst;
    sd.dt_inst = prm->dt_inst;
    sd.fx_inst = prm->fx_inst;
    if (nsub == 3) {
      sd.a = A3[k];
      sd.g = G3[k];
      sd.z = Z3[k];
    } else {
      sd.a = 1.0;
      sd.g = 1.0;
      sd.z = 0.0;
    }
    fcsph_status st = substep(c, s, sd, 1);
    if (st != FCSPH_OK) return st;
  }
  return FCSPH_OK;
}

// Instance groups of the step graph: the batch is split into G groups of
// nearly equal size, and each group's kernels form their own chain (a branch
// of the graph on its own capture stream).  A pass of one group then runs
// while another group's previous pass is still draining, so the partial last
// wave of CTAs of one launch overlaps with the next launch of another group.
// PPE refinement reduces over the whole batch between passes and keeps one
// chain.
static int step_groups(const fcsph_ctx* c, const fcsph_step_params* prm) {
  (void)prm;
  int G = c->groups;
  if (c->prec.fft_prec == FCSPH_F32 && c->prec.ppe_refine_iters > 0) G = 1;
  if (G > c->gd.batch) G = c->gd.batch;
  return G < 1 ? 1 : G;
}

static fcsph_status ensure_group_streams(fcsph_ctx* c, int G) {
  while ((int)c->grp_streams.size() < G) {
    cudaStream_t st = nullptr;
    FCSPH_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "group stream");
    c->grp_streams.push_back(st);
  }
  while ((int)c->grp_events.size() < G + 1) {
    cudaEvent_t ev = nullptr;
    FCSPH_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "group event");
    c->grp_events.push_back(ev);
  }
  return FCSPH_OK;
}

// Inside a capture on c->cap_stream: forks G group streams off it, records one
// step of instances [b0, b0 + nb) on each, and joins them back.  Every forked
// stream is joined even when a launch fails, so the capture can end.
static fcsph_status capture_groups(fcsph_ctx* c, const fcsph_state* s, const fcsph_step_params* prm, int G) {
  const int B = c->gd.batch;
  cudaEvent_t fork = c->grp_events[0];
  fcsph_status st = FCSPH_OK;
  if (cudaEventRecord(fork, c->cap_stream) != cudaSuccess) return fail(c, FCSPH_ECUDA, "group fork");
  int forked = 0;
  for (int k = 0; k < G; ++k) {
    if (cudaStreamWaitEvent(c->grp_streams[k], fork, 0) != cudaSuccess) {
      st = fail(c, FCSPH_ECUDA, "group fork wait");
      break;
    }
    forked = k + 1;
    const int b0 = (int)((long long)B * k / G), b1 = (int)((long long)B * (k + 1) / G);
    c->stream = c->grp_streams[k];
    c->gd.b0 = b0;
    c->gd.nb = b1 - b0;
    st = one_step(c, s, prm);
    if (st != FCSPH_OK) break;
  }
  c->gd.b0 = 0;
  c->gd.nb = B;
  c->stream = c->cap_stream;
  for (int k = 0; k < forked; ++k) {
    cudaEvent_t join = c->grp_events[k + 1];
    if ((cudaEventRecord(join, c->grp_streams[k]) != cudaSuccess ||
         cudaStreamWaitEvent(c->cap_stream, join, 0) != cudaSuccess) && st == FCSPH_OK)
      st = fail(c, FCSPH_ECUDA, "group join");
  }
  return st;
}

// The arguments a recorded step depends on (device pointers and parameters).
static std::vector<double> step_key(const fcsph_state* s, const fcsph_step_params* prm) {
  return {(double)(uintptr_t)s->u, (double)(uintptr_t)s->v, (double)(uintptr_t)s->p,
          (double)(uintptr_t)s->fu, (double)(uintptr_t)s->fv, prm->nu, prm->rho, prm->dt,
          prm->force_x, prm->force_y, prm->u_bottom, prm->u_top, (double)prm->scheme,
          (double)(uintptr_t)prm->nu_inst, (double)(uintptr_t)prm->fx_inst,
          (double)(uintptr_t)s->w, (double)(uintptr_t)s->fw, prm->force_z,
          (double)(uintptr_t)prm->active, (double)(uintptr_t)prm->dt_inst};
}

// nsteps steps, each one launch of the persistent kernel over the recorded
// passes of one step (after the forward transform isph_step launched).
static fcsph_status persistent_steps(fcsph_ctx* c, const fcsph_state* s, int nsteps, const fcsph_step_params* prm) {
  std::vector<double> key = step_key(s, prm);
  if (!c->pplan || key != c->pplan_key) {
    persist_destroy(c->pplan);
    c->pplan = persist_create(c->prec.fft_prec);
    fcsph_status st = record_isph_step(c, s, prm, persist_add_class(c->pplan, c->gd.batch), 0);
    if (st != FCSPH_OK) {
      persist_destroy(c->pplan);
      c->pplan = nullptr;
      return st;
    }
    std::string err;
    cudaError_t e = persist_finalize(c->pplan, &err);
    if (e != cudaSuccess) {
      persist_destroy(c->pplan);
      c->pplan = nullptr;
      return fail(c, FCSPH_ECUDA, "isph_step: " + err + ": " + cudaGetErrorString(e));
    }
    c->pplan_key = key;
  }
  for (int it = 0; it < nsteps; ++it)
    FCSPH_CK(persist_launch(c->pplan, c->stream, c->cap_stream, 1000000000ll, -1), "persistent step");
  c->launches += nsteps;
  return FCSPH_OK;
}

// Sets the context's instance mask for the duration of one isph_step call.
struct ActiveScope {
  fcsph_ctx* c;
  ActiveScope(fcsph_ctx* ctx, const unsigned char* active) : c(ctx) { c->gd.active = active; }
  ~ActiveScope() { c->gd.active = nullptr; }
};

static fcsph_status isph_step_masked(fcsph_ctx* c, const fcsph_state* s, int nsteps, const fcsph_step_params* prm);

fcsph_status isph_step(fcsph_ctx* c, const fcsph_state* s, int nsteps, const fcsph_step_params* prm) {
  TraceRange tr(c, "fcsph isph_step");
  if (!c || !s || !prm || nsteps < 0) return fail(c, FCSPH_EINVAL, "isph_step: bad argument");
  if (prm->active && c->prec.fft_prec == FCSPH_F32 && c->prec.ppe_refine_iters > 0)
    return fail(c, FCSPH_EUNSUPPORTED, "isph_step: an instance mask with PPE refinement");
  ActiveScope scope(c, prm->active);
  return isph_step_masked(c, s, nsteps, prm);
}

static fcsph_status isph_step_masked(fcsph_ctx* c, const fcsph_state* s, int nsteps, const fcsph_step_params* prm) {
  if (!s->u || !s->v || !s->p || !s->fu || !s->fv) return fail(c, FCSPH_EINVAL, "isph_step: null state pointer");
  if (c->gd.nz > 1 && (!s->w || !s->fw)) return fail(c, FCSPH_EINVAL, "isph_step: a 3D grid needs w and fw");
  if (prm->scheme != FCSPH_SCHEME_FOP && prm->scheme != FCSPH_SCHEME_RK3)
    return fail(c, FCSPH_EINVAL, "isph_step: bad scheme");
  if (!(prm->dt > 0) || !(prm->rho > 0) || !(prm->nu >= 0)) return fail(c, FCSPH_EINVAL, "isph_step: need dt, rho > 0, nu >= 0");
  if (nsteps == 0) return FCSPH_OK;
  const void* uvw[3] = {s->u, s->v, s->w};
  FCSPH_CK(launch_col_fwd(c, c->prec.fft_prec, c->gd.nz > 1 ? 3 : 2, uvw, 1, FCSPH_DIRICHLET, c->spec_in, 0),
           "step initial fwd");
  if (!prm->use_graph) {
    for (int it = 0; it < nsteps; ++it) {
      fcsph_status st = one_step(c, s, prm);
      if (st != FCSPH_OK) return st;
    }
    return FCSPH_OK;
  }
  if (c->persist) return persistent_steps(c, s, nsteps, prm);
  std::vector<double> key = step_key(s, prm);
  if (!c->gexec || key != c->graph_key) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    cudaStream_t user = c->stream;
    const int prof = c->prof_on;
    c->prof_on = 0;
    const int G = step_groups(c, prm);
    if (G > 1) {
      fcsph_status gst = ensure_group_streams(c, G);
      if (gst != FCSPH_OK) {
        c->prof_on = prof;
        return gst;
      }
    }
    c->stream = c->cap_stream;
    FCSPH_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
    const long long before = c->launches;
    fcsph_status st = G > 1 ? capture_groups(c, s, prm, G) : one_step(c, s, prm);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->stream = user;
    c->prof_on = prof;
    c->graph_kernels = c->launches - before;
    c->launches = before;  // captured launches are counted at replay
    if (st != FCSPH_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    c->graph_key = key;
  }
  for (int it = 0; it < nsteps; ++it) FCSPH_CK(cudaGraphLaunch(c->gexec, c->stream), "graph launch");
  c->launches += (long long)nsteps * c->graph_kernels;
  return FCSPH_OK;
}

// One RK3 (or FOP) step of every instance recorded as pass descriptors for
// the persistent multi-class launch (2D, FP64 or FP32x2).
fcsph_status record_isph_step(fcsph_ctx* c, const fcsph_state* s, const fcsph_step_params* prm, PersistRec* rec,
                              int with_fwd) {
  if (!c || !s || !prm || !rec) return fail(c, FCSPH_EINVAL, "record_isph_step: bad argument");
  if (c->gd.nz > 1 || c->prec.fft_prec == FCSPH_F32)
    return fail(c, FCSPH_EUNSUPPORTED, "persistent step: 2D FP64 or FP32x2 contexts only");
  if (!s->u || !s->v || !s->p || !s->fu || !s->fv) return fail(c, FCSPH_EINVAL, "record_isph_step: null state pointer");
  ActiveScope scope(c, prm->active);
  const int prof = c->prof_on;
  c->prof_on = 0;
  c->rec = rec;
  const void* uvw[3] = {s->u, s->v, s->w};
  cudaError_t e = with_fwd ? launch_col_fwd(c, c->prec.fft_prec, 2, uvw, 1, FCSPH_DIRICHLET, c->spec_in, 0) : cudaSuccess;
  fcsph_status st = e == cudaSuccess ? one_step(c, s, prm) : cuda_fail(c, e, "record step");
  c->rec = nullptr;
  c->prof_on = prof;
  return st;
}

fcsph_status fcsph_sync(fcsph_ctx* c) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_sync: null context");
  FCSPH_CK(cudaStreamSynchronize(c->stream), "sync");
  if (c->pplan) {
    int ps = 0;
    FCSPH_CK(persist_status(c->pplan, c->stream, &ps), "persistent status");
    if (ps) return fail(c, FCSPH_ETIMEOUT, "a dependency wait of the persistent step ran out");
  }
  int st = 0;
  FCSPH_CK(cudaMemcpy(&st, c->dstatus, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (st & 2) {
    cudaMemset(c->dstatus, 0, sizeof(int));
    return fail(c, FCSPH_ETIMEOUT, "a bulk-copy wait of a column pass ran out");
  }
  if (st & 1) {
    cudaMemset(c->dstatus, 0, sizeof(int));
    return fail(c, FCSPH_ENONFINITE, "non-finite value in the time-step state");
  }
  return FCSPH_OK;
}

fcsph_status fcsph_set_tracing(fcsph_ctx* c, int on) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_tracing: null context");
  c->trace_on = on ? 1 : 0;
  return FCSPH_OK;
}

fcsph_status fcsph_set_tma(fcsph_ctx* c, int on) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_tma: null context");
  c->tma = on ? 1 : 0;
  return FCSPH_OK;
}

fcsph_status fcsph_dft(int n, int nlines, int dir, int prec, const void* in, void* out, void* stream) {
  if (n < 1 || n > 65536 || nlines < 0 || (dir != -1 && dir != 1) || (prec != FCSPH_F64 && prec != FCSPH_F32 && prec != FCSPH_F32X2) || !in || !out)
    return fail(nullptr, FCSPH_EINVAL, "fcsph_dft: bad argument");
  if (nlines == 0) return FCSPH_OK;
  fcsph_ctx tmp;  // only for error reporting inside helpers
  fcsph_ctx* c = &tmp;
  Pool pool;
  std::vector<Fill> fills;
  FftPlan P = plan_for(n, &pool, &fills);
  double2* d64 = nullptr;
  float2* d32 = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  if (init_kernel_attributes() != cudaSuccess) return fail(nullptr, FCSPH_ECUDA, "fcsph_dft: kernel attributes");
  fcsph_status s = upload_pool(c, pool, fills, &d64, &d32, st);
  if (s != FCSPH_OK) {
    cudaFree(d64);
    cudaFree(d32);
    return fail(nullptr, s, c->err);
  }
  void* dff = nullptr;
  cudaError_t e = cudaSuccess;
  if (prec == FCSPH_F32X2) e = pool_ff_copy(d64, pool.re.size(), &dff);
  if (e == cudaSuccess)
    e = launch_dft_lines(n, nlines, dir, prec, in, out, st, P,
                         prec == FCSPH_F64 ? (const void*)d64 : prec == FCSPH_F32 ? (const void*)d32 : dff);
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(d64);
  cudaFree(d32);
  cudaFree(dff);
  if (e != cudaSuccess) return fail(nullptr, FCSPH_ECUDA, std::string("fcsph_dft: ") + cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(nullptr, FCSPH_ECUDA, std::string("fcsph_dft: ") + cudaGetErrorString(e2));
  return FCSPH_OK;
}

long long fcsph_launch_count(const fcsph_ctx* c) { return c ? c->launches : -1; }

static void drop_graph(fcsph_ctx* c) {
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->graph_key.clear();
  c->pplan_key.clear();  // a persistent step is recorded again with the new launch shape
}

fcsph_status fcsph_set_tiling(fcsph_ctx* c, int row_lines, int col_pairs) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_tiling: null context");
  if (row_lines < 1 || row_lines > 8 || col_pairs < 1 || col_pairs > 8)
    return fail(c, FCSPH_EINVAL, "fcsph_set_tiling: row_lines and col_pairs must be in 1..8");
  if (tiling_smem(c, row_lines, col_pairs) > tiling_smem_limit())
    return fail(c, FCSPH_EUNSUPPORTED, "fcsph_set_tiling: tiles exceed the shared memory of one CTA");
  if (row_lines != c->row_lines || col_pairs != c->col_pairs) drop_graph(c);
  c->row_lines = row_lines;
  c->col_pairs = col_pairs;
  return FCSPH_OK;
}

fcsph_status fcsph_set_cta_threads(fcsph_ctx* c, int row_threads, int col_threads) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_cta_threads: null context");
  auto ok = [](int t) { return t == 32 || t == 64 || t == 128; };
  if (!ok(row_threads) || !ok(col_threads))
    return fail(c, FCSPH_EINVAL, "fcsph_set_cta_threads: widths must be 32, 64 or 128");
  if (row_threads != c->row_threads || col_threads != c->col_threads) drop_graph(c);
  c->row_threads = row_threads;
  c->col_threads = col_threads;
  return FCSPH_OK;
}

fcsph_status fcsph_get_cta_threads(const fcsph_ctx* c, int* row_threads, int* col_threads) {
  if (!c || !row_threads || !col_threads) return fail(nullptr, FCSPH_EINVAL, "fcsph_get_cta_threads: bad argument");
  *row_threads = c->row_threads;
  *col_threads = c->col_threads;
  return FCSPH_OK;
}

fcsph_status fcsph_get_tiling(const fcsph_ctx* c, int* row_lines, int* col_pairs) {
  if (!c || !row_lines || !col_pairs) return fail(nullptr, FCSPH_EINVAL, "fcsph_get_tiling: bad argument");
  *row_lines = c->row_lines;
  *col_pairs = c->col_pairs;
  return FCSPH_OK;
}

fcsph_status fcsph_set_step_groups(fcsph_ctx* c, int groups) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_step_groups: null context");
  if (groups < 1 || groups > 16) return fail(c, FCSPH_EINVAL, "fcsph_set_step_groups: groups must be in 1..16");
  if (groups != c->groups) drop_graph(c);
  c->groups = groups;
  return FCSPH_OK;
}

fcsph_status fcsph_set_step_persistent(fcsph_ctx* c, int on) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_step_persistent: null context");
  if (on && (c->gd.nz > 1 || c->prec.fft_prec == FCSPH_F32))
    return fail(c, FCSPH_EUNSUPPORTED, "fcsph_set_step_persistent: 2D FP64 or FP32x2 contexts only");
  c->persist = on ? 1 : 0;
  if (!on && c->pplan) {
    cudaStreamSynchronize(c->stream);
    persist_destroy(c->pplan);
    c->pplan = nullptr;
    c->pplan_key.clear();
  }
  return FCSPH_OK;
}

fcsph_status fcsph_get_step_persistent(const fcsph_ctx* c, int* on) {
  if (!c || !on) return fail(nullptr, FCSPH_EINVAL, "fcsph_get_step_persistent: bad argument");
  *on = c->persist;
  return FCSPH_OK;
}

fcsph_status fcsph_get_step_groups(const fcsph_ctx* c, int* groups) {
  if (!c || !groups) return fail(nullptr, FCSPH_EINVAL, "fcsph_get_step_groups: bad argument");
  *groups = c->groups;
  return FCSPH_OK;
}

fcsph_status fcsph_autotune(fcsph_ctx* c, const fcsph_step_params* prm, int steps, double* best_ms_out) {
  if (!c || !prm || steps < 1) return fail(c, FCSPH_EINVAL, "fcsph_autotune: bad argument");
  const size_t n = field_elems(c);
  const int nf = c->gd.nz > 1 ? 7 : 5;
  double* buf = nullptr;
  FCSPH_CK(cudaMalloc((void**)&buf, nf * n * sizeof(double)), "autotune state");
  fcsph_state s{buf, buf + n, buf + 2 * n, buf + 3 * n, buf + 4 * n, nullptr, nullptr};
  if (nf == 7) {
    s.w = buf + 5 * n;
    s.fw = buf + 6 * n;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int cand[3] = {1, 2, 4};
  int best_r = c->row_lines, best_c = c->col_pairs;
  float best = -1.f;
  fcsph_status st = FCSPH_OK;
  cudaError_t e = cudaMemsetAsync(buf, 0, nf * n * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) st = cuda_fail(c, e, "autotune setup");
  // ms of `steps` steps in the context's current launch shape (after one
  // untimed step, which also captures the step graph); < 0 on failure
  auto time_steps = [&]() -> float {
    if ((st = isph_step(c, &s, 1, prm)) != FCSPH_OK) return -1.f;
    if ((e = cudaEventRecord(e0, c->stream)) != cudaSuccess) { st = cuda_fail(c, e, "autotune event"); return -1.f; }
    if ((st = isph_step(c, &s, steps, prm)) != FCSPH_OK) return -1.f;
    if ((e = cudaEventRecord(e1, c->stream)) != cudaSuccess) { st = cuda_fail(c, e, "autotune event"); return -1.f; }
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { st = cuda_fail(c, e, "autotune sync"); return -1.f; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  // The row passes and the column passes are separate kernels: their shapes
  // (lines per CTA x CTA width) are swept one family at a time, each over all
  // nine pairs, since lines per CTA and width trade against each other (two
  // lines on a 64-thread CTA fill as many warps per SM as one line on a
  // 32-thread CTA, with half the CTAs).
  int best_rt = c->row_threads, best_ct = c->col_threads;
  const int widths[3] = {32, 64, 128};
  auto try_shape = [&](int r, int cp, int rt, int ct) -> bool {
    if (tiling_smem(c, r, cp) > tiling_smem_limit()) return false;
    if ((st = fcsph_set_tiling(c, r, cp)) != FCSPH_OK) return false;
    if ((st = fcsph_set_cta_threads(c, rt, ct)) != FCSPH_OK) return false;
    const float ms = time_steps();
    if (st != FCSPH_OK) return false;
    if (best < 0.f || ms < best) {
      best = ms;
      best_r = r;
      best_c = cp;
      best_rt = rt;
      best_ct = ct;
    }
    return true;
  };
  for (int li = 0; li < 3 && st == FCSPH_OK; ++li)  // rows per CTA x row width
    for (int wi = 0; wi < 3 && st == FCSPH_OK; ++wi) try_shape(cand[li], best_c, widths[wi], best_ct);
  const int ccand[4] = {1, 2, 4, 8};  // a column pair's lines take half a row's shared memory
  auto sweep_cols = [&]() {  // column pairs per CTA x column width
    for (int li = 0; li < 4 && st == FCSPH_OK; ++li)
      for (int wi = 0; wi < 3 && st == FCSPH_OK; ++wi) try_shape(best_r, ccand[li], best_rt, widths[wi]);
    if (st == FCSPH_OK) st = fcsph_set_tiling(c, best_r, best_c);
    if (st == FCSPH_OK) st = fcsph_set_cta_threads(c, best_rt, best_ct);
  };
  // the instance groups of the step graph in the current shape
  int best_g = c->groups;
  const int gcand[6] = {1, 2, 3, 4, 6, 8};
  auto sweep_groups = [&]() {
    for (int gi = 0; gi < 6 && st == FCSPH_OK; ++gi) {
      if (gcand[gi] > c->gd.batch) continue;
      if ((st = fcsph_set_step_groups(c, gcand[gi])) != FCSPH_OK) break;
      const float ms = time_steps();
      if (st != FCSPH_OK) break;
      if (ms < best) {
        best = ms;
        best_g = gcand[gi];
      }
    }
    if (st == FCSPH_OK) st = fcsph_set_step_groups(c, best_g);
  };
  // the column shape and the groups interact (how the partial waves of one
  // group's launches overlap the next group's): two rounds of each
  for (int round = 0; round < 2 && st == FCSPH_OK; ++round) {
    sweep_cols();
    sweep_groups();
  }
  // then one persistent launch per step instead of the graph (2D FP64 / FP32x2)
  if (st == FCSPH_OK && c->gd.nz == 1 && c->prec.fft_prec != FCSPH_F32) {
    bool keep = false;
    if ((st = fcsph_set_step_persistent(c, 1)) == FCSPH_OK) {
      const float ms = time_steps();
      if (st == FCSPH_OK && ms < best) {
        best = ms;
        keep = true;
      }
    }
    // the autotuner's own state is freed below: the plan recorded for it goes
    fcsph_status st2 = fcsph_set_step_persistent(c, 0);
    if (st == FCSPH_OK) st = st2;
    if (st == FCSPH_OK && keep) st = fcsph_set_step_persistent(c, 1);
  }
  drop_graph(c);
  cudaStreamSynchronize(c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (st == FCSPH_OK && best_ms_out) *best_ms_out = best / steps;
  return st;
}

fcsph_status fcsph_set_profiling(fcsph_ctx* c, int on) {
  if (!c) return fail(nullptr, FCSPH_EINVAL, "fcsph_set_profiling: null context");
  c->prof_on = on ? 1 : 0;
  return FCSPH_OK;
}

fcsph_status fcsph_get_profile(fcsph_ctx* c, double* ms, long long* cnt, int nk) {
  if (!c || !ms || !cnt || nk < 1) return fail(c, FCSPH_EINVAL, "fcsph_get_profile: bad argument");
  FCSPH_CK(cudaStreamSynchronize(c->stream), "profile sync");
  for (auto& p : c->pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.kind] += t;
      c->prof_n[p.kind] += 1;
    }
    c->ev_free.push_back(p.a);
    c->ev_free.push_back(p.b);
  }
  c->pending.clear();
  for (int k = 0; k < nk && k < FCSPH_PROF_KINDS; ++k) {
    ms[k] = c->prof_ms[k];
    cnt[k] = c->prof_n[k];
    c->prof_ms[k] = 0;
    c->prof_n[k] = 0;
  }
  return FCSPH_OK;
}

fcsph_status fcsph_last_error(const fcsph_ctx* c, char* buf, size_t n) {
  if (!buf || n == 0) return FCSPH_EINVAL;
  std::string s;
  if (c) {
    s = c->err;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    s = g_err;
  }
  snprintf(buf, n, "%s", s.c_str());
  return FCSPH_OK;
}

}  // extern "C"
