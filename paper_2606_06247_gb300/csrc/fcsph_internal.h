// Internal types shared by the host table/plan builder, the C ABI layer and
// the CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fcsph.h"

namespace fcsph {

constexpr int kMaxStages = 12;
// Largest prime factor handled by a direct Stockham stage.  A prime length p
// whose p - 1 factors into such stages uses Rader's algorithm; other lengths
// with a larger prime factor go through Bluestein's chirp-z convolution.
constexpr int kMaxDirectPrime = 31;
// FP32 transform lines at least this long (shared-memory line length) get
// multi-warp CTAs by default (fcsph_set_cta_threads).
constexpr int kWideLine = 768;

// Division by a fixed d (< 2^31 dividends) as (umulhi(x, m) + x) >> l.
struct FastDiv {
  unsigned m = 1;
  int l = 0;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  int l = 0;
  while ((1ull << l) < d) ++l;
  f.l = l;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  return f;
}

// One Stockham decomposition n = radix[0] * radix[1] * ...; `tw` is the offset
// (in complex elements) of the n roots exp(-2 pi i e / n), e < n, in the pool.
// dnb[s], dns[s]: reciprocals of n/radix[s] and of Ns (product of the radices
// before stage s); dn: reciprocal of n.
struct Plan1 {
  int n = 0;
  int nst = 0;
  int tw = 0;
  int radix[kMaxStages] = {0};
  FastDiv dnb[kMaxStages];
  FastDiv dns[kMaxStages];
  FastDiv dn;
};
// Fills n, nst, radix, dnb, dns, dn from an ordered radix list.
inline void plan_set_radices(Plan1* p, int n, const int* rad, int nr) {
  p->n = n;
  p->nst = nr;
  p->dn = make_fastdiv((unsigned)n);
  int ns = 1;
  for (int i = 0; i < nr; ++i) {
    p->radix[i] = rad[i];
    p->dnb[i] = make_fastdiv((unsigned)(n / rad[i]));
    p->dns[i] = make_fastdiv((unsigned)ns);
    ns *= rad[i];
  }
}

// A length-n complex DFT: direct (bs = rd = 0, `base` holds the stages),
// Bluestein (bs = 1: base.n = n; `sub` is the smooth length-m plan; `chirp`
// holds exp(i pi j^2 / n), j < n; `bhat` holds FFT_m(b)/m of the chirp
// filter), or Rader for a prime n whose n - 1 factors directly (rd = 1: `sub`
// has length n - 1; `gidx[q]` = g^q mod n and `sidx[q]` = g^-q mod n for a
// primitive root g, stored as the real parts of pool entries; `bhat` holds
// FFT_{n-1}(b)/(n-1) of b_s = exp(-2 pi i g^-s / n)).
struct FftPlan {
  Plan1 base;
  int bs = 0;
  int rd = 0;
  Plan1 sub;
  int chirp = 0;
  int bhat = 0;
  int gidx = 0;
  int sidx = 0;
  // smem line length: Rader keeps x_0 and the sum term in two extra slots
  int line_len() const { return rd ? base.n + 2 : (bs ? sub.n : base.n); }
};

// Host-side twiddle/chirp pool (FP64 master, FP32 copy made at upload).
struct Pool {
  std::vector<double> re, im;
  int add(const std::vector<double>& r, const std::vector<double>& i) {
    int off = (int)re.size();
    re.insert(re.end(), r.begin(), r.end());
    im.insert(im.end(), i.begin(), i.end());
    return off;
  }
};

// Host builders (fcsph_tables.cpp).
bool factor_direct(int n, Plan1* p);
int smooth_at_least(int n);
// Builds the plan; Bluestein filters that need an FFT are left for the caller
// (bhat_src gets the length-m filter b in natural order, zero-padded).
FftPlan make_plan(int n, Pool* pool, std::vector<double>* bhat_src_re, std::vector<double>* bhat_src_im);
int fc_table_build(const fcsph_fc* fc, int bc, std::vector<double>* E, std::string* err);
std::vector<double> gauss_axis(int m, double d, double h, int count);
std::vector<double> what_table(const std::vector<double>& ex, const std::vector<double>& ey,
                               const std::vector<double>& ez, int mx, int my, int nz, int hy, double dx, double dy,
                               double dz, double h, int family);

}  // namespace fcsph

// Operator descriptors for the spectral row pass: output o is
// sum_{t < nterm[o]} symbol(op[o][t]) * spectrum(field[o][t]).
enum { SYM_W = 0, SYM_DX = 1, SYM_DY = 2, SYM_LAP = 3, SYM_DZ = 4,
       // Leray projection on the extended grid (spectral_project): 1, and
       // -gx^2/|g|^2, -gx gy/|g|^2, -gy^2/|g|^2 with g the gradient symbols'
       // wavevector (each component zero on its own Nyquist line), 0 where g = 0
       SYM_ONE = 5, SYM_NPXX = 6, SYM_NPXY = 7, SYM_NPYY = 8 };
constexpr int kMaxRowOut = 12;   // 3D momentum: 3 components x (3 gradients + Laplacian)
constexpr int kMaxRowTerms = 3;  // 3D divergence
struct RowOps {
  int nin;               // input spectra per instance
  int nout;              // output spectra per instance
  int nterm[kMaxRowOut];
  int field[kMaxRowOut][kMaxRowTerms];
  int op[kMaxRowOut][kMaxRowTerms];
};

// Everything a kernel needs about the grid and the method's constants.
struct GridDev {
  int nx, ny, batch, x_walls;
  // 3D channel: nz > 1 z nodes (periodic); every (x, z) pair is a wall-normal
  // column, ncol = nx * nz per instance (ncol = nx, nz = 1 in 2D)
  int nz, ncol;
  double dz;
  int ez_off, lz2_off;   // pool offsets: exp(-kz^2 h^2/4) and lam_z^2, index < nz
  int mx, my, hy;        // extended lengths, y half-spectrum rows
  int n_match, n_cont;
  int rows;              // spectrum rows allocated per field (max(hy, ny))
  double dx, dy, lx, ly, h;
  int family;
  // pool offsets of exp(-kx^2 h^2/4), kx index < mx, and exp(-ky^2 h^2/4),
  // ky < hy (real parts): the symbol's Gaussian factor is their product
  int ex_off, ey_off;
  // pool offsets of the PPE eigenvalues lam_k^2 (k < nx) and lam_l^2 (l < ny)
  int lx2_off, ly2_off;
  // isph_step only: device [batch] flags, instance b is advanced where
  // active[b] != 0 (null: every instance); null outside isph_step
  const unsigned char* active = nullptr;
  // Instances b0 .. b0 + nb - 1 are the ones a launch covers (grid dimension
  // nb, instance index b0 + block index).  isph_step captures the batch as
  // several such groups on parallel branches of its graph; every other call
  // covers the whole batch (b0 = 0, nb = batch).
  int b0 = 0, nb = 0;
  // FP32 constants of the register passes, computed once on the host in FP64
  // and rounded (the same values the kernels would get, without per-thread
  // FP64 divisions): 2 pi / (mx dx), 2 pi / (my dy), 2 pi / (nz dz), h^2 / 4, 1 / my
  float ckx_f = 0.f, cky_f = 0.f, ckz_f = 0.f, hh_f = 0.f, inv_my_f = 0.f;
  // the same in FP64, for the kernels of every precision
  double ckx_d = 0.0, cky_d = 0.0, ckz_d = 0.0, hh_d = 0.0;
};

// CTAs of an instance left out of the step return at once (uniform per CTA,
// before any barrier).
__host__ __device__ inline bool inactive(const GridDev& g, int b) { return g.active && !g.active[b]; }

struct StepDev {
  double nu, rho, dt, fx, fy, fz, u_bottom, u_top;
  double a, g, z;        // substep coefficients
  const double* nu_inst; // per-instance overrides (device) or null
  const double* fx_inst;
  const double* dt_inst; // per-instance time step (device) or null
};

// A recording of isph_step passes (fcsph_kernels.cu) and a persistent
// multi-class step built from such recordings.
struct PersistRec;
struct PersistPlan;

struct fcsph_ctx {
  fcsph_grid grid;
  fcsph_fc fc;
  fcsph_kernel kern;
  fcsph_precision prec;
  GridDev gd;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  fcsph::FftPlan plan_y, plan_x, plan_py, plan_px;  // FC-y, FC/periodic-x, PPE-y (DCT), PPE-x
  fcsph::FftPlan plan_z;                            // 3D: periodic z (operators and PPE)
  double* dE = nullptr;         // device [2][n_cont][2 n_match] (Dirichlet, Neumann)
  void* dEff = nullptr;         // the same in FP32 pairs (FP32x2 contexts)
  void* dW = nullptr;           // W_hat on the extended grid, [hy * nz][mx], in the transform type
  int row_lines = 1;            // rows per CTA of the row passes
  int col_pairs = 1;            // column pairs per CTA of the column passes
  int row_threads = 32;         // CTA width of the row (and z) passes: 32, 64 or 128
  int col_threads = 32;         // CTA width of the column passes
  int groups = 1;               // instance groups of the isph_step graph (parallel branches)
  PersistRec* rec = nullptr;    // set: the step's launchers record pass descriptors instead of launching
  int persist = 0;              // isph_step (use_graph = 1) as one persistent launch per step
  int tma = 1;                  // FP32 column passes stage their loads with bulk async copies (TMA)
  PersistPlan* pplan = nullptr; // its plan, valid for pplan_key
  std::vector<double> pplan_key;
  std::vector<cudaStream_t> grp_streams;  // one capture stream per group
  std::vector<cudaEvent_t> grp_events;    // fork event + one join event per group
  std::vector<double> hE[2];    // host copies
  double2* pool64 = nullptr;
  float2* pool32 = nullptr;
  void* poolff = nullptr;       // FP32x2 copy of the pool (hi, lo per component)
  void* spec_in = nullptr;      // [batch][2][rows][nx] complex (T)
  void* spec_out = nullptr;     // [batch][6][rows][nx] complex (T)
  void* spec_ppe = nullptr;     // [batch][rows][nx] complex (T) scratch for PPE refinement
  double* work = nullptr;       // 6 real double fields: u*, v*, b, phi_tmp, r, delta
  void* io_tmp = nullptr;       // scratch for F32 PPE refinement (float fields)
  double* dred = nullptr;       // reduction scratch
  int* dstatus = nullptr;       // device status word (bit 0: non-finite state)
  long long launches = 0;
  std::string err;
  // CUDA graph of one isph step, valid for `graph_key`
  cudaGraphExec_t gexec = nullptr;
  std::vector<double> graph_key;
  long long graph_kernels = 0;  // kernels in one replay of the step graph
  // per-kind event timing (eager launches only)
  int prof_on = 0;
  int trace_on = 0;             // NVTX ranges around every call and pass
  std::vector<cudaEvent_t> ev_free;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double prof_ms[FCSPH_PROF_KINDS] = {0};
  long long prof_n[FCSPH_PROF_KINDS] = {0};
};

// Records an event pair around one launch when profiling is on.
struct ProfScope {
  fcsph_ctx* c;
  int kind;
  cudaEvent_t b = nullptr;
  bool traced = false;
  ProfScope(fcsph_ctx* ctx, int k);
  ~ProfScope();
};

// Raises every kernel's dynamic shared-memory limit (called before any capture).
cudaError_t init_kernel_attributes();

// Kernel launchers (fcsph_kernels.cu); return cudaGetLastError().
cudaError_t launch_fc_extend(fcsph_ctx* c, const void* f, void* fext, int bc);
cudaError_t launch_col_fwd(fcsph_ctx* c, int prec, int nf, const void* const* fields, int fields_double, int bc,
                           void* spec, int dct);
size_t tiling_smem(const fcsph_ctx* c, int row_lines, int col_pairs);
size_t tiling_smem_limit();
cudaError_t launch_line_op(fcsph_ctx* c, const void* f, const int* ops, int nout, int bc, void* const* outs);
cudaError_t launch_row_sym(fcsph_ctx* c, int prec, const void* spec_in, void* spec_out, const RowOps& ops,
                           double scale, int bc, int kind);
cudaError_t launch_col_out(fcsph_ctx* c, const void* spec, int nout, void* const* outs);
cudaError_t launch_row_ppe(fcsph_ctx* c, int prec, void* spec, int apply);
cudaError_t launch_col_ppe_inv(fcsph_ctx* c, int prec, const void* spec, void* phi, int phi_double, double* phi64,
                               int mode, const double* rhs, int neumann_fwd, void* spec_fwd);
cudaError_t launch_step_mom(fcsph_ctx* c, const StepDev& s, const void* spec_mom, const double* const* vel,
                            double* const* Fp, double* const* vs, void* spec_next);
cudaError_t launch_step_div(fcsph_ctx* c, const StepDev& s, const void* spec1, double* b, void* spec_dct);
cudaError_t launch_step_corr(fcsph_ctx* c, const StepDev& s, const void* spec_grad, double* const* vs,
                             double* const* vo, void* spec_next);
cudaError_t launch_zpass(fcsph_ctx* c, int prec, void* spec, int nf, size_t bstride, int rows_used, int inv);
cudaError_t launch_dft_lines(int n, int nlines, int dir, int prec, const void* in, void* out, cudaStream_t st,
                             const fcsph::FftPlan& plan, const void* pool);
// Dynamic shared memory launch_dft_lines asks for with this plan and precision,
// and the most any CTA may have; a launch beyond it fails.
size_t dft_lines_smem(int prec, const fcsph::FftPlan& plan);
size_t dft_smem_max();
// Text returned by fcsph_last_error(NULL, ...) (context-free calls).
void set_global_error(const std::string& msg);
// out2[0] = sum over instances of sum (r - instance mean)^2, out2[1] = sum b^2
cudaError_t launch_resid_norm(fcsph_ctx* c, const double* r, const double* b, double* out2);
cudaError_t launch_axpy(fcsph_ctx* c, double* y, const double* x, const float* xf, int n, double a);
cudaError_t launch_sub(fcsph_ctx* c, double* r, const double* b, const double* lb, int n);
cudaError_t launch_narrow(fcsph_ctx* c, float* y, const double* x, int n);

// Persistent multi-class step (fcsph_kernels.cu).  persist_add_class returns
// a recording owned by the plan; record_isph_step (fcsph_api.cpp) records one
// step of a context into it; persist_finalize builds the work list on the
// device; persist_launch enqueues one launch on st (cap: an idle stream for
// the graph capture); persist_status reads and clears the status word (bit 1:
// a dependency wait ran out).
PersistPlan* persist_create(int prec);
void persist_destroy(PersistPlan* p);
PersistRec* persist_add_class(PersistPlan* p, int instances);
cudaError_t persist_finalize(PersistPlan* p, std::string* err);
cudaError_t persist_launch(PersistPlan* p, cudaStream_t st, cudaStream_t cap, long long wait_ns, int stall);
cudaError_t persist_status(PersistPlan* p, cudaStream_t st, int* status);
long long persist_items(const PersistPlan* p);
int persist_grid(const PersistPlan* p);
extern "C" fcsph_status record_isph_step(fcsph_ctx* c, const fcsph_state* s, const fcsph_step_params* prm,
                                         PersistRec* rec, int with_fwd);
