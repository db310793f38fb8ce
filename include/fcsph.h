/*
 * fcsph.h -- C ABI of the GB300 (sm_103a) hot path of the FC-based spectral
 * incompressible SPH scheme (Lin, Fourtakas & Rogers).
 *
 * One call chain per projection (sub)step (Sec. 5.2, Eqs. 5-9):
 *   FC extension of each wall-normal line (Sec. 4, Eq. 30)
 *   -> forward FFT over the extended periodic grid (Eqs. 11, 13)
 *   -> multiplication by the kernel's Fourier symbol per operator (Eq. 16)
 *      and the spectral PPE division (Eqs. 31-33)
 *   -> inverse FFT and truncation to the physical nodes (Eq. 30).
 *
 * Conventions shared by every entry point
 * --------------------------------------
 * Grid.  y always has walls on its first and last node (dy = Ly/(ny-1)).
 *   x is periodic (dx = Lx/nx, "channel") or has walls too (dx = Lx/(nx-1),
 *   "cavity").  A field is a dense array f[batch][nx][ny], y contiguous,
 *   holding `batch` independent instances of the same grid.
 * Extended grid.  my = ny + n_cont; mx = nx (periodic x) or nx + n_cont.
 * Pointers.  Every field pointer is a DEVICE pointer owned by the caller and
 *   must stay valid until the work queued on the context's stream finishes.
 *   Field element type: double when the context precision is FCSPH_F64 or
 *   FCSPH_F32X2, float when FCSPH_F32 -- except the time-stepping state of
 *   isph_step, which is always double.  Host pointers are marked "host".
 * Asynchrony.  Calls enqueue work on the stream given at fcsph_create and
 *   return; fcsph_sync waits and reports device-side errors.  No call aborts
 *   the process and no kernel traps.
 * Errors.  Every call returns an fcsph_status; on failure the context keeps
 *   a message (fcsph_last_error).  Invalid arguments are rejected before any
 *   work is queued (FCSPH_EINVAL); CUDA errors map to FCSPH_ECUDA.
 */
#ifndef FCSPH_H
#define FCSPH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FCSPH_OK = 0,
  FCSPH_EINVAL = 1,      /* bad argument or unsupported size                 */
  FCSPH_ENOMEM = 2,      /* device or host allocation failed                  */
  FCSPH_ECUDA = 3,       /* a CUDA runtime call failed                        */
  FCSPH_ETIMEOUT = 4,    /* a bounded device-side wait gave up                */
  FCSPH_ENONFINITE = 5,  /* a non-finite value reached the time-step state    */
  FCSPH_EUNSUPPORTED = 6 /* valid request the library does not implement      */
} fcsph_status;

/* arithmetic of FFTs and symbols: FP64; FP32; FP32x2 = double-float (value =
 * hi + lo, two FP32 numbers, 48-bit significand) run on the FP32 units.
 * F32X2 contexts use double fields like F64 ones. */
enum { FCSPH_F64 = 0, FCSPH_F32 = 1, FCSPH_F32X2 = 2 };
enum { FCSPH_FC_GRAM = 0, FCSPH_FC_PAPER = 1 };         /* FC table construction          */
enum { FCSPH_DIRICHLET = 0, FCSPH_NEUMANN = 1 };        /* boundary data type (Sec. 4.4)  */
enum { FCSPH_G2 = 1, FCSPH_G4 = 2, FCSPH_G6 = 3, FCSPH_G8 = 4, FCSPH_G10 = 5 }; /* Gaussian order 2n */
enum { FCSPH_OP_W = 1u, FCSPH_OP_DX = 2u, FCSPH_OP_DY = 4u, FCSPH_OP_LAP = 8u,
       FCSPH_OP_DZ = 16u };                             /* spectral_op mask (DZ: 3D grids) */
enum { FCSPH_SCHEME_FOP = 0, FCSPH_SCHEME_RK3 = 1 };    /* Sec. 2.2                       */

typedef struct {
  int nx, ny;      /* physical nodes per instance (nx >= 4, ny >= 2*n_match)    */
  double lx, ly;   /* domain lengths (see Grid above)                          */
  int x_walls;     /* 0: x periodic; 1: walls at both x ends                   */
  int batch;       /* independent instances per call (1 .. 65535)              */
  int nz;          /* 3D channel: nodes in z (periodic, like x); <= 1 = 2D     */
  double lz;       /* 3D channel: z period (dz = lz / nz)                      */
} fcsph_grid;

typedef struct {
  int variant;     /* FCSPH_FC_GRAM (default) or FCSPH_FC_PAPER                 */
  int n_match;     /* wall-adjacent points per wall (Gram: d; paper: C, Eq. 14) */
  int n_cont;      /* continuation points appended (Gram: C; paper: d, Eq. 21)  */
  int poly_deg;    /* FCSPH_FC_PAPER only: fitted degree p (Eq. 16), < n_match  */
} fcsph_fc;

typedef struct {
  int family;      /* FCSPH_G4 ... (Sec. 3.3, Appendix A)                       */
  double h_over_dx;/* smoothing length h in units of dx                         */
} fcsph_kernel;

typedef struct {
  int fft_prec;        /* FCSPH_F64 or FCSPH_F32                                 */
  int ppe_refine_iters;/* extra FP64-residual / FP32-correction PPE sweeps       */
} fcsph_precision;

typedef struct fcsph_ctx fcsph_ctx;

/* Time-stepping state of isph_step.  All device pointers to double arrays
 * [batch][nx][ny] (2D) or [batch][nx][nz][ny] (3D), owned by the caller.
 * fu, fv (fw) hold F^{k-1} between RK3 substeps (Eq. 5); their content on
 * entry is ignored at the first substep.  w, fw: 3D grids only (else NULL). */
typedef struct {
  double *u, *v;   /* velocity, updated in place                              */
  double *p;       /* out: pressure phi of the last substep (Eq. 8)           */
  double *fu, *fv; /* scratch: F^{k-1} of Eq. 5                               */
  double *w, *fw;  /* 3D: z velocity and its F^{k-1}                          */
} fcsph_state;

typedef struct {
  double nu, rho, dt;  /* viscosity, density, time step                        */
  double force_x, force_y; /* body force f of Eq. 1 (constant)                */
  double u_bottom, u_top;  /* tangential wall velocity at y = 0 and y = Ly    */
  int scheme;          /* FCSPH_SCHEME_FOP or FCSPH_SCHEME_RK3                 */
  int use_graph;       /* 1: capture one step in a CUDA graph and replay it   */
  const double* nu_inst;   /* device [batch] or NULL: per-instance viscosity (overrides nu) */
  const double* fx_inst;   /* device [batch] or NULL: per-instance body force x (overrides force_x) */
  double force_z;      /* 3D: body force in z                                  */
  /* device [batch] or NULL (every instance): instance b advances only where
   * active[b] != 0; the state of the others is not read or written (their
   * CTAs return at once).  The contents may change between calls and between
   * replays of the captured graph (the pointer is part of the graph's key).
   * Not with FP32 PPE refinement (FCSPH_EUNSUPPORTED).  Lets a batch hold
   * empty slots (serving) without computing them. */
  const unsigned char* active;
  /* device [batch] or NULL: per-instance time step (overrides dt); lets
   * instances of one grid but different viscosity each run within their own
   * explicit viscous limit */
  const double* dt_inst;
} fcsph_step_params;

/* Create a context for one grid shape: builds the FC tables (Sec. 4; FP64,
 * or quad precision for FC(Gram)), FFT plans and twiddles for every length
 * the path needs, and device workspace for `grid->batch` instances.
 *   fc_table_dir / fc_table_neu (host, nullable): caller-supplied FC tables,
 *     row-major [n_cont][2*n_match], columns = the n_match values nearest the
 *     y_max wall (in index order) then the n_match values nearest y = 0; NULL
 *     builds them.  The same table serves both axes.
 *   stream: cudaStream_t (NULL = legacy default stream).  */
fcsph_status fcsph_create(const fcsph_grid* grid, const fcsph_fc* fc, const fcsph_kernel* kernel,
                          const fcsph_precision* prec, const double* fc_table_dir,
                          const double* fc_table_neu, void* stream, fcsph_ctx** out);
fcsph_status fcsph_destroy(fcsph_ctx* ctx);

/* FC table used by a context (host out, [n_cont][2*n_match] doubles). */
fcsph_status fcsph_get_fc_table(const fcsph_ctx* ctx, int bc, double* out_host, size_t n_out);

/* Build an FC table on the host without a context (Sec. 4 / Sec. 4.5).
 * FC(Gram): the blend-to-zero trigonometric least squares solved in quad
 * precision; paper variant: Eqs. 14-29 in FP64.  out_host: [n_cont][2*n_match]. */
fcsph_status fcsph_fc_table(const fcsph_fc* fc, int bc, double* out_host, size_t n_out);

/* Eq. 30: write the FC-extended field f_ext[batch][mx][my] of f (both of the
 * context's element type).  Continuation along y for every x column, then
 * (walled x) along x for every extended y row.  bc: FCSPH_DIRICHLET/NEUMANN. */
fcsph_status fc_extend(fcsph_ctx* ctx, const void* f, void* f_ext, int bc);

/* Eqs. 11/13/16: for each bit set in op_mask (in the order W, DX, DY, LAP,
 * DZ), outs[k] receives that operator of f on the physical nodes.  outs has
 * one device pointer per set bit.  FC with the Dirichlet (bc=0) or Neumann
 * table.  3D grids (nz > 1): f and outs are [batch][nx][nz][ny], the
 * transforms run in y (FC), z and x, and DZ is allowed; 2D grids reject DZ. */
fcsph_status spectral_op(fcsph_ctx* ctx, const void* f, unsigned op_mask, int bc, void* const* outs);

/* The wall-normal operators of Eqs. 11/13/16 on independent lines: every
 * column f[b][i][0..ny) of the context's grid is one line with walls at both
 * ends, FC-extended on its own (table bc) and transformed in y only; each bit
 * of op_mask (order W, DX, DY, LAP) gives the symbol at kx = 0, i.e.
 * smoothing, 0 (DX), d/dy and d^2/dy^2 of the line.  outs as in spectral_op
 * (one device pointer per set bit, the context's I/O type).  Lines need not
 * have x neighbours: nx is only the count of lines per instance.  One kernel
 * per call; every line's FC, transforms and outputs stay on chip. */
fcsph_status line_op(fcsph_ctx* ctx, const void* f, unsigned op_mask, int bc, void* const* outs);

/* div(fx, fy) = IFFT( S_x FFT(Fx) + S_y FFT(Fy) ) on the physical nodes.
 * 2D grids only (FCSPH_EUNSUPPORTED on a 3D grid). */
fcsph_status spectral_div(fcsph_ctx* ctx, const void* fx, const void* fy, void* out);

/* The projection on the FC-extended periodic grid, the alternative to the
 * physical-domain PPE of Sec. 5.1 that Sec. 5.2 names and leaves for future
 * work.  Both components are FC-extended (Dirichlet table) and transformed;
 * with g = (kx, ky) the wavevector of the gradient symbols S_x = i kx W_hat,
 * S_y = i ky W_hat (each component zero on its own Nyquist line), every mode
 * is projected onto the null space of the extended divergence S_x U + S_y V:
 *   (U, V) <- (U, V) - g (g . (U, V)) / |g|^2     (modes with g = 0 kept),
 * i.e. phi_hat = (S_x U + S_y V)/(S_x^2 + S_y^2) and (U, V) -= (S_x, S_y) phi_hat;
 * then inverse transforms and truncation to the physical nodes.  The
 * extended field it truncates has zero discrete divergence at round-off.
 * fx, fy, out_x, out_y: [batch][nx][ny] in the context's I/O type (out may
 * not alias the inputs).  2D grids only (FCSPH_EUNSUPPORTED on a 3D grid).
 * Note: used inside a time step (truncate, reset the walls, re-extend) this
 * projection is unstable; isph_step keeps the physical-domain solve. */
fcsph_status spectral_project(fcsph_ctx* ctx, const void* fx, const void* fy, void* out_x, void* out_y);

/* Eqs. 31-33: phi with lap(phi) = rhs under the DFT(x) x DCT-I(y) (periodic x)
 * or DCT-I x DCT-I (walled x) diagonalisation; the (0,0) mode of phi is 0.
 * With ppe_refine_iters > 0 (F32 contexts) each sweep forms the residual in
 * FP64 and adds an FP32 correction.  resid_out (host, nullable): relative
 * residual ||L phi - rhs + mean mode|| / ||rhs||, computed on the device in
 * FP64 (synchronises the stream when non-NULL).  3D grids: DFT(x) x DFT(z) x
 * DCT-I(y), the (0,0,0) mode is 0 (no refinement). */
fcsph_status ppe_solve(fcsph_ctx* ctx, const void* rhs, void* phi, double* resid_out);

/* Advance `nsteps` projection steps (Eqs. 5-9; FOP = 1 substep, RK3 = 3)
 * of every instance.  Velocity uses the Dirichlet table, phi the Neumann one.
 * 3D grids advance (u, v, w): the y walls take u = u_bottom / u_top and
 * v = w = 0; state->w and state->fw are required. */
fcsph_status isph_step(fcsph_ctx* ctx, const fcsph_state* state, int nsteps, const fcsph_step_params* params);

/* Wait for the context's stream; report device-side errors (non-finite state). */
fcsph_status fcsph_sync(fcsph_ctx* ctx);

/* Batched complex DFT of `nlines` contiguous lines of length n with the
 * library's FFT engine (mixed radix Stockham / Bluestein), for testing the
 * engine.  dir = -1 forward (exp(-2 pi i k m/n)), +1 inverse (unscaled).
 * in/out: device arrays of nlines*n complex (interleaved re, im) doubles
 * (prec FCSPH_F64, or FCSPH_F32X2: double-float arithmetic, double I/O) or
 * floats (FCSPH_F32); in-place allowed. */
fcsph_status fcsph_dft(int n, int nlines, int dir, int prec, const void* in, void* out, void* stream);

/* ------------------------------------------------------------------------
 * Continuous batching of independent solves (serving).  Not part of the
 * paper's method: a scheduling layer over isph_step for many requests of
 * different sizes.  Requests are grouped into size classes (kind, n, kernel
 * family); a class owns one context of `slots` instances on its own stream,
 * with device-resident state for every slot.  The library allocates and owns
 * all device memory of the classes and copies each finished request's state
 * to host memory it owns.  A request's result does not depend on the other
 * requests in its class or in the batch (same precision: bitwise).
 *   Per request: Re -> nu = 1/Re; lid cavity on [0,1]^2 with lid speed 1
 *   (G8); channel (2D, or 3D with x and z periodic) with u_max = 1, body
 *   force 8 nu, G4 below Re 625 else G8; h = 1.3 dx; low-storage RK3 from
 *   the fluid at rest with dt = min(1e-3, 0.25 dx^2 Re) (the explicit
 *   viscous limit of the smoothed Laplacian is about 0.6 dx^2 / nu at
 *   h = 1.3 dx); FC(Gram) d = 5.
 * Not thread-safe: one batch is driven by one host thread. */
enum { FCSPH_REQ_CAVITY = 0, FCSPH_REQ_CHANNEL = 1, FCSPH_REQ_CHANNEL3D = 2 };
enum { FCSPH_REQ_QUEUED = 0, FCSPH_REQ_RUNNING = 1, FCSPH_REQ_DONE = 2, FCSPH_REQ_CANCELLED = 3 };
typedef struct {
  int kind;      /* FCSPH_REQ_CAVITY, _CHANNEL or _CHANNEL3D                    */
  int n;         /* particles per axis: n x n (3D n^3); 16..4096 (3D 16..256)   */
  double re;     /* Reynolds number, > 0                                        */
  int steps;     /* RK3 steps to run, >= 1                                      */
} fcsph_request;
typedef struct {
  int state;             /* FCSPH_REQ_*                                         */
  int done_steps;        /* steps completed                                     */
  double last_step_ms;   /* device time of its class's last step (CUDA events)  */
  double total_step_ms;  /* sum over its steps                                  */
} fcsph_request_info;
typedef struct fcsph_batch fcsph_batch;

/* prec: FCSPH_F64, FCSPH_F32 or FCSPH_F32X2.  slots: instances per size
 * class (1..1024).  mem_budget_bytes: a new class is created only while the
 * estimated device footprint of all classes stays within it (0: 80 % of the
 * device memory free at this call).  n_cont: FC continuation length of every
 * class (>= 4), or 0 for the per-size choice (25 where n + 25 has only prime
 * factors <= 17, else the length in [20, 40] nearest 25 with n + C 7-smooth).
 * Touches the device only when mem_budget_bytes is 0. */
fcsph_status fcsph_batch_create(int prec, int slots, double mem_budget_bytes, int n_cont, fcsph_batch** out);
/* Waits for every class's stream and frees all device and host memory. */
fcsph_status fcsph_batch_destroy(fcsph_batch* batch);
/* Queues a request; *id receives its handle (> 0).  No device work. */
fcsph_status fcsph_batch_add(fcsph_batch* batch, const fcsph_request* req, long long* id);
/* Cancels a request: a queued one at once, a running one when its class's
 * step in flight is done (its slot then frees); finished requests stay. */
fcsph_status fcsph_batch_remove(fcsph_batch* batch, long long id);
/* One scheduling tick: classes whose step is done (block = 1: wait for every
 * class in flight first) count the step for their occupied slots, copy the
 * finished requests' u, v (w), p to host and free their slots; queued
 * requests are admitted into free slots of classes not in flight (new
 * classes within the budget; classes with no occupied slot are dropped when
 * requests wait); every class with occupied slots that is not in flight
 * launches its next RK3 step (one graph replay) on its stream.  Returns
 * without waiting for those steps; *in_flight (nullable) receives the number
 * of classes with a step in flight.  FCSPH_ENONFINITE if a retired step
 * flagged a non-finite value (the batch stays usable). */
fcsph_status fcsph_batch_run(fcsph_batch* batch, int block, int* in_flight);
/* Persistent mode (on = 1; FP64 and FP32x2 batches of 2D requests): each
 * tick of fcsph_batch_run steps every class in ONE launch of a persistent
 * kernel (replayed from a CUDA graph) instead of one graph per class.  One RK3
 * step of every class is recorded once per set of classes as pass
 * descriptors; a work item is one CTA's share of one pass (one column pair
 * or spectrum row of one instance), and the CTAs take the items of all
 * classes pass by pass from an atomic counter.  An item waits until every
 * tile of the previous pass of its own instance is done, so the passes of
 * different instances and sizes overlap and no class runs alone.  Results
 * equal those of the per-class graphs bitwise.  Every such wait is bounded by
 * wait_limit_s (in (0, 60] seconds; and a spin count): a wait that runs out
 * makes the rest of that launch skip its items and fcsph_batch_run return
 * FCSPH_ETIMEOUT once, after which the batch stays usable (the requests of
 * that step hold undefined state).  Switching needs no step in flight;
 * on = 1 refuses FP32 batches and open 3D classes or queued 3D requests,
 * and fcsph_batch_add then refuses 3D requests (FCSPH_EUNSUPPORTED).  The
 * batching of uneven sizes is this library's serving layer; the paper has no
 * counterpart. */
fcsph_status fcsph_batch_set_persistent(fcsph_batch* batch, int on, double wait_limit_s);
/* Stream priorities by class size (on = 1; default off): classes created
 * from now on step on streams of high priority when an instance has at least
 * 512^2 nodes, middle priority from 256^2, low below, so that the longest
 * steps (which set the tail of the step latency) are scheduled first when
 * classes compete for the GPU.  Results are unchanged.  No device work. */
fcsph_status fcsph_batch_set_size_priorities(fcsph_batch* batch, int on);
/* Fault injection for tests of the bounded wait (persistent mode): in the
 * next launch the last work item waits for a count that never comes, so its
 * wait runs out after wait_limit_s.  Plants nothing on the device that could
 * fault: the wait gives up and the kernel returns. */
fcsph_status fcsph_batch_inject_stall(fcsph_batch* batch);
fcsph_status fcsph_batch_poll(fcsph_batch* batch, long long id, fcsph_request_info* info);
/* Host copies of a finished request's fields, each n_each >= n^2 (3D n^3)
 * doubles in [x][y] ([x][z][y]) order; any pointer may be NULL; w only for
 * 3D requests.  FCSPH_EINVAL unless the request is FCSPH_REQ_DONE. */
fcsph_status fcsph_batch_result(fcsph_batch* batch, long long id, double* u, double* v, double* w, double* p,
                                size_t n_each);
/* Classes alive, requests queued, estimated device bytes of the classes. */
fcsph_status fcsph_batch_info(const fcsph_batch* batch, int* classes, int* queued, double* used_bytes);
/* Message of the last failure of this batch (NULL: of fcsph_batch_create). */
fcsph_status fcsph_batch_last_error(const fcsph_batch* batch, char* buf, size_t n);

/* fcsph_dft without any allocation.  For callers that cannot allocate device
 * memory -- an application whose memory pool owns all device memory, a
 * plugin or a host thread that must not call into the CUDA allocator -- this
 * variant keeps its scratch (roots of unity, Bluestein chirp and filter) in
 * one fixed file-scope device array of FCSPH_NOALLOC_SCRATCH_BYTES per GPU
 * instead of allocating it.  The paper has no counterpart: this is a
 * deployment convenience, not part of the method.
 *   Arguments, layout and results as fcsph_dft (up to rounding of the roots,
 *   which are computed on the device), for prec FCSPH_F64 or FCSPH_F32 only
 *   (FCSPH_F32X2 returns FCSPH_EINVAL).  The caller allocates in and out.
 *   Limits: the scratch holds 24 bytes per pool entry; the pool has n entries
 *   when n factors into primes <= 31, else 2m + n (Bluestein, m the smallest
 *   2^a 3^b 5^c 7^d >= 2n - 1).  Every transform line must also fit in one
 *   CTA's 227 KB of shared memory: direct lengths n <= 7264 (FCSPH_F64) or
 *   n <= 14528 (FCSPH_F32); Bluestein m <= 7264 in both precisions (its
 *   filter is transformed in FP64), i.e. n up to about 3600.  Any other n
 *   returns FCSPH_EINVAL before anything is queued.
 *   Errors: FCSPH_ECUDA for a failed launch, or when a CUDA error from
 *   earlier work is already pending on the calling thread (reported, not
 *   cleared); fcsph_last_error(NULL, ...) gives the text.
 *   Set-up: the first call on each device, with that device current, looks
 *   up the array's device address (cudaGetSymbolAddress) and raises the
 *   kernels' shared-memory limits; neither allocates.  Make that first call
 *   before any stream capture.
 *   Sharing: all calls use the same array and every call rewrites the parts
 *   it reads, so calls whose work overlaps on the GPU race; serialise them.
 *   The array stays resident on every GPU that loaded the library until exit. */
#define FCSPH_NOALLOC_SCRATCH_BYTES (1u << 20)
fcsph_status fcsph_dft_noalloc(int n, int nlines, int dir, int prec, const void* in, void* out, void* stream);

/* Tiling of the FFT passes: row_lines rows per CTA of the x
 * passes, col_pairs column pairs per CTA of the wall-normal passes (each
 * 1..8).  More lines per CTA fill more lanes of each butterfly stage but hold
 * more shared memory, so fewer CTAs fit on an SM; the best choice depends on
 * the precision and the transform lengths.  Takes effect at the next call
 * (a captured isph_step graph is dropped).  FCSPH_EUNSUPPORTED if a CTA
 * would exceed the shared memory of an SM.  Engineering choice of this
 * library; the paper has no counterpart. */
fcsph_status fcsph_set_tiling(fcsph_ctx* ctx, int row_lines, int col_pairs);
fcsph_status fcsph_get_tiling(const fcsph_ctx* ctx, int* row_lines, int* col_pairs);

/* CTA width of the FFT passes: row_threads threads per CTA of the x (and z)
 * passes, col_threads per CTA of the wall-normal passes, each 32, 64 or 128
 * (else FCSPH_EINVAL); the threads of a CTA share its lines.  Wider CTAs
 * carry each line with more threads, which pays when a pass has too few
 * lines to fill the GPU, and hold less shared memory per warp, which pays for
 * long FP32 lines.  The result does not depend on the widths.  A context
 * starts, per pass, at 128 threads if its one-warp CTAs (rows or column pairs
 * of all instances) would fill at most a quarter of the GPU's 152 x 12, at 64
 * if at most half, else at 32; FP32 passes whose transform lines hold >= 768
 * points take at least 64 (row) and 128 (column) threads.  Takes effect at
 * the next call (a captured isph_step graph is dropped).  Engineering choice
 * of this library; the paper has no counterpart. */
fcsph_status fcsph_set_cta_threads(fcsph_ctx* ctx, int row_threads, int col_threads);
fcsph_status fcsph_get_cta_threads(const fcsph_ctx* ctx, int* row_threads, int* col_threads);

/* Instance groups of the isph_step graph (use_graph = 1): the batch is split
 * into `groups` (1..16) groups of nearly equal size whose kernels run as
 * parallel branches of the step graph, so that one group's launch fills the
 * SMs left idle by the last, partial wave of CTAs of another group's launch.
 * Results do not depend on it (each instance's arithmetic is unchanged).
 * Default 1; eager steps (use_graph = 0) and FP32 contexts with PPE
 * refinement always run one chain.  A change drops the captured graph.
 * Engineering choice of this library; the paper has no counterpart. */
fcsph_status fcsph_set_step_groups(fcsph_ctx* ctx, int groups);
fcsph_status fcsph_get_step_groups(const fcsph_ctx* ctx, int* groups);

/* Persistent step (on = 1; 2D FP64 or FP32x2 contexts, else
 * FCSPH_EUNSUPPORTED): with use_graph = 1, every step of isph_step is ONE
 * launch of a persistent kernel over the step's recorded passes instead of a
 * graph of ~25 kernels.  A work item is one CTA's share of one pass for one
 * instance; an item waits (bounded: 1 s, and a spin count) until every tile
 * of the previous pass of its own instance is done, so the passes of
 * different instances overlap and no launch ends in a partial wave.  Results
 * equal the graph's bitwise.  A wait that runs out makes the rest of that
 * launch skip its items and the next fcsph_sync return FCSPH_ETIMEOUT once.
 * The recording is redone when isph_step's pointers or parameters change.
 * Engineering choice of this library; the paper has no counterpart. */
fcsph_status fcsph_set_step_persistent(fcsph_ctx* ctx, int on);

/* TMA staging (on = 1, the default) of the FP32 register column passes
 * (extended wall-normal lengths 540 and 1050): the output pass gathers each
 * column pair's half-spectrum rows with 2D tiled bulk copies
 * (cp.async.bulk.tensor) one unit ahead of its inverse transform; on = 0
 * keeps the per-thread loads.  Needs an even number of columns and no
 * instance mask, else the per-thread path runs.  A copy whose wait runs out
 * (bounded) makes fcsph_sync return FCSPH_ETIMEOUT.  Results are identical
 * either way.  Engineering choice of this library; the paper has no
 * counterpart. */
fcsph_status fcsph_set_tma(fcsph_ctx* ctx, int on);

/* Tracing (on = 1; default off): NVTX ranges ("fcsph <call>" around every
 * call of this header that takes the context, "fcsph <pass>" around every
 * kernel launch, named as the FCSPH_PROF_* kinds) for a profiler's timeline
 * or for ncu --nvtx filters.  Host-side markers only: they cost nothing on
 * the device, and nothing at all unless a tool is attached.  Engineering
 * aid of this library; the paper has no counterpart. */
fcsph_status fcsph_set_tracing(fcsph_ctx* ctx, int on);
fcsph_status fcsph_get_step_persistent(const fcsph_ctx* ctx, int* on);

/* Autotuner: times `steps` isph_step calls with *prm on a zero state the
 * call allocates and frees (2D: 5 fields of the context's batch, 3D: 7).
 * First the row-pass shape: every rows-per-CTA in {1, 2, 4} with every row
 * CTA width in {32, 64, 128}, keeping the fastest; then the column-pass shape
 * the same way (column pairs per CTA in {1, 2, 4, 8} x column CTA width);
 * shapes whose shared memory does not fit are skipped.  Then the instance
 * groups 1, 2, 3, 4, 6, 8 (at most the batch) of the step graph in that
 * shape, keeping the fastest; the column sweep and the groups sweep then run
 * once more at the chosen groups; then
 * (2D FP64 / FP32x2) the persistent step, kept if faster still.  best_ms_out
 * (nullable, host): its milliseconds per step.
 * Synchronises the context's stream.  Engineering choice of this library;
 * the paper has no counterpart. */
fcsph_status fcsph_autotune(fcsph_ctx* ctx, const fcsph_step_params* prm, int steps, double* best_ms_out);

/* Kernel launches this context has queued since creation (for bookkeeping). */
long long fcsph_launch_count(const fcsph_ctx* ctx);

/* Per-kernel timing with CUDA events recorded on the context's stream around
 * every launch (eager launches only; isph_step with use_graph = 0).  Kinds:
 * FCSPH_PROF_* below.  fcsph_get_profile synchronises the stream, returns the
 * summed milliseconds and launch counts per kind since the last call (arrays
 * of n_kinds entries, host) and resets them. */
enum {
  FCSPH_PROF_COL_FWD = 0,   /* FC (or DCT) + forward FFT of wall-normal lines     */
  FCSPH_PROF_ROW_MOM = 1,   /* x pass: 2 spectra -> 6 (grad, lap of u and v)      */
  FCSPH_PROF_ROW_DIV = 2,   /* x pass: 2 spectra -> divergence                    */
  FCSPH_PROF_ROW_GRAD = 3,  /* x pass: phi spectrum -> grad phi                   */
  FCSPH_PROF_ROW_OP = 4,    /* x pass of spectral_op / spectral_div               */
  FCSPH_PROF_COL_MOM = 5,   /* inverse + momentum update + forward of u*, v*      */
  FCSPH_PROF_COL_DIV = 6,   /* inverse + PPE right-hand side + DCT forward        */
  FCSPH_PROF_COL_CORR = 7,  /* inverse + projection + forward of u, v             */
  FCSPH_PROF_COL_OUT = 8,   /* inverse + store (spectral_op / spectral_div)       */
  FCSPH_PROF_ROW_PPE = 9,   /* PPE x transform, division, inverse                 */
  FCSPH_PROF_COL_PPE = 10,  /* PPE inverse DCT (+ Neumann FC forward of phi)      */
  FCSPH_PROF_OTHER = 11,    /* fc_extend, reductions, conversions                 */
  FCSPH_PROF_KINDS = 12
};
fcsph_status fcsph_set_profiling(fcsph_ctx* ctx, int on);
fcsph_status fcsph_get_profile(fcsph_ctx* ctx, double* ms_out, long long* count_out, int n_kinds);

/* Copy the last error message of ctx (or of context-free calls if ctx is NULL). */
fcsph_status fcsph_last_error(const fcsph_ctx* ctx, char* buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* FCSPH_H */
