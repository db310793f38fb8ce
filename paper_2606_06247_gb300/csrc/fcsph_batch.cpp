// Continuous batching of independent wall-bounded solves behind the C ABI
// (fcsph_batch_*).  Not part of the paper's method: a serving layer over
// isph_step.
//
// A size class (kind, n, kernel family) owns one context with `slots`
// instances, its own stream, device-resident state for every slot, per-slot
// viscosity / body force and an instance mask.  fcsph_batch_run is one
// scheduling tick: classes whose last step has finished retire the requests
// that are done (their state is copied to host memory the batch owns), queued
// requests are admitted into free slots (a new class only while the estimated
// device footprint of all classes fits the memory budget), and every class
// with occupied slots that is not in flight launches its next step (one CUDA
// graph replay) on its own stream, so classes overlap on the GPU and never
// wait for one another.  Empty slots are masked out of the step.  A slot's
// result does not depend on the other slots.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fcsph_internal.h"

namespace {

constexpr double kDt = 1e-3;
constexpr double kHOverDx = 1.3;

struct Req {
  fcsph_request r;
  int state = FCSPH_REQ_QUEUED;
  int done_steps = 0;
  double last_ms = 0.0, sum_ms = 0.0;
  int cls = -1, slot = -1;
  bool cancel = false;
  std::vector<double> u, v, w, p;
};

struct Class {
  int kind = 0, n = 0, family = 0, n_cont = 25, capacity = 0;
  fcsph_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  double *u = nullptr, *v = nullptr, *p = nullptr, *fu = nullptr, *fv = nullptr, *w = nullptr, *fw = nullptr;
  double *nu = nullptr, *fx = nullptr, *dt = nullptr;
  unsigned char* active = nullptr;
  std::vector<long long> slots;  // request id or -1
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool pending = false;
  size_t footprint = 0;
  bool d3() const { return kind == FCSPH_REQ_CHANNEL3D; }
  size_t cells() const { return d3() ? (size_t)n * n * n : (size_t)n * n; }
  int occupied() const {
    int k = 0;
    for (long long id : slots) k += id >= 0;
    return k;
  }
};

}  // namespace

struct fcsph_batch {
  int prec = FCSPH_F32X2;
  int slots = 8;
  double budget = 0;
  int n_cont = 25;  // 0: per-size choice
  std::vector<Class*> classes;
  std::deque<long long> queue;
  std::map<long long, Req> reqs;
  long long next_id = 1;
  std::string err;
  bool size_priorities = false;  // class streams prioritised by class size (fcsph_batch_set_size_priorities)
  // persistent mode: one launch steps every class (fcsph_batch_set_persistent)
  bool persistent = false;
  double wait_s = 1.0;
  bool stall_next = false;
  PersistPlan* plan = nullptr;
  long long gen = 0, plan_gen = -1;  // class-set generation and the plan's
  cudaStream_t tick_st = nullptr, cap_st = nullptr;
  cudaEvent_t tick_end = nullptr;
  bool tick_pending = false;
};

namespace {

std::mutex g_batch_err_mu;
std::string g_batch_err;

fcsph_status bfail(fcsph_batch* b, fcsph_status st, const std::string& msg) {
  if (b) {
    b->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_batch_err_mu);
    g_batch_err = msg;
  }
  return st;
}

fcsph_status bcuda(fcsph_batch* b, cudaError_t e, const char* where) {
  return bfail(b, FCSPH_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool factors_over(int m, std::initializer_list<int> primes) {
  for (int q : primes)
    while (m % q == 0) m /= q;
  return m == 1;
}

// Continuation length for n wall-normal nodes: 25 if n + 25 factors into the
// engine's register radices (2..17); else the length in [20, 40] nearest 25
// (the smaller on a tie) whose n + C is 7-smooth; else 25.
int smooth_n_cont(int n) {
  const int base = 25, lo = 20, hi = 40;
  if (factors_over(n + base, {2, 3, 5, 7, 11, 13, 17})) return base;
  for (int d = 1; d <= std::max(base - lo, hi - base); ++d)
    for (int c : {base - d, base + d})
      if (c >= lo && c <= hi && factors_over(n + c, {2, 3, 5, 7})) return c;
  return base;
}

// Time step of a request: min(1e-3, 0.25 dx^2 Re), within the explicit
// viscous limit (about 0.6 dx^2 / nu for the smoothed Laplacian at h = 1.3 dx).
double request_dt(const fcsph_request& r) {
  const double dx = 1.0 / (r.n - 1);
  return std::min(kDt, 0.25 * dx * dx * r.re);
}

// Kernel family per the paper's guidance: G4 at low Re, G8 at high Re (the
// lid cavity always G8).
int family_for(int kind, double re) {
  if (kind == FCSPH_REQ_CAVITY) return FCSPH_G8;
  return re < 625 ? FCSPH_G4 : FCSPH_G8;
}

// Device bytes of a class: state, workspace and spectra per slot (2D: 5 + 6
// fields and 8 spectra; 3D: 7 + 7 fields and 15 spectra).
size_t footprint(int kind, int n, int capacity, int prec, int n_cont) {
  const size_t my = n + n_cont, hy = my / 2 + 1, rows = std::max<size_t>(hy, n);
  const size_t cb = prec == FCSPH_F32 ? 8 : 16;
  const bool d3 = kind == FCSPH_REQ_CHANNEL3D;
  const size_t ncol = d3 ? (size_t)n * n : n;
  const size_t fields = d3 ? 14 : 11, specs = d3 ? 15 : 8;
  return (size_t)capacity * (fields * ncol * n * 8 + specs * rows * ncol * cb + rows * ncol * 16);
}

void destroy_class(Class* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->ctx) fcsph_destroy(c->ctx);
  for (void* p : {(void*)c->u, (void*)c->v, (void*)c->p, (void*)c->fu, (void*)c->fv, (void*)c->w, (void*)c->fw,
                  (void*)c->nu, (void*)c->fx, (void*)c->dt, (void*)c->active})
    if (p) cudaFree(p);
  if (c->e0) cudaEventDestroy(c->e0);
  if (c->e1) cudaEventDestroy(c->e1);
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

fcsph_status create_class(fcsph_batch* b, int kind, int n, int family, Class** out) {
  Class* c = new Class();
  c->kind = kind;
  c->n = n;
  c->family = family;
  c->capacity = b->slots;
  c->n_cont = b->n_cont > 0 ? b->n_cont : smooth_n_cont(n);
  c->footprint = footprint(kind, n, b->slots, b->prec, c->n_cont);
  c->slots.assign(b->slots, -1);
  auto cleanup = [&](fcsph_status st) {
    destroy_class(c);
    return st;
  };
  // with size priorities on, the classes with the most nodes per instance run
  // on the highest-priority streams (their steps are the longest, and set the
  // tail of the step latency), the smallest on the lowest
  int prio = 0;
  if (b->size_priorities) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess) {
      const size_t cells = c->cells();
      prio = cells >= (size_t)512 * 512 ? greatest : (cells >= (size_t)256 * 256 ? (least + greatest) / 2 : least);
    }
  }
  cudaError_t e = cudaStreamCreateWithPriority(&c->st, cudaStreamNonBlocking, prio);
  if (e != cudaSuccess) return cleanup(bcuda(b, e, "fcsph_batch: stream"));
  if ((e = cudaEventCreate(&c->e0)) != cudaSuccess || (e = cudaEventCreate(&c->e1)) != cudaSuccess)
    return cleanup(bcuda(b, e, "fcsph_batch: events"));
  const double dy = 1.0 / (n - 1);
  fcsph_grid g;
  memset(&g, 0, sizeof(g));
  g.nx = n;
  g.ny = n;
  g.ly = 1.0;
  g.x_walls = kind == FCSPH_REQ_CAVITY;
  g.lx = g.x_walls ? 1.0 : n * dy;
  g.batch = b->slots;
  g.nz = c->d3() ? n : 1;
  g.lz = c->d3() ? n * dy : 0.0;
  fcsph_fc fc = {FCSPH_FC_GRAM, 5, c->n_cont, 0};
  fcsph_kernel kern = {family, kHOverDx};
  fcsph_precision pr = {b->prec, 0};
  fcsph_status st = fcsph_create(&g, &fc, &kern, &pr, nullptr, nullptr, c->st, &c->ctx);
  if (st != FCSPH_OK) {
    char buf[256];
    fcsph_last_error(nullptr, buf, sizeof(buf));
    return cleanup(bfail(b, st, std::string("fcsph_batch: class context: ") + buf));
  }
  const size_t bytes = (size_t)b->slots * c->cells() * sizeof(double);
  double** fields[7] = {&c->u, &c->v, &c->p, &c->fu, &c->fv, &c->w, &c->fw};
  for (int k = 0; k < (c->d3() ? 7 : 5); ++k) {
    if ((e = cudaMalloc(fields[k], bytes)) != cudaSuccess) return cleanup(bfail(b, FCSPH_ENOMEM, "fcsph_batch: state"));
    if ((e = cudaMemsetAsync(*fields[k], 0, bytes, c->st)) != cudaSuccess) return cleanup(bcuda(b, e, "fcsph_batch: clear"));
  }
  if (cudaMalloc(&c->nu, b->slots * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->fx, b->slots * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&c->dt, b->slots * sizeof(double)) != cudaSuccess || cudaMalloc(&c->active, b->slots) != cudaSuccess)
    return cleanup(bfail(b, FCSPH_ENOMEM, "fcsph_batch: slot parameters"));
  if ((e = cudaMemsetAsync(c->active, 0, b->slots, c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->nu, 0, b->slots * sizeof(double), c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->fx, 0, b->slots * sizeof(double), c->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->dt, 0, b->slots * sizeof(double), c->st)) != cudaSuccess)
    return cleanup(bcuda(b, e, "fcsph_batch: clear slot parameters"));
  *out = c;
  return FCSPH_OK;
}

size_t used_bytes(const fcsph_batch* b) {
  size_t s = 0;
  for (const Class* c : b->classes) s += c->footprint;
  return s;
}

int find_class(const fcsph_batch* b, int kind, int n, int family) {
  for (size_t i = 0; i < b->classes.size(); ++i) {
    const Class* c = b->classes[i];
    if (c->kind == kind && c->n == n && c->family == family) return (int)i;
  }
  return -1;
}

// Puts request r into slot s of class c: zero state, per-slot nu and body force, mask on.
fcsph_status admit(fcsph_batch* b, int ci, int s, long long id, Req& r) {
  Class* c = b->classes[ci];
  const size_t cells = c->cells();
  double* fields[7] = {c->u, c->v, c->p, c->fu, c->fv, c->w, c->fw};
  cudaError_t e;
  for (int k = 0; k < (c->d3() ? 7 : 5); ++k)
    if ((e = cudaMemsetAsync(fields[k] + (size_t)s * cells, 0, cells * sizeof(double), c->st)) != cudaSuccess)
      return bcuda(b, e, "fcsph_batch: slot clear");
  const double nu = 1.0 / r.r.re;
  const double fx = r.r.kind == FCSPH_REQ_CAVITY ? 0.0 : 8.0 * nu;
  const double dt = request_dt(r.r);
  const unsigned char one = 1;
  if ((e = cudaMemcpyAsync(c->nu + s, &nu, sizeof(double), cudaMemcpyHostToDevice, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->fx + s, &fx, sizeof(double), cudaMemcpyHostToDevice, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->dt + s, &dt, sizeof(double), cudaMemcpyHostToDevice, c->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->active + s, &one, 1, cudaMemcpyHostToDevice, c->st)) != cudaSuccess)
    return bcuda(b, e, "fcsph_batch: slot parameters");
  // the copies read host stack values: finish them before returning
  if ((e = cudaStreamSynchronize(c->st)) != cudaSuccess) return bcuda(b, e, "fcsph_batch: admit");
  c->slots[s] = id;
  r.state = FCSPH_REQ_RUNNING;
  r.cls = ci;
  r.slot = s;
  return FCSPH_OK;
}

// Frees slot s of class c (mask off; the class is not in flight).
fcsph_status release(fcsph_batch* b, Class* c, int s) {
  const unsigned char zero = 0;
  cudaError_t e = cudaMemcpyAsync(c->active + s, &zero, 1, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch: release");
  c->slots[s] = -1;
  return FCSPH_OK;
}

// Copies slot s of class c to the request's host result.
fcsph_status retire(fcsph_batch* b, Class* c, int s, Req& r) {
  const size_t cells = c->cells();
  r.u.resize(cells);
  r.v.resize(cells);
  r.p.resize(cells);
  if (c->d3()) r.w.resize(cells);
  cudaError_t e = cudaSuccess;
  const size_t off = (size_t)s * cells, bytes = cells * sizeof(double);
  if ((e = cudaMemcpyAsync(r.u.data(), c->u + off, bytes, cudaMemcpyDeviceToHost, c->st)) == cudaSuccess &&
      (e = cudaMemcpyAsync(r.v.data(), c->v + off, bytes, cudaMemcpyDeviceToHost, c->st)) == cudaSuccess &&
      (e = cudaMemcpyAsync(r.p.data(), c->p + off, bytes, cudaMemcpyDeviceToHost, c->st)) == cudaSuccess && c->d3())
    e = cudaMemcpyAsync(r.w.data(), c->w + off, bytes, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch: result copy");
  r.state = FCSPH_REQ_DONE;
  return release(b, c, s);
}

// Retires the finished step of class ci: step accounting, finished and
// cancelled requests leave their slots.
fcsph_status finish_step(fcsph_batch* b, int ci) {
  Class* c = b->classes[ci];
  float ms = 0.f;
  cudaError_t e = cudaEventElapsedTime(&ms, c->e0, c->e1);
  if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch: step time");
  c->pending = false;
  fcsph_status st = fcsph_sync(c->ctx);  // device-side status of the step (non-finite state)
  if (st != FCSPH_OK) {
    char buf[256];
    fcsph_last_error(c->ctx, buf, sizeof(buf));
    bfail(b, st, std::string("fcsph_batch: step: ") + buf);
  }
  for (int s = 0; s < c->capacity; ++s) {
    const long long id = c->slots[s];
    if (id < 0) continue;
    Req& r = b->reqs[id];
    if (r.cancel) {
      r.state = FCSPH_REQ_CANCELLED;
      fcsph_status rs = release(b, c, s);
      if (rs != FCSPH_OK) return rs;
      continue;
    }
    r.done_steps++;
    r.last_ms = ms;
    r.sum_ms += ms;
    if (r.done_steps >= r.r.steps) {
      fcsph_status rs = retire(b, c, s, r);
      if (rs != FCSPH_OK) return rs;
    }
  }
  return st;
}

// Step parameters of a class: per-slot viscosity, body force and time step,
// the slot mask, RK3.
fcsph_step_params class_params(const Class* c) {
  fcsph_step_params prm;
  memset(&prm, 0, sizeof(prm));
  prm.nu = 1e-2;
  prm.rho = 1.0;
  prm.dt = kDt;
  prm.u_top = c->kind == FCSPH_REQ_CAVITY ? 1.0 : 0.0;
  prm.scheme = FCSPH_SCHEME_RK3;
  prm.use_graph = 1;
  prm.nu_inst = c->nu;
  prm.fx_inst = c->fx;
  prm.active = c->active;
  prm.dt_inst = c->dt;
  return prm;
}

fcsph_status launch_step(fcsph_batch* b, Class* c) {
  cudaError_t e = cudaEventRecord(c->e0, c->st);
  if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch: event");
  fcsph_state s = {c->u, c->v, c->p, c->fu, c->fv, c->w, c->fw};
  fcsph_step_params prm = class_params(c);
  fcsph_status st = isph_step(c->ctx, &s, 1, &prm);
  if (st != FCSPH_OK) {
    char buf[256];
    fcsph_last_error(c->ctx, buf, sizeof(buf));
    return bfail(b, st, std::string("fcsph_batch: step launch: ") + buf);
  }
  if ((e = cudaEventRecord(c->e1, c->st)) != cudaSuccess) return bcuda(b, e, "fcsph_batch: event");
  c->pending = true;
  return FCSPH_OK;
}

// Queued requests into free slots (new classes within the budget).
fcsph_status admit_queued(fcsph_batch* b) {
  std::deque<long long> waiting;
  while (!b->queue.empty()) {
    const long long id = b->queue.front();
    b->queue.pop_front();
    Req& r = b->reqs[id];
    if (r.cancel) {
      r.state = FCSPH_REQ_CANCELLED;
      continue;
    }
    const int fam = family_for(r.r.kind, r.r.re);
    int ci = find_class(b, r.r.kind, r.r.n, fam);
    if (ci < 0) {
      const int nc = b->n_cont > 0 ? b->n_cont : smooth_n_cont(r.r.n);
      if ((double)(used_bytes(b) + footprint(r.r.kind, r.r.n, b->slots, b->prec, nc)) > b->budget) {
        waiting.push_back(id);
        continue;
      }
      Class* c = nullptr;
      fcsph_status st = create_class(b, r.r.kind, r.r.n, fam, &c);
      if (st != FCSPH_OK) {
        for (long long w : b->queue) waiting.push_back(w);
        waiting.push_front(id);
        b->queue.swap(waiting);
        return st;
      }
      b->classes.push_back(c);
      b->gen++;
      ci = (int)b->classes.size() - 1;
    }
    Class* c = b->classes[ci];
    int slot = -1;
    for (int s = 0; s < c->capacity && slot < 0; ++s)
      if (c->slots[s] < 0) slot = s;
    if (slot < 0 || c->pending) {  // a class in flight takes new requests once its step is done
      waiting.push_back(id);
      continue;
    }
    fcsph_status st = admit(b, ci, slot, id, r);
    if (st != FCSPH_OK) return st;
  }
  b->queue.swap(waiting);
  return FCSPH_OK;
}

// Drops classes with no occupied slot and no queued request of their kind.
void evict_idle(fcsph_batch* b) {
  std::vector<Class*> keep;
  for (size_t i = 0; i < b->classes.size(); ++i) {
    Class* c = b->classes[i];
    bool wanted = false;
    for (long long id : b->queue) {
      const Req& r = b->reqs[id];
      if (r.r.kind == c->kind && r.r.n == c->n && family_for(r.r.kind, r.r.re) == c->family) wanted = true;
    }
    if (!c->pending && c->occupied() == 0 && !wanted)
      destroy_class(c);
    else
      keep.push_back(c);
  }
  if (keep.size() != b->classes.size()) {
    b->classes.swap(keep);
    b->gen++;
    for (size_t i = 0; i < b->classes.size(); ++i)
      for (int s = 0; s < b->classes[i]->capacity; ++s)
        if (b->classes[i]->slots[s] >= 0) b->reqs[b->classes[i]->slots[s]].cls = (int)i;
  }
}

// Records one step of every class into a new persistent plan.
fcsph_status build_plan(fcsph_batch* b) {
  if (b->plan) {
    persist_destroy(b->plan);
    b->plan = nullptr;
  }
  b->plan = persist_create(b->prec);
  for (Class* c : b->classes) {
    PersistRec* r = persist_add_class(b->plan, c->capacity);
    fcsph_state s = {c->u, c->v, c->p, c->fu, c->fv, c->w, c->fw};
    fcsph_step_params prm = class_params(c);
    fcsph_status st = record_isph_step(c->ctx, &s, &prm, r, 1);
    if (st != FCSPH_OK) {
      char buf[256];
      fcsph_last_error(c->ctx, buf, sizeof(buf));
      return bfail(b, st, std::string("fcsph_batch: persistent step: ") + buf);
    }
  }
  std::string err;
  cudaError_t e = persist_finalize(b->plan, &err);
  if (e != cudaSuccess) return bfail(b, FCSPH_ECUDA, "fcsph_batch: " + err + ": " + cudaGetErrorString(e));
  b->plan_gen = b->gen;
  return FCSPH_OK;
}

// One tick of the persistent mode: retire the finished launch, admit, and
// step every class in one launch.
fcsph_status run_persistent(fcsph_batch* b, int block, int* in_flight) {
  fcsph_status first = FCSPH_OK;
  auto pending_count = [&]() {
    int k = 0;
    for (const Class* c : b->classes) k += c->pending;
    return k;
  };
  if (b->tick_pending) {
    cudaError_t e = block ? cudaEventSynchronize(b->tick_end) : cudaEventQuery(b->tick_end);
    if (e == cudaErrorNotReady) {
      if (in_flight) *in_flight = pending_count();
      return FCSPH_OK;
    }
    if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch_run: persistent step event");
    b->tick_pending = false;
    int ps = 0;
    if ((e = persist_status(b->plan, b->tick_st, &ps)) != cudaSuccess) return bcuda(b, e, "fcsph_batch_run: status");
    if (ps)
      first = bfail(b, FCSPH_ETIMEOUT, "fcsph_batch_run: a dependency wait of the persistent step ran out");
    for (size_t i = 0; i < b->classes.size(); ++i) {
      if (!b->classes[i]->pending) continue;
      fcsph_status st = finish_step(b, (int)i);
      if (st != FCSPH_OK && first == FCSPH_OK) first = st;
    }
  }
  fcsph_status st = admit_queued(b);
  if (st != FCSPH_OK) return st;
  if (!b->queue.empty()) {
    evict_idle(b);
    if ((st = admit_queued(b)) != FCSPH_OK) return st;
  }
  bool any = false;
  for (const Class* c : b->classes) any = any || c->occupied() > 0;
  if (any) {
    if (b->plan_gen != b->gen && (st = build_plan(b)) != FCSPH_OK) return st;
    cudaError_t e = cudaSuccess;
    for (Class* c : b->classes)
      if ((e = cudaEventRecord(c->e0, b->tick_st)) != cudaSuccess) return bcuda(b, e, "fcsph_batch: event");
    const int stall = b->stall_next ? (int)persist_items(b->plan) - 1 : -1;
    b->stall_next = false;
    e = persist_launch(b->plan, b->tick_st, b->cap_st, (long long)(b->wait_s * 1e9), stall);
    if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch: persistent launch");
    for (Class* c : b->classes) {
      if ((e = cudaEventRecord(c->e1, b->tick_st)) != cudaSuccess) return bcuda(b, e, "fcsph_batch: event");
      c->pending = c->occupied() > 0;
    }
    if ((e = cudaEventRecord(b->tick_end, b->tick_st)) != cudaSuccess) return bcuda(b, e, "fcsph_batch: event");
    b->tick_pending = true;
  }
  if (in_flight) *in_flight = pending_count();
  return first;
}

}  // namespace

extern "C" {

fcsph_status fcsph_batch_create(int prec, int slots, double mem_budget_bytes, int n_cont, fcsph_batch** out) {
  if (!out) return bfail(nullptr, FCSPH_EINVAL, "fcsph_batch_create: null output");
  *out = nullptr;
  if ((prec != FCSPH_F64 && prec != FCSPH_F32 && prec != FCSPH_F32X2) || slots < 1 || slots > 1024 || n_cont < 0 ||
      (n_cont > 0 && n_cont < 4) || n_cont > 256 || !(mem_budget_bytes >= 0))
    return bfail(nullptr, FCSPH_EINVAL, "fcsph_batch_create: bad precision, slots (1..1024), n_cont or budget");
  double budget = mem_budget_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) return bcuda(nullptr, e, "fcsph_batch_create: cudaMemGetInfo");
    budget = 0.8 * (double)fr;
  }
  fcsph_batch* b = new fcsph_batch();
  b->prec = prec;
  b->slots = slots;
  b->budget = budget;
  b->n_cont = n_cont;
  *out = b;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_destroy(fcsph_batch* b) {
  if (!b) return FCSPH_EINVAL;
  if (b->tick_st) cudaStreamSynchronize(b->tick_st);
  persist_destroy(b->plan);
  if (b->tick_end) cudaEventDestroy(b->tick_end);
  if (b->tick_st) cudaStreamDestroy(b->tick_st);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  for (Class* c : b->classes) destroy_class(c);
  delete b;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_add(fcsph_batch* b, const fcsph_request* req, long long* id) {
  if (!b || !req || !id) return bfail(b, FCSPH_EINVAL, "fcsph_batch_add: null argument");
  const bool d3 = req->kind == FCSPH_REQ_CHANNEL3D;
  if (req->kind < FCSPH_REQ_CAVITY || req->kind > FCSPH_REQ_CHANNEL3D || req->n < 16 || req->n > (d3 ? 256 : 4096) ||
      !(req->re > 0) || req->steps < 1)
    return bfail(b, FCSPH_EINVAL, "fcsph_batch_add: kind, n (16..4096; 3D 16..256), re > 0, steps >= 1");
  if (d3 && b->persistent)
    return bfail(b, FCSPH_EUNSUPPORTED, "fcsph_batch_add: the persistent step runs 2D requests only");
  const long long k = b->next_id++;
  Req r;
  r.r = *req;
  b->reqs[k] = r;
  b->queue.push_back(k);
  *id = k;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_remove(fcsph_batch* b, long long id) {
  if (!b) return FCSPH_EINVAL;
  auto it = b->reqs.find(id);
  if (it == b->reqs.end()) return bfail(b, FCSPH_EINVAL, "fcsph_batch_remove: unknown request");
  Req& r = it->second;
  if (r.state == FCSPH_REQ_DONE || r.state == FCSPH_REQ_CANCELLED) return FCSPH_OK;
  r.cancel = true;
  if (r.state == FCSPH_REQ_QUEUED) {
    r.state = FCSPH_REQ_CANCELLED;
    b->queue.erase(std::remove(b->queue.begin(), b->queue.end(), id), b->queue.end());
  } else if (r.cls >= 0 && !b->classes[r.cls]->pending) {
    r.state = FCSPH_REQ_CANCELLED;
    return release(b, b->classes[r.cls], r.slot);
  }
  return FCSPH_OK;  // a request in flight leaves its slot when its class's step is done
}

fcsph_status fcsph_batch_set_persistent(fcsph_batch* b, int on, double wait_limit_s) {
  if (!b) return bfail(nullptr, FCSPH_EINVAL, "fcsph_batch_set_persistent: null batch");
  if (!(wait_limit_s > 0) || wait_limit_s > 60)
    return bfail(b, FCSPH_EINVAL, "fcsph_batch_set_persistent: wait limit must be in (0, 60] s");
  if (b->tick_pending) return bfail(b, FCSPH_EINVAL, "fcsph_batch_set_persistent: a step is in flight");
  for (const Class* c : b->classes)
    if (c->pending) return bfail(b, FCSPH_EINVAL, "fcsph_batch_set_persistent: a step is in flight");
  if (on) {
    if (b->prec == FCSPH_F32)
      return bfail(b, FCSPH_EUNSUPPORTED, "fcsph_batch_set_persistent: FP64 or FP32x2 batches only");
    for (const Class* c : b->classes)
      if (c->d3()) return bfail(b, FCSPH_EUNSUPPORTED, "fcsph_batch_set_persistent: a 3D class is open");
    for (long long id : b->queue)
      if (b->reqs[id].r.kind == FCSPH_REQ_CHANNEL3D)
        return bfail(b, FCSPH_EUNSUPPORTED, "fcsph_batch_set_persistent: a 3D request is queued");
    cudaError_t e = cudaSuccess;
    if (!b->tick_st && (e = cudaStreamCreateWithFlags(&b->tick_st, cudaStreamNonBlocking)) != cudaSuccess)
      return bcuda(b, e, "fcsph_batch_set_persistent: stream");
    if (!b->cap_st && (e = cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking)) != cudaSuccess)
      return bcuda(b, e, "fcsph_batch_set_persistent: stream");
    if (!b->tick_end && (e = cudaEventCreateWithFlags(&b->tick_end, cudaEventDisableTiming)) != cudaSuccess)
      return bcuda(b, e, "fcsph_batch_set_persistent: event");
  }
  b->persistent = on != 0;
  b->wait_s = wait_limit_s;
  b->plan_gen = -1;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_set_size_priorities(fcsph_batch* b, int on) {
  if (!b) return bfail(nullptr, FCSPH_EINVAL, "fcsph_batch_set_size_priorities: null batch");
  b->size_priorities = on != 0;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_inject_stall(fcsph_batch* b) {
  if (!b) return bfail(nullptr, FCSPH_EINVAL, "fcsph_batch_inject_stall: null batch");
  if (!b->persistent) return bfail(b, FCSPH_EINVAL, "fcsph_batch_inject_stall: persistent mode only");
  b->stall_next = true;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_run(fcsph_batch* b, int block, int* in_flight) {
  if (!b) return FCSPH_EINVAL;
  if (b->persistent) return run_persistent(b, block, in_flight);
  fcsph_status first = FCSPH_OK;
  for (size_t i = 0; i < b->classes.size(); ++i) {
    Class* c = b->classes[i];
    if (!c->pending) continue;
    cudaError_t e = block ? cudaEventSynchronize(c->e1) : cudaEventQuery(c->e1);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) return bcuda(b, e, "fcsph_batch_run: step event");
    fcsph_status st = finish_step(b, (int)i);
    if (st != FCSPH_OK && first == FCSPH_OK) first = st;
  }
  fcsph_status st = admit_queued(b);
  if (st != FCSPH_OK) return st;
  for (Class* c : b->classes)
    if (!c->pending && c->occupied() > 0 && (st = launch_step(b, c)) != FCSPH_OK) return st;
  if (!b->queue.empty()) {
    evict_idle(b);
    if ((st = admit_queued(b)) != FCSPH_OK) return st;
    for (Class* c : b->classes)
      if (!c->pending && c->occupied() > 0 && (st = launch_step(b, c)) != FCSPH_OK) return st;
  }
  if (in_flight) {
    int k = 0;
    for (const Class* c : b->classes) k += c->pending;
    *in_flight = k;
  }
  return first;
}

fcsph_status fcsph_batch_poll(fcsph_batch* b, long long id, fcsph_request_info* info) {
  if (!b || !info) return FCSPH_EINVAL;
  auto it = b->reqs.find(id);
  if (it == b->reqs.end()) return bfail(b, FCSPH_EINVAL, "fcsph_batch_poll: unknown request");
  const Req& r = it->second;
  info->state = r.state;
  info->done_steps = r.done_steps;
  info->last_step_ms = r.last_ms;
  info->total_step_ms = r.sum_ms;
  return FCSPH_OK;
}

fcsph_status fcsph_batch_result(fcsph_batch* b, long long id, double* u, double* v, double* w, double* p, size_t n_each) {
  if (!b) return FCSPH_EINVAL;
  auto it = b->reqs.find(id);
  if (it == b->reqs.end()) return bfail(b, FCSPH_EINVAL, "fcsph_batch_result: unknown request");
  const Req& r = it->second;
  if (r.state != FCSPH_REQ_DONE) return bfail(b, FCSPH_EINVAL, "fcsph_batch_result: request not finished");
  if (n_each < r.u.size()) return bfail(b, FCSPH_EINVAL, "fcsph_batch_result: output too small");
  const size_t bytes = r.u.size() * sizeof(double);
  if (u) memcpy(u, r.u.data(), bytes);
  if (v) memcpy(v, r.v.data(), bytes);
  if (p) memcpy(p, r.p.data(), bytes);
  if (w && !r.w.empty()) memcpy(w, r.w.data(), bytes);
  return FCSPH_OK;
}

fcsph_status fcsph_batch_info(const fcsph_batch* b, int* classes, int* queued, double* used_bytes_out) {
  if (!b) return FCSPH_EINVAL;
  if (classes) *classes = (int)b->classes.size();
  if (queued) *queued = (int)b->queue.size();
  if (used_bytes_out) *used_bytes_out = (double)used_bytes(b);
  return FCSPH_OK;
}

fcsph_status fcsph_batch_last_error(const fcsph_batch* b, char* buf, size_t n) {
  if (!buf || n == 0) return FCSPH_EINVAL;
  std::string s;
  if (b) {
    s = b->err;
  } else {
    std::lock_guard<std::mutex> lk(g_batch_err_mu);
    s = g_batch_err;
  }
  snprintf(buf, n, "%s", s.c_str());
  return FCSPH_OK;
}

}  // extern "C"
