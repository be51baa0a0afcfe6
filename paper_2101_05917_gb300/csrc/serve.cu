// Serving of rollout-plus-gradient requests on one GPU (see diffpd.h).
//
// Each request is the paper's differentiable simulation end to end: a forward
// rollout of T implicit-Euler steps solved by PD + L-BFGS (Alg. 1, Sec. 4), the
// loss L = sum(loss_w * x_T), and the backward pass (Alg. 2 per step, Sec. 4.3)
// to dL/dv0 and dL/dact.  The server adds no arithmetic of its own: every step
// runs through the public entry points pd_create_mesh / pd_factorize /
// pd_forward / pd_backward on the slot's stream.
//
// Continuous admission: worker slots take requests first-in first-out as soon as
// they are free and the request's device-memory estimate fits in the budget next
// to the running ones; there is no batch boundary, so a short request never waits
// for a long one to finish.  The kernels of the running requests interleave on the
// GPU (one non-blocking stream per slot); the persistent solve of each request is
// capped at its share of the resident CTAs so that the solves of several requests
// run side by side instead of queueing behind one another.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "pd_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// Cache keys for geometry and factor inputs: the full byte string of the inputs
// plus its FNV-1a hash; a lookup compares the hash first and then every byte, so
// two different inputs never share a cache entry.
struct Hasher {
  uint64_t h = 1469598103934665603ull;
  std::vector<unsigned char> key;
  void bytes(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    key.insert(key.end(), c, c + n);
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
  bool same(uint64_t hash, const std::vector<unsigned char>& k) const { return hash == h && k == key; }
  template <typename T>
  void pod(const T& v) {
    bytes(&v, sizeof(T));
  }
  template <typename T>
  void vec(const std::vector<T>& v) {
    pod(v.size());
    if (!v.empty()) bytes(v.data(), sizeof(T) * v.size());
  }
};

// an owned copy of a pd_request
struct Job {
  uint64_t ticket = 0;
  int32_t nx = 0, ny = 0, nz = 0;
  double dx = 0, origin[3] = {0, 0, 0}, density = 0;
  std::vector<uint8_t> mask, dirichlet, contact;
  std::vector<double> wc, wv, wm, fiber;
  double h = 0, gravity[3] = {0, 0, 0}, k_contact = 0, mu = 0;
  int32_t precision = PD_PREC_FP64;
  int32_t T = 0;
  std::vector<double> x0, v0, fext, act, loss_w;
  pd_solver_opts opts{};
  int64_t n = 0, e = 0;   // kept nodes / cells
  size_t est_bytes = 0;
  Clock::time_point t_submit;
};

struct Done {
  pd_result r{};
  std::vector<double> x_final, g_v0, g_act;
};

// device buffer that only grows
struct DevBuf {
  double* p = nullptr;
  size_t cap = 0;
  cudaError_t reserve(size_t count) {
    if (count <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)&p, sizeof(double) * std::max<size_t>(count, 1));
    if (e == cudaSuccess) cap = count;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct CachedMesh {
  uint64_t geom = 0;
  std::vector<unsigned char> geom_key;
  uint64_t factor = 0;   // 0 = not factorised
  std::vector<unsigned char> factor_key;
  pd_mesh mesh = nullptr;
};

constexpr size_t kMeshCache = 8;   // meshes kept per slot (least recently used evicted)

struct Slot {
  int id = 0;
  std::thread th;
  cudaStream_t stream = nullptr;
  std::list<CachedMesh> cache;   // front = most recent
  DevBuf x0, v0, fext, act, xs, vs, dldx, gv0, gact, wc, wv, wm, fib;
};

}  // namespace

struct pd_server_s {
  int device = 0;
  size_t budget = 0;
  int solve_share = 0;   // persistent-solve CTAs per request
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Job>> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Done>> done;
  std::unordered_set<uint64_t> active;   // tickets queued or running
  size_t mem_running = 0;
  int running = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::vector<std::unique_ptr<Slot>> slots;
};

namespace {

// Device memory of one running request, estimated from its node and cell counts:
// the factor panels (FP64, FP32 and the FP32 solve tiles of both sweeps, about
// 8 + 4 + 9 bytes per entry) of a 3D nested-dissection ordering grow like n^(4/3);
// trajectories (T+1) x n x 3 positions and velocities; about 40 work vectors of
// 3n.  Used for admission only.
size_t estimate_bytes(const Job& j) {
  const double n = (double)j.n;
  const double panels = 21.0 * 8.0 * n * std::cbrt(n) * 4.0;
  const double traj = 2.0 * (j.T + 1.0) * 3.0 * n * 8.0;
  const double vecs = 40.0 * 3.0 * n * 8.0 + 8.0 * 24.0 * j.e + (double)j.T * j.e * 16.0;
  return (size_t)(panels + traj + vecs);
}

int64_t count_kept_nodes(const Job& j, int64_t* cells) {
  const int64_t nx = j.nx, ny = j.ny, nz = j.nz;
  if (j.mask.empty()) {
    *cells = nx * ny * nz;
    return (nx + 1) * (ny + 1) * (nz + 1);
  }
  std::vector<uint8_t> used((size_t)((nx + 1) * (ny + 1) * (nz + 1)), 0);
  int64_t c = 0;
  for (int64_t i = 0; i < nx; ++i)
    for (int64_t jj = 0; jj < ny; ++jj)
      for (int64_t k = 0; k < nz; ++k) {
        if (!j.mask[(size_t)((i * ny + jj) * nz + k)]) continue;
        ++c;
        for (int a = 0; a < 8; ++a) {
          const int64_t ii = i + (a >> 2), jb = jj + ((a >> 1) & 1), kk = k + (a & 1);
          used[(size_t)((ii * (ny + 1) + jb) * (nz + 1) + kk)] = 1;
        }
      }
  *cells = c;
  int64_t n = 0;
  for (uint8_t u : used) n += u;
  return n;
}

template <typename T>
bool copy_opt(const T* src, size_t count, std::vector<T>& dst) {
  if (!src) {
    dst.clear();
    return false;
  }
  dst.assign(src, src + count);
  return true;
}

// the slot's mesh for this geometry (created on a miss), factorised for these
// materials (refactorised when they differ from the cached factor)
pd_status prepare_mesh(pd_server s, Slot& sl, const Job& j, pd_mesh* out, int* mesh_hit, int* factor_hit) {
  Hasher g;
  g.pod(j.nx), g.pod(j.ny), g.pod(j.nz), g.pod(j.dx), g.bytes(j.origin, sizeof(j.origin)), g.pod(j.density);
  g.vec(j.mask), g.vec(j.dirichlet), g.vec(j.contact);
  Hasher f;
  f.vec(j.wc), f.vec(j.wv), f.vec(j.wm), f.vec(j.fiber);
  f.pod(j.h), f.bytes(j.gravity, sizeof(j.gravity)), f.pod(j.k_contact), f.pod(j.precision);
  const uint64_t fkey = f.h | 1ull;   // never 0
  auto it = std::find_if(sl.cache.begin(), sl.cache.end(),
                         [&](const CachedMesh& c) { return g.same(c.geom, c.geom_key); });
  *mesh_hit = it != sl.cache.end();
  if (it == sl.cache.end()) {
    pd_mesh_desc d{};
    d.nx = j.nx;
    d.ny = j.ny;
    d.nz = j.nz;
    d.dx = j.dx;
    for (int i = 0; i < 3; ++i) d.origin[i] = j.origin[i];
    d.density = j.density;
    d.cell_mask = j.mask.empty() ? nullptr : j.mask.data();
    d.dirichlet = j.dirichlet.empty() ? nullptr : j.dirichlet.data();
    d.contact = j.contact.empty() ? nullptr : j.contact.data();
    d.leaf_max = 0;
    d.device = s->device;
    pd_mesh m = nullptr;
    pd_status st = pd_create_mesh(&d, &m);
    if (st != PD_OK) return st;
    pd::limit_solve_ctas(m, s->solve_share);
    if (sl.cache.size() >= kMeshCache) {
      cudaStreamSynchronize(sl.stream);
      pd_mesh_destroy(sl.cache.back().mesh);
      sl.cache.pop_back();
    }
    sl.cache.push_front(CachedMesh{g.h, g.key, 0, {}, m});
  } else if (it != sl.cache.begin()) {
    sl.cache.splice(sl.cache.begin(), sl.cache, it);
  }
  CachedMesh& c = sl.cache.front();
  const bool fhit = c.factor == fkey && c.factor_key == f.key;
  *factor_hit = fhit;
  if (!fhit) {
    const size_t e = (size_t)j.e;
    auto up = [&](DevBuf& b, const std::vector<double>& v) -> const double* {
      if (v.empty()) return nullptr;
      if (b.reserve(v.size()) != cudaSuccess) return nullptr;
      cudaMemcpyAsync(b.p, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, sl.stream);
      return b.p;
    };
    const double* wc = up(sl.wc, j.wc);
    const double* wv = up(sl.wv, j.wv);
    const double* wm = up(sl.wm, j.wm);
    const double* fb = up(sl.fib, j.fiber);
    if ((!j.wc.empty() && !wc) || (!j.wv.empty() && !wv) || (!j.wm.empty() && !wm) ||
        (!j.fiber.empty() && !fb) || e == 0) {
      pd::set_error("serve: device allocation for the material weights failed");
      return PD_ERR_OOM;
    }
    pd_factor_opts fo{};
    fo.h = j.h;
    for (int i = 0; i < 3; ++i) fo.gravity[i] = j.gravity[i];
    fo.k_contact = j.k_contact;
    fo.precision = j.precision;
    c.factor = 0;
    c.factor_key.clear();
    pd_status st = pd_factorize(c.mesh, wc, wv, wm, fb, &fo, sl.stream);
    if (st != PD_OK) return st;
    c.factor = fkey;
    c.factor_key = std::move(f.key);
  }
  *out = c.mesh;
  return PD_OK;
}

// runs one request on the slot; fills d (status inside)
void run_job(pd_server s, Slot& sl, const Job& j, Done& d) {
  pd_result& r = d.r;
  r.n_nodes = j.n;
  r.n_elems = j.e;
  r.T = j.T;
  r.slot = sl.id;
  pd_mesh m = nullptr;
  int mesh_hit = 0, factor_hit = 0;
  pd_status st = prepare_mesh(s, sl, j, &m, &mesh_hit, &factor_hit);
  r.mesh_cached = mesh_hit;
  r.factor_cached = factor_hit;
  if (st != PD_OK) {
    r.status = st;
    return;
  }
  const size_t n3 = 3 * (size_t)j.n, T = (size_t)j.T, e = (size_t)j.e;
  auto fail = [&](cudaError_t ce) {
    pd::set_error(std::string("serve: ") + cudaGetErrorString(ce));
    r.status = ce == cudaErrorMemoryAllocation ? PD_ERR_OOM : PD_ERR_CUDA;
  };
  cudaError_t ce;
  DevBuf* bufs[] = {&sl.x0, &sl.v0, &sl.dldx, &sl.gv0};
  for (DevBuf* b : bufs)
    if ((ce = b->reserve(n3)) != cudaSuccess) return fail(ce);
  if ((ce = sl.xs.reserve((T + 1) * n3)) != cudaSuccess) return fail(ce);
  if ((ce = sl.vs.reserve((T + 1) * n3)) != cudaSuccess) return fail(ce);
  if (!j.fext.empty() && (ce = sl.fext.reserve(n3)) != cudaSuccess) return fail(ce);
  if (!j.act.empty()) {
    if ((ce = sl.act.reserve(T * e)) != cudaSuccess) return fail(ce);
    if ((ce = sl.gact.reserve(T * e)) != cudaSuccess) return fail(ce);
  }
  cudaStream_t q = sl.stream;
  cudaMemcpyAsync(sl.x0.p, j.x0.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, q);
  cudaMemcpyAsync(sl.v0.p, j.v0.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, q);
  cudaMemcpyAsync(sl.dldx.p, j.loss_w.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, q);
  const double* fext = nullptr;
  const double* act = nullptr;
  if (!j.fext.empty()) {
    cudaMemcpyAsync(sl.fext.p, j.fext.data(), sizeof(double) * n3, cudaMemcpyHostToDevice, q);
    fext = sl.fext.p;
  }
  if (!j.act.empty()) {
    cudaMemcpyAsync(sl.act.p, j.act.data(), sizeof(double) * T * e, cudaMemcpyHostToDevice, q);
    act = sl.act.p;
  }
  pd_solver_opts o = j.opts;
  o.checkpoint_every = 0;
  o.profile = 0;
  o.step_ms = nullptr;   // the request's host pointers do not outlive the submit call
  o.step_iters = nullptr;
  o.fext_per_step = 0;   // a request carries one (n,3) force for the whole rollout
  pd_stats fs{}, bs{};
  st = pd_forward(m, sl.x0.p, sl.v0.p, fext, act, j.mu, j.T, &o, sl.xs.p, sl.vs.p, &fs, q);
  r.fwd_iters = fs.fwd_iters;
  if (st != PD_OK && st != PD_ERR_NOT_CONVERGED) {
    r.status = st;
    return;
  }
  pd_status st_f = st;
  d.x_final.resize(n3);
  cudaMemcpyAsync(d.x_final.data(), sl.xs.p + T * n3, sizeof(double) * n3, cudaMemcpyDeviceToHost, q);
  st = pd_backward(m, sl.xs.p, sl.vs.p, fext, act, j.mu, j.T, sl.dldx.p, nullptr, 0, &o, nullptr, sl.gv0.p,
                   nullptr, nullptr, nullptr, nullptr, act ? sl.gact.p : nullptr, nullptr, &bs, q);
  r.bwd_iters = bs.bwd_iters;
  if (st != PD_OK && st != PD_ERR_NOT_CONVERGED) {
    r.status = st;
    return;
  }
  d.g_v0.resize(n3);
  cudaMemcpyAsync(d.g_v0.data(), sl.gv0.p, sizeof(double) * n3, cudaMemcpyDeviceToHost, q);
  if (act) {
    d.g_act.resize(T * e);
    cudaMemcpyAsync(d.g_act.data(), sl.gact.p, sizeof(double) * T * e, cudaMemcpyDeviceToHost, q);
  }
  if ((ce = cudaStreamSynchronize(q)) != cudaSuccess) return fail(ce);
  // loss in a fixed order on the host
  double loss = 0;
  for (size_t i = 0; i < n3; ++i) loss += j.loss_w[i] * d.x_final[i];
  r.loss = loss;
  r.x_final_host = d.x_final.data();
  r.g_v0_host = d.g_v0.data();
  r.g_act_host = act ? d.g_act.data() : nullptr;
  r.status = (st_f == PD_ERR_NOT_CONVERGED || st == PD_ERR_NOT_CONVERGED) ? PD_ERR_NOT_CONVERGED : PD_OK;
}

bool admissible(const pd_server s, const Job& j) {
  return s->running == 0 || s->mem_running + j.est_bytes <= s->budget;
}

void worker(pd_server s, Slot* sl) {
  cudaSetDevice(s->device);
  while (true) {
    std::unique_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || (!s->queue.empty() && admissible(s, *s->queue.front())); });
      if (s->stop) return;
      job = std::move(s->queue.front());
      s->queue.pop_front();
      s->running += 1;
      s->mem_running += job->est_bytes;
    }
    const Clock::time_point t_start = Clock::now();
    auto d = std::make_unique<Done>();
    run_job(s, *sl, *job, *d);
    const Clock::time_point t_end = Clock::now();
    d->r.queue_ms = ms_between(job->t_submit, t_start);
    d->r.latency_ms = ms_between(job->t_submit, t_end);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->running -= 1;
      s->mem_running -= job->est_bytes;
      s->done[job->ticket] = std::move(d);
      s->active.erase(job->ticket);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

pd_status validate(const pd_request* r) {
  auto bad = [](const char* m) {
    pd::set_error(std::string("pd_serve_submit: ") + m);
    return PD_ERR_INVALID_ARG;
  };
  if (!r) return bad("null request");
  if (r->nx <= 0 || r->ny <= 0 || r->nz <= 0) return bad("empty voxel box");
  if ((int64_t)r->nx * r->ny * r->nz > (int64_t)1 << 26) return bad("voxel box too large");
  if (!(r->dx > 0) || !(r->density > 0) || !(r->h > 0)) return bad("dx, density and h must be positive");
  if (r->T < 1) return bad("T must be at least 1");
  if (!r->x0_host || !r->v0_host || !r->loss_w_host) return bad("x0, v0 and loss_w are required");
  if (!r->w_corot_host && !r->w_vol_host && !r->w_muscle_host) return bad("at least one energy weight array");
  if (r->w_muscle_host && !r->fiber_host) return bad("fiber directions are required with w_muscle");
  if (r->precision != PD_PREC_FP64 && r->precision != PD_PREC_MIXED) return bad("unknown precision");
  if (r->k_contact < 0 || r->mu < 0) return bad("k_contact and mu must be non-negative");
  return PD_OK;
}

}  // namespace

extern "C" {

pd_status pd_serve_create(int32_t device, size_t mem_budget_bytes, int32_t max_slots, pd_server* out) {
  if (!out) {
    pd::set_error("pd_serve_create: null output");
    return PD_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64) {
    pd::set_error("pd_serve_create: max_slots must be in 1..64");
    return PD_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    pd::set_error("pd_serve_create: no CUDA device");
    return PD_ERR_NO_DEVICE;
  }
  if (device < 0 || device >= ndev) {
    pd::set_error("pd_serve_create: device ordinal out of range");
    return PD_ERR_INVALID_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  auto s = std::make_unique<pd_server_s>();
  s->device = device;
  s->budget = mem_budget_bytes;
  // a request's solve gets its share of the resident CTAs, at least one per SM
  // pair; the first solve of a mesh sizes it against the whole GPU otherwise
  s->solve_share = std::max(sms / 2, (sms * pd::solve_persistent_occupancy()) / max_slots);
  for (int i = 0; i < max_slots; ++i) {
    auto sl = std::make_unique<Slot>();
    sl->id = i;
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      pd::set_error("pd_serve_create: stream creation failed");
      for (auto& t : s->slots) cudaStreamDestroy(t->stream);
      cudaSetDevice(prev);
      return PD_ERR_CUDA;
    }
    s->slots.push_back(std::move(sl));
  }
  pd_server raw = s.release();
  for (auto& sl : raw->slots) sl->th = std::thread(worker, raw, sl.get());
  cudaSetDevice(prev);
  *out = raw;
  return PD_OK;
}

pd_status pd_serve_submit(pd_server s, const pd_request* r, uint64_t* ticket) {
  if (!s || !ticket) {
    pd::set_error("pd_serve_submit: null server or ticket");
    return PD_ERR_INVALID_ARG;
  }
  pd_status v = validate(r);
  if (v != PD_OK) return v;
  auto j = std::make_unique<Job>();
  j->t_submit = Clock::now();
  j->nx = r->nx;
  j->ny = r->ny;
  j->nz = r->nz;
  j->dx = r->dx;
  for (int i = 0; i < 3; ++i) j->origin[i] = r->origin[i];
  j->density = r->density;
  const size_t cells_box = (size_t)r->nx * r->ny * r->nz;
  copy_opt(r->cell_mask_host, cells_box, j->mask);
  j->n = count_kept_nodes(*j, &j->e);
  if (j->n == 0 || j->e == 0) {
    pd::set_error("pd_serve_submit: the cell mask keeps no cell");
    return PD_ERR_INVALID_ARG;
  }
  const size_t n = (size_t)j->n, e = (size_t)j->e, n3 = 3 * n;
  copy_opt(r->dirichlet_host, n, j->dirichlet);
  copy_opt(r->contact_host, n, j->contact);
  copy_opt(r->w_corot_host, e, j->wc);
  copy_opt(r->w_vol_host, e, j->wv);
  copy_opt(r->w_muscle_host, e, j->wm);
  copy_opt(r->fiber_host, 3 * e, j->fiber);
  j->h = r->h;
  for (int i = 0; i < 3; ++i) j->gravity[i] = r->gravity[i];
  j->k_contact = r->k_contact;
  j->mu = r->mu;
  j->precision = r->precision;
  j->T = r->T;
  copy_opt(r->x0_host, n3, j->x0);
  copy_opt(r->v0_host, n3, j->v0);
  copy_opt(r->f_ext_host, n3, j->fext);
  copy_opt(r->act_host, (size_t)r->T * e, j->act);
  copy_opt(r->loss_w_host, n3, j->loss_w);
  j->opts = r->opts;
  j->est_bytes = estimate_bytes(*j);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    j->ticket = s->next_ticket++;
    *ticket = j->ticket;
    s->active.insert(j->ticket);
    s->queue.push_back(std::move(j));
  }
  s->cv_work.notify_one();
  return PD_OK;
}

pd_status pd_serve_poll(pd_server s, uint64_t ticket, pd_result* out) {
  if (!s || !out) {
    pd::set_error("pd_serve_poll: null server or result");
    return PD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *out = it->second->r;
    return PD_OK;
  }
  if (s->active.count(ticket)) return PD_ERR_TIMEOUT;
  pd::set_error(ticket == 0 || ticket >= s->next_ticket ? "pd_serve_poll: unknown ticket"
                                                        : "pd_serve_poll: ticket was released");
  return PD_ERR_INVALID_ARG;
}

pd_status pd_serve_release(pd_server s, uint64_t ticket) {
  if (!s) {
    pd::set_error("pd_serve_release: null server");
    return PD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    pd::set_error("pd_serve_release: no finished request with this ticket");
    return PD_ERR_INVALID_ARG;
  }
  s->done.erase(it);
  return PD_OK;
}

pd_status pd_serve_drain(pd_server s) {
  if (!s) {
    pd::set_error("pd_serve_drain: null server");
    return PD_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->active.empty(); });
  return PD_OK;
}

void pd_serve_destroy(pd_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (const auto& j : s->queue) s->active.erase(j->ticket);
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto& sl : s->slots)
    if (sl->th.joinable()) sl->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (auto& sl : s->slots) {
    cudaStreamSynchronize(sl->stream);
    for (CachedMesh& c : sl->cache) pd_mesh_destroy(c.mesh);
    DevBuf* bufs[] = {&sl->x0, &sl->v0, &sl->fext, &sl->act, &sl->xs, &sl->vs, &sl->dldx,
                      &sl->gv0, &sl->gact, &sl->wc, &sl->wv, &sl->wm, &sl->fib};
    for (DevBuf* b : bufs) b->release();
    cudaStreamDestroy(sl->stream);
  }
  cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
