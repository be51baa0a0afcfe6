// C ABI of the differentiable PD solver and the host orchestration of the
// forward rollout (Alg. 1 + L-BFGS) and the backward rollout (Alg. 2 + L-BFGS).
// The host only launches kernels and polls one device flag per batch of
// iterations; every numerical decision is taken on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pd_internal.cuh"
#include "pd_vec.cuh"

namespace pd {

namespace {
thread_local std::string g_last_error;

template <typename T>
cudaError_t dalloc(MeshImpl* m, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
  if (e == cudaSuccess) {
    m->allocations.emplace_back((void*)*p, sizeof(T) * count);
    m->ws.bytes += sizeof(T) * count;
  }
  return e;
}

// frees a buffer made by dalloc (null is a no-op)
template <typename T>
void dfree(MeshImpl* m, T** p) {
  if (!*p) return;
  for (size_t i = 0; i < m->allocations.size(); ++i) {
    if (m->allocations[i].first != (void*)*p) continue;
    m->ws.bytes -= m->allocations[i].second;
    m->allocations.erase(m->allocations.begin() + (std::ptrdiff_t)i);
    cudaFree((void*)*p);
    break;
  }
  *p = nullptr;
}

template <typename T, typename S>
cudaError_t upload(MeshImpl* m, T** p, const std::vector<S>& v) {
  cudaError_t e = dalloc(m, p, v.size());
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  std::vector<T> tmp(v.begin(), v.end());
  return cudaMemcpy(*p, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice);
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev >= 0) {
      cudaGetDevice(&prev);
      if (prev != dev) cudaSetDevice(dev);
    }
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4096));
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace pd

struct pd_mesh_s {
  pd::MeshImpl impl;
};

namespace pd {

void drop_iteration_graphs(MeshImpl* m);

void limit_solve_ctas(pd_mesh m, int ctas) {
  if (!m || ctas <= 0) return;
  m->impl.solve_grid = std::max(1, std::min(m->impl.solve_grid, ctas));
  drop_iteration_graphs(&m->impl);   // the graphs captured the solve's grid
}

int solve_ctas(pd_mesh m) { return m ? m->impl.solve_grid : 0; }

size_t mesh_device_bytes(pd_mesh m) { return m ? m->impl.ws.bytes : 0; }

}  // namespace pd

using namespace pd;

namespace {

// NVTX range around a call or a time step (step index as payload), for profilers
// that attribute kernels to ranges (nsys, ncu --nvtx); a no-op without a tool
struct Range {
  explicit Range(const char* name, int64_t step = -1) {
    if (step < 0) {
      nvtxRangePushA(name);
      return;
    }
    nvtxEventAttributes_t a{};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    a.payloadType = NVTX_PAYLOAD_TYPE_INT64;
    a.payload.llValue = step;
    nvtxRangePushEx(&a);
  }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

pd_status ensure_workspace(MeshImpl* m, int lbfgs_m) {
  Workspace& w = m->ws;
  const int64_t n3 = 3 * m->h.n, nf3 = 3 * m->h.nf;
  if (!w.x) {
    double** vecs[] = {&w.x, &w.xt, &w.y, &w.xprev, &w.vprev, &w.grad, &w.gradt, &w.dir, &w.q, &w.r,
                       &w.z, &w.gs, &w.Hd, &w.ax, &w.av, &w.gbar, &w.fext, &w.ffric, &w.iox, &w.iov};
    for (double** v : vecs) {
      PD_CUDA_TRY(dalloc(m, v, (size_t)n3));
      PD_CUDA_TRY(cudaMemset(*v, 0, sizeof(double) * n3));
    }
    PD_CUDA_TRY(dalloc(m, (double**)&w.elembuf, (size_t)(24 * m->h.e)));
    const int64_t np = (int64_t)element_energy_partials(m) + 4 * (int64_t)gather_blocks(m) + 4 * 4096 + 64;
    PD_CUDA_TRY(dalloc(m, &w.partials, (size_t)np));
    PD_CUDA_TRY(dalloc(m, &w.lpart, (size_t)kMaxDots * kLbfgsMaxBlocks));
    PD_CUDA_TRY(dalloc(m, &w.act_cur, (size_t)std::max<int64_t>(m->h.e, 1)));
    PD_CUDA_TRY(dalloc(m, &w.xnext_cur, (size_t)n3));
    PD_CUDA_TRY(dalloc(m, &w.counters, 16));
    PD_CUDA_TRY(cudaMemset(w.counters, 0, 16 * sizeof(unsigned)));
    PD_CUDA_TRY(dalloc(m, &w.st, 1));
    PD_CUDA_TRY(cudaMallocHost((void**)&w.st_host, sizeof(IterState)));
    PD_CUDA_TRY(dalloc(m, &w.flags, 4));
    PD_CUDA_TRY(cudaMemset(w.flags, 0, 4 * sizeof(int)));
    PD_CUDA_TRY(dalloc(m, (double**)&w.solve_u, (size_t)nf3));
  }
  if (lbfgs_m > w.lbfgs_m) {
    // history buffers grow monotonically; old ones stay in the allocation list
    PD_CUDA_TRY(dalloc(m, &w.S, (size_t)lbfgs_m * nf3));
    PD_CUDA_TRY(dalloc(m, &w.Y, (size_t)lbfgs_m * nf3));
    w.lbfgs_m = lbfgs_m;
  }
  return PD_OK;
}

// The persistent solve counts tickets and finished blocks monotonically; a fresh
// start at every public call also recovers from an aborted solve.
cudaError_t reset_solve_counters(MeshImpl* m, cudaStream_t s) {
  const size_t n = 1 + 2 * (size_t)m->h.ns + m->sched.all.size();
  return cudaMemsetAsync(m->solve_counters, 0, sizeof(unsigned long long) * n, s);
}

pd_solver_opts default_opts() {
  pd_solver_opts o{};
  o.tol_fwd = 1e-9;
  o.tol_bwd = 1e-9;
  o.max_iter_fwd = 500;
  o.max_iter_bwd = 500;
  o.lbfgs_m = 5;
  o.ls_max = 10;
  o.checkpoint_every = 0;
  o.check_every = 4;
  return o;
}

pd_solver_opts fill_opts(const pd_solver_opts* o) {
  pd_solver_opts r = o ? *o : default_opts();
  const pd_solver_opts d = default_opts();
  if (!(r.tol_fwd > 0)) r.tol_fwd = d.tol_fwd;
  if (!(r.tol_bwd > 0)) r.tol_bwd = d.tol_bwd;
  if (r.max_iter_fwd <= 0) r.max_iter_fwd = d.max_iter_fwd;
  if (r.max_iter_bwd <= 0) r.max_iter_bwd = d.max_iter_bwd;
  if (r.lbfgs_m < 0) r.lbfgs_m = 0;
  if (r.lbfgs_m > kMaxHistory) r.lbfgs_m = kMaxHistory;
  if (r.ls_max < 0) r.ls_max = 0;
  if (r.check_every <= 0) r.check_every = d.check_every;
  return r;
}

// CUDA events bracketing selected launches (profile mode); elapsed times are
// summed after the call's final synchronisation.
struct EventTimer {
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  void record(cudaStream_t s) {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    cudaEventRecord(pool[used++], s);
  }
  int64_t pairs() const { return (int64_t)(used / 2); }
  double total_ms() {   // pairs (start, end)
    double t = 0;
    for (size_t i = 0; i + 1 < used; i += 2) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, pool[i], pool[i + 1]) == cudaSuccess) t += ms;
    }
    return t;
  }
  ~EventTimer() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

struct Ctx {
  MeshImpl* m;
  int64_t launches = 0, solves = 0, locals = 0;
  int64_t bwd_steps = 0;
  int last_kind = -1;   // 0 forward, 1 backward: L-BFGS pairs carry over within a kind
  // mixed forward: steps left that start with the strain-accurate FP32 local step
  // (set when a step's plain FP32 residual stopped halving above the tolerance)
  int acc_steps = 0;
  EventTimer* solve_t = nullptr;
  int dev_flags = 0;
  EventTimer* local_t = nullptr;
  cudaStream_t s;
  pd_solver_opts o;
  int64_t n, nf, n3f;
  int vb;          // vector kernel blocks
  int mx;          // compile-time bound of the L-BFGS history (2, 4, 5, 8, 10, 16)
  int lb;          // blocks of the L-BFGS kernels: at most two per SM (one completion counter)
  bool graphs;     // replay iteration chunks as CUDA graphs
  bool complementarity = false;   // contact by the active set on the prepared candidates
  VecCtx vc;
  double* pe;      // energy partials
  double* pg;      // gather partials
  int nbe, nbg;
};

Ctx make_ctx(MeshImpl* m, cudaStream_t s, const pd_solver_opts& o) {
  Ctx c;
  c.m = m;
  c.s = s;
  c.o = o;
  c.n = m->h.n;
  c.nf = m->h.nf;
  c.n3f = 3 * m->h.nf;
  c.vb = vec_blocks(c.n3f);
  c.mx = lbfgs_bound(o.lbfgs_m);
  c.lb = std::max(1, std::min(c.vb, 2 * m->sms));
  c.graphs = !o.no_graphs;
  c.complementarity = o.complementarity != 0;
  if (c.complementarity) c.graphs = false;   // the captured launches would fix the set size
  c.vc.n3 = c.n3f;
  c.vc.st = m->ws.st;
  c.vc.partials = m->ws.partials;
  c.vc.counter = m->ws.counters;
  c.vc.lpart = m->ws.lpart;
  c.vc.lcounter = m->ws.counters + 1;
  c.nbe = element_energy_partials(m);
  c.nbg = gather_blocks(m);
  c.pe = m->ws.partials;
  c.pg = m->ws.partials + c.nbe;
  return c;
}

pd_status poll(Ctx& c) {
  PD_CUDA_TRY(cudaMemcpyAsync(c.m->ws.st_host, c.m->ws.st, sizeof(IterState), cudaMemcpyDeviceToHost, c.s));
  PD_CUDA_TRY(cudaStreamSynchronize(c.s));
  return PD_OK;
}

// runs the statement with the constant MX bound to the context's history bound
#define PD_WITH_MX(mx, ...)          \
  switch (mx) {                      \
    case 2: {                        \
      constexpr int MX = 2;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 4: {                        \
      constexpr int MX = 4;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 5: {                        \
      constexpr int MX = 5;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 8: {                        \
      constexpr int MX = 8;          \
      __VA_ARGS__;                   \
    } break;                         \
    case 10: {                       \
      constexpr int MX = 10;         \
      __VA_ARGS__;                   \
    } break;                         \
    default: {                       \
      constexpr int MX = 16;         \
      __VA_ARGS__;                   \
    } break;                         \
  }

// runs the statement with MX bound as above and H to the L-BFGS history type: float
// in mixed precision (the history buffers, allocated as doubles, hold floats then),
// double otherwise
#define PD_WITH_MX_H(c, ...)                        \
  if ((c).m->precision == PD_PREC_MIXED) {          \
    using H = float;                                \
    PD_WITH_MX((c).mx, __VA_ARGS__);                \
  } else {                                          \
    using H = double;                               \
    PD_WITH_MX((c).mx, __VA_ARGS__);                \
  }

template <typename H>
H* hist(double* p) {
  return reinterpret_cast<H*>(p);
}

// Complementarity contact: the global step of an iteration restricted to the free
// nodes outside the held set (Alg. 3 / Alg. 5 global step, computed as in
// kernels_contact.cu with zero targets: held rows of the direction stay zero).
// Idempotent, so it is harmless when the gated solve was skipped.
cudaError_t held_correction(MeshImpl* m, double* r, cudaStream_t s) {
  if (!m->held_active || m->cset == 0) return cudaSuccess;
  return contact_correct(m->h.nf, m->Bc, m->cset_node, m->cset_cand, m->cset, m->cset_Q, m->cset_S, m->cset_a,
                         m->cset_u, m->cset_lam, r, m->cset_zero, r, s);
}

// one forward iteration: evaluate the trial point, decide, commit and the
// next direction (two-loop recursion around the global solve)
pd_status launch_fwd_iteration(Ctx& c, int prec, const double* act_t) {
  MeshImpl* m = c.m;
  Workspace& w = m->ws;
  IterState* st = w.st;
  LocalArgs la{m, st, w.xt, nullptr, act_t, prec};
  // timed: the local steps of the iteration precision (not the FP64 convergence checks)
  const bool timed = c.local_t && prec == m->precision;
  if (timed) c.local_t->record(c.s);
  PD_CUDA_TRY(launch_element_forces(la, w.elembuf, c.pe, w.flags, c.s));
  if (timed) c.local_t->record(c.s);
  PD_CUDA_TRY(launch_gather_grad(m, st, w.elembuf, prec, w.xt, w.y, w.dir, w.gradt, c.pg, c.s));
  decide_fwd_kernel<<<1, 256, 0, c.s>>>(st, c.pe, c.nbe, c.pg, c.nbg);
  PD_WITH_MX_H(c, lbfgs_commit_fwd_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, w.x, w.xt, w.grad, w.gradt,
                                                                         hist<H>(w.S), hist<H>(w.Y)));
  PD_WITH_MX_H(c, lbfgs_q_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, w.grad, hist<H>(w.Y), w.q));
  if (c.solve_t) c.solve_t->record(c.s);
  PD_CUDA_TRY(solve_A(m, st, w.q, w.r, m->precision, c.s));
  if (c.solve_t) c.solve_t->record(c.s);
  PD_CUDA_TRY(held_correction(m, w.r, c.s));
  PD_WITH_MX_H(c, lbfgs_post_dots_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, w.grad, hist<H>(w.Y), w.r));
  PD_WITH_MX_H(c, lbfgs_dir_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, hist<H>(w.S), w.r, w.dir, w.x, w.xt));
  c.launches += 9;
  c.solves += 1;
  c.locals += 1;
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

// one backward iteration: apply the previous step and the two-loop recursion
// around the global solve, then the Hessian product and the line search
pd_status launch_bwd_iteration(Ctx& c, int prec, const double* xnext, const double* act_t) {
  MeshImpl* m = c.m;
  Workspace& w = m->ws;
  IterState* st = w.st;
  PD_WITH_MX_H(c, lbfgs_commit_bwd_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, w.dir, w.Hd, w.z, w.gs,
                                                                         hist<H>(w.S), hist<H>(w.Y)));
  PD_WITH_MX_H(c, lbfgs_q_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, w.gs, hist<H>(w.Y), w.q));
  if (c.solve_t) c.solve_t->record(c.s);
  PD_CUDA_TRY(solve_A(m, st, w.q, w.r, m->precision, c.s));
  if (c.solve_t) c.solve_t->record(c.s);
  PD_CUDA_TRY(held_correction(m, w.r, c.s));
  PD_WITH_MX_H(c, lbfgs_post_dots_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, w.gs, hist<H>(w.Y), w.r));
  PD_WITH_MX_H(c, lbfgs_dir_kernel<MX, H><<<c.lb, 256, 0, c.s>>>(c.vc, hist<H>(w.S), w.r, w.dir, nullptr, nullptr));
  c.launches += 9;
  c.solves += 1;
  LocalArgs la{m, st, xnext, w.dir, act_t, prec};
  PD_CUDA_TRY(launch_element_hvp(la, w.elembuf, w.flags, c.s));
  PD_CUDA_TRY(launch_gather_hvp(m, st, w.elembuf, prec, xnext, w.dir, w.gs, w.Hd, c.pg, c.s));
  decide_bwd_kernel<<<1, 256, 0, c.s>>>(st, c.pg, c.nbg);
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

// ------------------------------------------------------------ CUDA graphs
// A chunk of kGraphIters iterations is captured once per mesh, direction and
// precision (on the mesh's capture stream, so any caller stream works, the legacy
// default stream included) and replayed with one launch.  The captured launches
// read the step's inputs from fixed buffers (ws.act_cur, ws.xnext_cur) and decide
// everything else from the device-side iteration state, exactly as the direct
// launches do; the results are the same.  If a capture fails the chunk is simply
// launched directly.
constexpr int kGraphIters = 4;


}  // namespace

namespace pd {

void drop_iteration_graphs(MeshImpl* m) {
  for (auto& dir : m->iter_graph)
    for (auto& prec : dir)
      for (cudaGraphExec_t& g : prec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

}  // namespace pd

namespace {

cudaGraphExec_t iteration_graph(Ctx& c, int dir, int prec, bool with_act, int variant) {
  MeshImpl* m = c.m;
  const int pi = prec == PD_PREC_MIXED ? 1 : (prec == kPrecMixedAcc ? 2 : (prec == kPrecRefined ? 3 : 0));
  const int iters = kGraphIters - variant;
  cudaGraphExec_t& g = m->iter_graph[dir][pi][variant];
  if (g && m->iter_graph_act[dir][pi][variant] == with_act) return g;
  if (g) cudaGraphExecDestroy(g);
  g = nullptr;
  if (!m->cap_stream && cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  Ctx cc = c;
  cc.s = m->cap_stream;
  cc.solve_t = nullptr;
  cc.local_t = nullptr;
  cc.launches = cc.solves = cc.locals = 0;
  if (cudaStreamBeginCapture(cc.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  pd_status st = PD_OK;
  for (int k = 0; k < iters && st == PD_OK; ++k)
    st = dir == 0 ? launch_fwd_iteration(cc, prec, with_act ? m->ws.act_cur : nullptr)
                  : launch_bwd_iteration(cc, prec, m->ws.xnext_cur, with_act ? m->ws.act_cur : nullptr);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cc.s, &graph);
  if (st != PD_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  e = cudaGraphInstantiate(&g, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g = nullptr;
    cudaGetLastError();
    return nullptr;
  }
  m->iter_graph_act[dir][pi][variant] = with_act;
  m->iter_graph_counts[dir][pi][variant][0] = cc.launches;
  m->iter_graph_counts[dir][pi][variant][1] = cc.solves;
  m->iter_graph_counts[dir][pi][variant][2] = cc.locals;
  return g;
}

// `count` iterations of one direction: whole chunks from the captured graph, the
// rest (and everything when graphs are off) launched directly.  act / xnext are
// the fixed per-step buffers.
pd_status run_iterations(Ctx& c, int dir, int prec, const double* act, const double* xnext, int count) {
  auto direct = [&]() {
    return dir == 0 ? launch_fwd_iteration(c, prec, act) : launch_bwd_iteration(c, prec, xnext, act);
  };
  int done = 0;
  if (c.graphs && count >= kGraphIters) {
    // profiled: a graph of all but one iteration, then the last one launched directly
    // with its timing events (the GPU is still busy with the graph when they are
    // recorded, so they time the kernels, not the host launch latency)
    const int variant = (c.solve_t || c.local_t) ? 1 : 0;
    cudaGraphExec_t g = iteration_graph(c, dir, prec, act != nullptr, variant);
    if (g) {
      const int64_t* gc =
          c.m->iter_graph_counts[dir][prec == PD_PREC_MIXED ? 1 : (prec == kPrecMixedAcc ? 2 : (prec == kPrecRefined ? 3 : 0))][variant];
      for (; done + kGraphIters <= count; done += kGraphIters) {
        PD_CUDA_TRY(cudaGraphLaunch(g, c.s));
        c.launches += gc[0];
        c.solves += gc[1];
        c.locals += gc[2];
        if (variant) {
          pd_status e = direct();
          if (e != PD_OK) return e;
        }
      }
    }
  }
  for (; done < count; ++done) {
    pd_status e = direct();
    if (e != PD_OK) return e;
  }
  return PD_OK;
}

struct StepInfo {
  int iters = 0, fp64_iters = 0, ls = 0;
  double rel = 0;
  bool converged = true;
  bool nan = false;   // a residual was non-finite (the call reports PD_ERR_NAN)
};

// One implicit-Euler step from the internal state (w.xprev, w.vprev): on return
// w.x holds x_{t+1}; finalize writes the trajectory and advances the state.
pd_status contact_apply(MeshImpl* m, const std::vector<int32_t>& node, cudaStream_t s);

// Complementarity contact (Alg. 3): the contact set of a step and its targets on
// the ground z = 0, updated until stable: a candidate whose ray x_t + s v_t
// reaches z = 0 within the step is held at the intersection (height exactly 0),
// one already touching or joining later at (x_t, y_t, 0); nodes whose contact force
// r_z = [M (x - y)/h^2 + grad E]_z is below -tau_r leave (at most once per step),
// candidates below -tau_z join.  `iterate` runs the inner PD + L-BFGS solve.
template <typename It>
pd_status contact_rounds(Ctx& c, const StateCfg& cfg, const PredParams& pp, const double* act_c, int step,
                         It& iterate, int& total_iters) {
  MeshImpl* m = c.m;
  Workspace& w = m->ws;
  const HostMesh& h = m->h;
  const int64_t nc = m->ncand;
  const double hs = m->h_step;
  auto rows = [&](const double* a, std::vector<double>& out) -> cudaError_t {
    out.resize((size_t)(3 * nc));
    cudaError_t e = contact_pack_rows(m->cand, nc, a, m->cand_buf, c.s);
    if (e != cudaSuccess) return e;
    if (nc) e = cudaMemcpyAsync(out.data(), m->cand_buf, sizeof(double) * 3 * nc, cudaMemcpyDeviceToHost, c.s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(c.s);
  };
  std::vector<double> xc, vc, xn, rn;
  PD_CUDA_TRY(rows(w.xprev, xc));
  PD_CUDA_TRY(rows(w.vprev, vc));
  std::vector<int32_t> C;       // candidate indices
  std::vector<uint8_t> ray;     // 1 = ray target, 0 = drop target
  for (int64_t k = 0; k < nc; ++k) {
    const double z = xc[3 * k + 2], vz = vc[3 * k + 2];
    if (z <= 0.0) {
      C.push_back((int32_t)k), ray.push_back(0);
    } else if (z + hs * vz <= 0.0) {
      C.push_back((int32_t)k), ray.push_back(1);
    }
  }
  double mmax = 0;
  for (double mm : h.mass) mmax = std::max(mmax, mm);
  const double tau_r = 1e-8 * mmax * std::sqrt(m->grav[0] * m->grav[0] + m->grav[1] * m->grav[1] +
                                                m->grav[2] * m->grav[2]);
  const double tau_z = 1e-9 * h.dx;
  std::vector<uint8_t> left((size_t)nc, 0), locked((size_t)nc, 0), inC((size_t)nc, 0);
  constexpr int kMaxRounds = 64;
  for (int round = 1;; ++round) {
    const int64_t cs = (int64_t)C.size();
    std::vector<int32_t> node((size_t)cs);
    std::vector<double> xs((size_t)(3 * cs));
    for (int64_t i = 0; i < cs; ++i) {
      const int64_t k = C[i];
      node[i] = m->cand_host[k];
      const double* xt = &xc[3 * k];
      const double* vt = &vc[3 * k];
      if (ray[i]) {   // on the ground by the choice of s: height exactly 0
        const double sr = xt[2] / (-vt[2]);
        xs[3 * i] = xt[0] + sr * vt[0], xs[3 * i + 1] = xt[1] + sr * vt[1], xs[3 * i + 2] = 0.0;
      } else {
        xs[3 * i] = xt[0], xs[3 * i + 1] = xt[1], xs[3 * i + 2] = 0.0;
      }
    }
    pd_status e = contact_apply(m, node, c.s);
    if (e != PD_OK) return e;
    if (cs) {
      PD_CUDA_TRY(cudaMemcpyAsync(m->cset_xstar, xs.data(), sizeof(double) * 3 * cs, cudaMemcpyHostToDevice, c.s));
    }
    if (round > 1) {   // restart from the last solution with the new set
      state_reset_kernel<<<1, 1, 0, c.s>>>(w.st, cfg);
      predictor_kernel<<<grid_for(c.n), 256, 0, c.s>>>(pp);
      copy_kernel<<<c.vb, 256, 0, c.s>>>(c.n3f, w.x, w.xt);
      c.launches += 3;
    }
    PD_CUDA_TRY(contact_set_targets(m->cset_node, cs, m->cset_xstar, w.xt, c.s));
    m->held_active = true;
    e = iterate();
    m->held_active = false;
    if (e != PD_OK) return e;
    total_iters += w.st_host->iters;
    // contact forces and positions at the candidates: unmasked FP64 gradient at x
    LocalArgs la{m, nullptr, w.x, nullptr, act_c, PD_PREC_FP64};
    PD_CUDA_TRY(launch_element_forces(la, w.elembuf, c.pe, w.flags, c.s));
    PD_CUDA_TRY(launch_gather_grad(m, nullptr, w.elembuf, PD_PREC_FP64, w.x, w.y, nullptr, w.Hd, c.pg, c.s));
    c.launches += 2;
    PD_CUDA_TRY(rows(w.Hd, rn));
    PD_CUDA_TRY(rows(w.x, xn));
    std::fill(inC.begin(), inC.end(), 0);
    for (int32_t k : C) inC[k] = 1;
    std::vector<int32_t> keepC;
    std::vector<uint8_t> keepR;
    bool leave = false;
    for (int64_t i = 0; i < cs; ++i) {
      const int32_t k = C[i];
      if (rn[3 * k + 2] < -tau_r && !locked[k]) {
        leave = true;
        left[k] = 1;
      } else {
        keepC.push_back(k), keepR.push_back(ray[i]);
      }
    }
    bool join = false;
    for (int64_t k = 0; k < nc; ++k) {
      if (inC[k] || !(xn[3 * k + 2] < -tau_z)) continue;
      join = true;
      if (left[k]) locked[k] = 1;
      keepC.push_back((int32_t)k), keepR.push_back(0);
    }
    if ((!leave && !join) || round == kMaxRounds) break;
    // left marks are only final for nodes that actually left in this round
    C.swap(keepC);
    ray.swap(keepR);
  }
  if (step >= 0 && step < (int)m->contact_log_node.size()) {
    std::vector<int32_t> node(C.size());
    for (size_t i = 0; i < C.size(); ++i) node[i] = m->cand_host[C[i]];
    m->contact_log_node[step] = node;
    m->contact_log_rule[step] = ray;
  }
  return PD_OK;
}

pd_status forward_step(Ctx& c, const double* act_t, const double* fext_int, double mu,
                       double* traj_x, double* traj_v, StepInfo& info, int& guess, int step) {
  MeshImpl* m = c.m;
  Workspace& w = m->ws;
  StateCfg cfg{c.o.tol_fwd, m->precision == PD_PREC_MIXED ? 1e-6 : 1e-12, c.o.lbfgs_m, c.o.ls_max,
               c.o.max_iter_fwd, 0, (c.o.warm_start && c.last_kind == 0) ? 1 : 0};
  c.last_kind = 0;
  state_reset_kernel<<<1, 1, 0, c.s>>>(w.st, cfg);
  PredParams pp{};
  pp.n = c.n;
  pp.nf = c.nf;
  pp.xi = w.xprev;
  pp.vi = w.vprev;
  pp.fext = fext_int;
  pp.mass = m->mass;
  pp.X = m->X;
  pp.contact = m->k_contact > 0 ? m->contact : nullptr;
  pp.k = m->k_contact;
  pp.mu = mu;
  pp.h = m->h_step;
  for (int i = 0; i < 3; ++i) pp.grav[i] = m->grav[i];
  pp.y = w.y;
  pp.xt = w.xt;
  pp.x = w.x;
  pp.partials = w.partials;
  pp.counter = w.counters;
  pp.st = w.st;
  predictor_kernel<<<grid_for(c.n), 256, 0, c.s>>>(pp);
  PD_CUDA_TRY(cudaGetLastError());
  c.launches += 2;
  // MIXED: iterate with FP32 local steps; when the FP32 residual meets the
  // tolerance, re-evaluate the gradient at the accepted point with an FP64 local
  // step (the convergence check; kPrecRefined: FP64-accurate from an FP32 SVD
  // refined in FP64).  If it fails the FP32 iteration continues from
  // the FP64 gradient; after kMaxChecks failed checks the FP64 local step is used
  // for the remaining iterations.  When the FP32 residual stops halving above the
  // tolerance (its rounding floor: under large rotations H = F - I is of the order
  // of the rotation angle, and forming the strain from it in FP32 cancels bits),
  // the iteration continues with the strain-accurate FP32 local step
  // (kPrecMixedAcc), and only when that stalls too with FP64 local steps; the next
  // steps then start with the strain-accurate one.
  const bool mixed = m->precision == PD_PREC_MIXED;
  int fp64_launched = 0;
  constexpr int kMaxChecks = 3;
  const int hard_cap = 3 * c.o.max_iter_fwd + 64;
  info = StepInfo{};
  const double* act_c = nullptr;   // the step's actuation in the fixed buffer the graphs read
  if (act_t) {
    PD_CUDA_TRY(cudaMemcpyAsync(w.act_cur, act_t, sizeof(double) * m->h.e, cudaMemcpyDeviceToDevice, c.s));
    act_c = w.act_cur;
  }
  // The first chunk of iterations is launched without polling; its length comes
  // from the previous step: the iterations its FP32 phase took until it met the
  // tolerance, or until the residual stopped halving (the start of the stall
  // window, not the switch to FP64 after it).  Counting the whole previous step
  // instead would feed every stall window into the next step's blind chunk.
  int fp32_end = -1;
  // the PD + L-BFGS iteration from the trial in w.xt (iteration state reset)
  bool used_acc = false;
  auto iterate = [&]() -> pd_status {
    int prec = mixed ? (c.acc_steps > 0 ? kPrecMixedAcc : PD_PREC_MIXED) : PD_PREC_FP64;
    int launched = 0, checks = 0, stall = 0;
    double best_rel = 1e300;
    int chunk = std::max(guess, 1);
    while (true) {
      pd_status er = run_iterations(c, 0, prec, act_c, nullptr, chunk);
      if (er != PD_OK) return er;
      launched += chunk;
      if (mixed && prec == kPrecRefined) fp64_launched += chunk;
      if (chunk > 0) {
        clear_checked_kernel<<<1, 1, 0, c.s>>>(w.st);
        c.launches += 1;
      }
      pd_status e = poll(c);
      if (e != PD_OK) return e;
      const IterState& sh = *w.st_host;
      if (sh.status & DEV_ERR_NAN) {
        info.converged = false;
        info.nan = true;
        break;
      }
      if (sh.converged) {
        if (mixed && prec != kPrecRefined && !sh.hit_max && !sh.fp64_checked) {
          // FP64 convergence check at the accepted point
          if (fp32_end < 0) fp32_end = sh.iters;
          ++checks;
          if (checks > kMaxChecks) prec = kPrecRefined;
          force_accept_kernel<<<1, 1, 0, c.s>>>(w.st);
          copy_kernel<<<c.vb, 256, 0, c.s>>>(c.n3f, w.x, w.xt);
          pd_status e2 = launch_fwd_iteration(c, kPrecRefined, act_c);
          if (e2 != PD_OK) return e2;
          fp64_launched += 1;
          mark_checked_kernel<<<1, 1, 0, c.s>>>(w.st);
          c.launches += 3;
          chunk = 0;
          continue;
        }
        info.converged = !sh.hit_max;
        break;
      }
      // FP32 floor above the tolerance: no halving of the residual over three polls
      if (mixed && prec != kPrecRefined && sh.ref2 > 0) {
        const double rel = std::sqrt(sh.gn2_acc / sh.ref2);
        if (rel < 0.5 * best_rel) {
          best_rel = rel;
          stall = 0;
        } else if (++stall >= 3) {
          if (fp32_end < 0) fp32_end = std::max(1, sh.iters - 3 * c.o.check_every);
          if (prec == PD_PREC_MIXED && m->h.rule == PD_ELEM_HEX8 && !m->neohookean) {
            prec = kPrecMixedAcc;
            used_acc = true;
          } else {
            prec = kPrecRefined;
          }
          best_rel = rel;
          stall = 0;
        }
      }
      if (launched >= hard_cap) {
        info.converged = false;
        break;
      }
      chunk = c.o.check_every;
    }
    return PD_OK;
  };
  int total_iters = 0;
  if (!c.complementarity) {
    pd_status e = iterate();
    if (e != PD_OK) return e;
    total_iters = w.st_host->iters;
  } else {
    pd_status e = contact_rounds(c, cfg, pp, act_c, step, iterate, total_iters);
    if (e != PD_OK) return e;
  }
  const IterState& sh = *w.st_host;
  info.iters = total_iters;
  info.ls = sh.ls_total;
  info.fp64_iters = fp64_launched;
  info.rel = sh.ref2 > 0 ? std::sqrt(sh.gn2_acc / sh.ref2) : 0.0;
  guess = std::max(1, (fp32_end >= 0 ? fp32_end : sh.iters) - 1);
  // the strain-accurate local step stays on for the next 8 steps once it was needed
  if (used_acc) c.acc_steps = 8;
  else if (c.acc_steps > 0) --c.acc_steps;
  finalize_fwd_kernel<<<grid_for(c.n), 256, 0, c.s>>>(c.n, w.x, w.xprev, w.vprev, 1.0 / m->h_step,
                                                      m->kept_of_internal, traj_x, traj_v);
  c.launches += 1;
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

void accumulate(pd_stats* st, const StepInfo& i, bool fwd) {
  if (!st) return;
  if (fwd) {
    st->fwd_iters += i.iters;
    st->fwd_fp64_iters += i.fp64_iters;
    st->fwd_line_search += i.ls;
    st->max_fwd_iters_step = std::max(st->max_fwd_iters_step, i.iters);
    st->max_fwd_rel_residual = std::max(st->max_fwd_rel_residual, i.rel);
  } else {
    st->bwd_iters += i.iters;
    st->bwd_fp64_iters += i.fp64_iters;
    st->max_bwd_iters_step = std::max(st->max_bwd_iters_step, i.iters);
    st->max_bwd_rel_residual = std::max(st->max_bwd_rel_residual, i.rel);
  }
  if (!i.converged) st->not_converged_steps += 1;
}

void finish_stats(Ctx& c, pd_stats* st) {
  if (!st) return;
  st->kernel_launches = c.launches;
  st->solves = c.solves;
  st->local_steps = c.locals;
  st->solve_ms = c.solve_t ? c.solve_t->total_ms() : 0.0;
  st->local_ms = c.local_t ? c.local_t->total_ms() : 0.0;
  st->solves_timed = c.solve_t ? c.solve_t->pairs() : 0;
  st->local_steps_timed = c.local_t ? c.local_t->pairs() : 0;
}

pd_status check_flags(Ctx& c, pd_stats* stats) {
  int flags = 0;
  PD_CUDA_TRY(cudaMemcpyAsync(&flags, c.m->ws.flags, sizeof(int), cudaMemcpyDeviceToHost, c.s));
  PD_CUDA_TRY(cudaStreamSynchronize(c.s));
  if (stats && (flags & DEV_ERR_INVERTED)) stats->inverted = 1;
  c.dev_flags = flags;
  return PD_OK;
}

// Adjoint of one step at x_{t+1} (w.x holds x_{t+1} internal; w.xprev/w.vprev hold x_t, v_t).
// Complementarity contact: the held set takes part in the gathers only while a
// scope is open
struct HeldScope {
  MeshImpl* m;
  HeldScope(MeshImpl* mm, bool on) : m(mm) { m->held_active = on; }
  ~HeldScope() { m->held_active = false; }
};

pd_status backward_step(Ctx& c, const double* xnext, const double* xt_, const double* vt_,
                        const double* act_t, double mu, const double* gx_t, const double* gv_t,
                        double* gfext_int, double* g_wc, double* g_wv, double* g_wm, double* g_act_t,
                        double* g_mu, StepInfo& info, int& guess, int step) {
  MeshImpl* m = c.m;
  Workspace& w = m->ws;
  const double inv_h = 1.0 / m->h_step;
  // complementarity contact (Alg. 5): the step's final contact set from the
  // forward pass; its rows of the adjoint are zero (H_{C'C'} z_{C'} = gbar_{C'})
  const uint8_t* held = nullptr;
  if (c.complementarity) {
    const std::vector<int32_t>& node = m->contact_log_node[step];
    const std::vector<uint8_t>& rule = m->contact_log_rule[step];
    pd_status e = contact_apply(m, node, c.s);
    if (e != PD_OK) return e;
    if (m->cset > 0) {
      PD_CUDA_TRY(cudaMemcpyAsync(m->cset_rule, rule.data(), rule.size(), cudaMemcpyHostToDevice, c.s));
    }
    held = m->held;
  }
  HeldScope scope(m, c.complementarity);
  const bool warm = c.o.warm_start && c.bwd_steps > 0;   // w.z holds the previous adjoint
  StateCfg cfg{c.o.tol_bwd, 0.0, c.o.lbfgs_m, c.o.ls_max, c.o.max_iter_bwd, 1,
               (c.o.warm_start && c.last_kind == 1) ? 1 : 0};
  c.bwd_steps += 1;
  c.last_kind = 1;
  state_reset_kernel<<<1, 1, 0, c.s>>>(w.st, cfg);
  bwd_step_init_kernel<<<c.vb, 256, 0, c.s>>>(c.vc, w.ax, w.av, inv_h, w.z, w.gs, w.q, warm ? 1 : 0, held);
  c.launches += 2;
  if (warm) {
    // start from the previous step's adjoint: gs = H z - gbar at that z
    const int p0 = m->precision == PD_PREC_MIXED ? PD_PREC_MIXED : PD_PREC_FP64;
    LocalArgs la0{m, nullptr, xnext, w.z, act_t, p0};
    PD_CUDA_TRY(launch_element_hvp(la0, w.elembuf, w.flags, c.s));
    PD_CUDA_TRY(launch_gather_hvp(m, nullptr, w.elembuf, p0, xnext, w.z, nullptr, w.Hd, c.pg, c.s));
    residual_replace_kernel<<<c.vb, 256, 0, c.s>>>(c.vc, w.Hd, w.ax, w.av, inv_h, w.gs, w.q, held);
    c.launches += 3;
  }
  // Hessian products in the factor's precision; at convergence of the recursively
  // updated residual, the true residual H z - gbar is evaluated with an FP64
  // product and replaces it (iterative refinement); the iteration continues
  // until the true residual meets the tolerance.
  const int prec = m->precision == PD_PREC_MIXED ? PD_PREC_MIXED : PD_PREC_FP64;
  // the FP64 true residual: refined from the FP32 SVD in mixed precision
  const int p64 = m->precision == PD_PREC_MIXED ? kPrecRefined : PD_PREC_FP64;
  int launched = 0, fp64_launched = 0, checks = 0;
  int chunk = std::max(guess, 1);
  const int hard_cap = 3 * c.o.max_iter_bwd + 64;
  info = StepInfo{};
  // the step's inputs in the fixed buffers the graphs read
  PD_CUDA_TRY(cudaMemcpyAsync(w.xnext_cur, xnext, sizeof(double) * 3 * c.n, cudaMemcpyDeviceToDevice, c.s));
  const double* act_c = nullptr;
  if (act_t) {
    PD_CUDA_TRY(cudaMemcpyAsync(w.act_cur, act_t, sizeof(double) * m->h.e, cudaMemcpyDeviceToDevice, c.s));
    act_c = w.act_cur;
  }
  while (true) {
    pd_status er = run_iterations(c, 1, prec, act_c, w.xnext_cur, chunk);
    if (er != PD_OK) return er;
    launched += chunk;
    pd_status e = poll(c);
    if (e != PD_OK) return e;
    const IterState* sh = w.st_host;
    if (sh->status & DEV_ERR_NAN) {
      info.converged = false;
      info.nan = true;
      break;
    }
    if (sh->converged) {
      if (sh->hit_max) {
        info.converged = false;
        break;
      }
      // the step's first refined check stores each point's refined rotation and
      // stretch at x_{t+1}, the later ones reuse them (the same values)
      LocalArgs la{m, nullptr, xnext, w.z, act_t, p64, checks == 0 ? 1 : 2};
      PD_CUDA_TRY(launch_element_hvp(la, w.elembuf, w.flags, c.s));
      PD_CUDA_TRY(launch_gather_hvp(m, nullptr, w.elembuf, p64, xnext, w.z, nullptr, w.Hd, c.pg, c.s));
      residual_replace_kernel<<<c.vb, 256, 0, c.s>>>(c.vc, w.Hd, w.ax, w.av, inv_h, w.gs, w.q, held);
      fp64_launched += 1;
      c.launches += 3;
      e = poll(c);
      if (e != PD_OK) return e;
      ++checks;
      if (w.st_host->converged || checks > 8) {
        info.converged = w.st_host->converged != 0;
        break;
      }
      chunk = c.o.check_every;
      continue;
    }
    if (launched >= hard_cap) {
      info.converged = false;
      break;
    }
    chunk = c.o.check_every;
  }
  const IterState* sh = w.st_host;
  info.iters = sh->iters;
  info.ls = sh->ls_total;
  info.fp64_iters = fp64_launched;
  info.rel = sh->ref2 > 0 ? std::sqrt(sh->gn2_acc / sh->ref2) : 0.0;
  guess = std::max(1, sh->iters - 1);
  const int64_t cs = c.complementarity ? m->cset : 0;
  m->held_active = false;
  if (cs > 0) {
    // dL/dx* = gbar_C - (H z)_C with the unmasked FP64 product, through the targets
    LocalArgs lh{m, nullptr, xnext, w.z, act_t, PD_PREC_FP64};
    PD_CUDA_TRY(launch_element_hvp(lh, w.elembuf, w.flags, c.s));
    PD_CUDA_TRY(launch_gather_hvp(m, nullptr, w.elembuf, PD_PREC_FP64, xnext, w.z, nullptr, w.Hd, c.pg, c.s));
    PD_CUDA_TRY(contact_target_vjp(m->cset_node, m->cset_rule, cs, xt_, vt_, w.ax, w.av, w.Hd, inv_h,
                                   m->cset_gx, m->cset_gv, c.s));
    c.launches += 3;
  }
  // parameter gradients at x_{t+1} (per-element products in the factor's precision,
  // FP64 accumulation over steps), then the state adjoint of step t
  LocalArgs la{m, nullptr, xnext, w.z, act_t, prec == PD_PREC_MIXED ? kPrecMixedAcc : prec};
  PD_CUDA_TRY(launch_element_param_grads(la, g_wc, g_wv, g_wm, g_act_t, c.s));
  BwdStateParams bp{};
  bp.n = c.n;
  bp.nf = c.nf;
  bp.z = w.z;
  bp.mass = m->mass;
  bp.xi = xt_;
  bp.vi = vt_;
  bp.contact = m->k_contact > 0 ? m->contact : nullptr;
  bp.k = m->k_contact;
  bp.mu = mu;
  bp.h = m->h_step;
  bp.inv_h = inv_h;
  bp.inv_h2 = inv_h * inv_h;
  bp.ax = w.ax;
  bp.av = w.av;
  bp.gfext = gfext_int;
  bp.gx_t = gx_t;
  bp.gv_t = gv_t;
  bp.kept_of_internal = m->kept_of_internal;
  bp.gmu = g_mu;
  bp.partials = w.partials;
  bp.counter = w.counters;
  bwd_state_kernel<<<grid_for(c.n), 256, 0, c.s>>>(bp);
  PD_CUDA_TRY(cudaGetLastError());
  c.launches += 2;
  if (cs > 0) {
    PD_CUDA_TRY(contact_add_rows(m->cset_node, cs, m->cset_gx, m->cset_gv, w.ax, w.av, c.s));
    c.launches += 1;
  }
  return PD_OK;
}

// status of the solve's device flags: a rejected tile descriptor is an internal
// inconsistency, a bounded wait that gave up a timeout
pd_status solve_flags_status(const char* who, int flags) {
  if (flags & DEV_ERR_LAYOUT) {
    set_error(std::string(who) + ": a solve tile descriptor failed its size / alignment check");
    return PD_ERR_INTERNAL;
  }
  if (flags & DEV_ERR_TIMEOUT) {
    set_error(std::string(who) + ": a bounded device-side wait in the solve gave up");
    return PD_ERR_TIMEOUT;
  }
  return PD_OK;
}

pd_status check_mesh(pd_mesh m, bool need_factor) {
  if (!m) {
    set_error("null mesh");
    return PD_ERR_INVALID_ARG;
  }
  if (m->impl.device < 0) {
    set_error("mesh was created without a device");
    return PD_ERR_NO_DEVICE;
  }
  if (need_factor && !m->impl.factorized) {
    set_error("pd_factorize has not succeeded on this mesh");
    return PD_ERR_INVALID_ARG;
  }
  return PD_OK;
}

}  // namespace

extern "C" {

const char* pd_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// Builds the host analysis with `analyse_fn`, then (device >= 0) uploads the mesh
// and its solve structures: the common part of pd_create_mesh and pd_create_tet_mesh.
template <typename Desc, typename AnalyseFn>
pd_status create_mesh_common(const Desc* desc, pd_mesh* out, AnalyseFn analyse_fn) {
  if (!desc || !out) {
    set_error("pd_create_mesh: null argument");
    return PD_ERR_INVALID_ARG;
  }
  *out = nullptr;
  pd_mesh m = new (std::nothrow) pd_mesh_s;
  if (!m) {
    set_error("pd_create_mesh: host allocation failed");
    return PD_ERR_OOM;
  }
  MeshImpl& I = m->impl;
  std::string err;
  try {
    err = analyse_fn(*desc, I.h);
  } catch (const std::bad_alloc&) {
    err = "pd_create_mesh: host allocation failed";
  }
  if (!err.empty()) {
    set_error(err);
    delete m;
    return PD_ERR_INVALID_ARG;
  }
  I.device = desc->device;
  if (I.device < 0) {
    *out = m;
    return PD_OK;
  }
  DeviceGuard g(I.device);
  const HostMesh& h = I.h;
  for (int64_t L = 0; L < h.nlev; ++L)
    if (h.level_ptr[L + 1] - h.level_ptr[L] > 65535) {
      set_error("pd_create_mesh: a tree level has more than 65535 supernodes");
      delete m;
      return PD_ERR_INVALID_ARG;
    }
  auto fail = [&](cudaError_t e) {
    set_error(std::string("pd_create_mesh: ") + cudaGetErrorString(e));
    pd_mesh_destroy(m);
    return e == cudaErrorMemoryAllocation ? PD_ERR_OOM : PD_ERR_CUDA;
  };
  cudaError_t e;
#define UP(dst, src) if ((e = upload(&I, &I.dst, h.src)) != cudaSuccess) return fail(e)
  UP(elems, elems);
  UP(inc_ptr, inc_ptr);
  UP(inc, inc);
  UP(kept_of_internal, kept_of_internal);
  UP(X, X);
  UP(mass, mass);
  UP(contact, contact);
  UP(snode_first, snode_first);
  UP(row_ptr, row_ptr);
  UP(panel_off, panel_off);
  UP(rel_ptr, rel_ptr);
  UP(gath_ptr, gath_ptr);
  UP(front_off, front_off);
  UP(level_list, level_list);
  UP(child_ptr, child_ptr);
  UP(child_list, child_list);
  UP(rows, rows);
  UP(gath, gath);
  UP(rel, rel);
  UP(la_target, la_target);
  UP(la_cptr, la_cptr);
  UP(la_diag_node, la_diag_node);
  UP(la_contrib, la_contrib);
  if (h.rule == PD_ELEM_TETU) {
    UP(tet_grad, tet_grad);
    UP(tet_grad_f, tet_grad);
    UP(tet_vol, tet_vol);
    UP(tet_vol_f, tet_vol);
  }
#undef UP
  build_solve_schedule(h, I.sched);
  {
    const SolveSchedule& S = I.sched;
    // fixed-width slots per parent position (max fan-in of the forward-solve
    // assembly): child update row gath[g] of position k goes to slot k w + (g - gath_ptr[k])
    int64_t w = 1;
    for (size_t k = 0; k + 1 < h.gath_ptr.size(); ++k) w = std::max<int64_t>(w, h.gath_ptr[k + 1] - h.gath_ptr[k]);
    I.slot_w = (int)w;
    const int64_t wrows = h.rel_ptr.empty() ? 0 : h.rel_ptr.back();
    std::vector<int32_t> dest((size_t)std::max<int64_t>(wrows, 1), 0);
    for (size_t k = 0; k + 1 < h.gath_ptr.size(); ++k)
      for (int64_t g = h.gath_ptr[k]; g < h.gath_ptr[k + 1]; ++g)
        dest[h.gath[g]] = (int32_t)(k * w + (g - h.gath_ptr[k]));
    if ((e = upload(&I, &I.wdest, dest)) != cudaSuccess) return fail(e);
    const size_t nslot = 3 * (size_t)std::max<int64_t>((int64_t)(h.gath_ptr.size() - 1) * w, 1);
    if ((e = dalloc(&I, &I.W32, nslot)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&I, &I.W64, nslot)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(I.W32, 0, sizeof(float) * nslot)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(I.W64, 0, sizeof(double) * nslot)) != cudaSuccess) return fail(e);
    if ((e = upload(&I, &I.nfb, S.nfb)) != cudaSuccess) return fail(e);
    if ((e = upload(&I, &I.nbb, S.nbb)) != cudaSuccess) return fail(e);
    if ((e = upload(&I, &I.parent, h.parent)) != cudaSuccess) return fail(e);
    if ((e = dalloc(&I, &I.all_tiles, S.all.size())) != cudaSuccess) return fail(e);
    if (!S.all.empty() && (e = cudaMemcpy(I.all_tiles, S.all.data(), sizeof(SolveTile) * S.all.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    const size_t ncount = 1 + 2 * (size_t)h.ns + S.all.size();
    if ((e = dalloc(&I, &I.solve_counters, ncount)) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(I.solve_counters, 0, sizeof(unsigned long long) * ncount)) != cudaSuccess) return fail(e);
    {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      I.solve_grid = sms * solve_persistent_occupancy();
      I.sms = std::max(1, sms);
    }
    if ((e = dalloc(&I, (char**)&I.ws.solve_partial, std::max<size_t>(solve_partial_bytes(S), 16))) != cudaSuccess)
      return fail(e);
    // bounded-wait settings and the test hook that makes one wait run out
    if (const char* ev = std::getenv("PD_SOLVE_SPIN_LIMIT")) {
      const long long v = std::atoll(ev);
      if (v > 0) I.solve_spin_limit = v;
    }
    if (const char* ev = std::getenv("PD_TEST_SOLVE_STALLS")) I.test_stall_solves = std::max(0, std::atoi(ev));
    for (int64_t k = (int64_t)S.fwd.size() - 1; k >= 0; --k)
      if (S.all[k].ndep > 0) {   // the last forward tile that waits for children
        I.stall_tile = k;
        break;
      }
  }
  I.flevels.assign(h.nlev, FactorLevel{});
  for (int64_t L = 0; L < h.nlev; ++L) {
    FactorLevel& f = I.flevels[L];
    f.list_off = h.level_ptr[L];
    f.count = h.level_ptr[L + 1] - h.level_ptr[L];
    for (int64_t i = h.level_ptr[L]; i < h.level_ptr[L + 1]; ++i) {
      const int64_t s = h.level_list[i];
      f.max_nc = std::max(f.max_nc, h.nc(s));
      f.max_nr = std::max(f.max_nr, h.nr(s));
      f.max_children = std::max(f.max_children, h.child_ptr[s + 1] - h.child_ptr[s]);
      for (int64_t ci = h.child_ptr[s]; ci < h.child_ptr[s + 1]; ++ci) {
        const int64_t t = h.child_list[ci];
        const int64_t nb = h.nr(t) - h.nc(t);
        f.max_child_nb2 = std::max(f.max_child_nb2, nb * nb);
      }
    }
  }
  pd_status ws = ensure_workspace(&I, 5);
  if (ws != PD_OK) {
    pd_mesh_destroy(m);
    return ws;
  }
  *out = m;
  return PD_OK;
}

}  // namespace

extern "C" {

pd_status pd_create_mesh(const pd_mesh_desc* desc, pd_mesh* out) {
  return create_mesh_common(desc, out, [](const pd_mesh_desc& d, HostMesh& h) { return analyse(d, h); });
}

pd_status pd_create_tet_mesh(const pd_tet_mesh_desc* desc, pd_mesh* out) {
  return create_mesh_common(desc, out, [](const pd_tet_mesh_desc& d, HostMesh& h) { return analyse_tet(d, h); });
}

void pd_mesh_destroy(pd_mesh m) {
  if (!m) return;
  MeshImpl& I = m->impl;
  if (I.device >= 0) {
    DeviceGuard g(I.device);
    cudaDeviceSynchronize();
    drop_iteration_graphs(&I);
    if (I.cap_stream) cudaStreamDestroy(I.cap_stream);
    for (auto& a : I.allocations) cudaFree(a.first);
    if (I.ws.st_host) cudaFreeHost(I.ws.st_host);
  }
  delete m;
}

pd_status pd_mesh_query(pd_mesh m, pd_mesh_info* info) {
  if (!m || !info) {
    set_error("pd_mesh_query: null argument");
    return PD_ERR_INVALID_ARG;
  }
  const HostMesh& h = m->impl.h;
  std::memset(info, 0, sizeof(*info));
  info->n_nodes = h.n;
  info->n_elems = h.e;
  info->n_free = h.nf;
  info->n_snodes = h.ns;
  info->n_levels = h.nlev;
  info->factor_nnz = h.factor_nnz();
  for (int64_t s = 0; s < h.ns; ++s) {
    info->max_rows = std::max(info->max_rows, h.nr(s));
    info->max_cols = std::max(info->max_cols, h.nc(s));
  }
  info->front_entries = h.front_entries();
  info->update_entries = h.rel_ptr.empty() ? 0 : h.rel_ptr.back();
  info->factorized = m->impl.factorized ? 1 : 0;
  info->precision = m->impl.precision;
  return PD_OK;
}

pd_status pd_plan_checkpoints(pd_mesh m, int32_t T, size_t mem_cap_bytes, int32_t* checkpoint_every) {
  if (!m || !checkpoint_every || T < 0) {
    set_error("pd_plan_checkpoints: null argument or T < 0");
    return PD_ERR_INVALID_ARG;
  }
  const MeshImpl& I = m->impl;
  size_t budget = mem_cap_bytes;
  if (budget == 0) {
    if (I.device < 0) {
      set_error("pd_plan_checkpoints: a host-only mesh needs an explicit memory cap");
      return PD_ERR_INVALID_ARG;
    }
    DeviceGuard g(I.device);
    size_t free_b = 0, total_b = 0;
    PD_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    budget = free_b / 10 * 8;   // leave a fifth of the free memory to everything else
  }
  // bytes of one stored state: x and v, (n, 3) doubles each
  const double state = 2.0 * 3.0 * 8.0 * (double)I.h.n;
  if ((double)(T + 1) * state <= (double)budget) {
    *checkpoint_every = 0;
    return PD_OK;
  }
  // smallest K dividing T whose checkpoints (T/K + 1 states, caller memory) and
  // recomputed segment (K + 1 states, pd_backward's buffer) fit
  for (int32_t K = 2; K <= T; ++K) {
    if (T % K) continue;
    if ((double)(T / K + 1 + K + 1) * state <= (double)budget) {
      *checkpoint_every = K;
      return PD_OK;
    }
  }
  set_error("pd_plan_checkpoints: no checkpoint interval fits the memory cap");
  return PD_ERR_OOM;
}

pd_status pd_mesh_export(pd_mesh m, int32_t what, int64_t* host_out, int64_t capacity, int64_t* count) {
  if (!m) {
    set_error("pd_mesh_export: null mesh");
    return PD_ERR_INVALID_ARG;
  }
  const HostMesh& h = m->impl.h;
  std::vector<int64_t> v;
  switch (what) {
    case PD_EXPORT_INC_PTR: v = h.inc_ptr_kept; break;
    case PD_EXPORT_INC: v = h.inc_kept; break;
    case PD_EXPORT_PERM: v = h.perm; break;
    case PD_EXPORT_SNODE_FIRST: v = h.snode_first; break;
    case PD_EXPORT_ROW_PTR: v = h.row_ptr; break;
    case PD_EXPORT_ROWS: v.assign(h.rows.begin(), h.rows.end()); break;
    case PD_EXPORT_PARENT: v = h.parent; break;
    case PD_EXPORT_LEVEL: v = h.level; break;
    case PD_EXPORT_REL: v.assign(h.rel.begin(), h.rel.end()); break;
    case PD_EXPORT_LEVEL_PTR: v = h.level_ptr; break;
    case PD_EXPORT_LEVEL_LIST: v = h.level_list; break;
    case PD_EXPORT_SOLVE_TILES: {
      SolveSchedule S;   // host-only meshes have none built: derive it here
      const SolveSchedule* sp = &m->impl.sched;
      if (m->impl.device < 0) {
        build_solve_schedule(h, S);
        sp = &S;
      }
      v.reserve(10 * sp->all.size());
      for (const SolveTile& t : sp->all) {
        const int64_t row[10] = {t.s, t.kind, t.a, t.chunk0, t.nchunks, t.soff, t.cbytes, t.lbytes, t.lld, t.ntile};
        v.insert(v.end(), row, row + 10);
      }
      break;
    }
    default:
      set_error("pd_mesh_export: unknown structure");
      return PD_ERR_INVALID_ARG;
  }
  if (count) *count = (int64_t)v.size();
  if (host_out) {
    if (capacity < (int64_t)v.size()) {
      set_error("pd_mesh_export: capacity too small");
      return PD_ERR_INVALID_ARG;
    }
    std::copy(v.begin(), v.end(), host_out);
  }
  return PD_OK;
}

pd_status pd_factorize(pd_mesh mesh, const double* w_corot, const double* w_vol, const double* w_muscle,
                       const double* fiber, const pd_factor_opts* opts, void* stream) {
  const Range range("pd_factorize");
  pd_status ck = check_mesh(mesh, false);
  if (ck != PD_OK) return ck;
  if (!opts || !(opts->h > 0)) {
    set_error("pd_factorize: opts->h must be positive");
    return PD_ERR_INVALID_ARG;
  }
  if (!w_corot && !w_vol && !w_muscle) {
    set_error("pd_factorize: at least one energy weight array is required");
    return PD_ERR_INVALID_ARG;
  }
  if (w_muscle && !fiber) {
    set_error("pd_factorize: fiber directions are required with w_muscle");
    return PD_ERR_INVALID_ARG;
  }
  if (opts->precision != PD_PREC_FP64 && opts->precision != PD_PREC_MIXED) {
    set_error("pd_factorize: unknown precision");
    return PD_ERR_INVALID_ARG;
  }
  if (opts->neohookean && (!w_corot || !w_vol)) {
    set_error("pd_factorize: the Neo-Hookean material needs w_corot (2 mu) and w_vol (lambda)");
    return PD_ERR_INVALID_ARG;
  }
  if (opts->neohookean && mesh->impl.h.rule != PD_ELEM_HEX8) {
    set_error("pd_factorize: the Neo-Hookean material is implemented for hexahedra");
    return PD_ERR_INVALID_ARG;
  }
  if (w_muscle && mesh->impl.h.rule == PD_ELEM_TETU) {
    set_error("pd_factorize: the muscle energy is implemented for voxel meshes");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl& I = mesh->impl;
  DeviceGuard g(I.device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t e = I.h.e;
  // the library keeps its own copies of the material arrays for the local steps
  auto own = [&](double** buf, double** dst, const double* src, int64_t count) -> pd_status {
    *dst = nullptr;
    if (!src) return PD_OK;
    if (!*buf) PD_CUDA_TRY(dalloc(&I, buf, (size_t)count));
    PD_CUDA_TRY(cudaMemcpyAsync(*buf, src, sizeof(double) * count, cudaMemcpyDeviceToDevice, s));
    *dst = *buf;
    return PD_OK;
  };
  pd_status st;
  if ((st = own(&I.wc_buf, &I.wc, w_corot, e)) != PD_OK) return st;
  if ((st = own(&I.wv_buf, &I.wv, w_vol, e)) != PD_OK) return st;
  if ((st = own(&I.wm_buf, &I.wm, w_muscle, e)) != PD_OK) return st;
  if ((st = own(&I.fiber_buf, &I.fiber, fiber, 3 * e)) != PD_OK) return st;
  I.h_step = opts->h;
  for (int i = 0; i < 3; ++i) I.grav[i] = opts->gravity[i];
  I.k_contact = opts->k_contact;
  I.precision = opts->precision;
  I.neohookean = opts->neohookean != 0;
  const int64_t nnz = I.h.factor_nnz();
  if (!I.Q64) PD_CUDA_TRY(dalloc(&I, &I.Q64, (size_t)nnz));
  if (I.precision == PD_PREC_MIXED && !I.Q32) PD_CUDA_TRY(dalloc(&I, &I.Q32, (size_t)nnz));
  if (I.precision == PD_PREC_MIXED && !I.Qs) PD_CUDA_TRY(dalloc(&I, &I.Qs, (size_t)I.sched.stream_elems));
  drop_iteration_graphs(&I);   // they captured the weights, panels and precision
  I.factor_gen += 1;           // contact candidate columns of the old factor are stale
  I.factorized = false;
  pd_status r = factorize_device(&I, s);
  if (r == PD_OK) I.factorized = true;
  return r;
}

pd_status pd_forward(pd_mesh mesh, const double* x0, const double* v0, const double* f_ext, const double* act,
                     double mu, int32_t T, const pd_solver_opts* opts, double* x_traj, double* v_traj,
                     pd_stats* stats, void* stream) {
  const Range range("pd_forward");
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  if (!x0 || !v0 || T < 0) {
    set_error("pd_forward: x0 and v0 are required and T must be >= 0");
    return PD_ERR_INVALID_ARG;
  }
  const pd_solver_opts o = fill_opts(opts);
  if (o.checkpoint_every < 0 || (o.checkpoint_every > 0 && T % o.checkpoint_every != 0)) {
    set_error("pd_forward: checkpoint_every must be >= 0 (pd_plan_checkpoints chooses one) and divide T");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  DeviceGuard g(m->device);
  const auto t0 = std::chrono::steady_clock::now();
  pd_status ws = ensure_workspace(m, o.lbfgs_m);
  if (ws != PD_OK) return ws;
  cudaStream_t s = (cudaStream_t)stream;
  if (o.complementarity) {
    if (m->contact_gen != m->factor_gen || m->k_contact > 0) {
      set_error("pd_forward: complementarity contact needs pd_contact_prepare after the last pd_factorize "
                "and no penalty contact (k_contact = 0)");
      return PD_ERR_INVALID_ARG;
    }
    m->contact_log_node.assign((size_t)T, {});
    m->contact_log_rule.assign((size_t)T, {});
  }
  Ctx c = make_ctx(m, s, o);
  EventTimer tsolve, tlocal;
  if (o.profile) {
    c.solve_t = &tsolve;
    c.local_t = &tlocal;
  }
  Workspace& w = m->ws;
  const int64_t n = m->h.n;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  PD_CUDA_TRY(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
  PD_CUDA_TRY(reset_solve_counters(m, s));
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x0, w.xprev);
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, v0, w.vprev);
  const double* fext_int = nullptr;
  if (f_ext) {
    kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, f_ext, w.fext);
    fext_int = w.fext;
  }
  const int K = o.checkpoint_every;
  if (x_traj) PD_CUDA_TRY(cudaMemcpyAsync(x_traj, x0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
  if (v_traj) PD_CUDA_TRY(cudaMemcpyAsync(v_traj, v0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
  int guess = 4;
  bool all_ok = true, any_nan = false;
  m->acc_log.assign((size_t)T, 0);
  m->guess_log.assign((size_t)T, 0);
  for (int t = 0; t < T; ++t) {
    const double* act_t = act ? act + (int64_t)t * m->h.e : nullptr;
    m->acc_log[t] = c.acc_steps;
    m->guess_log[t] = guess;
    if (f_ext && o.fext_per_step && t > 0)
      kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, f_ext + (int64_t)t * 3 * n, w.fext);
    double* tx = nullptr;
    double* tv = nullptr;
    if (K <= 0) {
      tx = x_traj ? x_traj + (int64_t)(t + 1) * 3 * n : nullptr;
      tv = v_traj ? v_traj + (int64_t)(t + 1) * 3 * n : nullptr;
    } else if ((t + 1) % K == 0) {
      tx = x_traj ? x_traj + (int64_t)((t + 1) / K) * 3 * n : nullptr;
      tv = v_traj ? v_traj + (int64_t)((t + 1) / K) * 3 * n : nullptr;
    }
    StepInfo info;
    const auto ts = std::chrono::steady_clock::now();
    const Range step_range("forward step", t);
    pd_status e = forward_step(c, act_t, fext_int, mu, tx, tv, info, guess, t);
    if (o.step_ms) o.step_ms[t] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
    if (o.step_iters) o.step_iters[t] = info.iters;
    if (e != PD_OK) return e;
    accumulate(stats, info, true);
    if (!info.converged) all_ok = false;
    if (info.nan) any_nan = true;
  }
  PD_CUDA_TRY(cudaStreamSynchronize(s));
  check_flags(c, stats);
  finish_stats(c, stats);
  if (stats) stats->fwd_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (c.dev_flags & (DEV_ERR_TIMEOUT | DEV_ERR_LAYOUT)) return solve_flags_status("pd_forward", c.dev_flags);
  // a step whose residual was non-finite stops there and the later steps restart
  // from stale values: the call reports it even when the last step converged
  if (any_nan || (w.st_host->status & DEV_ERR_NAN)) {
    set_error("pd_forward: non-finite residual");
    return PD_ERR_NAN;
  }
  if (!all_ok) {
    set_error("pd_forward: some steps reached the iteration cap");
    return PD_ERR_NOT_CONVERGED;
  }
  return PD_OK;
}

pd_status pd_backward(pd_mesh mesh, const double* x_traj, const double* v_traj, const double* f_ext,
                      const double* act, double mu, int32_t T, const double* dL_dx, const double* dL_dv,
                      int32_t loss_states, const pd_solver_opts* opts, double* g_x0, double* g_v0,
                      double* g_fext, double* g_w_corot, double* g_w_vol, double* g_w_muscle, double* g_act,
                      double* g_mu, pd_stats* stats, void* stream) {
  const Range range("pd_backward");
  if (loss_states != 0 && loss_states != 1 && loss_states != T + 1) {
    set_error("pd_backward: loss_states must be 1 (final state) or T+1 (every state), got " +
              std::to_string(loss_states));
    return PD_ERR_INVALID_ARG;
  }
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  if (!x_traj || !v_traj || !dL_dx || T < 0) {
    set_error("pd_backward: x_traj, v_traj and dL_dx are required");
    return PD_ERR_INVALID_ARG;
  }
  const bool loss_all_steps = loss_states == T + 1 && T + 1 != 1;
  const pd_solver_opts o = fill_opts(opts);
  const int K = o.checkpoint_every;
  if (K < 0 || (K > 0 && T % K != 0)) {
    set_error("pd_backward: checkpoint_every must be >= 0 and divide T");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  DeviceGuard g(m->device);
  const auto t0 = std::chrono::steady_clock::now();
  {
    // the Hessian products' SVD cache (before any iteration graph is captured); the
    // adjoint solves run without it when it does not fit in memory
    int64_t slots, fields;
    svd_cache_layout(m, &slots, &fields);
    if (fields > m->svd_cache_fields) {
      dfree(m, &m->svd_cache);
      m->svd_cache_fields = 0;
      if (dalloc(m, &m->svd_cache, (size_t)(slots * fields)) == cudaSuccess) m->svd_cache_fields = fields;
      else cudaGetLastError();
    }
    int64_t rd;
    if (!m->ref_cache && ref_cache_applies(m, &rd) && dalloc(m, &m->ref_cache, (size_t)rd) != cudaSuccess)
      cudaGetLastError();
  }
  pd_status ws = ensure_workspace(m, o.lbfgs_m);
  if (ws != PD_OK) return ws;
  cudaStream_t s = (cudaStream_t)stream;
  if (o.complementarity && (m->contact_gen != m->factor_gen || (int64_t)m->contact_log_node.size() != T)) {
    set_error("pd_backward: complementarity contact needs the contact sets of a pd_forward of the same T");
    return PD_ERR_INVALID_ARG;
  }
  Ctx c = make_ctx(m, s, o);
  EventTimer tsolve, tlocal;
  if (o.profile) {
    c.solve_t = &tsolve;
    c.local_t = &tlocal;
  }
  Workspace& w = m->ws;
  const int64_t n = m->h.n, e = m->h.e;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  PD_CUDA_TRY(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
  PD_CUDA_TRY(reset_solve_counters(m, s));
  // segment storage for recomputed states (internal order): K+1 states of x and v
  double* seg = nullptr;
  if (K > 0) PD_CUDA_TRY(cudaMallocAsync((void**)&seg, sizeof(double) * 6 * n * (size_t)(K + 1), s));
  double* gfext_int = w.gbar;   // reuse: accumulated dL/df_ext (internal order)
  const bool per_step_g = g_fext && o.fext_per_step;   // one gradient block per step
  PD_CUDA_TRY(cudaMemsetAsync(gfext_int, 0, sizeof(double) * 3 * n, s));
  if (g_w_corot) PD_CUDA_TRY(cudaMemsetAsync(g_w_corot, 0, sizeof(double) * e, s));
  if (g_w_vol) PD_CUDA_TRY(cudaMemsetAsync(g_w_vol, 0, sizeof(double) * e, s));
  if (g_w_muscle) PD_CUDA_TRY(cudaMemsetAsync(g_w_muscle, 0, sizeof(double) * e, s));
  if (g_mu) PD_CUDA_TRY(cudaMemsetAsync(g_mu, 0, sizeof(double), s));
  const double* fext_int = nullptr;
  if (f_ext) {
    kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, f_ext, w.fext);
    fext_int = w.fext;
  }
  auto loss_x = [&](int t) -> const double* {
    if (loss_all_steps) return dL_dx + (int64_t)t * 3 * n;
    return t == T ? dL_dx : nullptr;
  };
  auto loss_v = [&](int t) -> const double* {
    if (!dL_dv) return nullptr;
    if (loss_all_steps) return dL_dv + (int64_t)t * 3 * n;
    return t == T ? dL_dv : nullptr;
  };
  // upstream of the final state
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, loss_x(T), w.ax);
  if (loss_v(T)) kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, loss_v(T), w.av);
  else PD_CUDA_TRY(cudaMemsetAsync(w.av, 0, sizeof(double) * 3 * n, s));
  int guess_f = 4, guess_b = 4;
  bool all_ok = true, any_nan = false;
  // scratch for x_{t+1}, x_t, v_t in internal order
  double* xn_int = w.iox;     // x_{t+1}
  double* xt_int = w.xprev;   // x_t
  double* vt_int = w.vprev;   // v_t
  const int nseg = K > 0 ? T / K : 1;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int ta = K > 0 ? sg * K : 0;
    const int tb = K > 0 ? ta + K : T;
    if (K > 0) {
      // recompute states ta..tb-1 from the checkpoint (bit-identical to the forward)
      kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x_traj + (int64_t)sg * 3 * n, w.xprev);
      kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, v_traj + (int64_t)sg * 3 * n, w.vprev);
      copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, w.xprev, seg);
      copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, w.vprev, seg + 3 * n);
      for (int t = ta; t < tb - 1; ++t) {
        StepInfo info;
        const double* act_t = act ? act + (int64_t)t * e : nullptr;
        // the forward pass's driver state at this step (bit-identical recomputation)
        if ((int64_t)m->acc_log.size() == T) {
          c.acc_steps = m->acc_log[t];
          guess_f = m->guess_log[t];
        }
        if (f_ext && o.fext_per_step)
          kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, f_ext + (int64_t)t * 3 * n, w.fext);
        const Range step_range("recompute step", t);
        const auto ts = std::chrono::steady_clock::now();
        pd_status er = forward_step(c, act_t, fext_int, mu, nullptr, nullptr, info, guess_f, t);
        if (o.step_ms)
          o.step_ms[t] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
        if (er != PD_OK) return er;
        copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, w.xprev, seg + (int64_t)(t + 1 - ta) * 6 * n);
        copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, w.vprev, seg + (int64_t)(t + 1 - ta) * 6 * n + 3 * n);
      }
    }
    for (int t = tb - 1; t >= ta; --t) {
      const double* act_t = act ? act + (int64_t)t * e : nullptr;
      if (K > 0) {
        if (t + 1 == tb)
          kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x_traj + (int64_t)(sg + 1) * 3 * n, xn_int);
        else
          copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, seg + (int64_t)(t + 1 - ta) * 6 * n, xn_int);
        copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, seg + (int64_t)(t - ta) * 6 * n, xt_int);
        copy_kernel<<<grid_for(3 * n), 256, 0, s>>>(3 * n, seg + (int64_t)(t - ta) * 6 * n + 3 * n, vt_int);
      } else {
        kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x_traj + (int64_t)(t + 1) * 3 * n, xn_int);
        kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x_traj + (int64_t)t * 3 * n, xt_int);
        kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, v_traj + (int64_t)t * 3 * n, vt_int);
      }
      StepInfo info;
      const auto ts = std::chrono::steady_clock::now();
      const Range step_range("adjoint step", t);
      if (per_step_g) PD_CUDA_TRY(cudaMemsetAsync(gfext_int, 0, sizeof(double) * 3 * n, s));
      pd_status er = backward_step(c, xn_int, xt_int, vt_int, act_t, mu, loss_x(t), loss_v(t), gfext_int,
                                   g_w_corot, g_w_vol, g_w_muscle, g_act ? g_act + (int64_t)t * e : nullptr,
                                   g_mu, info, guess_b, t);
      if (o.step_ms)
        o.step_ms[t] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ts).count();
      if (o.step_iters) o.step_iters[t] = info.iters;
      if (er != PD_OK) return er;
      if (per_step_g)
        internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, n, m->kept_of_internal, gfext_int,
                                                            g_fext + (int64_t)t * 3 * n);
      accumulate(stats, info, false);
      if (!info.converged) all_ok = false;
      if (info.nan) any_nan = true;
    }
  }
  if (g_x0) internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, n, m->kept_of_internal, w.ax, g_x0);
  if (g_v0) internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, n, m->kept_of_internal, w.av, g_v0);
  if (g_fext && !per_step_g)
    internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, n, m->kept_of_internal, gfext_int, g_fext);
  if (seg) PD_CUDA_TRY(cudaFreeAsync(seg, s));
  PD_CUDA_TRY(cudaStreamSynchronize(s));
  check_flags(c, stats);
  finish_stats(c, stats);
  if (stats) stats->bwd_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (c.dev_flags & (DEV_ERR_TIMEOUT | DEV_ERR_LAYOUT)) return solve_flags_status("pd_backward", c.dev_flags);
  if (any_nan || (w.st_host->status & DEV_ERR_NAN)) {
    set_error("pd_backward: non-finite residual");
    return PD_ERR_NAN;
  }
  if (!all_ok) {
    set_error("pd_backward: some steps reached the iteration cap");
    return PD_ERR_NOT_CONVERGED;
  }
  return PD_OK;
}

pd_status pd_local_step(pd_mesh mesh, const double* x, const double* act, int32_t precision, double* grad_E,
                        double* energy, void* stream) {
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  if (!x) {
    set_error("pd_local_step: x is required");
    return PD_ERR_INVALID_ARG;
  }
  if (precision != PD_PREC_FP64 && precision != PD_PREC_MIXED && precision != PD_PREC_MIXED_STRAIN &&
      precision != PD_PREC_FP64_REFINED) {
    set_error("pd_local_step: unknown precision");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = m->ws;
  const int64_t n = m->h.n;
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x, w.iox);
  LocalArgs la{m, nullptr, w.iox, nullptr, act, precision};
  double* pe = w.partials;
  PD_CUDA_TRY(launch_element_forces(la, w.elembuf, pe, w.flags, s));
  const int nbe = element_energy_partials(m);
  double* etot = w.partials + nbe + 8;
  sum_partials_kernel<<<1, 256, 0, s>>>(pe, nbe, etot);
  double* gi = w.iov;
  const int gb = grid_for(n);
  if (local_is_fp32(precision))
    gather_all_kernel<float><<<gb, 256, 0, s>>>(n, m->inc_ptr, m->inc, w.elembuf, w.iox,
                                                m->k_contact > 0 ? m->contact : nullptr, m->k_contact, gi,
                                                w.partials + nbe + 16, w.counters + 1, etot);
  else
    gather_all_kernel<double><<<gb, 256, 0, s>>>(n, m->inc_ptr, m->inc, w.elembuf, w.iox,
                                                 m->k_contact > 0 ? m->contact : nullptr, m->k_contact, gi,
                                                 w.partials + nbe + 16, w.counters + 1, etot);
  if (grad_E) internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, n, m->kept_of_internal, gi, grad_E);
  if (energy) PD_CUDA_TRY(cudaMemcpyAsync(energy, etot, sizeof(double), cudaMemcpyDeviceToDevice, s));
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

pd_status pd_hessian_vector(pd_mesh mesh, const double* x, const double* act, const double* v, int32_t precision,
                            double* Hv, void* stream) {
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  if (!x || !v || !Hv) {
    set_error("pd_hessian_vector: x, v and Hv are required");
    return PD_ERR_INVALID_ARG;
  }
  if (precision != PD_PREC_FP64 && precision != PD_PREC_MIXED && precision != PD_PREC_MIXED_STRAIN &&
      precision != PD_PREC_FP64_REFINED) {
    set_error("pd_hessian_vector: unknown precision");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = m->ws;
  const int64_t n = m->h.n;
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, x, w.iox);
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, v, w.iov);
  LocalArgs la{m, nullptr, w.iox, w.iov, act, precision};
  PD_CUDA_TRY(launch_element_hvp(la, w.elembuf, w.flags, s));
  PD_CUDA_TRY(launch_gather_hvp(m, nullptr, w.elembuf, precision, w.iox, w.iov, nullptr, w.Hd,
                                w.partials + element_energy_partials(m), s));
  internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, m->h.nf, m->kept_of_internal, w.Hd, Hv);
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

pd_status pd_solve_A(pd_mesh mesh, const double* b, double* x, int32_t precision, void* stream) {
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  if (!b || !x) {
    set_error("pd_solve_A: b and x are required");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  if (precision == PD_PREC_MIXED && !m->Q32) {
    set_error("pd_solve_A: FP32 panels exist only after a PD_PREC_MIXED factorisation");
    return PD_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = m->ws;
  const int64_t n = m->h.n;
  PD_CUDA_TRY(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, b, w.iov);
  PD_CUDA_TRY(reset_solve_counters(m, s));
  PD_CUDA_TRY(solve_A(m, nullptr, w.iov, w.iox, precision, s));
  internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, m->h.nf, m->kept_of_internal, w.iox, x);
  PD_CUDA_TRY(cudaGetLastError());
  int flags = 0;
  PD_CUDA_TRY(cudaMemcpyAsync(&flags, w.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  PD_CUDA_TRY(cudaStreamSynchronize(s));
  return solve_flags_status("pd_solve_A", flags);
}

}  // extern "C"

// ------------------------------------------------------------ complementarity contact
namespace {

// Makes `node` (internal ids, distinct candidates) the contact set: index lists,
// the held mask, S = (L_A^-1)_{CC} and Q = L^-1 of S = L L^T on the device
// (c^3/3 multiply-adds each for the factor and the inverse).  Synchronises.
pd_status contact_apply(MeshImpl* m, const std::vector<int32_t>& node, cudaStream_t s) {
  const HostMesh& h = m->h;
  const int64_t c = (int64_t)node.size();
  std::vector<int32_t> cidx(c);
  std::vector<uint8_t> seen(m->ncand, 0);
  for (int64_t k = 0; k < c; ++k) {
    const int32_t ci = (node[k] >= 0 && node[k] < h.n) ? m->cand_of_internal[node[k]] : -1;
    if (ci < 0 || seen[ci]) {
      set_error("contact set: every node must be a distinct contact candidate");
      return PD_ERR_INVALID_ARG;
    }
    seen[ci] = 1;
    cidx[k] = ci;
  }
  if (c > m->cset_cap) {
    // grow geometrically (at most the candidate count): few reallocations when a
    // set grows node by node
    const int64_t cap = std::min<int64_t>(m->ncand, std::max<int64_t>(c, 2 * m->cset_cap));
    PD_CUDA_TRY(cudaStreamSynchronize(s));   // the last set's solves may still read them
    dfree(m, &m->cset_node);
    dfree(m, &m->cset_cand);
    dfree(m, &m->cset_S);
    dfree(m, &m->cset_Q);
    dfree(m, &m->cset_a);
    dfree(m, &m->cset_u);
    dfree(m, &m->cset_lam);
    dfree(m, &m->cset_zero);
    dfree(m, &m->cset_xstar);
    dfree(m, &m->cset_rule);
    dfree(m, &m->cset_gx);
    dfree(m, &m->cset_gv);
    PD_CUDA_TRY(dalloc(m, &m->cset_node, (size_t)cap));
    PD_CUDA_TRY(dalloc(m, &m->cset_cand, (size_t)cap));
    PD_CUDA_TRY(dalloc(m, &m->cset_S, (size_t)(cap * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_Q, (size_t)(cap * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_a, (size_t)(3 * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_u, (size_t)(3 * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_lam, (size_t)(3 * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_zero, (size_t)(3 * cap)));
    PD_CUDA_TRY(cudaMemsetAsync(m->cset_zero, 0, sizeof(double) * 3 * cap, s));
    PD_CUDA_TRY(dalloc(m, &m->cset_xstar, (size_t)(3 * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_rule, (size_t)cap));
    PD_CUDA_TRY(dalloc(m, &m->cset_gx, (size_t)(3 * cap)));
    PD_CUDA_TRY(dalloc(m, &m->cset_gv, (size_t)(3 * cap)));
    m->cset_cap = cap;
  }
  std::vector<uint8_t> held((size_t)h.nf, 0);
  for (int32_t in : node) held[in] = 1;
  PD_CUDA_TRY(cudaMemcpyAsync(m->held, held.data(), (size_t)h.nf, cudaMemcpyHostToDevice, s));
  m->cset = 0;
  if (c == 0) return cudaStreamSynchronize(s) == cudaSuccess ? PD_OK : PD_ERR_CUDA;
  PD_CUDA_TRY(cudaMemcpyAsync(m->cset_node, node.data(), sizeof(int32_t) * c, cudaMemcpyHostToDevice, s));
  PD_CUDA_TRY(cudaMemcpyAsync(m->cset_cand, cidx.data(), sizeof(int32_t) * c, cudaMemcpyHostToDevice, s));
  PD_CUDA_TRY(contact_gather_S(h.nf, m->Bc, m->cset_node, m->cset_cand, c, m->cset_S, s));
  if (!m->cset_meta) PD_CUDA_TRY(dalloc(m, &m->cset_meta, 4));
  if (!m->cset_flags) PD_CUDA_TRY(dalloc(m, &m->cset_flags, 1));
  pd_status e = dense_cholesky_inverse(m->cset_S, c, m->cset_Q, m->cset_S, m->cset_meta, m->cset_flags, s);
  if (e != PD_OK) return e;
  int flags = 0;
  PD_CUDA_TRY(cudaMemcpyAsync(&flags, m->cset_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  PD_CUDA_TRY(cudaStreamSynchronize(s));
  if (flags & DEV_ERR_NOT_SPD) {
    set_error("contact set: (A^-1)_CC is not positive definite");
    return PD_ERR_NOT_SPD;
  }
  if (flags & DEV_ERR_NAN) {
    set_error("contact set: non-finite entry in the inverse factor of (A^-1)_CC");
    return PD_ERR_NAN;
  }
  m->cset = c;
  return PD_OK;
}

}  // namespace

extern "C" {

pd_status pd_contact_prepare(pd_mesh mesh, const uint8_t* candidates_host, void* stream) {
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  if (!candidates_host) {
    set_error("pd_contact_prepare: candidates are required");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const HostMesh& h = m->h;
  std::vector<int32_t> cand;
  m->cand_of_internal.assign(h.n, -1);
  for (int64_t k = 0; k < h.n; ++k) {
    if (!candidates_host[k]) continue;
    const int32_t in = h.internal_of_kept[k];
    if (in >= h.nf) continue;   // fixed nodes are never in contact
    m->cand_of_internal[in] = (int32_t)cand.size();
    cand.push_back(in);
  }
  m->ncand = (int64_t)cand.size();
  m->cand_host = cand;
  PD_CUDA_TRY(cudaStreamSynchronize(s));   // earlier work may still read the old buffers
  dfree(m, &m->cand);
  dfree(m, &m->Bc);
  dfree(m, &m->cand_buf);
  PD_CUDA_TRY(upload(m, &m->cand, cand));
  PD_CUDA_TRY(dalloc(m, &m->Bc, (size_t)std::max<int64_t>(h.nf * m->ncand, 1)));
  PD_CUDA_TRY(dalloc(m, &m->cand_buf, (size_t)std::max<int64_t>(3 * m->ncand, 3)));
  if (!m->held) PD_CUDA_TRY(dalloc(m, &m->held, (size_t)std::max<int64_t>(h.nf, 1)));
  Workspace& w = m->ws;
  for (int64_t k0 = 0; k0 < m->ncand; k0 += 3) {
    const int count = (int)std::min<int64_t>(3, m->ncand - k0);
    PD_CUDA_TRY(contact_unit_rhs(h.nf, m->cand, k0, count, w.iov, s));
    PD_CUDA_TRY(reset_solve_counters(m, s));
    PD_CUDA_TRY(solve_A(m, nullptr, w.iov, w.iox, PD_PREC_FP64, s));
    PD_CUDA_TRY(contact_extract_columns(h.nf, w.iox, k0, count, m->Bc, s));
  }
  PD_CUDA_TRY(cudaStreamSynchronize(s));
  m->contact_gen = m->factor_gen;
  m->cset = 0;
  return PD_OK;
}

pd_status pd_contact_set(pd_mesh mesh, const int32_t* nodes_host, int64_t c, void* stream) {
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  MeshImpl* m = &mesh->impl;
  if (m->contact_gen != m->factor_gen) {
    set_error("pd_contact_set: call pd_contact_prepare after the last pd_factorize");
    return PD_ERR_INVALID_ARG;
  }
  if (c < 0 || (c > 0 && !nodes_host) || c > m->ncand) {
    set_error("pd_contact_set: invalid contact set size");
    return PD_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  const HostMesh& h = m->h;
  std::vector<int32_t> node(c);
  for (int64_t k = 0; k < c; ++k) {
    const int32_t kept = nodes_host[k];
    if (kept < 0 || kept >= h.n) {
      set_error("pd_contact_set: node id out of range");
      return PD_ERR_INVALID_ARG;
    }
    node[k] = h.internal_of_kept[kept];
  }
  return contact_apply(m, node, (cudaStream_t)stream);
}

pd_status pd_contact_step_set(pd_mesh mesh, int32_t t, int32_t* nodes_host, uint8_t* rules_host, int64_t cap,
                              int64_t* count) {
  if (!mesh || !count) {
    set_error("pd_contact_step_set: null argument");
    return PD_ERR_INVALID_ARG;
  }
  MeshImpl* m = &mesh->impl;
  *count = 0;
  if (t < 0 || t >= (int32_t)m->contact_log_node.size()) {
    set_error("pd_contact_step_set: no such step in the last complementarity forward pass");
    return PD_ERR_INVALID_ARG;
  }
  const std::vector<int32_t>& node = m->contact_log_node[t];
  const std::vector<uint8_t>& rule = m->contact_log_rule[t];
  *count = (int64_t)node.size();
  if (cap < *count || (*count > 0 && !nodes_host)) {
    set_error("pd_contact_step_set: output capacity too small");
    return PD_ERR_INVALID_ARG;
  }
  for (size_t k = 0; k < node.size(); ++k) {
    nodes_host[k] = m->h.kept_of_internal[node[k]];
    if (rules_host) rules_host[k] = rule[k];
  }
  return PD_OK;
}

pd_status pd_solve_A_contact(pd_mesh mesh, const double* b, const double* x_star, double* x, int32_t precision,
                             void* stream) {
  pd_status ck = check_mesh(mesh, true);
  if (ck != PD_OK) return ck;
  MeshImpl* m = &mesh->impl;
  if (!b || !x || (m->cset > 0 && !x_star)) {
    set_error("pd_solve_A_contact: b, x and (with a contact set) x_star are required");
    return PD_ERR_INVALID_ARG;
  }
  if (m->contact_gen != m->factor_gen) {
    set_error("pd_solve_A_contact: call pd_contact_prepare after the last pd_factorize");
    return PD_ERR_INVALID_ARG;
  }
  if (precision == PD_PREC_MIXED && !m->Q32) {
    set_error("pd_solve_A_contact: FP32 panels exist only after a PD_PREC_MIXED factorisation");
    return PD_ERR_INVALID_ARG;
  }
  DeviceGuard g(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = m->ws;
  const int64_t n = m->h.n;
  kept_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, m->kept_of_internal, b, w.iov);
  PD_CUDA_TRY(reset_solve_counters(m, s));
  PD_CUDA_TRY(solve_A(m, nullptr, w.iov, w.iox, precision, s));
  PD_CUDA_TRY(contact_correct(m->h.nf, m->Bc, m->cset_node, m->cset_cand, m->cset, m->cset_Q, m->cset_S,
                              m->cset_a, m->cset_u, m->cset_lam, w.iox, x_star, w.iov, s));
  internal_to_kept_kernel<<<grid_for(n), 256, 0, s>>>(n, m->h.nf, m->kept_of_internal, w.iov, x);
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

}  // extern "C"
