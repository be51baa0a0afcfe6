// Global step of PD (Alg. 1) and of the adjoint iteration (Alg. 2):
// x = A^-1 b with the prefactorised A (Sec. 3, "each global step requires
// back-substitution only").  A = I_3 (x) L_A, so one scalar factor serves the
// three coordinate columns, stored node-major (3 values per column).
//
// With the solve panels Q_s = [L11^-1; L21 L11^-1] (kernels_factor.cu) the
// substitutions of supernode s are dense products:
//   forward  (leaves -> root):  rhs = b[cols] - (children updates on cols)
//                               [u_s; w_s] = Q_s rhs,  W_s = w_s + (children
//                               updates on the below rows)
//   backward (root -> leaves):  x_s = Q_s^T [u_s; -x(below rows)]
// The panels are cut into 2D tiles (forward: 64 rows x 128 columns, backward:
// 256 rows x 32 columns; all-zero tiles of the triangular L11^-1 block are
// skipped), so that even the single root supernode spreads over many SMs, and
// every thread keeps many independent panel loads in flight.  Tiles sharing an
// output block write partial sums; the last tile to finish (integer ticket) adds
// them in tile order, so the result does not depend on scheduling and no float
// atomics run.  Both sweeps run in one persistent launch scheduled by the
// supernodal tree dependencies (below).
#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kThreads = 256;
constexpr int kFR = 64;     // forward tile rows
constexpr int kFC = 128;    // forward tile columns (8 warps x 16)
constexpr int kBR = 256;    // backward tile rows (32 lanes x 8)
constexpr int kBC = 32;     // backward tile columns (8 warps x 4)

struct SolveParams {
  const IterState* gate;
  const int32_t *rows, *slots;  // slots: (positions x slot_w) W-row sources, -1 = none
  int slot_w;
  const SolveTile* tiles;
  // persistent kernel
  int64_t ntiles;               // forward tiles then backward tiles
  unsigned long long* gticket;  // tile tickets (grid + ntiles consumed per solve)
  unsigned long long* otick;    // per output block (64-bit, monotone)
  unsigned long long* fdone;    // per supernode: finished forward output blocks
  unsigned long long* bdone;    // per supernode: finished backward output blocks
  const int32_t *nfb, *nbb;     // per supernode: forward / backward output blocks
  const int64_t *child_ptr, *child_list, *parent;
  int* err;
  void* partial;                // per tile partial sums (T)
  const void* Q;
  const double* b;
  void* u;       // (3 nf) T
  void* W;       // (3 * below rows) T
  double* x;     // (3 nf)
};

__device__ __forceinline__ SolveTile load_tile(const SolveTile* t, int64_t i) {
  const int4* p = reinterpret_cast<const int4*>(t + i);
  SolveTile r;
  int4* q = reinterpret_cast<int4*>(&r);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(SolveTile) / 16); ++k) q[k] = __ldg(p + k);
  return r;
}

// ------------------------------------------------------------ persistent
// Whole solve (forward and backward sweeps) in one launch.  CTAs take tiles in
// ticket order; a forward tile waits for its supernode's children to finish
// their forward outputs, a backward tile for its parent's backward outputs (the
// root for its own forward outputs).  Every awaited tile has an earlier ticket
// and is held by a running CTA, so the waits end; they are also bounded (error
// flag DEV_ERR_TIMEOUT).  Counters only grow: a solve consumes ntiles + grid
// tickets (every CTA draws one ticket past the end), so ticket t belongs to
// solve t / (ntiles + grid).
constexpr long long kSpinLimit = 1ll << 20;   // about a second of polling

__device__ __forceinline__ unsigned long long vload(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ bool wait_count(const unsigned long long* c, unsigned long long target, int* err) {
  long long it = 0;
  while (vload(c) < target) {
    if (++it > kSpinLimit) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

template <typename T>
__device__ __forceinline__ void gather_W_cg(const SolveParams& p, const T* W, int64_t pos, double& v0, double& v1,
                                            double& v2) {
  for (int k = 0; k < p.slot_w; ++k) {
    const int32_t g = __ldg(p.slots + pos * p.slot_w + k);
    if (g >= 0) {
      v0 += (double)__ldcg(W + 3 * (int64_t)g);
      v1 += (double)__ldcg(W + 3 * (int64_t)g + 1);
      v2 += (double)__ldcg(W + 3 * (int64_t)g + 2);
    }
  }
}

struct __align__(16) PersistSmem {
  double rhs_d[kFC][3];
  double red_d[kThreads / 32][kFR][3];
  double v_d[kBR][3];
  double res_d[kBC][3];
  int flag;
};

template <typename T>
__device__ void fwd_tile_body(const SolveParams& p, const SolveTile& tl, int64_t tid_g,
                              unsigned long long epoch, PersistSmem& sm) {
  T (*rhs)[3] = reinterpret_cast<T (*)[3]>(sm.rhs_d);
  T (*red)[kFR][3] = reinterpret_cast<T (*)[kFR][3]>(sm.red_d);
  const int64_t row0 = tl.a, col0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr, pos = tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* W = reinterpret_cast<const T*>(p.W);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cn = min((int64_t)kFC, nc - col0);
  const int64_t ra = row0 + lane, rb = row0 + 32 + lane;
  T qa[16], qb[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t j = col0 + warp * 16 + k;
    const bool jv = (warp * 16 + k) < cn;
    qa[k] = (jv && ra < nr && (ra >= nc || j <= ra)) ? __ldg(Q + ra + j * nr) : T(0);
    qb[k] = (jv && rb < nr && (rb >= nc || j <= rb)) ? __ldg(Q + rb + j * nr) : T(0);
  }
  // the children's update rows must be final
  if (threadIdx.x == 0) {
    for (int64_t ci = p.child_ptr[tl.s]; ci < p.child_ptr[tl.s + 1]; ++ci) {
      const int64_t c = p.child_list[ci];
      wait_count(p.fdone + c, (epoch + 1) * (unsigned long long)p.nfb[c], p.err);
    }
    __threadfence();
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < kFC; jj += kThreads) {
    T r0 = T(0), r1 = T(0), r2 = T(0);
    if (jj < cn) {
      const int64_t j = col0 + jj, c = first + j;
      double w0 = 0, w1 = 0, w2 = 0;
      gather_W_cg<T>(p, W, pos + j, w0, w1, w2);
      r0 = (T)(p.b[3 * c] - w0);
      r1 = (T)(p.b[3 * c + 1] - w1);
      r2 = (T)(p.b[3 * c + 2] - w2);
    }
    rhs[jj][0] = r0; rhs[jj][1] = r1; rhs[jj][2] = r2;
  }
  __syncthreads();
  T a0[3] = {T(0), T(0), T(0)}, a1[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int jj = warp * 16 + k;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a0[i] += qa[k] * rhs[jj][i];
      a1[i] += qb[k] * rhs[jj][i];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    red[warp][lane][i] = a0[i];
    red[warp][lane + 32][i] = a1[i];
  }
  __syncthreads();
  const int ntile = tl.ntile;
  T* part = reinterpret_cast<T*>(p.partial) + tid_g * (kFR * 3);
  for (int idx = threadIdx.x; idx < kFR * 3; idx += kThreads) {
    const int r = idx / 3, i = idx % 3;
    T t = T(0);
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += red[w][r][i];
    if (ntile == 1) red[0][r][i] = t;
    else part[idx] = t;
  }
  if (ntile > 1) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned long long v = atomicAdd(p.otick + tl.out, 1ull);
      sm.flag = ((v + 1) % (unsigned long long)ntile) == 0;
    }
    __syncthreads();
    if (!sm.flag) return;
    __threadfence();
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * (kFR * 3);
    for (int idx = threadIdx.x; idx < kFR * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * (kFR * 3) + idx);
      red[0][idx / 3][idx % 3] = t;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < kFR; r += kThreads) {
    const int64_t row = row0 + r;
    if (row >= nr) continue;
    if (row < nc) {
      T* uo = reinterpret_cast<T*>(p.u) + 3 * (first + row);
      uo[0] = red[0][r][0]; uo[1] = red[0][r][1]; uo[2] = red[0][r][2];
    } else {
      double v0 = (double)red[0][r][0], v1 = (double)red[0][r][1], v2 = (double)red[0][r][2];
      gather_W_cg<T>(p, W, pos + row, v0, v1, v2);
      T* Wo = reinterpret_cast<T*>(p.W) + 3 * (tl.relp + (row - nc));
      Wo[0] = (T)v0; Wo[1] = (T)v1; Wo[2] = (T)v2;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(p.fdone + tl.s, 1ull);
}

template <typename T>
__device__ void bwd_tile_body(const SolveParams& p, const SolveTile& tl, int64_t tid_g,
                              unsigned long long epoch, PersistSmem& sm) {
  T (*v)[3] = reinterpret_cast<T (*)[3]>(sm.v_d);
  T (*res)[3] = reinterpret_cast<T (*)[3]>(sm.res_d);
  const int64_t col0 = tl.a, row0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr;
  const int32_t* srows = p.rows + tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* u = reinterpret_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kPerWarp = kBC / (kThreads / 32);
  T q[kPerWarp][8];
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) {
    const int64_t j = col0 + warp * kPerWarp + c;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t r = row0 + lane + 32 * k;
      q[c][k] = (j < nc && r < nr && (r >= nc || r >= j)) ? __ldg(Q + r + j * nr) : T(0);
    }
  }
  // the parent's solution (the root: its own forward outputs) must be final
  if (threadIdx.x == 0) {
    const int64_t par = p.parent[tl.s];
    if (par >= 0) wait_count(p.bdone + par, (epoch + 1) * (unsigned long long)p.nbb[par], p.err);
    else wait_count(p.fdone + tl.s, (epoch + 1) * (unsigned long long)p.nfb[tl.s], p.err);
    __threadfence();
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < kBR; rr += kThreads) {
    const int64_t r = row0 + rr;
    T v0 = T(0), v1 = T(0), v2 = T(0);
    if (r < nr) {
      if (r < nc) {
        const T* ur = u + 3 * (first + r);
        v0 = __ldcg(ur); v1 = __ldcg(ur + 1); v2 = __ldcg(ur + 2);
      } else {
        const int64_t g = __ldg(srows + r);
        v0 = (T)(-__ldcg(p.x + 3 * g)); v1 = (T)(-__ldcg(p.x + 3 * g + 1)); v2 = (T)(-__ldcg(p.x + 3 * g + 2));
      }
    }
    v[rr][0] = v0; v[rr][1] = v1; v[rr][2] = v2;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) {
    const int jl = warp * kPerWarp + c;
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) acc[i] += q[c][k] * v[lane + 32 * k][i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T t = acc[i];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (lane == 0) res[jl][i] = t;
    }
  }
  __syncthreads();
  const int ntile = tl.ntile;
  if (ntile > 1) {
    T* part = reinterpret_cast<T*>(p.partial) + tid_g * (kFR * 3);
    for (int idx = threadIdx.x; idx < kBC * 3; idx += kThreads) part[idx] = res[idx / 3][idx % 3];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned long long vv = atomicAdd(p.otick + tl.out, 1ull);
      sm.flag = ((vv + 1) % (unsigned long long)ntile) == 0;
    }
    __syncthreads();
    if (!sm.flag) return;
    __threadfence();
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * (kFR * 3);
    for (int idx = threadIdx.x; idx < kBC * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * (kFR * 3) + idx);
      res[idx / 3][idx % 3] = t;
    }
    __syncthreads();
  }
  for (int jl = threadIdx.x; jl < kBC; jl += kThreads) {
    const int64_t j = col0 + jl;
    if (j >= nc) continue;
    p.x[3 * (first + j)] = (double)res[jl][0];
    p.x[3 * (first + j) + 1] = (double)res[jl][1];
    p.x[3 * (first + j) + 2] = (double)res[jl][2];
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(p.bdone + tl.s, 1ull);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) solve_persistent_kernel(SolveParams p) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  __shared__ PersistSmem sm;
  __shared__ unsigned long long tk;
  const unsigned long long per = (unsigned long long)p.ntiles + gridDim.x;
  while (true) {
    __syncthreads();   // shared memory of the previous tile is no longer in use
    if (threadIdx.x == 0) tk = atomicAdd(p.gticket, 1ull);
    __syncthreads();
    const unsigned long long t = tk;
    const unsigned long long epoch = t / per;
    const int64_t tile = (int64_t)(t % per);
    if (tile >= p.ntiles) return;
    const SolveTile tl = load_tile(p.tiles, tile);
    if (tl.pad0 == 0) fwd_tile_body<T>(p, tl, tile, epoch, sm);
    else bwd_tile_body<T>(p, tl, tile, epoch, sm);
  }
}

}  // namespace

// Builds the per-level tile lists (host) -- called once per mesh.  Tiles of one
// output block are contiguous, so part_base indexes their partial sums.
void build_solve_schedule(const HostMesh& h, SolveSchedule& S) {
  S.fwd.clear();
  S.bwd.clear();
  S.n_fwd_out = S.n_bwd_out = 0;
  S.levels.assign(h.nlev, SolveLevel{});
  auto base = [&](int64_t s) {
    SolveTile t{};
    t.panel_off = h.panel_off[s];
    t.s = (int32_t)s;
    t.first = (int32_t)h.snode_first[s];
    t.nc = (int32_t)h.nc(s);
    t.nr = (int32_t)h.nr(s);
    t.pos = (int32_t)h.row_ptr[s];
    t.relp = (int32_t)h.rel_ptr[s];
    return t;
  };
  for (int64_t L = 0; L < h.nlev; ++L) {
    SolveLevel& sl = S.levels[L];
    sl.fwd_off = (int64_t)S.fwd.size();
    sl.bwd_off = (int64_t)S.bwd.size();
    for (int64_t i = h.level_ptr[L]; i < h.level_ptr[L + 1]; ++i) {
      const int64_t s = h.level_list[i];
      const int64_t nr = h.nr(s), nc = h.nc(s);
      for (int64_t r0 = 0; r0 < nr; r0 += kFR) {
        const int32_t out = (int32_t)S.n_fwd_out++;
        const size_t b0 = S.fwd.size();
        // rows < nc of the L11^-1 block need columns <= row only
        const int64_t cmax = (r0 + kFR <= nc) ? r0 + kFR : nc;
        for (int64_t c0 = 0; c0 < cmax; c0 += kFC) {
          SolveTile t = base(s);
          t.a = (int32_t)r0;
          t.b = (int32_t)c0;
          t.out = out;
          t.part_base = (int64_t)b0;
          S.fwd.push_back(t);
        }
        for (size_t k = b0; k < S.fwd.size(); ++k) S.fwd[k].ntile = (int32_t)(S.fwd.size() - b0);
      }
      for (int64_t c0 = 0; c0 < nc; c0 += kBC) {
        const int32_t out = (int32_t)S.n_bwd_out++;
        const size_t b0 = S.bwd.size();
        // column c of L11^-1 is zero above row c
        for (int64_t r0 = (c0 / kBR) * kBR; r0 < nr; r0 += kBR) {
          SolveTile t = base(s);
          t.a = (int32_t)c0;
          t.b = (int32_t)r0;
          t.out = out;
          t.part_base = (int64_t)b0;
          S.bwd.push_back(t);
        }
        for (size_t k = b0; k < S.bwd.size(); ++k) S.bwd[k].ntile = (int32_t)(S.bwd.size() - b0);
      }
    }
    sl.fwd_cnt = (int64_t)S.fwd.size() - sl.fwd_off;
    sl.bwd_cnt = (int64_t)S.bwd.size() - sl.bwd_off;
  }
  S.nfb.assign(h.ns, 0);
  S.nbb.assign(h.ns, 0);
  for (int64_t s2 = 0; s2 < h.ns; ++s2) {
    S.nfb[s2] = (int32_t)((h.nr(s2) + kFR - 1) / kFR);
    S.nbb[s2] = (int32_t)((h.nc(s2) + kBC - 1) / kBC);
  }
  // persistent order: forward tiles by ascending level, backward tiles by
  // descending level (tiles of one output block stay contiguous); output ids of
  // backward blocks follow the forward ones; partial slots use the global index
  S.all.clear();
  for (const SolveTile& t : S.fwd) {
    SolveTile u = t;
    u.pad0 = 0;
    S.all.push_back(u);
  }
  for (int64_t L = h.nlev - 1; L >= 0; --L) {
    const SolveLevel& sl = S.levels[L];
    const int64_t shift = (int64_t)S.all.size() - sl.bwd_off;
    for (int64_t k = sl.bwd_off; k < sl.bwd_off + sl.bwd_cnt; ++k) {
      SolveTile u = S.bwd[k];
      u.pad0 = 1;
      u.out += (int32_t)S.n_fwd_out;
      u.part_base += shift;
      S.all.push_back(u);
    }
  }
}

size_t solve_partial_bytes(const SolveSchedule& S) {
  return std::max(S.fwd.size() * kFR * 3, (S.fwd.size() + S.bwd.size()) * kFR * 3) * sizeof(double);
}

int solve_persistent_occupancy() {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_persistent_kernel<float>, kThreads, 0);
  int occ2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, solve_persistent_kernel<double>, kThreads, 0);
  return std::max(1, std::min(occ, occ2));
}

cudaError_t solve_A(const MeshImpl* m, const IterState* gate, const double* b, double* out,
                    int precision, cudaStream_t st) {
  SolveParams p{};
  p.gate = gate;
  p.rows = m->rows;
  p.slots = m->gath_slots;
  p.slot_w = m->slot_w;
  p.b = b;
  p.u = m->ws.solve_u;
  p.W = m->ws.solve_W;
  p.partial = m->ws.solve_partial;
  p.x = out;
  const bool f32 = precision == PD_PREC_MIXED;
  p.Q = f32 ? (const void*)m->Q32 : (const void*)m->Q64;
  const int64_t ntiles = (int64_t)m->sched.all.size();
  if (ntiles == 0) return cudaSuccess;
  p.tiles = m->all_tiles;
  p.ntiles = ntiles;
  const int64_t nout = m->sched.n_fwd_out + m->sched.n_bwd_out;
  p.gticket = m->solve_counters;
  p.otick = m->solve_counters + 1;
  p.fdone = m->solve_counters + 1 + nout;
  p.bdone = m->solve_counters + 1 + nout + m->h.ns;
  p.nfb = m->nfb;
  p.nbb = m->nbb;
  p.child_ptr = m->child_ptr;
  p.child_list = m->child_list;
  p.parent = m->parent;
  p.err = m->ws.flags;
  const unsigned grid = (unsigned)std::min<int64_t>(m->solve_grid, ntiles);
  if (f32) solve_persistent_kernel<float><<<grid, kThreads, 0, st>>>(p);
  else solve_persistent_kernel<double><<<grid, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace pd
