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
constexpr int kFR = 256;    // forward tile rows (one thread per row)
constexpr int kFC = 256;    // forward tile columns
constexpr int kBR = 1024;   // backward tile rows (32 lanes x 32)
constexpr int kBC = 32;     // backward tile columns (8 warps x 4)
constexpr int kPart = kFR * 3;   // partial-sum slots per tile

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
  double rhs_d[kFC][3];   // forward: right-hand side of the tile's columns
  double v_d[kBR][3];     // backward: [u_s; -x(below rows)] of the tile's rows
  double res_d[kBC][3];
  int flag;
};

// last of the tiles of an output block?  (then the partial sums are complete)
__device__ __forceinline__ bool last_of_block(const SolveParams& p, const SolveTile& tl, PersistSmem& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long v = atomicAdd(p.otick + tl.out, 1ull);
    const bool last = ((v + 1) % (unsigned long long)tl.ntile) == 0;
    if (last) __threadfence();
    sm.flag = last;
  }
  __syncthreads();
  return sm.flag != 0;
}

__device__ __forceinline__ void signal_done(unsigned long long* c) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(c, 1ull);
  }
}

// Forward tile: rows [a, a + kFR) x columns [b, b + kFC) of panel s; thread t
// owns row a + t and accumulates its whole dot product over the tile's columns
// (coalesced: consecutive threads read consecutive rows of one column).
template <typename T>
__device__ void fwd_tile_body(const SolveParams& p, const SolveTile& tl, int64_t tid_g, unsigned long long epoch,
                              PersistSmem& sm) {
  T (*rhs)[3] = reinterpret_cast<T (*)[3]>(sm.rhs_d);
  const int64_t row0 = tl.a, col0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr, pos = tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* W = reinterpret_cast<const T*>(p.W);
  const int64_t cn = min((int64_t)kFC, nc - col0);
  const int64_t r = row0 + threadIdx.x;
  const bool valid = r < nr;
  // L11^-1 is lower triangular: rows < nc use columns <= row only
  const int64_t jend = !valid ? 0 : (r < nc ? min(cn, r - col0 + 1) : cn);
  const T* Qr = Q + r + col0 * nr;
  // the first panel values load while the dependencies are awaited
  constexpr int kPre = 16;
  T pre[kPre];
#pragma unroll
  for (int k = 0; k < kPre; ++k) pre[k] = (k < jend) ? __ldg(Qr + (int64_t)k * nr) : T(0);
  if (threadIdx.x == 0) {
    for (int64_t ci = __ldg(p.child_ptr + tl.s); ci < __ldg(p.child_ptr + tl.s + 1); ++ci) {
      const int64_t c = __ldg(p.child_list + ci);
      wait_count(p.fdone + c, (epoch + 1) * (unsigned long long)__ldg(p.nfb + c), p.err);
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
  T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    a0 += pre[k] * rhs[k][0];
    a1 += pre[k] * rhs[k][1];
    a2 += pre[k] * rhs[k][2];
  }
  for (int64_t j = kPre; j < jend; j += 16) {
    T q[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) q[k] = (j + k < jend) ? __ldg(Qr + (j + k) * nr) : T(0);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int64_t jj = min(j + k, (int64_t)kFC - 1);
      a0 += q[k] * rhs[jj][0];
      a1 += q[k] * rhs[jj][1];
      a2 += q[k] * rhs[jj][2];
    }
  }
  const int ntile = tl.ntile;
  if (ntile > 1) {
    T* part = reinterpret_cast<T*>(p.partial) + tid_g * kPart;
    part[3 * threadIdx.x] = a0;
    part[3 * threadIdx.x + 1] = a1;
    part[3 * threadIdx.x + 2] = a2;
    if (!last_of_block(p, tl, sm)) return;
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * kPart;
    a0 = a1 = a2 = T(0);
    for (int k = 0; k < ntile; ++k) {
      a0 += __ldcg(parts + (int64_t)k * kPart + 3 * threadIdx.x);
      a1 += __ldcg(parts + (int64_t)k * kPart + 3 * threadIdx.x + 1);
      a2 += __ldcg(parts + (int64_t)k * kPart + 3 * threadIdx.x + 2);
    }
  }
  if (valid) {
    if (r < nc) {
      T* uo = reinterpret_cast<T*>(p.u) + 3 * (first + r);
      uo[0] = a0; uo[1] = a1; uo[2] = a2;
    } else {
      double v0 = (double)a0, v1 = (double)a1, v2 = (double)a2;
      gather_W_cg<T>(p, W, pos + r, v0, v1, v2);
      T* Wo = reinterpret_cast<T*>(p.W) + 3 * (tl.relp + (r - nc));
      Wo[0] = (T)v0; Wo[1] = (T)v1; Wo[2] = (T)v2;
    }
  }
  signal_done(p.fdone + tl.s);
}

// Backward tile: columns [a, a + kBC) x rows [b, b + kBR) of panel s; warp w owns
// 4 columns, lanes stride the rows of a column (contiguous, coalesced).
template <typename T>
__device__ void bwd_tile_body(const SolveParams& p, const SolveTile& tl, int64_t tid_g, unsigned long long epoch,
                              PersistSmem& sm) {
  T (*v)[3] = reinterpret_cast<T (*)[3]>(sm.v_d);
  T (*res)[3] = reinterpret_cast<T (*)[3]>(sm.res_d);
  const int64_t col0 = tl.a, row0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr;
  const int32_t* srows = p.rows + tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* u = reinterpret_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kPerWarp = kBC / (kThreads / 32);
  const int64_t rn = min((int64_t)kBR, nr - row0);
  // first rows of each column load while the dependencies are awaited
  T pre[kPerWarp];
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) {
    const int64_t j = col0 + warp * kPerWarp + c;
    const int64_t rr = row0 + lane;
    pre[c] = (j < nc && lane < rn && (rr >= nc || rr >= j)) ? __ldg(Q + rr + j * nr) : T(0);
  }
  if (threadIdx.x == 0) {
    const int64_t par = __ldg(p.parent + tl.s);
    if (par >= 0) wait_count(p.bdone + par, (epoch + 1) * (unsigned long long)__ldg(p.nbb + par), p.err);
    else wait_count(p.fdone + tl.s, (epoch + 1) * (unsigned long long)__ldg(p.nfb + tl.s), p.err);
    __threadfence();
  }
  __syncthreads();
  for (int64_t rr = threadIdx.x; rr < rn; rr += kThreads) {
    const int64_t r = row0 + rr;
    T v0, v1, v2;
    if (r < nc) {
      const T* ur = u + 3 * (first + r);
      v0 = __ldcg(ur); v1 = __ldcg(ur + 1); v2 = __ldcg(ur + 2);
    } else {
      const int64_t g = __ldg(srows + r);
      v0 = (T)(-__ldcg(p.x + 3 * g)); v1 = (T)(-__ldcg(p.x + 3 * g + 1)); v2 = (T)(-__ldcg(p.x + 3 * g + 2));
    }
    v[rr][0] = v0; v[rr][1] = v1; v[rr][2] = v2;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) {
    const int jl = warp * kPerWarp + c;
    const int64_t j = col0 + jl;
    const int64_t l0 = min((int64_t)lane, rn - 1);
    T a0 = pre[c] * v[l0][0], a1 = pre[c] * v[l0][1], a2 = pre[c] * v[l0][2];
    if (j < nc) {
      // column j of L11^-1 is zero above row j
      const int64_t rs = max((int64_t)32, (j - row0) & ~(int64_t)31);
      const T* Qj = Q + j * nr + row0;
      for (int64_t base = rs; base < rn; base += 32 * 8) {
        T q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int64_t rr = base + lane + 32 * k;
          q[k] = (rr < rn && (row0 + rr >= nc || row0 + rr >= j)) ? __ldg(Qj + rr) : T(0);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          // rows past the tile carry q = 0; read a filled row so no stale value enters
          const int64_t rr = min(base + lane + 32 * k, rn - 1);
          a0 += q[k] * v[rr][0];
          a1 += q[k] * v[rr][1];
          a2 += q[k] * v[rr][2];
        }
      }
    }
    T t0 = a0, t1 = a1, t2 = a2;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      t0 += __shfl_xor_sync(0xffffffffu, t0, off);
      t1 += __shfl_xor_sync(0xffffffffu, t1, off);
      t2 += __shfl_xor_sync(0xffffffffu, t2, off);
    }
    if (lane == 0) { res[jl][0] = t0; res[jl][1] = t1; res[jl][2] = t2; }
  }
  __syncthreads();
  const int ntile = tl.ntile;
  if (ntile > 1) {
    T* part = reinterpret_cast<T*>(p.partial) + tid_g * kPart;
    for (int idx = threadIdx.x; idx < kBC * 3; idx += kThreads) part[idx] = res[idx / 3][idx % 3];
    if (!last_of_block(p, tl, sm)) return;
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * kPart;
    for (int idx = threadIdx.x; idx < kBC * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * kPart + idx);
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
  signal_done(p.bdone + tl.s);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) solve_persistent_kernel(SolveParams p) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  __shared__ PersistSmem sm;
  __shared__ unsigned long long tk[2];
  const unsigned long long per = (unsigned long long)p.ntiles + gridDim.x;
  if (threadIdx.x == 0) tk[0] = atomicAdd(p.gticket, 1ull);
  __syncthreads();
  int slot = 0;
  unsigned long long t = tk[0];
  while (true) {
    const int64_t tile = (int64_t)(t % per);
    if (tile >= p.ntiles) return;
    const unsigned long long epoch = t / per;
    // The next ticket is drawn now, so its latency overlaps this tile.  A CTA
    // holds at most one drawn-but-unstarted ticket, always above the one it is
    // working on, so the lowest unfinished ticket is always being worked on and
    // its dependencies (lower tickets) are done: the schedule cannot deadlock.
    // The two slots alternate: the slot written here was last read before the
    // barrier that ended the previous tile.
    if (threadIdx.x == 0) tk[slot ^ 1] = atomicAdd(p.gticket, 1ull);
    const SolveTile tl = load_tile(p.tiles, tile);
    if (tl.pad0 == 0) fwd_tile_body<T>(p, tl, tile, epoch, sm);
    else bwd_tile_body<T>(p, tl, tile, epoch, sm);
    __syncthreads();   // shared memory of this tile is free; the drawn ticket is visible
    slot ^= 1;
    t = tk[slot];
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
        // column c of L11^-1 is zero above row c: start at the row block holding c0
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
  return (S.fwd.size() + S.bwd.size()) * (size_t)kPart * sizeof(double);
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
