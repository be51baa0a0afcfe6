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
// One launch per tree level and direction.  Each level is cut into 2D tiles of
// the panels (forward: 64 rows x 128 columns, backward: 256 rows x 32 columns,
// all-zero tiles of the triangular L11^-1 block skipped), so that even the
// single root supernode spreads over many SMs; every thread keeps many
// independent panel loads in flight.  Tiles sharing an output block write
// partial sums; the last tile to finish (integer ticket) adds them in tile
// order, so the result does not depend on scheduling and no float atomics run.
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
  unsigned* tickets;            // per output block
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

// sum of the update-vector rows landing on position `pos` (fixed slot order)
template <typename T>
__device__ __forceinline__ void gather_W(const SolveParams& p, const T* W, int64_t pos, double& v0, double& v1,
                                         double& v2) {
  for (int k = 0; k < p.slot_w; ++k) {
    const int32_t g = __ldg(p.slots + pos * p.slot_w + k);
    if (g >= 0) {
      v0 += (double)W[3 * (int64_t)g];
      v1 += (double)W[3 * (int64_t)g + 1];
      v2 += (double)W[3 * (int64_t)g + 2];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) fwd_tile_kernel(SolveParams p, int64_t tile_off) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  const int64_t tid_g = tile_off + blockIdx.x;
  const SolveTile tl = load_tile(p.tiles, tid_g);
  const int64_t row0 = tl.a, col0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr, pos = tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* W = reinterpret_cast<const T*>(p.W);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ T rhs[kFC][3];
  __shared__ T red[kThreads / 32][kFR][3];
  __shared__ int is_last;
  const int64_t cn = min((int64_t)kFC, nc - col0);
  // 1) panel loads first: their addresses depend on the descriptor only
  // warp w: columns col0 + 16w .. +16, lanes: rows row0 + lane, row0 + 32 + lane
  const int64_t ra = row0 + lane, rb = row0 + 32 + lane;
  T qa[16], qb[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int64_t j = col0 + warp * 16 + k;
    const bool jv = (warp * 16 + k) < cn;
    // L11^-1 is lower triangular: rows < nc only use columns <= row
    qa[k] = (jv && ra < nr && (ra >= nc || j <= ra)) ? __ldg(Q + ra + j * nr) : T(0);
    qb[k] = (jv && rb < nr && (rb >= nc || j <= rb)) ? __ldg(Q + rb + j * nr) : T(0);
  }
  // 2) right-hand side of the tile's columns: b minus the children's updates
  for (int jj = threadIdx.x; jj < kFC; jj += kThreads) {
    T r0 = T(0), r1 = T(0), r2 = T(0);
    if (jj < cn) {
      const int64_t j = col0 + jj, c = first + j;
      double w0 = 0, w1 = 0, w2 = 0;
      gather_W<T>(p, W, pos + j, w0, w1, w2);
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
  // tile partial: sum of the 8 warps
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
      const unsigned t = atomicAdd(p.tickets + tl.out, 1u);
      is_last = (t == (unsigned)ntile - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * (kFR * 3);
    for (int idx = threadIdx.x; idx < kFR * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * (kFR * 3) + idx);
      red[0][idx / 3][idx % 3] = t;
    }
    if (threadIdx.x == 0) p.tickets[tl.out] = 0u;
  }
  __syncthreads();
  // outputs: u on the supernode's columns, W on its below rows
  for (int r = threadIdx.x; r < kFR; r += kThreads) {
    const int64_t row = row0 + r;
    if (row >= nr) continue;
    if (row < nc) {
      T* uo = reinterpret_cast<T*>(p.u) + 3 * (first + row);
      uo[0] = red[0][r][0]; uo[1] = red[0][r][1]; uo[2] = red[0][r][2];
    } else {
      double v0 = (double)red[0][r][0], v1 = (double)red[0][r][1], v2 = (double)red[0][r][2];
      gather_W<T>(p, W, pos + row, v0, v1, v2);
      T* Wo = reinterpret_cast<T*>(p.W) + 3 * (tl.relp + (row - nc));
      Wo[0] = (T)v0; Wo[1] = (T)v1; Wo[2] = (T)v2;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) bwd_tile_kernel(SolveParams p, int64_t tile_off) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  const int64_t tid_g = tile_off + blockIdx.x;
  const SolveTile tl = load_tile(p.tiles, tid_g);
  const int64_t col0 = tl.a, row0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr;
  const int32_t* srows = p.rows + tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* u = reinterpret_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kPerWarp = kBC / (kThreads / 32);   // 4 columns per warp
  __shared__ T v[kBR][3];
  __shared__ T res[kBC][3];
  __shared__ int is_last;
  // 1) panel loads first; warp w: columns col0 + 4w .. +4; lane: rows row0 + lane + 32k
  T q[kPerWarp][8];
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) {
    const int64_t j = col0 + warp * kPerWarp + c;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t r = row0 + lane + 32 * k;
      // column j of L11^-1 is zero above row j
      q[c][k] = (j < nc && r < nr && (r >= nc || r >= j)) ? __ldg(Q + r + j * nr) : T(0);
    }
  }
  // 2) v = [u_s; -x(below rows)]
  for (int rr = threadIdx.x; rr < kBR; rr += kThreads) {
    const int64_t r = row0 + rr;
    T v0 = T(0), v1 = T(0), v2 = T(0);
    if (r < nr) {
      if (r < nc) {
        const T* ur = u + 3 * (first + r);
        v0 = ur[0]; v1 = ur[1]; v2 = ur[2];
      } else {
        const int64_t g = __ldg(srows + r);
        v0 = (T)(-p.x[3 * g]); v1 = (T)(-p.x[3 * g + 1]); v2 = (T)(-p.x[3 * g + 2]);
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
    T* part = reinterpret_cast<T*>(p.partial) + tid_g * (kBC * 3);
    for (int idx = threadIdx.x; idx < kBC * 3; idx += kThreads) part[idx] = res[idx / 3][idx % 3];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(p.tickets + tl.out, 1u);
      is_last = (t == (unsigned)ntile - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * (kBC * 3);
    for (int idx = threadIdx.x; idx < kBC * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * (kBC * 3) + idx);
      res[idx / 3][idx % 3] = t;
    }
    if (threadIdx.x == 0) p.tickets[tl.out] = 0u;
    __syncthreads();
  }
  for (int jl = threadIdx.x; jl < kBC; jl += kThreads) {
    const int64_t j = col0 + jl;
    if (j >= nc) continue;
    p.x[3 * (first + j)] = (double)res[jl][0];
    p.x[3 * (first + j) + 1] = (double)res[jl][1];
    p.x[3 * (first + j) + 2] = (double)res[jl][2];
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
}

size_t solve_partial_bytes(const SolveSchedule& S) {
  return std::max(S.fwd.size() * kFR * 3, S.bwd.size() * kBC * 3) * sizeof(double);
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
  const int64_t nlev = (int64_t)m->sched.levels.size();
  p.tiles = m->fwd_tiles;
  p.tickets = m->ws.solve_tickets;
  for (int64_t L = 0; L < nlev; ++L) {
    const SolveLevel& sl = m->sched.levels[L];
    if (sl.fwd_cnt == 0) continue;
    if (f32) fwd_tile_kernel<float><<<(unsigned)sl.fwd_cnt, kThreads, 0, st>>>(p, sl.fwd_off);
    else fwd_tile_kernel<double><<<(unsigned)sl.fwd_cnt, kThreads, 0, st>>>(p, sl.fwd_off);
  }
  p.tiles = m->bwd_tiles;
  p.tickets = m->ws.solve_tickets + m->sched.n_fwd_out;
  for (int64_t L = nlev - 1; L >= 0; --L) {
    const SolveLevel& sl = m->sched.levels[L];
    if (sl.bwd_cnt == 0) continue;
    if (f32) bwd_tile_kernel<float><<<(unsigned)sl.bwd_cnt, kThreads, 0, st>>>(p, sl.bwd_off);
    else bwd_tile_kernel<double><<<(unsigned)sl.bwd_cnt, kThreads, 0, st>>>(p, sl.bwd_off);
  }
  return cudaGetLastError();
}

}  // namespace pd
