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
// One launch per level and direction; each CTA owns a block of panel rows
// (forward) or columns (backward), reads its panel block once with coalesced
// column-major loads and writes disjoint outputs, so no atomics are needed and
// every sum runs in a fixed order.
#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerTask = 64;    // forward: rows per CTA (4 column groups)
constexpr int kColsPerTask = 32;    // backward: columns per CTA (8 warps x 4)
constexpr int kChunk = 512;         // staged vector chunk

struct SolveParams {
  const IterState* gate;
  const int64_t *snode_first, *row_ptr, *panel_off, *rel_ptr, *gath_ptr;
  const int32_t *rows, *gath;
  const int2* tasks;
  const void* Q;
  const double* b;
  void* u;       // (3 nf) T
  void* W;       // (3 * below rows) T
  double* x;     // (3 nf)
};

template <typename T>
__global__ void __launch_bounds__(kThreads) fwd_level_kernel(SolveParams p, int64_t task_off) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  const int2 task = p.tasks[task_off + blockIdx.x];
  const int64_t s = task.x, row0 = task.y;
  const int64_t first = p.snode_first[s];
  const int64_t nc = p.snode_first[s + 1] - first;
  const int64_t nr = p.row_ptr[s + 1] - p.row_ptr[s];
  const int64_t pos = p.row_ptr[s];
  const T* Q = reinterpret_cast<const T*>(p.Q) + p.panel_off[s];
  const T* W = reinterpret_cast<const T*>(p.W);
  const int rl = threadIdx.x % kRowsPerTask;
  const int grp = threadIdx.x / kRowsPerTask;     // 0..3
  const int64_t r = row0 + rl;
  const bool valid = r < nr;
  // columns that can be nonzero for the task's rows (L11^-1 is lower triangular)
  const int64_t jmax = (row0 + kRowsPerTask <= nc) ? row0 + kRowsPerTask : nc;
  __shared__ T rhs[kChunk][3];
  __shared__ T red[kThreads / kRowsPerTask][kRowsPerTask][3];
  T acc0 = T(0), acc1 = T(0), acc2 = T(0);
  for (int64_t j0 = 0; j0 < jmax; j0 += kChunk) {
    const int64_t jn = min((int64_t)kChunk, jmax - j0);
    __syncthreads();
    for (int64_t jj = threadIdx.x; jj < jn; jj += kThreads) {
      const int64_t j = j0 + jj;
      const int64_t c = first + j;
      double v0 = p.b[3 * c], v1 = p.b[3 * c + 1], v2 = p.b[3 * c + 2];
      for (int64_t g = p.gath_ptr[pos + j]; g < p.gath_ptr[pos + j + 1]; ++g) {
        const int64_t wr = (int64_t)p.gath[g] * 3;
        v0 -= (double)W[wr];
        v1 -= (double)W[wr + 1];
        v2 -= (double)W[wr + 2];
      }
      rhs[jj][0] = (T)v0;
      rhs[jj][1] = (T)v1;
      rhs[jj][2] = (T)v2;
    }
    __syncthreads();
    if (valid) {
      const int64_t jend = (r < nc) ? min(jn, r - j0 + 1) : jn;
      for (int64_t jj = grp; jj < jend; jj += kThreads / kRowsPerTask) {
        const T q = Q[r + (j0 + jj) * nr];
        acc0 += q * rhs[jj][0];
        acc1 += q * rhs[jj][1];
        acc2 += q * rhs[jj][2];
      }
    }
  }
  red[grp][rl][0] = acc0;
  red[grp][rl][1] = acc1;
  red[grp][rl][2] = acc2;
  __syncthreads();
  if (grp == 0 && valid) {
    T o[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T t = red[0][rl][i];
#pragma unroll
      for (int g = 1; g < kThreads / kRowsPerTask; ++g) t += red[g][rl][i];
      o[i] = t;
    }
    if (r < nc) {
      T* u = reinterpret_cast<T*>(p.u) + 3 * (first + r);
      u[0] = o[0];
      u[1] = o[1];
      u[2] = o[2];
    } else {
      double v0 = (double)o[0], v1 = (double)o[1], v2 = (double)o[2];
      for (int64_t g = p.gath_ptr[pos + r]; g < p.gath_ptr[pos + r + 1]; ++g) {
        const int64_t wr = (int64_t)p.gath[g] * 3;
        v0 += (double)W[wr];
        v1 += (double)W[wr + 1];
        v2 += (double)W[wr + 2];
      }
      T* Wo = reinterpret_cast<T*>(p.W) + 3 * (p.rel_ptr[s] + (r - nc));
      Wo[0] = (T)v0;
      Wo[1] = (T)v1;
      Wo[2] = (T)v2;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) bwd_level_kernel(SolveParams p, int64_t task_off) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  const int2 task = p.tasks[task_off + blockIdx.x];
  const int64_t s = task.x, col0 = task.y;
  const int64_t first = p.snode_first[s];
  const int64_t nc = p.snode_first[s + 1] - first;
  const int64_t nr = p.row_ptr[s + 1] - p.row_ptr[s];
  const int32_t* srows = p.rows + p.row_ptr[s];
  const T* Q = reinterpret_cast<const T*>(p.Q) + p.panel_off[s];
  const T* u = reinterpret_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kPerWarp = kColsPerTask / (kThreads / 32);   // 4
  __shared__ T v[kChunk][3];
  T acc[kPerWarp][3];
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) acc[c][0] = acc[c][1] = acc[c][2] = T(0);
  // column j of L11^-1 is zero above row j
  for (int64_t r0 = col0; r0 < nr; r0 += kChunk) {
    const int64_t rn = min((int64_t)kChunk, nr - r0);
    __syncthreads();
    for (int64_t rr = threadIdx.x; rr < rn; rr += kThreads) {
      const int64_t r = r0 + rr;
      if (r < nc) {
        const T* ur = u + 3 * (first + r);
        v[rr][0] = ur[0];
        v[rr][1] = ur[1];
        v[rr][2] = ur[2];
      } else {
        const int64_t g = srows[r];
        v[rr][0] = (T)(-p.x[3 * g]);
        v[rr][1] = (T)(-p.x[3 * g + 1]);
        v[rr][2] = (T)(-p.x[3 * g + 2]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kPerWarp; ++c) {
      const int64_t j = col0 + warp * kPerWarp + c;
      if (j >= nc) continue;
      const T* Qj = Q + j * nr;
      const int64_t rstart = max((int64_t)0, j - r0);
      for (int64_t rr = rstart + lane; rr < rn; rr += 32) {
        const T q = Qj[r0 + rr];
        acc[c][0] += q * v[rr][0];
        acc[c][1] += q * v[rr][1];
        acc[c][2] += q * v[rr][2];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kPerWarp; ++c) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T t = acc[c][i];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      acc[c][i] = t;
    }
    const int64_t j = col0 + warp * kPerWarp + c;
    if (lane == 0 && j < nc) {
      p.x[3 * (first + j)] = (double)acc[c][0];
      p.x[3 * (first + j) + 1] = (double)acc[c][1];
      p.x[3 * (first + j) + 2] = (double)acc[c][2];
    }
  }
}

}  // namespace

// Builds the per-level task lists (host) -- called once per mesh.
void build_solve_schedule(const HostMesh& h, std::vector<int2>& fwd, std::vector<int2>& bwd,
                          std::vector<SolveLevel>& levels) {
  fwd.clear();
  bwd.clear();
  levels.assign(h.nlev, SolveLevel{});
  for (int64_t L = 0; L < h.nlev; ++L) {
    SolveLevel& sl = levels[L];
    sl.fwd_off = (int64_t)fwd.size();
    sl.bwd_off = (int64_t)bwd.size();
    for (int64_t i = h.level_ptr[L]; i < h.level_ptr[L + 1]; ++i) {
      const int64_t s = h.level_list[i];
      for (int64_t r = 0; r < h.nr(s); r += kRowsPerTask) fwd.push_back(make_int2((int)s, (int)r));
      for (int64_t c = 0; c < h.nc(s); c += kColsPerTask) bwd.push_back(make_int2((int)s, (int)c));
    }
    sl.fwd_cnt = (int64_t)fwd.size() - sl.fwd_off;
    sl.bwd_cnt = (int64_t)bwd.size() - sl.bwd_off;
  }
}

cudaError_t solve_A(const MeshImpl* m, const IterState* gate, const double* b, double* out,
                    int precision, cudaStream_t st) {
  SolveParams p{};
  p.gate = gate;
  p.snode_first = m->snode_first;
  p.row_ptr = m->row_ptr;
  p.panel_off = m->panel_off;
  p.rel_ptr = m->rel_ptr;
  p.gath_ptr = m->gath_ptr;
  p.rows = m->rows;
  p.gath = m->gath;
  p.b = b;
  p.u = m->ws.solve_u;
  p.W = m->ws.solve_W;
  p.x = out;
  const bool f32 = precision == PD_PREC_MIXED;
  p.Q = f32 ? (const void*)m->Q32 : (const void*)m->Q64;
  const int64_t nlev = (int64_t)m->slevels.size();
  p.tasks = m->fwd_tasks;
  for (int64_t L = 0; L < nlev; ++L) {
    const SolveLevel& sl = m->slevels[L];
    if (sl.fwd_cnt == 0) continue;
    if (f32) fwd_level_kernel<float><<<(unsigned)sl.fwd_cnt, kThreads, 0, st>>>(p, sl.fwd_off);
    else fwd_level_kernel<double><<<(unsigned)sl.fwd_cnt, kThreads, 0, st>>>(p, sl.fwd_off);
  }
  p.tasks = m->bwd_tasks;
  for (int64_t L = nlev - 1; L >= 0; --L) {
    const SolveLevel& sl = m->slevels[L];
    if (sl.bwd_cnt == 0) continue;
    if (f32) bwd_level_kernel<float><<<(unsigned)sl.bwd_cnt, kThreads, 0, st>>>(p, sl.bwd_off);
    else bwd_level_kernel<double><<<(unsigned)sl.bwd_cnt, kThreads, 0, st>>>(p, sl.bwd_off);
  }
  return cudaGetLastError();
}

}  // namespace pd
