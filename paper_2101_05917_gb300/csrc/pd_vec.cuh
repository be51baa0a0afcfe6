// Iteration control of PD forward (Alg. 1 + L-BFGS, Sec. 4 "Further acceleration
// with quasi-Newton methods") and of the adjoint solve (Alg. 2 + L-BFGS), with
// every decision taken on the device so that the host only polls one flag.
//
// Vectors are FP64, internal node order, the free DoFs first (3 nf entries).
// Reductions: each block writes one partial; the last block to finish (integer
// ticket) sums the partials in index order, so results do not depend on block
// scheduling.
#pragma once

#include "pd_internal.cuh"
#include "pd_iter.cuh"

namespace pd {

struct StateCfg {
  double tol, noise;
  int m, ls_max, max_iter, accepted;
  int keep_history;   // keep the L-BFGS pairs of the previous solve
};

struct VecCtx {
  int64_t n3;
  IterState* st;
  double* partials;
  unsigned* counter;
  double* lpart;       // L-BFGS products: kMaxDots per block
  unsigned* lcounter;
};

struct PredParams {
  int64_t n, nf;
  const double *xi, *vi, *fext, *mass, *X;
  const uint8_t* contact;
  double k, mu, h, grav[3];
  double *y, *xt, *x;
  double* partials;
  unsigned* counter;
  IterState* st;
};

struct BwdStateParams {
  int64_t n, nf;
  const double *z, *mass, *xi, *vi;
  const uint8_t* contact;
  double k, mu, h, inv_h, inv_h2;
  double *ax, *av, *gfext;
  const double *gx_t, *gv_t;     // kept order, may be null
  const int32_t* kept_of_internal;
  double* gmu;
  double* partials;
  unsigned* counter;
};

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kT / 32; ++i) t += sh[i];
  return t;   // valid in thread 0
}

// Returns true in thread 0 of the last block, with *total = sum of all block partials.
__device__ __forceinline__ bool grid_sum(double part, double* partials, unsigned* counter, double* total) {
  const double b = block_sum(part);
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = b;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kT) acc += __ldcg(partials + i);
  const double tot = block_sum(acc);
  if (threadIdx.x == 0) {
    *counter = 0u;
    *total = tot;
  }
  return threadIdx.x == 0;
}

__device__ __forceinline__ int idx_newest(const IterState* st, int k) {
  return (st->head + st->count - 1 - k + 2 * st->m) % st->m;
}
__device__ __forceinline__ int idx_oldest(const IterState* st, int k) { return (st->head + k) % st->m; }

// reduce up to `n` values at stride `stride` (fixed order), single block
__device__ __forceinline__ double block_reduce_strided(const double* a, int64_t n, int stride, int off) {
  double acc = 0;
  // eight loads in flight per thread, added in index order
  for (int64_t i0 = threadIdx.x; i0 < n; i0 += 8 * kT) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = i0 + (int64_t)u * kT;
      v[u] = i < n ? a[i * stride + off] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  return block_sum(acc);
}

}  // namespace

inline int vec_blocks(int64_t n3) {
  int64_t b = (n3 + kT * 4 - 1) / (kT * 4);
  if (b < 1) b = 1;
  if (b > 1184) b = 1184;   // 8 x 148; partial buffers hold at least this many
  return (int)b;
}

__global__ void state_reset_kernel(IterState* st, StateCfg cfg) {
  st->alpha = 1.0;
  st->slope = 0.0;
  st->g_acc = 0.0;
  st->gn2_acc = 0.0;
  st->ref2 = 0.0;
  st->refM2 = 0.0;
  st->tol2 = cfg.tol * cfg.tol;
  st->c1 = 1e-4;
  st->noise = cfg.noise;
  if (!cfg.keep_history || st->m != cfg.m) {
    st->head = 0;
    st->count = 0;
  }
  st->m = cfg.m;
  st->pslot = 0;
  st->push = 0;
  st->iters = 0;
  st->evals = 0;
  st->ls_tries = 0;
  st->ls_total = 0;
  st->ls_max = cfg.ls_max;
  st->max_iter = cfg.max_iter;
  st->accepted = cfg.accepted;
  st->converged = 0;
  st->hit_max = 0;
  st->force_accept = 0;
  st->fp64_checked = 0;
  st->pending = 0;
  st->status = 0;
  st->svd_cached = 0;
}

// ---------------------------------------------------------------- forward
// y = x + h v + h^2 (g + (f_ext + f_fric)/m); trial xt = y on free nodes, rest
// position on Dirichlet nodes; friction from the state at the start of the step
// (Sec. 5.1: penalty friction is added to f_ext).
__global__ void predictor_kernel(PredParams p) {
  double part = 0;
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < p.n; c += (int64_t)gridDim.x * kT) {
    const double m = p.mass[c];
    double f[3] = {0, 0, 0};
    if (p.fext) { f[0] = p.fext[3 * c]; f[1] = p.fext[3 * c + 1]; f[2] = p.fext[3 * c + 2]; }
    if (p.contact && p.contact[c]) {
      const double z = p.xi[3 * c + 2];
      const double vx = p.vi[3 * c], vy = p.vi[3 * c + 1];
      const double nv = sqrt(vx * vx + vy * vy);
      if (z < 0.0 && nv > 0.0) {
        const double fn = p.k * (-z);
        const double mag = fmin(p.mu * fn, m * nv / p.h);
        f[0] -= mag * vx / nv;
        f[1] -= mag * vy / nv;
      }
    }
    if (c < p.nf) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double yv = p.xi[3 * c + i] + p.h * p.vi[3 * c + i] + p.h * p.h * (p.grav[i] + f[i] / m);
        p.y[3 * c + i] = yv;
        p.xt[3 * c + i] = yv;
        const double my = m * yv / (p.h * p.h);
        part += my * my;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        p.y[3 * c + i] = p.X[3 * c + i];
        p.xt[3 * c + i] = p.X[3 * c + i];
        p.x[3 * c + i] = p.X[3 * c + i];
      }
    }
  }
  double tot;
  if (grid_sum(part, p.partials, p.counter, &tot)) p.st->refM2 = tot;
}

__global__ void decide_fwd_kernel(IterState* st, const double* energy_partials, int64_t nbe,
                                  const double* gather_partials, int64_t nbg) {
  const double e = block_reduce_strided(energy_partials, nbe, 1, 0);
  const double kin = block_reduce_strided(gather_partials, nbg, 4, 0);
  const double gn2 = block_reduce_strided(gather_partials, nbg, 4, 1);
  const double gd = block_reduce_strided(gather_partials, nbg, 4, 2);
  if (threadIdx.x != 0) return;
  if (st->converged) return;
  const double g = e + kin;
  st->g_t = g;
  st->gn2_t = gn2;
  st->gd_t = gd;
  if (!isfinite(g) || !isfinite(gn2)) {
    st->status |= DEV_ERR_NAN;
    st->converged = 1;
    st->accepted = 0;
    return;
  }
  const bool first = st->evals == 0 || st->force_accept;
  if (st->evals == 0) st->ref2 = fmax(gn2, st->refM2);
  st->evals += 1;
  bool acc = first;
  if (!first) {
    acc = g <= st->g_acc + st->c1 * st->alpha * st->slope + st->noise * fabs(st->g_acc);
    if (!acc && st->ls_tries >= st->ls_max) acc = true;
  }
  if (acc) {
    st->push = 0;
    if (!first && st->m > 0) {
      const double sy = st->alpha * (gd - st->slope);   // s = alpha d, y = grad_t - grad
      if (sy > 0.0) {
        int slot;
        if (st->count < st->m) {
          slot = (st->head + st->count) % st->m;
          st->count += 1;
        } else {
          slot = st->head;
          st->head = (st->head + 1) % st->m;
        }
        st->rho[slot] = 1.0 / sy;
        st->pslot = slot;
        st->push = 1;
      }
    }
    st->g_acc = g;
    st->gn2_acc = gn2;
    st->accepted = 1;
    st->ls_tries = 0;
    st->force_accept = 0;
    if (!first) st->iters += 1;
    st->alpha = 1.0;
    if (gn2 <= st->tol2 * st->ref2) {
      st->converged = 1;
    } else if (st->iters >= st->max_iter) {
      st->converged = 1;
      st->hit_max = 1;
    }
  } else {
    st->accepted = 0;
    st->alpha *= 0.5;
    st->ls_tries += 1;
    st->ls_total += 1;
  }
}

// ---------------------------------------------------------------- L-BFGS
// The two-loop recursion around A^-1 (Sec. 4, quasi-Newton acceleration) in
// compact form: every inner product of a loop is expressed through products
// that do not depend on the loop's own updates,
//   s_i . q_i = s_i . g - sum_{j newer than i} al_j (s_i . y_j)
//   y_i . r_i = y_i . r0 + sum_{j older than i} (al_j - be_j) (s_j . y_i)
// with the matrix SY_ij = s_i . y_j of the stored pairs kept on the device (one
// new row and column per stored pair).  So each loop is one pass that forms all
// its products at once (every thread loads an entry of every history vector
// together, then a fixed-order reduction), a scalar recursion of m steps in the
// last block, and one pass that combines the vectors:
//   commit (+ products s_i . g, new SY entries) -> q = g - sum al_i y_i -> solve
//   -> products y_i . r0, r0 . g -> d = -(r0 + sum (al_i - be_i) s_i)
// The recursion visits the pairs in the order of the two-loop recursion, so the
// result equals it up to rounding.  MX is a compile-time bound on the history
// length (2, 4, 5, 8, 10 or 16) so that the per-pair accumulators live in registers.
constexpr int kMaxDots = 3 * kMaxHistory + 2;

#define PD_FOR_MINE(i) \
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n3; i += (int64_t)gridDim.x * kT)

// warp sum of one product into sh[k][warp]
__device__ __forceinline__ void dot_to_shared(double v, double (*sh)[kT / 32], int k) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
}

// Block sums of products 0..K-1 to partials; true (all threads) in the last
// block to finish, with the grid totals in tot[0..K) summed in block order.
__device__ bool finish_dots(int K, double (*sh)[kT / 32], double* partials, unsigned* counter, double* tot) {
  __shared__ int is_last;
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += kT) {
    double t = 0;
#pragma unroll
    for (int w = 0; w < kT / 32; ++w) t += sh[k][w];
    partials[(int64_t)blockIdx.x * kMaxDots + k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // warp w sums products k = w, w + 8, ...; lane l the blocks l, l + 32, ... (eight
  // loads in flight per lane, added in block order)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = (int)gridDim.x;
  for (int k = warp; k < K; k += kT / 32) {
    double t = 0;
    for (int b0 = 0; b0 < nb; b0 += 32 * 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = b0 + lane + 32 * u;
        v[u] = b < nb ? __ldcg(partials + (int64_t)b * kMaxDots + k) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) t += v[u];
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) tot[k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ring slots newest first / oldest first (uniform over the grid)
template <int MX>
__device__ __forceinline__ void ring_newest(const IterState* st, int* idx) {
#pragma unroll
  for (int k = 0; k < MX; ++k) idx[k] = k < st->count ? idx_newest(st, k) : 0;
}
template <int MX>
__device__ __forceinline__ void ring_oldest(const IterState* st, int* idx) {
#pragma unroll
  for (int k = 0; k < MX; ++k) idx[k] = k < st->count ? idx_oldest(st, k) : 0;
}

// The scalar state of the recursions (the Gram matrix, rho, al, cf, s_i . g),
// staged in shared memory by the last block: one cooperative load, the m-step
// recursion on one thread from shared memory, one cooperative store.
struct LbfgsScalars {
  double SY[kMaxHistory][kMaxHistory];
  double rho[kMaxHistory], al[kMaxHistory], cf[kMaxHistory], sg[kMaxHistory];
  int head, count, m;
};

__device__ __forceinline__ void scalars_load(const IterState* st, LbfgsScalars& L) {
  for (int i = threadIdx.x; i < kMaxHistory * kMaxHistory; i += kT)
    L.SY[i / kMaxHistory][i % kMaxHistory] = st->SY[i / kMaxHistory][i % kMaxHistory];
  for (int i = threadIdx.x; i < kMaxHistory; i += kT) {
    L.rho[i] = st->rho[i];
    L.al[i] = st->al[i];
    L.cf[i] = st->cf[i];
    L.sg[i] = st->sg[i];
  }
  if (threadIdx.x == 0) {
    L.head = st->head;
    L.count = st->count;
    L.m = st->m;
  }
  __syncthreads();
}

__device__ __forceinline__ void scalars_store(IterState* st, const LbfgsScalars& L) {
  __syncthreads();
  for (int i = threadIdx.x; i < kMaxHistory * kMaxHistory; i += kT)
    st->SY[i / kMaxHistory][i % kMaxHistory] = L.SY[i / kMaxHistory][i % kMaxHistory];
  for (int i = threadIdx.x; i < kMaxHistory; i += kT) {
    st->al[i] = L.al[i];
    st->cf[i] = L.cf[i];
    st->sg[i] = L.sg[i];
  }
}

__device__ __forceinline__ int ring_newest_s(const LbfgsScalars& L, int k) {
  return (L.head + L.count - 1 - k + 2 * L.m) % L.m;
}
__device__ __forceinline__ int ring_oldest_s(const LbfgsScalars& L, int k) { return (L.head + k) % L.m; }

// one thread: store the products (s_i . g and the new SY entries)
__device__ __forceinline__ void store_products(LbfgsScalars& L, const double* tot, bool push, int slot) {
  const int cnt = L.count;
  for (int k = 0; k < cnt; ++k) L.sg[ring_newest_s(L, k)] = tot[k];
  if (push) {
    for (int k = 0; k < cnt; ++k) {
      const int i = ring_newest_s(L, k);
      L.SY[i][slot] = tot[cnt + 2 * k];
      L.SY[slot][i] = tot[cnt + 2 * k + 1];
    }
  }
}

// one thread: al_i newest -> oldest
__device__ __forceinline__ void first_loop_coefficients(LbfgsScalars& L) {
  const int cnt = L.count;
  for (int k = 0; k < cnt; ++k) {
    const int i = ring_newest_s(L, k);
    double acc = L.sg[i];
    for (int kk = 0; kk < k; ++kk) {
      const int j = ring_newest_s(L, kk);
      acc -= L.al[j] * L.SY[i][j];
    }
    L.al[i] = L.rho[i] * acc;
  }
}

// Products of the first loop at the new gradient gn, accumulated per entry:
// s_i . gn over the stored pairs (newest first) and, after a push into `slot`,
// s_i . y_slot and s_slot . y_i.  The pushed pair's own entries (ss, ys) come from
// registers; every other history entry was loaded before the entry's stores.
template <int MX, typename H>
__device__ __forceinline__ void accumulate_first_loop(const int* idx, int cnt, bool push, int slot,
                                                      const H* si, const H* yi, H gn, H ss,
                                                      H ys, H* sg, H* a, H* b) {
#pragma unroll
  for (int k = 0; k < MX; ++k) {
    const bool fresh = push && k < cnt && idx[k] == slot;
    const H sk = fresh ? ss : si[k];
    const H yk = fresh ? ys : yi[k];
    sg[k] += sk * gn;
    a[k] += sk * ys;
    b[k] += ss * yk;
  }
}

template <int MX, typename H>
__device__ __forceinline__ int first_loop_to_shared(int cnt, bool push, const H* sg, const H* a,
                                                    const H* b, double (*sh)[kT / 32], int k0) {
  int K = k0;
#pragma unroll
  for (int k = 0; k < MX; ++k)
    if (k < cnt) dot_to_shared((double)sg[k], sh, K++);
  if (push) {
#pragma unroll
    for (int k = 0; k < MX; ++k) {
      if (k < cnt) {
        dot_to_shared((double)a[k], sh, K++);
        dot_to_shared((double)b[k], sh, K++);
      }
    }
  }
  return K;
}

// History storage H: double in FP64 meshes; float in mixed precision, where the
// history only shapes the search direction (the iterate, gradient and convergence
// test stay FP64) and the per-thread products are formed in FP32 (GB300's FP64
// pipe is a small fraction of its FP32 pipe), then reduced in FP64.

// forward, before the solve: commit an accepted trial (history pair, x, grad) and
// form the first-loop products in the same pass; then the coefficients
template <int MX, typename H>
__global__ void __launch_bounds__(kT) lbfgs_commit_fwd_kernel(VecCtx c, double* x, const double* xt, double* grad,
                                                             const double* gradt, H* S, H* Y) {
  IterState* st = c.st;
  if (!st->accepted) return;
  const int64_t n3 = c.n3;
  const int push = st->push, slot = st->pslot, cnt = st->count;
  const bool conv = st->converged;
  int idx[MX];
  ring_newest<MX>(st, idx);
  const H* sp[MX];
  const H* yp[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) {   // unused entries read slot 0 of S (a valid address)
    sp[k] = k < cnt ? S + (int64_t)idx[k] * n3 : S;
    yp[k] = (k < cnt && push) ? Y + (int64_t)idx[k] * n3 : S;
  }
  H sg[MX], a[MX], b[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) sg[k] = a[k] = b[k] = H(0);
  // two entries per iteration, every load of both issued before any store
  const int64_t stride = (int64_t)gridDim.x * kT;
  for (int64_t e0 = (int64_t)blockIdx.x * kT + threadIdx.x; e0 < n3; e0 += 2 * stride) {
    const int64_t e1 = e0 + stride;
    const bool v1 = e1 < n3;
    const int64_t f1 = v1 ? e1 : e0;
    double xn[2], gn[2], xo[2], go[2];
    H si[2][MX], yi[2][MX];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t e = u ? f1 : e0;
      xn[u] = xt[e];
      gn[u] = gradt[e];
      xo[u] = x[e];
      go[u] = grad[e];
#pragma unroll
      for (int k = 0; k < MX; ++k) {   // entries past the count are not used
        si[u][k] = k < cnt ? sp[k][e] : H(0);
        yi[u][k] = (k < cnt && push) ? yp[k][e] : H(0);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !v1) break;
      const int64_t e = u ? e1 : e0;
      const H ss = (H)(xn[u] - xo[u]), ys = (H)(gn[u] - go[u]);
      if (push) {
        S[(int64_t)slot * n3 + e] = ss;
        Y[(int64_t)slot * n3 + e] = ys;
      }
      x[e] = xn[u];
      grad[e] = gn[u];
      accumulate_first_loop<MX, H>(idx, cnt, push != 0, slot, si[u], yi[u], (H)gn[u], ss, ys, sg, a, b);
    }
  }
  // a converged solve still records the new pair's products (history kept for the next step)
  if (conv && !push) return;
  __shared__ double sh[kMaxDots][kT / 32];
  __shared__ double tot[kMaxDots];
  const int K = first_loop_to_shared<MX, H>(cnt, push != 0, sg, a, b, sh, 0);
  if (!finish_dots(K, sh, c.lpart, c.lcounter, tot)) return;
  __shared__ LbfgsScalars L;
  scalars_load(st, L);
  if (threadIdx.x == 0) {
    store_products(L, tot, push != 0, slot);
    if (!conv) first_loop_coefficients(L);
  }
  scalars_store(st, L);
}

// backward, before the solve: apply the previous step z += alpha d,
// gs += alpha Hd (history pair alpha (d, Hd)) and test |gs| for convergence, with
// the first-loop products in the same pass; then the coefficients.  The first
// iteration of a step (or the one after a residual replacement) has no step to apply.
template <int MX, typename H>
__global__ void __launch_bounds__(kT) lbfgs_commit_bwd_kernel(VecCtx c, const double* d, const double* Hd, double* z,
                                                             double* gs, H* S, H* Y) {
  IterState* st = c.st;
  if (st->converged) return;
  const int64_t n3 = c.n3;
  const int pending = st->pending;
  const int push = pending ? st->push : 0, slot = st->pslot, cnt = st->count;
  const double al = pending ? st->alpha : 0.0;
  int idx[MX];
  ring_newest<MX>(st, idx);
  const H* sp[MX];
  const H* yp[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) {
    sp[k] = k < cnt ? S + (int64_t)idx[k] * n3 : S;
    yp[k] = (k < cnt && push) ? Y + (int64_t)idx[k] * n3 : S;
  }
  H sg[MX], a[MX], b[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) sg[k] = a[k] = b[k] = H(0);
  double part = 0;
  const int64_t stride = (int64_t)gridDim.x * kT;
  for (int64_t e0 = (int64_t)blockIdx.x * kT + threadIdx.x; e0 < n3; e0 += 2 * stride) {
    const int64_t e1 = e0 + stride;
    const bool v1 = e1 < n3;
    const int64_t f1 = v1 ? e1 : e0;
    double go[2], dd[2], hh[2], zz[2];
    H si[2][MX], yi[2][MX];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t e = u ? f1 : e0;
      go[u] = gs[e];
      dd[u] = pending ? d[e] : 0.0;
      hh[u] = pending ? Hd[e] : 0.0;
      zz[u] = pending ? z[e] : 0.0;
#pragma unroll
      for (int k = 0; k < MX; ++k) {   // entries past the count are not used
        si[u][k] = k < cnt ? sp[k][e] : H(0);
        yi[u][k] = (k < cnt && push) ? yp[k][e] : H(0);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !v1) break;
      const int64_t e = u ? e1 : e0;
      double gn = go[u], ad = 0.0, ah = 0.0;
      if (pending) {
        ad = al * dd[u];
        ah = al * hh[u];
        z[e] = zz[u] + ad;
        gn = go[u] + ah;
        gs[e] = gn;
        if (push) {
          S[(int64_t)slot * n3 + e] = (H)ad;
          Y[(int64_t)slot * n3 + e] = (H)ah;
        }
        part += gn * gn;
      }
      accumulate_first_loop<MX, H>(idx, cnt, push != 0, slot, si[u], yi[u], (H)gn, (H)ad, (H)ah, sg, a, b);
    }
  }
  __shared__ double sh[kMaxDots][kT / 32];
  __shared__ double tot[kMaxDots];
  int K0 = 0;
  if (pending) {
    dot_to_shared(part, sh, 0);
    K0 = 1;
  }
  const int K = first_loop_to_shared<MX, H>(cnt, push != 0, sg, a, b, sh, K0);
  if (!finish_dots(K, sh, c.lpart, c.lcounter, tot)) return;
  __shared__ LbfgsScalars L;
  scalars_load(st, L);
  if (threadIdx.x == 0) {
    store_products(L, tot + K0, push != 0, slot);
    bool stop = false;
    if (pending) {
      const double gn2 = tot[0];
      const bool conv = gn2 <= st->tol2 * st->ref2;
      st->iters += 1;
      const bool cap = !conv && st->iters >= st->max_iter;
      st->gn2_acc = gn2;
      st->pending = 0;
      if (conv || cap) {
        st->converged = 1;
        st->hit_max = cap ? 1 : 0;
        stop = true;
      }
    }
    if (!stop) first_loop_coefficients(L);
  }
  scalars_store(st, L);
}

// q = g - sum al_i y_i (newest first, as the first loop subtracts them)
template <int MX, typename H>
__global__ void __launch_bounds__(kT) lbfgs_q_kernel(VecCtx c, const double* g, const H* Y, double* q) {
  const IterState* st = c.st;
  if (st->converged || !st->accepted) return;
  const int64_t n3 = c.n3;
  const int cnt = st->count;
  int idx[MX];
  H al[MX];
  ring_newest<MX>(st, idx);
#pragma unroll
  for (int k = 0; k < MX; ++k) al[k] = k < cnt ? (H)st->al[idx[k]] : H(0);
  const H* yp[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) yp[k] = k < cnt ? Y + (int64_t)idx[k] * n3 : Y;   // al = 0 past the count
  PD_FOR_MINE(e) {
    H yv[MX];
#pragma unroll
    for (int k = 0; k < MX; ++k) yv[k] = k < cnt ? yp[k][e] : H(0);
    if constexpr (sizeof(H) == 8) {
      double v = g[e];
#pragma unroll
      for (int k = 0; k < MX; ++k) v -= al[k] * yv[k];
      q[e] = v;
    } else {
      H u = H(0);
#pragma unroll
      for (int k = 0; k < MX; ++k) u += al[k] * yv[k];
      q[e] = g[e] - (double)u;
    }
  }
}

// after the solve r0 = A^-1 q: products y_i . r0 and r0 . g, then be_i oldest ->
// newest, the coefficients cf_i = al_i - be_i and the slope d . g of
// d = -(r0 + sum cf_i s_i)
template <int MX, typename H>
__global__ void __launch_bounds__(kT) lbfgs_post_dots_kernel(VecCtx c, const double* g, const H* Y,
                                                            const double* r) {
  IterState* st = c.st;
  if (st->converged || !st->accepted) return;
  const int64_t n3 = c.n3;
  const int cnt = st->count;
  __shared__ double sh[kMaxDots][kT / 32];
  __shared__ double tot[kMaxDots];
  int idx[MX];
  ring_oldest<MX>(st, idx);
  H yr[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) yr[k] = H(0);
  double rg = 0.0;
  const H* yp[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) yp[k] = k < cnt ? Y + (int64_t)idx[k] * n3 : Y;
  const int64_t stride = (int64_t)gridDim.x * kT;
  for (int64_t e0 = (int64_t)blockIdx.x * kT + threadIdx.x; e0 < n3; e0 += 2 * stride) {
    const int64_t e1 = e0 + stride;
    const bool v1 = e1 < n3;
    const int64_t f1 = v1 ? e1 : e0;
    double re[2], ge[2];
    H yv[2][MX];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t e = u ? f1 : e0;
      re[u] = r[e];
      ge[u] = g[e];
#pragma unroll
      for (int k = 0; k < MX; ++k) yv[u][k] = k < cnt ? yp[k][e] : H(0);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !v1) break;
      rg += re[u] * ge[u];
      const H rh = (H)re[u];
#pragma unroll
      for (int k = 0; k < MX; ++k) yr[k] += yv[u][k] * rh;
    }
  }
#pragma unroll
  for (int k = 0; k < MX; ++k)
    if (k < cnt) dot_to_shared((double)yr[k], sh, k);
  dot_to_shared(rg, sh, cnt);
  if (!finish_dots(cnt + 1, sh, c.lpart, c.lcounter, tot)) return;
  __shared__ LbfgsScalars L;
  scalars_load(st, L);
  if (threadIdx.x == 0) {
    double slope = tot[cnt];
    for (int k = 0; k < cnt; ++k) {
      const int i = ring_oldest_s(L, k);
      double acc = tot[k];
      for (int kk = 0; kk < k; ++kk) {
        const int j = ring_oldest_s(L, kk);
        acc += L.cf[j] * L.SY[j][i];
      }
      L.cf[i] = L.al[i] - L.rho[i] * acc;
      slope += L.cf[i] * L.sg[i];
    }
    st->slope = -slope;
  }
  scalars_store(st, L);
}

// d = -(r0 + sum cf_i s_i) (oldest first, as the second loop adds them); forward:
// trial xt = x + d, or xt = x + alpha d after a rejected trial
template <int MX, typename H>
__global__ void __launch_bounds__(kT) lbfgs_dir_kernel(VecCtx c, const H* S, const double* r, double* d,
                                                      const double* x, double* xt) {
  const IterState* st = c.st;
  if (st->converged) return;
  const int64_t n3 = c.n3;
  if (!st->accepted) {
    const double a = st->alpha;
    if (xt) PD_FOR_MINE(e) xt[e] = x[e] + a * d[e];
    return;
  }
  const int cnt = st->count;
  int idx[MX];
  H cf[MX];
  ring_oldest<MX>(st, idx);
#pragma unroll
  for (int k = 0; k < MX; ++k) cf[k] = k < cnt ? (H)st->cf[idx[k]] : H(0);
  const H* sp[MX];
#pragma unroll
  for (int k = 0; k < MX; ++k) sp[k] = k < cnt ? S + (int64_t)idx[k] * n3 : S;   // cf = 0 past the count
  PD_FOR_MINE(e) {
    H sv[MX];
#pragma unroll
    for (int k = 0; k < MX; ++k) sv[k] = k < cnt ? sp[k][e] : H(0);
    double v;
    if constexpr (sizeof(H) == 8) {
      v = r[e];
#pragma unroll
      for (int k = 0; k < MX; ++k) v += cf[k] * sv[k];
    } else {
      H u = H(0);
#pragma unroll
      for (int k = 0; k < MX; ++k) u += cf[k] * sv[k];
      v = r[e] + (double)u;
    }
    d[e] = -v;
    if (xt) xt[e] = x[e] - v;
  }
}
#undef PD_FOR_MINE

// compile-time history bound for a history length m (<= kMaxHistory)
// blocks of the L-BFGS kernels: one entry per thread up to the partial-sum capacity
constexpr int kLbfgsMaxBlocks = 2048;
inline int lbfgs_blocks(int64_t n3) {
  const int64_t b = (n3 + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > kLbfgsMaxBlocks ? kLbfgsMaxBlocks : b));
}

inline int lbfgs_bound(int m) {
  return m <= 2 ? 2 : (m <= 4 ? 4 : (m <= 5 ? 5 : (m <= 8 ? 8 : (m <= 10 ? 10 : 16))));
}

// v_{t+1} = (x - x_t)/h, state advance, trajectory write in kept order
__global__ void finalize_fwd_kernel(int64_t n, const double* x, double* xi, double* vi, double inv_h,
                                    const int32_t* kept_of_internal, double* traj_x, double* traj_v) {
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < n; c += (int64_t)gridDim.x * kT) {
    const int64_t k = kept_of_internal[c];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double xn = x[3 * c + i];
      const double vn = (xn - xi[3 * c + i]) * inv_h;
      xi[3 * c + i] = xn;
      vi[3 * c + i] = vn;
      if (traj_x) traj_x[3 * k + i] = xn;
      if (traj_v) traj_v[3 * k + i] = vn;
    }
  }
}

// ---------------------------------------------------------------- backward
// gbar = ax + av/h, z = 0, gs = grad s(0) = -gbar, q = gs; ref2 = |gbar|^2.
// Rows of held nodes (complementarity contact, may be null) take no part: their
// right-hand side and z are zero.
__global__ void bwd_step_init_kernel(VecCtx c, const double* ax, const double* av, double inv_h,
                                     double* z, double* gs, double* q, int keep_z, const uint8_t* held) {
  double part = 0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < c.n3; i += (int64_t)gridDim.x * kT) {
    const bool h = held && held[i / 3];
    const double gb = h ? 0.0 : ax[i] + av[i] * inv_h;
    if (!keep_z || h) z[i] = 0.0;
    gs[i] = -gb;
    q[i] = -gb;
    part += gb * gb;
  }
  double tot;
  if (grid_sum(part, c.partials, c.counter, &tot)) {
    c.st->ref2 = tot;
    c.st->gn2_acc = tot;
    c.st->converged = (tot == 0.0);
  }
}

// line search on the quadratic s along d with the curvature d.Hd (exact values,
// no extra Hessian products), then the history pair (s, y) = alpha (d, Hd)
__global__ void decide_bwd_kernel(IterState* st, const double* gather_partials, int64_t nbg) {
  const double dHd = block_reduce_strided(gather_partials, nbg, 4, 0);
  if (threadIdx.x != 0) return;
  if (st->converged) return;
  st->svd_cached = 1;   // this iteration's Hessian product ran: its point SVDs are cached
  st->dHd = dHd;
  st->evals += 1;
  st->pending = 1;
  if (!isfinite(dHd)) {
    st->status |= DEV_ERR_NAN;
    st->converged = 1;
    st->alpha = 0.0;
    st->push = 0;
    return;
  }
  const double slope = st->slope;
  if (!(slope < 0.0)) {   // not a descent direction: drop the history, no step
    st->count = 0;
    st->head = 0;
    st->alpha = 0.0;
    st->push = 0;
    return;
  }
  // s is quadratic along d: its exact minimiser is alpha* = -slope / d.Hd when the
  // curvature is positive (with a fixed preconditioner this makes the L-BFGS
  // iteration generate the preconditioned conjugate-gradient iterates); otherwise
  // Armijo backtracking from alpha = 1 on the closed-form decrease.
  double a = 1.0;
  if (dHd > 0.0) {
    a = -slope / dHd;
  } else {
    for (int t = 0; t < st->ls_max; ++t) {
      if (a * slope + 0.5 * a * a * dHd <= st->c1 * a * slope) break;
      a *= 0.5;
      st->ls_total += 1;
    }
  }
  st->alpha = a;
  st->push = 0;
  const double sy = a * a * dHd;
  if (st->m > 0 && sy > 0.0) {
    int slot;
    if (st->count < st->m) {
      slot = (st->head + st->count) % st->m;
      st->count += 1;
    } else {
      slot = st->head;
      st->head = (st->head + 1) % st->m;
    }
    st->rho[slot] = 1.0 / sy;
    st->pslot = slot;
    st->push = 1;
  }
}

// gs = Hz - gbar from an exact product Hz (true-residual replacement); held rows
// (may be null) are zero
__global__ void residual_replace_kernel(VecCtx c, const double* Hz, const double* ax, const double* av,
                                        double inv_h, double* gs, double* q, const uint8_t* held) {
  double part = 0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < c.n3; i += (int64_t)gridDim.x * kT) {
    const double g = (held && held[i / 3]) ? 0.0 : Hz[i] - (ax[i] + av[i] * inv_h);
    gs[i] = g;
    q[i] = g;
    part += g * g;
  }
  double tot;
  if (grid_sum(part, c.partials, c.counter, &tot)) {
    c.st->gn2_acc = tot;
    c.st->converged = tot <= c.st->tol2 * c.st->ref2 ? 1 : 0;
    c.st->accepted = 1;
  }
}

// Adjoint of one step (Eqns 10-12) -> upstream gradients of the previous state:
//   dL/dy = M z/h^2, ax <- dL/dy - av/h (+ friction), av <- h dL/dy (+ friction),
//   g_fext += z, then the direct loss terms of step t are added.
__global__ void bwd_state_kernel(BwdStateParams p) {
  double part = 0;
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < p.n; c += (int64_t)gridDim.x * kT) {
    double nax[3] = {0, 0, 0}, nav[3] = {0, 0, 0};
    if (c < p.nf) {
      const double m = p.mass[c];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double zi = p.z[3 * c + i];
        const double dldy = m * zi * p.inv_h2;
        nax[i] = dldy - p.av[3 * c + i] * p.inv_h;
        nav[i] = p.h * dldy;
        if (p.gfext) p.gfext[3 * c + i] += zi;
      }
      if (p.contact && p.contact[c]) {
        // friction f_t(x_t, v_t, mu) entered f_ext of this step: dL/df = z
        const double zc = p.xi[3 * c + 2];
        const double vx = p.vi[3 * c], vy = p.vi[3 * c + 1];
        const double nv = sqrt(vx * vx + vy * vy);
        if (zc < 0.0 && nv > 0.0) {
          const double m = p.mass[c];
          const double tx = vx / nv, ty = vy / nv;
          const double gx = p.z[3 * c], gy = p.z[3 * c + 1];
          if (p.mu * p.k * (-zc) < m * nv / p.h) {
            const double gt = gx * tx + gy * ty;
            nax[2] += p.mu * p.k * gt;
            part += p.k * zc * gt;
            const double s = p.mu * p.k * zc / nv;
            nav[0] += s * (gx - tx * gt);
            nav[1] += s * (gy - ty * gt);
          } else {
            nav[0] += -m / p.h * gx;
            nav[1] += -m / p.h * gy;
          }
        }
      }
    }
    const int64_t k = p.kept_of_internal[c];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (p.gx_t) nax[i] += p.gx_t[3 * k + i];
      if (p.gv_t) nav[i] += p.gv_t[3 * k + i];
      p.ax[3 * c + i] = nax[i];
      p.av[3 * c + i] = nav[i];
    }
  }
  double tot;
  if (grid_sum(part, p.partials, p.counter, &tot) && p.gmu) *p.gmu += tot;
}

// ---------------------------------------------------------------- misc
__global__ void kept_to_internal_kernel(int64_t n, const int32_t* kept_of_internal, const double* in,
                                        double* out) {
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < n; c += (int64_t)gridDim.x * kT) {
    const int64_t k = kept_of_internal[c];
    out[3 * c] = in[3 * k];
    out[3 * c + 1] = in[3 * k + 1];
    out[3 * c + 2] = in[3 * k + 2];
  }
}

__global__ void internal_to_kept_kernel(int64_t n, int64_t nvalid, const int32_t* kept_of_internal,
                                        const double* in, double* out) {
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < n; c += (int64_t)gridDim.x * kT) {
    const int64_t k = kept_of_internal[c];
    const bool v = c < nvalid;
    out[3 * k] = v ? in[3 * c] : 0.0;
    out[3 * k + 1] = v ? in[3 * c + 1] : 0.0;
    out[3 * k + 2] = v ? in[3 * c + 2] : 0.0;
  }
}

// grad E over all nodes from the element buffer (local-step entry point) and
// the contact energy partials.
template <typename T>
__global__ void gather_all_kernel(int64_t n, const int32_t* inc_ptr, const int32_t* inc, const void* eb,
                                  const double* x, const uint8_t* contact, double k, double* out,
                                  double* partials, unsigned* counter, double* energy_total) {
  const T* e = reinterpret_cast<const T*>(eb);
  double part = 0;
  for (int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x; c < n; c += (int64_t)gridDim.x * kT) {
    double g[3] = {0, 0, 0};
    for (int32_t q = inc_ptr[c]; q < inc_ptr[c + 1]; ++q) {
      const int64_t slot = (int64_t)inc[q] * 3;
      g[0] += (double)e[slot];
      g[1] += (double)e[slot + 1];
      g[2] += (double)e[slot + 2];
    }
    if (contact && contact[c] && x[3 * c + 2] < 0.0) {
      const double z = x[3 * c + 2];
      g[2] += k * z;
      part += 0.5 * k * z * z;
    }
    if (out) {
      out[3 * c] = g[0];
      out[3 * c + 1] = g[1];
      out[3 * c + 2] = g[2];
    }
  }
  double tot;
  if (grid_sum(part, partials, counter, &tot) && energy_total) *energy_total += tot;
}

__global__ void sum_partials_kernel(const double* partials, int64_t n, double* out) {
  const double t = block_reduce_strided(partials, n, 1, 0);
  if (threadIdx.x == 0) *out = t;
}

__global__ void copy_kernel(int64_t n, const double* in, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) out[i] = in[i];
}

__global__ void mark_checked_kernel(IterState* st) { st->fp64_checked = 1; }
__global__ void clear_checked_kernel(IterState* st) { st->fp64_checked = 0; }

__global__ void force_accept_kernel(IterState* st) {
  st->force_accept = 1;
  st->converged = 0;
  st->hit_max = 0;
  st->accepted = 0;
}

}  // namespace pd
