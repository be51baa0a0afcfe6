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
// The panels are cut into 2D tiles of at most 256 x 48 panel entries (48 KB in
// FP32), shaped per supernode so that each of the 256 tile-body threads owns up to
// 48 entries: forward tiles are R rows x (256 / R) column groups of 48 columns
// (R = 256, 128 or 64, whichever covers the supernode's columns with the fewest
// idle groups); backward tiles are BC columns x min(12288 / BC, 1024) rows (BC =
// 64, 32, 16 or 8).  All-zero tiles of the triangular L11^-1 block are skipped.
// In FP32 every tile's panel values are also stored contiguously, in the order
// the tile body reads them (MeshImpl::Qs, packed once per factorisation), and
// reach shared memory by one bulk copy (cp.async.bulk, completion on an
// mbarrier) issued by a producer warp into one of two stages per CTA while the
// body warps work on the previous tile, so a CTA keeps the next tile's copy in
// flight throughout (per-thread register loads are limited by the requests an SM
// can have outstanding).  The stored layout adds zeros for the upper triangle of
// L11^-1 and for ragged tile edges.  The FP64 kernel keeps per-thread register
// loads.  Tiles sharing an output block write partial sums; the last tile to
// finish (integer ticket) adds them in tile order, so the result does not depend
// on scheduling and no float atomics run.  Both sweeps run in one persistent
// launch scheduled by the supernodal tree dependencies (below).
#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kThreads = 256;         // tile-body threads per CTA (8 warps); 2 CTAs per SM
constexpr int kWarps = kThreads / 32;
constexpr int kCols = 48;             // forward: columns per thread; backward: loads per lane
constexpr int kTileElems = kThreads * kCols;   // panel entries per tile at most (48 KB in FP32)
constexpr int kPart = kThreads * 3;   // partial-sum slots per tile
constexpr int kMaxC = 4 * kCols;       // widest forward tile (4 column groups)
// backward tile rows for BC columns: kTileElems / BC, at most 1024 (32 rows per lane)
__host__ __device__ constexpr int bwd_tile_rows(int bc) { return kTileElems / bc < 1024 ? kTileElems / bc : 1024; }
constexpr int kMaxBR = 1024;
constexpr int kPreSlots = 4;          // W-row sources per position held in registers
constexpr int kStreamBytes = kTileElems * 4;   // one shared-memory stage of the FP32 kernel
constexpr int kStages = 2;                     // FP32 kernel: stages per CTA (copy of the next tile in flight)
constexpr int kPipeThreads = kThreads + 32;    // FP32 kernel: + one producer warp

// loads issued back to back per thread in the FP64 kernel: batches of 16 (register
// budget); the FP32 kernel reads its panel values from shared memory
template <typename T>
struct Batch {
  static constexpr int kLoads = sizeof(T) == 4 ? 64 : 16;
};

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
  long long spin_limit;         // polls of a dependency wait before it gives up
  int64_t stall_tile;           // test support: this tile's first wait target is raised by one (-1: none)
  void* partial;                // per tile partial sums (T)
  const void* Q;
  const float* Qs;              // FP32: tiles stored contiguously (SolveTile::soff)
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
// flag DEV_ERR_TIMEOUT after SolveParams::spin_limit polls, about a second by
// default).  Counters only grow: a solve consumes ntiles + grid
// tickets (every CTA draws one ticket past the end), so ticket t belongs to
// solve t / (ntiles + grid).

// Message passing between CTAs: a producer's tile writes, then (after a CTA
// barrier) one thread's release reduction on a counter; a consumer's thread polls
// the counter with acquire loads, then a CTA barrier, then the CTA reads (through
// L2).  The barriers carry the ordering to the other threads of both CTAs
// (cumulativity); no fence waits for the consumer's own panel loads in flight.
__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void add_release(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long add_acq_rel(unsigned long long* p) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], 1;" : "=l"(old) : "l"(p) : "memory");
  return old;
}

__device__ __forceinline__ bool wait_count(const unsigned long long* c, unsigned long long target, int* err,
                                           long long limit) {
  long long it = 0;
  while (load_acquire(c) < target) {
    if (++it > limit) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// Barrier of the 256 tile-body threads (named barrier 1).  In the FP32 kernel the
// producer warp never joins it; the FP64 kernel has no producer and uses the same
// barrier.
__device__ __forceinline__ void body_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// shared memory of one tile body: forward rhs[kMaxC][3] + red[kThreads][3];
// backward v[kMaxBR][3] + res[64][3] (as T)
template <typename T>
struct __align__(16) TileSmem {
  T buf[(kMaxBR + 64) * 3];
  int flag;
};

// last of the tiles of an output block?  (then the partial sums are complete)
template <typename T>
__device__ __forceinline__ bool last_of_block(const SolveParams& p, const SolveTile& tl, TileSmem<T>& sm) {
  body_sync();
  if (threadIdx.x == 0) {
    const unsigned long long v = add_acq_rel(p.otick + tl.out);
    sm.flag = ((v + 1) % (unsigned long long)tl.ntile) == 0;
  }
  body_sync();
  return sm.flag != 0;
}

__device__ __forceinline__ void signal_done(unsigned long long* c) {
  body_sync();
  if (threadIdx.x == 0) add_release(c);
}

// ------------------------------------------------------------ mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// waits (at most about limit_ns) for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned phase, unsigned long long limit_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// W-row sources of a position, loaded before the dependency wait (they are static)
struct Slots {
  int32_t g[kPreSlots];
};

__device__ __forceinline__ Slots load_slots(const SolveParams& p, int64_t pos, bool valid) {
  Slots sl;
#pragma unroll
  for (int k = 0; k < kPreSlots; ++k)
    sl.g[k] = (valid && k < p.slot_w) ? __ldg(p.slots + pos * p.slot_w + k) : -1;
  return sl;
}

// sum of the children's updates of a position (W rows written earlier in this solve)
template <typename T>
__device__ __forceinline__ void add_W(const SolveParams& p, const Slots& sl, int64_t pos, double& v0, double& v1,
                                      double& v2) {
  const T* W = reinterpret_cast<const T*>(p.W);
#pragma unroll
  for (int k = 0; k < kPreSlots; ++k) {
    if (sl.g[k] >= 0) {
      v0 += (double)__ldcg(W + 3 * (int64_t)sl.g[k]);
      v1 += (double)__ldcg(W + 3 * (int64_t)sl.g[k] + 1);
      v2 += (double)__ldcg(W + 3 * (int64_t)sl.g[k] + 2);
    }
  }
  for (int k = kPreSlots; k < p.slot_w; ++k) {
    const int32_t g = __ldg(p.slots + pos * p.slot_w + k);
    if (g >= 0) {
      v0 += (double)__ldcg(W + 3 * (int64_t)g);
      v1 += (double)__ldcg(W + 3 * (int64_t)g + 1);
      v2 += (double)__ldcg(W + 3 * (int64_t)g + 2);
    }
  }
}

// Forward tile: rows [a, a + R) x columns [b, b + G * 64) of panel s, G = kThreads / R.
// Thread (row rl, group g) owns row a + rl and columns b + 64 g ... + 63; a warp
// reads 32 consecutive rows of one column per load (coalesced).  The group sums
// are added in group order.
template <typename T, int R>
__device__ void fwd_tile_body(const SolveParams& p, const SolveTile& tl, int64_t tid_g, unsigned long long epoch,
                              TileSmem<T>& sm, const float* stage) {
  constexpr bool kStream = sizeof(T) == 4;   // FP32: panel values in the shared-memory stage (null: copy failed)
  constexpr int G = kThreads / R;
  constexpr int C = G * kCols;
  constexpr int B = Batch<T>::kLoads;
  T (*rhs)[3] = reinterpret_cast<T (*)[3]>(sm.buf);
  T (*red)[3] = reinterpret_cast<T (*)[3]>(sm.buf) + kMaxC;   // after the widest rhs
  const int64_t row0 = tl.a, col0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr, pos = tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const int rl = threadIdx.x % R, g = threadIdx.x / R;
  const int64_t r = row0 + rl;
  const int64_t cg0 = col0 + (int64_t)g * kCols;
  // L11^-1 is lower triangular: rows < nc use columns <= row only
  const int64_t cend = r >= nr ? cg0 : (r < nc ? min(nc, r + 1) : nc);
  const int cnt = (int)max((int64_t)0, min((int64_t)kCols, cend - cg0));
  const T* Qr = Q + r + cg0 * nr;
  // static data first: panel values, right-hand side, W-row sources
  T q[kStream ? 1 : B];
  if constexpr (!kStream) {
#pragma unroll
    for (int k = 0; k < B; ++k) q[k] = (k < cnt) ? __ldg(Qr + (int64_t)k * nr) : T(0);
  }
  // rhs columns of this thread: col0 + threadIdx.x + kThreads * i
  constexpr int CPT = (C + kThreads - 1) / kThreads;
  double bb[CPT][3];
  Slots sc[CPT];
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int jj = threadIdx.x + kThreads * i;
    const int64_t jc = col0 + jj;
    const bool has_c = jj < C && jc < nc;
    bb[i][0] = has_c ? __ldg(p.b + 3 * (first + jc)) : 0.0;
    bb[i][1] = has_c ? __ldg(p.b + 3 * (first + jc) + 1) : 0.0;
    bb[i][2] = has_c ? __ldg(p.b + 3 * (first + jc) + 2) : 0.0;
    sc[i] = load_slots(p, pos + jc, has_c);
  }
  const bool out_w = g == 0 && r < nr && r >= nc;
  const Slots sr = load_slots(p, pos + r, out_w);
  if (threadIdx.x == 0) {
    // the children's forward outputs (inline in the descriptor; more from the tree)
    const int nd = tl.ndep;
    for (int k = 0; k < nd && k < kTileDeps; ++k)
      wait_count(p.fdone + tl.dep[k],
                 (epoch + 1) * (unsigned long long)tl.dep_blocks[k] + (k == 0 && tid_g == p.stall_tile ? 1 : 0),
                 p.err, p.spin_limit);
    if (nd > kTileDeps) {
      for (int64_t ci = __ldg(p.child_ptr + tl.s) + kTileDeps; ci < __ldg(p.child_ptr + tl.s + 1); ++ci) {
        const int64_t c = __ldg(p.child_list + ci);
        wait_count(p.fdone + c, (epoch + 1) * (unsigned long long)__ldg(p.nfb + c), p.err, p.spin_limit);
      }
    }
  }
  body_sync();
  // children's updates of the output row (below rows), read in the same round
  // trip as those of the right-hand side
  double o0 = 0, o1 = 0, o2 = 0;
  if (out_w) add_W<T>(p, sr, pos + r, o0, o1, o2);
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    const int jj = threadIdx.x + kThreads * i;
    if (jj >= C) continue;
    const int64_t jc = col0 + jj;
    const bool has_c = jc < nc;
    double w0 = 0, w1 = 0, w2 = 0;
    if (has_c) add_W<T>(p, sc[i], pos + jc, w0, w1, w2);
    // zero past the supernode's columns (their panel values are zero too)
    rhs[jj][0] = has_c ? (T)(bb[i][0] - w0) : T(0);
    rhs[jj][1] = has_c ? (T)(bb[i][1] - w1) : T(0);
    rhs[jj][2] = has_c ? (T)(bb[i][2] - w2) : T(0);
  }
  body_sync();
  T a0 = T(0), a1 = T(0), a2 = T(0);
  const T(*rg)[3] = rhs + g * kCols;
  if constexpr (kStream) {
    // stored layout [group][column k < kmax][row rl < rv], zeros past each row's
    // columns: the same products in the same order as the masked register loads of
    // the FP64 path.  (Staging the values into registers first, as the backward
    // tile does, was measured slower here.)
    const int kmax = tl.sld;
    const int rv = (int)min((int64_t)R, nr - row0);
    // products only from a completed copy (a rejected or timed-out copy leaves zeros)
    if (rl < rv && stage) {
      const float* qs = stage + g * kmax * rv + rl;
#pragma unroll 8
      for (int k = 0; k < kmax; ++k) {
        const float qk = qs[k * rv];
        a0 += qk * rg[k][0];
        a1 += qk * rg[k][1];
        a2 += qk * rg[k][2];
      }
    }
  } else {
    constexpr int NB = kCols / B;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      if (nb > 0) {   // FP64: the next batch of columns
#pragma unroll
        for (int k = 0; k < B; ++k) q[k] = (nb * B + k < cnt) ? __ldg(Qr + (int64_t)(nb * B + k) * nr) : T(0);
      }
#pragma unroll
      for (int k = 0; k < B; ++k) {
        a0 += q[k] * rg[nb * B + k][0];
        a1 += q[k] * rg[nb * B + k][1];
        a2 += q[k] * rg[nb * B + k][2];
      }
    }
  }
  if (G > 1) {
    red[threadIdx.x][0] = a0;
    red[threadIdx.x][1] = a1;
    red[threadIdx.x][2] = a2;
    body_sync();
    if (g == 0) {
#pragma unroll
      for (int k = 1; k < G; ++k) {
        a0 += red[k * R + rl][0];
        a1 += red[k * R + rl][1];
        a2 += red[k * R + rl][2];
      }
    }
  }
  const int ntile = tl.ntile;
  if (ntile > 1) {
    T* part = reinterpret_cast<T*>(p.partial) + tid_g * kPart;
    if (g == 0) {
      part[3 * rl] = a0;
      part[3 * rl + 1] = a1;
      part[3 * rl + 2] = a2;
    }
    if (!last_of_block(p, tl, sm)) return;
    if (g == 0) {
      const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * kPart + 3 * rl;
      a0 = a1 = a2 = T(0);
      for (int k = 0; k < ntile; ++k) {
        a0 += __ldcg(parts + (int64_t)k * kPart);
        a1 += __ldcg(parts + (int64_t)k * kPart + 1);
        a2 += __ldcg(parts + (int64_t)k * kPart + 2);
      }
    }
  }
  if (g == 0 && r < nr) {
    if (r < nc) {
      T* uo = reinterpret_cast<T*>(p.u) + 3 * (first + r);
      uo[0] = a0; uo[1] = a1; uo[2] = a2;
    } else {
      T* Wo = reinterpret_cast<T*>(p.W) + 3 * (tl.relp + (r - nc));
      Wo[0] = (T)((double)a0 + o0);
      Wo[1] = (T)((double)a1 + o1);
      Wo[2] = (T)((double)a2 + o2);
    }
  }
  signal_done(p.fdone + tl.s);
}

// Backward tile: columns [a, a + BC) x rows [b, b + BR) of panel s, BR = min(kTileElems / BC, 1024).
// Warp w owns columns a + w CW ... (CW = BC / 8), its lanes the rows b + lane + 32 i;
// per column the lanes' sums are added by a fixed shuffle tree.
template <typename T, int BC>
__device__ void bwd_tile_body(const SolveParams& p, const SolveTile& tl, int64_t tid_g, unsigned long long epoch,
                              TileSmem<T>& sm, const float* stage) {
  constexpr bool kStream = sizeof(T) == 4;   // FP32: panel values in the shared-memory stage (null: copy failed)
  constexpr int CW = BC / kWarps;
  constexpr int BR = bwd_tile_rows(BC);
  constexpr int RL = BR / 32;           // rows per lane
  constexpr int B = Batch<T>::kLoads;
  constexpr int NB = CW * RL > B ? CW * RL / B : 1;   // load batches
  constexpr int RB = RL / NB;           // rows per lane per batch
  T (*v)[3] = reinterpret_cast<T (*)[3]>(sm.buf);
  T (*res)[3] = reinterpret_cast<T (*)[3]>(sm.buf) + kMaxBR;
  const int64_t col0 = tl.a, row0 = tl.b;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr;
  const int32_t* srows = p.rows + tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* u = reinterpret_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t rn = min((int64_t)BR, nr - row0);
  T q[CW][RB];
  auto load_batch = [&](int nb) {
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const int64_t j = col0 + warp * CW + c;
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int64_t rr = lane + 32 * (nb * RB + i);
        const int64_t row = row0 + rr;
        // column j of L11^-1 is zero above row j
        q[c][i] = (j < nc && rr < rn && (row >= nc || row >= j)) ? __ldg(Q + row + j * nr) : T(0);
      }
    }
  };
  if constexpr (!kStream) load_batch(0);
  // global rows of the tile's below rows (static)
  constexpr int VR = (BR + kThreads - 1) / kThreads;   // rows of v per thread (BR need not divide)
  int32_t gidx[VR];
#pragma unroll
  for (int k = 0; k < VR; ++k) {
    const int64_t rr = threadIdx.x + (int64_t)k * kThreads;
    const int64_t row = row0 + rr;
    gidx[k] = (rr < BR && rr < rn && row >= nc) ? __ldg(srows + row) : -1;
  }
  if (threadIdx.x == 0) {
    // the parent's backward outputs; the root waits for its own forward outputs
    const int32_t d = tl.dep[0];
    if (d >= 0) wait_count(p.bdone + d, (epoch + 1) * (unsigned long long)tl.dep_blocks[0], p.err, p.spin_limit);
    else wait_count(p.fdone + (-d - 1), (epoch + 1) * (unsigned long long)tl.dep_blocks[0], p.err, p.spin_limit);
  }
  body_sync();
  // v = [u_s; -x(below rows)] on the tile's rows, zero past the panel
#pragma unroll
  for (int k = 0; k < VR; ++k) {
    const int64_t rr = threadIdx.x + (int64_t)k * kThreads;
    if (rr >= BR) continue;
    const int64_t row = row0 + rr;
    T v0 = T(0), v1 = T(0), v2 = T(0);
    if (rr < rn) {
      if (row < nc) {
        const T* ur = u + 3 * (first + row);
        v0 = __ldcg(ur); v1 = __ldcg(ur + 1); v2 = __ldcg(ur + 2);
      } else {
        const int64_t gr = gidx[k];
        v0 = (T)(-__ldcg(p.x + 3 * gr)); v1 = (T)(-__ldcg(p.x + 3 * gr + 1)); v2 = (T)(-__ldcg(p.x + 3 * gr + 2));
      }
    }
    v[rr][0] = v0; v[rr][1] = v1; v[rr][2] = v2;
  }
  body_sync();
  T acc[CW][3];
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c][0] = acc[c][1] = acc[c][2] = T(0);
  if constexpr (kStream) {
    // stored layout [column c < bcv][row rr < rn], zeros above the diagonal of
    // L11^-1.  Staged into registers first (all shared loads in flight together;
    // reading them inside the product loop was measured ~2.5 us slower per tile),
    // then the same products in the same order as the masked register loads of the
    // FP64 path.
    const int rs = (int)rn;
    // products only from a completed copy (a rejected or timed-out copy leaves zeros)
    const int bcv = stage ? (int)min((int64_t)BC, nc - col0) : 0;
    const float* tile = stage ? stage : reinterpret_cast<const float*>(sm.buf);
    T qq[CW][RL];
#pragma unroll
    for (int c = 0; c < CW; ++c)
#pragma unroll
      for (int i = 0; i < RL; ++i) {
        const int rr = lane + 32 * i, cc = warp * CW + c;
        qq[c][i] = (rr < rs && cc < bcv) ? tile[cc * rs + rr] : T(0);
      }
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      const int rr = lane + 32 * i;
#pragma unroll
      for (int c = 0; c < CW; ++c) {
        acc[c][0] += qq[c][i] * v[rr][0];
        acc[c][1] += qq[c][i] * v[rr][1];
        acc[c][2] += qq[c][i] * v[rr][2];
      }
    }
  } else {
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      if (nb > 0) load_batch(nb);
#pragma unroll
      for (int i = 0; i < RB; ++i) {
        const int rr = lane + 32 * (nb * RB + i);
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          acc[c][0] += q[c][i] * v[rr][0];
          acc[c][1] += q[c][i] * v[rr][1];
          acc[c][2] += q[c][i] * v[rr][2];
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CW; ++c) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      acc[c][0] += __shfl_xor_sync(0xffffffffu, acc[c][0], off);
      acc[c][1] += __shfl_xor_sync(0xffffffffu, acc[c][1], off);
      acc[c][2] += __shfl_xor_sync(0xffffffffu, acc[c][2], off);
    }
    if (lane == 0) {
      res[warp * CW + c][0] = acc[c][0];
      res[warp * CW + c][1] = acc[c][1];
      res[warp * CW + c][2] = acc[c][2];
    }
  }
  body_sync();
  const int ntile = tl.ntile;
  if (ntile > 1) {
    T* part = reinterpret_cast<T*>(p.partial) + tid_g * kPart;
    for (int idx = threadIdx.x; idx < BC * 3; idx += kThreads) part[idx] = res[idx / 3][idx % 3];
    if (!last_of_block(p, tl, sm)) return;
    const T* parts = reinterpret_cast<const T*>(p.partial) + tl.part_base * kPart;
    for (int idx = threadIdx.x; idx < BC * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * kPart + idx);
      res[idx / 3][idx % 3] = t;
    }
    body_sync();
  }
  for (int jl = threadIdx.x; jl < BC; jl += kThreads) {
    const int64_t j = col0 + jl;
    if (j >= nc) continue;
    p.x[3 * (first + j)] = (double)res[jl][0];
    p.x[3 * (first + j) + 1] = (double)res[jl][1];
    p.x[3 * (first + j) + 2] = (double)res[jl][2];
  }
  signal_done(p.bdone + tl.s);
}

// tile kinds (SolveTile::pad0): forward with 1 / 2 / 4 column groups (R = kThreads,
// kThreads / 2, kThreads / 4 rows), backward with BC = 64 / 32 / 16 / 8 columns
enum TileKind { kF1 = 0, kF2 = 1, kF4 = 2, kB64 = 3, kB32 = 4, kB16 = 5, kB8 = 6 };

template <typename T>
__device__ __forceinline__ void run_tile(const SolveParams& p, const SolveTile& tl, int64_t tile,
                                         unsigned long long epoch, TileSmem<T>& sm, const float* stage) {
  switch (tl.pad0) {
    case kF1: fwd_tile_body<T, kThreads>(p, tl, tile, epoch, sm, stage); break;
    case kF2: fwd_tile_body<T, kThreads / 2>(p, tl, tile, epoch, sm, stage); break;
    case kF4: fwd_tile_body<T, kThreads / 4>(p, tl, tile, epoch, sm, stage); break;
    case kB64: bwd_tile_body<T, 64>(p, tl, tile, epoch, sm, stage); break;
    case kB32: bwd_tile_body<T, 32>(p, tl, tile, epoch, sm, stage); break;
    case kB16: bwd_tile_body<T, 16>(p, tl, tile, epoch, sm, stage); break;
    default: bwd_tile_body<T, 8>(p, tl, tile, epoch, sm, stage); break;
  }
}

// FP64 solve: every CTA draws its tickets itself and loads each tile's panel
// values into registers (batches of 16 loads per thread).
__global__ void __launch_bounds__(kThreads, 1) solve_persistent_kernel(SolveParams p) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  __shared__ TileSmem<double> sm;
  __shared__ unsigned long long tk[2];
  const unsigned long long per = (unsigned long long)p.ntiles + gridDim.x;
  if (threadIdx.x == 0) tk[0] = atomicAdd(p.gticket, 1ull);
  body_sync();
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
    run_tile<double>(p, tl, tile, epoch, sm, nullptr);
    body_sync();   // shared memory of this tile is free; the drawn ticket is visible
    slot ^= 1;
    t = tk[slot];
  }
}

// FP32 solve: a producer warp and kStages shared-memory stages per CTA.  The
// producer (one lane) draws the CTA's tickets in increasing order, loads each
// tile's descriptor and starts one bulk copy (cp.async.bulk, completion on the
// stage's "full" mbarrier) of the tile's streamed panel values into a free stage,
// so the copies of the next tiles are in flight while the 8 body warps work on
// the current one.  The body warps take the stages in the same order and return
// each one on its "empty" mbarrier.  A CTA holds at most kStages tickets and
// works on them in increasing order, so the lowest unfinished ticket is always the
// one a CTA is working on, and the schedule cannot deadlock.  Every wait is
// bounded: a dependency wait after SolveParams::spin_limit polls, a stage wait
// after about a second (DEV_ERR_TIMEOUT); a rejected descriptor (DEV_ERR_LAYOUT)
// is not copied and its tile skips its products.  A body wait that gives up
// leaves after waiting once more, bounded, for that stage's copy; the producer
// stops at the first stage wait that gives up.
struct PipeStage {
  SolveTile tl;
  int64_t tile;                  // tile index, -1 = no more tiles
  unsigned long long epoch;
  int copied;                    // 1 = the stage holds the tile's panel values
};

// dynamic shared memory of the FP32 kernel: kStages stages of kStreamBytes
extern __shared__ __align__(128) unsigned char solve_dsm[];

__global__ void __launch_bounds__(kPipeThreads, 2) solve_pipe_kernel(SolveParams p) {
  if (p.gate && (p.gate->converged || !p.gate->accepted)) return;
  __shared__ TileSmem<float> sm;
  __shared__ PipeStage stg[kStages];
  __shared__ __align__(8) unsigned long long full[kStages], empty[kStages];
  __shared__ int abort_flag;
  float* stage_buf = reinterpret_cast<float*>(solve_dsm);
  if (threadIdx.x == 0) {
    for (int k = 0; k < kStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();   // the only barrier of all 288 threads: the mbarriers are ready
  const unsigned long long per = (unsigned long long)p.ntiles + gridDim.x;
  // stage waits outlast a dependency wait (~1 s), which a tile may sit in
  constexpr unsigned long long kStageWaitNs = 4000000000ull;
  if (threadIdx.x >= kThreads) {
    // ---------------------------------------------------------------- producer
    if (threadIdx.x != kThreads) return;
    for (int k = 0;; ++k) {
      const int st = k % kStages;
      const unsigned ph = (unsigned)(k / kStages) & 1u;
      if (k >= kStages && !mbar_wait(&empty[st], ph ^ 1u, kStageWaitNs)) {
        atomicOr(p.err, DEV_ERR_TIMEOUT);
        return;   // the body warps time out on this stage in turn
      }
      PipeStage& sg = stg[st];
      const unsigned long long t = atomicAdd(p.gticket, 1ull);
      const int64_t tile = (int64_t)(t % per);
      if (tile >= p.ntiles || *(volatile int*)&abort_flag) {
        sg.tile = -1;
        mbar_arrive(&full[st]);
        return;
      }
      sg.tl = load_tile(p.tiles, tile);
      sg.tile = tile;
      sg.epoch = t / per;
      const float* src = p.Qs + sg.tl.soff;
      const uint32_t bytes = (uint32_t)sg.tl.sbytes;
      float* dst = stage_buf + (size_t)st * kTileElems;
      const bool ok = bytes > 0u && bytes <= (uint32_t)kStreamBytes && !(bytes & 15u) &&
                      !(smem_u32(dst) & 15u) && !(reinterpret_cast<uintptr_t>(src) & 15u);
      sg.copied = ok ? 1 : 0;
      if (!ok) {
        atomicOr(p.err, DEV_ERR_LAYOUT);   // nothing copied: the tile skips its products
        mbar_arrive(&full[st]);
        continue;
      }
      mbar_arrive_tx(&full[st], bytes);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(&full[st]))
                   : "memory");
    }
  }
  // ------------------------------------------------------------------ body warps
  for (int k = 0;; ++k) {
    const int st = k % kStages;
    const unsigned ph = (unsigned)(k / kStages) & 1u;
    if (!mbar_wait(&full[st], ph, kStageWaitNs)) {
      // the stage's copy may still be writing shared memory: it reads a source
      // range checked by the producer, so it completes; wait for it once more,
      // bounded, before the CTA retires
      if (threadIdx.x == 0) {
        atomicOr(p.err, DEV_ERR_TIMEOUT);
        abort_flag = 1;
      }
      mbar_wait(&full[st], ph, 2 * kStageWaitNs);
      return;
    }
    const PipeStage& sg = stg[st];
    if (sg.tile < 0) return;
    const SolveTile tl = sg.tl;
    run_tile<float>(p, tl, sg.tile, sg.epoch, sm, sg.copied ? stage_buf + (size_t)st * kTileElems : nullptr);
    body_sync();   // every body thread is done with the stage and its descriptor
    if (threadIdx.x == 0) mbar_arrive(&empty[st]);
  }
}

// forward rows per tile for a supernode: fewest idle column groups
int fwd_rows(int64_t nc) {
  if (nc <= kCols) return kThreads;
  if (nc <= 2 * kCols) return kThreads / 2;
  return kThreads / 4;
}

// backward columns per tile: the narrowest BC >= nc (64 at most), so a supernode
// of up to 64 columns is one column block
int bwd_cols(int64_t nc) {
  if (nc > 32) return 64;
  if (nc > 16) return 32;
  if (nc > 8) return 16;
  return 8;
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
  // output blocks per supernode (the counts a dependent tile waits for)
  S.nfb.assign(h.ns, 0);
  S.nbb.assign(h.ns, 0);
  for (int64_t s = 0; s < h.ns; ++s) {
    const int R = fwd_rows(h.nc(s));
    const int BC = bwd_cols(h.nc(s));
    S.nfb[s] = (int32_t)((h.nr(s) + R - 1) / R);
    S.nbb[s] = (int32_t)((h.nc(s) + BC - 1) / BC);
  }
  auto fwd_deps = [&](int64_t s, SolveTile& t) {
    t.ndep = (int32_t)(h.child_ptr[s + 1] - h.child_ptr[s]);
    for (int k = 0; k < kTileDeps && k < t.ndep; ++k) {
      const int64_t c = h.child_list[h.child_ptr[s] + k];
      t.dep[k] = (int32_t)c;
      t.dep_blocks[k] = S.nfb[c];
    }
  };
  auto bwd_deps = [&](int64_t s, SolveTile& t) {
    const int64_t par = h.parent[s];
    t.ndep = 1;
    t.dep[0] = par >= 0 ? (int32_t)par : (int32_t)(-s - 1);
    t.dep_blocks[0] = par >= 0 ? S.nbb[par] : S.nfb[s];
  };
  for (int64_t L = 0; L < h.nlev; ++L) {
    SolveLevel& sl = S.levels[L];
    sl.fwd_off = (int64_t)S.fwd.size();
    sl.bwd_off = (int64_t)S.bwd.size();
    for (int64_t i = h.level_ptr[L]; i < h.level_ptr[L + 1]; ++i) {
      const int64_t s = h.level_list[i];
      const int64_t nr = h.nr(s), nc = h.nc(s);
      const int R = fwd_rows(nc);
      const int C = (kThreads / R) * kCols;
      const int32_t fkind = R == kThreads ? kF1 : (R == kThreads / 2 ? kF2 : kF4);
      for (int64_t r0 = 0; r0 < nr; r0 += R) {
        const int32_t out = (int32_t)S.n_fwd_out++;
        const size_t b0 = S.fwd.size();
        // rows < nc of the L11^-1 block need columns <= row only
        const int64_t cmax = (r0 + R <= nc) ? r0 + R : nc;
        for (int64_t c0 = 0; c0 < cmax; c0 += C) {
          SolveTile t = base(s);
          t.a = (int32_t)r0;
          t.b = (int32_t)c0;
          t.out = out;
          t.part_base = (int64_t)b0;
          t.pad0 = fkind;
          fwd_deps(s, t);
          S.fwd.push_back(t);
        }
        for (size_t k = b0; k < S.fwd.size(); ++k) S.fwd[k].ntile = (int32_t)(S.fwd.size() - b0);
      }
      const int BC = bwd_cols(nc);
      const int BR = bwd_tile_rows(BC);
      const int32_t bkind = BC == 64 ? kB64 : (BC == 32 ? kB32 : (BC == 16 ? kB16 : kB8));
      for (int64_t c0 = 0; c0 < nc; c0 += BC) {
        const int32_t out = (int32_t)S.n_bwd_out++;
        const size_t b0 = S.bwd.size();
        // column c of L11^-1 is zero above row c: start at the row block holding c0
        for (int64_t r0 = (c0 / BR) * BR; r0 < nr; r0 += BR) {
          SolveTile t = base(s);
          t.a = (int32_t)c0;
          t.b = (int32_t)r0;
          t.out = out;
          t.part_base = (int64_t)b0;
          t.pad0 = bkind;
          bwd_deps(s, t);
          S.bwd.push_back(t);
        }
        for (size_t k = b0; k < S.bwd.size(); ++k) S.bwd[k].ntile = (int32_t)(S.bwd.size() - b0);
      }
    }
    sl.fwd_cnt = (int64_t)S.fwd.size() - sl.fwd_off;
    sl.bwd_cnt = (int64_t)S.bwd.size() - sl.bwd_off;
  }
  // persistent order: forward tiles by ascending level, backward tiles by
  // descending level (tiles of one output block stay contiguous); output ids of
  // backward blocks follow the forward ones; partial slots use the global index
  S.all.clear();
  for (const SolveTile& t : S.fwd) S.all.push_back(t);
  for (int64_t L = h.nlev - 1; L >= 0; --L) {
    const SolveLevel& sl = S.levels[L];
    const int64_t shift = (int64_t)S.all.size() - sl.bwd_off;
    for (int64_t k = sl.bwd_off; k < sl.bwd_off + sl.bwd_cnt; ++k) {
      SolveTile u = S.bwd[k];
      u.out += (int32_t)S.n_fwd_out;
      u.part_base += shift;
      S.all.push_back(u);
    }
  }
  // streamed FP32 layout, tile after tile in persistent order, each start 16-byte
  // aligned: forward [group][column k < kmax][row < rv], kmax = the columns of the
  // tile's last row inside its first group (the most of any thread); backward
  // [column < bcv][row < rn]
  int64_t off = 0;
  for (SolveTile& t : S.all) {
    int64_t elems = 0;
    if (t.pad0 <= kF4) {
      const int R = t.pad0 == kF1 ? kThreads : (t.pad0 == kF2 ? kThreads / 2 : kThreads / 4);
      const int64_t rv = std::min<int64_t>(R, (int64_t)t.nr - t.a);
      const int64_t rmax = t.a + rv - 1;
      const int64_t cend = rmax < t.nc ? std::min<int64_t>(t.nc, rmax + 1) : t.nc;
      const int64_t kmax = std::max<int64_t>(0, std::min<int64_t>(kCols, cend - t.b));
      t.sld = (int32_t)kmax;
      elems = (kThreads / R) * kmax * rv;
    } else {
      const int BC = t.pad0 == kB64 ? 64 : (t.pad0 == kB32 ? 32 : (t.pad0 == kB16 ? 16 : 8));
      const int64_t rn = std::min<int64_t>(bwd_tile_rows(BC), (int64_t)t.nr - t.b);
      const int64_t bcv = std::min<int64_t>(BC, (int64_t)t.nc - t.a);
      t.sld = (int32_t)rn;
      elems = bcv * rn;
    }
    const int64_t padded = (elems + 3) / 4 * 4;
    t.soff = off;
    t.sbytes = (int32_t)(padded * 4);
    off += padded;
  }
  S.stream_elems = off;
}

// Copies the FP32 panels into the streamed layout, one block per tile (the same
// index rules as the tile bodies' masked loads: zeros above the diagonal of L11^-1
// and past the panel).
__global__ void pack_stream_kernel(const SolveTile* tiles, const float* Q, float* Qs) {
  const SolveTile tl = load_tile(tiles, blockIdx.x);
  const int64_t nr = tl.nr, nc = tl.nc;
  const float* P = Q + tl.panel_off;
  float* out = Qs + tl.soff;
  int64_t total;
  if (tl.pad0 <= kF4) {
    const int R = tl.pad0 == kF1 ? kThreads : (tl.pad0 == kF2 ? kThreads / 2 : kThreads / 4);
    const int64_t rv = min((int64_t)R, nr - tl.a);
    const int64_t kmax = tl.sld;
    total = (kThreads / R) * kmax * rv;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
      const int64_t rl = i % rv, gk = i / rv;
      const int64_t k = gk % kmax, g = gk / kmax;
      const int64_t r = tl.a + rl, col = tl.b + g * kCols + k;
      const int64_t cend = r < nc ? min(nc, r + 1) : nc;
      out[i] = col < cend ? P[r + col * nr] : 0.0f;
    }
  } else {
    const int BC = tl.pad0 == kB64 ? 64 : (tl.pad0 == kB32 ? 32 : (tl.pad0 == kB16 ? 16 : 8));
    const int64_t rn = tl.sld;
    const int64_t bcv = min((int64_t)BC, nc - tl.a);
    total = bcv * rn;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
      const int64_t rr = i % rn, c = i / rn;
      const int64_t row = tl.b + rr, j = tl.a + c;
      out[i] = (row >= nc || row >= j) ? P[row + j * nr] : 0.0f;
    }
  }
  for (int64_t i = total + threadIdx.x; i < tl.sbytes / 4; i += blockDim.x) out[i] = 0.0f;
}

size_t solve_partial_bytes(const SolveSchedule& S) {
  return (S.fwd.size() + S.bwd.size()) * (size_t)kPart * sizeof(double);
}

// CTAs per SM of the FP32 (pipelined) kernel.  Both precisions launch this many
// CTAs per SM, so every solve consumes the same number of tickets; the FP64
// kernel has fewer resident at a time, which the ticket order tolerates (a CTA
// draws tickets only once it runs).
int solve_persistent_occupancy() {
  // the FP32 kernel's stages; set on the current device (meshes and servers call
  // this on their device before any solve)
  cudaFuncSetAttribute(solve_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStages * kStreamBytes);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_pipe_kernel, kPipeThreads, kStages * kStreamBytes);
  return std::max(1, occ);
}

cudaError_t pack_solve_stream(const MeshImpl* m, cudaStream_t st) {
  const int64_t ntiles = (int64_t)m->sched.all.size();
  if (!m->Qs || !m->Q32 || ntiles == 0) return cudaSuccess;
  pack_stream_kernel<<<(unsigned)ntiles, 256, 0, st>>>(m->all_tiles, m->Q32, m->Qs);
  return cudaGetLastError();
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
  p.Qs = f32 ? m->Qs : nullptr;
  if (f32 && !m->Qs) return cudaErrorInvalidValue;
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
  p.spin_limit = m->solve_spin_limit;
  p.stall_tile = -1;
  if (m->test_stall_solves > 0 && m->stall_tile >= 0) {
    p.stall_tile = m->stall_tile;
    --m->test_stall_solves;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(m->solve_grid, ntiles);
  if (f32) solve_pipe_kernel<<<grid, kPipeThreads, kStages * kStreamBytes, st>>>(p);
  else solve_persistent_kernel<<<grid, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace pd
