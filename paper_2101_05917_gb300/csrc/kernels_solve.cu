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
//
// Tiles.  A forward tile is one row block of a panel (R = 256, 128 or 64 rows,
// whichever covers the supernode's columns with the fewest idle column groups)
// over every column its rows need; a backward tile is one column block (BC = 64,
// 32, 16 or 8 columns, the narrowest covering the supernode) over every row from
// its first column down.  A tile is processed by one CTA from start to end.  In a
// level with few blocks (the top of the tree) a block is split into several tiles,
// runs of its consecutive chunks: each writes its partial sums to its own slots and
// the last to arrive (an arrival counter) adds them in tile order, so the result
// does not depend on scheduling either way.  The
// panel values of a tile flow through the CTA in chunks of at most 256 x 32
// entries: forward chunks are ranges of 32 columns per row group (256 / R
// groups), backward chunks ranges of 8192 / BC rows (at most 256).
//
// FP32: every chunk is stored contiguously in the order the tile body reads it
// (MeshImpl::Qs, packed once per factorisation; zeros for the upper triangle of
// L11^-1 and ragged edges) and reaches shared memory by one bulk copy
// (cp.async.bulk, completion on an mbarrier) that a producer warp issues into one
// of two stages per CTA, so the next chunk -- of the same tile or of the CTA's
// next tile -- is in flight while the body warps multiply the current one.  The
// right-hand-side rows a chunk needs are gathered one chunk ahead.  FP64 tiles
// load their chunks into registers (batches of 16 per thread).  Both sweeps run in
// one persistent launch scheduled by the supernodal tree dependencies (below).
#include <algorithm>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kThreads = 256;         // tile-body threads per CTA (8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kCols = 32;             // forward: columns per thread and chunk
constexpr int kChunkElems = kThreads * kCols;   // panel entries per chunk at most (32 KB in FP32)
constexpr int kMaxC = 4 * kCols;      // widest forward chunk (4 column groups)
// backward chunk rows for BC columns: kChunkElems / BC, at most 256 (8 rows per lane;
// the double-buffered right-hand side of three CTAs then fits beside their stages)
constexpr int kMaxBR = 256;
__host__ __device__ constexpr int bwd_chunk_rows(int bc) { return kChunkElems / bc < kMaxBR ? kChunkElems / bc : kMaxBR; }
constexpr int kPreSlots = 4;          // W-row sources per position held in registers
constexpr int kPart = kThreads * 3;   // partial-sum slots per tile (forward rows / backward columns x 3)
// tiles a level is cut into at least, where its blocks have enough chunks: blocks
// are split into runs of consecutive chunks until the level has this many tiles
// (more than the 456 resident CTAs of a 152-SM part; each split costs its tiles a
// partial-sum round trip, so a level is not cut finer than that)
constexpr int64_t kLevelTiles = 608;
constexpr int kStageBytes = kChunkElems * 4;   // one shared-memory stage of the FP32 kernel
constexpr int kStages = 2;                     // FP32 kernel: stages per CTA
constexpr int kPipeThreads = kThreads + 32;    // FP32 kernel: + one producer warp

// FP64 register loads issued back to back per thread (register budget)
constexpr int kBatch64 = 16;

struct SolveParams {
  const IterState* gate;
  const int32_t *rows;          // row structure of the supernodes
  const int32_t* wdest;         // per child update row: its slot in the parent's layout
  int slot_w;                   // slots per position
  const SolveTile* tiles;
  int64_t ntiles;               // forward tiles then backward tiles
  unsigned long long* gticket;  // tile tickets (grid + ntiles consumed per solve)
  unsigned long long* fdone;    // per supernode: finished forward row blocks
  unsigned long long* bdone;    // per supernode: finished backward column blocks
  const int32_t *nfb, *nbb;     // per supernode: forward / backward blocks
  unsigned long long* otick;    // per block (at its first tile's index): tiles finished, monotone
  void* partial;                // per tile partial sums of split blocks (kPart values of T)
  const int64_t *child_ptr, *child_list;
  int* err;
  long long spin_limit;         // polls of a dependency wait before it gives up
  int64_t stall_tile;           // test support: this tile's first wait target is raised by one (-1: none)
  const void* Q;
  const float* Qs;              // FP32: chunks stored contiguously (SolveTile::soff)
  const double* b;
  void* u;       // (3 nf) T
  void* W;       // (positions x slot_w x 3) T, children's updates in the parents' layout
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
// their forward row blocks, a backward tile for its parent's backward column
// blocks (the root for its own forward row blocks).  Every awaited tile has an
// earlier ticket and is held by a running CTA, so the waits end; they are also
// bounded (error flag DEV_ERR_TIMEOUT after SolveParams::spin_limit polls, about
// a second by default).  Counters only grow: a solve consumes ntiles + grid
// tickets (every CTA draws one ticket past the end), so ticket t belongs to
// solve t / (ntiles + grid).

// Message passing between CTAs: a producer's tile writes, then (after a CTA
// barrier) one thread's release reduction on a counter; a consumer's thread polls
// the counter with acquire loads, then a CTA barrier, then the CTA reads (through
// L2).  The barriers carry the ordering to the other threads of both CTAs
// (cumulativity).
__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void add_release(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
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

// true on every body thread when v is true on any of them (the barrier's reduction)
__device__ __forceinline__ bool body_any(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((unsigned)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ unsigned long long add_acq_rel(unsigned long long* p) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], 1;" : "=l"(old) : "l"(p) : "memory");
  return old;
}

// the last tile of a split block to finish?  (then every partial sum is written)
__device__ __forceinline__ bool last_of_block(const SolveParams& p, const SolveTile& tl, int64_t tile, int* flag) {
  body_sync();
  if (threadIdx.x == 0) {
    const unsigned long long v = add_acq_rel(p.otick + (tile - tl.tib));
    *flag = ((v + 1) % (unsigned long long)tl.ntile) == 0;
  }
  body_sync();
  return *flag != 0;
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

// ------------------------------------------------------------ L2 hints
// Every line of [base, base + bytes) into L2 (each address issued lies inside the
// range).
__device__ __forceinline__ void prefetch_l2(const void* base, size_t bytes) {
  if (bytes == 0) return;
  const char* c = static_cast<const char*>(base);
  for (size_t o = 0; o < bytes; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
  asm volatile("prefetch.global.L2 [%0];" ::"l"(c + bytes - 1));
}

// L2 policy for the panel chunks: each is read once per solve, so its lines go
// first, ahead of the right-hand side, update and solution rows the tiles gather.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// ------------------------------------------------------------ stage ring (FP32)
// One entry per stage: the chunk it holds, written by the producer before it arms
// the stage's "full" barrier.
struct PipeStage {
  SolveTile tl;                  // the tile's descriptor (read for a tile's first chunk)
  int64_t tile;                  // tile index, -1 = no more tiles
  unsigned long long epoch;
  int copied;                    // 1 = the stage holds the chunk's panel values
  int chunk;
};

// stage waits outlast a dependency wait (~1 s), which a tile may sit in
constexpr unsigned long long kStageWaitNs = 4000000000ull;

// The body warps' view of the ring: k counts the chunks taken so far.
struct Ring {
  float* buf;
  PipeStage* meta;
  unsigned long long* full;
  unsigned long long* empty;
  int* abort_flag;
  int* err;
  int k;
  // waits for chunk k's copy (bounded); false on every body thread when the wait
  // gave up on any of them
  __device__ __forceinline__ bool wait() {
    const int st = k % kStages;
    const bool ok = mbar_wait(&full[st], (unsigned)(k / kStages) & 1u, kStageWaitNs);
    if (!body_any(!ok)) return true;
    if (threadIdx.x == 0) {
      atomicOr(err, DEV_ERR_TIMEOUT);
      *abort_flag = 1;
    }
    // the copy may still be writing shared memory: it reads a source range checked
    // by the producer, so it completes; wait once more, bounded, before the CTA
    // retires
    mbar_wait(&full[st], (unsigned)(k / kStages) & 1u, 2 * kStageWaitNs);
    return false;
  }
  __device__ __forceinline__ const PipeStage& cur() const { return meta[k % kStages]; }
  __device__ __forceinline__ const float* data() const {
    return meta[k % kStages].copied ? buf + (size_t)(k % kStages) * kChunkElems : nullptr;
  }
  // every body thread is done with chunk k: hand its stage back to the producer
  __device__ __forceinline__ void release() {
    body_sync();
    if (threadIdx.x == 0) mbar_arrive(&empty[k % kStages]);
    ++k;
  }
};

// ------------------------------------------------------------ gathers
// The children's updates of a position: slot_w consecutive slots (unused ones are
// zero), summed in slot order.  Loaded into registers first (up to kPreSlots
// slots; more are added directly), so a chunk can issue them ahead.
template <typename T>
struct WRow {
  T w[kPreSlots][3];
};

template <typename T>
__device__ __forceinline__ void load_W(const SolveParams& p, int64_t position, bool valid, WRow<T>& r) {
  const T* W = reinterpret_cast<const T*>(p.W) + 3 * position * p.slot_w;
#pragma unroll
  for (int k = 0; k < kPreSlots; ++k) {
    const bool v = valid && k < p.slot_w;
    r.w[k][0] = v ? __ldcg(W + 3 * k) : T(0);
    r.w[k][1] = v ? __ldcg(W + 3 * k + 1) : T(0);
    r.w[k][2] = v ? __ldcg(W + 3 * k + 2) : T(0);
  }
}

// Sums in T: the FP32 tiles keep every gather and sum in FP32 (GB300's FP64 pipe
// is a small fraction of its FP32 pipe, and FP64 work here sat on each tile's
// critical path).
template <typename T>
__device__ __forceinline__ void sum_W(const SolveParams& p, int64_t position, bool valid, const WRow<T>& r,
                                      T& v0, T& v1, T& v2) {
#pragma unroll
  for (int k = 0; k < kPreSlots; ++k) {
    v0 += r.w[k][0];
    v1 += r.w[k][1];
    v2 += r.w[k][2];
  }
  if (!valid) return;
  const T* W = reinterpret_cast<const T*>(p.W) + 3 * position * p.slot_w;
  for (int k = kPreSlots; k < p.slot_w; ++k) {
    v0 += __ldcg(W + 3 * k);
    v1 += __ldcg(W + 3 * k + 1);
    v2 += __ldcg(W + 3 * k + 2);
  }
}

// shared memory of one tile body (as T): forward rhs[2][kMaxC][3] (double buffer)
// + red[kThreads][3]; backward v[2][kMaxBR][3] (double buffer) + res[64][3]
constexpr int kTileSmemElems = (2 * kMaxBR + 64) * 3 > 2 * kMaxC * 4 + kThreads * 3
                                   ? (2 * kMaxBR + 64) * 3 : 2 * kMaxC * 4 + kThreads * 3;
template <typename T>
struct __align__(16) TileSmem {
  T buf[kTileSmemElems];   // the larger of the backward and forward layouts above
  int flag;
};

// ------------------------------------------------------------ forward tile
// Row block [a, a + rv) of panel s, rv <= R, over its chunks of G * 32 columns
// (G = kThreads / R).  Thread (row rl, group g) owns row a + rl and, in a chunk,
// the group's columns 32 g ... (fewer in a block's last chunk: its L columns fill
// the groups in order).  Chunks are added in order, the group sums in group order
// at the end.
//
// The chunk's right-hand side rows rhs = b - (children's updates) are loaded one
// chunk ahead: thread jj < G 32 owns column jj of the next chunk.
template <typename T, int R>
__device__ void fwd_tile(const SolveParams& p, const SolveTile& tl, int64_t tile, unsigned long long epoch,
                         TileSmem<T>& sm, Ring* ring) {
  constexpr bool kStream = sizeof(T) == 4;
  constexpr int G = kThreads / R;
  constexpr int CW = G * kCols;       // columns per chunk
  // right-hand side rows, double-buffered: FP32 as float4 (one shared load per
  // column), FP64 as 3 doubles
  float4 (*rhs4)[kMaxC] = reinterpret_cast<float4 (*)[kMaxC]>(sm.buf);
  T (*rhs)[kMaxC][3] = reinterpret_cast<T (*)[kMaxC][3]>(sm.buf);
  T (*red)[3] = reinterpret_cast<T (*)[3]>(sm.buf + 2 * kMaxC * 4);
  const int64_t row0 = tl.a;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr, pos = tl.pos;
  const int nch = tl.nchunks;
  const int rl = threadIdx.x % R, g = threadIdx.x / R;
  const int64_t r = row0 + rl;
  const int rv = (int)min((int64_t)R, nr - row0);
  // L11^-1 is lower triangular: rows < nc use columns <= row only
  const int64_t cend_r = r >= nr ? 0 : (r < nc ? min(nc, r + 1) : nc);
  const T* Qr = reinterpret_cast<const T*>(p.Q) + tl.panel_off + r;
  const bool own_col = (int)threadIdx.x < CW;
  const bool kids = tl.ndep > 0;      // leaves have no children's updates
  auto col_of = [&](int c) -> int64_t { return (int64_t)(tl.chunk0 + c) * CW + threadIdx.x; };
  // static data first: the output row's slot in the parent, the first chunk's b rows
  const bool out_w = g == 0 && r < nr && r >= nc;
  const int32_t wd = out_w ? __ldg(p.wdest + tl.relp + (r - nc)) : 0;
  double bb0 = 0, bb1 = 0, bb2 = 0;
  bool has = own_col && col_of(0) < nc;
  if (has) {
    const double* bp = p.b + 3 * (first + col_of(0));
    bb0 = __ldg(bp), bb1 = __ldg(bp + 1), bb2 = __ldg(bp + 2);
  }
  if (threadIdx.x < 32) {
    // the children's forward outputs: those inline in the descriptor polled in
    // parallel, one lane each; more (rare) from the tree by lane 0
    const int nd = tl.ndep, lane = threadIdx.x;
    int32_t dk = 0, bk = 0;
#pragma unroll
    for (int k = 0; k < kTileDeps; ++k)
      if (lane == k) {
        dk = tl.dep[k];
        bk = tl.dep_blocks[k];
      }
    if (lane < nd && lane < kTileDeps)
      wait_count(p.fdone + dk, (epoch + 1) * (unsigned long long)bk + (lane == 0 && tile == p.stall_tile ? 1 : 0),
                 p.err, p.spin_limit);
    if (nd > kTileDeps && lane == 0) {
      for (int64_t ci = __ldg(p.child_ptr + tl.s) + kTileDeps; ci < __ldg(p.child_ptr + tl.s + 1); ++ci) {
        const int64_t c = __ldg(p.child_list + ci);
        wait_count(p.fdone + c, (epoch + 1) * (unsigned long long)__ldg(p.nfb + c), p.err, p.spin_limit);
      }
    }
  }
  body_sync();
  // children's updates of the output row (below rows) and of the first chunk's columns
  WRow<T> wc;
  T o0 = T(0), o1 = T(0), o2 = T(0);
  {
    WRow<T> wo;
    load_W<T>(p, pos + r, out_w && kids, wo);
    load_W<T>(p, pos + col_of(0), has && kids, wc);
    sum_W<T>(p, pos + r, out_w && kids, wo, o0, o1, o2);
  }
  auto put_rhs = [&](int buf, bool h, const WRow<T>& wr, int64_t col) {
    T w0 = T(0), w1 = T(0), w2 = T(0);
    sum_W<T>(p, pos + col, h && kids, wr, w0, w1, w2);
    const T v0 = h ? (T)bb0 - w0 : T(0), v1 = h ? (T)bb1 - w1 : T(0), v2 = h ? (T)bb2 - w2 : T(0);
    if constexpr (kStream) rhs4[buf][threadIdx.x] = make_float4(v0, v1, v2, 0.0f);
    else {
      rhs[buf][threadIdx.x][0] = v0;
      rhs[buf][threadIdx.x][1] = v1;
      rhs[buf][threadIdx.x][2] = v2;
    }
  };
  if (own_col) put_rhs(0, has, wc, col_of(0));
  body_sync();
  T a0 = T(0), a1 = T(0), a2 = T(0);
  for (int c = 0; c < nch; ++c) {
    // next chunk's rhs rows: every load issued now, added after the products
    const bool nxt = c + 1 < nch;
    const int64_t jn = col_of(c + 1);
    has = nxt && own_col && jn < nc;
    if (has) {
      const double* bp = p.b + 3 * (first + jn);
      bb0 = __ldg(bp), bb1 = __ldg(bp + 1), bb2 = __ldg(bp + 2);
    }
    load_W<T>(p, pos + jn, has && kids, wc);
    if constexpr (kStream) {
      // stored layout [group][column k < kmax_g][row rl < rv]: group g holds
      // kmax_g = clamp(L - 32 g, 0, 32) of the chunk's L columns; zeros past each
      // row's columns
      if (c > 0 && !ring->wait()) return;
      const float* stage = ring->data();
      const int L = c + 1 < nch ? CW : tl.lld;
      const int kmax = max(0, min(kCols, L - g * kCols));
      const float4* rg = rhs4[c & 1] + g * kCols;
      if (rl < rv && stage) {
        const float* qs = stage + min(L, g * kCols) * rv + rl;
#pragma unroll 8
        for (int k = 0; k < kmax; ++k) {
          const float qk = qs[k * rv];
          const float4 b4 = rg[k];
          a0 += qk * b4.x;
          a1 += qk * b4.y;
          a2 += qk * b4.z;
        }
      }
    } else {
      const T(*rg)[3] = rhs[c & 1] + g * kCols;
      const int64_t cg0 = (int64_t)(tl.chunk0 + c) * CW + (int64_t)g * kCols;
      const int cnt = (int)max((int64_t)0, min((int64_t)kCols, cend_r - cg0));
      const T* Qc = Qr + cg0 * nr;
#pragma unroll
      for (int nb = 0; nb < kCols / kBatch64; ++nb) {
        T q[kBatch64];
#pragma unroll
        for (int k = 0; k < kBatch64; ++k)
          q[k] = (nb * kBatch64 + k < cnt) ? __ldg(Qc + (int64_t)(nb * kBatch64 + k) * nr) : T(0);
#pragma unroll
        for (int k = 0; k < kBatch64; ++k) {
          a0 += q[k] * rg[nb * kBatch64 + k][0];
          a1 += q[k] * rg[nb * kBatch64 + k][1];
          a2 += q[k] * rg[nb * kBatch64 + k][2];
        }
      }
    }
    if (nxt && own_col) put_rhs((c + 1) & 1, has, wc, jn);
    if constexpr (kStream) ring->release();   // includes the barrier
    else body_sync();
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
    // split block: this tile's sums, then the last tile adds all in tile order
    T* part = reinterpret_cast<T*>(p.partial) + tile * kPart;
    if (g == 0) {
      part[3 * rl] = a0;
      part[3 * rl + 1] = a1;
      part[3 * rl + 2] = a2;
    }
    if (!last_of_block(p, tl, tile, &sm.flag)) return;
    if (g == 0) {
      const T* parts = reinterpret_cast<const T*>(p.partial) + (tile - tl.tib) * kPart + 3 * rl;
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
      // this row's update into its slot of the parent's position
      T* Wo = reinterpret_cast<T*>(p.W) + 3 * (int64_t)wd;
      Wo[0] = a0 + o0;
      Wo[1] = a1 + o1;
      Wo[2] = a2 + o2;
    }
  }
  signal_done(p.fdone + tl.s);
}

// ------------------------------------------------------------ backward tile
// Column block [a, a + bcv) of panel s, bcv <= BC, over rows [a, nr) in chunks of
// BR = min(8192 / BC, 256) rows.  Warp w owns columns a + w CW ... (CW = BC / 8),
// its lanes the chunk's rows lane + 32 i; per column the lanes' sums are added by
// a fixed shuffle tree at the end.  v = [u_s; -x(below rows)] of the next chunk's
// rows is gathered one chunk ahead (thread t owns rows t + 256 k of a chunk).
template <typename T, int BC>
__device__ void bwd_tile(const SolveParams& p, const SolveTile& tl, int64_t tile, unsigned long long epoch,
                         TileSmem<T>& sm, Ring* ring) {
  constexpr bool kStream = sizeof(T) == 4;
  constexpr int CW = BC / kWarps;
  constexpr int BR = bwd_chunk_rows(BC);
  constexpr int RL = BR / 32;           // rows per lane and chunk
  constexpr int VR = (BR + kThreads - 1) / kThreads;   // v rows per thread and chunk
  T (*v)[kMaxBR][3] = reinterpret_cast<T (*)[kMaxBR][3]>(sm.buf);
  T (*res)[3] = reinterpret_cast<T (*)[3]>(sm.buf + 2 * kMaxBR * 3);
  const int64_t col0 = tl.a;
  const int64_t first = tl.first, nc = tl.nc, nr = tl.nr;
  const int32_t* srows = p.rows + tl.pos;
  const T* Q = reinterpret_cast<const T*>(p.Q) + tl.panel_off;
  const T* u = reinterpret_cast<const T*>(p.u);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nch = tl.nchunks;
  const int bcv = (int)min((int64_t)BC, nc - col0);
  auto chunk_row0 = [&](int c) -> int64_t { return col0 + (int64_t)(tl.chunk0 + c) * BR; };
  // global rows of a chunk's below rows (static)
  int32_t gidx[VR];
  auto load_gidx = [&](int c) {
    const int64_t r0 = chunk_row0(c);
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int64_t row = r0 + threadIdx.x + (int64_t)k * kThreads;
      gidx[k] = ((int)threadIdx.x + k * kThreads < BR && row < nr && row >= nc) ? __ldg(srows + row) : -1;
    }
  };
  // v rows of a chunk into registers (u rows now, x rows written by the parent)
  T vv[VR][3];
  auto load_v = [&](int c) {
    const int64_t r0 = chunk_row0(c);
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int64_t row = r0 + threadIdx.x + (int64_t)k * kThreads;
      T v0 = T(0), v1 = T(0), v2 = T(0);
      if ((int)threadIdx.x + k * kThreads < BR && row < nr) {
        if (row < nc) {
          const T* ur = u + 3 * (first + row);
          v0 = __ldcg(ur); v1 = __ldcg(ur + 1); v2 = __ldcg(ur + 2);
        } else {
          const int64_t gr = gidx[k];
          v0 = -(T)__ldcg(p.x + 3 * gr); v1 = -(T)__ldcg(p.x + 3 * gr + 1); v2 = -(T)__ldcg(p.x + 3 * gr + 2);
        }
      }
      vv[k][0] = v0; vv[k][1] = v1; vv[k][2] = v2;
    }
  };
  auto store_v = [&](int buf) {
#pragma unroll
    for (int k = 0; k < VR; ++k) {
      const int rr = threadIdx.x + k * kThreads;
      if (rr < BR) {
        v[buf][rr][0] = vv[k][0]; v[buf][rr][1] = vv[k][1]; v[buf][rr][2] = vv[k][2];
      }
    }
  };
  load_gidx(0);
  if (threadIdx.x == 0) {
    // the parent's backward outputs; the root waits for its own forward outputs
    const int32_t d = tl.dep[0];
    if (d >= 0) wait_count(p.bdone + d, (epoch + 1) * (unsigned long long)tl.dep_blocks[0], p.err, p.spin_limit);
    else wait_count(p.fdone + (-d - 1), (epoch + 1) * (unsigned long long)tl.dep_blocks[0], p.err, p.spin_limit);
  }
  body_sync();
  load_v(0);
  store_v(0);
  body_sync();
  T acc[CW][3];
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[c][0] = acc[c][1] = acc[c][2] = T(0);
  for (int c = 0; c < nch; ++c) {
    const bool nxt = c + 1 < nch;
    if (nxt) load_gidx(c + 1);
    const int64_t r0 = chunk_row0(c);
    const int rn = (int)min((int64_t)BR, nr - r0);
    const T(*vc)[3] = v[c & 1];
    if constexpr (kStream) {
      // stored layout [column c < bcv][row rr < rn], zeros above the diagonal of
      // L11^-1.  Staged into registers first (all shared loads in flight together),
      // then the same products in the same order as the masked register loads of
      // the FP64 path.
      if (c > 0 && !ring->wait()) return;
      const float* stage = ring->data();
      const int cols = stage ? bcv : 0;   // products only from a completed copy
      if (nxt) load_v(c + 1);
      // in batches of at most 16 staged values per thread (register budget)
      constexpr int NB = CW * RL > 16 ? CW * RL / 16 : 1;
      constexpr int RB = RL / NB;
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) {
        T qq[CW][RB];
#pragma unroll
        for (int cc = 0; cc < CW; ++cc)
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            const int rr = lane + 32 * (nb * RB + i), col = warp * CW + cc;
            qq[cc][i] = (rr < rn && col < cols) ? stage[col * rn + rr] : T(0);
          }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int rr = lane + 32 * (nb * RB + i);
          const T v0 = vc[rr][0], v1 = vc[rr][1], v2 = vc[rr][2];
#pragma unroll
          for (int cc = 0; cc < CW; ++cc) {
            acc[cc][0] += qq[cc][i] * v0;
            acc[cc][1] += qq[cc][i] * v1;
            acc[cc][2] += qq[cc][i] * v2;
          }
        }
      }
    } else {
      if (nxt) load_v(c + 1);
      constexpr int NB = CW * RL > kBatch64 ? CW * RL / kBatch64 : 1;   // load batches
      constexpr int RB = RL / NB;                                          // rows per lane per batch
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) {
        T q[CW][RB];
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) {
          const int64_t j = col0 + warp * CW + cc;
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            const int rr = lane + 32 * (nb * RB + i);
            const int64_t row = r0 + rr;
            // column j of L11^-1 is zero above row j
            q[cc][i] = (j < nc && rr < rn && (row >= nc || row >= j)) ? __ldg(Q + row + j * nr) : T(0);
          }
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          const int rr = lane + 32 * (nb * RB + i);
#pragma unroll
          for (int cc = 0; cc < CW; ++cc) {
            acc[cc][0] += q[cc][i] * vc[rr][0];
            acc[cc][1] += q[cc][i] * vc[rr][1];
            acc[cc][2] += q[cc][i] * vc[rr][2];
          }
        }
      }
    }
    if (nxt) store_v((c + 1) & 1);
    if constexpr (kStream) ring->release();   // includes the barrier
    else body_sync();
  }
#pragma unroll
  for (int cc = 0; cc < CW; ++cc) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      acc[cc][0] += __shfl_xor_sync(0xffffffffu, acc[cc][0], off);
      acc[cc][1] += __shfl_xor_sync(0xffffffffu, acc[cc][1], off);
      acc[cc][2] += __shfl_xor_sync(0xffffffffu, acc[cc][2], off);
    }
    if (lane == 0) {
      res[warp * CW + cc][0] = acc[cc][0];
      res[warp * CW + cc][1] = acc[cc][1];
      res[warp * CW + cc][2] = acc[cc][2];
    }
  }
  body_sync();
  const int ntile = tl.ntile;
  if (ntile > 1) {
    // split block: this tile's sums, then the last tile adds all in tile order
    T* part = reinterpret_cast<T*>(p.partial) + tile * kPart;
    for (int idx = threadIdx.x; idx < BC * 3; idx += kThreads) part[idx] = res[idx / 3][idx % 3];
    if (!last_of_block(p, tl, tile, &sm.flag)) return;
    const T* parts = reinterpret_cast<const T*>(p.partial) + (tile - tl.tib) * kPart;
    for (int idx = threadIdx.x; idx < BC * 3; idx += kThreads) {
      T t = T(0);
      for (int k = 0; k < ntile; ++k) t += __ldcg(parts + (int64_t)k * kPart + idx);
      res[idx / 3][idx % 3] = t;
    }
    body_sync();
  }
  for (int jl = threadIdx.x; jl < bcv; jl += kThreads) {
    const int64_t j = col0 + jl;
    p.x[3 * (first + j)] = (double)res[jl][0];
    p.x[3 * (first + j) + 1] = (double)res[jl][1];
    p.x[3 * (first + j) + 2] = (double)res[jl][2];
  }
  signal_done(p.bdone + tl.s);
}

// tile kinds (SolveTile::kind): forward row blocks of 256 / 128 / 64 rows (1 / 2 /
// 4 column groups), backward column blocks of 64 / 32 / 16 / 8 columns
enum TileKind { kF1 = 0, kF2 = 1, kF4 = 2, kB64 = 3, kB32 = 4, kB16 = 5, kB8 = 6 };

template <typename T>
__device__ __forceinline__ void run_tile(const SolveParams& p, const SolveTile& tl, int64_t tile,
                                         unsigned long long epoch, TileSmem<T>& sm, Ring* ring) {
  switch (tl.kind) {
    case kF1: fwd_tile<T, kThreads>(p, tl, tile, epoch, sm, ring); break;
    case kF2: fwd_tile<T, kThreads / 2>(p, tl, tile, epoch, sm, ring); break;
    case kF4: fwd_tile<T, kThreads / 4>(p, tl, tile, epoch, sm, ring); break;
    case kB64: bwd_tile<T, 64>(p, tl, tile, epoch, sm, ring); break;
    case kB32: bwd_tile<T, 32>(p, tl, tile, epoch, sm, ring); break;
    case kB16: bwd_tile<T, 16>(p, tl, tile, epoch, sm, ring); break;
    default: bwd_tile<T, 8>(p, tl, tile, epoch, sm, ring); break;
  }
}

// FP64 solve: every CTA draws its tickets itself and loads each chunk's panel
// values into registers.
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

// The static rows a chunk's body reads beside its panel values, into L2 when the
// chunk's copy is issued (a stage or more before the body reaches it): forward,
// the right-hand side rows of the chunk's columns and, with the first chunk, the
// parent slots of the block's update rows; backward, the global indices of the
// chunk's update rows and its own u rows.
__device__ __forceinline__ void prefetch_chunk_rows(const SolveParams& p, const SolveTile& tl, int c) {
  const int64_t nc = tl.nc, nr = tl.nr;
  if (tl.kind <= kF4) {
    const int G = 1 << tl.kind;
    const int64_t CW = (int64_t)G * kCols;
    const int64_t c0 = (int64_t)(tl.chunk0 + c) * CW, c1 = min(nc, c0 + CW);
    if (c1 > c0) prefetch_l2(p.b + 3 * ((int64_t)tl.first + c0), (size_t)(c1 - c0) * 3 * sizeof(double));
    if (c == 0) {
      const int64_t r0 = max((int64_t)tl.a, nc), r1 = min((int64_t)tl.a + kThreads / G, nr);
      if (r1 > r0) prefetch_l2(p.wdest + tl.relp + (r0 - nc), (size_t)(r1 - r0) * sizeof(int32_t));
    }
  } else {
    const int BR = bwd_chunk_rows(64 >> (tl.kind - kB64));
    const int64_t r0 = (int64_t)tl.a + (int64_t)(tl.chunk0 + c) * BR, r1 = min(r0 + BR, nr);
    const int64_t g0 = max(r0, nc);
    if (r1 > g0) prefetch_l2(p.rows + tl.pos + g0, (size_t)(r1 - g0) * sizeof(int32_t));
    const int64_t u1 = min(r1, nc);
    if (u1 > r0)
      prefetch_l2(static_cast<const float*>(p.u) + 3 * ((int64_t)tl.first + r0), (size_t)(u1 - r0) * 3 * sizeof(float));
  }
}

// dynamic shared memory of the FP32 kernel: kStages stages of kStageBytes
extern __shared__ __align__(128) unsigned char solve_dsm[];

// FP32 solve: a producer warp and kStages shared-memory stages per CTA.  The
// producer (one lane) draws the CTA's tickets in increasing order, loads each
// tile's descriptor and streams the tile's chunks, one bulk copy per chunk, into
// the stages as they come free; the 8 body warps take the stages in the same
// order.  A CTA holds at most kStages tickets and works on them in increasing
// order, so the lowest unfinished ticket is always the one a CTA is working on,
// and the schedule cannot deadlock.  Every wait is bounded: a dependency wait
// after SolveParams::spin_limit polls, a stage wait after a few seconds
// (DEV_ERR_TIMEOUT); a rejected chunk (DEV_ERR_LAYOUT) is not copied and the tile
// skips its products.  A body wait that gives up leaves after waiting once more,
// bounded, for that stage's copy; the producer stops at the first stage wait that
// gives up, or when the body has given up.
// Three CTAs of 288 threads per SM (72 registers per thread, 2 x 32 KB stages and
// 7.4 KB of tile-body buffers each): more tiles in flight per SM hide more of each
// tile's dependency, gather and release latency (the 64x64x128 beam's solve pair
// took 11 % less time than with two CTAs of 2 x 48 KB stages).
__global__ void __launch_bounds__(kPipeThreads, 3) solve_pipe_kernel(SolveParams p) {
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
  if (threadIdx.x >= kThreads) {
    // ---------------------------------------------------------------- producer
    if (threadIdx.x != kThreads) return;
    int k = 0;   // chunks issued
    const uint64_t pol = evict_first_policy();
    auto take = [&](int st) -> bool {   // wait until stage st is free again
      if (k < kStages) return true;
      if (mbar_wait(&empty[st], ((unsigned)(k / kStages) & 1u) ^ 1u, kStageWaitNs)) return true;
      atomicOr(p.err, DEV_ERR_TIMEOUT);
      return false;
    };
    while (true) {
      const int st0 = k % kStages;
      if (!take(st0)) return;   // the body warps time out on this stage in turn
      const unsigned long long t = atomicAdd(p.gticket, 1ull);
      const int64_t tile = (int64_t)(t % per);
      if (tile >= p.ntiles || *(volatile int*)&abort_flag) {
        stg[st0].tile = -1;
        mbar_arrive(&full[st0]);
        return;
      }
      const SolveTile tl = load_tile(p.tiles, tile);
      for (int c = 0; c < tl.nchunks; ++c) {
        const int st = k % kStages;
        if (c > 0 && !take(st)) return;
        prefetch_chunk_rows(p, tl, c);
        PipeStage& sg = stg[st];
        if (c == 0) sg.tl = tl;
        sg.tile = tile;
        sg.epoch = t / per;
        sg.chunk = c;
        const bool last = c + 1 == tl.nchunks;
        const float* src = p.Qs + tl.soff + (int64_t)c * (tl.cbytes / 4);
        const uint32_t bytes = (uint32_t)(last ? tl.lbytes : tl.cbytes);
        float* dst = stage_buf + (size_t)st * kChunkElems;
        const bool ok = bytes > 0u && bytes <= (uint32_t)kStageBytes && !(bytes & 15u) &&
                        !(smem_u32(dst) & 15u) && !(reinterpret_cast<uintptr_t>(src) & 15u);
        sg.copied = ok ? 1 : 0;
        ++k;
        if (!ok) {
          atomicOr(p.err, DEV_ERR_LAYOUT);   // nothing copied: the tile skips its products
          mbar_arrive(&full[st]);
          continue;
        }
        mbar_arrive_tx(&full[st], bytes);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
            ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(&full[st])), "l"(pol)
            : "memory");
      }
    }
  }
  // ------------------------------------------------------------------ body warps
  Ring ring{stage_buf, stg, full, empty, &abort_flag, p.err, 0};
  while (true) {
    if (!ring.wait()) return;   // the next tile's first chunk, or the end marker
    const PipeStage& sg = ring.cur();
    if (sg.tile < 0) return;
    const SolveTile tl = sg.tl;
    const int64_t tile = sg.tile;
    const unsigned long long epoch = sg.epoch;
    const int k0 = ring.k;
    run_tile<float>(p, tl, tile, epoch, sm, &ring);
    if (ring.k != k0 + tl.nchunks) return;   // a chunk wait gave up inside the tile
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

// Builds the tile lists (host) -- called once per mesh.
void build_solve_schedule(const HostMesh& h, SolveSchedule& S) {
  S.fwd.clear();
  S.bwd.clear();
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
  // blocks per supernode (the counts a dependent tile waits for)
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
  // a block as a whole (nchunks = its chunks, lld = its last chunk's dimension),
  // cut into runs of at most kc chunks
  auto split = [](const SolveTile& blk, int64_t kc, int last_full_ld, std::vector<SolveTile>& out) {
    const int nt = (int)((blk.nchunks + kc - 1) / kc);
    for (int k = 0; k < nt; ++k) {
      SolveTile t = blk;
      t.chunk0 = (int32_t)(k * kc);
      t.nchunks = (int32_t)std::min<int64_t>(kc, blk.nchunks - k * kc);
      const bool has_last = t.chunk0 + t.nchunks == blk.nchunks;
      t.lld = has_last ? blk.lld : last_full_ld;
      t.ntile = nt;
      t.tib = k;
      out.push_back(t);
    }
  };
  for (int64_t L = 0; L < h.nlev; ++L) {
    SolveLevel& sl = S.levels[L];
    sl.fwd_off = (int64_t)S.fwd.size();
    sl.bwd_off = (int64_t)S.bwd.size();
    std::vector<SolveTile> fb, bb;   // the level's blocks
    for (int64_t i = h.level_ptr[L]; i < h.level_ptr[L + 1]; ++i) {
      const int64_t s = h.level_list[i];
      const int64_t nr = h.nr(s), nc = h.nc(s);
      const int R = fwd_rows(nc);
      const int G = kThreads / R;
      const int64_t CW = (int64_t)G * kCols;
      const int32_t fkind = R == kThreads ? kF1 : (R == kThreads / 2 ? kF2 : kF4);
      for (int64_t r0 = 0; r0 < nr; r0 += R) {
        SolveTile t = base(s);
        t.kind = fkind;
        t.a = (int32_t)r0;
        // rows < nc of the L11^-1 block need columns <= row only
        const int64_t rv = std::min<int64_t>(R, nr - r0);
        const int64_t rmax = r0 + rv - 1;
        const int64_t cend = rmax < nc ? std::min<int64_t>(nc, rmax + 1) : nc;
        t.nchunks = (int32_t)((cend + CW - 1) / CW);
        // the last chunk's columns (they fill the groups in order)
        t.lld = (int32_t)(cend - (int64_t)(t.nchunks - 1) * CW);
        fwd_deps(s, t);
        fb.push_back(t);
      }
      const int BC = bwd_cols(nc);
      const int BR = bwd_chunk_rows(BC);
      const int32_t bkind = BC == 64 ? kB64 : (BC == 32 ? kB32 : (BC == 16 ? kB16 : kB8));
      for (int64_t c0 = 0; c0 < nc; c0 += BC) {
        SolveTile t = base(s);
        t.kind = bkind;
        t.a = (int32_t)c0;
        // column c of L11^-1 is zero above row c: rows from c0 on
        const int64_t rows = nr - c0;
        t.nchunks = (int32_t)((rows + BR - 1) / BR);
        t.lld = (int32_t)(rows - (int64_t)(t.nchunks - 1) * BR);
        bwd_deps(s, t);
        bb.push_back(t);
      }
    }
    // chunks per tile: the most for which the level still has kLevelTiles tiles
    // (whole blocks when it has that many blocks)
    auto chunks_per_tile = [](const std::vector<SolveTile>& blocks) -> int64_t {
      int64_t total = 0, most = 1;
      for (const SolveTile& t : blocks) total += t.nchunks, most = std::max<int64_t>(most, t.nchunks);
      if ((int64_t)blocks.size() >= kLevelTiles) return most;
      return std::max<int64_t>(1, std::min<int64_t>(most, total / kLevelTiles));
    };
    const int64_t kcf = chunks_per_tile(fb), kcb = chunks_per_tile(bb);
    for (const SolveTile& t : fb) {
      const int R = t.kind == kF1 ? kThreads : (t.kind == kF2 ? kThreads / 2 : kThreads / 4);
      split(t, kcf, (kThreads / R) * kCols, S.fwd);
    }
    for (const SolveTile& t : bb) {
      const int BC = t.kind == kB64 ? 64 : (t.kind == kB32 ? 32 : (t.kind == kB16 ? 16 : 8));
      split(t, kcb, bwd_chunk_rows(BC), S.bwd);
    }
    sl.fwd_cnt = (int64_t)S.fwd.size() - sl.fwd_off;
    sl.bwd_cnt = (int64_t)S.bwd.size() - sl.bwd_off;
  }
  // persistent order: forward tiles by ascending level, backward tiles by
  // descending level (the tiles of a block stay consecutive)
  S.all.clear();
  for (const SolveTile& t : S.fwd) S.all.push_back(t);
  for (int64_t L = h.nlev - 1; L >= 0; --L) {
    const SolveLevel& sl = S.levels[L];
    for (int64_t k = sl.bwd_off; k < sl.bwd_off + sl.bwd_cnt; ++k) S.all.push_back(S.bwd[k]);
  }
  // streamed FP32 layout, tile after tile in persistent order, chunk after chunk,
  // each chunk 16-byte aligned: forward [group][column k < kmax_g][row < rv] with
  // kmax_g = clamp(L - 32 g, 0, 32) for a chunk of L columns, backward [column <
  // bcv][row < rn]
  int64_t off = 0, chunks = 0;
  for (SolveTile& t : S.all) {
    int64_t full = 0, last = 0;
    if (t.kind <= kF4) {
      const int R = t.kind == kF1 ? kThreads : (t.kind == kF2 ? kThreads / 2 : kThreads / 4);
      const int G = kThreads / R;
      const int64_t rv = std::min<int64_t>(R, (int64_t)t.nr - t.a);
      full = (int64_t)G * kCols * rv;
      last = (int64_t)t.lld * rv;
    } else {
      const int BC = t.kind == kB64 ? 64 : (t.kind == kB32 ? 32 : (t.kind == kB16 ? 16 : 8));
      const int64_t bcv = std::min<int64_t>(BC, (int64_t)t.nc - t.a);
      full = bcv * bwd_chunk_rows(BC);
      last = bcv * t.lld;
    }
    const int64_t lpad = (last + 3) / 4 * 4;
    t.soff = off;
    t.cbytes = (int32_t)(full * 4);
    t.lbytes = (int32_t)(lpad * 4);
    off += full * (t.nchunks - 1) + lpad;
    chunks += t.nchunks;
  }
  S.stream_elems = off;
  S.chunks = chunks;
}

size_t solve_partial_bytes(const SolveSchedule& S) {
  return S.all.size() * (size_t)kPart * sizeof(double);
}

// Copies the FP32 panels into the streamed layout, one block per tile (the same
// index rules as the tile bodies' masked loads: zeros above the diagonal of L11^-1
// and past the panel).
__global__ void pack_stream_kernel(const SolveTile* tiles, const float* Q, float* Qs) {
  const SolveTile tl = load_tile(tiles, blockIdx.x);
  const int64_t nr = tl.nr, nc = tl.nc;
  const float* P = Q + tl.panel_off;
  for (int c = 0; c < tl.nchunks; ++c) {
    float* out = Qs + tl.soff + (int64_t)c * (tl.cbytes / 4);
    const bool last = c + 1 == tl.nchunks;
    int64_t total;
    if (tl.kind <= kF4) {
      const int R = tl.kind == kF1 ? kThreads : (tl.kind == kF2 ? kThreads / 2 : kThreads / 4);
      const int G = kThreads / R;
      const int64_t rv = min((int64_t)R, nr - tl.a);
      const int64_t L = last ? tl.lld : (int64_t)G * kCols;
      total = L * rv;
      for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        // groups before the chunk's last nonempty one hold 32 columns each
        const int64_t g = i / (kCols * rv), j = i - g * kCols * rv;
        const int64_t k = j / rv, rl = j % rv;
        const int64_t r = tl.a + rl, col = (int64_t)(tl.chunk0 + c) * G * kCols + g * kCols + k;
        const int64_t cend = r < nc ? min(nc, r + 1) : nc;
        out[i] = col < cend ? P[r + col * nr] : 0.0f;
      }
    } else {
      const int BC = tl.kind == kB64 ? 64 : (tl.kind == kB32 ? 32 : (tl.kind == kB16 ? 16 : 8));
      const int BR = bwd_chunk_rows(BC);
      const int64_t rn = last ? tl.lld : BR;
      const int64_t bcv = min((int64_t)BC, nc - tl.a);
      total = bcv * rn;
      for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int64_t rr = i % rn, cc = i / rn;
        const int64_t row = tl.a + (int64_t)(tl.chunk0 + c) * BR + rr, j = tl.a + cc;
        out[i] = (row >= nc || row >= j) ? P[row + j * nr] : 0.0f;
      }
    }
    const int64_t padded = last ? tl.lbytes / 4 : tl.cbytes / 4;
    for (int64_t i = total + threadIdx.x; i < padded; i += blockDim.x) out[i] = 0.0f;
  }
}

// CTAs per SM of the FP32 (pipelined) kernel.  Both precisions launch this many
// CTAs per SM, so every solve consumes the same number of tickets; the FP64
// kernel has fewer resident at a time, which the ticket order tolerates (a CTA
// draws tickets only once it runs).
int solve_persistent_occupancy() {
  // the FP32 kernel's stages; set on the current device (meshes and servers call
  // this on their device before any solve)
  cudaFuncSetAttribute(solve_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStages * kStageBytes);
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_pipe_kernel, kPipeThreads, kStages * kStageBytes);
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
  p.wdest = m->wdest;
  p.slot_w = m->slot_w;
  p.b = b;
  p.u = m->ws.solve_u;
  p.W = precision == PD_PREC_MIXED ? (void*)m->W32 : (void*)m->W64;
  p.x = out;
  const bool f32 = precision == PD_PREC_MIXED;
  p.Q = f32 ? (const void*)m->Q32 : (const void*)m->Q64;
  p.Qs = f32 ? m->Qs : nullptr;
  if (f32 && !m->Qs) return cudaErrorInvalidValue;
  const int64_t ntiles = (int64_t)m->sched.all.size();
  if (ntiles == 0) return cudaSuccess;
  p.tiles = m->all_tiles;
  p.ntiles = ntiles;
  p.gticket = m->solve_counters;
  p.fdone = m->solve_counters + 1;
  p.bdone = m->solve_counters + 1 + m->h.ns;
  p.otick = m->solve_counters + 1 + 2 * m->h.ns;
  p.partial = m->ws.solve_partial;
  p.nfb = m->nfb;
  p.nbb = m->nbb;
  p.child_ptr = m->child_ptr;
  p.child_list = m->child_list;
  p.err = m->ws.flags;
  p.spin_limit = m->solve_spin_limit;
  p.stall_tile = -1;
  if (m->test_stall_solves > 0 && m->stall_tile >= 0) {
    p.stall_tile = m->stall_tile;
    --m->test_stall_solves;
  }
  const unsigned grid = (unsigned)std::min<int64_t>(m->solve_grid, ntiles);
  if (f32) solve_pipe_kernel<<<grid, kPipeThreads, kStages * kStageBytes, st>>>(p);
  else solve_persistent_kernel<<<grid, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace pd
