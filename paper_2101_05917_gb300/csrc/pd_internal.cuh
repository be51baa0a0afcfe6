// Internal declarations shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "diffpd.h"
#include "pd_host.h"
#include "pd_iter.cuh"

namespace pd {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);

// Mesh handles (abi.cu) as seen by the server: cap the persistent solve's CTAs
// (takes effect from the next pd_forward / pd_backward / pd_solve_A call) and the
// device bytes the mesh holds.
void limit_solve_ctas(pd_mesh m, int ctas);
int solve_ctas(pd_mesh m);
size_t mesh_device_bytes(pd_mesh m);
#define PD_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) {                                                     \
      ::pd::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
      return PD_ERR_CUDA;                                                        \
    }                                                                            \
  } while (0)

// Local-step precision beside PD_PREC_FP64 / PD_PREC_MIXED (internal): the FP32
// local step with the displacement gradient H = F - I and the Green strain formed
// in FP64, so its stresses stay accurate relative to the strain under large
// rotations (hexahedra; the tetrahedral rule runs the plain FP32 step).
constexpr int kPrecMixedAcc = PD_PREC_MIXED_STRAIN;
// FP64-accurate local step from an FP32 SVD refined in FP64 (hexahedra, corotated +
// muscle energies; otherwise the plain FP64 step runs)
constexpr int kPrecRefined = PD_PREC_FP64_REFINED;
inline bool local_is_fp32(int precision) { return precision == PD_PREC_MIXED || precision == kPrecMixedAcc; }

// Device status bits raised by kernels (integer atomicOr; never on data).
enum : int {
  DEV_ERR_NOT_SPD = 1,
  DEV_ERR_INVERTED = 2,
  DEV_ERR_NAN = 4,
  DEV_ERR_TIMEOUT = 8,   // a bounded device-side wait gave up
  DEV_ERR_LAYOUT = 16,   // an internal descriptor failed its size / alignment check
};

// ---------------------------------------------------------------- buffers
template <typename T>
struct DArr {
  T* p = nullptr;
  size_t n = 0;
};

// Solve schedule: per level, ranges of tiles.  An output block is one row block
// of a supernode's panel over all the columns it needs (forward) or one column
// block over all its rows (backward); its panel values are streamed in chunks
// (a chunk is what one shared-memory stage holds: at most 256 x 48 entries), and
// a tile is a run of at most a level-dependent number of consecutive chunks of
// one block.  A block split into several tiles adds their partial sums in tile
// order (its last tile to finish does, after an integer ticket).
struct SolveLevel {
  int64_t fwd_off = 0, fwd_cnt = 0;
  int64_t bwd_off = 0, bwd_cnt = 0;
};
// Everything one tile needs, loaded with eight 16-byte loads.
constexpr int kTileDeps = 6;   // dependencies carried inside a tile descriptor
struct alignas(16) SolveTile {
  int64_t panel_off;   // offset of the supernode's panel (column-major nr x nc)
  int64_t soff;        // FP32 streamed copy: offset (floats, 16-byte aligned) of the tile's first chunk
  int32_t s;           // supernode
  int32_t kind;        // forward 0/1/2: 256/128/64 rows; backward 3/4/5/6: 64/32/16/8 columns
  int32_t a;           // forward: first row of the row block; backward: first column of the block
  int32_t first, nc, nr;   // first column, columns, rows of the supernode
  int32_t pos;         // row_ptr[s]: start of its row structure / positions
  int32_t relp;        // rel_ptr[s]: start of its update-vector rows
  int32_t ndep;        // dependencies: forward = children, backward = parent (root: itself)
  int32_t nchunks;     // chunks of this tile (forward: column ranges, backward: row ranges)
  int32_t cbytes;      // FP32 stream: bytes of every chunk but the tile's last
  int32_t lbytes;      // FP32 stream: bytes of the tile's last chunk (a multiple of 16)
  int32_t lld;         // the tile's last chunk's leading dimension: forward columns per group, backward rows
  int32_t chunk0;      // index of the tile's first chunk within its block
  // the first kTileDeps dependencies inline: counter index (supernode id; backward
  // dependencies on a forward counter are stored as -(id + 1)) and the number of
  // output blocks that counter reaches per solve; more are read from the tree arrays
  int32_t dep[kTileDeps];
  int32_t dep_blocks[kTileDeps];
  int32_t ntile;       // tiles of its block
  int32_t tib;         // index of this tile within its block (the block's tiles are consecutive)
};
static_assert(sizeof(SolveTile) == 128, "tile descriptors are 128 bytes");
struct SolveSchedule {
  std::vector<SolveTile> fwd, bwd;
  std::vector<SolveTile> all;      // persistent order: forward tiles, then backward tiles by descending level
  int64_t stream_elems = 0;        // floats of the streamed FP32 chunks (both sweeps)
  int64_t chunks = 0;              // chunks of one solve (both sweeps)
  std::vector<int32_t> nfb, nbb;   // per supernode: forward row blocks / backward column blocks
  std::vector<SolveLevel> levels;
};

// Factorisation schedule for one level.
struct FactorLevel {
  int64_t list_off = 0, count = 0;    // supernode ids in level_list (device copy)
  int64_t max_nc = 0, max_nr = 0, max_child_nb2 = 0, max_children = 0;
};


struct Workspace {
  // per-node / per-DoF vectors (FP64, internal order)
  double *x = nullptr, *xt = nullptr, *y = nullptr, *xprev = nullptr, *vprev = nullptr;
  double *grad = nullptr, *gradt = nullptr, *dir = nullptr, *q = nullptr, *r = nullptr;
  double *S = nullptr, *Y = nullptr;          // L-BFGS history (m x 3nf each)
  double *z = nullptr, *gs = nullptr, *Hd = nullptr;   // backward
  double *ax = nullptr, *av = nullptr, *gbar = nullptr, *fext = nullptr, *ffric = nullptr;
  double *iox = nullptr, *iov = nullptr;      // kept-order staging
  void* elembuf = nullptr;                    // (8e x 3) T
  double* partials = nullptr;                 // block partial sums
  double* lpart = nullptr;                    // L-BFGS inner products, per block
  unsigned int* counters = nullptr;           // last-block counters
  IterState* st = nullptr;                    // device iteration state
  IterState* st_host = nullptr;               // pinned mirror
  int* flags = nullptr;                       // device status bits
  void* solve_u = nullptr;                    // (3 nf) T
  void* solve_partial = nullptr;              // per tile partial sums of split blocks
  double* act_cur = nullptr;                  // (e) actuation of the current step
  double* xnext_cur = nullptr;                // (3n) x_{t+1} of the current adjoint step
  int lbfgs_m = 0;
  size_t bytes = 0;
};

struct MeshImpl {
  HostMesh h;
  int device = -1;
  // geometry / topology (device)
  int32_t *elems = nullptr, *inc_ptr = nullptr, *inc = nullptr, *kept_of_internal = nullptr;
  double *X = nullptr, *mass = nullptr;
  uint8_t* contact = nullptr;
  // solve structure (device)
  int64_t *snode_first = nullptr, *row_ptr = nullptr, *panel_off = nullptr, *rel_ptr = nullptr;
  int64_t *gath_ptr = nullptr, *front_off = nullptr, *level_list = nullptr, *child_ptr = nullptr,
          *child_list = nullptr;
  int32_t *rows = nullptr, *gath = nullptr, *rel = nullptr;
  SolveTile* all_tiles = nullptr;
  int32_t *nfb = nullptr, *nbb = nullptr;
  int64_t* parent = nullptr;
  unsigned long long* solve_counters = nullptr;   // gticket | fdone[ns] | bdone[ns] | otick[tiles]
  int solve_grid = 0;
  // polls of a solve dependency wait before it gives up (~1 s by default); the
  // environment variable PD_SOLVE_SPIN_LIMIT, read at mesh creation, lowers it
  long long solve_spin_limit = 1ll << 20;
  // test support (PD_TEST_SOLVE_STALLS at mesh creation): the next solves raise one
  // forward dependency target by one, so that wait runs out and reports
  // DEV_ERR_TIMEOUT; each such solve decrements the count
  mutable int test_stall_solves = 0;
  int64_t stall_tile = -1;         // the forward tile whose wait is raised
  int sms = 1;                     // SMs of the device
  // forward-solve update vectors in the parent's layout: child update row i (of
  // rel_ptr.back()) goes to slot wdest[i] = position x slot_w + rank of the
  // parent's positions (ranks in child order); unused slots stay zero
  int32_t* wdest = nullptr;
  int slot_w = 1;
  float* W32 = nullptr;            // (positions x slot_w x 3), zero-initialised
  double* W64 = nullptr;
  SolveSchedule sched;
  std::vector<FactorLevel> flevels;
  // assembly map (device)
  int64_t *la_target = nullptr, *la_cptr = nullptr;
  int32_t *la_diag_node = nullptr, *la_contrib = nullptr;
  // unstructured tetrahedra (PD_ELEM_TETU): barycentric gradients (12 per element,
  // vertex-major) and volumes, in FP64 and FP32
  double *tet_grad = nullptr, *tet_vol = nullptr;
  float *tet_grad_f = nullptr, *tet_vol_f = nullptr;
  // iteration chunks replayed as CUDA graphs: [forward/backward][precision index],
  // captured on cap_stream with the per-step inputs read from ws.act_cur /
  // ws.xnext_cur; dropped whenever a captured argument could change
  cudaStream_t cap_stream = nullptr;
  // [direction][precision][variant]: variant 1 holds one iteration fewer (profiled
  // chunks launch their first iteration directly, with timing events)
  // [direction][local-step precision: FP64, MIXED, kPrecMixedAcc, kPrecRefined][variant]
  cudaGraphExec_t iter_graph[2][4][2] = {};
  bool iter_graph_act[2][4][2] = {};
  int64_t iter_graph_counts[2][4][2][3] = {};   // kernels, solves, local steps per replay
  // complementarity contact (contact.cu): A^-1 columns of the candidate nodes and
  // the current contact set
  int64_t factor_gen = 0;              // bumped by every factorisation
  int64_t contact_gen = -1;            // factor_gen the candidate columns belong to
  int64_t ncand = 0;
  int32_t* cand = nullptr;             // (ncand) internal free-node ids
  std::vector<int32_t> cand_host;      // the same on the host
  std::vector<int32_t> cand_of_internal;   // host: internal id -> candidate index, -1
  double* Bc = nullptr;                // (nf x ncand) column-major: L_A^-1 e_j
  int64_t cset = 0, cset_cap = 0;      // contact set size / buffer capacity
  int32_t *cset_node = nullptr, *cset_cand = nullptr;   // (cset) internal id, candidate index
  double* cset_S = nullptr;            // (cset x cset) S = (L_A^-1)_{CC}, factored in place; then Q^T
  double* cset_Q = nullptr;            // (cset x cset) Q = L^-1 of S = L L^T (column-major, lower)
  double* cset_a = nullptr;            // (cset x 3) scratch: (a1)_C
  double* cset_u = nullptr;            // (cset x 3) scratch: Q (a1)_C
  int64_t* cset_meta = nullptr;        // (4) one-supernode tree of S for the dense factorisation
  int* cset_flags = nullptr;           // SPD / finite flags of that factorisation
  double* cset_lam = nullptr;          // (cset x 3) multipliers of the current solve
  double* cset_zero = nullptr;         // (cset x 3) zeros: targets of the iteration's directions
  double* cset_xstar = nullptr;        // (cset x 3) targets of the current set
  uint8_t* cset_rule = nullptr;        // (cset) 1 = ray target, 0 = drop target (backward)
  double* cset_gx = nullptr;           // (cset x 3) adjoint of the targets into x_t (backward)
  double* cset_gv = nullptr;           // (cset x 3) adjoint of the targets into v_t (backward)
  double* cand_buf = nullptr;          // (ncand x 3) scratch for candidate rows
  uint8_t* held = nullptr;             // (nf) 1 = node held at its contact target
  bool held_active = false;            // gathers mask held rows (complementarity steps)
  // per time step of the last complementarity rollout: contact set (internal ids),
  // target rule (1 = ray, 0 = drop) -- read by the backward pass
  std::vector<std::vector<int32_t>> contact_log_node;
  std::vector<std::vector<uint8_t>> contact_log_rule;
  // per time step of the last pd_forward: the strain-accurate tier's remaining steps
  // and the length of the first chunk of iterations at the start of the step, so that
  // a checkpointed recomputation polls at the same iterations and takes the same
  // local-step precision at every step as the forward pass did
  std::vector<int32_t> acc_log, guess_log;
  // material state
  bool factorized = false;
  int precision = PD_PREC_FP64;
  bool neohookean = false;   // Neo-Hookean material (mu = wc/2, lambda = wv) in the local steps
  // point SVDs (and volume projections) shared by the FP32 Hessian products of one
  // adjoint solve (svd_cache_layout); allocated by pd_backward when it applies
  float* svd_cache = nullptr;
  int64_t svd_cache_fields = 0;
  // the refined FP64 rotation and stretch of every point (18 doubles), shared by the
  // refined FP64 residual checks of one adjoint step (ref_cache_applies)
  double* ref_cache = nullptr;
  double h_step = 0, grav[3] = {0, 0, 0}, k_contact = 0;
  double *wc = nullptr, *wv = nullptr, *wm = nullptr, *fiber = nullptr;   // null = energy absent
  double *wc_buf = nullptr, *wv_buf = nullptr, *wm_buf = nullptr, *fiber_buf = nullptr;
  // factor panels Q_s = [L11^-1 ; L21 L11^-1] (column-major nr x nc)
  double* Q64 = nullptr;
  float* Q32 = nullptr;
  // the FP32 panels again, cut into the solve's tiles and stored tile after tile in
  // the order each tile body reads them (SolveTile::soff), for one bulk copy per tile
  float* Qs = nullptr;
  Workspace ws;
  std::vector<std::pair<void*, size_t>> allocations;   // device buffers and their bytes
};

// ------------------------------------------------------------------ launchers
// Local steps (kernels_local.cu).  Vectors are internal-order node-major.
struct LocalArgs {
  const MeshImpl* m;
  const IterState* gate;   // skip the launch's work once gate->converged is set (may be null)
  const double* x;       // (n,3) positions
  const double* v;       // (n,3) direction for HVP / adjoint for param grads
  const double* act;     // (e) contraction or null
  int precision;         // PD_PREC_FP64 / PD_PREC_MIXED (float local step)
  int ref_cache = 0;     // refined FP64 Hessian products: 1 write m->ref_cache, 2 read it
};
// forces into ws.elembuf; energy block partials into partials[0..nblk)
cudaError_t launch_element_forces(const LocalArgs& a, void* elembuf, double* energy_partials,
                                  int* flags, cudaStream_t s);
cudaError_t launch_element_hvp(const LocalArgs& a, void* elembuf, int* flags, cudaStream_t s);
// floats per field of the Hessian-product SVD cache (the element kernel's grid
// threads) and the fields the mesh needs; 0 fields when the cache does not apply
// (not FP32 hexahedra, the Neo-Hookean or the muscle energy)
void svd_cache_layout(const MeshImpl* m, int64_t* slots, int64_t* fields);
// whether the refined FP64 Hessian products of the mesh can share m->ref_cache
// (mixed-precision hexahedra of the corotated energy alone), and its doubles
bool ref_cache_applies(const MeshImpl* m, int64_t* doubles);
cudaError_t launch_element_param_grads(const LocalArgs& a, double* g_wc, double* g_wv,
                                       double* g_wm, double* g_act, cudaStream_t s);
// blocks of the element kernels: 8 threads per element record (voxel rules) or one
// thread per element (unstructured tetrahedra); each force launch writes one
// energy partial per block
int element_blocks(const MeshImpl* m);
int element_energy_partials(const MeshImpl* m);

// Gathers (K2): out[c] = sum over incidence of elembuf + node terms, for c < nf
// (gradient mode: + m (x - y)/h^2 + contact force; hvp mode: + m v/h^2 + contact).
cudaError_t launch_gather_grad(const MeshImpl* m, const IterState* gate, const void* elembuf,
                               int precision, const double* x, const double* y, const double* dir,
                               double* grad, double* partials, cudaStream_t s);
cudaError_t launch_gather_hvp(const MeshImpl* m, const IterState* gate, const void* elembuf,
                              int precision, const double* x, const double* v, const double* gs,
                              double* Hv, double* partials, cudaStream_t s);
int gather_blocks(const MeshImpl* m);
// Threads per block of the element kernels (8 lanes per cell): the raw force
// launch writes one energy partial per block, raw_element_blocks(ne) of them.
constexpr int kElemBlockThreads = 256;
constexpr int64_t raw_element_blocks(int64_t ne) { return (ne * 8 + kElemBlockThreads - 1) / kElemBlockThreads; }
cudaError_t launch_element_forces_raw(int64_t ne, const int32_t* elems, const double* x, const double* act,
                                      const double* wc, const double* wv, const double* wm, const double* fiber,
                                      double dx, int precision, void* elembuf, double* energy_partials,
                                      int* flags, cudaStream_t s);

// Factorisation (kernels_factor.cu)
pd_status factorize_device(MeshImpl* m, cudaStream_t s);

// Triangular solves (kernels_solve.cu): out = A^-1 b on the free DoFs
// (internal order, 3 nf entries each).
// gate: skipped when gate->converged or !gate->accepted (may be null).
// Complementarity contact (kernels_contact.cu); vectors in internal node order.
cudaError_t contact_unit_rhs(int64_t nf, const int32_t* cand, int64_t k0, int count, double* b, cudaStream_t s);
cudaError_t contact_extract_columns(int64_t nf, const double* x, int64_t k0, int count, double* Bc,
                                    cudaStream_t s);
cudaError_t contact_gather_S(int64_t nf, const double* Bc, const int32_t* node, const int32_t* cidx, int64_t c,
                             double* S, cudaStream_t s);
cudaError_t contact_correct(int64_t nf, const double* Bc, const int32_t* node, const int32_t* cidx, int64_t c,
                            const double* Q, const double* QT, double* abuf, double* ubuf, double* lam,
                            const double* a1, const double* xstar, double* x, cudaStream_t s);
// Q = L^-1 and QT = Q^T for S = L L^T (c x c, factored in place; QT may alias S);
// meta: 4 device int64; flags gets DEV_ERR_NOT_SPD / DEV_ERR_NAN
pd_status dense_cholesky_inverse(double* S, int64_t c, double* Q, double* QT, int64_t* meta, int* flags,
                                 cudaStream_t st);

cudaError_t contact_pack_rows(const int32_t* rows, int64_t c, const double* a, double* out, cudaStream_t s);
cudaError_t contact_set_targets(const int32_t* node, int64_t c, const double* xstar, double* x, cudaStream_t s);
cudaError_t contact_target_vjp(const int32_t* node, const uint8_t* ray, int64_t c, const double* xt,
                               const double* vt, const double* ax, const double* av, const double* Hz, double inv_h,
                               double* gx, double* gv, cudaStream_t s);
cudaError_t contact_add_rows(const int32_t* node, int64_t c, const double* gx, const double* gv, double* ax,
                             double* av, cudaStream_t s);

cudaError_t solve_A(const MeshImpl* m, const IterState* gate, const double* b, double* out,
                    int precision, cudaStream_t s);
void build_solve_schedule(const HostMesh& h, SolveSchedule& S);
size_t solve_partial_bytes(const SolveSchedule& S);
int solve_persistent_occupancy();
// fills m->Qs from m->Q32 (after every mixed-precision factorisation)
cudaError_t pack_solve_stream(const MeshImpl* m, cudaStream_t s);

}  // namespace pd
