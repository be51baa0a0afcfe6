/*
 * diffpd.h -- C ABI of a GB300-native differentiable Projective Dynamics solver.
 *
 * The library simulates voxel meshes (hexahedra, or six tetrahedra per cell)
 * and unstructured tetrahedral meshes with implicit Euler solved by
 * Projective Dynamics (Sec. 3, Alg. 1 of "DiffPD: Differentiable Projective
 * Dynamics", arXiv 2101.05917) and back-propagates through the rollout with the
 * adjoint splitting iteration  A z_{k+1} = Delta A z_k + dL/dx  (Sec. 4, Eqn 23,
 * Alg. 2), both accelerated by L-BFGS with the constant matrix A as initial
 * Hessian (Sec. 4, "Further acceleration with quasi-Newton methods").
 *
 * Conventions shared by every entry point
 *   - Pointers named *_host are host memory; every other array pointer is CUDA
 *     device memory on the mesh's device, owned by the caller.  The library never
 *     frees caller memory and never keeps a caller pointer past the call.
 *   - Per-node arrays are node-major (n, 3) FP64 in kept-node order: the nodes
 *     touched by at least one kept cell, in increasing grid id, where grid node
 *     (i, j, k) has id (i*(ny+1)+j)*(nz+1)+k and i runs along x.  On an
 *     unstructured tetrahedral mesh (pd_create_tet_mesh) the kept nodes are the
 *     caller's nodes in the caller's order.
 *   - Per-element arrays follow kept-cell order (increasing cell id
 *     (ci*ny+cj)*nz+ck), or the caller's tetrahedron order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are stream-ordered; entry points that return statistics synchronise
 *     the stream before returning.
 *   - Errors: every call returns a pd_status; pd_last_error() gives a
 *     thread-local message for the last failing call.  Non-convergence returns
 *     PD_ERR_NOT_CONVERGED with valid (partially converged) outputs and filled
 *     statistics.
 *   - Determinism: no floating-point atomics are used on any data path; every
 *     reduction runs in a fixed order, so identical inputs give bit-identical
 *     outputs on the same GPU.
 */
#ifndef DIFFPD_H
#define DIFFPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PD_OK = 0,
  PD_ERR_INVALID_ARG = 1,   /* bad size, NULL where required, wrong state */
  PD_ERR_OOM = 2,           /* device allocation failed / admission refused */
  PD_ERR_NOT_SPD = 3,       /* non-positive pivot while factoring A */
  PD_ERR_NOT_CONVERGED = 4, /* iteration cap reached before the tolerance */
  PD_ERR_INVERTED = 5,      /* an element with det F <= 0 was seen */
  PD_ERR_NAN = 6,           /* non-finite value in a residual */
  PD_ERR_TIMEOUT = 7,       /* serving: result not ready yet; solves: a bounded
                               device-side wait (about 1 s) gave up */
  PD_ERR_CUDA = 8,          /* CUDA runtime error */
  PD_ERR_NO_DEVICE = 9,     /* mesh created without a device */
  PD_ERR_INTERNAL = 10      /* an internal descriptor failed a device-side check
                               (a library defect, not an input error) */
} pd_status;

enum {
  PD_PREC_FP64 = 0,
  PD_PREC_MIXED = 1,
  /* pd_local_step / pd_hessian_vector only: the FP32 local step with the
     displacement gradient F - I and the Green strain F^T F - I formed in FP64, so
     that the stresses stay accurate relative to the strain under large rotations
     (hexahedra; the tetrahedral rules run the plain FP32 step).  The mixed-precision
     rollouts switch to it when the plain FP32 residual stops decreasing. */
  PD_PREC_MIXED_STRAIN = 2,
  /* pd_local_step / pd_hessian_vector only: FP64-accurate results from an FP32 SVD
     of the FP64 strain whose rotation (and its derivative) is refined in FP64
     without eigenvectors; hexahedra with the corotated and muscle energies (a mesh
     with the volume energy, or a tetrahedral rule, runs the plain FP64 step).
     The mixed-precision rollouts use it for their FP64 convergence checks. */
  PD_PREC_FP64_REFINED = 3
};

typedef struct pd_mesh_s* pd_mesh;

/* Element rules: the first two on the kept cells of the voxel grid. */
enum {
  PD_ELEM_HEX8 = 0,  /* trilinear hexahedron, 2x2x2 Gauss points of weight dx^3/8 each;
                        lumped mass rho dx^3/8 per cell corner */
  PD_ELEM_TET6 = 1,  /* six linear tetrahedra per cell, one for each order of the axes
                        along the path from corner (0,0,0) to corner (1,1,1) (conforming
                        between cells), one point of weight dx^3/6 each; lumped mass
                        rho V/4 per tetrahedron vertex.  Stands in for the tetrahedral
                        meshes of Secs. 5.1 and 7; per-element inputs (weights, fibres,
                        actuation, their gradients) stay per cell and are shared by its
                        six tetrahedra */
  PD_ELEM_TETU = 2   /* unstructured linear tetrahedra (pd_create_tet_mesh): one point of
                        weight V per tetrahedron, lumped mass rho V/4 per vertex */
};

/* Voxel mesh description.  All pointers are host memory, read during the call. */
typedef struct {
  int32_t nx, ny, nz;           /* cells along x, y, z */
  double dx;                    /* cell edge [m] */
  double origin[3];             /* position of grid node (0,0,0) [m] */
  double density;               /* [kg/m^3]; lumped mass rho dx^3/8 per cell corner */
  const uint8_t* cell_mask;     /* nx*ny*nz in cell-id order (nonzero = kept), NULL = full box */
  const uint8_t* dirichlet;     /* per kept node: fixed at its rest position, NULL = none */
  const uint8_t* contact;       /* per kept node: ground-penalty candidate, NULL = none */
  int32_t leaf_max;             /* nested-dissection leaf size, 0 = 64 */
  int32_t device;               /* CUDA device ordinal, -1 = host analysis only */
  int32_t element_rule;         /* PD_ELEM_HEX8 (0) or PD_ELEM_TET6 */
} pd_mesh_desc;

typedef struct {
  int64_t n_nodes, n_elems, n_free;
  int64_t n_snodes, n_levels;
  int64_t factor_nnz;           /* entries of all supernode panels (rows x cols) */
  int64_t max_rows, max_cols;   /* largest supernode panel */
  int64_t front_entries;        /* sum of rows^2 over supernodes (factor workspace) */
  int64_t update_entries;       /* forward-solve update vector entries */
  int32_t factorized;           /* pd_factorize succeeded */
  int32_t precision;            /* precision of the last factorisation */
} pd_mesh_info;

/* Builds the mesh, its node/element incidence, the nested-dissection ordering
 * and the supernodal structure of A on the host (C++), and uploads them to
 * `device`.  Ownership of *out passes to the caller (pd_mesh_destroy). */
pd_status pd_create_mesh(const pd_mesh_desc* desc, pd_mesh* out);

/* Unstructured tetrahedral mesh (the tetrahedral meshes of Secs. 5.1 and 7, with
 * their own node sets).  All pointers are host memory, read during the call. */
typedef struct {
  int64_t n_nodes, n_tets;      /* every node must be a vertex of a tetrahedron;
                                   n_tets < 2^25 (32-bit assembly codes) */
  const double* X;              /* (n_nodes, 3) rest positions [m] */
  const int32_t* tets;          /* (n_tets, 4) vertex indices, either orientation;
                                   four distinct nodes, |det(edge matrix)| above
                                   1e-12 x (longest edge from vertex 0)^3 */
  double density;               /* [kg/m^3]; lumped mass rho V/4 per vertex */
  const uint8_t* dirichlet;     /* per node: fixed at its rest position, NULL = none */
  const uint8_t* contact;       /* per node: ground-penalty candidate, NULL = none */
  int32_t leaf_max;             /* nested-dissection leaf size, 0 = 64 */
  int32_t device;               /* CUDA device ordinal, -1 = host analysis only */
} pd_tet_mesh_desc;

/* Builds an unstructured tetrahedral mesh (element rule PD_ELEM_TETU): per
 * tetrahedron the gradients of its barycentric coordinates (rows of the inverse
 * of its edge matrix) and its volume, the node incidence, a nested-dissection
 * ordering of the free nodes by coordinate bisection with vertex separators of
 * the mesh graph (a set of more than leaf_max free nodes is sorted by its
 * coordinate of largest extent -- ties x, y, z -- then by node index, and halved;
 * the separator is the first half's nodes adjacent to the second half; the order
 * is first half without the separator, second half, separator), and the
 * supernodal structure of A as pd_create_mesh builds it for voxel meshes.  The
 * mesh then serves every entry point that takes a pd_mesh, with per-element
 * arrays per tetrahedron, except the muscle energy and the Neo-Hookean material
 * (pd_factorize rejects them on this rule).  PD_EXPORT_INC entries are
 * e*8 + vertex (vertex < 4): element records keep the stride of eight.
 * Errors: PD_ERR_INVALID_ARG for a vertex out of range or repeated, a degenerate
 * tetrahedron, a node in no tetrahedron or no free node; PD_ERR_OOM / PD_ERR_CUDA
 * as pd_create_mesh.  Ownership of *out passes to the caller (pd_mesh_destroy). */
pd_status pd_create_tet_mesh(const pd_tet_mesh_desc* desc, pd_mesh* out);
void pd_mesh_destroy(pd_mesh m);
pd_status pd_mesh_query(pd_mesh m, pd_mesh_info* info);

/* Copies one host-side index structure into host_out (capacity in elements).
 * Integer structures are int64.  Used to check the native index construction
 * bit for bit against an independent re-derivation. */
enum {
  PD_EXPORT_INC_PTR = 0,   /* (n+1): kept-node -> (element, corner) CSR pointers */
  PD_EXPORT_INC = 1,       /* (8e; 4e on an unstructured tetrahedral mesh): entries
                              e*8+corner, ascending per node */
  PD_EXPORT_PERM = 2,      /* (n_free): column -> free-node index (free nodes in kept order) */
  PD_EXPORT_SNODE_FIRST = 3, /* (n_snodes+1): first column of each supernode */
  PD_EXPORT_ROW_PTR = 4,   /* (n_snodes+1) */
  PD_EXPORT_ROWS = 5,      /* row structure of every supernode, ascending */
  PD_EXPORT_PARENT = 6,    /* (n_snodes): supernodal etree parent or -1 */
  PD_EXPORT_LEVEL = 7,     /* (n_snodes) */
  PD_EXPORT_REL = 8,       /* positions of each supernode's below rows in its parent */
  PD_EXPORT_LEVEL_PTR = 9, /* (n_levels+1) into PD_EXPORT_LEVEL_LIST */
  PD_EXPORT_LEVEL_LIST = 10, /* (n_snodes) supernodes grouped by level, ascending ids */
  PD_EXPORT_SOLVE_TILES = 11 /* 10 per triangular-solve tile, in the persistent solve's order
                                (forward tiles by ascending level, then backward tiles by
                                descending level): supernode, kind (0-2 forward row blocks of
                                256/128/64 rows, 3-6 backward column blocks of 64/32/16/8
                                columns), first row (forward) or column (backward) of its
                                block, index of its first chunk within the block, its chunks
                                (forward: column ranges of 32 columns per row group; backward:
                                row ranges of min(8192 / columns, 256) rows), offset of its
                                first chunk in the FP32 streamed copy (floats), bytes of each
                                chunk but its last, bytes of its last chunk, the last chunk's
                                columns (forward; they fill the row groups in order) or rows
                                (backward), and the tiles of its block */
};
pd_status pd_mesh_export(pd_mesh m, int32_t what, int64_t* host_out, int64_t capacity,
                         int64_t* count);

/* Material state and the one-time factorisation of
 *   A = M/h^2 + sum_c w_c G_c^T G_c   (Sec. 3, Eqn 19).
 * w_corot, w_vol, w_muscle: (e) stiffness per unit volume [Pa] of the corotated,
 * volume-preserving and muscle-fibre energies (NULL = energy absent); each
 * Gauss point of a cell carries w * dx^3/8 (w * dx^3/6 per tetrahedron of the
 * six-way split, w * V per unstructured tetrahedron).  fiber: (e, 3) unit fibre
 * directions (required when w_muscle is given).  The numeric supernodal Cholesky runs on
 * the device in FP64; with PD_PREC_MIXED an FP32 copy of the solve panels is kept
 * for the triangular solves.  Copies of the weights are kept for the local
 * steps.  Returns PD_ERR_NOT_SPD on a non-positive pivot; PD_ERR_INVALID_ARG for
 * the Neo-Hookean option without both w_corot and w_vol or on a tetrahedral mesh,
 * and for w_muscle on an unstructured tetrahedral mesh. */
typedef struct {
  double h;                     /* time step [s] */
  double gravity[3];            /* [m/s^2] */
  double k_contact;             /* ground penalty stiffness [N/m] on contact candidates */
  int32_t precision;            /* PD_PREC_FP64 or PD_PREC_MIXED */
  int32_t neohookean;           /* nonzero: Neo-Hookean material (Sec. 8, hexahedra only): the
                                   local steps evaluate psi = mu/2 (tr F^T F - 3) - mu log J +
                                   lambda/2 (log J)^2 with mu = w_corot / 2 and lambda = w_vol
                                   (both required) instead of the corotated and volume energies;
                                   A is still assembled from w_corot and w_vol (the PD matrix
                                   of the same material, the L-BFGS initial Hessian) */
} pd_factor_opts;

pd_status pd_factorize(pd_mesh m, const double* w_corot, const double* w_vol,
                       const double* w_muscle, const double* fiber,
                       const pd_factor_opts* opts, void* stream);

typedef struct {
  double tol_fwd;               /* |grad g| <= tol_fwd * max(|grad g(y)|, |M y/h^2|) */
  double tol_bwd;               /* |Hess g z - gbar| <= tol_bwd * |gbar| */
  int32_t max_iter_fwd, max_iter_bwd;
  int32_t lbfgs_m;              /* history length (0 = plain PD / plain splitting iteration) */
  int32_t ls_max;               /* Armijo backtracking tries (Sec. 6 uses 10) */
  int32_t checkpoint_every;     /* 0 = every state stored; K > 0 = store states t % K == 0 */
  int32_t check_every;          /* iterations between host convergence polls (0 = 4); with
                                   PD_PREC_MIXED the local steps run in FP32 and the convergence
                                   test is confirmed by an FP64 residual */
  int32_t profile;              /* nonzero: time solve and local-step launches with CUDA events
                                   on the launching stream (pd_stats.*_ms, *_timed); with
                                   graphs on, the last iteration of every chunk of 4 is
                                   launched directly and timed, the others replayed */
  int32_t warm_start;           /* nonzero: keep the L-BFGS pairs from one time step to the
                                   next and start each adjoint solve from the previous
                                   step's z (fixed points unchanged) */
  int32_t no_graphs;            /* nonzero: launch every kernel directly; by default chunks of
                                   iterations are captured once per mesh as CUDA graphs and
                                   replayed */
  int32_t complementarity;      /* nonzero: complementarity contact on the ground z = 0 (Sec. 5.2,
                                   Alg. 3 forward / Alg. 5 backward) for the candidates given to
                                   pd_contact_prepare; needs k_contact = 0; CUDA graphs are not
                                   used.  Per step the contact set starts with the candidates
                                   touching the ground (target (x_t, y_t, 0), "drop") or whose
                                   ray x_t + s v_t reaches it within h (target: the
                                   intersection, "ray"); after each solve nodes whose normal
                                   contact force [M (x - y)/h^2 + grad E]_z is below
                                   -1e-8 max(m) |g| leave (once per step: a node that leaves
                                   and then sinks again stays), candidates below -1e-9 dx join
                                   (drop), until the set is stable (at most 64 solves).
                                   pd_backward uses the sets of the last pd_forward (same T);
                                   a checkpointed backward recomputes them identically. */
  double* step_ms;              /* optional host array of T entries: pd_forward stores the
                                   host wall time of each step [ms], pd_backward adds the
                                   time of the step's adjoint and, with checkpointing, of its
                                   recomputation (so after both calls entry t holds the
                                   fwd+bwd latency of step t); NULL = none */
  int32_t* step_iters;          /* optional host array of T entries: pd_forward stores the
                                   iterations of each step, pd_backward those of each step's
                                   adjoint solve (it overwrites the entries); NULL = none */
  int32_t fext_per_step;        /* nonzero: f_ext holds one external force per step, (T, n, 3)
                                   (step t's predictor uses slice t), and pd_backward's g_fext
                                   receives one gradient per step, (T, n, 3); 0: f_ext is (n, 3),
                                   the same every step, and g_fext (n, 3) is summed over steps */
} pd_solver_opts;

typedef struct {
  int64_t fwd_iters, bwd_iters;         /* total iterations over the rollout */
  int64_t fwd_fp64_iters, bwd_fp64_iters;
  int64_t fwd_line_search;              /* rejected trial steps */
  int32_t max_fwd_iters_step, max_bwd_iters_step;
  double max_fwd_rel_residual, max_bwd_rel_residual;
  int32_t inverted;                     /* det F <= 0 seen */
  int32_t not_converged_steps;
  double fwd_ms, bwd_ms;                /* host wall time of the call */
  int64_t kernel_launches;              /* kernels this call launched */
  int64_t solves;                       /* global-step solves (forward + backward sweep pairs) */
  double solve_ms;                      /* profile: summed device time of the solves */
  int64_t local_steps;                  /* forward local steps (FP32 or FP64) */
  double local_ms;                      /* profile: summed device time of the forward local steps */
  int64_t solves_timed;                 /* profile: solves timed by events (solve_ms covers these) */
  int64_t local_steps_timed;            /* profile: forward local steps timed by events (those in
                                           the factor's precision, not the FP64 checks) */
} pd_stats;

/* Forward rollout of T implicit-Euler steps (Sec. 3 Eqns 1-4, Alg. 1).
 * x0, v0: (n,3).  f_ext: external force added to gravity, or NULL: (n,3) the
 * same every step, or (T, n, 3) one per step with opts->fext_per_step (y of step t
 * = x_t + h v_t + h^2 M^-1 (f_ext[t] + M g), Eqn 1).  act: (T, e) muscle
 * contraction per step, or NULL.  mu: friction
 * coefficient of the ground penalty contact (Sec. 5.1).
 * x_traj, v_traj: ((S, n, 3)) with S = T+1, or with checkpointing
 * S = T/K + 1 (T must be a multiple of K) holding states 0, K, 2K, ...
 * Status: PD_OK; PD_ERR_NOT_CONVERGED when a step reached the iteration cap
 * (outputs and statistics are still written); PD_ERR_NAN when a residual of any
 * step was non-finite (that step stops, later steps restart from the last finite
 * iterate: the outputs are not a trajectory); PD_ERR_TIMEOUT when a bounded
 * device-side wait gave up; PD_ERR_INVALID_ARG before pd_factorize succeeded.
 * An element with det F <= 0 sets stats->inverted. */
pd_status pd_forward(pd_mesh m, const double* x0, const double* v0, const double* f_ext,
                     const double* act, double mu, int32_t T, const pd_solver_opts* opts,
                     double* x_traj, double* v_traj, pd_stats* stats, void* stream);

/* Checkpoint interval for a rollout of T steps (Sec. 4 back-propagates through
 * every step; states that do not fit are recomputed per segment).  The budget is
 * mem_cap_bytes, or (0) four fifths of the device's free memory.  *checkpoint_every
 * = 0 when all T+1 states (x and v, 48 n bytes each) fit; otherwise the smallest
 * K > 1 dividing T for which the T/K + 1 checkpointed states (the caller's x_traj,
 * v_traj) plus the K + 1 states of one recomputed segment (pd_backward's buffer)
 * fit.  PD_ERR_OOM when no K fits; PD_ERR_INVALID_ARG for a host-only mesh
 * without a cap.  Does not allocate. */
pd_status pd_plan_checkpoints(pd_mesh m, int32_t T, size_t mem_cap_bytes, int32_t* checkpoint_every);

/* Backward rollout (Sec. 4, Alg. 2 with L-BFGS; Eqns 10-12 per step).
 * x_traj, v_traj, f_ext, act, mu, T: exactly as given to / produced by pd_forward
 * (with checkpointing the missing states are recomputed segment by segment).
 * dL_dx, dL_dv: direct loss gradients of loss_states states: loss_states = 1
 * (or 0) means (n, 3) for the final state x_T / v_T only; loss_states = T+1 means
 * (T+1, n, 3), one block per state t = 0..T (with checkpointing as well: a loss
 * on the checkpointed states only puts zeros in the other blocks).  Any other
 * value returns PD_ERR_INVALID_ARG before anything is read.  dL_dv may be NULL.
 * Outputs (each may be NULL): g_x0, g_v0 (n,3); g_fext (n,3) summed over steps,
 * or (T, n, 3) per step with opts->fext_per_step (dL/df_ext[t] = z_t, the adjoint
 * of step t: y depends on f_ext through h^2 M^-1, dL/dy = M z / h^2);
 * g_w_corot, g_w_vol, g_w_muscle (e) = dL/dw per unit volume; g_act (T, e);
 * g_mu (1).  Status as pd_forward (PD_ERR_NOT_CONVERGED for an adjoint solve that
 * reached its cap, PD_ERR_NAN for a non-finite residual in any step). */
pd_status pd_backward(pd_mesh m, const double* x_traj, const double* v_traj,
                      const double* f_ext, const double* act, double mu, int32_t T,
                      const double* dL_dx, const double* dL_dv, int32_t loss_states,
                      const pd_solver_opts* opts, double* g_x0, double* g_v0,
                      double* g_fext, double* g_w_corot, double* g_w_vol,
                      double* g_w_muscle, double* g_act, double* g_mu,
                      pd_stats* stats, void* stream);

/* Kernel-level entry points (same conventions; used by tests and tools). */

/* Local step (Sec. 3): grad_E = sum_c w_c G_c^T (G_c x - p_c) (Eqn 20, (n,3),
 * Dirichlet rows included) and energy = sum_c w_c/2 |G_c x - p_c|^2 (1 scalar),
 * at positions x (n,3) with contraction act (e) or NULL. */
pd_status pd_local_step(pd_mesh m, const double* x, const double* act, int32_t precision,
                        double* grad_E, double* energy, void* stream);

/* Hessian-vector product (A - Delta A) v = Hess g(x) v (Eqn 22) on the free
 * DoFs of v (n,3); Dirichlet rows of Hv are set to zero. */
pd_status pd_hessian_vector(pd_mesh m, const double* x, const double* act, const double* v,
                            int32_t precision, double* Hv, void* stream);

/* Global step (Eqn 19): x = A^-1 b on the free DoFs (b, x: (n,3); Dirichlet
 * rows of x are set to zero) with the prefactorised supernodal factor.
 * Synchronises the stream and reads the solve's device flags: PD_ERR_TIMEOUT
 * when a bounded dependency or copy wait gave up (the results are then not
 * valid; the mesh stays usable), PD_ERR_INTERNAL for a rejected tile
 * descriptor.  The environment variable PD_SOLVE_SPIN_LIMIT (polls, read by
 * pd_create_mesh) shortens the dependency waits' bound; PD_TEST_SOLVE_STALLS=k
 * (test support, read by pd_create_mesh) makes the first k solves of the mesh
 * wait for one block more than a forward dependency delivers, so that wait
 * runs out. */
pd_status pd_solve_A(pd_mesh m, const double* b, double* x, int32_t precision, void* stream);

/* Complementarity contact (Sec. 5.2): the global step with the contact set C held
 * fixed -- the solve inside Alg. 3, which Alg. 4 evaluates with a low-rank update
 * of the prefactorised A.  Every node j in C is held at its target x*_j; the other
 * free nodes C' solve A_{C'C'} x_{C'} = b_{C'}.
 *
 * pd_contact_prepare: after pd_factorize, computes the columns L_A^-1 e_j of every
 * candidate node (candidates_host: per kept node, nonzero = candidate; fixed nodes
 * are never candidates) in FP64, three per solve; memory nf x (candidates) doubles.
 * A later pd_factorize makes them stale (PD_ERR_INVALID_ARG until prepared again). */
pd_status pd_contact_prepare(pd_mesh m, const uint8_t* candidates_host, void* stream);

/* Fixes the contact set: c distinct kept node ids (host), each a candidate; forms
 * S = (L_A^-1)_{CC} and factors it on the device, S = L L^T with Q = L^-1 (FP64,
 * c^3/3 multiply-adds for each; PD_ERR_NOT_SPD if a pivot is not positive).  Device
 * memory 2 c^2 doubles, kept for later sets.  c = 0 clears the set.  Synchronises
 * the stream. */
pd_status pd_contact_set(pd_mesh m, const int32_t* nodes_host, int64_t c, void* stream);

/* x (n,3) with x_C = x* and A_{C'C'} x_{C'} = b_{C'}: one solve of A (precision as
 * pd_solve_A) then x = a1 - B_{.,C} Q^T Q (a1)_C in FP64.  b, x: (n,3) device, kept
 * order (Dirichlet rows of x are zero); x_star: (c,3) device, in the order given to
 * pd_contact_set (NULL when c = 0). */
pd_status pd_solve_A_contact(pd_mesh m, const double* b, const double* x_star, double* x, int32_t precision,
                             void* stream);

/* The final contact set of step t (0 <= t < T) of the last pd_forward with
 * complementarity contact: *count nodes (kept ids, in the order they joined) into
 * nodes_host and their targets into rules_host (1 = ray, 0 = drop; may be NULL),
 * both host arrays of capacity cap.  PD_ERR_INVALID_ARG if there is no such step
 * or cap < *count (*count is still set). */
pd_status pd_contact_step_set(pd_mesh m, int32_t t, int32_t* nodes_host, uint8_t* rules_host, int64_t cap,
                              int64_t* count);

/* Local step that allocates no device memory (the paper has no counterpart).
 * For callers that cannot call cudaMalloc -- e.g. code under a device-memory
 * budget fixed in advance, or behind an allocator the library cannot reach --
 * this variant of pd_local_step takes every array
 * from the caller and keeps its scratch (corner forces, partial sums, a status
 * word) in one fixed-size device array owned by the library; every GPU that
 * loads the library holds that array (6.3 MB) until the process exits.
 * Computes grad_E (n_nodes, 3) and energy (1 scalar, may be NULL) exactly as
 * pd_local_step on a PD_ELEM_HEX8 mesh, on the current device and `stream`, for at most
 * PD_NOALLOC_MAX_CELLS cells and 8 x PD_NOALLOC_MAX_CELLS nodes (larger meshes
 * return PD_ERR_INVALID_ARG).  Inputs (device): elems (n_elems, 8) node ids with
 * corner a = 4 di + 2 dj + dk of a cube of edge dx; inc_ptr (n_nodes + 1) and inc
 * (8 n_elems, entries e*8+a) the node -> corner incidence (pd_mesh_export gives
 * it for a pd_mesh); x (n_nodes, 3); act (n_elems) or NULL; w_* (n_elems) per
 * unit volume as in pd_factorize; fiber (n_elems, 3) with w_muscle; contact
 * (n_nodes) uint8 or NULL with penalty k_contact.  The first call on a device
 * looks up the scratch address there: make it before any stream capture.
 * Calls share the scratch: calls that overlap on the GPU race (keep them on one
 * stream).  The scratch keeps the last call's contents; each call clears what
 * must start at zero.
 * status_flags (device, one int32, may be NULL): set in stream order, once the
 * call's kernels have run, to the OR of PD_LOCAL_FLAG_INVERTED (an element with
 * det F <= 0) and PD_LOCAL_FLAG_NAN (a non-finite gradient entry); 0 when
 * neither happened.  The returned pd_status reports argument and launch errors
 * only: it cannot wait for the kernels.  With status_flags NULL these two
 * conditions are not reported. */
#define PD_NOALLOC_MAX_CELLS 32768
#define PD_LOCAL_FLAG_INVERTED 2
#define PD_LOCAL_FLAG_NAN 4
pd_status pd_local_step_noalloc(int64_t n_nodes, int64_t n_elems, const int32_t* elems,
                                const int32_t* inc_ptr, const int32_t* inc, double dx,
                                const double* x, const double* act, const double* w_corot,
                                const double* w_vol, const double* w_muscle, const double* fiber,
                                const uint8_t* contact, double k_contact, int32_t precision,
                                double* grad_E, double* energy, int32_t* status_flags,
                                void* stream);

/* Serving: rollout-plus-gradient requests on one GPU (no counterpart in the
 * paper, whose method this wraps: each request is one forward rollout of T
 * implicit-Euler steps (Alg. 1), the loss L = sum(loss_w * x_T), and one
 * backward pass (Alg. 2 per step, Sec. 4.3) to dL/dv0 and dL/dact).
 *
 * A server owns `max_slots` worker slots; each is a host thread with its own
 * CUDA stream and a small cache of meshes (keyed by geometry) and factors (keyed
 * by material weights, h, gravity, contact stiffness and precision).  Requests
 * are admitted first-in first-out as soon as a slot is free and their estimated
 * device memory fits in `mem_budget_bytes` next to the requests already running
 * (a request that fits nowhere runs alone).  The kernels of all running requests
 * share the GPU; the solve of a request is limited to its share of the SMs so
 * that several small solves run side by side.  A request's result does not
 * depend on what else runs: every reduction has a fixed order, and each request
 * has its own mesh workspace.
 *
 * All arrays of a request are host memory, copied during pd_serve_submit (the
 * caller may free them on return); node arrays are in kept-node order. */
typedef struct pd_server_s* pd_server;

typedef struct {
  /* geometry (as pd_mesh_desc) */
  int32_t nx, ny, nz;
  double dx, origin[3], density;
  const uint8_t* cell_mask_host;   /* nx*ny*nz or NULL */
  const uint8_t* dirichlet_host;   /* per kept node or NULL */
  const uint8_t* contact_host;     /* per kept node or NULL (contact needs k_contact > 0) */
  /* material and dynamics (as pd_factorize) */
  const double* w_corot_host;      /* (e) or NULL */
  const double* w_vol_host;        /* (e) or NULL */
  const double* w_muscle_host;     /* (e) or NULL */
  const double* fiber_host;        /* (e,3), required with w_muscle_host */
  double h, gravity[3], k_contact, mu;
  int32_t precision;               /* PD_PREC_FP64 or PD_PREC_MIXED */
  /* rollout */
  int32_t T;                       /* steps, >= 1 */
  const double* x0_host;           /* (n,3) */
  const double* v0_host;           /* (n,3) */
  const double* f_ext_host;        /* (n,3) constant over the rollout, or NULL */
  const double* act_host;          /* (T,e) or NULL */
  const double* loss_w_host;       /* (n,3) */
  pd_solver_opts opts;
} pd_request;

typedef struct {
  pd_status status;                /* the request's own status (PD_OK, PD_ERR_NOT_CONVERGED, ...) */
  double loss;                     /* sum(loss_w * x_T) */
  int64_t n_nodes, n_elems, T;
  const double* x_final_host;      /* (n,3) x_T */
  const double* g_v0_host;         /* (n,3) dL/dv0 */
  const double* g_act_host;        /* (T,e) dL/dact, NULL without actuation */
  double queue_ms;                 /* submit -> start on a slot (host clock) */
  double latency_ms;               /* submit -> completion (host clock) */
  int64_t fwd_iters, bwd_iters;
  int32_t slot;                    /* worker slot that ran it */
  int32_t mesh_cached, factor_cached;   /* 1 if the slot's cache served them */
} pd_result;

/* device: CUDA ordinal; mem_budget_bytes: device memory the running requests'
 * estimates may add up to; max_slots: concurrent requests (1..64). */
pd_status pd_serve_create(int32_t device, size_t mem_budget_bytes, int32_t max_slots,
                          pd_server* out);
/* Non-blocking: validates and copies the request, returns its ticket.
 * PD_ERR_INVALID_ARG for a malformed request (nothing is queued). */
pd_status pd_serve_submit(pd_server s, const pd_request* r, uint64_t* ticket);
/* PD_OK with *out filled once the request has finished (out->status holds the
 * request's own status; pd_last_error-style text is not kept), PD_ERR_TIMEOUT
 * while it is queued or running, PD_ERR_INVALID_ARG for an unknown or released
 * ticket.  The arrays in *out stay valid until pd_serve_release of the ticket
 * or pd_serve_destroy. */
pd_status pd_serve_poll(pd_server s, uint64_t ticket, pd_result* out);
/* Frees a finished request's result. */
pd_status pd_serve_release(pd_server s, uint64_t ticket);
/* Blocks until every submitted request has finished. */
pd_status pd_serve_drain(pd_server s);
/* Finishes the running requests, drops the queued ones, frees everything. */
void pd_serve_destroy(pd_server s);

const char* pd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DIFFPD_H */
