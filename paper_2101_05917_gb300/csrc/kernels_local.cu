// Local steps of PD forward (Alg. 1) and of the adjoint splitting iteration
// (Alg. 2), plus the node gathers that turn element contributions into
// grad g = M (x - y)/h^2 + sum_c w_c G_c^T (G_c x - p_c)      (Eqn 20)
// and   Hess g v = M v/h^2 + sum_c w_c G_c^T (I - dp_c/dx) G_c v   (Eqns 21-22).
//
// Layout: one warp handles 4 hex cells; lane = 8*cell + k.  For loads and
// stores k is a corner; for the per-Gauss-point math k is the Gauss point
// (2x2x2 rule).  Corner data moves between the two roles with warp shuffles,
// so there is no shared memory and no atomics: each cell writes its 8 corner
// forces to an element buffer, and the gather sums them per node in the fixed
// incidence order (bit-reproducible).  Unstructured tetrahedra (one point each)
// take one thread per element instead (tet_element_kernel), with the same element
// buffer layout and gathers.
#include "pd_internal.cuh"
#include "pd_math.cuh"

namespace pd {

namespace {

constexpr int kElemThreads = kElemBlockThreads;   // 8 warps = 32 cells per block
constexpr int kGatherThreads = 256;

__device__ __forceinline__ int cbit(int a, int d) { return (a >> (2 - d)) & 1; }

// d N_a / d X at Gauss point q, component d, for a cube of edge dx:
// (s_ad / dx) * prod_{d' != d} (1 + s_ad' xi_qd') / 2, xi = +-1/sqrt(3).
template <typename T>
__device__ __forceinline__ T gradN(int a, int q, int d, T inv_dx) {
  const T g = T(0.57735026918962576451);
  const T wp = T(0.5) * (T(1) + g), wm = T(0.5) * (T(1) - g);
  T prod = inv_dx;
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    if (dd == d) continue;
    prod *= (cbit(a, dd) == cbit(q, dd)) ? wp : wm;
  }
  return cbit(a, d) ? prod : -prod;
}

// Tetrahedral rule: tetrahedron q < 6 runs from corner 0 along axes p1, p2, p3 to
// corner 7 (q = 2 p1 + [p2 is the larger of the other two]); the gradients of its
// barycentric coordinates are (-e_p1, e_p1 - e_p2, e_p2 - e_p3, e_p3) / dx at corners
// 0, c1 = {p1}, c2 = {p1, p2}, 7, zero at the other corners; q = 6, 7 are unused.
template <typename T>
__device__ __forceinline__ T gradN_tet(int a, int q, int d, T inv_dx) {
  if (q >= 6) return T(0);
  const int p1 = q >> 1, lo = p1 == 0 ? 1 : 0, hi = p1 == 2 ? 1 : 2;
  const int p2 = (q & 1) ? hi : lo, p3 = 3 - p1 - p2;
  const int c1 = 4 >> p1, c2 = c1 + (4 >> p2);
  int g = 0;
  if (a == 0) g = -(d == p1);
  else if (a == c1) g = (d == p1) - (d == p2);
  else if (a == c2) g = (d == p2) - (d == p3);
  else if (a == 7) g = (d == p3);
  return T(g) * inv_dx;
}

enum { RULE_HEX8 = 0, RULE_TET6 = 1 };

// Hexahedron: the shape gradients factor over the three axes, so the sums over
// the 8 corners (F at a Gauss point) and over the 8 Gauss points (corner forces)
// are Kronecker products of 2 x 2 matrices applied across the cell's 8 lanes: one
// butterfly stage per axis, exchanging with the lane whose index differs in that
// axis' bit (d = 0, 1, 2 <-> lane bit 4, 2, 1).  Per axis, with w(equal bits) =
// (1 + 1/sqrt3)/2 and w(different bits) = (1 - 1/sqrt3)/2:
//   W (an axis other than the derivative's): v' = w+ v + w- v_partner
//   D (the derivative axis, corners -> point): v' = v[bit 1] - v[bit 0]
//   S (the derivative axis, points -> corner): v' = sign(own bit) (v + v_partner)
// which reproduces sum_a v_a dN_a/dX_j(xi_q) (and its transpose) with the factor
// 1/dx applied once at the end.
template <typename T>
struct HexW {
  static constexpr double kWp = 0.78867513459481288225;   // (1 + 1/sqrt3) / 2
  static constexpr double kWm = 0.21132486540518711775;   // (1 - 1/sqrt3) / 2
};

template <typename T, int MASK>
__device__ __forceinline__ T bf_w(T v) {
  const T p = __shfl_xor_sync(0xffffffffu, v, MASK);
  return T(HexW<T>::kWp) * v + T(HexW<T>::kWm) * p;
}
template <typename T, int MASK>
__device__ __forceinline__ T bf_d(T v, int k) {
  const T p = __shfl_xor_sync(0xffffffffu, v, MASK);
  return (k & MASK) ? v - p : p - v;
}
template <typename T, int MASK>
__device__ __forceinline__ T bf_s(T v, int k) {
  const T t = v + __shfl_xor_sync(0xffffffffu, v, MASK);
  return (k & MASK) ? t : -t;
}

// G[i][j] += inv_dx * sum_a v_a[i] dN_a/dX_j at the lane's Gauss point k (v: the
// lane's corner value, corner a = lane k)
template <typename T>
__device__ __forceinline__ void hex_grad(const T (&v)[3], int k, T inv_dx, T (&G)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T p0 = __shfl_xor_sync(0xffffffffu, v[i], 4);
    const T w0 = T(HexW<T>::kWp) * v[i] + T(HexW<T>::kWm) * p0;
    const T d0 = (k & 4) ? v[i] - p0 : p0 - v[i];
    const T pw = __shfl_xor_sync(0xffffffffu, w0, 2);
    const T pd = __shfl_xor_sync(0xffffffffu, d0, 2);
    const T d0w1 = T(HexW<T>::kWp) * d0 + T(HexW<T>::kWm) * pd;
    const T w0d1 = (k & 2) ? w0 - pw : pw - w0;
    const T w0w1 = T(HexW<T>::kWp) * w0 + T(HexW<T>::kWm) * pw;
    G[i][0] += inv_dx * bf_w<T, 1>(d0w1);
    G[i][1] += inv_dx * bf_w<T, 1>(w0d1);
    G[i][2] += inv_dx * bf_d<T, 1>(w0w1, k);
  }
}

// f[i] = inv_dx * sum_q sum_j S_q[i][j] dN_k/dX_j(xi_q) for the lane's corner k
// (S: the lane's Gauss-point stress)
template <typename T>
__device__ __forceinline__ void hex_forces(const T (&S)[3][3], int k, T inv_dx, T (&f)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T u0 = bf_s<T, 4>(S[i][0], k);
    const T u1 = bf_w<T, 4>(S[i][1]);
    const T u2 = bf_w<T, 4>(S[i][2]);
    const T v0 = bf_w<T, 2>(u0);
    const T v1 = bf_s<T, 2>(u1, k);
    const T v2 = bf_w<T, 2>(u2);
    f[i] = inv_dx * (bf_w<T, 1>(v0 + v1) + bf_s<T, 1>(v2, k));
  }
}

template <typename T, int RULE>
__device__ __forceinline__ T shape_grad(int a, int q, int d, T inv_dx) {
  return RULE == RULE_TET6 ? gradN_tet<T>(a, q, d, inv_dx) : gradN<T>(a, q, d, inv_dx);
}

enum { MODE_FORCE = 0, MODE_HVP = 1, MODE_PGRAD = 2 };

// det(I + H) - 1 without the cancellation of forming det(I + H): the trace, the
// principal 2x2 minors and det H
template <typename T>
__device__ __forceinline__ T det_minus_one(const T (&H)[3][3]) {
  const T tr = H[0][0] + H[1][1] + H[2][2];
  const T m2 = H[0][0] * H[1][1] - H[0][1] * H[1][0] + H[0][0] * H[2][2] - H[0][2] * H[2][0] +
               H[1][1] * H[2][2] - H[1][2] * H[2][1];
  const T d3 = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) - H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
               H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
  return tr + m2 + d3;
}

// x - log(1 + x): its Taylor series for small |x| (the direct form cancels), else
// directly
template <typename T>
__device__ __forceinline__ T x_minus_log1p(T x) {
  const T lim = sizeof(T) == 4 ? T(0.1) : T(0.01);
  if (fabs(x) < lim) {
    // x^2/2 - x^3/3 + ... - x^11/11, Horner in x
    T s = T(0);
#pragma unroll
    for (int k = 11; k >= 2; --k) s = s * x + ((k & 1) ? T(1) : T(-1)) * (T(1) / T(k)) * T(-1);
    return s * x * x;
  }
  return x - (sizeof(T) == 4 ? (T)log1pf((float)x) : (T)log1p((double)x));
}

// One Gauss point of the Neo-Hookean material (Sec. 8),
//   psi = mu/2 (tr F^T F - 3) - mu log J + lambda/2 (log J)^2,
//   P   = mu (F - F^-T) + lambda log J F^-T,
//   dP  = mu dF + (mu - lambda log J) F^-T dF^T F^-T + lambda tr(F^-1 dF) F^-T,
// with F = I + H, in forms that keep the accuracy relative to the strain:
// F - F^-T = (H + H^T + H H^T) F^-T, log J = log1p(det(I + H) - 1) and
// tr F^T F - 3 - 2 log J = |H|^2 + 2 (tr H - log J).  FORCE adds V P to S and
// V psi to energy, HVP adds V dP(dF), PGRAD sets the adjoint products of
// dP/dw_corot = (F - F^-T)/2 and dP/dw_vol = log J F^-T with dF = G z.
template <typename T, int MODE>
__device__ __forceinline__ void neohookean_point(const T (&H)[3][3], const T (&dF)[3][3], T mu, T lam, T V,
                                                 T (&S)[3][3], T& energy, T& gwc, T& gwv) {
  const T F[3][3] = {{T(1) + H[0][0], H[0][1], H[0][2]},
                     {H[1][0], T(1) + H[1][1], H[1][2]},
                     {H[2][0], H[2][1], T(1) + H[2][2]}};
  const T j1 = det_minus_one<T>(H);
  const T invJ = T(1) / (T(1) + j1);
  const T logJ = sizeof(T) == 4 ? (T)log1pf((float)j1) : (T)log1p((double)j1);
  // F^-T = cof(F) / J
  T Fit[3][3];
  Fit[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) * invJ;
  Fit[0][1] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) * invJ;
  Fit[0][2] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) * invJ;
  Fit[1][0] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * invJ;
  Fit[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * invJ;
  Fit[1][2] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * invJ;
  Fit[2][0] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * invJ;
  Fit[2][1] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * invJ;
  Fit[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * invJ;
  if constexpr (MODE == MODE_HVP) {
    // tr(F^-1 dF) = F^-T : dF;  F^-T dF^T F^-T
    T tr = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tr += Fit[i][j] * dF[i][j];
    T A[3][3];   // dF^T F^-T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A[i][j] = dF[0][i] * Fit[0][j] + dF[1][i] * Fit[1][j] + dF[2][i] * Fit[2][j];
    const T c1 = mu - lam * logJ, c2 = lam * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T FA = Fit[i][0] * A[0][j] + Fit[i][1] * A[1][j] + Fit[i][2] * A[2][j];
        S[i][j] += V * (mu * dF[i][j] + c1 * FA + c2 * Fit[i][j]);
      }
  } else {
    // B = H + H^T + H H^T = F F^T - I;  F - F^-T = B F^-T
    T B[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) B[i][j] = H[i][j] + H[j][i] + H[i][0] * H[j][0] + H[i][1] * H[j][1] + H[i][2] * H[j][2];
    T D[3][3];   // F - F^-T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) D[i][j] = B[i][0] * Fit[0][j] + B[i][1] * Fit[1][j] + B[i][2] * Fit[2][j];
    if (MODE == MODE_FORCE) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[i][j] += V * (mu * D[i][j] + lam * logJ * Fit[i][j]);
      // tr H - log J = (tr H - j1) + (j1 - log1p(j1))
      const T trH = H[0][0] + H[1][1] + H[2][2];
      T hh = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) hh += H[i][j] * H[i][j];
      const T trh_logj = (trH - j1) + x_minus_log1p<T>(j1);
      energy += V * (T(0.5) * mu * hh + mu * trh_logj + T(0.5) * lam * logJ * logJ);
    } else {
      T a = T(0), b = T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          a += dF[i][j] * D[i][j];
          b += dF[i][j] * Fit[i][j];
        }
      gwc = -V * T(0.5) * a;
      gwv = -V * logJ * b;
    }
  }
}

struct ElemParams {
  const IterState* gate;
  int64_t ne;
  const int32_t* elems;
  const double* x;
  const double* v;
  const double* act;
  const double *wc, *wv, *wm, *fiber;
  double dx, Vq, inv_dx;
  float dx_f, Vq_f, inv_dx_f;   // the same in FP32 (the FP32 kernels take no FP64 arithmetic for them)
  void* out;            // elembuf (T) for FORCE/HVP
  double* energy;       // block partials (FORCE)
  double *g_wc, *g_wv, *g_wm, *g_act;   // PGRAD outputs
  int* flags;
  // FP32 hexahedral Hessian products inside an adjoint solve (gate set): the point
  // SVDs (and volume projections) at x_{t+1}, shared by the solve's products;
  // kSvdFields (+ kVolFields with the volume energy) fields of n_gp floats each
  float* svd_cache;
  int64_t n_gp;
  // refined FP64 Hessian products of one adjoint step (REF): each point's refined
  // rotation and stretch (18 doubles, field stride n_gp), written by the step's first
  // residual check (ref_mode 1) and read by the later ones (ref_mode 2)
  double* ref_cache;
  int ref_mode;
  // unstructured tetrahedra (tet_element_kernel): node rest positions (internal
  // order) and per element the barycentric gradients (12, vertex-major) and volume
  const double* Xrest;
  const double *tgrad, *tvol;
  const float *tgrad_f, *tvol_f;
};

constexpr int kRefFields = 18;   // R (9), S (9)

constexpr int kSvdFields = 24;   // U, V, sigma, sigma - 1
constexpr int kVolFields = 11;   // lambda, s, gap, a, and whether the projection applies

// ACC (FP32 hexahedra only): H and the Green strain in FP64, the rest in FP32.
// REF (FP64 hexahedra with the corotated and muscle energies only): the SVD runs
// in FP32 on the FP64 strain, and the rotation and its derivative are refined to
// FP64 without eigenvectors (polar_refine / polar_solve); every quantity that
// enters the gradient or the Hessian product is then FP64-accurate.
// NH (hexahedra): the Neo-Hookean material (Sec. 8) with mu = w_corot / 2 and
// lambda = w_vol in place of the corotated and volume energies; no SVD.
template <typename T, int MODE, int RULE = RULE_HEX8, bool ACC = false, bool REF = false, bool NH = false>
__global__ void __launch_bounds__(kElemThreads, sizeof(T) == 8 ? 1 : (MODE == MODE_FORCE && !ACC ? 3 : 2))
element_kernel(ElemParams p) {
  static_assert(!REF || (sizeof(T) == 8 && RULE == RULE_HEX8 && MODE != MODE_PGRAD), "refined: FP64 hexahedra");
  static_assert(!NH || (RULE == RULE_HEX8 && !ACC && !REF), "Neo-Hookean: hexahedra, plain FP32 / FP64");
  if (p.gate && p.gate->converged) return;
  __shared__ double wsum[kElemThreads / 32];
  __shared__ unsigned arrived;
  if (MODE == MODE_FORCE) {
    if (threadIdx.x == 0) arrived = 0u;
    __syncthreads();   // at entry all warps are together: no wait
  }
  const int lane = threadIdx.x & 31;
  const int base = lane & ~7;
  const int k = lane & 7;
  const int64_t e = ((int64_t)blockIdx.x * kElemThreads + threadIdx.x) >> 3;
  const bool valid = e < p.ne;
  const T inv_dx = sizeof(T) == 4 ? T(p.inv_dx_f) : T(p.inv_dx);
  // The Hessian products of one adjoint solve are all taken at x_{t+1}: the solve's
  // first product writes every point's SVD (and volume projection) to the cache, the
  // later ones read it instead of forming H and the SVD again (same values, so the
  // same results).  Uniform over the grid: 0 none, 1 write, 2 read.
  constexpr bool kCache = MODE == MODE_HVP && sizeof(T) == 4 && RULE == RULE_HEX8 && !ACC && !REF && !NH;
  int cmode = 0;
  if constexpr (kCache) {
    if (p.svd_cache && p.gate && !p.wm) cmode = p.gate->svd_cached ? 2 : 1;
  }
  // every thread of the grid owns a slot (n_gp = the grid's threads), tail threads too
  float* cache = (kCache && cmode != 0) ? p.svd_cache + ((int64_t)blockIdx.x * kElemThreads + threadIdx.x) : nullptr;
  const int64_t cs = p.n_gp;   // field stride
  constexpr bool kRefCache = REF && MODE == MODE_HVP;
  const int rmode = (kRefCache && p.ref_cache) ? p.ref_mode : 0;
  double* rcache = rmode ? p.ref_cache + ((int64_t)blockIdx.x * kElemThreads + threadIdx.x) : nullptr;
  const bool skip_x = cmode == 2 || rmode == 2;   // the cached point data replace x and H
  // volume weight of this lane's point (the tetrahedral rule leaves lanes 6, 7 idle)
  const T Vq = (RULE == RULE_TET6 && k >= 6) ? T(0) : (sizeof(T) == 4 ? T(p.Vq_f) : T(p.Vq));

  // ---- corner loads: relative displacement of corner k w.r.t. corner 0
  int node = valid ? p.elems[e * 8 + k] : 0;
  T dk[3] = {T(0), T(0), T(0)};
  double dkd[3] = {0, 0, 0};
  if (!skip_x) {
    double xk[3] = {0, 0, 0};
    if (valid) {
      xk[0] = p.x[3 * (int64_t)node + 0];
      xk[1] = p.x[3 * (int64_t)node + 1];
      xk[2] = p.x[3 * (int64_t)node + 2];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double x0 = __shfl_sync(0xffffffffu, xk[i], base);
      dkd[i] = (xk[i] - x0) - (cbit(k, i) ? p.dx : 0.0);
      dk[i] = (T)dkd[i];
    }
  }
  T vk[3] = {T(0), T(0), T(0)};
  if (MODE != MODE_FORCE && valid) {
    vk[0] = (T)p.v[3 * (int64_t)node + 0];
    vk[1] = (T)p.v[3 * (int64_t)node + 1];
    vk[2] = (T)p.v[3 * (int64_t)node + 2];
  }

  // ---- per Gauss point (q = k): H = F - I and, when needed, dF = G_q v
  T H[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  T dF[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  // ACC: the Green strain of this point formed in FP64 (for the SVD below)
  T Eacc[3][3];
  if constexpr (RULE == RULE_HEX8 && ACC) {
    double Hd[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    hex_grad<double>(dkd, k, 1.0 / p.dx, Hd);
    double Ed[3][3];
    green_strain<double>(Hd, Ed);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        H[i][j] = (T)Hd[i][j];
        Eacc[i][j] = (T)Ed[i][j];
      }
    if (MODE != MODE_FORCE) hex_grad<T>(vk, k, inv_dx, dF);
  } else if constexpr (RULE == RULE_HEX8) {
    if (!skip_x) hex_grad<T>(dk, k, inv_dx, H);
    if (MODE != MODE_FORCE) hex_grad<T>(vk, k, inv_dx, dF);
  } else {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      T da[3], va[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        da[i] = __shfl_sync(0xffffffffu, dk[i], base + a);
        if (MODE != MODE_FORCE) va[i] = __shfl_sync(0xffffffffu, vk[i], base + a);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T gN = shape_grad<T, RULE>(a, k, j, inv_dx);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          H[i][j] += da[i] * gN;
          if (MODE != MODE_FORCE) dF[i][j] += va[i] * gN;
        }
      }
    }
  }

  const T wc = (valid && p.wc) ? (T)p.wc[e] : T(0);
  const T wv = (valid && p.wv) ? (T)p.wv[e] : T(0);
  const T wm = (valid && p.wm) ? (T)p.wm[e] : T(0);
  const T act = (valid && p.act) ? (T)p.act[e] : T(0);

  T S[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  T energy = T(0);
  T gwc = T(0), gwv = T(0), gwm = T(0), gact = T(0);

  SVD3<T> sv;
  double Rr[3][3], Sr[3][3];   // REF: refined rotation and symmetric factor
  if constexpr (NH) {
    neohookean_point<T, MODE>(H, dF, T(0.5) * wc, wv, Vq, S, energy, gwc, gwv);
    if (valid && !(T(1) + det_minus_one<T>(H) > T(0))) atomicOr(p.flags, DEV_ERR_INVERTED);
  } else if (REF && rmode == 2) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Rr[i][j] = __ldcs(rcache + (3 * i + j) * cs);
        Sr[i][j] = __ldcs(rcache + (9 + 3 * i + j) * cs);
      }
  } else if constexpr (REF) {
    double Ed[3][3];
    green_strain<double>(H, Ed);
    float H32[3][3], E32[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        H32[i][j] = (float)H[i][j];
        E32[i][j] = (float)Ed[i][j];
      }
    SVD3<float> s32;
    svd3_from_HE<float>(H32, E32, s32);
    const bool ok = polar_refine(s32.U, s32.V, H, Rr, Sr);
    if (valid && (!(s32.sig[2] > 0.0f) || !ok)) atomicOr(p.flags, DEV_ERR_INVERTED);
    if (rmode == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          rcache[(3 * i + j) * cs] = Rr[i][j];
          rcache[(9 + 3 * i + j) * cs] = Sr[i][j];
        }
    }
  } else if (cmode == 2) {
    if constexpr (kCache) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          sv.U[i][j] = (T)__ldcs(cache + (3 * i + j) * cs);
          sv.V[i][j] = (T)__ldcs(cache + (9 + 3 * i + j) * cs);
        }
        sv.sig[i] = (T)__ldcs(cache + (18 + i) * cs);
        sv.sm1[i] = (T)__ldcs(cache + (21 + i) * cs);
      }
    }
  } else {
    if constexpr (RULE == RULE_HEX8 && ACC) svd3_from_HE<T>(H, Eacc, sv);
    else svd3_from_H<T>(H, sv);
    if (valid && !(sv.sig[2] > T(0))) atomicOr(p.flags, DEV_ERR_INVERTED);
    if constexpr (kCache) {
      if (cmode == 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            cache[(3 * i + j) * cs] = (float)sv.U[i][j];
            cache[(9 + 3 * i + j) * cs] = (float)sv.V[i][j];
          }
          cache[(18 + i) * cs] = (float)sv.sig[i];
          cache[(21 + i) * cs] = (float)sv.sm1[i];
        }
      }
    }
  }
  T M[3][3];
  if (MODE != MODE_FORCE && !REF && !NH) rotate_in<T>(sv.U, dF, sv.V, M);

  if constexpr (NH) {
    // done above
  } else if constexpr (REF) {
    if (wc != T(0)) {
      if (MODE == MODE_FORCE) {
        // F - R with F = I + H
        T en = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const double d = (i == j ? 1.0 : 0.0) + H[i][j] - Rr[i][j];
            S[i][j] += wc * Vq * d;
            en += d * d;
          }
        energy += T(0.5) * wc * Vq * en;
      } else {
        // dF - dR, dR = R skew(w), w = 2 (tr(S) I - S)^-1 axial(skew(R^T dF))
        double RtdF[3][3], k[3], w[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) RtdF[i][j] = Rr[0][i] * dF[0][j] + Rr[1][i] * dF[1][j] + Rr[2][i] * dF[2][j];
        skew_axial(RtdF, k);
        polar_solve(Sr, k, w);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          // (R skew(w))_ij = sum_k R_ik skew(w)_kj
          const double dR0 = Rr[i][1] * w[2] - Rr[i][2] * w[1];
          const double dR1 = Rr[i][2] * w[0] - Rr[i][0] * w[2];
          const double dR2 = Rr[i][0] * w[1] - Rr[i][1] * w[0];
          S[i][0] += wc * Vq * (dF[i][0] - dR0);
          S[i][1] += wc * Vq * (dF[i][1] - dR1);
          S[i][2] += wc * Vq * (dF[i][2] - dR2);
        }
      }
    }
  } else if (wc != T(0)) {
    if (MODE == MODE_FORCE) {
      add_UdVt<T>(S, sv.U, sv.sm1, sv.V, wc * Vq);
      energy += T(0.5) * wc * Vq * (sv.sm1[0] * sv.sm1[0] + sv.sm1[1] * sv.sm1[1] + sv.sm1[2] * sv.sm1[2]);
    } else if (MODE == MODE_HVP) {
      T K[3][3];
      corot_hvp_frame<T>(sv, M, K);
      add_UKVt<T>(S, sv.U, K, sv.V, wc * Vq);
    } else {
      gwc = -Vq * (M[0][0] * sv.sm1[0] + M[1][1] * sv.sm1[1] + M[2][2] * sv.sm1[2]);
    }
  }
  if (!REF && !NH && __any_sync(0xffffffffu, wv != T(0))) {   // REF runs without the volume energy
    VolProj<T> vp;
    bool vok;
    if (cmode == 2) {
      float* vc = cache + kSvdFields * cs;
      vp.lam = (T)__ldcs(vc);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vp.s[i] = (T)__ldcs(vc + (1 + i) * cs);
        vp.gap[i] = (T)__ldcs(vc + (4 + i) * cs);
        vp.a[i] = (T)__ldcs(vc + (7 + i) * cs);
      }
      vok = __ldcs(vc + 10 * cs) != 0.0f;
    } else {
      vok = volume_project<T>(sv, vp, wv != T(0));
      if (cmode == 1) {
        float* vc = cache + kSvdFields * cs;
        vc[0] = (float)vp.lam;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          vc[(1 + i) * cs] = (float)vp.s[i];
          vc[(4 + i) * cs] = (float)vp.gap[i];
          vc[(7 + i) * cs] = (float)vp.a[i];
        }
        vc[10 * cs] = vok ? 1.0f : 0.0f;
      }
    }
    if (vok) {
      if (MODE == MODE_FORCE) {
        add_UdVt<T>(S, sv.U, vp.gap, sv.V, wv * Vq);
        energy += T(0.5) * wv * Vq * (vp.gap[0] * vp.gap[0] + vp.gap[1] * vp.gap[1] + vp.gap[2] * vp.gap[2]);
      } else if (MODE == MODE_HVP) {
        T K[3][3];
        vol_hvp_frame<T>(sv, vp, M, K);
        add_UKVt<T>(S, sv.U, K, sv.V, wv * Vq);
      } else {
        gwv = -Vq * (M[0][0] * vp.gap[0] + M[1][1] * vp.gap[1] + M[2][2] * vp.gap[2]);
      }
    }
  }
  // dL/dw_muscle exists for every element with a fibre, also where w_muscle = 0
  const bool musc = (MODE == MODE_PGRAD) ? (valid && p.wm != nullptr) : (wm != T(0));
  if (musc) {
    const T m0 = (T)p.fiber[3 * e + 0], m1 = (T)p.fiber[3 * e + 1], m2 = (T)p.fiber[3 * e + 2];
    const T mv[3] = {m0, m1, m2};
    T f[3], Hm[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Hm[i] = H[i][0] * m0 + H[i][1] * m1 + H[i][2] * m2;
      f[i] = mv[i] + Hm[i];
    }
    // m^T E m with E = H + H^T + H^T H  ->  2 m.Hm + |Hm|^2
    const T mEm = T(2) * (m0 * Hm[0] + m1 * Hm[1] + m2 * Hm[2]) + Hm[0] * Hm[0] + Hm[1] * Hm[1] + Hm[2] * Hm[2];
    const T fn = tsqrt<T>(T(1) + mEm);
    const T fnm1 = mEm / (T(1) + fn);            // |f| - 1
    const T fh[3] = {f[0] / fn, f[1] / fn, f[2] / fn};
    const T ex = fnm1 + act;                     // |f| - (1 - a)
    if (MODE == MODE_FORCE) {
      const T c = wm * Vq * ex;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[i][j] += c * fh[i] * mv[j];
      energy += T(0.5) * wm * Vq * ex * ex;
    } else {
      T df[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) df[i] = dF[i][0] * m0 + dF[i][1] * m1 + dF[i][2] * m2;
      const T fd = fh[0] * df[0] + fh[1] * df[1] + fh[2] * df[2];
      if (MODE == MODE_HVP) {
        const T c1 = ex / fn, c2 = (T(1) - act) / fn * fd;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const T r = wm * Vq * (c1 * df[i] + c2 * fh[i]);
#pragma unroll
          for (int j = 0; j < 3; ++j) S[i][j] += r * mv[j];
        }
      } else {
        gwm = -Vq * ex * fd;
        gact = -wm * Vq * fd;
      }
    }
  }

  if (MODE == MODE_PGRAD) {
    // reduce over the 8 Gauss points of the cell (fixed butterfly)
#pragma unroll
    for (int off = 4; off >= 1; off >>= 1) {
      gwc += __shfl_xor_sync(0xffffffffu, gwc, off);
      gwv += __shfl_xor_sync(0xffffffffu, gwv, off);
      gwm += __shfl_xor_sync(0xffffffffu, gwm, off);
      gact += __shfl_xor_sync(0xffffffffu, gact, off);
    }
    if (valid && k == 0) {
      if (p.g_wc) p.g_wc[e] += (double)gwc;
      if (p.g_wv) p.g_wv[e] += (double)gwv;
      if (p.g_wm) p.g_wm[e] += (double)gwm;
      if (p.g_act) p.g_act[e] = (double)gact;
    }
    return;
  }

  // ---- corner forces f_a = sum_q S_q gradN_a(q), lane k acting as corner a = k
  T fa[3] = {T(0), T(0), T(0)};
  if constexpr (RULE == RULE_HEX8) {
    hex_forces<T>(S, k, inv_dx, fa);
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      T Sq[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Sq[i][j] = __shfl_sync(0xffffffffu, S[i][j], base + q);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const T gN = shape_grad<T, RULE>(k, q, j, inv_dx);
#pragma unroll
        for (int i = 0; i < 3; ++i) fa[i] += Sq[i][j] * gN;
      }
    }
  }
  if (valid) {
    T* out = reinterpret_cast<T*>(p.out) + (e * 8 + k) * 3;
    out[0] = fa[0];
    out[1] = fa[1];
    out[2] = fa[2];
  }
  if (MODE == MODE_FORCE) {
    // block energy partial without a block barrier: the cell's 8 points are added
    // in T, the warp's 4 cells in FP64; each warp deposits its sum, the last warp to
    // arrive adds the 8 deposits in warp order
    T ec = valid ? energy : T(0);
#pragma unroll
    for (int off = 4; off >= 1; off >>= 1) ec += __shfl_xor_sync(0xffffffffu, ec, off);
    double en = (double)ec;
#pragma unroll
    for (int off = 16; off >= 8; off >>= 1) en += __shfl_xor_sync(0xffffffffu, en, off);
    if (lane == 0) {
      wsum[threadIdx.x >> 5] = en;
      __threadfence_block();
      const unsigned t = atomicAdd(&arrived, 1u);
      if (t == kElemThreads / 32 - 1) {
        __threadfence_block();
        double tot = 0;
        for (int w = 0; w < kElemThreads / 32; ++w) tot += ((volatile double*)wsum)[w];
        p.energy[blockIdx.x] = tot;
      }
    }
  }
}

// Unstructured linear tetrahedra (PD_ELEM_TETU), one element per thread: F - I =
// sum over vertices a = 1..3 of (x_a - x_0 - (X_a - X_0)) (outer) grad N_a with the
// element's own barycentric gradients, dF = sum over a = 0..3 of v_a (outer) grad N_a,
// the corotated and volume projections of element_kernel at the element's one
// point (weight V), and the vertex forces f_a = S grad N_a into slots 0..3 of the
// element's record (slots 4..7 have no incidence entries and are not written).
// Every thread of the grid reaches the SVD and the volume projection (their
// full-warp votes); tail threads carry F = I and zero weights.
template <typename T, int MODE>
__global__ void __launch_bounds__(kElemThreads, sizeof(T) == 8 ? 1 : 2)
tet_element_kernel(ElemParams p) {
  if (p.gate && p.gate->converged) return;
  __shared__ double wsum[kElemThreads / 32];
  __shared__ unsigned arrived;
  if (MODE == MODE_FORCE) {
    if (threadIdx.x == 0) arrived = 0u;
    __syncthreads();   // at entry all warps are together: no wait
  }
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * kElemThreads + threadIdx.x;
  const bool valid = e < p.ne;
  T g[4][3];
  T H[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  T dF[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  T Vq = T(0);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int j = 0; j < 3; ++j) g[a][j] = T(0);
  if (valid) {
    int node[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) node[a] = p.elems[e * 8 + a];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if constexpr (sizeof(T) == 4) g[a][j] = p.tgrad_f[12 * e + 3 * a + j];
        else g[a][j] = p.tgrad[12 * e + 3 * a + j];
      }
    if constexpr (sizeof(T) == 4) Vq = p.tvol_f[e];
    else Vq = p.tvol[e];
    double x0[3], X0[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x0[i] = p.x[3 * (int64_t)node[0] + i];
      X0[i] = p.Xrest[3 * (int64_t)node[0] + i];
    }
#pragma unroll
    for (int a = 1; a < 4; ++a) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int64_t k = 3 * (int64_t)node[a] + i;
        const T d = (T)((p.x[k] - x0[i]) - (p.Xrest[k] - X0[i]));
#pragma unroll
        for (int j = 0; j < 3; ++j) H[i][j] += d * g[a][j];
      }
    }
    if (MODE != MODE_FORCE) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const T va = (T)p.v[3 * (int64_t)node[a] + i];
#pragma unroll
          for (int j = 0; j < 3; ++j) dF[i][j] += va * g[a][j];
        }
    }
  }
  const T wc = (valid && p.wc) ? (T)p.wc[e] : T(0);
  const T wv = (valid && p.wv) ? (T)p.wv[e] : T(0);

  T S[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
  T energy = T(0);
  T gwc = T(0), gwv = T(0);
  SVD3<T> sv;
  svd3_from_H<T>(H, sv);
  if (valid && !(sv.sig[2] > T(0))) atomicOr(p.flags, DEV_ERR_INVERTED);
  T M[3][3];
  if (MODE != MODE_FORCE) rotate_in<T>(sv.U, dF, sv.V, M);
  if (wc != T(0)) {
    if (MODE == MODE_FORCE) {
      add_UdVt<T>(S, sv.U, sv.sm1, sv.V, wc * Vq);
      energy += T(0.5) * wc * Vq * (sv.sm1[0] * sv.sm1[0] + sv.sm1[1] * sv.sm1[1] + sv.sm1[2] * sv.sm1[2]);
    } else if (MODE == MODE_HVP) {
      T K[3][3];
      corot_hvp_frame<T>(sv, M, K);
      add_UKVt<T>(S, sv.U, K, sv.V, wc * Vq);
    } else {
      gwc = -Vq * (M[0][0] * sv.sm1[0] + M[1][1] * sv.sm1[1] + M[2][2] * sv.sm1[2]);
    }
  }
  if (__any_sync(0xffffffffu, wv != T(0))) {
    VolProj<T> vp;
    if (volume_project<T>(sv, vp, wv != T(0))) {
      if (MODE == MODE_FORCE) {
        add_UdVt<T>(S, sv.U, vp.gap, sv.V, wv * Vq);
        energy += T(0.5) * wv * Vq * (vp.gap[0] * vp.gap[0] + vp.gap[1] * vp.gap[1] + vp.gap[2] * vp.gap[2]);
      } else if (MODE == MODE_HVP) {
        T K[3][3];
        vol_hvp_frame<T>(sv, vp, M, K);
        add_UKVt<T>(S, sv.U, K, sv.V, wv * Vq);
      } else {
        gwv = -Vq * (M[0][0] * vp.gap[0] + M[1][1] * vp.gap[1] + M[2][2] * vp.gap[2]);
      }
    }
  }

  if (MODE == MODE_PGRAD) {
    if (valid) {
      if (p.g_wc) p.g_wc[e] += (double)gwc;
      if (p.g_wv) p.g_wv[e] += (double)gwv;
      if (p.g_act) p.g_act[e] = 0.0;   // no muscle energy on this rule
    }
    return;
  }

  if (valid) {
    T* out = reinterpret_cast<T*>(p.out) + e * 8 * 3;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) out[3 * a + i] = S[i][0] * g[a][0] + S[i][1] * g[a][1] + S[i][2] * g[a][2];
  }
  if (MODE == MODE_FORCE) {
    // block energy partial as in element_kernel: the warp's 32 elements in FP64,
    // each warp deposits its sum, the last warp to arrive adds the deposits in order
    double en = valid ? (double)energy : 0.0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) en += __shfl_xor_sync(0xffffffffu, en, off);
    if (lane == 0) {
      wsum[threadIdx.x >> 5] = en;
      __threadfence_block();
      const unsigned t = atomicAdd(&arrived, 1u);
      if (t == kElemThreads / 32 - 1) {
        __threadfence_block();
        double tot = 0;
        for (int w = 0; w < kElemThreads / 32; ++w) tot += ((volatile double*)wsum)[w];
        p.energy[blockIdx.x] = tot;
      }
    }
  }
}

// Fixed-order block reduction of NV values per thread into partials[blk*4 + i].
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* partials) {
  __shared__ double red[NV][kGatherThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = v[i];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) red[i][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0;
    for (int k = 0; k < kGatherThreads / 32; ++k) t += red[threadIdx.x][k];
    partials[blockIdx.x * 4 + threadIdx.x] = t;
  }
}

struct GatherParams {
  const IterState* gate;
  int64_t nf;
  const int32_t *inc_ptr, *inc;
  const double* mass;
  const uint8_t* contact;
  double inv_h2, k_contact;
  const void* elembuf;
  const double* x;      // positions (contact)
  const double* y;      // predictor (grad mode)
  const double* v;      // dir (grad mode, for g.dir) / input vector (hvp mode)
  const double* aux;    // hvp mode: second vector for a dot product (may be null)
  double* out;
  double* partials;
  const uint8_t* held;  // nodes held at contact targets: gradient / product rows are zero
};

// sum of a node's corner values in incidence order.  FP32 values are added in
// FP32 with Kahan compensation (the sum of an FP64 accumulation without its FP64
// additions, which GB300 runs at a small fraction of the FP32 rate), FP64 values
// in FP64.
template <typename T>
__device__ __forceinline__ void corner_sum(const GatherParams& p, int64_t c, double (&g)[3]) {
  const T* eb = reinterpret_cast<const T*>(p.elembuf);
  const int32_t q0 = p.inc_ptr[c], q1 = p.inc_ptr[c + 1];
  if constexpr (sizeof(T) == 8) {
    g[0] = g[1] = g[2] = 0.0;
    for (int32_t q = q0; q < q1; ++q) {
      const int64_t slot = (int64_t)p.inc[q] * 3;
      g[0] += eb[slot + 0];
      g[1] += eb[slot + 1];
      g[2] += eb[slot + 2];
    }
  } else {
    float sm[3] = {0.f, 0.f, 0.f}, cp[3] = {0.f, 0.f, 0.f};
    for (int32_t q = q0; q < q1; ++q) {
      const int64_t slot = (int64_t)p.inc[q] * 3;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float y = eb[slot + i] - cp[i];
        const float t = sm[i] + y;
        cp[i] = (t - sm[i]) - y;
        sm[i] = t;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] = (double)sm[i] - (double)cp[i];
  }
}

// grad g at x: partials = [kinetic + contact energy, |g|^2, g.dir, 0]
template <typename T>
__global__ void __launch_bounds__(kGatherThreads) gather_grad_kernel(GatherParams p) {
  if (p.gate && p.gate->converged) return;
  const int64_t c = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x;
  double acc[4] = {0, 0, 0, 0};
  if (c < p.nf) {
    double g[3];
    corner_sum<T>(p, c, g);
    const double m = p.mass[c];
    double kin = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double d = p.x[3 * c + i] - p.y[3 * c + i];
      g[i] += m * d * p.inv_h2;
      kin += 0.5 * m * d * d * p.inv_h2;
    }
    if (p.contact && p.contact[c]) {
      const double z = p.x[3 * c + 2];
      if (z < 0.0) {
        g[2] += p.k_contact * z;
        kin += 0.5 * p.k_contact * z * z;
      }
    }
    if (p.held && p.held[c]) g[0] = g[1] = g[2] = 0.0;
    double gd = 0, gg = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      p.out[3 * c + i] = g[i];
      gg += g[i] * g[i];
      if (p.v) gd += g[i] * p.v[3 * c + i];
    }
    acc[0] = kin;
    acc[1] = gg;
    acc[2] = gd;
  }
  block_partials<4>(acc, p.partials);
}

// Hv = M v/h^2 + sum elembuf + contact; partials = [v.Hv, aux.Hv, |Hv|^2, 0]
template <typename T>
__global__ void __launch_bounds__(kGatherThreads) gather_hvp_kernel(GatherParams p) {
  if (p.gate && p.gate->converged) return;
  const int64_t c = (int64_t)blockIdx.x * kGatherThreads + threadIdx.x;
  double acc[4] = {0, 0, 0, 0};
  if (c < p.nf) {
    double g[3];
    corner_sum<T>(p, c, g);
    const double m = p.mass[c];
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] += m * p.v[3 * c + i] * p.inv_h2;
    if (p.contact && p.contact[c] && p.x[3 * c + 2] < 0.0) g[2] += p.k_contact * p.v[3 * c + 2];
    if (p.held && p.held[c]) g[0] = g[1] = g[2] = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      p.out[3 * c + i] = g[i];
      acc[0] += g[i] * p.v[3 * c + i];
      if (p.aux) acc[1] += g[i] * p.aux[3 * c + i];
      acc[2] += g[i] * g[i];
    }
  }
  block_partials<4>(acc, p.partials);
}

void set_cell_size(ElemParams& p, double dx, double points_per_cell) {
  p.dx = dx;
  p.Vq = dx * dx * dx / points_per_cell;
  p.inv_dx = 1.0 / dx;
  p.dx_f = (float)p.dx;
  p.Vq_f = (float)p.Vq;
  p.inv_dx_f = (float)p.inv_dx;
}

ElemParams make_params(const LocalArgs& a) {
  ElemParams p{};
  p.gate = a.gate;
  p.ne = a.m->h.e;
  p.elems = a.m->elems;
  p.x = a.x;
  p.v = a.v;
  p.act = a.act;
  p.wc = a.m->wc;
  p.wv = a.m->wv;
  p.wm = a.m->wm;
  p.fiber = a.m->fiber;
  set_cell_size(p, a.m->h.dx, a.m->h.rule == PD_ELEM_TET6 ? 6.0 : 8.0);
  p.Xrest = a.m->X;
  p.tgrad = a.m->tet_grad;
  p.tvol = a.m->tet_vol;
  p.tgrad_f = a.m->tet_grad_f;
  p.tvol_f = a.m->tet_vol_f;
  return p;
}

// element_kernel<T, MODE, rule of the mesh>
// grid of the element kernels: 8 threads per element record (voxel rules), one
// thread per element (unstructured tetrahedra)
int64_t element_grid(const MeshImpl* m) {
  const int64_t threads = m->h.rule == PD_ELEM_TETU ? m->h.e : m->h.e * 8;
  return (threads + kElemThreads - 1) / kElemThreads;
}

template <int MODE>
void launch_elem(const MeshImpl* m, int precision, const ElemParams& p, cudaStream_t s) {
  const int nb = (int)element_grid(m);
  if (m->h.rule == PD_ELEM_TETU) {   // corotated and volume energies only (no muscles, not Neo-Hookean)
    if (local_is_fp32(precision)) tet_element_kernel<float, MODE><<<nb, kElemThreads, 0, s>>>(p);
    else tet_element_kernel<double, MODE><<<nb, kElemThreads, 0, s>>>(p);
    return;
  }
  const bool tet = m->h.rule == PD_ELEM_TET6;
  if (m->neohookean && !tet) {
    // Neo-Hookean: FP32 for the mixed tiers, FP64 for the FP64 and refined ones
    if (local_is_fp32(precision))
      element_kernel<float, MODE, RULE_HEX8, false, false, true><<<nb, kElemThreads, 0, s>>>(p);
    else
      element_kernel<double, MODE, RULE_HEX8, false, false, true><<<nb, kElemThreads, 0, s>>>(p);
    return;
  }
  if (local_is_fp32(precision)) {
    if (tet) element_kernel<float, MODE, RULE_TET6><<<nb, kElemThreads, 0, s>>>(p);
    else if (precision == kPrecMixedAcc) element_kernel<float, MODE, RULE_HEX8, true><<<nb, kElemThreads, 0, s>>>(p);
    else element_kernel<float, MODE, RULE_HEX8><<<nb, kElemThreads, 0, s>>>(p);
  } else if (MODE != MODE_PGRAD && precision == kPrecRefined && !tet && !p.wv) {
    if constexpr (MODE != MODE_PGRAD)
      element_kernel<double, MODE, RULE_HEX8, false, true><<<nb, kElemThreads, 0, s>>>(p);
  } else {
    if (tet) element_kernel<double, MODE, RULE_TET6><<<nb, kElemThreads, 0, s>>>(p);
    else element_kernel<double, MODE, RULE_HEX8><<<nb, kElemThreads, 0, s>>>(p);
  }
}

GatherParams make_gather(const MeshImpl* m) {
  GatherParams p{};
  p.nf = m->h.nf;
  p.inc_ptr = m->inc_ptr;
  p.inc = m->inc;
  p.mass = m->mass;
  p.contact = m->k_contact > 0 ? m->contact : nullptr;
  p.inv_h2 = 1.0 / (m->h_step * m->h_step);
  p.k_contact = m->k_contact;
  p.held = m->held_active ? m->held : nullptr;
  return p;
}

}  // namespace

int element_blocks(const MeshImpl* m) { return (int)element_grid(m); }
int element_energy_partials(const MeshImpl* m) { return element_blocks(m); }
int gather_blocks(const MeshImpl* m) {
  return (int)((m->h.nf + kGatherThreads - 1) / kGatherThreads);
}

cudaError_t launch_element_forces(const LocalArgs& a, void* elembuf, double* energy_partials,
                                  int* flags, cudaStream_t s) {
  ElemParams p = make_params(a);
  p.out = elembuf;
  p.energy = energy_partials;
  p.flags = flags;
  launch_elem<MODE_FORCE>(a.m, a.precision, p, s);
  return cudaGetLastError();
}

bool ref_cache_applies(const MeshImpl* m, int64_t* doubles) {
  const int64_t nb = (m->h.e * 8 + kElemThreads - 1) / kElemThreads;
  *doubles = nb * kElemThreads * kRefFields;
  return m->precision == PD_PREC_MIXED && m->h.rule == PD_ELEM_HEX8 && !m->neohookean && !m->wv && !m->wm;
}

void svd_cache_layout(const MeshImpl* m, int64_t* slots, int64_t* fields) {
  const int64_t nb = (m->h.e * 8 + kElemThreads - 1) / kElemThreads;
  *slots = nb * kElemThreads;
  const bool applies = m->precision == PD_PREC_MIXED && m->h.rule == PD_ELEM_HEX8 && !m->neohookean && !m->wm;
  *fields = applies ? kSvdFields + (m->wv ? kVolFields : 0) : 0;
}

cudaError_t launch_element_hvp(const LocalArgs& a, void* elembuf, int* flags, cudaStream_t s) {
  ElemParams p = make_params(a);
  p.out = elembuf;
  p.flags = flags;
  int64_t slots, fields;
  svd_cache_layout(a.m, &slots, &fields);
  if (a.gate && a.m->svd_cache && fields > 0 && a.m->svd_cache_fields >= fields && a.precision == PD_PREC_MIXED) {
    p.svd_cache = a.m->svd_cache;
    p.n_gp = slots;
  }
  int64_t rd;
  if (a.ref_cache && a.m->ref_cache && ref_cache_applies(a.m, &rd) && a.precision == kPrecRefined) {
    p.ref_cache = a.m->ref_cache;
    p.ref_mode = a.ref_cache;
    p.n_gp = slots;
  }
  launch_elem<MODE_HVP>(a.m, a.precision, p, s);
  return cudaGetLastError();
}

cudaError_t launch_element_param_grads(const LocalArgs& a, double* g_wc, double* g_wv,
                                       double* g_wm, double* g_act, cudaStream_t s) {
  ElemParams p = make_params(a);
  p.g_wc = g_wc;
  p.g_wv = g_wv;
  p.g_wm = g_wm;
  p.g_act = g_act;
  p.flags = a.m->ws.flags;
  // per-element products in the requested precision, accumulated over the steps in FP64
  launch_elem<MODE_PGRAD>(a.m, a.precision, p, s);
  return cudaGetLastError();
}

cudaError_t launch_gather_grad(const MeshImpl* m, const IterState* gate, const void* elembuf,
                               int precision, const double* x, const double* y, const double* dir,
                               double* grad, double* partials, cudaStream_t s) {
  GatherParams p = make_gather(m);
  p.gate = gate;
  p.elembuf = elembuf;
  p.x = x;
  p.y = y;
  p.v = dir;
  p.out = grad;
  p.partials = partials;
  const int nb = gather_blocks(m);
  if (local_is_fp32(precision))
    gather_grad_kernel<float><<<nb, kGatherThreads, 0, s>>>(p);
  else
    gather_grad_kernel<double><<<nb, kGatherThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gather_hvp(const MeshImpl* m, const IterState* gate, const void* elembuf,
                              int precision, const double* x, const double* v, const double* aux,
                              double* Hv, double* partials, cudaStream_t s) {
  GatherParams p = make_gather(m);
  p.gate = gate;
  p.elembuf = elembuf;
  p.x = x;
  p.v = v;
  p.aux = aux;
  p.out = Hv;
  p.partials = partials;
  const int nb = gather_blocks(m);
  if (local_is_fp32(precision))
    gather_hvp_kernel<float><<<nb, kGatherThreads, 0, s>>>(p);
  else
    gather_hvp_kernel<double><<<nb, kGatherThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pd

namespace pd {

// Force-mode local step on caller-provided topology and weights (no mesh object).
cudaError_t launch_element_forces_raw(int64_t ne, const int32_t* elems, const double* x, const double* act,
                                      const double* wc, const double* wv, const double* wm, const double* fiber,
                                      double dx, int precision, void* elembuf, double* energy_partials,
                                      int* flags, cudaStream_t s) {
  ElemParams p{};
  p.ne = ne;
  p.elems = elems;
  p.x = x;
  p.act = act;
  p.wc = wc;
  p.wv = wv;
  p.wm = wm;
  p.fiber = fiber;
  set_cell_size(p, dx, 8.0);
  p.out = elembuf;
  p.energy = energy_partials;
  p.flags = flags;
  const int nb = (int)raw_element_blocks(ne);
  if (precision == PD_PREC_MIXED)
    element_kernel<float, MODE_FORCE><<<nb, kElemThreads, 0, s>>>(p);
  else
    element_kernel<double, MODE_FORCE><<<nb, kElemThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pd
