// Complementarity contact (Sec. 5.2): the global step with the contact set C held
// fixed (Alg. 3's inner solve, computed by Alg. 4 with a low-rank update of the
// prefactorised A).
//
// A = I_3 (x) L_A, so everything is scalar per coordinate.  With the columns
// B_j = L_A^-1 e_j of every contact candidate j precomputed once per
// factorisation, the solution with x_C = x* and L_{C'C'} x_{C'} = b_{C'} is
//   a1 = L_A^-1 b,  lambda = S^-1 (a1)_C  with S = (L_A^-1)_{CC} = B_{C,C},
//   x  = a1 - B_{.,C} lambda,  then x_C = x*.
// (Multipliers lambda on the rows of C make (a1 - B lambda)_C = 0, and the rows
// C' of L_A x + E_C lambda = b are the reduced system.)  This is the same rank-|C|
// update of A as the paper's Woodbury identity, written with the |C| x |C| matrix
// S instead of its 2|C| x 2|C| one; the result is identical in exact arithmetic.
// S is factored once per contact set on the device (S = L L^T, Q = L^-1), so
// lambda = Q^T (Q (a1)_C): two triangular matrix-vector products.  Per solve the
// update costs one solve of A plus O(nf |C| + |C|^2) memory traffic.
#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int kT = 256;

// b = 0 except b[3 cand[k0 + i] + i] = 1, i < count (<= 3): three unit right-hand
// sides, one per coordinate column
__global__ void unit_rhs_kernel(const int32_t* cand, int64_t k0, int count, double* b) {
  const int i = threadIdx.x;
  if (i < count) b[3 * (int64_t)cand[k0 + i] + i] = 1.0;
}

// Bc[:, k0 + j] = x[:, j] (coordinate column j of the solve), j < count
__global__ void extract_columns_kernel(int64_t nf, const double* x, int64_t k0, int count, double* Bc) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= nf) return;
  for (int j = 0; j < count; ++j) Bc[(k0 + j) * nf + i] = x[3 * i + j];
}

// S[r][k] = (L_A^-1)[node[r], node[k]] from the candidate columns, averaged over
// the two columns that hold it (they come from different solves): symmetric
__global__ void gather_S_kernel(int64_t nf, const double* Bc, const int32_t* node, const int32_t* cidx, int64_t c,
                                double* S) {
  const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (t >= c * c) return;
  const int64_t r = t / c, k = t % c;
  S[t] = 0.5 * (Bc[(int64_t)cidx[k] * nf + node[r]] + Bc[(int64_t)cidx[r] * nf + node[k]]);
}

// out[r] = sum_k M[k + r c] in[k] over k <= r (kPrefix) or k >= r, three columns:
// one warp per output row, reading column r of M contiguously.  With M = Q^T
// (prefix) this is Q in for lower-triangular Q; with M = Q (suffix), Q^T in.
template <bool kPrefix>
__global__ void tri_matvec_kernel(const double* M, int64_t c, const double* in, double* out) {
  const int64_t r = ((int64_t)blockIdx.x * kT + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (r >= c) return;
  const int64_t k0 = kPrefix ? 0 : r, k1 = kPrefix ? r + 1 : c;
  const double* col = M + r * c;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t k = k0 + lane; k < k1; k += 32) {
    const double q = col[k];
    a0 += q * in[3 * k];
    a1 += q * in[3 * k + 1];
    a2 += q * in[3 * k + 2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
    a1 += __shfl_down_sync(0xffffffffu, a1, o);
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) {
    out[3 * r] = a0;
    out[3 * r + 1] = a1;
    out[3 * r + 2] = a2;
  }
}

// x[i] = a1[i] - sum_k Bc[cidx[k]][i] lambda[k] for the free nodes i; the
// multipliers pass through shared memory in chunks
constexpr int kChunk = 512;
__global__ void correct_kernel(int64_t nf, const double* Bc, const int32_t* cidx, int64_t c, const double* lam,
                               const double* a1, double* x) {
  __shared__ double sl[kChunk][3];
  __shared__ int32_t sc[kChunk];
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  double x0 = 0, x1 = 0, x2 = 0;
  for (int64_t k0 = 0; k0 < c; k0 += kChunk) {
    const int64_t kn = c - k0 < kChunk ? c - k0 : kChunk;
    __syncthreads();
    for (int64_t k = threadIdx.x; k < kn; k += kT) {
      sl[k][0] = lam[3 * (k0 + k)];
      sl[k][1] = lam[3 * (k0 + k) + 1];
      sl[k][2] = lam[3 * (k0 + k) + 2];
      sc[k] = cidx[k0 + k];
    }
    __syncthreads();
    if (i < nf) {
      for (int64_t k = 0; k < kn; ++k) {
        const double bv = Bc[(int64_t)sc[k] * nf + i];
        x0 += bv * sl[k][0];
        x1 += bv * sl[k][1];
        x2 += bv * sl[k][2];
      }
    }
  }
  if (i < nf) {
    x[3 * i] = a1[3 * i] - x0;
    x[3 * i + 1] = a1[3 * i + 1] - x1;
    x[3 * i + 2] = a1[3 * i + 2] - x2;
  }
}

// x[node[k]] = xstar[k]
__global__ void set_targets_kernel(const int32_t* node, int64_t c, const double* xstar, double* x) {
  const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (k >= c) return;
  const int64_t g = 3 * (int64_t)node[k];
  x[g] = xstar[3 * k];
  x[g + 1] = xstar[3 * k + 1];
  x[g + 2] = xstar[3 * k + 2];
}

// out[k] = a[rows[k]] (3 values per row)
__global__ void pack_rows_kernel(const int32_t* rows, int64_t c, const double* a, double* out) {
  const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (k >= c) return;
  const int64_t g = 3 * (int64_t)rows[k];
  out[3 * k] = a[g];
  out[3 * k + 1] = a[g + 1];
  out[3 * k + 2] = a[g + 2];
}

// Adjoint of the targets (Alg. 5): with z_C = 0, dL/dx*_j = gbar_j - (H z)_j for
// every held node j, gbar = ax + av/h, chained into (x_t, v_t) of that node.
//   ray  x* = x_t + s v_t, s = z_t / (-v_z):  the height of x* is identically 0;
//        ds/dz_t = -1/v_z, ds/dv_z = -s/v_z, so with w = -(g_x v_x + g_y v_y)/v_z
//        dL/dx_t = (g_x, g_y, w), dL/dv_t = s (g_x, g_y, w)
//   drop x* = (x_t, y_t, 0):  dL/dx_t = (g_x, g_y, 0), dL/dv_t = 0
__global__ void target_vjp_kernel(const int32_t* node, const uint8_t* ray, int64_t c, const double* xt,
                                  const double* vt, const double* ax, const double* av, const double* Hz,
                                  double inv_h, double* gx, double* gv) {
  const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (k >= c) return;
  const int64_t j = 3 * (int64_t)node[k];
  const double g0 = ax[j] + av[j] * inv_h - Hz[j];
  const double g1 = ax[j + 1] + av[j + 1] * inv_h - Hz[j + 1];
  double dx2 = 0, s = 0;
  if (ray[k]) {
    const double vz = vt[j + 2];
    s = xt[j + 2] / (-vz);
    dx2 = -(g0 * vt[j] + g1 * vt[j + 1]) / vz;
  }
  gx[3 * k] = g0;
  gx[3 * k + 1] = g1;
  gx[3 * k + 2] = dx2;
  gv[3 * k] = s * g0;
  gv[3 * k + 1] = s * g1;
  gv[3 * k + 2] = s * dx2;
}

// ax[node[k]] += gx[k], av[node[k]] += gv[k]
__global__ void add_rows_kernel(const int32_t* node, int64_t c, const double* gx, const double* gv, double* ax,
                                double* av) {
  const int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (k >= c) return;
  const int64_t j = 3 * (int64_t)node[k];
  for (int d = 0; d < 3; ++d) {
    ax[j + d] += gx[3 * k + d];
    av[j + d] += gv[3 * k + d];
  }
}

unsigned blocks(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

}  // namespace

cudaError_t contact_unit_rhs(int64_t nf, const int32_t* cand, int64_t k0, int count, double* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b, 0, sizeof(double) * 3 * nf, s);
  if (e != cudaSuccess) return e;
  unit_rhs_kernel<<<1, 32, 0, s>>>(cand, k0, count, b);
  return cudaGetLastError();
}

cudaError_t contact_extract_columns(int64_t nf, const double* x, int64_t k0, int count, double* Bc,
                                    cudaStream_t s) {
  extract_columns_kernel<<<blocks(nf), kT, 0, s>>>(nf, x, k0, count, Bc);
  return cudaGetLastError();
}

cudaError_t contact_gather_S(int64_t nf, const double* Bc, const int32_t* node, const int32_t* cidx, int64_t c,
                             double* S, cudaStream_t s) {
  if (c == 0) return cudaSuccess;
  gather_S_kernel<<<blocks(c * c), kT, 0, s>>>(nf, Bc, node, cidx, c, S);
  return cudaGetLastError();
}

cudaError_t contact_correct(int64_t nf, const double* Bc, const int32_t* node, const int32_t* cidx, int64_t c,
                            const double* Q, const double* QT, double* abuf, double* ubuf, double* lam,
                            const double* a1, const double* xstar, double* x, cudaStream_t s) {
  if (c > 0) {
    pack_rows_kernel<<<blocks(c), kT, 0, s>>>(node, c, a1, abuf);
    tri_matvec_kernel<true><<<blocks(32 * c), kT, 0, s>>>(QT, c, abuf, ubuf);
    tri_matvec_kernel<false><<<blocks(32 * c), kT, 0, s>>>(Q, c, ubuf, lam);
  }
  correct_kernel<<<blocks(nf), kT, 0, s>>>(nf, Bc, cidx, c, lam, a1, x);
  if (c > 0) set_targets_kernel<<<blocks(c), kT, 0, s>>>(node, c, xstar, x);
  return cudaGetLastError();
}

cudaError_t contact_pack_rows(const int32_t* rows, int64_t c, const double* a, double* out, cudaStream_t s) {
  if (c == 0) return cudaSuccess;
  pack_rows_kernel<<<blocks(c), kT, 0, s>>>(rows, c, a, out);
  return cudaGetLastError();
}

cudaError_t contact_set_targets(const int32_t* node, int64_t c, const double* xstar, double* x, cudaStream_t s) {
  if (c == 0) return cudaSuccess;
  set_targets_kernel<<<blocks(c), kT, 0, s>>>(node, c, xstar, x);
  return cudaGetLastError();
}

cudaError_t contact_target_vjp(const int32_t* node, const uint8_t* ray, int64_t c, const double* xt,
                               const double* vt, const double* ax, const double* av, const double* Hz, double inv_h,
                               double* gx, double* gv, cudaStream_t s) {
  if (c == 0) return cudaSuccess;
  target_vjp_kernel<<<blocks(c), kT, 0, s>>>(node, ray, c, xt, vt, ax, av, Hz, inv_h, gx, gv);
  return cudaGetLastError();
}

cudaError_t contact_add_rows(const int32_t* node, int64_t c, const double* gx, const double* gv, double* ax,
                             double* av, cudaStream_t s) {
  if (c == 0) return cudaSuccess;
  add_rows_kernel<<<blocks(c), kT, 0, s>>>(node, c, gx, gv, ax, av);
  return cudaGetLastError();
}

}  // namespace pd
