// One-time numeric factorisation of the PD matrix on the device (FP64).
//
// Sec. 3: A = M/h^2 + sum_c w_c G_c^T G_c is constant and SPD, so its Cholesky
// factor is computed once and every global step is a back-substitution.
// A = I_3 (x) L_A, so only the scalar free-node matrix L_A is factored.
//
// Method (this implementation's design, not the paper's Eigen call):
// multifrontal supernodal Cholesky over the nested-dissection tree.  For every
// supernode s the dense front (nr x nr, column-major, lower triangle) is
//   assembled from L_A entries of its columns + the update matrices of its
//   children (extend-add in ascending child order, no atomics),
//   partially factored on its nc pivot columns with a blocked right-looking
//   Cholesky (NB = 32 diagonal blocks, row-parallel panel solves, 64x64-tile
//   Schur updates),
// level by level from the leaves.  Finally every panel [L11; L21] is turned into
// the solve panel Q = [L11^-1; L21 L11^-1] by the right triangular solve
// Q L11 = [I; L21], so each supernode's forward and backward substitution
// becomes a dense matrix-vector product that all SMs can share.
#include <algorithm>
#include <cmath>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int NB = 32;
constexpr int TILE = 64;

struct AsmParams {
  int64_t nnz;
  const int64_t* target;
  const int64_t* cptr;
  const int32_t* contrib;
  const int32_t* diag_node;
  const double *wc, *wv, *wm, *fiber;
  const double* mass;
  const uint8_t* contact;
  double inv_h2, k;
  double Kref[64];
  double gN[8][8][3];   // dN_a/dX at Gauss point q: gN[q][a][d]
  double Vq;
  // unstructured tetrahedra: per-element barycentric gradients (12, vertex-major) and
  // volumes in place of the voxel rule's reference matrix Kref
  const double *tet_grad, *tet_vol;
  double* front;
};

__global__ void assemble_la_kernel(AsmParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.nnz) return;
  double v = 0.0;
  for (int64_t c = p.cptr[i]; c < p.cptr[i + 1]; ++c) {
    const int32_t code = p.contrib[c];
    const int32_t e = code >> 6, a = (code >> 3) & 7, b = code & 7;
    const double w = (p.wc ? p.wc[e] : 0.0) + (p.wv ? p.wv[e] : 0.0);
    if (p.tet_grad) {
      // V_e w grad N_a . grad N_b (one point per tetrahedron; a, b < 4)
      const double* ga = p.tet_grad + 12 * (int64_t)e + 3 * a;
      const double* gb = p.tet_grad + 12 * (int64_t)e + 3 * b;
      v += w * p.tet_vol[e] * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
    } else {
      v += w * p.Kref[a * 8 + b];
    }
    if (p.wm && p.wm[e] != 0.0) {
      const double m0 = p.fiber[3 * e], m1 = p.fiber[3 * e + 1], m2 = p.fiber[3 * e + 2];
      double s = 0.0;
      for (int q = 0; q < 8; ++q) {
        const double ga = p.gN[q][a][0] * m0 + p.gN[q][a][1] * m1 + p.gN[q][a][2] * m2;
        const double gb = p.gN[q][b][0] * m0 + p.gN[q][b][1] * m1 + p.gN[q][b][2] * m2;
        s += ga * gb;
      }
      v += p.wm[e] * p.Vq * s;
    }
  }
  const int32_t dn = p.diag_node[i];
  if (dn >= 0) {
    v += p.mass[dn] * p.inv_h2;
    if (p.contact && p.contact[dn]) v += p.k;
  }
  p.front[p.target[i]] = v;
}

struct TreeView {
  const int64_t *level_list, *snode_first, *row_ptr, *front_off, *child_ptr, *child_list,
      *rel_ptr, *panel_off;
  const int32_t* rel;
  double* front;
};

__device__ __forceinline__ int64_t snr(const TreeView& t, int64_t s) { return t.row_ptr[s + 1] - t.row_ptr[s]; }
__device__ __forceinline__ int64_t snc(const TreeView& t, int64_t s) { return t.snode_first[s + 1] - t.snode_first[s]; }

// front(s) += update matrix of its ci-th child, mapped through rel
__global__ void extend_add_kernel(TreeView t, int64_t list_off, int ci) {
  const int64_t s = t.level_list[list_off + blockIdx.y];
  if (t.child_ptr[s + 1] - t.child_ptr[s] <= ci) return;
  const int64_t c = t.child_list[t.child_ptr[s] + ci];
  const int64_t nrc = snr(t, c), ncc = snc(t, c), nb = nrc - ncc;
  const double* U = t.front + t.front_off[c] + ncc + ncc * nrc;
  const int32_t* rl = t.rel + t.rel_ptr[c];
  double* F = t.front + t.front_off[s];
  const int64_t nrs = snr(t, s);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nb * nb;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / nb, i = idx - j * nb;
    if (i < j) continue;
    F[rl[i] + (int64_t)rl[j] * nrs] += U[i + j * nrc];
  }
}

// Cholesky of the kb-th diagonal block of every front of the level.
__global__ void potrf_diag_kernel(TreeView t, int64_t list_off, int kb, int* flags) {
  const int64_t s = t.level_list[list_off + blockIdx.x];
  const int64_t nc = snc(t, s), nr = snr(t, s);
  const int64_t k0 = (int64_t)kb * NB;
  if (k0 >= nc) return;
  const int nb = (int)min((int64_t)NB, nc - k0);
  double* A = t.front + t.front_off[s] + k0 + k0 * nr;
  __shared__ double L[NB][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    L[i][j] = (i < nb && j < nb && i >= j) ? A[i + (int64_t)j * nr] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = L[j][j];
      if (!(d > 0.0)) {
        atomicOr(flags, DEV_ERR_NOT_SPD);
        d = 1.0;
      }
      L[j][j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) L[i][j] /= L[j][j];
    __syncthreads();
    const int m = nb - j - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = j + 1 + idx % m, k = j + 1 + idx / m;
      if (i >= k) L[i][k] -= L[i][j] * L[k][j];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, j = idx / nb;
    if (i >= j) A[i + (int64_t)j * nr] = L[i][j];
  }
}

// rows below the diagonal block: A[i, blk] <- A[i, blk] L_D^-T
__global__ void trsm_panel_kernel(TreeView t, int64_t list_off, int kb) {
  const int64_t s = t.level_list[list_off + blockIdx.y];
  const int64_t nc = snc(t, s), nr = snr(t, s);
  const int64_t k0 = (int64_t)kb * NB;
  if (k0 >= nc) return;
  const int nb = (int)min((int64_t)NB, nc - k0);
  double* F = t.front + t.front_off[s];
  __shared__ double L[NB][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    L[i][j] = (i < nb && j < nb && i >= j) ? F[(k0 + i) + (k0 + j) * nr] : 0.0;
  }
  __syncthreads();
  const int64_t i = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  double x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) x[j] = j < nb ? F[i + (k0 + j) * nr] : 0.0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < nb) {
      double v = x[j];
#pragma unroll
      for (int l = 0; l < NB; ++l)
        if (l < j) v -= x[l] * L[j][l];
      x[j] = v / L[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nb) F[i + (k0 + j) * nr] = x[j];
}

__device__ __forceinline__ void tri_index(int64_t idx, int64_t& ti, int64_t& tj) {
  // idx -> (ti, tj), ti >= tj, row-major over the lower triangle
  int64_t r = (int64_t)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= idx) ++r;
  while (r * (r + 1) / 2 > idx) --r;
  ti = r;
  tj = idx - r * (r + 1) / 2;
}

// trailing update: A[i, j] -= sum_l A[i, k0+l] A[j, k0+l], i >= j >= k1
__global__ void __launch_bounds__(256) syrk_update_kernel(TreeView t, int64_t list_off, int kb) {
  const int64_t s = t.level_list[list_off + blockIdx.y];
  const int64_t nc = snc(t, s), nr = snr(t, s);
  const int64_t k0 = (int64_t)kb * NB;
  if (k0 >= nc) return;
  const int nb = (int)min((int64_t)NB, nc - k0);
  const int64_t k1 = k0 + nb;
  const int64_t ntr = (nr - k1 + TILE - 1) / TILE;
  if ((int64_t)blockIdx.x >= ntr * (ntr + 1) / 2) return;
  int64_t ti, tj;
  tri_index(blockIdx.x, ti, tj);
  const int64_t r0 = k1 + ti * TILE, c0 = k1 + tj * TILE;
  double* F = t.front + t.front_off[s];
  __shared__ double Ai[TILE][NB + 1];
  __shared__ double Aj[TILE][NB + 1];
  for (int idx = threadIdx.x; idx < TILE * NB; idx += blockDim.x) {
    const int r = idx % TILE, l = idx / TILE;
    Ai[r][l] = (l < nb && r0 + r < nr) ? F[(r0 + r) + (k0 + l) * nr] : 0.0;
    Aj[r][l] = (l < nb && c0 + r < nr) ? F[(c0 + r) + (k0 + l) * nr] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int l = 0; l < nb; ++l) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a[u] = Ai[tx + 16 * u][l]; b[u] = Aj[ty + 16 * u][l]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[u][w] += a[u] * b[w];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int64_t row = r0 + tx + 16 * u, col = c0 + ty + 16 * w;
      if (row < nr && col < nr && row >= col) F[row + col * nr] -= acc[u][w];
    }
}

// Q_s = [I; L21] (nr x nc, column-major) from the factored front
__global__ void init_Q_kernel(TreeView t, double* Q, int64_t list_off) {
  const int64_t s = t.level_list[list_off + blockIdx.y];
  const int64_t nc = snc(t, s), nr = snr(t, s);
  const double* F = t.front + t.front_off[s];
  double* Qs = Q + t.panel_off[s];
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nr * nc;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / nr, i = idx - j * nr;
    Qs[idx] = i < nc ? (i == j ? 1.0 : 0.0) : F[i + j * nr];
  }
}

// Right solve on column block jb (counted from the right, rb): X[:, blk] <- X[:, blk] L_D^-1
__global__ void trsm_right_diag_kernel(TreeView t, double* Q, int64_t list_off, int rb) {
  const int64_t s = t.level_list[list_off + blockIdx.y];
  const int64_t nc = snc(t, s), nr = snr(t, s);
  const int64_t nblk = (nc + NB - 1) / NB;
  const int64_t jb = nblk - 1 - rb;
  if (jb < 0) return;
  const int64_t j0 = jb * NB;
  const int nb = (int)min((int64_t)NB, nc - j0);
  const double* F = t.front + t.front_off[s];
  __shared__ double L[NB][NB + 1];
  for (int idx = threadIdx.x; idx < NB * NB; idx += blockDim.x) {
    const int i = idx % NB, j = idx / NB;
    L[i][j] = (i < nb && j < nb && i >= j) ? F[(j0 + i) + (j0 + j) * nr] : 0.0;
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nr) return;
  double* Qs = Q + t.panel_off[s];
  double x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) x[j] = j < nb ? Qs[i + (j0 + j) * nr] : 0.0;
  // x L_D = b  ->  x_k = (b_k - sum_{l > k} x_l L[l][k]) / L[k][k]
#pragma unroll
  for (int k = NB - 1; k >= 0; --k) {
    if (k < nb) {
      double v = x[k];
#pragma unroll
      for (int l = 0; l < NB; ++l)
        if (l > k && l < nb) v -= x[l] * L[l][k];
      x[k] = v / L[k][k];
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nb) Qs[i + (j0 + j) * nr] = x[j];
}

// X[:, 0:j0] -= X[:, blk] L11[blk, 0:j0]
__global__ void __launch_bounds__(256) gemm_right_update_kernel(TreeView t, double* Q,
                                                                int64_t list_off, int rb) {
  const int64_t s = t.level_list[list_off + blockIdx.z];
  const int64_t nc = snc(t, s), nr = snr(t, s);
  const int64_t nblk = (nc + NB - 1) / NB;
  const int64_t jb = nblk - 1 - rb;
  if (jb <= 0) return;
  const int64_t j0 = jb * NB;
  const int nb = (int)min((int64_t)NB, nc - j0);
  const int64_t rt = blockIdx.x, ct = blockIdx.y;
  if (rt * TILE >= nr || ct * TILE >= j0) return;
  const int64_t r0 = rt * TILE, c0 = ct * TILE;
  const double* F = t.front + t.front_off[s];
  double* Qs = Q + t.panel_off[s];
  __shared__ double Xs[TILE][NB + 1];
  __shared__ double Ls[NB][TILE + 1];
  for (int idx = threadIdx.x; idx < TILE * NB; idx += blockDim.x) {
    const int r = idx % TILE, l = idx / TILE;
    Xs[r][l] = (l < nb && r0 + r < nr) ? Qs[(r0 + r) + (j0 + l) * nr] : 0.0;
    const int cc = idx % TILE, ll = idx / TILE;
    Ls[ll][cc] = (ll < nb && c0 + cc < j0) ? F[(j0 + ll) + (c0 + cc) * nr] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int l = 0; l < nb; ++l) {
    double a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { a[u] = Xs[tx + 16 * u][l]; b[u] = Ls[l][ty + 16 * u]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[u][w] += a[u] * b[w];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int64_t row = r0 + tx + 16 * u, col = c0 + ty + 16 * w;
      if (row < nr && col < j0) Qs[row + col * nr] -= acc[u][w];
    }
}

__global__ void to_float_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void nan_scan_kernel(const double* a, int64_t n, int* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) { atomicOr(flags, DEV_ERR_NAN); return; }
}

// QT = Q^T for a c x c column-major matrix (32 x 32 tiles through shared memory)
__global__ void transpose_kernel(const double* Q, int64_t c, double* QT) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + threadIdx.x, j = j0 + r;
    t[r][threadIdx.x] = (i < c && j < c) ? Q[i + j * c] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + threadIdx.x, i = i0 + r;
    if (i < c && j < c) QT[j + i * c] = t[threadIdx.x][r];
  }
}

}  // namespace

// Dense SPD matrix as a tree of one supernode (nr = nc = c, no children): the
// same blocked Cholesky and right solve as the fronts, giving Q = L^-1.
pd_status dense_cholesky_inverse(double* S, int64_t c, double* Q, double* QT, int64_t* meta, int* flags,
                                 cudaStream_t st) {
  if (c <= 0) return PD_OK;
  // level_list = front_off = panel_off = {0}; snode_first = row_ptr = {0, c}; child_ptr = {0, 0}
  const int64_t host_meta[4] = {0, c, 0, 0};
  PD_CUDA_TRY(cudaMemcpyAsync(meta, host_meta, sizeof(host_meta), cudaMemcpyHostToDevice, st));
  PD_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), st));
  TreeView tv{meta, meta, meta, meta, meta + 2, nullptr, meta, meta, nullptr, S};
  const int nkb = (int)((c + NB - 1) / NB);
  for (int kb = 0; kb < nkb; ++kb) {
    potrf_diag_kernel<<<1, 256, 0, st>>>(tv, 0, kb, flags);
    const int64_t rows = std::max<int64_t>(c - (int64_t)kb * NB, 1);
    trsm_panel_kernel<<<dim3((unsigned)((rows + 127) / 128), 1), 128, 0, st>>>(tv, 0, kb);
    const int64_t ntr = (rows + TILE - 1) / TILE;
    syrk_update_kernel<<<dim3((unsigned)std::max<int64_t>(ntr * (ntr + 1) / 2, 1), 1), 256, 0, st>>>(tv, 0, kb);
    PD_CUDA_TRY(cudaGetLastError());
  }
  init_Q_kernel<<<dim3((unsigned)std::min<int64_t>((c * c + 255) / 256, 2048), 1), 256, 0, st>>>(tv, Q, 0);
  const int64_t row_tiles = (c + TILE - 1) / TILE;
  for (int rb = 0; rb < nkb; ++rb) {
    trsm_right_diag_kernel<<<dim3((unsigned)((c + 127) / 128), 1), 128, 0, st>>>(tv, Q, 0, rb);
    const int64_t j0max = (int64_t)(nkb - 1 - rb) * NB;
    if (j0max > 0) {
      gemm_right_update_kernel<<<dim3((unsigned)row_tiles, (unsigned)((j0max + TILE - 1) / TILE), 1), 256, 0, st>>>(
          tv, Q, 0, rb);
    }
    PD_CUDA_TRY(cudaGetLastError());
  }
  const unsigned tb = (unsigned)((c + 31) / 32);
  transpose_kernel<<<dim3(tb, tb), dim3(32, 8), 0, st>>>(Q, c, QT);
  nan_scan_kernel<<<256, 256, 0, st>>>(Q, c * c, flags);
  PD_CUDA_TRY(cudaGetLastError());
  return PD_OK;
}

pd_status factorize_device(MeshImpl* m, cudaStream_t st) {
  const HostMesh& h = m->h;
  double* front = nullptr;
  PD_CUDA_TRY(cudaMallocAsync((void**)&front, sizeof(double) * (size_t)h.front_entries(), st));
  PD_CUDA_TRY(cudaMemsetAsync(front, 0, sizeof(double) * (size_t)h.front_entries(), st));
  PD_CUDA_TRY(cudaMemsetAsync(m->ws.flags, 0, sizeof(int), st));

  // ---- assembly of L_A into the fronts
  AsmParams ap{};
  ap.nnz = (int64_t)h.la_target.size();
  ap.target = m->la_target;
  ap.cptr = m->la_cptr;
  ap.contrib = m->la_contrib;
  ap.diag_node = m->la_diag_node;
  ap.wc = m->wc; ap.wv = m->wv; ap.wm = m->wm; ap.fiber = m->fiber;
  ap.mass = m->mass;
  ap.contact = m->contact;
  ap.inv_h2 = 1.0 / (m->h_step * m->h_step);
  ap.k = m->k_contact;
  ap.Vq = h.dx * h.dx * h.dx / (h.rule == PD_ELEM_TET6 ? 6.0 : 8.0);
  if (h.rule == PD_ELEM_TET6) {
    // tetrahedron q < 6: the path from corner 0 along axes p1, p2, p3 to corner 7;
    // barycentric gradients (-e_p1, e_p1 - e_p2, e_p2 - e_p3, e_p3) / dx at its four
    // corners, zero elsewhere; points 6 and 7 unused (zero)
    for (int q = 0; q < 8; ++q)
      for (int a = 0; a < 8; ++a)
        for (int d = 0; d < 3; ++d) ap.gN[q][a][d] = 0.0;
    for (int q = 0; q < 6; ++q) {
      const int p1 = q >> 1, lo = p1 == 0 ? 1 : 0, hi = p1 == 2 ? 1 : 2;
      const int p2 = (q & 1) ? hi : lo, p3 = 3 - p1 - p2;
      const int c1 = 4 >> p1, c2 = c1 + (4 >> p2);
      const double s = 1.0 / h.dx;
      ap.gN[q][0][p1] -= s;
      ap.gN[q][c1][p1] += s;
      ap.gN[q][c1][p2] -= s;
      ap.gN[q][c2][p2] += s;
      ap.gN[q][c2][p3] -= s;
      ap.gN[q][7][p3] += s;
    }
  } else {
    const double g = 1.0 / std::sqrt(3.0);
    for (int q = 0; q < 8; ++q)
      for (int a = 0; a < 8; ++a)
        for (int d = 0; d < 3; ++d) {
          double prod = 1.0 / h.dx;
          for (int dd = 0; dd < 3; ++dd) {
            if (dd == d) continue;
            const int ba = (a >> (2 - dd)) & 1, bq = (q >> (2 - dd)) & 1;
            prod *= (ba == bq) ? 0.5 * (1 + g) : 0.5 * (1 - g);
          }
          ap.gN[q][a][d] = ((a >> (2 - d)) & 1) ? prod : -prod;
        }
  }
  {
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) {
        double s = 0;
        for (int q = 0; q < 8; ++q)
          for (int d = 0; d < 3; ++d) s += ap.gN[q][a][d] * ap.gN[q][b][d];
        ap.Kref[a * 8 + b] = ap.Vq * s;
      }
  }
  if (h.rule == PD_ELEM_TETU) {
    ap.tet_grad = m->tet_grad;
    ap.tet_vol = m->tet_vol;
  }
  ap.front = front;
  if (ap.nnz > 0) {
    assemble_la_kernel<<<(unsigned)((ap.nnz + 255) / 256), 256, 0, st>>>(ap);
    PD_CUDA_TRY(cudaGetLastError());
  }

  TreeView tv{m->level_list, m->snode_first, m->row_ptr, m->front_off, m->child_ptr, m->child_list,
              m->rel_ptr, m->panel_off, m->rel, front};

  // ---- level-by-level partial factorisation
  for (const FactorLevel& L : m->flevels) {
    for (int ci = 0; ci < L.max_children; ++ci) {
      const int64_t blocks = std::min<int64_t>(std::max<int64_t>((L.max_child_nb2 + 255) / 256, 1), 4096);
      dim3 grid((unsigned)blocks, (unsigned)L.count);
      extend_add_kernel<<<grid, 256, 0, st>>>(tv, L.list_off, ci);
      PD_CUDA_TRY(cudaGetLastError());
    }
    const int nkb = (int)((L.max_nc + NB - 1) / NB);
    for (int kb = 0; kb < nkb; ++kb) {
      potrf_diag_kernel<<<(unsigned)L.count, 256, 0, st>>>(tv, L.list_off, kb, m->ws.flags);
      const int64_t k1 = (int64_t)kb * NB;   // rows below the block start after k1 + nb
      const int64_t rows = std::max<int64_t>(L.max_nr - k1, 1);
      dim3 g2((unsigned)((rows + 127) / 128), (unsigned)L.count);
      trsm_panel_kernel<<<g2, 128, 0, st>>>(tv, L.list_off, kb);
      const int64_t ntr = (rows + TILE - 1) / TILE;
      dim3 g3((unsigned)std::max<int64_t>(ntr * (ntr + 1) / 2, 1), (unsigned)L.count);
      syrk_update_kernel<<<g3, 256, 0, st>>>(tv, L.list_off, kb);
      PD_CUDA_TRY(cudaGetLastError());
    }
  }

  // ---- solve panels Q = [L11^-1; L21 L11^-1] via Q L11 = [I; L21], per level
  for (const FactorLevel& L : m->flevels) {
    {
      dim3 g((unsigned)std::min<int64_t>(std::max<int64_t>((L.max_nr * L.max_nc + 255) / 256, 1), 2048),
             (unsigned)L.count);
      init_Q_kernel<<<g, 256, 0, st>>>(tv, m->Q64, L.list_off);
      PD_CUDA_TRY(cudaGetLastError());
    }
    const int maxblk = (int)((L.max_nc + NB - 1) / NB);
    const int64_t row_tiles = (L.max_nr + TILE - 1) / TILE;
    for (int rb = 0; rb < maxblk; ++rb) {
      dim3 g1((unsigned)((L.max_nr + 127) / 128), (unsigned)L.count);
      trsm_right_diag_kernel<<<g1, 128, 0, st>>>(tv, m->Q64, L.list_off, rb);
      // the largest remaining left block of any panel is j0 = (nblk - 1 - rb) * NB
      const int64_t j0max = std::max<int64_t>((int64_t)(maxblk - 1 - rb) * NB, 0);
      if (j0max > 0) {
        dim3 g2((unsigned)row_tiles, (unsigned)((j0max + TILE - 1) / TILE), (unsigned)L.count);
        gemm_right_update_kernel<<<g2, 256, 0, st>>>(tv, m->Q64, L.list_off, rb);
      }
      PD_CUDA_TRY(cudaGetLastError());
    }
  }
  const int64_t nnz = h.factor_nnz();
  nan_scan_kernel<<<1024, 256, 0, st>>>(m->Q64, nnz, m->ws.flags);
  if (m->Q32) {
    to_float_kernel<<<2048, 256, 0, st>>>(m->Q64, m->Q32, nnz);
    PD_CUDA_TRY(cudaGetLastError());
    PD_CUDA_TRY(pack_solve_stream(m, st));   // the FP32 solve's tile-contiguous copy
  }
  PD_CUDA_TRY(cudaFreeAsync(front, st));
  int flags = 0;
  PD_CUDA_TRY(cudaMemcpyAsync(&flags, m->ws.flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  PD_CUDA_TRY(cudaStreamSynchronize(st));
  if (flags & DEV_ERR_NOT_SPD) {
    set_error("pd_factorize: non-positive pivot (A is not SPD)");
    return PD_ERR_NOT_SPD;
  }
  if (flags & DEV_ERR_NAN) {
    set_error("pd_factorize: non-finite entry in the factor");
    return PD_ERR_NAN;
  }
  return PD_OK;
}

}  // namespace pd
