// Per-Gauss-point math of the local steps: 3x3 SVD, PD projections (supplement,
// "Energy Definitions") and the action of their Jacobians (Sec. 4, Eqn 21).
//
// Everything is written for relative accuracy at small strain, so that the FP32
// local step resolves stresses to FP32 precision relative to the strain rather
// than to |F| ~ 1:
//   * the input is the displacement gradient H = F - I, not F;
//   * the SVD runs cyclic Jacobi (Golub & Van Loan, symmetric Schur
//     decomposition) on the Green-strain matrix E = F^T F - I = H + H^T + H^T H,
//     whose eigenvalues e_i give sigma_i - 1 = e_i / (1 + sqrt(1 + e_i)) without
//     cancellation; U follows from a Givens QR of F V (McAdams et al. 2011 use the
//     same Jacobi-then-QR structure);
//   * stresses are formed as R V diag(.) V^T (polar form), never as F - P.
#pragma once

#include <cuda_runtime.h>

namespace pd {

template <typename T> __device__ __forceinline__ T tsqrt(T x);
template <> __device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ T tlog1p(T x);
template <> __device__ __forceinline__ float tlog1p<float>(float x) { return log1pf(x); }
template <> __device__ __forceinline__ double tlog1p<double>(double x) { return log1p(x); }
template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float v = 1.1920929e-7f; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

// One Jacobi rotation annihilating S[p][q]; r is the remaining index.  Written
// without branches: with d = (S_qq - S_pp)/2 the tangent of the rotation angle is
// t = sign(d) S_pq / (|d| + sqrt(d^2 + S_pq^2)) (sign(0) = +1), which is 0 when
// S_pq = 0 and 1 (45 degrees) when d = 0 (Golub & Van Loan, symmetric Schur).
template <typename T, int p, int q, int r>
__device__ __forceinline__ void jacobi_rot(T (&S)[3][3], T (&V)[3][3]) {
  const T apq = S[p][q];
  const T d = T(0.5) * (S[q][q] - S[p][p]);
  const T den = fabs(d) + tsqrt<T>(d * d + apq * apq);
  const T t = den > T(0) ? (d >= T(0) ? apq : -apq) / den : T(0);
  const T c = T(1) / tsqrt<T>(T(1) + t * t);
  const T s = t * c;
  const T arp = S[r][p], arq = S[r][q];
  S[p][p] -= t * apq;
  S[q][q] += t * apq;
  S[p][q] = S[q][p] = T(0);
  const T nrp = c * arp - s * arq, nrq = s * arp + c * arq;
  S[r][p] = S[p][r] = nrp;
  S[r][q] = S[q][r] = nrq;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T vp = V[i][p], vq = V[i][q];
    V[i][p] = c * vp - s * vq;
    V[i][q] = s * vp + c * vq;
  }
}

// Givens rotation of rows (i, k) of B zeroing B[k][j]; accumulates U <- U G^T.
template <typename T, int i, int k, int j>
__device__ __forceinline__ void givens_qr(T (&B)[3][3], T (&U)[3][3]) {
  const T a = B[i][j], b = B[k][j];
  const T rr = tsqrt<T>(a * a + b * b);
  const T inv = rr > T(0) ? T(1) / rr : T(0);
  const T c = rr > T(0) ? a * inv : T(1);
  const T s = b * inv;
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const T bi = B[i][col], bk = B[k][col];
    B[i][col] = c * bi + s * bk;
    B[k][col] = -s * bi + c * bk;
  }
  B[k][j] = T(0);
#pragma unroll
  for (int row = 0; row < 3; ++row) {
    const T ui = U[row][i], uk = U[row][k];
    U[row][i] = c * ui + s * uk;
    U[row][k] = -s * ui + c * uk;
  }
}

template <typename T>
struct SVD3 {
  T U[3][3], V[3][3];
  T sig[3];   // signed singular values, |sig| descending, sig[2] < 0 iff det F < 0
  T sm1[3];   // sig - 1, accurate at small strain
};

// Green strain E = F^T F - I = H + H^T + H^T H from H = F - I
template <typename S>
__device__ __forceinline__ void green_strain(const S (&H)[3][3], S (&E)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      S v = H[i][j] + H[j][i];
#pragma unroll
      for (int k = 0; k < 3; ++k) v += H[k][i] * H[k][j];
      E[i][j] = v;
    }
}

// SVD of F = I + H given H and its Green strain E (which svd3_from_H forms in T;
// a caller may form it in higher precision: under a large rotation H is of the
// order of the rotation angle while E is of the order of the strain, and the
// cancellation in H + H^T + H^T H then costs the bits that separate the two)
template <typename T>
__device__ __forceinline__ void svd3_from_HE(const T (&H)[3][3], const T (&Ein)[3][3], SVD3<T>& o) {
  T E[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) E[i][j] = Ein[i][j];
  T V[3][3] = {{T(1), T(0), T(0)}, {T(0), T(1), T(0)}, {T(0), T(0), T(1)}};
  const T nrm2 = E[0][0] * E[0][0] + E[1][1] * E[1][1] + E[2][2] * E[2][2] +
                 T(2) * (E[0][1] * E[0][1] + E[0][2] * E[0][2] + E[1][2] * E[1][2]);
  const T thr = nrm2 * Eps<T>::v * Eps<T>::v;
  // all lanes of a warp run the same number of sweeps (no divergence); a sweep
  // on an already diagonal matrix leaves it unchanged
  for (int sweep = 0; sweep < 12; ++sweep) {
    const T off = E[0][1] * E[0][1] + E[0][2] * E[0][2] + E[1][2] * E[1][2];
    if (!__any_sync(0xffffffffu, off > thr)) break;
    jacobi_rot<T, 0, 1, 2>(E, V);
    jacobi_rot<T, 0, 2, 1>(E, V);
    jacobi_rot<T, 1, 2, 0>(E, V);
  }
  T e[3] = {E[0][0], E[1][1], E[2][2]};
  // sort descending; each swap negates one column to keep det V = +1
  auto swapcol = [&](int a, int b) {
    T t = e[a]; e[a] = e[b]; e[b] = t;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T va = V[i][a];
      V[i][a] = V[i][b];
      V[i][b] = -va;
    }
  };
  if (e[0] < e[1]) swapcol(0, 1);
  if (e[0] < e[2]) swapcol(0, 2);
  if (e[1] < e[2]) swapcol(1, 2);
  // B = F V = V + H V
  T B[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T v = V[i][j];
#pragma unroll
      for (int k = 0; k < 3; ++k) v += H[i][k] * V[k][j];
      B[i][j] = v;
    }
  T U[3][3] = {{T(1), T(0), T(0)}, {T(0), T(1), T(0)}, {T(0), T(0), T(1)}};
  givens_qr<T, 0, 1, 0>(B, U);
  givens_qr<T, 0, 2, 0>(B, U);
  givens_qr<T, 1, 2, 1>(B, U);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o.sig[i] = B[i][i];
    if (B[i][i] > T(0)) {
      const T ei = e[i] > T(-1) ? e[i] : T(-1);
      o.sm1[i] = ei / (T(1) + tsqrt<T>(T(1) + ei));
    } else {
      o.sm1[i] = B[i][i] - T(1);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) { o.U[i][j] = U[i][j]; o.V[i][j] = V[i][j]; }
}

template <typename T>
__device__ __forceinline__ void svd3_from_H(const T (&H)[3][3], SVD3<T>& o) {
  T E[3][3];
  green_strain<T>(H, E);
  svd3_from_HE<T>(H, E, o);
}

// ---------------------------------------------------------------- polar refinement
// FP64 rotation of F = R S (S symmetric) from a rotation R0 accurate to FP32,
// without eigenvectors.  Two identities carry it:
//   * Newton-Schulz, R <- R (3 I - R^T R) / 2, squares the distance of R from the
//     orthogonal matrices (1e-7 -> 1e-14);
//   * for symmetric S and skew W = skew(w): W S + S W = skew((tr(S) I - S) w), so
//     the rotation R exp(W) that makes (R exp(W))^T F symmetric to first order has
//     w = 2 (tr(S0) I - S0)^-1 k with S0 = sym(R^T F), k = axial(skew(R^T F))
//     (tr(S0) I - S0 has the eigenvalues s_i + s_j > 0 of S0's pairs);
//     one step squares the error of R again.
// The same 3 x 3 solve gives the derivative of the polar rotation:
//   dR = R skew(w) with w = 2 (tr(S) I - S)^-1 axial(skew(R^T dF)).
__device__ __forceinline__ void skew_axial(const double (&A)[3][3], double (&k)[3]) {
  // axial vector of skew(A) = (A - A^T)/2: skew(k) has [2][1] = k0, [0][2] = k1, [1][0] = k2
  k[0] = 0.5 * (A[2][1] - A[1][2]);
  k[1] = 0.5 * (A[0][2] - A[2][0]);
  k[2] = 0.5 * (A[1][0] - A[0][1]);
}

// w = 2 (tr(S) I - S)^-1 k for symmetric S (returns false when the matrix is singular)
__device__ __forceinline__ bool polar_solve(const double (&S)[3][3], const double (&k)[3], double (&w)[3]) {
  const double t = S[0][0] + S[1][1] + S[2][2];
  const double a00 = t - S[0][0], a11 = t - S[1][1], a22 = t - S[2][2];
  const double a01 = -0.5 * (S[0][1] + S[1][0]), a02 = -0.5 * (S[0][2] + S[2][0]), a12 = -0.5 * (S[1][2] + S[2][1]);
  // adjugate of the symmetric matrix
  const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
  const double c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
  const double det = a00 * c00 + a01 * c01 + a02 * c02;
  if (!(fabs(det) > 1e-300)) {
    w[0] = w[1] = w[2] = 0.0;
    return false;
  }
  const double id = 2.0 / det;
  w[0] = id * (c00 * k[0] + c01 * k[1] + c02 * k[2]);
  w[1] = id * (c01 * k[0] + c11 * k[1] + c12 * k[2]);
  w[2] = id * (c02 * k[0] + c12 * k[1] + c22 * k[2]);
  return true;
}

// R <- R (I + skew(w) + skew(w)^2 / 2)
__device__ __forceinline__ void rotate_by(double (&R)[3][3], const double (&w)[3]) {
  const double W2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double G[3][3];
  G[0][0] = 1.0 + 0.5 * (w[0] * w[0] - W2);
  G[1][1] = 1.0 + 0.5 * (w[1] * w[1] - W2);
  G[2][2] = 1.0 + 0.5 * (w[2] * w[2] - W2);
  G[0][1] = -w[2] + 0.5 * w[0] * w[1];
  G[1][0] = w[2] + 0.5 * w[0] * w[1];
  G[0][2] = w[1] + 0.5 * w[0] * w[2];
  G[2][0] = -w[1] + 0.5 * w[0] * w[2];
  G[1][2] = -w[0] + 0.5 * w[1] * w[2];
  G[2][1] = w[0] + 0.5 * w[1] * w[2];
  double T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) T[i][j] = R[i][0] * G[0][j] + R[i][1] * G[1][j] + R[i][2] * G[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[i][j] = T[i][j];
}

// R from the FP32 rotation R0 and F = I + H (FP64), refined as above; S gets the
// symmetric factor R^T F.  Returns false if a solve was singular (inverted or
// degenerate elements).
__device__ __forceinline__ bool polar_refine(const float (&U)[3][3], const float (&V)[3][3], const double (&H)[3][3],
                                             double (&R)[3][3], double (&S)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      R[i][j] = (double)U[i][0] * (double)V[j][0] + (double)U[i][1] * (double)V[j][1] +
                (double)U[i][2] * (double)V[j][2];
  // Newton-Schulz
  double RtR[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) RtR[i][j] = R[0][i] * R[0][j] + R[1][i] * R[1][j] + R[2][i] * R[2][j];
  double T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      T[i][j] = 1.5 * R[i][j] - 0.5 * (R[i][0] * RtR[0][j] + R[i][1] * RtR[1][j] + R[i][2] * RtR[2][j]);
  // one polar correction: M = R^T F = R^T + R^T H
  double M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = T[j][i] + T[0][i] * H[0][j] + T[1][i] * H[1][j] + T[2][i] * H[2][j];
  double k[3], w[3];
  skew_axial(M, k);
  const bool ok = polar_solve(M, k, w);
  rotate_by(T, w);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[i][j] = T[i][j];
  // S = sym(R^T F)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = R[j][i] + R[0][i] * H[0][j] + R[1][i] * H[1][j] + R[2][i] * H[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) S[i][j] = 0.5 * (M[i][j] + M[j][i]);
  return ok;
}

// out += c * U diag(d) V^T   (c scalar)
template <typename T>
__device__ __forceinline__ void add_UdVt(T (&out)[3][3], const T (&U)[3][3], const T* d,
                                         const T (&V)[3][3], T c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      out[i][j] += c * (U[i][0] * d[0] * V[j][0] + U[i][1] * d[1] * V[j][1] + U[i][2] * d[2] * V[j][2]);
}

// out += c * U K V^T
template <typename T>
__device__ __forceinline__ void add_UKVt(T (&out)[3][3], const T (&U)[3][3], const T (&K)[3][3],
                                         const T (&V)[3][3], T c) {
  T KV[3][3];   // K V^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) KV[i][j] = K[i][0] * V[j][0] + K[i][1] * V[j][1] + K[i][2] * V[j][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) out[i][j] += c * (U[i][0] * KV[0][j] + U[i][1] * KV[1][j] + U[i][2] * KV[2][j]);
}

// M = U^T dF V
template <typename T>
__device__ __forceinline__ void rotate_in(const T (&U)[3][3], const T (&dF)[3][3], const T (&V)[3][3],
                                          T (&M)[3][3]) {
  T FV[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) FV[i][j] = dF[i][0] * V[0][j] + dF[i][1] * V[1][j] + dF[i][2] * V[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i][j] = U[0][i] * FV[0][j] + U[1][i] * FV[1][j] + U[2][i] * FV[2][j];
}

// Volume-preserving projection in singular-value space (supplement, volume
// energy): s = sigma + d*, d* = argmin |d|^2 s.t. prod s = 1.  The KKT
// conditions give d_i = -lam / s_i, i.e. s_i^2 - sigma_i s_i + lam = 0, so
// s_i(lam) = sigma_i (1 + sqrt(1 - 4 lam / sigma_i^2)) / 2 and lam solves the
// scalar equation sum_i log s_i(lam) = 0 (Newton from lam = 0).
// Returns false when some sigma_i <= 0 (inverted element).
template <typename T>
struct VolProj {
  T lam;
  T s[3];
  T gap[3];   // sigma_i - s_i = lam / s_i
  T a[3];     // 1 / (2 s_i - sigma_i)
};

// Must be called by all 32 lanes of the warp together (full-warp votes).  Lanes
// with active == false (or an inverted element) get a dummy result and false.
template <typename T>
__device__ __forceinline__ bool volume_project(const SVD3<T>& d, VolProj<T>& o, bool active) {
  const bool ok = active && d.sig[0] > T(0) && d.sig[1] > T(0) && d.sig[2] > T(0);
  const T sg[3] = {ok ? d.sig[0] : T(1), ok ? d.sig[1] : T(1), ok ? d.sig[2] : T(1)};
  const T sm[3] = {ok ? d.sm1[0] : T(0), ok ? d.sm1[1] : T(0), ok ? d.sm1[2] : T(0)};
  T lam = T(0);
  // the branch s_i(lam) exists for lam <= sigma_min^2 / 4: Newton steps that
  // overshoot it are pulled back halfway to the bound
  const T smin = fmin(sg[0], fmin(sg[1], sg[2]));
  const T lmax = T(0.25) * smin * smin;
  // lam is of the order of the principal strains: converge relative to that
  // scale (a test relative to |lam| alone never triggers when det F = 1)
  const T scale = fabs(sm[0]) + fabs(sm[1]) + fabs(sm[2]) + T(1e-30);
  for (int it = 0; it < 40; ++it) {
    T phi = T(0), dphi = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T q = T(1) - T(4) * lam / (sg[i] * sg[i]);
      const T rq = tsqrt<T>(q > T(0) ? q : T(0));
      const T gap = T(2) * lam / (sg[i] * (T(1) + rq));
      const T sm1 = sm[i] - gap;
      const T s = T(1) + sm1;
      phi += tlog1p<T>(sm1);
      dphi += -T(1) / ((T(2) * s - sg[i]) * s);
    }
    const T step = phi / dphi;
    const T lold = lam;
    lam -= step;
    if (lam >= lmax) lam = T(0.5) * (lold + lmax);
    // warp-uniform exit: converged lanes keep taking (vanishing) Newton steps
    if (!__any_sync(0xffffffffu, fabs(step) > T(4) * Eps<T>::v * (fabs(lam) + scale))) break;
  }
  o.lam = lam;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T q = T(1) - T(4) * lam / (sg[i] * sg[i]);
    const T rq = tsqrt<T>(q > T(0) ? q : T(0));
    o.gap[i] = T(2) * lam / (sg[i] * (T(1) + rq));
    o.s[i] = sg[i] - o.gap[i];
    o.a[i] = T(1) / (T(2) * o.s[i] - sg[i]);
  }
  return ok;
}

// dF - dR(F)[dF] for the corotated energy, as a matrix in the rotated frame:
// K = sym(M) + skew(M) o (sm1_i + sm1_j)/(sig_i + sig_j), diagonal M_ii.
template <typename T>
__device__ __forceinline__ void corot_hvp_frame(const SVD3<T>& d, const T (&M)[3][3], T (&K)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) { K[i][j] = M[i][i]; continue; }
      const T sym = T(0.5) * (M[i][j] + M[j][i]);
      const T skw = T(0.5) * (M[i][j] - M[j][i]);
      K[i][j] = sym + skw * (d.sm1[i] + d.sm1[j]) / (d.sig[i] + d.sig[j]);
    }
}

// dF - dD(F)[dF] for the volume energy in the rotated frame:
//   off-diagonal: sym * (-lam / (s_i s_j - lam)) + skw * (gap_i + gap_j) / (sig_i + sig_j)
//   diagonal:     sum_j (delta_ij - ds_i/dsig_j) M_jj with
//                 ds_i/dsig_j = a_i (s_i delta_ij - a_j / sum_k a_k / s_k)
template <typename T>
__device__ __forceinline__ void vol_hvp_frame(const SVD3<T>& d, const VolProj<T>& v, const T (&M)[3][3],
                                              T (&K)[3][3]) {
  const T den = v.a[0] / v.s[0] + v.a[1] / v.s[1] + v.a[2] / v.s[2];
  const T am = (v.a[0] * M[0][0] + v.a[1] * M[1][1] + v.a[2] * M[2][2]) / den;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (i == j) {
        K[i][i] = -(v.gap[i]) * v.a[i] * M[i][i] + v.a[i] * am;
        continue;
      }
      const T sym = T(0.5) * (M[i][j] + M[j][i]);
      const T skw = T(0.5) * (M[i][j] - M[j][i]);
      K[i][j] = sym * (-v.lam / (v.s[i] * v.s[j] - v.lam)) +
                skw * (v.gap[i] + v.gap[j]) / (d.sig[i] + d.sig[j]);
    }
}

}  // namespace pd
