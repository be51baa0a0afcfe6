// Host-side mesh analysis (C++).  The definitions below are the canonical ones
// of this implementation; they are reproduced bit for bit by an independent
// re-derivation in the test suite.
//
//  incidence   kept node -> entries e*8+a (cell e, corner a), ascending.
//  ordering    nested dissection over grid boxes of free nodes: a box with more
//              than leaf_max free nodes splits along its longest axis (ties x, y,
//              z) at node plane mid = floor((lo+hi)/2); left part [lo, mid-1]
//              first, then right part [mid+1, hi], then the plane's free nodes in
//              grid-id order.  Boxes with 1..leaf_max free nodes are leaves in
//              grid-id order.
//  supernodes  every leaf and every non-empty separator plane.
//  unstructured tetrahedral meshes (analyse_tet): kept nodes and elements are the
//              caller's; incidence entries e*8+a for vertices a < 4; ordering by
//              coordinate bisection of free-node sets with vertex separators of
//              the mesh graph (GraphNDBuilder); supernodes every leaf and every
//              non-empty separator.
//  structure   rows(s) = cols(s) + {r >= first(s) adjacent to a column of s} +
//              below(t) of every child t; parent(s) = owner of min below(s).
//  levels      0 for supernodes without children, else 1 + max over children.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "pd_host.h"

namespace pd {
namespace {

struct NDBuilder {
  const HostMesh& m;
  const std::vector<int64_t>& fi, &fj, &fk;   // grid coordinates of free nodes
  std::vector<int64_t>& perm;
  std::vector<int64_t>& firsts;
  int leaf_max;

  // `ids`: free-node indices inside the box, ascending grid id (== ascending index)
  void rec(const int64_t lo[3], const int64_t hi[3], std::vector<int64_t>& ids) {
    if (ids.empty()) return;
    if ((int64_t)ids.size() <= leaf_max) {
      firsts.push_back((int64_t)perm.size());
      perm.insert(perm.end(), ids.begin(), ids.end());
      return;
    }
    int64_t ext[3] = {hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
    int d = 0;
    if (ext[1] > ext[d]) d = 1;
    if (ext[2] > ext[d]) d = 2;
    const int64_t mid = (lo[d] + hi[d]) / 2;   // lo, hi >= 0
    std::vector<int64_t> left, right, sep;
    for (int64_t f : ids) {
      const int64_t c = d == 0 ? fi[f] : (d == 1 ? fj[f] : fk[f]);
      if (c < mid) left.push_back(f);
      else if (c > mid) right.push_back(f);
      else sep.push_back(f);
    }
    ids.clear();
    ids.shrink_to_fit();
    int64_t lhi[3] = {hi[0], hi[1], hi[2]};
    lhi[d] = mid - 1;
    int64_t rlo[3] = {lo[0], lo[1], lo[2]};
    rlo[d] = mid + 1;
    rec(lo, lhi, left);
    rec(rlo, hi, right);
    if (!sep.empty()) {
      firsts.push_back((int64_t)perm.size());
      perm.insert(perm.end(), sep.begin(), sep.end());
    }
  }
};

// Unstructured meshes: coordinate bisection with vertex separators of the mesh
// graph.  `ids` ascending free-node indices.
struct GraphNDBuilder {
  const std::vector<double>& P;                     // (3 nf) free-node rest positions
  const std::vector<std::vector<int32_t>>& adj;     // free-node adjacency
  std::vector<int64_t>& perm;
  std::vector<int64_t>& firsts;
  std::vector<uint8_t>& in_right;                   // scratch, all zero between calls
  int leaf_max;

  void rec(std::vector<int64_t>& ids) {
    if (ids.empty()) return;
    if ((int64_t)ids.size() <= leaf_max) {
      firsts.push_back((int64_t)perm.size());
      perm.insert(perm.end(), ids.begin(), ids.end());
      return;
    }
    double lo[3], hi[3];
    for (int c = 0; c < 3; ++c) lo[c] = hi[c] = P[3 * ids[0] + c];
    for (int64_t f : ids)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], P[3 * f + c]);
        hi[c] = std::max(hi[c], P[3 * f + c]);
      }
    const double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    int d = 0;
    if (ext[1] > ext[d]) d = 1;
    if (ext[2] > ext[d]) d = 2;
    std::vector<int64_t> order(ids);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      const double pa = P[3 * a + d], pb = P[3 * b + d];
      return pa < pb || (pa == pb && a < b);
    });
    const size_t half = ids.size() / 2;
    for (size_t i = half; i < order.size(); ++i) in_right[order[i]] = 1;
    std::vector<int64_t> left, sep, right(order.begin() + (std::ptrdiff_t)half, order.end());
    for (size_t i = 0; i < half; ++i) {
      const int64_t f = order[i];
      bool touches = false;
      for (int32_t o : adj[f])
        if (in_right[o]) {
          touches = true;
          break;
        }
      (touches ? sep : left).push_back(f);
    }
    for (int64_t f : right) in_right[f] = 0;
    ids.clear();
    ids.shrink_to_fit();
    order.clear();
    order.shrink_to_fit();
    std::sort(left.begin(), left.end());
    std::sort(sep.begin(), sep.end());
    std::sort(right.begin(), right.end());
    rec(left);
    rec(right);
    if (!sep.empty()) {
      firsts.push_back((int64_t)perm.size());
      perm.insert(perm.end(), sep.begin(), sep.end());
    }
  }
};

}  // namespace

std::string build_structure(HostMesh& m);

std::string analyse(const pd_mesh_desc& d, HostMesh& m) {
  if (d.nx <= 0 || d.ny <= 0 || d.nz <= 0) return "mesh: nx, ny, nz must be positive";
  if (!(d.dx > 0)) return "mesh: dx must be positive";
  if (!(d.density > 0)) return "mesh: density must be positive";
  m.nx = d.nx; m.ny = d.ny; m.nz = d.nz; m.dx = d.dx; m.density = d.density;
  for (int c = 0; c < 3; ++c) m.origin[c] = d.origin[c];
  m.leaf_max = d.leaf_max > 0 ? d.leaf_max : 64;
  if (d.element_rule != PD_ELEM_HEX8 && d.element_rule != PD_ELEM_TET6) return "mesh: unknown element rule";
  m.rule = d.element_rule;
  m.corners = 8;
  const int64_t nx = d.nx, ny = d.ny, nz = d.nz;
  const int64_t ncell = nx * ny * nz;
  const int64_t ngrid = (nx + 1) * (ny + 1) * (nz + 1);
  if (ngrid >= (int64_t)1 << 31) return "mesh: grid too large for 32-bit node ids";

  // ---- kept cells and nodes
  std::vector<int64_t> cell_corner;   // grid ids
  cell_corner.reserve(8 * ncell);
  for (int64_t ci = 0; ci < nx; ++ci)
    for (int64_t cj = 0; cj < ny; ++cj)
      for (int64_t ck = 0; ck < nz; ++ck) {
        const int64_t cid = (ci * ny + cj) * nz + ck;
        if (d.cell_mask && !d.cell_mask[cid]) continue;
        for (int a = 0; a < 8; ++a) {
          const int64_t di = (a >> 2) & 1, dj = (a >> 1) & 1, dk = a & 1;
          cell_corner.push_back(((ci + di) * (ny + 1) + (cj + dj)) * (nz + 1) + (ck + dk));
        }
      }
  m.e = (int64_t)cell_corner.size() / 8;
  if (m.e == 0) return "mesh: no kept cells";
  std::vector<int32_t> kept_of_grid(ngrid, -1);
  for (int64_t g : cell_corner) kept_of_grid[g] = 0;
  m.grid.clear();
  for (int64_t g = 0; g < ngrid; ++g)
    if (kept_of_grid[g] == 0) {
      kept_of_grid[g] = (int32_t)m.grid.size();
      m.grid.push_back(g);
    }
  m.n = (int64_t)m.grid.size();
  m.elems_kept.resize(8 * m.e);
  for (int64_t i = 0; i < 8 * m.e; ++i) m.elems_kept[i] = kept_of_grid[cell_corner[i]];
  m.dirichlet_kept.assign(m.n, 0);
  m.contact_kept.assign(m.n, 0);
  if (d.dirichlet) for (int64_t i = 0; i < m.n; ++i) m.dirichlet_kept[i] = d.dirichlet[i] ? 1 : 0;
  if (d.contact) for (int64_t i = 0; i < m.n; ++i) m.contact_kept[i] = d.contact[i] ? 1 : 0;

  // ---- incidence (kept order)
  m.inc_ptr_kept.assign(m.n + 1, 0);
  for (int64_t i = 0; i < 8 * m.e; ++i) m.inc_ptr_kept[m.elems_kept[i] + 1]++;
  for (int64_t i = 0; i < m.n; ++i) m.inc_ptr_kept[i + 1] += m.inc_ptr_kept[i];
  m.inc_kept.assign(8 * m.e, 0);
  {
    std::vector<int64_t> fill(m.inc_ptr_kept.begin(), m.inc_ptr_kept.end() - 1);
    for (int64_t i = 0; i < 8 * m.e; ++i) m.inc_kept[fill[m.elems_kept[i]]++] = i;  // i = e*8+a ascending
  }

  // ---- free nodes and nested dissection
  std::vector<int64_t> free_kept;   // free index -> kept index
  for (int64_t i = 0; i < m.n; ++i)
    if (!m.dirichlet_kept[i]) free_kept.push_back(i);
  m.nf = (int64_t)free_kept.size();
  if (m.nf == 0) return "mesh: every node is fixed";
  std::vector<int64_t> fi(m.nf), fj(m.nf), fk(m.nf);
  for (int64_t f = 0; f < m.nf; ++f) {
    const int64_t g = m.grid[free_kept[f]];
    fk[f] = g % (nz + 1);
    fj[f] = (g / (nz + 1)) % (ny + 1);
    fi[f] = g / ((nz + 1) * (ny + 1));
  }
  m.perm.clear();
  m.snode_first.clear();
  {
    std::vector<int64_t> ids(m.nf);
    std::iota(ids.begin(), ids.end(), 0);
    NDBuilder b{m, fi, fj, fk, m.perm, m.snode_first, m.leaf_max};
    const int64_t lo[3] = {0, 0, 0}, hi[3] = {nx, ny, nz};
    b.rec(lo, hi, ids);
  }
  m.snode_first.push_back(m.nf);
  m.ns = (int64_t)m.snode_first.size() - 1;

  // ---- internal numbering
  m.internal_of_kept.assign(m.n, -1);
  m.kept_of_internal.assign(m.n, -1);
  for (int64_t c = 0; c < m.nf; ++c) {
    const int64_t k = free_kept[m.perm[c]];
    m.internal_of_kept[k] = (int32_t)c;
    m.kept_of_internal[c] = (int32_t)k;
  }
  {
    int64_t next = m.nf;
    for (int64_t k = 0; k < m.n; ++k)
      if (m.dirichlet_kept[k]) {
        m.internal_of_kept[k] = (int32_t)next;
        m.kept_of_internal[next] = (int32_t)k;
        ++next;
      }
  }
  m.elems.resize(8 * m.e);
  for (int64_t i = 0; i < 8 * m.e; ++i) m.elems[i] = m.internal_of_kept[m.elems_kept[i]];
  m.X.resize(3 * m.n);
  m.contact.assign(m.n, 0);
  for (int64_t in = 0; in < m.n; ++in) {
    const int64_t g = m.grid[m.kept_of_internal[in]];
    const int64_t k = g % (nz + 1), j = (g / (nz + 1)) % (ny + 1), i = g / ((nz + 1) * (ny + 1));
    m.X[3 * in + 0] = d.origin[0] + d.dx * (double)i;
    m.X[3 * in + 1] = d.origin[1] + d.dx * (double)j;
    m.X[3 * in + 2] = d.origin[2] + d.dx * (double)k;
    m.contact[in] = m.contact_kept[m.kept_of_internal[in]];
  }
  m.mass.assign(m.n, 0.0);
  if (m.rule == PD_ELEM_HEX8) {
    const double mcorner = d.density * d.dx * d.dx * d.dx / 8.0;
    for (int64_t i = 0; i < 8 * m.e; ++i) m.mass[m.elems[i]] += mcorner;
  } else {
    // rho V / 4 to each vertex of each tetrahedron, V = dx^3 / 6: the two corners on
    // the cell diagonal belong to all six tetrahedra, the other six corners to two
    const double share = d.density * d.dx * d.dx * d.dx / 24.0;
    for (int64_t c = 0; c < m.e; ++c)
      for (int a = 0; a < 8; ++a) m.mass[m.elems[8 * c + a]] += (a == 0 || a == 7 ? 6.0 : 2.0) * share;
  }
  m.inc_ptr.assign(m.n + 1, 0);
  for (int64_t i = 0; i < 8 * m.e; ++i) m.inc_ptr[m.elems[i] + 1]++;
  for (int64_t i = 0; i < m.n; ++i) m.inc_ptr[i + 1] += m.inc_ptr[i];
  m.inc.assign(8 * m.e, 0);
  {
    std::vector<int32_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
    for (int64_t i = 0; i < 8 * m.e; ++i) m.inc[fill[m.elems[i]]++] = (int32_t)i;
  }

  return build_structure(m);
}

std::string analyse_tet(const pd_tet_mesh_desc& d, HostMesh& m) {
  if (d.n_nodes <= 0 || d.n_tets <= 0) return "tet mesh: n_nodes and n_tets must be positive";
  if (!d.X || !d.tets) return "tet mesh: X and tets are required";
  if (!(d.density > 0)) return "tet mesh: density must be positive";
  if (d.n_nodes >= (int64_t)1 << 31) return "tet mesh: too many nodes for 32-bit node ids";
  if (d.n_tets >= (int64_t)1 << 25) return "tet mesh: too many tetrahedra for 32-bit assembly codes";
  m.rule = PD_ELEM_TETU;
  m.corners = 4;
  m.nx = m.ny = m.nz = 0;
  m.density = d.density;
  m.leaf_max = d.leaf_max > 0 ? d.leaf_max : 64;
  m.n = d.n_nodes;
  m.e = d.n_tets;
  for (int64_t i = 0; i < 3 * m.n; ++i)
    if (!std::isfinite(d.X[i])) return "tet mesh: non-finite rest position";

  // ---- elements (kept order = the caller's), barycentric gradients and volumes
  m.elems_kept.assign(8 * m.e, 0);
  m.tet_grad.assign(12 * m.e, 0.0);
  m.tet_vol.assign(m.e, 0.0);
  std::vector<uint8_t> used(m.n, 0);
  double vsum = 0.0;
  for (int64_t t = 0; t < m.e; ++t) {
    int32_t v[4];
    for (int a = 0; a < 4; ++a) {
      v[a] = d.tets[4 * t + a];
      if (v[a] < 0 || v[a] >= m.n) return "tet mesh: vertex index out of range in tetrahedron " + std::to_string(t);
      for (int b = 0; b < a; ++b)
        if (v[b] == v[a]) return "tet mesh: repeated vertex in tetrahedron " + std::to_string(t);
      used[v[a]] = 1;
    }
    for (int a = 0; a < 8; ++a) m.elems_kept[8 * t + a] = v[a < 4 ? a : 0];
    // edge matrix D (columns X_a - X_0, a = 1..3) and its inverse by cofactors; row
    // a-1 of D^-1 is the gradient of barycentric coordinate a, coordinate 0 takes
    // minus their sum
    double D[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) D[r][c] = d.X[3 * (int64_t)v[c + 1] + r] - d.X[3 * (int64_t)v[0] + r];
    const double C00 = D[1][1] * D[2][2] - D[1][2] * D[2][1];
    const double C01 = D[1][2] * D[2][0] - D[1][0] * D[2][2];
    const double C02 = D[1][0] * D[2][1] - D[1][1] * D[2][0];
    const double det = D[0][0] * C00 + D[0][1] * C01 + D[0][2] * C02;
    // degenerate: a volume below 1e-12 of the cube of its longest edge from vertex 0
    // (the barycentric gradients would then overflow the FP32 tables)
    double L2 = 0.0;
    for (int c = 0; c < 3; ++c) L2 = std::max(L2, D[0][c] * D[0][c] + D[1][c] * D[1][c] + D[2][c] * D[2][c]);
    if (!std::isfinite(det) || !(std::fabs(det) > 1e-12 * L2 * std::sqrt(L2)))
      return "tet mesh: degenerate tetrahedron " + std::to_string(t);
    double inv[3][3];   // inv = adj(D) / det, adj(D)[i][j] = cofactor C_ji
    inv[0][0] = C00 / det;
    inv[1][0] = C01 / det;
    inv[2][0] = C02 / det;
    inv[0][1] = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) / det;
    inv[1][1] = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) / det;
    inv[2][1] = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) / det;
    inv[0][2] = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) / det;
    inv[1][2] = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) / det;
    inv[2][2] = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) / det;
    double* g = m.tet_grad.data() + 12 * t;
    for (int j = 0; j < 3; ++j) {
      g[3 * 1 + j] = inv[0][j];
      g[3 * 2 + j] = inv[1][j];
      g[3 * 3 + j] = inv[2][j];
      g[j] = -(inv[0][j] + inv[1][j] + inv[2][j]);
    }
    m.tet_vol[t] = std::fabs(det) / 6.0;
    vsum += m.tet_vol[t];
  }
  for (int64_t i = 0; i < m.n; ++i)
    if (!used[i]) return "tet mesh: node " + std::to_string(i) + " belongs to no tetrahedron";
  // a length scale for tolerances that voxel meshes take from dx: the edge of a cube
  // of six times the mean tetrahedron volume
  m.dx = std::cbrt(6.0 * vsum / (double)m.e);
  m.grid.resize(m.n);
  std::iota(m.grid.begin(), m.grid.end(), 0);
  m.dirichlet_kept.assign(m.n, 0);
  m.contact_kept.assign(m.n, 0);
  if (d.dirichlet) for (int64_t i = 0; i < m.n; ++i) m.dirichlet_kept[i] = d.dirichlet[i] ? 1 : 0;
  if (d.contact) for (int64_t i = 0; i < m.n; ++i) m.contact_kept[i] = d.contact[i] ? 1 : 0;

  // ---- incidence (kept order): entries e*8+a for the four vertices
  m.inc_ptr_kept.assign(m.n + 1, 0);
  for (int64_t t = 0; t < m.e; ++t)
    for (int a = 0; a < 4; ++a) m.inc_ptr_kept[m.elems_kept[8 * t + a] + 1]++;
  for (int64_t i = 0; i < m.n; ++i) m.inc_ptr_kept[i + 1] += m.inc_ptr_kept[i];
  m.inc_kept.assign(4 * m.e, 0);
  {
    std::vector<int64_t> fill(m.inc_ptr_kept.begin(), m.inc_ptr_kept.end() - 1);
    for (int64_t t = 0; t < m.e; ++t)
      for (int a = 0; a < 4; ++a) m.inc_kept[fill[m.elems_kept[8 * t + a]]++] = 8 * t + a;
  }

  // ---- free nodes, their adjacency and the nested dissection
  std::vector<int64_t> free_kept;
  std::vector<int64_t> free_of(m.n, -1);
  for (int64_t i = 0; i < m.n; ++i)
    if (!m.dirichlet_kept[i]) {
      free_of[i] = (int64_t)free_kept.size();
      free_kept.push_back(i);
    }
  m.nf = (int64_t)free_kept.size();
  if (m.nf == 0) return "tet mesh: every node is fixed";
  std::vector<std::vector<int32_t>> fadj(m.nf);
  for (int64_t t = 0; t < m.e; ++t)
    for (int a = 0; a < 4; ++a) {
      const int64_t fa = free_of[m.elems_kept[8 * t + a]];
      if (fa < 0) continue;
      for (int b = 0; b < 4; ++b) {
        const int64_t fb = free_of[m.elems_kept[8 * t + b]];
        if (fb >= 0 && fb != fa) fadj[fa].push_back((int32_t)fb);
      }
    }
  std::vector<double> P(3 * m.nf);
  for (int64_t f = 0; f < m.nf; ++f)
    for (int c = 0; c < 3; ++c) P[3 * f + c] = d.X[3 * free_kept[f] + c];
  m.perm.clear();
  m.snode_first.clear();
  {
    std::vector<int64_t> ids(m.nf);
    std::iota(ids.begin(), ids.end(), 0);
    std::vector<uint8_t> in_right(m.nf, 0);
    GraphNDBuilder b{P, fadj, m.perm, m.snode_first, in_right, m.leaf_max};
    b.rec(ids);
  }
  m.snode_first.push_back(m.nf);
  m.ns = (int64_t)m.snode_first.size() - 1;

  // ---- internal numbering: columns in ND order, then the fixed nodes
  m.internal_of_kept.assign(m.n, -1);
  m.kept_of_internal.assign(m.n, -1);
  for (int64_t c = 0; c < m.nf; ++c) {
    const int64_t k = free_kept[m.perm[c]];
    m.internal_of_kept[k] = (int32_t)c;
    m.kept_of_internal[c] = (int32_t)k;
  }
  {
    int64_t next = m.nf;
    for (int64_t k = 0; k < m.n; ++k)
      if (m.dirichlet_kept[k]) {
        m.internal_of_kept[k] = (int32_t)next;
        m.kept_of_internal[next] = (int32_t)k;
        ++next;
      }
  }
  m.elems.resize(8 * m.e);
  for (int64_t i = 0; i < 8 * m.e; ++i) m.elems[i] = m.internal_of_kept[m.elems_kept[i]];
  m.X.resize(3 * m.n);
  m.contact.assign(m.n, 0);
  for (int64_t in = 0; in < m.n; ++in) {
    const int64_t k = m.kept_of_internal[in];
    for (int c = 0; c < 3; ++c) m.X[3 * in + c] = d.X[3 * k + c];
    m.contact[in] = m.contact_kept[k];
  }
  m.mass.assign(m.n, 0.0);
  for (int64_t t = 0; t < m.e; ++t)
    for (int a = 0; a < 4; ++a) m.mass[m.elems[8 * t + a]] += d.density * m.tet_vol[t] / 4.0;
  m.inc_ptr.assign(m.n + 1, 0);
  for (int64_t t = 0; t < m.e; ++t)
    for (int a = 0; a < 4; ++a) m.inc_ptr[m.elems[8 * t + a] + 1]++;
  for (int64_t i = 0; i < m.n; ++i) m.inc_ptr[i + 1] += m.inc_ptr[i];
  m.inc.assign(4 * m.e, 0);
  {
    std::vector<int32_t> fill(m.inc_ptr.begin(), m.inc_ptr.end() - 1);
    for (int64_t t = 0; t < m.e; ++t)
      for (int a = 0; a < 4; ++a) m.inc[fill[m.elems[8 * t + a]]++] = (int32_t)(8 * t + a);
  }
  return build_structure(m);
}

// Everything that follows from the internal numbering, the element records and
// the incidence: the adjacency of L_A, the supernodal structure, levels, relative
// indices, panel / front offsets, the forward-solve gather lists and the L_A
// assembly map (contribution code e*64 + a*8 + b for element corners a, b).
std::string build_structure(HostMesh& m) {
  const int nco = m.corners;
  // ---- adjacency of L_A over columns (free nodes share an element), sorted
  std::vector<int64_t> adj_ptr(m.nf + 1, 0);
  std::vector<int32_t> adj;
  {
    std::vector<int64_t> mark(m.nf, -1);
    std::vector<int32_t> tmp;
    for (int64_t c = 0; c < m.nf; ++c) {
      tmp.clear();
      for (int32_t p = m.inc_ptr[c]; p < m.inc_ptr[c + 1]; ++p) {
        const int32_t e = m.inc[p] / 8;
        for (int b = 0; b < nco; ++b) {
          const int32_t o = m.elems[8 * e + b];
          if (o < m.nf && mark[o] != c) {
            mark[o] = c;
            tmp.push_back(o);
          }
        }
      }
      std::sort(tmp.begin(), tmp.end());
      adj.insert(adj.end(), tmp.begin(), tmp.end());
      adj_ptr[c + 1] = (int64_t)adj.size();
    }
  }

  // ---- supernodal structure
  std::vector<int64_t> owner(m.nf);
  for (int64_t s = 0; s < m.ns; ++s)
    for (int64_t c = m.snode_first[s]; c < m.snode_first[s + 1]; ++c) owner[c] = s;
  m.parent.assign(m.ns, -1);
  std::vector<std::vector<int64_t>> children(m.ns);
  m.row_ptr.assign(m.ns + 1, 0);
  m.rows.clear();
  {
    std::vector<int64_t> mark(m.nf, -1);
    std::vector<int32_t> tmp;
    for (int64_t s = 0; s < m.ns; ++s) {
      const int64_t f = m.snode_first[s], l = m.snode_first[s + 1];
      tmp.clear();
      auto add = [&](int64_t r) {
        if (r >= f && mark[r] != s) {
          mark[r] = s;
          tmp.push_back((int32_t)r);
        }
      };
      for (int64_t c = f; c < l; ++c) {
        add(c);
        for (int64_t p = adj_ptr[c]; p < adj_ptr[c + 1]; ++p) add(adj[p]);
      }
      for (int64_t t : children[s])
        for (int64_t p = m.row_ptr[t]; p < m.row_ptr[t + 1]; ++p)
          if (m.rows[p] >= m.snode_first[t + 1]) add(m.rows[p]);
      std::sort(tmp.begin(), tmp.end());
      m.rows.insert(m.rows.end(), tmp.begin(), tmp.end());
      m.row_ptr[s + 1] = (int64_t)m.rows.size();
      const int64_t nrs = (int64_t)tmp.size(), ncs = l - f;
      if (nrs > ncs) {
        const int64_t p = owner[tmp[ncs]];
        m.parent[s] = p;
        children[p].push_back(s);
      }
    }
  }
  m.level.assign(m.ns, 0);
  for (int64_t s = 0; s < m.ns; ++s)
    for (int64_t t : children[s]) m.level[s] = std::max(m.level[s], m.level[t] + 1);
  m.nlev = 0;
  for (int64_t s = 0; s < m.ns; ++s) m.nlev = std::max(m.nlev, m.level[s] + 1);
  m.level_ptr.assign(m.nlev + 1, 0);
  for (int64_t s = 0; s < m.ns; ++s) m.level_ptr[m.level[s] + 1]++;
  for (int64_t L = 0; L < m.nlev; ++L) m.level_ptr[L + 1] += m.level_ptr[L];
  m.level_list.assign(m.ns, 0);
  {
    std::vector<int64_t> fill(m.level_ptr.begin(), m.level_ptr.end() - 1);
    for (int64_t s = 0; s < m.ns; ++s) m.level_list[fill[m.level[s]]++] = s;
  }
  m.child_ptr.assign(m.ns + 1, 0);
  m.child_list.clear();
  for (int64_t s = 0; s < m.ns; ++s) {
    m.child_list.insert(m.child_list.end(), children[s].begin(), children[s].end());
    m.child_ptr[s + 1] = (int64_t)m.child_list.size();
  }
  // relative indices of below rows in the parent
  m.rel_ptr.assign(m.ns + 1, 0);
  m.rel.clear();
  for (int64_t s = 0; s < m.ns; ++s) {
    const int64_t p = m.parent[s];
    const int64_t ncs = m.nc(s);
    if (p >= 0) {
      const int32_t* pr = m.rows.data() + m.row_ptr[p];
      const int64_t pn = m.nr(p);
      for (int64_t q = m.row_ptr[s] + ncs; q < m.row_ptr[s + 1]; ++q) {
        const int32_t* it = std::lower_bound(pr, pr + pn, m.rows[q]);
        if (it == pr + pn || *it != m.rows[q]) return "internal: below row missing in parent";
        m.rel.push_back((int32_t)(it - pr));
      }
    }
    m.rel_ptr[s + 1] = (int64_t)m.rel.size();
  }
  // panel / front offsets
  m.panel_off.assign(m.ns + 1, 0);
  m.front_off.assign(m.ns + 1, 0);
  for (int64_t s = 0; s < m.ns; ++s) {
    m.panel_off[s + 1] = m.panel_off[s] + m.nr(s) * m.nc(s);
    m.front_off[s + 1] = m.front_off[s] + m.nr(s) * m.nr(s);
  }
  // forward-solve gather lists per supernode position
  m.pos_off = m.row_ptr;
  const int64_t npos = m.row_ptr[m.ns];
  m.gath_ptr.assign(npos + 1, 0);
  for (int64_t s = 0; s < m.ns; ++s) {
    const int64_t p = m.parent[s];
    if (p < 0) continue;
    for (int64_t i = 0; i < m.rel_ptr[s + 1] - m.rel_ptr[s]; ++i)
      m.gath_ptr[m.pos_off[p] + m.rel[m.rel_ptr[s] + i] + 1]++;
  }
  for (int64_t k = 0; k < npos; ++k) m.gath_ptr[k + 1] += m.gath_ptr[k];
  m.gath.assign(m.gath_ptr[npos], 0);
  {
    std::vector<int64_t> fill(m.gath_ptr.begin(), m.gath_ptr.end() - 1);
    for (int64_t p = 0; p < m.ns; ++p)            // parents ascending
      for (int64_t ci = m.child_ptr[p]; ci < m.child_ptr[p + 1]; ++ci) {   // children ascending
        const int64_t s = m.child_list[ci];
        for (int64_t i = 0; i < m.rel_ptr[s + 1] - m.rel_ptr[s]; ++i) {
          const int64_t k = m.pos_off[p] + m.rel[m.rel_ptr[s] + i];
          m.gath[fill[k]++] = (int32_t)(m.rel_ptr[s] + i);
        }
      }
  }

  // ---- L_A assembly map (lower triangle, per column in supernode order)
  m.la_target.clear();
  m.la_diag_node.clear();
  m.la_cptr.assign(1, 0);
  m.la_contrib.clear();
  {
    std::vector<std::vector<int32_t>> contrib_of_row;   // scratch per column
    for (int64_t s = 0; s < m.ns; ++s) {
      const int32_t* sr = m.rows.data() + m.row_ptr[s];
      const int64_t nrs = m.nr(s);
      for (int64_t c = m.snode_first[s]; c < m.snode_first[s + 1]; ++c) {
        // rows r >= c adjacent to c, with their element contributions
        std::vector<std::pair<int32_t, int32_t>> items;   // (row, e*64+a*8+b)
        for (int32_t p = m.inc_ptr[c]; p < m.inc_ptr[c + 1]; ++p) {
          const int32_t e = m.inc[p] / 8, b = m.inc[p] % 8;
          for (int a = 0; a < nco; ++a) {
            const int32_t r = m.elems[8 * e + a];
            if (r < m.nf && r >= c) items.push_back({r, e * 64 + a * 8 + b});
          }
        }
        std::sort(items.begin(), items.end());
        const int64_t pc = c - m.snode_first[s];
        size_t i = 0;
        while (i < items.size()) {
          const int32_t r = items[i].first;
          const int32_t* it = std::lower_bound(sr, sr + nrs, r);
          if (it == sr + nrs || *it != r) return "internal: L_A row outside supernode structure";
          m.la_target.push_back(m.front_off[s] + (int64_t)(it - sr) + pc * nrs);
          m.la_diag_node.push_back(r == c ? (int32_t)c : -1);
          while (i < items.size() && items[i].first == r) m.la_contrib.push_back(items[i++].second);
          m.la_cptr.push_back((int64_t)m.la_contrib.size());
        }
      }
    }
  }
  return "";
}

}  // namespace pd
