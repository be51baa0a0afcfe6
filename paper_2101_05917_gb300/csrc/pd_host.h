// Host-side mesh analysis: voxel or tetrahedral mesh, incidence, nested-dissection ordering and
// the supernodal structure of the scalar matrix L_A with A = I_3 (x) L_A
// (Eqn 19: G_c maps each coordinate identically, so A never couples x, y, z).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "diffpd.h"

namespace pd {

struct HostMesh {
  int nx = 0, ny = 0, nz = 0;
  double dx = 0, origin[3] = {0, 0, 0}, density = 0;
  int leaf_max = 64;
  int rule = 0;                        // PD_ELEM_HEX8 / PD_ELEM_TET6 / PD_ELEM_TETU
  // element corners in use; element records keep a stride of 8 entries (a
  // tetrahedron of an unstructured mesh fills slots 0..3 and repeats vertex 0 in
  // slots 4..7, which carry zero shape gradients and no incidence entries)
  int corners = 8;
  int64_t n = 0, e = 0, nf = 0;       // kept nodes, kept cells, free nodes

  // kept order (increasing grid id / cell id)
  std::vector<int64_t> grid;           // (n) grid id of each kept node
  std::vector<int32_t> elems_kept;     // (8e) kept-node index of each corner
  std::vector<uint8_t> dirichlet_kept, contact_kept;
  std::vector<int64_t> inc_ptr_kept, inc_kept;   // node -> e*8+a, ascending

  // nested dissection over the free nodes
  std::vector<int64_t> perm;           // (nf) column -> free index (kept order among free)

  // internal node numbering: columns 0..nf-1 in ND order, then Dirichlet nodes
  std::vector<int32_t> internal_of_kept, kept_of_internal;
  std::vector<int32_t> elems;          // (8e) internal ids
  std::vector<double> X;               // (3n) rest positions, internal order
  std::vector<double> mass;            // (n) lumped mass, internal order
  std::vector<uint8_t> contact;        // (n) internal order
  std::vector<int32_t> inc_ptr, inc;   // incidence over internal nodes
  // unstructured tetrahedra: per element the gradients of the four barycentric
  // coordinates (12 doubles, vertex-major) and the volume
  std::vector<double> tet_grad, tet_vol;

  // supernodes (ND-tree nodes: leaves and separator planes)
  int64_t ns = 0, nlev = 0;
  std::vector<int64_t> snode_first;    // (ns+1)
  std::vector<int64_t> row_ptr;        // (ns+1)
  std::vector<int32_t> rows;           // ascending row structure per supernode
  std::vector<int64_t> parent, level, level_ptr, level_list;
  std::vector<int64_t> rel_ptr;        // (ns+1) into rel (below-row count per supernode)
  std::vector<int32_t> rel;            // position of each below row inside rows(parent)
  std::vector<int64_t> panel_off;      // (ns+1) offsets of nr x nc panels
  std::vector<int64_t> front_off;      // (ns+1) offsets of nr x nr fronts
  std::vector<int64_t> child_ptr, child_list;   // supernodal etree children, ascending

  // forward-solve assembly: for every position k of every supernode (global
  // position index pos_off[s] + k) the update-vector rows W[rel_ptr[t] + i]
  // that land on it, children in ascending order.
  std::vector<int64_t> pos_off;        // == row_ptr
  std::vector<int64_t> gath_ptr;       // (sum nr + 1)
  std::vector<int32_t> gath;           // W row index

  // assembly of the lower triangle of L_A into the fronts: one entry per
  // nonzero (r >= c), target = front_off[s] + pos_r + pos_c * nr, with the
  // element contributions (e*64 + a*8 + b) and an optional diagonal node.
  std::vector<int64_t> la_target;      // (nnz)
  std::vector<int32_t> la_diag_node;   // (nnz) internal node for diagonals, -1 otherwise
  std::vector<int64_t> la_cptr;        // (nnz+1)
  std::vector<int32_t> la_contrib;     // e*64 + a*8 + b

  int64_t factor_nnz() const { return panel_off.empty() ? 0 : panel_off.back(); }
  int64_t front_entries() const { return front_off.empty() ? 0 : front_off.back(); }
  int64_t nr(int64_t s) const { return row_ptr[s + 1] - row_ptr[s]; }
  int64_t nc(int64_t s) const { return snode_first[s + 1] - snode_first[s]; }
};

// Returns "" on success, else an error message.
std::string analyse(const pd_mesh_desc& d, HostMesh& m);
std::string analyse_tet(const pd_tet_mesh_desc& d, HostMesh& m);

}  // namespace pd
