// Internal declarations shared by the host C++ and CUDA translation units of
// libfs.  Nothing here is part of the C ABI (see include/fs.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fs.h"

namespace fs {

constexpr int kMaxLoc = 10;  // P2 nodes per tetrahedron
constexpr int kMaxRestart = 32;
constexpr int kExtrapMax = 4;  // previous states kept for a step's starting guess

// Thread-local error message behind fs_last_error().
void set_error(const std::string& msg);

// A host CSR matrix (pattern plus optional values).
struct HostCsr {
  int64_t nrow = 0, ncol = 0;
  std::vector<int32_t> rowptr;  // nrow + 1
  std::vector<int32_t> col;
  std::vector<double> val;      // empty when pattern-only
  int64_t nnz() const { return (int64_t)col.size(); }
};

// One structured instance of a (possibly batched) mesh: its description and
// where its vertices, edge nodes and cells sit in the union numbering.
struct Instance {
  fs_mesh_desc desc{};
  int64_t voff = 0, nv = 0;   // vertices [voff, voff + nv)
  int64_t eoff = 0, ne = 0;   // edge nodes [nv_total + eoff, ... + ne)
  int64_t coff = 0, ncell = 0;
  int64_t n2() const { return nv + ne; }
};

struct Mesh {
  fs_mesh_desc desc{};              // instance 0 (the only one unless batched)
  std::vector<Instance> inst;       // >= 1 instance; union = disjoint meshes
  int dim = 0, nloc = 0, nb = 0;    // nb = vertices per simplex
  int64_t nv = 0, ne = 0, n2 = 0, ncell = 0;
  std::vector<double> coords;       // nv x dim
  std::vector<double> p2xyz;        // n2 x dim
  std::vector<int32_t> c2d;         // ncell x nloc
  std::vector<int32_t> edges;       // ne x 2
  std::vector<uint8_t> dirichlet;   // n2
  std::vector<int32_t> dlist;       // Dirichlet P2 node ids
  HostCsr A, B, BT, Kp;             // patterns: P2-P2, P1-P2, P2-P1, P1-P1
  std::vector<uint8_t> posA;        // ncell x nloc x nloc
  std::vector<uint8_t> posB;        // ncell x nb x nloc
  std::vector<uint8_t> posBT;       // ncell x nloc x nb
  std::vector<uint8_t> posKp;       // ncell x nb x nb
  // P2 nodes are numbered internally with the edge nodes of every instance
  // grouped by the parity class of their doubled-lattice position (see
  // build_local); node_nat[q] is the paper-order (vertices, then edges ranked
  // lexicographically) id of internal node q.  Vertices keep their ids.
  std::vector<int32_t> node_nat;    // n2
  // Cells grouped by colour: no two cells of one colour share a P2 node, so
  // the cells of a colour add their element matrices into the block values
  // without atomics, and the colours run in a fixed order: every assembled
  // value is summed in the same order on every run.  Colour c holds the
  // cells color_cells[color_ptr[c] .. color_ptr[c + 1]), ascending.
  std::vector<int32_t> color_cells;
  std::vector<int64_t> color_ptr;
};

// The DOF map in paper order (the numbering of fs_dof_map): cell-to-node
// table, Dirichlet flags and the monolithic CSR pattern.
void natural_dof_map(const Mesh& m, std::vector<int32_t>* c2d, std::vector<uint8_t>* dir,
                     std::vector<int64_t>* rowptr, std::vector<int32_t>* col);

// Builds the mesh tables; returns an fs_status.
int build_mesh(const fs_mesh_desc& d, Mesh& m);
// Union of several structured meshes (no shared nodes), numbered as one mesh:
// all vertices (instance by instance), then all edge nodes, then cells.
int build_batch_mesh(const fs_mesh_desc* d, int count, Mesh& m);
// Local P2 node id of instance i -> union node id, and its inverse pieces.
inline int64_t union_node(const Mesh& m, int i, int64_t local) {
  const Instance& I = m.inst[i];
  return local < I.nv ? I.voff + local : m.nv + I.eoff + (local - I.nv);
}

// Monolithic CSR row pointers / columns from the block patterns.
void monolithic_pattern(const Mesh& m, std::vector<int64_t>& rowptr,
                        std::vector<int32_t>& col);

// Reference-simplex integrals of the P2/P1 basis, by a Grundmann-Moeller
// degree-5 rule (exact for the polynomial integrands).
struct RefTensors {
  int dim = 0, nloc = 0, nb = 0, npair = 0;
  // (j, r) pairs with d phi_j / d lambda_r != 0 (vertex j: r = j;
  // edge (a,b): r = a and r = b)
  int pair_j[16], pair_r[16];
  double mass[kMaxLoc][kMaxLoc];            // int phi_i phi_j
  double stiff[kMaxLoc][kMaxLoc][4][4];     // int d_r phi_i d_s phi_j
  double conv[kMaxLoc][kMaxLoc][16];        // int phi_i phi_k d_{r(p)} phi_{j(p)}
  double div[4][kMaxLoc][4];                // int lambda_q d_r phi_j
  double pmass[4][kMaxLoc];                 // int lambda_q phi_k
};
void ref_tensors(int dim, RefTensors& R);

// Taylor-Hood P3/P2 on a single 2D mesh (fs_p3.cpp): the P3 velocity map
// c2u (ncell x 10) and P2 pressure map c2p (ncell x 6), node coordinates,
// velocity Dirichlet flags, the block patterns A (P3-P3), B (P2-P3), BT
// (P3-P2), Kp (P2-P2) and their slot tables (layouts as Mesh's).
struct P3Tables {
  int64_t n3 = 0, np = 0, ncell = 0;
  std::vector<int32_t> c2u, c2p;
  std::vector<double> xyz;      // n3 x 2 velocity node coordinates
  std::vector<double> pxyz;     // np x 2 pressure node coordinates
  std::vector<uint8_t> dir;     // n3
  std::vector<int32_t> dlist;
  HostCsr A, B, BT, Kp;
  std::vector<uint8_t> posA, posB, posBT, posK;
};
int build_p3_tables(const Mesh& m, P3Tables& T);

// Reference-triangle integrals of the P3/P2 basis (local orders of
// fs_p3.cpp), by a Grundmann-Moeller rule of degree 9:
//   mass[i][j] = int phi_i phi_j, stiff[i][j][r][t] = int d_r phi_i d_t phi_j,
//   conv[i][k][j][r] = int phi_i phi_k d_r phi_j, div[q][j][r] = int psi_q
//   d_r phi_j, pstiff[q][s][r][t] = int d_r psi_q d_t psi_s
// (d_r = derivative in the barycentric coordinate lambda_r).
struct RefP3 {
  double mass[10][10];
  double stiff[10][10][3][3];
  double conv[10][10][10][3];
  double div[6][10][3];
  double pstiff[6][6][3][3];
};
void p3_ref_tensors(RefP3& R);

// Multigrid hierarchy on the host (values FP64), built once per problem.
struct HostLevel {
  HostCsr A;          // level operator
  HostCsr P;          // prolongation to this level from the next coarser one
  HostCsr R;          // restriction = P^T
  std::vector<double> dinv;
  double lmax = 0;    // estimate of the largest eigenvalue of D^-1 A
  int grid[3] = {1, 1, 1};  // structured mesh of the level (cells per axis)
  bool p2 = false;          // the level is the P2 space of that mesh
};
// Coarsest operators of at most this many rows are inverted on the host at
// set-up; larger ones (single problems only) are inverted on the device.
constexpr int64_t kHostInverseMax = 800;

struct HostHierarchy {
  std::vector<HostLevel> levels;   // levels[0] finest; last = coarsest
  std::vector<double> coarse_inv;  // dense inverse of the coarsest operator
  int64_t ncoarse = 0;
  // Level-0 rows of a P2 hierarchy are stored grouped by node class (see
  // the multigrid builder); order0[r] is the mesh-numbered row of level-0 row r.
  std::vector<int32_t> order0;
};
// Builds a hierarchy: A0 (square CSR with values), the structured mesh size
// n0 (cells per axis) of the P1 levels, whether level 0 is the P2 space of
// that mesh (then the first prolongation is P1 -> P2 on the same mesh), and
// the fine rows whose prolongation rows are zeroed (fixed values).
void build_hierarchy(const Mesh& m, const HostCsr& A0, bool p2_fine,
                     const std::vector<int32_t>& fixed_rows,
                     int64_t coarse_max, HostHierarchy& H);

// Hierarchy of a batched (union) mesh: one hierarchy per instance (built in
// parallel), combined level by level into block-diagonal operators.  An
// instance with fewer levels repeats its coarsest operator with identity
// transfers down to the common depth; the coarsest level is solved with the
// block-diagonal of the instances' dense inverses.
//   A0: union operator (rows = union P2 nodes when p2_fine, else vertices);
//   fixed: union fine rows whose prolongation rows are zeroed.
struct UnionHierarchy {
  HostHierarchy H;                   // block-diagonal levels; coarse_inv unused
  std::vector<int64_t> blk_row;      // coarsest level: row offset per instance
  std::vector<int64_t> blk_n;        // ... block size per instance
  std::vector<int64_t> blk_dense;    // ... offset of its dense inverse
  std::vector<double> dense;         // concatenated dense inverses (row-major);
                                     // empty: invert the coarsest level's A
                                     // on the device (one block above
                                     // kHostInverseMax rows)
  std::vector<int32_t> row_blk;      // coarsest row -> instance
  // per level: first row of each instance (instance count + 1 entries;
  // every level is block-diagonal in instance order)
  std::vector<std::vector<int64_t>> inst_off;
  // level-0 rows are in instance-major (block) order, each instance's rows
  // in class order; perm[r] is the union row of block row r (empty when
  // the two orders agree)
  std::vector<int32_t> perm;
};
void build_union_hierarchy(const Mesh& m, const std::vector<Mesh>& local,
                           const HostCsr& A0, bool p2_fine,
                           const std::vector<int32_t>& fixed, int64_t coarse_max,
                           UnionHierarchy& U);

}  // namespace fs
