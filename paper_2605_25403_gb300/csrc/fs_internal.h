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

struct Mesh {
  fs_mesh_desc desc{};
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
};

// Builds the mesh tables; returns an fs_status.
int build_mesh(const fs_mesh_desc& d, Mesh& m);

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
};
void ref_tensors(int dim, RefTensors& R);

// Multigrid hierarchy on the host (values FP64), built once per problem.
struct HostLevel {
  HostCsr A;          // level operator
  HostCsr P;          // prolongation to this level from the next coarser one
  HostCsr R;          // restriction = P^T
  std::vector<double> dinv;
  double lmax = 0;    // estimate of the largest eigenvalue of D^-1 A
};
struct HostHierarchy {
  std::vector<HostLevel> levels;   // levels[0] finest; last = coarsest
  std::vector<double> coarse_inv;  // dense inverse of the coarsest operator
  int64_t ncoarse = 0;
};
// Builds a hierarchy: A0 (square CSR with values), the structured mesh size
// n0 (cells per axis) of the P1 levels, whether level 0 is the P2 space of
// that mesh (then the first prolongation is P1 -> P2 on the same mesh), and
// the fine rows whose prolongation rows are zeroed (fixed values).
void build_hierarchy(const Mesh& m, const HostCsr& A0, bool p2_fine,
                     const std::vector<int32_t>& fixed_rows,
                     int64_t coarse_max, HostHierarchy& H);

}  // namespace fs
