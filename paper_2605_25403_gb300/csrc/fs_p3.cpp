// Host tables of the Taylor-Hood P3/P2 pair on triangles (paper Sec. 4.1,
// the P3-P2 convergence experiment, which the paper solves by IPCS): the P3
// velocity and P2 pressure DOF maps of a structured triangle mesh, their
// block CSR patterns with per-element slot tables, and the reference-element
// integrals of the P3/P2 basis.
//
// Numbering: velocity P3 nodes are the vertices, then two nodes per edge in
// the lexicographic order of the edges (the one nearer the edge's smaller
// vertex id first), then one interior node per cell; pressure P2 nodes are
// the vertices, then one node per edge, in the paper order of fs_dof_map.
// Local P3 order: vertices 0, 1, 2; for each of the edges (1,2), (2,0),
// (0,1) the node nearer its first vertex, then the other; the interior node.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "fs_internal.h"

namespace fs {

namespace {

constexpr int kP3Edge[3][2] = {{1, 2}, {2, 0}, {0, 1}};

// Block pattern of the rows of table R (nr local nodes per cell, nrow rows)
// against the columns of table C (nc per cell), columns ascending, and the
// slot table pos[(e nr + i) nc + j] = position of C's node j in the row of
// R's node i.  False when a row is longer than 256 entries.
bool pattern_and_slots(int64_t ncell, int64_t nrow, const std::vector<int32_t>& R, int nr,
                       const std::vector<int32_t>& C, int nc, HostCsr& P,
                       std::vector<uint8_t>& pos) {
  std::vector<std::vector<int32_t>> rows(nrow);
  for (int64_t e = 0; e < ncell; ++e)
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nc; ++j) rows[R[e * nr + i]].push_back(C[e * nc + j]);
  P.nrow = nrow;
  P.rowptr.assign(nrow + 1, 0);
  P.col.clear();
  for (int64_t r = 0; r < nrow; ++r) {
    auto& v = rows[r];
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    if (v.size() > 256) return false;
    P.col.insert(P.col.end(), v.begin(), v.end());
    P.rowptr[r + 1] = (int32_t)P.col.size();
  }
  pos.resize(ncell * nr * nc);
  for (int64_t e = 0; e < ncell; ++e)
    for (int i = 0; i < nr; ++i) {
      const int32_t r = R[e * nr + i];
      const int32_t* b = P.col.data() + P.rowptr[r];
      const int32_t* en = P.col.data() + P.rowptr[r + 1];
      for (int j = 0; j < nc; ++j)
        pos[(e * nr + i) * nc + j] = (uint8_t)(std::lower_bound(b, en, C[e * nc + j]) - b);
    }
  return true;
}

// P3 basis values and derivatives d phi / d lambda_r at barycentric point l.
void p3_eval(const double* l, double (&phi)[10], double (&d)[10][3]) {
  for (auto& row : d) row[0] = row[1] = row[2] = 0;
  for (int v = 0; v < 3; ++v) {
    const double x = l[v];
    phi[v] = 0.5 * x * (3 * x - 1) * (3 * x - 2);
    d[v][v] = 0.5 * (27 * x * x - 18 * x + 2);
  }
  for (int le = 0; le < 3; ++le) {
    const int a = kP3Edge[le][0], b = kP3Edge[le][1];
    for (int h = 0; h < 2; ++h) {
      const int near = h == 0 ? a : b, k = 3 + 2 * le + h;
      const double f = 3 * l[near] - 1;
      phi[k] = 4.5 * l[a] * l[b] * f;
      d[k][a] = 4.5 * (l[b] * f + (near == a ? 3 * l[a] * l[b] : 0.0));
      d[k][b] = 4.5 * (l[a] * f + (near == b ? 3 * l[a] * l[b] : 0.0));
    }
  }
  phi[9] = 27 * l[0] * l[1] * l[2];
  d[9][0] = 27 * l[1] * l[2];
  d[9][1] = 27 * l[0] * l[2];
  d[9][2] = 27 * l[0] * l[1];
}

void p2_eval(const double* l, double (&psi)[6], double (&d)[6][3]) {
  for (auto& row : d) row[0] = row[1] = row[2] = 0;
  for (int v = 0; v < 3; ++v) {
    psi[v] = l[v] * (2 * l[v] - 1);
    d[v][v] = 4 * l[v] - 1;
  }
  for (int le = 0; le < 3; ++le) {
    const int a = kP3Edge[le][0], b = kP3Edge[le][1];
    psi[3 + le] = 4 * l[a] * l[b];
    d[3 + le][a] = 4 * l[b];
    d[3 + le][b] = 4 * l[a];
  }
}

void compositions3(int total, int parts, std::vector<int>& cur,
                   std::vector<std::vector<int>>& out) {
  if (parts == 1) {
    cur.push_back(total);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int k = 0; k <= total; ++k) {
    cur.push_back(k);
    compositions3(total - k, parts - 1, cur, out);
    cur.pop_back();
  }
}

double factorial(int k) {
  double f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

}  // namespace

int build_p3_tables(const Mesh& m, P3Tables& T) {
  if (m.dim != 2 || m.inst.size() != 1) {
    set_error("P3/P2 problems need a single 2D mesh");
    return FS_ERR_UNSUPPORTED;
  }
  std::vector<int32_t> c2d;
  std::vector<uint8_t> dir;
  natural_dof_map(m, &c2d, &dir, nullptr, nullptr);  // P2 map in the paper order
  const int64_t nv = m.nv, ne = m.ne, nc = m.ncell;
  T.ncell = nc;
  T.n3 = nv + 2 * ne + nc;
  T.np = nv + ne;
  T.c2p.assign(c2d.begin(), c2d.end());
  T.c2u.resize(nc * 10);
  T.dir.assign(T.n3, 0);
  for (int64_t q = 0; q < nv; ++q) T.dir[q] = dir[q];
  for (int64_t e = 0; e < nc; ++e) {
    const int32_t* g = &c2d[e * 6];
    int32_t* u = &T.c2u[e * 10];
    for (int v = 0; v < 3; ++v) u[v] = g[v];
    for (int le = 0; le < 3; ++le) {
      const int64_t r = g[3 + le] - nv;  // edge rank
      const bool lo_first = g[kP3Edge[le][0]] < g[kP3Edge[le][1]];
      u[3 + 2 * le] = (int32_t)(nv + 2 * r + (lo_first ? 0 : 1));
      u[4 + 2 * le] = (int32_t)(nv + 2 * r + (lo_first ? 1 : 0));
      T.dir[nv + 2 * r] = T.dir[nv + 2 * r + 1] = dir[g[3 + le]];
    }
    u[9] = (int32_t)(nv + 2 * ne + e);
  }
  T.dlist.clear();
  for (int64_t q = 0; q < T.n3; ++q)
    if (T.dir[q]) T.dlist.push_back((int32_t)q);
  // node coordinates: barycentric positions of the local nodes
  T.xyz.assign(T.n3 * 2, 0.0);
  T.pxyz.assign(T.np * 2, 0.0);
  for (int64_t e = 0; e < nc; ++e) {
    const int32_t* u = &T.c2u[e * 10];
    double X[3][2];
    for (int v = 0; v < 3; ++v)
      for (int a = 0; a < 2; ++a) X[v][a] = m.coords[(int64_t)u[v] * 2 + a];
    for (int k = 0; k < 10; ++k) {
      double l[3] = {0, 0, 0};
      if (k < 3) {
        l[k] = 1;
      } else if (k < 9) {
        const int le = (k - 3) / 2, h = (k - 3) % 2;
        const int a = kP3Edge[le][0], b = kP3Edge[le][1];
        l[h == 0 ? a : b] = 2.0 / 3.0;
        l[h == 0 ? b : a] = 1.0 / 3.0;
      } else {
        l[0] = l[1] = l[2] = 1.0 / 3.0;
      }
      for (int a = 0; a < 2; ++a)
        T.xyz[(int64_t)u[k] * 2 + a] = l[0] * X[0][a] + l[1] * X[1][a] + l[2] * X[2][a];
    }
    const int32_t* g = &c2d[e * 6];
    for (int v = 0; v < 3; ++v)
      for (int a = 0; a < 2; ++a) T.pxyz[(int64_t)g[v] * 2 + a] = X[v][a];
    for (int le = 0; le < 3; ++le)
      for (int a = 0; a < 2; ++a)
        T.pxyz[(int64_t)g[3 + le] * 2 + a] =
            0.5 * (X[kP3Edge[le][0]][a] + X[kP3Edge[le][1]][a]);
  }
  if (!pattern_and_slots(nc, T.n3, T.c2u, 10, T.c2u, 10, T.A, T.posA) ||
      !pattern_and_slots(nc, T.np, T.c2p, 6, T.c2u, 10, T.B, T.posB) ||
      !pattern_and_slots(nc, T.n3, T.c2u, 10, T.c2p, 6, T.BT, T.posBT) ||
      !pattern_and_slots(nc, T.np, T.c2p, 6, T.c2p, 6, T.Kp, T.posK)) {
    set_error("P3/P2 tables: a CSR row is longer than 256 entries");
    return FS_ERR_INVALID_MESH;
  }
  T.A.ncol = T.n3;
  T.B.ncol = T.n3;
  T.BT.ncol = T.np;
  T.Kp.ncol = T.np;
  return FS_OK;
}

// Reference-triangle integrals by the Grundmann-Moeller rule of degree 9
// (s = 4; exact for the degree-8 convection integrand).
void p3_ref_tensors(RefP3& R) {
  R = RefP3{};
  const int s = 4, deg = 2 * s + 1, n = 2;
  for (int i = 0; i <= s; ++i) {
    const double w = ((i % 2) ? -1.0 : 1.0) * std::ldexp(1.0, -2 * s) *
                     std::pow((double)(deg + n - 2 * i), deg) /
                     (factorial(i) * factorial(deg + n - i));
    std::vector<std::vector<int>> betas;
    std::vector<int> cur;
    compositions3(s - i, n + 1, cur, betas);
    for (auto& b : betas) {
      double l[3];
      for (int k = 0; k <= n; ++k) l[k] = (2.0 * b[k] + 1.0) / (double)(deg + n - 2 * i);
      double phi[10], dphi[10][3], psi[6], dpsi[6][3];
      p3_eval(l, phi, dphi);
      p2_eval(l, psi, dpsi);
      for (int a = 0; a < 10; ++a)
        for (int c = 0; c < 10; ++c) {
          R.mass[a][c] += w * phi[a] * phi[c];
          for (int r = 0; r < 3; ++r)
            for (int t = 0; t < 3; ++t) R.stiff[a][c][r][t] += w * dphi[a][r] * dphi[c][t];
          for (int j = 0; j < 10; ++j)
            for (int r = 0; r < 3; ++r) R.conv[a][c][j][r] += w * phi[a] * phi[c] * dphi[j][r];
        }
      for (int q = 0; q < 6; ++q) {
        for (int j = 0; j < 10; ++j)
          for (int r = 0; r < 3; ++r) R.div[q][j][r] += w * psi[q] * dphi[j][r];
        for (int q2 = 0; q2 < 6; ++q2)
          for (int r = 0; r < 3; ++r)
            for (int t = 0; t < 3; ++t) R.pstiff[q][q2][r][t] += w * dpsi[q][r] * dpsi[q2][t];
      }
    }
  }
}

}  // namespace fs
