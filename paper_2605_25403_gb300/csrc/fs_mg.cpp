// Host-side construction of the multigrid hierarchies used by the block
// preconditioner (not in the paper, which names no preconditioner; see the
// Cahouet-Chabard reading in the design notes).  Prolongations are linear
// interpolation in the index space of the structured simplicial meshes:
// P1 on mesh n_{l+1} -> P1 on mesh n_l with n_{l+1} = ceil(n_l / 4) cells
// per axis (nested when 4 divides n_l), and, for the velocity block,
// P1 -> P2 on the finest mesh.  Coarsening by 4 per axis halves the number
// of levels against 2 (each level costs eight dependent passes of a V-cycle);
// the Chebyshev(3) interval [lmax/8, 1.1 lmax] of the smoother reaches down
// to the smallest eigenvalues (~0.15 lmax) of the modes a coarser grid of
// 4h spacing cannot represent.  Coarse operators are
// Galerkin products R A P with R = P^T.  The coarsest operator is inverted
// densely.  Built once per problem; the values are FP64.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <atomic>
#include <random>

#include "fs_internal.h"

namespace fs {

namespace {

HostCsr transpose(const HostCsr& P) {
  HostCsr R;
  R.nrow = P.ncol;
  R.ncol = P.nrow;
  R.rowptr.assign(R.nrow + 1, 0);
  for (int32_t c : P.col) R.rowptr[c + 1]++;
  for (int64_t r = 0; r < R.nrow; ++r) R.rowptr[r + 1] += R.rowptr[r];
  R.col.resize(P.nnz());
  R.val.resize(P.nnz());
  std::vector<int32_t> f(R.rowptr.begin(), R.rowptr.end() - 1);
  for (int64_t r = 0; r < P.nrow; ++r)
    for (int32_t k = P.rowptr[r]; k < P.rowptr[r + 1]; ++k) {
      int32_t dst = f[P.col[k]]++;
      R.col[dst] = (int32_t)r;
      R.val[dst] = P.val[k];
    }
  return R;
}

// C = A B (Gustavson, dense accumulator), columns sorted per row.
HostCsr spgemm(const HostCsr& A, const HostCsr& B) {
  HostCsr C;
  C.nrow = A.nrow;
  C.ncol = B.ncol;
  C.rowptr.assign(C.nrow + 1, 0);
  std::vector<double> acc(B.ncol, 0.0);
  std::vector<int32_t> mark(B.ncol, -1), cols;
  for (int64_t i = 0; i < A.nrow; ++i) {
    cols.clear();
    for (int32_t ka = A.rowptr[i]; ka < A.rowptr[i + 1]; ++ka) {
      int32_t k = A.col[ka];
      double a = A.val[ka];
      for (int32_t kb = B.rowptr[k]; kb < B.rowptr[k + 1]; ++kb) {
        int32_t j = B.col[kb];
        if (mark[j] != (int32_t)i) {
          mark[j] = (int32_t)i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * B.val[kb];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int32_t j : cols) {
      C.col.push_back(j);
      C.val.push_back(acc[j]);
    }
    C.rowptr[i + 1] = (int32_t)C.col.size();
  }
  return C;
}

// Linear interpolation from the structured simplicial mesh nc to nf (cells
// per axis) in index space: fine vertex i sits at i nc / nf on the coarse
// grid; its weights are the barycentric coordinates in the coarse Kuhn
// simplex (triangle) that contains it.
HostCsr p1_interp(int dim, const int* nf, const int* nc) {
  int64_t sf[3] = {nf[0] + 1, nf[1] + 1, dim == 3 ? nf[2] + 1 : 1};
  int64_t scn[3] = {nc[0] + 1, nc[1] + 1, dim == 3 ? nc[2] + 1 : 1};
  HostCsr P;
  P.nrow = sf[0] * sf[1] * sf[2];
  P.ncol = scn[0] * scn[1] * scn[2];
  P.rowptr.assign(P.nrow + 1, 0);
  for (int64_t v = 0; v < P.nrow; ++v) {
    int64_t fi[3] = {v % sf[0], (v / sf[0]) % sf[1], v / (sf[0] * sf[1])};
    int64_t I[3] = {0, 0, 0};
    double s[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      // exact rational position fi * nc / nf
      int64_t num = fi[a] * nc[a];
      I[a] = std::min<int64_t>(num / nf[a], nc[a] - 1);
      s[a] = (double)(num - I[a] * nf[a]) / (double)nf[a];
    }
    int ord[3] = {0, 1, 2};
    std::stable_sort(ord, ord + dim, [&](int x, int y) { return s[x] > s[y]; });
    std::vector<std::pair<int32_t, double>> ent;
    int64_t cur[3] = {I[0], I[1], I[2]};
    auto cid = [&](const int64_t* c) {
      return (int32_t)(c[0] + scn[0] * (c[1] + scn[1] * c[2]));
    };
    double w0 = 1.0 - s[ord[0]];
    if (w0 > 1e-14) ent.push_back({cid(cur), w0});
    for (int k = 0; k < dim; ++k) {
      cur[ord[k]] += 1;
      double w = s[ord[k]] - (k + 1 < dim ? s[ord[k + 1]] : 0.0);
      if (w > 1e-14) ent.push_back({cid(cur), w});
    }
    std::sort(ent.begin(), ent.end());
    for (auto& e : ent) {
      P.col.push_back(e.first);
      P.val.push_back(e.second);
    }
    P.rowptr[v + 1] = (int32_t)P.col.size();
  }
  return P;
}

// P1 -> P2 on the same mesh: vertices copy, edge midpoints average.
HostCsr p2_from_p1(const Mesh& m) {
  HostCsr P;
  P.nrow = m.n2;
  P.ncol = m.nv;
  P.rowptr.assign(P.nrow + 1, 0);
  for (int64_t v = 0; v < m.nv; ++v) {
    P.col.push_back((int32_t)v);
    P.val.push_back(1.0);
    P.rowptr[v + 1] = (int32_t)P.col.size();
  }
  for (int64_t e = 0; e < m.ne; ++e) {
    int32_t a = m.edges[2 * e], b = m.edges[2 * e + 1];
    P.col.push_back(std::min(a, b));
    P.val.push_back(0.5);
    P.col.push_back(std::max(a, b));
    P.val.push_back(0.5);
    P.rowptr[m.nv + e + 1] = (int32_t)P.col.size();
  }
  return P;
}

void finish_level(HostLevel& L) {
  const HostCsr& A = L.A;
  L.dinv.assign(A.nrow, 1.0);
  for (int64_t i = 0; i < A.nrow; ++i)
    for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k)
      if (A.col[k] == i && A.val[k] != 0.0) L.dinv[i] = 1.0 / A.val[k];
  // largest eigenvalue of D^-1 A by power iteration (30 steps)
  std::vector<double> v(A.nrow), w(A.nrow);
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (auto& x : v) x = U(g);
  double lam = 0;
  for (int it = 0; it < 30; ++it) {
    double nw = 0, nv = 0;
    for (int64_t i = 0; i < A.nrow; ++i) {
      double s = 0;
      for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) s += A.val[k] * v[A.col[k]];
      w[i] = L.dinv[i] * s;
      nw += w[i] * w[i];
      nv += v[i] * v[i];
    }
    lam = std::sqrt(nw / nv);
    double inv = 1.0 / std::sqrt(nw);
    for (int64_t i = 0; i < A.nrow; ++i) v[i] = w[i] * inv;
  }
  L.lmax = lam;
}

// Gauss-Jordan inverse with partial pivoting (n small).
bool dense_inverse(const HostCsr& A, std::vector<double>& inv) {
  int64_t n = A.nrow;
  std::vector<double> M(n * n, 0.0);
  inv.assign(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    for (int32_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) M[i * n + A.col[k]] += A.val[k];
    inv[i * n + i] = 1.0;
  }
  for (int64_t c = 0; c < n; ++c) {
    int64_t p = c;
    for (int64_t r = c + 1; r < n; ++r)
      if (std::fabs(M[r * n + c]) > std::fabs(M[p * n + c])) p = r;
    if (M[p * n + c] == 0.0) return false;
    if (p != c)
      for (int64_t j = 0; j < n; ++j) {
        std::swap(M[p * n + j], M[c * n + j]);
        std::swap(inv[p * n + j], inv[c * n + j]);
      }
    double d = 1.0 / M[c * n + c];
    for (int64_t j = 0; j < n; ++j) {
      M[c * n + j] *= d;
      inv[c * n + j] *= d;
    }
    for (int64_t r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = M[r * n + c];
      if (f == 0.0) continue;
      for (int64_t j = 0; j < n; ++j) {
        M[r * n + j] -= f * M[c * n + j];
        inv[r * n + j] -= f * inv[c * n + j];
      }
    }
  }
  return true;
}

// Order of the rows of a P2 level: the nodes sit on the doubled lattice of
// the mesh (a vertex at twice its grid indices, an edge node at the sum of its
// end points' indices); they are grouped by the parity class of their
// doubled coordinates (vertices, then each edge direction) and ordered
// lexicographically (x fastest) within a class.  Rows of one class along a
// grid line then have the same stencil shifted by one, so the neighbours that
// 32 consecutive rows read at one matrix slot are contiguous.  Returns sigma
// (new row -> mesh row); vertices keep their numbers.
std::vector<int32_t> class_order(const Mesh& m, const HostLevel& L) {
  const int dim = m.dim;
  const int64_t sx = L.grid[0] + 1, sy = L.grid[1] + 1, sz = dim == 3 ? L.grid[2] + 1 : 1;
  const int64_t nv = sx * sy * sz;
  auto ijk = [&](int64_t v, int64_t* c) {
    c[0] = v % sx;
    c[1] = (v / sx) % sy;
    c[2] = v / (sx * sy);
  };
  const int64_t n = L.A.nrow;
  const int64_t X = 2 * sx, Y = 2 * sy;
  std::vector<std::pair<int64_t, int32_t>> key(n);
  for (int64_t r = 0; r < n; ++r) {
    int64_t c[3];
    if (r < nv) {
      ijk(r, c);
      for (int a = 0; a < 3; ++a) c[a] *= 2;
    } else {
      int64_t ca[3], cb[3];
      ijk(m.edges[2 * (r - nv)], ca);
      ijk(m.edges[2 * (r - nv) + 1], cb);
      for (int a = 0; a < 3; ++a) c[a] = ca[a] + cb[a];
    }
    const int64_t cls = (c[0] & 1) | (c[1] & 1) << 1 | (c[2] & 1) << 2;
    key[r] = {((cls * (2 * sz) + c[2]) * Y + c[1]) * X + c[0], (int32_t)r};
  }
  std::sort(key.begin(), key.end());
  std::vector<int32_t> sigma(n);
  for (int64_t r = 0; r < n; ++r) sigma[r] = key[r].second;
  return sigma;
}

// M' with M'[r] = M[rows[r]] and columns renumbered by cinv (old -> new),
// columns sorted per row.
HostCsr permute(const HostCsr& M, const std::vector<int32_t>& rows,
                const std::vector<int32_t>& cinv) {
  HostCsr O;
  O.nrow = M.nrow;
  O.ncol = M.ncol;
  O.rowptr.assign(O.nrow + 1, 0);
  O.col.reserve(M.nnz());
  O.val.reserve(M.nnz());
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t r = 0; r < O.nrow; ++r) {
    const int32_t o = rows[r];
    row.clear();
    for (int32_t k = M.rowptr[o]; k < M.rowptr[o + 1]; ++k)
      row.push_back({cinv[M.col[k]], M.val[k]});
    std::sort(row.begin(), row.end());
    for (auto& e : row) {
      O.col.push_back(e.first);
      O.val.push_back(e.second);
    }
    O.rowptr[r + 1] = (int32_t)O.col.size();
  }
  return O;
}

std::vector<int32_t> inverse(const std::vector<int32_t>& sigma) {
  std::vector<int32_t> inv(sigma.size());
  for (size_t r = 0; r < sigma.size(); ++r) inv[sigma[r]] = (int32_t)r;
  return inv;
}

// Renumbers the rows of a P2 finest level in class order (a symmetric
// permutation of its operator, with the transfer to the next level and the
// diagonal following); P1 levels keep the grid numbering, which already has
// that property.
void class_order_hierarchy(const Mesh& m, HostHierarchy& H) {
  H.order0.clear();
  HostLevel& L = H.levels[0];
  if (!L.p2) {
    H.order0.resize(L.A.nrow);
    std::iota(H.order0.begin(), H.order0.end(), 0);
    return;
  }
  std::vector<int32_t> sg = class_order(m, L), inv = inverse(sg);
  L.A = permute(L.A, sg, inv);
  std::vector<double> d(L.dinv.size());
  for (size_t r = 0; r < d.size(); ++r) d[r] = L.dinv[sg[r]];
  L.dinv.swap(d);
  if (H.levels.size() > 1) {
    std::vector<int32_t> id(L.P.ncol);
    std::iota(id.begin(), id.end(), 0);
    L.P = permute(L.P, sg, id);
    L.R = permute(L.R, id, inv);
  } else if (!H.coarse_inv.empty()) {
    const int64_t nc = H.ncoarse;
    std::vector<double> ci(nc * nc);
    for (int64_t r = 0; r < nc; ++r)
      for (int64_t c = 0; c < nc; ++c) ci[r * nc + c] = H.coarse_inv[sg[r] * nc + sg[c]];
    H.coarse_inv.swap(ci);
  }
  H.order0 = sg;
}

}  // namespace

void build_hierarchy(const Mesh& m, const HostCsr& A0, bool p2_fine,
                     const std::vector<int32_t>& fixed_rows,
                     int64_t coarse_max, HostHierarchy& H) {
  H.levels.clear();
  H.levels.emplace_back();
  H.levels[0].A = A0;
  int dim = m.dim;
  int ncur[3] = {m.desc.n[0], m.desc.n[1], dim == 3 ? m.desc.n[2] : 1};
  for (int a = 0; a < 3; ++a) H.levels[0].grid[a] = ncur[a];
  H.levels[0].p2 = p2_fine;
  bool first = true;
  while (H.levels.back().A.nrow > coarse_max) {
    HostLevel& fine = H.levels.back();
    HostCsr P;
    if (first && p2_fine) {
      P = p2_from_p1(m);  // coarse = P1 on the same mesh
    } else {
      int nn[3] = {ncur[0], ncur[1], ncur[2]};
      bool changed = false;
      for (int a = 0; a < dim; ++a) {
        nn[a] = std::max(1, (ncur[a] + 3) / 4);
        changed = changed || nn[a] != ncur[a];
      }
      if (!changed) break;
      P = p1_interp(dim, ncur, nn);
      for (int a = 0; a < dim; ++a) ncur[a] = nn[a];
    }
    if (first)
      for (int32_t r : fixed_rows)
        for (int32_t k = P.rowptr[r]; k < P.rowptr[r + 1]; ++k) P.val[k] = 0.0;
    first = false;
    HostCsr R = transpose(P);
    HostCsr Ac = spgemm(R, spgemm(fine.A, P));
    for (int64_t i = 0; i < Ac.nrow; ++i) {
      bool has = false;
      for (int32_t k = Ac.rowptr[i]; k < Ac.rowptr[i + 1]; ++k)
        if (Ac.col[k] == i && Ac.val[k] != 0.0) has = true;
      if (!has) {  // an unreachable coarse node: make its row the identity
        for (int32_t k = Ac.rowptr[i]; k < Ac.rowptr[i + 1]; ++k) Ac.val[k] = 0.0;
        bool found = false;
        for (int32_t k = Ac.rowptr[i]; k < Ac.rowptr[i + 1]; ++k)
          if (Ac.col[k] == i) { Ac.val[k] = 1.0; found = true; }
        if (!found) {  // insert a diagonal entry
          HostCsr B2 = Ac;
          B2.col.insert(B2.col.begin() + Ac.rowptr[i], (int32_t)i);
          B2.val.insert(B2.val.begin() + Ac.rowptr[i], 1.0);
          for (int64_t r = i + 1; r <= Ac.nrow; ++r) B2.rowptr[r]++;
          // keep the row sorted
          auto b = B2.col.begin() + B2.rowptr[i], e = B2.col.begin() + B2.rowptr[i + 1];
          std::vector<std::pair<int32_t, double>> row;
          for (auto it = b; it != e; ++it)
            row.push_back({*it, B2.val[it - B2.col.begin()]});
          std::sort(row.begin(), row.end());
          for (size_t k = 0; k < row.size(); ++k) {
            B2.col[B2.rowptr[i] + k] = row[k].first;
            B2.val[B2.rowptr[i] + k] = row[k].second;
          }
          Ac = B2;
        }
      }
    }
    fine.P = P;
    fine.R = R;
    H.levels.emplace_back();
    H.levels.back().A = Ac;
    for (int a = 0; a < 3; ++a) H.levels.back().grid[a] = ncur[a];
  }
  for (auto& L : H.levels) finish_level(L);
  H.ncoarse = H.levels.back().A.nrow;
  if (H.ncoarse > kHostInverseMax) {
    H.coarse_inv.clear();  // inverted on the device after the upload
  } else if (!dense_inverse(H.levels.back().A, H.coarse_inv)) {
    // singular coarsest operator: fall back to its Jacobi inverse
    H.coarse_inv.assign(H.ncoarse * H.ncoarse, 0.0);
    for (int64_t i = 0; i < H.ncoarse; ++i)
      H.coarse_inv[i * H.ncoarse + i] = H.levels.back().dinv[i];
  }
  class_order_hierarchy(m, H);
}

}  // namespace fs

// ---------------------------------------------------------------------------
// Batched (union) hierarchies
// ---------------------------------------------------------------------------
#include <thread>

namespace fs {

namespace {

// Edges/sizes of instance i in its own numbering (what build_hierarchy needs).
Mesh local_view(const Mesh& m, int i) {
  const Instance& I = m.inst[i];
  Mesh L;
  L.desc = I.desc;
  L.dim = m.dim;
  L.nb = m.nb;
  L.nloc = m.nloc;
  L.nv = I.nv;
  L.ne = I.ne;
  L.n2 = I.nv + I.ne;
  L.ncell = I.ncell;
  L.edges.resize(2 * I.ne);
  for (int64_t e = 0; e < I.ne; ++e) {
    L.edges[2 * e] = (int32_t)(m.edges[2 * (I.eoff + e)] - I.voff);
    L.edges[2 * e + 1] = (int32_t)(m.edges[2 * (I.eoff + e) + 1] - I.voff);
  }
  return L;
}

HostCsr identity(int64_t n) {
  HostCsr I;
  I.nrow = I.ncol = n;
  I.rowptr.resize(n + 1);
  I.col.resize(n);
  I.val.assign(n, 1.0);
  for (int64_t i = 0; i <= n; ++i) I.rowptr[i] = (int32_t)i;
  for (int64_t i = 0; i < n; ++i) I.col[i] = (int32_t)i;
  return I;
}

// Block-diagonal concatenation.
HostCsr block_diag(const std::vector<const HostCsr*>& blocks) {
  HostCsr C;
  for (auto* b : blocks) {
    C.nrow += b->nrow;
    C.ncol += b->ncol;
  }
  C.rowptr.assign(C.nrow + 1, 0);
  int64_t r0 = 0, c0 = 0;
  for (auto* b : blocks) {
    for (int64_t r = 0; r < b->nrow; ++r) {
      for (int32_t k = b->rowptr[r]; k < b->rowptr[r + 1]; ++k) {
        C.col.push_back((int32_t)(c0 + b->col[k]));
        C.val.push_back(b->val[k]);
      }
      C.rowptr[r0 + r + 1] = (int32_t)C.col.size();
    }
    r0 += b->nrow;
    c0 += b->ncol;
  }
  return C;
}

}  // namespace

void build_union_hierarchy(const Mesh& m, const std::vector<Mesh>& /*local*/,
                           const HostCsr& A0, bool p2_fine,
                           const std::vector<int32_t>& fixed, int64_t coarse_max,
                           UnionHierarchy& U) {
  const int K = (int)m.inst.size();
  // union row -> (instance, local row)
  std::vector<int32_t> owner(A0.nrow, -1);
  std::vector<int64_t> local(A0.nrow, -1);
  for (int i = 0; i < K; ++i) {
    const Instance& I = m.inst[i];
    int64_t n = p2_fine ? I.n2() : I.nv;
    for (int64_t j = 0; j < n; ++j) {
      int64_t g = p2_fine ? union_node(m, i, j) : I.voff + j;
      owner[g] = i;
      local[g] = j;
    }
  }
  std::vector<HostHierarchy> H(K);
  auto work = [&](int i) {
    const Instance& I = m.inst[i];
    Mesh L = local_view(m, i);
    HostCsr Ai;
    Ai.nrow = Ai.ncol = p2_fine ? I.n2() : I.nv;
    Ai.rowptr.assign(Ai.nrow + 1, 0);
    for (int64_t j = 0; j < Ai.nrow; ++j) {
      int64_t g = p2_fine ? union_node(m, i, j) : I.voff + j;
      for (int32_t k = A0.rowptr[g]; k < A0.rowptr[g + 1]; ++k) {
        // block-diagonal: every column belongs to the same instance, and the
        // union order restricted to one instance is its local order
        Ai.col.push_back((int32_t)local[A0.col[k]]);
        Ai.val.push_back(A0.val[k]);
      }
      Ai.rowptr[j + 1] = (int32_t)Ai.col.size();
    }
    std::vector<int32_t> fx;
    for (int32_t g : fixed)
      if (owner[g] == i) fx.push_back((int32_t)local[g]);
    build_hierarchy(L, Ai, p2_fine, fx, coarse_max, H[i]);
  };
  int nthr = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u);
  if (K == 1 || nthr == 1) {
    for (int i = 0; i < K; ++i) work(i);
  } else {
    std::vector<std::thread> pool;
    std::atomic<int> next{0};
    for (int t = 0; t < std::min(nthr, K); ++t)
      pool.emplace_back([&]() {
        for (int i = next++; i < K; i = next++) work(i);
      });
    for (auto& th : pool) th.join();
  }
  int depth = 0;
  for (int i = 0; i < K; ++i) depth = std::max(depth, (int)H[i].levels.size());
  U.H.levels.assign(depth, HostLevel());
  U.inst_off.clear();
  for (int l = 0; l < depth; ++l) {
    std::vector<const HostCsr*> As, Ps, Rs;
    std::vector<HostCsr> ids;
    ids.reserve(K);
    HostLevel& UL = U.H.levels[l];
    UL.lmax = 0;
    for (int i = 0; i < K; ++i) {
      int li = std::min(l, (int)H[i].levels.size() - 1);
      const HostLevel& hl = H[i].levels[li];
      As.push_back(&hl.A);
      UL.dinv.insert(UL.dinv.end(), hl.dinv.begin(), hl.dinv.end());
      UL.lmax = std::max(UL.lmax, hl.lmax);
      if (l + 1 < depth) {
        if (l + 1 < (int)H[i].levels.size()) {
          Ps.push_back(&hl.P);
          Rs.push_back(&hl.R);
        } else {
          ids.push_back(identity(hl.A.nrow));
          Ps.push_back(&ids.back());
          Rs.push_back(&ids.back());
        }
      }
    }
    UL.A = block_diag(As);
    std::vector<int64_t> off(1, 0);
    for (const HostCsr* a : As) off.push_back(off.back() + a->nrow);
    U.inst_off.push_back(off);
    if (l + 1 < depth) {
      UL.P = block_diag(Ps);
      UL.R = block_diag(Rs);
    }
  }
  // level-0 rows (instance blocks, each in Z-order) vs the union numbering
  U.perm.clear();
  U.perm.reserve(A0.nrow);
  bool identity = true;
  for (int i = 0; i < K; ++i)
    for (int32_t j : H[i].order0) {
      const int32_t g = (int32_t)(p2_fine ? union_node(m, i, j) : m.inst[i].voff + j);
      identity = identity && g == (int32_t)U.perm.size();
      U.perm.push_back(g);
    }
  if (identity) U.perm.clear();
  // coarsest: block-diagonal dense inverses
  U.blk_row.assign(K, 0);
  U.blk_n.assign(K, 0);
  U.blk_dense.assign(K, 0);
  U.dense.clear();
  U.row_blk.clear();
  int64_t row = 0;
  for (int i = 0; i < K; ++i) {
    U.blk_row[i] = row;
    U.blk_n[i] = H[i].ncoarse;
    U.blk_dense[i] = (int64_t)U.dense.size();
    if (H[i].coarse_inv.empty() && K > 1 &&
        !dense_inverse(H[i].levels.back().A, H[i].coarse_inv)) {
      // (batches keep their coarsest blocks small; a large one is inverted
      // here, singular ones fall back to Jacobi)
      H[i].coarse_inv.assign(H[i].ncoarse * H[i].ncoarse, 0.0);
      for (int64_t q = 0; q < H[i].ncoarse; ++q)
        H[i].coarse_inv[q * H[i].ncoarse + q] = H[i].levels.back().dinv[q];
    }
    U.dense.insert(U.dense.end(), H[i].coarse_inv.begin(), H[i].coarse_inv.end());
    for (int64_t r = 0; r < H[i].ncoarse; ++r) U.row_blk.push_back(i);
    row += H[i].ncoarse;
  }
  U.H.ncoarse = row;
}

}  // namespace fs
