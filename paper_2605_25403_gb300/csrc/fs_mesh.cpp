// Host-side mesh, P2/P1 DOF map, block CSR patterns and per-element slot
// tables; reference-simplex integrals by a Grundmann-Moeller rule.
//
// Paper: Sec. 2.2.1 (conforming simplicial mesh, Taylor-Hood spaces V_h, Q_h
// with k = 2) and Sec. 3.1 (Common level: meshes, function spaces; Simulation
// base class: DOF management).  The mesh generator plays the role of the
// paper's init_mesh['uniform_tri'](nx, ny) of Sec. 3.3, extended to Kuhn
// tetrahedra in 3D.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "fs_internal.h"

namespace fs {

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): one output of the generator whose
// state is `s` before the step.
uint64_t splitmix64_next(uint64_t s) {
  s += 0x9E3779B97F4A7C15ULL;
  s = (s ^ (s >> 30)) * 0xBF58476D1CE4E5B9ULL;
  s = (s ^ (s >> 27)) * 0x94D049BB133111EBULL;
  return s ^ (s >> 31);
}

double unit_draw(uint64_t seed, uint64_t key) {
  return std::ldexp((double)(splitmix64_next(seed ^ key) >> 11), -53);
}

const int kTriEdge[3][2] = {{1, 2}, {2, 0}, {0, 1}};
const int kTetEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

// Rows = local nodes [r0, r0 + nr) of each cell, columns = [c0, c0 + nc).
void cell_pattern(const Mesh& m, int64_t nrow, int r0, int nr, int c0, int nc,
                  HostCsr& out) {
  out.nrow = nrow;
  std::vector<int64_t> cnt(nrow + 1, 0);
  for (int64_t c = 0; c < m.ncell; ++c)
    for (int a = 0; a < nr; ++a) cnt[m.c2d[c * m.nloc + r0 + a] + 1] += nc;
  for (int64_t r = 0; r < nrow; ++r) cnt[r + 1] += cnt[r];
  std::vector<int32_t> buf(cnt[nrow]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int64_t c = 0; c < m.ncell; ++c) {
    const int32_t* g = &m.c2d[c * m.nloc];
    for (int a = 0; a < nr; ++a) {
      int32_t row = g[r0 + a];
      for (int b = 0; b < nc; ++b) buf[fill[row]++] = g[c0 + b];
    }
  }
  out.rowptr.assign(nrow + 1, 0);
  out.col.clear();
  out.col.reserve(cnt[nrow] / 4 + 16);
  for (int64_t r = 0; r < nrow; ++r) {
    auto b = buf.begin() + cnt[r], e = buf.begin() + cnt[r + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    out.col.insert(out.col.end(), b, e);
    out.rowptr[r + 1] = (int32_t)out.col.size();
  }
}

// Position of each (row node, col node) pair of every cell in its CSR row.
bool cell_slots(const Mesh& m, const HostCsr& P, int r0, int nr, int c0,
                int nc, std::vector<uint8_t>& pos) {
  pos.assign((size_t)m.ncell * nr * nc, 0);
  for (int64_t c = 0; c < m.ncell; ++c) {
    const int32_t* g = &m.c2d[c * m.nloc];
    for (int a = 0; a < nr; ++a) {
      int32_t row = g[r0 + a];
      const int32_t* b0 = P.col.data() + P.rowptr[row];
      const int32_t* b1 = P.col.data() + P.rowptr[row + 1];
      for (int b = 0; b < nc; ++b) {
        const int32_t* it = std::lower_bound(b0, b1, g[c0 + b]);
        int64_t off = it - b0;
        if (it == b1 || *it != g[c0 + b] || off > 255) return false;
        pos[((size_t)c * nr + a) * nc + b] = (uint8_t)off;
      }
    }
  }
  return true;
}

}  // namespace

namespace {
int build_local(const fs_mesh_desc& d, Mesh& m);
int finalize_patterns(Mesh& m);
}  // namespace

int build_mesh(const fs_mesh_desc& d, Mesh& m) {
  int rc = build_local(d, m);
  if (rc != FS_OK) return rc;
  Instance I;
  I.desc = d;
  I.voff = 0;
  I.nv = m.nv;
  I.eoff = 0;
  I.ne = m.ne;
  I.coff = 0;
  I.ncell = m.ncell;
  m.inst.assign(1, I);
  return finalize_patterns(m);
}

int build_batch_mesh(const fs_mesh_desc* d, int count, Mesh& m) {
  if (count < 1 || !d) {
    set_error("fs_mesh_create_batch: need at least one description");
    return FS_ERR_INVALID_ARG;
  }
  std::vector<Mesh> loc(count);
  for (int i = 0; i < count; ++i) {
    if (d[i].dim != d[0].dim) {
      set_error("fs_mesh_create_batch: all instances must have the same dimension");
      return FS_ERR_INVALID_ARG;
    }
    int rc = build_local(d[i], loc[i]);
    if (rc != FS_OK) return rc;
  }
  const int dim = d[0].dim;
  m = Mesh();
  m.desc = d[0];
  m.dim = dim;
  m.nb = dim + 1;
  m.nloc = dim == 2 ? 6 : 10;
  m.inst.resize(count);
  for (int i = 0; i < count; ++i) {
    Instance& I = m.inst[i];
    I.desc = d[i];
    I.voff = m.nv;
    I.nv = loc[i].nv;
    I.eoff = m.ne;
    I.ne = loc[i].ne;
    I.coff = m.ncell;
    I.ncell = loc[i].ncell;
    m.nv += I.nv;
    m.ne += I.ne;
    m.ncell += I.ncell;
  }
  m.n2 = m.nv + m.ne;
  if (m.ncell * (dim == 2 ? 36 : 100) >= (int64_t)1 << 31) {
    set_error("fs_mesh_create_batch: batch too large for int32 CSR offsets");
    return FS_ERR_INVALID_ARG;
  }
  m.coords.resize(m.nv * dim);
  m.p2xyz.resize(m.n2 * dim);
  m.c2d.resize(m.ncell * m.nloc);
  m.edges.resize(m.ne * 2);
  m.dirichlet.resize(m.n2);
  m.node_nat.resize(m.n2);
  for (int i = 0; i < count; ++i) {
    const Mesh& L = loc[i];
    const Instance& I = m.inst[i];
    for (int64_t j = 0; j < L.n2; ++j)
      m.node_nat[union_node(m, i, j)] = (int32_t)union_node(m, i, L.node_nat[j]);
    std::memcpy(&m.coords[I.voff * dim], L.coords.data(), sizeof(double) * L.nv * dim);
    for (int64_t j = 0; j < L.n2; ++j) {
      int64_t g = union_node(m, i, j);
      for (int a = 0; a < dim; ++a) m.p2xyz[g * dim + a] = L.p2xyz[j * dim + a];
      m.dirichlet[g] = L.dirichlet[j];
    }
    for (int64_t e = 0; e < L.ne; ++e) {
      m.edges[2 * (I.eoff + e)] = (int32_t)(I.voff + L.edges[2 * e]);
      m.edges[2 * (I.eoff + e) + 1] = (int32_t)(I.voff + L.edges[2 * e + 1]);
    }
    for (int64_t c = 0; c < L.ncell; ++c)
      for (int a = 0; a < m.nloc; ++a)
        m.c2d[(I.coff + c) * m.nloc + a] = (int32_t)union_node(m, i, L.c2d[c * m.nloc + a]);
  }
  m.dlist.clear();
  for (int64_t i = 0; i < m.n2; ++i)
    if (m.dirichlet[i]) m.dlist.push_back((int32_t)i);
  return finalize_patterns(m);
}

namespace {

int build_local(const fs_mesh_desc& d, Mesh& m) {
  if (d.dim != 2 && d.dim != 3) {
    set_error("fs_mesh_create: dim must be 2 or 3");
    return FS_ERR_INVALID_ARG;
  }
  int64_t cells_total = 1;
  for (int a = 0; a < d.dim; ++a) {
    if (d.n[a] < 1 || !(d.hi[a] > d.lo[a])) {
      set_error("fs_mesh_create: need n >= 1 and hi > lo on every axis");
      return FS_ERR_INVALID_ARG;
    }
    cells_total *= d.n[a];
  }
  if (!(d.jitter >= 0.0 && d.jitter < 0.25)) {
    set_error("fs_mesh_create: jitter must be in [0, 0.25)");
    return FS_ERR_INVALID_ARG;
  }
  const int dim = d.dim;
  m.desc = d;
  m.dim = dim;
  m.nb = dim + 1;
  m.nloc = dim == 2 ? 6 : 10;
  int n[3] = {d.n[0], d.n[1], dim == 3 ? d.n[2] : 0};
  m.ncell = cells_total * (dim == 2 ? 2 : 6);
  // 2^31 guard: int32 node ids and CSR offsets
  if (m.ncell * (dim == 2 ? 36 : 100) >= (int64_t)1 << 31) {
    set_error("fs_mesh_create: mesh too large for int32 CSR offsets");
    return FS_ERR_INVALID_ARG;
  }
  const int64_t sx = n[0] + 1, sy = n[1] + 1;
  m.nv = sx * sy * (dim == 3 ? (n[2] + 1) : 1);
  double h[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) h[a] = (d.hi[a] - d.lo[a]) / (double)n[a];

  // vertices: x = lo + i h, interior ones jittered
  m.coords.resize(m.nv * dim);
  for (int64_t v = 0; v < m.nv; ++v) {
    int64_t ijk[3] = {v % sx, (v / sx) % sy, dim == 3 ? v / (sx * sy) : 0};
    bool inner = true;
    for (int a = 0; a < dim; ++a) inner = inner && ijk[a] > 0 && ijk[a] < n[a];
    for (int a = 0; a < dim; ++a) {
      double x = d.lo[a] + (double)ijk[a] * h[a];
      if (inner && d.jitter != 0.0) {
        double U = unit_draw(d.seed, (uint64_t)(3 * v + a));
        x = x + d.jitter * h[a] * (2.0 * U - 1.0);
      }
      m.coords[v * dim + a] = x;
    }
  }

  // cells, P1 part of c2d
  m.c2d.assign(m.ncell * m.nloc, 0);
  {
    int64_t c = 0;
    if (dim == 2) {
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int32_t a = (int32_t)(i + sx * j);
          int32_t quad[4] = {a, a + 1, (int32_t)(a + 1 + sx), (int32_t)(a + sx)};
          // along the diagonal quad[0]-quad[2]
          int32_t* t = &m.c2d[(c++) * m.nloc];
          t[0] = quad[0]; t[1] = quad[1]; t[2] = quad[2];
          t = &m.c2d[(c++) * m.nloc];
          t[0] = quad[0]; t[1] = quad[2]; t[2] = quad[3];
        }
    } else {
      // the 6 axis orders, lexicographic
      const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                               {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
      const int64_t stride[3] = {1, sx, sx * sy};
      for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
          for (int i = 0; i < n[0]; ++i) {
            int64_t base = i + sx * j + sx * sy * k;
            for (int s = 0; s < 6; ++s) {
              int32_t* t = &m.c2d[(c++) * m.nloc];
              int64_t cur = base;
              t[0] = (int32_t)cur;
              for (int st = 0; st < 3; ++st) {
                cur += stride[order[s][st]];
                t[st + 1] = (int32_t)cur;
              }
            }
          }
    }
  }

  // degenerate-element check
  {
    double hd = 1;
    for (int a = 0; a < dim; ++a) hd *= h[a];
    for (int64_t c = 0; c < m.ncell; ++c) {
      const int32_t* t = &m.c2d[c * m.nloc];
      double J[3][3];
      for (int r = 0; r < dim; ++r)
        for (int a = 0; a < dim; ++a)
          J[a][r] = m.coords[(int64_t)t[r + 1] * dim + a] - m.coords[(int64_t)t[0] * dim + a];
      double det = dim == 2 ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                            : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                  J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                  J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      if (!(std::fabs(det) > 1e-12 * hd)) {
        set_error("fs_mesh_create: degenerate simplex " + std::to_string(c));
        return FS_ERR_INVALID_MESH;
      }
    }
  }

  // edges: per lower vertex, the sorted set of higher neighbours
  const int nle = dim == 2 ? 3 : 6;
  const int(*le)[2] = dim == 2 ? kTriEdge : kTetEdge;
  std::vector<int64_t> eoff(m.nv + 1, 0);
  for (int64_t c = 0; c < m.ncell; ++c)
    for (int e = 0; e < nle; ++e) {
      int32_t a = m.c2d[c * m.nloc + le[e][0]], b = m.c2d[c * m.nloc + le[e][1]];
      eoff[std::min(a, b) + 1]++;
    }
  for (int64_t v = 0; v < m.nv; ++v) eoff[v + 1] += eoff[v];
  std::vector<int32_t> hiv(eoff[m.nv]);
  {
    std::vector<int64_t> f(eoff.begin(), eoff.end() - 1);
    for (int64_t c = 0; c < m.ncell; ++c)
      for (int e = 0; e < nle; ++e) {
        int32_t a = m.c2d[c * m.nloc + le[e][0]], b = m.c2d[c * m.nloc + le[e][1]];
        hiv[f[std::min(a, b)]++] = std::max(a, b);
      }
  }
  std::vector<int64_t> first(m.nv + 1, 0);  // first edge id of each lower vertex
  std::vector<int32_t> uniq;
  uniq.reserve(hiv.size() / 2);
  for (int64_t v = 0; v < m.nv; ++v) {
    auto b = hiv.begin() + eoff[v], e = hiv.begin() + eoff[v + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    first[v] = (int64_t)uniq.size();
    uniq.insert(uniq.end(), b, e);
  }
  first[m.nv] = (int64_t)uniq.size();
  m.ne = (int64_t)uniq.size();
  m.n2 = m.nv + m.ne;
  m.edges.resize(m.ne * 2);
  for (int64_t v = 0; v < m.nv; ++v)
    for (int64_t e = first[v]; e < first[v + 1]; ++e) {
      m.edges[2 * e] = (int32_t)v;
      m.edges[2 * e + 1] = uniq[e];
    }
  for (int64_t c = 0; c < m.ncell; ++c) {
    int32_t* g = &m.c2d[c * m.nloc];
    for (int e = 0; e < nle; ++e) {
      int32_t a = g[le[e][0]], b = g[le[e][1]];
      int32_t lo = std::min(a, b), hi = std::max(a, b);
      auto it = std::lower_bound(uniq.begin() + first[lo], uniq.begin() + first[lo + 1], hi);
      g[m.nb + e] = (int32_t)(m.nv + (it - uniq.begin()));
    }
  }
  // Internal order of the edge nodes: grouped by the parity class of their
  // position on the doubled lattice (the sum of their end points' grid
  // indices: one class per edge direction), lexicographic (x fastest) within a
  // class.  Consecutive nodes of a class along a grid line then have the same
  // stencil shifted by one, so the neighbours that a warp's rows read at one
  // matrix slot are contiguous.  node_nat keeps the paper order.
  {
    const int64_t X = 2 * sx, Y = 2 * sy, Z = 2 * (dim == 3 ? n[2] + 1 : 1);
    std::vector<std::pair<int64_t, int32_t>> key(m.ne);
    for (int64_t e = 0; e < m.ne; ++e) {
      int64_t c[3] = {0, 0, 0};
      for (int end = 0; end < 2; ++end) {
        const int64_t v = m.edges[2 * e + end];
        c[0] += v % sx;
        c[1] += (v / sx) % sy;
        c[2] += dim == 3 ? v / (sx * sy) : 0;
      }
      const int64_t cls = (c[0] & 1) | (c[1] & 1) << 1 | (c[2] & 1) << 2;
      key[e] = {((cls * Z + c[2]) * Y + c[1]) * X + c[0], (int32_t)e};
    }
    std::sort(key.begin(), key.end());
    std::vector<int32_t> newid(m.ne), ed(2 * m.ne);
    m.node_nat.resize(m.n2);
    for (int64_t v = 0; v < m.nv; ++v) m.node_nat[v] = (int32_t)v;
    for (int64_t e = 0; e < m.ne; ++e) {
      const int32_t old = key[e].second;
      newid[old] = (int32_t)e;
      ed[2 * e] = m.edges[2 * old];
      ed[2 * e + 1] = m.edges[2 * old + 1];
      m.node_nat[m.nv + e] = (int32_t)(m.nv + old);
    }
    m.edges.swap(ed);
    for (int64_t c = 0; c < m.ncell; ++c)
      for (int e = 0; e < nle; ++e) {
        int32_t& g = m.c2d[c * m.nloc + m.nb + e];
        g = (int32_t)(m.nv + newid[g - m.nv]);
      }
  }
  m.p2xyz.resize(m.n2 * dim);
  std::memcpy(m.p2xyz.data(), m.coords.data(), sizeof(double) * m.nv * dim);
  for (int64_t e = 0; e < m.ne; ++e)
    for (int a = 0; a < dim; ++a)
      m.p2xyz[(m.nv + e) * dim + a] =
          0.5 * (m.coords[(int64_t)m.edges[2 * e] * dim + a] +
                 m.coords[(int64_t)m.edges[2 * e + 1] * dim + a]);

  // Dirichlet P2 nodes: vertices on a Dirichlet side; edge midpoints whose
  // two ends lie on one common Dirichlet side
  auto side_bits = [&](int64_t v) {
    int64_t ijk[3] = {v % sx, (v / sx) % sy, dim == 3 ? v / (sx * sy) : 0};
    int bits = 0;
    for (int a = 0; a < dim; ++a) {
      if (ijk[a] == 0) bits |= 1 << (2 * a);
      if (ijk[a] == n[a]) bits |= 1 << (2 * a + 1);
    }
    return bits & d.dirichlet_sides;
  };
  m.dirichlet.assign(m.n2, 0);
  for (int64_t v = 0; v < m.nv; ++v) m.dirichlet[v] = side_bits(v) ? 1 : 0;
  for (int64_t e = 0; e < m.ne; ++e)
    m.dirichlet[m.nv + e] =
        (side_bits(m.edges[2 * e]) & side_bits(m.edges[2 * e + 1])) ? 1 : 0;
  m.dlist.clear();
  for (int64_t i = 0; i < m.n2; ++i)
    if (m.dirichlet[i]) m.dlist.push_back((int32_t)i);
  return FS_OK;
}

// Greedy colouring of the cells by shared P2 nodes, in cell order: a cell
// takes the lowest colour that no cell holding one of its nodes has taken
// (node colour sets as 128-bit masks).  Structured triangle meshes take
// 6-8 colours, Kuhn tetrahedra about twice as many.
bool color_cells(Mesh& m) {
  const int nl = m.nloc;
  std::vector<uint64_t> used(2 * (size_t)m.n2, 0);
  std::vector<int> col(m.ncell);
  int ncol = 0;
  for (int64_t e = 0; e < m.ncell; ++e) {
    uint64_t lo = 0, hi = 0;
    for (int k = 0; k < nl; ++k) {
      const int64_t q = m.c2d[e * nl + k];
      lo |= used[2 * q];
      hi |= used[2 * q + 1];
    }
    int c;
    if (~lo != 0)
      c = __builtin_ctzll(~lo);
    else if (~hi != 0)
      c = 64 + __builtin_ctzll(~hi);
    else
      return false;
    col[e] = c;
    ncol = std::max(ncol, c + 1);
    for (int k = 0; k < nl; ++k) {
      const int64_t q = m.c2d[e * nl + k];
      used[2 * q + c / 64] |= 1ull << (c % 64);
    }
  }
  m.color_ptr.assign(ncol + 1, 0);
  for (int64_t e = 0; e < m.ncell; ++e) m.color_ptr[col[e] + 1]++;
  for (int c = 0; c < ncol; ++c) m.color_ptr[c + 1] += m.color_ptr[c];
  m.color_cells.resize(m.ncell);
  std::vector<int64_t> next(m.color_ptr.begin(), m.color_ptr.end() - 1);
  for (int64_t e = 0; e < m.ncell; ++e) m.color_cells[next[col[e]]++] = (int32_t)e;
  return true;
}

int finalize_patterns(Mesh& m) {
  if (!color_cells(m)) {
    set_error("fs_mesh_create: more than 128 cell colours");
    return FS_ERR_INVALID_MESH;
  }

  // block patterns and slot tables
  cell_pattern(m, m.n2, 0, m.nloc, 0, m.nloc, m.A);
  cell_pattern(m, m.nv, 0, m.nb, 0, m.nloc, m.B);
  cell_pattern(m, m.n2, 0, m.nloc, 0, m.nb, m.BT);
  cell_pattern(m, m.nv, 0, m.nb, 0, m.nb, m.Kp);
  m.A.ncol = m.n2; m.B.ncol = m.n2; m.BT.ncol = m.nv; m.Kp.ncol = m.nv;
  if (!cell_slots(m, m.A, 0, m.nloc, 0, m.nloc, m.posA) ||
      !cell_slots(m, m.B, 0, m.nb, 0, m.nloc, m.posB) ||
      !cell_slots(m, m.BT, 0, m.nloc, 0, m.nb, m.posBT) ||
      !cell_slots(m, m.Kp, 0, m.nb, 0, m.nb, m.posKp)) {
    set_error("fs_mesh_create: a CSR row is longer than 256 entries");
    return FS_ERR_INVALID_MESH;
  }
  return FS_OK;
}

}  // namespace

void monolithic_pattern(const Mesh& m, std::vector<int64_t>& rowptr,
                        std::vector<int32_t>& col) {
  const int dim = m.dim;
  const int64_t ndof = dim * m.n2 + m.nv;
  rowptr.assign(ndof + 1, 0);
  col.clear();
  col.reserve(dim * (m.A.nnz() + 2 * m.B.nnz()) + m.nv);
  for (int c = 0; c < dim; ++c)
    for (int64_t i = 0; i < m.n2; ++i) {
      for (int32_t k = m.A.rowptr[i]; k < m.A.rowptr[i + 1]; ++k)
        col.push_back((int32_t)(c * m.n2 + m.A.col[k]));
      for (int32_t k = m.BT.rowptr[i]; k < m.BT.rowptr[i + 1]; ++k)
        col.push_back((int32_t)(dim * m.n2 + m.BT.col[k]));
      rowptr[c * m.n2 + i + 1] = (int64_t)col.size();
    }
  for (int64_t q = 0; q < m.nv; ++q) {
    for (int c = 0; c < dim; ++c)
      for (int32_t k = m.B.rowptr[q]; k < m.B.rowptr[q + 1]; ++k)
        col.push_back((int32_t)(c * m.n2 + m.B.col[k]));
    col.push_back((int32_t)(dim * m.n2 + q));
    rowptr[dim * m.n2 + q + 1] = (int64_t)col.size();
  }
}

void natural_dof_map(const Mesh& m, std::vector<int32_t>* c2d, std::vector<uint8_t>* dir,
                     std::vector<int64_t>* rowptr, std::vector<int32_t>* col) {
  Mesh nm;
  nm.dim = m.dim;
  nm.nloc = m.nloc;
  nm.nb = m.nb;
  nm.nv = m.nv;
  nm.ne = m.ne;
  nm.n2 = m.n2;
  nm.ncell = m.ncell;
  nm.c2d.resize(m.c2d.size());
  for (size_t k = 0; k < m.c2d.size(); ++k) nm.c2d[k] = m.node_nat[m.c2d[k]];
  if (dir) {
    dir->assign(m.n2, 0);
    for (int64_t q = 0; q < m.n2; ++q) (*dir)[m.node_nat[q]] = m.dirichlet[q];
  }
  if (rowptr || col) {
    cell_pattern(nm, nm.n2, 0, nm.nloc, 0, nm.nloc, nm.A);
    cell_pattern(nm, nm.nv, 0, nm.nb, 0, nm.nloc, nm.B);
    cell_pattern(nm, nm.n2, 0, nm.nloc, 0, nm.nb, nm.BT);
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    monolithic_pattern(nm, rp, ci);
    if (rowptr) rowptr->swap(rp);
    if (col) col->swap(ci);
  }
  if (c2d) c2d->swap(nm.c2d);
}

// ---------------------------------------------------------------------------
// Grundmann-Moeller rule of degree 2s+1 on the n-simplex (Grundmann and
// Moeller, SIAM J. Numer. Anal. 15 (1978)): points with barycentric
// coordinates (2 beta_k + 1)/(d + n - 2i) for |beta| = s - i, weights
// (-1)^i 2^{-2s} (d + n - 2i)^d / (i! (d + n - i)!), d = 2s + 1.  The weights
// sum to the volume 1/n! of the unit simplex.
// ---------------------------------------------------------------------------
namespace {

void compositions(int total, int parts, std::vector<int>& cur,
                  std::vector<std::vector<int>>& out) {
  if (parts == 1) {
    cur.push_back(total);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int k = 0; k <= total; ++k) {
    cur.push_back(k);
    compositions(total - k, parts - 1, cur, out);
    cur.pop_back();
  }
}

double fact(int k) {
  double f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

}  // namespace

void ref_tensors(int dim, RefTensors& R) {
  R = RefTensors{};  // every table zero
  R.dim = dim;
  R.nb = dim + 1;
  R.nloc = dim == 2 ? 6 : 10;
  const int(*le)[2] = dim == 2 ? kTriEdge : kTetEdge;
  R.npair = 0;
  for (int j = 0; j < R.nloc; ++j) {
    if (j < R.nb) {
      R.pair_j[R.npair] = j; R.pair_r[R.npair++] = j;
    } else {
      R.pair_j[R.npair] = j; R.pair_r[R.npair++] = le[j - R.nb][0];
      R.pair_j[R.npair] = j; R.pair_r[R.npair++] = le[j - R.nb][1];
    }
  }
  const int s = 2, deg = 2 * s + 1, n = dim;
  std::vector<std::array<double, 4>> pts;
  std::vector<double> wts;
  for (int i = 0; i <= s; ++i) {
    double w = ((i % 2) ? -1.0 : 1.0) * std::ldexp(1.0, -2 * s) *
               std::pow((double)(deg + n - 2 * i), deg) / (fact(i) * fact(deg + n - i));
    std::vector<std::vector<int>> betas;
    std::vector<int> cur;
    compositions(s - i, n + 1, cur, betas);
    for (auto& b : betas) {
      std::array<double, 4> l{0, 0, 0, 0};
      for (int k = 0; k <= n; ++k) l[k] = (2.0 * b[k] + 1.0) / (double)(deg + n - 2 * i);
      pts.push_back(l);
      wts.push_back(w);
    }
  }
  for (size_t q = 0; q < pts.size(); ++q) {
    const double* l = pts[q].data();
    double w = wts[q];
    double phi[kMaxLoc], dphi[kMaxLoc][4];
    for (int j = 0; j < R.nloc; ++j) {
      for (int r = 0; r < 4; ++r) dphi[j][r] = 0;
      if (j < R.nb) {
        phi[j] = l[j] * (2.0 * l[j] - 1.0);
        dphi[j][j] = 4.0 * l[j] - 1.0;
      } else {
        int a = le[j - R.nb][0], b = le[j - R.nb][1];
        phi[j] = 4.0 * l[a] * l[b];
        dphi[j][a] = 4.0 * l[b];
        dphi[j][b] = 4.0 * l[a];
      }
    }
    for (int i = 0; i < R.nloc; ++i)
      for (int j = 0; j < R.nloc; ++j) {
        R.mass[i][j] += w * phi[i] * phi[j];
        for (int r = 0; r < R.nb; ++r)
          for (int t = 0; t < R.nb; ++t) R.stiff[i][j][r][t] += w * dphi[i][r] * dphi[j][t];
      }
    for (int i = 0; i < R.nloc; ++i)
      for (int k = 0; k < R.nloc; ++k)
        for (int p = 0; p < R.npair; ++p)
          R.conv[i][k][p] += w * phi[i] * phi[k] * dphi[R.pair_j[p]][R.pair_r[p]];
    for (int qv = 0; qv < R.nb; ++qv)
      for (int j = 0; j < R.nloc; ++j) {
        for (int r = 0; r < R.nb; ++r) R.div[qv][j][r] += w * l[qv] * dphi[j][r];
        R.pmass[qv][j] += w * l[qv] * phi[j];
      }
  }
}

}  // namespace fs
