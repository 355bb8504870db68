/*
 * fs_oracle.c -- the oracle: a plain, slow, FP64 CPU reference for one
 * backward-Euler Oseen step of the Taylor-Hood P2/P1 finite element
 * discretisation of the incompressible Navier-Stokes equations.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product library
 * (the CUDA path) never includes, links or calls anything in this directory,
 * and this file includes nothing from the product.
 *
 * What it follows (paper: "A High-Performance, Cross-Platform Open-Source
 * Solver for the Incompressible Navier-Stokes Equations in FEALPy"):
 *   - Sec. 2.1, Eq. (3) (unsteady NS) and Eq. (2) (steady NS);
 *   - Sec. 2.2.1, the spaces V_h = [P_2]^d and Q_h = P_1 (Taylor-Hood, k = 2);
 *   - Sec. 2.2.1, the Oseen linearisation: with the convecting velocity
 *     lagged (w = u_h^n) and one linear solve per step,
 *       ((u - u^n)/dt, v) + ((w.grad) u, v) + nu (grad u, grad v)
 *         - (p, div v) = (f^{n+1}, v),      (div u, q) = 0;
 *   - Sec. 3.3 / 4.1: the manufactured solutions (steady polynomial example
 *     of Sec. 3.3, the unsteady benchmark of Sec. 4.1).
 * Where the paper is silent this file reads it as follows: the load (f, v) is taken as (I_h f, v) = M I_h f with P2
 * nodal interpolation; Dirichlet rows are replaced by identity rows keeping
 * their pattern; when all of the boundary is Dirichlet the row of pressure
 * DOF 0 is replaced by an identity row holding p_exact(x_0, t).
 *
 * Element integrals are exact: every integrand is expanded in barycentric
 * monomials and integrated with int_K l^a = a! d! |K| / (|a| + d)!.
 * Global assembly goes through sorted COO triplets (the definition of a sum
 * of element contributions), not through precomputed slots.
 *
 * Floating point: compile with -ffp-contract=off so that the mesh
 * coordinates come out bit-identical on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014), used as a counter-based hash.  */
/* ------------------------------------------------------------------ */
static uint64_t splitmix64(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* U in [0,1): 53 high bits of SplitMix64(seed XOR key). */
double or_uniform(uint64_t seed, uint64_t key) {
  return (double)(splitmix64(seed ^ key) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* Structured simplicial meshes.                                        */
/* 2D: (n0+1)(n1+1) vertices, vertex id i + (n0+1) j; square (i,j) is   */
/* split along v00-v11 into (v00,v10,v11) and (v00,v11,v01).            */
/* 3D: vertex id i + (n0+1)(j + (n1+1) k); cube split into the 6 Kuhn   */
/* tetrahedra, one per axis permutation taken in lexicographic order;   */
/* the tetrahedron walks from the cube's low corner along the axes in   */
/* permutation order.  Cells ordered by square/cube index (x fastest),  */
/* then by split index.                                                 */
/* ------------------------------------------------------------------ */
int64_t or_mesh_nvert(int dim, const int* n) {
  return dim == 2 ? (int64_t)(n[0] + 1) * (n[1] + 1)
                  : (int64_t)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
}
int64_t or_mesh_ncell(int dim, const int* n) {
  return dim == 2 ? 2LL * n[0] * n[1] : 6LL * n[0] * n[1] * n[2];
}

int or_mesh(int dim, const int* n, const double* lo, const double* hi,
            double jitter, uint64_t seed, double* coords, int32_t* cells) {
  if (dim != 2 && dim != 3) return 1;
  double h[3];
  int m[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 1) return 1;
    h[a] = (hi[a] - lo[a]) / (double)n[a];
    m[a] = n[a];
  }
  int64_t nv = or_mesh_nvert(dim, n);
  for (int64_t v = 0; v < nv; ++v) {
    int64_t idx[3];
    idx[0] = v % (m[0] + 1);
    idx[1] = (v / (m[0] + 1)) % (m[1] + 1);
    idx[2] = dim == 3 ? v / ((int64_t)(m[0] + 1) * (m[1] + 1)) : 0;
    int interior = 1;
    for (int a = 0; a < dim; ++a)
      if (idx[a] == 0 || idx[a] == m[a]) interior = 0;
    for (int a = 0; a < dim; ++a) {
      double x = lo[a] + (double)idx[a] * h[a];
      if (interior && jitter != 0.0) {
        double U = or_uniform(seed, (uint64_t)(3 * v + a));
        x = x + jitter * h[a] * (2.0 * U - 1.0);
      }
      coords[v * dim + a] = x;
    }
  }
  if (dim == 2) {
    int64_t c = 0;
    for (int j = 0; j < m[1]; ++j)
      for (int i = 0; i < m[0]; ++i) {
        int32_t v00 = i + (m[0] + 1) * j, v10 = v00 + 1;
        int32_t v01 = v00 + (m[0] + 1), v11 = v01 + 1;
        int32_t* t0 = cells + 3 * (c++);
        t0[0] = v00; t0[1] = v10; t0[2] = v11;
        int32_t* t1 = cells + 3 * (c++);
        t1[0] = v00; t1[1] = v11; t1[2] = v01;
      }
  } else {
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                    {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int64_t c = 0;
    for (int k = 0; k < m[2]; ++k)
      for (int j = 0; j < m[1]; ++j)
        for (int i = 0; i < m[0]; ++i)
          for (int s = 0; s < 6; ++s) {
            int p[3] = {i, j, k};
            int32_t* t = cells + 4 * (c++);
            for (int step = 0; step <= 3; ++step) {
              if (step > 0) p[perms[s][step - 1]] += 1;
              t[step] = (int32_t)(p[0] + (m[0] + 1) * (p[1] + (m[1] + 1) * p[2]));
            }
          }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* P2 DOF map.  Local P2 order: vertices, then edges; triangle edges    */
/* (1,2),(2,0),(0,1); tetrahedron edges (0,1),(0,2),(0,3),(1,2),(1,3),  */
/* (2,3).  Global edge id = rank of (min,max) in lexicographic order;   */
/* P2 node id = nvert + edge id.                                        */
/* ------------------------------------------------------------------ */
static const int tri_edges[3][2] = {{1, 2}, {2, 0}, {0, 1}};
static const int tet_edges[6][2] = {{0, 1}, {0, 2}, {0, 3},
                                    {1, 2}, {1, 3}, {2, 3}};

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Returns the number of unique edges; edges_out may be NULL (count only).
 * cell2dof: ncell x nloc, filled when non-NULL. */
int64_t or_dofmap(int dim, int64_t nv, int64_t ncell, const int32_t* cells,
                  int32_t* edges_out, int32_t* cell2dof) {
  int nle = dim == 2 ? 3 : 6, nlv = dim + 1;
  const int(*le)[2] = dim == 2 ? tri_edges : tet_edges;
  int64_t nk = ncell * nle;
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nk ? nk : 1));
  for (int64_t c = 0; c < ncell; ++c)
    for (int e = 0; e < nle; ++e) {
      uint64_t a = (uint64_t)cells[c * nlv + le[e][0]];
      uint64_t b = (uint64_t)cells[c * nlv + le[e][1]];
      uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
      keys[c * nle + e] = lo * (uint64_t)nv + hi;
    }
  uint64_t* uniq = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nk ? nk : 1));
  memcpy(uniq, keys, sizeof(uint64_t) * (size_t)nk);
  qsort(uniq, (size_t)nk, sizeof(uint64_t), cmp_u64);
  int64_t ne = 0;
  for (int64_t i = 0; i < nk; ++i)
    if (i == 0 || uniq[i] != uniq[i - 1]) uniq[ne++] = uniq[i];
  if (edges_out)
    for (int64_t e = 0; e < ne; ++e) {
      edges_out[2 * e] = (int32_t)(uniq[e] / (uint64_t)nv);
      edges_out[2 * e + 1] = (int32_t)(uniq[e] % (uint64_t)nv);
    }
  if (cell2dof) {
    int nloc = nlv + nle;
    for (int64_t c = 0; c < ncell; ++c) {
      for (int v = 0; v < nlv; ++v) cell2dof[c * nloc + v] = cells[c * nlv + v];
      for (int e = 0; e < nle; ++e) {
        uint64_t key = keys[c * nle + e];
        int64_t lo = 0, hi = ne - 1;
        while (lo < hi) {
          int64_t mid = (lo + hi) / 2;
          if (uniq[mid] < key) lo = mid + 1; else hi = mid;
        }
        cell2dof[c * nloc + nlv + e] = (int32_t)(nv + lo);
      }
    }
  }
  free(keys);
  free(uniq);
  return ne;
}

/* P2 node coordinates: vertices, then straight-edge midpoints. */
void or_p2_coords(int dim, int64_t nv, int64_t ne, const double* coords,
                  const int32_t* edges, double* out) {
  memcpy(out, coords, sizeof(double) * (size_t)(nv * dim));
  for (int64_t e = 0; e < ne; ++e)
    for (int a = 0; a < dim; ++a)
      out[(nv + e) * dim + a] =
          0.5 * (coords[(int64_t)edges[2 * e] * dim + a] +
                 coords[(int64_t)edges[2 * e + 1] * dim + a]);
}

/* Dirichlet P2 nodes of a structured mesh.  Sides are numbered
 * 0: x=lo, 1: x=hi, 2: y=lo, 3: y=hi, 4: z=lo, 5: z=hi; side_mask selects
 * the Dirichlet sides.  A vertex is Dirichlet when it lies on a selected
 * side; an edge midpoint is Dirichlet when both ends lie on one common
 * selected side (then the whole straight edge lies in that side). */
static int vertex_sides(int dim, const int* n, int64_t v) {
  int64_t i = v % (n[0] + 1);
  int64_t j = (v / (n[0] + 1)) % (n[1] + 1);
  int64_t k = dim == 3 ? v / ((int64_t)(n[0] + 1) * (n[1] + 1)) : -1;
  int s = 0;
  if (i == 0) s |= 1;
  if (i == n[0]) s |= 2;
  if (j == 0) s |= 4;
  if (j == n[1]) s |= 8;
  if (dim == 3) {
    if (k == 0) s |= 16;
    if (k == n[2]) s |= 32;
  }
  return s;
}

void or_dirichlet_mask(int dim, const int* n, int side_mask, int64_t nv,
                       int64_t ne, const int32_t* edges, uint8_t* mask) {
  for (int64_t v = 0; v < nv; ++v)
    mask[v] = (vertex_sides(dim, n, v) & side_mask) ? 1 : 0;
  for (int64_t e = 0; e < ne; ++e) {
    int sa = vertex_sides(dim, n, edges[2 * e]);
    int sb = vertex_sides(dim, n, edges[2 * e + 1]);
    mask[nv + e] = (sa & sb & side_mask) ? 1 : 0;
  }
}

/* ------------------------------------------------------------------ */
/* Manufactured solutions and their loads f = u_t - nu Lap u            */
/* + (w.grad) u + grad p, where w = u (Navier-Stokes) except for the    */
/* polynomial Oseen problem whose w is a given constant vector.         */
/* ------------------------------------------------------------------ */
enum {
  OR_JOHN = 0,         /* Sec. 4.1 unsteady benchmark, 2D                */
  OR_STEADY_POLY = 1,  /* Sec. 3.3 steady example, 2D (no time)          */
  OR_CHANNEL = 2,      /* Poiseuille profile, U_max 1.5, H 0.41, L 2.2   */
  OR_CUBE = 3,         /* 3D: u = sin t curl(Phi (1,1,1)), Phi=prod sin^2 */
  OR_POLY_OSEEN = 4,   /* u in P2 div-free, p in P1, constant w           */
  OR_POLY_OSEEN_T = 5, /* (1 + t) times the fields of OR_POLY_OSEEN       */
  OR_POLY3 = 6         /* 2D: u in P3 div-free, p in P2, constant w       */
};

/* g(s) = sin^2(pi s) and its derivatives up to order 3. */
static double g_der(int order, double s) {
  const double pi = 3.14159265358979323846;
  switch (order) {
    case 0: { double v = sin(pi * s); return v * v; }
    case 1: return pi * sin(2.0 * pi * s);
    case 2: return 2.0 * pi * pi * cos(2.0 * pi * s);
    default: return -4.0 * pi * pi * pi * sin(2.0 * pi * s);
  }
}
/* D^(a,b,c) Phi for Phi(x,y,z) = g(x) g(y) g(z). */
static double phi_der(int a, int b, int c, const double* x) {
  return g_der(a, x[0]) * g_der(b, x[1]) * g_der(c, x[2]);
}

/* u, grad u (du[i*dim+j] = d u_i / d x_j), Laplacian, u_t, p, grad p. */
static void exact_fields(int problem, int dim, double t, const double* x,
                         double* u, double* du, double* lap, double* ut,
                         double* p, double* dp) {
  const double pi = 3.14159265358979323846;
  double X = x[0], Y = x[1];
  for (int i = 0; i < dim; ++i) {
    u[i] = 0; ut[i] = 0; lap[i] = 0; dp[i] = 0;
    for (int j = 0; j < dim; ++j) du[i * dim + j] = 0;
  }
  *p = 0;
  switch (problem) {
    case OR_JOHN: {
      double S = sin(t), C = cos(t);
      double sa = sin(pi * X), s2a = sin(2 * pi * X), c2a = cos(2 * pi * X);
      double sb = sin(pi * Y), s2b = sin(2 * pi * Y), c2b = cos(2 * pi * Y);
      /* u1 = pi S sin^2(pi x) sin(2 pi y); u2 = -pi S sin(2 pi x) sin^2(pi y) */
      u[0] = pi * S * sa * sa * s2b;
      u[1] = -pi * S * s2a * sb * sb;
      ut[0] = pi * C * sa * sa * s2b;
      ut[1] = -pi * C * s2a * sb * sb;
      du[0] = pi * pi * S * s2a * s2b;
      du[1] = 2 * pi * pi * S * sa * sa * c2b;
      du[2] = -2 * pi * pi * S * c2a * sb * sb;
      du[3] = -pi * pi * S * s2a * s2b;
      lap[0] = 2 * pi * pi * pi * S * c2a * s2b - 4 * pi * pi * pi * S * sa * sa * s2b;
      lap[1] = 4 * pi * pi * pi * S * s2a * sb * sb - 2 * pi * pi * pi * S * s2a * c2b;
      *p = 20 * S * (X * X * Y - 1.0 / 6.0);
      dp[0] = 40 * S * X * Y;
      dp[1] = 20 * S * X * X;
      break;
    }
    case OR_STEADY_POLY: {
      /* u = 10 x^2 (x-1)^2 y (y-1)(2y-1), v = -10 x (x-1)(2x-1) y^2 (y-1)^2,
       * p = 10 (2x-1)(2y-1).  Written as products a(x) b(y). */
      double ax = X * X * (X - 1) * (X - 1);             /* x^2 (x-1)^2 */
      double ax1 = 2 * X * (X - 1) * (2 * X - 1);        /* d/dx        */
      double ax2 = 12 * X * X - 12 * X + 2;              /* d2/dx2      */
      double by = Y * (Y - 1) * (2 * Y - 1);             /* = 2y^3-3y^2+y */
      double by1 = 6 * Y * Y - 6 * Y + 1;
      double by2 = 12 * Y - 6;
      double cx = X * (X - 1) * (2 * X - 1);
      double cx1 = 6 * X * X - 6 * X + 1;
      double cx2 = 12 * X - 6;
      double dy = Y * Y * (Y - 1) * (Y - 1);
      double dy1 = 2 * Y * (Y - 1) * (2 * Y - 1);
      double dy2 = 12 * Y * Y - 12 * Y + 2;
      u[0] = 10 * ax * by;
      u[1] = -10 * cx * dy;
      du[0] = 10 * ax1 * by;  du[1] = 10 * ax * by1;
      du[2] = -10 * cx1 * dy; du[3] = -10 * cx * dy1;
      lap[0] = 10 * (ax2 * by + ax * by2);
      lap[1] = -10 * (cx2 * dy + cx * dy2);
      *p = 10 * (2 * X - 1) * (2 * Y - 1);
      dp[0] = 20 * (2 * Y - 1);
      dp[1] = 20 * (2 * X - 1);
      break;
    }
    case OR_CHANNEL: {
      const double H = 0.41, L = 2.2, Um = 1.5;
      u[0] = 4 * Um * Y * (H - Y) / (H * H);
      du[1] = 4 * Um * (H - 2 * Y) / (H * H);
      lap[0] = -8 * Um / (H * H);
      /* pressure for nu = 1 scaled later: p = 8 nu Um (L - x) / H^2 */
      *p = 8 * Um * (L - X) / (H * H);
      dp[0] = -8 * Um / (H * H);
      break;
    }
    case OR_CUBE: {
      double S = sin(t), C = cos(t);
      /* u = S (Phi_y - Phi_z, Phi_z - Phi_x, Phi_x - Phi_y) */
      static const int comp_plus[3] = {1, 2, 0}, comp_minus[3] = {2, 0, 1};
      for (int i = 0; i < 3; ++i) {
        int ep[3] = {0, 0, 0}, em[3] = {0, 0, 0};
        ep[comp_plus[i]] = 1;
        em[comp_minus[i]] = 1;
        double val = phi_der(ep[0], ep[1], ep[2], x) - phi_der(em[0], em[1], em[2], x);
        u[i] = S * val;
        ut[i] = C * val;
        double l = 0;
        for (int j = 0; j < 3; ++j) {
          int fp[3] = {ep[0], ep[1], ep[2]}, fm[3] = {em[0], em[1], em[2]};
          fp[j] += 1; fm[j] += 1;
          du[i * 3 + j] = S * (phi_der(fp[0], fp[1], fp[2], x) - phi_der(fm[0], fm[1], fm[2], x));
          fp[j] += 1; fm[j] += 1;
          l += phi_der(fp[0], fp[1], fp[2], x) - phi_der(fm[0], fm[1], fm[2], x);
        }
        lap[i] = S * l;
      }
      double Z = x[2];
      *p = S * (X * X * Y * Z - 1.0 / 12.0);
      dp[0] = S * 2 * X * Y * Z;
      dp[1] = S * X * X * Z;
      dp[2] = S * X * X * Y;
      break;
    }
    case OR_POLY_OSEEN:
    case OR_POLY_OSEEN_T: {
      /* 2D: u = (x^2, -2xy), p = x + y - 1.
       * 3D: u = (x^2, -2xy, xy), p = x + y + z - 1.
       * OR_POLY_OSEEN_T multiplies u and p by (1 + t), so u_t is the
       * spatial field itself: affine in time, which backward Euler
       * differentiates exactly. */
      u[0] = X * X;
      u[1] = -2 * X * Y;
      du[0 * dim + 0] = 2 * X;
      du[1 * dim + 0] = -2 * Y;
      du[1 * dim + 1] = -2 * X;
      lap[0] = 2;
      *p = X + Y - 1;
      dp[0] = 1; dp[1] = 1;
      if (dim == 3) {
        u[2] = X * Y;
        du[2 * 3 + 0] = Y;
        du[2 * 3 + 1] = X;
        *p = X + Y + x[2] - 1;
        dp[2] = 1;
      }
      if (problem == OR_POLY_OSEEN_T) {
        double s = 1.0 + t;
        for (int i = 0; i < dim; ++i) {
          ut[i] = u[i];
          u[i] *= s;
          lap[i] *= s;
          dp[i] *= s;
          for (int j = 0; j < dim; ++j) du[i * dim + j] *= s;
        }
        *p *= s;
      }
      break;
    }
    case OR_POLY3: {
      /* u = (x^3, -3 x^2 y) (div u = 3x^2 - 3x^2 = 0), p = x^2 - y^2 */
      u[0] = X * X * X;
      u[1] = -3 * X * X * Y;
      du[0] = 3 * X * X;
      du[1] = 0;
      du[2] = -6 * X * Y;
      du[3] = -3 * X * X;
      lap[0] = 6 * X;
      lap[1] = -6 * Y;
      *p = X * X - Y * Y;
      dp[0] = 2 * X;
      dp[1] = -2 * Y;
      break;
    }
  }
}

/* Exact velocity u, pressure p and load f at one point.  nu scales the
 * viscous term; for the channel the pressure is scaled by nu as well so
 * that the Poiseuille pair solves -nu Lap u + grad p = 0. */
void or_exact(int problem, int dim, double t, double nu, const double* wconst,
              const double* x, double* u, double* p, double* f) {
  double du[9], lap[3], ut[3], dp[3], uu[3], pp;
  exact_fields(problem, dim, t, x, uu, du, lap, ut, &pp, dp);
  if (problem == OR_CHANNEL) {
    pp *= nu;
    for (int i = 0; i < dim; ++i) dp[i] *= nu;
  }
  double w[3];
  for (int i = 0; i < dim; ++i)
    w[i] = ((problem == OR_POLY_OSEEN || problem == OR_POLY_OSEEN_T ||
             problem == OR_POLY3) && wconst)
               ? wconst[i] : uu[i];
  if (u) for (int i = 0; i < dim; ++i) u[i] = uu[i];
  if (p) *p = pp;
  if (f)
    for (int i = 0; i < dim; ++i) {
      double conv = 0;
      for (int j = 0; j < dim; ++j) conv += w[j] * du[i * dim + j];
      double time_term = (problem == OR_STEADY_POLY) ? 0.0 : ut[i];
      f[i] = time_term - nu * lap[i] + conv + dp[i];
    }
}

/* Vectorised helper for the Python side: npts points, AoS layout. */
void or_exact_many(int problem, int dim, double t, double nu,
                   const double* wconst, int64_t npts, const double* x,
                   double* u, double* p, double* f) {
  for (int64_t i = 0; i < npts; ++i)
    or_exact(problem, dim, t, nu, wconst, x + i * dim, u ? u + i * dim : NULL,
             p ? p + i : NULL, f ? f + i * dim : NULL);
}

/* ------------------------------------------------------------------ */
/* Barycentric polynomial algebra and exact reference integrals.        */
/* ------------------------------------------------------------------ */
#define BP_MAXT 96
typedef struct {
  int n;
  int e[BP_MAXT][4];
  double c[BP_MAXT];
} bpoly;

static void bp_add_term(bpoly* p, const int* e, double c) {
  for (int t = 0; t < p->n; ++t)
    if (p->e[t][0] == e[0] && p->e[t][1] == e[1] && p->e[t][2] == e[2] &&
        p->e[t][3] == e[3]) {
      p->c[t] += c;
      return;
    }
  if (p->n >= BP_MAXT) abort();
  for (int r = 0; r < 4; ++r) p->e[p->n][r] = e[r];
  p->c[p->n] = c;
  p->n++;
}

static void bp_mul(const bpoly* a, const bpoly* b, bpoly* out) {
  out->n = 0;
  for (int i = 0; i < a->n; ++i)
    for (int j = 0; j < b->n; ++j) {
      int e[4];
      for (int r = 0; r < 4; ++r) e[r] = a->e[i][r] + b->e[j][r];
      bp_add_term(out, e, a->c[i] * b->c[j]);
    }
}

static void bp_diff(const bpoly* a, int r, bpoly* out) {
  out->n = 0;
  for (int i = 0; i < a->n; ++i)
    if (a->e[i][r] > 0) {
      int e[4] = {a->e[i][0], a->e[i][1], a->e[i][2], a->e[i][3]};
      double c = a->c[i] * e[r];
      e[r] -= 1;
      bp_add_term(out, e, c);
    }
}

static double factorial(int k) {
  double f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

/* (1/|K|) int_K p  =  sum_a c_a  a! d! / (|a| + d)!  */
static double bp_mean(const bpoly* p, int dim) {
  double s = 0;
  for (int t = 0; t < p->n; ++t) {
    int tot = 0;
    double num = factorial(dim);
    for (int r = 0; r < 4; ++r) {
      num *= factorial(p->e[t][r]);
      tot += p->e[t][r];
    }
    s += p->c[t] * num / factorial(tot + dim);
  }
  return s;
}

/* P2 Lagrange basis in barycentric form: vertex v: l_v (2 l_v - 1);
 * edge (a,b): 4 l_a l_b. */
static void p2_basis(int dim, int i, bpoly* out) {
  out->n = 0;
  int nlv = dim + 1;
  int e[4] = {0, 0, 0, 0};
  if (i < nlv) {
    e[i] = 2; bp_add_term(out, e, 2.0);
    e[i] = 1; bp_add_term(out, e, -1.0);
  } else {
    const int* ed = dim == 2 ? tri_edges[i - nlv] : tet_edges[i - nlv];
    e[ed[0]] = 1; e[ed[1]] = 1;
    bp_add_term(out, e, 4.0);
  }
}

typedef struct {
  int ready;
  double M[10][10];        /* mean of phi_i phi_j                    */
  double K[10][10][4][4];  /* mean of d_r phi_i d_s phi_j             */
  double N[10][10][10][4]; /* mean of phi_i phi_k d_r phi_j           */
  double B[4][10][4];      /* mean of l_q d_r phi_j                   */
  double P1M[4][4];        /* mean of l_q l_s (P1 mass)               */
} reftens;
static reftens REF[2];

static const reftens* ref_tensors(int dim) {
  reftens* R = &REF[dim - 2];
  if (R->ready) return R;
  int nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  static bpoly phi[10], dphi[10][4], tmp, tmp2;
  for (int i = 0; i < nloc; ++i) {
    p2_basis(dim, i, &phi[i]);
    for (int r = 0; r < nb; ++r) bp_diff(&phi[i], r, &dphi[i][r]);
  }
  for (int i = 0; i < nloc; ++i)
    for (int j = 0; j < nloc; ++j) {
      bp_mul(&phi[i], &phi[j], &tmp);
      R->M[i][j] = bp_mean(&tmp, dim);
      for (int r = 0; r < nb; ++r)
        for (int s = 0; s < nb; ++s) {
          bp_mul(&dphi[i][r], &dphi[j][s], &tmp);
          R->K[i][j][r][s] = bp_mean(&tmp, dim);
        }
      for (int k = 0; k < nloc; ++k) {
        bp_mul(&phi[i], &phi[k], &tmp2);
        for (int r = 0; r < nb; ++r) {
          bp_mul(&tmp2, &dphi[j][r], &tmp);
          R->N[i][j][k][r] = bp_mean(&tmp, dim);
        }
      }
    }
  for (int q = 0; q < nb; ++q) {
    bpoly lq;
    lq.n = 0;
    int e[4] = {0, 0, 0, 0};
    e[q] = 1;
    bp_add_term(&lq, e, 1.0);
    for (int j = 0; j < nloc; ++j)
      for (int r = 0; r < nb; ++r) {
        bp_mul(&lq, &dphi[j][r], &tmp);
        R->B[q][j][r] = bp_mean(&tmp, dim);
      }
    for (int s = 0; s < nb; ++s) {
      bpoly ls;
      ls.n = 0;
      int f[4] = {0, 0, 0, 0};
      f[s] = 1;
      bp_add_term(&ls, f, 1.0);
      bp_mul(&lq, &ls, &tmp);
      R->P1M[q][s] = bp_mean(&tmp, dim);
    }
  }
  R->ready = 1;
  return R;
}

/* Reference tensors exported for tests (means over the simplex). */
void or_ref_tensors(int dim, double* M, double* K, double* N, double* B) {
  const reftens* R = ref_tensors(dim);
  int nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  for (int i = 0; i < nloc; ++i)
    for (int j = 0; j < nloc; ++j) {
      if (M) M[i * nloc + j] = R->M[i][j];
      for (int r = 0; r < nb; ++r)
        for (int s = 0; s < nb; ++s)
          if (K) K[((i * nloc + j) * nb + r) * nb + s] = R->K[i][j][r][s];
      for (int k = 0; k < nloc; ++k)
        for (int r = 0; r < nb; ++r)
          if (N) N[((i * nloc + j) * nloc + k) * nb + r] = R->N[i][j][k][r];
    }
  for (int q = 0; q < nb; ++q)
    for (int j = 0; j < nloc; ++j)
      for (int r = 0; r < nb; ++r)
        if (B) B[(q * nloc + j) * nb + r] = R->B[q][j][r];
}

/* ------------------------------------------------------------------ */
/* Element matrices on one affine simplex.                              */
/*   xv: (d+1) x d vertex coordinates; w: nloc x d nodal convecting     */
/*   velocity or NULL.  Outputs (each optional):                        */
/*   A = mass_coef M + nu K + N(w)       nloc x nloc                    */
/*   M (P2 mass), K (P2 stiffness), N (convection)                      */
/*   B[c][q][j] = int psi_q d_c phi_j    d x (d+1) x nloc               */
/*   Mp[q][s]   = int psi_q psi_s        (d+1) x (d+1)                  */
/* Returns the signed determinant of J = [x1-x0, ..., xd-x0].           */
/* ------------------------------------------------------------------ */
double or_element(int dim, const double* xv, const double* w,
                  double mass_coef, double nu, double* A, double* M,
                  double* K, double* N, double* B, double* Kp, double* Mp) {
  const reftens* R = ref_tensors(dim);
  int nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  double J[3][3], Ji[3][3], det;
  for (int a = 0; a < dim; ++a)
    for (int b = 0; b < dim; ++b) J[a][b] = xv[(b + 1) * dim + a] - xv[a];
  if (dim == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;  Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  }
  /* grad l_r for r >= 1 is row r-1 of J^{-1}; grad l_0 = -sum. */
  double gl[4][3];
  for (int a = 0; a < dim; ++a) {
    gl[0][a] = 0;
    for (int r = 1; r <= dim; ++r) {
      gl[r][a] = Ji[r - 1][a];
      gl[0][a] -= Ji[r - 1][a];
    }
  }
  double vol = fabs(det) / (dim == 2 ? 2.0 : 6.0);
  double G[4][4];
  for (int r = 0; r < nb; ++r)
    for (int s = 0; s < nb; ++s) {
      G[r][s] = 0;
      for (int a = 0; a < dim; ++a) G[r][s] += gl[r][a] * gl[s][a];
    }
  double cw[10][4];
  if (w)
    for (int k = 0; k < nloc; ++k)
      for (int r = 0; r < nb; ++r) {
        cw[k][r] = 0;
        for (int a = 0; a < dim; ++a) cw[k][r] += w[k * dim + a] * gl[r][a];
      }
  for (int i = 0; i < nloc; ++i)
    for (int j = 0; j < nloc; ++j) {
      double m = vol * R->M[i][j];
      double kk = 0;
      for (int r = 0; r < nb; ++r)
        for (int s = 0; s < nb; ++s) kk += G[r][s] * R->K[i][j][r][s];
      kk *= vol;
      double nn = 0;
      if (w)
        for (int k = 0; k < nloc; ++k)
          for (int r = 0; r < nb; ++r) nn += cw[k][r] * R->N[i][j][k][r];
      nn *= vol;
      if (M) M[i * nloc + j] = m;
      if (K) K[i * nloc + j] = kk;
      if (N) N[i * nloc + j] = nn;
      if (A) A[i * nloc + j] = mass_coef * m + nu * kk + nn;
    }
  if (B)
    for (int c = 0; c < dim; ++c)
      for (int q = 0; q < nb; ++q)
        for (int j = 0; j < nloc; ++j) {
          double s = 0;
          for (int r = 0; r < nb; ++r) s += gl[r][c] * R->B[q][j][r];
          B[(c * nb + q) * nloc + j] = vol * s;
        }
  if (Kp)
    for (int q = 0; q < nb; ++q)
      for (int s = 0; s < nb; ++s) Kp[q * nb + s] = vol * G[q][s];
  if (Mp)
    for (int q = 0; q < nb; ++q)
      for (int s = 0; s < nb; ++s) Mp[q * nb + s] = vol * R->P1M[q][s];
  return det;
}

/* ------------------------------------------------------------------ */
/* Global assembly of the monolithic saddle-point matrix                */
/*   [ A  0 -Bx^T ]        unknowns [u_x | u_y | (u_z) | p],            */
/*   [ 0  A -By^T ]        A = mass_coef M + nu K + N(w) (per component)*/
/*   [ Bx By  D   ]        D = explicit zero pressure diagonal          */
/* through COO triplets sorted by (row, col, element order).            */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t key, ord;
  double v;
} triplet;

static int cmp_triplet(const void* a, const void* b) {
  const triplet* x = (const triplet*)a;
  const triplet* y = (const triplet*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->ord < y->ord ? -1 : (x->ord > y->ord ? 1 : 0);
}

int64_t or_assemble_capacity(int dim, int64_t ncell, int64_t nv) {
  int nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  return ncell * (int64_t)(dim * nloc * nloc + 2 * dim * nb * nloc) + nv;
}

/* w: convecting velocity, component-blocked dim x n2, or NULL.
 * rowptr: ndof+1 (int64); col, val: capacity entries.  Returns nnz. */
int64_t or_assemble(int dim, int64_t nv, int64_t n2, int64_t ncell,
                    const int32_t* c2d, const double* p2xyz, const double* w,
                    double mass_coef, double nu, int64_t* rowptr,
                    int32_t* col, double* val) {
  int nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  int64_t ndof = dim * n2 + nv;
  int64_t cap = or_assemble_capacity(dim, ncell, nv);
  triplet* T = (triplet*)malloc(sizeof(triplet) * (size_t)cap);
  int64_t nt = 0;
  double xv[12], wl[30], A[100], B[120];
  for (int64_t c = 0; c < ncell; ++c) {
    const int32_t* g = c2d + c * nloc;
    for (int v = 0; v < nb; ++v)
      for (int a = 0; a < dim; ++a) xv[v * dim + a] = p2xyz[(int64_t)g[v] * dim + a];
    if (w)
      for (int k = 0; k < nloc; ++k)
        for (int a = 0; a < dim; ++a) wl[k * dim + a] = w[a * n2 + g[k]];
    or_element(dim, xv, w ? wl : NULL, mass_coef, nu, A, NULL, NULL, NULL, B, NULL, NULL);
    for (int comp = 0; comp < dim; ++comp) {
      int64_t off = comp * n2;
      for (int i = 0; i < nloc; ++i)
        for (int j = 0; j < nloc; ++j) {
          T[nt].key = (off + g[i]) * ndof + (off + g[j]);
          T[nt].ord = nt;
          T[nt].v = A[i * nloc + j];
          nt++;
        }
      for (int q = 0; q < nb; ++q)
        for (int j = 0; j < nloc; ++j) {
          int64_t prow = dim * n2 + g[q];
          int64_t ucol = off + g[j];
          double bv = B[(comp * nb + q) * nloc + j];
          T[nt].key = prow * ndof + ucol;
          T[nt].ord = nt;
          T[nt].v = bv;
          nt++;
          T[nt].key = ucol * ndof + prow;
          T[nt].ord = nt;
          T[nt].v = -bv;
          nt++;
        }
    }
  }
  for (int64_t q = 0; q < nv; ++q) {
    int64_t r = dim * n2 + q;
    T[nt].key = r * ndof + r;
    T[nt].ord = nt;
    T[nt].v = 0.0;
    nt++;
  }
  qsort(T, (size_t)nt, sizeof(triplet), cmp_triplet);
  int64_t nnz = 0;
  for (int64_t r = 0; r <= ndof; ++r) rowptr[r] = 0;
  for (int64_t t = 0; t < nt; ++t) {
    if (t > 0 && T[t].key == T[t - 1].key) {
      val[nnz - 1] += T[t].v;
    } else {
      int64_t r = T[t].key / ndof;
      col[nnz] = (int32_t)(T[t].key % ndof);
      val[nnz] = T[t].v;
      rowptr[r + 1]++;
      nnz++;
    }
  }
  for (int64_t r = 0; r < ndof; ++r) rowptr[r + 1] += rowptr[r];
  free(T);
  return nnz;
}

/* Right-hand side b_u = M (inv_dt u^n + I_h f(t)), b_p = 0, assembled
 * element by element.  u_prev: component-blocked dim x n2 (or NULL = 0). */
void or_rhs(int dim, int64_t nv, int64_t n2, int64_t ncell, const int32_t* c2d,
            const double* p2xyz, const double* u_prev, int problem, double t,
            double nu, const double* wconst, double inv_dt, double* b) {
  int nloc = dim == 2 ? 6 : 10, nb = dim + 1;
  int64_t ndof = dim * n2 + nv;
  for (int64_t i = 0; i < ndof; ++i) b[i] = 0;
  double xv[12], M[100], g_l[30];
  for (int64_t c = 0; c < ncell; ++c) {
    const int32_t* g = c2d + c * nloc;
    for (int v = 0; v < nb; ++v)
      for (int a = 0; a < dim; ++a) xv[v * dim + a] = p2xyz[(int64_t)g[v] * dim + a];
    or_element(dim, xv, NULL, 0.0, 0.0, NULL, M, NULL, NULL, NULL, NULL, NULL);
    for (int j = 0; j < nloc; ++j) {
      double fj[3];
      or_exact(problem, dim, t, nu, wconst, p2xyz + (int64_t)g[j] * dim, NULL, NULL, fj);
      for (int a = 0; a < dim; ++a)
        g_l[j * dim + a] = (u_prev ? inv_dt * u_prev[a * n2 + g[j]] : 0.0) + fj[a];
    }
    for (int a = 0; a < dim; ++a)
      for (int i = 0; i < nloc; ++i) {
        double s = 0;
        for (int j = 0; j < nloc; ++j) s += M[i * nloc + j] * g_l[j * dim + a];
        b[a * n2 + g[i]] += s;
      }
  }
}

/* Dirichlet row replacement (pattern kept, off-diagonals set to zero):
 * velocity rows of masked P2 nodes take u_exact(x_i, t); when pin_p0 is
 * set, the row of pressure DOF 0 takes p_exact(x_0, t). */
void or_apply_bc(int dim, int64_t nv, int64_t n2, const int64_t* rowptr,
                 const int32_t* col, double* val, double* b,
                 const uint8_t* mask, const double* p2xyz, int problem,
                 double t, double nu, const double* wconst, int pin_p0) {
  for (int64_t i = 0; i < n2; ++i) {
    if (!mask[i]) continue;
    double u[3];
    or_exact(problem, dim, t, nu, wconst, p2xyz + i * dim, u, NULL, NULL);
    for (int a = 0; a < dim; ++a) {
      int64_t r = a * n2 + i;
      for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k)
        val[k] = (col[k] == r) ? 1.0 : 0.0;
      if (b) b[r] = u[a];
    }
  }
  if (pin_p0) {
    int64_t r = dim * n2;
    double p;
    or_exact(problem, dim, t, nu, wconst, p2xyz, NULL, &p, NULL);
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k)
      val[k] = (col[k] == r) ? 1.0 : 0.0;
    if (b) b[r] = p;
  }
}

/* y = A x for a CSR matrix with int64 row pointers. */
void or_spmv(int64_t n, const int64_t* rowptr, const int32_t* col,
             const double* val, const double* x, double* y) {
  for (int64_t r = 0; r < n; ++r) {
    double s = 0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += val[k] * x[col[k]];
    y[r] = s;
  }
}

/* ------------------------------------------------------------------ */
/* Linear solvers.                                                      */
/* ------------------------------------------------------------------ */

/* Dense LU with partial pivoting; A (n x n row-major) and b overwritten;
 * the solution is returned in b.  Returns 0, or 1 on a zero pivot. */
int or_dense_solve(int64_t n, double* A, double* b) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t piv = k;
    double best = fabs(A[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); piv = i; }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (int64_t j = 0; j < n; ++j) {
        double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int64_t i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      if (l == 0.0) continue;
      A[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int64_t j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  return 0;
}

/* ILU(0) on the CSR pattern (columns sorted ascending). */
static int ilu0(int64_t n, const int64_t* rp, const int32_t* ci, double* lu,
                int64_t* diag) {
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) pos[j] = -1;
  int rc = 0;
  for (int64_t i = 0; i < n && !rc; ++i) {
    diag[i] = -1;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      pos[ci[k]] = k;
      if (ci[k] == i) diag[i] = k;
    }
    for (int64_t k = rp[i]; k < rp[i + 1] && ci[k] < i; ++k) {
      int64_t kr = ci[k];
      double l = lu[k] / lu[diag[kr]];
      lu[k] = l;
      for (int64_t p = diag[kr] + 1; p < rp[kr + 1]; ++p)
        if (pos[ci[p]] >= 0) lu[pos[ci[p]]] -= l * lu[p];
    }
    if (diag[i] < 0 || lu[diag[i]] == 0.0) rc = 1;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) pos[ci[k]] = -1;
  }
  free(pos);
  return rc;
}

static void ilu0_apply(int64_t n, const int64_t* rp, const int32_t* ci,
                       const double* lu, const int64_t* diag, const double* r,
                       double* z) {
  for (int64_t i = 0; i < n; ++i) {
    double s = r[i];
    for (int64_t k = rp[i]; k < diag[i]; ++k) s -= lu[k] * z[ci[k]];
    z[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = z[i];
    for (int64_t k = diag[i] + 1; k < rp[i + 1]; ++k) s -= lu[k] * z[ci[k]];
    z[i] = s / lu[diag[i]];
  }
}

static double dotv(int64_t n, const double* a, const double* b) {
  double s = 0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Right-preconditioned restarted GMRES with ILU(0) and modified
 * Gram-Schmidt; stops when the TRUE residual ||b - Ax|| <= rtol ||b||
 * (recomputed at every restart).  x holds the initial guess on entry.
 * Returns 0 on convergence, 1 if the ILU broke down, 2 if maxit was hit,
 * 3 if a restart cycle stagnated (rounding floor reached). */
int or_gmres_ilu0(int64_t n, const int64_t* rp, const int32_t* ci,
                  const double* val, const double* b, double* x, int restart,
                  int maxit, double rtol, int* iters_out, double* relres_out) {
  int64_t nnz = rp[n];
  double* lu = (double*)malloc(sizeof(double) * (size_t)nnz);
  int64_t* diag = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  memcpy(lu, val, sizeof(double) * (size_t)nnz);
  if (ilu0(n, rp, ci, lu, diag)) {
    free(lu); free(diag);
    return 1;
  }
  int m = restart;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* Z = (double*)malloc(sizeof(double) * (size_t)n * m);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double*)malloc(sizeof(double) * m), *sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double bn = sqrt(dotv(n, b, b));
  if (bn == 0) bn = 1;
  int it = 0, rc = 2;
  double relres = 0, prev = INFINITY;
  while (1) {
    or_spmv(n, rp, ci, val, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    double beta = sqrt(dotv(n, r, r));
    relres = beta / bn;
    if (relres <= rtol) { rc = 0; break; }
    if (it >= maxit) break;
    /* a whole restart cycle that did not halve the true residual means the
     * iteration has reached the rounding floor of the problem */
    if (relres > 0.5 * prev) { rc = 3; break; }
    prev = relres;
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (int j = 0; j <= m; ++j) g[j] = 0;
    g[0] = beta;
    int j;
    for (j = 0; j < m && it < maxit; ++j, ++it) {
      double* z = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      ilu0_apply(n, rp, ci, lu, diag, V + (size_t)j * n, z);
      or_spmv(n, rp, ci, val, z, w);
      for (int i = 0; i <= j; ++i) {
        double h = dotv(n, w, V + (size_t)i * n);
        H[i * m + j] = h;
        for (int64_t k = 0; k < n; ++k) w[k] -= h * V[(size_t)i * n + k];
      }
      double hn = sqrt(dotv(n, w, w));
      H[(j + 1) * m + j] = hn;
      if (hn != 0)
        for (int64_t k = 0; k < n; ++k) w[k] /= hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double den = sqrt(a * a + c * c);
      cs[j] = den == 0 ? 1 : a / den;
      sn[j] = den == 0 ? 0 : c / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (fabs(g[j + 1]) <= 0.1 * rtol * bn) { ++j; ++it; break; }
    }
    /* x += Z y with H y = g (upper triangular, size j) */
    double* y = (double*)malloc(sizeof(double) * (j > 0 ? j : 1));
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < j; ++i)
      for (int64_t k = 0; k < n; ++k) x[k] += y[i] * Z[(size_t)i * n + k];
    free(y);
  }
  *iters_out = it;
  *relres_out = relres;
  free(lu); free(diag); free(V); free(Z); free(H); free(cs); free(sn); free(g); free(r);
  return rc;
}
