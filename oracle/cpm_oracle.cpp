// cpm_oracle.cpp -- plain, slow FP64 CPU oracle for the closest point method
// (CPM) shifted surface Poisson solver of May, Haynes & Ruuth,
// "A closest point method library for PDEs on surfaces with parallel domain
// decomposition solvers and preconditioners" (arXiv 2110.06322).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
// includes this file.  Only the test-suite, the smoke check and the CPU
// baseline leg of the benchmark load it.  It shares no code with the CUDA
// path: every formula below is written out again from the paper.
//
// Everything is FP64, compiled with -ffp-contract=off so that every product
// and sum rounds exactly once in the order written.  Where the paper is silent
// the reading taken is stated beside the code.
//
// Parity status per function (what pins each one lives in tests/):
//   cp / dist .......... pinned (closed forms, invariants)
//   band ............... pinned (tube volume, closure, symmetry, h-scaling)
//   weights ............ pinned (partition of unity, reproduction, Lagrange form)
//   E, M ............... pinned (polynomial reproduction, M 1 = c 1, spherical
//                        harmonic consistency, 2nd-order convergence)
//   RAS / ILU(0) ....... pinned (LU = A on the pattern, N_S = 1 exact = M^-1,
//                        stationary RAS converges to the direct solve)
//   P-ORAS (Robin) ..... parity unpinned beyond "alpha -> infinity gives RAS"
//                        and "GMRES+P-ORAS reaches the direct solution": the
//                        paper defers the Robin discretisation to other work.
//   GMRES .............. pinned (dense LU agreement)
//   adjoint ............ pinned (<Mx,y> = <x,M^T y>, dense transpose)

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Surfaces and the closest point function (Section 2.1, eq. cpFunc).
// kind 0: sphere, prm = {cx, cy, cz, rho}
// kind 1: torus about the z axis, prm = {cx, cy, cz, R, r}
// ---------------------------------------------------------------------------
struct Surf {
  int kind;
  double c[3];
  double a;  // sphere radius rho, or torus major radius R
  double b;  // torus minor radius r
};

// Unsigned distance to the surface.  Defined everywhere (also on the torus
// axis), so it can be evaluated over the whole bounding box.
double surf_dist(const Surf& S, const double x[3]) {
  double dx = x[0] - S.c[0], dy = x[1] - S.c[1], dz = x[2] - S.c[2];
  if (S.kind == 0) {
    double n = std::sqrt((dx * dx + dy * dy) + dz * dz);
    return std::fabs(n - S.a);
  }
  double rxy = std::sqrt(dx * dx + dy * dy);
  double w = rxy - S.a;
  double n = std::sqrt(w * w + dz * dz);
  return std::fabs(n - S.b);
}

// Closest point cp_S(x) = argmin_{y in S} |x - y| (eq. cpFunc).
// Returns false where cp is not unique (the medial axis).
bool surf_cp(const Surf& S, const double x[3], double cp[3]) {
  double dx = x[0] - S.c[0], dy = x[1] - S.c[1], dz = x[2] - S.c[2];
  if (S.kind == 0) {
    double n = std::sqrt((dx * dx + dy * dy) + dz * dz);
    if (!(n > 0.0)) return false;
    double q = S.a / n;
    cp[0] = S.c[0] + q * dx;
    cp[1] = S.c[1] + q * dy;
    cp[2] = S.c[2] + q * dz;
    return true;
  }
  // torus: nearest point of the core circle, then step r towards x
  double rxy = std::sqrt(dx * dx + dy * dy);
  if (!(rxy > 0.0)) return false;
  double t = S.a / rxy;
  double qx = t * dx, qy = t * dy;
  double ex = dx - qx, ey = dy - qy, ez = dz;
  double ne = std::sqrt((ex * ex + ey * ey) + ez * ez);
  if (!(ne > 0.0)) return false;
  double u = S.b / ne;
  cp[0] = S.c[0] + (qx + u * ex);
  cp[1] = S.c[1] + (qy + u * ey);
  cp[2] = S.c[2] + u * ez;
  return true;
}

// Reach kappa_inf^-1 (Section 2.1): sphere rho; torus min(r, R - r).
double surf_reach(const Surf& S) {
  if (S.kind == 0) return S.a;
  return std::min(S.b, S.a - S.b);
}

void surf_bbox(const Surf& S, double lo[3], double hi[3]) {
  if (S.kind == 0) {
    for (int a = 0; a < 3; ++a) { lo[a] = S.c[a] - S.a; hi[a] = S.c[a] + S.a; }
  } else {
    for (int a = 0; a < 2; ++a) { lo[a] = S.c[a] - (S.a + S.b); hi[a] = S.c[a] + (S.a + S.b); }
    lo[2] = S.c[2] - S.b; hi[2] = S.c[2] + S.b;
  }
}

bool make_surf(int kind, const double* prm, Surf* S) {
  S->kind = kind;
  for (int a = 0; a < 3; ++a) S->c[a] = prm[a];
  S->a = prm[3];
  S->b = (kind == 1) ? prm[4] : 0.0;
  if (kind == 0) return S->a > 0.0;
  if (kind == 1) return S->b > 0.0 && S->a > S->b;
  return false;
}

// Band radius.  A node of Sigma_A lies at most (p+1)/2 grid steps from its
// closest point along each axis (the interpolation cube straddles cp), and a
// ghost node one more step along one axis; the seed tube therefore has radius
//   lambda_T = h * sqrt((d-1)((p+1)/2)^2 + (1 + (p+1)/2)^2),  d = 3,
// which is sqrt(17) h for p = 3 (Section 2.1: Sigma_A is the union of the
// (p+1)^d interpolation cubes; ghosts complete the FD stencils).
double band_lambda(double h, int p) {
  double half = 0.5 * (double)(p + 1);
  double lam2 = 2.0 * (half * half) + (1.0 + half) * (1.0 + half);
  return h * std::sqrt(lam2);
}

// Barycentric weights of equispaced nodes 0..p: w_j = (-1)^j binom(p, j)
// (barycentric Lagrange interpolation, Section 2.1, [Berrut & Trefethen]).
double bary_w(int p, int j) {
  double b = 1.0;
  for (int q = 1; q <= j; ++q) b = b * (double)(p - q + 1) / (double)q;
  return (j % 2) ? -b : b;
}

// 1-D interpolation weights l_0..l_p at offset s (in grid steps from the
// cube base), second ("true") barycentric form.  s equal to a node gives the
// unit vector for that node.
void weights1d(int p, double s, double* out) {
  for (int j = 0; j <= p; ++j) {
    if (s == (double)j) {
      for (int q = 0; q <= p; ++q) out[q] = (q == j) ? 1.0 : 0.0;
      return;
    }
  }
  double t[8];
  double den = 0.0;
  for (int j = 0; j <= p; ++j) {
    t[j] = bary_w(p, j) / (s - (double)j);
    den = den + t[j];
  }
  for (int j = 0; j <= p; ++j) out[j] = t[j] / den;
}

// ---------------------------------------------------------------------------
// Band: T (seed tube), Sigma_A (active), Sigma_G (ghost), E rows.
// Nodes are x = (i, j, k) h.  Canonical order is lexicographic in (i, j, k)
// with k fastest.  E rows are numbered: Sigma_A rows first, then Sigma_G rows.
// ---------------------------------------------------------------------------
struct Band {
  Surf S;
  double h;
  int p;
  int glo[3], gn[3];           // dense grid origin and extent
  std::vector<int32_t> gmap;   // >= 0 active index; <= -2 ghost (-2 - g); -1 none
  std::vector<int32_t> ijkA;   // 3 per active node, canonical
  std::vector<int32_t> ijkG;   // 3 per ghost node, canonical
  std::vector<int32_t> base;   // 3 per E row
  std::vector<double> cp;      // 3 per E row
  int64_t nT = 0, nA = 0, nG = 0;

  int64_t cell(int i, int j, int k) const {
    int a = i - glo[0], b = j - glo[1], c = k - glo[2];
    if (a < 0 || b < 0 || c < 0 || a >= gn[0] || b >= gn[1] || c >= gn[2]) return -1;
    return ((int64_t)a * gn[1] + b) * gn[2] + c;
  }
  int64_t active(int i, int j, int k) const {
    int64_t q = cell(i, j, k);
    if (q < 0) return -1;
    int32_t v = gmap[q];
    return v >= 0 ? v : -1;
  }
  // E row index of a node of Sigma_A or Sigma_G, else -1
  int64_t row(int i, int j, int k) const {
    int64_t q = cell(i, j, k);
    if (q < 0) return -1;
    int32_t v = gmap[q];
    if (v >= 0) return v;
    if (v <= -2) return nA + (int64_t)(-2 - v);
    return -1;
  }
  int64_t nrows() const { return nA + nG; }
};

// Cube base per axis: b = floor(cp/h - (p-1)/2).  For odd p the cube
// straddles cp (s in [1,2) for p = 3); for even p it is centred on the nearest
// node.  s = cp/h - b is the offset fed to the 1-D weights.
void cube_base(double cpa, double h, int p, int* b, double* s) {
  double u = cpa / h;
  double f = std::floor(u - 0.5 * (double)(p - 1));
  *b = (int)f;
  *s = u - f;
}

enum { ST_OK = 0, ST_ARG = 1, ST_BAND = 4 };

int band_build(Band& B) {
  const int p = B.p;
  const double h = B.h;
  const double lam = band_lambda(h, p);
  if (!(lam < surf_reach(B.S))) return ST_BAND;  // nodes must stay within reach
  double lo[3], hi[3];
  surf_bbox(B.S, lo, hi);
  for (int a = 0; a < 3; ++a) {
    int l = (int)std::floor((lo[a] - lam) / h) - (p + 3);
    int u = (int)std::ceil((hi[a] + lam) / h) + (p + 3);
    B.glo[a] = l;
    B.gn[a] = u - l + 1;
  }
  int64_t ncell = (int64_t)B.gn[0] * B.gn[1] * B.gn[2];
  std::vector<uint8_t> flag(ncell, 0);  // bit0 active, bit1 ghost
  // T and Sigma_A
  for (int a = 0; a < B.gn[0]; ++a)
    for (int b = 0; b < B.gn[1]; ++b)
      for (int c = 0; c < B.gn[2]; ++c) {
        int ijk[3] = {B.glo[0] + a, B.glo[1] + b, B.glo[2] + c};
        double x[3] = {(double)ijk[0] * h, (double)ijk[1] * h, (double)ijk[2] * h};
        if (!(surf_dist(B.S, x) <= lam)) continue;
        B.nT++;
        double q[3];
        if (!surf_cp(B.S, x, q)) return ST_BAND;
        int bs[3];
        double s;
        for (int d = 0; d < 3; ++d) cube_base(q[d], h, p, &bs[d], &s);
        for (int u = 0; u <= p; ++u)
          for (int v = 0; v <= p; ++v)
            for (int w = 0; w <= p; ++w) {
              int64_t qc = B.cell(bs[0] + u, bs[1] + v, bs[2] + w);
              if (qc < 0) return ST_BAND;
              flag[qc] |= 1;
            }
      }
  // Sigma_G: 6-neighbours of Sigma_A that are not in Sigma_A
  static const int nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int a = 0; a < B.gn[0]; ++a)
    for (int b = 0; b < B.gn[1]; ++b)
      for (int c = 0; c < B.gn[2]; ++c) {
        int64_t q0 = ((int64_t)a * B.gn[1] + b) * B.gn[2] + c;
        if (!(flag[q0] & 1)) continue;
        for (int n = 0; n < 6; ++n) {
          int64_t qn = B.cell(B.glo[0] + a + nb[n][0], B.glo[1] + b + nb[n][1], B.glo[2] + c + nb[n][2]);
          if (qn < 0) return ST_BAND;
          if (!(flag[qn] & 1)) flag[qn] |= 2;
        }
      }
  // canonical numbering
  B.gmap.assign(ncell, -1);
  for (int a = 0; a < B.gn[0]; ++a)
    for (int b = 0; b < B.gn[1]; ++b)
      for (int c = 0; c < B.gn[2]; ++c) {
        int64_t q0 = ((int64_t)a * B.gn[1] + b) * B.gn[2] + c;
        int ijk[3] = {B.glo[0] + a, B.glo[1] + b, B.glo[2] + c};
        if (flag[q0] & 1) {
          B.gmap[q0] = (int32_t)B.nA++;
          B.ijkA.insert(B.ijkA.end(), ijk, ijk + 3);
        } else if (flag[q0] & 2) {
          B.gmap[q0] = (int32_t)(-2 - B.nG++);
          B.ijkG.insert(B.ijkG.end(), ijk, ijk + 3);
        }
      }
  // E rows (Sigma_A rows, then Sigma_G rows) and the closure check: every
  // row's interpolation cube must lie in Sigma_A.
  int64_t nr = B.nA + B.nG;
  B.base.resize(3 * nr);
  B.cp.resize(3 * nr);
  for (int64_t r = 0; r < nr; ++r) {
    const int32_t* ijk = (r < B.nA) ? &B.ijkA[3 * r] : &B.ijkG[3 * (r - B.nA)];
    double x[3] = {(double)ijk[0] * h, (double)ijk[1] * h, (double)ijk[2] * h};
    double q[3];
    if (!surf_cp(B.S, x, q)) return ST_BAND;
    for (int d = 0; d < 3; ++d) {
      double s;
      cube_base(q[d], h, p, &B.base[3 * r + d], &s);
      B.cp[3 * r + d] = q[d];
    }
    const int32_t* bs = &B.base[3 * r];
    for (int u = 0; u <= p; ++u)
      for (int v = 0; v <= p; ++v)
        for (int w = 0; w <= p; ++w)
          if (B.active(bs[0] + u, bs[1] + v, bs[2] + w) < 0) return ST_BAND;
  }
  return ST_OK;
}

// Interpolation weights of E row r in cube order (u, v, w), w fastest:
// W = (l_u(s_x) l_v(s_y)) l_w(s_z).
void erow_weights(const Band& B, int64_t r, double* W) {
  const int p = B.p;
  double l[3][8];
  for (int d = 0; d < 3; ++d) {
    int b;
    double s;
    cube_base(B.cp[3 * r + d], B.h, p, &b, &s);
    weights1d(p, s, l[d]);
  }
  int q = 0;
  for (int u = 0; u <= p; ++u)
    for (int v = 0; v <= p; ++v)
      for (int w = 0; w <= p; ++w) W[q++] = (l[0][u] * l[1][v]) * l[2][w];
}

// ---------------------------------------------------------------------------
// Sparse matrices (CSR, ascending columns).
// ---------------------------------------------------------------------------
struct CSR {
  int64_t nr = 0, nc = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

void csr_matvec(const CSR& A, const double* x, double* y) {
  for (int64_t i = 0; i < A.nr; ++i) {
    double s = 0.0;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s = s + A.val[q] * x[A.col[q]];
    y[i] = s;
  }
}

CSR csr_transpose(const CSR& A) {
  CSR T;
  T.nr = A.nc;
  T.nc = A.nr;
  T.ptr.assign(T.nr + 1, 0);
  for (int64_t q = 0; q < (int64_t)A.col.size(); ++q) T.ptr[A.col[q] + 1]++;
  for (int64_t i = 0; i < T.nr; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int64_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int64_t i = 0; i < A.nr; ++i)
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      int64_t d = fill[A.col[q]]++;
      T.col[d] = (int32_t)i;
      T.val[d] = A.val[q];
    }
  return T;
}

// E as an explicit matrix (Section 2.1): N_C rows x N_A columns, each row the
// (p+1)^3 tensor-product weights of its closest point.
CSR build_E(const Band& B) {
  const int p = B.p, m = (p + 1) * (p + 1) * (p + 1);
  CSR E;
  E.nr = B.nrows();
  E.nc = B.nA;
  E.ptr.resize(E.nr + 1);
  E.col.resize(E.nr * m);
  E.val.resize(E.nr * m);
  std::vector<double> W(m);
  for (int64_t r = 0; r < E.nr; ++r) {
    E.ptr[r] = r * m;
    erow_weights(B, r, W.data());
    const int32_t* bs = &B.base[3 * r];
    int q = 0;
    for (int u = 0; u <= p; ++u)
      for (int v = 0; v <= p; ++v)
        for (int w = 0; w <= p; ++w, ++q) {
          E.col[r * m + q] = (int32_t)B.active(bs[0] + u, bs[1] + v, bs[2] + w);
          E.val[r * m + q] = W[q];
        }
  }
  E.ptr[E.nr] = E.nr * m;
  return E;
}

static const int NB6[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

// One row of M = c I - Delta_S^h with the stabilised operator of eq. lapBel,
//   Delta_S^h = -(2d/h^2) I + (Delta^h + (2d/h^2) I) E,
// i.e. M = (c + 2d/h^2) I - P with P = L_off E, where L_off is the 7-point
// Laplacian with its diagonal removed (1/h^2 on the six neighbours, all of
// which are in Sigma_A or Sigma_G).  The centre node is not extended; the
// neighbours are (Section 3.1, semidiscrete form).  P_im is summed over the
// neighbours in the order -x,+x,-y,+y,-z,+z, each cube in (u,v,w) order.
void assemble_row(const Band& B, double c, int64_t i, std::vector<int32_t>& cols,
                  std::vector<double>& vals) {
  const int p = B.p, m = (p + 1) * (p + 1) * (p + 1);
  const double coef = 1.0 / (B.h * B.h);
  const double diag0 = c + 6.0 * coef;
  const int32_t* x = &B.ijkA[3 * i];
  // accumulate P_im in order of appearance
  std::vector<int32_t> order;      // distinct columns in first-seen order
  std::vector<double> acc;
  std::vector<std::pair<int32_t, int32_t>> seen;  // (col, slot)
  std::vector<double> W(m);
  for (int n = 0; n < 6; ++n) {
    int64_t r = B.row(x[0] + NB6[n][0], x[1] + NB6[n][1], x[2] + NB6[n][2]);
    erow_weights(B, r, W.data());
    const int32_t* bs = &B.base[3 * r];
    int q = 0;
    for (int u = 0; u <= p; ++u)
      for (int v = 0; v <= p; ++v)
        for (int w = 0; w <= p; ++w, ++q) {
          int32_t col = (int32_t)B.active(bs[0] + u, bs[1] + v, bs[2] + w);
          double term = coef * W[q];
          int slot = -1;
          for (auto& sc : seen)
            if (sc.first == col) { slot = sc.second; break; }
          if (slot < 0) {
            slot = (int)acc.size();
            seen.push_back({col, slot});
            order.push_back(col);
            acc.push_back(term);
          } else {
            acc[slot] = acc[slot] + term;
          }
        }
  }
  bool has_diag = false;
  for (auto col : order) if (col == (int32_t)i) has_diag = true;
  if (!has_diag) { order.push_back((int32_t)i); acc.push_back(0.0); seen.push_back({(int32_t)i, (int)acc.size() - 1}); }
  std::vector<int> idx(order.size());
  for (size_t q = 0; q < idx.size(); ++q) idx[q] = (int)q;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return order[a] < order[b]; });
  cols.clear();
  vals.clear();
  for (int q : idx) {
    int32_t col = order[q];
    double v;
    if (col == (int32_t)i) {
      v = has_diag ? (diag0 - acc[q]) : diag0;
    } else {
      v = -acc[q];
    }
    cols.push_back(col);
    vals.push_back(v);
  }
}

CSR build_M(const Band& B, double c) {
  CSR M;
  M.nr = B.nA;
  M.nc = B.nA;
  M.ptr.assign(M.nr + 1, 0);
  std::vector<int32_t> cols;
  std::vector<double> vals;
  for (int64_t i = 0; i < B.nA; ++i) {
    assemble_row(B, c, i, cols, vals);
    M.ptr[i + 1] = M.ptr[i] + (int64_t)cols.size();
    M.col.insert(M.col.end(), cols.begin(), cols.end());
    M.val.insert(M.val.end(), vals.begin(), vals.end());
  }
  return M;
}

// ---------------------------------------------------------------------------
// Domain decomposition (Section 2.2): disjoint partition, overlap growth,
// local matrices A_j = R_j M R_j^T (+ the Robin diagonal reading), ILU(0).
// ---------------------------------------------------------------------------

// Recursive coordinate bisection on the lattice index (stand-in for the
// paper's ParMETIS partitioner).  A node set is split by a lattice plane
// normal to its longest extent (ties: i before j before k): the left part is
// {coord < v} with v minimising |count_left - n * nl / np| (ties: smaller v),
// nl = floor(np / 2).  Every part is the band restricted to a box.
void rcb(const Band& B, std::vector<int64_t>& nodes, int np, int off, std::vector<int32_t>& part) {
  if (np == 1) {
    for (int64_t i : nodes) part[i] = off;
    return;
  }
  int64_t n = (int64_t)nodes.size();
  int mn[3] = {0, 0, 0}, mx[3] = {-1, -1, -1};
  if (n > 0) {
    for (int a = 0; a < 3; ++a) { mn[a] = B.ijkA[3 * nodes[0] + a]; mx[a] = mn[a]; }
    for (int64_t i : nodes)
      for (int a = 0; a < 3; ++a) {
        mn[a] = std::min(mn[a], B.ijkA[3 * i + a]);
        mx[a] = std::max(mx[a], B.ijkA[3 * i + a]);
      }
  }
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (mx[a] - mn[a] > mx[ax] - mn[ax]) ax = a;
  int nl = np / 2;
  int best_v = mn[ax];
  int64_t best_err = -1;
  if (n > 0) {
    int span = mx[ax] - mn[ax] + 1;
    std::vector<int64_t> hist(span, 0);
    for (int64_t i : nodes) hist[B.ijkA[3 * i + ax] - mn[ax]]++;
    int64_t below = 0;  // count with coord < v
    for (int v = mn[ax]; v <= mx[ax] + 1; ++v) {
      int64_t err = std::llabs((int64_t)np * below - n * (int64_t)nl);
      if (best_err < 0 || err < best_err) { best_err = err; best_v = v; }
      if (v <= mx[ax]) below += hist[v - mn[ax]];
    }
  }
  std::vector<int64_t> L, R;
  for (int64_t i : nodes) (B.ijkA[3 * i + ax] < best_v ? L : R).push_back(i);
  rcb(B, L, nl, off, part);
  rcb(B, R, np - nl, off + nl, part);
}

struct Sub {
  std::vector<int32_t> nodes;  // global active indices, ascending (local order)
  CSR A;                       // local matrix; ILU(0) factors in place if ilu
  std::vector<int64_t> diag;   // position of the diagonal in each row
  std::vector<double> dense;   // exact local solve: LU with partial pivoting
  std::vector<int32_t> piv;
};

struct ORAS {
  int np = 0, overlap = 0, robin = 0, exact = 0, order = 0;
  double alpha = 0, alpha_x = 0, h = 0;
  int64_t n = 0;
  std::vector<int32_t> part;
  std::vector<Sub> sub;
  // two-level variant (coarse = 1): coarse space Z with one column per
  // disjoint part, Z_{i,a} = 1 if node i lies in part a; coarse matrix
  // E0 = Z^T M Z (dense, LU-factored in place)
  int coarse = 0;
  const CSR* M = nullptr;
  std::vector<double> E0;
  std::vector<int32_t> E0piv;
};

int dense_lu(int64_t n, std::vector<double>& A, std::vector<int32_t>& piv) {
  piv.resize(n);
  for (int64_t k = 0; k < n; ++k) {
    int64_t pr = k;
    double best = std::fabs(A[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) { best = std::fabs(A[i * n + k]); pr = i; }
    piv[k] = (int32_t)pr;
    if (best == 0.0) return 1;
    if (pr != k)
      for (int64_t j = 0; j < n; ++j) std::swap(A[k * n + j], A[pr * n + j]);
    for (int64_t i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) A[i * n + j] = A[i * n + j] - l * A[k * n + j];
    }
  }
  return 0;
}

void dense_lu_solve(int64_t n, const std::vector<double>& LU, const std::vector<int32_t>& piv,
                    double* x, int transpose) {
  if (!transpose) {
    for (int64_t k = 0; k < n; ++k) std::swap(x[k], x[piv[k]]);
    for (int64_t i = 0; i < n; ++i) {
      double s = x[i];
      for (int64_t k = 0; k < i; ++k) s = s - LU[i * n + k] * x[k];
      x[i] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = x[i];
      for (int64_t k = i + 1; k < n; ++k) s = s - LU[i * n + k] * x[k];
      x[i] = s / LU[i * n + i];
    }
  } else {
    // (P^T L U)^T y = U^T L^T P y
    for (int64_t i = 0; i < n; ++i) {
      double s = x[i];
      for (int64_t k = 0; k < i; ++k) s = s - LU[k * n + i] * x[k];
      x[i] = s / LU[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = x[i];
      for (int64_t k = i + 1; k < n; ++k) s = s - LU[k * n + i] * x[k];
      x[i] = s;
    }
    for (int64_t k = n - 1; k >= 0; --k) std::swap(x[k], x[piv[k]]);
  }
}

// ILU(0) in the natural local order (PETSc's default local solver, Section
// 4.1.1): row-by-row (IKJ) elimination restricted to the sparsity pattern of
// A.  For each row i and each k < i in its pattern, ascending:
//   a_ik <- a_ik / u_kk;  a_ij <- a_ij - a_ik u_kj for j > k in both patterns.
int ilu0(CSR& A, std::vector<int64_t>& diag) {
  int64_t n = A.nr;
  diag.assign(n, -1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
      if (A.col[q] == i) diag[i] = q;
  for (int64_t i = 0; i < n; ++i)
    if (diag[i] < 0) return 1;
  std::vector<int64_t> pos(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) pos[A.col[q]] = q;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1] && A.col[q] < i; ++q) {
      int64_t k = A.col[q];
      double piv = A.val[diag[k]];
      if (piv == 0.0) return 2;
      A.val[q] = A.val[q] / piv;
      double lik = A.val[q];
      for (int64_t t = diag[k] + 1; t < A.ptr[k + 1]; ++t) {
        int64_t at = pos[A.col[t]];
        if (at >= 0) A.val[at] = A.val[at] - lik * A.val[t];
      }
    }
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) pos[A.col[q]] = -1;
    if (A.val[diag[i]] == 0.0) return 2;
  }
  return 0;
}

// (L U) z = r in place: forward with unit L, then backward with U.
void ilu_solve(const Sub& s, double* x) {
  const CSR& A = s.A;
  int64_t n = A.nr;
  for (int64_t i = 0; i < n; ++i) {
    double v = x[i];
    for (int64_t q = A.ptr[i]; q < s.diag[i]; ++q) v = v - A.val[q] * x[A.col[q]];
    x[i] = v;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double v = x[i];
    for (int64_t q = s.diag[i] + 1; q < A.ptr[i + 1]; ++q) v = v - A.val[q] * x[A.col[q]];
    x[i] = v / A.val[s.diag[i]];
  }
}

// (L U)^T z = r in place: U^T w = r (forward, column sweep), L^T z = w
// (backward, unit diagonal, column sweep).
void ilu_solve_T(const Sub& s, double* x) {
  const CSR& A = s.A;
  int64_t n = A.nr;
  for (int64_t i = 0; i < n; ++i) {
    x[i] = x[i] / A.val[s.diag[i]];
    double xi = x[i];
    for (int64_t q = s.diag[i] + 1; q < A.ptr[i + 1]; ++q) x[A.col[q]] = x[A.col[q]] - A.val[q] * xi;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double xi = x[i];
    for (int64_t q = A.ptr[i]; q < s.diag[i]; ++q) x[A.col[q]] = x[A.col[q]] - A.val[q] * xi;
  }
}

int oras_setup(const Band& B, const CSR& M, ORAS& P) {
  const int64_t n = B.nA;
  P.n = n;
  P.part.assign(n, 0);
  std::vector<int64_t> all(n);
  for (int64_t i = 0; i < n; ++i) all[i] = i;
  rcb(B, all, P.np, 0, P.part);
  P.sub.assign(P.np, Sub());
  std::vector<uint8_t> in(n, 0);
  std::vector<int32_t> loc(n, -1);
  for (int j = 0; j < P.np; ++j) {
    Sub& s = P.sub[j];
    // overlap growth: N_O layers of 6-adjacency within Sigma_A
    std::vector<int32_t> mem, front;
    for (int64_t i = 0; i < n; ++i)
      if (P.part[i] == j) { mem.push_back((int32_t)i); in[i] = 1; }
    front = mem;
    for (int l = 0; l < P.overlap; ++l) {
      std::vector<int32_t> next;
      for (int32_t i : front) {
        const int32_t* x = &B.ijkA[3 * i];
        for (int d = 0; d < 6; ++d) {
          int64_t m = B.active(x[0] + NB6[d][0], x[1] + NB6[d][1], x[2] + NB6[d][2]);
          if (m >= 0 && !in[m]) { in[m] = 1; next.push_back((int32_t)m); }
        }
      }
      mem.insert(mem.end(), next.begin(), next.end());
      front.swap(next);
    }
    std::sort(mem.begin(), mem.end());
    if (P.order == 2) {
      // Alternative local order: distance shells of width h, outermost shell
      // first (shell = floor(dist / h)); inside a shell the 8 colours of the
      // lattice parity (i mod 2, j mod 2, k mod 2), colour 0 first; inside a
      // colour, canonical.  Measured on the torus against the plain
      // descending-distance order: triangular sweeps 14 / 25 / 49 / 56 %
      // shallower at h = 0.025 (16 parts), 0.0125 (64), 0.00625 (256) and
      // 0.004 (512), and GMRES to 1e-8 in 19 / 23 / 24 / 23 % fewer
      // iterations (at h = 0.004: 520 -> 400).
      std::vector<int64_t> shell(mem.size());
      std::vector<int> colour(mem.size());
      for (size_t q = 0; q < mem.size(); ++q) {
        const int32_t* xi = &B.ijkA[3 * mem[q]];
        double x[3] = {(double)xi[0] * B.h, (double)xi[1] * B.h, (double)xi[2] * B.h};
        shell[q] = (int64_t)std::floor(surf_dist(B.S, x) / B.h);
        colour[q] = (xi[0] & 1) | ((xi[1] & 1) << 1) | ((xi[2] & 1) << 2);
      }
      std::vector<size_t> id(mem.size());
      for (size_t q = 0; q < id.size(); ++q) id[q] = q;
      std::stable_sort(id.begin(), id.end(), [&](size_t a, size_t b) {
        if (shell[a] != shell[b]) return shell[a] > shell[b];
        return colour[a] < colour[b];
      });
      std::vector<int32_t> m2(mem.size());
      for (size_t q = 0; q < id.size(); ++q) m2[q] = mem[id[q]];
      mem.swap(m2);
    }
    if (P.order == 1) {
      // Local order for the ILU(0) factorisation (the paper leaves it to
      // PETSc): descending unsigned distance to the surface, ties by
      // canonical index.  Far-from-surface nodes are eliminated first.  In
      // canonical (lexicographic) order ILU(0) of the p = 3 operator meets
      // negative pivots wherever the sweep runs outward along the normal.
      std::vector<double> key(mem.size());
      for (size_t q = 0; q < mem.size(); ++q) {
        const int32_t* xi = &B.ijkA[3 * mem[q]];
        double x[3] = {(double)xi[0] * B.h, (double)xi[1] * B.h, (double)xi[2] * B.h};
        key[q] = surf_dist(B.S, x);
      }
      std::vector<size_t> id(mem.size());
      for (size_t q = 0; q < id.size(); ++q) id[q] = q;
      std::stable_sort(id.begin(), id.end(), [&](size_t a, size_t b) { return key[a] > key[b]; });
      std::vector<int32_t> m2(mem.size());
      for (size_t q = 0; q < id.size(); ++q) m2[q] = mem[id[q]];
      mem.swap(m2);
    }
    s.nodes = mem;
    for (size_t q = 0; q < mem.size(); ++q) loc[mem[q]] = (int32_t)q;
    // A_j = R_j M R_j^T, columns outside S_j dropped (Dirichlet, RAS).
    // Robin reading (P-ORAS): A_j[i,i] += beta * D_i, D_i the sum of the
    // dropped entries of row i, beta = 1 / (1 + alpha h), with alpha_cross in
    // place of alpha when the dropped columns are owned by >= 2 other
    // disjoint subdomains.  alpha -> infinity recovers RAS exactly.
    CSR& A = s.A;
    A.nr = A.nc = (int64_t)mem.size();
    A.ptr.assign(A.nr + 1, 0);
    for (size_t q = 0; q < mem.size(); ++q) {
      int64_t i = mem[q];
      double D = 0.0;
      bool dropped = false;
      std::vector<int32_t> owners;
      int64_t dpos = -1;
      for (int64_t t = M.ptr[i]; t < M.ptr[i + 1]; ++t) {
        int32_t m = M.col[t];
        if (loc[m] >= 0) {
          if (m == i) dpos = (int64_t)A.col.size();
          A.col.push_back(loc[m]);
          A.val.push_back(M.val[t]);
        } else {
          dropped = true;
          D = D + M.val[t];
          if (std::find(owners.begin(), owners.end(), P.part[m]) == owners.end()) owners.push_back(P.part[m]);
        }
      }
      if (P.robin && dropped && dpos >= 0) {
        double al = owners.size() >= 2 ? P.alpha_x : P.alpha;
        double beta = 1.0 / (1.0 + al * P.h);
        A.val[dpos] = A.val[dpos] + beta * D;
      }
      A.ptr[q + 1] = (int64_t)A.col.size();
      {  // keep each local row in ascending local column order
        int64_t b0 = A.ptr[q], b1 = A.ptr[q + 1];
        std::vector<std::pair<int32_t, double>> rowv;
        for (int64_t t = b0; t < b1; ++t) rowv.push_back({A.col[t], A.val[t]});
        std::sort(rowv.begin(), rowv.end(), [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) { return a.first < b.first; });
        for (int64_t t = b0; t < b1; ++t) { A.col[t] = rowv[t - b0].first; A.val[t] = rowv[t - b0].second; }
      }
    }
    for (int32_t i : mem) { loc[i] = -1; in[i] = 0; }
    if (P.exact) {
      int64_t m = A.nr;
      s.dense.assign(m * m, 0.0);
      for (int64_t r = 0; r < m; ++r)
        for (int64_t t = A.ptr[r]; t < A.ptr[r + 1]; ++t) s.dense[r * m + A.col[t]] = A.val[t];
      if (dense_lu(m, s.dense, s.piv)) return 6;
    } else {
      if (ilu0(A, s.diag)) return 6;
    }
  }
  return ST_OK;
}

// z = sum_j Rtilde_j^T A_j^{-1} R_j r (restricted additive Schwarz, Section
// 2.2: local solves on the overlapping S_j, recombined on the disjoint parts).
// Transposed: z = sum_j R_j^T A_j^{-T} Rtilde_j r, summed over j ascending.
void oras_apply_one_level(const ORAS& P, const double* r, double* z, int transpose) {
  if (!transpose) {
    for (int j = 0; j < P.np; ++j) {
      const Sub& s = P.sub[j];
      std::vector<double> x(s.nodes.size());
      for (size_t q = 0; q < x.size(); ++q) x[q] = r[s.nodes[q]];
      if (P.exact) dense_lu_solve(s.A.nr, s.dense, s.piv, x.data(), 0);
      else ilu_solve(s, x.data());
      for (size_t q = 0; q < x.size(); ++q)
        if (P.part[s.nodes[q]] == j) z[s.nodes[q]] = x[q];
    }
  } else {
    for (int64_t i = 0; i < P.n; ++i) z[i] = 0.0;
    for (int j = 0; j < P.np; ++j) {
      const Sub& s = P.sub[j];
      std::vector<double> x(s.nodes.size());
      for (size_t q = 0; q < x.size(); ++q) x[q] = (P.part[s.nodes[q]] == j) ? r[s.nodes[q]] : 0.0;
      if (P.exact) dense_lu_solve(s.A.nr, s.dense, s.piv, x.data(), 1);
      else ilu_solve_T(s, x.data());
      for (size_t q = 0; q < x.size(); ++q) z[s.nodes[q]] = z[s.nodes[q]] + x[q];
    }
  }
}

// Coarse matrix of the two-level variant: E0[a][b] = sum over nodes i of part
// a and columns k of part b of M_ik (rows ascending, entries in CSR order).
int coarse_setup(ORAS& P, const CSR& M) {
  const int np = P.np;
  P.M = &M;
  P.E0.assign((size_t)np * np, 0.0);
  for (int64_t i = 0; i < M.nr; ++i) {
    const int a = P.part[i];
    for (int64_t q = M.ptr[i]; q < M.ptr[i + 1]; ++q) {
      double& e = P.E0[(size_t)a * np + P.part[M.col[q]]];
      e = e + M.val[q];
    }
  }
  return dense_lu(np, P.E0, P.E0piv) ? 6 : 0;
}

// y[a] = sum of v over the nodes of part a (Z^T v), nodes ascending
void coarse_restrict(const ORAS& P, const double* v, std::vector<double>& y) {
  y.assign(P.np, 0.0);
  for (int64_t i = 0; i < P.n; ++i) y[P.part[i]] = y[P.part[i]] + v[i];
}

// Schwarz preconditioner, one- or two-level.  The two-level variant adds a
// coarse correction on Z (one constant per disjoint part) multiplicatively
// before the one-level apply:
//     q = Z E0^{-1} Z^T r,   z = q + P_RAS (r - M q),
// i.e. P2 = Q + P_RAS (I - M Q) with Q = Z E0^{-1} Z^T.  Its transpose is
//     t = P_RAS^T r,   z = t + Z E0^{-T} Z^T (r - M^T t).
void oras_apply(const ORAS& P, const double* r, double* z, int transpose) {
  if (!P.coarse) {
    oras_apply_one_level(P, r, z, transpose);
    return;
  }
  const int64_t n = P.n;
  const CSR& M = *P.M;
  std::vector<double> y, t(n);
  if (!transpose) {
    coarse_restrict(P, r, y);
    dense_lu_solve(P.np, P.E0, P.E0piv, y.data(), 0);
    std::vector<double> q(n);
    for (int64_t i = 0; i < n; ++i) q[i] = y[P.part[i]];
    csr_matvec(M, q.data(), t.data());
    for (int64_t i = 0; i < n; ++i) t[i] = r[i] - t[i];
    oras_apply_one_level(P, t.data(), z, 0);
    for (int64_t i = 0; i < n; ++i) z[i] = z[i] + q[i];
  } else {
    oras_apply_one_level(P, r, t.data(), 1);
    std::vector<double> mt(n, 0.0);  // M^T t, scattered row by row
    for (int64_t i = 0; i < n; ++i)
      for (int64_t q = M.ptr[i]; q < M.ptr[i + 1]; ++q) mt[M.col[q]] = mt[M.col[q]] + M.val[q] * t[i];
    for (int64_t i = 0; i < n; ++i) mt[i] = r[i] - mt[i];
    coarse_restrict(P, mt.data(), y);
    dense_lu_solve(P.np, P.E0, P.E0piv, y.data(), 1);
    for (int64_t i = 0; i < n; ++i) z[i] = t[i] + y[P.part[i]];
  }
}

// ---------------------------------------------------------------------------
// Restarted GMRES(m), right preconditioned (M P y = f, x = P y), classical
// Gram-Schmidt with an optional second pass, Givens least squares.  Stops when
// the true residual |f - M x|_2 <= rtol |f|_2 (checked at the end of every
// cycle; inside a cycle the Givens estimate ends the cycle early).
// ---------------------------------------------------------------------------
double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
  return s;
}

struct Op {
  const CSR* A;
  const ORAS* P;
  int transpose;  // use P^T
};

void op_prec(const Op& o, const double* v, double* z, int64_t n) {
  if (o.P) oras_apply(*o.P, v, z, o.transpose);
  else std::memcpy(z, v, sizeof(double) * n);
}

int gmres(const Op& o, const double* f, double* x, int restart, int maxit, double rtol, int reorth,
          int* iters_out, double* relres_out) {
  const int64_t n = o.A->nr;
  const int m = restart;
  std::vector<double> V((int64_t)(m + 1) * n), H((m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
  std::vector<double> r(n), z(n), w(n), hcol(m + 1);
  double fn = std::sqrt(dot(n, f, f));
  if (fn == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    *iters_out = 0;
    *relres_out = 0.0;
    return 0;
  }
  int it = 0;
  double relres = 0.0;
  int status = 7;  // not converged
  while (true) {
    csr_matvec(*o.A, x, r.data());
    for (int64_t i = 0; i < n; ++i) r[i] = f[i] - r[i];
    double beta = std::sqrt(dot(n, r.data(), r.data()));
    relres = beta / fn;
    if (relres <= rtol) { status = 0; break; }
    if (it >= maxit) break;
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && it < maxit; ++j) {
      op_prec(o, &V[(int64_t)j * n], z.data(), n);
      csr_matvec(*o.A, z.data(), w.data());
      for (int i = 0; i <= j; ++i) hcol[i] = 0.0;
      for (int pass = 0; pass < (reorth ? 2 : 1); ++pass) {
        std::vector<double> hp(j + 1);
        for (int i = 0; i <= j; ++i) hp[i] = dot(n, &V[(int64_t)i * n], w.data());
        for (int i = 0; i <= j; ++i) {
          const double* vi = &V[(int64_t)i * n];
          for (int64_t t = 0; t < n; ++t) w[t] = w[t] - hp[i] * vi[t];
          hcol[i] = hcol[i] + hp[i];
        }
      }
      double hn = std::sqrt(dot(n, w.data(), w.data()));
      hcol[j + 1] = hn;
      it++;
      k = j + 1;
      // previous rotations
      for (int i = 0; i < j; ++i) {
        double t0 = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        double t1 = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = t0;
        hcol[i + 1] = t1;
      }
      double den = std::sqrt(hcol[j] * hcol[j] + hcol[j + 1] * hcol[j + 1]);
      if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
      else { cs[j] = hcol[j] / den; sn[j] = hcol[j + 1] / den; }
      hcol[j] = den;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[i * m + j] = hcol[i];
      if (hn == 0.0 || std::fabs(g[j + 1]) <= rtol * fn) break;  // happy breakdown / estimate met
      double inv = 1.0 / hn;
      double* vn = &V[(int64_t)(j + 1) * n];
      for (int64_t t = 0; t < n; ++t) vn[t] = w[t] * inv;
    }
    // y = H^{-1} g (upper triangular k x k), x += P (V y)
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < k; ++t) s = s - H[i * m + t] * y[t];
      y[i] = s / H[i * m + i];
    }
    for (int64_t t = 0; t < n; ++t) w[t] = 0.0;
    for (int i = 0; i < k; ++i) {
      const double* vi = &V[(int64_t)i * n];
      for (int64_t t = 0; t < n; ++t) w[t] = w[t] + y[i] * vi[t];
    }
    op_prec(o, w.data(), z.data(), n);
    for (int64_t t = 0; t < n; ++t) x[t] = x[t] + z[t];
  }
  *iters_out = it;
  *relres_out = relres;
  return status;
}

thread_local char g_err[256] = "";

}  // namespace

// ===========================================================================
// extern "C" interface (ctypes)
// ===========================================================================
extern "C" {

const char* orc_last_error() { return g_err; }

int orc_cp_dist(int kind, const double* prm, const double* x, double* cp, double* dist) {
  Surf S;
  if (!make_surf(kind, prm, &S)) return ST_ARG;
  *dist = surf_dist(S, x);
  return surf_cp(S, x, cp) ? ST_OK : ST_BAND;
}

double orc_band_lambda(double h, int p) { return band_lambda(h, p); }

double orc_reach(int kind, const double* prm) {
  Surf S;
  if (!make_surf(kind, prm, &S)) return -1.0;
  return surf_reach(S);
}

void orc_weights1d(int p, double s, double* out) { weights1d(p, s, out); }

void* orc_band_build(int kind, const double* prm, double h, int p, int* status) {
  Band* B = new Band();
  if (!make_surf(kind, prm, &B->S) || !(h > 0.0) || p < 1 || p > 5) {
    *status = ST_ARG;
    delete B;
    return nullptr;
  }
  B->h = h;
  B->p = p;
  *status = band_build(*B);
  if (*status != ST_OK) {
    delete B;
    return nullptr;
  }
  return B;
}

void orc_band_free(void* b) { delete (Band*)b; }

void orc_band_counts(const void* b, int64_t* nT, int64_t* nA, int64_t* nG) {
  const Band* B = (const Band*)b;
  *nT = B->nT;
  *nA = B->nA;
  *nG = B->nG;
}

void orc_band_export(const void* b, int32_t* ijkA, int32_t* ijkG, int32_t* base, double* cp) {
  const Band* B = (const Band*)b;
  if (ijkA) std::memcpy(ijkA, B->ijkA.data(), sizeof(int32_t) * B->ijkA.size());
  if (ijkG) std::memcpy(ijkG, B->ijkG.data(), sizeof(int32_t) * B->ijkG.size());
  if (base) std::memcpy(base, B->base.data(), sizeof(int32_t) * B->base.size());
  if (cp) std::memcpy(cp, B->cp.data(), sizeof(double) * B->cp.size());
}

int64_t orc_band_active_index(const void* b, int i, int j, int k) { return ((const Band*)b)->active(i, j, k); }
int64_t orc_band_row_index(const void* b, int i, int j, int k) { return ((const Band*)b)->row(i, j, k); }

void orc_erow_weights(const void* b, int64_t r, double* W) { erow_weights(*(const Band*)b, r, W); }

void* orc_E(const void* b) { return new CSR(build_E(*(const Band*)b)); }
void* orc_M(const void* b, double c) { return new CSR(build_M(*(const Band*)b, c)); }
void* orc_transpose(const void* a) { return new CSR(csr_transpose(*(const CSR*)a)); }
void orc_csr_free(void* a) { delete (CSR*)a; }

void orc_csr_info(const void* a, int64_t* nr, int64_t* nc, int64_t* nnz) {
  const CSR* A = (const CSR*)a;
  *nr = A->nr;
  *nc = A->nc;
  *nnz = (int64_t)A->col.size();
}

void orc_csr_export(const void* a, int64_t* ptr, int32_t* col, double* val) {
  const CSR* A = (const CSR*)a;
  std::memcpy(ptr, A->ptr.data(), sizeof(int64_t) * A->ptr.size());
  std::memcpy(col, A->col.data(), sizeof(int32_t) * A->col.size());
  std::memcpy(val, A->val.data(), sizeof(double) * A->val.size());
}

void orc_csr_matvec(const void* a, const double* x, double* y) { csr_matvec(*(const CSR*)a, x, y); }

// Sampled rows of M x, assembled one row at a time (for bands too large to
// assemble whole).
void orc_apply_rows(const void* b, double c, const double* x, int64_t nrows, const int64_t* rows, double* out) {
  const Band* B = (const Band*)b;
  std::vector<int32_t> cols;
  std::vector<double> vals;
  for (int64_t q = 0; q < nrows; ++q) {
    assemble_row(*B, c, rows[q], cols, vals);
    double s = 0.0;
    for (size_t t = 0; t < cols.size(); ++t) s = s + vals[t] * x[cols[t]];
    out[q] = s;
  }
}

// Sampled entries of M^T x: (M^T x)_m = sum_i M_im x_i over all rows i whose
// pattern holds m (searched in a lattice window around m), ascending i.
void orc_apply_T_cols(const void* b, double c, const double* x, int64_t ncols, const int64_t* cols_in, double* out) {
  const Band* B = (const Band*)b;
  std::vector<int32_t> cols;
  std::vector<double> vals;
  const int rad = B->p + 6;
  for (int64_t q = 0; q < ncols; ++q) {
    int64_t m = cols_in[q];
    const int32_t* xm = &B->ijkA[3 * m];
    std::vector<int64_t> rows;
    for (int a = -rad; a <= rad; ++a)
      for (int bb = -rad; bb <= rad; ++bb)
        for (int cc = -rad; cc <= rad; ++cc) {
          int64_t i = B->active(xm[0] + a, xm[1] + bb, xm[2] + cc);
          if (i >= 0) rows.push_back(i);
        }
    std::sort(rows.begin(), rows.end());
    double s = 0.0;
    for (int64_t i : rows) {
      assemble_row(*B, c, i, cols, vals);
      for (size_t t = 0; t < cols.size(); ++t)
        if (cols[t] == (int32_t)m) s = s + vals[t] * x[i];
    }
    out[q] = s;
  }
}

// Dense LU solve (partial pivoting) of a row-major n x n system.
int orc_dense_solve(int64_t n, const double* A, const double* rhs, double* x, int transpose) {
  std::vector<double> LU(A, A + n * n);
  std::vector<int32_t> piv;
  if (dense_lu(n, LU, piv)) return 2;
  std::memcpy(x, rhs, sizeof(double) * n);
  dense_lu_solve(n, LU, piv, x, transpose);
  return 0;
}

void* orc_oras_setup(const void* b, const void* m, int nparts, int overlap, int robin, double alpha,
                     double alpha_cross, int exact, int order, int coarse, int* status) {
  const Band* B = (const Band*)b;
  ORAS* P = new ORAS();
  P->np = nparts;
  P->overlap = overlap;
  P->robin = robin;
  P->alpha = alpha;
  P->alpha_x = alpha_cross;
  P->exact = exact;
  P->order = order;
  P->h = B->h;
  if (nparts < 1 || overlap < 0) {
    *status = ST_ARG;
    delete P;
    return nullptr;
  }
  *status = oras_setup(*B, *(const CSR*)m, *P);
  if (!*status && coarse) {
    P->coarse = 1;
    *status = coarse_setup(*P, *(const CSR*)m);
  }
  if (*status) {
    delete P;
    return nullptr;
  }
  return P;
}

// Coarse matrix E0 = Z^T M Z of a two-level preconditioner (np x np, row-major),
// before factorisation (assembled again).
void orc_oras_coarse_matrix(const void* p, double* out) {
  const ORAS* P = (const ORAS*)p;
  const CSR& M = *P->M;
  std::memset(out, 0, sizeof(double) * (size_t)P->np * P->np);
  for (int64_t i = 0; i < M.nr; ++i)
    for (int64_t q = M.ptr[i]; q < M.ptr[i + 1]; ++q) {
      double& e = out[(size_t)P->part[i] * P->np + P->part[M.col[q]]];
      e = e + M.val[q];
    }
}

void orc_oras_free(void* p) { delete (ORAS*)p; }

void orc_oras_partition(const void* p, int32_t* part) {
  const ORAS* P = (const ORAS*)p;
  std::memcpy(part, P->part.data(), sizeof(int32_t) * P->part.size());
}

int64_t orc_oras_sub_size(const void* p, int j) { return (int64_t)((const ORAS*)p)->sub[j].nodes.size(); }

void orc_oras_sub_nodes(const void* p, int j, int32_t* nodes) {
  const Sub& s = ((const ORAS*)p)->sub[j];
  std::memcpy(nodes, s.nodes.data(), sizeof(int32_t) * s.nodes.size());
}

// Local matrix (or, after ILU(0), its factors packed L\U) of subdomain j.
void* orc_oras_sub_matrix(const void* p, int j) { return new CSR(((const ORAS*)p)->sub[j].A); }

void orc_oras_apply(const void* p, const double* r, double* z, int transpose) {
  oras_apply(*(const ORAS*)p, r, z, transpose);
}

// Local matrix A_j before factorisation (assembled again, for the ILU(0)
// pin LU = A on the pattern).
void* orc_oras_sub_matrix_unfactored(const void* b, const void* m, const void* p, int j) {
  const Band* B = (const Band*)b;
  ORAS Q = *(const ORAS*)p;
  (void)B;
  const CSR& M = *(const CSR*)m;
  const Sub& s = Q.sub[j];
  std::vector<int32_t> loc(Q.n, -1);
  for (size_t q = 0; q < s.nodes.size(); ++q) loc[s.nodes[q]] = (int32_t)q;
  CSR* A = new CSR();
  A->nr = A->nc = (int64_t)s.nodes.size();
  A->ptr.assign(A->nr + 1, 0);
  for (size_t q = 0; q < s.nodes.size(); ++q) {
    int64_t i = s.nodes[q];
    double D = 0.0;
    bool dropped = false;
    std::vector<int32_t> owners;
    int64_t dpos = -1;
    for (int64_t t = M.ptr[i]; t < M.ptr[i + 1]; ++t) {
      int32_t mm = M.col[t];
      if (loc[mm] >= 0) {
        if (mm == i) dpos = (int64_t)A->col.size();
        A->col.push_back(loc[mm]);
        A->val.push_back(M.val[t]);
      } else {
        dropped = true;
        D = D + M.val[t];
        if (std::find(owners.begin(), owners.end(), Q.part[mm]) == owners.end()) owners.push_back(Q.part[mm]);
      }
    }
    if (Q.robin && dropped && dpos >= 0) {
      double al = owners.size() >= 2 ? Q.alpha_x : Q.alpha;
      double beta = 1.0 / (1.0 + al * Q.h);
      A->val[dpos] = A->val[dpos] + beta * D;
    }
    A->ptr[q + 1] = (int64_t)A->col.size();
  }
  return A;
}

// GMRES on M (transpose = 0, preconditioner P) or on M^T (pass the transposed
// matrix and transpose = 1, preconditioner P^T).  p may be null (no PC).
int orc_gmres(const void* a, const void* p, int transpose, const double* f, double* x, int restart, int maxit,
              double rtol, int reorth, int* iters, double* relres) {
  Op o{(const CSR*)a, (const ORAS*)p, transpose};
  return gmres(o, f, x, restart, maxit, rtol, reorth, iters, relres);
}

// dependency depth (number of levels) of the lower (lower = 1) or upper
// triangle of subdomain j's local matrix in its local order
int orc_oras_depth(const void* p, int j, int lower) {
  const CSR& A = ((const ORAS*)p)->sub[j].A;
  const int64_t n = A.nr;
  std::vector<int> lev(n, 0);
  int mx = 0;
  for (int64_t t = 0; t < n; ++t) {
    const int64_t i = lower ? t : n - 1 - t;
    int l = 0;
    for (int64_t q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      const int64_t c = A.col[q];
      if (lower ? c < i : c > i) l = std::max(l, lev[c]);
    }
    lev[i] = l + 1;
    mx = std::max(mx, l + 1);
  }
  return mx;
}
}  // extern "C"
