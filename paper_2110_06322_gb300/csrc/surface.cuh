// surface.cuh -- device closest point function, distance and 1-D
// barycentric weights (Section 2.1), every FP64 operation written with an
// explicit round-to-nearest intrinsic in a fixed order (no contraction).
#pragma once

#include "common.cuh"

namespace cpm {
namespace {

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsb(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddv(double a, double b) { return __ddiv_rn(a, b); }

struct SurfDev {
  int kind;
  double c[3];
  double a, b;
};

// unsigned distance to the surface (defined everywhere)
__device__ double surf_dist(const SurfDev& S, double x0, double x1, double x2) {
  double dx = dsb(x0, S.c[0]), dy = dsb(x1, S.c[1]), dz = dsb(x2, S.c[2]);
  if (S.kind == 0) {
    double n = __dsqrt_rn(da(da(dm(dx, dx), dm(dy, dy)), dm(dz, dz)));
    return fabs(dsb(n, S.a));
  }
  double rxy = __dsqrt_rn(da(dm(dx, dx), dm(dy, dy)));
  double w = dsb(rxy, S.a);
  double n = __dsqrt_rn(da(dm(w, w), dm(dz, dz)));
  return fabs(dsb(n, S.b));
}

// closest point (eq. cpFunc): sphere -- radial projection; torus -- nearest
// point of the core circle, then r along the direction to x
__device__ bool surf_cp(const SurfDev& S, double x0, double x1, double x2, double cp[3]) {
  double dx = dsb(x0, S.c[0]), dy = dsb(x1, S.c[1]), dz = dsb(x2, S.c[2]);
  if (S.kind == 0) {
    double n = __dsqrt_rn(da(da(dm(dx, dx), dm(dy, dy)), dm(dz, dz)));
    if (!(n > 0.0)) return false;
    double q = ddv(S.a, n);
    cp[0] = da(S.c[0], dm(q, dx));
    cp[1] = da(S.c[1], dm(q, dy));
    cp[2] = da(S.c[2], dm(q, dz));
    return true;
  }
  double rxy = __dsqrt_rn(da(dm(dx, dx), dm(dy, dy)));
  if (!(rxy > 0.0)) return false;
  double t = ddv(S.a, rxy);
  double qx = dm(t, dx), qy = dm(t, dy);
  double ex = dsb(dx, qx), ey = dsb(dy, qy), ez = dz;
  double ne = __dsqrt_rn(da(da(dm(ex, ex), dm(ey, ey)), dm(ez, ez)));
  if (!(ne > 0.0)) return false;
  double u = ddv(S.b, ne);
  cp[0] = da(S.c[0], da(qx, dm(u, ex)));
  cp[1] = da(S.c[1], da(qy, dm(u, ey)));
  cp[2] = da(S.c[2], dm(u, ez));
  return true;
}

// cube base b = floor(cp/h - (p-1)/2) and offset s = cp/h - b
__device__ __forceinline__ void cube_base(double cpa, double h, int p, int* b, double* s) {
  double u = ddv(cpa, h);
  double f = floor(dsb(u, 0.5 * (double)(p - 1)));
  *b = (int)f;
  *s = dsb(u, f);
}

// barycentric weights of equispaced nodes: (-1)^j binom(p, j)
__device__ __forceinline__ double bary_w(int p, int j) {
  double b = 1.0;
  for (int q = 1; q <= j; ++q) b = ddv(dm(b, (double)(p - q + 1)), (double)q);
  return (j & 1) ? -b : b;
}

// 1-D weights, second (true) barycentric form; an exact node hit gives e_j
__device__ void weights1d(int p, double s, double* out) {
  for (int j = 0; j <= p; ++j)
    if (s == (double)j) {
      for (int q = 0; q <= p; ++q) out[q] = (q == j) ? 1.0 : 0.0;
      return;
    }
  double t[4];
  double den = 0.0;
  for (int j = 0; j <= p; ++j) {
    t[j] = ddv(bary_w(p, j), dsb(s, (double)j));
    den = da(den, t[j]);
  }
  for (int j = 0; j <= p; ++j) out[j] = ddv(t[j], den);
}


}  // namespace
}  // namespace cpm
