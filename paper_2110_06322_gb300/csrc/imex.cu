// imex.cu -- the explicit part of one semi-implicit Euler (IMEX) step of the
// Schnakenberg reaction-diffusion system on the band (Section 4.1.6, eq. schnack):
//
//   u_t = D_u Delta_S u + f(u, v),   f = delta1 - u + u^2 v + lambda v
//   v_t = D_v Delta_S v + g(u, v),   g = delta2 - u^2 v - lambda v
//
// Diffusion is implicit and the reaction explicit, so one step solves
//   (c_u I - Delta_S^h) u' = c_u (u + dt f(u, v)),   c_u = 1 / (D_u dt)
// and the same for v with c_v = 1 / (D_v dt): the shifted Poisson problem of
// Section 1 with one right-hand side per species.  This file forms those
// right-hand sides and, for the adjoint (reverse) sweep, the transposed
// Jacobian products and the per-step contributions to dL/dc (accumulated).
//
// Reverse step.  With lam_u = M_u^{-T} du' (the adjoint solve of the step),
//   dL/du += c_u lam_u (1 + dt f_u) + c_v lam_v dt g_u
//   dL/dv += c_u lam_u dt f_v       + c_v lam_v (1 + dt g_v)
//   dL/dc_u += <lam_u, u + dt f - u'>   (b_u = c_u (u + dt f), u' = M_u^{-1} b_u)
// with f_u = -1 + 2uv, f_v = u^2 + lambda, g_u = -2uv, g_v = -u^2 - lambda.
#include "kernels.cuh"

namespace cpm {

namespace {

constexpr int IMX_THREADS = 256;
constexpr int IMX_BLOCKS = 152 * 4;  // fixed grid: the dL/dc sums are reproducible

struct Rx {
  double d1, d2, lam, dt, cu, cv;
  int model;  // 0 Schnakenberg reaction, 1 none (heat equation)
};

__device__ __forceinline__ double rx_f(const Rx& R, double u, double v) {
  return R.model ? 0.0 : R.d1 - u + u * u * v + R.lam * v;
}
__device__ __forceinline__ double rx_g(const Rx& R, double u, double v) {
  return R.model ? 0.0 : R.d2 - u * u * v - R.lam * v;
}

// ARS(2,2,2) coefficients (gamma = 1 - 1/sqrt(2), delta = 1 - 1/(2 gamma))
constexpr double ARS_G = 0.29289321881345247560;
constexpr double ARS_D = -0.70710678118654752440;

__global__ void __launch_bounds__(IMX_THREADS)
    k_imex_rhs(Rx R, int64_t n, const double* __restrict__ u, const double* __restrict__ v, double* bu, double* bv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ui = u[i], vi = v[i];
    bu[i] = R.cu * (ui + R.dt * rx_f(R, ui, vi));
    bv[i] = R.cv * (vi + R.dt * rx_g(R, ui, vi));
  }
}

// stage right-hand sides of one ARS(2,2,2) step (R.cu, R.cv: 1 / (gamma D dt))
__global__ void __launch_bounds__(IMX_THREADS)
    k_imex2_rhs(Rx R, int stage, int64_t n, const double* __restrict__ u, const double* __restrict__ v,
                const double* __restrict__ u2, const double* __restrict__ v2, double* bu, double* bv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ui = u[i], vi = v[i];
    const double f1 = rx_f(R, ui, vi), g1 = rx_g(R, ui, vi);
    if (stage == 2) {
      bu[i] = R.cu * (ui + ARS_G * R.dt * f1);
      bv[i] = R.cv * (vi + ARS_G * R.dt * g1);
    } else {
      const double a = u2[i], b = v2[i];
      const double f2 = rx_f(R, a, b), g2 = rx_g(R, a, b);
      const double gu2 = (a - ui - ARS_G * R.dt * f1) / ARS_G;  // dt D_u Delta u2
      const double gv2 = (b - vi - ARS_G * R.dt * g1) / ARS_G;
      bu[i] = R.cu * (ui + R.dt * (ARS_D * f1 + (1.0 - ARS_D) * f2) + (1.0 - ARS_G) * gu2);
      bv[i] = R.cv * (vi + R.dt * (ARS_D * g1 + (1.0 - ARS_D) * g2) + (1.0 - ARS_G) * gv2);
    }
  }
}

__device__ __forceinline__ double blk_sum(double x, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int q = 0; q < IMX_THREADS / 32; ++q) t += sh[q];
  return t;
}

__global__ void __launch_bounds__(IMX_THREADS)
    k_imex_adj(Rx R, int64_t n, const double* __restrict__ u, const double* __restrict__ v,
               const double* __restrict__ u1, const double* __restrict__ v1, const double* __restrict__ lu,
               const double* __restrict__ lv, double* ubar, double* vbar, double* partial) {
  __shared__ double sh[IMX_THREADS / 32];
  double su = 0, sv = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ui = u[i], vi = v[i], a = lu[i], b = lv[i];
    const double uv = ui * vi, uu = ui * ui;
    const double fu = R.model ? 0.0 : -1.0 + 2.0 * uv, fv = R.model ? 0.0 : uu + R.lam;
    const double gu = R.model ? 0.0 : -2.0 * uv, gv = R.model ? 0.0 : -uu - R.lam;
    ubar[i] = R.cu * a * (1.0 + R.dt * fu) + R.cv * b * (R.dt * gu);
    vbar[i] = R.cu * a * (R.dt * fv) + R.cv * b * (1.0 + R.dt * gv);
    su += a * (ui + R.dt * rx_f(R, ui, vi) - u1[i]);
    sv += b * (vi + R.dt * rx_g(R, ui, vi) - v1[i]);
  }
  su = blk_sum(su, sh);
  sv = blk_sum(sv, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = su;
    partial[gridDim.x + blockIdx.x] = sv;
  }
}

// out[t] (+)= sum over b of partial[t * nb + b], in a fixed order; block t
// reduces value t
__global__ void __launch_bounds__(IMX_THREADS)
    k_imex_reduce(const double* __restrict__ partial, int nb, double* out, int accumulate) {
  __shared__ double sh[IMX_THREADS / 32];
  double x = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) x += partial[blockIdx.x * nb + b];
  x = blk_sum(x, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = accumulate ? out[blockIdx.x] + x : x;
}

__global__ void __launch_bounds__(IMX_THREADS)
    k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* partial) {
  __shared__ double sh[IMX_THREADS / 32];
  double x = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x += a[i] * b[i];
  x = blk_sum(x, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = x;
}

Rx make_rx(const cpm_schnakenberg* p) {
  Rx R;
  R.d1 = p->delta1;
  R.d2 = p->delta2;
  R.lam = p->lambda;
  R.dt = p->dt;
  R.cu = 1.0 / (p->Du * p->dt);
  R.cv = 1.0 / (p->Dv * p->dt);
  R.model = p->model;
  return R;
}

}  // namespace

cpm_status imex_rhs(const cpm_schnakenberg* prm, int64_t n, const double* u, const double* v, double* bu, double* bv,
                    cudaStream_t s) {
  KL(k_imex_rhs<<<grid_for(n, IMX_THREADS), IMX_THREADS, 0, s>>>(make_rx(prm), n, u, v, bu, bv));
  CPM_CUDA(cudaGetLastError());
  return CPM_OK;
}

cpm_status imex2_rhs(const cpm_schnakenberg* prm, int stage, int64_t n, const double* u, const double* v,
                     const double* u2, const double* v2, double* bu, double* bv, cudaStream_t s) {
  Rx R = make_rx(prm);
  R.cu = 1.0 / (ARS_G * prm->Du * prm->dt);
  R.cv = 1.0 / (ARS_G * prm->Dv * prm->dt);
  KL(k_imex2_rhs<<<grid_for(n, IMX_THREADS), IMX_THREADS, 0, s>>>(R, stage, n, u, v, u2, v2, bu, bv));
  CPM_CUDA(cudaGetLastError());
  return CPM_OK;
}

cpm_status imex_rhs_adjoint(const cpm_schnakenberg* prm, int64_t n, const double* u, const double* v,
                            const double* u1, const double* v1, const double* lu, const double* lv, double* ubar,
                            double* vbar, double* dc, cudaStream_t s) {
  double* partial = nullptr;
  CPM_TRY(dalloc(&partial, 2 * IMX_BLOCKS, s));
  KL(k_imex_adj<<<IMX_BLOCKS, IMX_THREADS, 0, s>>>(make_rx(prm), n, u, v, u1, v1, lu, lv, ubar, vbar, partial));
  KL(k_imex_reduce<<<2, IMX_THREADS, 0, s>>>(partial, IMX_BLOCKS, dc, 1));
  cudaError_t e = cudaGetLastError();
  dfree(partial, s);
  if (e != cudaSuccess) return cuda_fail(e, "IMEX adjoint kernels", __FILE__, __LINE__);
  return CPM_OK;
}

cpm_status dot(int64_t n, const double* a, const double* b, double* out, cudaStream_t s) {
  double* partial = nullptr;
  CPM_TRY(dalloc(&partial, IMX_BLOCKS, s));
  KL(k_dot2<<<IMX_BLOCKS, IMX_THREADS, 0, s>>>(n, a, b, partial));
  KL(k_imex_reduce<<<1, IMX_THREADS, 0, s>>>(partial, IMX_BLOCKS, out, 0));
  cudaError_t e = cudaGetLastError();
  dfree(partial, s);
  if (e != cudaSuccess) return cuda_fail(e, "dot kernels", __FILE__, __LINE__);
  return CPM_OK;
}

}  // namespace cpm
