// solve.cu -- restarted GMRES(m), right preconditioned by the Schwarz
// preconditioner (Section 4.1.1: GMRES is the default Krylov method), and
// FP64 iterative refinement around an FP32-operator inner GMRES.
//
// One iteration j:  z = P v_j;  w = M z;  classical Gram-Schmidt against
// v_0..v_j (optionally a second pass);  h_{j+1,j} = |w|;  v_{j+1} = w / |w|;
// Givens rotations update the least-squares problem on the device (one
// thread, FP64) and publish the residual estimate |g_{j+1}|.  At the end of a
// cycle x += P (V y) and the true residual |f - M x| (FP64) decides.
//
// All reductions are two-stage with a fixed grid and a fixed summation order,
// so a solve is bitwise reproducible on the same device.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "oras.cuh"
#include "reduce.cuh"

namespace cpm {

namespace {

constexpr int RED_BLOCKS = 152 * 8;

// partial[b] = block b's share of <a, b>
__global__ void __launch_bounds__(RED_THREADS)
    k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* partial) {
  __shared__ double sh[RED_THREADS / 32];
  double acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Gram-Schmidt pass kernels over nv <= NV basis vectors V_t = V + t ld.
//   MODE 0: dots     partial <- <V_t, w>
//   MODE 1: update   w -= sum_t coef[t] V_t
//   MODE 2: update, then dots of the V_t with the updated w (the second
//           classical pass's projection fused with the first one's
//           subtraction: each V_t is read once for both)
//   MODE 3: update, then partial <- |w|^2
template <int NV, int MODE>
__global__ void __launch_bounds__(RED_THREADS)
    k_gs(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ coef, double* w, int64_t n,
         double* partial) {
  __shared__ double cf[NV];
  if (MODE != 0) {
    if (threadIdx.x < NV) cf[threadIdx.x] = threadIdx.x < nv ? coef[threadIdx.x] : 0.0;
    __syncthreads();
  }
  constexpr int NA = MODE == 3 ? 1 : NV;
  double acc[NA];
#pragma unroll
  for (int t = 0; t < NA; ++t) acc[t] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = t < nv ? V[t * ld + i] : 0.0;
    double wi = w[i];
    if (MODE != 0) {
#pragma unroll
      for (int t = 0; t < NV; ++t)
        if (t < nv) wi -= cf[t] * v[t];
      w[i] = wi;
    }
    if (MODE == 0 || MODE == 2) {
#pragma unroll
      for (int t = 0; t < NA; ++t)
        if (t < nv) acc[t] += v[t] * wi;
    }
    if (MODE == 3) acc[0] += wi * wi;
  }
  if constexpr (MODE == 0 || MODE == 2) block_partials<NA>(acc, nv, partial);
  if constexpr (MODE == 3) block_partials<1>(acc, 1, partial);
}

// Blocks of one Gram-Schmidt pass kernel: the SM count times the blocks that
// fit on one SM, fixed per device so that the summation order (and thus the
// result) does not change between calls.
template <int NV, int MODE>
int gs_blocks() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gs<NV, MODE>, RED_THREADS, 0);
    int b = sms * (per > 0 ? per : 1);
    cache[dev] = b < 1 ? 1 : (b > RED_BLOCKS ? RED_BLOCKS : b);
  }
  return cache[dev];
}

// Launch k_gs for nv <= 16 vectors with the smaller of 8, 16 that holds them;
// returns the grid used (the number of partial sums per value).
template <int MODE>
int launch_gs(const double* V, int64_t ld, int nv, const double* coef, double* w, int64_t n, double* partial,
              cudaStream_t s) {
  int g = 0;
  if (nv <= 8) {
    g = gs_blocks<8, MODE>();
    KL(k_gs<8, MODE><<<g, RED_THREADS, 0, s>>>(V, ld, nv, coef, w, n, partial));
  } else {
    g = gs_blocks<16, MODE>();
    KL(k_gs<16, MODE><<<g, RED_THREADS, 0, s>>>(V, ld, nv, coef, w, n, partial));
  }
  return g;
}

// out[t] (+)= sum_b partial[t * nb + b] in a fixed order; block t reduces value t
__global__ void k_reduce(const double* __restrict__ partial, int nvals, int nb, double* out, int accumulate) {
  __shared__ double sh[RED_THREADS / 32];
  const int t = blockIdx.x;
  double v = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partial[t * nb + b];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) out[t] = accumulate ? out[t] + s : s;
}

// y[t] = sum_b partial[t * nb + b] in a fixed order; hc[t] = y[t] (acc 0)
// or hc[t] += y[t] (acc 1).  Block t reduces value t.
__global__ void k_reduce_gs(const double* __restrict__ partial, int nb, double* y, double* hc, int acc) {
  __shared__ double sh[RED_THREADS / 32];
  const int t = blockIdx.x;
  double v = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partial[t * nb + b];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) {
    y[t] = s;
    hc[t] = acc ? hc[t] + s : s;
  }
}

// v = w * (*inv)
__global__ void k_scale(const double* __restrict__ w, const double* __restrict__ inv, double* v, int64_t n) {
  const double a = *inv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = w[i] * a;
}

// out[0] = 1 / sqrt(in[0]) (one thread)
__global__ void k_rsqrt1(const double* __restrict__ in, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = 1.0 / sqrt(in[0]);
}

__global__ void k_sub(const double* __restrict__ f, double* r, int64_t n) {  // r = f - r
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = f[i] - r[i];
}

__global__ void k_axpy(const double* __restrict__ z, double* x, int64_t n) {  // x += z
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += z[i];
}

// x += sum_t y[t] Z_t with Z_t = Z + t ld in FP32 (the preconditioned basis
// vectors of a flexible cycle), accumulated in FP64 in a fixed order
__global__ void k_flex_update(const float* __restrict__ Z, int64_t ld, int k, const double* __restrict__ y, double* x,
                              int64_t n) {
  __shared__ double ys[256];
  for (int t = threadIdx.x; t < k; t += blockDim.x) ys[t] = y[t];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0;
    for (int t = 0; t < k; ++t) acc += ys[t] * (double)Z[t * ld + i];
    x[i] += acc;
  }
}

__global__ void k_d2f(const double* __restrict__ a, float* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(const float* __restrict__ a, double* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// Givens update of column j (one thread).  hc[0..j+1] holds the new column
// (its last entry the squared norm of w).  Publishes {|g_{j+1}|, h_{j+1,j}}.
__global__ void k_givens(double* H, int m, const double* __restrict__ hc, double* cs, double* sn, double* g, int j,
                         double* pub) {
  if (threadIdx.x || blockIdx.x) return;
  double col[258];
  for (int i = 0; i <= j; ++i) col[i] = hc[i];
  const double hn = sqrt(hc[j + 1]);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
    const double t1 = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t0;
    col[i + 1] = t1;
  }
  const double den = sqrt(col[j] * col[j] + col[j + 1] * col[j + 1]);
  if (den == 0.0) {
    cs[j] = 1.0;
    sn[j] = 0.0;
  } else {
    cs[j] = col[j] / den;
    sn[j] = col[j + 1] / den;
  }
  col[j] = den;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  for (int i = 0; i <= j; ++i) H[i * m + j] = col[i];
  pub[0] = fabs(g[j + 1]);
  pub[1] = hn;
  pub[2] = hn > 0.0 ? 1.0 / hn : 0.0;  // scale of the next basis vector
}

// y = H(0:k,0:k)^{-1} g (upper triangular), one thread
__global__ void k_trisolve(const double* __restrict__ H, int m, const double* __restrict__ g, int k, double* y) {
  if (threadIdx.x || blockIdx.x) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int t = i + 1; t < k; ++t) s -= H[i * m + t] * y[t];
    y[i] = s / H[i * m + i];
  }
}

__global__ void k_negate(const double* __restrict__ a, double* b, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = -a[i];
}

__global__ void k_init_g(double* g, int m, const double* __restrict__ nrm2) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = 0.0;
  if (threadIdx.x == 0) g[0] = sqrt(*nrm2);
}

struct Work {
  int64_t n = 0;
  int m = 0;
  double *V = nullptr, *w = nullptr, *z = nullptr, *t = nullptr, *r = nullptr;
  float *v32 = nullptr, *z32 = nullptr, *w32 = nullptr;
  float* Z32 = nullptr;  // m x n: preconditioned basis vectors of a flexible (mixed-precision) cycle
  double *H = nullptr, *hc = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *ny = nullptr;
  double *partial = nullptr, *scal = nullptr;  // partial: (32 + 1) x RED_BLOCKS
  double* pub = nullptr;  // pinned host: two slots of {|g_{j+1}|, h_{j+1,j}, 1/h_{j+1,j}} at 0 and 4
  cudaEvent_t ev[2] = {nullptr, nullptr};  // iteration j's slot has landed
  cpm_status alloc(int64_t n_, int m_, bool f32, cudaStream_t s) {
    n = n_;
    m = m_;
    CPM_TRY(dalloc(&V, (size_t)(m + 1) * n, s));
    CPM_TRY(dalloc(&w, n, s));
    CPM_TRY(dalloc(&z, n, s));
    CPM_TRY(dalloc(&t, n, s));
    CPM_TRY(dalloc(&r, n, s));
    if (f32) {
      CPM_TRY(dalloc(&v32, n, s));
      CPM_TRY(dalloc(&z32, n, s));
      CPM_TRY(dalloc(&Z32, (size_t)m * n, s));
      CPM_TRY(dalloc(&w32, n, s));
    }
    CPM_TRY(dalloc(&H, (size_t)(m + 1) * m, s));
    CPM_TRY(dalloc(&hc, m + 2, s));
    CPM_TRY(dalloc(&cs, m, s));
    CPM_TRY(dalloc(&sn, m, s));
    CPM_TRY(dalloc(&g, m + 1, s));
    CPM_TRY(dalloc(&y, m, s));
    CPM_TRY(dalloc(&ny, m, s));
    CPM_TRY(dalloc(&partial, (size_t)(32 + 1) * RED_BLOCKS, s));
    CPM_TRY(dalloc(&scal, 8, s));
    CPM_CUDA(cudaMallocHost((void**)&pub, 8 * sizeof(double)));
    for (int q = 0; q < 2; ++q) CPM_CUDA(cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming));
    return CPM_OK;
  }
  void release(cudaStream_t s) {
    for (double** p : {&V, &w, &z, &t, &r, &H, &hc, &cs, &sn, &g, &y, &ny, &partial, &scal}) dfree(*p, s);
    dfree(v32, s);
    dfree(z32, s);
    dfree(Z32, s);
    dfree(w32, s);
    if (pub) cudaFreeHost(pub);
    pub = nullptr;
    for (int q = 0; q < 2; ++q)
      if (ev[q]) cudaEventDestroy(ev[q]);
    ev[0] = ev[1] = nullptr;
  }
};

struct Timing {
  bool on = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double ms_P = 0, ms_M = 0;
  int nP = 0, nM = 0;
  void start(cudaStream_t s) {
    if (on) cudaEventRecord(e0, s);
  }
  void stop(cudaStream_t s, bool prec) {
    if (!on) return;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (prec) {
      ms_P += ms;
      nP++;
    } else {
      ms_M += ms;
      nM++;
    }
  }
};

struct Ops {
  const cpm_band* B;
  const oras_pc* P;
  double c;
  int transpose;
  int f32;  // operator and preconditioner in FP32
  Timing* tm;
  // flexible cycle (FP32 applies with a preconditioner): z_j = P v_j is kept
  // (in FP32, as computed) and the cycle ends with x += Z y, so the update is
  // made of exactly the vectors the Arnoldi relation M Z = V H was built from
  bool flex() const { return f32 && P; }
};

const int GB = RED_BLOCKS;

// out = M x (FP64 or FP32 operator)
cpm_status op_M(const Ops& o, const double* x, double* out, Work& W, cudaStream_t s) {
  if (!o.f32) {
    o.tm->start(s);
    CPM_TRY(apply_op(o.B, &o.c, x, out, CPM_F64, 1, o.transpose, s));
    o.tm->stop(s, false);
    return CPM_OK;
  }
  KL(k_d2f<<<grid_for(W.n, 256), 256, 0, s>>>(x, W.v32, W.n));
  o.tm->start(s);
  CPM_TRY(apply_op(o.B, &o.c, W.v32, W.w32, CPM_F32, 1, o.transpose, s));
  o.tm->stop(s, false);
  KL(k_f2d<<<grid_for(W.n, 256), 256, 0, s>>>(W.w32, out, W.n));
  return CPM_OK;
}

// out = P v
cpm_status op_P(const Ops& o, const double* v, double* out, Work& W, cudaStream_t s) {
  if (!o.P) {
    CPM_CUDA(cudaMemcpyAsync(out, v, W.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return CPM_OK;
  }
  if (!o.f32) {
    o.tm->start(s);
    CPM_TRY(oras_run(o.P, v, out, CPM_F64, 1, o.transpose, s));
    o.tm->stop(s, true);
    return CPM_OK;
  }
  KL(k_d2f<<<grid_for(W.n, 256), 256, 0, s>>>(v, W.v32, W.n));
  o.tm->start(s);
  CPM_TRY(oras_run(o.P, W.v32, W.z32, CPM_F32, 1, o.transpose, s));
  o.tm->stop(s, true);
  KL(k_f2d<<<grid_for(W.n, 256), 256, 0, s>>>(W.z32, out, W.n));
  return CPM_OK;
}

// w = M P v_j.  In FP32 the preconditioned vector stays FP32 between the two
// applies (its FP64 copy would round back to the same FP32 values) and is
// kept as column j of the flexible basis Z.
cpm_status op_MP(const Ops& o, const double* v, double* w, int j, Work& W, cudaStream_t s) {
  if (!o.flex()) {
    CPM_TRY(op_P(o, v, W.z, W, s));
    return op_M(o, W.z, w, W, s);
  }
  float* zj = W.Z32 + (int64_t)j * W.n;
  KL(k_d2f<<<grid_for(W.n, 256), 256, 0, s>>>(v, W.v32, W.n));
  o.tm->start(s);
  CPM_TRY(oras_run(o.P, W.v32, zj, CPM_F32, 1, o.transpose, s));
  o.tm->stop(s, true);
  o.tm->start(s);
  CPM_TRY(apply_op(o.B, &o.c, zj, W.w32, CPM_F32, 1, o.transpose, s));
  o.tm->stop(s, false);
  KL(k_f2d<<<grid_for(W.n, 256), 256, 0, s>>>(W.w32, w, W.n));
  return CPM_OK;
}

// out[0] = <a, a>
cpm_status norm2(const double* a, int64_t n, double* out, Work& W, cudaStream_t s) {
  KL(k_dot<<<GB, RED_THREADS, 0, s>>>(a, a, n, W.partial));
  KL(k_reduce<<<1, RED_THREADS, 0, s>>>(W.partial, 1, GB, out, 0));
  return CPM_OK;
}

// Classical Gram-Schmidt of w against V_0..V_j; hc[0..j] = coefficients,
// hc[j+1] = |w|^2 after orthogonalisation.  reorth: 0 one pass; 1 a second
// pass when the first one shrank |w| below 1/sqrt(2) of its value (the
// Daniel-Gragg-Kaufman-Stewart criterion); 2 always two passes.
//
// One pass is h = V^T w (kernel MODE 0), then w -= V h (MODE 1 or 3).  With
// two passes the first pass's subtraction and the second pass's projection
// run as one kernel (MODE 2), so V is streamed three times instead of four.
// Bases wider than GS_MAX vectors are processed in chunks of at most GS_MAX
// (balanced: 20 vectors run as 10 + 10): the 16-vector kernels keep enough
// warps per SM to stream V at close to full bandwidth, where a 32-vector
// kernel's register use leaves one block per SM.
constexpr int GS_MAX = 16;
inline int gs_chunk(int nv) {
  const int nch = (nv + GS_MAX - 1) / GS_MAX;
  return (nv + nch - 1) / nch;
}

// dots of w with V_0..V_{nv-1}: y = V^T w and hc = y (acc 0) or hc += y (acc 1)
cpm_status gs_dots(int nv, bool acc, Work& W, cudaStream_t s) {
  const int cs = gs_chunk(nv);
  for (int t0 = 0; t0 < nv; t0 += cs) {
    const int nc = nv - t0 < cs ? nv - t0 : cs;
    const int g = launch_gs<0>(W.V + (int64_t)t0 * W.n, W.n, nc, nullptr, W.w, W.n, W.partial, s);
    KL(k_reduce_gs<<<nc, RED_THREADS, 0, s>>>(W.partial, g, W.y + t0, W.hc + t0, acc ? 1 : 0));
  }
  return CPM_OK;
}

// w -= V y over V_0..V_{nv-1}; hc[nv] = |w|^2 afterwards
cpm_status gs_subtract_norm(int nv, Work& W, cudaStream_t s) {
  int g = 0;
  const int cs = gs_chunk(nv);
  for (int t0 = 0; t0 < nv; t0 += cs) {
    const int nc = nv - t0 < cs ? nv - t0 : cs;
    const double* Vt = W.V + (int64_t)t0 * W.n;
    if (t0 + cs >= nv) g = launch_gs<3>(Vt, W.n, nc, W.y + t0, W.w, W.n, W.partial, s);
    else launch_gs<1>(Vt, W.n, nc, W.y + t0, W.w, W.n, W.partial, s);
  }
  KL(k_reduce<<<1, RED_THREADS, 0, s>>>(W.partial, 1, g, W.hc + nv, 0));
  return CPM_OK;
}

cpm_status gram_schmidt(int j, int reorth, Work& W, cudaStream_t s) {
  const int nv = j + 1;
  if (reorth == 1) {
    CPM_TRY(norm2(W.w, W.n, W.scal + 6, W, s));
    CPM_TRY(gs_dots(nv, false, W, s));
    CPM_TRY(gs_subtract_norm(nv, W, s));
    double nn[2];
    CPM_CUDA(cudaMemcpyAsync(&nn[0], W.scal + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaMemcpyAsync(&nn[1], W.hc + j + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
    if (nn[1] < 0.5 * nn[0]) {
      CPM_TRY(gs_dots(nv, true, W, s));
      CPM_TRY(gs_subtract_norm(nv, W, s));
    }
    return CPM_OK;
  }
  CPM_TRY(gs_dots(nv, false, W, s));
  if (reorth == 2) {
    if (nv <= GS_MAX) {  // fused: w -= V h1 and h2 = V^T w in one sweep
      const int g = launch_gs<2>(W.V, W.n, nv, W.y, W.w, W.n, W.partial, s);
      KL(k_reduce_gs<<<nv, RED_THREADS, 0, s>>>(W.partial, g, W.y, W.hc, 1));
    } else {
      const int cs = gs_chunk(nv);
      for (int t0 = 0; t0 < nv; t0 += cs) {
        const int nc = nv - t0 < cs ? nv - t0 : cs;
        launch_gs<1>(W.V + (int64_t)t0 * W.n, W.n, nc, W.y + t0, W.w, W.n, W.partial, s);
      }
      CPM_TRY(gs_dots(nv, true, W, s));
    }
  }
  CPM_TRY(gs_subtract_norm(nv, W, s));
  CPM_CUDA(cudaGetLastError());
  return CPM_OK;
}

struct GmresOut {
  int iters = 0, cycles = 0;
  double relres = 0;
  cpm_status status = CPM_OK;
};

// one_cycle: x must be zero on entry; run a single cycle from r = f and
// return (the inner solve of iterative refinement).
cpm_status gmres(const Ops& o, const double* f, double* x, int m, int maxit, double rtol, int reorth, Work& W,
                 GmresOut& out, cudaStream_t s, bool one_cycle = false) {
  const int64_t n = W.n;
  const int G = grid_for(n, 256);
  CPM_TRY(norm2(f, n, W.scal, W, s));
  double fn2 = 0;
  CPM_CUDA(cudaMemcpyAsync(&fn2, W.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  const double fn = std::sqrt(fn2);
  if (!std::isfinite(fn)) {
    out.status = CPM_ERR_NAN;
    return fail(CPM_ERR_NAN, "right-hand side holds NaN or Inf");
  }
  if (fn == 0.0) {
    CPM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    out.relres = 0;
    out.status = CPM_OK;
    return CPM_OK;
  }
  bool first = true;
  while (true) {
    if (one_cycle && !first) {
      out.status = CPM_OK;
      return CPM_OK;
    }
    first = false;
    // r = f - M x
    if (one_cycle) {
      CPM_CUDA(cudaMemcpyAsync(W.r, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      CPM_TRY(op_M(o, x, W.r, W, s));
      KL(k_sub<<<G, 256, 0, s>>>(f, W.r, n));
    }
    CPM_TRY(norm2(W.r, n, W.scal + 1, W, s));
    double b2 = 0;
    CPM_CUDA(cudaMemcpyAsync(&b2, W.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
    if (o.P) {  // a Schwarz apply of the last cycle ran out of a bounded wait: its output is not usable
      const cpm_status te = oras_take_error(o.P, s);
      if (te != CPM_OK) {
        out.status = te;
        return te;
      }
    }
    const double beta = std::sqrt(b2);
    out.relres = beta / fn;
    if (!std::isfinite(beta)) {
      out.status = CPM_ERR_NAN;
      return fail(CPM_ERR_NAN, "residual became NaN or Inf");
    }
    if (out.relres <= rtol) {
      out.status = CPM_OK;
      return CPM_OK;
    }
    if (out.iters >= maxit) {
      out.status = CPM_ERR_NOT_CONVERGED;
      return CPM_OK;
    }
    out.cycles++;
    KL(k_rsqrt1<<<1, 32, 0, s>>>(W.scal + 1, W.scal + 5));
    KL(k_scale<<<G, 256, 0, s>>>(W.r, W.scal + 5, W.V, n));
    KL(k_init_g<<<1, 256, 0, s>>>(W.g, m, W.scal + 1));
    // Iteration j's residual estimate is read on the host while iteration j+1
    // already runs (the host waits on j's event after queueing j+1), so the
    // GPU never idles on the convergence test.  When the test stops the cycle
    // at j, the speculative iteration j+1 is discarded: k = j + 1 columns are
    // used, and nothing of column j+1 (its H column, its rotation, g[j+2])
    // enters the least-squares solution.
    int k = 0;
    const int jmax = std::min(m, maxit - out.iters);
    auto check = [&](int j, bool& stop) -> cpm_status {
      CPM_CUDA(cudaEventSynchronize(W.ev[j & 1]));
      const double* pj = W.pub + 4 * (j & 1);
      const double est = pj[0], hn = pj[1];
      k = j + 1;
      if (!std::isfinite(est)) {
        out.status = CPM_ERR_NAN;
        return fail(CPM_ERR_NAN, "Krylov iteration produced NaN or Inf");
      }
      stop = hn == 0.0 || est <= rtol * fn;
      return CPM_OK;
    };
    bool stop = false;
    for (int j = 0; j < jmax && !stop; ++j) {
      double* vj = W.V + (int64_t)j * n;
      CPM_TRY(op_MP(o, vj, W.w, j, W, s));
      CPM_TRY(gram_schmidt(j, reorth, W, s));
      KL(k_givens<<<1, 1, 0, s>>>(W.H, m, W.hc, W.cs, W.sn, W.g, j, W.scal + 2));
      CPM_CUDA(cudaMemcpyAsync(W.pub + 4 * (j & 1), W.scal + 2, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CPM_CUDA(cudaEventRecord(W.ev[j & 1], s));
      if (j + 1 < m) KL(k_scale<<<G, 256, 0, s>>>(W.w, W.scal + 4, W.V + (int64_t)(j + 1) * n, n));
      CPM_CUDA(cudaGetLastError());
      if (j > 0) CPM_TRY(check(j - 1, stop));
    }
    if (!stop && jmax > 0) CPM_TRY(check(jmax - 1, stop));
    out.iters += k;
    KL(k_trisolve<<<1, 1, 0, s>>>(W.H, m, W.g, k, W.y));
    if (o.flex()) {  // x += Z y
      KL(k_flex_update<<<G, 256, 0, s>>>(W.Z32, n, k, W.y, x, n));
      CPM_CUDA(cudaGetLastError());
      continue;
    }
    // x += P (V y)
    CPM_CUDA(cudaMemsetAsync(W.t, 0, n * sizeof(double), s));
    KL(k_negate<<<1, 256, 0, s>>>(W.y, W.ny, k));
    const int cs = gs_chunk(k);
    for (int t0 = 0; t0 < k; t0 += cs) {
      const int nc = k - t0 < cs ? k - t0 : cs;
      launch_gs<1>(W.V + (int64_t)t0 * n, n, nc, W.ny + t0, W.t, n, nullptr, s);
    }
    CPM_TRY(op_P(o, W.t, W.z, W, s));
    KL(k_axpy<<<G, 256, 0, s>>>(W.z, x, n));
    CPM_CUDA(cudaGetLastError());
  }
}

}  // namespace

cpm_status solve_run(const cpm_band* B, const oras_pc* P, double c, const double* f, double* u,
                     const cpm_solve_params* prm, cpm_solve_info* info, int transpose, cudaStream_t s) {
  *info = cpm_solve_info{};
  const int64_t n = B->nA;
  if (prm->mixed && P && P->store == CPM_F64)
    return fail(CPM_ERR_ARG, "mixed precision needs FP32 or BF16 factors (oras_params.store)");
  Work W;
  cpm_status st = W.alloc(n, prm->restart, prm->mixed != 0, s);
  if (st != CPM_OK) {
    W.release(s);
    return st;
  }
  Timing tm;
  tm.on = prm->timing != 0;
  if (tm.on) {
    cudaEventCreate(&tm.e0);
    cudaEventCreate(&tm.e1);
  }
  Ops o64{B, P, c, transpose, 0, &tm};
  GmresOut out;
  if (!prm->mixed) {
    st = gmres(o64, f, u, prm->restart, prm->maxit, prm->rtol, prm->reorth, W, out, s);
  } else {
    // FP64 iterative refinement: r = f - M u (FP64); one GMRES(m) cycle on
    // M d = r with the FP32 operator and preconditioner (FP64 basis and least
    // squares); u += d.  Every restart residual is thus an FP64 residual.
    Ops o32{B, P, c, transpose, 1, &tm};
    double *r = nullptr, *d = nullptr;
    st = dalloc(&r, n, s);
    if (st == CPM_OK) st = dalloc(&d, n, s);
    double fn2 = 0;
    if (st == CPM_OK) st = norm2(f, n, W.scal + 4, W, s);
    if (st == CPM_OK) {
      cudaMemcpyAsync(&fn2, W.scal + 4, sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
    }
    const double fn = std::sqrt(fn2);
    const double inner = prm->inner_rtol > 0 ? prm->inner_rtol : 1e-4;
    while (st == CPM_OK) {
      st = op_M(o64, u, r, W, s);
      if (st != CPM_OK) break;
      KL(k_sub<<<grid_for(n, 256), 256, 0, s>>>(f, r, n));
      st = norm2(r, n, W.scal + 5, W, s);
      double r2 = 0;
      cudaMemcpyAsync(&r2, W.scal + 5, sizeof(double), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      out.relres = fn > 0 ? std::sqrt(r2) / fn : 0.0;
      if (P) {
        st = oras_take_error(P, s);
        if (st != CPM_OK) {
          out.status = st;
          break;
        }
      }
      if (!std::isfinite(out.relres)) {
        st = fail(CPM_ERR_NAN, "residual became NaN or Inf");
        out.status = CPM_ERR_NAN;
        break;
      }
      if (out.relres <= prm->rtol) {
        out.status = CPM_OK;
        break;
      }
      if (out.iters >= prm->maxit) {
        out.status = CPM_ERR_NOT_CONVERGED;
        break;
      }
      cudaMemsetAsync(d, 0, n * sizeof(double), s);
      GmresOut in;
      // the inner cycle may stop once its estimate is well below what the
      // outer tolerance still asks for (half of it: FP32 applies make the
      // estimate and the FP64 residual differ slightly)
      const double rn = std::sqrt(r2);
      const double tol_in = std::max(inner, rn > 0 ? 0.5 * prm->rtol * fn / rn : inner);
      st = gmres(o32, r, d, prm->restart, prm->maxit - out.iters, tol_in, prm->reorth, W, in, s, true);
      out.iters += in.iters;
      out.cycles += in.cycles;
      info->ir_steps++;
      if (st != CPM_OK) break;
      KL(k_axpy<<<grid_for(n, 256), 256, 0, s>>>(d, u, n));
    }
    dfree(r, s);
    dfree(d, s);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (P && e == cudaSuccess) {
    // a timed-out apply makes every later result meaningless: it takes
    // precedence over whatever the iteration concluded from it
    const cpm_status te = oras_take_error(P, s);
    if (te != CPM_OK) st = te;
  }
  W.release(s);
  cudaStreamSynchronize(s);
  info->iters = out.iters;
  info->restarts = out.cycles;
  info->rel_residual = out.relres;
  info->status = st != CPM_OK ? st : out.status;
  info->ms_precond = tm.ms_P;
  info->ms_operator = tm.ms_M;
  info->n_precond = tm.nP;
  info->n_operator = tm.nM;
  if (tm.on) {
    cudaEventDestroy(tm.e0);
    cudaEventDestroy(tm.e1);
  }
  if (e != cudaSuccess) return cuda_fail(e, "solver", __FILE__, __LINE__);
  if (st != CPM_OK) return st;
  if (out.status == CPM_ERR_NOT_CONVERGED)
    return fail(CPM_ERR_NOT_CONVERGED, "not converged: relative residual %.3e after %d iterations", out.relres,
                out.iters);
  return out.status;
}

}  // namespace cpm
