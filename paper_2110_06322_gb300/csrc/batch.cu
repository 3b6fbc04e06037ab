// batch.cu -- restarted GMRES(m) over a batch of independent systems
//   (c_p I - Delta_S^h(p)) u_{p,r} = f_{p,r}
// for problems p (each its own band, Schwarz preconditioner and shift c_p)
// and right-hand sides r of each problem, advanced in lockstep.
//
// All systems' vectors are concatenated into one vector of N = sum n_s
// doubles: problem-major, right-hand side within problem (so a problem's
// right-hand sides sit one after another, the nrhs layout of cpm_apply and
// oras_apply).  A Krylov basis vector is such a concatenation too, and the
// vector kernels run over the whole batch at once: the grid's blocks are
// shared out among the systems in proportion to their lengths, each block
// knowing its system, so dot products are segmented sums with one partial per
// block and a fixed reduction order (reproducible).  The per-system scalars
// -- Hessenberg columns, Givens rotations, residual estimates -- live on the
// device, one thread per system.
//
// A system that reaches its tolerance inside a cycle is frozen on the device
// (its next basis vectors are zero, so nothing of it changes any more) and
// records how many columns it uses; the host does not look at the cycle until
// it ends.  Each cycle ends with the true residual of every system
// (FP64), as in the single-system solver.
//
// The operator and the preconditioner apply once per problem per iteration,
// with all its right-hand sides in one launch; the problems' launches go to
// eight side streams, so that small problems run side by side.  With mixed = 1 they run in
// FP32 inside FP64 iterative refinement (one flexible inner cycle per
// refinement step), as cpm_solve does for one system.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "oras.cuh"
#include "reduce.cuh"

namespace cpm {

cpm_status oras_run(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose, cudaStream_t s);

namespace {

constexpr int BGS = 16;  // basis vectors per segmented Gram-Schmidt kernel

// Block b of a batched vector kernel covers elements [lo[b], hi[b]) of the
// concatenated vector, all inside system sys[b].  When act is set, blocks of
// systems with act[sys] == 0 (stopped) skip their elements: their partial
// sums are zero and their vectors are left as they are (nothing reads them
// any more in this cycle).
struct Seg {
  const int32_t* sys;
  const int64_t* lo;
  const int64_t* hi;
  const int32_t* act;
  __device__ __forceinline__ bool skip(int b) const { return act && !act[sys[b]]; }
};

// partial[t * gridDim.x + b] = block b's share of <V_t, w>, t < nv
template <int NV>
__global__ void __launch_bounds__(RED_THREADS)
    kb_dots(Seg G, const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w, double* partial) {
  double acc[NV];
#pragma unroll
  for (int t = 0; t < NV; ++t) acc[t] = 0;
  const int64_t lo = G.lo[blockIdx.x], hi = G.skip(blockIdx.x) ? lo : G.hi[blockIdx.x];
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int t = 0; t < NV; ++t)
      if (t < nv) acc[t] += V[t * ld + i] * wi;
  }
  block_partials<NV>(acc, nv, partial);
}

// w -= sum_t coef[sys][t] V_t (t < nv); NORM: partial[b] = block b's share of |w|^2
template <int NV, bool NORM>
__global__ void __launch_bounds__(RED_THREADS)
    kb_update(Seg G, const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ coef, int ldc,
              double* w, double* partial) {
  __shared__ double cf[NV];
  const int s = G.sys[blockIdx.x];
  if (threadIdx.x < NV) cf[threadIdx.x] = threadIdx.x < nv ? coef[(int64_t)s * ldc + threadIdx.x] : 0.0;
  __syncthreads();
  double acc[1] = {0.0};
  const int64_t lo = G.lo[blockIdx.x], hi = G.skip(blockIdx.x) ? lo : G.hi[blockIdx.x];
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double wi = w[i];
#pragma unroll
    for (int t = 0; t < NV; ++t)
      if (t < nv) wi -= cf[t] * V[t * ld + i];
    w[i] = wi;
    acc[0] += wi * wi;
  }
  if (NORM) block_partials<1>(acc, 1, partial);
}

// out[s * ldo + t] (+)= sum over system s's blocks of partial[t * nb + b];
// grid (nv, S), one block per value
__global__ void __launch_bounds__(RED_THREADS)
    kb_reduce(const double* __restrict__ partial, int nb, const int32_t* __restrict__ sb, double* out, int ldo,
              int accumulate) {
  __shared__ double sh[RED_THREADS / 32];
  const int t = blockIdx.x, s = blockIdx.y;
  double v = 0;
  for (int b = sb[s] + threadIdx.x; b < sb[s + 1]; b += blockDim.x) v += partial[(int64_t)t * nb + b];
  const double tot = block_sum(v, sh);
  if (threadIdx.x == 0) {
    double* o = out + (int64_t)s * ldo + t;
    *o = accumulate ? *o + tot : tot;
  }
}

// v = w * scale[sys]
__global__ void __launch_bounds__(RED_THREADS)
    kb_scale(Seg G, const double* __restrict__ w, const double* __restrict__ scale, double* v) {
  const double a = scale[G.sys[blockIdx.x]];
  const int64_t lo = G.lo[blockIdx.x], hi = G.skip(blockIdx.x) ? lo : G.hi[blockIdx.x];
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) v[i] = w[i] * a;
}

struct SysState {
  double* H;      // [S][m+1][m] (row i, column j at i * m + j)
  double* hc;     // [S][m+2]: new column, |w|^2 last
  double* cs;     // [S][m]
  double* sn;     // [S][m]
  double* g;      // [S][m+1]
  double* y;      // [S][m]
  double* scale;  // [S] scale of the next basis vector (0 when frozen)
  double* rr;     // [S] |r|^2 at the start of a cycle
  double* fn;     // [S] |f|_2 (refinement: |f| of the outer system)
  double* tol;    // [S] absolute tolerance of the current cycle
  int32_t* active;
  int32_t* kk;    // [S] columns used in the current cycle
  int32_t* its;   // [S] iterations so far
};

// start of a cycle: beta = |r|; the system takes part if beta > tol and it
// has iterations left
__global__ void kb_cycle_init(int S, int m, SysState X, int maxit, double rtol, int inner) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double beta = sqrt(X.rr[s]);
  const double tol = inner ? rtol * beta : rtol * X.fn[s];
  const bool go = beta > 0.0 && (inner ? true : beta > tol) && X.its[s] < maxit;
  X.tol[s] = tol;
  X.active[s] = go ? 1 : 0;
  X.kk[s] = 0;
  X.scale[s] = go ? 1.0 / beta : 0.0;
  double* g = X.g + (int64_t)s * (m + 1);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
}

// Givens update of column j of every active system; a system whose residual
// estimate reaches its tolerance (or whose Krylov space is exhausted) stops
// and keeps j + 1 columns
__global__ void kb_givens(int S, int m, int j, SysState X, int maxit) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || !X.active[s]) return;
  double* H = X.H + (int64_t)s * (m + 1) * m;
  const double* hc = X.hc + (int64_t)s * (m + 2);
  double* cs = X.cs + (int64_t)s * m;
  double* sn = X.sn + (int64_t)s * m;
  double* g = X.g + (int64_t)s * (m + 1);
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
  X.kk[s] = j + 1;
  X.its[s] += 1;
  const bool stop = hn == 0.0 || !(fabs(g[j + 1]) > X.tol[s]) || X.its[s] >= maxit;
  X.active[s] = stop ? 0 : 1;
  X.scale[s] = stop ? 0.0 : 1.0 / hn;
}

// y = H(0:k,0:k)^{-1} g per system; -y into ny (the coefficients of t -= V (-y))
__global__ void kb_trisolve(int S, int m, SysState X, double* ny, int ldn) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int k = X.kk[s];
  const double* H = X.H + (int64_t)s * (m + 1) * m;
  const double* g = X.g + (int64_t)s * (m + 1);
  double* y = X.y + (int64_t)s * m;
  for (int i = k - 1; i >= 0; --i) {
    double a = g[i];
    for (int t = i + 1; t < k; ++t) a -= H[i * m + t] * y[t];
    y[i] = a / H[i * m + i];
  }
  for (int i = 0; i < ldn; ++i) ny[(int64_t)s * ldn + i] = i < k ? -y[i] : 0.0;
}

__global__ void kb_sub(const double* __restrict__ f, double* r, int64_t n) {  // r = f - r
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = f[i] - r[i];
}
__global__ void kb_axpy(const double* __restrict__ z, double* x, int64_t n) {  // x += z
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += z[i];
}
__global__ void kb_d2f(const double* __restrict__ a, float* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void kb_f2d(const float* __restrict__ a, double* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

struct Batch {
  int P = 0, S = 0, m = 0, NB = 0;
  int64_t N = 0;
  std::vector<const cpm_band*> band;
  std::vector<const oras_pc*> pc;
  std::vector<double> c;
  std::vector<int> nrhs;
  std::vector<int64_t> po;  // problem offsets [P+1]
  std::vector<char> live;   // problems with a system still iterating (this cycle)
  std::vector<char> zeroed; // finished problems whose z and w segments are zero
  // side streams: the per-problem operator and preconditioner launches of one
  // iteration run concurrently (small problems fill only a few SMs each)
  static constexpr int NSTREAM = 8;
  cudaStream_t ss[NSTREAM] = {};
  cudaStream_t cap = nullptr;  // private stream the cycle graph is captured on (the caller's
                               // stream may be the legacy default stream, which cannot capture)
  cudaEvent_t fork = nullptr, join[NSTREAM] = {};
  cpm_status make_streams() {
    for (int k = 0; k < NSTREAM; ++k) {
      CPM_CUDA(cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking));
      CPM_CUDA(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
    }
    CPM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CPM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    return CPM_OK;
  }
  void free_streams() {
    for (int k = 0; k < NSTREAM; ++k) {
      if (ss[k]) cudaStreamDestroy(ss[k]);
      if (join[k]) cudaEventDestroy(join[k]);
      ss[k] = nullptr;
      join[k] = nullptr;
    }
    if (fork) cudaEventDestroy(fork);
    fork = nullptr;
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
  }
  // side streams start after everything queued on s so far
  cpm_status fan_out(cudaStream_t s) {
    CPM_CUDA(cudaEventRecord(fork, s));
    for (int k = 0; k < NSTREAM; ++k) CPM_CUDA(cudaStreamWaitEvent(ss[k], fork, 0));
    return CPM_OK;
  }
  // s continues after all side-stream work
  cpm_status fan_in(cudaStream_t s) {
    for (int k = 0; k < NSTREAM; ++k) {
      CPM_CUDA(cudaEventRecord(join[k], ss[k]));
      CPM_CUDA(cudaStreamWaitEvent(s, join[k], 0));
    }
    return CPM_OK;
  }
  cudaStream_t side(int p) const { return ss[p % NSTREAM]; }
  Seg G{};   // every block works
  Seg GA{};  // blocks of stopped systems skip (act = X.active)
  int32_t* sb = nullptr;  // [S+1] first block of each system
  double *V = nullptr, *w = nullptr, *z = nullptr, *t = nullptr, *r = nullptr, *ny = nullptr, *partial = nullptr;
  // mixed precision: the preconditioned vectors z_j = P v_j of the inner
  // cycle (m x N), kept so that the correction is sum_j y_j z_j (flexible
  // GMRES): it is built from exactly the vectors of the Arnoldi relation, and
  // the cycle needs no preconditioner apply after the last column
  double* Z = nullptr;
  float *x32 = nullptr, *y32 = nullptr;
  SysState X{};
  std::vector<void*> owned;
  // CUDA graph of one cycle: a cycle is a fixed sequence of launches (systems
  // stop on the device), so it is captured once per set of live problems and
  // replayed; the first cycle of a solve runs uncaptured, since first uses
  // (factor packing, transposed structures) synchronise.
  cudaGraphExec_t cycle_exec = nullptr;
  std::vector<char> cycle_live;
  const double* cycle_x = nullptr;
  bool cycle_f32 = false;
  int cycle_inner = 0;
  long long cycle_kernels = 0;  // kernels in the captured cycle (counted at each replay)
  bool warm = false;
  int graph_replays = 0, graph_captures = 0;

  template <typename T>
  cpm_status get(T** p, size_t n, cudaStream_t s) {
    CPM_TRY(dalloc(p, n, s));
    owned.push_back((void*)*p);
    return CPM_OK;
  }
  void release(cudaStream_t s) {
    if (cycle_exec) cudaGraphExecDestroy(cycle_exec);
    cycle_exec = nullptr;
    for (void* p : owned) cudaFreeAsync(p, s);
    owned.clear();
    free_streams();
  }
};

// the batch's blocks: each system gets a share of NB in proportion to its
// length (at least one), and its elements are split evenly over them
cpm_status make_segments(Batch& Bt, const std::vector<int64_t>& so, cudaStream_t s) {
  const int S = Bt.S;
  const int64_t N = so[S];
  const int target = std::max(152 * 8, S);
  std::vector<int> nbs(S);
  int NB = 0;
  for (int q = 0; q < S; ++q) {
    const int64_t n = so[q + 1] - so[q];
    int k = (int)std::max<int64_t>(1, (int64_t)((double)target * (double)n / (double)std::max<int64_t>(N, 1)));
    k = (int)std::min<int64_t>(k, std::max<int64_t>(1, (n + 255) / 256));
    nbs[q] = k;
    NB += k;
  }
  std::vector<int32_t> sys(NB), sb(S + 1);
  std::vector<int64_t> lo(NB), hi(NB);
  int b = 0;
  for (int q = 0; q < S; ++q) {
    sb[q] = b;
    const int64_t n = so[q + 1] - so[q];
    for (int k = 0; k < nbs[q]; ++k, ++b) {
      sys[b] = q;
      lo[b] = so[q] + n * k / nbs[q];
      hi[b] = so[q] + n * (k + 1) / nbs[q];
    }
  }
  sb[S] = NB;
  Bt.NB = NB;
  int32_t *dsys = nullptr, *dsb = nullptr;
  int64_t *dlo = nullptr, *dhi = nullptr;
  CPM_TRY(Bt.get(&dsys, NB, s));
  CPM_TRY(Bt.get(&dlo, NB, s));
  CPM_TRY(Bt.get(&dhi, NB, s));
  CPM_TRY(Bt.get(&dsb, S + 1, s));
  CPM_CUDA(cudaMemcpyAsync(dsys, sys.data(), NB * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CPM_CUDA(cudaMemcpyAsync(dlo, lo.data(), NB * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CPM_CUDA(cudaMemcpyAsync(dhi, hi.data(), NB * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CPM_CUDA(cudaMemcpyAsync(dsb, sb.data(), (S + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CPM_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  Bt.G = Seg{dsys, dlo, dhi, nullptr};
  Bt.sb = dsb;
  return CPM_OK;
}

int grid_n(int64_t n) { return grid_for(n, 256); }

// partial sums and per-system reductions of <V_t, w>, t in [t0, t0 + nc)
cpm_status seg_dots(Batch& Bt, const Seg& G, const double* V, int nc, const double* w, double* out, int ldo,
                    int acc, cudaStream_t s) {
  if (nc <= 8) KL(kb_dots<8><<<Bt.NB, RED_THREADS, 0, s>>>(G, V, Bt.N, nc, w, Bt.partial));
  else KL(kb_dots<16><<<Bt.NB, RED_THREADS, 0, s>>>(G, V, Bt.N, nc, w, Bt.partial));
  KL(kb_reduce<<<dim3(nc, Bt.S), RED_THREADS, 0, s>>>(Bt.partial, Bt.NB, Bt.sb, out, ldo, acc));
  return CPM_OK;
}

// w -= V_{t0..t0+nc} coef; with norm, out[s * ldo] = |w_s|^2
cpm_status seg_update(Batch& Bt, const Seg& G, const double* V, int nc, const double* coef, int ldc, double* w,
                      bool norm, double* out, int ldo, cudaStream_t s) {
  if (nc <= 8) {
    if (norm) KL(kb_update<8, true><<<Bt.NB, RED_THREADS, 0, s>>>(G, V, Bt.N, nc, coef, ldc, w, Bt.partial));
    else KL(kb_update<8, false><<<Bt.NB, RED_THREADS, 0, s>>>(G, V, Bt.N, nc, coef, ldc, w, nullptr));
  } else {
    if (norm) KL(kb_update<16, true><<<Bt.NB, RED_THREADS, 0, s>>>(G, V, Bt.N, nc, coef, ldc, w, Bt.partial));
    else KL(kb_update<16, false><<<Bt.NB, RED_THREADS, 0, s>>>(G, V, Bt.N, nc, coef, ldc, w, nullptr));
  }
  if (norm) KL(kb_reduce<<<dim3(1, Bt.S), RED_THREADS, 0, s>>>(Bt.partial, Bt.NB, Bt.sb, out, ldo, 0));
  return CPM_OK;
}

inline int chunk_of(int nv) {
  const int nch = (nv + BGS - 1) / BGS;
  return (nv + nch - 1) / nch;
}

// out = M x per problem (FP64, or FP32 through the conversion buffers).
// Problems with no live system are skipped: the solver zeroes their segments
// of the outputs (z, w) once when they finish, and nothing else writes them,
// so a batch does not keep paying for the systems that have finished.
cpm_status batch_M(Batch& Bt, const double* x, double* out, bool f32, int transpose, cudaStream_t s,
                   bool all = false) {
  CPM_TRY(Bt.fan_out(s));
  for (int p = 0; p < Bt.P; ++p) {
    cudaStream_t sp = Bt.side(p);
    std::vector<double> cs(Bt.nrhs[p], Bt.c[p]);
    const int64_t o = Bt.po[p], len = Bt.po[p + 1] - o;
    if (!all && !Bt.live[p]) continue;  // its output segment was zeroed when it finished
    if (f32) {
      KL(kb_d2f<<<grid_n(len), 256, 0, sp>>>(x + o, Bt.x32 + o, len));
      CPM_TRY(apply_op(Bt.band[p], cs.data(), Bt.x32 + o, Bt.y32 + o, CPM_F32, Bt.nrhs[p], transpose, sp));
      KL(kb_f2d<<<grid_n(len), 256, 0, sp>>>(Bt.y32 + o, out + o, len));
    } else {
      CPM_TRY(apply_op(Bt.band[p], cs.data(), x + o, out + o, CPM_F64, Bt.nrhs[p], transpose, sp));
    }
  }
  return Bt.fan_in(s);
}

// out = P x per problem (identity where a problem has no preconditioner;
// zero for problems with no live system); conversions per live problem
cpm_status batch_P(Batch& Bt, const double* x, double* out, bool f32, int transpose, cudaStream_t s) {
  CPM_TRY(Bt.fan_out(s));
  for (int p = 0; p < Bt.P; ++p) {
    cudaStream_t sp = Bt.side(p);
    const int64_t o = Bt.po[p], len = Bt.po[p + 1] - o;
    if (!Bt.live[p]) continue;  // its output segment was zeroed when it finished
    if (!Bt.pc[p]) {
      CPM_CUDA(cudaMemcpyAsync(out + o, x + o, len * sizeof(double), cudaMemcpyDeviceToDevice, sp));
      continue;
    }
    if (f32) {
      KL(kb_d2f<<<grid_n(len), 256, 0, sp>>>(x + o, Bt.x32 + o, len));
      CPM_TRY(oras_run(Bt.pc[p], Bt.x32 + o, Bt.y32 + o, CPM_F32, Bt.nrhs[p], transpose, sp));
      KL(kb_f2d<<<grid_n(len), 256, 0, sp>>>(Bt.y32 + o, out + o, len));
    } else {
      CPM_TRY(oras_run(Bt.pc[p], x + o, out + o, CPM_F64, Bt.nrhs[p], transpose, sp));
    }
  }
  return Bt.fan_in(s);
}

// One GMRES(m) cycle for every active system on M d = b (x += P V y, or
// x += Z y with the kept z_j = P v_j in the mixed cycle), from the residual
// vector r (overwritten).  inner: tolerances relative to |r|
// (refinement), else to |f|.
cpm_status batch_cycle(Batch& Bt, double* x, bool f32, int transpose, int maxit, double rtol, int inner,
                       cudaStream_t s) {
  const int S = Bt.S, m = Bt.m;
  const int gs = (S + 127) / 128;
  // |r_s|^2, v_0 = r / |r|
  CPM_TRY(seg_dots(Bt, Bt.G, Bt.r, 1, Bt.r, Bt.X.rr, 1, 0, s));
  KL(kb_cycle_init<<<gs, 128, 0, s>>>(S, m, Bt.X, maxit, rtol, inner));
  KL(kb_scale<<<Bt.NB, RED_THREADS, 0, s>>>(Bt.G, Bt.r, Bt.X.scale, Bt.V));
  const bool flex = f32 && Bt.Z;
  for (int j = 0; j < m; ++j) {
    double* vj = Bt.V + (int64_t)j * Bt.N;
    double* zj = flex ? Bt.Z + (int64_t)j * Bt.N : Bt.z;
    CPM_TRY(batch_P(Bt, vj, zj, f32, transpose, s));
    CPM_TRY(batch_M(Bt, zj, Bt.w, f32, transpose, s));
    // classical Gram-Schmidt, one pass: hc = V^T w; w -= V hc; hc[j+1] = |w|^2
    const int nv = j + 1, cs = chunk_of(nv);
    for (int t0 = 0; t0 < nv; t0 += cs) {
      const int nc = std::min(cs, nv - t0);
      CPM_TRY(seg_dots(Bt, Bt.GA, Bt.V + (int64_t)t0 * Bt.N, nc, Bt.w, Bt.X.hc + t0, m + 2, 0, s));
    }
    for (int t0 = 0; t0 < nv; t0 += cs) {
      const int nc = std::min(cs, nv - t0);
      const bool last = t0 + cs >= nv;
      CPM_TRY(seg_update(Bt, Bt.GA, Bt.V + (int64_t)t0 * Bt.N, nc, Bt.X.hc + t0, m + 2, Bt.w, last, Bt.X.hc + nv,
                         m + 2, s));
    }
    KL(kb_givens<<<gs, 128, 0, s>>>(S, m, j, Bt.X, maxit));
    if (j + 1 < m) KL(kb_scale<<<Bt.NB, RED_THREADS, 0, s>>>(Bt.GA, Bt.w, Bt.X.scale, Bt.V + (int64_t)(j + 1) * Bt.N));
    CPM_CUDA(cudaGetLastError());
  }
  // x += P (V y), or x += Z y when flexible; y per system over its kk columns
  KL(kb_trisolve<<<gs, 128, 0, s>>>(S, m, Bt.X, Bt.ny, m));
  CPM_CUDA(cudaMemsetAsync(Bt.t, 0, Bt.N * sizeof(double), s));
  const int cs = chunk_of(m);
  const double* basis = flex ? Bt.Z : Bt.V;
  for (int t0 = 0; t0 < m; t0 += cs) {
    const int nc = std::min(cs, m - t0);
    CPM_TRY(seg_update(Bt, Bt.G, basis + (int64_t)t0 * Bt.N, nc, Bt.ny + t0, m, Bt.t, false, nullptr, 0, s));
  }
  if (flex) {
    KL(kb_axpy<<<grid_n(Bt.N), 256, 0, s>>>(Bt.t, x, Bt.N));
  } else {
    CPM_TRY(batch_P(Bt, Bt.t, Bt.z, f32, transpose, s));
    KL(kb_axpy<<<grid_n(Bt.N), 256, 0, s>>>(Bt.z, x, Bt.N));
  }
  CPM_CUDA(cudaGetLastError());
  return CPM_OK;
}

// One cycle through the graph cache: replay the captured cycle when the live
// problems, the solution vector and the precision are those it was captured
// with; otherwise capture this cycle (after one uncaptured warm-up cycle).
// Capture runs on the batch's private stream; the graph is launched on s.
cpm_status run_cycle(Batch& Bt, double* x, bool f32, int transpose, int maxit, double rtol, int inner,
                     cudaStream_t s) {
  if (Bt.cycle_exec && Bt.cycle_live == Bt.live && Bt.cycle_x == x && Bt.cycle_f32 == f32 &&
      Bt.cycle_inner == inner) {
    CPM_CUDA(cudaGraphLaunch(Bt.cycle_exec, s));
    g_launches.fetch_add(Bt.cycle_kernels, std::memory_order_relaxed);
    Bt.graph_replays++;
    return CPM_OK;
  }
  if (!Bt.warm) {
    Bt.warm = true;
    return batch_cycle(Bt, x, f32, transpose, maxit, rtol, inner, s);
  }
  if (Bt.cycle_exec) cudaGraphExecDestroy(Bt.cycle_exec);
  Bt.cycle_exec = nullptr;
  const long long k0 = g_launches.load();
  CPM_CUDA(cudaStreamBeginCapture(Bt.cap, cudaStreamCaptureModeThreadLocal));
  const cpm_status st = batch_cycle(Bt, x, f32, transpose, maxit, rtol, inner, Bt.cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(Bt.cap, &g);
  if (st != CPM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "capture of a batched GMRES cycle", __FILE__, __LINE__);
  const cudaError_t e2 = cudaGraphInstantiate(&Bt.cycle_exec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return cuda_fail(e2, "instantiation of a batched GMRES cycle", __FILE__, __LINE__);
  Bt.cycle_kernels = g_launches.load() - k0;
  Bt.cycle_live = Bt.live;
  Bt.cycle_x = x;
  Bt.cycle_f32 = f32;
  Bt.cycle_inner = inner;
  Bt.graph_captures++;
  CPM_CUDA(cudaGraphLaunch(Bt.cycle_exec, s));
  return CPM_OK;
}

}  // namespace

namespace {
// one group of problems solved in lockstep
cpm_status solve_group(int nprob, const cpm_band* const* bands, const oras_pc* const* pcs, const double* c,
                       const int32_t* nrhs, const double* f, double* u, const cpm_solve_params* prm,
                       cpm_solve_info* info, int transpose, cudaStream_t s) {
  Batch Bt;
  Bt.P = nprob;
  Bt.m = prm->restart;
  Bt.po.assign(nprob + 1, 0);
  std::vector<int64_t> so(1, 0);
  for (int p = 0; p < nprob; ++p) {
    Bt.band.push_back(bands[p]);
    Bt.pc.push_back(pcs ? pcs[p] : nullptr);
    Bt.c.push_back(c[p]);
    Bt.nrhs.push_back(nrhs[p]);
    const int64_t n = bands[p]->nA;
    for (int q = 0; q < nrhs[p]; ++q) so.push_back(so.back() + n);
    Bt.po[p + 1] = Bt.po[p] + (int64_t)nrhs[p] * n;
  }
  Bt.S = (int)so.size() - 1;
  Bt.N = so.back();
  std::vector<int> sys_prob;
  for (int p = 0; p < nprob; ++p)
    for (int q = 0; q < nrhs[p]; ++q) sys_prob.push_back(p);
  const int S = Bt.S, m = Bt.m;
  const bool mixed = prm->mixed != 0;
  for (int p = 0; p < nprob; ++p)
    if (mixed && Bt.pc[p] && Bt.pc[p]->store == CPM_F64)
      return fail(CPM_ERR_ARG, "mixed precision needs FP32 or BF16 factors (problem %d)", p);
  cpm_status st = make_segments(Bt, so, s);
  if (st == CPM_OK) st = Bt.make_streams();
  auto bail = [&](cpm_status e) {
    Bt.release(s);
    cudaStreamSynchronize(s);
    return e;
  };
  if (st != CPM_OK) return bail(st);
#define BTRY(x)                      \
  do {                               \
    cpm_status e_ = (x);             \
    if (e_ != CPM_OK) return bail(e_); \
  } while (0)
  BTRY(Bt.get(&Bt.V, (size_t)(m + 1) * Bt.N, s));
  // a stopped system's later basis vectors are left as they are (finite: an
  // older vector or these zeros) and enter the correction with coefficient 0
  BTRY(cudaMemsetAsync(Bt.V, 0, (size_t)(m + 1) * Bt.N * sizeof(double), s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
  BTRY(Bt.get(&Bt.w, Bt.N, s));
  BTRY(Bt.get(&Bt.z, Bt.N, s));
  BTRY(Bt.get(&Bt.t, Bt.N, s));
  BTRY(Bt.get(&Bt.r, Bt.N, s));
  BTRY(Bt.get(&Bt.ny, (size_t)S * m, s));
  BTRY(Bt.get(&Bt.partial, (size_t)BGS * Bt.NB, s));
  if (mixed) {
    BTRY(Bt.get(&Bt.x32, Bt.N, s));
    BTRY(Bt.get(&Bt.y32, Bt.N, s));
    // finished problems' columns keep finite values (these zeros or older
    // vectors) and enter the correction with coefficient 0
    BTRY(Bt.get(&Bt.Z, (size_t)m * Bt.N, s));
    BTRY(cudaMemsetAsync(Bt.Z, 0, (size_t)m * Bt.N * sizeof(double), s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
  }
  SysState& X = Bt.X;
  BTRY(Bt.get(&X.H, (size_t)S * (m + 1) * m, s));
  BTRY(Bt.get(&X.hc, (size_t)S * (m + 2), s));
  BTRY(Bt.get(&X.cs, (size_t)S * m, s));
  BTRY(Bt.get(&X.sn, (size_t)S * m, s));
  BTRY(Bt.get(&X.g, (size_t)S * (m + 1), s));
  BTRY(Bt.get(&X.y, (size_t)S * m, s));
  BTRY(Bt.get(&X.scale, S, s));
  BTRY(Bt.get(&X.rr, S, s));
  BTRY(Bt.get(&X.fn, S, s));
  BTRY(Bt.get(&X.tol, S, s));
  BTRY(Bt.get(&X.active, S, s));
  BTRY(Bt.get(&X.kk, S, s));
  BTRY(Bt.get(&X.its, S, s));
  double* d = nullptr;  // refinement correction
  if (mixed) BTRY(Bt.get(&d, Bt.N, s));
  BTRY(cudaMemsetAsync(X.its, 0, S * sizeof(int32_t), s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
  // |f_s|
  Bt.GA = Seg{Bt.G.sys, Bt.G.lo, Bt.G.hi, X.active};
  BTRY(seg_dots(Bt, Bt.G, f, 1, f, X.rr, 1, 0, s));
  std::vector<double> h2(S), fn(S);
  BTRY(cudaMemcpyAsync(h2.data(), X.rr, S * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess ? CPM_OK
                                                                                                  : CPM_ERR_CUDA);
  BTRY(cudaStreamSynchronize(s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
  for (int q = 0; q < S; ++q) {
    fn[q] = std::sqrt(h2[q]);
    if (!std::isfinite(fn[q])) return bail(fail(CPM_ERR_NAN, "right-hand side %d holds NaN or Inf", q));
  }
  BTRY(cudaMemcpyAsync(X.fn, fn.data(), S * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess ? CPM_OK
                                                                                                   : CPM_ERR_CUDA);
  std::vector<int32_t> its(S, 0);
  std::vector<double> rel(S, 0.0);
  const double inner = prm->inner_rtol > 0 ? prm->inner_rtol : 1e-4;
  int cycles = 0, ir = 0;
  while (true) {
    // true residual of every system (FP64): r = f - M u
    BTRY(batch_M(Bt, u, Bt.r, false, transpose, s, true));
    KL(kb_sub<<<grid_n(Bt.N), 256, 0, s>>>(f, Bt.r, Bt.N));
    BTRY(seg_dots(Bt, Bt.G, Bt.r, 1, Bt.r, X.rr, 1, 0, s));
    BTRY(cudaMemcpyAsync(h2.data(), X.rr, S * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess
             ? CPM_OK
             : CPM_ERR_CUDA);
    BTRY(cudaMemcpyAsync(its.data(), X.its, S * sizeof(int32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess
             ? CPM_OK
             : CPM_ERR_CUDA);
    BTRY(cudaStreamSynchronize(s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
    bool any = false;
    Bt.live.assign(nprob, 0);
    for (int q = 0; q < S; ++q) {
      const double rn = std::sqrt(h2[q]);
      if (!std::isfinite(rn)) return bail(fail(CPM_ERR_NAN, "residual of system %d became NaN or Inf", q));
      rel[q] = fn[q] > 0 ? rn / fn[q] : 0.0;
      if (rel[q] > prm->rtol && its[q] < prm->maxit) {
        any = true;
        Bt.live[sys_prob[q]] = 1;
      }
    }
    if (!any) break;
    Bt.zeroed.resize(nprob, 0);
    for (int p = 0; p < nprob; ++p)
      if (!Bt.live[p] && !Bt.zeroed[p]) {
        const int64_t o = Bt.po[p], len = Bt.po[p + 1] - o;
        BTRY(cudaMemsetAsync(Bt.z + o, 0, len * sizeof(double), s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
        BTRY(cudaMemsetAsync(Bt.w + o, 0, len * sizeof(double), s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
        Bt.zeroed[p] = 1;
      }
    ++cycles;
    if (!mixed) {
      BTRY(run_cycle(Bt, u, false, transpose, prm->maxit, prm->rtol, 0, s));
    } else {
      // refinement step: systems already at rtol get no correction (their
      // residual is zeroed, which freezes them in the inner cycle)
      ++ir;
      std::vector<double> keep(S);
      for (int q = 0; q < S; ++q) keep[q] = (rel[q] > prm->rtol && its[q] < prm->maxit) ? 1.0 : 0.0;
      BTRY(cudaMemcpyAsync(X.scale, keep.data(), S * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess
               ? CPM_OK
               : CPM_ERR_CUDA);
      KL(kb_scale<<<Bt.NB, RED_THREADS, 0, s>>>(Bt.G, Bt.r, X.scale, Bt.r));
      BTRY(cudaMemsetAsync(d, 0, Bt.N * sizeof(double), s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);
      BTRY(run_cycle(Bt, d, true, transpose, prm->maxit, inner, 1, s));
      KL(kb_axpy<<<grid_n(Bt.N), 256, 0, s>>>(d, u, Bt.N));
      BTRY(cudaStreamSynchronize(s) == cudaSuccess ? CPM_OK : CPM_ERR_CUDA);  // keep is read by the copy
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batched solve", __FILE__, __LINE__));
  for (int p = 0; p < nprob; ++p)
    if (Bt.pc[p]) {
      const cpm_status te = oras_take_error(Bt.pc[p], s);
      if (te != CPM_OK) return bail(te);
    }
  cpm_status all = CPM_OK;
  for (int q = 0; q < S; ++q) {
    info[q] = cpm_solve_info{};
    info[q].iters = its[q];
    info[q].restarts = cycles;
    info[q].ir_steps = mixed ? ir : 0;
    info[q].rel_residual = rel[q];
    info[q].status = rel[q] <= prm->rtol ? CPM_OK : CPM_ERR_NOT_CONVERGED;
    if (info[q].status != CPM_OK) all = CPM_ERR_NOT_CONVERGED;
  }
#undef BTRY
  Bt.release(s);
  cudaStreamSynchronize(s);
  return all;
}
}  // namespace

// Memory-bounded batching: the lockstep solver holds its Krylov basis and
// work vectors for every system at once ((restart + 7) doubles per unknown,
// 2 restart + 7 with the preconditioned vectors of the mixed cycle),
// so the problems are cut, in order, into consecutive groups whose storage
// fits min(32 GB, 40 % of the device's free memory) and the groups are
// solved one after another.
cpm_status solve_batch(int nprob, const cpm_band* const* bands, const oras_pc* const* pcs, const double* c,
                       const int32_t* nrhs, const double* f, double* u, const cpm_solve_params* prm,
                       cpm_solve_info* info, int transpose, cudaStream_t s) {
  size_t freeb = 0, totalb = 0;
  CPM_CUDA(cudaMemGetInfo(&freeb, &totalb));
  const double budget = std::min(32e9, 0.4 * (double)freeb);
  const double per_unknown = 8.0 * ((prm->mixed ? 2 * prm->restart : prm->restart) + 7);
  cpm_status all = CPM_OK;
  int p0 = 0;
  int64_t off = 0, sys0 = 0;
  while (p0 < nprob) {
    int p1 = p0;
    double bytes = 0;
    int64_t len = 0, nsys = 0;
    do {
      bytes += per_unknown * (double)nrhs[p1] * (double)bands[p1]->nA;
      len += (int64_t)nrhs[p1] * bands[p1]->nA;
      nsys += nrhs[p1];
      ++p1;
    } while (p1 < nprob && bytes + per_unknown * (double)nrhs[p1] * (double)bands[p1]->nA <= budget);
    const cpm_status st = solve_group(p1 - p0, bands + p0, pcs ? pcs + p0 : nullptr, c + p0, nrhs + p0, f + off,
                                      u + off, prm, info + sys0, transpose, s);
    if (st == CPM_ERR_NOT_CONVERGED) all = CPM_ERR_NOT_CONVERGED;
    else if (st != CPM_OK) return st;
    off += len;
    sys0 += nsys;
    p0 = p1;
  }
  return all;
}

}  // namespace cpm
