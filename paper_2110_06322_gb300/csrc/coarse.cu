// coarse.cu -- two-level Schwarz preconditioner: a coarse correction added to
// the one-level apply.  The paper's preconditioners are one-level and it
// names a coarse grid correction as future work (Section 4.1.1); the reading
// built here:
//
//   coarse space  Z, one column per disjoint part a: Z_{i,a} = 1 if node i
//                 lies in part a (a constant per part)
//   coarse matrix E0 = Z^T M Z   (np x np, dense; its inverse is kept)
//   apply         q = Z E0^{-1} Z^T r,   z = q + P_RAS (r - M q)
//                 (P2 = Q + P_RAS (I - M Q), Q = Z E0^{-1} Z^T: the coarse
//                 correction first, then the one-level apply on what is left)
//   transposed    t = P_RAS^T r,   z = t + Z E0^{-T} Z^T (r - M^T t)
//
// M q for a piecewise-constant q = Z y is a short sum per node: the rows of
// M Z (for each node, the parts its matrix row reaches and the row's sum over
// each of them) are built once at set-up and give both E0 (summed over the
// nodes of each part) and, in every apply, r - M Z y without touching M.
// The transposed apply forms M^T t with the matrix-free transposed operator.
// Every sum runs in a fixed order, so the applies are reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "oras.cuh"

namespace cpm {

cpm_status oras_run_one_level(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose,
                              cudaStream_t s);

namespace {

constexpr int KMZ = 64;    // most parts one matrix row may reach (a row spans a few lattice cells)
constexpr int NBMAX = 64;  // parts one part's rows reach, summed warp-parallel (more: by one lane)

// rows of M Z: for node i, the distinct parts of its row's columns (in order
// of first appearance along the ascending columns) and the row's sum over
// each.  count pass (out == nullptr) or fill pass.
__global__ void k_mz(int64_t nA, const int64_t* __restrict__ mptr, const int32_t* __restrict__ mcol,
                     const double* __restrict__ mval, const int32_t* __restrict__ part, int32_t* cnt,
                     const int64_t* __restrict__ optr, int32_t* opart, double* oval, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nA; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t pp[KMZ];
    double vv[KMZ];
    int k = 0;
    for (int64_t q = mptr[i]; q < mptr[i + 1]; ++q) {
      const int32_t b = part[mcol[q]];
      int t = 0;
      while (t < k && pp[t] != b) ++t;
      if (t == k) {
        if (k == KMZ) {
          atomicExch(err, CPM_ERR_ARG);
          break;
        }
        pp[k] = b;
        vv[k] = 0.0;
        ++k;
      }
      vv[t] += mval[q];
    }
    if (!optr) {
      cnt[i] = k;
    } else {
      const int64_t o = optr[i];
      for (int t = 0; t < k; ++t) {
        opart[o + t] = pp[t];
        oval[o + t] = vv[t];
      }
    }
  }
}

// E0 row a = sum over the nodes of part a (the owned rows of subdomain a, in
// local order) of their M Z rows.  One warp per part: the distinct parts
// reached are collected in a bitmap and listed ascending; lane l sums the
// part's nodes l, l + 32, ... into its own slots; slot s is then summed over
// lanes 0..31 in order.
__global__ void __launch_bounds__(32) k_coarse_e0(int np, const int64_t* __restrict__ sptr,
                                                  const int32_t* __restrict__ snode, const uint8_t* __restrict__ owned,
                                                  const int64_t* __restrict__ mzptr, const int32_t* __restrict__ mzpart,
                                                  const double* __restrict__ mzval, double* E0, int* err) {
  extern __shared__ unsigned int bm[];  // np bits
  __shared__ int32_t nbr[NBMAX];
  __shared__ int nn;
  __shared__ double acc[32][NBMAX + 1];
  const int a = blockIdx.x, lane = threadIdx.x;
  const int nw = (np + 31) / 32;
  for (int w = lane; w < nw; w += 32) bm[w] = 0u;
  for (int t = 0; t < NBMAX; ++t) acc[lane][t] = 0.0;
  __syncwarp();
  const int64_t b0 = sptr[a], b1 = sptr[a + 1];
  for (int64_t q = b0 + lane; q < b1; q += 32)
    if (owned[q]) {
      const int64_t i = snode[q];
      for (int64_t e = mzptr[i]; e < mzptr[i + 1]; ++e) atomicOr(&bm[mzpart[e] >> 5], 1u << (mzpart[e] & 31));
    }
  __syncwarp();
  if (lane == 0) {
    int k = 0;
    for (int w = 0; w < nw; ++w) {
      unsigned int bits = bm[w];
      while (bits) {
        const int bit = __ffs(bits) - 1;
        bits &= bits - 1;
        if (k < NBMAX) nbr[k] = w * 32 + bit;
        ++k;
      }
    }
    nn = k;
  }
  __syncwarp();
  const int n = nn;
  if (n == 0) {  // an empty part: a decoupled unit row keeps E0 regular (its Z^T r is 0)
    if (lane == 0) E0[(int64_t)a * np + a] = 1.0;
    return;
  }
  if (n > NBMAX) {
    // a small part among many tiny ones reaches more parts than there are
    // slots: one lane sums its rows in order straight into the zeroed E0 row
    if (lane == 0)
      for (int64_t q = b0; q < b1; ++q)
        if (owned[q]) {
          const int64_t i = snode[q];
          for (int64_t e = mzptr[i]; e < mzptr[i + 1]; ++e) E0[(int64_t)a * np + mzpart[e]] += mzval[e];
        }
    return;
  }
  for (int64_t q = b0 + lane; q < b1; q += 32)
    if (owned[q]) {
      const int64_t i = snode[q];
      for (int64_t e = mzptr[i]; e < mzptr[i + 1]; ++e) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (nbr[mid] < mzpart[e]) lo = mid + 1;
          else hi = mid;
        }
        acc[lane][lo] += mzval[e];
      }
    }
  __syncwarp();
  for (int t = lane; t < n; t += 32) {
    double sum = 0.0;
    for (int l = 0; l < 32; ++l) sum += acc[l][t];
    E0[(int64_t)a * np + nbr[t]] = sum;
  }
}

// Gauss-Jordan elimination with partial pivoting on [A | X], X = I on entry:
// one launch per column k.  k_gj_pivot (one block) finds the pivot row
// (largest |A_ik|, i >= k, ties by the smaller i), swaps it into row k of A
// and X and scales row k by 1 / A_kk.
__global__ void __launch_bounds__(256) k_gj_pivot(int n, int k, double* A, double* X, int* err) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  double best = -1.0;
  int bidx = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(A[(int64_t)i * n + k]);
    if (v > best) {
      best = v;
      bidx = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = bv[threadIdx.x + o];
      const int i2 = bi[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const int p = bi[0];
  if (bv[0] <= 0.0) {
    if (threadIdx.x == 0) atomicExch(err, CPM_ERR_BREAKDOWN);
    return;
  }
  if (p != k)
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = A[(int64_t)k * n + j];
      A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
      A[(int64_t)p * n + j] = t;
      t = X[(int64_t)k * n + j];
      X[(int64_t)k * n + j] = X[(int64_t)p * n + j];
      X[(int64_t)p * n + j] = t;
    }
  __syncthreads();
  const double inv = 1.0 / A[(int64_t)k * n + k];
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    A[(int64_t)k * n + j] *= inv;
    X[(int64_t)k * n + j] *= inv;
  }
}

// rows i != k: row_i -= A_ik row_k (A_ik read before the update: column k of
// row i is saved first, since the kernel rewrites it).
__global__ void k_gj_elim(int n, int k, double* A, double* X, const double* __restrict__ colk) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i == k) continue;
    const double f = colk[i];
    A[e] -= f * A[(int64_t)k * n + j];
    X[e] -= f * X[(int64_t)k * n + j];
  }
}
__global__ void k_gj_col(int n, int k, const double* __restrict__ A, double* colk) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) colk[i] = A[(int64_t)i * n + k];
}
__global__ void k_eye(int n, double* X) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// y0[rhs][a] = sum over the nodes i of part a of (v_i - w_i) (w may be null),
// owned rows of subdomain a in local order, fixed block reduction
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(int np, int64_t nA, const int64_t* __restrict__ sptr,
                                                  const int32_t* __restrict__ snode, const uint8_t* __restrict__ owned,
                                                  const T* __restrict__ v, const T* __restrict__ w, double* y0) {
  __shared__ double sh[8];
  const int a = blockIdx.x, rhs = blockIdx.y;
  v += (int64_t)rhs * nA;
  if (w) w += (int64_t)rhs * nA;
  double acc = 0.0;
  for (int64_t q = sptr[a] + threadIdx.x; q < sptr[a + 1]; q += blockDim.x)
    if (owned[q]) {
      const int64_t i = snode[q];
      acc += w ? (double)v[i] - (double)w[i] : (double)v[i];
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < 8; ++q) t += sh[q];
    y0[(int64_t)rhs * np + a] = t;
  }
}

// y[rhs] = E0^{-1} y0[rhs] (transpose: E0^{-T}); one warp per row
__global__ void k_coarse_mv(int np, const double* __restrict__ Einv, const double* __restrict__ y0, double* y,
                            int transpose) {
  const int rhs = blockIdx.y, lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= np) return;
  y0 += (int64_t)rhs * np;
  double acc = 0.0;
  for (int c = lane; c < np; c += 32)
    acc += (transpose ? Einv[(int64_t)c * np + row] : Einv[(int64_t)row * np + c]) * y0[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[(int64_t)rhs * np + row] = acc;
}

// t_i = r_i - (M Z y)_i, the residual left after the coarse correction.  The
// coefficients and the sum stay FP64 in FP32 applies too: y is of size |r| / c
// on the coarse space, so (M Z y)_i cancels against r_i to a value ~c / |M|
// times its terms, and FP32-rounded coefficients would leave an error of
// eps_32 |M| / c relative to t (percents for small shifts on fine grids).
template <typename T>
__global__ void k_coarse_res(int64_t nA, int np, const int64_t* __restrict__ mzptr, const int32_t* __restrict__ mzpart,
                             const double* __restrict__ mzval, const double* __restrict__ y, const T* __restrict__ r,
                             T* __restrict__ t) {
  const int rhs = blockIdx.y;
  r += (int64_t)rhs * nA;
  t += (int64_t)rhs * nA;
  y += (int64_t)rhs * np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nA; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t e = mzptr[i]; e < mzptr[i + 1]; ++e) acc += mzval[e] * y[mzpart[e]];
    t[i] = (T)((double)r[i] - acc);
  }
}

// z_i = (base ? base_i : z_i) + y[part(i)]
template <typename T>
__global__ void k_coarse_add(int64_t nA, int np, const int32_t* __restrict__ part, const double* __restrict__ y,
                             const T* __restrict__ base, T* z) {
  const int rhs = blockIdx.y;
  z += (int64_t)rhs * nA;
  if (base) base += (int64_t)rhs * nA;
  y += (int64_t)rhs * np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nA; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = (T)((double)(base ? base[i] : z[i]) + y[part[i]]);
}

template <typename T>
cpm_status coarse_apply_t(const oras_pc* P, const T* r, T* z, int nrhs, int transpose, cudaStream_t s) {
  const cpm_dtype dt = sizeof(T) == 8 ? CPM_F64 : CPM_F32;
  const int np = P->np;
  const int64_t nA = P->nA;
  T* t = nullptr;
  double* y = nullptr;
  CPM_TRY(dalloc(&t, (size_t)nrhs * nA, s));
  cpm_status st = dalloc(&y, (size_t)2 * nrhs * np, s);
  if (st != CPM_OK) {
    dfree(t, s);
    return st;
  }
  double* y0 = y + (int64_t)nrhs * np;
  const dim3 gP(np, nrhs), gN(grid_for(nA, 256), nrhs), gC((np * 32 + 255) / 256, nrhs);
  if (!transpose) {
    KL(k_restrict<T><<<gP, 256, 0, s>>>(np, nA, P->sptr, P->snode, P->owned, r, nullptr, y0));
    KL(k_coarse_mv<<<gC, 256, 0, s>>>(np, P->E0inv, y0, y, 0));
    KL(k_coarse_res<T><<<gN, 256, 0, s>>>(nA, np, P->mzptr, P->mzpart, P->mzval, y, r, t));
    st = oras_run_one_level(P, t, z, dt, nrhs, 0, s);
    if (st == CPM_OK) KL(k_coarse_add<T><<<gN, 256, 0, s>>>(nA, np, P->part, y, nullptr, z));
  } else {
    // t = P_RAS^T r;  z = M^T t;  y0 = Z^T (r - z);  z = t + Z E0^{-T} y0
    st = oras_run_one_level(P, r, t, dt, nrhs, 1, s);
    if (st == CPM_OK) {
      std::vector<double> cs(nrhs, P->c);
      st = apply_op(P->band, cs.data(), t, z, dt, nrhs, 1, s);
    }
    if (st == CPM_OK) {
      KL(k_restrict<T><<<gP, 256, 0, s>>>(np, nA, P->sptr, P->snode, P->owned, r, z, y0));
      KL(k_coarse_mv<<<gC, 256, 0, s>>>(np, P->E0inv, y0, y, 1));
      KL(k_coarse_add<T><<<gN, 256, 0, s>>>(nA, np, P->part, y, t, z));
    }
  }
  cudaError_t e = cudaGetLastError();
  dfree(t, s);
  dfree(y, s);
  if (st != CPM_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "coarse correction kernels", __FILE__, __LINE__);
  return CPM_OK;
}

}  // namespace

// Coarse structures of a two-level preconditioner from the assembled M
// (CSR, columns ascending in every row): rows of M Z, E0 = Z^T M Z and its
// inverse.
cpm_status coarse_build(oras_pc* P, const int64_t* mptr, const int32_t* mcol, const double* mval, cudaStream_t s) {
  const int np = P->np;
  const int64_t nA = P->nA;
  int32_t* cnt = nullptr;
  int* err = nullptr;
  double *E = nullptr, *colk = nullptr;
  auto done = [&](cpm_status st) {
    dfree(cnt, s);
    dfree(err, s);
    dfree(E, s);
    dfree(colk, s);
    return st;
  };
  cpm_status st;
  if ((st = dalloc(&cnt, nA, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&err, 1, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&P->mzptr, nA + 1, s)) != CPM_OK) return done(st);
  CPM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  const int G = grid_for(nA, 256);
  KL(k_mz<<<G, 256, 0, s>>>(nA, mptr, mcol, mval, P->part, cnt, nullptr, nullptr, nullptr, err));
  if ((st = scan_exclusive_i32(cnt, P->mzptr, nA, s)) != CPM_OK) return done(st);
  int64_t nmz = 0;
  CPM_CUDA(cudaMemcpyAsync(&nmz, P->mzptr + nA, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if ((st = dalloc(&P->mzpart, nmz, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&P->mzval, nmz, s)) != CPM_OK) return done(st);
  KL(k_mz<<<G, 256, 0, s>>>(nA, mptr, mcol, mval, P->part, nullptr, P->mzptr, P->mzpart, P->mzval, err));
  // E0 and its inverse
  const int64_t nn = (int64_t)np * np;
  if ((st = dalloc(&E, nn, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&P->E0inv, nn, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&colk, np, s)) != CPM_OK) return done(st);
  CPM_CUDA(cudaMemsetAsync(E, 0, nn * sizeof(double), s));
  const size_t bmb = (size_t)((np + 31) / 32) * sizeof(unsigned int);
  if (bmb > 48 * 1024) return done(fail(CPM_ERR_ARG, "two-level preconditioner supports at most 393216 parts"));
  KL(k_coarse_e0<<<np, 32, bmb, s>>>(np, P->sptr, P->snode, P->owned, P->mzptr, P->mzpart, P->mzval, E, err));
  int herr = 0;
  CPM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if (herr) return done(fail(CPM_ERR_ARG, "a matrix row reaches more than %d parts", KMZ));
  const int GE = grid_for(nn, 256);
  KL(k_eye<<<GE, 256, 0, s>>>(np, P->E0inv));
  for (int k = 0; k < np; ++k) {
    KL(k_gj_pivot<<<1, 256, 0, s>>>(np, k, E, P->E0inv, err));
    KL(k_gj_col<<<(np + 255) / 256, 256, 0, s>>>(np, k, E, colk));
    KL(k_gj_elim<<<GE, 256, 0, s>>>(np, k, E, P->E0inv, colk));
  }
  CPM_CUDA(cudaGetLastError());
  CPM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if (herr) return done(fail(CPM_ERR_BREAKDOWN, "the coarse matrix Z^T M Z is singular"));
  return done(CPM_OK);
}

void coarse_free(oras_pc* P, cudaStream_t s) {
  dfree(P->mzptr, s);
  dfree(P->mzpart, s);
  dfree(P->mzval, s);
  dfree(P->E0inv, s);
}

cpm_status coarse_apply(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose,
                        cudaStream_t s) {
  if (dt == CPM_F64) return coarse_apply_t<double>(P, (const double*)r, (double*)z, nrhs, transpose, s);
  return coarse_apply_t<float>(P, (const float*)r, (float*)z, nrhs, transpose, s);
}

}  // namespace cpm
