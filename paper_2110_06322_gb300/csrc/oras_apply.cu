// oras_apply.cu -- z = sum_j Rtilde_j^T (L_j U_j)^{-1} R_j r  (Section 2.2).
//
// One CTA per subdomain (the paper's MPI subdomains become blocks of one
// launch).  The CTA gathers R_j r into a local vector -- in shared memory
// when the subdomain fits, else in a global scratch slice -- and runs the
// forward (unit L) and backward (U) substitutions level by level: the rows of
// one level are independent, one warp per row, a CTA barrier between levels.
// The factor data of a row (columns, values, diagonal) do not depend on the
// solution, so each warp loads its next row's data into registers BEFORE the
// level barrier; after the barrier only shared-memory gathers, FMAs and a
// shuffle reduction remain on the critical path.  Only the rows of the
// subdomain's own disjoint part are written back (restricted prolongation),
// so every output element has exactly one writer.
//
// Transposed: z = sum_j R_j^T (L_j U_j)^{-T} Rtilde_j r.  The factors are
// transposed once (U^T lower with U's diagonal, L^T unit upper); the local
// results of all subdomains holding a node are summed in ascending subdomain
// order by a gather (no atomics).
#include "kernels.cuh"
#include "oras.cuh"

namespace cpm {

cpm_status oras_build_transpose(oras_pc* P, cudaStream_t s);

namespace {

constexpr int SW_WARPS = 16;
constexpr int SW_K = 4;  // factor entries per lane held in registers (a row prefix of 128)
constexpr size_t SW_SMEM_MAX = 100 * 1024;  // keeps two or more CTAs per SM

template <typename V>
__device__ __forceinline__ float ldv(const V* p);
template <>
__device__ __forceinline__ float ldv<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

template <typename T, typename V>
__device__ __forceinline__ T ldval(const V* val, int64_t e) {
  if constexpr (sizeof(T) == 8) return __ldg((const double*)val + e);
  else return ldv<V>(val + e);
}

struct Sched {
  const int32_t* lvsub;
  const int64_t* lvptr;
  const int32_t* lvrow;
};

struct SwArgs {
  const int64_t* sptr;
  const int32_t* snode;
  const uint8_t* owned;
  const int64_t* rptr;
  const int32_t* col;
  const int32_t* dpos;
  Sched fwd, bwd;
  int fwd_div, bwd_div;  // divide by the diagonal in the forward / backward sweep
  int transpose;
  int64_t nA, nloc;
};

// registers describing one row of a sweep
template <typename T>
struct RowRegs {
  int64_t idx;  // position in lvrow this data belongs to (-1: none)
  int32_t q;    // local row (subdomain-local index)
  int64_t e0, e1;
  int32_t c[SW_K];
  T v[SW_K];
  T diag;
};

template <typename T, typename V>
__device__ __forceinline__ void load_row(const SwArgs& A, const V* __restrict__ val, const Sched& S, int64_t idx,
                                         int64_t base, bool lower, bool div, RowRegs<T>& R) {
  const int lane = threadIdx.x & 31;
  R.idx = idx;
  const int64_t qg = S.lvrow[idx];
  R.q = (int32_t)(qg - base);
  const int64_t r0 = A.rptr[qg], d = r0 + A.dpos[qg];
  R.e0 = lower ? r0 : d + 1;
  R.e1 = lower ? d : A.rptr[qg + 1];
#pragma unroll
  for (int k = 0; k < SW_K; ++k) {
    const int64_t e = R.e0 + lane + 32 * k;
    if (e < R.e1) {
      R.c[k] = __ldg(A.col + e);
      R.v[k] = ldval<T, V>(val, e);
    } else {
      R.c[k] = 0;
      R.v[k] = (T)0;
    }
  }
  R.diag = div ? ldval<T, V>(val, d) : (T)1;
}

template <typename T, typename V>
__device__ void sweep(const SwArgs& A, const V* __restrict__ val, const Sched& S, int j, int64_t base, T* xs,
                      bool lower, bool div) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t L0 = S.lvsub[j], L1 = S.lvsub[j + 1];
  RowRegs<T> R;
  R.idx = -1;
  for (int32_t L = L0; L < L1; ++L) {
    const int64_t i1 = S.lvptr[L + 1];
    // this warp's first row of the next level (-1: none)
    const int64_t nfirst = (L + 1 < L1 && S.lvptr[L + 1] + wid < S.lvptr[L + 2]) ? S.lvptr[L + 1] + wid : -1;
    int64_t idx = S.lvptr[L] + wid;
    if (idx >= i1 && nfirst >= 0 && R.idx != nfirst) load_row<T, V>(A, val, S, nfirst, base, lower, div, R);
    for (; idx < i1; idx += SW_WARPS) {
      if (R.idx != idx) load_row<T, V>(A, val, S, idx, base, lower, div, R);
      T s = 0;
#pragma unroll
      for (int k = 0; k < SW_K; ++k) s += R.v[k] * xs[R.c[k]];
      for (int64_t e = R.e0 + 32 * SW_K + lane; e < R.e1; e += 32) s += ldval<T, V>(val, e) * xs[__ldg(A.col + e)];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const int32_t q = R.q;
      const T dg = R.diag;
      const int64_t nxt = idx + SW_WARPS < i1 ? idx + SW_WARPS : nfirst;
      if (lane == 0) xs[q] = (xs[q] - s) / dg;
      // the factor data do not depend on the solution: fetch the next row now
      if (nxt >= 0) load_row<T, V>(A, val, S, nxt, base, lower, div, R);
    }
    __syncthreads();
  }
}

template <typename T, typename V, bool SMEM>
__global__ void __launch_bounds__(SW_WARPS * 32)
    k_schwarz(SwArgs A, const V* __restrict__ val, const T* __restrict__ r, T* __restrict__ z, T* xglob) {
  extern __shared__ __align__(16) unsigned char sw_smem[];
  const int j = blockIdx.x, rhs = blockIdx.y;
  r += (int64_t)rhs * A.nA;
  z += (int64_t)rhs * A.nA;
  const int64_t base = A.sptr[j], n = A.sptr[j + 1] - base;
  T* xs = SMEM ? reinterpret_cast<T*>(sw_smem) : xglob + (int64_t)rhs * A.nloc + base;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) {
    const T v = r[A.snode[base + q]];
    xs[q] = (A.transpose && !A.owned[base + q]) ? (T)0 : v;
  }
  __syncthreads();
  sweep<T, V>(A, val, A.fwd, j, base, xs, true, A.fwd_div);
  sweep<T, V>(A, val, A.bwd, j, base, xs, false, A.bwd_div);
  if (!A.transpose) {
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x)
      if (A.owned[base + q]) z[A.snode[base + q]] = xs[q];
  } else if (SMEM) {
    T* xg = xglob + (int64_t)rhs * A.nloc + base;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) xg[q] = xs[q];
  }
}

// adjoint prolongation: z_m = sum over the subdomains holding m (ascending)
template <typename T>
__global__ void k_gather_T(int64_t nA, int64_t nloc, const int32_t* __restrict__ mcnt,
                           const int32_t* __restrict__ mloc, const T* __restrict__ xloc, T* __restrict__ z) {
  const int rhs = blockIdx.y;
  xloc += (int64_t)rhs * nloc;
  z += (int64_t)rhs * nA;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < nA; m += (int64_t)gridDim.x * blockDim.x) {
    T acc = 0;
    for (int t = 0; t < mcnt[m]; ++t) acc = acc + xloc[mloc[m * KMEM + t]];
    z[m] = acc;
  }
}

template <typename T, typename V>
cpm_status run_typed(const oras_pc* P, const V* val, const T* r, T* z, int nrhs, int transpose, cudaStream_t s) {
  SwArgs A{};
  A.sptr = P->sptr;
  A.snode = P->snode;
  A.owned = P->owned;
  A.nA = P->nA;
  A.nloc = P->nloc;
  A.transpose = transpose;
  if (!transpose) {
    A.rptr = P->rptr;
    A.col = P->col;
    A.dpos = P->dpos;
    A.fwd = {P->lvsub_f, P->lvptr_f, P->lvrow_f};
    A.bwd = {P->lvsub_b, P->lvptr_b, P->lvrow_b};
    A.fwd_div = 0;
    A.bwd_div = 1;
  } else {
    A.rptr = P->tptr;
    A.col = P->tcol;
    A.dpos = P->tdpos;
    A.fwd = {P->lvsub_tf, P->lvptr_tf, P->lvrow_tf};
    A.bwd = {P->lvsub_tb, P->lvptr_tb, P->lvrow_tb};
    A.fwd_div = 1;
    A.bwd_div = 0;
  }
  const size_t smem = (size_t)P->max_rows * sizeof(T);
  const bool use_smem = smem <= SW_SMEM_MAX;
  T* xloc = nullptr;
  if (!use_smem || transpose) CPM_TRY(dalloc(&xloc, (size_t)nrhs * P->nloc, s));
  for (int r0 = 0; r0 < nrhs; r0 += 65535) {
    const int nr = nrhs - r0 < 65535 ? nrhs - r0 : 65535;
    dim3 g(P->np, nr);
    T* xl = xloc ? xloc + (int64_t)r0 * P->nloc : nullptr;
    if (use_smem) {
      CPM_CUDA(cudaFuncSetAttribute(k_schwarz<T, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      KL(k_schwarz<T, V, true><<<g, SW_WARPS * 32, smem, s>>>(A, val, r + (int64_t)r0 * P->nA,
                                                           z + (int64_t)r0 * P->nA, xl));
    } else {
      KL(k_schwarz<T, V, false><<<g, SW_WARPS * 32, 0, s>>>(A, val, r + (int64_t)r0 * P->nA, z + (int64_t)r0 * P->nA,
                                                          xl));
    }
    if (transpose) {
      dim3 g2(grid_for(P->nA, 256), nr);
      KL(k_gather_T<T><<<g2, 256, 0, s>>>(P->nA, P->nloc, P->mcnt, P->mloc, xl, z + (int64_t)r0 * P->nA));
    }
  }
  cudaError_t e = cudaGetLastError();
  dfree(xloc, s);
  if (e != cudaSuccess) return cuda_fail(e, "Schwarz kernels", __FILE__, __LINE__);
  return CPM_OK;
}

}  // namespace

cpm_status oras_run(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose, cudaStream_t s) {
  if (transpose) CPM_TRY(oras_build_transpose(const_cast<oras_pc*>(P), s));
  if (dt == CPM_F64) {
    const double* v = transpose ? P->tval : P->val;
    return run_typed<double, double>(P, v, (const double*)r, (double*)z, nrhs, transpose, s);
  }
  if (transpose) return run_typed<float, float>(P, P->tval32, (const float*)r, (float*)z, nrhs, 1, s);
  if (P->val16) return run_typed<float, __nv_bfloat16>(P, P->val16, (const float*)r, (float*)z, nrhs, 0, s);
  if (!P->val32) return fail(CPM_ERR_ARG, "FP32 apply needs factors stored as CPM_F32 or CPM_BF16");
  return run_typed<float, float>(P, P->val32, (const float*)r, (float*)z, nrhs, 0, s);
}

}  // namespace cpm
