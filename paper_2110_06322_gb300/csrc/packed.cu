// packed.cu -- level-packed ILU(0) factors and the TMA-streamed Schwarz apply.
//
// Set-up repacks the factors of every subdomain in the order the triangular
// sweeps consume them: the forward rows (strict lower part) level by level,
// then the backward rows (diagonal first, then the strict upper part) level by
// level.  Consecutive rows of one level are cut into chunks of at most
// CHUNK_BYTES; a chunk never spans two levels.  A chunk is
//     [row headers: {local row, entry offset, entry count, pad} x nrows]
//     [16-bit local columns x ne, padded to 16 bytes]
//     [values x ne, padded to 16 bytes]
// so a whole chunk is one contiguous, 16-byte aligned copy.
//
// The apply runs one CTA per subdomain: thread 0 streams the chunk sequence
// (forward then backward) into a ring of NSTAGE shared-memory buffers with
// cp.async.bulk (the 1-D TMA copy) and mbarrier transaction counts, NSTAGE-1
// chunks ahead; all warps consume the current chunk from shared memory (one
// warp per row: gather the local vector, multiply, shuffle-reduce) and meet at
// one CTA barrier per chunk, which is also the level barrier.  The local
// vector lives in shared memory when it fits, else in a global slice.  Every
// mbarrier wait is bounded; a wait that runs out sets an error flag, the CTA
// drains its copies in flight (bounded) and returns.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "oras.cuh"

namespace cpm {

cpm_status oras_build_transpose(oras_pc* P, cudaStream_t s);

namespace {

constexpr int CHUNK_BYTES = 16384;
constexpr int NSTAGE = 3;
constexpr int PK_WARPS = 16;
constexpr unsigned WAIT_LIMIT = 1u << 26;  // polls of one mbarrier before giving up

__host__ __device__ inline int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }

template <typename V>
__host__ __device__ inline int64_t chunk_bytes(int64_t nrows, int64_t ne) {
  return 16 * nrows + pad16(2 * ne) + pad16((int64_t)sizeof(V) * ne);
}

// ---------------------------------------------------------------- packing
struct SweepSrc {
  const int64_t* rptr;
  const int32_t* col;
  const int32_t* dpos;
  const double* val;
  const int32_t* lvsub;
  const int64_t* lvptr;
  const int32_t* lvrow;
  int lower, div;
};

__device__ __forceinline__ int64_t row_entries(const SweepSrc& S, int64_t q) {
  const int64_t n = S.rptr[q + 1] - S.rptr[q], d = S.dpos[q];
  return (S.lower ? d : n - d - 1) + (S.div ? 1 : 0);
}

// pass A: one thread per subdomain walks its schedule and cuts chunks.
// mode 0: count chunks; mode 1: write chunk records and row placements.
template <typename V>
__global__ void k_pack_plan(int np, SweepSrc S, int mode, int32_t* nchunks, const int64_t* __restrict__ chbase,
                            ChunkRec* rec, int32_t* row_chunk, int32_t* row_slot, int32_t* row_eoff, int kindflag) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  int64_t c = mode ? chbase[j] : 0;
  int32_t cnt = 0;
  for (int32_t L = S.lvsub[j]; L < S.lvsub[j + 1]; ++L) {
    int64_t nrows = 0, ne = 0;
    for (int64_t idx = S.lvptr[L]; idx < S.lvptr[L + 1]; ++idx) {
      const int64_t q = S.lvrow[idx];
      const int64_t e = row_entries(S, q);
      if (nrows > 0 && chunk_bytes<V>(nrows + 1, ne + e) > CHUNK_BYTES) {
        if (mode) {
          rec[c].bytes = (int32_t)chunk_bytes<V>(nrows, ne);
          rec[c].nrows = (int32_t)nrows;
          rec[c].ne = (int32_t)ne;
          rec[c].div = kindflag;
        }
        ++c;
        ++cnt;
        nrows = 0;
        ne = 0;
      }
      if (mode) {
        row_chunk[idx] = (int32_t)c;
        row_slot[idx] = (int32_t)nrows;
        row_eoff[idx] = (int32_t)ne;
      }
      ++nrows;
      ne += e;
    }
    if (nrows > 0) {
      if (mode) {
        rec[c].bytes = (int32_t)chunk_bytes<V>(nrows, ne);
        rec[c].nrows = (int32_t)nrows;
        rec[c].ne = (int32_t)ne;
        rec[c].div = kindflag;
      }
      ++c;
      ++cnt;
    }
  }
  if (!mode) nchunks[j] = cnt;
}

__global__ void k_chunk_sizes(int64_t n, const ChunkRec* __restrict__ rec, int64_t* sz) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    sz[c] = rec[c].bytes;
}
__global__ void k_chunk_offsets(int64_t n, const int64_t* __restrict__ off, ChunkRec* rec) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    rec[c].off = off[c];
}

// pass B: one warp per scheduled row writes its header and entries
template <typename V>
__global__ void k_pack_write(int64_t nrow, SweepSrc S, const int64_t* __restrict__ sptr,
                             const int32_t* __restrict__ lsub, const ChunkRec* __restrict__ rec,
                             const int32_t* __restrict__ row_chunk, const int32_t* __restrict__ row_slot,
                             const int32_t* __restrict__ row_eoff, uint8_t* data) {
  const int lane = threadIdx.x & 31;
  for (int64_t idx = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; idx < nrow;
       idx += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t q = S.lvrow[idx];
    const ChunkRec R = rec[row_chunk[idx]];
    uint8_t* base = data + R.off;
    int32_t* hdr = reinterpret_cast<int32_t*>(base) + 4 * row_slot[idx];
    uint16_t* cols = reinterpret_cast<uint16_t*>(base + 16 * (int64_t)R.nrows);
    V* vals = reinterpret_cast<V*>(base + 16 * (int64_t)R.nrows + pad16(2 * (int64_t)R.ne));
    const int64_t eo = row_eoff[idx];
    const int64_t r0 = S.rptr[q], d = r0 + S.dpos[q], r1 = S.rptr[q + 1];
    const int64_t e0 = S.lower ? r0 : d + 1, e1 = S.lower ? d : r1;
    const int64_t off = S.div ? 1 : 0;
    if (lane == 0) {
      hdr[0] = (int32_t)(q - sptr[lsub[q]]);
      hdr[1] = (int32_t)eo;
      hdr[2] = (int32_t)(e1 - e0 + off);
      hdr[3] = 0;
      if (S.div) {
        cols[eo] = 0;
        vals[eo] = (V)S.val[d];
      }
    }
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      cols[eo + off + (e - e0)] = (uint16_t)S.col[e];
      vals[eo + off + (e - e0)] = (V)S.val[e];
    }
  }
}

template <>
__global__ void k_pack_write<__nv_bfloat16>(int64_t nrow, SweepSrc S, const int64_t* __restrict__ sptr,
                                            const int32_t* __restrict__ lsub, const ChunkRec* __restrict__ rec,
                                            const int32_t* __restrict__ row_chunk, const int32_t* __restrict__ row_slot,
                                            const int32_t* __restrict__ row_eoff, uint8_t* data) {
  const int lane = threadIdx.x & 31;
  for (int64_t idx = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; idx < nrow;
       idx += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t q = S.lvrow[idx];
    const ChunkRec R = rec[row_chunk[idx]];
    uint8_t* base = data + R.off;
    int32_t* hdr = reinterpret_cast<int32_t*>(base) + 4 * row_slot[idx];
    uint16_t* cols = reinterpret_cast<uint16_t*>(base + 16 * (int64_t)R.nrows);
    __nv_bfloat16* vals = reinterpret_cast<__nv_bfloat16*>(base + 16 * (int64_t)R.nrows + pad16(2 * (int64_t)R.ne));
    const int64_t eo = row_eoff[idx];
    const int64_t r0 = S.rptr[q], d = r0 + S.dpos[q], r1 = S.rptr[q + 1];
    const int64_t e0 = S.lower ? r0 : d + 1, e1 = S.lower ? d : r1;
    const int64_t off = S.div ? 1 : 0;
    if (lane == 0) {
      hdr[0] = (int32_t)(q - sptr[lsub[q]]);
      hdr[1] = (int32_t)eo;
      hdr[2] = (int32_t)(e1 - e0 + off);
      hdr[3] = 0;
      if (S.div) {
        cols[eo] = 0;
        vals[eo] = __float2bfloat16_rn((float)S.val[d]);
      }
    }
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      cols[eo + off + (e - e0)] = (uint16_t)S.col[e];
      vals[eo + off + (e - e0)] = __float2bfloat16_rn((float)S.val[e]);
    }
  }
}

template <typename V>
cpm_status pack_one(oras_pc* P, const SweepSrc* sw, PackedFactors& out, cudaStream_t s) {
  const int np = P->np;
  const int64_t nloc = P->nloc;
  int32_t* cnt = nullptr;
  int64_t* chbase[2] = {nullptr, nullptr};
  int32_t *rc = nullptr, *rs = nullptr, *re = nullptr;
  int64_t* sz = nullptr;
  int64_t* off = nullptr;
  CPM_TRY(dalloc(&cnt, np, s));
  // chunk counts per subdomain for both sweeps; layout: subdomain j owns the
  // chunks [chsub[j], chsub[j+1]): its forward chunks, then its backward chunks
  std::vector<int32_t> hc[2];
  for (int w = 0; w < 2; ++w) {
    KL(k_pack_plan<V><<<(np + 127) / 128, 128, 0, s>>>(np, sw[w], 0, cnt, nullptr, nullptr, nullptr, nullptr,
                                                       nullptr, sw[w].div));
    hc[w].resize(np);
    CPM_CUDA(cudaMemcpyAsync(hc[w].data(), cnt, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  }
  CPM_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> chsub(np + 1, 0), hbase[2];
  hbase[0].resize(np);
  hbase[1].resize(np);
  for (int j = 0; j < np; ++j) {
    hbase[0][j] = chsub[j];
    hbase[1][j] = chsub[j] + hc[0][j];
    chsub[j + 1] = chsub[j] + hc[0][j] + hc[1][j];
  }
  const int64_t nch = chsub[np];
  out.nchunks = nch;
  CPM_TRY(dalloc(&out.rec, nch, s));
  CPM_TRY(dalloc(&out.chsub, np + 1, s));
  CPM_CUDA(cudaMemcpyAsync(out.chsub, chsub.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CPM_TRY(dalloc(&rc, nloc, s));
  CPM_TRY(dalloc(&rs, nloc, s));
  CPM_TRY(dalloc(&re, nloc, s));
  for (int w = 0; w < 2; ++w) {
    CPM_TRY(dalloc(&chbase[w], np, s));
    CPM_CUDA(cudaMemcpyAsync(chbase[w], hbase[w].data(), np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  }
  CPM_TRY(dalloc(&sz, nch, s));
  CPM_TRY(dalloc(&off, nch + 1, s));
  // chunk records of both sweeps, then their byte offsets
  for (int w = 0; w < 2; ++w)
    KL(k_pack_plan<V><<<(np + 127) / 128, 128, 0, s>>>(np, sw[w], 1, nullptr, chbase[w], out.rec, rc, rs, re,
                                                       sw[w].div));
  KL(k_chunk_sizes<<<grid_for(nch, 256), 256, 0, s>>>(nch, out.rec, sz));
  CPM_TRY(scan_exclusive_i64(sz, off, nch, s));
  KL(k_chunk_offsets<<<grid_for(nch, 256), 256, 0, s>>>(nch, off, out.rec));
  CPM_CUDA(cudaMemcpyAsync(&out.bytes, off + nch, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  CPM_TRY(dalloc(&out.data, out.bytes, s));
  for (int w = 0; w < 2; ++w) {
    // row placements (per schedule position) of sweep w, then its data; the
    // re-plan rewrites the same records and leaves their offsets in place
    KL(k_pack_plan<V><<<(np + 127) / 128, 128, 0, s>>>(np, sw[w], 1, nullptr, chbase[w], out.rec, rc, rs, re,
                                                       sw[w].div));
    KL(k_pack_write<V><<<grid_for(nloc * 32, 256), 256, 0, s>>>(nloc, sw[w], P->sptr, P->lsub, out.rec, rc, rs, re,
                                                               out.data));
  }
  CPM_CUDA(cudaGetLastError());
  CPM_CUDA(cudaStreamSynchronize(s));
  dfree(cnt, s);
  dfree(chbase[0], s);
  dfree(chbase[1], s);
  dfree(rc, s);
  dfree(rs, s);
  dfree(re, s);
  dfree(sz, s);
  dfree(off, s);
  return CPM_OK;
}

// ---------------------------------------------------------------- apply
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

template <typename V, typename T>
__device__ __forceinline__ T cvt(V v) {
  if constexpr (std::is_same<V, __nv_bfloat16>::value) return (T)__bfloat162float(v);
  else return (T)v;
}

struct PkArgs {
  const int64_t* sptr;
  const int32_t* snode;
  const uint8_t* owned;
  const int64_t* chsub;
  const ChunkRec* rec;
  const uint8_t* data;
  int transpose;
  int64_t nA, nloc;
  int* err;
};

template <typename T, typename V, bool SMEMX>
__global__ void __launch_bounds__(PK_WARPS * 32)
    k_schwarz_pk(PkArgs A, const T* __restrict__ r, T* __restrict__ z, T* xglob) {
  extern __shared__ __align__(128) unsigned char pk_smem[];
  __shared__ uint64_t full[NSTAGE];
  __shared__ int abort_flag;
  const int j = blockIdx.x, rhs = blockIdx.y;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  r += (int64_t)rhs * A.nA;
  z += (int64_t)rhs * A.nA;
  unsigned char* ring = pk_smem;
  const int64_t base = A.sptr[j], n = A.sptr[j + 1] - base;
  T* xs = SMEMX ? reinterpret_cast<T*>(pk_smem + NSTAGE * CHUNK_BYTES) : xglob + (int64_t)rhs * A.nloc + base;
  const int64_t c0 = A.chsub[j], nch = A.chsub[j + 1] - c0;
  if (tid == 0) {
    abort_flag = 0;
    for (int q = 0; q < NSTAGE; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int64_t c = 0; c < nch && c < NSTAGE; ++c) {
      const ChunkRec R = A.rec[c0 + c];
      mbar_expect_tx(&full[c], (uint32_t)R.bytes);
      bulk_g2s(ring + c * CHUNK_BYTES, A.data + R.off, (uint32_t)R.bytes, &full[c]);
    }
  for (int64_t q = tid; q < n; q += blockDim.x) {
    const T v = r[A.snode[base + q]];
    xs[q] = (A.transpose && !A.owned[base + q]) ? (T)0 : v;
  }
  __syncthreads();
  int64_t issued = nch < NSTAGE ? nch : NSTAGE;
  for (int64_t c = 0; c < nch; ++c) {
    const int st = (int)(c % NSTAGE);
    const uint32_t par = (uint32_t)((c / NSTAGE) & 1);
    unsigned polls = 0;
    while (!mbar_try_wait(&full[st], par)) {
      if (++polls > WAIT_LIMIT) {
        abort_flag = 1;
        break;
      }
    }
    const ChunkRec R = A.rec[c0 + c];
    const unsigned char* buf = ring + st * CHUNK_BYTES;
    const int32_t* hdr = reinterpret_cast<const int32_t*>(buf);
    const uint16_t* cols = reinterpret_cast<const uint16_t*>(buf + 16 * (int64_t)R.nrows);
    const V* vals = reinterpret_cast<const V*>(buf + 16 * (int64_t)R.nrows + pad16(2 * (int64_t)R.ne));
    if (!abort_flag) {
      for (int rr = wid; rr < R.nrows; rr += PK_WARPS) {
        const int4 h = reinterpret_cast<const int4*>(hdr)[rr];
        const int q = h.x, eo = h.y, cnt = h.z;
        const int e0 = R.div ? 1 : 0;
        T s = 0;
        for (int e = e0 + lane; e < cnt; e += 32) s += cvt<V, T>(vals[eo + e]) * xs[cols[eo + e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
          T v = xs[q] - s;
          if (R.div) v = v / cvt<V, T>(vals[eo]);
          xs[q] = v;
        }
      }
    }
    __syncthreads();
    if (abort_flag) break;
    // refill the stage just consumed (only thread 0 issues copies)
    if (tid == 0 && issued < nch) {
      const int st2 = (int)(issued % NSTAGE);
      const ChunkRec R2 = A.rec[c0 + issued];
      fence_proxy_async();
      mbar_expect_tx(&full[st2], (uint32_t)R2.bytes);
      bulk_g2s(ring + st2 * CHUNK_BYTES, A.data + R2.off, (uint32_t)R2.bytes, &full[st2]);
      ++issued;
    }
  }
  if (abort_flag) {
    if (tid == 0) {
      atomicExch(A.err, CPM_ERR_TIMEOUT);
      // drain copies in flight (bounded) before the shared memory goes away
      for (int64_t c = 0; c < issued; ++c) {
        unsigned polls = 0;
        while (!mbar_try_wait(&full[c % NSTAGE], (uint32_t)((c / NSTAGE) & 1)) && ++polls < WAIT_LIMIT) {
        }
      }
    }
    return;
  }
  if (!A.transpose) {
    for (int64_t q = tid; q < n; q += blockDim.x)
      if (A.owned[base + q]) z[A.snode[base + q]] = xs[q];
  } else if (SMEMX) {
    T* xg = xglob + (int64_t)rhs * A.nloc + base;
    for (int64_t q = tid; q < n; q += blockDim.x) xg[q] = xs[q];
  }
}

template <typename T>
__global__ void k_gather_T2(int64_t nA, int64_t nloc, const int32_t* __restrict__ mcnt,
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

}  // namespace

// Build the level-packed factors (forward rows, then backward rows) with
// values of type V from the CSR factors; transposed selects the transposed
// factors (U^T with its diagonal first, then L^T).
cpm_status pack_factors(oras_pc* P, int transposed, cpm_dtype vt, PackedFactors& out, cudaStream_t s) {
  if (P->max_rows > 65535) return fail(CPM_ERR_ARG, "subdomain of %lld rows exceeds 16-bit local columns", (long long)P->max_rows);
  SweepSrc sw[2];
  if (!transposed) {
    sw[0] = {P->rptr, P->col, P->dpos, P->val, P->lvsub_f, P->lvptr_f, P->lvrow_f, 1, 0};
    sw[1] = {P->rptr, P->col, P->dpos, P->val, P->lvsub_b, P->lvptr_b, P->lvrow_b, 0, 1};
  } else {
    sw[0] = {P->tptr, P->tcol, P->tdpos, P->tval, P->lvsub_tf, P->lvptr_tf, P->lvrow_tf, 1, 1};
    sw[1] = {P->tptr, P->tcol, P->tdpos, P->tval, P->lvsub_tb, P->lvptr_tb, P->lvrow_tb, 0, 0};
  }
  out.vtype = vt;
  if (vt == CPM_F64) return pack_one<double>(P, sw, out, s);
  if (vt == CPM_F32) return pack_one<float>(P, sw, out, s);
  return pack_one<__nv_bfloat16>(P, sw, out, s);
}

void packed_free(PackedFactors& pf, cudaStream_t s) {
  dfree(pf.data, s);
  dfree(pf.rec, s);
  dfree(pf.chsub, s);
  pf.nchunks = 0;
  pf.bytes = 0;
}

template <typename T, typename V>
static cpm_status run_pk(const oras_pc* P, const PackedFactors& pf, const T* r, T* z, int nrhs, int transpose,
                         cudaStream_t s) {
  PkArgs A{};
  A.sptr = P->sptr;
  A.snode = P->snode;
  A.owned = P->owned;
  A.chsub = pf.chsub;
  A.rec = pf.rec;
  A.data = pf.data;
  A.transpose = transpose;
  A.nA = P->nA;
  A.nloc = P->nloc;
  A.err = P->err;
  const size_t ring = (size_t)NSTAGE * CHUNK_BYTES;
  const size_t xsb = (size_t)P->max_rows * sizeof(T);
  const bool smemx = ring + xsb <= 113 * 1024;  // two CTAs per SM
  T* xloc = nullptr;
  if (!smemx || transpose) CPM_TRY(dalloc(&xloc, (size_t)nrhs * P->nloc, s));
  for (int r0 = 0; r0 < nrhs; r0 += 65535) {
    const int nr = nrhs - r0 < 65535 ? nrhs - r0 : 65535;
    dim3 g(P->np, nr);
    T* xl = xloc ? xloc + (int64_t)r0 * P->nloc : nullptr;
    if (smemx) {
      const size_t sm = ring + xsb;
      CPM_CUDA(cudaFuncSetAttribute(k_schwarz_pk<T, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      KL(k_schwarz_pk<T, V, true><<<g, PK_WARPS * 32, sm, s>>>(A, r + (int64_t)r0 * P->nA, z + (int64_t)r0 * P->nA,
                                                               xl));
    } else {
      CPM_CUDA(cudaFuncSetAttribute(k_schwarz_pk<T, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ring));
      KL(k_schwarz_pk<T, V, false><<<g, PK_WARPS * 32, ring, s>>>(A, r + (int64_t)r0 * P->nA,
                                                                  z + (int64_t)r0 * P->nA, xl));
    }
    if (transpose) {
      dim3 g2(grid_for(P->nA, 256), nr);
      KL(k_gather_T2<T><<<g2, 256, 0, s>>>(P->nA, P->nloc, P->mcnt, P->mloc, xl, z + (int64_t)r0 * P->nA));
    }
  }
  cudaError_t e = cudaGetLastError();
  dfree(xloc, s);
  if (e != cudaSuccess) return cuda_fail(e, "packed Schwarz kernels", __FILE__, __LINE__);
  return CPM_OK;
}

cpm_status oras_run(const oras_pc* Pc, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose, cudaStream_t s) {
  oras_pc* P = const_cast<oras_pc*>(Pc);
  if (dt == CPM_F32 && !transpose && P->store == CPM_F64)
    return fail(CPM_ERR_ARG, "FP32 apply needs factors stored as CPM_F32 or CPM_BF16");
  if (transpose) CPM_TRY(oras_build_transpose(P, s));
  const int slot = (transpose ? 2 : 0) + (dt == CPM_F32 ? 1 : 0);
  PackedFactors& pf = P->packed[slot];
  if (!pf.data) {
    const cpm_dtype vt = dt == CPM_F64 ? CPM_F64 : (transpose ? CPM_F32 : (cpm_dtype)P->store);
    CPM_TRY(pack_factors(P, transpose, vt, pf, s));
  }
  if (dt == CPM_F64) return run_pk<double, double>(P, pf, (const double*)r, (double*)z, nrhs, transpose, s);
  if (pf.vtype == CPM_BF16)
    return run_pk<float, __nv_bfloat16>(P, pf, (const float*)r, (float*)z, nrhs, transpose, s);
  return run_pk<float, float>(P, pf, (const float*)r, (float*)z, nrhs, transpose, s);
}

}  // namespace cpm
