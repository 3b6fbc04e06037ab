// packed.cu -- level-packed ILU(0) factors and the TMA-streamed Schwarz apply.
//
// Set-up repacks the factors of every subdomain in the order the triangular
// sweeps consume them: the forward rows (strict lower part) level by level,
// then the backward rows (reciprocal diagonal first, then the strict upper
// part) level by level.  Consecutive rows of one level are cut into chunks of at most
// CHUNK_BYTES; a chunk never spans two levels.  A chunk is
//     [chunk header: {nrows, ne, scale-by-diagonal flag, pad}]
//     [row headers: {local row, entry offset, entry count, pad} x nrows]
//     [16-bit local columns x ne, padded to 16 bytes]
//     [values x ne, padded to 16 bytes]
// so a whole chunk is one contiguous, 16-byte aligned copy that describes
// itself; the chunks of one subdomain are contiguous, and a table of their
// sizes (in 16-byte units) lets the copying thread walk them without reading
// global metadata on the critical path.
//
// The apply runs one CTA per subdomain: one lane of a producer warp streams
// the chunk sequence (forward then backward) into a ring of NSTAGE
// shared-memory buffers with
// cp.async.bulk (the 1-D TMA copy) and mbarrier transaction counts, NSTAGE-1
// chunks ahead; all warps consume the current chunk from shared memory
// (SW_LPR lanes per row: gather the local vector, multiply, shuffle-reduce;
// 32 / SW_LPR rows share each shuffle), release each stage warp by warp and
// meet at one barrier per level (at the level's last chunk).  The local
// vector lives in shared memory when it fits, else in a global slice.  Every
// mbarrier wait is bounded.  A wait that runs out sets an error flag; the
// producer then stops issuing, and before the CTA returns it waits (bounded)
// for the last copy it issued into each ring stage -- the only copies that
// can still be in flight, since every earlier copy into a stage was waited
// for by the consumers before the stage was refilled.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "kernels.cuh"
#include "oras.cuh"

namespace cpm {

cpm_status oras_build_transpose(oras_pc* P, cudaStream_t s);

namespace {

constexpr int CHUNK_BYTES = 24576;
constexpr int NSTAGE = 2;
constexpr int PK_WARPS = 12;       // consumer warps of a CTA (two CTAs per SM)
constexpr int PK_WARPS_FOUR = 6;   // consumer warps in the four-CTAs-per-SM mode (global slices)
constexpr unsigned WAIT_LIMIT = 1u << 22;  // polls of one mbarrier before giving up (seconds at most)

__host__ __device__ inline int64_t pad16(int64_t b) { return (b + 15) & ~(int64_t)15; }

__host__ __device__ inline int64_t chunk_bytes(int64_t nrows, int64_t ne, int vsize) {
  return 16 + 16 * nrows + pad16(2 * ne) + pad16((int64_t)vsize * ne);
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

// pass A: one thread per level cuts its rows into chunks (a chunk never spans
// two levels, so levels are independent).
// mode 0: lcnt[L] = chunks of level L.
// mode 1: write chunk records and row placements; level L of subdomain j
//         starts at chunk chbase[j] + lbase[L] - lbase[lvsub[j]].
__global__ void k_pack_plan(int32_t nl, int np, SweepSrc S, int vsize, int mode, int32_t* lcnt,
                            const int64_t* __restrict__ lbase, const int64_t* __restrict__ chbase, ChunkRec* rec,
                            int32_t* row_chunk, int32_t* row_slot, int32_t* row_eoff, int kindflag) {
  for (int32_t L = blockIdx.x * blockDim.x + threadIdx.x; L < nl; L += gridDim.x * blockDim.x) {
    int64_t c = 0;
    if (mode) {
      int lo = 0, hi = np - 1;  // the subdomain of level L: the last j with lvsub[j] <= L
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.lvsub[mid] <= L) lo = mid;
        else hi = mid - 1;
      }
      c = chbase[lo] + (lbase[L] - lbase[S.lvsub[lo]]);
    }
    int32_t cnt = 0;
    int64_t nrows = 0, ne = 0;
    for (int64_t idx = S.lvptr[L]; idx < S.lvptr[L + 1]; ++idx) {
      const int64_t q = S.lvrow[idx];
      const int64_t e = row_entries(S, q);
      if (nrows > 0 && chunk_bytes(nrows + 1, ne + e, vsize) > CHUNK_BYTES) {
        if (mode) {
          rec[c].bytes = (int32_t)chunk_bytes(nrows, ne, vsize);
          rec[c].nrows = (int32_t)nrows;
          rec[c].ne = (int32_t)ne;
          rec[c].div = kindflag;
          rec[c].lend = 0;  // more chunks of this level follow
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
        rec[c].bytes = (int32_t)chunk_bytes(nrows, ne, vsize);
        rec[c].nrows = (int32_t)nrows;
        rec[c].ne = (int32_t)ne;
        rec[c].div = kindflag;
        rec[c].lend = 1;  // the level's last chunk
      }
      ++cnt;
    }
    if (!mode) lcnt[L] = cnt;
  }
}

// chunks of subdomain j in one sweep
__global__ void k_sub_chunks(int np, const int32_t* __restrict__ lvsub, const int64_t* __restrict__ lbase,
                             int32_t* cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < np) cnt[j] = (int32_t)(lbase[lvsub[j + 1]] - lbase[lvsub[j]]);
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
    int32_t* hdr = reinterpret_cast<int32_t*>(base + 16) + 4 * row_slot[idx];
    uint16_t* cols = reinterpret_cast<uint16_t*>(base + 16 + 16 * (int64_t)R.nrows);
    if (lane == 0 && row_slot[idx] == 0) {
      int32_t* ch = reinterpret_cast<int32_t*>(base);
      ch[0] = R.nrows;
      ch[1] = R.ne;
      ch[2] = R.div;
      ch[3] = 0;
    }
    V* vals = reinterpret_cast<V*>(base + 16 + 16 * (int64_t)R.nrows + pad16(2 * (int64_t)R.ne));
    const int64_t eo = row_eoff[idx];
    const int64_t r0 = S.rptr[q], d = r0 + S.dpos[q], r1 = S.rptr[q + 1];
    const int64_t e0 = S.lower ? r0 : d + 1, e1 = S.lower ? d : r1;
    const int64_t off = S.div ? 1 : 0;
    if (lane == 0) {
      hdr[0] = (int32_t)(q - sptr[lsub[q]]);
      hdr[1] = (int32_t)eo;
      hdr[2] = (int32_t)(e1 - e0 + off);
      hdr[3] = 0;
      if (S.div) {  // the diagonal is stored as its reciprocal
        cols[eo] = 0;
        vals[eo] = (V)(1.0 / S.val[d]);
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
    int32_t* hdr = reinterpret_cast<int32_t*>(base + 16) + 4 * row_slot[idx];
    uint16_t* cols = reinterpret_cast<uint16_t*>(base + 16 + 16 * (int64_t)R.nrows);
    if (lane == 0 && row_slot[idx] == 0) {
      int32_t* ch = reinterpret_cast<int32_t*>(base);
      ch[0] = R.nrows;
      ch[1] = R.ne;
      ch[2] = R.div;
      ch[3] = 0;
    }
    __nv_bfloat16* vals = reinterpret_cast<__nv_bfloat16*>(base + 16 + 16 * (int64_t)R.nrows + pad16(2 * (int64_t)R.ne));
    const int64_t eo = row_eoff[idx];
    const int64_t r0 = S.rptr[q], d = r0 + S.dpos[q], r1 = S.rptr[q + 1];
    const int64_t e0 = S.lower ? r0 : d + 1, e1 = S.lower ? d : r1;
    const int64_t off = S.div ? 1 : 0;
    if (lane == 0) {
      hdr[0] = (int32_t)(q - sptr[lsub[q]]);
      hdr[1] = (int32_t)eo;
      hdr[2] = (int32_t)(e1 - e0 + off);
      hdr[3] = 0;
      if (S.div) {  // the diagonal is stored as its reciprocal
        cols[eo] = 0;
        vals[eo] = __float2bfloat16_rn((float)(1.0 / S.val[d]));
      }
    }
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      cols[eo + off + (e - e0)] = (uint16_t)S.col[e];
      vals[eo + off + (e - e0)] = __float2bfloat16_rn((float)S.val[e]);
    }
  }
}

__global__ void k_chunk_sizes_v(int64_t n, const ChunkRec* __restrict__ plan, int vsize, int64_t* sz) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    sz[c] = chunk_bytes(plan[c].nrows, plan[c].ne, vsize);
}
__global__ void k_chunk_place(int64_t n, const ChunkRec* __restrict__ plan, const int64_t* __restrict__ off,
                              const int64_t* __restrict__ sz, ChunkRec* rec, uint16_t* csz, int* err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    if (sz[c] > CHUNK_BYTES) atomicExch(err, 1);  // a single row larger than a stage buffer
    ChunkRec R = plan[c];
    R.off = off[c];
    R.bytes = (int32_t)sz[c];
    rec[c] = R;
    // size in 16-byte units (at most CHUNK_BYTES / 16 = 1536), top bit: the
    // chunk ends its level
    csz[c] = (uint16_t)((sz[c] >> 4) | (plan[c].lend ? 0x8000 : 0));
  }
}

// Chunk plan shared by every value type: cut with the FP64 sizes, so the
// chunks of narrower types fit the budget too.
struct Plan {
  int64_t nch = 0, max_chunks = 0;
  ChunkRec* rec = nullptr;   // nrows, ne, div per chunk
  int64_t* chsub = nullptr;  // [np+1]
  int32_t* rc[2] = {nullptr, nullptr};  // per sweep and schedule position: chunk, slot, entry offset
  int32_t* rs[2] = {nullptr, nullptr};
  int32_t* re[2] = {nullptr, nullptr};
  void release(cudaStream_t s) {
    dfree(rec, s);
    dfree(chsub, s);
    for (int w = 0; w < 2; ++w) {
      dfree(rc[w], s);
      dfree(rs[w], s);
      dfree(re[w], s);
    }
  }
};

cpm_status make_plan(oras_pc* P, const SweepSrc* sw, int vsize, Plan& pl, cudaStream_t s) {
  const int np = P->np;
  const int64_t nloc = P->nloc;
  int32_t* cnt = nullptr;
  int32_t* lcnt[2] = {nullptr, nullptr};
  int64_t* lbase[2] = {nullptr, nullptr};
  int64_t* chbase[2] = {nullptr, nullptr};
  int32_t nl[2] = {0, 0};
  CPM_TRY(dalloc(&cnt, np, s));
  std::vector<int32_t> hc[2];
  for (int w = 0; w < 2; ++w) {
    CPM_CUDA(cudaMemcpyAsync(&nl[w], sw[w].lvsub + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
    CPM_TRY(dalloc(&lcnt[w], std::max<int32_t>(nl[w], 1), s));
    CPM_TRY(dalloc(&lbase[w], (int64_t)nl[w] + 1, s));
    if (nl[w] > 0)
      KL(k_pack_plan<<<grid_for(nl[w], 128), 128, 0, s>>>(nl[w], np, sw[w], vsize, 0, lcnt[w], nullptr, nullptr,
                                                          nullptr, nullptr, nullptr, nullptr, sw[w].div));
    CPM_TRY(scan_exclusive_i32(lcnt[w], lbase[w], nl[w], s));
    KL(k_sub_chunks<<<(np + 127) / 128, 128, 0, s>>>(np, sw[w].lvsub, lbase[w], cnt));
    hc[w].resize(np);
    CPM_CUDA(cudaMemcpyAsync(hc[w].data(), cnt, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int64_t> chsub(np + 1, 0), hbase[2];
  pl.max_chunks = 0;
  hbase[0].resize(np);
  hbase[1].resize(np);
  for (int j = 0; j < np; ++j) {
    hbase[0][j] = chsub[j];
    hbase[1][j] = chsub[j] + hc[0][j];
    chsub[j + 1] = chsub[j] + hc[0][j] + hc[1][j];
    pl.max_chunks = std::max<int64_t>(pl.max_chunks, hc[0][j] + hc[1][j]);
  }
  pl.nch = chsub[np];
  CPM_TRY(dalloc(&pl.rec, std::max<int64_t>(pl.nch, 1), s));
  CPM_TRY(dalloc(&pl.chsub, np + 1, s));
  CPM_CUDA(cudaMemcpyAsync(pl.chsub, chsub.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  for (int w = 0; w < 2; ++w) {
    CPM_TRY(dalloc(&chbase[w], np, s));
    CPM_CUDA(cudaMemcpyAsync(chbase[w], hbase[w].data(), np * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CPM_TRY(dalloc(&pl.rc[w], nloc, s));
    CPM_TRY(dalloc(&pl.rs[w], nloc, s));
    CPM_TRY(dalloc(&pl.re[w], nloc, s));
    if (nl[w] > 0)
      KL(k_pack_plan<<<grid_for(nl[w], 128), 128, 0, s>>>(nl[w], np, sw[w], vsize, 1, nullptr, lbase[w], chbase[w],
                                                          pl.rec, pl.rc[w], pl.rs[w], pl.re[w], sw[w].div));
  }
  CPM_CUDA(cudaGetLastError());
  CPM_CUDA(cudaStreamSynchronize(s));
  dfree(cnt, s);
  for (int w = 0; w < 2; ++w) {
    dfree(lcnt[w], s);
    dfree(lbase[w], s);
    dfree(chbase[w], s);
  }
  return CPM_OK;
}

template <typename V>
cpm_status emit(oras_pc* P, const SweepSrc* sw, const Plan& pl, PackedFactors& out, cudaStream_t s) {
  const int np = P->np;
  const int64_t nch = pl.nch;
  int64_t *sz = nullptr, *off = nullptr;
  CPM_TRY(dalloc(&sz, nch, s));
  CPM_TRY(dalloc(&off, nch + 1, s));
  CPM_TRY(dalloc(&out.rec, nch, s));
  CPM_TRY(dalloc(&out.csz, nch, s));
  out.max_chunks = pl.max_chunks;
  CPM_TRY(dalloc(&out.chsub, np + 1, s));
  CPM_CUDA(cudaMemcpyAsync(out.chsub, pl.chsub, (np + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  {
    // launch order: longest subdomains first, so the last wave holds the short ones
    std::vector<int64_t> hs(np + 1);
    CPM_CUDA(cudaMemcpyAsync(hs.data(), pl.chsub, (np + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> ord(np);
    for (int q = 0; q < np; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int32_t a, int32_t b) { return hs[a + 1] - hs[a] > hs[b + 1] - hs[b]; });
    CPM_TRY(dalloc(&out.order, np, s));
    CPM_CUDA(cudaMemcpyAsync(out.order, ord.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CPM_CUDA(cudaStreamSynchronize(s));
  }
  KL(k_chunk_sizes_v<<<grid_for(nch, 256), 256, 0, s>>>(nch, pl.rec, (int)sizeof(V), sz));
  CPM_TRY(scan_exclusive_i64(sz, off, nch, s));
  int* err = nullptr;
  CPM_TRY(dalloc(&err, 1, s));
  CPM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  KL(k_chunk_place<<<grid_for(nch, 256), 256, 0, s>>>(nch, pl.rec, off, sz, out.rec, out.csz, err));
  int herr = 0;
  CPM_CUDA(cudaMemcpyAsync(&out.bytes, off + nch, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  dfree(err, s);
  if (herr) return fail(CPM_ERR_ARG, "a factor row does not fit one %d-byte chunk", CHUNK_BYTES);
  out.nchunks = nch;
  CPM_TRY(dalloc(&out.data, out.bytes, s));
  for (int w = 0; w < 2; ++w)
    KL(k_pack_write<V><<<grid_for(P->nloc * 32, 256), 256, 0, s>>>(P->nloc, sw[w], P->sptr, P->lsub, out.rec,
                                                                  pl.rc[w], pl.rs[w], pl.re[w], out.data));
  CPM_CUDA(cudaGetLastError());
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
  else if constexpr (std::is_same<V, __half>::value) return (T)__half2float(v);
  else return (T)v;
}
// store a sweep value in the local vector's type (FP16: round to nearest)
template <typename X, typename T>
__device__ __forceinline__ X to_x(T v) {
  if constexpr (std::is_same<X, __half>::value) return __float2half_rn((float)v);
  else return (X)v;
}

// FP16 local vector: the entries of R_j r are scaled by a power of two that
// puts the largest one in [2^(XS_EXP-1), 2^XS_EXP) = [1, 2), which leaves a
// factor of about 2^15 of FP16's range (largest finite 65504) for growth in
// the sweeps -- smooth vectors grow 25-65x through the ILU(0) sweeps of the
// torus at h = 0.0125, and more on finer grids -- while entries down to 2^-14
// of the largest keep FP16's full precision.
constexpr int XS_EXP = 1;
__device__ __forceinline__ float pow2_scale(float amax) {
  const int be = (__float_as_int(amax) >> 23) & 0xff;  // biased exponent: amax in [2^(be-127), 2^(be-126))
  if (!(amax > 0.f) || be == 0xff) return 1.f;
  const int k = max(-120, min(120, XS_EXP + 126 - be));
  return __int_as_float((127 + k) << 23);
}

struct PkArgs {
  const int32_t* order;  // subdomains by decreasing chunk count (longest first)
  const uint16_t* csz;
  int64_t csz_bytes;  // shared-memory bytes reserved for the chunk-size table
  const int64_t* sptr;
  const int32_t* snode;
  const uint8_t* owned;
  const int64_t* chsub;
  const ChunkRec* rec;
  const uint8_t* data;
  int transpose;
  int64_t nA, nloc;
  int* err;
  uint32_t wait_limit;  // polls of each consumer-side wait before it gives up
  int probe;            // failure-path test: the first chunk wait waits on a barrier nothing completes
  int natural;          // subdomains in partition order instead of longest first
  float xsigma;         // FP16 local vector: power of two at the binade of the diagonal scale c + 6/h^2
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// barrier among the NW consumer warps only (named barrier 1)
template <int NW>
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NW * 32) : "memory");
}
// the same barrier, returning the OR of every consumer thread's v: all
// consumers get the same answer, so they stop at the same chunk
template <int NW>
__device__ __forceinline__ bool consumer_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NW * 32)
      : "memory");
  return r != 0;
}

// partial dot product of one packed row with the local vector: lane `sub`
// of the row's LPR lanes takes entries e0 + sub, e0 + sub + LPR, ...  UNR
// entries are loaded before they are used, so UNR gathers of the local
// vector are in flight at once: a few for a local vector in shared memory
// (short latency), enough to cover a whole row when it lives in a global
// slice (one L2 round trip per row instead of several).
template <typename T, typename V, int LPR, int UNR, typename X>
__device__ __forceinline__ T row_dot(const int4 h, int e0, int sub, const V* vals, const uint16_t* cols,
                                     const X* xs) {
  T s = 0;
#pragma unroll UNR
  for (int e = e0 + sub; e < h.z; e += LPR) s += cvt<V, T>(vals[h.y + e]) * cvt<X, T>(xs[cols[h.y + e]]);
  return s;
}

// lanes per factor row in the Schwarz sweeps (a run-time choice among 4, 8
// and 16): 32 / LPR rows share each shuffle of the row reductions.  Lower
// and upper rows hold ~60 entries each.
constexpr int SW_LPR_SMEM = 8;    // local vector in shared memory: measured best on the 512-part torus
constexpr int SW_LPR_GLOBAL = 8;  // global slice: 8 also measured best (4 lanes: 1.3x slower at h = 0.002)

// Warps 0..PK_WARPS-1 consume chunks; warp PK_WARPS produces them (one lane
// issues the bulk copies).  full[s]: a chunk landed in stage s (transaction
// count); empty[s]: the consumers finished with stage s.
//
// XT is the type of the local vector: T, or FP16 (in shared memory only, for
// FP32 applies whose subdomains do not fit there in FP32).  With FP16 the
// entries of R_j r are scaled by alpha (pow2_scale) and the rows that carry a
// reciprocal pivot d compute (x_i * sigma - sum) * d, with sigma the power of
// two at the binade of the diagonal scale c + 6/h^2 (the ILU(0) pivots lie
// within a small factor of it), so that their results (x_i / pivot ~ 1e-6 x_i
// on the benchmark grids) stay in FP16's normal range; the output is unscaled
// by 1 / (alpha * sigma), both powers of two.  sigma comes from the host, so
// the rounding does not depend on the order of rows within a level.
template <int NW, typename XT>
constexpr int pk_min_blocks() {
  return NW == PK_WARPS_FOUR ? 4 : (std::is_same<XT, __half>::value ? 1 : 2);
}

template <typename T, typename V, bool SMEMX, int SW_LPR, int NW = PK_WARPS, typename XT = T>
__global__ void __launch_bounds__((NW + 1) * 32, pk_min_blocks<NW, XT>())
    k_schwarz_pk(PkArgs A, const T* __restrict__ r, T* __restrict__ z, T* xglob) {
  constexpr bool HX = std::is_same<XT, __half>::value;
  static_assert(SMEMX || std::is_same<XT, T>::value, "a global slice holds the apply's own type");
  extern __shared__ __align__(128) unsigned char pk_smem[];
  __shared__ uint64_t full[NSTAGE], empty[NSTAGE], probe_bar;
  __shared__ int abort_flag;
  __shared__ float xred[HX ? NW : 1];  // FP16: per-warp maxima of |R_j r|
  __shared__ T xout;                   // FP16: 1 / (alpha * sigma), set by consumer thread 0
  int64_t issued = 0;  // chunks the producer lane has issued (used by its drain)
  const int j = A.natural ? (int)blockIdx.x : A.order[blockIdx.x], rhs = blockIdx.y;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const bool producer = wid == NW;
  r += (int64_t)rhs * A.nA;
  z += (int64_t)rhs * A.nA;
  unsigned char* ring = pk_smem;
  uint16_t* csz = reinterpret_cast<uint16_t*>(pk_smem + NSTAGE * CHUNK_BYTES);  // chunk sizes / 16
  const int64_t base = A.sptr[j], n = A.sptr[j + 1] - base;
  XT* xs = SMEMX ? reinterpret_cast<XT*>(pk_smem + NSTAGE * CHUNK_BYTES + A.csz_bytes)
                 : reinterpret_cast<XT*>(xglob + (int64_t)rhs * A.nloc + base);
  const int64_t c0 = A.chsub[j], nch = A.chsub[j + 1] - c0;
  for (int64_t c = tid; c < nch; c += blockDim.x) csz[c] = A.csz[c0 + c];
  if (tid == 0) {
    abort_flag = 0;
    for (int q = 0; q < NSTAGE; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], NW);  // one arrival per consumer warp
    }
    mbar_init(&probe_bar, 1);  // never arrived on: a wait on it can only run out
    fence_mbar_init();
  }
  __syncthreads();
  if (producer) {
    if (lane == 0) {
      int64_t off = nch > 0 ? A.rec[c0].off : 0;
      for (int64_t c = 0; c < nch; ++c) {
        const int st = (int)(c % NSTAGE);
        if (c >= NSTAGE) {  // wait until the consumers released this stage
          unsigned polls = 0;
          bool ok = true;
          while (!mbar_try_wait(&empty[st], (uint32_t)(((c / NSTAGE) - 1) & 1)))
            if (++polls > WAIT_LIMIT) {
              ok = false;
              break;
            }
          if (!ok || *(volatile int*)&abort_flag) {
            abort_flag = 1;
            break;
          }
        }
        const uint32_t bytes = (uint32_t)(csz[c] & 0x7fff) << 4;
        fence_proxy_async();
        mbar_expect_tx(&full[st], bytes);
        bulk_g2s(ring + st * CHUNK_BYTES, A.data + off, bytes, &full[st]);
        off += bytes;
        ++issued;
      }
    }
  } else {
    T alpha = 1, sigma = 1;  // FP16 scales (1 otherwise)
    if constexpr (HX) {
      sigma = A.xsigma;
      float amax = 0.f;
      for (int64_t q = tid; q < n; q += NW * 32)
        if (!(A.transpose && !A.owned[base + q])) amax = fmaxf(amax, fabsf((float)r[A.snode[base + q]]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      if (lane == 0) xred[wid] = amax;
      consumer_sync<NW>();
      amax = 0.f;
      for (int w = 0; w < NW; ++w) amax = fmaxf(amax, xred[w]);
      alpha = pow2_scale(amax);
    }
    for (int64_t q = tid; q < n; q += NW * 32) {
      T v = r[A.snode[base + q]];
      if constexpr (HX) v = v * alpha;
      xs[q] = to_x<XT>((A.transpose && !A.owned[base + q]) ? (T)0 : v);
    }
    consumer_sync<NW>();
    for (int64_t c = 0; c < nch; ++c) {
      const int st = (int)(c % NSTAGE);
      const bool probe = A.probe && c == 0;
      uint64_t* bar = probe ? &probe_bar : &full[st];
      const uint32_t par = probe ? 0u : (uint32_t)((c / NSTAGE) & 1);
      unsigned polls = 0;
      while (!mbar_try_wait(bar, par)) {
        if (++polls > A.wait_limit) {
          abort_flag = 1;
          break;
        }
      }
      const unsigned char* buf = ring + st * CHUNK_BYTES;
      const int4 ch = *reinterpret_cast<const int4*>(buf);  // {nrows, ne, scale-by-diagonal flag, pad}
      const int4* hdr = reinterpret_cast<const int4*>(buf + 16);
      const uint16_t* cols = reinterpret_cast<const uint16_t*>(buf + 16 + 16 * (int64_t)ch.x);
      const V* vals = reinterpret_cast<const V*>(buf + 16 + 16 * (int64_t)ch.x + pad16(2 * (int64_t)ch.y));
      // skip the chunk when this warp saw the abort (decided per warp, so
      // that either all lanes or none reach the shuffles below)
      if (!__any_sync(0xffffffffu, *(volatile int*)&abort_flag != 0)) {
        constexpr int LPR = SW_LPR, RPW = 32 / LPR;  // lanes per row, rows per warp
        const int e0 = ch.z ? 1 : 0, sub = lane & (LPR - 1);
        // rows rb + RPW * wid + lane / LPR; the loop is warp-uniform so that
        // every lane reaches the shuffles
        for (int rb = 0; rb < ch.x; rb += RPW * NW) {
          const int rr = rb + RPW * wid + lane / LPR;
          const bool has = rr < ch.x;
          int4 h = make_int4(0, 0, 0, 0);
          T sdot = 0;
          if (has) {
            h = hdr[rr];
            sdot = row_dot<T, V, LPR, (SMEMX ? 4 : 64 / LPR), XT>(h, e0, sub, vals, cols, xs);
          }
#pragma unroll
          for (int o = LPR / 2; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
          if (has && sub == 0) {
            T v = cvt<XT, T>(xs[h.x]);
            if constexpr (HX) {
              if (ch.z) v = v * sigma;
            }
            v = v - sdot;
            if (ch.z) v = v * cvt<V, T>(vals[h.y]);
            xs[h.x] = to_x<XT>(v);
          }
        }
      }
      // this warp is done reading the stage
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      // Rows of one level are independent, so the consumers meet only at the
      // last chunk of a level (the next level reads its results), and take one
      // abort decision there for all of them: the producer may set the flag at
      // any time.  The level ends come from the chunk-size table that every
      // thread copied before the loop, so all warps meet at the same chunks
      // even when a wait ran out.
      if (csz[c] >> 15) {
        const bool stop = consumer_sync_or<NW>(*(volatile int*)&abort_flag != 0);
        if (stop) {
          abort_flag = 1;
          break;
        }
      }
    }
    if constexpr (HX) {
      if (tid == 0) xout = ((T)1 / alpha) * ((T)1 / sigma);  // powers of two: exact
    }
  }
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) atomicExch(A.err, CPM_ERR_TIMEOUT);
    // Drain before the shared memory goes away.  Chunk c went into stage
    // c % NSTAGE and completes phase c / NSTAGE of full[stage].  Only the
    // last chunk issued into each stage can still be in flight (the producer
    // refills a stage only after the consumers released it, and they stop at
    // the first wait that runs out), so wait for that chunk's phase.
    if (producer && lane == 0)
      for (int q = 0; q < NSTAGE && q < issued; ++q) {
        const int64_t last = q + (int64_t)NSTAGE * ((issued - 1 - q) / NSTAGE);
        const uint32_t par = (uint32_t)((last / NSTAGE) & 1);
        unsigned polls = 0;
        while (!mbar_try_wait(&full[q], par) && ++polls < WAIT_LIMIT) {
        }
      }
    return;
  }
  T unscale = 1;
  if constexpr (HX) unscale = xout;
  if (!A.transpose) {
    for (int64_t q = tid; q < n; q += blockDim.x)
      if (A.owned[base + q]) z[A.snode[base + q]] = cvt<XT, T>(xs[q]) * unscale;
  } else if (SMEMX) {
    T* xg = xglob + (int64_t)rhs * A.nloc + base;
    for (int64_t q = tid; q < n; q += blockDim.x) xg[q] = cvt<XT, T>(xs[q]) * unscale;
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

// Build level-packed factors (forward rows, then backward rows) from the CSR
// factors, one packed stream per requested value type (nout of them, types
// vt[]); transposed selects the transposed factors (U^T with its diagonal
// first, then L^T).
cpm_status pack_factors(oras_pc* P, int transposed, const cpm_dtype* vt, PackedFactors* out, int nout,
                        cudaStream_t s) {
  if (P->max_rows > 65535)
    return fail(CPM_ERR_ARG, "subdomain of %lld rows exceeds 16-bit local columns", (long long)P->max_rows);
  SweepSrc sw[2];
  if (!transposed) {
    sw[0] = {P->rptr, P->col, P->dpos, P->val, P->lvsub_f, P->lvptr_f, P->lvrow_f, 1, 0};
    sw[1] = {P->rptr, P->col, P->dpos, P->val, P->lvsub_b, P->lvptr_b, P->lvrow_b, 0, 1};
  } else {
    sw[0] = {P->tptr, P->tcol, P->tdpos, P->tval, P->lvsub_tf, P->lvptr_tf, P->lvrow_tf, 1, 1};
    sw[1] = {P->tptr, P->tcol, P->tdpos, P->tval, P->lvsub_tb, P->lvptr_tb, P->lvrow_tb, 0, 0};
  }
  cpm_status st = CPM_OK;
  for (int k = 0; k < nout && st == CPM_OK; ++k) {
    // chunks are cut per value type so that every type fills the budget
    const int vsize = vt[k] == CPM_F64 ? 8 : (vt[k] == CPM_F32 ? 4 : 2);
    Plan pl;
    st = make_plan(P, sw, vsize, pl, s);
    out[k].vtype = vt[k];
    if (st == CPM_OK) {
      if (vt[k] == CPM_F64) st = emit<double>(P, sw, pl, out[k], s);
      else if (vt[k] == CPM_F32) st = emit<float>(P, sw, pl, out[k], s);
      else st = emit<__nv_bfloat16>(P, sw, pl, out[k], s);
    }
    cudaStreamSynchronize(s);
    pl.release(s);
  }
  return st;
}

void packed_free(PackedFactors& pf, cudaStream_t s) {
  dfree(pf.data, s);
  dfree(pf.order, s);
  dfree(pf.rec, s);
  dfree(pf.csz, s);
  dfree(pf.chsub, s);
  pf.nchunks = 0;
  pf.bytes = 0;
}

// Largest dynamic shared memory a Schwarz CTA asks for: the ring and the
// chunk-size table, plus the local vector when it lives in shared memory
// (at most 113 KB in total, so that two CTAs fit on one SM).
constexpr size_t PK_SMEM_MAX = 113 * 1024;
// ... and with an FP16 local vector (one CTA per SM): up to the 227 KB a CTA
// may have, less a margin for the kernel's static shared memory
constexpr size_t PK_SMEM_HALF = 226 * 1024;
constexpr int PK_WARPS_WIDE = 24;  // consumer warps of the FP16 variant with xplace 3

// Raise the kernels' dynamic shared-memory limit once per device (the
// attribute is a ceiling; each launch asks for what it needs).
template <typename T, typename V>
static cpm_status allow_pk_smem(cudaStream_t) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  CPM_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return CPM_OK;
  const void* fns[6] = {(const void*)k_schwarz_pk<T, V, true, 4>,  (const void*)k_schwarz_pk<T, V, true, 8>,
                        (const void*)k_schwarz_pk<T, V, true, 16>, (const void*)k_schwarz_pk<T, V, false, 4>,
                        (const void*)k_schwarz_pk<T, V, false, 8>, (const void*)k_schwarz_pk<T, V, false, 16>};
  for (const void* f : fns)
    CPM_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PK_SMEM_MAX));
  CPM_CUDA(cudaFuncSetAttribute((const void*)k_schwarz_pk<T, V, false, 8, PK_WARPS_FOUR>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PK_SMEM_MAX));
  if constexpr (std::is_same<T, float>::value) {
    CPM_CUDA(cudaFuncSetAttribute((const void*)k_schwarz_pk<float, V, true, 8, PK_WARPS, __half>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PK_SMEM_HALF));
    CPM_CUDA(cudaFuncSetAttribute((const void*)k_schwarz_pk<float, V, true, 8, PK_WARPS_WIDE, __half>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PK_SMEM_HALF));
  }
  done.fetch_or(bit);
  return CPM_OK;
}

// Shared-memory carve-out of the one-CTA-per-SM mode (percent of the largest
// carve-out: 28 % is the 64 KB configuration) and the dynamic shared memory
// it requests so that a second CTA cannot fit beside the first.
constexpr int PK_CARVE_ONE = 28;
constexpr size_t PK_SMEM_ONE = 60 * 1024;

template <typename T, typename V, bool SMEMX, int L, int NW = PK_WARPS, typename XT = T>
static void launch_pk_l(int carve, dim3 g, size_t sm, cudaStream_t s, const PkArgs& A, const T* r, T* z, T* xl) {
  constexpr int NT = (NW + 1) * 32;
  cudaFuncSetAttribute(k_schwarz_pk<T, V, SMEMX, L, NW, XT>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
  KL(k_schwarz_pk<T, V, SMEMX, L, NW, XT><<<g, NT, sm, s>>>(A, r, z, xl));
}

// ctas 4 (global slices only): four CTAs per SM of PK_WARPS_FOUR consumer
// warps each, 8 lanes per row, so that up to 608 subdomains run at once
template <typename T, typename V, bool SMEMX>
static void launch_pk(int lanes, int ctas, int carve, dim3 g, size_t sm, cudaStream_t s, const PkArgs& A, const T* r,
                      T* z, T* xl) {
  if (!SMEMX && ctas == 4) launch_pk_l<T, V, false, 8, PK_WARPS_FOUR>(carve, g, sm, s, A, r, z, xl);
  else if (lanes == 4) launch_pk_l<T, V, SMEMX, 4>(carve, g, sm, s, A, r, z, xl);
  else if (lanes == 16) launch_pk_l<T, V, SMEMX, 16>(carve, g, sm, s, A, r, z, xl);
  else launch_pk_l<T, V, SMEMX, 8>(carve, g, sm, s, A, r, z, xl);
}

// FP16 local vector (FP32 applies only): 8 lanes per row, 12 or (wide) 24
// consumer warps, one CTA per SM
template <typename T, typename V>
static void launch_pk_half(bool wide, int carve, dim3 g, size_t sm, cudaStream_t s, const PkArgs& A, const T* r,
                           T* z, T* xl) {
  if constexpr (std::is_same<T, float>::value) {
    if (wide) launch_pk_l<float, V, true, 8, PK_WARPS_WIDE, __half>(carve, g, sm, s, A, r, z, xl);
    else launch_pk_l<float, V, true, 8, PK_WARPS, __half>(carve, g, sm, s, A, r, z, xl);
  }
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
  A.order = pf.order;
  A.csz = pf.csz;
  A.csz_bytes = pad16(2 * pf.max_chunks);
  A.wait_limit = P->wait_polls > 0 ? (uint32_t)std::min<int64_t>(P->wait_polls, 0xffffffffll) : WAIT_LIMIT;
  A.probe = P->probe_timeout;
  A.natural = P->schedule == 1;
  {  // 2^(e-1) <= c + 6/h^2 < 2^e
    int e = 0;
    std::frexp(std::fabs(P->c) + 6.0 / (P->band->h * P->band->h), &e);
    A.xsigma = (float)std::ldexp(1.0, std::max(-100, std::min(100, e - 1)));
  }
  const size_t ring = (size_t)NSTAGE * CHUNK_BYTES + A.csz_bytes;
  const size_t xsb = (size_t)P->max_rows * sizeof(T);
  // local vector in shared memory when it fits beside the ring with two CTAs
  // per SM, unless the caller asked for the global slice
  const bool smemx = P->xplace != 1 && ring + xsb <= PK_SMEM_MAX;
  // else, for FP32 applies with xplace 2 or 3, an FP16 local vector in shared
  // memory (one CTA per SM) when that fits
  const bool smemh = std::is_same<T, float>::value && !smemx && (P->xplace == 2 || P->xplace == 3) &&
                     ring + (size_t)P->max_rows * 2 <= PK_SMEM_HALF;
  // one CTA per SM with a small shared-memory carve-out (the rest of the SM's
  // memory is L1, which then holds most of one subdomain's global slice)
  // CTAs per SM for global slices: one by default (measured 9 % faster than two
  // at h = 0.002, where two 230 KB slices per SM overflow L1)
  const int ctas = P->ctas ? P->ctas : 1;
  const bool one_cta = !smemx && !smemh && ctas == 1 && ring <= PK_SMEM_ONE;
  const bool four = !smemx && !smemh && ctas == 4 && 4 * ring <= 220 * 1024;
  const size_t sm = smemh ? ring + pad16((int64_t)P->max_rows * 2)
                          : (smemx ? ring + xsb : (one_cta ? PK_SMEM_ONE : ring));
  const int carve = one_cta ? PK_CARVE_ONE
                            : ((four || smemh) ? (int)cudaSharedmemCarveoutMaxShared : (int)cudaSharedmemCarveoutDefault);
  if (sm > (smemh ? PK_SMEM_HALF : PK_SMEM_MAX))
    return fail(CPM_ERR_ARG, "Schwarz apply needs %zu bytes of shared memory", sm);
  CPM_TRY((allow_pk_smem<T, V>(s)));
  T* xloc = nullptr;
  if ((!smemx && !smemh) || transpose) CPM_TRY(dalloc(&xloc, (size_t)nrhs * P->nloc, s));
  for (int r0 = 0; r0 < nrhs; r0 += 65535) {
    const int nr = nrhs - r0 < 65535 ? nrhs - r0 : 65535;
    dim3 g(P->np, nr);
    T* xl = xloc ? xloc + (int64_t)r0 * P->nloc : nullptr;
    const int lanes = P->lanes ? P->lanes : (smemx ? SW_LPR_SMEM : SW_LPR_GLOBAL);
    const T* rr = r + (int64_t)r0 * P->nA;
    T* zz = z + (int64_t)r0 * P->nA;
    if (smemh) launch_pk_half<T, V>(P->xplace == 3, carve, g, sm, s, A, rr, zz, xl);
    else if (smemx) launch_pk<T, V, true>(lanes, 0, carve, g, sm, s, A, rr, zz, xl);
    else launch_pk<T, V, false>(lanes, four ? 4 : 0, carve, g, sm, s, A, rr, zz, xl);
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

// Autotuner of the apply: every (placement, lanes, schedule) combination
// that the preconditioner allows, timed on reps forward applies of a zero
// vector (the sweeps' work does not depend on the values), fastest kept.
cpm_status oras_tune(oras_pc* P, cpm_dtype dt, int reps, cudaStream_t s, oras_tuning* best, double* best_ms) {
  if (dt == CPM_F32 && P->store == CPM_F64)
    return fail(CPM_ERR_ARG, "FP32 applies need factors stored as CPM_F32 or CPM_BF16");
  const size_t esz = dt == CPM_F64 ? 8 : 4;
  const int saved_probe = P->probe_timeout;
  P->probe_timeout = 0;
  void *r = nullptr, *z = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto done = [&](cpm_status st) {
    dfree(r, s);
    dfree(z, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    P->probe_timeout = saved_probe;
    return st;
  };
  cpm_status st;
  if ((st = dalloc((uint8_t**)&r, P->nA * esz, s)) != CPM_OK) return done(st);
  if ((st = dalloc((uint8_t**)&z, P->nA * esz, s)) != CPM_OK) return done(st);
  if (cudaMemsetAsync(r, 0, P->nA * esz, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    return done(fail(CPM_ERR_CUDA, "autotune set-up failed"));
  oras_tuning keep{P->xplace, P->lanes, P->schedule, P->ctas, 0, P->wait_polls}, win = keep;
  double win_ms = 1e300;
  const int lanes[3] = {4, 8, 16};
  if ((st = oras_run(P, r, z, dt, 1, 0, s)) != CPM_OK) return done(st);  // packs this precision if needed
  const size_t ring = (size_t)NSTAGE * CHUNK_BYTES + pad16(2 * P->packed[dt == CPM_F64 ? 0 : 1].max_chunks);
  const bool fits = ring + (size_t)P->max_rows * esz <= PK_SMEM_MAX;
  for (int xp = 0; xp < 2; ++xp)
    for (int li = 0; li < 3; ++li)
      for (int sc = 0; sc < 2; ++sc)
        for (int ci = 0; ci < 3; ++ci) {
        const int ctas = ci == 0 ? 2 : (ci == 1 ? 1 : 4);
        if (ctas != 2 && xp == 0 && fits) continue;  // CTAs per SM only vary for global slices
        if (ctas == 4 && lanes[li] != 8) continue;    // the four-CTA kernel uses 8 lanes per row
        P->xplace = xp;
        P->lanes = lanes[li];
        P->schedule = sc;
        P->ctas = ctas;
        if ((st = oras_run(P, r, z, dt, 1, 0, s)) != CPM_OK) return done(st);  // warm-up (packs on first use)
        cudaEventRecord(e0, s);
        for (int q = 0; q < reps; ++q)
          if ((st = oras_run(P, r, z, dt, 1, 0, s)) != CPM_OK) return done(st);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return done(fail(CPM_ERR_CUDA, "autotune timing failed"));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < win_ms) {
          win_ms = ms / reps;
          win = oras_tuning{xp, lanes[li], sc, ctas, 0, keep.wait_polls};
        }
      }
  if ((st = oras_take_error(P, s)) != CPM_OK) {
    P->xplace = keep.xplace;
    P->lanes = keep.lanes;
    P->schedule = keep.schedule;
    P->ctas = keep.ctas;
    return done(st);
  }
  P->xplace = win.xplace;
  P->lanes = win.lanes;
  P->schedule = win.schedule;
  P->ctas = win.ctas;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return done(CPM_OK);
}

cpm_status oras_take_error(const oras_pc* P, cudaStream_t s) {
  if (!P) return CPM_OK;
  int herr = 0;
  CPM_CUDA(cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if (!herr) return CPM_OK;
  CPM_CUDA(cudaMemsetAsync(P->err, 0, sizeof(int), s));
  CPM_CUDA(cudaStreamSynchronize(s));
  return fail(CPM_ERR_TIMEOUT, "a bounded wait in the Schwarz apply ran out");
}

cpm_status oras_run(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose, cudaStream_t s) {
  if (dt == CPM_F32 && !transpose && P->store == CPM_F64)
    return fail(CPM_ERR_ARG, "FP32 apply needs factors stored as CPM_F32 or CPM_BF16");
  if (P->coarse) return coarse_apply(P, r, z, dt, nrhs, transpose, s);
  return oras_run_one_level(P, r, z, dt, nrhs, transpose, s);
}

cpm_status oras_run_one_level(const oras_pc* Pc, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose,
                              cudaStream_t s) {
  oras_pc* P = const_cast<oras_pc*>(Pc);
  if (dt == CPM_F32 && !transpose && P->store == CPM_F64)
    return fail(CPM_ERR_ARG, "FP32 apply needs factors stored as CPM_F32 or CPM_BF16");
  if (transpose) CPM_TRY(oras_build_transpose(P, s));
  const int slot = (transpose ? 2 : 0) + (dt == CPM_F32 ? 1 : 0);
  PackedFactors& pf = P->packed[slot];
  if (!pf.data) {
    const cpm_dtype vt = dt == CPM_F64 ? CPM_F64 : (transpose ? CPM_F32 : (cpm_dtype)P->store);
    CPM_TRY(pack_factors(P, transpose, &vt, &pf, 1, s));
  }
  if (dt == CPM_F64) return run_pk<double, double>(P, pf, (const double*)r, (double*)z, nrhs, transpose, s);
  if (pf.vtype == CPM_BF16)
    return run_pk<float, __nv_bfloat16>(P, pf, (const float*)r, (float*)z, nrhs, transpose, s);
  return run_pk<float, float>(P, pf, (const float*)r, (float*)z, nrhs, transpose, s);
}

}  // namespace cpm
