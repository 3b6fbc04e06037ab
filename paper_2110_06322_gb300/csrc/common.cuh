// common.cuh -- internal definitions shared by the libcpm translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "cpm.h"

namespace cpm {

// every kernel launch of the library goes through KL(...) so that callers can
// count the kernels of a region (cpm_kernel_launches)
extern std::atomic<long long> g_launches;
extern std::atomic<long long> g_allocs;  // device allocations made (cpm_device_allocations)
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
#define KL(...) ::cpm::count_launch(), __VA_ARGS__

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
cpm_status fail(cpm_status st, const char* fmt, ...);
cpm_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define CPM_CUDA(call)                                                     \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return ::cpm::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define CPM_TRY(expr)                    \
  do {                                   \
    cpm_status s_ = (expr);              \
    if (s_ != CPM_OK) return s_;         \
  } while (0)

// Raise the release threshold of the current device's default memory pool
// (once per device), so freed working memory stays in the pool for reuse.
void keep_pool_memory();

// Device allocation that reports CPM_ERR_OOM.  Stream-ordered.
template <typename T>
cpm_status dalloc(T** p, size_t n, cudaStream_t s) {
  *p = nullptr;
  if (n == 0) n = 1;
  keep_pool_memory();
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaMallocAsync((void**)p, n * sizeof(T), s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(CPM_ERR_OOM, "device allocation of %zu bytes failed", n * sizeof(T));
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
  return CPM_OK;
}

template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync((void*)p, s);
  p = nullptr;
}

// two buffers of `bytes` bytes each, starting at a and b, share a byte
inline bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return bytes > 0 && pa < pb + bytes && pb < pa + bytes;
}

inline int grid_for(int64_t n, int block, int64_t cap = 152 * 64) {
  int64_t g = (n + block - 1) / block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// ------------------------------------------------------------------ lattice bitmaps
// A set of lattice cells stored as one bit per cell over a dense box grid
// (origin glo, extents gn), k fastest.  Each k-column is padded to whole
// 64-bit words; `pre` holds the number of set bits before the word, so the
// canonical rank of a member cell is pre + popcount of the bits below it.
struct __align__(16) BitWord {
  unsigned long long bits;
  int32_t pre;
  int32_t pad;
};

struct Grid {
  int glo[3];
  int gn[3];
  int nkw;  // 64-bit words per k-column
  __host__ __device__ int64_t nwords() const { return (int64_t)gn[0] * gn[1] * nkw; }
};

// rank of lattice cell (i,j,k) in a bitmap, or -1 when absent / outside
__device__ __forceinline__ int32_t bm_rank(const BitWord* __restrict__ bm, const Grid& g, int i, int j, int k) {
  int a = i - g.glo[0], b = j - g.glo[1], c = k - g.glo[2];
  if ((unsigned)a >= (unsigned)g.gn[0] || (unsigned)b >= (unsigned)g.gn[1] || (unsigned)c >= (unsigned)(g.nkw * 64))
    return -1;
  int64_t w = ((int64_t)a * g.gn[1] + b) * g.nkw + (c >> 6);
  BitWord bw = bm[w];
  unsigned long long bit = 1ull << (c & 63);
  if (!(bw.bits & bit)) return -1;
  return bw.pre + __popcll(bw.bits & (bit - 1));
}

// rank of a cell known to be present (no membership test)
__device__ __forceinline__ int32_t bm_rank_known(const BitWord* __restrict__ bm, const Grid& g, int i, int j, int k) {
  int a = i - g.glo[0], b = j - g.glo[1], c = k - g.glo[2];
  int64_t w = ((int64_t)a * g.gn[1] + b) * g.nkw + (c >> 6);
  BitWord bw = bm[w];
  return bw.pre + __popcll(bw.bits & ((1ull << (c & 63)) - 1));
}

}  // namespace cpm

// ------------------------------------------------------------------ handles
struct cpm_band {
  int device = 0;
  cpm_surface surf{};
  double h = 0, lam = 0;
  int p = 3;
  cpm::Grid grid{};
  int64_t nT = 0, nA = 0, nG = 0, nR = 0;
  cpm::BitWord* amap = nullptr;  // Sigma_A
  cpm::BitWord* rmap = nullptr;  // Sigma_A u Sigma_G ("rows")
  int32_t* ijkA = nullptr;       // [nA][3] canonical
  int32_t* arow = nullptr;       // [nA] row (rank in rmap) of each active node
  int32_t* rijk = nullptr;       // [nR][3] row nodes, canonical in rmap order
  int32_t* rexp = nullptr;       // [nR] export position (active rows, then ghost rows)
  int32_t* rbase = nullptr;      // [nR][3] interpolation cube base
  double* rcp = nullptr;         // [nR][3] closest point (FP64)
  double* w1d = nullptr;         // [nR][3][p+1] barycentric 1-D weights (FP64)
  float* s32 = nullptr;          // [nR][3] cube offsets s = cp/h - base (FP32)
  // transpose map (built on first transposed apply): for each active m, the
  // (row, cube position) pairs whose cube holds m, ascending row
  int64_t* tptr = nullptr;       // [nA + 1]
  uint32_t* tent = nullptr;      // packed row * 64 + position
  double* tw64 = nullptr;        // tensor weight of each entry, (w_u w_v) w_w in FP64
  float* tw32 = nullptr;         // the same rounded to FP32
  // E rows grouped by interpolation cube (FP32 apply): rows sharing a cube
  // base are consecutive in grow; a work item is at most EGROUP_MAX of them
  int64_t nitem = 0;
  int32_t* gitem = nullptr;      // [nitem][2] {first position << 4 | (rows - 1), base node (canonical rank)}
  int32_t* grow = nullptr;       // [nR] E rows in cube-base order (set-up only)
  float* grec = nullptr;         // [nR][4] per row in that order: FP32 offsets s_x, s_y, s_z and the row
                                 // index (as the bits of the fourth float), one 16-byte record
  // tile-staged FP32 apply: bricks of 16^3 cells holding active nodes, each
  // with the E rows its stencils need, grouped by cube
  int64_t ntile = 0, ntrec = 0;
  int32_t* thead = nullptr;      // [ntile][8] brick origin, work items, box origin, box extents
  int64_t* troff = nullptr;      // [ntile + 1] first record of each brick
  float* trec = nullptr;         // [ntrec][4] {s_x, s_y, s_z, slot of the row in the grown brick (bits)}
  uint32_t* titem = nullptr;     // [ntrec] work items (the first nitem of each brick's range)
  int32_t tmaxbox = 0;           // cells of the largest box
  // scratch for the operator apply
  void* wbuf = nullptr;          // [nR] E x values (FP64 room)
  size_t wbuf_bytes = 0;
};
