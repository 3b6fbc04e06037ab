// scan.cu -- deterministic device-wide exclusive prefix sums (three passes:
// tile sums, a scan of the tile sums, tile-local scans plus offsets).
#include "kernels.cuh"

namespace cpm {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ int64_t block_exclusive(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[SCAN_THREADS / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t ws = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += y;
    }
    if (lane < SCAN_THREADS / 32) warp_sums[lane] = ws;
  }
  __syncthreads();
  int64_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
  *total = warp_sums[SCAN_THREADS / 32 - 1];
  __syncthreads();
  return before;
}

template <typename T>
__global__ void k_tile_sums(const T* __restrict__ in, int64_t n, int64_t* tsum) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v = 0;
  for (int q = 0; q < SCAN_ITEMS; ++q)
    if (base + q < n) v += (int64_t)in[base + q];
  int64_t tot;
  block_exclusive<T>(v, &tot);
  if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in place
__global__ void k_scan_tiles(int64_t* tsum, int64_t nt) {
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nt; b0 += SCAN_THREADS) {
    int64_t i = b0 + threadIdx.x;
    int64_t v = i < nt ? tsum[i] : 0;
    int64_t tot;
    int64_t e = block_exclusive<int64_t>(v, &tot);
    if (i < nt) tsum[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) tsum[nt] = carry;
}

template <typename T>
__global__ void k_tile_scan(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ tsum, int64_t* out,
                            int64_t nt) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t vals[SCAN_ITEMS];
  int64_t v = 0;
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    vals[q] = (base + q < n) ? (int64_t)in[base + q] : 0;
    v += vals[q];
  }
  int64_t tot;
  int64_t run = tsum[blockIdx.x] + block_exclusive<T>(v, &tot);
  for (int q = 0; q < SCAN_ITEMS; ++q) {
    if (base + q < n) out[base + q] = run;
    run += vals[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tsum[nt];
}

template <typename T>
cpm_status scan_impl(const T* in, int64_t* out, int64_t n, cudaStream_t s) {
  int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nt == 0) {
    CPM_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return CPM_OK;
  }
  int64_t* tsum = nullptr;
  CPM_TRY(dalloc(&tsum, nt + 1, s));
  KL(k_tile_sums<T><<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tsum));
  KL(k_scan_tiles<<<1, SCAN_THREADS, 0, s>>>(tsum, nt));
  KL(k_tile_scan<T><<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, n, tsum, out, nt));
  cudaError_t e = cudaGetLastError();
  dfree(tsum, s);
  if (e != cudaSuccess) return cuda_fail(e, "scan kernels", __FILE__, __LINE__);
  return CPM_OK;
}

}  // namespace

cpm_status scan_exclusive_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, n, s);
}
cpm_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return scan_impl<int64_t>(in, out, n, s);
}

}  // namespace cpm
