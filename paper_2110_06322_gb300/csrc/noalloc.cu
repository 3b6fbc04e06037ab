// noalloc.cu -- cpm_apply_noalloc: the forward operator apply without any
// device allocation, for callers that cannot allocate device memory.
//
// cpm_apply takes its scratch (one value pair per E row) from the stream-
// ordered allocator on every call.  Some callers cannot do that: processes
// whose device memory is owned by another allocator (a framework's caching
// pool that has reserved the device, so a foreign cudaMalloc fails or
// fragments it), and latency-bounded loops in which an allocation may block
// or synchronise.  This entry point uses instead one fixed scratch array that
// lives in this file as a static __device__ variable: every GPU on which a
// band has been built holds it (16 MiB) until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current.  Under CUDA's
// lazy module loading that lookup is also what loads this file's module and
// so commits the 16 MiB on the device; cpm_band_build therefore does it
// (noalloc_prepare) when it builds a band, while the caller is still in its
// allocating phase, and the entry point only reads the cached address.  All
// calls share the array: calls whose kernels overlap on the GPU (two
// streams, two threads) race on it.  Nothing in the scratch needs to start
// at zero -- every call writes each entry it reads.
#include <mutex>

#include "kernels.cuh"

namespace cpm {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;  // 16 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// device address of the scratch array on the current device (set-up on first use)
cpm_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(CPM_ERR_ARG, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)", __FILE__, __LINE__);
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CPM_OK;
}

}  // namespace

// Commit the scratch array on the current device and cache its address
// (called by cpm_band_build for the band's device).
cpm_status noalloc_prepare() {
  int dev = 0;
  CPM_CUDA(cudaGetDevice(&dev));
  void* p = nullptr;
  return scratch_address(dev, &p);
}

}  // namespace cpm

using namespace cpm;

extern "C" cpm_status cpm_apply_noalloc(const cpm_band* band, const double* c, const void* x, void* y,
                                        cpm_dtype dtype, int nrhs, void* stream) {
  if (!band || !c || !x || !y) return fail(CPM_ERR_ARG, "null argument");
  if (nrhs < 1) return fail(CPM_ERR_ARG, "nrhs must be >= 1");
  if (dtype != CPM_F64 && dtype != CPM_F32) return fail(CPM_ERR_ARG, "dtype must be CPM_F64 or CPM_F32");
  if (ranges_overlap(x, y, (size_t)nrhs * (size_t)band->nA * (dtype == CPM_F64 ? 8u : 4u)))
    return fail(CPM_ERR_ARG, "x and y must not overlap");
  for (int q = 0; q < nrhs; ++q)
    if (!(c[q] == c[q]) || c[q] - c[q] != 0.0) return fail(CPM_ERR_NAN, "shift c[%d] is not finite", q);
  int dev = 0;
  CPM_CUDA(cudaGetDevice(&dev));
  if (dev != band->device) return fail(CPM_ERR_ARG, "the band lives on device %d, current device is %d", band->device, dev);
  // scratch: 8 bytes per E row and right-hand side, for up to 16 right-hand sides at a time
  const int chunk = nrhs < 16 ? nrhs : 16;
  const size_t need = (size_t)chunk * (size_t)band->nR * 8u;
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(CPM_ERR_ARG,
                "cpm_apply_noalloc needs %zu bytes of scratch (%d right-hand sides x %lld E rows x 8 bytes) but its "
                "fixed scratch holds %zu bytes: use cpm_apply or fewer right-hand sides",
                need, chunk, (long long)band->nR, NOALLOC_SCRATCH_BYTES);
  void* scratch = nullptr;
  CPM_TRY(scratch_address(dev, &scratch));
  return apply_op_scratch(band, c, x, y, dtype, nrhs, scratch, (cudaStream_t)stream);
}
