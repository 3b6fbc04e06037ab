// oras.cu -- placeholder (filled in next)
#include "kernels.cuh"
#include "oras.cuh"
namespace cpm {
cpm_status oras_build(const cpm_band*, const oras_params*, double, cudaStream_t, oras_pc**) { return fail(CPM_ERR_ARG, "not built yet"); }
cpm_status oras_run(const oras_pc*, const void*, void*, cpm_dtype, int, int, cudaStream_t) { return fail(CPM_ERR_ARG, "not built yet"); }
void oras_destroy(oras_pc* P, cudaStream_t) { delete P; }
}
