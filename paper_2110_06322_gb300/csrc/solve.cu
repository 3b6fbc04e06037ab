// solve.cu -- placeholder (filled in next)
#include "kernels.cuh"
#include "oras.cuh"
namespace cpm {
cpm_status solve_run(const cpm_band*, const oras_pc*, double, const double*, double*, const cpm_solve_params*, cpm_solve_info*, int, cudaStream_t) { return fail(CPM_ERR_ARG, "not built yet"); }
}
