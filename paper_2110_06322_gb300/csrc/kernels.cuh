// kernels.cuh -- cross-translation-unit entry points of libcpm (internal).
#pragma once

#include "common.cuh"

namespace cpm {

// scan.cu: exclusive prefix sums, out[0..n] (out[n] = total), deterministic
cpm_status scan_exclusive_i32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
cpm_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

// band.cu
cpm_status band_build(const cpm_surface* surf, double h, int p, cudaStream_t s, cpm_band** out);
void band_free(cpm_band* B, cudaStream_t s);
cpm_status band_export(const cpm_band* B, int32_t* ijkA, int32_t* ijkG, int32_t* ebase, double* ecp, int64_t* perm,
                       cudaStream_t s);
cpm_status band_weights(const cpm_band* B, double* w, cudaStream_t s);
cpm_status bitmap_prefix(BitWord* bm, int64_t nw, int64_t* total, cudaStream_t s);

// apply.cu: y = M x or M^T x for nrhs vectors of type T (double or float)
cpm_status apply_op(const cpm_band* B, const double* c, const void* x, void* y, cpm_dtype dt, int nrhs, int transpose,
                    cudaStream_t s);
// E x for all rows (into B->wbuf) followed by the stencil; exposed so that
// the solver can reuse it with device-side c.
cpm_status build_transpose_map(cpm_band* B, cudaStream_t s);
// group the E rows by interpolation cube for the FP32 apply (band build)
cpm_status build_erow_groups(cpm_band* B, cudaStream_t s);
// tile.cu: the FP32 forward apply staged through shared memory by bricks
cpm_status build_tiles(cpm_band* B, cudaStream_t s);
void free_tiles(cpm_band* B, cudaStream_t s);
cpm_status tile_apply_f32(const cpm_band* B, const double* c, const float* x, float* y, int nrhs, cudaStream_t s);
cpm_status apply_op_scratch(const cpm_band* B, const double* c, const void* x, void* y, cpm_dtype dt, int nrhs,
                            void* scratch, cudaStream_t s);

// noalloc.cu: commit the fixed scratch of cpm_apply_noalloc on the current device
cpm_status noalloc_prepare();

// batch.cu: lockstep GMRES over many systems
cpm_status solve_batch(int nprob, const cpm_band* const* bands, const oras_pc* const* pcs, const double* c,
                       const int32_t* nrhs, const double* f, double* u, const cpm_solve_params* prm,
                       cpm_solve_info* info, int transpose, cudaStream_t s);

// imex.cu: reaction-diffusion step right-hand sides, their adjoint, dot product
cpm_status imex_rhs(const cpm_schnakenberg* prm, int64_t n, const double* u, const double* v, double* bu, double* bv,
                    cudaStream_t s);
cpm_status imex2_rhs(const cpm_schnakenberg* prm, int stage, int64_t n, const double* u, const double* v,
                     const double* u2, const double* v2, double* bu, double* bv, cudaStream_t s);
cpm_status imex_rhs_adjoint(const cpm_schnakenberg* prm, int64_t n, const double* u, const double* v,
                            const double* u1, const double* v1, const double* lu, const double* lv, double* ubar,
                            double* vbar, double* dc, cudaStream_t s);
cpm_status dot(int64_t n, const double* a, const double* b, double* out, cudaStream_t s);

}  // namespace cpm
