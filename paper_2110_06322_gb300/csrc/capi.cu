// capi.cu -- extern "C" entry points of libcpm (declared in include/cpm.h).
// Argument checking and error reporting live here; the work is in band.cu,
// apply.cu, oras.cu and solve.cu.
#include <cmath>
#include <cstring>

#include "kernels.cuh"
#include "oras.cuh"

namespace cpm {

static thread_local char g_err[512] = "";
std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

cpm_status fail(cpm_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

void keep_pool_memory() {
  static std::atomic<unsigned long long> done{0};  // one bit per device (devices 0..63)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  const unsigned long long bit = 1ull << dev;
  if (done.load() & bit) return;
  cudaMemPool_t pool;
  uint64_t thr = 64ull << 30;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess ||
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess)
    cudaGetLastError();  // not fatal: allocations still work, only slower
  done.fetch_or(bit);
}

cpm_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_err, sizeof(g_err), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  return e == cudaErrorMemoryAllocation ? CPM_ERR_OOM : CPM_ERR_CUDA;
}

}  // namespace cpm

using namespace cpm;

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

extern "C" {

const char* cpm_last_error(void) { return g_err; }

int64_t cpm_kernel_launches(void) { return (int64_t)g_launches.load(); }

int64_t cpm_device_allocations(void) { return (int64_t)g_allocs.load(); }

cpm_status cpm_band_build(const cpm_surface* surf, double h, int p, void* stream, cpm_band** out) {
  g_err[0] = 0;
  cpm_status st = band_build(surf, h, p, as_stream(stream), out);
  if (st != CPM_OK) return st;
  // commit cpm_apply_noalloc's fixed scratch on this device now, while the
  // caller is still allocating (lazy module loading would otherwise commit
  // it at the first cpm_apply_noalloc call)
  st = noalloc_prepare();
  if (st != CPM_OK) {
    band_free(*out, as_stream(stream));
    *out = nullptr;
  }
  return st;
}

cpm_status cpm_band_info(const cpm_band* band, int64_t* n_active, int64_t* n_ghost, int64_t* n_tube) {
  if (!band) return fail(CPM_ERR_ARG, "null band");
  if (n_active) *n_active = band->nA;
  if (n_ghost) *n_ghost = band->nG;
  if (n_tube) *n_tube = band->nT;
  return CPM_OK;
}

cpm_status cpm_band_export(const cpm_band* band, int32_t* ijk_active, int32_t* ijk_ghost, int32_t* erow_base,
                           double* erow_cp, int64_t* perm, void* stream) {
  if (!band) return fail(CPM_ERR_ARG, "null band");
  return band_export(band, ijk_active, ijk_ghost, erow_base, erow_cp, perm, as_stream(stream));
}

cpm_status cpm_band_weights(const cpm_band* band, double* w1d, void* stream) {
  if (!band || !w1d) return fail(CPM_ERR_ARG, "null argument");
  return band_weights(band, w1d, as_stream(stream));
}

cpm_status cpm_apply(const cpm_band* band, const double* c, const void* x, void* y, cpm_dtype dtype, int nrhs,
                     int transpose, void* stream) {
  if (!band || !c || !x || !y) return fail(CPM_ERR_ARG, "null argument");
  if (nrhs < 1) return fail(CPM_ERR_ARG, "nrhs must be >= 1");
  if (ranges_overlap(x, y, (size_t)nrhs * (size_t)band->nA * (dtype == CPM_F64 ? 8u : 4u)))
    return fail(CPM_ERR_ARG, "x and y must not overlap");
  for (int q = 0; q < nrhs; ++q)
    if (!std::isfinite(c[q])) return fail(CPM_ERR_NAN, "shift c[%d] is not finite", q);
  return apply_op(band, c, x, y, dtype, nrhs, transpose ? 1 : 0, as_stream(stream));
}

cpm_status oras_setup(const cpm_band* band, const oras_params* prm, double c, void* stream, oras_pc** out) {
  if (!band || !prm || !out) return fail(CPM_ERR_ARG, "null argument");
  *out = nullptr;
  if (prm->nparts < 1 || prm->nparts > band->nA) return fail(CPM_ERR_ARG, "nparts must be in [1, N_A]");
  if (prm->overlap < 0 || prm->overlap > 16) return fail(CPM_ERR_ARG, "overlap must be in [0, 16]");
  if (prm->robin && !(prm->alpha >= 0.0 && prm->alpha_cross >= 0.0))
    return fail(CPM_ERR_ARG, "Robin parameters must be >= 0 (infinity allowed)");
  if (prm->store != CPM_F32 && prm->store != CPM_BF16 && prm->store != CPM_F64)
    return fail(CPM_ERR_ARG, "store must be CPM_F64, CPM_F32 or CPM_BF16");
  if (prm->order < 0 || prm->order > 2)
    return fail(CPM_ERR_ARG, "order must be 0 (by degree), 1 (distance) or 2 (shells)");
  if (prm->coarse != 0 && prm->coarse != 1) return fail(CPM_ERR_ARG, "coarse must be 0 or 1");
  if (!std::isfinite(c)) return fail(CPM_ERR_NAN, "shift c is not finite");
  g_err[0] = 0;
  oras_params q = *prm;
  if (q.order == 0) q.order = band->p == 3 ? 2 : 1;  // the order measured best for each degree
  return oras_build(band, &q, c, as_stream(stream), out);
}

cpm_status oras_apply(const oras_pc* pc, const void* r, void* z, cpm_dtype dtype, int nrhs, int transpose,
                      void* stream) {
  if (!pc || !r || !z) return fail(CPM_ERR_ARG, "null argument");
  if (nrhs < 1) return fail(CPM_ERR_ARG, "nrhs must be >= 1");
  if (dtype != CPM_F64 && dtype != CPM_F32) return fail(CPM_ERR_ARG, "oras_apply supports CPM_F64 and CPM_F32");
  if (ranges_overlap(r, z, (size_t)nrhs * (size_t)pc->nA * (dtype == CPM_F64 ? 8u : 4u)))
    return fail(CPM_ERR_ARG, "r and z must not overlap");
  return oras_run(pc, r, z, dtype, nrhs, transpose ? 1 : 0, as_stream(stream));
}

cpm_status oras_set_tuning(oras_pc* pc, const oras_tuning* t) {
  if (!pc || !t) return fail(CPM_ERR_ARG, "null argument");
  if (t->xplace < 0 || t->xplace > 3) return fail(CPM_ERR_ARG, "xplace must be 0, 1, 2 or 3");
  if (t->lanes != 0 && t->lanes != 4 && t->lanes != 8 && t->lanes != 16)
    return fail(CPM_ERR_ARG, "lanes must be 0, 4, 8 or 16");
  if (t->schedule != 0 && t->schedule != 1) return fail(CPM_ERR_ARG, "schedule must be 0 or 1");
  if (t->ctas != 0 && t->ctas != 1 && t->ctas != 2 && t->ctas != 4)
    return fail(CPM_ERR_ARG, "ctas must be 0, 1, 2 or 4");
  if (t->probe_timeout != 0 && t->probe_timeout != 1) return fail(CPM_ERR_ARG, "probe_timeout must be 0 or 1");
  if (t->wait_polls < 0 || t->wait_polls > 0xffffffffll) return fail(CPM_ERR_ARG, "wait_polls must be in [0, 2^32)");
  pc->xplace = t->xplace;
  pc->lanes = t->lanes;
  pc->schedule = t->schedule;
  pc->ctas = t->ctas;
  pc->probe_timeout = t->probe_timeout;
  pc->wait_polls = t->wait_polls;
  return CPM_OK;
}

cpm_status oras_get_tuning(const oras_pc* pc, oras_tuning* t) {
  if (!pc || !t) return fail(CPM_ERR_ARG, "null argument");
  *t = oras_tuning{pc->xplace, pc->lanes, pc->schedule, pc->ctas, pc->probe_timeout, pc->wait_polls};
  return CPM_OK;
}

cpm_status oras_autotune(oras_pc* pc, cpm_dtype dtype, int reps, void* stream, oras_tuning* best, double* best_ms) {
  if (!pc) return fail(CPM_ERR_ARG, "null preconditioner");
  if (dtype != CPM_F32 && dtype != CPM_F64) return fail(CPM_ERR_ARG, "dtype must be CPM_F32 or CPM_F64");
  if (reps < 1 || reps > 1000) return fail(CPM_ERR_ARG, "reps must be in [1, 1000]");
  return oras_tune(pc, dtype, reps, as_stream(stream), best, best_ms);
}

cpm_status oras_info(const oras_pc* pc, int32_t* nparts, int64_t* total_rows, int64_t* total_nnz,
                     int32_t* max_levels) {
  if (!pc) return fail(CPM_ERR_ARG, "null preconditioner");
  if (nparts) *nparts = pc->np;
  if (total_rows) *total_rows = pc->nloc;
  if (total_nnz) *total_nnz = pc->nnz;
  if (max_levels) *max_levels = pc->max_levels;
  return CPM_OK;
}

cpm_status oras_export(const oras_pc* pc, int32_t* part, int64_t* sub_ptr, int32_t* sub_nodes, void* stream) {
  if (!pc) return fail(CPM_ERR_ARG, "null preconditioner");
  cudaStream_t s = as_stream(stream);
  if (part) CPM_CUDA(cudaMemcpyAsync(part, pc->part, pc->nA * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (sub_ptr) CPM_CUDA(cudaMemcpyAsync(sub_ptr, pc->sptr, (pc->np + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  if (sub_nodes) CPM_CUDA(cudaMemcpyAsync(sub_nodes, pc->snode, pc->nloc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return CPM_OK;
}

cpm_status cpm_solve_batch(int32_t nprob, const cpm_band* const* bands, const oras_pc* const* pcs, const double* c,
                           const int32_t* nrhs, const double* f, double* u, const cpm_solve_params* prm,
                           cpm_solve_info* info, int32_t transpose, void* stream) {
  if (nprob < 1 || !bands || !c || !nrhs || !f || !u || !prm || !info) return fail(CPM_ERR_ARG, "null argument");
  if (prm->restart < 1 || prm->restart > 256 || prm->maxit < 0 || !(prm->rtol > 0.0))
    return fail(CPM_ERR_ARG, "restart in [1, 256], maxit >= 0 and rtol > 0 required");
  int64_t S = 0;
  for (int p = 0; p < nprob; ++p) {
    if (!bands[p]) return fail(CPM_ERR_ARG, "null band for problem %d", p);
    if (nrhs[p] < 1) return fail(CPM_ERR_ARG, "nrhs[%d] must be >= 1", p);
    if (!std::isfinite(c[p])) return fail(CPM_ERR_NAN, "shift c[%d] is not finite", p);
    if (pcs && pcs[p] && pcs[p]->band != bands[p]) return fail(CPM_ERR_ARG, "pcs[%d] belongs to another band", p);
    S += nrhs[p];
  }
  if (S > 65535) return fail(CPM_ERR_ARG, "at most 65535 systems per batch");
  if (f == u) return fail(CPM_ERR_ARG, "f and u must not overlap");
  g_err[0] = 0;
  return solve_batch(nprob, bands, pcs, c, nrhs, f, u, prm, info, transpose ? 1 : 0, as_stream(stream));
}

static cpm_status check_rx(const cpm_schnakenberg* p) {
  if (!p) return fail(CPM_ERR_ARG, "null reaction parameters");
  if (!(p->Du > 0.0) || !(p->Dv > 0.0) || !(p->dt > 0.0))
    return fail(CPM_ERR_ARG, "Du, Dv and dt must be > 0");
  if (!std::isfinite(p->delta1) || !std::isfinite(p->delta2) || !std::isfinite(p->lambda) || !std::isfinite(p->Du) ||
      !std::isfinite(p->Dv) || !std::isfinite(p->dt))
    return fail(CPM_ERR_NAN, "reaction parameters must be finite");
  if (p->model != 0 && p->model != 1) return fail(CPM_ERR_ARG, "model must be 0 (Schnakenberg) or 1 (no reaction)");
  return CPM_OK;
}

cpm_status cpm_imex_rhs(const cpm_band* band, const cpm_schnakenberg* prm, const double* u, const double* v,
                        double* bu, double* bv, void* stream) {
  if (!band || !u || !v || !bu || !bv) return fail(CPM_ERR_ARG, "null argument");
  if (bu == u || bu == v || bv == u || bv == v || bu == bv) return fail(CPM_ERR_ARG, "outputs must not alias inputs");
  CPM_TRY(check_rx(prm));
  return imex_rhs(prm, band->nA, u, v, bu, bv, as_stream(stream));
}

cpm_status cpm_imex2_rhs(const cpm_band* band, const cpm_schnakenberg* prm, int32_t stage, const double* u,
                         const double* v, const double* u2, const double* v2, double* bu, double* bv, void* stream) {
  if (!band || !u || !v || !bu || !bv) return fail(CPM_ERR_ARG, "null argument");
  if (stage != 2 && stage != 3) return fail(CPM_ERR_ARG, "stage must be 2 or 3");
  if (stage == 3 && (!u2 || !v2)) return fail(CPM_ERR_ARG, "stage 3 needs the stage-2 solutions");
  const size_t bytes = (size_t)band->nA * sizeof(double);
  for (const double* in : {u, v, u2, v2})
    if (in && (ranges_overlap(in, bu, bytes) || ranges_overlap(in, bv, bytes)))
      return fail(CPM_ERR_ARG, "outputs must not overlap the inputs");
  if (ranges_overlap(bu, bv, bytes)) return fail(CPM_ERR_ARG, "bu and bv must not overlap");
  CPM_TRY(check_rx(prm));
  return imex2_rhs(prm, stage, band->nA, u, v, u2, v2, bu, bv, as_stream(stream));
}

cpm_status cpm_imex_rhs_adjoint(const cpm_band* band, const cpm_schnakenberg* prm, const double* u, const double* v,
                                const double* u1, const double* v1, const double* lu, const double* lv,
                                double* ubar, double* vbar, double* dc, void* stream) {
  if (!band || !u || !v || !u1 || !v1 || !lu || !lv || !ubar || !vbar || !dc)
    return fail(CPM_ERR_ARG, "null argument");
  CPM_TRY(check_rx(prm));
  return imex_rhs_adjoint(prm, band->nA, u, v, u1, v1, lu, lv, ubar, vbar, dc, as_stream(stream));
}

cpm_status cpm_dot(const cpm_band* band, const double* a, const double* b, double* out, void* stream) {
  if (!band || !a || !b || !out) return fail(CPM_ERR_ARG, "null argument");
  return dot(band->nA, a, b, out, as_stream(stream));
}

cpm_status cpm_solve(const cpm_band* band, const oras_pc* pc, double c, const double* f, double* u,
                     const cpm_solve_params* prm, cpm_solve_info* info, void* stream) {
  if (!band || !f || !u || !prm || !info) return fail(CPM_ERR_ARG, "null argument");
  if (prm->restart < 1 || prm->restart > 256 || prm->maxit < 0 || !(prm->rtol > 0.0))
    return fail(CPM_ERR_ARG, "restart in [1, 256], maxit >= 0 and rtol > 0 required");
  if (!std::isfinite(c)) return fail(CPM_ERR_NAN, "shift c is not finite");
  if (pc && pc->band != band) return fail(CPM_ERR_ARG, "preconditioner was built for another band");
  g_err[0] = 0;
  return solve_run(band, pc, c, f, u, prm, info, 0, as_stream(stream));
}

cpm_status cpm_solve_adjoint(const cpm_band* band, const oras_pc* pc, double c, const double* g, double* lambda,
                             const cpm_solve_params* prm, cpm_solve_info* info, void* stream) {
  if (!band || !g || !lambda || !prm || !info) return fail(CPM_ERR_ARG, "null argument");
  if (prm->restart < 1 || prm->restart > 256 || prm->maxit < 0 || !(prm->rtol > 0.0))
    return fail(CPM_ERR_ARG, "restart in [1, 256], maxit >= 0 and rtol > 0 required");
  if (!std::isfinite(c)) return fail(CPM_ERR_NAN, "shift c is not finite");
  if (pc && pc->band != band) return fail(CPM_ERR_ARG, "preconditioner was built for another band");
  g_err[0] = 0;
  return solve_run(band, pc, c, g, lambda, prm, info, 1, as_stream(stream));
}

void cpm_band_free(cpm_band* band) {
  if (!band) return;
  cudaDeviceSynchronize();
  band_free(band, 0);
  cudaDeviceSynchronize();
}

void oras_free(oras_pc* pc) {
  if (!pc) return;
  cudaDeviceSynchronize();
  oras_destroy(pc, 0);
  cudaDeviceSynchronize();
}

}  // extern "C"
