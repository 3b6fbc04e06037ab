// oras.cuh -- Schwarz preconditioner handle and solver entry points (internal).
#pragma once

#include "common.cuh"

// One chunk of level-packed factor rows (see packed.cu): byte offset and size
// in the packed stream, its rows and entries, whether its rows are scaled by a
// stored reciprocal diagonal, and whether it is the last chunk of its level.
struct ChunkRec {
  int64_t off;
  int32_t bytes, nrows, ne, div;
  int32_t lend, pad;
};

struct PackedFactors {
  uint8_t* data = nullptr;
  int64_t bytes = 0;
  ChunkRec* rec = nullptr;
  int64_t* chsub = nullptr;  // [np+1] chunk range of each subdomain (forward, then backward)
  uint16_t* csz = nullptr;   // [nchunks] chunk sizes in 16-byte units
  int32_t* order = nullptr;  // [np] subdomains by decreasing chunk count (launch order)
  int64_t nchunks = 0, max_chunks = 0;
  cpm_dtype vtype = CPM_F64;
};

// Restricted additive Schwarz preconditioner (Section 2.2).  Local rows of all
// subdomains are numbered globally ("local rows"): subdomain j owns local
// rows sptr[j] .. sptr[j+1]-1, in its local order.  Column indices in the
// factors are local to the subdomain (0 .. |S_j|-1).
struct oras_pc {
  const cpm_band* band = nullptr;
  int device = 0;
  int np = 0, overlap = 0, robin = 0, store = CPM_F32;
  int order = 1;  // local order of the factorisation: 1 distance, 2 shells + lattice colours
  double alpha = 0, alpha_x = 0, c = 0;
  int64_t nA = 0;
  int32_t* part = nullptr;    // [nA] disjoint part of each active node
  int64_t nloc = 0;           // sum_j |S_j|
  int64_t max_rows = 0;       // max_j |S_j|
  int64_t* sptr = nullptr;    // [np+1]
  int32_t* snode = nullptr;   // [nloc] canonical node of each local row
  uint8_t* owned = nullptr;   // [nloc] node lies in the subdomain's own disjoint part
  int64_t nnz = 0;
  int64_t* rptr = nullptr;    // [nloc+1] CSR of the local matrices / ILU(0) factors (L\U packed)
  int32_t* col = nullptr;     // [nnz] local column (within the subdomain)
  int32_t* dpos = nullptr;    // [nloc] offset of the diagonal within its row
  double* val = nullptr;      // [nnz] FP64 factors (CSR; the applies use the packed copies)
  // level schedules: for subdomain j, forward levels lvptr_f[lvsub_f[j] .. lvsub_f[j+1]]
  // index ranges of lvrow_f (local rows, ascending within a level)
  int32_t* lvsub_f = nullptr;  // [np+1]
  int64_t* lvptr_f = nullptr;  // [nlev_f + 1]
  int32_t* lvrow_f = nullptr;  // [nloc]
  int32_t* lvsub_b = nullptr;
  int64_t* lvptr_b = nullptr;
  int32_t* lvrow_b = nullptr;
  int32_t max_levels = 0;
  // transposed factors (adjoint): CSR of L^T and U^T, built on first use
  int64_t* tptr = nullptr;
  int32_t* tcol = nullptr;
  double* tval = nullptr;
  int32_t* tdpos = nullptr;
  int32_t* lvsub_tf = nullptr;  // level schedules of the transposed factors
  int64_t* lvptr_tf = nullptr;
  int32_t* lvrow_tf = nullptr;
  int32_t* lvsub_tb = nullptr;
  int64_t* lvptr_tb = nullptr;
  int32_t* lvrow_tb = nullptr;
  // node -> subdomains holding it (ascending) and its local row there
  int32_t* mcnt = nullptr;    // [nA]
  int32_t* memb = nullptr;    // [nA][KMEM]
  int32_t* mloc = nullptr;    // [nA][KMEM] local row (global numbering)
  int32_t* lsub = nullptr;    // [nloc] subdomain of each local row
  // level-packed factors: [0] FP64, [1] store type, [2] transposed FP64, [3] transposed FP32
  PackedFactors packed[4];
  int* err = nullptr;         // device flag: a bounded wait of the apply ran out
  // run-time settings of the apply (oras_set_tuning)
  int xplace = 0;             // 0 local vector in shared memory when it fits, 1 always a global slice
  int lanes = 0;              // lanes per factor row in the sweeps (0: by placement)
  int schedule = 0;           // 0 subdomains longest first, 1 in partition order
  int ctas = 0;               // global-slice path: CTAs per SM, 1 (larger L1), 2 or 4 (6 consumer warps); 0 = 1
  int probe_timeout = 0;      // failure-path test: the first chunk wait can only run out
  int64_t wait_polls = 0;     // polls of each consumer-side wait (0: the default)
  // two-level variant (coarse correction on one constant per disjoint part)
  int coarse = 0;
  int64_t* mzptr = nullptr;   // [nA+1] rows of M Z: the parts each node's row reaches
  int32_t* mzpart = nullptr;  // [nmz] part
  double* mzval = nullptr;    // [nmz] the row's sum over that part (FP64)
  double* E0inv = nullptr;    // [np][np] inverse of Z^T M Z, row-major
};

namespace cpm {
constexpr int KMEM = 16;  // most subdomains one node may belong to
}

namespace cpm {
cpm_status oras_build(const cpm_band* B, const oras_params* prm, double c, cudaStream_t s, oras_pc** out);
cpm_status oras_run(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose, cudaStream_t s);
cpm_status oras_run_one_level(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose,
                              cudaStream_t s);
// coarse.cu: the two-level variant
cpm_status coarse_build(oras_pc* P, const int64_t* mptr, const int32_t* mcol, const double* mval, cudaStream_t s);
void coarse_free(oras_pc* P, cudaStream_t s);
cpm_status coarse_apply(const oras_pc* P, const void* r, void* z, cpm_dtype dt, int nrhs, int transpose,
                        cudaStream_t s);
cpm_status pack_factors(oras_pc* P, int transposed, const cpm_dtype* vt, PackedFactors* out, int nout,
                        cudaStream_t s);
void packed_free(PackedFactors& pf, cudaStream_t s);
void oras_destroy(oras_pc* P, cudaStream_t s);
// Read and clear the preconditioner's timeout flag (synchronises the stream):
// CPM_ERR_TIMEOUT if a bounded wait of an apply since the last check ran out.
cpm_status oras_take_error(const oras_pc* P, cudaStream_t s);
// time the equivalent apply kernels and keep the fastest (oras_autotune)
cpm_status oras_tune(oras_pc* P, cpm_dtype dt, int reps, cudaStream_t s, oras_tuning* best, double* best_ms);
cpm_status solve_run(const cpm_band* B, const oras_pc* P, double c, const double* f, double* u,
                     const cpm_solve_params* prm, cpm_solve_info* info, int transpose, cudaStream_t s);
}  // namespace cpm
