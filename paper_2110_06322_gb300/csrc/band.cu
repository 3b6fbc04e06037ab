// band.cu -- narrow-band construction on the GPU (Section 2.1).
//
//   K1 tube_mark   seed tube T = {x : dist(x,S) <= lambda} over a dense box
//                  grid (FP32 pre-filter, exact FP64 test), and for every x in
//                  T the (p+1)^3 interpolation cube at cp(x) OR-ed into the
//                  Sigma_A bitmap (idempotent, so the result is deterministic)
//   K2 dilate      Sigma_G = 6-neighbours of Sigma_A outside it; R = A u G
//   K3 scan        word prefix counts -> canonical ranks (bitmap order is the
//                  lexicographic order, k fastest)
//   K4 enumerate   node lists, row numbering, export positions
//   K5 erow        per row: cp (FP64), cube base, 1-D barycentric weights,
//                  FP32 offsets, and the closure check (cube inside Sigma_A)
//
// Every FP64 operation of the band (closest points, bases, weights) is
// written with explicit round-to-nearest intrinsics in a fixed order, so the
// band and the stencil weights are bit-identical to a plain IEEE evaluation
// of the same formulas.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"
#include "surface.cuh"

namespace cpm {

namespace {

struct TubeArgs {
  SurfDev S;
  double h, lam;
  int p;
  Grid g;
  // FP32 pre-filter: x_rel = (i - ic) * hf - off
  int ic[3];
  float off[3], hf, lam_hi;
};

__device__ __forceinline__ void or_bits(unsigned long long* bits, const Grid& g, int i, int j, int k, int len,
                                        int* err) {
  int a = i - g.glo[0], b = j - g.glo[1], c = k - g.glo[2];
  if (a < 0 || b < 0 || c < 0 || a >= g.gn[0] || b >= g.gn[1] || c + len > g.gn[2]) {
    atomicExch(err, CPM_ERR_BAND);
    return;
  }
  int64_t w = ((int64_t)a * g.gn[1] + b) * g.nkw + (c >> 6);
  int sh = c & 63;
  unsigned long long m = ((1ull << len) - 1ull);
  atomicOr(bits + 2 * w, m << sh);  // BitWord = {bits, pre|pad}: bits at even 8-byte slots
  if (sh + len > 64) atomicOr(bits + 2 * (w + 1), m >> (64 - sh));
}

// K1: seed tube and cube marks.  One thread per grid cell.
__global__ void k_tube_mark(TubeArgs A, BitWord* amap, unsigned long long* nT, int* err) {
  const Grid& g = A.g;
  int64_t ncell = (int64_t)g.gn[0] * g.gn[1] * g.gn[2];
  unsigned long long cnt = 0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ncell; q += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(q % g.gn[2]);
    int64_t ab = q / g.gn[2];
    int b = (int)(ab % g.gn[1]);
    int a = (int)(ab / g.gn[1]);
    int ijk[3] = {g.glo[0] + a, g.glo[1] + b, g.glo[2] + c};
    // FP32 pre-filter with a generous margin; the FP64 test decides
    float xr[3];
    for (int d = 0; d < 3; ++d) xr[d] = (float)(ijk[d] - A.ic[d]) * A.hf - A.off[d];
    float d32;
    if (A.S.kind == 0) {
      d32 = fabsf(sqrtf(xr[0] * xr[0] + xr[1] * xr[1] + xr[2] * xr[2]) - (float)A.S.a);
    } else {
      float w = sqrtf(xr[0] * xr[0] + xr[1] * xr[1]) - (float)A.S.a;
      d32 = fabsf(sqrtf(w * w + xr[2] * xr[2]) - (float)A.S.b);
    }
    if (d32 > A.lam_hi) continue;
    double x0 = dm((double)ijk[0], A.h), x1 = dm((double)ijk[1], A.h), x2 = dm((double)ijk[2], A.h);
    if (!(surf_dist(A.S, x0, x1, x2) <= A.lam)) continue;
    cnt++;
    double cp[3];
    if (!surf_cp(A.S, x0, x1, x2, cp)) {
      atomicExch(err, CPM_ERR_BAND);
      continue;
    }
    int bs[3];
    double s;
    for (int d = 0; d < 3; ++d) cube_base(cp[d], A.h, A.p, &bs[d], &s);
    for (int u = 0; u <= A.p; ++u)
      for (int v = 0; v <= A.p; ++v)
        or_bits(reinterpret_cast<unsigned long long*>(amap), g, bs[0] + u, bs[1] + v, bs[2], A.p + 1, err);
  }
  // warp-aggregated count
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(nT, cnt);
}

// K2: ghosts = 6-dilation of A minus A; rmap = A | G.  One thread per word.
__global__ void k_dilate(const BitWord* __restrict__ amap, BitWord* rmap, Grid g) {
  int64_t nw = g.nwords();
  int64_t colw = g.nkw, planew = (int64_t)g.gn[1] * g.nkw;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    int kw = (int)(w % g.nkw);
    int64_t ab = w / g.nkw;
    int b = (int)(ab % g.gn[1]);
    int a = (int)(ab / g.gn[1]);
    unsigned long long A = amap[w].bits;
    unsigned long long up = (kw + 1 < g.nkw) ? amap[w + 1].bits : 0ull;
    unsigned long long dn = (kw > 0) ? amap[w - 1].bits : 0ull;
    unsigned long long n = (A << 1) | (dn >> 63) | (A >> 1) | (up << 63);
    if (b > 0) n |= amap[w - colw].bits;
    if (b + 1 < g.gn[1]) n |= amap[w + colw].bits;
    if (a > 0) n |= amap[w - planew].bits;
    if (a + 1 < g.gn[0]) n |= amap[w + planew].bits;
    int valid = g.gn[2] - kw * 64;
    unsigned long long vm = valid >= 64 ? ~0ull : (valid <= 0 ? 0ull : ((1ull << valid) - 1ull));
    rmap[w].bits = (A | (n & ~A)) & vm;
  }
}

__global__ void k_popc(const BitWord* __restrict__ bm, int32_t* cnt, int64_t nw) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popcll(bm[w].bits);
}

__global__ void k_set_pre(BitWord* bm, const int64_t* pre, int64_t nw) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
    bm[w].pre = (int32_t)pre[w];
}

// K4: enumerate rows (A u G) in canonical order.  One thread per word.
__global__ void k_enumerate(const BitWord* __restrict__ amap, const BitWord* __restrict__ rmap, Grid g, int64_t nA,
                            int32_t* ijkA, int32_t* arow, int32_t* rijk, int32_t* rexp) {
  int64_t nw = g.nwords();
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    BitWord R = rmap[w];
    if (!R.bits) continue;
    BitWord Aw = amap[w];
    int kw = (int)(w % g.nkw);
    int64_t ab = w / g.nkw;
    int b = (int)(ab % g.gn[1]);
    int a = (int)(ab / g.gn[1]);
    unsigned long long bits = R.bits;
    while (bits) {
      int bit = __ffsll((long long)bits) - 1;
      bits &= bits - 1;
      unsigned long long below = (1ull << bit) - 1ull;
      int32_t r = R.pre + __popcll(R.bits & below);
      int32_t na_before = Aw.pre + __popcll(Aw.bits & below);
      int i = g.glo[0] + a, j = g.glo[1] + b, k = g.glo[2] + kw * 64 + bit;
      rijk[3 * (int64_t)r + 0] = i;
      rijk[3 * (int64_t)r + 1] = j;
      rijk[3 * (int64_t)r + 2] = k;
      if (Aw.bits & (1ull << bit)) {
        int32_t q = na_before;
        ijkA[3 * (int64_t)q + 0] = i;
        ijkA[3 * (int64_t)q + 1] = j;
        ijkA[3 * (int64_t)q + 2] = k;
        arow[q] = r;
        rexp[r] = q;
      } else {
        rexp[r] = (int32_t)(nA + (r - na_before));
      }
    }
  }
}

// K5: E-row geometry and closure.  One thread per row.
__global__ void k_erow(SurfDev S, double h, int p, Grid g, const BitWord* __restrict__ amap, int64_t nR,
                       const int32_t* __restrict__ rijk, int32_t* rbase, double* rcp, double* w1d, float* s32,
                       int* err) {
  const int P1 = p + 1;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nR; r += (int64_t)gridDim.x * blockDim.x) {
    double x0 = dm((double)rijk[3 * r], h), x1 = dm((double)rijk[3 * r + 1], h), x2 = dm((double)rijk[3 * r + 2], h);
    double cp[3];
    if (!surf_cp(S, x0, x1, x2, cp)) {
      atomicExch(err, CPM_ERR_BAND);
      continue;
    }
    int bs[3];
    for (int d = 0; d < 3; ++d) {
      double s;
      cube_base(cp[d], h, p, &bs[d], &s);
      rbase[3 * r + d] = bs[d];
      rcp[3 * r + d] = cp[d];
      s32[3 * r + d] = (float)s;
      double wl[4];
      weights1d(p, s, wl);
      for (int q = 0; q < P1; ++q) w1d[(3 * r + d) * P1 + q] = wl[q];
    }
    // closure: the whole cube must be active
    for (int u = 0; u <= p; ++u)
      for (int v = 0; v <= p; ++v)
        for (int w = 0; w <= p; ++w)
          if (bm_rank(amap, g, bs[0] + u, bs[1] + v, bs[2] + w) < 0) atomicExch(err, CPM_ERR_BAND);
  }
}

__global__ void k_export(int64_t nR, int64_t nA, const int32_t* __restrict__ rexp, const int32_t* __restrict__ rijk,
                         const int32_t* __restrict__ rbase, const double* __restrict__ rcp, int32_t* ijkG,
                         int32_t* ebase, double* ecp) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nR; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = rexp[r];
    for (int d = 0; d < 3; ++d) {
      if (ebase) ebase[3 * e + d] = rbase[3 * r + d];
      if (ecp) ecp[3 * e + d] = rcp[3 * r + d];
      if (ijkG && e >= nA) ijkG[3 * (e - nA) + d] = rijk[3 * r + d];
    }
  }
}

__global__ void k_export_w(int64_t nR, int P1, const int32_t* __restrict__ rexp, const double* __restrict__ w1d,
                           double* out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nR; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = rexp[r];
    for (int q = 0; q < 3 * P1; ++q) out[e * 3 * P1 + q] = w1d[r * 3 * P1 + q];
  }
}

__global__ void k_iota64(int64_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = i;
}

// Host copy of the band radius formula (exact for the p used here).
double band_lambda(double h, int p) {
  double half = 0.5 * (double)(p + 1);
  double lam2 = 2.0 * (half * half) + (1.0 + half) * (1.0 + half);
  return h * std::sqrt(lam2);
}

}  // namespace

cpm_status bitmap_prefix(BitWord* bm, int64_t nw, int64_t* total, cudaStream_t s) {
  int32_t* cnt = nullptr;
  int64_t* pre = nullptr;
  CPM_TRY(dalloc(&cnt, nw, s));
  CPM_TRY(dalloc(&pre, nw + 1, s));
  KL(k_popc<<<grid_for(nw, 256), 256, 0, s>>>(bm, cnt, nw));
  CPM_TRY(scan_exclusive_i32(cnt, pre, nw, s));
  KL(k_set_pre<<<grid_for(nw, 256), 256, 0, s>>>(bm, pre, nw));
  CPM_CUDA(cudaMemcpyAsync(total, pre + nw, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  dfree(cnt, s);
  dfree(pre, s);
  return CPM_OK;
}

cpm_status band_build(const cpm_surface* surf, double h, int p, cudaStream_t s, cpm_band** out) {
  if (!surf || !out) return fail(CPM_ERR_ARG, "null argument");
  *out = nullptr;
  if (!(h > 0.0) || !std::isfinite(h)) return fail(CPM_ERR_ARG, "grid spacing must be positive");
  if (p != 2 && p != 3) return fail(CPM_ERR_ARG, "interpolation degree p must be 2 or 3");
  SurfDev S{};
  S.kind = surf->kind;
  for (int d = 0; d < 3; ++d) S.c[d] = surf->param[d];
  S.a = surf->param[3];
  S.b = surf->kind == 1 ? surf->param[4] : 0.0;
  double reach, scale;
  double lo[3], hi[3];
  if (S.kind == 0) {
    if (!(S.a > 0.0)) return fail(CPM_ERR_ARG, "sphere radius must be positive");
    reach = S.a;
    scale = S.a;
    for (int d = 0; d < 3; ++d) { lo[d] = S.c[d] - S.a; hi[d] = S.c[d] + S.a; }
  } else if (S.kind == 1) {
    if (!(S.b > 0.0 && S.a > S.b)) return fail(CPM_ERR_ARG, "torus needs R > r > 0");
    reach = std::min(S.b, S.a - S.b);
    scale = S.a + S.b;
    for (int d = 0; d < 2; ++d) { lo[d] = S.c[d] - (S.a + S.b); hi[d] = S.c[d] + (S.a + S.b); }
    lo[2] = S.c[2] - S.b;
    hi[2] = S.c[2] + S.b;
  } else {
    return fail(CPM_ERR_ARG, "surface kind %d is not supported (0 sphere, 1 torus)", surf->kind);
  }
  double lam = band_lambda(h, p);
  if (!(lam < reach))
    return fail(CPM_ERR_BAND, "band radius %.6g is not inside the surface reach %.6g: refine h", lam, reach);
  Grid g{};
  for (int d = 0; d < 3; ++d) {
    double l = std::floor((lo[d] - lam) / h) - (p + 3);
    double u = std::ceil((hi[d] + lam) / h) + (p + 3);
    if (!(u - l < 2.0e6)) return fail(CPM_ERR_ARG, "grid too large (h too small for the surface)");
    g.glo[d] = (int)l;
    g.gn[d] = (int)(u - l) + 1;
  }
  g.nkw = (g.gn[2] + 63) / 64;
  int64_t nw = g.nwords();
  if ((double)nw * 16.0 > 64.0e9) return fail(CPM_ERR_ARG, "grid too large (h too small for the surface)");

  cpm_band* B = new cpm_band();
  CPM_CUDA(cudaGetDevice(&B->device));
  B->surf = *surf;
  B->h = h;
  B->p = p;
  B->lam = lam;
  B->grid = g;
  int* err = nullptr;
  unsigned long long* nT = nullptr;
  auto cleanup = [&](cpm_status st) {
    dfree(err, s);
    dfree(nT, s);
    if (st != CPM_OK) band_free(B, s);
    return st;
  };
  cpm_status st;
  if ((st = dalloc(&B->amap, nw, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->rmap, nw, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&err, 1, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&nT, 1, s)) != CPM_OK) return cleanup(st);
  CPM_CUDA(cudaMemsetAsync(B->amap, 0, nw * sizeof(BitWord), s));
  CPM_CUDA(cudaMemsetAsync(B->rmap, 0, nw * sizeof(BitWord), s));
  CPM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  CPM_CUDA(cudaMemsetAsync(nT, 0, sizeof(unsigned long long), s));

  TubeArgs A{};
  A.S = S;
  A.h = h;
  A.lam = lam;
  A.p = p;
  A.g = g;
  A.hf = (float)h;
  for (int d = 0; d < 3; ++d) {
    A.ic[d] = (int)std::llround(S.c[d] / h);
    A.off[d] = (float)(S.c[d] - (double)A.ic[d] * h);
  }
  A.lam_hi = (float)(lam * 1.0001 + 1e-5 * scale);
  int64_t ncell = (int64_t)g.gn[0] * g.gn[1] * g.gn[2];
  KL(k_tube_mark<<<grid_for(ncell, 256, 152 * 32), 256, 0, s>>>(A, B->amap, nT, err));
  CPM_CUDA(cudaGetLastError());
  KL(k_dilate<<<grid_for(nw, 256), 256, 0, s>>>(B->amap, B->rmap, g));
  CPM_CUDA(cudaGetLastError());
  int64_t nA = 0, nR = 0;
  if ((st = bitmap_prefix(B->amap, nw, &nA, s)) != CPM_OK) return cleanup(st);
  if ((st = bitmap_prefix(B->rmap, nw, &nR, s)) != CPM_OK) return cleanup(st);
  int herr = 0;
  unsigned long long hT = 0;
  CPM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaMemcpyAsync(&hT, nT, sizeof(hT), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if (herr) return cleanup(fail(CPM_ERR_BAND, "interpolation cube left the grid"));
  if (nR >= (1ll << 26) || nA == 0)
    return cleanup(fail(CPM_ERR_ARG, "band of %lld rows is outside the supported range [1, 2^26)", (long long)nR));
  B->nT = (int64_t)hT;
  B->nA = nA;
  B->nR = nR;
  B->nG = nR - nA;
  const int P1 = p + 1;
  if ((st = dalloc(&B->ijkA, 3 * nA, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->arow, nA, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->rijk, 3 * nR, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->rexp, nR, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->rbase, 3 * nR, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->rcp, 3 * nR, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->w1d, 3 * P1 * nR, s)) != CPM_OK) return cleanup(st);
  if ((st = dalloc(&B->s32, 3 * nR, s)) != CPM_OK) return cleanup(st);
  KL(k_enumerate<<<grid_for(nw, 256), 256, 0, s>>>(B->amap, B->rmap, g, nA, B->ijkA, B->arow, B->rijk, B->rexp));
  CPM_CUDA(cudaGetLastError());
  KL(k_erow<<<grid_for(nR, 128), 128, 0, s>>>(S, h, p, g, B->amap, nR, B->rijk, B->rbase, B->rcp, B->w1d, B->s32, err));
  CPM_CUDA(cudaGetLastError());
  CPM_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if (herr) return cleanup(fail(CPM_ERR_BAND, "an interpolation cube is not inside the active set"));
  if ((st = build_erow_groups(B, s)) != CPM_OK) return cleanup(st);
  if ((st = build_tiles(B, s)) != CPM_OK) return cleanup(st);
  *out = B;
  return cleanup(CPM_OK);
}

void band_free(cpm_band* B, cudaStream_t s) {
  if (!B) return;
  dfree(B->amap, s);
  dfree(B->rmap, s);
  dfree(B->ijkA, s);
  dfree(B->arow, s);
  dfree(B->rijk, s);
  dfree(B->rexp, s);
  dfree(B->rbase, s);
  dfree(B->rcp, s);
  dfree(B->w1d, s);
  dfree(B->s32, s);
  dfree(B->tptr, s);
  dfree(B->tent, s);
  dfree(B->tw64, s);
  dfree(B->tw32, s);
  dfree(B->gitem, s);
  dfree(B->grow, s);
  dfree(B->grec, s);
  free_tiles(B, s);
  if (B->wbuf) cudaFreeAsync(B->wbuf, s);
  B->wbuf = nullptr;
  delete B;
}

cpm_status band_export(const cpm_band* B, int32_t* ijkA, int32_t* ijkG, int32_t* ebase, double* ecp, int64_t* perm,
                       cudaStream_t s) {
  if (ijkA) CPM_CUDA(cudaMemcpyAsync(ijkA, B->ijkA, 3 * B->nA * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (ijkG || ebase || ecp) {
    KL(k_export<<<grid_for(B->nR, 256), 256, 0, s>>>(B->nR, B->nA, B->rexp, B->rijk, B->rbase, B->rcp, ijkG, ebase, ecp));
    CPM_CUDA(cudaGetLastError());
  }
  if (perm) {
    KL(k_iota64<<<grid_for(B->nA, 256), 256, 0, s>>>(perm, B->nA));
    CPM_CUDA(cudaGetLastError());
  }
  return CPM_OK;
}

cpm_status band_weights(const cpm_band* B, double* w, cudaStream_t s) {
  KL(k_export_w<<<grid_for(B->nR, 256), 256, 0, s>>>(B->nR, B->p + 1, B->rexp, B->w1d, w));
  CPM_CUDA(cudaGetLastError());
  return CPM_OK;
}

}  // namespace cpm
