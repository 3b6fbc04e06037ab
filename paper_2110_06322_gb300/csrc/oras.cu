// oras.cu -- set-up of the restricted additive Schwarz preconditioner
// (Section 2.2; defaults of Section 4.1.1) on the GPU:
//
//   assemble   M = (c + 6/h^2) I - L_off E as CSR, one warp per row: the six
//              neighbour cubes (already in ascending column order) are merged
//              by rank counting, duplicates summed in neighbour/cube order,
//              so M is bit-identical to a sequential assembly
//   partition  recursive coordinate bisection of Sigma_A by lattice planes
//              (per level: boxes and histograms on the device, cut choice on
//              the host)
//   overlap    N_O layers of 6-adjacency within Sigma_A: each node carries the
//              sorted list of subdomains it belongs to
//   order      each subdomain sorted by descending distance to the surface
//              (ties: canonical index), a bitonic sort per subdomain
//   local      A_j = R_j M R_j^T; Robin reading: A_j[i,i] += beta D_i with D_i
//              the sum of the dropped entries of row i, beta = 1/(1 + alpha h)
//   levels     dependency levels of the lower and upper triangles
//   ilu0       level-scheduled ILU(0) (row-by-row IKJ elimination restricted
//              to the pattern), one CTA per subdomain, one warp per row
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "oras.cuh"
#include "surface.cuh"

namespace cpm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int lower_b(const int32_t* a, int n, int32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (a[m] < v) lo = m + 1;
    else hi = m;
  }
  return lo;
}
__device__ __forceinline__ int upper_b(const int32_t* a, int n, int32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int m = (lo + hi) >> 1;
    if (a[m] <= v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// ------------------------------------------------------------------ assemble M
struct AsmArgs {
  Grid g;
  const BitWord* amap;
  const BitWord* rmap;
  const int32_t* ijkA;
  const int32_t* rbase;
  const double* w1d;
  int64_t nA;
  double coef, diag0;
};

constexpr int ASM_WARPS = 4;

template <int P>
__global__ void __launch_bounds__(ASM_WARPS * 32)
    k_assemble(AsmArgs A, const int64_t* __restrict__ mptr, int32_t* cnt, int32_t* ocol, double* oval) {
  constexpr int P1 = P + 1, NC = P1 * P1 * P1, NL = 6 * NC + 1;
  __shared__ int32_t s_lcol[ASM_WARPS][NL];
  __shared__ double s_lterm[ASM_WARPS][NL];
  __shared__ int32_t s_mcol[ASM_WARPS][NL];
  __shared__ int16_t s_mpos[ASM_WARPS][NL];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* lcol = s_lcol[wid];
  double* lterm = s_lterm[wid];
  int32_t* mcol = s_mcol[wid];
  int16_t* mpos = s_mpos[wid];
  for (int64_t i = (int64_t)blockIdx.x * ASM_WARPS + wid; i < A.nA; i += (int64_t)gridDim.x * ASM_WARPS) {
    const int x0 = A.ijkA[3 * i], x1 = A.ijkA[3 * i + 1], x2 = A.ijkA[3 * i + 2];
    // list entries: neighbour n (-x,+x,-y,+y,-z,+z), cube position (u,v,t)
    for (int pc = lane; pc < 6 * P1 * P1; pc += 32) {
      const int n = pc / (P1 * P1), uv = pc % (P1 * P1), u = uv / P1, v = uv % P1;
      const int dx = n == 0 ? -1 : (n == 1 ? 1 : 0), dy = n == 2 ? -1 : (n == 3 ? 1 : 0),
                dz = n == 4 ? -1 : (n == 5 ? 1 : 0);
      const int32_t r = bm_rank_known(A.rmap, A.g, x0 + dx, x1 + dy, x2 + dz);
      const int32_t* b = A.rbase + 3 * (int64_t)r;
      const int32_t q0 = bm_rank_known(A.amap, A.g, b[0] + u, b[1] + v, b[2]);
      const double* w = A.w1d + (int64_t)r * 3 * P1;
      const double wuv = mptr ? dm(w[u], w[P1 + v]) : 0.0;  // the counting pass needs columns only
#pragma unroll
      for (int t = 0; t < P1; ++t) {
        const int pos = n * NC + uv * P1 + t;
        lcol[pos] = q0 + t;
        if (mptr) lterm[pos] = dm(A.coef, dm(wuv, w[2 * P1 + t]));
      }
    }
    if (lane == 0) {  // diagonal marker, last in list order
      lcol[6 * NC] = (int32_t)i;
      lterm[6 * NC] = 0.0;
    }
    __syncwarp();
    // stable merge of the 7 sorted runs by rank counting
    for (int e = lane; e < NL; e += 32) {
      const int a = e / NC, t = e - a * NC;
      const int32_t c = lcol[e];
      int rank = t;
#pragma unroll
      for (int b = 0; b < 7; ++b) {
        if (b == a) continue;
        const int nb = b == 6 ? 1 : NC;
        rank += (b < a) ? upper_b(lcol + b * NC, nb, c) : lower_b(lcol + b * NC, nb, c);
      }
      mcol[rank] = c;
      mpos[rank] = (int16_t)e;
    }
    __syncwarp();
    int nout = 0;
    for (int b0 = 0; b0 < NL; b0 += 32) {
      const int e = b0 + lane;
      const bool head = e < NL && (e == 0 || mcol[e] != mcol[e - 1]);
      const unsigned bal = __ballot_sync(FULL, head);
      if (head && mptr) {
        double sacc = lterm[mpos[e]];
        for (int f = e + 1; f < NL && mcol[f] == mcol[e]; ++f) sacc = da(sacc, lterm[mpos[f]]);
        const int32_t c = mcol[e];
        const double v = (c == (int32_t)i) ? dsb(A.diag0, sacc) : -sacc;
        const int64_t o = mptr[i] + nout + __popc(bal & ((1u << lane) - 1u));
        ocol[o] = c;
        oval[o] = v;
      }
      nout += __popc(bal);
    }
    if (!mptr && lane == 0) cnt[i] = nout;
    __syncwarp();
  }
}

// ------------------------------------------------------------------ partition
__global__ void k_seg_box(int64_t nA, const int32_t* __restrict__ ijkA, const int32_t* __restrict__ segof,
                          const int32_t* __restrict__ segnp, int* box, int* cnt) {
  // grid-stride over whole warps so that every lane takes part in the shuffles
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); q0 < nA; q0 += stride) {
    const int64_t q = q0 + lane;
    const bool in = q < nA;
    const int s = in ? segof[q] : -1;
    const bool act = in && segnp[s] > 1;
    int v[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    if (act)
      for (int d = 0; d < 3; ++d) v[d] = v[3 + d] = ijkA[3 * q + d];
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    if (__all_sync(0xffffffffu, s == s0 && act)) {
      // one segment for the whole warp: reduce, then one lane updates
      for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; ++d) {
          v[d] = min(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
          v[3 + d] = max(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
        }
      if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
          atomicMin(&box[6 * s0 + d], v[d]);
          atomicMax(&box[6 * s0 + 3 + d], v[3 + d]);
        }
        atomicAdd(&cnt[s0], 32);
      }
    } else if (act) {
      for (int d = 0; d < 3; ++d) {
        atomicMin(&box[6 * s + d], v[d]);
        atomicMax(&box[6 * s + 3 + d], v[3 + d]);
      }
      atomicAdd(&cnt[s], 1);
    }
  }
}

__global__ void k_seg_hist(int64_t nA, const int32_t* __restrict__ ijkA, const int32_t* __restrict__ segof,
                           const int32_t* __restrict__ sax, const int32_t* __restrict__ smin,
                           const int64_t* __restrict__ shoff, int32_t* hist) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    int s = segof[q];
    if (sax[s] < 0) continue;
    atomicAdd(&hist[shoff[s] + ijkA[3 * q + sax[s]] - smin[s]], 1);
  }
}

__global__ void k_seg_split(int64_t nA, const int32_t* __restrict__ ijkA, int32_t* segof,
                            const int32_t* __restrict__ sax, const int32_t* __restrict__ scut,
                            const int32_t* __restrict__ sleft, const int32_t* __restrict__ sright) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    int s = segof[q];
    if (sax[s] < -1) continue;  // final segment
    segof[q] = ijkA[3 * q + (sax[s] < 0 ? 0 : sax[s])] < scut[s] ? sleft[s] : sright[s];
  }
}

__global__ void k_seg_final(int64_t nA, const int32_t* __restrict__ segof, const int32_t* __restrict__ segoff,
                            int32_t* part) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x)
    part[q] = segoff[segof[q]];
}

template <typename T>
cpm_status upload(T** d, const std::vector<T>& h, cudaStream_t s) {
  CPM_TRY(dalloc(d, h.size(), s));
  if (!h.empty()) CPM_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return CPM_OK;
}

// Recursive coordinate bisection by lattice planes: a set is cut normal to
// its longest extent (ties: i, j, k) at the plane v minimising
// |count(coord < v) - n * nl / np| (ties: smaller v), nl = floor(np / 2).
cpm_status partition_rcb(const cpm_band* B, int np, int32_t* part, cudaStream_t s) {
  const int64_t nA = B->nA;
  struct Seg {
    int np, off;
  };
  std::vector<Seg> segs{{np, 0}};
  int32_t* segof = nullptr;
  CPM_TRY(dalloc(&segof, nA, s));
  CPM_CUDA(cudaMemsetAsync(segof, 0, nA * sizeof(int32_t), s));
  const int G = grid_for(nA, 256);
  while (true) {
    const int ns = (int)segs.size();
    bool any = false;
    for (auto& sg : segs) any |= sg.np > 1;
    if (!any) break;
    std::vector<int32_t> hnp(ns), hbox(6 * ns), hcnt(ns, 0);
    for (int q = 0; q < ns; ++q) {
      hnp[q] = segs[q].np;
      for (int d = 0; d < 3; ++d) { hbox[6 * q + d] = INT_MAX; hbox[6 * q + 3 + d] = INT_MIN; }
    }
    int32_t *dnp = nullptr, *dbox = nullptr, *dcnt = nullptr;
    CPM_TRY(upload(&dnp, hnp, s));
    CPM_TRY(upload(&dbox, hbox, s));
    CPM_TRY(upload(&dcnt, hcnt, s));
    KL(k_seg_box<<<G, 256, 0, s>>>(nA, B->ijkA, segof, dnp, dbox, dcnt));
    CPM_CUDA(cudaMemcpyAsync(hbox.data(), dbox, hbox.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaMemcpyAsync(hcnt.data(), dcnt, hcnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
    // axis and histogram layout per splitting segment
    std::vector<int32_t> sax(ns, -2), smin(ns, 0), scut(ns, 0), sleft(ns, 0), sright(ns, 0);
    std::vector<int64_t> shoff(ns, 0);
    int64_t htot = 0;
    for (int q = 0; q < ns; ++q) {
      if (segs[q].np <= 1) continue;
      if (hcnt[q] == 0) {
        sax[q] = -1;  // empty: all (none) go right
        continue;
      }
      int ax = 0;
      for (int a = 1; a < 3; ++a)
        if (hbox[6 * q + 3 + a] - hbox[6 * q + a] > hbox[6 * q + 3 + ax] - hbox[6 * q + ax]) ax = a;
      sax[q] = ax;
      smin[q] = hbox[6 * q + ax];
      shoff[q] = htot;
      htot += hbox[6 * q + 3 + ax] - hbox[6 * q + ax] + 1;
    }
    int32_t *dax = nullptr, *dmin = nullptr, *dhist = nullptr;
    int64_t* dhoff = nullptr;
    CPM_TRY(upload(&dax, sax, s));
    CPM_TRY(upload(&dmin, smin, s));
    CPM_TRY(upload(&dhoff, shoff, s));
    CPM_TRY(dalloc(&dhist, htot, s));
    CPM_CUDA(cudaMemsetAsync(dhist, 0, std::max<int64_t>(htot, 1) * sizeof(int32_t), s));
    KL(k_seg_hist<<<G, 256, 0, s>>>(nA, B->ijkA, segof, dax, dmin, dhoff, dhist));
    std::vector<int32_t> hh(std::max<int64_t>(htot, 1));
    CPM_CUDA(cudaMemcpyAsync(hh.data(), dhist, hh.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CPM_CUDA(cudaStreamSynchronize(s));
    std::vector<Seg> next = segs;
    for (int q = 0; q < ns; ++q) {
      if (segs[q].np <= 1) continue;
      const int npq = segs[q].np, nl = npq / 2;
      const int64_t n = hcnt[q];
      int best_v = 0;
      if (sax[q] >= 0) {
        const int ax = sax[q], mn = hbox[6 * q + ax], mx = hbox[6 * q + 3 + ax];
        int64_t best_err = -1, below = 0;
        best_v = mn;
        for (int v = mn; v <= mx + 1; ++v) {
          int64_t err = std::llabs((int64_t)npq * below - n * (int64_t)nl);
          if (best_err < 0 || err < best_err) { best_err = err; best_v = v; }
          if (v <= mx) below += hh[shoff[q] + (v - mn)];
        }
      }
      scut[q] = best_v;
      sleft[q] = (int32_t)next.size();
      next.push_back({nl, segs[q].off});
      sright[q] = (int32_t)next.size();
      next.push_back({npq - nl, segs[q].off + nl});
      next[q].np = 0;  // split: no longer a leaf
    }
    int32_t *dcut = nullptr, *dl = nullptr, *dr = nullptr;
    CPM_TRY(upload(&dcut, scut, s));
    CPM_TRY(upload(&dl, sleft, s));
    CPM_TRY(upload(&dr, sright, s));
    KL(k_seg_split<<<G, 256, 0, s>>>(nA, B->ijkA, segof, dax, dcut, dl, dr));
    CPM_CUDA(cudaGetLastError());
    CPM_CUDA(cudaStreamSynchronize(s));
    for (auto* p : {dnp, dbox, dcnt, dax, dmin, dhist, dcut, dl, dr}) cudaFreeAsync(p, s);
    cudaFreeAsync(dhoff, s);
    segs.swap(next);
  }
  std::vector<int32_t> off(segs.size());
  for (size_t q = 0; q < segs.size(); ++q) off[q] = segs[q].off;
  int32_t* doff = nullptr;
  CPM_TRY(upload(&doff, off, s));
  KL(k_seg_final<<<G, 256, 0, s>>>(nA, segof, doff, part));
  CPM_CUDA(cudaGetLastError());
  dfree(doff, s);
  dfree(segof, s);
  return CPM_OK;
}

// ------------------------------------------------------------------ overlap
__global__ void k_memb_init(int64_t nA, const int32_t* __restrict__ part, int32_t* memb, int32_t* mcnt) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    memb[q * KMEM] = part[q];
    mcnt[q] = 1;
  }
}

// one layer of 6-adjacency growth: union of the node's list and its active
// neighbours' lists (all sorted ascending)
__global__ void k_memb_layer(Grid g, const BitWord* __restrict__ amap, const int32_t* __restrict__ ijkA, int64_t nA,
                             const int32_t* __restrict__ mi, const int32_t* __restrict__ ci, int32_t* mo, int32_t* co,
                             int* err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    int32_t L[KMEM];
    int n = ci[q];
    for (int t = 0; t < n; ++t) L[t] = mi[q * KMEM + t];
    const int i = ijkA[3 * q], j = ijkA[3 * q + 1], k = ijkA[3 * q + 2];
    const int nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int d = 0; d < 6; ++d) {
      int32_t m = bm_rank(amap, g, i + nb[d][0], j + nb[d][1], k + nb[d][2]);
      if (m < 0) continue;
      for (int t = 0; t < ci[m]; ++t) {
        int32_t v = mi[(int64_t)m * KMEM + t];
        int pos = 0;
        while (pos < n && L[pos] < v) ++pos;
        if (pos < n && L[pos] == v) continue;
        if (n == KMEM) {
          atomicExch(err, CPM_ERR_ARG);
          continue;
        }
        for (int u = n; u > pos; --u) L[u] = L[u - 1];
        L[pos] = v;
        ++n;
      }
    }
    for (int t = 0; t < n; ++t) mo[q * KMEM + t] = L[t];
    co[q] = n;
  }
}

__global__ void k_sub_count(int64_t nA, const int32_t* __restrict__ memb, const int32_t* __restrict__ mcnt,
                            int32_t* scnt) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x)
    for (int t = 0; t < mcnt[q]; ++t) atomicAdd(&scnt[memb[q * KMEM + t]], 1);
}

__global__ void k_sub_fill(int64_t nA, const int32_t* __restrict__ memb, const int32_t* __restrict__ mcnt,
                           const int64_t* __restrict__ sptr, int32_t* cursor, int32_t* snode) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x)
    for (int t = 0; t < mcnt[q]; ++t) {
      int32_t j = memb[q * KMEM + t];
      int32_t slot = atomicAdd(&cursor[j], 1);
      snode[sptr[j] + slot] = (int32_t)q;
    }
}

// sort keys: descending distance (bit pattern of a non-negative double is
// monotone), then ascending canonical index
// Sort keys of the local order (ascending key, ties by canonical index):
// order 1: descending distance to the surface;
// order 2: distance shells of width h, outermost first (shell = floor(dist / h),
//          correctly rounded division as in the oracle), then the 8 colours of
//          the lattice parity (i mod 2, j mod 2, k mod 2).
__global__ void k_sort_prep(SurfDev S, double h, int order, const int32_t* __restrict__ ijkA, int np,
                            const int64_t* __restrict__ sptr, const int64_t* __restrict__ poff,
                            const int32_t* __restrict__ snode, unsigned long long* key, int32_t* val) {
  const int j = blockIdx.x;
  const int64_t n = sptr[j + 1] - sptr[j], N = poff[j + 1] - poff[j];
  for (int64_t t = threadIdx.x; t < N; t += blockDim.x) {
    if (t < n) {
      const int32_t q = snode[sptr[j] + t];
      const double d = surf_dist(S, dm((double)ijkA[3 * q], h), dm((double)ijkA[3 * q + 1], h),
                                 dm((double)ijkA[3 * q + 2], h));
      if (order == 2) {
        const unsigned long long shell = (unsigned long long)floor(ddv(d, h));
        const unsigned colour = (unsigned)((ijkA[3 * q] & 1) | ((ijkA[3 * q + 1] & 1) << 1) | ((ijkA[3 * q + 2] & 1) << 2));
        key[poff[j] + t] = ((0xFFFFFFFFull - shell) << 3) | colour;
      } else {
        key[poff[j] + t] = ~(unsigned long long)__double_as_longlong(d);
      }
      val[poff[j] + t] = q;
    } else {
      key[poff[j] + t] = ~0ull;
      val[poff[j] + t] = INT_MAX;
    }
  }
}

__global__ void __launch_bounds__(1024) k_bitonic_sub(const int64_t* __restrict__ poff, unsigned long long* key,
                                                      int32_t* val) {
  const int j = blockIdx.x;
  const int64_t N = poff[j + 1] - poff[j];
  unsigned long long* K = key + poff[j];
  int32_t* V = val + poff[j];
  for (int64_t k = 2; k <= N; k <<= 1)
    for (int64_t jj = k >> 1; jj > 0; jj >>= 1) {
      for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const int64_t l = i ^ jj;
        if (l > i) {
          const bool up = (i & k) == 0;
          const unsigned long long ka = K[i], kb = K[l];
          const int32_t va = V[i], vb = V[l];
          const bool gt = ka > kb || (ka == kb && va > vb);
          if (gt == up) {
            K[i] = kb;
            K[l] = ka;
            V[i] = vb;
            V[l] = va;
          }
        }
      }
      __syncthreads();
    }
}

__global__ void k_sort_back(int np, const int64_t* __restrict__ sptr, const int64_t* __restrict__ poff,
                            const int32_t* __restrict__ val, const int32_t* __restrict__ part, int32_t* snode,
                            uint8_t* owned, int32_t* lsub) {
  const int j = blockIdx.x;
  const int64_t n = sptr[j + 1] - sptr[j];
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    const int32_t q = val[poff[j] + t];
    snode[sptr[j] + t] = q;
    owned[sptr[j] + t] = part[q] == j;
    lsub[sptr[j] + t] = j;
  }
}

__global__ void k_mloc(int64_t nloc, const int32_t* __restrict__ snode, const int32_t* __restrict__ lsub,
                       const int32_t* __restrict__ memb, const int32_t* __restrict__ mcnt, int32_t* mloc) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nloc; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = snode[q];
    for (int t = 0; t < mcnt[m]; ++t)
      if (memb[m * KMEM + t] == lsub[q]) mloc[m * KMEM + t] = (int32_t)q;
  }
}

// ------------------------------------------------------------------ local matrices
constexpr int LOC_WARPS = 2;
constexpr int MAXROW = 512;

struct LocArgs {
  int64_t nloc;
  const int32_t* snode;
  const int32_t* lsub;
  const int64_t* sptr;
  const int32_t* part;
  const int32_t* memb;
  const int32_t* mcnt;
  const int32_t* mloc;
  const int64_t* mptr;  // global M
  const int32_t* mcol;
  const double* mval;
  int robin;
  double beta, beta_x;
};

__device__ __forceinline__ int32_t local_col(const LocArgs& A, int32_t m, int32_t j) {
  for (int t = 0; t < A.mcnt[m]; ++t)
    if (A.memb[(int64_t)m * KMEM + t] == j) return A.mloc[(int64_t)m * KMEM + t];
  return -1;
}

__global__ void __launch_bounds__(LOC_WARPS * 32)
    k_local(LocArgs A, const int64_t* __restrict__ rptr, int32_t* cnt, int32_t* lcol, double* lval, int32_t* dpos,
            int* err) {
  __shared__ int32_t s_col[LOC_WARPS][MAXROW];
  __shared__ double s_val[LOC_WARPS][MAXROW];
  __shared__ double s_drop[LOC_WARPS][MAXROW];
  __shared__ int32_t s_own[LOC_WARPS][MAXROW];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* scol = s_col[wid];
  double* sval = s_val[wid];
  double* sdrop = s_drop[wid];
  int32_t* sown = s_own[wid];
  for (int64_t q = (int64_t)blockIdx.x * LOC_WARPS + wid; q < A.nloc; q += (int64_t)gridDim.x * LOC_WARPS) {
    const int32_t i = A.snode[q], j = A.lsub[q];
    const int64_t base = A.sptr[j];
    const int64_t e0 = A.mptr[i], e1 = A.mptr[i + 1];
    if (e1 - e0 > MAXROW) {
      if (lane == 0) {
        atomicExch(err, CPM_ERR_ARG);
        if (!rptr) cnt[q] = 0;
      }
      continue;
    }
    int nk = 0, nd = 0;
    for (int64_t b0 = e0; b0 < e1; b0 += 32) {
      const int64_t e = b0 + lane;
      int32_t lc = -1;
      if (e < e1) lc = local_col(A, A.mcol[e], j);
      const bool kept = e < e1 && lc >= 0, drop = e < e1 && lc < 0;
      const unsigned bk = __ballot_sync(FULL, kept), bd = __ballot_sync(FULL, drop);
      const unsigned below = (1u << lane) - 1u;
      if (kept) {
        const int o = nk + __popc(bk & below);
        scol[o] = (int32_t)(lc - base);
        sval[o] = A.mval[e];
      }
      if (drop) {
        const int o = nd + __popc(bd & below);
        sdrop[o] = A.mval[e];
        sown[o] = A.part[A.mcol[e]];
      }
      nk += __popc(bk);
      nd += __popc(bd);
    }
    __syncwarp();
    if (!rptr) {
      if (lane == 0) cnt[q] = nk;
      __syncwarp();
      continue;
    }
    if (lane == 0 && A.robin && nd > 0) {
      double D = 0.0;
      bool cross = false;
      for (int t = 0; t < nd; ++t) {
        D = da(D, sdrop[t]);
        cross |= sown[t] != sown[0];
      }
      const int32_t me = (int32_t)(q - base);
      for (int t = 0; t < nk; ++t)
        if (scol[t] == me) sval[t] = da(sval[t], dm(cross ? A.beta_x : A.beta, D));
    }
    __syncwarp();
    // sort the kept entries by local column (bitonic, padded)
    int N = 1;
    while (N < nk) N <<= 1;
    for (int t = nk + lane; t < N; t += 32) scol[t] = INT_MAX;
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1)
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int t = lane; t < N; t += 32) {
          const int l = t ^ jj;
          if (l > t) {
            const bool up = (t & k) == 0;
            const int32_t ca = scol[t], cb = scol[l];
            if ((ca > cb) == up) {
              scol[t] = cb;
              scol[l] = ca;
              const double va = sval[t];
              sval[t] = sval[l];
              sval[l] = va;
            }
          }
        }
        __syncwarp();
      }
    const int64_t o = rptr[q];
    for (int t = lane; t < nk; t += 32) {
      lcol[o + t] = scol[t];
      lval[o + t] = sval[t];
      if (scol[t] == (int32_t)(q - base)) dpos[q] = t;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ level schedules
// One warp per subdomain.  lower = 1: dependencies are the entries left of
// the diagonal (rows in ascending order); lower = 0: right of the diagonal
// (rows in descending order).
__global__ void k_levels(int np, const int64_t* __restrict__ sptr, const int64_t* __restrict__ rptr,
                         const int32_t* __restrict__ col, const int32_t* __restrict__ dpos, int lower, int32_t* lev,
                         int32_t* nlev) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= np) return;
  const int64_t base = sptr[j], n = sptr[j + 1] - base;
  int32_t mx = 0;
  for (int64_t t = 0; t < n; ++t) {
    const int64_t q = base + (lower ? t : n - 1 - t);
    const int64_t e0 = lower ? rptr[q] : rptr[q] + dpos[q] + 1;
    const int64_t e1 = lower ? rptr[q] + dpos[q] : rptr[q + 1];
    int32_t l = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) l = max(l, lev[base + col[e]]);
    for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(FULL, l, o));
    if (lane == 0) lev[q] = l + 1;
    mx = max(mx, l + 1);
    __syncwarp();
  }
  if (lane == 0) nlev[j] = mx;
}

// The same with the subdomain's levels in shared memory (16-bit: a level is
// at most the row count, below 2^15 here) and the next row's bounds and
// columns loaded while the current row is reduced: one warp per subdomain,
// one warp per block, so many subdomains share an SM.
constexpr int LEV_PF = 3;  // dependency columns per lane fetched a row ahead
__global__ void __launch_bounds__(32)
    k_levels_smem(const int64_t* __restrict__ sptr, const int64_t* __restrict__ rptr,
                  const int32_t* __restrict__ col, const int32_t* __restrict__ dpos, int lower, int32_t* lev,
                  int32_t* nlev) {
  extern __shared__ uint16_t slev[];  // levels <= rows <= 65535 (16-bit local columns)
  const int lane = threadIdx.x;
  const int j = blockIdx.x;
  const int64_t base = sptr[j], n = sptr[j + 1] - base;
  auto bounds = [&](int64_t t, int64_t& e0, int64_t& e1) {
    const int64_t q = base + (lower ? t : n - 1 - t);
    e0 = lower ? rptr[q] : rptr[q] + dpos[q] + 1;
    e1 = lower ? rptr[q] + dpos[q] : rptr[q + 1];
  };
  int64_t e0 = 0, e1 = 0;
  int32_t c[LEV_PF];
  if (n > 0) {
    bounds(0, e0, e1);
#pragma unroll
    for (int k = 0; k < LEV_PF; ++k) c[k] = e0 + lane + 32 * k < e1 ? col[e0 + lane + 32 * k] : -1;
  }
  int32_t mx = 0;
  for (int64_t t = 0; t < n; ++t) {
    int64_t f0 = 0, f1 = 0;
    int32_t cn[LEV_PF];
    if (t + 1 < n) {
      bounds(t + 1, f0, f1);
#pragma unroll
      for (int k = 0; k < LEV_PF; ++k) cn[k] = f0 + lane + 32 * k < f1 ? col[f0 + lane + 32 * k] : -1;
    }
    int32_t l = 0;
#pragma unroll
    for (int k = 0; k < LEV_PF; ++k)
      if (c[k] >= 0) l = max(l, (int32_t)slev[c[k]]);
    for (int64_t e = e0 + lane + 32 * LEV_PF; e < e1; e += 32) l = max(l, (int32_t)slev[col[e]]);
    for (int o = 16; o > 0; o >>= 1) l = max(l, __shfl_xor_sync(FULL, l, o));
    const int64_t tl = lower ? t : n - 1 - t;
    if (lane == 0) {
      slev[tl] = (uint16_t)(l + 1);
      lev[base + tl] = l + 1;
    }
    mx = max(mx, l + 1);
    __syncwarp();
    e0 = f0;
    e1 = f1;
#pragma unroll
    for (int k = 0; k < LEV_PF; ++k) c[k] = cn[k];
  }
  if (lane == 0) nlev[j] = mx;
}

__global__ void k_level_count(int64_t nloc, const int32_t* __restrict__ lsub, const int32_t* __restrict__ lvsub,
                              const int32_t* __restrict__ lev, int32_t* lcnt) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nloc; q += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&lcnt[lvsub[lsub[q]] + lev[q] - 1], 1);
}

__global__ void k_level_fill(int64_t nloc, const int32_t* __restrict__ lsub, const int32_t* __restrict__ lvsub,
                             const int32_t* __restrict__ lev, const int64_t* __restrict__ lvptr, int32_t* cursor,
                             int32_t* lvrow) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nloc; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t L = lvsub[lsub[q]] + lev[q] - 1;
    const int32_t slot = atomicAdd(&cursor[L], 1);
    lvrow[lvptr[L] + slot] = (int32_t)q;
  }
}

// ------------------------------------------------------------------ ILU(0)
constexpr int ILU_WARPS = 16;
constexpr int ILU_PF = 4;  // entries per lane of the next pivot row held in registers

struct PivotRow {
  double rpiv;  // 1 / u_kk
  int64_t kd, k1;
  int32_t c[ILU_PF];
  double u[ILU_PF];
};

// strict upper part of pivot row kq (final: computed in an earlier level)
__device__ __forceinline__ void load_pivot(const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                                           const int32_t* __restrict__ dpos, const double* val, const double* rinv,
                                           int64_t kq, int lane, PivotRow& R) {
  R.kd = rptr[kq] + dpos[kq];
  R.k1 = rptr[kq + 1];
  R.rpiv = rinv[kq];
#pragma unroll
  for (int k = 0; k < ILU_PF; ++k) {
    const int64_t e = R.kd + 1 + lane + 32 * k;
    R.c[k] = e < R.k1 ? col[e] : -1;
    R.u[k] = e < R.k1 ? val[e] : 0.0;
  }
}

// One CTA per subdomain, one warp per row of the current level.  Row i is
// eliminated in shared memory: for each k < i of its pattern (ascending),
// a_ik *= 1 / u_kk, then a_ij -= a_ik u_kj (one fused multiply-add) for the
// j > k of row k's pattern that row i also holds (binary search), in FP64.
// A finished row stores the reciprocal of its pivot for the rows below it,
// so each row costs one division; the factors agree with the division-and-
// separate-rounding form to a few units in the last place.  FP64 throughput is
// the bound here: every warp-wide FP64 instruction costs the same whether one
// lane or 32 use it.
__global__ void __launch_bounds__(ILU_WARPS * 32)
    k_ilu0(const int64_t* __restrict__ sptr, const int32_t* __restrict__ lvsub, const int64_t* __restrict__ lvptr,
           const int32_t* __restrict__ lvrow, const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
           const int32_t* __restrict__ dpos, double* val, double* rinv, int* err) {
  extern __shared__ __align__(16) unsigned char ilu_smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* sval = reinterpret_cast<double*>(ilu_smem) + wid * MAXROW;
  int32_t* scol = reinterpret_cast<int32_t*>(ilu_smem + ILU_WARPS * MAXROW * sizeof(double)) + wid * MAXROW;
  const int j = blockIdx.x;
  const int64_t base = sptr[j];
  for (int32_t L = lvsub[j]; L < lvsub[j + 1]; ++L) {
    for (int64_t idx = lvptr[L] + wid; idx < lvptr[L + 1]; idx += ILU_WARPS) {
      const int64_t q = lvrow[idx];
      const int64_t e0 = rptr[q];
      const int n = (int)(rptr[q + 1] - e0), d = dpos[q];
      for (int t = lane; t < n; t += 32) {
        scol[t] = col[e0 + t];
        sval[t] = val[e0 + t];
      }
      __syncwarp();
      PivotRow cur, nxt;
      if (d > 0) load_pivot(rptr, col, dpos, val, rinv, base + scol[0], lane, cur);
      for (int t = 0; t < d; ++t) {
        if (t + 1 < d) load_pivot(rptr, col, dpos, val, rinv, base + scol[t + 1], lane, nxt);
        const double l = dm(sval[t], cur.rpiv);
        __syncwarp();
        if (lane == 0) sval[t] = l;
#pragma unroll
        for (int k = 0; k < ILU_PF; ++k) {
          const int32_t c = cur.c[k];
          if (c >= 0) {
            const int pos = lower_b(scol, n, c);
            if (pos < n && scol[pos] == c) sval[pos] = __fma_rn(-l, cur.u[k], sval[pos]);
          }
        }
        for (int64_t e = cur.kd + 1 + 32 * ILU_PF + lane; e < cur.k1; e += 32) {
          const int32_t c = col[e];
          const int pos = lower_b(scol, n, c);
          if (pos < n && scol[pos] == c) sval[pos] = __fma_rn(-l, val[e], sval[pos]);
        }
        __syncwarp();
        cur = nxt;
      }
      if (lane == 0) {
        if (sval[d] == 0.0) atomicExch(err, CPM_ERR_BREAKDOWN);
        rinv[q] = ddv(1.0, sval[d]);
      }
      for (int t = lane; t < n; t += 32) val[e0 + t] = sval[t];
      __syncwarp();
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ transposed factors
__global__ void k_tcount_f(int64_t nloc, const int64_t* __restrict__ sptr, const int32_t* __restrict__ lsub,
                           const int64_t* __restrict__ rptr, const int32_t* __restrict__ col, int32_t* cnt) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nloc; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = sptr[lsub[q]];
    for (int64_t e = rptr[q]; e < rptr[q + 1]; ++e) atomicAdd(&cnt[base + col[e]], 1);
  }
}
__global__ void k_tfill_f(int64_t nloc, const int64_t* __restrict__ sptr, const int32_t* __restrict__ lsub,
                          const int64_t* __restrict__ rptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const int64_t* __restrict__ tptr, int32_t* cursor,
                          int32_t* tcol, double* tval) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nloc; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = sptr[lsub[q]];
    for (int64_t e = rptr[q]; e < rptr[q + 1]; ++e) {
      const int64_t r = base + col[e];
      const int32_t slot = atomicAdd(&cursor[r], 1);
      tcol[tptr[r] + slot] = (int32_t)(q - base);
      tval[tptr[r] + slot] = val[e];
    }
  }
}
// Sort each transposed row by local column and record its diagonal's place.
// One warp per row: the columns of a row are distinct, so an entry's place is
// the number of smaller columns (counted from a shared-memory copy); rows
// longer than the staging buffer fall back to an insertion sort by one lane.
constexpr int TSORT_WARPS = 4, TSORT_CAP = 512;
__global__ void __launch_bounds__(TSORT_WARPS * 32)
    k_tsort_f(int64_t nloc, const int64_t* __restrict__ sptr, const int32_t* __restrict__ lsub,
              const int64_t* __restrict__ tptr, int32_t* tcol, double* tval, int32_t* tdpos) {
  __shared__ int32_t sc[TSORT_WARPS][TSORT_CAP];
  __shared__ double sv[TSORT_WARPS][TSORT_CAP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nloc;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t a = tptr[q];
    const int n = (int)(tptr[q + 1] - a);
    const int32_t me = (int32_t)(q - sptr[lsub[q]]);
    if (n <= TSORT_CAP) {
      for (int i = lane; i < n; i += 32) {
        sc[wid][i] = tcol[a + i];
        sv[wid][i] = tval[a + i];
      }
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        const int32_t c = sc[wid][i];
        int r = 0;
        for (int k = 0; k < n; ++k) r += sc[wid][k] < c ? 1 : 0;
        tcol[a + r] = c;
        tval[a + r] = sv[wid][i];
        if (c == me) tdpos[q] = r;
      }
      __syncwarp();
    } else if (lane == 0) {
      for (int64_t i = a + 1; i < a + n; ++i) {
        const int32_t c = tcol[i];
        const double v = tval[i];
        int64_t k = i - 1;
        while (k >= a && tcol[k] > c) {
          tcol[k + 1] = tcol[k];
          tval[k + 1] = tval[k];
          --k;
        }
        tcol[k + 1] = c;
        tval[k + 1] = v;
      }
      for (int64_t i = a; i < a + n; ++i)
        if (tcol[i] == me) tdpos[q] = (int32_t)(i - a);
    }
    __syncwarp();
  }
}

cpm_status build_schedule(oras_pc* P, const int64_t* rptr, const int32_t* col, const int32_t* dpos, int lower,
                          int32_t** lvsub_out, int64_t** lvptr_out, int32_t** lvrow_out, int32_t* maxlev,
                          cudaStream_t s) {
  const int np = P->np;
  const int64_t nloc = P->nloc;
  int32_t *lev = nullptr, *nlev = nullptr;
  CPM_TRY(dalloc(&lev, nloc, s));
  CPM_TRY(dalloc(&nlev, np, s));
  if (P->max_rows <= 65535 && P->max_rows * (int64_t)sizeof(uint16_t) <= 200 * 1024) {
    const int sm = (int)std::max<int64_t>(P->max_rows * (int64_t)sizeof(uint16_t), 16);
    CPM_CUDA(cudaFuncSetAttribute(k_levels_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    KL(k_levels_smem<<<np, 32, sm, s>>>(P->sptr, rptr, col, dpos, lower, lev, nlev));
  } else {
    KL(k_levels<<<(np + 3) / 4, 128, 0, s>>>(np, P->sptr, rptr, col, dpos, lower, lev, nlev));
  }
  CPM_CUDA(cudaGetLastError());
  std::vector<int32_t> hn(np);
  CPM_CUDA(cudaMemcpyAsync(hn.data(), nlev, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> lvsub(np + 1, 0);
  for (int j = 0; j < np; ++j) {
    lvsub[j + 1] = lvsub[j] + hn[j];
    *maxlev = std::max(*maxlev, hn[j]);
  }
  const int64_t nl = lvsub[np];
  int32_t *dlvsub = nullptr, *lcnt = nullptr, *lvrow = nullptr;
  int64_t* lvptr = nullptr;
  CPM_TRY(upload(&dlvsub, lvsub, s));
  CPM_TRY(dalloc(&lcnt, nl, s));
  CPM_TRY(dalloc(&lvptr, nl + 1, s));
  CPM_TRY(dalloc(&lvrow, nloc, s));
  CPM_CUDA(cudaMemsetAsync(lcnt, 0, std::max<int64_t>(nl, 1) * sizeof(int32_t), s));
  KL(k_level_count<<<grid_for(nloc, 256), 256, 0, s>>>(nloc, P->lsub, dlvsub, lev, lcnt));
  CPM_TRY(scan_exclusive_i32(lcnt, lvptr, nl, s));
  CPM_CUDA(cudaMemsetAsync(lcnt, 0, std::max<int64_t>(nl, 1) * sizeof(int32_t), s));
  KL(k_level_fill<<<grid_for(nloc, 256), 256, 0, s>>>(nloc, P->lsub, dlvsub, lev, lvptr, lcnt, lvrow));
  CPM_CUDA(cudaGetLastError());
  dfree(lev, s);
  dfree(nlev, s);
  dfree(lcnt, s);
  *lvsub_out = dlvsub;
  *lvptr_out = lvptr;
  *lvrow_out = lvrow;
  return CPM_OK;
}

int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

}  // namespace

// Transposed factors and their schedules (for the adjoint), built once.
cpm_status oras_build_transpose(oras_pc* P, cudaStream_t s) {
  if (P->tptr) return CPM_OK;
  const int64_t nloc = P->nloc;
  int32_t* cnt = nullptr;
  CPM_TRY(dalloc(&cnt, nloc, s));
  CPM_CUDA(cudaMemsetAsync(cnt, 0, nloc * sizeof(int32_t), s));
  const int G = grid_for(nloc, 256);
  KL(k_tcount_f<<<G, 256, 0, s>>>(nloc, P->sptr, P->lsub, P->rptr, P->col, cnt));
  CPM_TRY(dalloc(&P->tptr, nloc + 1, s));
  CPM_TRY(scan_exclusive_i32(cnt, P->tptr, nloc, s));
  CPM_TRY(dalloc(&P->tcol, P->nnz, s));
  CPM_TRY(dalloc(&P->tval, P->nnz, s));
  CPM_TRY(dalloc(&P->tdpos, nloc, s));
  CPM_CUDA(cudaMemsetAsync(cnt, 0, nloc * sizeof(int32_t), s));
  KL(k_tfill_f<<<G, 256, 0, s>>>(nloc, P->sptr, P->lsub, P->rptr, P->col, P->val, P->tptr, cnt, P->tcol, P->tval));
  KL(k_tsort_f<<<grid_for(nloc * 32, TSORT_WARPS * 32), TSORT_WARPS * 32, 0, s>>>(nloc, P->sptr, P->lsub,
                                                                                   P->tptr, P->tcol, P->tval, P->tdpos));
  CPM_CUDA(cudaGetLastError());
  dfree(cnt, s);
  int32_t ml = 0;
  CPM_TRY(build_schedule(P, P->tptr, P->tcol, P->tdpos, 1, &P->lvsub_tf, &P->lvptr_tf, &P->lvrow_tf, &ml, s));
  CPM_TRY(build_schedule(P, P->tptr, P->tcol, P->tdpos, 0, &P->lvsub_tb, &P->lvptr_tb, &P->lvrow_tb, &ml, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  return CPM_OK;
}

cpm_status oras_build(const cpm_band* B, const oras_params* prm, double c, cudaStream_t s, oras_pc** out) {
  oras_pc* P = new oras_pc();
  P->band = B;
  P->device = B->device;
  P->np = prm->nparts;
  P->overlap = prm->overlap;
  P->robin = prm->robin;
  P->order = prm->order;
  P->coarse = prm->coarse;
  P->alpha = prm->alpha;
  P->alpha_x = prm->alpha_cross;
  P->store = prm->store;
  P->c = c;
  P->nA = B->nA;
  const int64_t nA = B->nA;
  const int np = P->np;
  int64_t* mptr = nullptr;
  int32_t* mcol = nullptr;
  double* mval = nullptr;
  int32_t *tmp32 = nullptr, *memb2 = nullptr, *mcnt2 = nullptr, *err = nullptr;
  unsigned long long* skey = nullptr;
  int32_t* sval = nullptr;
  int64_t* poff = nullptr;
  auto cleanup = [&](cpm_status st) {
    dfree(mptr, s);
    dfree(mcol, s);
    dfree(mval, s);
    dfree(tmp32, s);
    dfree(memb2, s);
    dfree(mcnt2, s);
    dfree(err, s);
    dfree(skey, s);
    dfree(sval, s);
    dfree(poff, s);
    if (st != CPM_OK) oras_destroy(P, s);
    else *out = P;
    cudaStreamSynchronize(s);
    return st;
  };
#define TRY(x)                                 \
  do {                                         \
    cpm_status st_ = (x);                      \
    if (st_ != CPM_OK) return cleanup(st_);    \
  } while (0)
#define TRYC(x)                                                              \
  do {                                                                       \
    cudaError_t e_ = (x);                                                    \
    if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, #x, __FILE__, __LINE__)); \
  } while (0)
  TRY(dalloc(&err, 1, s));
  TRYC(cudaMemsetAsync(err, 0, sizeof(int), s));
  // ---- global M
  {
    AsmArgs A{B->grid, B->amap, B->rmap, B->ijkA, B->rbase, B->w1d, nA, 0.0, 0.0};
    A.coef = 1.0 / (B->h * B->h);
    A.diag0 = c + 6.0 * A.coef;
    TRY(dalloc(&tmp32, nA, s));
    TRY(dalloc(&mptr, nA + 1, s));
    const int G = grid_for(nA, ASM_WARPS * 32, 152 * 16);
    if (B->p == 3) KL(k_assemble<3><<<G, ASM_WARPS * 32, 0, s>>>(A, nullptr, tmp32, nullptr, nullptr));
    else KL(k_assemble<2><<<G, ASM_WARPS * 32, 0, s>>>(A, nullptr, tmp32, nullptr, nullptr));
    TRYC(cudaGetLastError());
    TRY(scan_exclusive_i32(tmp32, mptr, nA, s));
    int64_t mnnz = 0;
    TRYC(cudaMemcpyAsync(&mnnz, mptr + nA, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRYC(cudaStreamSynchronize(s));
    TRY(dalloc(&mcol, mnnz, s));
    TRY(dalloc(&mval, mnnz, s));
    if (B->p == 3) KL(k_assemble<3><<<G, ASM_WARPS * 32, 0, s>>>(A, mptr, nullptr, mcol, mval));
    else KL(k_assemble<2><<<G, ASM_WARPS * 32, 0, s>>>(A, mptr, nullptr, mcol, mval));
    TRYC(cudaGetLastError());
    dfree(tmp32, s);
  }
  // ---- partition and overlap
  TRY(dalloc(&P->part, nA, s));
  TRY(partition_rcb(B, np, P->part, s));
  TRY(dalloc(&P->memb, nA * KMEM, s));
  TRY(dalloc(&P->mcnt, nA, s));
  TRY(dalloc(&P->mloc, nA * KMEM, s));
  TRY(dalloc(&memb2, nA * KMEM, s));
  TRY(dalloc(&mcnt2, nA, s));
  const int GA = grid_for(nA, 256);
  KL(k_memb_init<<<GA, 256, 0, s>>>(nA, P->part, P->memb, P->mcnt));
  for (int l = 0; l < P->overlap; ++l) {
    KL(k_memb_layer<<<GA, 256, 0, s>>>(B->grid, B->amap, B->ijkA, nA, P->memb, P->mcnt, memb2, mcnt2, err));
    std::swap(P->memb, memb2);
    std::swap(P->mcnt, mcnt2);
  }
  TRYC(cudaGetLastError());
  dfree(memb2, s);
  dfree(mcnt2, s);
  // ---- subdomain node lists, sorted into the local order
  TRY(dalloc(&tmp32, np, s));
  TRYC(cudaMemsetAsync(tmp32, 0, np * sizeof(int32_t), s));
  KL(k_sub_count<<<GA, 256, 0, s>>>(nA, P->memb, P->mcnt, tmp32));
  TRY(dalloc(&P->sptr, np + 1, s));
  TRY(scan_exclusive_i32(tmp32, P->sptr, np, s));
  std::vector<int64_t> hsptr(np + 1);
  TRYC(cudaMemcpyAsync(hsptr.data(), P->sptr, (np + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  P->nloc = hsptr[np];
  const int64_t nloc = P->nloc;
  if (nloc >= INT_MAX) return cleanup(fail(CPM_ERR_ARG, "too many local rows"));
  for (int j = 0; j < np; ++j) P->max_rows = std::max<int64_t>(P->max_rows, hsptr[j + 1] - hsptr[j]);
  for (int j = 0; j < np; ++j)
    if (hsptr[j + 1] - hsptr[j] > (1 << 24))
      return cleanup(fail(CPM_ERR_ARG, "subdomain %d has %lld rows: use more parts", j,
                          (long long)(hsptr[j + 1] - hsptr[j])));
  TRY(dalloc(&P->snode, nloc, s));
  TRYC(cudaMemsetAsync(tmp32, 0, np * sizeof(int32_t), s));
  KL(k_sub_fill<<<GA, 256, 0, s>>>(nA, P->memb, P->mcnt, P->sptr, tmp32, P->snode));
  dfree(tmp32, s);
  std::vector<int64_t> hpoff(np + 1, 0);
  for (int j = 0; j < np; ++j) hpoff[j + 1] = hpoff[j] + next_pow2(hsptr[j + 1] - hsptr[j]);
  TRY(upload(&poff, hpoff, s));
  TRY(dalloc(&skey, hpoff[np], s));
  TRY(dalloc(&sval, hpoff[np], s));
  {
    SurfDev S{};
    S.kind = B->surf.kind;
    for (int d = 0; d < 3; ++d) S.c[d] = B->surf.param[d];
    S.a = B->surf.param[3];
    S.b = B->surf.kind == 1 ? B->surf.param[4] : 0.0;
    KL(k_sort_prep<<<np, 256, 0, s>>>(S, B->h, P->order, B->ijkA, np, P->sptr, poff, P->snode, skey, sval));
  }
  KL(k_bitonic_sub<<<np, 1024, 0, s>>>(poff, skey, sval));
  TRY(dalloc(&P->owned, nloc, s));
  TRY(dalloc(&P->lsub, nloc, s));
  KL(k_sort_back<<<np, 256, 0, s>>>(np, P->sptr, poff, sval, P->part, P->snode, P->owned, P->lsub));
  TRYC(cudaGetLastError());
  dfree(skey, s);
  dfree(sval, s);
  dfree(poff, s);
  const int GL = grid_for(nloc, 256);
  KL(k_mloc<<<GL, 256, 0, s>>>(nloc, P->snode, P->lsub, P->memb, P->mcnt, P->mloc));
  // ---- local matrices
  {
    LocArgs A{nloc, P->snode, P->lsub, P->sptr, P->part, P->memb, P->mcnt, P->mloc, mptr, mcol, mval, P->robin,
              0.0, 0.0};
    A.beta = 1.0 / (1.0 + P->alpha * B->h);
    A.beta_x = 1.0 / (1.0 + P->alpha_x * B->h);
    TRY(dalloc(&tmp32, nloc, s));
    const int G = grid_for(nloc, LOC_WARPS * 32, 152 * 32);
    KL(k_local<<<G, LOC_WARPS * 32, 0, s>>>(A, nullptr, tmp32, nullptr, nullptr, nullptr, err));
    TRY(dalloc(&P->rptr, nloc + 1, s));
    TRY(scan_exclusive_i32(tmp32, P->rptr, nloc, s));
    TRYC(cudaMemcpyAsync(&P->nnz, P->rptr + nloc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRYC(cudaStreamSynchronize(s));
    dfree(tmp32, s);
    TRY(dalloc(&P->col, P->nnz, s));
    TRY(dalloc(&P->val, P->nnz, s));
    TRY(dalloc(&P->dpos, nloc, s));
    TRYC(cudaMemsetAsync(P->dpos, 0xff, nloc * sizeof(int32_t), s));
    KL(k_local<<<G, LOC_WARPS * 32, 0, s>>>(A, P->rptr, nullptr, P->col, P->val, P->dpos, err));
    TRYC(cudaGetLastError());
    if (P->coarse) TRY(coarse_build(P, mptr, mcol, mval, s));
    dfree(mptr, s);
    dfree(mcol, s);
    dfree(mval, s);
  }
  int herr = 0;
  TRYC(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  if (herr) return cleanup(fail((cpm_status)herr, "subdomain structure exceeds the supported limits"));
  // ---- level schedules and ILU(0)
  TRY(build_schedule(P, P->rptr, P->col, P->dpos, 1, &P->lvsub_f, &P->lvptr_f, &P->lvrow_f, &P->max_levels, s));
  TRY(build_schedule(P, P->rptr, P->col, P->dpos, 0, &P->lvsub_b, &P->lvptr_b, &P->lvrow_b, &P->max_levels, s));
  {
    const int sm = ILU_WARPS * MAXROW * (int)(sizeof(double) + sizeof(int32_t));
    TRYC(cudaFuncSetAttribute(k_ilu0, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    double* rinv = nullptr;
    TRY(dalloc(&rinv, std::max<int64_t>(P->nloc, 1), s));
    KL(k_ilu0<<<np, ILU_WARPS * 32, sm, s>>>(P->sptr, P->lvsub_f, P->lvptr_f, P->lvrow_f, P->rptr, P->col, P->dpos,
                                            P->val, rinv, err));
    dfree(rinv, s);
  }
  TRYC(cudaGetLastError());
  TRYC(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRYC(cudaStreamSynchronize(s));
  if (herr) return cleanup(fail(CPM_ERR_BREAKDOWN, "zero pivot in the ILU(0) factorisation"));
  // level-packed factors for the applies in the stored precision; the FP64
  // stream is packed on the first FP64 apply (mixed-precision solves never
  // need it, and it is the largest copy of the factors)
  TRY(dalloc(&P->err, 1, s));
  TRYC(cudaMemsetAsync(P->err, 0, sizeof(int), s));
  {
    const cpm_dtype vt = (cpm_dtype)P->store;
    PackedFactors tmp;
    TRY(pack_factors(P, 0, &vt, &tmp, 1, s));
    P->packed[vt == CPM_F64 ? 0 : 1] = tmp;
  }
  TRYC(cudaGetLastError());
#undef TRY
#undef TRYC
  return cleanup(CPM_OK);
}

void oras_destroy(oras_pc* P, cudaStream_t s) {
  if (!P) return;
  dfree(P->part, s);
  dfree(P->sptr, s);
  dfree(P->snode, s);
  dfree(P->owned, s);
  dfree(P->rptr, s);
  dfree(P->col, s);
  dfree(P->dpos, s);
  dfree(P->val, s);
  dfree(P->lvsub_f, s);
  dfree(P->lvptr_f, s);
  dfree(P->lvrow_f, s);
  dfree(P->lvsub_b, s);
  dfree(P->lvptr_b, s);
  dfree(P->lvrow_b, s);
  dfree(P->tptr, s);
  dfree(P->tcol, s);
  dfree(P->tval, s);
  dfree(P->tdpos, s);
  dfree(P->lvsub_tf, s);
  dfree(P->lvptr_tf, s);
  dfree(P->lvrow_tf, s);
  dfree(P->lvsub_tb, s);
  dfree(P->lvptr_tb, s);
  dfree(P->lvrow_tb, s);
  dfree(P->mcnt, s);
  dfree(P->memb, s);
  dfree(P->mloc, s);
  dfree(P->lsub, s);
  for (auto& pf : P->packed) packed_free(pf, s);
  coarse_free(P, s);
  dfree(P->err, s);
  delete P;
}

}  // namespace cpm
