// apply.cu -- matrix-free CPM operator (Section 2.1, eq. lapBel):
//
//   y_i = (c + 6/h^2) x_i - (1/h^2) * sum_{n in N6(i)} (E x)_n
//
// Pass 1 (k_erow_apply) evaluates (E x)_r once for every row r of Sigma_A u
// Sigma_G: a (p+1)^3 tensor-product interpolation, contracted axis by axis
// (z, then y, then x).  The cube's nodes along k are consecutive in the
// canonical order, so each (u, v) pencil costs one bitmap rank lookup.
// Pass 2 (k_stencil) forms the 7-point stencil from those values; the +-k
// neighbours of a row are the adjacent rows.
//
// FP32 uses a difference form: the weights of an E row sum to one, so
//   (E x)_n - x_i = sum_m W_nm (x_m - x_ref(n)) + (x_ref(n) - x_i)
// with x_ref(n) a node of row n's own cube.  Rounding then scales with the
// local differences of x instead of |x| * 6/h^2, which keeps the FP32
// operator accurate for smooth vectors on fine grids (at h = 0.004 the direct
// form loses about 4e-3 of relative accuracy to cancellation).
//
// The transposed apply uses y = (c + 6/h^2) x - (1/h^2) E^T (L_off^T x):
// v_r = sum of x over the active neighbours of row r, then E^T v gathered
// through a transpose map (for each active m, its (row, position) pairs in
// ascending row order) -- no atomics, so the sum order is fixed.
#include "kernels.cuh"

namespace cpm {

namespace {

struct ApplyGeom {
  Grid g;
  const BitWord* amap;
  const BitWord* rmap;
  const int32_t* ijkA;
  const int32_t* arow;
  const int32_t* rbase;
  const double* w1d;
  const float* s32;
  int64_t nA, nR;
  double coef;  // 1/h^2
};

constexpr int MAXRHS = 16;
struct Shifts {
  double c[MAXRHS];
};

// Lagrange weights of nodes 0..P at s (product form; used for the FP32 apply)
template <int P>
__device__ __forceinline__ void lagrange_f32(float s, float* l) {
#pragma unroll
  for (int j = 0; j <= P; ++j) {
    float num = 1.0f, den = 1.0f;
#pragma unroll
    for (int k = 0; k <= P; ++k)
      if (k != j) {
        num *= (s - (float)k);
        den *= (float)(j - k);
      }
    l[j] = num / den;
  }
}

template <typename T, int P>
__device__ __forceinline__ void row_weights(const ApplyGeom& G, int64_t r, T (&l)[3][P + 1]);

template <>
__device__ __forceinline__ void row_weights<double, 3>(const ApplyGeom& G, int64_t r, double (&l)[3][4]) {
  const double* w = G.w1d + r * 12;
#pragma unroll
  for (int q = 0; q < 12; ++q) l[q / 4][q % 4] = w[q];
}
template <>
__device__ __forceinline__ void row_weights<double, 2>(const ApplyGeom& G, int64_t r, double (&l)[3][3]) {
  const double* w = G.w1d + r * 9;
#pragma unroll
  for (int q = 0; q < 9; ++q) l[q / 3][q % 3] = w[q];
}
template <>
__device__ __forceinline__ void row_weights<float, 3>(const ApplyGeom& G, int64_t r, float (&l)[3][4]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) lagrange_f32<3>(G.s32[3 * r + d], l[d]);
}
template <>
__device__ __forceinline__ void row_weights<float, 2>(const ApplyGeom& G, int64_t r, float (&l)[3][3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) lagrange_f32<2>(G.s32[3 * r + d], l[d]);
}

// Pass 1: w_r = (E x)_r for all rows (FP64), or the difference-form pair
// (sum_m W_rm (x_m - x_ref), x_ref) (FP32).
template <typename T, int P>
__global__ void __launch_bounds__(256) k_erow_apply(ApplyGeom G, const T* __restrict__ x, T* __restrict__ w) {
  constexpr bool DIFF = sizeof(T) == 4;
  const int rhs = blockIdx.y;
  x += (int64_t)rhs * G.nA;
  w += (int64_t)rhs * G.nR * (DIFF ? 2 : 1);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < G.nR; r += (int64_t)gridDim.x * blockDim.x) {
    T l[3][P + 1];
    row_weights<T, P>(G, r, l);
    int b0 = G.rbase[3 * r], b1 = G.rbase[3 * r + 1], b2 = G.rbase[3 * r + 2];
    T xref = 0;
    if (DIFF) xref = __ldg(x + bm_rank_known(G.amap, G.g, b0 + 1, b1 + 1, b2) + 1);
    T acc = 0;
#pragma unroll
    for (int u = 0; u <= P; ++u) {
      T au = 0;
#pragma unroll
      for (int v = 0; v <= P; ++v) {
        int32_t q = bm_rank_known(G.amap, G.g, b0 + u, b1 + v, b2);
        const T* xp = x + q;
        T av = 0;
#pragma unroll
        for (int t = 0; t <= P; ++t) av += l[2][t] * (__ldg(xp + t) - xref);
        au += l[1][v] * av;
      }
      acc += l[0][u] * au;
    }
    if (DIFF) {
      w[2 * r] = acc;
      w[2 * r + 1] = xref;
    } else {
      w[r] = acc;
    }
  }
}

// Pass 1 in FP32, grouped by cube: the rows that share an interpolation
// cube (about five per cube on the benchmark surfaces: the nodes along one
// surface normal) are consecutive in the cube-base order, and one thread
// takes a work item of up to EGROUP_MAX of them.  It gathers the (p+1)^3 cube
// values once into registers (minus the reference node's value, the
// difference form above), then evaluates each of its rows from registers with
// that row's weights.  The arithmetic per row is the one of k_erow_apply, in
// the same order; only the loads are shared.
constexpr int EGROUP_MAX = 16;
constexpr int EGROUP_WIN = 256;  // items are ordered by row count within windows of this many

// Each row of an item is one aligned 16-byte record {s_x, s_y, s_z, row}
// (offsets in the cube, row index as bits); the next row's record is loaded
// while the current row is evaluated, so the DRAM latency of the record
// stream overlaps the arithmetic instead of stalling every row.
template <int P>
__global__ void __launch_bounds__(EGROUP_WIN)
    k_erow_grp(ApplyGeom G, int64_t nitem, const int2* __restrict__ items, const float4* __restrict__ grec,
               const float* __restrict__ x, float* __restrict__ w) {
  const int rhs = blockIdx.y;
  x += (int64_t)rhs * G.nA;
  w += (int64_t)rhs * G.nR * 2;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nitem;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int2 I = items[it];
    const int start = I.x >> 4, rows = (I.x & 15) + 1;
    const int b0 = G.ijkA[3 * I.y], b1 = G.ijkA[3 * I.y + 1], b2 = G.ijkA[3 * I.y + 2];
    float X[P + 1][P + 1][P + 1];
#pragma unroll
    for (int u = 0; u <= P; ++u)
#pragma unroll
      for (int v = 0; v <= P; ++v) {
        const float* xp = x + bm_rank_known(G.amap, G.g, b0 + u, b1 + v, b2);
#pragma unroll
        for (int t = 0; t <= P; ++t) X[u][v][t] = __ldg(xp + t);
      }
    const float xref = X[1][1][1];
#pragma unroll
    for (int u = 0; u <= P; ++u)
#pragma unroll
      for (int v = 0; v <= P; ++v)
#pragma unroll
        for (int t = 0; t <= P; ++t) X[u][v][t] -= xref;
    float4 nxt = __ldg(grec + start);
    for (int k = 0; k < rows; ++k) {
      const float4 cur = nxt;
      if (k + 1 < rows) nxt = __ldg(grec + start + k + 1);
      const int32_t r = __float_as_int(cur.w);
      float l[3][P + 1];
      lagrange_f32<P>(cur.x, l[0]);
      lagrange_f32<P>(cur.y, l[1]);
      lagrange_f32<P>(cur.z, l[2]);
      float acc = 0;
#pragma unroll
      for (int u = 0; u <= P; ++u) {
        float au = 0;
#pragma unroll
        for (int v = 0; v <= P; ++v) {
          float av = 0;
#pragma unroll
          for (int t = 0; t <= P; ++t) av += l[2][t] * X[u][v][t];
          au += l[1][v] * av;
        }
        acc += l[0][u] * au;
      }
      w[2 * r] = acc;
      w[2 * r + 1] = xref;
    }
  }
}

// ---- grouping of the E rows by cube (set-up, at band build)
// key of row r: canonical rank of its cube base (a node of Sigma_A: the
// cube lies inside Sigma_A); count rows per key
__global__ void k_gkey(ApplyGeom G, int32_t* key, int32_t* cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < G.nR; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = bm_rank_known(G.amap, G.g, G.rbase[3 * r], G.rbase[3 * r + 1], G.rbase[3 * r + 2]);
    key[r] = q;
    atomicAdd(&cnt[q], 1);
  }
}
__global__ void k_gfill(int64_t nR, const int32_t* __restrict__ key, const int64_t* __restrict__ kptr,
                        int32_t* cursor, int32_t* grow) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nR; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t q = key[r];
    grow[kptr[q] + atomicAdd(&cursor[q], 1)] = (int32_t)r;
  }
}
// per cube: its rows ascending (the fill order above is not deterministic),
// and its number of work items
__global__ void k_gsort(int64_t nA, const int64_t* __restrict__ kptr, int32_t* grow, int32_t* icnt) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = kptr[q], n = kptr[q + 1] - a;
    for (int64_t i = a + 1; i < a + n; ++i) {
      const int32_t v = grow[i];
      int64_t j = i - 1;
      while (j >= a && grow[j] > v) {
        grow[j + 1] = grow[j];
        --j;
      }
      grow[j + 1] = v;
    }
    icnt[q] = (int32_t)((n + EGROUP_MAX - 1) / EGROUP_MAX);
  }
}
__global__ void k_gitems(int64_t nA, const int64_t* __restrict__ kptr, const int64_t* __restrict__ iptr, int2* items) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = kptr[q], n = kptr[q + 1] - a;
    int64_t o = iptr[q];
    for (int64_t c = 0; c < n; c += EGROUP_MAX, ++o) {
      const int64_t rows = n - c < EGROUP_MAX ? n - c : EGROUP_MAX;
      items[o] = make_int2((int)(((a + c) << 4) | (rows - 1)), (int)q);
    }
  }
}
// within each window of EGROUP_WIN consecutive items, order the items by
// row count (stable), so that the threads of a warp loop over similar counts
// while the window keeps its spatial locality
__global__ void __launch_bounds__(EGROUP_WIN) k_gwin(int64_t nitem, const int2* __restrict__ in, int2* out) {
  __shared__ int2 sh[EGROUP_WIN];
  const int64_t w0 = (int64_t)blockIdx.x * EGROUP_WIN;
  const int n = (int)(nitem - w0 < EGROUP_WIN ? nitem - w0 : EGROUP_WIN);
  const int t = threadIdx.x;
  if (t < n) sh[t] = in[w0 + t];
  __syncthreads();
  if (t < n) {
    const int mine = sh[t].x & 15;
    int pos = 0;
    for (int k = 0; k < n; ++k) {
      const int o = sh[k].x & 15;
      pos += (o < mine || (o == mine && k < t)) ? 1 : 0;
    }
    out[w0 + pos] = sh[t];
  }
}
__global__ void k_grec(int64_t nR, const int32_t* __restrict__ grow, const float* __restrict__ s32, float4* rec) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nR; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = grow[p];
    rec[p] = make_float4(s32[3 * (int64_t)r], s32[3 * (int64_t)r + 1], s32[3 * (int64_t)r + 2], __int_as_float(r));
  }
}

// Pass 2: y_i = (c + 6/h^2) x_i - (1/h^2) sum_n w_n.
template <typename T>
__global__ void __launch_bounds__(256) k_stencil(ApplyGeom G, Shifts S, const T* __restrict__ x,
                                                 const T* __restrict__ w, T* __restrict__ y) {
  const int rhs = blockIdx.y;
  x += (int64_t)rhs * G.nA;
  y += (int64_t)rhs * G.nA;
  constexpr bool DIFF = sizeof(T) == 4;
  w += (int64_t)rhs * G.nR * (DIFF ? 2 : 1);
  const T diag = (T)(S.c[rhs] + 6.0 * G.coef), coef = (T)G.coef, cshift = (T)S.c[rhs];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < G.nA; q += (int64_t)gridDim.x * blockDim.x) {
    int i = G.ijkA[3 * q], j = G.ijkA[3 * q + 1], k = G.ijkA[3 * q + 2];
    int32_t r = G.arow[q];
    int32_t rjm = bm_rank_known(G.rmap, G.g, i, j - 1, k), rjp = bm_rank_known(G.rmap, G.g, i, j + 1, k);
    int32_t rim = bm_rank_known(G.rmap, G.g, i - 1, j, k), rip = bm_rank_known(G.rmap, G.g, i + 1, j, k);
    const T xi = x[q];
    if (DIFF) {
      auto d = [&](int32_t n) { return w[2 * n] + (w[2 * n + 1] - xi); };
      T s = ((d(rim) + d(rip)) + (d(rjm) + d(rjp))) + (d(r - 1) + d(r + 1));
      y[q] = cshift * xi - coef * s;
    } else {
      T s = ((w[rim] + w[rip]) + (w[rjm] + w[rjp])) + (w[r - 1] + w[r + 1]);
      y[q] = diag * xi - coef * s;
    }
  }
}

// ---- transposed apply
template <typename T>
__global__ void k_loff_T(ApplyGeom G, const T* __restrict__ x, const int32_t* __restrict__ rijk, T* __restrict__ v) {
  const int rhs = blockIdx.y;
  x += (int64_t)rhs * G.nA;
  v += (int64_t)rhs * G.nR;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < G.nR; r += (int64_t)gridDim.x * blockDim.x) {
    int i = rijk[3 * r], j = rijk[3 * r + 1], k = rijk[3 * r + 2];
    const int nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    T s = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      int32_t m = bm_rank(G.amap, G.g, i + nb[d][0], j + nb[d][1], k + nb[d][2]);
      if (m >= 0) s += x[m];
    }
    v[r] = s;
  }
}

// LPN lanes per active node: the node's transpose-map entries (ascending
// row) are split over its lanes and shuffle-reduced in a fixed tree, so the
// sum order is fixed and the result deterministic.  FP64 uses few lanes per
// node (the reduction costs FP64 adds); FP32 uses more lanes for coalescing.
// Each lane issues the loads of U entries before it uses any of them (the
// row index, then the gather of v through it), so U chains are in flight;
// entries past the node's end read row 0 with weight 0, which leaves the sum
// unchanged.
constexpr int ET_UNROLL = 4;
template <typename T, int LPN, int U>
__global__ void __launch_bounds__(256) k_ET(ApplyGeom G, Shifts S, const int64_t* __restrict__ tptr,
                                            const uint32_t* __restrict__ tent, const T* __restrict__ tw,
                                            const T* __restrict__ x, const T* __restrict__ v, T* __restrict__ y) {
  constexpr int NPW = 32 / LPN;  // nodes per warp
  const int rhs = blockIdx.y, lane = threadIdx.x & 31, sub = lane & (LPN - 1);
  x += (int64_t)rhs * G.nA;
  y += (int64_t)rhs * G.nA;
  v += (int64_t)rhs * G.nR;
  const T diag = (T)(S.c[rhs] + 6.0 * G.coef), coef = (T)G.coef;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // warp-uniform loop over groups of NPW nodes
  for (int64_t wb = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * NPW; wb < G.nA; wb += nwarps * NPW) {
    const int64_t m = wb + lane / LPN;
    T acc = 0;
    if (m < G.nA) {
      const int64_t e1 = tptr[m + 1];
      for (int64_t e = tptr[m] + sub; e < e1; e += LPN * U) {
        uint32_t k[U];
        T w[U], vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t ee = e + u * LPN;
          k[u] = ee < e1 ? __ldg(tent + ee) : 0u;
          w[u] = ee < e1 ? __ldg(tw + ee) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) vv[u] = v[k[u] >> 6];
#pragma unroll
        for (int u = 0; u < U; ++u) acc += w[u] * vv[u];
      }
    }
#pragma unroll
    for (int o = LPN / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (sub == 0 && m < G.nA) y[m] = diag * x[m] - coef * acc;
  }
}

// tensor weight of every transpose-map entry, in the order (w_u w_v) w_w
__global__ void k_tweights(int64_t n, int P, const uint32_t* __restrict__ tent, const double* __restrict__ w1d,
                           double* tw64, float* tw32) {
  const int P1 = P + 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t pk = tent[e];
    const int64_t r = pk >> 6;
    const int pos = pk & 63, u = pos / (P1 * P1), vv = (pos / P1) % P1, t = pos % P1;
    const double* w = w1d + r * 3 * P1;
    const double W = __dmul_rn(__dmul_rn(w[u], w[P1 + vv]), w[2 * P1 + t]);
    tw64[e] = W;
    tw32[e] = (float)W;
  }
}

// transpose map: counts, then fill, then sort each segment
__global__ void k_tcount(ApplyGeom G, int P, int32_t* cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < G.nR; r += (int64_t)gridDim.x * blockDim.x) {
    int b0 = G.rbase[3 * r], b1 = G.rbase[3 * r + 1], b2 = G.rbase[3 * r + 2];
    for (int u = 0; u <= P; ++u)
      for (int v = 0; v <= P; ++v) {
        int32_t q = bm_rank_known(G.amap, G.g, b0 + u, b1 + v, b2);
        for (int t = 0; t <= P; ++t) atomicAdd(&cnt[q + t], 1);
      }
  }
}

__global__ void k_tfill(ApplyGeom G, int P, const int64_t* __restrict__ tptr, int32_t* cursor, uint32_t* tent) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < G.nR; r += (int64_t)gridDim.x * blockDim.x) {
    int b0 = G.rbase[3 * r], b1 = G.rbase[3 * r + 1], b2 = G.rbase[3 * r + 2];
    int pos = 0;
    for (int u = 0; u <= P; ++u)
      for (int v = 0; v <= P; ++v) {
        int32_t q = bm_rank_known(G.amap, G.g, b0 + u, b1 + v, b2);
        for (int t = 0; t <= P; ++t, ++pos) {
          int32_t slot = atomicAdd(&cursor[q + t], 1);
          tent[tptr[q + t] + slot] = ((uint32_t)r << 6) | (uint32_t)pos;
        }
      }
  }
}

// Sort each node's (row, cube position) keys ascending.  One warp per node:
// the keys are distinct, so a key's place is the number of smaller keys in
// its segment (counted from a shared-memory copy); segments longer than the
// staging buffer fall back to an insertion sort by one lane.
constexpr int TSORT_WARPS = 4, TSORT_CAP = 512;
__global__ void __launch_bounds__(TSORT_WARPS * 32)
    k_tsort(int64_t nA, const int64_t* __restrict__ tptr, uint32_t* tent) {
  __shared__ uint32_t sk[TSORT_WARPS][TSORT_CAP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* buf = sk[wid];
  for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; m < nA;
       m += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t a = tptr[m];
    const int n = (int)(tptr[m + 1] - a);
    if (n <= TSORT_CAP) {
      for (int i = lane; i < n; i += 32) buf[i] = tent[a + i];
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        const uint32_t key = buf[i];
        int r = 0;
        for (int k = 0; k < n; ++k) r += buf[k] < key ? 1 : 0;
        tent[a + r] = key;
      }
      __syncwarp();
    } else if (lane == 0) {
      for (int64_t i = a + 1; i < a + n; ++i) {
        const uint32_t key = tent[i];
        int64_t j = i - 1;
        while (j >= a && tent[j] > key) {
          tent[j + 1] = tent[j];
          --j;
        }
        tent[j + 1] = key;
      }
    }
    __syncwarp();
  }
}

ApplyGeom geom_of(const cpm_band* B) {
  ApplyGeom G;
  G.g = B->grid;
  G.amap = B->amap;
  G.rmap = B->rmap;
  G.ijkA = B->ijkA;
  G.arow = B->arow;
  G.rbase = B->rbase;
  G.w1d = B->w1d;
  G.s32 = B->s32;
  G.nA = B->nA;
  G.nR = B->nR;
  G.coef = 1.0 / (B->h * B->h);
  return G;
}

// Pass 1 for nr right-hand sides: FP64 row by row (weights precomputed,
// FP64-ALU bound); FP32 grouped by cube.
template <typename T>
cpm_status erow_pass(const cpm_band* B, const ApplyGeom& G, const T* x, T* w, int nr, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    dim3 g1(grid_for(B->nitem, EGROUP_WIN), nr);
    const int2* it = reinterpret_cast<const int2*>(B->gitem);
    const float4* rec = reinterpret_cast<const float4*>(B->grec);
    if (B->p == 3) KL(k_erow_grp<3><<<g1, EGROUP_WIN, 0, s>>>(G, B->nitem, it, rec, x, w));
    else KL(k_erow_grp<2><<<g1, EGROUP_WIN, 0, s>>>(G, B->nitem, it, rec, x, w));
  } else {
    dim3 g1(grid_for(B->nR, 256), nr);
    if (B->p == 3) KL(k_erow_apply<T, 3><<<g1, 256, 0, s>>>(G, x, w));
    else KL(k_erow_apply<T, 2><<<g1, 256, 0, s>>>(G, x, w));
  }
  return CPM_OK;
}

template <typename T>
cpm_status apply_typed(const cpm_band* B, const double* c, const T* x, T* y, int nrhs, int transpose, cudaStream_t s) {
  ApplyGeom G = geom_of(B);
  if (transpose && !B->tptr) CPM_TRY(build_transpose_map(const_cast<cpm_band*>(B), s));
  for (int r0 = 0; r0 < nrhs; r0 += MAXRHS) {
    int nr = nrhs - r0 < MAXRHS ? nrhs - r0 : MAXRHS;
    const T* xr = x + (int64_t)r0 * B->nA;
    T* yr = y + (int64_t)r0 * B->nA;
    if constexpr (sizeof(T) == 4) {
      if (!transpose && B->ntile > 0) {  // staged through shared memory by bricks (tile.cu)
        CPM_TRY(tile_apply_f32(B, c + r0, xr, yr, nr, s));
        continue;
      }
    }
    Shifts S{};
    for (int q = 0; q < nr; ++q) S.c[q] = c[r0 + q];
    T* w = nullptr;
    CPM_TRY(dalloc(&w, (size_t)nr * B->nR * (sizeof(T) == 4 ? 2 : 1), s));
    if (!transpose) {
      CPM_TRY(erow_pass(B, G, xr, w, nr, s));
      dim3 g2(grid_for(B->nA, 256), nr);
      KL(k_stencil<T><<<g2, 256, 0, s>>>(G, S, xr, w, yr));
    } else {
      dim3 g1(grid_for(B->nR, 256), nr);
      KL(k_loff_T<T><<<g1, 256, 0, s>>>(G, xr, B->rijk, w));
      const T* tw = sizeof(T) == 8 ? (const T*)B->tw64 : (const T*)B->tw32;
      constexpr int LPN = sizeof(T) == 8 ? 4 : 16;
      dim3 g3(grid_for(B->nA * LPN, 256), nr);
      KL(k_ET<T, LPN, ET_UNROLL><<<g3, 256, 0, s>>>(G, S, B->tptr, B->tent, tw, xr, w, yr));
    }
    cudaError_t e = cudaGetLastError();
    dfree(w, s);
    if (e != cudaSuccess) return cuda_fail(e, "apply kernels", __FILE__, __LINE__);
  }
  return CPM_OK;
}

template <typename T>
cpm_status apply_fwd_scratch(const cpm_band* B, const double* c, const T* x, T* y, int nrhs, T* w, cudaStream_t s) {
  ApplyGeom G = geom_of(B);
  for (int r0 = 0; r0 < nrhs; r0 += MAXRHS) {
    int nr = nrhs - r0 < MAXRHS ? nrhs - r0 : MAXRHS;
    Shifts S{};
    for (int q = 0; q < nr; ++q) S.c[q] = c[r0 + q];
    const T* xr = x + (int64_t)r0 * B->nA;
    T* yr = y + (int64_t)r0 * B->nA;
    CPM_TRY(erow_pass(B, G, xr, w, nr, s));
    dim3 g2(grid_for(B->nA, 256), nr);
    KL(k_stencil<T><<<g2, 256, 0, s>>>(G, S, xr, w, yr));
    CPM_CUDA(cudaGetLastError());
  }
  return CPM_OK;
}

}  // namespace

// Forward operator with scratch supplied by the caller: at least
// min(nrhs, 16) * nR * 8 bytes, 8-byte aligned.  Allocates nothing.
cpm_status apply_op_scratch(const cpm_band* B, const double* c, const void* x, void* y, cpm_dtype dt, int nrhs,
                            void* scratch, cudaStream_t s) {
  if (dt == CPM_F64)
    return apply_fwd_scratch<double>(B, c, (const double*)x, (double*)y, nrhs, (double*)scratch, s);
  if (dt == CPM_F32) return apply_fwd_scratch<float>(B, c, (const float*)x, (float*)y, nrhs, (float*)scratch, s);
  return fail(CPM_ERR_ARG, "cpm_apply_noalloc supports CPM_F64 and CPM_F32 vectors");
}

cpm_status build_erow_groups(cpm_band* B, cudaStream_t s) {
  ApplyGeom G = geom_of(B);
  const int64_t nA = B->nA, nR = B->nR;
  int32_t *key = nullptr, *cnt = nullptr, *icnt = nullptr;
  int64_t *kptr = nullptr, *iptr = nullptr;
  int2* tmp = nullptr;
  auto done = [&](cpm_status st) {
    dfree(key, s);
    dfree(cnt, s);
    dfree(icnt, s);
    dfree(kptr, s);
    dfree(iptr, s);
    dfree(tmp, s);
    return st;
  };
  cpm_status st;
  if ((st = dalloc(&key, nR, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&cnt, nA, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&icnt, nA, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&kptr, nA + 1, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&iptr, nA + 1, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&B->grow, nR, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&B->grec, 4 * nR, s)) != CPM_OK) return done(st);
  CPM_CUDA(cudaMemsetAsync(cnt, 0, nA * sizeof(int32_t), s));
  KL(k_gkey<<<grid_for(nR, 256), 256, 0, s>>>(G, key, cnt));
  if ((st = scan_exclusive_i32(cnt, kptr, nA, s)) != CPM_OK) return done(st);
  CPM_CUDA(cudaMemsetAsync(cnt, 0, nA * sizeof(int32_t), s));
  KL(k_gfill<<<grid_for(nR, 256), 256, 0, s>>>(nR, key, kptr, cnt, B->grow));
  KL(k_gsort<<<grid_for(nA, 256), 256, 0, s>>>(nA, kptr, B->grow, icnt));
  if ((st = scan_exclusive_i32(icnt, iptr, nA, s)) != CPM_OK) return done(st);
  CPM_CUDA(cudaMemcpyAsync(&B->nitem, iptr + nA, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  if ((st = dalloc(&tmp, B->nitem, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&B->gitem, 2 * B->nitem, s)) != CPM_OK) return done(st);
  KL(k_gitems<<<grid_for(nA, 256), 256, 0, s>>>(nA, kptr, iptr, tmp));
  const int64_t nwin = (B->nitem + EGROUP_WIN - 1) / EGROUP_WIN;
  KL(k_gwin<<<(unsigned)nwin, EGROUP_WIN, 0, s>>>(B->nitem, tmp, reinterpret_cast<int2*>(B->gitem)));
  KL(k_grec<<<grid_for(nR, 256), 256, 0, s>>>(nR, B->grow, B->s32, reinterpret_cast<float4*>(B->grec)));
  dfree(B->grow, s);  // the records carry the row indices
  CPM_CUDA(cudaGetLastError());
  return done(CPM_OK);
}

cpm_status build_transpose_map(cpm_band* B, cudaStream_t s) {
  ApplyGeom G = geom_of(B);
  int P = B->p;
  int64_t nA = B->nA;
  int32_t* cnt = nullptr;
  CPM_TRY(dalloc(&cnt, nA, s));
  CPM_TRY(dalloc(&B->tptr, nA + 1, s));
  CPM_CUDA(cudaMemsetAsync(cnt, 0, nA * sizeof(int32_t), s));
  KL(k_tcount<<<grid_for(B->nR, 256), 256, 0, s>>>(G, P, cnt));
  CPM_TRY(scan_exclusive_i32(cnt, B->tptr, nA, s));
  int64_t total = 0;
  CPM_CUDA(cudaMemcpyAsync(&total, B->tptr + nA, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CPM_CUDA(cudaStreamSynchronize(s));
  CPM_TRY(dalloc(&B->tent, total, s));
  CPM_CUDA(cudaMemsetAsync(cnt, 0, nA * sizeof(int32_t), s));
  KL(k_tfill<<<grid_for(B->nR, 256), 256, 0, s>>>(G, P, B->tptr, cnt, B->tent));
  KL(k_tsort<<<grid_for(nA * 32, TSORT_WARPS * 32), TSORT_WARPS * 32, 0, s>>>(nA, B->tptr, B->tent));
  CPM_TRY(dalloc(&B->tw64, total, s));
  CPM_TRY(dalloc(&B->tw32, total, s));
  KL(k_tweights<<<grid_for(total, 256), 256, 0, s>>>(total, P, B->tent, B->w1d, B->tw64, B->tw32));
  CPM_CUDA(cudaGetLastError());
  dfree(cnt, s);
  return CPM_OK;
}

cpm_status apply_op(const cpm_band* B, const double* c, const void* x, void* y, cpm_dtype dt, int nrhs, int transpose,
                    cudaStream_t s) {
  if (dt == CPM_F64) return apply_typed<double>(B, c, (const double*)x, (double*)y, nrhs, transpose, s);
  if (dt == CPM_F32) return apply_typed<float>(B, c, (const float*)x, (float*)y, nrhs, transpose, s);
  return fail(CPM_ERR_ARG, "cpm_apply supports CPM_F64 and CPM_F32 vectors");
}

}  // namespace cpm
