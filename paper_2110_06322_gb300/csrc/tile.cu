// tile.cu -- the FP32 operator apply staged through shared memory by
// lattice bricks (Section 2.1, eq. lapBel):
//
//   y_i = c x_i - (1/h^2) sum_{n in N6(i)} ((E x)_n - x_i)
//
// The lattice is cut into bricks of TB^3 cells.  A brick's output nodes are
// its active nodes; the E rows it needs are their six neighbours (rows of
// Sigma_A u Sigma_G inside the brick grown by one cell), and the x values
// those rows interpolate lie in the bounding box of their cubes (at most 31
// cells per axis, since a row lies within a few h of its closest point).
// One CTA per brick
//   1. stages x over that box into shared memory: one thread per box column,
//      whose active cells in the box's k-window are a run of consecutive
//      canonical ranks (one bitmap word or two);
//   2. evaluates the brick's E rows from shared memory -- rows that share an
//      interpolation cube form one work item, whose cube is read once into
//      registers -- into a shared grid of (value, reference) pairs over the
//      grown brick (the difference form of the two-pass FP32 apply: the
//      weights of a row sum to one, so (E x)_n - x_i = sum_m W_nm (x_m -
//      x_ref) + (x_ref - x_i), with x_ref the cube's node (1,1,1));
//   3. forms the stencil of each active node from that grid and writes y.
// No intermediate goes through HBM and no gather needs a bitmap lookup.  The
// contraction order of a row and the stencil's sum order are those of the
// two-pass FP32 apply.  Rows that neighbour two bricks are evaluated by both (1.2-1.3
// records per E row at TB = 16 on the benchmark surfaces).
//
// Set-up (band build): bricks holding active nodes are listed in canonical
// brick order; each marks the grid slots of the rows its nodes need; one CTA
// per brick then ranks those rows, takes the bounding box of their cubes,
// sorts the rows by cube (bitonic, in shared memory), and writes one 16-byte
// record per row {s_x, s_y, s_z, slot} and one 32-bit word per work item
// {first record, rows - 1, cube base in the box}.
#include "kernels.cuh"

namespace cpm {

namespace {

constexpr int TB = 16;                       // brick edge (cells)
constexpr int TS = TB + 2;                   // slot grid edge: the brick grown by one cell
constexpr int TSLOTS = TS * TS * TS;         // 5832
constexpr int TMW = (TSLOTS + 31) / 32;      // 32-bit words of a brick's slot mask
constexpr int TBOX = 31;                     // largest box edge the item packing allows
constexpr int TSORT = 8192;                  // sort capacity (power of two >= TSLOTS)
constexpr int TITEM_MAX = 16;                // rows per work item
constexpr int TAPPLY_THREADS = TB * TB;      // one thread per brick column in the stencil
constexpr int TBUILD_THREADS = 512;

// header of brick t: {a0, b0, c0, nitem, oa, ob, oc, DI | DJ << 8 | DK << 16},
// grid-relative brick and box origins
struct TileHead {
  int a0, b0, c0, nitem, oa, ob, oc, dims;
};

__device__ __forceinline__ int64_t tile_word(const Grid& g, int a, int b, int c) {
  return ((int64_t)a * g.gn[1] + b) * g.nkw + (c >> 6);
}

// ---------------------------------------------------------------- set-up
__global__ void k_tb_flag(int64_t nA, const int32_t* __restrict__ ijkA, Grid g, int nbj, int nbk, int32_t* flag) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    const int a = ijkA[3 * q] - g.glo[0], b = ijkA[3 * q + 1] - g.glo[1], c = ijkA[3 * q + 2] - g.glo[2];
    flag[((int64_t)(a / TB) * nbj + b / TB) * nbk + c / TB] = 1;
  }
}
// per brick: the extent of its active nodes (grid-relative min and max per
// axis), so that the box holds every node whose stencil the brick forms
__global__ void k_tb_extent(int64_t nA, const int32_t* __restrict__ ijkA, Grid g, int nbj, int nbk,
                            const int64_t* __restrict__ tidx, int32_t* ext) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    const int a = ijkA[3 * q] - g.glo[0], b = ijkA[3 * q + 1] - g.glo[1], c = ijkA[3 * q + 2] - g.glo[2];
    int32_t* e = ext + 6 * tidx[((int64_t)(a / TB) * nbj + b / TB) * nbk + c / TB];
    atomicMin(&e[0], a);
    atomicMin(&e[1], b);
    atomicMin(&e[2], c);
    atomicMax(&e[3], a);
    atomicMax(&e[4], b);
    atomicMax(&e[5], c);
  }
}
__global__ void k_tb_ext_init(int64_t nt, int32_t* ext) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 6 * nt; q += (int64_t)gridDim.x * blockDim.x)
    ext[q] = (q % 6) < 3 ? INT_MAX : INT_MIN;
}
__global__ void k_tb_list(int64_t nb, const int32_t* __restrict__ flag, const int64_t* __restrict__ tidx,
                          int32_t* bid) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x)
    if (flag[q]) bid[tidx[q]] = (int32_t)q;
}
// every active node marks the slots of its six neighbours in its brick's mask
__global__ void k_tb_need(int64_t nA, const int32_t* __restrict__ ijkA, Grid g, int nbj, int nbk,
                          const int64_t* __restrict__ tidx, uint32_t* mask) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA; q += (int64_t)gridDim.x * blockDim.x) {
    const int a = ijkA[3 * q] - g.glo[0], b = ijkA[3 * q + 1] - g.glo[1], c = ijkA[3 * q + 2] - g.glo[2];
    const int64_t t = tidx[((int64_t)(a / TB) * nbj + b / TB) * nbk + c / TB];
    const int s0 = ((a % TB + 1) * TS + (b % TB + 1)) * TS + (c % TB + 1);
    const int nb[6] = {s0 - TS * TS, s0 + TS * TS, s0 - TS, s0 + TS, s0 - 1, s0 + 1};
    uint32_t* m = mask + t * TMW;
#pragma unroll
    for (int d = 0; d < 6; ++d) atomicOr(&m[nb[d] >> 5], 1u << (nb[d] & 31));
  }
}
__global__ void k_tb_count(int64_t nt, const uint32_t* __restrict__ mask, int32_t* cnt) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
    int c = 0;
    for (int w = 0; w < TMW; ++w) c += __popc(mask[t * TMW + w]);
    cnt[t] = c;
  }
}

// exclusive sum over the block (blockDim.x == TBUILD_THREADS) of one value per thread
__device__ int tb_block_exclusive(int v, int* red, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) red[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < TBUILD_THREADS / 32 ? red[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < TBUILD_THREADS / 32) red[lane] = s;
  }
  __syncthreads();
  const int before = (wid ? red[wid - 1] : 0) + x - v;
  *total = red[TBUILD_THREADS / 32 - 1];
  __syncthreads();
  return before;
}

struct TileBuildArgs {
  Grid g;
  const BitWord* rmap;
  const int32_t* rbase;  // [nR][3] global lattice coordinates of each row's cube base
  const float* s32;
  const int32_t* bid;
  const uint32_t* mask;
  const int32_t* ext;
  const int64_t* roff;
  int nbj, nbk, P;
  TileHead* head;
  float4* rec;
  uint32_t* item;
  int32_t* maxbox;
  int32_t* err;
};

// one CTA per brick
constexpr size_t TBUILD_SMEM = sizeof(uint32_t) * TSORT + sizeof(int32_t) * TSLOTS + sizeof(uint16_t) * TSLOTS;

__global__ void __launch_bounds__(TBUILD_THREADS) k_tb_build(TileBuildArgs A) {
  extern __shared__ __align__(16) unsigned char tb_smem[];
  uint32_t* keys = reinterpret_cast<uint32_t*>(tb_smem);                                  // [TSORT]
  int32_t* rows = reinterpret_cast<int32_t*>(tb_smem + sizeof(uint32_t) * TSORT);         // [TSLOTS]
  uint16_t* list = reinterpret_cast<uint16_t*>(tb_smem + sizeof(uint32_t) * TSORT + sizeof(int32_t) * TSLOTS);
  __shared__ int red[TBUILD_THREADS / 32];
  __shared__ int bmin[3], bmax[3];
  const int t = blockIdx.x, tid = threadIdx.x;
  const int id = A.bid[t];
  const int a0 = (id / (A.nbj * A.nbk)) * TB, b0 = ((id / A.nbk) % A.nbj) * TB, c0 = (id % A.nbk) * TB;
  const int64_t r0 = A.roff[t];
  const int n = (int)(A.roff[t + 1] - r0);
  if (tid < 3) {  // start from the extent of the brick's own active nodes
    bmin[tid] = A.ext[6 * (int64_t)t + tid];
    bmax[tid] = A.ext[6 * (int64_t)t + 3 + tid];
  }
  // the needed slots in ascending order
  const uint32_t w = tid < TMW ? A.mask[(int64_t)t * TMW + tid] : 0u;
  int total = 0;
  int o = tb_block_exclusive(__popc(w), red, &total);
  for (uint32_t m = w; m; m &= m - 1) list[o++] = (uint16_t)(tid * 32 + __ffs(m) - 1);
  __syncthreads();
  // rows and the bounding box of their cubes (grid-relative)
  for (int p = tid; p < n; p += TBUILD_THREADS) {
    const int sl = list[p];
    const int a = a0 + sl / (TS * TS) - 1, b = b0 + (sl / TS) % TS - 1, c = c0 + sl % TS - 1;
    const int32_t r = bm_rank_known(A.rmap, A.g, a + A.g.glo[0], b + A.g.glo[1], c + A.g.glo[2]);
    rows[p] = r;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int v = A.rbase[3 * (int64_t)r + d] - A.g.glo[d];
      atomicMin(&bmin[d], v);
      atomicMax(&bmax[d], v + A.P);
    }
  }
  __syncthreads();
  const int oa = bmin[0], ob = bmin[1], oc = bmin[2];
  const int DI = bmax[0] - oa + 1, DJ = bmax[1] - ob + 1, DK = bmax[2] - oc + 1;
  const bool ok = DI <= TBOX && DJ <= TBOX && DK <= TBOX;
  if (!ok) {
    if (tid == 0) atomicExch(A.err, 1);
    return;  // uniform over the block
  }
  // sort keys: box-local cube base, then position in the slot list
  int N = 1;
  while (N < n) N <<= 1;
  for (int p = tid; p < N; p += TBUILD_THREADS) {
    if (p < n) {
      const int32_t r = rows[p];
      const int ka = A.rbase[3 * (int64_t)r] - A.g.glo[0] - oa, kb = A.rbase[3 * (int64_t)r + 1] - A.g.glo[1] - ob,
                kc = A.rbase[3 * (int64_t)r + 2] - A.g.glo[2] - oc;
      keys[p] = ((uint32_t)((ka * DJ + kb) * DK + kc) << 16) | (uint32_t)p;
    } else {
      keys[p] = 0xffffffffu;
    }
  }
  __syncthreads();
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < N; i += TBUILD_THREADS) {
        const int ij = i ^ j;
        if (ij > i) {
          const uint32_t x = keys[i], y = keys[ij];
          if ((x > y) == ((i & k) == 0)) {
            keys[i] = y;
            keys[ij] = x;
          }
        }
      }
      __syncthreads();
    }
  // records in cube order
  for (int p = tid; p < n; p += TBUILD_THREADS) {
    const int q = (int)(keys[p] & 0xffffu);
    const int32_t r = rows[q];
    A.rec[r0 + p] = make_float4(A.s32[3 * (int64_t)r], A.s32[3 * (int64_t)r + 1], A.s32[3 * (int64_t)r + 2],
                                __int_as_float((int)list[q]));
  }
  // work items: runs of one cube, cut every TITEM_MAX rows; each thread takes
  // a contiguous span of positions so that items come out in order
  const int span = (n + TBUILD_THREADS - 1) / TBUILD_THREADS;
  const int p0 = tid * span, p1 = min(n, p0 + span);
  auto starts = [&](int p) {
    const uint32_t kp = keys[p] >> 16;
    int q = p;
    while (q > 0 && (keys[q - 1] >> 16) == kp) --q;
    return (p - q) % TITEM_MAX == 0;
  };
  int mine = 0;
  for (int p = p0; p < p1; ++p) mine += starts(p) ? 1 : 0;
  int nitem = 0;
  int io = tb_block_exclusive(mine, red, &nitem);
  for (int p = p0; p < p1; ++p)
    if (starts(p)) {
      const uint32_t kp = keys[p] >> 16;
      int e = p + 1;
      while (e < n && e - p < TITEM_MAX && (keys[e] >> 16) == kp) ++e;
      A.item[r0 + io++] = ((uint32_t)p << 19) | ((uint32_t)(e - p - 1) << 15) | kp;
    }
  if (tid == 0) {
    A.head[t] = TileHead{a0, b0, c0, nitem, oa, ob, oc, DI | (DJ << 8) | (DK << 16)};
    atomicMax(A.maxbox, DI * DJ * DK);
  }
}

// ---------------------------------------------------------------- apply
// Lagrange weights of nodes 0..P at s (product form).  The denominators are
// constants, so each weight is scaled by the rounded reciprocal of its
// denominator (one multiply instead of an IEEE division; at most an ulp apart).
template <int P>
__device__ __forceinline__ void tile_lagrange(float s, float* l) {
#pragma unroll
  for (int j = 0; j <= P; ++j) {
    float num = 1.0f;
    int den = 1;
#pragma unroll
    for (int k = 0; k <= P; ++k)
      if (k != j) {
        num *= (s - (float)k);
        den *= j - k;
      }
    l[j] = num * (1.0f / (float)den);
  }
}

struct TileApplyArgs {
  Grid g;
  const BitWord* amap;
  const TileHead* head;
  const int64_t* roff;
  const float4* rec;
  const uint32_t* item;
  int64_t nA;
  float coef;  // 1/h^2
  float c[16];
};

template <int P>
__global__ void __launch_bounds__(TAPPLY_THREADS, 2)
    k_tile_apply(TileApplyArgs A, const float* __restrict__ x, float* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char tile_smem[];
  float2* ws = reinterpret_cast<float2*>(tile_smem);                    // [TSLOTS] (value, reference)
  float* xb = reinterpret_cast<float*>(tile_smem + sizeof(float2) * TSLOTS);  // [DI][DJ][DK]
  const int t = blockIdx.x, rhs = blockIdx.y, tid = threadIdx.x;
  x += (int64_t)rhs * A.nA;
  y += (int64_t)rhs * A.nA;
  const TileHead H = A.head[t];
  const int DI = H.dims & 0xff, DJ = (H.dims >> 8) & 0xff, DK = H.dims >> 16;
  // 1. x over the box: one thread per column
  for (int col = tid; col < DI * DJ; col += TAPPLY_THREADS) {
    const int ca = col / DJ, cb = col - ca * DJ;
    const int a = H.oa + ca, b = H.ob + cb;
    float* dst = xb + (int64_t)col * DK - H.oc;  // indexed by grid-relative k
    const int w0 = H.oc >> 6, w1 = (H.oc + DK - 1) >> 6;
    for (int wd = w0; wd <= w1; ++wd) {
      const BitWord bw = A.amap[tile_word(A.g, a, b, wd * 64)];
      const int lo = max(H.oc - wd * 64, 0), hi = min(H.oc + DK - wd * 64, 64);
      unsigned long long m = bw.bits;
      if (lo > 0) m &= ~0ull << lo;
      if (hi < 64) m &= (1ull << hi) - 1;
      int32_t q = bw.pre + __popcll(bw.bits & (lo > 0 ? (1ull << lo) - 1 : 0ull));
      for (; m; m &= m - 1) dst[wd * 64 + __ffsll((long long)m) - 1] = __ldg(x + q++);
    }
  }
  __syncthreads();
  // 2. E rows by work item
  const int64_t r0 = A.roff[t];
  for (int it = tid; it < H.nitem; it += TAPPLY_THREADS) {
    const uint32_t I = A.item[r0 + it];
    const int start = (int)(I >> 19), rows = (int)((I >> 15) & 15) + 1, key = (int)(I & 0x7fff);
    const float* cb = xb + key;  // key = (ka * DJ + kb) * DK + kc
    float X[P + 1][P + 1][P + 1];
#pragma unroll
    for (int u = 0; u <= P; ++u)
#pragma unroll
      for (int v = 0; v <= P; ++v)
#pragma unroll
        for (int w = 0; w <= P; ++w) X[u][v][w] = cb[(u * DJ + v) * DK + w];
    const float xref = X[1][1][1];
#pragma unroll
    for (int u = 0; u <= P; ++u)
#pragma unroll
      for (int v = 0; v <= P; ++v)
#pragma unroll
        for (int w = 0; w <= P; ++w) X[u][v][w] -= xref;
    float4 nxt = __ldg(A.rec + r0 + start);
    for (int k = 0; k < rows; ++k) {
      const float4 cur = nxt;
      if (k + 1 < rows) nxt = __ldg(A.rec + r0 + start + k + 1);
      float l[3][P + 1];
      tile_lagrange<P>(cur.x, l[0]);
      tile_lagrange<P>(cur.y, l[1]);
      tile_lagrange<P>(cur.z, l[2]);
      float acc = 0;
#pragma unroll
      for (int u = 0; u <= P; ++u) {
        float au = 0;
#pragma unroll
        for (int v = 0; v <= P; ++v) {
          float av = 0;
#pragma unroll
          for (int w = 0; w <= P; ++w) av += l[2][w] * X[u][v][w];
          au += l[1][v] * av;
        }
        acc += l[0][u] * au;
      }
      ws[__float_as_int(cur.w)] = make_float2(acc, xref);
    }
  }
  __syncthreads();
  // 3. the stencil: one thread per brick column (TB consecutive k in one word)
  const int la = tid / TB, lb = tid % TB;
  const int a = H.a0 + la, b = H.b0 + lb;
  if (a < A.g.gn[0] && b < A.g.gn[1]) {
    const BitWord bw = A.amap[tile_word(A.g, a, b, H.c0)];
    const int sh = H.c0 & 63;
    unsigned long long m = (bw.bits >> sh) & ((1ull << TB) - 1);
    int32_t q = bw.pre + __popcll(bw.bits & (sh > 0 ? (1ull << sh) - 1 : 0ull));
    const float* xcol = xb + (int64_t)((a - H.oa) * DJ + (b - H.ob)) * DK - H.oc;
    const float cshift = A.c[rhs], coef = A.coef;
    for (; m; m &= m - 1, ++q) {
      const int lc = __ffsll((long long)m) - 1;
      const float xi = xcol[H.c0 + lc];
      const int s0 = ((la + 1) * TS + (lb + 1)) * TS + (lc + 1);
      auto d = [&](int sl) {
        const float2 v = ws[sl];
        return v.x + (v.y - xi);
      };
      const float s = ((d(s0 - TS * TS) + d(s0 + TS * TS)) + (d(s0 - TS) + d(s0 + TS))) + (d(s0 - 1) + d(s0 + 1));
      y[q] = cshift * xi - coef * s;
    }
  }
}

}  // namespace

void free_tiles(cpm_band* B, cudaStream_t s);

// Bricks, row records and work items of the tile-staged FP32 apply.
cpm_status build_tiles(cpm_band* B, cudaStream_t s) {
  const Grid g = B->grid;
  const int nbi = (g.gn[0] + TB - 1) / TB, nbj = (g.gn[1] + TB - 1) / TB, nbk = g.nkw * (64 / TB);
  const int64_t nb = (int64_t)nbi * nbj * nbk;
  int32_t *flag = nullptr, *bid = nullptr, *cnt = nullptr, *dmax = nullptr, *ext = nullptr;
  int64_t* tidx = nullptr;
  uint32_t* mask = nullptr;
  auto done = [&](cpm_status st) {
    dfree(flag, s);
    dfree(bid, s);
    dfree(cnt, s);
    dfree(dmax, s);
    dfree(ext, s);
    dfree(tidx, s);
    dfree(mask, s);
    if (st != CPM_OK) free_tiles(B, s);
    return st;
  };
  auto cu = [](cudaError_t e) { return e == cudaSuccess ? CPM_OK : fail(CPM_ERR_CUDA, "%s", cudaGetErrorString(e)); };
  cpm_status st;
  B->ntile = 0;
  if (B->nA == 0) return done(CPM_OK);
  if ((st = dalloc(&flag, nb, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&tidx, nb + 1, s)) != CPM_OK) return done(st);
  if ((st = cu(cudaMemsetAsync(flag, 0, nb * sizeof(int32_t), s))) != CPM_OK) return done(st);
  KL(k_tb_flag<<<grid_for(B->nA, 256), 256, 0, s>>>(B->nA, B->ijkA, g, nbj, nbk, flag));
  if ((st = scan_exclusive_i32(flag, tidx, nb, s)) != CPM_OK) return done(st);
  int64_t nt = 0;
  if ((st = cu(cudaMemcpyAsync(&nt, tidx + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, s))) != CPM_OK)
    return done(st);
  if ((st = cu(cudaStreamSynchronize(s))) != CPM_OK) return done(st);
  if (nt > INT32_MAX) return done(fail(CPM_ERR_ARG, "band of %lld bricks", (long long)nt));
  if ((st = dalloc(&bid, nt, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&mask, nt * TMW, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&cnt, nt, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&B->troff, nt + 1, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&ext, 6 * nt, s)) != CPM_OK) return done(st);
  KL(k_tb_list<<<grid_for(nb, 256), 256, 0, s>>>(nb, flag, tidx, bid));
  if ((st = cu(cudaMemsetAsync(mask, 0, nt * TMW * sizeof(uint32_t), s))) != CPM_OK) return done(st);
  KL(k_tb_ext_init<<<grid_for(6 * nt, 256), 256, 0, s>>>(nt, ext));
  KL(k_tb_extent<<<grid_for(B->nA, 256), 256, 0, s>>>(B->nA, B->ijkA, g, nbj, nbk, tidx, ext));
  KL(k_tb_need<<<grid_for(B->nA, 256), 256, 0, s>>>(B->nA, B->ijkA, g, nbj, nbk, tidx, mask));
  KL(k_tb_count<<<grid_for(nt, 256), 256, 0, s>>>(nt, mask, cnt));
  if ((st = scan_exclusive_i32(cnt, B->troff, nt, s)) != CPM_OK) return done(st);
  int64_t nrec = 0;
  if ((st = cu(cudaMemcpyAsync(&nrec, B->troff + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s))) != CPM_OK)
    return done(st);
  if ((st = cu(cudaStreamSynchronize(s))) != CPM_OK) return done(st);
  if ((st = dalloc(&B->thead, 8 * nt, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&B->trec, 4 * nrec, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&B->titem, nrec, s)) != CPM_OK) return done(st);
  if ((st = dalloc(&dmax, 2, s)) != CPM_OK) return done(st);
  if ((st = cu(cudaMemsetAsync(dmax, 0, 2 * sizeof(int32_t), s))) != CPM_OK) return done(st);
  TileBuildArgs A{g,       B->rmap, B->rbase, B->s32, bid, mask, ext, B->troff, nbj, nbk, B->p,
                  reinterpret_cast<TileHead*>(B->thead), reinterpret_cast<float4*>(B->trec), B->titem, dmax,
                  dmax + 1};
  if ((st = cu(cudaFuncSetAttribute(k_tb_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TBUILD_SMEM))) !=
      CPM_OK)
    return done(st);
  KL(k_tb_build<<<(unsigned)nt, TBUILD_THREADS, TBUILD_SMEM, s>>>(A));
  int32_t hv[2] = {0, 0};
  if ((st = cu(cudaMemcpyAsync(hv, dmax, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s))) != CPM_OK) return done(st);
  if ((st = cu(cudaStreamSynchronize(s))) != CPM_OK) return done(st);
  if (hv[1]) {  // a brick's box is wider than the item packing allows: keep the two-pass apply
    free_tiles(B, s);
    return done(CPM_OK);
  }
  if ((st = cu(cudaGetLastError())) != CPM_OK) return done(st);
  B->ntile = nt;
  B->tmaxbox = hv[0];
  B->ntrec = nrec;
  return done(CPM_OK);
}

void free_tiles(cpm_band* B, cudaStream_t s) {
  dfree(B->thead, s);
  dfree(B->troff, s);
  dfree(B->trec, s);
  dfree(B->titem, s);
  B->ntile = 0;
}

// y = M x in FP32 for nrhs (<= 16) right-hand sides with shifts c.
cpm_status tile_apply_f32(const cpm_band* B, const double* c, const float* x, float* y, int nrhs, cudaStream_t s) {
  if (B->ntile == 0) return CPM_OK;
  TileApplyArgs A{};
  A.g = B->grid;
  A.amap = B->amap;
  A.head = reinterpret_cast<const TileHead*>(B->thead);
  A.roff = B->troff;
  A.rec = reinterpret_cast<const float4*>(B->trec);
  A.item = B->titem;
  A.nA = B->nA;
  A.coef = (float)(1.0 / (B->h * B->h));
  for (int q = 0; q < nrhs; ++q) A.c[q] = (float)c[q];
  const size_t sm = sizeof(float2) * TSLOTS + sizeof(float) * (size_t)B->tmaxbox;
  const dim3 grid((unsigned)B->ntile, nrhs);
  if (B->p == 3) {
    CPM_CUDA(cudaFuncSetAttribute(k_tile_apply<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    KL(k_tile_apply<3><<<grid, TAPPLY_THREADS, sm, s>>>(A, x, y));
  } else {
    CPM_CUDA(cudaFuncSetAttribute(k_tile_apply<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    KL(k_tile_apply<2><<<grid, TAPPLY_THREADS, sm, s>>>(A, x, y));
  }
  CPM_CUDA(cudaGetLastError());
  return CPM_OK;
}

}  // namespace cpm
