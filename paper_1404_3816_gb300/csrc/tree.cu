// T1 tree build (uniform 2^d-tree in Morton order) and T2 source packing.
//
// The H^2 approach subdivides the domain recursively along a tree (Sec. 3.2);
// here the tree is uniform: a cube around the points' bounding box, depth L,
// points sorted by the Morton key of their leaf so that every box at every
// level owns a contiguous range of points.
#include <math.h>

#include <algorithm>
#include <vector>

#include "hikf_internal.cuh"

namespace hikf {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                       // items per thread per tile (radix sort)
constexpr int kTile = kThreads * kItems;        // items per block tile

// ---------------------------------------------------------------------------
// bounding box
// ---------------------------------------------------------------------------
__global__ void bbox_partial(const double* __restrict__ pts, int64_t m, int dim, double* __restrict__ part) {
  __shared__ double smin[3][kThreads];
  __shared__ double smax[3][kThreads];
  double lo[3] = {INFINITY, INFINITY, INFINITY};
  double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < dim; ++d) {
      double v = pts[i * dim + d];
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  }
  for (int d = 0; d < 3; ++d) {
    smin[d][threadIdx.x] = lo[d];
    smax[d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      for (int d = 0; d < 3; ++d) {
        smin[d][threadIdx.x] = fmin(smin[d][threadIdx.x], smin[d][threadIdx.x + s]);
        smax[d][threadIdx.x] = fmax(smax[d][threadIdx.x], smax[d][threadIdx.x + s]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; ++d) {
      part[blockIdx.x * 6 + d] = smin[d][0];
      part[blockIdx.x * 6 + 3 + d] = smax[d][0];
    }
  }
}

// ---------------------------------------------------------------------------
// leaf coordinates and Morton keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t morton_key(const int64_t* c, int dim, int depth) {
  uint64_t key = 0;
  for (int b = depth - 1; b >= 0; --b)
    for (int d = 0; d < dim; ++d) key = (key << 1) | (uint64_t)((c[d] >> b) & 1);
  return key;
}

__global__ void leaf_keys(const double* __restrict__ pts, int64_t m, int dim, int depth, double lo0, double lo1,
                          double lo2, double w, uint64_t* __restrict__ keys, int64_t* __restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double lo[3] = {lo0, lo1, lo2};
  const int64_t top = ((int64_t)1 << depth) - 1;
  int64_t c[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    // explicit round-to-nearest ops: no contraction, so the leaf of a point is
    // the IEEE value floor((x - lo) / w)
    double u = __ddiv_rn(__dsub_rn(pts[i * dim + d], lo[d]), w);
    int64_t k = (int64_t)floor(u);
    c[d] = k < 0 ? 0 : (k > top ? top : k);
  }
  keys[i] = morton_key(c, dim, depth);
  idx[i] = i;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, index), 8-bit digits
// ---------------------------------------------------------------------------
__global__ void radix_hist(const uint64_t* __restrict__ keys, int64_t m, int shift, int nblocks,
                           int64_t* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int c = 0; c < kItems; ++c) {
    int64_t i = base + (int64_t)c * kThreads + threadIdx.x;
    if (i < m) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void radix_scatter(const uint64_t* __restrict__ kin, const int64_t* __restrict__ vin,
                              uint64_t* __restrict__ kout, int64_t* __restrict__ vout, int64_t m, int shift,
                              int nblocks, const int64_t* __restrict__ offs) {
  __shared__ int64_t run[256];
  __shared__ int wcnt[kThreads / 32][256];
  __shared__ int total[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * kTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kItems; ++c) {
    for (int k = tid; k < (kThreads / 32) * 256; k += kThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    int64_t i = base + (int64_t)c * kThreads + tid;
    bool valid = i < m;
    uint64_t key = valid ? kin[i] : 0;
    int dg = valid ? (int)((key >> shift) & 255) : 256 + 0;
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    int rank = __popc(peers & lt);
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][dg] = __popc(peers);
    __syncthreads();
    {
      int s = 0;
      for (int w = 0; w < kThreads / 32; ++w) {
        int v = wcnt[w][tid];
        wcnt[w][tid] = s;
        s += v;
      }
      total[tid] = s;
    }
    __syncthreads();
    if (valid) {
      int64_t pos = run[dg] + wcnt[warp][dg] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    run[tid] += total[tid];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// exclusive scan (int64), two-level
// ---------------------------------------------------------------------------
__global__ void scan_blocks(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t* __restrict__ bsum,
                            int64_t count) {
  __shared__ int64_t s[kThreads];
  int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
  int64_t v[kItems];
  int64_t acc = 0;
  for (int k = 0; k < kItems; ++k) {
    int64_t i = base + k;
    v[k] = i < count ? in[i] : 0;
    acc += v[k];
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 1; off < kThreads; off <<= 1) {
    int64_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  int64_t run = s[threadIdx.x] - acc;
  for (int k = 0; k < kItems; ++k) {
    int64_t i = base + k;
    if (i < count) out[i] = run;
    run += v[k];
  }
  if (threadIdx.x == kThreads - 1 && bsum) bsum[blockIdx.x] = s[threadIdx.x];
}

__global__ void scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ boff, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] += boff[i / kTile];
}

__global__ void binary_starts(const uint64_t* __restrict__ sorted_keys, int64_t m, int64_t nleaf,
                              int64_t* __restrict__ start) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k > nleaf) return;
  int64_t lo = 0, hi = m;  // first index with key >= k
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (sorted_keys[mid] < (uint64_t)k) lo = mid + 1; else hi = mid;
  }
  start[k] = lo;
}

__global__ void gather_points(const double* __restrict__ pts, const int64_t* __restrict__ perm, int64_t m, int dim,
                              double* __restrict__ out, int64_t* __restrict__ iperm) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m) return;
  int64_t i = perm[s];
  for (int d = 0; d < dim; ++d) out[s * dim + d] = pts[i * dim + d];
  iperm[i] = s;
}

// ---------------------------------------------------------------------------
// sparse H in tree order
// ---------------------------------------------------------------------------
__global__ void map_cols(const int64_t* __restrict__ col, const int64_t* __restrict__ iperm, int64_t nnz,
                         int32_t* __restrict__ out, int64_t* __restrict__ count) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  int64_t c = iperm[col[k]];
  out[k] = (int32_t)c;
  atomicAdd(reinterpret_cast<unsigned long long*>(&count[c]), 1ull);
}

__global__ void transpose_scatter(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, int n, const int64_t* __restrict__ trowptr,
                                  int64_t* __restrict__ cursor, int32_t* __restrict__ tcol,
                                  double* __restrict__ tval) {
  int r = blockIdx.x;
  if (r >= n) return;
  for (int64_t k = rowptr[r] + threadIdx.x; k < rowptr[r + 1]; k += blockDim.x) {
    int32_t c = col[k];
    int64_t pos = trowptr[c] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[c]), 1ull);
    tcol[pos] = r;
    tval[pos] = val[k];
  }
}

// entries of one H^T row sorted by (ray, value): a deterministic layout
__global__ void sort_rows(const int64_t* __restrict__ trowptr, int64_t m, int32_t* __restrict__ tcol,
                          double* __restrict__ tval) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t a = trowptr[i], b = trowptr[i + 1];
  for (int64_t p = a + 1; p < b; ++p) {
    int32_t c = tcol[p];
    double v = tval[p];
    int64_t q = p - 1;
    while (q >= a && (tcol[q] > c || (tcol[q] == c && tval[q] > v))) {
      tcol[q + 1] = tcol[q];
      tval[q + 1] = tval[q];
      --q;
    }
    tcol[q + 1] = c;
    tval[q + 1] = v;
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// exclusive scan of `count` int64 values (count <= kTile^2); tmp holds >= 2 * ceil(count / kTile) + 1
Status exclusive_scan(const int64_t* in, int64_t* out, int64_t count, int64_t* tmp, cudaStream_t s) {
  if (count <= 0) return Status::Ok();
  int64_t nb = (count + kTile - 1) / kTile;
  if (nb > kTile) return make_status(HIKF_EINVAL, "scan longer than supported");
  int64_t* bsum = tmp;
  int64_t* boff = tmp + nb;
  scan_blocks<<<(unsigned)nb, kThreads, 0, s>>>(in, out, nb > 1 ? bsum : nullptr, count);
  HIKF_LAUNCH_CHECK("scan_blocks");
  if (nb > 1) {
    scan_blocks<<<1, kThreads, 0, s>>>(bsum, boff, nullptr, nb);
    HIKF_LAUNCH_CHECK("scan_blocks(2)");
    scan_add<<<nblk(count, kThreads), kThreads, 0, s>>>(out, boff, count);
    HIKF_LAUNCH_CHECK("scan_add");
  }
  return Status::Ok();
}

int auto_depth(int64_t m, int dim, int leaf_size) {
  int L = 0;
  while (m > (int64_t)leaf_size * ((int64_t)1 << (dim * L))) ++L;
  return L;
}

Status build_tree(Tree& t, Arena& arena, const double* d_pts, cudaStream_t s) {
  const int64_t m = t.m;
  const int dim = t.dim;
  // bounding box
  int nb = std::min<int64_t>(1024, (m + kThreads - 1) / kThreads);
  double* d_part = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&d_part, sizeof(double) * 6 * nb, s));
  bbox_partial<<<nb, kThreads, 0, s>>>(d_pts, m, dim, d_part);
  HIKF_LAUNCH_CHECK("bbox_partial");
  std::vector<double> part(6 * nb);
  HIKF_CUDA(cudaMemcpyAsync(part.data(), d_part, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, s));
  HIKF_CUDA(cudaStreamSynchronize(s));
  HIKF_CUDA(cudaFreeAsync(d_part, s));
  double pmin[3] = {INFINITY, INFINITY, INFINITY}, pmax[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b)
    for (int d = 0; d < dim; ++d) {
      pmin[d] = std::min(pmin[d], part[b * 6 + d]);
      pmax[d] = std::max(pmax[d], part[b * 6 + 3 + d]);
    }
  double side = 0.0;
  for (int d = 0; d < dim; ++d) side = std::max(side, pmax[d] - pmin[d]);
  if (!(side > 0.0)) side = 1.0;
  t.side = side;
  for (int d = 0; d < 3; ++d) t.lo[d] = d < dim ? 0.5 * (pmin[d] + pmax[d]) - 0.5 * side : 0.0;
  const double w = side / (double)((int64_t)1 << t.depth);
  t.nleaf = (int64_t)1 << (dim * t.depth);

  // keys, sort
  uint64_t *k0 = nullptr, *k1 = nullptr;
  int64_t *v0 = nullptr, *v1 = nullptr, *hist = nullptr, *tmp = nullptr;
  const int nbl = (int)((m + kTile - 1) / kTile);
  HIKF_CUDA(hikf::pool_malloc((void**)&k0, sizeof(uint64_t) * m, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&k1, sizeof(uint64_t) * m, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&v0, sizeof(int64_t) * m, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&v1, sizeof(int64_t) * m, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&hist, sizeof(int64_t) * 256 * (size_t)nbl * 2, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&tmp, sizeof(int64_t) * (2 * (256 * (size_t)nbl / kTile + 2) + 8), s));
  leaf_keys<<<nblk(m, kThreads), kThreads, 0, s>>>(d_pts, m, dim, t.depth, t.lo[0], t.lo[1], t.lo[2], w, k0, v0);
  HIKF_LAUNCH_CHECK("leaf_keys");
  const int bits = dim * t.depth;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist<<<nbl, kThreads, 0, s>>>(k0, m, shift, nbl, hist);
    HIKF_LAUNCH_CHECK("radix_hist");
    HIKF_TRY(exclusive_scan(hist, hist + 256 * (size_t)nbl, 256 * (int64_t)nbl, tmp, s));
    radix_scatter<<<nbl, kThreads, 0, s>>>(k0, v0, k1, v1, m, shift, nbl, hist + 256 * (size_t)nbl);
    HIKF_LAUNCH_CHECK("radix_scatter");
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  HIKF_TRY(arena_alloc(arena, &t.perm, m));
  HIKF_TRY(arena_alloc(arena, &t.iperm, m));
  HIKF_TRY(arena_alloc(arena, &t.leaf_start, t.nleaf + 1));
  HIKF_TRY(arena_alloc(arena, &t.pts, m * dim));
  HIKF_CUDA(cudaMemcpyAsync(t.perm, v0, sizeof(int64_t) * m, cudaMemcpyDeviceToDevice, s));
  binary_starts<<<nblk(t.nleaf + 1, kThreads), kThreads, 0, s>>>(k0, m, t.nleaf, t.leaf_start);
  HIKF_LAUNCH_CHECK("binary_starts");
  gather_points<<<nblk(m, kThreads), kThreads, 0, s>>>(d_pts, t.perm, m, dim, t.pts, t.iperm);
  HIKF_LAUNCH_CHECK("gather_points");
  HIKF_CUDA(cudaFreeAsync(k0, s));
  HIKF_CUDA(cudaFreeAsync(k1, s));
  HIKF_CUDA(cudaFreeAsync(v0, s));
  HIKF_CUDA(cudaFreeAsync(v1, s));
  HIKF_CUDA(cudaFreeAsync(hist, s));
  HIKF_CUDA(cudaFreeAsync(tmp, s));
  int64_t off = 0;
  for (int l = 0; l <= t.depth; ++l) {
    t.box_offset[l] = off;
    off += (int64_t)1 << (dim * l);
  }
  t.box_offset[t.depth + 1] = off;
  t.nbox_total = off;
  return Status::Ok();
}

Status build_sparse(SparseH& h, Arena& arena, const Tree& t, const int64_t* h_rowptr, const int64_t* h_col,
                    const double* h_val, int n, cudaStream_t s) {
  const int64_t nnz = h_rowptr[n];
  const int64_t m = t.m;
  h.n = n;
  h.nnz = nnz;
  HIKF_TRY(arena_alloc(arena, &h.rowptr, n + 1));
  HIKF_TRY(arena_alloc(arena, &h.col, std::max<int64_t>(nnz, 1)));
  HIKF_TRY(arena_alloc(arena, &h.val, std::max<int64_t>(nnz, 1)));
  HIKF_TRY(arena_alloc(arena, &h.trowptr, m + 1));
  HIKF_TRY(arena_alloc(arena, &h.tcol, std::max<int64_t>(nnz, 1)));
  HIKF_TRY(arena_alloc(arena, &h.tval, std::max<int64_t>(nnz, 1)));
  HIKF_CUDA(cudaMemcpyAsync(h.rowptr, h_rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  int64_t *d_col = nullptr, *count = nullptr, *cursor = nullptr, *tmp = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&d_col, sizeof(int64_t) * std::max<int64_t>(nnz, 1), s));
  HIKF_CUDA(hikf::pool_malloc((void**)&count, sizeof(int64_t) * (m + 1), s));
  HIKF_CUDA(hikf::pool_malloc((void**)&cursor, sizeof(int64_t) * (m + 1), s));
  HIKF_CUDA(hikf::pool_malloc((void**)&tmp, sizeof(int64_t) * (2 * ((m + 1) / kTile + 2) + 8), s));
  HIKF_CUDA(cudaMemsetAsync(count, 0, sizeof(int64_t) * (m + 1), s));
  HIKF_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int64_t) * (m + 1), s));
  if (nnz > 0) {
    HIKF_CUDA(cudaMemcpyAsync(d_col, h_col, sizeof(int64_t) * nnz, cudaMemcpyHostToDevice, s));
    HIKF_CUDA(cudaMemcpyAsync(h.val, h_val, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    map_cols<<<nblk(nnz, kThreads), kThreads, 0, s>>>(d_col, t.iperm, nnz, h.col, count);
    HIKF_LAUNCH_CHECK("map_cols");
  }
  HIKF_TRY(exclusive_scan(count, h.trowptr, m + 1, tmp, s));
  if (nnz > 0) {
    transpose_scatter<<<n, kThreads, 0, s>>>(h.rowptr, h.col, h.val, n, h.trowptr, cursor, h.tcol, h.tval);
    HIKF_LAUNCH_CHECK("transpose_scatter");
    sort_rows<<<nblk(m, kThreads), kThreads, 0, s>>>(h.trowptr, m, h.tcol, h.tval);
    HIKF_LAUNCH_CHECK("sort_rows");
  }
  HIKF_CUDA(cudaFreeAsync(d_col, s));
  HIKF_CUDA(cudaFreeAsync(count, s));
  HIKF_CUDA(cudaFreeAsync(cursor, s));
  HIKF_CUDA(cudaFreeAsync(tmp, s));
  return Status::Ok();
}

}  // namespace hikf
