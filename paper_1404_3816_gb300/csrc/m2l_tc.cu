// M2L (far-field translation of the H^2 product) on the tensor cores.
//
// At level l every target box B receives L_B = sum_{B' in IL(B)} K_{l, B'-B} W_{B'}
// (q x n, q = p^d Chebyshev nodes, n rays). Per target box this runs as the
// transposed product  L_B^T (n x q) = sum_{B'} W_{B'}^T (n x q) K^T (q x q)  with the
// rays as the MMA M dimension (128 per half, up to two halves), the operator rows as N
// and the source nodes as K. Operands are TF32 split into two pieces (rounded hi +
// exact remainder) and three products are accumulated in FP32 in TMEM:
//   A1 B1 + A1 B2 + A2 B1  (~2^-21 relative), no scaling needed (TF32 keeps FP32's range).
// W_{B'} is packed once per level into K-major core-matrix images, operators once per
// level; both are fed to shared memory by bulk copies (TMA engine) through a two-stage
// mbarrier pipeline. Warp 0 copies, warp 1 issues tcgen05.mma, warps 4-7 drain TMEM and
// write L (coalesced over the rays); two TMEM accumulators let the drain of one box
// overlap the MMAs of the next. Bounded waits as in the sweep kernel.
#include <math.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "m2l_tc.cuh"
#include "tc_ptx.cuh"

namespace hikf {

namespace {

using namespace tc;

constexpr int kKC = 32;       // K (source nodes) per chunk: 128-byte rows of FP32
constexpr int kStages = 2;
constexpr int kThreads = 256;

// byte offset of (row, k), k < 32, in a K-major FP32 core-matrix chunk (8 rows x 16 B cores)
__host__ __device__ __forceinline__ uint32_t off32(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
  const uint32_t u = (__float_as_uint(v) + 0x1000u) & 0xFFFFE000u;  // round to 10 mantissa bits
  hi = __uint_as_float(u);
  lo = v - hi;  // exact
}

struct Dims {
  int q, npad, nkc, ld, halves, ldp;  // ldp = 128 * halves
  int64_t a_box_bytes;                // one box: 2 pieces x nkc chunks x ldp x 128 B
  int64_t a_chunk_bytes;              // ldp x 128 B
  int64_t b_chunk_bytes;              // npad x 128 B
  int64_t b_off_bytes;                // one offset: 2 pieces x nkc chunks x npad x 128 B
};

// W[box][c][r] -> image[box][piece][chunk][core layout of (r, c mod 32)]
__global__ void pack_w_kernel(const float* __restrict__ W, int64_t box0, int64_t nboxes,
                              const int64_t* __restrict__ nsrc, Dims d, unsigned char* __restrict__ img) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_box = (int64_t)d.nkc * kKC * d.ldp;
  if (t >= nboxes * per_box) return;
  const int64_t b = t / per_box;
  if (nsrc[box0 + b] == 0) return;
  const int rem = (int)(t % per_box);
  const int c = rem / d.ldp, r = rem % d.ldp;
  const float v = (c < d.q && r < d.ld) ? W[(box0 + b) * (int64_t)d.q * d.ld + (int64_t)c * d.ld + r] : 0.f;
  float hi, lo;
  tf32_split(v, hi, lo);
  const int kc = c / kKC, kk = c % kKC;
  unsigned char* base = img + b * d.a_box_bytes + (int64_t)kc * d.a_chunk_bytes + off32(r, kk);
  *reinterpret_cast<float*>(base) = hi;
  *reinterpret_cast<float*>(base + (int64_t)d.nkc * d.a_chunk_bytes) = lo;
}

// operators K_off[a][c] (level slice of the FP32 table) -> image[off][piece][chunk][(a, c mod 32)]
__global__ void pack_k_kernel(const float* __restrict__ kop_level, int noff, Dims d, unsigned char* __restrict__ img) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_off = (int64_t)d.npad * d.nkc * kKC;
  if (t >= noff * per_off) return;
  const int off = (int)(t / per_off);
  const int rem = (int)(t % per_off);
  const int a = rem / (d.nkc * kKC), c = rem % (d.nkc * kKC);
  const float v = (a < d.q && c < d.q) ? kop_level[((int64_t)off * d.q + a) * d.q + c] : 0.f;
  float hi, lo;
  tf32_split(v, hi, lo);
  const int kc = c / kKC, kk = c % kKC;
  unsigned char* base = img + off * d.b_off_bytes + (int64_t)kc * d.b_chunk_bytes + off32(a, kk);
  *reinterpret_cast<float*>(base) = hi;
  *reinterpret_cast<float*>(base + (int64_t)d.nkc * d.b_chunk_bytes) = lo;
}

// interaction list of box B (Morton index at `lev`), deterministic order; returns count
__device__ int interaction_list(int64_t B, int lev, int dim, const int64_t* __restrict__ nsrc, int64_t box0,
                                int* __restrict__ src, int* __restrict__ offi) {
  int64_t cb[3] = {0, 0, 0};
  for (int bit = 0; bit < lev; ++bit)
    for (int d = 0; d < dim; ++d) cb[d] |= ((B >> (bit * dim + (dim - 1 - d))) & 1) << bit;
  int cnt = 0;
  const int ncand = dim == 2 ? 36 : 216;
  for (int t = 0; t < ncand; ++t) {
    int tt = t;
    int64_t cc[3] = {0, 0, 0};
    int o[3] = {0, 0, 0};
    bool ok = true, sep = false;
    for (int d = dim - 1; d >= 0; --d) {
      const int k = tt % 6;
      tt /= 6;
      cc[d] = 2 * (cb[d] >> 1) - 2 + k;
      o[d] = (int)(cc[d] - cb[d]);
      if (cc[d] < 0 || cc[d] >= ((int64_t)1 << lev)) ok = false;
      if (o[d] > 1 || o[d] < -1) sep = true;
    }
    if (!ok || !sep) continue;
    int64_t key = 0;
    for (int bit = lev - 1; bit >= 0; --bit)
      for (int d = 0; d < dim; ++d) key = (key << 1) | ((cc[d] >> bit) & 1);
    if (nsrc[box0 + key] == 0) continue;
    int oi = 0;
    for (int d = 0; d < dim; ++d) oi = oi * 7 + (o[d] + 3);
    src[cnt] = (int)key;
    offi[cnt] = oi;
    ++cnt;
  }
  return cnt;
}

__device__ bool has_interactions(int64_t B, int lev, int dim, const int64_t* __restrict__ nsrc, int64_t box0) {
  int64_t cb[3] = {0, 0, 0};
  for (int bit = 0; bit < lev; ++bit)
    for (int d = 0; d < dim; ++d) cb[d] |= ((B >> (bit * dim + (dim - 1 - d))) & 1) << bit;
  const int ncand = dim == 2 ? 36 : 216;
  for (int t = 0; t < ncand; ++t) {
    int tt = t;
    int64_t cc[3] = {0, 0, 0};
    bool ok = true, sep = false;
    for (int d = dim - 1; d >= 0; --d) {
      const int k = tt % 6;
      tt /= 6;
      cc[d] = 2 * (cb[d] >> 1) - 2 + k;
      const int o = (int)(cc[d] - cb[d]);
      if (cc[d] < 0 || cc[d] >= ((int64_t)1 << lev)) ok = false;
      if (o > 1 || o < -1) sep = true;
    }
    if (!ok || !sep) continue;
    int64_t key = 0;
    for (int bit = lev - 1; bit >= 0; --bit)
      for (int d = 0; d < dim; ++d) key = (key << 1) | ((cc[d] >> bit) & 1);
    if (nsrc[box0 + key] != 0) return true;
  }
  return false;
}

template <int NPAD, int HALVES>
__global__ void __launch_bounds__(kThreads, 1) m2l_tc_kernel(Dims d, int lev, int dim, int64_t box0, int64_t nbox,
                                                             const int64_t* __restrict__ nsrc,
                                                             const int64_t* __restrict__ npts,
                                                             const unsigned char* __restrict__ wimg,
                                                             const unsigned char* __restrict__ kimg,
                                                             float* __restrict__ Lx, int* __restrict__ err) {
  constexpr int LDP = 128 * HALVES;
  constexpr int A_CHUNK = LDP * 128;   // bytes of one A piece chunk
  constexpr int B_CHUNK = NPAD * 128;  // bytes of one B piece chunk
  constexpr int STAGE = 2 * A_CHUNK + 2 * B_CHUNK;
  constexpr int ACC_COLS = HALVES * NPAD;  // TMEM columns per accumulator buffer
  constexpr int TMEM_COLS = 2 * ACC_COLS <= 32 ? 32 : (2 * ACC_COLS <= 64 ? 64 : (2 * ACC_COLS <= 128 ? 128
                                                        : (2 * ACC_COLS <= 256 ? 256 : 512)));
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * STAGE);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (kStages + s); };
  const uint32_t acc_full0 = bar0 + 8u * (2 * kStages);
  const uint32_t acc_empty0 = acc_full0 + 16u;
  const uint32_t drain = acc_full0 + 32u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full0 + 8u * b, 1);
      mbar_init(acc_empty0 + 8u * b, 4);
    }
    mbar_init(drain, 1);
    *s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(s_tmem), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    int il_src[216], il_off[216];
    if (lane == 0) {
      int64_t j = 0;  // chunk counter across boxes
      bool ok = true;
      for (int64_t B = blockIdx.x; B < nbox && ok; B += gridDim.x) {
        if (npts[box0 + B] == 0) continue;
        const int nil = interaction_list(B, lev, dim, nsrc, box0, il_src, il_off);
        for (int e = 0; e < nil && ok; ++e) {
          for (int kc = 0; kc < d.nkc && ok; ++kc, ++j) {
            const int s = (int)(j % kStages);
            ok = mbar_wait(empty(s), (uint32_t)(((j / kStages) & 1) ^ 1), err, s_abort);
            if (!ok) break;
            const uint32_t dst = smem_u32(smem + s * STAGE);
            mbar_expect_tx(full(s), STAGE);
            const unsigned char* a = wimg + (int64_t)il_src[e] * d.a_box_bytes + (int64_t)kc * d.a_chunk_bytes;
            bulk_load(dst, a, A_CHUNK, full(s));
            bulk_load(dst + A_CHUNK, a + (int64_t)d.nkc * d.a_chunk_bytes, A_CHUNK, full(s));
            const unsigned char* bsrc = kimg + (int64_t)il_off[e] * d.b_off_bytes + (int64_t)kc * d.b_chunk_bytes;
            bulk_load(dst + 2 * A_CHUNK, bsrc, B_CHUNK, full(s));
            bulk_load(dst + 2 * A_CHUNK + B_CHUNK, bsrc + (int64_t)d.nkc * d.b_chunk_bytes, B_CHUNK, full(s));
          }
        }
      }
      if (!ok) {
        *s_abort = 1;
        const unsigned long long t0 = now_ns();
        while (now_ns() - t0 < 5000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    int il_src[216], il_off[216];
    if (lane == 0) {
      // kind::tf32: A, B TF32 (2), D F32; N = NPAD, M = 128; both K-major
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NPAD >> 3) << 17) | (8u << 24);
      int64_t j = 0, nb = 0;
      bool ok = true;
      for (int64_t B = blockIdx.x; B < nbox && ok; B += gridDim.x) {
        if (npts[box0 + B] == 0) continue;
        const int nil = interaction_list(B, lev, dim, nsrc, box0, il_src, il_off);
        if (nil == 0) continue;
        const int buf = (int)(nb & 1);
        ok = mbar_wait(acc_empty0 + 8u * buf, (uint32_t)(((nb >> 1) & 1) ^ 1), err, s_abort);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(buf * ACC_COLS);
        for (int e = 0; e < nil && ok; ++e) {
          for (int kc = 0; kc < d.nkc && ok; ++kc, ++j) {
            const int s = (int)(j % kStages);
            ok = mbar_wait(full(s), (uint32_t)((j / kStages) & 1), err, s_abort);
            if (!ok) break;
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * STAGE);
            for (int h = 0; h < HALVES; ++h) {
              for (int ks = 0; ks < kKC / 8; ++ks) {
                const uint64_t a1 = smem_desc(base + h * 16384 + ks * 256, 128, 1024);
                const uint64_t a2 = smem_desc(base + A_CHUNK + h * 16384 + ks * 256, 128, 1024);
                const uint64_t b1 = smem_desc(base + 2 * A_CHUNK + ks * 256, 128, 1024);
                const uint64_t b2 = smem_desc(base + 2 * A_CHUNK + B_CHUNK + ks * 256, 128, 1024);
                const uint32_t dd = dacc + (uint32_t)(h * NPAD);
                const uint32_t acc = (e > 0 || kc > 0 || ks > 0) ? 1u : 0u;
                tc_mma_tf32(dd, a2, b1, idesc, acc);
                tc_mma_tf32(dd, a1, b2, idesc, 1u);
                tc_mma_tf32(dd, a1, b1, idesc, 1u);
              }
            }
            tc_commit(empty(s));
          }
        }
        if (!ok) break;
        tc_commit(acc_full0 + 8u * buf);
        ++nb;
      }
      tc_commit(drain);
      mbar_wait_drain(drain, 0, err);
      if (!ok) *s_abort = 1;
    }
  } else if (warp >= 4) {
    // drain TMEM: thread = ray row (lane quarter q), writes L[B][a][r] coalesced over r
    const int q4 = warp & 3;
    int64_t nb = 0;
    bool ok = true;
    for (int64_t B = blockIdx.x; B < nbox && ok; B += gridDim.x) {
      if (npts[box0 + B] == 0) continue;
      if (!has_interactions(B, lev, dim, nsrc, box0)) continue;
      const int buf = (int)(nb & 1);
      ok = __all_sync(0xffffffffu, mbar_wait(acc_full0 + 8u * buf, (uint32_t)((nb >> 1) & 1), err, s_abort));
      if (!ok) break;
      tc_fence_after();
      float* Lb = Lx + (box0 + B) * (int64_t)d.q * d.ld;
      for (int h = 0; h < HALVES; ++h) {
        const int r = h * 128 + q4 * 32 + lane;
        for (int c0 = 0; c0 < NPAD; c0 += 32) {
          uint32_t v[32];
          tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * ACC_COLS + h * NPAD + c0), v);
          tmem_wait_ld();
          if (r < d.ld) {
#pragma unroll
            for (int u = 0; u < 32; ++u)
              if (c0 + u < d.q) Lb[(int64_t)(c0 + u) * d.ld + r] = __uint_as_float(v[u]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty0 + 8u * buf);
      ++nb;
    }
    if (!ok) *s_abort = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <int NPAD, int HALVES>
Status launch_m2l_tc(const Dims& d, int lev, int dim, int64_t box0, int64_t nbox, const int64_t* nsrc,
                     const int64_t* npts, const unsigned char* wimg, const unsigned char* kimg, float* Lx, int* err,
                     int sms, cudaStream_t s) {
  constexpr int STAGE = 2 * (128 * HALVES) * 128 + 2 * NPAD * 128;
  const int smem = kStages * STAGE + (2 * kStages + 5) * 8 + 64 + 1024;
  auto fn = m2l_tc_kernel<NPAD, HALVES>;
  HIKF_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int grid = (int)std::min<int64_t>(nbox, sms);
  fn<<<grid, kThreads, smem, s>>>(d, lev, dim, box0, nbox, nsrc, npts, wimg, kimg, Lx, err);
  HIKF_LAUNCH_CHECK("m2l_tc");
  return Status::Ok();
}

}  // namespace

bool m2l_tc_supported(int q, int ld) { return q <= 128 && ld <= 256; }

Status m2l_tc_level(const M2lTcArgs& a, cudaStream_t s) {
  Dims d;
  d.q = a.q;
  d.npad = a.q <= 32 ? 32 : (a.q <= 64 ? 64 : 128);  // MMA N of the instantiated kernel
  d.nkc = (a.q + kKC - 1) / kKC;
  d.ld = a.ld;
  d.halves = a.ld <= 128 ? 1 : 2;
  d.ldp = 128 * d.halves;
  d.a_chunk_bytes = (int64_t)d.ldp * 128;
  d.a_box_bytes = 2 * (int64_t)d.nkc * d.a_chunk_bytes;
  d.b_chunk_bytes = (int64_t)d.npad * 128;
  d.b_off_bytes = 2 * (int64_t)d.nkc * d.b_chunk_bytes;
  const int noff = a.dim == 2 ? 49 : 343;
  // images (stream-ordered scratch of this call)
  unsigned char *wimg = nullptr, *kimg = nullptr;
  HIKF_CUDA(cudaMallocAsync((void**)&wimg, (size_t)(a.nbox * d.a_box_bytes), s));
  HIKF_CUDA(cudaMallocAsync((void**)&kimg, (size_t)(noff * d.b_off_bytes), s));
  const int64_t wthreads = a.nbox * (int64_t)d.nkc * kKC * d.ldp;
  pack_w_kernel<<<nblk(wthreads, 256), 256, 0, s>>>(a.W, a.box0, a.nbox, a.nsrc, d, wimg);
  HIKF_LAUNCH_CHECK("pack_w");
  const int64_t kthreads = (int64_t)noff * d.npad * d.nkc * kKC;
  pack_k_kernel<<<nblk(kthreads, 256), 256, 0, s>>>(a.kop_level, noff, d, kimg);
  HIKF_LAUNCH_CHECK("pack_k");
  Status st;
  const int npad = d.npad;
  if (d.halves == 2) {
    if (npad <= 32) st = launch_m2l_tc<32, 2>(d, a.lev, a.dim, a.box0, a.nbox, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
    else if (npad <= 64) st = launch_m2l_tc<64, 2>(d, a.lev, a.dim, a.box0, a.nbox, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
    else st = launch_m2l_tc<128, 2>(d, a.lev, a.dim, a.box0, a.nbox, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
  } else {
    if (npad <= 32) st = launch_m2l_tc<32, 1>(d, a.lev, a.dim, a.box0, a.nbox, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
    else if (npad <= 64) st = launch_m2l_tc<64, 1>(d, a.lev, a.dim, a.box0, a.nbox, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
    else st = launch_m2l_tc<128, 1>(d, a.lev, a.dim, a.box0, a.nbox, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
  }
  HIKF_CUDA(cudaFreeAsync(wimg, s));
  HIKF_CUDA(cudaFreeAsync(kimg, s));
  return st;
}

}  // namespace hikf
