// M2L (far-field translation of the H^2 product) on the tensor cores.
//
// At level l every target box B receives L_B = sum_{B' in IL(B)} K_{l, B'-B} W_{B'}
// (q x n, q = p^d Chebyshev nodes, n rays). Per target box this runs as the
// transposed product  L_B^T (n x q) = sum_{B'} W_{B'}^T (n x q) K^T (q x q)  with the
// rays as the MMA M dimension (128 per half, up to two halves per pass, passes of 256
// rays), the operator rows as N (passes of up to 128 rows) and the source nodes as K.
// Operands are TF32 split into two pieces (hi rounded, then the remainder rounded) and
// three products are accumulated in FP32 in TMEM:
//   A1 B1 + A1 B2 + A2 B1  (~2^-21 relative), no scaling needed (TF32 keeps FP32's range).
// All levels go out in one persistent launch per pass: the work items are the
// (level, box) pairs of every level, W of all levels is packed once into K-major
// core-matrix images and the operators of all levels likewise; both are fed to shared
// memory by bulk copies (TMA engine) through a multi-stage mbarrier pipeline. Warp 0
// copies, warp 1 issues tcgen05.mma, warps 4-7 drain TMEM and write L (coalesced over
// the rays); two TMEM accumulators let the drain of one box overlap the MMAs of the
// next; the sources of a box are accumulated in groups (at most ~4096 products per
// output element per group) whose partials are summed on the CUDA cores, because the
// tensor core's FP32 accumulation drifts over long chains (3D boxes have up to 189
// sources of up to 512 nodes). A pipeline stage is one 128-ray half of a K chunk (with its
// operator chunk), so that up to four stages fit. The number of pipeline stages and of CTAs per SM are chosen by a small
// autotuner that times each feasible variant once per problem shape (the outputs of
// all variants are identical) and remembers the fastest for the process. Bounded
// waits as in the sweep kernel.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "hikf_internal.cuh"
#include "m2l_tc.cuh"
#include "tc_ptx.cuh"

namespace hikf {

namespace {

using namespace tc;

constexpr int kKC = 32;       // K (source nodes) per chunk: 128-byte rows of FP32
constexpr int kThreads = 256;

// byte offset of (row, k), k < 32, in a K-major FP32 core-matrix chunk (8 rows x 16 B cores)
__host__ __device__ __forceinline__ uint32_t off32(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_round(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);  // nearest, 10 mantissa bits
}

// v = hi + lo + O(2^-22 |v|): both pieces rounded to TF32, because kind::tf32 uses only
// the TF32 bits of an operand; an unrounded lo would be truncated, with a bias that grows
// with the length of the accumulation (thousands of terms per output in 3D)
__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
  hi = tf32_round(v);
  lo = tf32_round(v - hi);  // v - hi is exact
}

struct Dims {
  int q, npad, nkc, ld, halves, ldp;  // ldp = 128 * halves
  int r0, rw;                         // rays [r0, r0 + rw) of this pass (rw <= ldp)
  int a0, aw;                         // operator rows (target nodes) [a0, a0 + aw) of this pass (aw <= npad)
  int group;                          // source boxes accumulated in TMEM before a partial is drained
  int64_t a_box_bytes;                // one box: 2 pieces x nkc chunks x ldp x 128 B
  int64_t a_chunk_bytes;              // ldp x 128 B
  int64_t b_chunk_bytes;              // npad x 128 B
  int64_t b_off_bytes;                // one offset: 2 pieces x nkc chunks x npad x 128 B
};

// W[box][c][r] -> image[box][piece][chunk][core layout of (r, c mod 32)]
__global__ void pack_w_kernel(const float* __restrict__ W, int64_t box0, int64_t nboxes,
                              const int64_t* __restrict__ nsrc, Dims d, unsigned char* __restrict__ img) {
  // one thread: four consecutive nodes c (one 16-byte row of a core matrix) of one column
  // r; consecutive threads take consecutive columns, so the loads of W and the 16-byte
  // stores of both pieces are coalesced
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_box = (int64_t)d.nkc * (kKC / 4) * d.ldp;
  if (t >= nboxes * per_box) return;
  const int64_t b = t / per_box;
  if (nsrc[box0 + b] == 0) return;
  const int rem = (int)(t % per_box);
  const int cq = rem / d.ldp, r = rem % d.ldp;  // cq: index of the quad of nodes
  const int c0 = cq * 4;
  const float* Wb = W + (box0 + b) * (int64_t)d.q * d.ld + d.r0 + r;
  float4 hi, lo;
  float* h = &hi.x;
  float* l = &lo.x;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = c0 + u;
    const float v = (c < d.q && r < d.rw) ? Wb[(int64_t)c * d.ld] : 0.f;
    tf32_split(v, h[u], l[u]);
  }
  const int kc = c0 / kKC, kk = c0 % kKC;
  unsigned char* base = img + b * d.a_box_bytes + (int64_t)kc * d.a_chunk_bytes + off32(r, kk);
  *reinterpret_cast<float4*>(base) = hi;
  *reinterpret_cast<float4*>(base + (int64_t)d.nkc * d.a_chunk_bytes) = lo;
}

// operators K_off[a][c] (level slice of the FP32 table) -> image[off][piece][chunk][(a, c mod 32)]
__global__ void pack_k_kernel(const float* __restrict__ kop_level, int noff, Dims d, unsigned char* __restrict__ img) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_off = (int64_t)d.npad * d.nkc * kKC;
  if (t >= noff * per_off) return;
  const int off = (int)(t / per_off);
  const int rem = (int)(t % per_off);
  const int a = rem / (d.nkc * kKC), c = rem % (d.nkc * kKC);
  const float v = (a < d.aw && c < d.q) ? kop_level[((int64_t)off * d.q + d.a0 + a) * d.q + c] : 0.f;
  float hi, lo;
  tf32_split(v, hi, lo);
  const int kc = c / kKC, kk = c % kKC;
  unsigned char* base = img + off * d.b_off_bytes + (int64_t)kc * d.b_chunk_bytes + off32(a, kk);
  *reinterpret_cast<float*>(base) = hi;
  *reinterpret_cast<float*>(base + (int64_t)d.nkc * d.b_chunk_bytes) = lo;
}

// the work items of one launch: the boxes of levels lev[0] < lev[1] < ..., in order
constexpr int kMaxLevels = 16;
struct LevelTab {
  int nlev = 0;
  int lev[kMaxLevels];
  int64_t box0[kMaxLevels];        // first box of the level in the all-level arrays
  int64_t item0[kMaxLevels + 1];   // first work item of the level
};

__device__ __forceinline__ int item_level(const LevelTab& lt, int64_t it) {
  int li = 0;
  while (li + 1 < lt.nlev && it >= lt.item0[li + 1]) ++li;
  return li;
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

// number of boxes in the interaction list of box B (same test as interaction_list)
__device__ int interaction_count(int64_t B, int lev, int dim, const int64_t* __restrict__ nsrc, int64_t box0) {
  int64_t cb[3] = {0, 0, 0};
  for (int bit = 0; bit < lev; ++bit)
    for (int d = 0; d < dim; ++d) cb[d] |= ((B >> (bit * dim + (dim - 1 - d))) & 1) << bit;
  const int ncand = dim == 2 ? 36 : 216;
  int cnt = 0;
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
    if (nsrc[box0 + key] != 0) ++cnt;
  }
  return cnt;
}

// A pipeline stage holds one 128-ray half of a K chunk of W (two pieces) and the operator
// chunk (two pieces): the operator chunk, small, is copied once per half, so that a stage
// stays small enough for three or four of them in shared memory
template <int NPAD, int HALVES, int STAGES>
struct TcM2lCfg {
  static constexpr int A_HALF = 128 * 128;    // bytes of one A piece for one half (128 rays x 32 K)
  static constexpr int B_CHUNK = NPAD * 128;  // bytes of one B piece chunk
  static constexpr int STAGE = 2 * A_HALF + 2 * B_CHUNK;
  static constexpr int ACC_COLS = HALVES * NPAD;  // TMEM columns per accumulator buffer
  static constexpr int TMEM_COLS = 2 * ACC_COLS <= 32 ? 32 : (2 * ACC_COLS <= 64 ? 64 : (2 * ACC_COLS <= 128 ? 128
                                                         : (2 * ACC_COLS <= 256 ? 256 : 512)));
  static constexpr int NBARS = 2 * STAGES + 5;
  static constexpr int SMEM = STAGES * STAGE + NBARS * 8 + 64 + 1024;
};

template <int NPAD, int HALVES, int STAGES>
__global__ void __launch_bounds__(kThreads, 1) m2l_tc_kernel(Dims d, LevelTab lt, int dim, int64_t wbox0,
                                                             const int64_t* __restrict__ nsrc,
                                                             const int64_t* __restrict__ npts,
                                                             const unsigned char* __restrict__ wimg,
                                                             const unsigned char* __restrict__ kimg,
                                                             float* __restrict__ Lx, int* __restrict__ err) {
  using Cfg = TcM2lCfg<NPAD, HALVES, STAGES>;
  constexpr int A_HALF = Cfg::A_HALF, B_CHUNK = Cfg::B_CHUNK, STAGE = Cfg::STAGE;
  constexpr int ACC_COLS = Cfg::ACC_COLS, TMEM_COLS = Cfg::TMEM_COLS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + Cfg::NBARS);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (STAGES + s); };
  const uint32_t acc_full0 = bar0 + 8u * (2 * STAGES);
  const uint32_t acc_empty0 = acc_full0 + 16u;
  const uint32_t drain = acc_full0 + 32u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int noff = dim == 2 ? 49 : 343;
  const int64_t nitems = lt.item0[lt.nlev];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
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
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const int li = item_level(lt, it);
        const int lev = lt.lev[li];
        const int64_t B = it - lt.item0[li], box0 = lt.box0[li];
        if (npts[box0 + B] == 0) continue;
        const int nil = interaction_list(B, lev, dim, nsrc, box0, il_src, il_off);
        const unsigned char* wl = wimg + (box0 - wbox0) * d.a_box_bytes;
        const unsigned char* kl = kimg + (int64_t)(lev - 2) * noff * d.b_off_bytes;
        for (int e = 0; e < nil && ok; ++e) {
          for (int kc = 0; kc < d.nkc && ok; ++kc) {
            for (int h = 0; h < HALVES && ok; ++h, ++j) {
              const int s = (int)(j % STAGES);
              ok = mbar_wait(empty(s), (uint32_t)(((j / STAGES) & 1) ^ 1), err, s_abort);
              if (!ok) break;
              const uint32_t dst = smem_u32(smem + s * STAGE);
              mbar_expect_tx(full(s), STAGE);
              // the half's rows of the chunk: 128-row groups are contiguous in the image
              const unsigned char* a =
                  wl + (int64_t)il_src[e] * d.a_box_bytes + (int64_t)kc * d.a_chunk_bytes + (int64_t)h * A_HALF;
              bulk_load(dst, a, A_HALF, full(s));
              bulk_load(dst + A_HALF, a + (int64_t)d.nkc * d.a_chunk_bytes, A_HALF, full(s));
              const unsigned char* bsrc = kl + (int64_t)il_off[e] * d.b_off_bytes + (int64_t)kc * d.b_chunk_bytes;
              bulk_load(dst + 2 * A_HALF, bsrc, B_CHUNK, full(s));
              bulk_load(dst + 2 * A_HALF + B_CHUNK, bsrc + (int64_t)d.nkc * d.b_chunk_bytes, B_CHUNK, full(s));
            }
          }
        }
      }
      if (!ok) *s_abort = 1;
      // every copy issued (j of them) has landed before the CTA may exit
      drain_ring(full(0), STAGES, j, err);
    }
  } else if (warp == 1) {
    int il_src[216], il_off[216];
    if (lane == 0) {
      // kind::tf32: A, B TF32 (2), D F32; N = NPAD, M = 128; both K-major
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NPAD >> 3) << 17) | (8u << 24);
      int64_t j = 0, nb = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
        const int li = item_level(lt, it);
        const int lev = lt.lev[li];
        const int64_t B = it - lt.item0[li], box0 = lt.box0[li];
        if (npts[box0 + B] == 0) continue;
        const int nil = interaction_list(B, lev, dim, nsrc, box0, il_src, il_off);
        if (nil == 0) continue;
        uint32_t dacc = 0;
        int buf = 0;
        for (int e = 0; e < nil && ok; ++e) {
          const int ge = e % d.group;  // position in the current group of sources
          if (ge == 0) {
            buf = (int)(nb & 1);
            ok = mbar_wait(acc_empty0 + 8u * buf, (uint32_t)(((nb >> 1) & 1) ^ 1), err, s_abort);
            if (!ok) break;
            tc_fence_after();
            dacc = tmem + (uint32_t)(buf * ACC_COLS);
          }
          for (int kc = 0; kc < d.nkc && ok; ++kc) {
            for (int h = 0; h < HALVES && ok; ++h, ++j) {
              const int s = (int)(j % STAGES);
              ok = mbar_wait(full(s), (uint32_t)((j / STAGES) & 1), err, s_abort);
              if (!ok) break;
              tc_fence_after();
              const uint32_t base = smem_u32(smem + s * STAGE);
              for (int ks = 0; ks < kKC / 8; ++ks) {
                const uint64_t a1 = smem_desc(base + ks * 256, 128, 1024);
                const uint64_t a2 = smem_desc(base + A_HALF + ks * 256, 128, 1024);
                const uint64_t b1 = smem_desc(base + 2 * A_HALF + ks * 256, 128, 1024);
                const uint64_t b2 = smem_desc(base + 2 * A_HALF + B_CHUNK + ks * 256, 128, 1024);
                const uint32_t dd = dacc + (uint32_t)(h * NPAD);
                const uint32_t acc = (ge > 0 || kc > 0 || ks > 0) ? 1u : 0u;
                tc_mma_tf32(dd, a2, b1, idesc, acc);
                tc_mma_tf32(dd, a1, b2, idesc, 1u);
                tc_mma_tf32(dd, a1, b1, idesc, 1u);
              }
              tc_commit(empty(s));
            }
          }
          if (ok && (ge == d.group - 1 || e == nil - 1)) {
            tc_commit(acc_full0 + 8u * buf);  // a partial over this group of sources
            ++nb;
          }
        }
        if (!ok) break;
      }
      tc_commit(drain);
      mbar_wait_drain(drain, 0, err);
      if (!ok) *s_abort = 1;
    }
  } else if (warp >= 4) {
    // drain TMEM: thread = ray row (lane quarter q), writes L[B][a][r0 + r] coalesced over r
    const int q4 = warp & 3;
    int64_t nb = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < nitems && ok; it += gridDim.x) {
      const int li = item_level(lt, it);
      const int lev = lt.lev[li];
      const int64_t B = it - lt.item0[li], box0 = lt.box0[li];
      if (npts[box0 + B] == 0) continue;
      const int nil = interaction_count(B, lev, dim, nsrc, box0);
      const int ngroups = (nil + d.group - 1) / d.group;
      float* Lb = Lx + (box0 + B) * (int64_t)d.q * d.ld + (int64_t)d.a0 * d.ld + d.r0;
      for (int gi = 0; gi < ngroups && ok; ++gi) {
        const int buf = (int)(nb & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(acc_full0 + 8u * buf, (uint32_t)((nb >> 1) & 1), err, s_abort));
        if (!ok) break;
        tc_fence_after();
        // the first partial is written, later ones added (FP32, round to nearest): the
        // tensor-core accumulation chains stay short
        for (int h = 0; h < HALVES; ++h) {
          const int r = h * 128 + q4 * 32 + lane;
          for (int c0 = 0; c0 < NPAD; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * ACC_COLS + h * NPAD + c0), v);
            tmem_wait_ld();
            if (r < d.rw) {
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (c0 + u < d.aw) {
                  float* dst = Lb + (int64_t)(c0 + u) * d.ld + r;
                  *dst = gi == 0 ? __uint_as_float(v[u]) : *dst + __uint_as_float(v[u]);
                }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty0 + 8u * buf);
        ++nb;
      }
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

// one launch variant: pipeline stages and CTAs per SM
struct Variant {
  int stages = 2, per_sm = 1;
};

template <int NPAD, int HALVES, int STAGES>
Status launch_variant(const Dims& d, const LevelTab& lt, int dim, int64_t wbox0, const int64_t* nsrc,
                      const int64_t* npts, const unsigned char* wimg, const unsigned char* kimg, float* Lx, int* err,
                      int grid, cudaStream_t s) {
  using Cfg = TcM2lCfg<NPAD, HALVES, STAGES>;
  auto fn = m2l_tc_kernel<NPAD, HALVES, STAGES>;
  HIKF_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
  fn<<<grid, kThreads, Cfg::SMEM, s>>>(d, lt, dim, wbox0, nsrc, npts, wimg, kimg, Lx, err);
  HIKF_LAUNCH_CHECK("m2l_tc");
  return Status::Ok();
}

template <int NPAD, int HALVES>
Status launch_npad_halves(const Variant& v, const Dims& d, const LevelTab& lt, int dim, int64_t wbox0,
                          const int64_t* nsrc, const int64_t* npts, const unsigned char* wimg,
                          const unsigned char* kimg, float* Lx, int* err, int sms, cudaStream_t s) {
  const int64_t nitems = lt.item0[lt.nlev];
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nitems, (int64_t)sms * v.per_sm));
  if (v.stages == 4)
    return launch_variant<NPAD, HALVES, 4>(d, lt, dim, wbox0, nsrc, npts, wimg, kimg, Lx, err, grid, s);
  if (v.stages == 3)
    return launch_variant<NPAD, HALVES, 3>(d, lt, dim, wbox0, nsrc, npts, wimg, kimg, Lx, err, grid, s);
  return launch_variant<NPAD, HALVES, 2>(d, lt, dim, wbox0, nsrc, npts, wimg, kimg, Lx, err, grid, s);
}

Status launch(const Variant& v, const Dims& d, const LevelTab& lt, int dim, int64_t wbox0, const int64_t* nsrc,
              const int64_t* npts, const unsigned char* wimg, const unsigned char* kimg, float* Lx, int* err, int sms,
              cudaStream_t s) {
#define HIKF_M2L_CASE(NP, HV)                                                                              \
  if (d.npad == NP && d.halves == HV)                                                                      \
    return launch_npad_halves<NP, HV>(v, d, lt, dim, wbox0, nsrc, npts, wimg, kimg, Lx, err, sms, s);
  HIKF_M2L_CASE(32, 1)
  HIKF_M2L_CASE(64, 1)
  HIKF_M2L_CASE(128, 1)
  HIKF_M2L_CASE(32, 2)
  HIKF_M2L_CASE(64, 2)
  HIKF_M2L_CASE(128, 2)
#undef HIKF_M2L_CASE
  return make_status(HIKF_EINVAL, "tensor-core M2L: unsupported shape");
}

// shared memory and TMEM of one CTA of a variant (for the feasibility of stages and CTAs per SM)
void variant_footprint(int npad, int halves, int stages, int* smem, int* tmem_cols) {
  const int stage = 2 * 128 * 128 + 2 * npad * 128;
  *smem = stages * stage + (2 * stages + 5) * 8 + 64 + 1024;
  const int acc = 2 * halves * npad;
  *tmem_cols = acc <= 32 ? 32 : (acc <= 64 ? 64 : (acc <= 128 ? 128 : (acc <= 256 ? 256 : 512)));
}

std::vector<Variant> feasible_variants(int npad, int halves) {
  std::vector<Variant> out;
  for (int st = 2; st <= 4; ++st) {
    int smem = 0, tcols = 0;
    variant_footprint(npad, halves, st, &smem, &tcols);
    if (smem > 227 * 1024) continue;
    for (int per = 1; per <= 2; ++per) {
      if (per * (smem + 1024) > 228 * 1024 || per * tcols > 512) continue;
      out.push_back(Variant{st, per});
    }
  }
  return out;
}

// the autotuner's memory: (dim, npad, halves, work items) -> fastest variant
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int64_t>, Variant> g_tuned;

}  // namespace

bool m2l_tc_supported(int q, int ld) { return q >= 1 && ld >= 1; }

Status m2l_tc_all(const M2lTcAll& a, cudaStream_t s) {
  if (a.nlev < 1 || a.nlev > kMaxLevels) return make_status(HIKF_EINVAL, "tensor-core M2L: level count");
  LevelTab lt;
  lt.nlev = a.nlev;
  int64_t items = 0;
  for (int i = 0; i < a.nlev; ++i) {
    lt.lev[i] = a.lev[i];
    lt.box0[i] = a.box0[i];
    lt.item0[i] = items;
    items += a.nbox[i];
  }
  lt.item0[a.nlev] = items;
  const int64_t wbox0 = a.box0[0];
  const int64_t nboxes = items;  // the levels are contiguous in the all-level arrays
  const int noff = a.dim == 2 ? 49 : 343;
  const int nkc = (a.q + kKC - 1) / kKC;
  // operator images of all levels for one pass of up to 128 operator rows (MMA N)
  const int64_t b_chunk_max = 128 * 128, b_off_max = 2 * (int64_t)nkc * b_chunk_max;
  unsigned char* kimg = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&kimg, (size_t)((int64_t)a.nlev * noff * b_off_max), s));
  Status st;
  // passes of up to 256 rays (two 128-row MMA halves); W is packed once per ray pass
  for (int r0 = 0; r0 < a.ld && st.ok(); r0 += 256) {
    Dims d;
    d.q = a.q;
    d.nkc = nkc;
    d.ld = a.ld;
    d.r0 = r0;
    d.rw = std::min(256, a.ld - r0);
    d.halves = d.rw <= 128 ? 1 : 2;
    d.ldp = 128 * d.halves;
    d.a_chunk_bytes = (int64_t)d.ldp * 128;
    d.a_box_bytes = 2 * (int64_t)d.nkc * d.a_chunk_bytes;
    unsigned char* wimg = nullptr;
    HIKF_CUDA(hikf::pool_malloc((void**)&wimg, (size_t)(nboxes * d.a_box_bytes), s));
    const int64_t wthreads = nboxes * (int64_t)d.nkc * (kKC / 4) * d.ldp;
    pack_w_kernel<<<nblk(wthreads, 256), 256, 0, s>>>(a.W, wbox0, nboxes, a.nsrc, d, wimg);
    HIKF_LAUNCH_CHECK("pack_w");
    // sources per TMEM accumulation: at most ~4096 products per output element
    d.group = std::max(1, 4096 / (nkc * kKC));
    for (int a0 = 0; a0 < a.q && st.ok(); a0 += 128) {
      d.a0 = a0;
      d.aw = std::min(128, a.q - a0);
      d.npad = d.aw <= 32 ? 32 : (d.aw <= 64 ? 64 : 128);  // MMA N of the instantiated kernel
      d.b_chunk_bytes = (int64_t)d.npad * 128;
      d.b_off_bytes = 2 * (int64_t)nkc * d.b_chunk_bytes;
      const int64_t kthreads = (int64_t)a.nlev * noff * d.npad * nkc * kKC;
      pack_k_kernel<<<nblk(kthreads, 256), 256, 0, s>>>(a.kop, a.nlev * noff, d, kimg);
      HIKF_LAUNCH_CHECK("pack_k");
      // the variant: tuned once per shape (every variant writes the same L, so timing one
      // on the real data is harmless), then remembered
      const auto key = std::make_tuple(a.dim, d.npad, d.halves, items);
      Variant v;
      bool known = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto f = g_tuned.find(key);
        if (f != g_tuned.end()) {
          v = f->second;
          known = true;
        }
      }
      if (!known && a.autotune) {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        const std::vector<Variant> cands = feasible_variants(d.npad, d.halves);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        HIKF_CUDA(cudaEventCreate(&e0));
        HIKF_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        for (const Variant& c : cands) {
          HIKF_CUDA(cudaEventRecord(e0, s));
          st = launch(c, d, lt, a.dim, wbox0, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
          if (!st.ok()) break;
          HIKF_CUDA(cudaEventRecord(e1, s));
          HIKF_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          HIKF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            v = c;
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st.ok()) g_tuned[key] = v;  // L already holds this pass (every candidate wrote it)
      } else {
        st = launch(v, d, lt, a.dim, wbox0, a.nsrc, a.npts, wimg, kimg, a.L, a.err, a.sms, s);
      }
    }
    HIKF_CUDA(cudaFreeAsync(wimg, s));
  }
  HIKF_CUDA(cudaFreeAsync(kimg, s));
  return st;
}

}  // namespace hikf
