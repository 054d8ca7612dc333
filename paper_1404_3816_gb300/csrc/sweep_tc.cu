// The measurement-update sweep (S4) on the 5th-generation tensor cores.
//
// Per 128-row tile of the m x n cross-covariance (Alg. 2):
//   C_p = C + C_Q,  K = C_p M,  delta^2 += diag(Q) - sum_j K_ij C_p,ij,
//   x += C_p a,  C <- K R  (= C_p - K H C_p, Eq. KF_pred_new, since H C_p = S - R).
//
// K = C_p M is a dense (m x n) x (n x n) contraction. To keep FP32-level accuracy
// on FP16 tensor cores each operand is split into FP16 pieces after a power-of-two
// scaling (row scale alpha_i for C_p, one scale beta for M):
//   alpha C_p = A1 + A2 (22 significant bits),  beta M = B1 + B2 + B3 (33 bits),
//   K = (A1 B1 + A1 B2 + A2 B1 + A1 B3 + A2 B2) / (alpha beta),
// i.e. every product down to 2^-22 of the leading one; products are exact in the
// FP32 accumulator. Measured against the FP64 oracle, a third piece of C_p (a sixth
// product) changes neither the mean nor the variance error (the FP32 accumulation of
// the tensor core sets them); it would cost a sixth more tensor-core time, which sets
// the pace of a tile (each M=128, N=256, K=16 instruction takes ~72 ns). A well-
// conditioned update (cond S_t <= 3e3, decided at create) splits M into two pieces only:
// four products (A1 B3 left out), a fifth less tensor time, and a third less B traffic from
// L2 per chunk, which buys a three-stage B ring in the same shared memory. Two pieces of M
// are not enough in general: on an n = 100 case with cond S_t ~ 9e3 they lost the 1e-5
// bound on the variance.
// The row scale comes from a bound carried from the previous step:
// |C_p,ij| <= max_j |C_{t|t}| + max_j |C_Q|.
//
// Data path (one persistent CTA per SM, warp-specialised):
//   warp 0      TMA: raw FP32 tiles of C and C_Q (128 rows x 32 columns, 128B
//               swizzle)
//   warp 2      bulk copies of the pre-laid-out FP16 images of M (a producer of its
//               own, so the raw ring runs ahead of the MMAs)
//   warps 4-7   one thread per row: C_p = C + C_Q, x increment, split into FP16
//               pieces in the canonical no-swizzle K-major layout, C_p into TMEM;
//               after the MMAs: epilogue from TMEM (rowdot, C <- K R, row max)
//   warp 1      TMEM allocation and the single-thread tcgen05.mma issue
// TMEM (512 columns): accumulator K in columns [0, 256), C_p in [256, 512).
// Every wait is bounded (about two seconds); a timeout sets an error code,
// drains the copies and MMAs in flight, frees TMEM and returns. The cross-covariance
// is updated in place tile by tile, so after a timeout its state is undefined (the
// host reports HIKF_ETIMEOUT once and HIKF_ESTATE for every later call).
#include <cuda.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "sweep_tc.cuh"
#include "tc_ptx.cuh"

namespace hikf {

namespace {

constexpr int kBM = 128;                 // rows per tile (MMA M)
constexpr int kKC = 32;                  // K per stage
constexpr int kGroups = 2;               // converter/epilogue warp groups (4 warps each, one per TMEM lane quarter)
constexpr int kRawStages = 2;            // chunk j -> raw stage j % 2 (= its group)
constexpr int kPiecesA = 2;              // FP16 pieces of alpha C_p (2 x 11 bits)
constexpr int kAStages = 2;              // chunk j -> A stage j % 2 (= its group)
constexpr int kThreadsTc = 128 + 128 * kGroups;
constexpr int kRawBytes = kBM * kKC * 4;          // one FP32 raw tile (C or C_Q): 16 KB
constexpr int kAPieceBytes = kBM * kKC * 2;       // one FP16 A piece: 8 KB

// PB: FP16 pieces of beta M (3: five products per K step; 2: four, for a well-conditioned
// update); the B ring holds the same bytes either way: 2 stages of 3 pieces or 3 of 2
template <int NT, int PB>
struct TcLayout {
  static constexpr int BStages = PB == 3 ? 2 : 3;
  static constexpr int BPiece = NT * kKC * 2;                        // one FP16 B piece per stage
  static constexpr int RawOff = 0;
  static constexpr int AOff = RawOff + kRawStages * 2 * kRawBytes;
  static constexpr int BOff = AOff + kAStages * kPiecesA * kAPieceBytes;
  static constexpr int VecOff = BOff + BStages * PB * BPiece;        // a (NT floats), r (NT floats)
  static constexpr int RedOff = VecOff + 2 * NT * 4;                 // group-0 partials: 128 x {rd hi, rd lo, x hi, x lo, max}
  static constexpr int BarOff = RedOff + 128 * 5 * 4;
  static constexpr int NumBars = 2 * kRawStages + 2 * kAStages + 2 * BStages + 5;
  static constexpr int Total = BarOff + NumBars * 8 + 16;
  static constexpr int Smem = Total + 1024;                          // slack for 1024-B alignment
};

using namespace tc;

__device__ __forceinline__ int pow2_exp(float bound) {
  // e with bound < 2^e (bound > 0)
  int e;
  frexpf(bound, &e);
  return e;
}

// a + b = s + err exactly (Knuth's two-sum), in FP32
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
  return s;
}

// GROUPED: the tiles of several filters (args.items, in the order of their tile0) in one
// launch; every role walks the same flat tile order and finds a tile's filter with a cursor.
// A tile of a filter whose step was rejected is skipped by every role alike.
template <int NT, bool GROUPED, int PB>
__global__ void __launch_bounds__(kThreadsTc, 1) sweep_tc_kernel(const __grid_constant__ CUtensorMap tmC,
                                                          const __grid_constant__ CUtensorMap tmCQ,
                                                          const __grid_constant__ CUtensorMap tmCst, TcArgs args) {
  using Lay = TcLayout<NT, PB>;
  constexpr int kBStages = Lay::BStages;
  constexpr int NK = NT / kKC;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (!GROUPED) {
    if (*args.flag) return;  // a rejected step is a no-op
  }
  const TcItem* its = args.items;
  // the item of flat tile t (t never decreases along a role's cursor)
  auto item_of = [&](int64_t t, int& s) {
    if constexpr (GROUPED) {
      while (s + 1 < args.nitems && t >= its[s + 1].tile0) ++s;
    }
  };
  auto local_tile = [&](int64_t t, int s) -> int64_t {
    if constexpr (GROUPED) return t - its[s].tile0;
    return t;
  };
  auto skip = [&](int s) -> bool {
    if constexpr (GROUPED) return *its[s].flag != 0;
    return false;
  };

  float* s_a = reinterpret_cast<float*>(smem + Lay::VecOff);
  float* s_r = s_a + NT;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::BarOff);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + Lay::BarOff + Lay::NumBars * 8);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  const uint32_t bar0 = smem_u32(bars);
  auto raw_full = [&](int s) { return bar0 + 8u * s; };
  auto raw_empty = [&](int s) { return bar0 + 8u * (kRawStages + s); };
  auto a_full = [&](int s) { return bar0 + 8u * (2 * kRawStages + s); };
  auto a_empty = [&](int s) { return bar0 + 8u * (2 * kRawStages + kAStages + s); };
  auto b_full = [&](int s) { return bar0 + 8u * (2 * kRawStages + 2 * kAStages + s); };
  auto b_empty = [&](int s) { return bar0 + 8u * (2 * kRawStages + 2 * kAStages + kBStages + s); };
  const uint32_t acc_full = bar0 + 8u * (2 * kRawStages + 2 * kAStages + 2 * kBStages);
  const uint32_t acc_empty = acc_full + 8u;
  const uint32_t drain = acc_full + 16u;
  const uint32_t red_full = acc_full + 24u;   // group 1's row partials written (4 warp arrivals)
  const uint32_t red_empty = acc_full + 32u;  // group 0 has read them (4 warp arrivals)

  if constexpr (!GROUPED) {
    for (int j = threadIdx.x; j < NT; j += blockDim.x) {
      s_a[j] = j < args.n ? (float)args.a[j] : 0.f;
      s_r[j] = j < args.n ? (float)args.rd[j] : 0.f;
    }
  }
  int* s_err = reinterpret_cast<int*>(s_tmem + 2);  // grouped: a wait timed out in this CTA
  if (threadIdx.x == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(raw_full(s), 1);
      mbar_init(raw_empty(s), 4);  // the 4 warps of the consuming group
    }
    for (int s = 0; s < kAStages; ++s) {
      mbar_init(a_full(s), 4);
      mbar_init(a_empty(s), 1);
    }
    for (int s = 0; s < kBStages; ++s) {
      mbar_init(b_full(s), 1);
      mbar_init(b_empty(s), 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 4 * kGroups);
    mbar_init(drain, 1);
    mbar_init(red_full, 4);
    mbar_init(red_empty, 4);
    *s_abort = 0;
    *s_err = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(s_tmem), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  const int64_t ntiles = GROUPED ? args.ntiles_total : (args.m + kBM - 1) / kBM;
  const int beta_exp0 = GROUPED ? 0 : *args.beta_exp;
  const unsigned long long wlim = args.wait_ns;
  int* const errp = GROUPED ? s_err : args.err;  // a grouped launch reports to every item at the end

  if (warp == 0) {
    // ---------------- producer: raw tiles ----------------
    if (lane == 0) {
      int64_t j = 0;
      int is = 0, fenced = -1;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        item_of(tile, is);
        if (skip(is)) continue;
        if constexpr (GROUPED) {
          if (is != fenced) {
            tensormap_acquire(&its[is].mapC);
            tensormap_acquire(&its[is].mapCQ);
            fenced = is;
          }
        }
        const CUtensorMap* mC = GROUPED ? &its[is].mapC : &tmC;
        const CUtensorMap* mCQ = GROUPED ? &its[is].mapCQ : &tmCQ;
        const int row0 = (int)(local_tile(tile, is) * kBM);
        for (int kc = 0; kc < NK && ok; ++kc, ++j) {
          const int rs = (int)(j % kRawStages);
          const uint32_t rph = (uint32_t)((j / kRawStages) & 1);
          ok = mbar_wait(raw_empty(rs), rph ^ 1u, errp, s_abort, wlim);
          if (!ok) break;
          const uint32_t rbase = smem_u32(smem + Lay::RawOff + rs * 2 * kRawBytes);
          mbar_expect_tx(raw_full(rs), 2 * kRawBytes);
          tma_load_2d(rbase, mC, kc * kKC, row0, raw_full(rs));
          tma_load_2d(rbase + kRawBytes, mCQ, kc * kKC, row0, raw_full(rs));
        }
      }
      if (!ok) *s_abort = 1;
      // every copy this thread issued (j of them) has landed before the CTA may exit
      drain_ring(raw_full(0), kRawStages, j, errp);
    }
  } else if (warp == 2) {
    // ---------------- producer: B images (its own warp, so the raw ring runs ahead of
    // the MMAs instead of in step with the B ring) ----------------
    if (lane == 0) {
      int64_t j = 0;
      int is = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        item_of(tile, is);
        if (skip(is)) continue;
        const __half* bimg = GROUPED ? its[is].bimg : args.bimg;
        for (int kc = 0; kc < NK && ok; ++kc, ++j) {
          const int bs = (int)(j % kBStages);
          ok = mbar_wait(b_empty(bs), (uint32_t)(((j / kBStages) & 1) ^ 1), errp, s_abort, wlim);
          if (!ok) break;
          const uint32_t bbase = smem_u32(smem + Lay::BOff + bs * PB * Lay::BPiece);
          mbar_expect_tx(b_full(bs), PB * Lay::BPiece);
          for (int pc = 0; pc < PB; ++pc)
            bulk_load(bbase + pc * Lay::BPiece, bimg + ((size_t)pc * NK + kc) * (Lay::BPiece / 2), Lay::BPiece,
                      b_full(bs));
        }
      }
      if (!ok) *s_abort = 1;
      drain_ring(b_full(0), kBStages, j, errp);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0, eph = 0;
      int is = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        item_of(tile, is);
        if (skip(is)) continue;
        ok = mbar_wait(acc_empty, eph ^ 1u, errp, s_abort, wlim);
        eph ^= 1u;
        if (!ok) break;
        tc_fence_after();
        for (int kc = 0; kc < NK && ok; ++kc) {
          ok = mbar_wait(a_full(as), aph, errp, s_abort, wlim) && mbar_wait(b_full(bs), bph, errp, s_abort, wlim);
          if (!ok) break;
          tc_fence_after();
          const uint32_t abase = smem_u32(smem + Lay::AOff + as * kPiecesA * kAPieceBytes);
          const uint32_t bbase = smem_u32(smem + Lay::BOff + bs * PB * Lay::BPiece);
          for (int ks = 0; ks < kKC / 16; ++ks) {
            const uint64_t a1 = smem_desc(abase + ks * 256, 128, 512);
            const uint64_t a2 = smem_desc(abase + kAPieceBytes + ks * 256, 128, 512);
            const uint64_t b1 = smem_desc(bbase + ks * 256, 128, 512);
            const uint64_t b2 = smem_desc(bbase + Lay::BPiece + ks * 256, 128, 512);
            const uint64_t b3 = PB == 3 ? smem_desc(bbase + 2 * Lay::BPiece + ks * 256, 128, 512) : 0;
            // smallest terms first; the first product of a tile overwrites the accumulator
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            tc_mma_f16(tmem, a2, b2, idesc, acc);
            if constexpr (PB == 3) tc_mma_f16(tmem, a1, b3, idesc, 1u);
            tc_mma_f16(tmem, a2, b1, idesc, 1u);
            tc_mma_f16(tmem, a1, b2, idesc, 1u);
            tc_mma_f16(tmem, a1, b1, idesc, 1u);
          }
          tc_commit(a_empty(as));
          tc_commit(b_empty(bs));
          if (++as == kAStages) {
            as = 0;
            aph ^= 1u;
          }
          if (++bs == kBStages) {
            bs = 0;
            bph ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(acc_full);
      }
      // all issued MMAs complete before TMEM is released
      tc_commit(drain);
      mbar_wait_drain(drain, 0, errp);
      if (!ok) *s_abort = 1;
    }
  } else if (warp >= 4) {
    // ---------------- converter + epilogue (thread = row) ----------------
    // group g converts the K-chunks kc with kc % 2 == g and writes the output column
    // chunks [g NK/2, (g+1) NK/2); the two groups' row partials meet in shared memory.
    const int g = (warp - 4) / 4;
    const int q = warp & 3;  // TMEM lane quarter of this warp
    const int r = q * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    float* red = reinterpret_cast<float*>(smem + Lay::RedOff);
    uint32_t fph = 0, redph = 0;
    // group 1: the row results of the previous tile, finished during the next tile
    bool pend = false, p_valid = false;
    int64_t p_row = 0;
    int p_item = 0;
    float p_rs = 0.f, p_rc = 0.f, p_xs = 0.f, p_xc = 0.f, p_rmax = 0.f;
    double p_v = 0.0, p_x = 0.0;
    uint32_t p_ph = 0;
    // combine both groups' partials of the pending rows (group 0's come through shared memory)
    auto finish_rows = [&]() -> bool {
      if (!__all_sync(0xffffffffu, mbar_wait(red_full, p_ph, errp, s_abort, wlim))) return false;
      if (p_valid) {
        // the two groups' compensated sums are combined in FP32 (an exact two-sum of the
        // leading parts, the compensations added to the error term) and only the result
        // goes through FP64: an FP64 instruction holds its SM sub-partition for ~64 cycles
        float rd_lo, xi_lo;
        const float rd_hi = two_sum(p_rs, red[r * 5 + 0], rd_lo);
        const float xi_hi = two_sum(p_xs, red[r * 5 + 2], xi_lo);
        rd_lo -= p_rc + red[r * 5 + 1];
        xi_lo -= p_xc + red[r * 5 + 3];
        double* var = GROUPED ? its[p_item].var : args.var;
        double* xv = GROUPED ? its[p_item].x : args.x;
        float* cmax = GROUPED ? its[p_item].cmax : args.cmax;
        const double theta = GROUPED ? its[p_item].theta : args.theta;
        var[p_row] = (p_v + theta) - ((double)rd_hi + (double)rd_lo);
        xv[p_row] = p_x + ((double)xi_hi + (double)xi_lo);
        cmax[p_row] = fmaxf(p_rmax, red[r * 5 + 4]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(red_empty);
      pend = false;
      return true;
    };
    int64_t j = g;  // global chunk counter of this group (stride kGroups)
    bool ok = true;
    // row scalars of the next tile are loaded one tile ahead (hides their latency)
    float nb_c = 0.f, nb_q = 0.f;
    double nv = 0.0, nx = 0.0;
    if constexpr (!GROUPED) {
      const int64_t row = (int64_t)blockIdx.x * kBM + r;
      if (blockIdx.x < ntiles && row < args.m) {
        nb_c = args.cmax[row];
        nb_q = args.cqmax[row];
        if (g == 1) {
          nv = args.var[row];
          nx = args.x[row];
        }
      }
    }
    int is = 0, fenced = -1;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      item_of(tile, is);
      if (skip(is)) continue;
      if constexpr (GROUPED) {  // lane 0 issues the tile's stores through the item's map
        if (is != fenced) {
          if (lane == 0) tensormap_acquire(&its[is].mapCst);
          fenced = is;
        }
      }
      const int64_t row = local_tile(tile, is) * kBM + r;  // the row within its filter
      const int64_t mrows = GROUPED ? its[is].m : args.m;
      const bool valid = row < mrows;
      if constexpr (GROUPED) {  // a grouped launch reads the tile's row scalars when it starts it
        nb_c = valid ? its[is].cmax[row] : 0.f;
        nb_q = valid ? its[is].cqmax[row] : 0.f;
        nv = (g == 1 && valid) ? its[is].var[row] : 0.0;
        nx = (g == 1 && valid) ? its[is].x[row] : 0.0;
      }
      const float bound = valid ? nb_c + nb_q : 0.f;
      const double cur_v = nv, cur_x = nx;
      if constexpr (!GROUPED) {
        const int64_t nrow = (tile + gridDim.x) * kBM + r;
        if (tile + gridDim.x < ntiles && nrow < args.m) {
          nb_c = args.cmax[nrow];
          nb_q = args.cqmax[nrow];
          if (g == 1) {
            nv = args.var[nrow];
            nx = args.x[nrow];
          }
        }
      }
      const int ea = bound > 0.f ? max(-100, min(100, pow2_exp(bound))) : 0;
      const float alpha = ldexpf(1.f, 14 - ea);
      float xs = 0.f, xc = 0.f;
      for (int kc = g; kc < NK; kc += kGroups, j += kGroups) {
        const int rs = (int)(j % kRawStages);
        const uint32_t rph = (uint32_t)((j / kRawStages) & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(raw_full(rs), rph, errp, s_abort, wlim));
        if (!ok) break;
        const unsigned char* rc = smem + Lay::RawOff + rs * 2 * kRawBytes;
        float cp[kKC];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int phys = c ^ (r & 7);  // 128B swizzle of the TMA tile
          const float4 u = *reinterpret_cast<const float4*>(rc + r * 128 + phys * 16);
          const float4 v = *reinterpret_cast<const float4*>(rc + kRawBytes + r * 128 + phys * 16);
          cp[4 * c + 0] = u.x + v.x;
          cp[4 * c + 1] = u.y + v.y;
          cp[4 * c + 2] = u.z + v.z;
          cp[4 * c + 3] = u.w + v.w;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(raw_empty(rs));
        // x increment: chunk partial by FMA, chunks combined with compensation
        {
          float part = 0.f;
          // a grouped launch reads the item's FP32 copy of a (one address for all lanes)
          const float4* a4 = reinterpret_cast<const float4*>((GROUPED ? its[is].a32 : s_a) + kc * kKC);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 av = a4[c];
            part = fmaf(cp[4 * c + 0], av.x, part);
            part = fmaf(cp[4 * c + 1], av.y, part);
            part = fmaf(cp[4 * c + 2], av.z, part);
            part = fmaf(cp[4 * c + 3], av.w, part);
          }
          const float y = part - xc;
          const float t = xs + y;
          xc = (t - xs) - y;
          xs = t;
        }
        tmem_st32(tq + 256 + kc * kKC, reinterpret_cast<const uint32_t*>(cp));
        const int as = (int)(j % kAStages);
        const uint32_t aph = (uint32_t)((j / kAStages) & 1);
        ok = __all_sync(0xffffffffu, mbar_wait(a_empty(as), aph ^ 1u, errp, s_abort, wlim));
        if (!ok) break;
        if (kc == g) {
          // the A stage held this warp's output staging: its last tile stores have read it
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
        }
        unsigned char* ab = smem + Lay::AOff + as * kPiecesA * kAPieceBytes;
#pragma unroll
        for (int gg = 0; gg < kKC / 8; ++gg) {
          __align__(16) __half2 p1[4], p2[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 sv = make_float2(cp[8 * gg + 2 * u] * alpha, cp[8 * gg + 2 * u + 1] * alpha);
            const __half2 h1 = __float22half2_rn(sv);
            const float2 f1 = __half22float2(h1);
            p1[u] = h1;
            p2[u] = __float22half2_rn(make_float2(sv.x - f1.x, sv.y - f1.y));  // residual exact in FP32
          }
          const uint32_t off = core_off(r, 8 * gg);
          *reinterpret_cast<uint4*>(ab + off) = *reinterpret_cast<const uint4*>(p1);
          *reinterpret_cast<uint4*>(ab + kAPieceBytes + off) = *reinterpret_cast<const uint4*>(p2);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(a_full(as));
        if (pend) {
          ok = finish_rows();
          if (!ok) break;
        }
      }
      if (!ok) break;
      tmem_wait_st();
      // ---- epilogue: output column chunks [0, e0) for group 0, [e0, NK) for group 1 ----
      // (group 0 takes fewer: it converts the chunk the next tile's MMAs start with)
      ok = __all_sync(0xffffffffu, mbar_wait(acc_full, fph, errp, s_abort, wlim));
      fph ^= 1u;
      if (!ok) break;
      tc_fence_after();
      const int beta_exp = GROUPED ? *its[is].beta_exp : beta_exp0;
      const float inv = ldexpf(1.f, ea - 14 - beta_exp);  // 1 / (alpha beta)
      float rs_ = 0.f, rc_ = 0.f, rmax = 0.f;
      // output staging: this warp's 32 rows x 32 columns as two 16-row boxes (2 KB each,
      // 128B-swizzled like the C tensor map) in the bytes its own rows occupy in A pieces
      // 0 and 1 of the group's A stage; no MMA reads that stage during the epilogue, and
      // only this warp writes those bytes (its converter rows), so no other warp waits
      unsigned char* stg = smem + Lay::AOff + g * kPiecesA * kAPieceBytes + (lane >> 4) * kAPieceBytes + q * 2048;
      constexpr int e0 = NK / 4;
      for (int jc = g == 0 ? 0 : e0; jc < (g == 0 ? e0 : NK); ++jc) {
        uint32_t kv[32], cv[32];
        tmem_ld32(tq + jc * kKC, kv);
        tmem_ld32(tq + 256 + jc * kKC, cv);
        tmem_wait_ld();
        float out[32];
        float part = 0.f;
        const float4* r4 = reinterpret_cast<const float4*>((GROUPED ? its[is].rd32 : s_r) + jc * kKC);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 rv = r4[c];
          const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int u = 4 * c + w;
            const float k = __uint_as_float(kv[u]) * inv;
            part = fmaf(k, __uint_as_float(cv[u]), part);
            out[u] = k * rr[w];
            rmax = fmaxf(rmax, fabsf(out[u]));
          }
        }
        const float y = part - rc_;
        const float t = rs_ + y;
        rc_ = (t - rs_) - y;
        rs_ = t;
        const int col0 = jc * kKC;
        if (col0 < (GROUPED ? its[is].ld : args.ld)) {
          // the previous store from this buffer has been read out of shared memory
          if (lane == 0) bulk_wait_read0();
          __syncwarp();
#pragma unroll
          for (int u = 0; u < 8; ++u)
            *reinterpret_cast<float4*>(stg + (lane & 15) * 128 + ((u ^ (lane & 7)) * 16)) =
                make_float4(out[4 * u], out[4 * u + 1], out[4 * u + 2], out[4 * u + 3]);
          fence_proxy_async();
          __syncwarp();
          // rows past m are clipped by the tensor map
          if (lane == 0) {
            unsigned char* s0 = smem + Lay::AOff + g * kPiecesA * kAPieceBytes + q * 2048;
            const CUtensorMap* mst = GROUPED ? &its[is].mapCst : &tmCst;
            const int srow = (int)(local_tile(tile, is) * kBM + q * 32);
            tma_store_2d(mst, smem_u32(s0), col0, srow);
            tma_store_2d(mst, smem_u32(s0 + kAPieceBytes), col0, srow + 16);
            bulk_commit();
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty);
      // combine the two groups' row partials through shared memory (bounded mbarrier handoff);
      // group 1 finishes the rows, so group 0 can start converting the next tile's first
      // chunk (the first the next MMAs need) at once
      if (g == 0) {
        ok = __all_sync(0xffffffffu, mbar_wait(red_empty, redph ^ 1u, errp, s_abort, wlim));
        if (!ok) break;
        red[r * 5 + 0] = rs_;
        red[r * 5 + 1] = rc_;
        red[r * 5 + 2] = xs;
        red[r * 5 + 3] = xc;
        red[r * 5 + 4] = rmax;
        __syncwarp();
        if (lane == 0) mbar_arrive(red_full);
      } else {
        // group 1 finishes these rows later, after converting its first chunk of the next
        // tile: its FP64 work would otherwise hold the SM sub-partitions while group 0
        // converts the chunk the next tile's MMAs wait for
        pend = true;
        p_valid = valid;
        p_row = row;
        p_item = is;
        p_rs = rs_;
        p_rc = rc_;
        p_xs = xs;
        p_xc = xc;
        p_rmax = rmax;
        p_v = cur_v;
        p_x = cur_x;
        p_ph = redph;
      }
      redph ^= 1u;
    }
    if (ok && pend) ok = finish_rows();  // the last tile's rows
    if (!ok) *s_abort = 1;
    tmem_wait_st();  // an abort may leave this warp's C_p stores to TMEM unwaited
    if (lane == 0) bulk_wait0();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, 512);
  }
  if constexpr (GROUPED) {
    // a timed-out wait leaves every filter of the launch in an undefined state
    if (threadIdx.x == 0 && *s_err)
      for (int i = 0; i < args.nitems; ++i) atomicExch(its[i].err, 1);
  }
}

// B images: beta M split into FP16 hi / lo, K-major core-matrix layout per 32-K stage (see pack_b_dyn_kernel)
// max|M| over the n x n block: block b reduces rows b, b + kAbsBlocks, ... into out[b]
__global__ void absmax_kernel(const float* __restrict__ M, int nt, int n, unsigned* __restrict__ out) {
  float mx = 0.f;
  for (int i = blockIdx.x; i < n; i += gridDim.x)
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(M[(int64_t)i * nt + j]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    out[blockIdx.x] = __float_as_uint(fmaxf(red[0], mx));
  }
}

// beta exponent from the kAbsBlocks partial maxima of |M| (written where pack_b_kernel and the sweep read it)
__global__ void beta_kernel(const unsigned* __restrict__ mx, int* __restrict__ beta_exp) {
  float v = __uint_as_float(mx[threadIdx.x]);
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ float red[kAbsBlocks / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < kAbsBlocks / 32; ++w) v = fmaxf(v, red[w]);
    int e = 0;
    if (v > 0.f) frexpf(v, &e);
    *beta_exp = 14 - e;
  }
}

template <int NT>
__global__ void pack_b_dyn_kernel(const float* __restrict__ Msw, int nt_src, int n, const int* __restrict__ beta_exp,
                                  __half* __restrict__ img, const double* __restrict__ a,
                                  const double* __restrict__ rd, float* __restrict__ vec32,
                                  const int* __restrict__ flag, int pieces) {
  if (*flag) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)NT * NT) return;
  if (t < NT) {  // the FP32 vectors a grouped sweep reads (once per step, not per tile)
    vec32[t] = t < n ? (float)a[t] : 0.f;
    vec32[NT + t] = t < n ? (float)rd[t] : 0.f;
  }
  const int nidx = (int)(t / NT), k = (int)(t % NT);
  const float v = (nidx < n && k < n) ? Msw[(int64_t)nidx * nt_src + k] * ldexpf(1.f, *beta_exp) : 0.f;
  const __half h1 = __float2half_rn(v);
  const float r1 = v - __half2float(h1);  // exact in FP32
  const __half h2 = __float2half_rn(r1);
  const int kc = k / kKC, kk = k % kKC;
  const size_t chunk = (size_t)NT * kKC;                   // halves per piece per chunk
  const size_t off = (size_t)kc * chunk + core_off(nidx, kk) / 2;
  const size_t piece = (size_t)(NT / kKC) * chunk;         // halves per piece (all chunks)
  img[off] = h1;
  img[piece + off] = h2;
  if (pieces == 3) img[2 * piece + off] = __float2half_rn(r1 - __half2float(h2));
}

// per-row max |value| of an m x ld FP32 matrix (row scale bounds)
__global__ void rowmax_kernel(const float* __restrict__ A, int64_t m, int ld, float* __restrict__ out) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  float mx = 0.f;
  for (int j = lane; j < ld; j += 32) mx = fmaxf(mx, fabsf(A[row * ld + j]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) out[row] = mx;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

Status encode_map(CUtensorMap* map, const float* base, int64_t m, int ld, int box_rows = kBM) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    HIKF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) return make_status(HIKF_ECUDA, "cuTensorMapEncodeTiled unavailable");
    fn = (EncodeTiledFn)p;
  }
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return make_status(HIKF_ECUDA, "cuTensorMapEncodeTiled failed");
  return Status::Ok();
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// One instantiation of the sweep: its entry point and dynamic shared memory
struct TcKernel {
  const void* fn;
  int smem;
};
template <int NT, bool G, int PB>
TcKernel tc_kernel_of() {
  return {(const void*)sweep_tc_kernel<NT, G, PB>, TcLayout<NT, PB>::Smem};
}
TcKernel tc_kernel(int nt, bool grouped, int products) {
  const int pb = products == 4 ? 2 : 3;
  if (nt == 128) {
    if (grouped) return pb == 2 ? tc_kernel_of<128, true, 2>() : tc_kernel_of<128, true, 3>();
    return pb == 2 ? tc_kernel_of<128, false, 2>() : tc_kernel_of<128, false, 3>();
  }
  if (grouped) return pb == 2 ? tc_kernel_of<256, true, 2>() : tc_kernel_of<256, true, 3>();
  return pb == 2 ? tc_kernel_of<256, false, 2>() : tc_kernel_of<256, false, 3>();
}

Status tc_setup(TcState& tc, const float* C, const float* CQ, int64_t m, int ld, int n) {
  if (ld > 256) return make_status(HIKF_EINVAL, "MIXED precision supports n <= 256");
  tc.nt = ld <= 128 ? 128 : 256;
  HIKF_TRY(encode_map(&tc.mapC, C, m, ld));
  HIKF_TRY(encode_map(&tc.mapCst, C, m, ld, 16));
  HIKF_TRY(encode_map(&tc.mapCQ, CQ, m, ld));
  for (int grouped = 0; grouped < 2; ++grouped)
    for (int products = 4; products <= 5; ++products) {
      const TcKernel k = tc_kernel(tc.nt, grouped != 0, products);
      HIKF_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem));
    }
  return Status::Ok();
}

// Launch one instantiation (the arguments as the kernel's parameter list)
Status tc_launch(int nt, bool grouped, int products, int grid, const CUtensorMap& mC, const CUtensorMap& mCQ,
                 const CUtensorMap& mCst, const TcArgs& args, cudaStream_t s) {
  const TcKernel k = tc_kernel(nt, grouped, products);
  void* params[] = {(void*)&mC, (void*)&mCQ, (void*)&mCst, (void*)&args};
  HIKF_CUDA(cudaLaunchKernel(k.fn, dim3(grid), dim3(kThreadsTc), params, (size_t)k.smem, s));
  return Status::Ok();
}

Status tc_init_rows(const TcState& tc, const float* C, const float* CQ, int64_t m, int ld, cudaStream_t s) {
  rowmax_kernel<<<nblk(m, 8), 256, 0, s>>>(C, m, ld, tc.cmax);
  HIKF_LAUNCH_CHECK("rowmax");
  rowmax_kernel<<<nblk(m, 8), 256, 0, s>>>(CQ, m, ld, tc.cqmax);
  HIKF_LAUNCH_CHECK("rowmax");
  return Status::Ok();
}

Status tc_pack(const TcState& tc, const float* Msw, int nt_src, int n, const double* a, const double* rd,
               const int* flag, cudaStream_t s) {
  absmax_kernel<<<kAbsBlocks, 256, 0, s>>>(Msw, nt_src, n, tc.mmax);
  HIKF_LAUNCH_CHECK("absmax");
  beta_kernel<<<1, kAbsBlocks, 0, s>>>(tc.mmax, tc.beta_exp);
  HIKF_LAUNCH_CHECK("beta");
  const int64_t cnt = (int64_t)tc.nt * tc.nt;
  if (tc.nt == 128)
    pack_b_dyn_kernel<128><<<nblk(cnt, 256), 256, 0, s>>>(Msw, nt_src, n, tc.beta_exp, tc.bimg, a, rd, tc.vec32,
                                                          flag, tc.products == 4 ? 2 : 3);
  else
    pack_b_dyn_kernel<256><<<nblk(cnt, 256), 256, 0, s>>>(Msw, nt_src, n, tc.beta_exp, tc.bimg, a, rd, tc.vec32,
                                                          flag, tc.products == 4 ? 2 : 3);
  HIKF_LAUNCH_CHECK("pack_b");
  return Status::Ok();
}

namespace {
unsigned long long g_wait_ns = 0;  // 0: the default limit
}  // namespace

void tc_set_wait_limit(unsigned long long ns) { g_wait_ns = ns; }

Status tc_sweep(const TcState& tc, TcArgs args, int sms, cudaStream_t s) {
  args.wait_ns = g_wait_ns ? g_wait_ns : tc::kWaitNs;
  const int64_t ntiles = (args.m + kBM - 1) / kBM;
  const int grid = (int)std::min<int64_t>(ntiles, sms);
  args.bimg = tc.bimg;
  args.cmax = tc.cmax;
  args.cqmax = tc.cqmax;
  args.products = tc.products;
  return tc_launch(tc.nt, false, tc.products, grid, tc.mapC, tc.mapCQ, tc.mapCst, args, s);
}

int tc_nt(const TcState& tc) { return tc.nt; }
int64_t tc_tiles(int64_t m) { return (m + kBM - 1) / kBM; }

void tc_item(const TcState& tc, const TcArgs& args, TcItem* it) {
  it->mapC = tc.mapC;
  it->mapCQ = tc.mapCQ;
  it->mapCst = tc.mapCst;
  it->m = args.m;
  it->n = args.n;
  it->ld = args.ld;
  it->theta = args.theta;
  it->a32 = tc.vec32;
  it->rd32 = tc.vec32 + tc.nt;
  it->x = args.x;
  it->var = args.var;
  it->flag = args.flag;
  it->err = args.err;
  it->beta_exp = args.beta_exp;
  it->bimg = tc.bimg;
  it->cmax = tc.cmax;
  it->cqmax = tc.cqmax;
  it->tile0 = 0;
  it->products = tc.products;
}

Status tc_sweep_grouped(int nt, int products, const TcItem* items, int count, int64_t ntiles_total, int sms,
                        cudaStream_t s) {
  if (count < 1 || ntiles_total < 1) return Status::Ok();
  TcArgs args;
  args.items = items;
  args.nitems = count;
  args.ntiles_total = ntiles_total;
  args.wait_ns = g_wait_ns ? g_wait_ns : tc::kWaitNs;
  const int grid = (int)std::min<int64_t>(ntiles_total, sms);
  // the per-launch tensor-map parameters are unused by the grouped kernel (each item has its own)
  CUtensorMap unused;
  memset(&unused, 0, sizeof(unused));
  args.products = products;
  return tc_launch(nt, true, products, grid, unused, unused, unused, args, s);
}

}  // namespace hikf
