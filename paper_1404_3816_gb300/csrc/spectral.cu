// Spectral form of the n x n chain of the measurement update.
//
// With stationary H, Q, R (Sec. 2.2) the random-walk filter's innovation
// covariance obeys S_{t+1} = H C_Q + 2R - R S_t^{-1} R (because
// H C_{t+1|t} = H C_{t|t} + H C_Q and H C_{t|t} = R - R S_t^{-1} R). Scaling by
// D = R^{-1/2} gives  S~_{t+1} = B~ + 2I - S~_t^{-1}  with B~ = D sym(H C_Q) D.
// When P_0 = c Q (c >= 0, which includes P_0 = 0), S~_1 = (1 + c) B~ + I, so every
// S~_t is a function of B~: with B~ = V diag(lambda) V^T,
//     s_1 = (1 + c) lambda + 1,   s_{t+1} = lambda + 2 - 1 / s_t     (per eigenvalue)
//     M_t = S_t^{-1} = W diag(1 / s_t) W^T,   W = D V.
// One FP64 eigendecomposition at create replaces a Cholesky factorisation per
// step, whose FP64 cost and conditioning (cond(S) ~ 1e8 and more) would
// otherwise dominate the update.
//
// Eigensolver (FP64): parallel cyclic Jacobi (Golub & Van Loan, Sec. 8.5) on the full
// matrix. A sweep is N - 1 rounds of a round-robin ordering; a round rotates N / 2
// disjoint index pairs at once, so every 2 x 2 block of A and every pair of columns of V
// is updated independently. On this part an FP64 instruction occupies its SM
// sub-partition for 64 cycles whatever the number of active lanes, and a dependent
// divide or square root takes several hundred cycles. So the work is laid out to keep
// every lane of every sub-partition busy across all SMs, and serial FP64 chains are kept
// to one rotation per round. A QR algorithm on the tridiagonal form would chase its
// rotations one after another on a single thread.
#include <math.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "spectral.cuh"

namespace hikf {

namespace {

__device__ __forceinline__ unsigned long long tc_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over a cooperative launch (every CTA resident): a counter with a bounded
// wait (2 s), after which the CTA sets *err and *s_abort, and the caller leaves.
__device__ bool grid_barrier(unsigned* bar, unsigned& gen, int* err, volatile int* s_abort) {
  // arrive with a release add, wait with acquire loads: the CTA's writes (ordered before
  // thread 0 by the CTA barrier) are visible to every CTA that passes
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (gen + 1u) * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const unsigned long long t0 = tc_now_ns();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (tc_now_ns() - t0 > 2000000000ull) {
        atomicExch(err, 1);
        *s_abort = 1;
        break;
      }
    }
  }
  __syncthreads();
  ++gen;
  return *s_abort == 0;
}

// ---- parallel cyclic Jacobi ------------------------------------------------------------
// Round-robin ordering over N (even) indices: in round r, index N - 1 meets r, and every
// other index a meets (2r - a) mod (N - 1); pair 0 is (r, N - 1), pair k >= 1 is
// ((r + k), (r - k)) mod (N - 1). Over N - 1 rounds every pair meets once.
__device__ __forceinline__ int rr_mod(int a, int m) {
  a %= m;
  return a < 0 ? a + m : a;
}
__device__ __forceinline__ void rr_pair(int r, int k, int N, int& p, int& q) {
  if (k == 0) {
    p = r;
    q = N - 1;
  } else {
    p = rr_mod(r + k, N - 1);
    q = rr_mod(r - k, N - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}
// One Jacobi rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) with (J^T A J)_pq = 0:
// t = tan(phi) is the smaller root of t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 a_pq).
// With d = a_qq - a_pp, b = 2 a_pq, h = hypot(d, b), u = h + |d| this is t = sign(d) b / u,
// and c = u / sqrt(2 h u), s = sign(d) b / sqrt(2 h u) (c^2 + s^2 = (u^2 + b^2) / (2 h u) = 1),
// t = s / c = 2 h sign(d) b / (2 h u): two reciprocal square roots and no division, whose
// FP64 latency (~650 cycles on this part) would sit on every round's critical path. A pair
// whose off-diagonal entry is negligible (|a_pq| <= eps sqrt(|a_pp a_qq|), or below the
// absolute floor) is not rotated: t = 0.
__device__ __forceinline__ bool jacobi_rotation(double app, double aqq, double apq, double floor_abs, double& c,
                                                double& s, double& t) {
  c = 1.0;
  s = 0.0;
  t = 0.0;
  const double aa = fabs(apq), pa = fabs(app), qa = fabs(aqq);
  if (aa <= floor_abs) return false;
  if (pa < 1e150 && qa < 1e150 && aa > 1e-150) {  // squared: no square roots on the chain
    if (aa * aa <= 4.930380657631324e-32 * pa * qa) return false;
  } else if (aa <= 2.220446049250313e-16 * sqrt(pa) * sqrt(qa)) {
    return false;
  }
  const double d = aqq - app, b = 2.0 * apq;
  const double sb = d >= 0.0 ? b : -b;
  const double h2 = fma(d, d, b * b);
  if (h2 > 1e-290 && h2 < 1e290) {
    const double h = h2 * rsqrt(h2);
    const double u = h + fabs(d);
    const double r2 = rsqrt(2.0 * h * u);
    c = u * r2;
    s = sb * r2;
    t = 2.0 * h * s * r2;
  } else {
    const double h = hypot(d, b);
    t = sb / (fabs(d) + h);
    c = 1.0 / sqrt(fma(t, t, 1.0));
    s = t * c;
  }
  return true;
}

constexpr int kJacThreads = 256;

// Per index i, the effect of one round: the rotation of i's pair acts on rows (and on
// columns) as new_i = al_i old_i + be_i old_j with j = jp_i, its partner; td_i gives the
// rotated diagonal entry a_ii + td_i a_ij, and on_i whether the pair was rotated (its
// off-diagonal entry is then exactly zero).
struct JacRound {
  int jp[kMaxN];
  int on[kMaxN];
  double al[kMaxN], be[kMaxN], td[kMaxN];
};

__device__ __forceinline__ void jac_record(JacRound& R, int p, int q, bool on, double c, double s, double t) {
  R.jp[p] = q;
  R.jp[q] = p;
  R.on[p] = R.on[q] = on ? 1 : 0;
  R.al[p] = R.al[q] = c;
  R.be[p] = -s;  // new_p = c old_p - s old_q
  R.be[q] = s;   // new_q = s old_p + c old_q
  R.td[p] = -t;  // a_pp - t a_pq
  R.td[q] = t;   // a_qq + t a_pq
}

// Entry (x, y) of A after one round R, from the entries of A before it.
__device__ __forceinline__ double jac_after(const double* __restrict__ A, int N, const JacRound& R, int x, int y) {
  const int jx = R.jp[x];
  if (y == x) return fma(R.td[x], A[(int64_t)x * N + jx], A[(int64_t)x * N + x]);
  if (y == jx) return R.on[x] ? 0.0 : A[(int64_t)x * N + y];
  const int jy = R.jp[y];
  const double u = fma(R.be[y], A[(int64_t)x * N + jy], R.al[y] * A[(int64_t)x * N + y]);
  const double w = fma(R.be[y], A[(int64_t)jx * N + jy], R.al[y] * A[(int64_t)jx * N + y]);
  return fma(R.be[x], w, R.al[x] * u);
}

// A (N x N, row-major, symmetric) -> diag(lambda); VT (N x N) -> V^T (row j = eigenvector
// j). A and VT are parity double buffers (2 x N x N each; the input in parity 0): a step
// reads one parity and writes every entry of the other, so a CTA still reading never sees
// an entry change under it. One step applies two consecutive rounds of the cyclic order
// (round-robin pairing, every pair meeting once per N - 1 rounds) behind one grid barrier:
// every CTA forms the first round's rotations from A, then the second round's from the
// entries that the first round leaves on that round's pairs (each a combination of at most
// four entries of A), and the update writes A after both rounds as J2^T (J1^T A J1) J2 in
// blocks of the second round's pairs (each block's four entries from a 4 x 4 set of A).
// Every CTA forms the same rotations and the same decisions. Tasks: block row i of the
// second round's pairs (blocks j >= i, each with its mirror) or its column pair k of V.
// The iteration ends after N - 1 consecutive rounds without a rotation (no entry left
// above the thresholds) or max_sweeps x (N - 1) rounds. out[0] = 1 when it did not
// converge, out[1] = sweeps run (rounds / (N - 1), rounded up), out[4] = the parity that
// holds the result.
__global__ void __launch_bounds__(kJacThreads) eig_jacobi_kernel(double* __restrict__ A, double* __restrict__ VT,
                                                                 int N, int max_sweeps, unsigned* bar, int* err,
                                                                 int* out) {
  __shared__ JacRound R1;
  __shared__ int sp2[kMaxN / 2], sq2[kMaxN / 2], son2[kMaxN / 2];
  __shared__ double sc2[kMaxN / 2], ss2[kMaxN / 2], st2[kMaxN / 2];
  __shared__ double sapp[kMaxN / 2], saqq[kMaxN / 2], sapq[kMaxN / 2];
  __shared__ int s_rot1, s_rot2;
  __shared__ volatile int s_abort;
  __shared__ double s_dmax;
  const int P = N / 2;
  const int64_t NN = (int64_t)N * N;
  const int tid = threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid, gthreads = (int64_t)gridDim.x * blockDim.x;
  unsigned gen = 0;
  if (tid == 0) s_abort = 0;
  for (int64_t u = gtid; u < NN; u += gthreads) VT[u] = (u / N == u % N) ? 1.0 : 0.0;
  if (!grid_barrier(bar, gen, err, &s_abort)) return;
  // absolute floor for a negligible off-diagonal entry: eps max|a_ii| / N, so the entries
  // left out add up (Frobenius) to at most eps max|a_ii|, the backward error of any FP64
  // eigensolver. It ends the iteration on graded spectra (a smooth kernel's), where the
  // entries coupling the smallest eigenvalues carry rounding from rotations with the
  // largest ones and never fall below eps relative to their own diagonal.
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < N; ++i) m = fmax(m, fabs(A[(int64_t)i * N + i]));
    s_dmax = m;
  }
  __syncthreads();
  const double floor_abs = 2.220446049250313e-16 * s_dmax / N;
  const int64_t cycle = N - 1, max_rounds = (int64_t)max_sweeps * cycle;
  int par = 0;
  int64_t g = 0, quiet = 0;
  while (g < max_rounds && quiet < cycle) {
    const double* Ac = A + par * NN;
    const double* Vc = VT + par * NN;
    double* An = A + (par ^ 1) * NN;
    double* Vn = VT + (par ^ 1) * NN;
    const int r1 = (int)(g % cycle), r2 = (int)((g + 1) % cycle);
    if (tid == 0) {
      s_rot1 = 0;
      s_rot2 = 0;
    }
    __syncthreads();
    // round r1: rotations from A
    for (int k = tid; k < P; k += blockDim.x) {
      int p, q;
      rr_pair(r1, k, N, p, q);
      double c, s_, t;
      const bool on = jacobi_rotation(Ac[(int64_t)p * N + p], Ac[(int64_t)q * N + q], Ac[(int64_t)p * N + q],
                                      floor_abs, c, s_, t);
      if (on) atomicAdd(&s_rot1, 1);
      jac_record(R1, p, q, on, c, s_, t);
    }
    __syncthreads();
    // round r2: rotations from the entries round r1 leaves on r2's pairs
    for (int k = tid; k < P; k += blockDim.x) {
      int p, q;
      rr_pair(r2, k, N, p, q);
      const double app = jac_after(Ac, N, R1, p, p), aqq = jac_after(Ac, N, R1, q, q);
      const double apq = jac_after(Ac, N, R1, p, q);
      double c, s_, t;
      const bool on = jacobi_rotation(app, aqq, apq, floor_abs, c, s_, t);
      if (on) atomicAdd(&s_rot2, 1);
      sp2[k] = p;
      sq2[k] = q;
      son2[k] = on ? 1 : 0;
      sc2[k] = c;
      ss2[k] = s_;
      st2[k] = t;
      sapp[k] = app;
      saqq[k] = aqq;
      sapq[k] = apq;
    }
    __syncthreads();
    for (int task = blockIdx.x; task < 2 * P; task += gridDim.x) {
      if (task < P) {
        const int i = task, p = sp2[i], q = sq2[i];
        for (int j = i + tid; j < P; j += blockDim.x) {
          if (j == i) {  // diagonal block: a_pp - t a_pq, a_qq + t a_pq, a_pq -> 0
            double app = sapp[i], aqq = saqq[i], apq = sapq[i];
            if (son2[i]) {
              const double t = st2[i];
              app = fma(-t, apq, app);
              aqq = fma(t, apq, aqq);
              apq = 0.0;
            }
            An[(int64_t)p * N + p] = app;
            An[(int64_t)q * N + q] = aqq;
            An[(int64_t)p * N + q] = apq;
            An[(int64_t)q * N + p] = apq;
            continue;
          }
          const int u0 = sp2[j], v0 = sq2[j];
          double x00 = jac_after(Ac, N, R1, p, u0), x01 = jac_after(Ac, N, R1, p, v0);
          double x10 = jac_after(Ac, N, R1, q, u0), x11 = jac_after(Ac, N, R1, q, v0);
          if (son2[i] | son2[j]) {
            const double c1 = sc2[i], s1 = ss2[i], c2 = sc2[j], s2 = ss2[j];
            // rows: J_i^T X
            const double y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
            const double y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
            // columns: Y J_j
            x00 = c2 * y00 - s2 * y01;
            x01 = s2 * y00 + c2 * y01;
            x10 = c2 * y10 - s2 * y11;
            x11 = s2 * y10 + c2 * y11;
          }
          An[(int64_t)p * N + u0] = x00;
          An[(int64_t)p * N + v0] = x01;
          An[(int64_t)q * N + u0] = x10;
          An[(int64_t)q * N + v0] = x11;
          An[(int64_t)u0 * N + p] = x00;
          An[(int64_t)v0 * N + p] = x01;
          An[(int64_t)u0 * N + q] = x10;
          An[(int64_t)v0 * N + q] = x11;
        }
      } else {
        // rows p, q of V^T after both rounds (V <- V J1 J2)
        const int k = task - P, p = sp2[k], q = sq2[k];
        const int jp = R1.jp[p], jq = R1.jp[q];
        const double alp = R1.al[p], bep = R1.be[p], alq = R1.al[q], beq = R1.be[q];
        const double c = sc2[k], s_ = ss2[k];
        const bool on = son2[k] != 0;
        for (int comp = tid; comp < N; comp += blockDim.x) {
          const double a = fma(bep, Vc[(int64_t)jp * N + comp], alp * Vc[(int64_t)p * N + comp]);
          const double b = fma(beq, Vc[(int64_t)jq * N + comp], alq * Vc[(int64_t)q * N + comp]);
          Vn[(int64_t)p * N + comp] = on ? c * a - s_ * b : a;
          Vn[(int64_t)q * N + comp] = on ? s_ * a + c * b : b;
        }
      }
    }
    // the rotation counts were final at the CTA barrier before the update; every thread
    // reads them before the grid barrier, ahead of the next step's reset
    const int n1 = s_rot1, n2 = s_rot2;
    par ^= 1;
    if (!grid_barrier(bar, gen, err, &s_abort)) return;
    quiet = n1 ? 0 : quiet + 1;
    quiet = n2 ? 0 : quiet + 1;
    g += 2;
  }
  if (blockIdx.x == 0 && tid == 0) {
    out[0] = quiet >= cycle ? 0 : 1;
    out[1] = (int)((g + cycle - 1) / cycle);
    out[4] = par;
  }
}

// lambda_j = A_jj, V (n x n, row i = component i) from V^T (N x N), in the parity *par
__global__ void eig_jacobi_out_kernel(const double* __restrict__ A2, const double* __restrict__ VT2, int N, int n,
                                      const int* __restrict__ par, double* __restrict__ lam, double* __restrict__ V) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const double* A = A2 + (int64_t)*par * N * N;
  const double* VT = VT2 + (int64_t)*par * N * N;
  const int i = (int)(t / n), j = (int)(t % n);
  V[t] = VT[(int64_t)j * N + i];
  if (i == 0) lam[j] = A[(int64_t)j * N + j];
}

// B~ = D sym(HCQ) D with D = R^{-1/2}, into an N x N buffer (N >= n) padded with zeros
__global__ void scale_b_kernel(const double* __restrict__ hcq_sym, const double* __restrict__ rd, int n, int N,
                               double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  int i = (int)(t / N), j = (int)(t % N);
  out[t] = (i < n && j < n) ? hcq_sym[(int64_t)i * n + j] / sqrt(rd[i] * rd[j]) : 0.0;
}

// W = D V (FP64 and FP32 copies); s_1 = (1 + c) lambda + 1
__global__ void spec_init_kernel(const double* __restrict__ V, const double* __restrict__ lam,
                                 const double* __restrict__ rd, int n, double c, double* __restrict__ W64,
                                 float* __restrict__ W32, double* __restrict__ s, int* __restrict__ flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)n * n) {
    int i = (int)(t / n);
    double w = V[t] / sqrt(rd[i]);
    W64[t] = w;
    W32[t] = (float)w;
  }
  if (t < n) {
    double sv = (1.0 + c) * lam[t] + 1.0;
    s[t] = sv;
    if (!(sv > 0.0)) atomicOr(flag, 2);
  }
}

// u = (1/s) o (W^T e), one warp per output
__global__ void spec_u_kernel(const double* __restrict__ W64, const double* __restrict__ s,
                              const double* __restrict__ e, int n, double* __restrict__ u,
                              const int* __restrict__ flag) {
  if (*flag) return;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= n) return;
  double acc = 0.0;
  for (int i = lane; i < n; i += 32) acc += W64[(int64_t)i * n + k] * e[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) u[k] = acc / s[k];
}

// a = W u, one warp per output
__global__ void spec_a_kernel(const double* __restrict__ W64, const double* __restrict__ u, int n,
                              double* __restrict__ a, const int* __restrict__ flag) {
  if (*flag) return;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc += W64[(int64_t)i * n + k] * u[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) a[i] = acc;
}

// U = W diag(1/sqrt(s)) split into FP32 hi + lo, so that M = U U^T
__global__ void spec_split_kernel(const double* __restrict__ W64, const double* __restrict__ s, int n,
                                  float* __restrict__ Uhi, float* __restrict__ Ulo, const int* __restrict__ flag) {
  if (*flag) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int k = (int)(t % n);
  double u = W64[t] / sqrt(s[k]);
  float hi = (float)u;
  Uhi[t] = hi;
  Ulo[t] = (float)(u - (double)hi);
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// M = U U^T with U = Uhi + Ulo in compensated (double-float) FP32: the products
// Uhi_ik Uhi_jk are split exactly (FMA) and summed with error-free additions; the
// cross terms are ~2^-24 smaller and summed plainly. 16 x 16 output tiles.
template <typename T>
__global__ void spec_m_dd_kernel(const float* __restrict__ Uhi, const float* __restrict__ Ulo, int n, int nt,
                                 T* __restrict__ Msw, const int* __restrict__ flag) {
  if (*flag) return;
  __shared__ float hi_i[16][33], lo_i[16][33], hi_j[16][33], lo_j[16][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  float ps = 0.f, pc = 0.f;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int t = threadIdx.x; t < 16 * 32; t += 256) {
      int r = t / 32, kk = t % 32, k = k0 + kk;
      bool oi = i0 + r < n && k < n, oj = j0 + r < n && k < n;
      hi_i[r][kk] = oi ? Uhi[(int64_t)(i0 + r) * n + k] : 0.f;
      lo_i[r][kk] = oi ? Ulo[(int64_t)(i0 + r) * n + k] : 0.f;
      hi_j[r][kk] = oj ? Uhi[(int64_t)(j0 + r) * n + k] : 0.f;
      lo_j[r][kk] = oj ? Ulo[(int64_t)(j0 + r) * n + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      const float a = hi_i[ty][kk], b = hi_j[tx][kk];
      const float p = __fmul_rn(a, b);
      const float pe = __fmaf_rn(a, b, -p);
      float s2, e2;
      two_sum_f(ps, p, s2, e2);
      ps = s2;
      pc += e2 + pe + (a * lo_j[tx][kk] + lo_i[ty][kk] * b);
    }
    __syncthreads();
  }
  if (i0 + ty < n && j0 + tx < n) Msw[(int64_t)(i0 + ty) * nt + j0 + tx] = (T)((double)ps + (double)pc);
}

// FP64 operand (FP64 mode): M = W diag(1/s) W^T in FP64, 16 x 16 output tiles
__global__ void spec_m64_kernel(const double* __restrict__ W, const double* __restrict__ s, int n, int nt,
                                double* __restrict__ Msw, const int* __restrict__ flag) {
  if (*flag) return;
  __shared__ double wi[16][33], wj[16][33], g[32];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int t = threadIdx.x; t < 16 * 32; t += 256) {
      int r = t / 32, kk = t % 32, k = k0 + kk;
      wi[r][kk] = (i0 + r < n && k < n) ? W[(int64_t)(i0 + r) * n + k] : 0.0;
      wj[r][kk] = (j0 + r < n && k < n) ? W[(int64_t)(j0 + r) * n + k] : 0.0;
    }
    if (threadIdx.x < 32) g[threadIdx.x] = k0 + threadIdx.x < n ? 1.0 / s[k0 + threadIdx.x] : 0.0;
    __syncthreads();
    for (int kk = 0; kk < 32; ++kk) acc += wi[ty][kk] * g[kk] * wj[tx][kk];
    __syncthreads();
  }
  if (i0 + ty < n && j0 + tx < n) Msw[(int64_t)(i0 + ty) * nt + j0 + tx] = acc;
}

// s <- lambda + 2 - 1/s   (after an applied step)
__global__ void spec_next_kernel(const double* __restrict__ lam, int n, double* __restrict__ s,
                                 int* __restrict__ flag) {
  if (*flag) return;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  s[k] = lam[k] + 2.0 - 1.0 / s[k];
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

Status spectral_setup(SpectralState& sp, const double* hcq_sym, const double* rd, int n, double c, int* flag,
                      cudaStream_t s) {
  const int N = n + (n & 1);  // even; an odd n gets one zero row and column
  const int64_t nn = (int64_t)n * n, NN = (int64_t)N * N;
  constexpr int kMaxSweeps = 60;
  double *A = nullptr, *VT = nullptr, *V = nullptr;
  int* ints = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&A, sizeof(double) * 2 * NN, s));   // two parities
  HIKF_CUDA(hikf::pool_malloc((void**)&VT, sizeof(double) * 2 * NN, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&V, sizeof(double) * nn, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&ints, 8 * sizeof(int), s));  // info, sweeps, barrier, error, parity
  HIKF_CUDA(cudaMemsetAsync(ints, 0, 8 * sizeof(int), s));
  scale_b_kernel<<<nblk(NN, 256), 256, 0, s>>>(hcq_sym, rd, n, N, A);
  HIKF_LAUNCH_CHECK("scale_b");
  {
    // cooperative grid: one CTA per SM, all resident
    int dev = 0, sms = 1, per_sm = 0;
    HIKF_CUDA(cudaGetDevice(&dev));
    HIKF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HIKF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eig_jacobi_kernel, kJacThreads, 0));
    if (per_sm < 1) return make_status(HIKF_ECUDA, "the Jacobi eigensolver cannot be made resident");
    const int grid = std::max(1, std::min(sms, N));  // the 2 x N/2 update tasks of a round over all SMs
    double* Ap = A;
    double* Vp = VT;
    int Np = N, msw = kMaxSweeps;
    unsigned* bp = reinterpret_cast<unsigned*>(ints + 2);
    int* errp = ints + 3;
    int* outp = ints;
    void* args[] = {&Ap, &Vp, &Np, &msw, &bp, &errp, &outp};
    HIKF_CUDA(cudaLaunchCooperativeKernel((const void*)eig_jacobi_kernel, dim3(grid), dim3(kJacThreads), args, 0, s));
    HIKF_LAUNCH_CHECK("eig_jacobi");
  }
  eig_jacobi_out_kernel<<<nblk(nn, 256), 256, 0, s>>>(A, VT, N, n, ints + 4, sp.lam, V);
  HIKF_LAUNCH_CHECK("eig_jacobi_out");
  spec_init_kernel<<<nblk(nn, 256), 256, 0, s>>>(V, sp.lam, rd, n, c, sp.W64, sp.W32, sp.s, flag);
  HIKF_LAUNCH_CHECK("spec_init");
  int hinfo[4] = {0, 0, 0, 0};
  HIKF_CUDA(cudaMemcpyAsync(hinfo, ints, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  HIKF_CUDA(cudaStreamSynchronize(s));
  HIKF_CUDA(cudaFreeAsync(A, s));
  HIKF_CUDA(cudaFreeAsync(VT, s));
  HIKF_CUDA(cudaFreeAsync(V, s));
  HIKF_CUDA(cudaFreeAsync(ints, s));
  sp.sweeps = hinfo[1];
  if (hinfo[3]) return make_status(HIKF_ETIMEOUT, "a bounded grid barrier in the Jacobi eigensolver timed out");
  if (hinfo[0]) return make_status(HIKF_ECUDA, "Jacobi eigensolver did not converge in 60 sweeps");
  return Status::Ok();
}

template <typename T>
Status spectral_gain(const SpectralState& sp, int n, const double* e, double* a, T* Msw, int nt, const int* flag,
                     cudaStream_t s) {
  spec_u_kernel<<<nblk((int64_t)n * 32, 256), 256, 0, s>>>(sp.W64, sp.s, e, n, sp.u, flag);
  HIKF_LAUNCH_CHECK("spec_u");
  spec_a_kernel<<<nblk((int64_t)n * 32, 256), 256, 0, s>>>(sp.W64, sp.u, n, a, flag);
  HIKF_LAUNCH_CHECK("spec_a");
  dim3 grid((unsigned)((n + 15) / 16), (unsigned)((n + 15) / 16));
  if (sizeof(T) == 8) {
    spec_m64_kernel<<<grid, 256, 0, s>>>(sp.W64, sp.s, n, nt, (double*)Msw, flag);
  } else {
    spec_split_kernel<<<nblk((int64_t)n * n, 256), 256, 0, s>>>(sp.W64, sp.s, n, sp.Uhi, sp.Ulo, flag);
    HIKF_LAUNCH_CHECK("spec_split");
    spec_m_dd_kernel<T><<<grid, 256, 0, s>>>(sp.Uhi, sp.Ulo, n, nt, Msw, flag);
  }
  HIKF_LAUNCH_CHECK("spec_m");
  return Status::Ok();
}
template Status spectral_gain<float>(const SpectralState&, int, const double*, double*, float*, int, const int*,
                                     cudaStream_t);
template Status spectral_gain<double>(const SpectralState&, int, const double*, double*, double*, int, const int*,
                                      cudaStream_t);

Status spectral_next(const SpectralState& sp, int n, int* flag, cudaStream_t s) {
  spec_next_kernel<<<nblk(n, 256), 256, 0, s>>>(sp.lam, n, sp.s, flag);
  HIKF_LAUNCH_CHECK("spec_next");
  return Status::Ok();
}

}  // namespace hikf

// ---------------------------------------------------------------------------
// Eigenbasis form of the state (rotated cross-covariance G = C_{t|t} W, W = D V).
// Because W^T R W = V^T V = I, the update C_{t|t} = C_p W diag(g) W^T R becomes, with
// G_p = G + C_Q W the rotated prior,  G <- G_p diag(g), and
//   sum_j K_ij (C_p)_ij = sum_k g_k G_p,ik^2,   (C_p a)_i = sum_k G_p,ik u_k,
// with g = 1/s_t and u = g o (W^T e). One pass over G per step, O(m n);
// C_{t|t} = G W^T R is formed only on request.
// ---------------------------------------------------------------------------
namespace hikf {
namespace {

// (sh, sl) += (ph, pl) in double-float arithmetic (TwoSum, then renormalise)
__device__ __forceinline__ void df_add(float& sh, float& sl, float ph, float pl) {
  const float s = sh + ph;
  const float bb = s - sh;
  float e = (sh - (s - bb)) + (ph - bb);
  e += sl + pl;
  sh = s + e;
  sl = e - (sh - s);
}

// FP32: one warp per group of kRows rows; every load of the group is issued before
// any store (the rows' G, Gq, x and delta^2), so each warp keeps ~kRows x 2 KB in flight.
template <int VPL, int kRows>
__global__ void __launch_bounds__(256) eigen_sweep_f32_kernel(int64_t m, int ld, int n, float* __restrict__ G,
                                                              const float* __restrict__ Gq,
                                                              const double* __restrict__ s,
                                                              const double* __restrict__ u, double theta,
                                                              double* __restrict__ x, double* __restrict__ var,
                                                              const int* __restrict__ flag) {
  if (*flag) return;
  __shared__ __align__(16) float sg[kMaxN], su[kMaxN];
  for (int k = threadIdx.x; k < ld; k += blockDim.x) {
    sg[k] = k < n ? (float)(1.0 / s[k]) : 0.f;
    su[k] = k < n ? (float)u[k] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nv = ld / 128 + ((ld % 128) > lane * 4 ? 1 : 0);  // float4 vectors of this lane (ld % 32 == 0)
  const int64_t groups = (m + kRows - 1) / kRows;
  const int64_t gstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t grp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); grp < groups; grp += gstride) {
    const int64_t row0 = grp * kRows;
    float4 gv[kRows][VPL], qv[kRows][VPL];
    double vr = 0.0, xr = 0.0;
    const int64_t myrow = row0 + lane;
    if (lane < kRows && myrow < m) {
      vr = var[myrow];
      xr = x[myrow];
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int64_t row = row0 + r;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        if (v < nv && row < m) {
          gv[r][v] = *reinterpret_cast<const float4*>(G + row * ld + v * 128 + lane * 4);
          qv[r][v] = *reinterpret_cast<const float4*>(Gq + row * ld + v * 128 + lane * 4);
        }
      }
    }
    float rdh[kRows], rdl[kRows], xih[kRows], xil[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int64_t row = row0 + r;
      float rp = 0.f, xp = 0.f;  // at most 16 terms per lane: plain FMA partials
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        if (v < nv && row < m) {
          float* ga = reinterpret_cast<float*>(&gv[r][v]);
          const float* qa = reinterpret_cast<const float*>(&qv[r][v]);
          const float4 g4 = *reinterpret_cast<const float4*>(sg + v * 128 + lane * 4);
          const float4 u4 = *reinterpret_cast<const float4*>(su + v * 128 + lane * 4);
          const float gk[4] = {g4.x, g4.y, g4.z, g4.w};
          const float uk[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const float gp = ga[w] + qa[w];  // rotated prior
            rp = fmaf(gk[w] * gp, gp, rp);
            xp = fmaf(gp, uk[w], xp);
            ga[w] = gp * gk[w];
          }
          *reinterpret_cast<float4*>(G + row * ld + v * 128 + lane * 4) = gv[r][v];
        }
      }
      rdh[r] = rp;
      rdl[r] = 0.f;
      xih[r] = xp;
      xil[r] = 0.f;
    }
    // across the lanes in double-float (FP32 pairs): the FP64 rate of this part is low,
    // so only the row's final value is formed in FP64
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      for (int o = 16; o > 0; o >>= 1) {
        const float a = __shfl_xor_sync(0xffffffffu, rdh[r], o), al = __shfl_xor_sync(0xffffffffu, rdl[r], o);
        const float b = __shfl_xor_sync(0xffffffffu, xih[r], o), bl = __shfl_xor_sync(0xffffffffu, xil[r], o);
        df_add(rdh[r], rdl[r], a, al);
        df_add(xih[r], xil[r], b, bl);
      }
    }
    if (lane < kRows && myrow < m) {
      float rh = rdh[0], rl = rdl[0], xh = xih[0], xl = xil[0];
#pragma unroll
      for (int r = 1; r < kRows; ++r)
        if (lane == r) {
          rh = rdh[r];
          rl = rdl[r];
          xh = xih[r];
          xl = xil[r];
        }
      var[myrow] = vr + theta - ((double)rh + (double)rl);
      x[myrow] = xr + ((double)xh + (double)xl);
    }
  }
}

// FP64 (oracle-grade mode): one warp per row
__global__ void eigen_sweep_f64_kernel(int64_t m, int ld, int n, double* __restrict__ G,
                                       const double* __restrict__ Gq, const double* __restrict__ s,
                                       const double* __restrict__ u, double theta, double* __restrict__ x,
                                       double* __restrict__ var, const int* __restrict__ flag) {
  if (*flag) return;
  __shared__ double sg[kMaxN], su[kMaxN];
  for (int k = threadIdx.x; k < ld; k += blockDim.x) {
    sg[k] = k < n ? 1.0 / s[k] : 0.0;
    su[k] = k < n ? u[k] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < m; row += warps) {
    double* gr = G + row * ld;
    const double* qr = Gq + row * ld;
    double rd64 = 0.0, xd64 = 0.0;
    for (int k = lane; k < ld; k += 32) {
      const double gp = gr[k] + qr[k], gk = sg[k];
      rd64 += gk * gp * gp;
      xd64 += gp * su[k];
      gr[k] = gp * gk;
    }
    for (int o = 16; o > 0; o >>= 1) {
      rd64 += __shfl_xor_sync(0xffffffffu, rd64, o);
      xd64 += __shfl_xor_sync(0xffffffffu, xd64, o);
    }
    if (lane == 0) {
      var[row] += theta - rd64;
      x[row] += xd64;
    }
  }
}

// out (m x ldo) = A (m x lda, first kdim columns) * B (kdim x nout, row-major, ld ldb), 64 x 64 tiles
template <typename T, typename BT>
__global__ void gemm_tn_kernel(int64_t m, int kdim, int nout, const T* __restrict__ A, int lda,
                               const BT* __restrict__ Bm, int ldb, T* __restrict__ out, int ldo, int subtract_q,
                               const T* __restrict__ Aq) {
  __shared__ T As[16][65];
  __shared__ T Bs[16][64];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  for (int k0 = 0; k0 < kdim; k0 += 16) {
    for (int t = threadIdx.x; t < 64 * 16; t += 256) {
      int r = t / 16, kk = t % 16;
      int64_t gr = r0 + r;
      T v = (T)0;
      if (gr < m && k0 + kk < kdim) {
        v = A[gr * lda + k0 + kk];
        if (subtract_q) v -= Aq[gr * lda + k0 + kk];
      }
      As[kk][r] = v;
    }
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int kk = t / 64, c = t % 64;
      Bs[kk][c] = (k0 + kk < kdim && c0 + c < nout) ? (T)Bm[(int64_t)(k0 + kk) * ldb + c0 + c] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T a[4], b[4];
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    int64_t gr = r0 + ty * 4 + i;
    if (gr >= m) continue;
    for (int j = 0; j < 4; ++j) {
      int c = c0 + tx + 16 * j;
      if (c < ldo) out[gr * ldo + c] = c < nout ? acc[i][j] : (T)0;
    }
  }
}

// B = W^T R (n x n): B[k][j] = W[j][k] r_j
__global__ void wtr_kernel(const double* __restrict__ W64, const double* __restrict__ rd, int n,
                           double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int k = (int)(t / n), j = (int)(t % n);
  out[t] = W64[(int64_t)j * n + k] * rd[j];
}

template <typename T>
__global__ void scale_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t count, double f) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) dst[t] = (T)((double)src[t] * f);
}

inline int nb(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

template <typename T>
Status eigen_setup(const SpectralState& sp, const T* CQ, int64_t m, int ld, int n, double c, T* Gq, T* G,
                   cudaStream_t s) {
  dim3 grid((unsigned)((m + 63) / 64), (unsigned)((ld + 63) / 64));
  gemm_tn_kernel<T, double><<<grid, 256, 0, s>>>(m, n, n, CQ, ld, sp.W64, n, Gq, ld, 0, nullptr);
  HIKF_LAUNCH_CHECK("gemm Gq");
  if (G) {
    scale_copy_kernel<T><<<nb(m * ld, 256), 256, 0, s>>>(Gq, G, m * ld, c);  // C_0 W = c C_Q W
    HIKF_LAUNCH_CHECK("scale G");
  }
  return Status::Ok();
}
template Status eigen_setup<float>(const SpectralState&, const float*, int64_t, int, int, double, float*, float*,
                                   cudaStream_t);
template Status eigen_setup<double>(const SpectralState&, const double*, int64_t, int, int, double, double*,
                                    double*, cudaStream_t);

template <typename T>
Status eigen_step(const SpectralState& sp, int64_t m, int ld, int n, T* G, const T* Gq, double theta, double* x,
                  double* var, const int* flag, int sms, cudaStream_t s) {
  if (sizeof(T) == 4) {
    auto launch = [&](auto kern, int rows) {
      const int64_t groups = (m + rows - 1) / rows;
      const int64_t blocks = std::min<int64_t>((groups + 7) / 8, (int64_t)sms * 8);
      kern<<<(unsigned)blocks, 256, 0, s>>>(m, ld, n, (float*)G, (const float*)Gq, sp.s, sp.u, theta, x, var, flag);
    };
    if (ld <= 128) launch(eigen_sweep_f32_kernel<1, 4>, 4);
    else if (ld <= 256) launch(eigen_sweep_f32_kernel<2, 4>, 4);
    else launch(eigen_sweep_f32_kernel<4, 2>, 2);
  } else {
    const int64_t blocks = std::min<int64_t>((m + 7) / 8, (int64_t)sms * 8);
    eigen_sweep_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(m, ld, n, (double*)G, (const double*)Gq, sp.s, sp.u,
                                                            theta, x, var, flag);
  }
  HIKF_LAUNCH_CHECK("eigen_sweep");
  return Status::Ok();
}
template Status eigen_step<float>(const SpectralState&, int64_t, int, int, float*, const float*, double, double*,
                                  double*, const int*, int, cudaStream_t);
template Status eigen_step<double>(const SpectralState&, int64_t, int, int, double*, const double*, double, double*,
                                   double*, const int*, int, cudaStream_t);

Status eigen_u(const SpectralState& sp, int n, const double* e, const int* flag, cudaStream_t s) {
  spec_u_kernel<<<nb((int64_t)n * 32, 256), 256, 0, s>>>(sp.W64, sp.s, e, n, sp.u, flag);
  HIKF_LAUNCH_CHECK("spec_u");
  return Status::Ok();
}

// out (m x ld) = A (m x ld, first n columns) * B (n x n, FP64)
template <typename T>
Status gemm_rows_small(const T* A, int64_t m, int ld, int n, const double* B, T* out, cudaStream_t s) {
  dim3 grid((unsigned)((m + 63) / 64), (unsigned)((ld + 63) / 64));
  gemm_tn_kernel<T, double><<<grid, 256, 0, s>>>(m, n, n, A, ld, B, n, out, ld, 0, nullptr);
  HIKF_LAUNCH_CHECK("gemm");
  return Status::Ok();
}
template Status gemm_rows_small<float>(const float*, int64_t, int, int, const double*, float*, cudaStream_t);
template Status gemm_rows_small<double>(const double*, int64_t, int, int, const double*, double*, cudaStream_t);

// C_{t|t} = G W^T R  (output in the caller's T, m x ld)
template <typename T>
Status eigen_cross(const SpectralState& sp, const double* rd, int64_t m, int ld, int n, const T* G, const T* Gq,
                   T* out, cudaStream_t s) {
  double* B = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&B, sizeof(double) * (size_t)n * n, s));
  wtr_kernel<<<nb((int64_t)n * n, 256), 256, 0, s>>>(sp.W64, rd, n, B);
  HIKF_LAUNCH_CHECK("wtr");
  dim3 grid((unsigned)((m + 63) / 64), (unsigned)((ld + 63) / 64));
  gemm_tn_kernel<T, double><<<grid, 256, 0, s>>>(m, n, n, G, ld, B, n, out, ld, 0, nullptr);
  HIKF_LAUNCH_CHECK("gemm cross");
  HIKF_CUDA(cudaFreeAsync(B, s));
  return Status::Ok();
}
template Status eigen_cross<float>(const SpectralState&, const double*, int64_t, int, int, const float*, const float*,
                                   float*, cudaStream_t);
template Status eigen_cross<double>(const SpectralState&, const double*, int64_t, int, int, const double*,
                                    const double*, double*, cudaStream_t);

}  // namespace hikf
