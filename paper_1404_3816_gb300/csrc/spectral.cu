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
// index of the pair that holds a in round r, and a's partner
__device__ __forceinline__ int rr_slot(int r, int a, int N, int& partner) {
  if (a == N - 1 || a == r) {
    partner = a == r ? N - 1 : r;
    return 0;
  }
  partner = rr_mod(2 * r - a, N - 1);
  const int d = rr_mod(a - r, N - 1);
  return min(d, N - 1 - d);
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

// A (N x N, row-major, symmetric) -> diag(lambda) in place; VT (N x N) -> V^T (row j =
// eigenvector j). diag and pq are round-parity double buffers (2 x N and 2 x N/2): the
// rotations of a round read only them, and the round's updates write the other parity,
// so a CTA that is still forming rotations never sees A change under it, and one grid
// barrier per round suffices. Every CTA forms all N/2 rotations of a round itself (the
// same inputs give the same rotations and the same convergence decision in every CTA),
// with each index's slot and partner in the next round, which tell a block's thread
// which of its four new entries to export. The updates are dealt to the CTAs as tasks:
// block row i of A (blocks j >= i, the diagonal block included, each written with its
// mirror) or column pair k of V. Every entry of A and V has one writer per round.
// info[0] = 1 when max_sweeps sweeps did not converge; *sweeps = sweeps run.
__global__ void __launch_bounds__(kJacThreads) eig_jacobi_kernel(double* __restrict__ A, double* __restrict__ VT,
                                                                 int N, int max_sweeps,
                                                                 double* __restrict__ diag,
                                                                 double* __restrict__ pq,
                                                                 unsigned* bar, int* err, int* info,
                                                                 int* sweeps) {
  __shared__ double sc[kMaxN / 2], ssn[kMaxN / 2], st[kMaxN / 2];
  __shared__ int spi[kMaxN / 2], sqi[kMaxN / 2], son[kMaxN / 2];
  __shared__ int sslp[kMaxN / 2], sptp[kMaxN / 2], sslq[kMaxN / 2], sptq[kMaxN / 2];
  __shared__ int s_rot;
  __shared__ volatile int s_abort;
  const int P = N / 2;
  const int tid = threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid, gthreads = (int64_t)gridDim.x * blockDim.x;  // setup only
  unsigned gen = 0;
  if (tid == 0) s_abort = 0;
  // V = I; round-0 inputs into parity 0
  for (int64_t u = gtid; u < (int64_t)N * N; u += gthreads) VT[u] = (u / N == u % N) ? 1.0 : 0.0;
  for (int64_t u = gtid; u < N; u += gthreads) diag[u] = A[u * N + u];
  for (int64_t k = gtid; k < P; k += gthreads) {
    int p, q;
    rr_pair(0, (int)k, N, p, q);
    pq[k] = A[(int64_t)p * N + q];
  }
  if (!grid_barrier(bar, gen, err, &s_abort)) return;
  // absolute floor for a negligible off-diagonal entry: eps max|a_ii| / N, so the entries
  // left out add up (Frobenius) to at most eps max|a_ii|, the backward error of any FP64
  // eigensolver. It ends the iteration on graded spectra (a smooth kernel's), where the
  // entries coupling the smallest eigenvalues carry rounding from rotations with the
  // largest ones and never fall below eps relative to their own diagonal. Every CTA forms
  // the same value.
  __shared__ double s_dmax;
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < N; ++i) m = fmax(m, fabs(diag[i]));
    s_dmax = m;
  }
  __syncthreads();
  const double floor_abs = 2.220446049250313e-16 * s_dmax / N;
  int par = 0, sw = 0;
  bool converged = false;
  for (; sw < max_sweeps && !converged; ++sw) {
    if (tid == 0) s_rot = 0;
    for (int r = 0; r + 1 < N; ++r) {
      const int rn = r + 2 < N ? r + 1 : 0;  // the next round (wraps into the next sweep)
      const double* dg = diag + par * N;
      const double* pg = pq + par * P;
      double* dn = diag + (par ^ 1) * N;
      double* pn = pq + (par ^ 1) * P;
      __syncthreads();
      for (int k = tid; k < P; k += blockDim.x) {
        int p, q;
        rr_pair(r, k, N, p, q);
        double c, s_, t;
        const bool on = jacobi_rotation(dg[p], dg[q], pg[k], floor_abs, c, s_, t);
        if (on) atomicAdd(&s_rot, 1);
        sc[k] = c;
        ssn[k] = s_;
        st[k] = t;
        spi[k] = p;
        sqi[k] = q;
        son[k] = on ? 1 : 0;
        // where p and q go in the next round: the slot of their pair and their partner
        int pp, pq2;
        sslp[k] = rr_slot(rn, p, N, pp);
        sptp[k] = pp;
        sslq[k] = rr_slot(rn, q, N, pq2);
        sptq[k] = pq2;
      }
      __syncthreads();
      // updates: tasks 0 .. P-1 are the block rows i (blocks j >= i), tasks P .. 2P-1 the
      // column pairs of V; tasks are dealt to the CTAs in turn
      for (int task = blockIdx.x; task < 2 * P; task += gridDim.x) {
        if (task < P) {
          const int i = task, p = spi[i], q = sqi[i];
          for (int j = i + tid; j < P; j += blockDim.x) {
            if (j == i) {  // diagonal block: a_pp - t a_pq, a_qq + t a_pq, a_pq -> 0
              const double t = st[i], apq = A[(int64_t)p * N + q];
              const double app = A[(int64_t)p * N + p] - t * apq, aqq = A[(int64_t)q * N + q] + t * apq;
              A[(int64_t)p * N + p] = app;
              A[(int64_t)q * N + q] = aqq;
              A[(int64_t)p * N + q] = 0.0;
              A[(int64_t)q * N + p] = 0.0;
              dn[p] = app;
              dn[q] = aqq;
              if (sptp[i] == q) pn[sslp[i]] = 0.0;  // N = 2: the same pair meets again
              continue;
            }
            const int u0 = spi[j], v0 = sqi[j];
            double x00 = A[(int64_t)p * N + u0], x01 = A[(int64_t)p * N + v0];
            double x10 = A[(int64_t)q * N + u0], x11 = A[(int64_t)q * N + v0];
            if (son[i] | son[j]) {
              const double c1 = sc[i], s1 = ssn[i], c2 = sc[j], s2 = ssn[j];
              // rows: J_i^T X
              const double y00 = c1 * x00 - s1 * x10, y01 = c1 * x01 - s1 * x11;
              const double y10 = s1 * x00 + c1 * x10, y11 = s1 * x01 + c1 * x11;
              // columns: Y J_j
              x00 = c2 * y00 - s2 * y01;
              x01 = s2 * y00 + c2 * y01;
              x10 = c2 * y10 - s2 * y11;
              x11 = s2 * y10 + c2 * y11;
              A[(int64_t)p * N + u0] = x00;
              A[(int64_t)p * N + v0] = x01;
              A[(int64_t)q * N + u0] = x10;
              A[(int64_t)q * N + v0] = x11;
              A[(int64_t)u0 * N + p] = x00;
              A[(int64_t)v0 * N + p] = x01;
              A[(int64_t)u0 * N + q] = x10;
              A[(int64_t)v0 * N + q] = x11;
            }
            // export the entries that form a pair of the next round
            if (sptp[i] == u0) pn[sslp[i]] = x00;
            if (sptp[i] == v0) pn[sslp[i]] = x01;
            if (sptq[i] == u0) pn[sslq[i]] = x10;
            if (sptq[i] == v0) pn[sslq[i]] = x11;
          }
        } else {
          const int k = task - P;
          if (!son[k]) continue;
          const double c = sc[k], s_ = ssn[k];
          double* vp = VT + (int64_t)spi[k] * N;
          double* vq = VT + (int64_t)sqi[k] * N;
          for (int comp = tid; comp < N; comp += blockDim.x) {
            const double a = vp[comp], b = vq[comp];
            vp[comp] = c * a - s_ * b;
            vq[comp] = s_ * a + c * b;
          }
        }
      }
      par ^= 1;
      if (!grid_barrier(bar, gen, err, &s_abort)) return;
    }
    __syncthreads();
    converged = s_rot == 0;
    __syncthreads();  // every thread has read s_rot before thread 0 resets it for the next sweep
  }
  if (blockIdx.x == 0 && tid == 0) {
    *info = converged ? 0 : 1;
    *sweeps = sw;
  }
}

// lambda_j = A_jj, V (n x n, row i = component i) from V^T (N x N)
__global__ void eig_jacobi_out_kernel(const double* __restrict__ A, const double* __restrict__ VT, int N, int n,
                                      double* __restrict__ lam, double* __restrict__ V) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
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
  double *A = nullptr, *VT = nullptr, *V = nullptr, *dbuf = nullptr;
  int* ints = nullptr;
  HIKF_CUDA(cudaMallocAsync((void**)&A, sizeof(double) * NN, s));
  HIKF_CUDA(cudaMallocAsync((void**)&VT, sizeof(double) * NN, s));
  HIKF_CUDA(cudaMallocAsync((void**)&V, sizeof(double) * nn, s));
  HIKF_CUDA(cudaMallocAsync((void**)&dbuf, sizeof(double) * 3 * N, s));  // diag[2][N], pq[2][N/2]
  HIKF_CUDA(cudaMallocAsync((void**)&ints, 4 * sizeof(int), s));         // info, sweeps, barrier, error
  HIKF_CUDA(cudaMemsetAsync(ints, 0, 4 * sizeof(int), s));
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
    double* dp = dbuf;
    double* pp = dbuf + 2 * N;
    unsigned* bp = reinterpret_cast<unsigned*>(ints + 2);
    int* errp = ints + 3;
    int* infop = ints;
    int* swp = ints + 1;
    void* args[] = {&Ap, &Vp, &Np, &msw, &dp, &pp, &bp, &errp, &infop, &swp};
    HIKF_CUDA(cudaLaunchCooperativeKernel((const void*)eig_jacobi_kernel, dim3(grid), dim3(kJacThreads), args, 0, s));
    HIKF_LAUNCH_CHECK("eig_jacobi");
  }
  eig_jacobi_out_kernel<<<nblk(nn, 256), 256, 0, s>>>(A, VT, N, n, sp.lam, V);
  HIKF_LAUNCH_CHECK("eig_jacobi_out");
  spec_init_kernel<<<nblk(nn, 256), 256, 0, s>>>(V, sp.lam, rd, n, c, sp.W64, sp.W32, sp.s, flag);
  HIKF_LAUNCH_CHECK("spec_init");
  int hinfo[4] = {0, 0, 0, 0};
  HIKF_CUDA(cudaMemcpyAsync(hinfo, ints, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  HIKF_CUDA(cudaStreamSynchronize(s));
  HIKF_CUDA(cudaFreeAsync(A, s));
  HIKF_CUDA(cudaFreeAsync(VT, s));
  HIKF_CUDA(cudaFreeAsync(V, s));
  HIKF_CUDA(cudaFreeAsync(dbuf, s));
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
  HIKF_CUDA(cudaMallocAsync((void**)&B, sizeof(double) * (size_t)n * n, s));
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
