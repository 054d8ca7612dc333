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
// Eigensolver (FP64): Householder reduction to tridiagonal form on one CTA;
// implicit symmetric QR steps with Wilkinson shifts (Golub & Van Loan, Sec. 8.3)
// chased by one thread, which only records the rotations; then the eigenvectors
// V = Q G_1 G_2 ... row by row over many CTAs (rows are independent). The FP64
// rate per SM is low on this part, so the O(n^3) work is spread over SMs and
// the serial chase does O(n^2) work only.
#include <math.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "spectral.cuh"

namespace hikf {

namespace {

constexpr int kEigThreads = 1024;

__device__ __forceinline__ unsigned long long tc_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// ---- 1. Householder tridiagonalisation (one CTA) --------------------------
// A (n x n, row-major, symmetric; destroyed) -> T = Q^T A Q with diagonal d and
// sub-diagonal e; Q = H_0 H_1 ... H_{n-3}, H_k = I - 2 v_k v_k^T with v_k (unit,
// zero at indices <= k) stored as row k of hv.
__global__ void __launch_bounds__(kEigThreads) eig_tridiag_kernel(double* __restrict__ A, int n,
                                                                 double* __restrict__ d, double* __restrict__ e,
                                                                 double* __restrict__ hv) {
  __shared__ double red[32];
  __shared__ double sv[kMaxN], sw[kMaxN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    double part = 0.0;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) {
      double x = A[(int64_t)i * n + k];
      part += x * x;
    }
    const double ss = block_sum(part, red);
    const double x0 = A[(int64_t)(k + 1) * n + k];
    const double tail = ss - x0 * x0;
    double* vk = hv + (int64_t)k * n;
    if (tail <= 0.0) {  // already tridiagonal in this column: H_k = I
      for (int i = tid; i < n; i += blockDim.x) vk[i] = 0.0;
      if (tid == 0) e[k] = x0;
      __syncthreads();
      continue;
    }
    const double alpha = x0 >= 0.0 ? -sqrt(ss) : sqrt(ss);
    const double v0 = x0 - alpha;
    const double vn = sqrt(tail + v0 * v0);
    for (int i = tid; i < n; i += blockDim.x) {
      double v = 0.0;
      if (i == k + 1) v = v0 / vn;
      else if (i > k + 1) v = A[(int64_t)i * n + k] / vn;
      sv[i] = v;
      vk[i] = v;
    }
    if (tid == 0) e[k] = alpha;
    __syncthreads();
    // w = A_sub v (rows k+1..n-1), warp per row
    for (int i = k + 1 + warp; i < n; i += nw) {
      double s = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) s += A[(int64_t)i * n + j] * sv[j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sw[i] = s;
    }
    __syncthreads();
    double cp = 0.0;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) cp += sv[i] * sw[i];
    const double cc = block_sum(cp, red);
    for (int i = k + 1 + tid; i < n; i += blockDim.x) sw[i] = sw[i] - cc * sv[i];  // q = w - (v.w) v
    __syncthreads();
    const int len = n - k - 1;
    for (int64_t t = tid; t < (int64_t)len * len; t += blockDim.x) {
      int i = k + 1 + (int)(t / len), j = k + 1 + (int)(t % len);
      A[(int64_t)i * n + j] -= 2.0 * (sv[i] * sw[j] + sw[i] * sv[j]);
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) d[i] = A[(int64_t)i * n + i];
  if (tid == 0 && n >= 2) e[n - 2] = A[(int64_t)(n - 1) * n + (n - 2)];
}

// ---- 1'. the same reduction over a grid of co-resident CTAs --------------------
// Per column k: every CTA forms v (and the norm) redundantly; w = A_sub v is split by
// rows over the CTAs; after a grid barrier every CTA forms q = w - (v.w) v; the rank-2
// update A -= 2 (v q^T + q v^T) is split by rows; a second grid barrier ends the column.
// The FP64 work, O(n^3) in all, is spread over the SMs. The grid barrier is a counter
// with a bounded wait (2 s), after which the CTA sets *err and leaves; the launch is
// cooperative, so every CTA is resident.
constexpr int kTriThreads = 256;

__device__ bool grid_barrier(unsigned* bar, unsigned& gen, int* err, volatile int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned target = (gen + 1u) * gridDim.x;
    atomicAdd(bar, 1u);
    const unsigned long long t0 = tc_now_ns();
    while (*(volatile unsigned*)bar < target) {
      if (tc_now_ns() - t0 > 2000000000ull) {
        atomicExch(err, 1);
        *s_abort = 1;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  ++gen;
  return *s_abort == 0;
}

__global__ void __launch_bounds__(kTriThreads) eig_tridiag_grid_kernel(double* __restrict__ A, int n,
                                                                       double* __restrict__ d,
                                                                       double* __restrict__ e,
                                                                       double* __restrict__ hv,
                                                                       double* __restrict__ wbuf, unsigned* bar,
                                                                       int* __restrict__ err) {
  __shared__ double red[32];
  __shared__ double sv[kMaxN], sq[kMaxN];
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int rank = blockIdx.x, nblk = gridDim.x;
  if (tid == 0) s_abort = 0;
  __syncthreads();
  unsigned gen = 0;
  for (int k = 0; k + 2 < n; ++k) {
    double part = 0.0;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) {
      const double x = A[(int64_t)i * n + k];
      part += x * x;
    }
    const double ss = block_sum(part, red);
    const double x0 = A[(int64_t)(k + 1) * n + k];
    const double tail = ss - x0 * x0;
    if (tail <= 0.0) {  // already tridiagonal in this column: H_k = I (every CTA decides alike)
      if (rank == 0) {
        for (int i = tid; i < n; i += blockDim.x) hv[(int64_t)k * n + i] = 0.0;
        if (tid == 0) e[k] = x0;
      }
      __syncthreads();
      continue;
    }
    const double alpha = x0 >= 0.0 ? -sqrt(ss) : sqrt(ss);
    const double v0 = x0 - alpha;
    const double vn = sqrt(tail + v0 * v0);
    for (int i = tid; i < n; i += blockDim.x) {
      double v = 0.0;
      if (i == k + 1) v = v0 / vn;
      else if (i > k + 1) v = A[(int64_t)i * n + k] / vn;
      sv[i] = v;
      if (rank == 0) hv[(int64_t)k * n + i] = v;
    }
    if (rank == 0 && tid == 0) e[k] = alpha;
    __syncthreads();
    // w = A_sub v: rows k+1 .. n-1 over the CTAs, a warp per row
    for (int i = k + 1 + rank * nw + warp; i < n; i += nblk * nw) {
      double sacc = 0.0;
      for (int j = k + 1 + lane; j < n; j += 32) sacc += A[(int64_t)i * n + j] * sv[j];
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) wbuf[i] = sacc;
    }
    if (!grid_barrier(bar, gen, err, &s_abort)) return;
    double cp = 0.0;
    for (int i = k + 1 + tid; i < n; i += blockDim.x) cp += sv[i] * wbuf[i];
    const double cc = block_sum(cp, red);
    for (int i = k + 1 + tid; i < n; i += blockDim.x) sq[i] = wbuf[i] - cc * sv[i];  // q = w - (v.w) v
    __syncthreads();
    // A -= 2 (v q^T + q v^T) on this CTA's rows
    for (int i = k + 1 + rank; i < n; i += nblk) {
      const double vi = sv[i], qi = sq[i];
      for (int j = k + 1 + tid; j < n; j += blockDim.x) A[(int64_t)i * n + j] -= 2.0 * (vi * sq[j] + qi * sv[j]);
    }
    if (!grid_barrier(bar, gen, err, &s_abort)) return;
  }
  if (rank == 0) {
    for (int i = tid; i < n; i += blockDim.x) d[i] = A[(int64_t)i * n + i];
    if (tid == 0 && n >= 2) e[n - 2] = A[(int64_t)(n - 1) * n + (n - 2)];
  }
}

// ---- 2. implicit symmetric QR on (d, e), one thread, several bulges at once ----
// (Golub & Van Loan, Alg. 8.3.2 with deflation.) Each batch chases kBulges bulges down
// the active block [l, m], bulge b starting three columns behind bulge b-1, with shifts
// from the 2 x 2 diagonal blocks at the bottom of the block (a single Wilkinson-shifted
// bulge when the block is short). A rotation of one bulge depends only on its own
// previous rotation and on entries the bulge ahead has finished with, so the bulges'
// FP64 dependency chains overlap: the chase is latency-bound, and this part's FP64
// latency is long. The chase does not need the eigenvectors: it records every Givens
// rotation (c, s) and, per bulge, its block [l, m]. Recording bulge by bulge is a valid
// order for the back-transformation, because a rotation of bulge b on columns (k, k+1)
// that precedes one of bulge b-1 in time acts on columns at least three apart.
// Capacity: at most max_sweeps bulges of at most n - 1 rotations each.
// d and e live in shared memory; each bulge carries its d[k], e[k] and (x, z) in registers.
constexpr int kBulges = 4;

__device__ __forceinline__ void givens(double x, double z, double& r, double& c, double& s) {
  // r = |(x, z)|, c = x / r, s = z / r: one reciprocal square root where x^2 + z^2 is
  // safely inside the normal range (always, for the matrices of this library), hypot
  // and a division otherwise
  const double t2 = fma(x, x, z * z);
  c = 1.0;
  s = 0.0;
  if (t2 > 1e-290 && t2 < 1e290) {
    const double ir = rsqrt(t2);
    r = t2 * ir;
    c = x * ir;
    s = z * ir;
  } else {
    r = hypot(x, z);
    if (r > 0.0) {
      c = x / r;
      s = z / r;
    }
  }
}

__global__ void eig_qr_chase_kernel(double* __restrict__ dg, double* __restrict__ eg, int n, int max_sweeps,
                                    double2* __restrict__ rot, int2* __restrict__ sweep_lm,
                                    int* __restrict__ nsweeps, int* __restrict__ info) {
  __shared__ double d[kMaxN], e[kMaxN];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = dg[i];
    e[i] = eg[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double eps = 2.220446049250313e-16;
    int m = n - 1, ns = 0;
    int64_t nr = 0;
    int bad = 0;
    while (true) {
      while (m > 0 && fabs(e[m - 1]) <= eps * (fabs(d[m - 1]) + fabs(d[m]))) {
        e[m - 1] = 0.0;
        --m;
      }
      if (m == 0) break;
      int l = m - 1;
      while (l > 0 && fabs(e[l - 1]) > eps * (fabs(d[l - 1]) + fabs(d[l]))) --l;
      const int len = m - l;  // rotations per bulge
      const int kb = len >= 4 * kBulges ? kBulges : 1;
      if (ns + kb > max_sweeps) {
        bad = 1;
        break;
      }
      double mu[kBulges];
      if (kb == 1) {
        // Wilkinson shift from the trailing 2 x 2 block
        const double a = d[m - 1], b = e[m - 1], c2 = d[m];
        const double delta = 0.5 * (a - c2);
        const double sgn = delta >= 0.0 ? 1.0 : -1.0;
        mu[0] = c2 - b * b / (delta + sgn * hypot(delta, b));
      } else {
        // both eigenvalues of each of the kBulges/2 trailing 2 x 2 diagonal blocks
        for (int j = 0; j < kBulges / 2; ++j) {
          const int i1 = m - 2 * j;
          const double a = d[i1 - 1], b = e[i1 - 1], c2 = d[i1];
          const double mid = 0.5 * (a + c2), rad = hypot(0.5 * (a - c2), b);
          mu[2 * j] = mid - rad;
          mu[2 * j + 1] = mid + rad;
        }
      }
      // bulge state: carried d[k], e[k] and the (x, z) to annihilate
      double x[kBulges], z[kBulges], ak[kBulges], bk[kBulges];
      const int steps = len + 3 * (kb - 1);
      for (int st = 0; st < steps; ++st) {
#pragma unroll
        for (int bb = 0; bb < kBulges; ++bb) {
          if (bb >= kb) continue;
          const int k = l + st - 3 * bb;
          if (k < l || k >= m) continue;
          if (k == l) {  // the bulge enters the block
            ak[bb] = d[l];
            bk[bb] = e[l];
            x[bb] = d[l] - mu[bb];
            z[bb] = e[l];
          }
          const double ck = d[k + 1];
          const double f = k + 1 < m ? e[k + 1] : 0.0;
          double r, c, s;
          givens(x[bb], z[bb], r, c, s);
          if (k > l) e[k - 1] = r;
          const double cc = c * c, ss = s * s, cs = c * s;
          d[k] = ak[bb] * cc + 2.0 * bk[bb] * cs + ck * ss;
          const double dk1 = ak[bb] * ss - 2.0 * bk[bb] * cs + ck * cc;
          const double ek = (ck - ak[bb]) * cs + bk[bb] * (cc - ss);
          rot[nr + (int64_t)bb * len + (k - l)] = make_double2(c, s);
          x[bb] = ek;
          if (k + 1 < m) {
            z[bb] = f * s;
            bk[bb] = f * c;
          }
          e[k] = ek;
          ak[bb] = dk1;
          if (k == m - 1) d[m] = dk1;  // the bulge leaves the block
        }
      }
      for (int bb = 0; bb < kb; ++bb) sweep_lm[ns + bb] = make_int2(l, m);
      ns += kb;
      nr += (int64_t)kb * len;
    }
    *info = bad;
    *nsweeps = ns;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    dg[i] = d[i];
    eg[i] = e[i];
  }
}

// ---- 3. eigenvectors V = H_0 ... H_{n-3} G_1 G_2 ... , rows in parallel ----
// Row i of V is e_i^T times the product; each factor acts on a row independently. One
// thread carries kVecRows rows (held in shared memory) through the factors together, so
// the rows' FP64 dependency chains interleave; the row groups are spread over CTAs.
constexpr int kVecRows = 8;  // rows per thread (one thread per CTA)
__global__ void __launch_bounds__(32) eig_vectors_kernel(const double* __restrict__ hv,
                                                         const double2* __restrict__ rot,
                                                         const int2* __restrict__ sweep_lm,
                                                         const int* __restrict__ nsweeps,
                                                         const int* __restrict__ info, int n,
                                                         double* __restrict__ V) {
  extern __shared__ double srow[];  // kVecRows x (n + 1)
  if (threadIdx.x != 0 || *info) return;
  const int i0 = blockIdx.x * kVecRows;
  const int nr = min(kVecRows, n - i0);
  if (nr <= 0) return;
  const int ld = n + 1;
  for (int r = 0; r < kVecRows; ++r)
    for (int j = 0; j < n; ++j) srow[r * ld + j] = (r < nr && j == i0 + r) ? 1.0 : 0.0;
  // row <- row (I - 2 v_k v_k^T), k = 0 .. n-3
  for (int k = 0; k + 2 < n; ++k) {
    const double* vk = hv + (int64_t)k * n;
    double dot[kVecRows];
#pragma unroll
    for (int r = 0; r < kVecRows; ++r) dot[r] = 0.0;
    for (int j = k + 1; j < n; ++j) {
      const double v = vk[j];
#pragma unroll
      for (int r = 0; r < kVecRows; ++r) dot[r] = fma(srow[r * ld + j], v, dot[r]);
    }
    for (int j = k + 1; j < n; ++j) {
      const double v = vk[j];
#pragma unroll
      for (int r = 0; r < kVecRows; ++r) srow[r * ld + j] -= 2.0 * dot[r] * v;
    }
  }
  // row <- row G, sweep by sweep, rotations in recorded order
  const int ns = *nsweeps;
  int64_t off = 0;
  for (int sw = 0; sw < ns; ++sw) {
    const int2 lm = sweep_lm[sw];
    double vk[kVecRows];
#pragma unroll
    for (int r = 0; r < kVecRows; ++r) vk[r] = srow[r * ld + lm.x];
    for (int k = lm.x; k < lm.y; ++k) {
      const double2 cs = rot[off + (k - lm.x)];
#pragma unroll
      for (int r = 0; r < kVecRows; ++r) {
        const double vk1 = srow[r * ld + k + 1];
        srow[r * ld + k] = cs.x * vk[r] + cs.y * vk1;
        vk[r] = -cs.y * vk[r] + cs.x * vk1;
      }
    }
#pragma unroll
    for (int r = 0; r < kVecRows; ++r) srow[r * ld + lm.y] = vk[r];
    off += lm.y - lm.x;
  }
  for (int r = 0; r < nr; ++r)
    for (int j = 0; j < n; ++j) V[(int64_t)(i0 + r) * n + j] = srow[r * ld + j];
}

// B~ = D sym(HCQ) D with D = R^{-1/2}
__global__ void scale_b_kernel(const double* __restrict__ hcq_sym, const double* __restrict__ rd, int n,
                               double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  out[t] = hcq_sym[t] / sqrt(rd[i] * rd[j]);
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
  const int64_t nn = (int64_t)n * n;
  const int max_sweeps = 40 * n + 100;
  const int64_t max_rot = (int64_t)max_sweeps * std::max(1, n - 1);
  double *A = nullptr, *V = nullptr, *hv = nullptr, *e = nullptr;
  double2* rot = nullptr;
  int2* lm = nullptr;
  int* ints = nullptr;
  HIKF_CUDA(cudaMallocAsync((void**)&A, sizeof(double) * nn, s));
  HIKF_CUDA(cudaMallocAsync((void**)&V, sizeof(double) * nn, s));
  HIKF_CUDA(cudaMallocAsync((void**)&hv, sizeof(double) * nn, s));
  HIKF_CUDA(cudaMallocAsync((void**)&e, sizeof(double) * n, s));
  HIKF_CUDA(cudaMallocAsync((void**)&rot, sizeof(double2) * max_rot, s));
  HIKF_CUDA(cudaMallocAsync((void**)&lm, sizeof(int2) * max_sweeps, s));
  double* wbuf = nullptr;
  HIKF_CUDA(cudaMallocAsync((void**)&wbuf, sizeof(double) * n, s));
  HIKF_CUDA(cudaMallocAsync((void**)&ints, 4 * sizeof(int), s));  // info, nsweeps, barrier, tridiag error
  HIKF_CUDA(cudaMemsetAsync(ints, 0, 4 * sizeof(int), s));
  HIKF_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, s));
  scale_b_kernel<<<nblk(nn, 256), 256, 0, s>>>(hcq_sym, rd, n, A);
  HIKF_LAUNCH_CHECK("scale_b");
  {
    // cooperative grid: at most one CTA per SM, all resident
    int dev = 0, sms = 1, per_sm = 0;
    HIKF_CUDA(cudaGetDevice(&dev));
    HIKF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HIKF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eig_tridiag_grid_kernel, kTriThreads, 0));
    const int grid = std::max(1, std::min({64, sms * std::max(per_sm, 0), std::max(1, n / 4)}));
    if (per_sm >= 1) {
      double* Ap = A;
      double* dp = sp.lam;
      double* ep = e;
      double* hp = hv;
      double* wp = wbuf;
      unsigned* bp = reinterpret_cast<unsigned*>(ints + 2);
      int* errp = ints + 3;
      int nn_ = n;
      void* args[] = {&Ap, &nn_, &dp, &ep, &hp, &wp, &bp, &errp};
      HIKF_CUDA(cudaLaunchCooperativeKernel((const void*)eig_tridiag_grid_kernel, dim3(grid), dim3(kTriThreads), args,
                                            0, s));
    } else {
      eig_tridiag_kernel<<<1, kEigThreads, 0, s>>>(A, n, sp.lam, e, hv);
    }
    HIKF_LAUNCH_CHECK("eig_tridiag");
  }
  eig_qr_chase_kernel<<<1, 32, 0, s>>>(sp.lam, e, n, max_sweeps, rot, lm, ints + 1, ints);
  HIKF_LAUNCH_CHECK("eig_qr_chase");
  const size_t vsmem = sizeof(double) * kVecRows * (size_t)(n + 1);
  eig_vectors_kernel<<<nblk(n, kVecRows), 32, vsmem, s>>>(hv, rot, lm, ints + 1, ints, n, V);
  HIKF_LAUNCH_CHECK("eig_vectors");
  spec_init_kernel<<<nblk(nn, 256), 256, 0, s>>>(V, sp.lam, rd, n, c, sp.W64, sp.W32, sp.s, flag);
  HIKF_LAUNCH_CHECK("spec_init");
  int hinfo[4] = {0, 0, 0, 0};
  HIKF_CUDA(cudaMemcpyAsync(hinfo, ints, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  HIKF_CUDA(cudaStreamSynchronize(s));
  HIKF_CUDA(cudaFreeAsync(A, s));
  HIKF_CUDA(cudaFreeAsync(V, s));
  HIKF_CUDA(cudaFreeAsync(hv, s));
  HIKF_CUDA(cudaFreeAsync(e, s));
  HIKF_CUDA(cudaFreeAsync(rot, s));
  HIKF_CUDA(cudaFreeAsync(lm, s));
  HIKF_CUDA(cudaFreeAsync(ints, s));
  HIKF_CUDA(cudaFreeAsync(wbuf, s));
  if (hinfo[3]) return make_status(HIKF_ETIMEOUT, "a bounded grid barrier in the tridiagonalisation timed out");
  if (hinfo[0]) return make_status(HIKF_ECUDA, "eigensolver did not converge");
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

__device__ __forceinline__ void kahan_add(float v, float& s, float& c) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
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
