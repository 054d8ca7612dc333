// Measurement update of HiKF (Alg. 2, prediction + correction), per step:
//
//   n x n chain (S3): S_t = H C_{t|t-1} + R  ->  M_t = S_t^{-1}
//     FP32 Cholesky + triangular inverse on one CTA, then residual refinement
//     E = I - S M, M <- M + M E with the residual in compensated (double-float)
//     FP32 arithmetic over many CTAs; FP64 Cholesky fallback when the FP32
//     factor is not accurate enough. M is kept as an unevaluated sum Mh + Ml.
//   innovation (S2): e = y - H x  (sparse H, FP64)
//   a = M e
//   sweep (S4, the O(n^2 m) hot loop), one streaming pass over the m rows:
//     C_p = C + C_Q                            (Eq. KF_forecast_new)
//     K   = C_p M                              (Eq. kalmangin_new)
//     delta^2 += diag(Q) - sum_j K_ij C_p,ij   (variance update)
//     x   += C_p a                             (= K (y - H x))
//     C   <- K R                               (Eq. KF_pred_new: C_p - K H C_p = K R,
//                                                because H C_p = S - R)
//   next S (n-space recurrence): H C_{t+1|t} = H C_{t|t} + H C_Q = R - R M_t R + H C_Q,
//     so S_{t+1} = H C_Q + 2R - R M_t R needs no pass over C.
#include <math.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "step.cuh"

namespace hikf {

namespace {

constexpr int kThreads = 256;

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// double-float helpers (error-free transformations)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// ---------------------------------------------------------------------------
// H C gather: out[r][c] (+)= sum_{k in ray r} H_rk C[k][c]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gather_hc_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const T* __restrict__ C, int ld, int n,
                                 double* __restrict__ out, int accumulate) {
  const int r = blockIdx.x;
  if constexpr (sizeof(T) == 4) {
    // FP32 C: a double-float (hi + lo) sum of the products H_rk C_kc on the FP32 pipe (about
    // 2^-48 relative per term, far below the FP32 rounding already in C). The ray's entries
    // are split into FP32 pairs once, in shared memory, in chunks.
    constexpr int kG = 1024, kCols = kMaxN / 256;  // columns per thread (blockDim = 256)
    __shared__ float svh[kG], svl[kG];
    __shared__ int scol[kG];
    float sh[kCols], sl[kCols];
#pragma unroll
    for (int u = 0; u < kCols; ++u) sh[u] = sl[u] = 0.f;
    const int64_t e0 = rowptr[r], e1 = rowptr[r + 1];
    for (int64_t base = e0; base < e1; base += kG) {
      const int cnt = (int)min((int64_t)kG, e1 - base);
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        const double v = val[base + t];
        const float vh = (float)v;
        svh[t] = vh;
        svl[t] = (float)(v - (double)vh);
        scol[t] = col[base + t];
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < kCols; ++u) {
        const int c = threadIdx.x + u * blockDim.x;
        if (c >= n) break;
        float h = sh[u], l = sl[u];
        for (int t = 0; t < cnt; ++t) {
          const float vh = svh[t], x = (float)C[(int64_t)scol[t] * ld + c];
          const float p = vh * x;
          const float e = fmaf(vh, x, -p) + svl[t] * x;  // v x = p + e to about 2^-48
          const float s2 = h + p;                       // (h, l) += (p, e) by an exact two-sum
          const float bp = s2 - h;
          l += ((h - (s2 - bp)) + (p - bp)) + e;
          h = s2;
        }
        sh[u] = h;
        sl[u] = l;
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kCols; ++u) {
      const int c = threadIdx.x + u * blockDim.x;
      if (c >= n) break;
      const double acc = (double)sh[u] + (double)sl[u];
      if (accumulate) out[(int64_t)r * n + c] += acc; else out[(int64_t)r * n + c] = acc;
    }
  } else {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      double acc = 0.0;
      for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) acc += val[k] * (double)C[(int64_t)col[k] * ld + c];
      if (accumulate) out[(int64_t)r * n + c] += acc; else out[(int64_t)r * n + c] = acc;
    }
  }
}

// S = sym(A) + diag(R)
__global__ void form_s_kernel(const double* __restrict__ A, const double* __restrict__ rd, int n,
                              double* __restrict__ S) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  double v = 0.5 * (A[(int64_t)i * n + j] + A[(int64_t)j * n + i]);
  if (i == j) v += rd[i];
  S[t] = v;
}

// next S from the recurrence: S' = sym(HCQ) + 2R - R M R   (M = Mh + Ml); skipped when the step failed
__global__ void recur_kernel(const double* __restrict__ hcq_sym, const double* __restrict__ rd,
                             const float* __restrict__ Mh, const float* __restrict__ Ml, const double* __restrict__ M64,
                             int n, int ldm, const int* __restrict__ flag, double* __restrict__ S) {
  if (*flag) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  double mij, mji;
  if (M64) {
    mij = M64[(int64_t)i * ldm + j];
    mji = M64[(int64_t)j * ldm + i];
  } else {
    mij = (double)Mh[(int64_t)i * ldm + j] + (double)Ml[(int64_t)i * ldm + j];
    mji = (double)Mh[(int64_t)j * ldm + i] + (double)Ml[(int64_t)j * ldm + i];
  }
  double v = hcq_sym[t] - rd[i] * rd[j] * 0.5 * (mij + mji);
  if (i == j) v += 2.0 * rd[i];
  S[t] = v;
}

// ---------------------------------------------------------------------------
// single-CTA Cholesky + in-place triangular inverse of an SPD matrix.
// Storage: packed lower triangle in shared memory (n <= kSmemN) or a full
// row-major n x n scratch in global memory (larger n).
// ---------------------------------------------------------------------------
constexpr int kSmemN = 256;

template <typename T>
struct LowerTri {
  T* base;
  int n;
  bool packed;
  __device__ __forceinline__ T& operator()(int i, int j) const {
    return packed ? base[(int64_t)i * (i + 1) / 2 + j] : base[(int64_t)i * n + j];
  }
};

// Outer-product (LDL^T-style) Cholesky, one barrier per column; then L = column k scaled by 1/sqrt(d_k).
// Returns false (uniformly) when a pivot is not positive and finite.
template <typename T>
__device__ bool chol_lower(const LowerTri<T>& A, int n) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    const T dkk = A(k, k);
    if (!(dkk > (T)0) || !(dkk < (T)INFINITY)) return false;
    const T inv = (T)1 / dkk;
    for (int i = k + 1 + ty; i < n; i += nty) {
      const T aik = A(i, k) * inv;
      for (int j = k + 1 + tx; j <= i; j += 32) A(i, j) -= aik * A(j, k);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    // row i: L(i, k) = A(i, k) / sqrt(A(k, k)); done row-wise so no thread races on a column
    for (int k = 0; k < i; ++k) A(i, k) = A(i, k) / sqrt(A(k, k));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) A(k, k) = sqrt(A(k, k));
  __syncthreads();
  return true;
}

// In-place inverse of the lower-triangular L, column by column from the right:
//   X(j, j) = 1 / L(j, j);  X(i, j) = -X(j, j) sum_{k=j+1}^{i} X(i, k) L(k, j),  i > j
template <typename T>
__device__ void trtri_lower(const LowerTri<T>& A, int n, T* __restrict__ col) {
  const int part = threadIdx.x & 3, grp = threadIdx.x >> 2, ngrp = blockDim.x >> 2;
  for (int j = n - 1; j >= 0; --j) {
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) col[i] = A(i, j);
    __syncthreads();
    const T xjj = (T)1 / A(j, j);
    for (int ib = j + 1; ib < n; ib += ngrp) {
      const int i = ib + grp;
      T s = (T)0;
      if (i < n)
        for (int k = j + 1 + part; k <= i; k += 4) s += A(i, k) * col[k];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (i < n && part == 0) A(i, j) = -s * xjj;
    }
    if (threadIdx.x == 0) A(j, j) = xjj;
    __syncthreads();
  }
}

// FP32 factor: Shi/Slo split of S, Cholesky of Shi, X = L^{-1} (full n x n, lower part).
// flag[1] |= 4 on failure (the FP64 factor is wanted).
__global__ void __launch_bounds__(1024) chol32_kernel(const double* __restrict__ S, int n, float* __restrict__ Shi,
                                                      float* __restrict__ Slo, float* __restrict__ Lw,
                                                      float* __restrict__ X, int* __restrict__ flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool packed = n <= kSmemN;
  float* colbuf = reinterpret_cast<float*>(smem_raw);
  LowerTri<float> A{packed ? colbuf + 512 : Lw, n, packed};
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    double v = S[t];
    float hi = (float)v;
    Shi[t] = hi;
    Slo[t] = (float)(v - (double)hi);
    int i = (int)(t / n), j = (int)(t % n);
    if (j <= i) A(i, j) = hi;
  }
  __syncthreads();
  if (!chol_lower<float>(A, n)) {
    if (threadIdx.x == 0) atomicOr(flag + 1, 4);
    return;
  }
  trtri_lower<float>(A, n, colbuf);
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    int i = (int)(t / n), j = (int)(t % n);
    X[t] = j <= i ? A(i, j) : 0.f;
  }
}

// M0 = X^T X (X lower triangular), written as Mh, Ml = 0
__global__ void xtx_kernel(const float* __restrict__ X, int n, int ldm, float* __restrict__ Mh,
                           float* __restrict__ Ml, const int* __restrict__ flag) {
  if (flag[1] & 4) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  float s = 0.f;
  for (int k = max(i, j); k < n; ++k) s += X[(int64_t)k * n + i] * X[(int64_t)k * n + j];
  Mh[(int64_t)i * ldm + j] = s;
  Ml[(int64_t)i * ldm + j] = 0.f;
}

// residual E = I - S M in compensated FP32: S = Shi + Slo, M = Mh + Ml.
// Each thread owns one (i, j); a warp covers consecutive j.
__global__ void residual_kernel(const float* __restrict__ Shi, const float* __restrict__ Slo,
                                const float* __restrict__ Mh, const float* __restrict__ Ml, int n, int ldm,
                                float* __restrict__ E, unsigned* __restrict__ emax, int* __restrict__ flag) {
  if (flag[1] & (4 | 8)) return;  // factor failed / already converged
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  float p = 0.f, s = 0.f;
  for (int k = 0; k < n; ++k) {
    float a = Shi[(int64_t)i * n + k], al = Slo[(int64_t)i * n + k];
    float b = Mh[(int64_t)k * ldm + j], bl = Ml[(int64_t)k * ldm + j];
    float h, r, q;
    two_prod(a, b, h, r);
    two_sum(p, h, p, q);
    s += q + r + (a * bl + al * b);
  }
  // E = (delta_ij - p) - s ; delta_ij - p is exact when p ~ delta_ij
  float e = __fsub_rn(__fsub_rn(i == j ? 1.f : 0.f, p), s);
  E[t] = e;
  float ae = fabsf(e);
  if (!(ae <= 3.0e38f)) ae = 3.0e38f;  // NaN -> huge
  atomicMax(emax, __float_as_uint(ae));
}

// M <- M + M E (converged: max|E| below tol -> stop; diverged -> fallback wanted)
__global__ void correct_kernel(const float* __restrict__ Mh, const float* __restrict__ Ml, const float* __restrict__ E,
                               float* __restrict__ D, int n, int ldm, const unsigned* __restrict__ emax,
                               int* __restrict__ flag, float tol) {
  if (flag[1] & (4 | 8)) return;
  const float em = __uint_as_float(*emax);
  if (em < tol) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flag + 1, 8);
    return;
  }
  if (em > 0.25f) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flag + 1, 4);
    return;
  }
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  float d = 0.f;
  for (int k = 0; k < n; ++k)
    d += (Mh[(int64_t)i * ldm + k] + Ml[(int64_t)i * ldm + k]) * E[(int64_t)k * n + j];
  // other threads still read row i of M, so the correction goes to scratch D and is folded in next
  D[t] = d;
}

// after the last residual: accept the refined inverse or ask for the FP64 factor
__global__ void accept_kernel(const unsigned* __restrict__ emax, int* __restrict__ flag, float accept) {
  if (flag[1] & (4 | 8)) return;
  if (!(__uint_as_float(*emax) <= accept)) atomicOr(flag + 1, 4);
}

__global__ void fold_kernel(float* __restrict__ Mh, float* __restrict__ Ml, const float* __restrict__ D, int n,
                            int ldm, const unsigned* __restrict__ emax, const int* __restrict__ flag, float tol) {
  if (flag[1] & (4 | 8)) return;
  if (__uint_as_float(*emax) < tol) return;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  float h = Mh[(int64_t)i * ldm + j];
  float l = Ml[(int64_t)i * ldm + j] + D[t];
  float s, e;
  two_sum(h, l, s, e);
  Mh[(int64_t)i * ldm + j] = s;
  Ml[(int64_t)i * ldm + j] = e;
}

// FP64 Cholesky + inverse on one CTA (global scratch): the fallback of the FP32 path and the
// factor of FP64 mode. Runs only when `force` or the FP32 factor failed (flag[1] & 4).
__global__ void __launch_bounds__(1024) chol64_kernel(const double* __restrict__ S, int n, double* __restrict__ Lw,
                                                      double* __restrict__ X, double* __restrict__ M64, int ldm,
                                                      float* __restrict__ Mh, float* __restrict__ Ml,
                                                      int* __restrict__ flag, int force) {
  if (!force && !(flag[1] & 4)) return;
  __shared__ double colbuf[kMaxN];
  LowerTri<double> A{Lw, n, false};
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) Lw[t] = S[t];
  __syncthreads();
  if (!chol_lower<double>(A, n)) {
    if (threadIdx.x == 0) atomicOr(flag, 2);  // not positive definite: the step is rejected
    return;
  }
  trtri_lower<double>(A, n, colbuf);
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    int i = (int)(t / n), j = (int)(t % n);
    double s = 0.0;
    for (int k = max(i, j); k < n; ++k) s += A(k, i) * A(k, j);
    if (M64) M64[(int64_t)i * ldm + j] = s;
    if (Mh) {
      float h = (float)s;
      Mh[(int64_t)i * ldm + j] = h;
      Ml[(int64_t)i * ldm + j] = (float)(s - (double)h);
    }
  }
}

// ---------------------------------------------------------------------------
// innovation e = y - H x and a = M e
// ---------------------------------------------------------------------------
__global__ void innovation_kernel(const double* __restrict__ y, const int64_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                  const double* __restrict__ x, int n, double* __restrict__ e,
                                  int* __restrict__ flag) {
  __shared__ double red[kThreads];
  const int r = blockIdx.x;
  double acc = 0.0;
  for (int64_t k = rowptr[r] + threadIdx.x; k < rowptr[r + 1]; k += blockDim.x) acc += val[k] * x[col[k]];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double yv = y[r];
    if (!isfinite(yv)) atomicOr(flag, 1);
    e[r] = yv - red[0];
  }
}

// a = M e (one warp per row); also M32 = round(Mh + Ml) into the padded sweep operand
template <typename T>
__global__ void gemv_kernel(const float* __restrict__ Mh, const float* __restrict__ Ml,
                            const double* __restrict__ M64, int n, int ldm, const double* __restrict__ e,
                            double* __restrict__ a, T* __restrict__ Msw, int nt, const int* __restrict__ flag) {
  if (*flag) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int i = warp;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) {
    double mij = M64 ? M64[(int64_t)i * ldm + j] : (double)Mh[(int64_t)i * ldm + j] + (double)Ml[(int64_t)i * ldm + j];
    acc += mij * e[j];
    Msw[(int64_t)i * nt + j] = (T)mij;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) a[i] = acc;
}

// ---------------------------------------------------------------------------
// the sweep (S4), FP32/FP64 CUDA-core version
// ---------------------------------------------------------------------------
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int N = 4;
};
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int N = 2;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename T, int NT, int TM>
struct SweepCfg {
  static constexpr int VEC = Vec<T>::N;
  static constexpr int BM = 8 * TM;                                  // rows per tile
  static constexpr int TN = NT / 32;                                 // columns per thread
  static constexpr int G = TN / VEC;                                 // vector groups per thread
  static constexpr int BK = 32768 / (2 * NT * (int)sizeof(T));       // M rows per stage
  static constexpr int LDP = NT + VEC;                               // Cp row stride (elements)
  static constexpr size_t SMEM = sizeof(T) * ((size_t)BM * LDP + 2 * (size_t)BK * NT + NT + NT);
};

// Per tile of BM rows: Cp = C + CQ into smem, K = Cp M (M streamed in BK-row stages),
// epilogue: rowdot, x update, C <- K R.
// (sh, sl) += (ph, pl) in double-float arithmetic (TwoSum, then renormalise)
__device__ __forceinline__ void df_add(float& sh, float& sl, float ph, float pl) {
  const float s = sh + ph;
  const float bb = s - sh;
  float e = (sh - (s - bb)) + (ph - bb);
  e += sl + pl;
  sh = s + e;
  sl = e - (sh - s);
}

template <typename T, int NT, int TM>
__global__ void __launch_bounds__(256) sweep_kernel(int64_t m, int ld, int n, const T* __restrict__ CQ,
                                                    T* __restrict__ C, const T* __restrict__ Msw,
                                                    const double* __restrict__ a_in, const double* __restrict__ rd,
                                                    double theta, double* __restrict__ x,
                                                    double* __restrict__ var, const int* __restrict__ flag) {
  using Cfg = SweepCfg<T, NT, TM>;
  using V = typename Vec<T>::V;
  constexpr int VEC = Cfg::VEC, BM = Cfg::BM, TN = Cfg::TN, G = Cfg::G, BK = Cfg::BK, LDP = Cfg::LDP;
  if (*flag) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Cp = reinterpret_cast<T*>(smem_raw);   // BM x LDP
  T* Ms = Cp + BM * LDP;                    // 2 x BK x NT
  T* as = Ms + 2 * BK * NT;                 // NT: a
  T* rs = as + NT;                          // NT: diag R
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  for (int j = tid; j < NT; j += 256) {
    as[j] = j < n ? (T)a_in[j] : (T)0;
    rs[j] = j < n ? (T)rd[j] : (T)0;
  }
  const int64_t ntiles = (m + BM - 1) / BM;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * BM;
    __syncthreads();  // previous tile's smem reads are done
    // stage 0 of M
    auto load_m = [&](int stage, int k0) {
      T* dst = Ms + stage * BK * NT;
      for (int v = tid; v < BK * NT / VEC; v += 256) {
        int kk = v / (NT / VEC), cv = v % (NT / VEC);
        cp_async16(dst + kk * NT + cv * VEC, Msw + (int64_t)(k0 + kk) * NT + cv * VEC, 16);
      }
      cp_async_commit();
    };
    load_m(0, 0);
    // C tile -> smem (async), then add CQ
    for (int v = tid; v < BM * NT / VEC; v += 256) {
      int r = v / (NT / VEC), cv = v % (NT / VEC);
      int64_t grow = row0 + r;
      bool ok = grow < m && cv * VEC < ld;
      const T* src = ok ? C + grow * ld + cv * VEC : C;
      cp_async16(Cp + r * LDP + cv * VEC, src, ok ? 16 : 0);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll 4
    for (int v = tid; v < BM * NT / VEC; v += 256) {
      int r = v / (NT / VEC), cv = v % (NT / VEC);
      int64_t grow = row0 + r;
      if (grow < m && cv * VEC < ld) {
        V q = *reinterpret_cast<const V*>(CQ + grow * ld + cv * VEC);
        V* p = reinterpret_cast<V*>(Cp + r * LDP + cv * VEC);
        V c = *p;
        const T* qa = reinterpret_cast<const T*>(&q);
        T* ca = reinterpret_cast<T*>(&c);
#pragma unroll
        for (int w = 0; w < VEC; ++w) ca[w] += qa[w];
        *p = c;
      }
    }
    // (visibility of Cp is ensured by the __syncthreads inside the k loop)
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;
    constexpr int NK = NT / BK;
    for (int kb = 0; kb < NK; ++kb) {
      if (kb + 1 < NK) {
        load_m((kb + 1) & 1, (kb + 1) * BK);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const T* Mb = Ms + (kb & 1) * BK * NT;
#pragma unroll
      for (int kk = 0; kk < BK; kk += VEC) {
        T av[TM][VEC];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          V t = *reinterpret_cast<const V*>(Cp + (ty * TM + i) * LDP + kb * BK + kk);
          const T* ta = reinterpret_cast<const T*>(&t);
#pragma unroll
          for (int w = 0; w < VEC; ++w) av[i][w] = ta[w];
        }
#pragma unroll
        for (int w = 0; w < VEC; ++w) {
          T bv[TN];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            V t = *reinterpret_cast<const V*>(Mb + (kk + w) * NT + g * 32 * VEC + tx * VEC);
            const T* ta = reinterpret_cast<const T*>(&t);
#pragma unroll
            for (int u = 0; u < VEC; ++u) bv[g * VEC + u] = ta[u];
          }
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] += av[i][w] * bv[j];
        }
      }
      __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int r = ty * TM + i;
      const int64_t grow = row0 + r;
      // compensated sums of K_ij Cp_ij and Cp_ij a_j over this thread's columns
      T rd_s = (T)0, rd_c = (T)0, xi_s = (T)0, xi_c = (T)0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int c0 = g * 32 * VEC + tx * VEC;
        V t = *reinterpret_cast<const V*>(Cp + r * LDP + c0);
        const T* cp = reinterpret_cast<const T*>(&t);
        V out;
        T* oa = reinterpret_cast<T*>(&out);
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const T k = acc[i][g * VEC + u];
          T y1 = k * cp[u] - rd_c;
          T t1 = rd_s + y1;
          rd_c = (t1 - rd_s) - y1;
          rd_s = t1;
          T y2 = cp[u] * as[c0 + u] - xi_c;
          T t2 = xi_s + y2;
          xi_c = (t2 - xi_s) - y2;
          xi_s = t2;
          oa[u] = k * rs[c0 + u];
        }
        if (grow < m && c0 < ld) *reinterpret_cast<V*>(C + grow * ld + c0) = out;
      }
      double rdv, xiv;
      if (sizeof(T) == 4) {
        // across the lanes in double-float (FP32 pairs; the Kahan pair (s, c) holds s - c):
        // the FP64 rate of this part is low, so only the row's final value is FP64
        float rh = (float)rd_s, rl = -(float)rd_c, xh = (float)xi_s, xl = -(float)xi_c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float a = __shfl_xor_sync(0xffffffffu, rh, o), al = __shfl_xor_sync(0xffffffffu, rl, o);
          const float b = __shfl_xor_sync(0xffffffffu, xh, o), bl = __shfl_xor_sync(0xffffffffu, xl, o);
          df_add(rh, rl, a, al);
          df_add(xh, xl, b, bl);
        }
        rdv = (double)rh + (double)rl;
        xiv = (double)xh + (double)xl;
      } else {
        rdv = (double)rd_s - (double)rd_c;
        xiv = (double)xi_s - (double)xi_c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          rdv += __shfl_xor_sync(0xffffffffu, rdv, o);
          xiv += __shfl_xor_sync(0xffffffffu, xiv, o);
        }
      }
      if (tx == 0 && grow < m) {
        var[grow] += theta - rdv;
        x[grow] += xiv;
      }
    }
  }
}

template <typename T, int NT, int TM>
Status sweep_config(int* per_sm_out) {
  using Cfg = SweepCfg<T, NT, TM>;
  auto fn = sweep_kernel<T, NT, TM>;
  static int per_sm = 0;  // resolved once per instantiation, at create (outside any graph capture)
  if (per_sm == 0) {
    HIKF_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    int v = 1;
    HIKF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, 256, Cfg::SMEM));
    per_sm = std::max(v, 1);
  }
  *per_sm_out = per_sm;
  return Status::Ok();
}

template <typename T, int NT, int TM>
Status launch_sweep_t(const SweepArgs<T>& s, cudaStream_t st, int sms) {
  using Cfg = SweepCfg<T, NT, TM>;
  auto fn = sweep_kernel<T, NT, TM>;
  int per_sm = 1;
  HIKF_TRY((sweep_config<T, NT, TM>(&per_sm)));
  int64_t ntiles = (s.m + Cfg::BM - 1) / Cfg::BM;
  int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
  grid = std::max(grid, 1);
  fn<<<grid, 256, Cfg::SMEM, st>>>(s.m, s.ld, s.n, s.CQ, s.C, s.Msw, s.a, s.rd, s.theta, s.x, s.var, s.flag);
  HIKF_LAUNCH_CHECK("sweep");
  return Status::Ok();
}

}  // namespace

int sweep_nt(int ld) {
  if (ld <= 128) return 128;
  if (ld <= 256) return 256;
  return 512;
}

template <typename T>
Status launch_sweep(const SweepArgs<T>& s, cudaStream_t st, int sms) {
  const int nt = sweep_nt(s.ld);
  if (sizeof(T) == 4) {
    if (nt == 128) return launch_sweep_t<T, 128, 8>(s, st, sms);
    if (nt == 256) return launch_sweep_t<T, 256, 8>(s, st, sms);
    return launch_sweep_t<T, 512, 4>(s, st, sms);
  } else {
    if (nt == 128) return launch_sweep_t<T, 128, 8>(s, st, sms);
    if (nt == 256) return launch_sweep_t<T, 256, 4>(s, st, sms);
    return launch_sweep_t<T, 512, 2>(s, st, sms);
  }
}

template Status launch_sweep<float>(const SweepArgs<float>&, cudaStream_t, int);

template <typename T>
Status prepare_sweep(int ld) {
  const int nt = sweep_nt(ld);
  int v = 0;
  if (sizeof(T) == 4) {
    if (nt == 128) return sweep_config<T, 128, 8>(&v);
    if (nt == 256) return sweep_config<T, 256, 8>(&v);
    return sweep_config<T, 512, 4>(&v);
  }
  if (nt == 128) return sweep_config<T, 128, 8>(&v);
  if (nt == 256) return sweep_config<T, 256, 4>(&v);
  return sweep_config<T, 512, 2>(&v);
}
template Status prepare_sweep<float>(int);
template Status prepare_sweep<double>(int);

Status prepare_chain() {
  HIKF_CUDA(cudaFuncSetAttribute((const void*)chol32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * (512 + (size_t)kSmemN * (kSmemN + 1) / 2))));
  return Status::Ok();
}
template Status launch_sweep<double>(const SweepArgs<double>&, cudaStream_t, int);

template <typename T>
Status launch_gather_hc(const SparseH& h, const T* C, int ld, double* out, int accumulate, cudaStream_t s) {
  gather_hc_kernel<T><<<h.n, 256, 0, s>>>(h.rowptr, h.col, h.val, C, ld, h.n, out, accumulate);
  HIKF_LAUNCH_CHECK("gather_hc");
  return Status::Ok();
}
template Status launch_gather_hc<float>(const SparseH&, const float*, int, double*, int, cudaStream_t);
template Status launch_gather_hc<double>(const SparseH&, const double*, int, double*, int, cudaStream_t);

Status launch_form_s(const double* A, const double* rd, int n, double* S, cudaStream_t s) {
  form_s_kernel<<<nblk((int64_t)n * n, kThreads), kThreads, 0, s>>>(A, rd, n, S);
  HIKF_LAUNCH_CHECK("form_s");
  return Status::Ok();
}

Status launch_chain(const ChainArgs& c, cudaStream_t s) {
  const int n = c.n;
  const int64_t nn = (int64_t)n * n;
  HIKF_CUDA(cudaMemsetAsync(c.flag + 1, 0, sizeof(int), s));  // factor-path bits of this step
  if (c.fp64) {
    chol64_kernel<<<1, 1024, 0, s>>>(c.S, n, c.L64, c.X64, c.M64, c.ldm, nullptr, nullptr, c.flag, 1);
    HIKF_LAUNCH_CHECK("chol64");
    return Status::Ok();
  }
  {
    size_t sm = n <= kSmemN ? sizeof(float) * (512 + (size_t)n * (n + 1) / 2) : sizeof(float) * 512;
    chol32_kernel<<<1, 1024, sm, s>>>(c.S, n, c.Shi, c.Slo, c.L32, c.X32, c.flag);
  }
  HIKF_LAUNCH_CHECK("chol32");
  xtx_kernel<<<nblk(nn, kThreads), kThreads, 0, s>>>(c.X32, n, c.ldm, c.Mh, c.Ml, c.flag);
  HIKF_LAUNCH_CHECK("xtx");
  for (int it = 0; it < c.refine_iters; ++it) {
    HIKF_CUDA(cudaMemsetAsync(c.emax, 0, sizeof(unsigned), s));
    residual_kernel<<<nblk(nn, kThreads), kThreads, 0, s>>>(c.Shi, c.Slo, c.Mh, c.Ml, n, c.ldm, c.E, c.emax, c.flag);
    HIKF_LAUNCH_CHECK("residual");
    correct_kernel<<<nblk(nn, kThreads), kThreads, 0, s>>>(c.Mh, c.Ml, c.E, c.E + nn, n, c.ldm, c.emax, c.flag,
                                                           c.tol);
    HIKF_LAUNCH_CHECK("correct");
    fold_kernel<<<nblk(nn, kThreads), kThreads, 0, s>>>(c.Mh, c.Ml, c.E + nn, n, c.ldm, c.emax, c.flag, c.tol);
    HIKF_LAUNCH_CHECK("fold");
  }
  // the last residual must be small; otherwise fall back to FP64
  HIKF_CUDA(cudaMemsetAsync(c.emax, 0, sizeof(unsigned), s));
  residual_kernel<<<nblk(nn, kThreads), kThreads, 0, s>>>(c.Shi, c.Slo, c.Mh, c.Ml, n, c.ldm, c.E, c.emax, c.flag);
  HIKF_LAUNCH_CHECK("residual");
  accept_kernel<<<1, 1, 0, s>>>(c.emax, c.flag, c.accept);
  HIKF_LAUNCH_CHECK("accept");
  chol64_kernel<<<1, 1024, 0, s>>>(c.S, n, c.L64, c.X64, nullptr, c.ldm, c.Mh, c.Ml, c.flag, 0);
  HIKF_LAUNCH_CHECK("chol64");
  return Status::Ok();
}

}  // namespace hikf

namespace hikf {

Status launch_innovation(const double* y, const SparseH& h, const double* x, double* e, int* flag, cudaStream_t s) {
  innovation_kernel<<<h.n, kThreads, 0, s>>>(y, h.rowptr, h.col, h.val, x, h.n, e, flag);
  HIKF_LAUNCH_CHECK("innovation");
  return Status::Ok();
}

template <typename T>
Status launch_gemv(const float* Mh, const float* Ml, const double* M64, int n, int ldm, const double* e, double* a,
                   T* Msw, int nt, const int* flag, cudaStream_t s) {
  gemv_kernel<T><<<nblk((int64_t)n * 32, kThreads), kThreads, 0, s>>>(Mh, Ml, M64, n, ldm, e, a, Msw, nt, flag);
  HIKF_LAUNCH_CHECK("gemv");
  return Status::Ok();
}
template Status launch_gemv<float>(const float*, const float*, const double*, int, int, const double*, double*,
                                   float*, int, const int*, cudaStream_t);
template Status launch_gemv<double>(const float*, const float*, const double*, int, int, const double*, double*,
                                    double*, int, const int*, cudaStream_t);

Status launch_recur(const double* hcq_sym, const double* rd, const float* Mh, const float* Ml, const double* M64,
                    int n, int ldm, const int* flag, double* S, cudaStream_t s) {
  recur_kernel<<<nblk((int64_t)n * n, kThreads), kThreads, 0, s>>>(hcq_sym, rd, Mh, Ml, M64, n, ldm, flag, S);
  HIKF_LAUNCH_CHECK("recur");
  return Status::Ok();
}

}  // namespace hikf

namespace hikf {

// ---------------------------------------------------------------------------
// dense R: the whitening factors of R = L L^T (FP64, one CTA): L^T, L^{-1} and L^{-T}
// (full n x n, zeros outside the triangle); flag[0] |= 2 when R is not positive definite
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) whiten_factors_kernel(const double* __restrict__ R, int n,
                                                              double* __restrict__ W1, double* __restrict__ W2,
                                                              double* __restrict__ Linv, double* __restrict__ LinvT,
                                                              double* __restrict__ LT, int* __restrict__ flag) {
  __shared__ double colbuf[kMaxN];
  const int64_t nn = (int64_t)n * n;
  for (int64_t t = threadIdx.x; t < nn; t += blockDim.x) W1[t] = R[t];
  __syncthreads();
  LowerTri<double> A{W1, n, false};
  if (!chol_lower<double>(A, n)) {
    if (threadIdx.x == 0) atomicOr(flag, 2);
    return;
  }
  for (int64_t t = threadIdx.x; t < nn; t += blockDim.x) W2[t] = W1[t];
  __syncthreads();
  LowerTri<double> X{W2, n, false};
  trtri_lower<double>(X, n, colbuf);
  __syncthreads();
  for (int64_t t = threadIdx.x; t < nn; t += blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const double l = j <= i ? W1[t] : 0.0;
    const double li = j <= i ? W2[t] : 0.0;
    Linv[t] = li;
    LinvT[(int64_t)j * n + i] = li;
    LT[(int64_t)j * n + i] = l;
  }
}

// out = L^{-1} in (n-vectors, L^{-1} lower triangular): one warp per row
__global__ void whiten_vec_kernel(const double* __restrict__ Linv, const double* __restrict__ in, int n,
                                  double* __restrict__ out) {
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  double acc = 0.0;
  for (int j = lane; j <= i; j += 32) acc += Linv[(int64_t)i * n + j] * in[j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[i] = acc;
}

// out = L^{-1} A (n x n): one thread per output entry
__global__ void left_lower_kernel(const double* __restrict__ Linv, const double* __restrict__ A, int n,
                                  double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  double acc = 0.0;
  for (int k = 0; k <= i; ++k) acc += Linv[(int64_t)i * n + k] * A[(int64_t)k * n + j];
  out[t] = acc;
}

Status launch_whiten_factors(const double* R, int n, double* W1, double* W2, double* Linv, double* LinvT, double* LT,
                             int* flag, cudaStream_t s) {
  HIKF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * 2, s));
  whiten_factors_kernel<<<1, 1024, 0, s>>>(R, n, W1, W2, Linv, LinvT, LT, flag);
  HIKF_LAUNCH_CHECK("whiten_factors");
  return Status::Ok();
}

Status launch_whiten_vec(const double* Linv, const double* in, int n, double* out, cudaStream_t s) {
  whiten_vec_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(Linv, in, n, out);
  HIKF_LAUNCH_CHECK("whiten_vec");
  return Status::Ok();
}

Status launch_left_lower(const double* Linv, const double* A, int n, double* out, cudaStream_t s) {
  const int64_t nn = (int64_t)n * n;
  left_lower_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Linv, A, n, out);
  HIKF_LAUNCH_CHECK("left_lower");
  return Status::Ok();
}

Status spd_inverse_f64(const double* S, int n, double* M, double* scratch, int* flag, cudaStream_t s) {
  HIKF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * 2, s));
  // force = 1: factor S itself; the inverse goes to M (ldm = n)
  chol64_kernel<<<1, 1024, 0, s>>>(S, n, scratch, nullptr, M, n, nullptr, nullptr, flag, 1);
  HIKF_LAUNCH_CHECK("chol64");
  return Status::Ok();
}

}  // namespace hikf

// ---------------------------------------------------------------------------
// S^{-1} without device allocation: the scratch of the FP64 factor is a static
// device array (HIKF_NOALLOC_MAX_N^2 FP64) shared by all calls on a device.
// ---------------------------------------------------------------------------
#include <mutex>

namespace hikf {
namespace {

__device__ __align__(256) double g_noalloc_scratch[HIKF_NOALLOC_MAX_N * HIKF_NOALLOC_MAX_N];
__device__ __align__(256) int g_noalloc_flag[4];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_scratch_ptr[kMaxDevices];
int* g_noalloc_flag_ptr[kMaxDevices];

// device addresses of the static scratch on the current device, resolved once per device
Status noalloc_scratch(double** scratch, int** flag) {
  int dev = 0;
  HIKF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return make_status(HIKF_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_scratch_ptr[dev]) {
    void* a = nullptr;
    void* b = nullptr;
    HIKF_CUDA(cudaGetSymbolAddress(&a, g_noalloc_scratch));
    HIKF_CUDA(cudaGetSymbolAddress(&b, g_noalloc_flag));
    g_noalloc_scratch_ptr[dev] = (double*)a;
    g_noalloc_flag_ptr[dev] = (int*)b;
  }
  *scratch = g_noalloc_scratch_ptr[dev];
  *flag = g_noalloc_flag_ptr[dev];
  return Status::Ok();
}

}  // namespace
}  // namespace hikf

extern "C" hikf_status hikf_spd_inverse_noalloc(const double* d_S, int n, double* d_M, void* stream) {
  using hikf::Status;
  using hikf::make_status;
  using hikf::set_global_error;
  if (!d_S || !d_M) return set_global_error(make_status(HIKF_EINVAL, "null matrix pointer"));
  if (n < 1 || n > HIKF_NOALLOC_MAX_N)
    return set_global_error(make_status(HIKF_EINVAL, "n out of range [1, 256] (the size of the static scratch)"));
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  int* flag = nullptr;
  Status st = hikf::noalloc_scratch(&scratch, &flag);
  if (st.ok()) st = hikf::spd_inverse_f64(d_S, n, d_M, scratch, flag, s);  // clears the status word first
  int f[2] = {0, 0};
  if (st.ok()) {
    cudaError_t e = cudaMemcpyAsync(f, flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = hikf::cuda_status(e, "spd_inverse_noalloc", __FILE__, __LINE__);
  }
  if (!st.ok()) return set_global_error(st);
  if (f[0] & 2) return set_global_error(make_status(HIKF_ENOTPD, "matrix is not positive definite"));
  return HIKF_OK;
}
