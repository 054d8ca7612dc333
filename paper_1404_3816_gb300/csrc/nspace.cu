// n-space form of the filter (see below); the spectral state and the eigenbasis
// form it builds on are in spectral.cu.
#include <math.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "spectral.cuh"

// ---------------------------------------------------------------------------
// n-space form. Under the spectral condition with P_0 = c Q the rotated state is
// G_{t|t} = Gq diag(gamma_t) with Gq = C_Q W fixed: G_0 = c Gq, and one step maps
// G_p = G + Gq = Gq diag(gamma + 1) to G_p diag(g_t), so gamma_{t} = (gamma_{t-1} + 1) g_t.
// The mean and the variance then stay linear in Gq:
//   x_t = x_0 + Gq b_t,              b_t = b_{t-1} + (gamma_{t-1} + 1) o u_t,
//   delta^2_t = delta^2_0 + t theta - sum_k h_k,t Gq_ik^2,   h_t = h_{t-1} + g_t o (gamma_{t-1} + 1)^2,
// and the innovation needs only H x_t = H x_0 + (H Gq) b_t. A step is O(n^2) (two n x n
// products, no pass over the m rows); x and delta^2 are formed on request in one pass
// over Gq, and C_{t|t} = Gq diag(gamma) W^T R likewise.
// ---------------------------------------------------------------------------
namespace hikf {
namespace {

inline int nb(int64_t n, int t) { return (int)((n + t - 1) / t); }

// e = y - H x_0 - P b  (P = H Gq, n x n), one warp per row; non-finite y -> flag bit 1
__global__ void nspace_innovation_kernel(const double* __restrict__ y, const double* __restrict__ hx0,
                                         const double* __restrict__ P, const double* __restrict__ b, int n,
                                         double* __restrict__ e, int* __restrict__ flag) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= n) return;
  double acc = 0.0;
  for (int c = lane; c < n; c += 32) acc += P[(int64_t)r * n + c] * b[c];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const double yv = y[r];
    if (!isfinite(yv)) atomicOr(flag, 1);
    e[r] = yv - hx0[r] - acc;
  }
}

// per eigen-direction: b += (gamma + 1) u, h += g (gamma + 1)^2, gamma <- (gamma + 1) g,
// s <- lambda + 2 - g (u = g W^T e is already formed); counts the applied step
__global__ void nspace_update_kernel(const double* __restrict__ lam, double* __restrict__ s,
                                     const double* __restrict__ u, double* __restrict__ gam, double* __restrict__ b,
                                     double* __restrict__ h, int n, const int* __restrict__ flag,
                                     long long* __restrict__ step) {
  if (*flag) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) *step += 1;
  if (k >= n) return;
  const double g = 1.0 / s[k];
  const double gp = gam[k] + 1.0;
  b[k] += gp * u[k];
  h[k] += g * gp * gp;
  gam[k] = gp * g;
  s[k] = lam[k] + 2.0 - g;
}

// double-float helpers (FP32 pairs): error-free sum and product
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void dd_add(float& sh, float& sl, float ph, float pl) {
  float s, e;
  two_sum(sh, ph, s, e);
  e += sl + pl;
  sh = s + e;
  sl = e - (sh - s);
}

// x = x_0 + Gq b, delta^2 = delta^2_0 + t theta - sum_k h_k Gq_ik^2.
// FP32 Gq: four lanes per row, each lane takes float4 column groups 4 (lane & 3) + 16 j
// (so a warp reads 64 contiguous bytes of each of 8 rows per load; four such loads in
// flight per lane, since one at a time left the SM too few bytes in flight for HBM); Gq b by FP32 products
// with a compensated sum (b as an FP32 pair), h Gq^2 with the square exact (TwoProd) and a
// double-float sum, since delta^2_t is a small difference of large terms; FP64 result.
// FP64 Gq: one warp per row in FP64.
__global__ void __launch_bounds__(256) nspace_outputs_f32_kernel(const float* __restrict__ Gq, int64_t m, int ld,
                                                                 int n, const double* __restrict__ x0, double var0,
                                                                 double theta, const long long* __restrict__ step,
                                                                 const double* __restrict__ b,
                                                                 const double* __restrict__ h,
                                                                 double* __restrict__ x, double* __restrict__ var) {
  __shared__ __align__(16) float sbh[kMaxN], sbl[kMaxN], shh[kMaxN], shl[kMaxN];
  for (int k = threadIdx.x; k < kMaxN; k += blockDim.x) {
    const double bv = k < n ? b[k] : 0.0, hv = k < n ? h[k] : 0.0;
    sbh[k] = (float)bv;
    sbl[k] = (float)(bv - (double)sbh[k]);
    shh[k] = (float)hv;
    shl[k] = (float)(hv - (double)shh[k]);
  }
  __syncthreads();
  const double tq = (double)*step * theta;
  const int lane = threadIdx.x & 31, sub = lane & 3;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x >> 2);
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 2; i - (lane >> 2) < m; i += groups) {
    const bool live = i < m;
    float xs = 0.f, xc = 0.f, vh = 0.f, vl = 0.f;
    if (live) {
      const float4* gr = reinterpret_cast<const float4*>(Gq + i * ld);
      // four loads of the row in flight per lane (the sums then take them in column order)
      for (int c0 = 4 * sub; c0 < n; c0 += 64) {
        float4 gq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (c0 + 16 * k < n) gq[k] = __ldcs(gr + ((c0 + 16 * k) >> 2));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = c0 + 16 * k;
          if (c >= n) break;
          const float4 g4 = gq[k];
          const float4 bh = *reinterpret_cast<const float4*>(sbh + c);
          const float4 bl = *reinterpret_cast<const float4*>(sbl + c);
          const float4 hh = *reinterpret_cast<const float4*>(shh + c);
          const float4 hl = *reinterpret_cast<const float4*>(shl + c);
          const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
          const float bhv[4] = {bh.x, bh.y, bh.z, bh.w}, blv[4] = {bl.x, bl.y, bl.z, bl.w};
          const float hhv[4] = {hh.x, hh.y, hh.z, hh.w}, hlv[4] = {hl.x, hl.y, hl.z, hl.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            // x: FMA product, Kahan-compensated sum
            const float p = fmaf(gv[u], bhv[u], gv[u] * blv[u]);
            const float y = p - xc;
            const float t = xs + y;
            xc = (t - xs) - y;
            xs = t;
            // delta^2: (qh + ql) = Gq^2 exactly, times (hh + hl), double-float sum
            const float qh = gv[u] * gv[u];
            const float ql = fmaf(gv[u], gv[u], -qh);
            const float r = qh * hhv[u];
            dd_add(vh, vl, r, fmaf(qh, hhv[u], -r) + (qh * hlv[u] + ql * hhv[u]));
          }
        }
      }
    }
    // combine the four lanes of the row (the Kahan pair (xs, xc) holds xs - xc)
    float xl = -xc;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      const float oxs = __shfl_xor_sync(0xffffffffu, xs, o), oxl = __shfl_xor_sync(0xffffffffu, xl, o);
      const float ovh = __shfl_xor_sync(0xffffffffu, vh, o), ovl = __shfl_xor_sync(0xffffffffu, vl, o);
      dd_add(xs, xl, oxs, oxl);
      dd_add(vh, vl, ovh, ovl);
    }
    if (live && sub == 0) {
      x[i] = x0[i] + ((double)xs + (double)xl);
      var[i] = (var0 + tq) - ((double)vh + (double)vl);
    }
  }
}

__global__ void __launch_bounds__(256) nspace_outputs_f64_kernel(const double* __restrict__ Gq, int64_t m, int ld,
                                                                 int n, const double* __restrict__ x0, double var0,
                                                                 double theta, const long long* __restrict__ step,
                                                                 const double* __restrict__ b,
                                                                 const double* __restrict__ h,
                                                                 double* __restrict__ x, double* __restrict__ var) {
  const double tq = (double)*step * theta;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
    const double* gr = Gq + i * ld;
    double ax = 0.0, av = 0.0;
    for (int k = lane; k < n; k += 32) {
      const double gv = gr[k];
      ax = fma(gv, b[k], ax);
      av = fma(gv * gv, h[k], av);
    }
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      av += __shfl_xor_sync(0xffffffffu, av, o);
    }
    if (lane == 0) {
      x[i] = x0[i] + ax;
      var[i] = (var0 + tq) - av;
    }
  }
}

// B = diag(gamma) W^T R (n x n): B[k][j] = gamma_k W[j][k] r_j
__global__ void nspace_wtr_kernel(const double* __restrict__ W64, const double* __restrict__ rd,
                                  const double* __restrict__ gam, int n, double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  int k = (int)(t / n), j = (int)(t % n);
  out[t] = gam[k] * W64[(int64_t)j * n + k] * rd[j];
}

}  // namespace

Status nspace_step(const SpectralState& sp, const NspaceState& ns, int n, const double* y, double* e, int* flag,
                   long long* step, cudaStream_t s) {
  nspace_innovation_kernel<<<nb((int64_t)n * 32, 256), 256, 0, s>>>(y, ns.hx0, ns.P, ns.b, n, e, flag);
  HIKF_LAUNCH_CHECK("nspace_innovation");
  HIKF_TRY(eigen_u(sp, n, e, flag, s));
  nspace_update_kernel<<<nb(n, 256), 256, 0, s>>>(sp.lam, sp.s, sp.u, ns.gam, ns.b, ns.h, n, flag, step);
  HIKF_LAUNCH_CHECK("nspace_update");
  return Status::Ok();
}

template <typename T>
Status nspace_outputs(const NspaceState& ns, const T* Gq, int64_t m, int ld, int n, const double* x0, double var0,
                      double theta, const long long* step, double* x, double* var, int sms, cudaStream_t s) {
  if (sizeof(T) == 4) {
    const int64_t blocks = std::min<int64_t>((m + 63) / 64, (int64_t)sms * 8);
    nspace_outputs_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float*)Gq, m, ld, n, x0, var0, theta, step,
                                                              ns.b, ns.h, x, var);
  } else {
    const int64_t blocks = std::min<int64_t>((m + 7) / 8, (int64_t)sms * 8);
    nspace_outputs_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>((const double*)Gq, m, ld, n, x0, var0, theta, step,
                                                              ns.b, ns.h, x, var);
  }
  HIKF_LAUNCH_CHECK("nspace_outputs");
  return Status::Ok();
}
template Status nspace_outputs<float>(const NspaceState&, const float*, int64_t, int, int, const double*, double,
                                      double, const long long*, double*, double*, int, cudaStream_t);
template Status nspace_outputs<double>(const NspaceState&, const double*, int64_t, int, int, const double*, double,
                                       double, const long long*, double*, double*, int, cudaStream_t);

template <typename T>
Status nspace_cross(const SpectralState& sp, const NspaceState& ns, const double* rd, int64_t m, int ld, int n,
                    const T* Gq, T* out, cudaStream_t s) {
  double* B = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&B, sizeof(double) * (size_t)n * n, s));
  nspace_wtr_kernel<<<nb((int64_t)n * n, 256), 256, 0, s>>>(sp.W64, rd, ns.gam, n, B);
  HIKF_LAUNCH_CHECK("nspace_wtr");
  HIKF_TRY(gemm_rows_small<T>(Gq, m, ld, n, B, out, s));
  HIKF_CUDA(cudaFreeAsync(B, s));
  return Status::Ok();
}
template Status nspace_cross<float>(const SpectralState&, const NspaceState&, const double*, int64_t, int, int,
                                    const float*, float*, cudaStream_t);
template Status nspace_cross<double>(const SpectralState&, const NspaceState&, const double*, int64_t, int, int,
                                     const double*, double*, cudaStream_t);

}  // namespace hikf
