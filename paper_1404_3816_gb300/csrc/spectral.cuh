// Spectral form of the n x n chain (internal).
#pragma once

#include "hikf_internal.cuh"

namespace hikf {

struct SpectralState {
  double* lam = nullptr;  // n eigenvalues of D sym(H C_Q) D, D = R^{-1/2}
  int sweeps = 0;         // Jacobi sweeps the eigendecomposition took
  double* s = nullptr;    // n current s_t (eigenvalues of D S_t D)
  double* W64 = nullptr;  // n x n, D V
  float* W32 = nullptr;   // n x n, D V rounded to FP32
  float* Uhi = nullptr;   // n x n, W diag(s)^{-1/2} as FP32 hi + lo (per step)
  float* Ulo = nullptr;
  double* u = nullptr;    // n scratch
};

// Eigendecomposition of D sym(HCQ) D and s_1 = (1 + c) lambda + 1 (flag[0] |= 2 when some s_1 <= 0).
Status spectral_setup(SpectralState& sp, const double* hcq_sym, const double* rd, int n, double c, int* flag,
                      cudaStream_t s);
// a = M_t e and the sweep operand Msw = M_t (row stride nt), M_t = W diag(1/s_t) W^T.
template <typename T>
Status spectral_gain(const SpectralState& sp, int n, const double* e, double* a, T* Msw, int nt, const int* flag,
                     cudaStream_t s);
// s_{t+1} = lambda + 2 - 1/s_t (skipped when the step failed).
Status spectral_next(const SpectralState& sp, int n, int* flag, cudaStream_t s);

// Eigenbasis form of the state: Gq = C_Q W, G = C_0 W = c Gq at create; per step
// u = (W^T e) / s, then one pass G <- (G + Gq) diag(1/s) with the variance and mean updates.
template <typename T>
Status eigen_setup(const SpectralState& sp, const T* CQ, int64_t m, int ld, int n, double c, T* Gq, T* G,
                   cudaStream_t s);
Status eigen_u(const SpectralState& sp, int n, const double* e, const int* flag, cudaStream_t s);
template <typename T>
Status eigen_step(const SpectralState& sp, int64_t m, int ld, int n, T* G, const T* Gq, double theta, double* x,
                  double* var, const int* flag, int sms, cudaStream_t s);
// n-space form: G_{t|t} = Gq diag(gamma), x = x_0 + Gq b, delta^2 = delta^2_0 + t theta - Gq^2 h
struct NspaceState {
  double* gam = nullptr;  // n, gamma_t (gamma_0 = c)
  double* b = nullptr;    // n, mean coefficients
  double* h = nullptr;    // n, variance coefficients
  double* P = nullptr;    // n x n, H Gq
  double* hx0 = nullptr;  // n, H x_0
};
// one step: e = y - H x_0 - P b, u = (W^T e) / s, the coefficient updates and s_{t+1}
Status nspace_step(const SpectralState& sp, const NspaceState& ns, int n, const double* y, double* e, int* flag,
                   long long* step, cudaStream_t s);
// x and delta^2 of the current state, one pass over Gq
template <typename T>
Status nspace_outputs(const NspaceState& ns, const T* Gq, int64_t m, int ld, int n, const double* x0, double var0,
                      double theta, const long long* step, double* x, double* var, int sms, cudaStream_t s);
// C_{t|t} = Gq diag(gamma) W^T R
template <typename T>
Status nspace_cross(const SpectralState& sp, const NspaceState& ns, const double* rd, int64_t m, int ld, int n,
                    const T* Gq, T* out, cudaStream_t s);

// out (m x ld) = A (m x ld, first n columns) * B (n x n FP64), padding columns zeroed
template <typename T>
Status gemm_rows_small(const T* A, int64_t m, int ld, int n, const double* B, T* out, cudaStream_t s);

// the current C_{t|t} = G W^T R
template <typename T>
Status eigen_cross(const SpectralState& sp, const double* rd, int64_t m, int ld, int n, const T* G, const T* Gq,
                   T* out, cudaStream_t s);

}  // namespace hikf
