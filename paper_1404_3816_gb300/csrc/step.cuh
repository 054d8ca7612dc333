// Launchers of the measurement-update kernels (internal).
#pragma once

#include "hikf_internal.cuh"

namespace hikf {

// Arguments of the sweep (S4): all device pointers, tree order.
template <typename T>
struct SweepArgs {
  int64_t m = 0;
  int ld = 0;              // row stride of C and CQ (padded n)
  int n = 0;
  const T* CQ = nullptr;   // m x ld
  T* C = nullptr;          // m x ld, updated in place
  const T* Msw = nullptr;  // NT x NT (NT = sweep_nt(ld)), zero outside n x n
  const double* a = nullptr;   // n
  const double* rd = nullptr;  // n, diag R
  double theta = 0.0;          // diag Q
  double* x = nullptr;         // m
  double* var = nullptr;       // m
  const int* flag = nullptr;   // step error flag: nonzero -> no-op
};

// Arguments of the n x n chain (S3).
struct ChainArgs {
  int n = 0;
  int ldm = 0;               // row stride of Mh / Ml / M64
  const double* S = nullptr; // n x n
  float* Shi = nullptr;      // n x n
  float* Slo = nullptr;
  float* L32 = nullptr;      // n x n scratch
  float* X32 = nullptr;      // n x n scratch
  float* E = nullptr;        // 2 n x n scratch
  float* Mh = nullptr;       // n x ldm
  float* Ml = nullptr;
  double* L64 = nullptr;     // n x n scratch (FP64 factor)
  double* X64 = nullptr;
  double* M64 = nullptr;     // n x ldm (FP64 mode)
  unsigned* emax = nullptr;
  int* flag = nullptr;       // [0] step error bits, [1] factor-path bits
  int refine_iters = 3;
  float tol = 1e-9f;         // refinement stops below this max |I - S M|
  float accept = 1e-6f;      // larger final residual -> FP64 factor
  int fp64 = 0;
};

int sweep_nt(int ld);

template <typename T>
Status launch_sweep(const SweepArgs<T>& s, cudaStream_t st, int sms);
// launch attributes resolved at create (so that the update can be captured as a graph)
template <typename T>
Status prepare_sweep(int ld);
Status prepare_chain();

template <typename T>
Status launch_gather_hc(const SparseH& h, const T* C, int ld, double* out, int accumulate, cudaStream_t s);

Status launch_form_s(const double* A, const double* rd, int n, double* S, cudaStream_t s);
Status launch_chain(const ChainArgs& c, cudaStream_t s);
Status launch_innovation(const double* y, const SparseH& h, const double* x, double* e, int* flag, cudaStream_t s);
template <typename T>
Status launch_gemv(const float* Mh, const float* Ml, const double* M64, int n, int ldm, const double* e, double* a,
                   T* Msw, int nt, const int* flag, cudaStream_t s);
Status launch_recur(const double* hcq_sym, const double* rd, const float* Mh, const float* Ml, const double* M64,
                    int n, int ldm, const int* flag, double* S, cudaStream_t s);

// Dense R = L L^T: L^{-1}, L^{-T} and L^T (n x n FP64 each, zeros outside the triangle), W1 and W2
// n x n scratch; flag[0] & 2 when R is not positive definite.
Status launch_whiten_factors(const double* R, int n, double* W1, double* W2, double* Linv, double* LinvT, double* LT,
                             int* flag, cudaStream_t s);
// out = L^{-1} in (n-vectors; in != out)
Status launch_whiten_vec(const double* Linv, const double* in, int n, double* out, cudaStream_t s);
// out = L^{-1} A (n x n; A != out)
Status launch_left_lower(const double* Linv, const double* A, int n, double* out, cudaStream_t s);

// Standalone S^{-1} (FP64 Cholesky on one CTA): scratch n x n FP64, flag 2 ints (flag[0] & 2: not PD).
Status spd_inverse_f64(const double* S, int n, double* M, double* scratch, int* flag, cudaStream_t s);

}  // namespace hikf
