// Tensor-core sweep of the measurement update (internal).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "hikf_internal.cuh"

namespace hikf {

struct TcArgs {
  int64_t m = 0;
  int ld = 0;
  int n = 0;
  float* C = nullptr;           // m x ld, updated in place (written as K R)
  const double* a = nullptr;    // n
  const double* rd = nullptr;   // n, diag R
  double theta = 0.0;           // diag Q
  double* x = nullptr;          // m
  double* var = nullptr;        // m
  const int* flag = nullptr;    // step error flag: nonzero -> no-op
  int* err = nullptr;           // set to 1 when a bounded wait times out
  const int* beta_exp = nullptr;  // scale exponent of M (device)
  const __half* bimg = nullptr;   // 3 pieces x (n_t / 32) chunks of n_t x 32 FP16 images of beta M
  float* cmax = nullptr;        // m: max_j |C_ij| of the current C (row-scale bound)
  const float* cqmax = nullptr; // m: max_j |C_Q,ij|
  unsigned long long wait_ns = 0;  // limit of the abortable waits (set by tc_sweep)
};

struct TcState {
  int nt = 256;                 // MMA N (128 or 256)
  int smem = 0;
  CUtensorMap mapC, mapCQ;
  CUtensorMap mapCst;           // C, 32-column x 16-row boxes: the epilogue's tile stores
  __half* bimg = nullptr;       // 3 x nt x nt FP16 images of beta M (three pieces)
  float* cmax = nullptr;
  float* cqmax = nullptr;
  unsigned* mmax = nullptr;     // kAbsBlocks partial maxima of |M|
  int* beta_exp = nullptr;
};

constexpr int kAbsBlocks = 64;

Status tc_setup(TcState& tc, const float* C, const float* CQ, int64_t m, int ld, int n);
Status tc_init_rows(const TcState& tc, const float* C, const float* CQ, int64_t m, int ld, cudaStream_t s);
Status tc_pack(const TcState& tc, const float* Msw, int nt_src, int n, const int* flag, cudaStream_t s);
Status tc_sweep(const TcState& tc, TcArgs args, int sms, cudaStream_t s);

// Limit (ns) of the sweep's abortable waits for launches enqueued from now on; 0 restores
// the default (about two seconds). Test hook: a tiny limit makes a step time out.
void tc_set_wait_limit(unsigned long long ns);

}  // namespace hikf
