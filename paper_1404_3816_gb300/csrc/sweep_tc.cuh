// Tensor-core sweep of the measurement update (internal).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "hikf_internal.cuh"

namespace hikf {

// One filter's part of a grouped sweep (the updates of several filters in one launch): its
// tensor maps, sizes and state pointers, and the first tile of the launch's flat tile order.
struct TcItem {
  CUtensorMap mapC, mapCQ, mapCst;
  int64_t m = 0;
  int n = 0, ld = 0;
  double theta = 0.0;
  const float* a32 = nullptr;   // n_t: the gain vector a in FP32, zero past n (written by tc_pack)
  const float* rd32 = nullptr;  // n_t: diag R in FP32, zero past n
  double* x = nullptr;
  double* var = nullptr;
  const int* flag = nullptr;
  int* err = nullptr;
  const int* beta_exp = nullptr;
  const __half* bimg = nullptr;
  float* cmax = nullptr;
  const float* cqmax = nullptr;
  int64_t tile0 = 0;
  int products = 5;             // 5 or 4 (M in three or two pieces); one value per launch
};

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
  int products = 5;             // FP16 products per K step: 5 (M in three pieces) or 4 (two)
  // grouped sweep: the items (device) and the launch's tiles over all of them
  const TcItem* items = nullptr;
  int nitems = 0;
  int64_t ntiles_total = 0;
};

struct TcState {
  int nt = 256;                 // MMA N (128 or 256)
  CUtensorMap mapC, mapCQ;
  CUtensorMap mapCst;           // C, 32-column x 16-row boxes: the epilogue's tile stores
  __half* bimg = nullptr;       // 3 x nt x nt: FP16 images of beta M (three pieces, or two)
  float* cmax = nullptr;
  float* cqmax = nullptr;
  unsigned* mmax = nullptr;     // kAbsBlocks partial maxima of |M|
  int* beta_exp = nullptr;
  float* vec32 = nullptr;       // 2 x nt: a, then diag R, in FP32 (zero past n) for a grouped sweep
  int products = 5;             // FP16 products per K step: 5 (M in three pieces) or 4 (two; set at create)
};

constexpr int kAbsBlocks = 64;

Status tc_setup(TcState& tc, const float* C, const float* CQ, int64_t m, int ld, int n);
Status tc_init_rows(const TcState& tc, const float* C, const float* CQ, int64_t m, int ld, cudaStream_t s);
// The step's B images of beta M, and the FP32 copies of a and diag R (a grouped sweep's)
Status tc_pack(const TcState& tc, const float* Msw, int nt_src, int n, const double* a, const double* rd,
               const int* flag, cudaStream_t s);
Status tc_sweep(const TcState& tc, TcArgs args, int sms, cudaStream_t s);

// Fill a grouped-sweep item from one filter's sweep state and arguments (tile0 left 0).
void tc_item(const TcState& tc, const TcArgs& args, TcItem* item);
// The sweeps of several filters with the same n_t and product count in one launch: `items`
// (device, count items, tile0 set) and their total tiles; nt = 128 or 256, products = 4 or 5;
// a wait that timed out sets every item's err.
Status tc_sweep_grouped(int nt, int products, const TcItem* items, int count, int64_t ntiles_total, int sms,
                        cudaStream_t s);
int tc_nt(const TcState& tc);
// Row tiles of an m-row sweep (the units of a grouped launch's flat tile order).
int64_t tc_tiles(int64_t m);

// Limit (ns) of the sweep's abortable waits for launches enqueued from now on; 0 restores
// the default (about two seconds). Test hook: a tiny limit makes a step time out.
void tc_set_wait_limit(unsigned long long ns);

}  // namespace hikf
