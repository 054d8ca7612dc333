// Internal declarations of the HiKF CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hikf.h"

namespace hikf {

constexpr int kMaxN = 512;        // measurements (rays) per filter
constexpr int kMaxOrder2D = 12;   // Chebyshev nodes per axis, 2D
constexpr int kMaxOrder3D = 8;    // Chebyshev nodes per axis, 3D
constexpr int kMaxDepth2D = 15;
constexpr int kMaxDepth3D = 10;

// Status carried inside the library: code + message.
struct Status {
  hikf_status code = HIKF_OK;
  std::string msg;
  bool ok() const { return code == HIKF_OK; }
  static Status Ok() { return Status(); }
};

Status make_status(hikf_status c, const std::string& m);
Status cuda_status(cudaError_t e, const char* what, const char* file, int line);
// message returned by hikf_last_error(NULL) (calls that take no handle); returns s.code
hikf_status set_global_error(const Status& s);

#define HIKF_CUDA(call)                                                           \
  do {                                                                            \
    cudaError_t _e = (call);                                                      \
    if (_e != cudaSuccess) return ::hikf::cuda_status(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define HIKF_LAUNCH_CHECK(what)                                                   \
  do {                                                                            \
    cudaError_t _e = cudaGetLastError();                                          \
    if (_e != cudaSuccess) return ::hikf::cuda_status(_e, what, __FILE__, __LINE__); \
  } while (0)

#define HIKF_TRY(expr)                 \
  do {                                         \
    ::hikf::Status _s = (expr);                \
    if (!_s.ok()) return _s;                   \
  } while (0)

// Device memory arena of one handle: every buffer is cudaMalloc'ed at create
// and released at destroy.
// Device memory of the library comes from one stream-ordered pool per device that keeps up
// to kPoolKeepBytes of freed memory for reuse (the next create's scratch and state reuse it
// without mapping pages again); pool_trim_all() returns the cached memory to the device.
constexpr uint64_t kPoolKeepBytes = 16ull << 30;
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);
template <typename T>
inline cudaError_t pool_malloc(T** p, size_t bytes, cudaStream_t s) {
  return pool_malloc(reinterpret_cast<void**>(p), bytes, s);
}
cudaError_t pool_trim_all();

// A handle's long-lived buffers: allocated from the pool in the order of `stream`, released
// in that order by release() (the caller has synchronised the stream first).
struct Arena {
  void* ptrs[64];
  int count = 0;
  int64_t bytes = 0;
  cudaStream_t stream = nullptr;
  Status alloc(void** p, size_t nbytes);
  void release();
};

template <typename T>
inline Status arena_alloc(Arena& a, T** p, size_t count) {
  return a.alloc(reinterpret_cast<void**>(p), count * sizeof(T) + 0);
}

// ---------------------------------------------------------------------------
// Tree (uniform 2^d-tree, Morton order)
// ---------------------------------------------------------------------------
struct Tree {
  int dim = 2;
  int depth = 0;          // L
  int64_t m = 0;
  int64_t nleaf = 0;      // 2^(dim L)
  double lo[3] = {0, 0, 0};
  double side = 1.0;
  int64_t* perm = nullptr;      // [m] tree position -> caller index
  int64_t* iperm = nullptr;     // [m] caller index -> tree position
  int64_t* leaf_start = nullptr;  // [nleaf + 1]
  double* pts = nullptr;        // [m * dim] points in tree order
  int64_t box_offset[kMaxDepth2D + 2];  // first box of level l in the concatenated box arrays
  int64_t nbox_total = 0;
};

// Sparse H in two layouts, columns in tree order.
struct SparseH {
  int n = 0;
  int64_t nnz = 0;
  int64_t* rowptr = nullptr;   // [n+1]   H rows (rays)
  int32_t* col = nullptr;      // [nnz]   tree positions
  double* val = nullptr;       // [nnz]
  int64_t* trowptr = nullptr;  // [m+1]   H^T rows (points in tree order)
  int32_t* tcol = nullptr;     // [nnz]   ray index
  double* tval = nullptr;      // [nnz]
};

struct Workspace;  // scratch used by the build steps

Status build_tree(Tree& t, Arena& arena, const double* d_points_caller, cudaStream_t s);
Status build_sparse(SparseH& h, Arena& arena, const Tree& t, const int64_t* h_rowptr, const int64_t* h_col,
                    const double* h_val, int n, cudaStream_t s);

// ---------------------------------------------------------------------------
// H^2 product (black-box FMM)
// ---------------------------------------------------------------------------
struct FmmParams {
  int order = 8;     // p
  int pow = 1;
  double theta = 1.0;
  double length = 1.0;
  double shape = 1.0;       // GCF exponent p / LOG self-distance r0 (hikf_kernel.shape)
  bool tensor_m2l = false;  // M2L on the tensor cores (FP32 storage only)
  bool autotune = true;     // tensor-core M2L: time the launch variants once per shape
  int sms = 1;
};

// out: rows [row0, row1) of the m x ldc product in tree order (T = float or double), row row0
// first; columns >= n are zero. row1 < 0 means m. Only the target boxes that hold one of those
// rows take part in the downward pass (M2L, L2L, L2P, P2P); the upward pass covers every source.
template <typename T>
Status h2_product(const Tree& t, const SparseH& h, const FmmParams& fp, T* out, int ldc, cudaStream_t s,
                  int64_t row0 = 0, int64_t row1 = -1);

int auto_depth(int64_t m, int dim, int leaf_size);

// ---------------------------------------------------------------------------
// Measurement update
// ---------------------------------------------------------------------------
int padded_ld(int n);  // leading dimension of the m x n matrices

}  // namespace hikf
