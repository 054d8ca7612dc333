// C ABI of the HiKF library: handle lifetime, precomputation and the
// measurement update (Alg. 2), see include/hikf.h.
#include <math.h>
#include <string.h>

#include <mutex>

#include <algorithm>
#include <chrono>
#include <new>
#include <string>
#include <vector>

#include "hikf_internal.cuh"
#include "spectral.cuh"
#include "step.cuh"
#include "sweep_tc.cuh"

namespace hikf {

Status make_status(hikf_status c, const std::string& m) {
  Status s;
  s.code = c;
  s.msg = m;
  return s;
}

Status cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
  return make_status(e == cudaErrorMemoryAllocation ? HIKF_ENOMEM : HIKF_ECUDA, m);
}

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaError_t pool_for(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mutex);
  if (!g_pools[dev]) {
    cudaMemPoolProps pr;
    memset(&pr, 0, sizeof(pr));
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = cudaMemPoolCreate(&pool, &pr);
    if (e != cudaSuccess) return e;
    uint64_t keep = kPoolKeepBytes;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}
}  // namespace

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  if (e == cudaSuccess) e = pool_for(dev, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t pool_trim_all() {
  std::lock_guard<std::mutex> lk(g_pool_mutex);
  for (cudaMemPool_t pool : g_pools)
    if (pool) {
      cudaError_t e = cudaMemPoolTrimTo(pool, 0);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

Status Arena::alloc(void** p, size_t nbytes) {
  *p = nullptr;
  if (count >= 64) return make_status(HIKF_ENOMEM, "arena full");
  if (nbytes == 0) nbytes = 16;
  cudaError_t e = pool_malloc(p, nbytes, stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_status(e, "device allocation", __FILE__, __LINE__);
  }
  ptrs[count++] = *p;
  bytes += (int64_t)nbytes;
  return Status::Ok();
}

void Arena::release() {
  for (int i = 0; i < count; ++i) cudaFreeAsync(ptrs[i], stream);
  count = 0;
  bytes = 0;
}

int padded_ld(int n) { return (n + 31) / 32 * 32; }

namespace {

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <typename T>
__global__ void rows_to_tree(const double* __restrict__ src, const int64_t* __restrict__ perm, int64_t m, int n,
                             int ld, T* __restrict__ dst) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * ld) return;
  int64_t s = t / ld;
  int c = (int)(t % ld);
  dst[t] = c < n ? (T)src[perm[s] * n + c] : (T)0;
}

template <typename T>
__global__ void rows_to_caller(const T* __restrict__ src, const int64_t* __restrict__ perm, int64_t m, int n, int ld,
                               double* __restrict__ dst) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  int64_t s = t / n;
  int c = (int)(t % n);
  dst[(perm ? perm[s] : s) * n + c] = (double)src[s * ld + c];
}

__global__ void vec_to_caller(const double* __restrict__ src, const int64_t* __restrict__ perm, int64_t m,
                              double* __restrict__ dst) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) dst[perm[s]] = src[s];
}

// the same permutation as a gather (caller index i <- tree position iperm[i]): contiguous
// writes, for outputs written straight into mapped host memory
__global__ void vec_from_tree(const double* __restrict__ src, const int64_t* __restrict__ iperm, int64_t m,
                              double* __restrict__ dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) dst[i] = src[iperm[i]];
}

__global__ void vec_to_tree(const double* __restrict__ src, const int64_t* __restrict__ perm, int64_t m,
                            double* __restrict__ dst) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) dst[s] = src ? src[perm[s]] : 0.0;
}

__global__ void fill_kernel(double* __restrict__ v, int64_t m, double val) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) v[s] = val;
}

// dst = f src. FP32 data is scaled in FP32 (FP64 arithmetic costs this part 64 cycles an
// instruction): the same value as the FP64 product rounded to FP32 whenever f is exact in
// FP32, as the ratios of kernel amplitudes in use are (c = 100)
template <typename T>
__global__ void scale_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t count, T f) {
  // 16 bytes per thread when the buffers are 16-byte aligned (the m x ld matrices are)
  constexpr int kV = 16 / sizeof(T);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
  if (vec) {
    const int64_t i0 = t * kV;
    if (i0 + kV <= count) {
      struct alignas(16) V { T v[kV]; };
      V a = *reinterpret_cast<const V*>(src + i0);
#pragma unroll
      for (int k = 0; k < kV; ++k) a.v[k] *= f;
      *reinterpret_cast<V*>(dst + i0) = a;
    } else {
      for (int64_t i = i0; i < count; ++i) dst[i] = src[i] * f;
    }
  } else {
    for (int64_t i = t * kV; i < count && i < (t + 1) * kV; ++i) dst[i] = src[i] * f;
  }
}

__global__ void count_step(const int* __restrict__ flag, long long* __restrict__ step) {
  if (*flag == 0) *step += 1;
}

thread_local std::string g_create_error;

}  // namespace

hikf_status set_global_error(const Status& s) {
  g_create_error = s.msg;
  return s.code;
}

}  // namespace hikf

using hikf::Status;

struct hikf_handle {
  int dim = 2;
  int64_t m = 0;
  int n = 0;
  int ld = 0;
  int nt = 0;
  int prec = HIKF_PREC_FP32;
  int order = 8;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sms = 1;
  hikf::Arena arena;
  hikf::Tree tree;
  hikf::SparseH H;
  void* C = nullptr;
  void* CQ = nullptr;
  double* x = nullptr;
  double* var = nullptr;
  double theta_q = 0.0;
  double* rd = nullptr;
  double* hcq_sym = nullptr;
  double* S = nullptr;
  hikf::ChainArgs chain;
  bool spectral = false;
  hikf::SpectralState sp;
  hikf::TcState tc;
  bool eigen = false;
  bool nspace = false;       // n-space form (HIKF_FORM_NSPACE): G = Gq diag(gamma)
  hikf::NspaceState ns;
  double* x0t = nullptr;     // x_0 in tree order (n-space form)
  double var0 = 0.0;         // delta^2_0 = theta_0
  long long enq = 0;         // updates enqueued (host count)
  long long clean_at = -1;   // value of enq when the step flag was last read as clear
  long long outs_at = -1;    // value of enq when x, delta^2 were last formed (n-space form)
  void* G = nullptr;   // eigenbasis state (HIKF_FORM_EIGEN), m x ld
  void* Gq = nullptr;  // C_Q W
  void* Msw = nullptr;
  double* e = nullptr;
  double* a = nullptr;
  double* ybuf = nullptr;
  double* outbuf = nullptr;
  long long* dstep = nullptr;
  int* flag = nullptr;
  std::string err;
  // a bounded device wait ran out inside a step: the step wrote part of its tiles in place,
  // so the state is undefined from then on and every later call is refused (HIKF_ESTATE)
  bool dead = false;
  double cond_s = 0.0;       // estimate of cond(S_t) (hikf_info)
  bool qht_only = false;     // hikf_h2_qht: the H^2 product only, no filter state
  // row sharding (hikf_create_shard): the state holds the rank's rows [r0, r0 + m) of m_full
  bool shard = false;
  hikf_shard sh = {0, 1, nullptr, nullptr};
  int64_t r0 = 0, m_full = 0;
  hikf::SparseH Hfull;       // H over all m_full points (the H^2 product); H: the rank's columns
  const double* hx_ext = nullptr;  // step part 2: the summed H x_t
  double* yzero = nullptr;   // n zeros (the partial H x through the innovation kernel)
  // dense R = L L^T: the filter runs on L^{-1} y, L^{-1} H and R = I (hikf_create_dense_r)
  bool whiten = false;
  double* Linv = nullptr;    // n x n, L^{-1}
  double* LT = nullptr;      // n x n, L^T (back to the caller's C = C' L^T)
  double* eraw = nullptr;    // n, the innovation before whitening
  double* yw = nullptr;      // n, L^{-1} y (n-space form)
  double create_ms = 0.0;
  int launches = 0;
  // the update as a CUDA graph (HIKF options.graph)
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraphNode_t gnode[2] = {nullptr, nullptr};
  cudaGraphExec_t gpart[2] = {nullptr, nullptr};  // the step before / after a grouped sweep
  cudaEvent_t bev = nullptr;  // orders this handle's stream against a grouped sweep
  bool capturing = false;  // event records become graph event-record nodes
  // sweep timing (hikf_profile_enable)
  bool prof = false;
  int prof_count = 0;
  std::vector<cudaEvent_t> ev;

  int m2l = HIKF_M2L_AUTO;
  bool fp64() const { return prec == HIKF_PREC_FP64; }
  bool mixed() const { return prec == HIKF_PREC_MIXED; }
  bool tensor_m2l() const { return m2l == HIKF_M2L_TENSOR ? !fp64() : (m2l == HIKF_M2L_AUTO && mixed()); }
};

namespace {

hikf_status fail(hikf_t* h, const Status& s) {
  if (h) h->err = s.msg; else hikf::g_create_error = s.msg;
  return s.code;
}

Status validate_common(int dim, int64_t m, const double* points, int n, const int64_t* rowptr, const int64_t* col,
                       const double* val, const double* r_diag, const double* x0, const hikf_options& o) {
  using hikf::make_status;
  if (dim != 2 && dim != 3) return make_status(HIKF_EINVAL, "dim must be 2 or 3");
  if (m < 1 || m > 2147483647LL) return make_status(HIKF_EINVAL, "m out of range [1, 2^31-1]");
  if (n < 1 || n > hikf::kMaxN) return make_status(HIKF_EINVAL, "n out of range [1, 512]");
  if (!points || !rowptr || !r_diag) return make_status(HIKF_EINVAL, "null input pointer");
  if (rowptr[0] != 0) return make_status(HIKF_EINVAL, "h_rowptr[0] must be 0");
  for (int r = 0; r < n; ++r)
    if (rowptr[r + 1] < rowptr[r]) return make_status(HIKF_EINVAL, "h_rowptr not monotone");
  const int64_t nnz = rowptr[n];
  if (nnz > 0 && (!col || !val)) return make_status(HIKF_EINVAL, "null h_col/h_val");
  if (nnz > 2147483647LL) return make_status(HIKF_EINVAL, "nnz too large");
  for (int64_t k = 0; k < nnz; ++k) {
    if (col[k] < 0 || col[k] >= m) return make_status(HIKF_EINVAL, "h_col index out of range");
    if (!std::isfinite(val[k])) return make_status(HIKF_EINVAL, "non-finite h_val");
  }
  for (int64_t i = 0; i < m * dim; ++i)
    if (!std::isfinite(points[i])) return make_status(HIKF_EINVAL, "non-finite point coordinate");
  for (int r = 0; r < n; ++r)
    if (!(r_diag[r] > 0.0) || !std::isfinite(r_diag[r])) return make_status(HIKF_EINVAL, "r_diag must be > 0");
  if (x0)
    for (int64_t i = 0; i < m; ++i)
      if (!std::isfinite(x0[i])) return make_status(HIKF_EINVAL, "non-finite x0");
  const int pmax = dim == 2 ? hikf::kMaxOrder2D : hikf::kMaxOrder3D;
  if (o.cheb_order < 2 || o.cheb_order > pmax) return make_status(HIKF_EINVAL, "cheb_order out of range");
  if (o.leaf_size < 1) return make_status(HIKF_EINVAL, "leaf_size must be >= 1");
  const int dmax = dim == 2 ? hikf::kMaxDepth2D : hikf::kMaxDepth3D;
  if (o.max_depth > dmax) return make_status(HIKF_EINVAL, "max_depth too large");
  if (o.precision != HIKF_PREC_FP32 && o.precision != HIKF_PREC_FP64 && o.precision != HIKF_PREC_MIXED)
    return make_status(HIKF_EINVAL, "unknown precision");
  if (o.chain < HIKF_CHAIN_AUTO || o.chain > HIKF_CHAIN_SPECTRAL) return make_status(HIKF_EINVAL, "unknown chain");
  if (o.form != HIKF_FORM_CROSS && o.form != HIKF_FORM_EIGEN && o.form != HIKF_FORM_NSPACE &&
      o.form != HIKF_FORM_AUTO)
    return make_status(HIKF_EINVAL, "unknown form");
  if (o.m2l < HIKF_M2L_AUTO || o.m2l > HIKF_M2L_SIMT) return make_status(HIKF_EINVAL, "unknown m2l");
  if (o.sweep_products != 0 && o.sweep_products != 4 && o.sweep_products != 5)
    return make_status(HIKF_EINVAL, "sweep_products must be 0 (automatic), 4 or 5");
  if (o.m2l == HIKF_M2L_TENSOR && o.precision == HIKF_PREC_FP64)
    return make_status(HIKF_EINVAL, "the tensor-core M2L takes FP32 storage (FP32 or MIXED)");
  return Status::Ok();
}

Status validate_kernel(const hikf_kernel& k, bool allow_zero, bool allow_white, bool allow_log) {
  using hikf::make_status;
  const bool white = allow_white && k.pow == HIKF_KERNEL_WHITE;
  const bool fam = k.pow == HIKF_KERNEL_EXP || k.pow == HIKF_KERNEL_GAUSS || k.pow == HIKF_KERNEL_GCF ||
                   (allow_log && k.pow == HIKF_KERNEL_LOG);
  if (!white && !fam)
    return make_status(HIKF_EINVAL, k.pow == HIKF_KERNEL_LOG
                                        ? "the log kernel is a generalised covariance: hikf_h2_qht only"
                                        : (allow_white ? "kernel family must be WHITE, EXP, GAUSS or GCF"
                                                       : "kernel family must be EXP, GAUSS or GCF"));
  if (!std::isfinite(k.theta) || k.theta < 0.0 || (!allow_zero && k.theta == 0.0))
    return make_status(HIKF_EINVAL, "kernel theta out of range");
  if (!white && k.theta != 0.0 && (!(k.length > 0.0) || !std::isfinite(k.length)))
    return make_status(HIKF_EINVAL, "kernel length must be > 0");
  if (k.pow == HIKF_KERNEL_GCF && k.theta != 0.0 && !(k.shape > 0.0 && k.shape <= 2.0))
    return make_status(HIKF_EINVAL, "GCF exponent (shape) must be in (0, 2]");
  if (k.pow == HIKF_KERNEL_LOG && k.theta != 0.0 && !(k.shape > 0.0 && std::isfinite(k.shape)))
    return make_status(HIKF_EINVAL, "log kernel: the self-distance r0 (shape) must be > 0");
  return Status::Ok();
}

// the same covariance function up to its scale theta (P_0 = c Q)
bool same_shape(const hikf_kernel& a, const hikf_kernel& b) {
  return a.pow == b.pow && a.length == b.length && (a.pow != HIKF_KERNEL_GCF || a.shape == b.shape);
}

// C_0 = theta H^T (P_0 = theta I, Sec. 3.1): row i (tree order) gets theta times the
// entries of H^T's row i; one thread per row, rows are disjoint
template <typename T>
__global__ void white_c0_kernel(const int64_t* __restrict__ trowptr, const int32_t* __restrict__ tcol,
                                const double* __restrict__ tval, int64_t m, int ld, double theta,
                                T* __restrict__ C) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int64_t e = trowptr[i]; e < trowptr[i + 1]; ++e) C[i * ld + tcol[e]] += (T)(theta * tval[e]);
}

// Largest cond(S_t) the explicit-inverse sweep is claimed for (1e-5 relative on mean and
// variance): measured on the parity cases and the full-size workloads, the FP32 sweep's
// variance error grows about like eps_32 cond(S_t) / 30 and reaches 1e-5 near cond ~ 5e4; the
// split-FP16 tensor-core sweep (FP32 accumulation in the tensor core) about 5x earlier.
constexpr double kCondCrossFp32 = 5e4;
constexpr double kCondCrossMixed = 1e4;
// Largest cond(S_t) for which the tensor-core sweep splits M into two FP16 pieces instead of
// three (A1 B3, 2^-22 of the leading product, left out): measured against the oracle, the
// variance error moved by at most 1.3e-6 on every case below 3e3 (cond 71 to 2.5e3, including
// the m = 2^20, n = 256 workload over 100 steps, where it fell from 5.2e-6 to 4.7e-6), but two
// pieces of M put an n = 100 case at cond 9.3e3 above 1e-5.
constexpr double kCondFourProducts = 3e3;

// Spectral chain: with D = R^{-1/2}, D S_t D = V diag(s_t) V^T, s_1 = (1 + c) lambda + 1 and
// s_{t+1} = lambda + 2 - 1/s_t per eigenvalue, so cond(S_t) <= cond(R) max_k s_t,k / min_k s_t,k
// (equality for R = sigma^2 I). Both s_1 and the step map grow with lambda (c >= -1), so the
// order of the s_k never changes: the largest and the smallest eigenvalue carry max_k and
// min_k at every step, and only their two recurrences are run, until both have settled. Each
// moves monotonically to its fixed point s* = (lambda + 2 + sqrt(lambda^2 + 4 lambda)) / 2,
// so past the last step run the ratio is bounded by max(s_T, s*) / min(s_T, s*) of the two.
// The result bounds cond(S_t) for every t.
double spectral_cond_bound(const std::vector<double>& lam, const double* r_diag, int n, double c) {
  double lhi = 0.0, llo = INFINITY, rmax = 0.0, rmin = INFINITY;
  for (int k = 0; k < n; ++k) {
    const double l = std::max(lam[k], 0.0);
    lhi = std::max(lhi, l);
    llo = std::min(llo, l);
    rmax = std::max(rmax, r_diag[k]);
    rmin = std::min(rmin, r_diag[k]);
  }
  auto fixed = [](double l) { return 0.5 * (l + 2.0 + std::sqrt(l * l + 4.0 * l)); };
  double hi = (1.0 + c) * lhi + 1.0, lo = (1.0 + c) * llo + 1.0, worst = 0.0;
  for (int t = 0; t < 20000; ++t) {
    worst = std::max(worst, hi / lo);
    const double nh = lhi + 2.0 - 1.0 / hi, nl = llo + 2.0 - 1.0 / lo;
    const double move = std::max(std::fabs(nh - hi) / hi, std::fabs(nl - lo) / lo);
    hi = nh;
    lo = nl;
    if (move < 1e-13) break;
  }
  worst = std::max(worst, std::max(hi, fixed(lhi)) / std::min(lo, fixed(llo)));
  return (rmax / rmin) * worst;
}

// Factor chain: the 1-norm condition number ||S_1||_1 ||S_1^{-1}||_1 of the first step's S
// (within a factor n of the 2-norm one), S_1^{-1} by the library's FP64 Cholesky inverse.
Status factor_cond(const double* dS, int n, double* scratch, cudaStream_t s, double* cond) {
  double* dM = nullptr;
  int* dflag = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&dM, sizeof(double) * (size_t)n * n, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&dflag, sizeof(int) * 2, s));
  Status st = hikf::spd_inverse_f64(dS, n, dM, scratch, dflag, s);
  std::vector<double> S((size_t)n * n), M((size_t)n * n);
  int f[2] = {0, 0};
  if (st.ok()) {
    cudaError_t e = cudaMemcpyAsync(S.data(), dS, sizeof(double) * S.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.data(), dM, sizeof(double) * M.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, dflag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = hikf::cuda_status(e, "condition estimate", __FILE__, __LINE__);
  }
  cudaFreeAsync(dM, s);
  cudaFreeAsync(dflag, s);
  HIKF_TRY(st);
  if (f[0] & 2) {
    *cond = INFINITY;  // not positive definite: the first step reports HIKF_ENOTPD
    return Status::Ok();
  }
  double ns = 0.0, nm = 0.0;
  for (int j = 0; j < n; ++j) {
    double cs = 0.0, cm = 0.0;
    for (int i = 0; i < n; ++i) {
      cs += std::fabs(S[(size_t)i * n + j]);
      cm += std::fabs(M[(size_t)i * n + j]);
    }
    ns = std::max(ns, cs);
    nm = std::max(nm, cm);
  }
  *cond = ns * nm;
  return Status::Ok();
}

// The H^2 product into dst (the handle's rows, m x ld). H is replicated, so every rank has
// every source and runs the upward pass whole; the downward pass of a shard covers only the
// boxes that hold its rows [r0, r0 + m) of the tree order, and no rank forms another's rows.
template <typename T>
Status h2_rows(hikf_t* h, const hikf::FmmParams& fp, T* dst, int ld, cudaStream_t s) {
  if (!h->shard) return hikf::h2_product<T>(h->tree, h->Hfull, fp, dst, ld, s);
  return hikf::h2_product<T>(h->tree, h->Hfull, fp, dst, ld, s, h->r0, h->r0 + h->m);
}

template <typename T>
Status setup_state(hikf_t* h, const hikf_kernel& q, const hikf_kernel& p0, const double* x0, const double* cq,
                   const double* c0, const double* r_diag, const double* r_full, int chain_opt, int form_opt,
                   int sweep_products) {
  cudaStream_t s = h->stream;
  const int64_t m = h->m;
  const int n = h->n, ld = h->ld;
  T *C = nullptr, *CQ = nullptr;
  HIKF_TRY(hikf::arena_alloc(h->arena, &C, (size_t)m * ld));
  HIKF_TRY(hikf::arena_alloc(h->arena, &CQ, (size_t)m * ld));
  h->C = C;
  h->CQ = CQ;
  if (cq) {
    double* d = nullptr;
    HIKF_CUDA(hikf::pool_malloc((void**)&d, sizeof(double) * (size_t)m * n, s));
    HIKF_CUDA(cudaMemcpyAsync(d, cq, sizeof(double) * (size_t)m * n, cudaMemcpyHostToDevice, s));
    hikf::rows_to_tree<T><<<hikf::nblk(m * ld, 256), 256, 0, s>>>(d, h->tree.perm, m, n, ld, CQ);
    HIKF_LAUNCH_CHECK("rows_to_tree");
    HIKF_CUDA(cudaMemcpyAsync(d, c0, sizeof(double) * (size_t)m * n, cudaMemcpyHostToDevice, s));
    hikf::rows_to_tree<T><<<hikf::nblk(m * ld, 256), 256, 0, s>>>(d, h->tree.perm, m, n, ld, C);
    HIKF_LAUNCH_CHECK("rows_to_tree");
    HIKF_CUDA(cudaFreeAsync(d, s));
  } else {
    hikf::FmmParams fp;
    fp.order = h->order;
    fp.tensor_m2l = h->tensor_m2l();
    fp.sms = h->sms;
    fp.pow = q.pow;
    fp.theta = q.theta;
    fp.length = q.length;
    fp.shape = q.shape;
    HIKF_TRY(h2_rows<T>(h, fp, CQ, ld, s));
    if (h->qht_only) return Status::Ok();
    if (p0.theta == 0.0) {
      HIKF_CUDA(cudaMemsetAsync(C, 0, sizeof(T) * (size_t)m * ld, s));
    } else if (p0.pow == HIKF_KERNEL_WHITE) {
      HIKF_CUDA(cudaMemsetAsync(C, 0, sizeof(T) * (size_t)m * ld, s));
      white_c0_kernel<T><<<hikf::nblk(m, 256), 256, 0, s>>>(h->H.trowptr, h->H.tcol, h->H.tval, m, ld,
                                                                   p0.theta, C);
      HIKF_LAUNCH_CHECK("white_c0");
    } else if (same_shape(p0, q)) {
      // P_0 = (theta_0 / theta_Q) Q  =>  C_0 = P_0 H^T = (theta_0 / theta_Q) C_Q
      hikf::scale_kernel<T><<<hikf::nblk((m * ld + 16 / (int)sizeof(T) - 1) / (16 / (int)sizeof(T)), 256), 256, 0, s>>>(
          CQ, C, m * ld, (T)(p0.theta / q.theta));
      HIKF_LAUNCH_CHECK("scale");
    } else {
      hikf::FmmParams f0;
      f0.order = h->order;
      f0.tensor_m2l = h->tensor_m2l();
      f0.sms = h->sms;
      f0.pow = p0.pow;
      f0.theta = p0.theta;
      f0.length = p0.length;
      f0.shape = p0.shape;
      HIKF_TRY(h2_rows<T>(h, f0, C, ld, s));
    }
  }
  // dense R = L L^T: C_Q <- C_Q L^{-T}, C_0 <- C_0 L^{-T}; from here on the filter runs with
  // the measurement-space operators whitened and R = I (the diagonal-R path)
  std::vector<double> r_unit;
  if (r_full) {
    const size_t nn0 = (size_t)n * n;
    double *dR = nullptr, *w1 = nullptr, *w2 = nullptr, *linvT = nullptr;
    int* wflag = nullptr;
    HIKF_TRY(hikf::arena_alloc(h->arena, &h->Linv, nn0));
    HIKF_TRY(hikf::arena_alloc(h->arena, &h->LT, nn0));
    HIKF_TRY(hikf::arena_alloc(h->arena, &h->eraw, n));
    HIKF_TRY(hikf::arena_alloc(h->arena, &h->yw, n));
    HIKF_CUDA(hikf::pool_malloc((void**)&dR, sizeof(double) * nn0, s));
    HIKF_CUDA(hikf::pool_malloc((void**)&w1, sizeof(double) * nn0, s));
    HIKF_CUDA(hikf::pool_malloc((void**)&w2, sizeof(double) * nn0, s));
    HIKF_CUDA(hikf::pool_malloc((void**)&linvT, sizeof(double) * nn0, s));
    HIKF_CUDA(hikf::pool_malloc((void**)&wflag, sizeof(int) * 2, s));
    HIKF_CUDA(cudaMemcpyAsync(dR, r_full, sizeof(double) * nn0, cudaMemcpyHostToDevice, s));
    HIKF_TRY(hikf::launch_whiten_factors(dR, n, w1, w2, h->Linv, linvT, h->LT, wflag, s));
    int wf[2] = {0, 0};
    HIKF_CUDA(cudaMemcpyAsync(wf, wflag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    HIKF_CUDA(cudaStreamSynchronize(s));
    if (wf[0] & 2) return hikf::make_status(HIKF_EINVAL, "R is not positive definite");
    T* tmp = nullptr;
    HIKF_CUDA(hikf::pool_malloc((void**)&tmp, sizeof(T) * (size_t)m * ld, s));
    HIKF_TRY(hikf::gemm_rows_small<T>(CQ, m, ld, n, linvT, tmp, s));
    HIKF_CUDA(cudaMemcpyAsync(CQ, tmp, sizeof(T) * (size_t)m * ld, cudaMemcpyDeviceToDevice, s));
    HIKF_TRY(hikf::gemm_rows_small<T>(C, m, ld, n, linvT, tmp, s));
    HIKF_CUDA(cudaMemcpyAsync(C, tmp, sizeof(T) * (size_t)m * ld, cudaMemcpyDeviceToDevice, s));
    HIKF_CUDA(cudaFreeAsync(tmp, s));
    for (double* b : {dR, w1, w2, linvT}) HIKF_CUDA(cudaFreeAsync(b, s));
    HIKF_CUDA(cudaFreeAsync(wflag, s));
    r_unit.assign(n, 1.0);
    r_diag = r_unit.data();
    h->whiten = true;
  }
  // n x n products H A of the whitened operator: L^{-1} (H A), in place through a scratch
  double* wscr = nullptr;
  if (h->whiten) HIKF_CUDA(hikf::pool_malloc((void**)&wscr, sizeof(double) * (size_t)n * n, s));
  auto whiten_nn = [&](double* A) -> Status {
    if (!h->whiten) return Status::Ok();
    HIKF_TRY(hikf::launch_left_lower(h->Linv, A, n, wscr, s));
    HIKF_CUDA(cudaMemcpyAsync(A, wscr, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    return Status::Ok();
  };

  // mean, variance
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->x, m));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->var, m));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->outbuf, m));
  if (h->shard) {
    // x_0 of all points in tree order, then the rank's rows
    double *xc = nullptr, *xt = nullptr;
    const int64_t mf = h->m_full;
    HIKF_CUDA(hikf::pool_malloc((void**)&xc, sizeof(double) * mf, s));
    HIKF_CUDA(hikf::pool_malloc((void**)&xt, sizeof(double) * mf, s));
    if (x0) HIKF_CUDA(cudaMemcpyAsync(xc, x0, sizeof(double) * mf, cudaMemcpyHostToDevice, s));
    hikf::vec_to_tree<<<hikf::nblk(mf, 256), 256, 0, s>>>(x0 ? xc : nullptr, h->tree.perm, mf, xt);
    HIKF_LAUNCH_CHECK("vec_to_tree");
    HIKF_CUDA(cudaMemcpyAsync(h->x, xt + h->r0, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    HIKF_CUDA(cudaFreeAsync(xc, s));
    HIKF_CUDA(cudaFreeAsync(xt, s));
  } else if (x0) {
    HIKF_CUDA(cudaMemcpyAsync(h->outbuf, x0, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    hikf::vec_to_tree<<<hikf::nblk(m, 256), 256, 0, s>>>(h->outbuf, h->tree.perm, m, h->x);
  } else {
    hikf::vec_to_tree<<<hikf::nblk(m, 256), 256, 0, s>>>(nullptr, h->tree.perm, m, h->x);
  }
  HIKF_LAUNCH_CHECK("vec_to_tree");
  hikf::fill_kernel<<<hikf::nblk(m, 256), 256, 0, s>>>(h->var, m, p0.theta);
  HIKF_LAUNCH_CHECK("fill");
  h->theta_q = q.theta;

  // n x n state: S_1 = sym(H C_0 + H C_Q) + R, and sym(H C_Q) for the recurrence
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->rd, n));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->hcq_sym, (size_t)n * n));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->S, (size_t)n * n));
  HIKF_CUDA(cudaMemcpyAsync(h->rd, r_diag, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  double *hcq = nullptr, *a1 = nullptr, *zero = nullptr;
  HIKF_CUDA(hikf::pool_malloc((void**)&hcq, sizeof(double) * 2 * (size_t)n * n, s));  // [H C_Q | H C_1]
  a1 = hcq + (size_t)n * n;
  HIKF_CUDA(hikf::pool_malloc((void**)&zero, sizeof(double) * n, s));
  HIKF_CUDA(cudaMemsetAsync(zero, 0, sizeof(double) * n, s));
  HIKF_TRY(hikf::launch_gather_hc<T>(h->H, CQ, ld, hcq, 0, s));
  HIKF_TRY(hikf::launch_gather_hc<T>(h->H, C, ld, a1, 0, s));
  HIKF_TRY(hikf::launch_gather_hc<T>(h->H, CQ, ld, a1, 1, s));
  if (h->shard && h->sh.nranks > 1) {
    // the sums over the ranks' rows of H C_Q and H C_1 (the only create-time exchange)
    HIKF_CUDA(cudaStreamSynchronize(s));
    if (h->sh.allreduce(hcq, 2 * (int64_t)n * n, h->sh.ctx) != 0)
      return hikf::make_status(HIKF_ECUDA, "the caller's allreduce failed");
  }
  HIKF_TRY(whiten_nn(hcq));
  HIKF_TRY(hikf::launch_form_s(hcq, zero, n, h->hcq_sym, s));
  HIKF_TRY(whiten_nn(a1));
  HIKF_TRY(hikf::launch_form_s(a1, h->rd, n, h->S, s));
  HIKF_CUDA(cudaFreeAsync(hcq, s));
  HIKF_CUDA(cudaFreeAsync(zero, s));

  // chain scratch
  hikf::ChainArgs& c = h->chain;
  c.n = n;
  c.ldm = n;
  c.S = h->S;
  const size_t nn = (size_t)n * n;
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.Shi, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.Slo, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.L32, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.X32, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.E, 2 * nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.Mh, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.Ml, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.L64, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.X64, nn));
  if (h->fp64()) HIKF_TRY(hikf::arena_alloc(h->arena, &c.M64, nn));
  HIKF_TRY(hikf::arena_alloc(h->arena, &c.emax, 1));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->flag, 4));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->dstep, 1));
  HIKF_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int) * 4, s));
  HIKF_CUDA(cudaMemsetAsync(h->dstep, 0, sizeof(long long), s));
  c.flag = h->flag;
  c.fp64 = h->fp64() ? 1 : 0;
  T* msw = nullptr;
  HIKF_TRY(hikf::arena_alloc(h->arena, &msw, (size_t)h->nt * h->nt));
  HIKF_CUDA(cudaMemsetAsync(msw, 0, sizeof(T) * (size_t)h->nt * h->nt, s));
  h->Msw = msw;
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->e, n));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->a, n));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->ybuf, n));
  HIKF_TRY(hikf::prepare_sweep<T>(ld));
  HIKF_TRY(hikf::prepare_chain());

  // spectral chain when P_0 = c Q (c >= 0) and C_Q is our own H^2 product
  const bool p0_is_cq = p0.theta == 0.0 || same_shape(p0, q);
  const bool can_spec = cq == nullptr && p0_is_cq;
  if (chain_opt == HIKF_CHAIN_SPECTRAL && !can_spec)
    return hikf::make_status(HIKF_EINVAL, "spectral chain needs P0 = c Q and a computed C_Q");
  if ((form_opt == HIKF_FORM_EIGEN || form_opt == HIKF_FORM_NSPACE) && (!can_spec || chain_opt == HIKF_CHAIN_FACTOR))
    return hikf::make_status(HIKF_EINVAL,
                             "the eigenbasis and n-space forms need the spectral chain (P0 = c Q, computed C_Q)");
  h->spectral = can_spec && chain_opt != HIKF_CHAIN_FACTOR;
  if (!h->spectral) {
    HIKF_TRY(factor_cond(h->S, n, c.L64, s, &h->cond_s));
    if (form_opt == HIKF_FORM_AUTO) form_opt = HIKF_FORM_CROSS;  // no other form without the spectral chain
  }
  if (h->spectral) {
    hikf::SpectralState& sp = h->sp;
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.lam, n));
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.s, n));
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.u, n));
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.W64, nn));
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.W32, nn));
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.Uhi, nn));
    HIKF_TRY(hikf::arena_alloc(h->arena, &sp.Ulo, nn));
    const double cfac = p0.theta == 0.0 ? 0.0 : p0.theta / q.theta;
    HIKF_TRY(hikf::spectral_setup(sp, h->hcq_sym, h->rd, n, cfac, h->flag, s));
    int f[2] = {0, 0};
    HIKF_CUDA(cudaMemcpyAsync(f, h->flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
    HIKF_CUDA(cudaStreamSynchronize(s));
    if (f[0]) return hikf::make_status(HIKF_ENOTPD, "H C_1 + R is not positive definite");
    {
      std::vector<double> lam(n);
      HIKF_CUDA(cudaMemcpy(lam.data(), sp.lam, sizeof(double) * n, cudaMemcpyDeviceToHost));
      h->cond_s = spectral_cond_bound(lam, r_diag, n, cfac);
    }
    if (form_opt == HIKF_FORM_AUTO) {
      // the paper's cross-covariance form where its explicit inverse keeps 1e-5, else the
      // eigenbasis form (the same filter with a diagonal update, see include/hikf.h)
      const double lim = h->mixed() ? kCondCrossMixed : kCondCrossFp32;
      const bool tc_fits = h->ld <= 256;  // the tensor-core sweep's accumulator width
      form_opt = (!h->fp64() && (h->cond_s > lim || (h->mixed() && !tc_fits))) ? HIKF_FORM_EIGEN : HIKF_FORM_CROSS;
    }
    if (form_opt == HIKF_FORM_EIGEN) {
      T *G = nullptr, *Gq = nullptr;
      HIKF_TRY(hikf::arena_alloc(h->arena, &G, (size_t)m * ld));
      HIKF_TRY(hikf::arena_alloc(h->arena, &Gq, (size_t)m * ld));
      HIKF_TRY(hikf::eigen_setup<T>(sp, CQ, m, ld, n, cfac, Gq, G, s));
      h->G = G;
      h->Gq = Gq;
      h->eigen = true;
    } else if (form_opt == HIKF_FORM_NSPACE) {
      T* Gq = nullptr;
      HIKF_TRY(hikf::arena_alloc(h->arena, &Gq, (size_t)m * ld));
      HIKF_TRY(hikf::eigen_setup<T>(sp, CQ, m, ld, n, cfac, Gq, (T*)nullptr, s));
      h->Gq = Gq;
      hikf::NspaceState& ns = h->ns;
      HIKF_TRY(hikf::arena_alloc(h->arena, &ns.gam, n));
      HIKF_TRY(hikf::arena_alloc(h->arena, &ns.b, n));
      HIKF_TRY(hikf::arena_alloc(h->arena, &ns.h, n));
      HIKF_TRY(hikf::arena_alloc(h->arena, &ns.P, nn));
      HIKF_TRY(hikf::arena_alloc(h->arena, &ns.hx0, n));
      HIKF_TRY(hikf::arena_alloc(h->arena, &h->x0t, m));
      hikf::fill_kernel<<<hikf::nblk(n, 256), 256, 0, s>>>(ns.gam, n, cfac);
      HIKF_LAUNCH_CHECK("fill");
      HIKF_CUDA(cudaMemsetAsync(ns.b, 0, sizeof(double) * n, s));
      HIKF_CUDA(cudaMemsetAsync(ns.h, 0, sizeof(double) * n, s));
      HIKF_TRY(hikf::launch_gather_hc<T>(h->H, Gq, ld, ns.P, 0, s));
      HIKF_TRY(whiten_nn(ns.P));
      HIKF_CUDA(cudaMemcpyAsync(h->x0t, h->x, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
      // H x_0 = -(0 - H x_0)
      HIKF_CUDA(cudaMemsetAsync(h->ybuf, 0, sizeof(double) * n, s));
      HIKF_TRY(hikf::launch_innovation(h->ybuf, h->H, h->x, ns.hx0, h->flag, s));
      hikf::scale_kernel<double><<<hikf::nblk((n + 1) / 2, 256), 256, 0, s>>>(ns.hx0, ns.hx0, n, -1.0);
      HIKF_LAUNCH_CHECK("scale");
      if (h->whiten) {
        HIKF_CUDA(cudaMemcpyAsync(h->eraw, ns.hx0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        HIKF_TRY(hikf::launch_whiten_vec(h->Linv, h->eraw, n, ns.hx0, s));
      }
      h->var0 = p0.theta;
      h->nspace = true;
    }
  }
  if (h->mixed() && !h->eigen && !h->nspace) {
    hikf::TcState& tc = h->tc;
    HIKF_TRY(hikf::tc_setup(tc, (const float*)C, (const float*)CQ, m, ld, n));
    tc.products = sweep_products ? sweep_products : (h->cond_s <= kCondFourProducts ? 4 : 5);
    HIKF_TRY(hikf::arena_alloc(h->arena, &tc.bimg, (size_t)3 * tc.nt * tc.nt));
    HIKF_TRY(hikf::arena_alloc(h->arena, &tc.cmax, m));
    HIKF_TRY(hikf::arena_alloc(h->arena, &tc.cqmax, m));
    HIKF_TRY(hikf::arena_alloc(h->arena, &tc.mmax, hikf::kAbsBlocks));
    HIKF_TRY(hikf::arena_alloc(h->arena, &tc.beta_exp, 1));
    HIKF_TRY(hikf::arena_alloc(h->arena, &tc.vec32, (size_t)2 * tc.nt));
    HIKF_TRY(hikf::tc_init_rows(tc, (const float*)C, (const float*)CQ, m, ld, s));
  }
  if (wscr) HIKF_CUDA(cudaFreeAsync(wscr, s));
  return Status::Ok();
}

// e = y - H x; with a dense R, e = L^{-1} (y - H x) (the innovation of the whitened measurements)
// e = y - H x from the ranks' summed H x (sharded filter, step part 2)
__global__ void external_innovation_kernel(const double* __restrict__ y, const double* __restrict__ hx, int n,
                                           double* __restrict__ e, int* __restrict__ flag) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double yv = y[r];
  if (!isfinite(yv)) atomicOr(flag, 1);
  e[r] = yv - hx[r];
}

Status innovation(hikf_t* h, cudaStream_t s) {
  if (h->hx_ext) {
    external_innovation_kernel<<<hikf::nblk(h->n, 256), 256, 0, s>>>(h->ybuf, h->hx_ext, h->n, h->e, h->flag);
    HIKF_LAUNCH_CHECK("external_innovation");
    return Status::Ok();
  }
  if (!h->whiten) return hikf::launch_innovation(h->ybuf, h->H, h->x, h->e, h->flag, s);
  HIKF_TRY(hikf::launch_innovation(h->ybuf, h->H, h->x, h->eraw, h->flag, s));
  return hikf::launch_whiten_vec(h->Linv, h->eraw, h->n, h->e, s);
}

// Parts of one update: the whole step, or the grouped sweep's halves (everything before
// the tensor-core sweep, and everything after it).
enum StepPart { kStepAll = 0, kStepPre = 1, kStepPost = 2 };

// The tensor-core sweep's arguments of one handle (fixed pointers: the same every step)
hikf::TcArgs tc_args(const hikf_t* h) {
  hikf::TcArgs ta;
  ta.m = h->m;
  ta.ld = h->ld;
  ta.n = h->n;
  ta.C = (float*)h->C;
  ta.a = h->a;
  ta.rd = h->rd;
  ta.theta = h->theta_q;
  ta.x = h->x;
  ta.var = h->var;
  ta.flag = h->flag;
  ta.err = h->flag + 2;
  ta.beta_exp = h->tc.beta_exp;
  return ta;
}

// Whether a handle's sweep can join a grouped launch (hikf_assimilate_batch): the MIXED
// tensor-core sweep of the cross-covariance and spectral forms.
bool groupable(const hikf_t* h) { return h->mixed() && !h->eigen && !h->nspace && !h->shard; }

// One measurement update (or one part of it, see StepPart) on stream s. ev0/ev1 (may be
// null) bracket the sweep.
template <typename T>
Status enqueue_step(hikf_t* h, cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t s, int part) {
  hikf::ChainArgs& c = h->chain;
  int launches = 0;
  if (h->nspace) {
    if (ev0) HIKF_CUDA(cudaEventRecordWithFlags(ev0, s, h->capturing ? cudaEventRecordExternal : 0));
    const double* y = h->ybuf;
    if (h->whiten) {  // L^{-1} y against the whitened L^{-1} H x_0 and L^{-1} H G_Q
      HIKF_TRY(hikf::launch_whiten_vec(h->Linv, h->ybuf, h->n, h->yw, s));
      y = h->yw;
    }
    HIKF_TRY(hikf::nspace_step(h->sp, h->ns, h->n, y, h->e, h->flag, h->dstep, s));
    if (ev1) HIKF_CUDA(cudaEventRecordWithFlags(ev1, s, h->capturing ? cudaEventRecordExternal : 0));
    h->launches = 3;
    return Status::Ok();
  }
  if (h->eigen) {
    HIKF_TRY(innovation(h, s));
    HIKF_TRY(hikf::eigen_u(h->sp, h->n, h->e, h->flag, s));
    if (ev0) HIKF_CUDA(cudaEventRecordWithFlags(ev0, s, h->capturing ? cudaEventRecordExternal : 0));
    HIKF_TRY(hikf::eigen_step<T>(h->sp, h->m, h->ld, h->n, (T*)h->G, (const T*)h->Gq, h->theta_q, h->x, h->var,
                                 h->flag, h->sms, s));
    if (ev1) HIKF_CUDA(cudaEventRecordWithFlags(ev1, s, h->capturing ? cudaEventRecordExternal : 0));
    hikf::count_step<<<1, 1, 0, s>>>(h->flag, h->dstep);
    HIKF_LAUNCH_CHECK("count_step");
    HIKF_TRY(hikf::spectral_next(h->sp, h->n, h->flag, s));
    h->launches = 6;
    return Status::Ok();
  }
  if (part != kStepPost) {
    if (h->spectral) {
      HIKF_TRY(innovation(h, s));
      HIKF_TRY(hikf::spectral_gain<T>(h->sp, h->n, h->e, h->a, (T*)h->Msw, h->nt, h->flag, s));
      launches += sizeof(T) == 4 ? 5 : 4;
    } else {
      HIKF_TRY(hikf::launch_chain(c, s));
      launches += c.fp64 ? 1 : (2 + 3 * c.refine_iters + 3);
      HIKF_TRY(innovation(h, s));
      HIKF_TRY(hikf::launch_gemv<T>(c.Mh, c.Ml, c.M64, h->n, c.ldm, h->e, h->a, (T*)h->Msw, h->nt, h->flag, s));
      launches += 2;
    }
    if (h->mixed()) {
      HIKF_TRY(hikf::tc_pack(h->tc, (const float*)h->Msw, h->nt, h->n, h->a, h->rd, h->flag, s));
      launches += 3;
    }
    if (part == kStepPre) {
      h->launches = launches;
      return Status::Ok();
    }
    if (ev0) HIKF_CUDA(cudaEventRecordWithFlags(ev0, s, h->capturing ? cudaEventRecordExternal : 0));
    if (h->mixed()) {
      HIKF_TRY(hikf::tc_sweep(h->tc, tc_args(h), h->sms, s));
    } else {
      hikf::SweepArgs<T> sa;
      sa.m = h->m;
      sa.ld = h->ld;
      sa.n = h->n;
      sa.CQ = (const T*)h->CQ;
      sa.C = (T*)h->C;
      sa.Msw = (const T*)h->Msw;
      sa.a = h->a;
      sa.rd = h->rd;
      sa.theta = h->theta_q;
      sa.x = h->x;
      sa.var = h->var;
      sa.flag = h->flag;
      HIKF_TRY(hikf::launch_sweep<T>(sa, s, h->sms));
    }
    if (ev1) HIKF_CUDA(cudaEventRecordWithFlags(ev1, s, h->capturing ? cudaEventRecordExternal : 0));
    launches += 1;
  }
  hikf::count_step<<<1, 1, 0, s>>>(h->flag, h->dstep);
  HIKF_LAUNCH_CHECK("count_step");
  if (h->spectral)
    HIKF_TRY(hikf::spectral_next(h->sp, h->n, h->flag, s));
  else
    HIKF_TRY(hikf::launch_recur(h->hcq_sym, h->rd, c.Mh, c.Ml, c.M64, h->n, c.ldm, h->flag, h->S, s));
  launches += 2;
  h->launches = part == kStepPost ? h->launches + launches : launches;
  return Status::Ok();
}

Status enqueue_direct(hikf_t* h, cudaEvent_t ev0, cudaEvent_t ev1, int part = kStepAll) {
  return h->fp64() ? enqueue_step<double>(h, ev0, ev1, h->stream, part)
                   : enqueue_step<float>(h, ev0, ev1, h->stream, part);
}

// The update as one CUDA graph, captured on first use (thread-local capture mode, so
// other threads' allocations are not affected). Two event-record nodes bracket the
// sweep; they record placeholder events unless profiling points them at the record.
Status build_graph(hikf_t* h) {
  HIKF_CUDA(cudaEventCreate(&h->gev[0]));
  HIKF_CUDA(cudaEventCreate(&h->gev[1]));
  HIKF_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  Status st = enqueue_direct(h, h->gev[0], h->gev[1]);
  h->capturing = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (!st.ok()) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return hikf::cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  h->graph = g;
  HIKF_CUDA(cudaGraphInstantiate(&h->graph_exec, g, 0));
  size_t cnt = 0;
  HIKF_CUDA(cudaGraphGetNodes(g, nullptr, &cnt));
  std::vector<cudaGraphNode_t> nodes(cnt);
  HIKF_CUDA(cudaGraphGetNodes(g, nodes.data(), &cnt));
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    HIKF_CUDA(cudaGraphNodeGetType(nd, &ty));
    if (ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev = nullptr;
    HIKF_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
    if (ev == h->gev[0]) h->gnode[0] = nd;
    if (ev == h->gev[1]) h->gnode[1] = nd;
  }
  if (!h->gnode[0] || !h->gnode[1]) return hikf::make_status(HIKF_ECUDA, "graph event nodes not found");
  return Status::Ok();
}

// One half of a step around a grouped sweep (kStepPre / kStepPost) on the handle's stream,
// as a CUDA graph captured on first use when the handle uses graphs.
Status enqueue_part(hikf_t* h, int part) {
  if (!h->use_graph) return enqueue_direct(h, nullptr, nullptr, part);
  cudaGraphExec_t& ex = h->gpart[part - 1];
  if (!ex) {
    HIKF_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    Status st = enqueue_direct(h, nullptr, nullptr, part);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (!st.ok()) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return hikf::cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return hikf::cuda_status(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  HIKF_CUDA(cudaGraphLaunch(ex, h->stream));
  return Status::Ok();
}

Status enqueue(hikf_t* h) {
  const bool rec = h->prof && h->prof_count < (int)h->ev.size() / 2;
  cudaEvent_t ev0 = rec ? h->ev[2 * h->prof_count] : nullptr;
  cudaEvent_t ev1 = rec ? h->ev[2 * h->prof_count + 1] : nullptr;
  if (!h->use_graph) {
    HIKF_TRY(enqueue_direct(h, ev0, ev1));
  } else {
    if (!h->graph_exec) HIKF_TRY(build_graph(h));
    HIKF_CUDA(cudaGraphExecEventRecordNodeSetEvent(h->graph_exec, h->gnode[0], rec ? ev0 : h->gev[0]));
    HIKF_CUDA(cudaGraphExecEventRecordNodeSetEvent(h->graph_exec, h->gnode[1], rec ? ev1 : h->gev[1]));
    HIKF_CUDA(cudaGraphLaunch(h->graph_exec, h->stream));
  }
  if (rec) ++h->prof_count;
  ++h->enq;
  return Status::Ok();
}

// n-space form: form x and delta^2 of the current state (once per state)
Status form_outputs(hikf_t* h) {
  if (!h->nspace || h->outs_at == h->enq) return Status::Ok();
  HIKF_TRY(h->fp64() ? hikf::nspace_outputs<double>(h->ns, (const double*)h->Gq, h->m, h->ld, h->n, h->x0t,
                                                     h->var0, h->theta_q, h->dstep, h->x, h->var, h->sms, h->stream)
                     : hikf::nspace_outputs<float>(h->ns, (const float*)h->Gq, h->m, h->ld, h->n, h->x0t, h->var0,
                                                    h->theta_q, h->dstep, h->x, h->var, h->sms, h->stream));
  h->outs_at = h->enq;
  return Status::Ok();
}

Status read_flag(hikf_t* h, int* out) {
  int f[4] = {0, 0, 0, 0};
  HIKF_CUDA(cudaMemcpyAsync(f, h->flag, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream));
  HIKF_CUDA(cudaStreamSynchronize(h->stream));
  *out = f[0] | (f[2] ? 8 : 0);
  if (f[2]) h->dead = true;
  if (*out == 0) h->clean_at = h->enq;
  if (*out) HIKF_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int) * 4, h->stream));
  return Status::Ok();
}

// HIKF_ESTATE for every call on a handle whose state a timed-out step left undefined
bool refuse_dead(hikf_t* h, hikf_status* code) {
  if (!h->dead) return false;
  h->err = "the state is undefined after a timed-out step (HIKF_ETIMEOUT); destroy the handle and create a new one";
  *code = HIKF_ESTATE;
  return true;
}

Status flag_status(int f) {
  if (f & 8)
    return hikf::make_status(HIKF_ETIMEOUT,
                             "a bounded wait in the tensor-core sweep timed out; the state is now undefined");
  if (f & 1) return hikf::make_status(HIKF_EINVAL, "non-finite measurement y; step not applied");
  if (f & 2) return hikf::make_status(HIKF_ENOTPD, "H C + R is not positive definite; step not applied");
  return Status::Ok();
}

__global__ void iota_kernel(int64_t* __restrict__ a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

// The rank's rows [r0, r1) of the tree order (a balanced split) and H restricted to them
// (columns renumbered from r0): the state, the gathers and the innovation of the shard use
// this H; the H^2 product keeps the full one.
Status make_shard(hikf_t* h, const hikf_shard& sh) {
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n;
  const int64_t r0 = m * sh.rank / sh.nranks, r1 = m * (sh.rank + 1) / sh.nranks;
  const int64_t nnz = h->Hfull.nnz;
  std::vector<int64_t> rp(n + 1);
  std::vector<int32_t> cl(std::max<int64_t>(nnz, 1));
  std::vector<double> vl(std::max<int64_t>(nnz, 1));
  HIKF_CUDA(cudaMemcpyAsync(rp.data(), h->Hfull.rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
  if (nnz > 0) {
    HIKF_CUDA(cudaMemcpyAsync(cl.data(), h->Hfull.col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
    HIKF_CUDA(cudaMemcpyAsync(vl.data(), h->Hfull.val, sizeof(double) * nnz, cudaMemcpyDeviceToHost, s));
  }
  HIKF_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> lrp(n + 1, 0), lcl;
  std::vector<double> lvl;
  for (int64_t r = 0; r < n; ++r) {
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
      if (cl[k] >= r0 && cl[k] < r1) {
        lcl.push_back(cl[k] - r0);
        lvl.push_back(vl[k]);
      }
    lrp[r + 1] = (int64_t)lcl.size();
  }
  hikf::Tree local;  // the identity order over the rank's rows
  local.m = r1 - r0;
  HIKF_TRY(hikf::arena_alloc(h->arena, &local.iperm, local.m));
  iota_kernel<<<hikf::nblk(local.m, 256), 256, 0, s>>>(local.iperm, local.m);
  HIKF_LAUNCH_CHECK("iota");
  HIKF_TRY(hikf::build_sparse(h->H, h->arena, local, lrp.data(), lcl.data(), lvl.data(), (int)n, s));
  HIKF_TRY(hikf::arena_alloc(h->arena, &h->yzero, n));
  HIKF_CUDA(cudaMemsetAsync(h->yzero, 0, sizeof(double) * n, s));
  h->shard = true;
  h->sh = sh;
  h->r0 = r0;
  h->m_full = m;
  h->m = r1 - r0;
  h->use_graph = false;  // the step is split around the caller's exchange
  return Status::Ok();
}

hikf_status create_impl(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q, int n,
                        const int64_t* rowptr, const int64_t* col, const double* val, const double* r_diag,
                        const double* x0, hikf_kernel p0, const double* cq, const double* c0,
                        const hikf_options* opt, const double* r_full = nullptr, bool qht_only = false,
                        const hikf_shard* shard = nullptr) {
  auto t0 = std::chrono::steady_clock::now();
  if (!out) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "out is NULL"));
  *out = nullptr;
  hikf_options o;
  hikf_options_default(&o);
  if (opt) o = *opt;
  std::vector<double> r_from_full;
  if (r_full) {
    if (n < 1 || n > hikf::kMaxN) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "n out of range [1, 512]"));
    double rmax = 0.0;
    for (int64_t i = 0; i < (int64_t)n * n; ++i) {
      if (!std::isfinite(r_full[i])) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "non-finite R"));
      rmax = std::max(rmax, std::fabs(r_full[i]));
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j)
        if (std::fabs(r_full[(int64_t)i * n + j] - r_full[(int64_t)j * n + i]) > 1e-12 * rmax)
          return fail(nullptr, hikf::make_status(HIKF_EINVAL, "R is not symmetric"));
    r_from_full.resize(n);
    for (int i = 0; i < n; ++i) r_from_full[i] = r_full[(int64_t)i * n + i];
    r_diag = r_from_full.data();
  }
  Status st = validate_common(dim, m, points, n, rowptr, col, val, r_diag, x0, o);
  if (!st.ok()) return fail(nullptr, st);
  st = validate_kernel(q, cq != nullptr, false, qht_only);
  if (!st.ok()) return fail(nullptr, st);
  st = validate_kernel(p0, true, true, qht_only);
  if (!st.ok()) return fail(nullptr, st);
  if (cq && !c0) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "c0 is NULL"));
  if (shard) {
    if (shard->nranks < 1 || shard->rank < 0 || shard->rank >= shard->nranks)
      return fail(nullptr, hikf::make_status(HIKF_EINVAL, "shard rank / nranks out of range"));
    if (shard->nranks > 1 && !shard->allreduce)
      return fail(nullptr, hikf::make_status(HIKF_EINVAL, "a sharded filter over several ranks needs allreduce"));
    if (o.form == HIKF_FORM_NSPACE)
      return fail(nullptr, hikf::make_status(HIKF_EINVAL, "the n-space form is not sharded"));
    if (shard->nranks > m) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "more ranks than points"));
  }
  if (o.precision == HIKF_PREC_MIXED && o.form == HIKF_FORM_CROSS && hikf::padded_ld(n) > 256)
    return fail(nullptr, hikf::make_status(HIKF_EINVAL, "the tensor-core sweep (MIXED, cross form) supports n <= 256"));
  hikf_t* h = new (std::nothrow) hikf_handle();
  if (!h) return fail(nullptr, hikf::make_status(HIKF_ENOMEM, "host allocation failed"));
  auto bail = [&](const Status& s) {
    hikf::g_create_error = s.msg;
    hikf_destroy(h);
    return s.code;
  };
  h->dim = dim;
  h->m = m;
  h->n = n;
  h->ld = hikf::padded_ld(n);
  h->nt = hikf::sweep_nt(h->ld);
  h->prec = o.precision;
  h->order = o.cheb_order;
  h->use_graph = o.graph != 0;
  h->m2l = o.m2l;
  h->qht_only = qht_only;
  if (o.cuda_stream) {
    h->stream = (cudaStream_t)o.cuda_stream;
    if (h->stream == cudaStreamLegacy) h->use_graph = false;  // the legacy stream cannot be captured
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(hikf::cuda_status(e, "cudaStreamCreate", __FILE__, __LINE__));
    h->own_stream = true;
  }
  h->arena.stream = h->stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  h->tree.dim = dim;
  h->tree.m = m;
  h->tree.depth = o.max_depth >= 0 ? o.max_depth : hikf::auto_depth(m, dim, o.leaf_size);
  const int dmax = dim == 2 ? hikf::kMaxDepth2D : hikf::kMaxDepth3D;
  if (h->tree.depth > dmax) return bail(hikf::make_status(HIKF_EINVAL, "automatic depth too large; raise leaf_size"));
  double* d_pts = nullptr;
  cudaError_t e = hikf::pool_malloc((void**)&d_pts, sizeof(double) * (size_t)m * dim, h->stream);
  if (e != cudaSuccess) return bail(hikf::cuda_status(e, "device allocation", __FILE__, __LINE__));
  e = cudaMemcpyAsync(d_pts, points, sizeof(double) * (size_t)m * dim, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return bail(hikf::cuda_status(e, "cudaMemcpyAsync", __FILE__, __LINE__));
  st = hikf::build_tree(h->tree, h->arena, d_pts, h->stream);
  cudaFreeAsync(d_pts, h->stream);
  if (!st.ok()) return bail(st);
  st = hikf::build_sparse(h->H, h->arena, h->tree, rowptr, col, val, n, h->stream);
  if (!st.ok()) return bail(st);
  h->Hfull = h->H;
  if (shard) {
    st = make_shard(h, *shard);
    if (!st.ok()) return bail(st);
  }
  st = h->fp64() ? setup_state<double>(h, q, p0, x0, cq, c0, r_diag, r_full, o.chain, o.form, o.sweep_products)
                 : setup_state<float>(h, q, p0, x0, cq, c0, r_diag, r_full, o.chain, o.form, o.sweep_products);
  if (!st.ok()) return bail(st);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return bail(hikf::cuda_status(e, "create", __FILE__, __LINE__));
  h->create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return HIKF_OK;
}

}  // namespace

extern "C" {

hikf_status hikf_options_default(hikf_options* opt) {
  if (!opt) return HIKF_EINVAL;
  opt->cheb_order = 8;
  opt->leaf_size = 64;
  opt->max_depth = -1;
  opt->precision = HIKF_PREC_FP32;
  opt->cuda_stream = nullptr;
  opt->chain = HIKF_CHAIN_AUTO;
  opt->form = HIKF_FORM_AUTO;
  opt->graph = 1;
  opt->m2l = HIKF_M2L_AUTO;
  opt->sweep_products = 0;
  return HIKF_OK;
}

hikf_status hikf_create(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q, int n,
                        const int64_t* h_rowptr, const int64_t* h_col, const double* h_val, const double* r_diag,
                        const double* x0, hikf_kernel p0, const hikf_options* opt) {
  return create_impl(out, dim, m, points, q, n, h_rowptr, h_col, h_val, r_diag, x0, p0, nullptr, nullptr, opt);
}

hikf_status hikf_create_dense_r(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q, int n,
                                const int64_t* h_rowptr, const int64_t* h_col, const double* h_val,
                                const double* r_full, const double* x0, hikf_kernel p0, const hikf_options* opt) {
  if (!r_full) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "r_full is NULL"));
  return create_impl(out, dim, m, points, q, n, h_rowptr, h_col, h_val, nullptr, x0, p0, nullptr, nullptr, opt,
                     r_full);
}

hikf_status hikf_create_shard(hikf_t** out, const hikf_shard* shard, int dim, int64_t m, const double* points,
                              hikf_kernel q, int n, const int64_t* h_rowptr, const int64_t* h_col,
                              const double* h_val, const double* r_diag, const double* x0, hikf_kernel p0,
                              const hikf_options* opt) {
  if (!shard) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "shard is NULL"));
  return create_impl(out, dim, m, points, q, n, h_rowptr, h_col, h_val, r_diag, x0, p0, nullptr, nullptr, opt,
                     nullptr, false, shard);
}

hikf_status hikf_shard_rows(const hikf_t* h, int64_t* first, int64_t* count) {
  if (!h || !first || !count) return HIKF_EINVAL;
  *first = h->shard ? h->r0 : 0;
  *count = h->m;
  return HIKF_OK;
}

hikf_status hikf_shard_caller_index(hikf_t* h, int64_t* out) {
  if (!h || !out) return HIKF_EINVAL;
  cudaError_t e = cudaMemcpyAsync(out, h->tree.perm + h->r0, sizeof(int64_t) * h->m, cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "shard caller index", __FILE__, __LINE__));
  return HIKF_OK;
}

hikf_status hikf_shard_step_begin(hikf_t* h, const double* d_y, double* d_hx) {
  if (!h || !d_y || !d_hx) return h ? fail(h, hikf::make_status(HIKF_EINVAL, "null pointer")) : HIKF_EINVAL;
  if (!h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "not a sharded filter"));
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  cudaError_t e = cudaMemcpyAsync(h->ybuf, d_y, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "copy y", __FILE__, __LINE__));
  // H_r x_r = -(0 - H_r x_r) through the innovation kernel over the rank's columns
  Status st = hikf::launch_innovation(h->yzero, h->H, h->x, d_hx, h->flag, h->stream);
  if (st.ok()) {
    hikf::scale_kernel<double><<<hikf::nblk((h->n + 1) / 2, 256), 256, 0, h->stream>>>(d_hx, d_hx, h->n, -1.0);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = hikf::cuda_status(e, "scale", __FILE__, __LINE__);
  }
  if (!st.ok()) return fail(h, st);
  return HIKF_OK;
}

hikf_status hikf_shard_step_end(hikf_t* h, const double* d_hx) {
  if (!h || !d_hx) return h ? fail(h, hikf::make_status(HIKF_EINVAL, "d_hx is NULL")) : HIKF_EINVAL;
  if (!h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "not a sharded filter"));
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  h->hx_ext = d_hx;
  Status st = enqueue(h);
  h->hx_ext = nullptr;
  if (!st.ok()) return fail(h, st);
  return HIKF_OK;
}

static hikf_status shard_vec(hikf_t* h, const double* src, double* out) {
  if (!h || !out) return HIKF_EINVAL;
  if (!h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "not a sharded filter"));
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  cudaError_t e = cudaMemcpyAsync(out, src, sizeof(double) * h->m, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "shard output", __FILE__, __LINE__));
  return HIKF_OK;
}

hikf_status hikf_shard_get_mean(hikf_t* h, double* out) { return shard_vec(h, h ? h->x : nullptr, out); }
hikf_status hikf_shard_get_variance(hikf_t* h, double* out) { return shard_vec(h, h ? h->var : nullptr, out); }

hikf_status hikf_create_with_cq(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q, int n,
                                const int64_t* h_rowptr, const int64_t* h_col, const double* h_val,
                                const double* r_diag, const double* x0, hikf_kernel p0, const double* cq,
                                const double* c0, const hikf_options* opt) {
  if (!cq) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "cq is NULL"));
  return create_impl(out, dim, m, points, q, n, h_rowptr, h_col, h_val, r_diag, x0, p0, cq, c0, opt);
}

hikf_status hikf_assimilate(hikf_t* h, const double* y) {
  if (!h || !y) return h ? fail(h, hikf::make_status(HIKF_EINVAL, "y is NULL")) : HIKF_EINVAL;
  if (h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "a sharded filter: hikf_shard_step_begin / _end"));
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  for (int r = 0; r < h->n; ++r)
    if (!std::isfinite(y[r])) return fail(h, hikf::make_status(HIKF_EINVAL, "non-finite measurement y"));
  int f = 0;
  Status st;
  if (h->clean_at != h->enq) {  // steps were enqueued since the flag was last read clear
    st = read_flag(h, &f);
    if (!st.ok()) return fail(h, st);
    if (f) return fail(h, hikf::make_status(f & 8 ? HIKF_ETIMEOUT : HIKF_ESTATE,
                                            "an earlier asynchronous step failed: " + flag_status(f).msg));
  }
  cudaError_t e = cudaMemcpyAsync(h->ybuf, y, sizeof(double) * h->n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "copy y", __FILE__, __LINE__));
  st = enqueue(h);
  if (!st.ok()) return fail(h, st);
  st = read_flag(h, &f);
  if (!st.ok()) return fail(h, st);
  st = flag_status(f);
  if (!st.ok()) return fail(h, st);
  return HIKF_OK;
}

hikf_status hikf_assimilate_device(hikf_t* h, const double* d_y) {
  if (!h || !d_y) return h ? fail(h, hikf::make_status(HIKF_EINVAL, "d_y is NULL")) : HIKF_EINVAL;
  if (h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "a sharded filter: hikf_shard_step_begin / _end"));
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  cudaError_t e = cudaMemcpyAsync(h->ybuf, d_y, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "copy y", __FILE__, __LINE__));
  Status st = enqueue(h);
  if (!st.ok()) return fail(h, st);
  return HIKF_OK;
}

// An error of hikf_assimilate_batch: on the handle it concerns and for hikf_last_error(NULL)
static hikf_status bfail(hikf_t* h, const Status& st) {
  if (h) h->err = st.msg;
  return hikf::set_global_error(st);
}

hikf_status hikf_assimilate_batch(hikf_t* const* hs, const double* const* d_y, int count) {
  if (count < 0) return bfail(nullptr, hikf::make_status(HIKF_EINVAL, "count < 0"));
  if (count == 0) return HIKF_OK;
  if (!hs || !d_y) return bfail(nullptr, hikf::make_status(HIKF_EINVAL, "hs or d_y is NULL"));
  for (int i = 0; i < count; ++i) {
    hikf_t* h = hs[i];
    if (!h) return bfail(nullptr, hikf::make_status(HIKF_EINVAL, "a handle of the batch is NULL"));
    if (!d_y[i]) return bfail(h, hikf::make_status(HIKF_EINVAL, "d_y is NULL"));
    if (h->shard) return bfail(h, hikf::make_status(HIKF_ESTATE, "a sharded filter: hikf_shard_step_begin / _end"));
    hikf_status dead_code;
    if (refuse_dead(h, &dead_code)) return dead_code;
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return bfail(h, hikf::make_status(HIKF_EINVAL, "a handle appears twice in the batch"));
  }
  std::vector<hikf_t*> grp;
  for (int i = 0; i < count; ++i) {
    hikf_t* h = hs[i];
    cudaError_t e = cudaMemcpyAsync(h->ybuf, d_y[i], sizeof(double) * h->n, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return bfail(h, hikf::cuda_status(e, "copy y", __FILE__, __LINE__));
    if (groupable(h)) {
      grp.push_back(h);
      continue;
    }
    Status st = enqueue(h);  // its own step, as hikf_assimilate_device
    if (!st.ok()) return bfail(h, st);
  }
  if (grp.empty()) return HIKF_OK;
  if (grp.size() == 1) {  // nothing to group with
    Status st = enqueue(grp[0]);
    return st.ok() ? HIKF_OK : bfail(grp[0], st);
  }
  // the steps up to the sweep, each on its own stream; the sweeps run on the first
  // handle's stream once all of those have finished
  hikf_t* lead = grp[0];
  for (hikf_t* h : grp) {
    Status st = enqueue_part(h, kStepPre);
    if (!st.ok()) return bfail(h, st);
    cudaError_t e = h->bev ? cudaSuccess : cudaEventCreateWithFlags(&h->bev, cudaEventDisableTiming);
    if (e == cudaSuccess && h != lead) {
      e = cudaEventRecord(h->bev, h->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(lead->stream, h->bev, 0);
    }
    if (e != cudaSuccess) return bfail(h, hikf::cuda_status(e, "order the batch", __FILE__, __LINE__));
  }
  // one launch per MMA width n_t and product count over the tiles of all its filters
  for (int key = 0; key < 4; ++key) {
    const int nt = key < 2 ? 128 : 256, products = key % 2 == 0 ? 4 : 5;
    std::vector<hikf::TcItem> items;
    int64_t tiles = 0;
    for (hikf_t* h : grp) {
      if (hikf::tc_nt(h->tc) != nt || h->tc.products != products) continue;
      hikf::TcItem it;
      hikf::tc_item(h->tc, tc_args(h), &it);
      it.tile0 = tiles;
      tiles += hikf::tc_tiles(h->m);
      items.push_back(it);
    }
    if (items.empty()) continue;
    hikf::TcItem* d_items = nullptr;
    const size_t bytes = sizeof(hikf::TcItem) * items.size();
    cudaError_t e = hikf::pool_malloc((void**)&d_items, bytes, lead->stream);
    if (e == cudaSuccess)  // pageable source: staged before the call returns
      e = cudaMemcpyAsync(d_items, items.data(), bytes, cudaMemcpyHostToDevice, lead->stream);
    if (e != cudaSuccess) {
      if (d_items) cudaFreeAsync(d_items, lead->stream);
      return bfail(lead, hikf::cuda_status(e, "batch items", __FILE__, __LINE__));
    }
    Status st = hikf::tc_sweep_grouped(nt, products, d_items, (int)items.size(), tiles, lead->sms, lead->stream);
    cudaFreeAsync(d_items, lead->stream);
    if (!st.ok()) return bfail(lead, st);
  }
  cudaError_t e = cudaEventRecord(lead->bev, lead->stream);
  if (e != cudaSuccess) return bfail(lead, hikf::cuda_status(e, "order the batch", __FILE__, __LINE__));
  for (hikf_t* h : grp) {
    if (h != lead) {
      e = cudaStreamWaitEvent(h->stream, lead->bev, 0);
      if (e != cudaSuccess) return bfail(h, hikf::cuda_status(e, "order the batch", __FILE__, __LINE__));
    }
    Status st = enqueue_part(h, kStepPost);
    if (!st.ok()) return bfail(h, st);
    ++h->enq;
  }
  return HIKF_OK;
}

hikf_status hikf_sync(hikf_t* h) {
  if (!h) return HIKF_EINVAL;
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  int f = 0;
  Status st = read_flag(h, &f);
  if (!st.ok()) return fail(h, st);
  st = flag_status(f);
  if (!st.ok()) return fail(h, st);
  return HIKF_OK;
}

static hikf_status get_vec(hikf_t* h, const double* src, double* out, bool device) {
  if (!h || !out) return h ? fail(h, hikf::make_status(HIKF_EINVAL, "out is NULL")) : HIKF_EINVAL;
  if (h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "a sharded filter: hikf_shard_get_mean / _variance"));
  hikf_status dead_code;
  if (refuse_dead(h, &dead_code)) return dead_code;
  Status fs = form_outputs(h);
  if (!fs.ok()) return fail(h, fs);
  if (!device) {
    // page-locked host memory mapped into the device's address space (a pinned buffer): one
    // kernel writes it directly, with one wait, instead of a device copy and a transfer
    cudaPointerAttributes at;
    memset(&at, 0, sizeof(at));
    if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
      hikf::vec_from_tree<<<hikf::nblk(h->m, 256), 256, 0, h->stream>>>(src, h->tree.iperm, h->m,
                                                                         (double*)at.devicePointer);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "vec_from_tree", __FILE__, __LINE__));
      return HIKF_OK;
    }
    cudaGetLastError();  // an unregistered pointer may leave an error from the query
  }
  hikf::vec_to_caller<<<hikf::nblk(h->m, 256), 256, 0, h->stream>>>(src, h->tree.perm, h->m,
                                                                     device ? out : h->outbuf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "vec_to_caller", __FILE__, __LINE__));
  if (!device) {
    e = cudaMemcpyAsync(out, h->outbuf, sizeof(double) * h->m, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "copy out", __FILE__, __LINE__));
  }
  return HIKF_OK;
}

hikf_status hikf_get_mean(hikf_t* h, double* out) { return get_vec(h, h ? h->x : nullptr, out, false); }
hikf_status hikf_get_variance(hikf_t* h, double* out) { return get_vec(h, h ? h->var : nullptr, out, false); }
hikf_status hikf_get_mean_device(hikf_t* h, double* d_out) { return get_vec(h, h ? h->x : nullptr, d_out, true); }
hikf_status hikf_get_variance_device(hikf_t* h, double* d_out) {
  return get_vec(h, h ? h->var : nullptr, d_out, true);
}

static hikf_status get_mat(hikf_t* h, const void* src, double* out) {
  if (!h || !out) return h ? fail(h, hikf::make_status(HIKF_EINVAL, "out is NULL")) : HIKF_EINVAL;
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (size_t)h->m * h->n;
  // a shard returns its own rows in its order (hikf_shard_caller_index maps them)
  const int64_t* perm = h->shard ? nullptr : h->tree.perm;
  cudaError_t e = hikf::pool_malloc((void**)&d, bytes, h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "device allocation", __FILE__, __LINE__));
  void* unw = nullptr;
  if (h->whiten) {
    // the matrices are held in the whitened measurement space: C = C' L^T for the caller
    const size_t tb = (h->fp64() ? sizeof(double) : sizeof(float)) * (size_t)h->m * h->ld;
    e = hikf::pool_malloc(&unw, tb, h->stream);
    if (e != cudaSuccess) {
      cudaFreeAsync(d, h->stream);
      return fail(h, hikf::cuda_status(e, "device allocation", __FILE__, __LINE__));
    }
    Status st = h->fp64() ? hikf::gemm_rows_small<double>((const double*)src, h->m, h->ld, h->n, h->LT,
                                                          (double*)unw, h->stream)
                          : hikf::gemm_rows_small<float>((const float*)src, h->m, h->ld, h->n, h->LT, (float*)unw,
                                                         h->stream);
    if (!st.ok()) {
      cudaFreeAsync(d, h->stream);
      cudaFreeAsync(unw, h->stream);
      return fail(h, st);
    }
    src = unw;
  }
  if (h->fp64())
    hikf::rows_to_caller<double><<<hikf::nblk(h->m * h->n, 256), 256, 0, h->stream>>>(
        (const double*)src, perm, h->m, h->n, h->ld, d);
  else
    hikf::rows_to_caller<float><<<hikf::nblk(h->m * h->n, 256), 256, 0, h->stream>>>(
        (const float*)src, perm, h->m, h->n, h->ld, d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(d, h->stream);
  if (unw) cudaFreeAsync(unw, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "get matrix", __FILE__, __LINE__));
  return HIKF_OK;
}

hikf_status hikf_get_cq(hikf_t* h, double* out) { return get_mat(h, h ? h->CQ : nullptr, out); }
hikf_status hikf_get_cross(hikf_t* h, double* out) {
  hikf_status dead_code;
  if (h && refuse_dead(h, &dead_code)) return dead_code;
  if (h && h->eigen) {
    // C_{t|t} = (G - Gq) W^T R, formed on request into the C buffer (unused by this form)
    Status st = h->fp64() ? hikf::eigen_cross<double>(h->sp, h->rd, h->m, h->ld, h->n, (const double*)h->G,
                                                       (const double*)h->Gq, (double*)h->C, h->stream)
                          : hikf::eigen_cross<float>(h->sp, h->rd, h->m, h->ld, h->n, (const float*)h->G,
                                                      (const float*)h->Gq, (float*)h->C, h->stream);
    if (!st.ok()) return fail(h, st);
  }
  if (h && h->nspace) {
    // C_{t|t} = Gq diag(gamma) W^T R, formed on request into the C buffer (unused by this form)
    Status st = h->fp64() ? hikf::nspace_cross<double>(h->sp, h->ns, h->rd, h->m, h->ld, h->n, (const double*)h->Gq,
                                                        (double*)h->C, h->stream)
                          : hikf::nspace_cross<float>(h->sp, h->ns, h->rd, h->m, h->ld, h->n, (const float*)h->Gq,
                                                       (float*)h->C, h->stream);
    if (!st.ok()) return fail(h, st);
  }
  return get_mat(h, h ? h->C : nullptr, out);
}

hikf_status hikf_get_perm(hikf_t* h, int64_t* out) {
  if (!h || !out) return HIKF_EINVAL;
  if (h->shard) return fail(h, hikf::make_status(HIKF_ESTATE, "a sharded filter: hikf_shard_caller_index"));
  cudaError_t e = cudaMemcpyAsync(out, h->tree.perm, sizeof(int64_t) * h->m, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "get perm", __FILE__, __LINE__));
  return HIKF_OK;
}

hikf_status hikf_info(const hikf_t* h, hikf_info_t* info) {
  if (!h || !info) return HIKF_EINVAL;
  memset(info, 0, sizeof(*info));
  info->m = h->m;
  info->n = h->n;
  info->dim = h->dim;
  info->depth = h->tree.depth;
  info->cheb_order = h->order;
  info->precision = h->prec;
  long long st = 0;
  if (cudaMemcpyAsync(&st, h->dstep, sizeof(long long), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
      cudaStreamSynchronize(h->stream) == cudaSuccess)
    info->step = st;
  info->device_bytes = h->arena.bytes;
  info->create_ms = h->create_ms;
  info->sweep_launches = h->launches;
  info->chain = h->spectral ? HIKF_CHAIN_SPECTRAL : HIKF_CHAIN_FACTOR;
  info->form = h->nspace ? HIKF_FORM_NSPACE : (h->eigen ? HIKF_FORM_EIGEN : HIKF_FORM_CROSS);
  info->eig_sweeps = h->spectral ? h->sp.sweeps : 0;
  info->cond_s = h->cond_s;
  info->sweep_products = h->mixed() && !h->eigen && !h->nspace ? h->tc.products : 0;
  return HIKF_OK;
}

int64_t hikf_step(const hikf_t* h) {
  hikf_info_t i;
  if (hikf_info(h, &i) != HIKF_OK) return -1;
  return i.step;
}

hikf_status hikf_profile_enable(hikf_t* h, int enable) {
  if (!h) return HIKF_EINVAL;
  if (enable && h->ev.empty()) {
    h->ev.resize(2 * 4096);
    for (auto& e : h->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return fail(h, hikf::cuda_status(r, "cudaEventCreate", __FILE__, __LINE__));
    }
  }
  h->prof = enable != 0;
  h->prof_count = 0;
  return HIKF_OK;
}

hikf_status hikf_profile_read(hikf_t* h, double* sweep_ms, int64_t* sweep_launches) {
  if (!h || !sweep_ms || !sweep_launches) return HIKF_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "sync", __FILE__, __LINE__));
  double tot = 0.0;
  for (int i = 0; i < h->prof_count; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]);
    if (e != cudaSuccess) return fail(h, hikf::cuda_status(e, "cudaEventElapsedTime", __FILE__, __LINE__));
    tot += ms;
  }
  *sweep_ms = tot;
  *sweep_launches = h->prof_count;
  return HIKF_OK;
}

void* hikf_stream(const hikf_t* h) { return h ? (void*)h->stream : nullptr; }

const char* hikf_last_error(const hikf_t* h) {
  if (h) return h->err.c_str();
  return hikf::g_create_error.c_str();
}

void hikf_destroy(hikf_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (auto& g : h->gpart)
    if (g) cudaGraphExecDestroy(g);
  if (h->bev) cudaEventDestroy(h->bev);
  for (auto& e : h->gev)
    if (e) cudaEventDestroy(e);
  h->arena.release();
  if (h->stream) cudaStreamSynchronize(h->stream);  // the frees are done before the stream goes
  for (auto& e : h->ev) cudaEventDestroy(e);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

hikf_status hikf_release_cached_memory(void) {
  cudaError_t e = hikf::pool_trim_all();
  if (e != cudaSuccess) return fail(nullptr, hikf::cuda_status(e, "release cached memory", __FILE__, __LINE__));
  return HIKF_OK;
}

hikf_status hikf_spd_inverse(const double* d_S, int n, double* d_M, void* stream) {
  if (!d_S || !d_M) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "null matrix pointer"));
  if (n < 1 || n > hikf::kMaxN) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "n out of range [1, 512]"));
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  int* flag = nullptr;
  cudaError_t e = hikf::pool_malloc((void**)&scratch, sizeof(double) * (size_t)n * n, s);
  if (e == cudaSuccess) e = hikf::pool_malloc((void**)&flag, sizeof(int) * 2, s);
  if (e != cudaSuccess) return fail(nullptr, hikf::cuda_status(e, "device allocation", __FILE__, __LINE__));
  Status st = hikf::spd_inverse_f64(d_S, n, d_M, scratch, flag, s);
  int f[2] = {0, 0};
  if (st.ok()) {
    e = cudaMemcpyAsync(f, flag, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = hikf::cuda_status(e, "spd_inverse", __FILE__, __LINE__);
  }
  cudaFreeAsync(scratch, s);
  cudaFreeAsync(flag, s);
  if (!st.ok()) return fail(nullptr, st);
  if (f[0] & 2) return fail(nullptr, hikf::make_status(HIKF_ENOTPD, "matrix is not positive definite"));
  return HIKF_OK;
}

hikf_status hikf_test_set_wait_limit(uint64_t ns) {
  hikf::tc_set_wait_limit((unsigned long long)ns);
  return HIKF_OK;
}

hikf_status hikf_h2_qht(int dim, int64_t m, const double* points, hikf_kernel k, int n, const int64_t* h_rowptr,
                        const int64_t* h_col, const double* h_val, const hikf_options* opt, double* out) {
  if (!out) return fail(nullptr, hikf::make_status(HIKF_EINVAL, "out is NULL"));
  std::vector<double> rd(std::max(n, 1), 1.0);
  hikf_kernel zero = {k.pow, 0.0, 1.0, k.shape};
  hikf_t* h = nullptr;
  hikf_status s = create_impl(&h, dim, m, points, k, n, h_rowptr, h_col, h_val, rd.data(), nullptr, zero, nullptr,
                              nullptr, opt, nullptr, true);
  if (s != HIKF_OK) return s;
  s = hikf_get_cq(h, out);
  if (s != HIKF_OK) hikf::g_create_error = h->err;
  hikf_destroy(h);
  return s;
}

}  // extern "C"
