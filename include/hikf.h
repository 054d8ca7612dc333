/*
 * hikf.h — C ABI of the GB300 HiKF library (libhikf.so).
 *
 * HiKF (Li, Ambikasaran, Darve, Kitanidis, "A Kalman filter powered by
 * H^2-matrices for quasi-continuous data assimilation problems") is the
 * random-walk Kalman filter (Sec. 2.1, Eq. random_walk: x_t = x_{t-1} + w_t;
 * Eq. measurement: z_t = H x_t + v_t; w ~ N(0,Q), v ~ N(0,R)) carried by the
 * m x n cross-covariance C = P H^T instead of the m x m covariance P
 * (Alg. 2). The model-error cross-covariance C_Q = Q H^T is computed once by a
 * black-box FMM (Chebyshev-interpolated H^2 product, Sec. 3.2-3.3), and each
 * measurement update costs O(n^2 m) (Alg. 2's cost column; Sec. 3.1 and 3.3).
 *
 * Conventions shared by every call:
 *   - All pointers are plain host or device pointers as stated per argument;
 *     no C++ or torch types cross this interface.
 *   - Every input is copied during the call; the caller keeps ownership of
 *     its buffers and may free them when the call returns (for the *_device
 *     and *_async calls: when the handle's stream has passed the call).
 *   - Vectors over the m grid points are in the CALLER's point order (the
 *     order of `points` given to hikf_create); the library's internal tree
 *     order never leaks out.
 *   - Every call returns a status; nothing aborts or throws across the ABI.
 *     hikf_last_error() gives a one-line message for the last failure.
 *   - A handle is used by one host thread at a time; distinct handles are
 *     independent (they may share a device and run concurrently).
 *   - All device memory of a handle is allocated in hikf_create and freed in
 *     hikf_destroy; a measurement update allocates nothing.
 */
#ifndef HIKF_H
#define HIKF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hikf_handle hikf_t; /* opaque; owns all of its device memory */

typedef enum {
  HIKF_OK = 0,
  HIKF_EINVAL = 1,   /* invalid argument: null pointer, size out of range, non-finite value */
  HIKF_ENOMEM = 2,   /* a device or pinned-host allocation failed */
  HIKF_ECUDA = 3,    /* a CUDA runtime call failed (message in hikf_last_error) */
  HIKF_ENOTPD = 4,   /* H C_{t+1|t} + R was not positive definite; the step was not applied */
  HIKF_ETIMEOUT = 5, /* a bounded device-side wait ran out */
  HIKF_ESTATE = 6    /* the handle holds an unreported error or the call is out of order */
} hikf_status;

/* Kernel families (the field `pow` of hikf_kernel):
 *   HIKF_KERNEL_EXP    K(r) = theta exp(-r / l)        (Sec. 3.3, kernel 2)
 *   HIKF_KERNEL_GAUSS  K(r) = theta exp(-r^2 / l^2)    (Sec. 3.3, kernel 1)
 *   HIKF_KERNEL_GCF    K(r) = theta exp(-(r / l)^p), the generalised covariance
 *                      function of Eq. Q with any exponent 0 < p <= 2 (shape = p;
 *                      p = 1 and p = 2 are the two kernels above)
 *   HIKF_KERNEL_LOG    K(r) = theta log(l / r) for r > 0, i.e. A log r with A = -theta < 0
 *                      (Sec. 3.3, kernel 3) plus the constant theta log l; the kernel is
 *                      singular at r = 0, so its diagonal is stated: K(0) = theta log(l / r0)
 *                      with r0 = shape > 0 (e.g. r0 = half a cell). A generalised covariance,
 *                      not a covariance: accepted by hikf_h2_qht only, not as Q or P_0.
 *   HIKF_KERNEL_WHITE  (P_0 only) P_0 = theta I, the initialisation of Sec. 3.1 (cells
 *                      uncorrelated; length and shape ignored).
 * theta = 0 gives the zero kernel. */
enum {
  HIKF_KERNEL_WHITE = 0,
  HIKF_KERNEL_EXP = 1,
  HIKF_KERNEL_GAUSS = 2,
  HIKF_KERNEL_GCF = 3,
  HIKF_KERNEL_LOG = 4
};

typedef struct {
  int pow;       /* kernel family HIKF_KERNEL_* (HIKF_KERNEL_WHITE: p0 only; LOG: hikf_h2_qht only) */
  double theta;  /* scale, >= 0 (for the covariances theta = K(0) = diag of the covariance) */
  double length; /* correlation length l > 0, in the units of `points` */
  double shape;  /* HIKF_KERNEL_GCF: the exponent p, 0 < p <= 2; HIKF_KERNEL_LOG: r0 > 0;
                    ignored by the other families */
} hikf_kernel;

/* Arithmetic of the device path.
 *   FP32:  C, C_Q and the H^2 product in FP32 on the CUDA cores; the n x n
 *          solve refined to FP64-level accuracy; diag(P) and the state in FP64.
 *   MIXED: as FP32, with the per-step O(n^2 m) product on the tensor cores
 *          (tcgen05; each FP32 operand split into three FP16 pieces, FP32
 *          accumulation) and the M2L translations of the H^2 product on the
 *          tensor cores (tcgen05, FP32 operands split into two TF32 pieces).
 *   FP64:  everything in FP64 (small problems; the FP64 rate of this part is low). */
enum { HIKF_PREC_FP32 = 0, HIKF_PREC_MIXED = 1, HIKF_PREC_FP64 = 2 };

typedef struct {
  int cheb_order;    /* Chebyshev nodes per axis p, 2..12 (3D: 2..8). Default 8. */
  int leaf_size;     /* target points per leaf for the automatic depth. Default 64. */
  int max_depth;     /* uniform tree depth L; -1 = automatic (smallest L with
                        m <= leaf_size * 2^(dim L)). Default -1. */
  int precision;     /* HIKF_PREC_*. Default HIKF_PREC_FP32. */
  void* cuda_stream; /* cudaStream_t the handle runs on; NULL = a stream the handle
                        creates and owns. A caller's stream must outlive the handle
                        (hikf_destroy frees the handle's memory in its order). Default NULL. */
  int chain;         /* how S_t^{-1} = (H C_{t|t-1} + R)^{-1} is formed each step:
                        HIKF_CHAIN_AUTO (default): spectral when P_0 = c Q (c >= 0,
                        including P_0 = 0) and C_Q is computed, else factor;
                        HIKF_CHAIN_FACTOR: a Cholesky factorisation every step;
                        HIKF_CHAIN_SPECTRAL: one eigendecomposition of
                        R^{-1/2} H C_Q R^{-1/2} at create, then an O(n) recurrence per
                        step (HIKF_EINVAL when P_0 is not c Q). */
  int form;          /* the state the update sweeps over each step:
                        HIKF_FORM_CROSS (default): the cross-covariance C = P H^T of
                        Alg. 2, one (m x n)(n x n) contraction per step, O(n^2 m);
                        HIKF_FORM_EIGEN: the same filter carried as G = C_{t|t} R^{-1/2} V
                        (V: eigenvectors of R^{-1/2} H C_Q R^{-1/2}); the update is
                        then diagonal, O(n m) per step, and the variance reduction a
                        sum of squares. Needs the spectral chain (P_0 = c Q) and
                        FP32/FP64. hikf_get_cross forms C_{t|t} = G V^T R^{1/2} on request;
                        HIKF_FORM_NSPACE: with P_0 = c Q the eigenbasis state stays
                        G_{t|t} = C_Q R^{-1/2} V diag(gamma_t), so the filter is carried by
                        three n-vectors (x_t = x_0 + G_Q b_t, delta^2_t = delta^2_0 +
                        t theta - G_Q^2 h_t, G_Q = C_Q R^{-1/2} V) and one step costs O(n^2)
                        with no pass over the m rows. hikf_get_mean / hikf_get_variance
                        (and the _device forms) form x and delta^2 in one pass over G_Q
                        when the state has changed since the last call; hikf_get_cross
                        forms C_{t|t}. Same conditions as HIKF_FORM_EIGEN.
                        HIKF_FORM_AUTO (default): HIKF_FORM_CROSS, unless the spectral chain
                        is in use, the precision is FP32 or MIXED and the bound on cond(S_t)
                        (hikf_info's cond_s) is above what the cross form's explicit FP32
                        inverse carries to 1e-5 (5e4 for FP32, 1e4 for MIXED; or n > 256 for
                        MIXED): then HIKF_FORM_EIGEN, whose update is a sum of positive terms
                        and keeps FP32 accuracy at any cond(S). hikf_info reports the form
                        chosen. With MIXED the eigenbasis and n-space sweeps run on the CUDA
                        cores (FP32); the H^2 product still uses the tensor cores. */
  int graph;         /* 1 (default): each update is replayed as one CUDA graph, captured on
                        the first update; 0: kernels are launched one by one. */
  int m2l;           /* where the M2L translations of the H^2 product run:
                        HIKF_M2L_AUTO (default): on the tensor cores for MIXED, on the
                        CUDA cores otherwise; HIKF_M2L_TENSOR: on the tensor cores
                        (tcgen05, FP32 operands split into two TF32 pieces, all levels in
                        one launch per pass of 256 rays x 128 operator rows, launch
                        variant autotuned once per shape) for FP32 and MIXED
                        (HIKF_EINVAL for FP64); HIKF_M2L_SIMT: on the CUDA cores. */
  int sweep_products; /* MIXED tensor-core sweep, FP16 products per K step: 0 (default) = 4
                        when cond_s <= 3e3, else 5 (see hikf_info_t.sweep_products); 4 or 5
                        to choose; anything else is HIKF_EINVAL. */
} hikf_options;

enum { HIKF_CHAIN_AUTO = 0, HIKF_CHAIN_FACTOR = 1, HIKF_CHAIN_SPECTRAL = 2 };
enum { HIKF_FORM_CROSS = 0, HIKF_FORM_EIGEN = 1, HIKF_FORM_NSPACE = 2, HIKF_FORM_AUTO = 3 };
enum { HIKF_M2L_AUTO = 0, HIKF_M2L_TENSOR = 1, HIKF_M2L_SIMT = 2 };

/* Fill *opt with the defaults listed above. */
hikf_status hikf_options_default(hikf_options* opt);

/*
 * hikf_create — precomputation of Alg. 2 (C_Q = Q H^T by the H^2 approach) and
 * initialisation (Sec. 3.1: x_{0|0}, C_{0|0} = P_0 H^T; delta^2_{0|0} = diag(P_0)).
 *
 *   out       receives the new handle (set to NULL on failure).
 *   dim       2 or 3.
 *   m         number of grid points (state size), 1 <= m <= 2^31 - 1.
 *   points    host, m x dim FP64, row-major: point i is points[i*dim .. i*dim+dim-1].
 *   q         model-error covariance kernel Q (Eq. Q); theta > 0.
 *   n         number of measurements (rays), 1 <= n <= 512.
 *   h_rowptr  host, n+1 int64: CSR row pointers of H (n x m), h_rowptr[0] = 0.
 *   h_col     host, nnz int64 column indices in [0, m) (any order within a row;
 *             duplicates are summed).
 *   h_val     host, nnz FP64 values (Sec. 4.1: H_ij = length of ray i in cell j).
 *   r_diag    host, n FP64 > 0: the diagonal of R (Eq. R: R = sigma^2 I).
 *   x0        host, m FP64 initial mean x_{0|0}; NULL = zero (Sec. 4.2).
 *   p0        initial covariance kernel P_0; theta = 0 gives P_0 = 0 (Sec. 4.2).
 *             If p0 has q's pow and length, C_0 = (p0.theta / q.theta) C_Q and no
 *             second H^2 product is run. pow = HIKF_KERNEL_WHITE gives P_0 = theta I
 *             (Sec. 3.1): C_0 = theta H^T, and the gain chain factors S_t every step
 *             (the spectral chain, and with it the eigenbasis and n-space forms, needs
 *             P_0 = c Q).
 *   opt       NULL = defaults.
 * Errors: HIKF_EINVAL (sizes, null pointers, non-finite or negative values,
 * column index out of range), HIKF_ENOMEM, HIKF_ECUDA.
 */
hikf_status hikf_create(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q, int n,
                        const int64_t* h_rowptr, const int64_t* h_col, const double* h_val,
                        const double* r_diag, const double* x0, hikf_kernel p0, const hikf_options* opt);

/*
 * hikf_create_dense_r — as hikf_create, with a full measurement-error covariance R
 * (Eq. R generalised from sigma^2 I to correlated errors) instead of its diagonal:
 *   r_full  host, n x n FP64, row-major, symmetric positive definite.
 * The filter is run in the whitened measurement space: with R = L L^T (FP64 Cholesky on
 * the device), the measurements L^{-1} y, the operator L^{-1} H and the error covariance
 * I give the same posterior mean and variance (Alg. 1 and 2 are invariant under this
 * change of measurement coordinates). C_Q and C_{0|0} are transformed once at create
 * (C L^{-T}) and each innovation by L^{-1}; the O(n^2 m) update itself is the diagonal-R
 * one. hikf_get_cq and hikf_get_cross return the untransformed C_Q and C_{t|t}; hikf_info's
 * cond_s refers to the whitened S_t = L^{-1} (H C_{t|t-1} + R) L^{-T}.
 * Errors: as hikf_create; HIKF_EINVAL also when r_full is not finite, not symmetric
 * (|R_ij - R_ji| > 1e-12 max |R|) or not positive definite.
 */
hikf_status hikf_create_dense_r(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q, int n,
                                const int64_t* h_rowptr, const int64_t* h_col, const double* h_val,
                                const double* r_full, const double* x0, hikf_kernel p0, const hikf_options* opt);

/*
 * hikf_create_with_cq — as hikf_create, but C_Q and C_{0|0} are given instead
 * of computed (host, m x n FP64 row-major, caller's point order). Use it to
 * check the measurement update separately from the H^2 product. The kernel q
 * only provides diag(Q) = q.theta and p0 only delta^2_0 = p0.theta.
 */
hikf_status hikf_create_with_cq(hikf_t** out, int dim, int64_t m, const double* points, hikf_kernel q,
                                int n, const int64_t* h_rowptr, const int64_t* h_col, const double* h_val,
                                const double* r_diag, const double* x0, hikf_kernel p0,
                                const double* cq, const double* c0, const hikf_options* opt);

/*
 * hikf_assimilate — one prediction + correction step of Alg. 2 with the
 * measurement y_{t+1} (host, n FP64):
 *   C_{t+1|t} = C_{t|t} + C_Q;  delta^2_{t+1|t} = delta^2_{t|t} + diag(Q)
 *   K = C_{t+1|t} (H C_{t+1|t} + R)^{-1}
 *   x_{t+1|t+1} = x_{t+1|t} + K (y_{t+1} - H x_{t+1|t})
 *   delta^2_{t+1|t+1} = delta^2_{t+1|t} - sum_j K_ij (C_{t+1|t})_ij
 *   C_{t+1|t+1} = C_{t+1|t} - K H C_{t+1|t}
 * Synchronous: returns when the step is complete. Transactional: on HIKF_EINVAL
 * (a non-finite y) and HIKF_ENOTPD the state is unchanged.
 * HIKF_ETIMEOUT (a bounded wait inside the tensor-core sweep ran out) is different:
 * the sweep updates C, x and delta^2 in place tile by tile, so the state is then
 * undefined. The timeout is reported once; from then on every call on the handle
 * that reads or advances the state returns HIKF_ESTATE, until the handle is
 * destroyed and created again.
 */
hikf_status hikf_assimilate(hikf_t* h, const double* y);

/*
 * hikf_assimilate_device — the same step with y (n FP64) in DEVICE memory,
 * enqueued on the handle's stream without waiting. A failure inside the step
 * (non-finite y, HIKF_ENOTPD) leaves the state unchanged, turns the following
 * enqueued steps into no-ops, and is reported by the next hikf_sync (or any
 * synchronous call), after which the handle works again. A timed-out step
 * (HIKF_ETIMEOUT, reported the same way) leaves the state undefined, and later
 * calls return HIKF_ESTATE as for hikf_assimilate.
 */
hikf_status hikf_assimilate_device(hikf_t* h, const double* d_y);

/*
 * hikf_assimilate_batch — one step of each of `count` filters (Alg. 2 per filter, each
 * with its own y: d_y[i], DEVICE memory, n_i FP64 of filter hs[i]), enqueued without
 * waiting. The tensor-core sweeps (the O(m n^2) update of C, x and delta^2) of the filters
 * in MIXED precision and the cross-covariance or spectral form run as ONE launch per MMA
 * width (n_t = 128 or 256) over the row tiles of all of them, so that many small filters
 * fill the SMs together; the rest of each step runs on the filter's own stream, and the
 * other filters take their ordinary step (hikf_assimilate_device); filters of different
 * sweep_products (hikf_info) go in separate launches. Every filter's result
 * is bit-identical to hikf_assimilate_device with the same y. The filters' streams are
 * ordered against the shared launch by events (it runs on the first grouped filter's
 * stream); each handle's stream has passed its step once hikf_sync of that handle returns.
 * Errors inside a step are per filter and reported as for hikf_assimilate_device; a
 * timed-out wait in a shared launch marks every filter of that launch (HIKF_ETIMEOUT, then
 * HIKF_ESTATE). The sweep timing of hikf_profile_enable does not cover a shared launch.
 * Argument errors (count < 0, a NULL pointer, a handle twice, a sharded or dead handle)
 * return before anything is enqueued. The message of any failure is given by
 * hikf_last_error(NULL) (and by the handle it concerns). hs and d_y are read during the
 * call only.
 */
hikf_status hikf_assimilate_batch(hikf_t* const* hs, const double* const* d_y, int count);

/* Wait for the handle's stream; return and clear a latched step error. */
hikf_status hikf_sync(hikf_t* h);

/* Posterior mean x_{t|t} / variance delta^2_{t|t} (Alg. 2) into host `out`
 * (m FP64, caller's point order). Synchronous. */
hikf_status hikf_get_mean(hikf_t* h, double* out);
hikf_status hikf_get_variance(hikf_t* h, double* out);

/* The same into DEVICE `d_out` (m FP64, caller's order), enqueued on the stream. */
hikf_status hikf_get_mean_device(hikf_t* h, double* d_out);
hikf_status hikf_get_variance_device(hikf_t* h, double* d_out);

/* Test hooks: the H^2 product C_Q and the current C_{t|t} (host, m x n FP64,
 * row-major, caller's order; on a sharded filter the rank's rows, count x n, in the
 * rank's order of hikf_shard_caller_index); the tree permutation (host, m int64:
 * entry s is the caller index of the s-th point in tree order; not on a shard).
 * Synchronous. */
hikf_status hikf_get_cq(hikf_t* h, double* out);
hikf_status hikf_get_cross(hikf_t* h, double* out);
hikf_status hikf_get_perm(hikf_t* h, int64_t* out);

typedef struct {
  int64_t m;
  int n;
  int dim;
  int depth;          /* uniform tree depth L */
  int cheb_order;     /* p */
  int precision;      /* HIKF_PREC_* */
  int64_t step;       /* measurement updates applied */
  int64_t device_bytes; /* device memory held by the handle */
  double create_ms;   /* wall time of the precomputation */
  int sweep_launches; /* kernel launches of one measurement update */
  int chain;          /* HIKF_CHAIN_FACTOR or HIKF_CHAIN_SPECTRAL: the form in use */
  int form;           /* HIKF_FORM_CROSS, HIKF_FORM_EIGEN or HIKF_FORM_NSPACE */
  int eig_sweeps;     /* Jacobi sweeps of the create-time eigendecomposition (0: factor chain) */
  double cond_s;      /* conditioning of S_t = H C_{t|t-1} + R, the matrix the gain inverts
                         (Eq. kalmangin_new): spectral chain, a bound on the 2-norm condition
                         number valid for every step, cond(R) max s / min s over the eigenvalue
                         recurrences; factor chain, the 1-norm condition number of S_1. The
                         cross form's explicit FP32 inverse loses accuracy in proportion to it
                         (see HIKF_FORM_AUTO); INFINITY when S_1 is not positive definite. */
  int sweep_products; /* MIXED tensor-core sweep: FP16 products per K step (C_p and M split into
                         two and three pieces: 5; M in two pieces when cond_s <= 3e3, where the
                         third does not move the result past 1e-5: 4; or as
                         hikf_options.sweep_products chose); 0 for the other paths */
} hikf_info_t;

hikf_status hikf_info(const hikf_t* h, hikf_info_t* info);

/* Measurement updates applied so far (hikf_info's `step`); -1 when h is NULL or the
 * count cannot be read. Waits for the handle's stream. */
int64_t hikf_step(const hikf_t* h);

/* Timing of the sweep, the O(n^2 m) pass of every update: while enabled,
 * CUDA events on the handle's stream bracket each sweep launch (up to 4096
 * launches; later ones are not recorded). Enabling resets the record. */
hikf_status hikf_profile_enable(hikf_t* h, int enable);

/* Total duration (ms) of the recorded sweep launches and their number.
 * Synchronous. */
hikf_status hikf_profile_read(hikf_t* h, double* sweep_ms, int64_t* sweep_launches);

/* The CUDA stream of the handle (a cudaStream_t). */
void* hikf_stream(const hikf_t* h);

/* One-line message for the last failure on this handle (h != NULL) or of the
 * last failed hikf_create on this thread (h == NULL). Never NULL. */
const char* hikf_last_error(const hikf_t* h);

/* Free the handle and all of its device memory (back to the library's pool, in the order
 * of the handle's stream, after waiting for the stream's work). NULL is ignored. */
void hikf_destroy(hikf_t* h);

/*
 * Row sharding — the filter split over `nranks` processes (one GPU each) by rows of the
 * state. Alg. 2 is row-wise except for H C_{t+1|t} and H s_{t+1|t}, which sum over the rows
 * on the support of H; the cost analysis of Alg. 2 and the O(mn) storage of Table 3 make the
 * m x n state the quantity to split. Each rank owns a contiguous range of rows in the tree
 * (Morton) order: its rows of C, C_Q, x and delta^2. The n x n quantities of the gain chain are
 * replicated (every rank forms the same ones from the same sums), so the ranks exchange:
 *   at create, once: the sums over ranks of the partial n x n products H_r C_Q,r and
 *                    H_r C_1,r (2 n^2 doubles), through the caller's all-reduce callback;
 *   every step:      the sum over ranks of the partial n-vector H_r x_r (the innovation),
 *                    done by the caller between hikf_shard_step_begin and _end.
 * H is small and replicated, so every rank runs the upward pass of the H^2 product over all
 * sources (no multipole halo is exchanged) and the downward pass (M2L, L2L, L2P, P2P) only
 * for the boxes that hold its rows: no rank forms another rank's rows of C_Q. Forms: cross and eigen (HIKF_FORM_NSPACE is
 * refused); diagonal R only. Updates are enqueued on the handle's stream without a graph.
 */
typedef int (*hikf_allreduce_fn)(double* d_buf, int64_t count, void* ctx); /* sum in place over the ranks,
                                                                               device buffer; 0 = success */
typedef struct {
  int rank;                    /* 0 <= rank < nranks */
  int nranks;                  /* >= 1 */
  hikf_allreduce_fn allreduce; /* called from hikf_create_shard with the stream synchronized;
                                  may be NULL when nranks == 1 */
  void* ctx;                   /* passed through to allreduce */
} hikf_shard;

/* hikf_create with the filter split by rows as described above; the other arguments as
 * in hikf_create (every rank passes the same problem). HIKF_EINVAL for a bad rank/nranks,
 * HIKF_FORM_NSPACE, or a missing allreduce with nranks > 1; HIKF_ECUDA when allreduce fails. */
hikf_status hikf_create_shard(hikf_t** out, const hikf_shard* shard, int dim, int64_t m, const double* points,
                              hikf_kernel q, int n, const int64_t* h_rowptr, const int64_t* h_col,
                              const double* h_val, const double* r_diag, const double* x0, hikf_kernel p0,
                              const hikf_options* opt);

/* The rank's rows: tree-order positions [*first, *first + *count) of the m points. */
hikf_status hikf_shard_rows(const hikf_t* h, int64_t* first, int64_t* count);
/* host, count int64: the caller's index of each of the rank's rows (in the rank's order). */
hikf_status hikf_shard_caller_index(hikf_t* h, int64_t* out);

/* Step of a sharded filter, part 1: y_{t+1} (device, n FP64) is taken in, and the rank's
 * partial H_r x_r is written to d_hx (device, n FP64). Enqueued on the handle's stream: the
 * caller synchronises it, sums d_hx over the ranks in place, and calls part 2. */
hikf_status hikf_shard_step_begin(hikf_t* h, const double* d_y, double* d_hx);
/* Part 2: the rest of the step (Alg. 2 with H x_t = the summed d_hx, device n FP64) on the
 * rank's rows. Enqueued; errors are latched and reported by hikf_sync as for
 * hikf_assimilate_device. d_hx must stay valid until the stream has passed the call. */
hikf_status hikf_shard_step_end(hikf_t* h, const double* d_hx);
/* The rank's rows of x_{t|t} / delta^2_{t|t} (host, count FP64, the rank's order). Synchronous. */
hikf_status hikf_shard_get_mean(hikf_t* h, double* out);
hikf_status hikf_shard_get_variance(hikf_t* h, double* out);

/* Test hook: the limit (ns) of the tensor-core sweep's abortable device-side waits
 * for launches captured or enqueued from now on (process-wide); 0 restores the
 * default of about two seconds. A tiny limit makes the next MIXED step time out
 * (HIKF_ETIMEOUT) through the sweep's normal abort path: it drains its copies and
 * tensor-core work in flight, frees its tensor memory and returns. */
hikf_status hikf_test_set_wait_limit(uint64_t ns);

/* Device memory: the filters' state and the scratch of a create come from one
 * stream-ordered pool per device that the library owns. Freed memory stays cached in it,
 * up to 16 GiB, so that the next create reuses it without mapping pages again (a handle's
 * buffers return to it at hikf_destroy). This returns every cached byte to the device;
 * memory held by live handles is not affected. HIKF_ECUDA on a CUDA error. */
hikf_status hikf_release_cached_memory(void);

/*
 * hikf_h2_qht — the H^2 product alone (Alg. 2 precomputation, Sec. 3.2:
 * Q H^T = [Q h^(1) ... Q h^(n)]), without a filter. Arguments as in
 * hikf_create (any kernel family, HIKF_KERNEL_LOG included); `out` is host m x n FP64,
 * row-major, caller's point order.
 * Allocates its device memory for the call and frees it before returning.
 */
hikf_status hikf_h2_qht(int dim, int64_t m, const double* points, hikf_kernel k, int n,
                        const int64_t* h_rowptr, const int64_t* h_col, const double* h_val,
                        const hikf_options* opt, double* out);

/*
 * hikf_spd_inverse — M = S^{-1} for a symmetric positive-definite n x n matrix
 * by an FP64 Cholesky factorisation S = L L^T and the inverse of L: the
 * (H C_{t+1|t} + R)^{-1} of the gain (Eq. kalmangin_new), the factor path of
 * the update used when P_0 is not a multiple of Q.
 *   d_S     device, n x n FP64 row-major (only the lower triangle is read).
 *   n       1 <= n <= 512.
 *   d_M     device, n x n FP64 row-major output (full symmetric matrix).
 *   stream  cudaStream_t, NULL = the default stream.
 * Allocates n x n FP64 of device scratch for the call (stream-ordered) and
 * frees it before returning. Synchronous. HIKF_ENOTPD when a pivot is not
 * positive (d_M is then unspecified), HIKF_EINVAL for bad sizes or pointers.
 */
hikf_status hikf_spd_inverse(const double* d_S, int n, double* d_M, void* stream);

/*
 * hikf_spd_inverse_noalloc — hikf_spd_inverse without any device allocation,
 * for callers that must not call cudaMalloc/cudaFree (or an allocating library
 * routine) on this path: processes that reserve all of their device memory up
 * front and hand out fixed slices of it (a server dividing HBM among filter
 * handles, for example), and latency-bound loops in which an allocation could
 * synchronise the device or fail under fragmentation. It has no counterpart in
 * the paper; it runs the same kernel as hikf_spd_inverse.
 *   d_S, d_M, stream  as in hikf_spd_inverse (caller-owned device buffers).
 *   n       1 <= n <= HIKF_NOALLOC_MAX_N; larger n returns HIKF_EINVAL.
 * Scratch is a static device array of HIKF_NOALLOC_MAX_N^2 FP64 (512 KB) plus
 * a status word, which every GPU that loads the library holds until the
 * process exits. The first call on a device resolves the array's device
 * address on that device (cudaGetSymbolAddress). All calls share the array and
 * it keeps the last call's contents: calls whose work overlaps on the GPU (from
 * several host threads or streams) race and must be serialised by the caller.
 * Synchronous. HIKF_ENOTPD when a pivot is not positive (d_M unspecified).
 */
#define HIKF_NOALLOC_MAX_N 256
hikf_status hikf_spd_inverse_noalloc(const double* d_S, int n, double* d_M, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HIKF_H */
