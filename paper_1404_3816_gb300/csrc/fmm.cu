// H^2 product C_Q = Q H^T by a black-box FMM with tensor Chebyshev
// interpolation (Sec. 3.2-3.3; Alg. 2 precomputation).
//
// Q H^T = [Q h^(1) ... Q h^(n)]: the n columns of H^T are n source vectors of
// one FMM. Far-field kernel blocks between well-separated boxes B, B' are
// replaced by their Chebyshev interpolant
//     K(x, y) ~ sum_{a,c} S(x; B, a) K(xbar_a^B, ybar_c^B') S(y; B', c),
// with first-kind nodes cos((2k-1)pi/(2p)) per axis and the 1-D weight
// s_p(u, xi) = 1/p + (2/p) sum_{j=1}^{p-1} T_j(u) T_j(xi).
// Passes: P2M (leaf anterpolation), M2M (upward, nested interpolation), M2L
// (interaction lists), L2L (downward), L2P + P2P (near field, exact kernel).
//
// Layout in HBM: the boxes of all levels are concatenated (level l starts at
// box_offset[l], boxes in Morton order); multipole W and local L arrays hold
// [box][q][ld] with the n ray columns contiguous (ld = padded n), so every
// pass streams whole 128-byte rows of n values.
#include <math.h>

#include <algorithm>

#include "hikf_internal.cuh"
#include "m2l_tc.cuh"

namespace hikf {

namespace {

constexpr int kThreads = 256;
constexpr int kPMax = 12;
constexpr int kPT = 64;   // points per chunk in P2M / L2P / P2P
constexpr int kNzStage = 512;   // H^T entries of one source chunk staged in shared memory (P2P)

struct Geo {
  double lo[3];
  double side;
  int dim, depth, p, q, ld, n;
  int pow;                    // HIKF_KERNEL_EXP / GAUSS / GCF / LOG
  double theta, length;
  double shape;               // GCF: the exponent p of Eq. Q; LOG: the self-distance r0
  double kdiag;               // LOG: the value at r = 0, theta log(length / r0)
  double wl;                  // leaf width side / 2^depth (host-computed: no FP64 division per thread)
  double inv_len, inv_len2;   // 1 / length, 1 / length^2
};

__host__ __device__ inline int64_t cmin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t cmax64(int64_t a, int64_t b) { return a > b ? a : b; }

__host__ __device__ constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }

__host__ __device__ inline int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
// tab layout (double): [0, p*p): Tj(xi_k) at [j*p + k]; then T1[c][a'][a] (2*p*p)
__global__ void cheb_tables(int p, double* __restrict__ tab) {
  int t = threadIdx.x;
  const double pi = 3.141592653589793238462643383279502884;
  if (t < p * p) {
    int j = t / p, k = t % p;
    double xi = cos((2.0 * (k + 1) - 1.0) * pi / (2.0 * p));
    tab[t] = cos(j * acos(xi));  // T_j(xi) = cos(j arccos xi)
  }
  __syncthreads();
  if (t < 2 * p * p) {
    int c = t / (p * p), ap = (t / p) % p, a = t % p;
    double xi_ap = cos((2.0 * (ap + 1) - 1.0) * pi / (2.0 * p));
    double u = 0.5 * (xi_ap + (c ? 1.0 : -1.0));  // child node in parent-local coordinates
    // s_p(u, xi_a)
    double s = 1.0 / p, tprev = 1.0, tcur = u;
    for (int j = 1; j < p; ++j) {
      s += (2.0 / p) * tcur * tab[j * p + a];
      double tn = 2.0 * u * tcur - tprev;
      tprev = tcur;
      tcur = tn;
    }
    tab[p * p + t] = s;
  }
}

// K(r) of the kernel families (r2 = r^2):
//   EXP    theta exp(-r / l)            GAUSS  theta exp(-r^2 / l^2)        (Sec. 3.3, kernels 1-2)
//   GCF    theta exp(-(r / l)^p)        (Eq. Q, 0 < p <= 2)
//   LOG    theta log(l / r), r > 0; theta log(l / r0) at r = 0   (Sec. 3.3, kernel 3: A log r
//          with A = -theta < 0, shifted by the constant theta log l; r0 is the stated diagonal)
__device__ __forceinline__ double kernel_value_d(double r2, int fam, double theta, double length, double shape,
                                                 double kdiag) {
  if (fam == HIKF_KERNEL_GAUSS) return theta * exp(-r2 / (length * length));
  if (fam == HIKF_KERNEL_GCF) return theta * exp(-pow(sqrt(r2) / length, shape));
  if (fam == HIKF_KERNEL_LOG) return r2 > 0.0 ? -0.5 * theta * log(r2 / (length * length)) : kdiag;
  return theta * exp(-sqrt(r2) / length);
}

template <typename T>
__device__ __forceinline__ T kernel_value(T r2, int fam, T theta, T inv_len, T inv_len2, T shape, T kdiag);

template <>
__device__ __forceinline__ float kernel_value<float>(float r2, int fam, float theta, float inv_len, float inv_len2,
                                                    float shape, float kdiag) {
  if (fam == HIKF_KERNEL_GAUSS) return theta * expf(-r2 * inv_len2);
  if (fam == HIKF_KERNEL_GCF) return theta * expf(-powf(sqrtf(r2) * inv_len, shape));
  if (fam == HIKF_KERNEL_LOG) return r2 > 0.f ? -0.5f * theta * logf(r2 * inv_len2) : kdiag;
  return theta * expf(-sqrtf(r2) * inv_len);
}
template <>
__device__ __forceinline__ double kernel_value<double>(double r2, int fam, double theta, double inv_len,
                                                       double inv_len2, double shape, double kdiag) {
  if (fam == HIKF_KERNEL_GAUSS) return theta * exp(-r2 * inv_len2);
  if (fam == HIKF_KERNEL_GCF) return theta * exp(-pow(sqrt(r2) * inv_len, shape));
  if (fam == HIKF_KERNEL_LOG) return r2 > 0.0 ? -0.5 * theta * log(r2 * inv_len2) : kdiag;
  return theta * exp(-sqrt(r2) * inv_len);
}

// M2L operator table: kop[(lev-2)][off][a][c] = K(xbar_a^B - ybar_c^{B+off})
template <typename T>
__global__ void m2l_table(Geo g, const double* __restrict__ tab, T* __restrict__ kop, int64_t total) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int q = g.q, p = g.p, dim = g.dim;
  const int noff = ipow(7, dim);
  int c = (int)(t % q);
  int a = (int)((t / q) % q);
  int off = (int)((t / ((int64_t)q * q)) % noff);
  int lev = 2 + (int)(t / ((int64_t)q * q * noff));
  const double pi = 3.141592653589793238462643383279502884;
  double s = g.side / (double)(1 << lev);
  double r2 = 0.0;
  int aa = a, cc = c, oo = off;
  for (int d = dim - 1; d >= 0; --d) {
    int ad = aa % p, cd = cc % p, od = oo % 7 - 3;
    aa /= p;
    cc /= p;
    oo /= 7;
    double xa = cos((2.0 * (ad + 1) - 1.0) * pi / (2.0 * p));
    double xc = cos((2.0 * (cd + 1) - 1.0) * pi / (2.0 * p));
    double diff = 0.5 * s * (xa - xc) - s * od;
    r2 += diff * diff;
  }
  kop[t] = (T)kernel_value_d(r2, g.pow, g.theta, g.length, g.shape, g.kdiag);
}

// per-box count of H^T nonzeros (sources) below the box, and of the box's target points in
// the rows [row0, row1) being formed
__global__ void box_sources(const int64_t* __restrict__ leaf_start, const int64_t* __restrict__ trowptr,
                            const int64_t* __restrict__ box_offset_d, int depth, int dim, int64_t nbox,
                            int64_t row0, int64_t row1, int64_t* __restrict__ nsrc, int64_t* __restrict__ npts) {
  int64_t gb = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gb >= nbox) return;
  int lev = 0;
  while (lev < depth && gb >= box_offset_d[lev + 1]) ++lev;
  int64_t b = gb - box_offset_d[lev];
  int64_t span = (int64_t)1 << (dim * (depth - lev));
  int64_t p0 = leaf_start[b * span], p1 = leaf_start[(b + 1) * span];
  nsrc[gb] = trowptr[p1] - trowptr[p0];
  npts[gb] = max((int64_t)0, min(p1, row1) - max(p0, row0));
}

// 1-D weights s_p(u, xi_k) for k < p, u in [-1, 1]
template <typename T>
__device__ __forceinline__ void weights_1d(T u, int p, const T* __restrict__ tj, T* __restrict__ w) {
  // tj[j*p + k] = T_j(xi_k)
  T tprev = (T)1, tcur = u;
  const T inv = (T)1 / (T)p;
  for (int k = 0; k < p; ++k) w[k] = inv;
  for (int j = 1; j < p; ++j) {
    const T f = (T)2 * inv * tcur;
    for (int k = 0; k < p; ++k) w[k] += f * tj[j * p + k];
    T tn = (T)2 * u * tcur - tprev;
    tprev = tcur;
    tcur = tn;
  }
}

// S[i][a] for the points [ps, ps+cnt) in the leaf with Morton index b; smem out (kPT x q)
template <typename T>
__device__ void leaf_weights(const Geo& g, const double* __restrict__ pts, int64_t ps, int cnt, int64_t b,
                             const T* __restrict__ tj, T* __restrict__ w1 /* kPT*3*kPMax */, T* __restrict__ S) {
  const int p = g.p, dim = g.dim, q = g.q;
  // leaf coordinates of box b from its Morton index
  int64_t c[3] = {0, 0, 0};
  for (int bit = 0; bit < g.depth; ++bit)
    for (int d = 0; d < dim; ++d) c[d] |= ((b >> (bit * dim + (dim - 1 - d))) & 1) << bit;
  const double wl = g.wl;
  for (int t = threadIdx.x; t < cnt * dim; t += blockDim.x) {
    int i = t / dim, d = t % dim;
    double ctr = g.lo[d] + ((double)c[d] + 0.5) * wl;
    T u = (T)((pts[(ps + i) * dim + d] - ctr) / (0.5 * wl));
    weights_1d<T>(u, p, tj, w1 + (i * 3 + d) * kPMax);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < cnt * q; t += blockDim.x) {
    int i = t / q, a = t % q;
    T s = (T)1;
    int aa = a;
    for (int d = dim - 1; d >= 0; --d) {
      s *= w1[(i * 3 + d) * kPMax + aa % p];
      aa /= p;
    }
    S[i * q + a] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// P2M: W_b = S_b^T H^T_b at the leaves
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) p2m_kernel(Geo g, const double* __restrict__ pts,
                                                       const int64_t* __restrict__ leaf_start,
                                                       const int64_t* __restrict__ trowptr,
                                                       const int32_t* __restrict__ tcol,
                                                       const double* __restrict__ tval,
                                                       const double* __restrict__ tab,
                                                       const int64_t* __restrict__ nsrc, int64_t leaf_box0, int nch,
                                                       T* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tj = reinterpret_cast<T*>(smem_raw);                // p*p
  T* w1 = tj + kPMax * kPMax;                            // kPT*3*kPMax
  T* S = w1 + kPT * 3 * kPMax;                           // kPT*q
  T* Hd = S + kPT * g.q;                                 // kPT*nch
  int* act = reinterpret_cast<int*>(Hd + kPT * nch);     // flags (nch), count, active columns (nch)
  const int64_t b = blockIdx.x;
  if (nsrc[leaf_box0 + b] == 0) return;
  const int p = g.p, q = g.q, ld = g.ld;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) tj[t] = (T)tab[t];
  T* Wb = W + (leaf_box0 + b) * (int64_t)q * ld;
  const int64_t p0 = leaf_start[b], p1 = leaf_start[b + 1];
  __syncthreads();
  for (int64_t ps = p0; ps < p1; ps += kPT) {
    const int cnt = (int)cmin64(kPT, p1 - ps);
    leaf_weights<T>(g, pts, ps, cnt, b, tj, w1, S);
    for (int r0 = 0; r0 < ld; r0 += nch) {
      for (int t = threadIdx.x; t < kPT * nch; t += blockDim.x) Hd[t] = (T)0;
      for (int t = threadIdx.x; t < nch; t += blockDim.x) act[t] = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        for (int64_t e = trowptr[ps + i]; e < trowptr[ps + i + 1]; ++e) {
          int r = tcol[e] - r0;
          if (r >= 0 && r < nch) {
            Hd[i * nch + r] += (T)tval[e];
            act[r] = 1;
          }
        }
      }
      __syncthreads();
      // the columns (rays) with a source among these points, in column order; the
      // product below runs over them only (most rays miss a given leaf)
      if (threadIdx.x < 32) {
        int base = 0;
        for (int c0 = 0; c0 < nch; c0 += 32) {
          const int c = c0 + (int)threadIdx.x;
          const bool on = c < nch && act[c] != 0;
          const unsigned bal = __ballot_sync(0xffffffffu, on);
          __syncwarp();
          if (on) act[nch + 1 + base + __popc(bal & ((1u << threadIdx.x) - 1u))] = c;
          base += __popc(bal);
        }
        if (threadIdx.x == 0) act[nch] = base;
      }
      __syncthreads();
      const int nact = act[nch];
      const int* cols = act + nch + 1;
      for (int t = threadIdx.x; t < q * nact; t += blockDim.x) {
        const int a = t / nact, r = cols[t % nact];
        if (r0 + r >= ld) continue;
        T acc = (T)0;
        for (int i = 0; i < cnt; ++i) acc += S[i * q + a] * Hd[i * nch + r];
        Wb[(int64_t)a * ld + r0 + r] += acc;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// separable application of the 1-D transfer along one axis (smem -> smem)
//   dst[a][r] = sum_k M[k][a_ax] src[a with a_ax := k][r]   (forward: M = T1[c] as [child][parent])
//   transposed: dst[a][r] = sum_k M[a_ax][k] src[...k...][r]
// ---------------------------------------------------------------------------
template <typename T>
__device__ void apply_axis(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ M, int p, int q,
                           int dim, int ax, int nch, bool transposed) {
  const int stride = ipow(p, dim - 1 - ax);
  for (int t = threadIdx.x; t < q * nch; t += blockDim.x) {
    int a = t / nch, r = t % nch;
    int aax = (a / stride) % p;
    int base = a - aax * stride;
    T acc = (T)0;
    for (int k = 0; k < p; ++k) {
      T mv = transposed ? M[aax * p + k] : M[k * p + aax];
      acc += mv * src[(base + k * stride) * nch + r];
    }
    dst[t] = acc;
  }
  __syncthreads();
}

// M2M: W_parent = sum_children (T1[c_0] x ... x T1[c_{d-1}])^T W_child
template <typename T>
__global__ void __launch_bounds__(kThreads) m2m_kernel(Geo g, int lev, const double* __restrict__ tab,
                                                       const int64_t* __restrict__ nsrc, int64_t box0,
                                                       int64_t child0, int nch, T* __restrict__ W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = g.p, q = g.q, ld = g.ld, dim = g.dim;
  T* t1 = reinterpret_cast<T*>(smem_raw);  // 2*p*p
  T* acc = t1 + 2 * kPMax * kPMax;         // q*nch
  T* bufA = acc + q * nch;
  T* bufB = bufA + q * nch;
  const int64_t P = blockIdx.x;
  if (nsrc[box0 + P] == 0) return;
  for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) t1[t] = (T)tab[p * p + t];
  const int nchild = 1 << dim;
  for (int r0 = 0; r0 < ld; r0 += nch) {
    const int w = min(nch, ld - r0);
    for (int t = threadIdx.x; t < q * nch; t += blockDim.x) acc[t] = (T)0;
    __syncthreads();
    for (int c = 0; c < nchild; ++c) {
      const int64_t cb = child0 + P * nchild + c;
      if (nsrc[cb] == 0) continue;
      const T* Wc = W + cb * (int64_t)q * ld;
      for (int t = threadIdx.x; t < q * nch; t += blockDim.x) {
        int a = t / nch, r = t % nch;
        bufA[t] = r < w ? Wc[(int64_t)a * ld + r0 + r] : (T)0;
      }
      __syncthreads();
      T* s = bufA;
      T* d = bufB;
      for (int ax = 0; ax < dim; ++ax) {
        int cax = (c >> (dim - 1 - ax)) & 1;
        apply_axis<T>(s, d, t1 + cax * p * p, p, q, dim, ax, nch, false);
        T* tmp = s;
        s = d;
        d = tmp;
      }
      for (int t = threadIdx.x; t < q * nch; t += blockDim.x) acc[t] += s[t];
      __syncthreads();
    }
    T* Wp = W + (box0 + P) * (int64_t)q * ld;
    for (int t = threadIdx.x; t < q * nch; t += blockDim.x) {
      int a = t / nch, r = t % nch;
      if (r < w) Wp[(int64_t)a * ld + r0 + r] = acc[t];
    }
    __syncthreads();
  }
}

// L2L: L_child += (T1[c_0] x ... ) L_parent
template <typename T>
__global__ void __launch_bounds__(kThreads) l2l_kernel(Geo g, int lev, const double* __restrict__ tab,
                                                       const int64_t* __restrict__ npts, int64_t box0,
                                                       int64_t child0, int nch, T* __restrict__ Lx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = g.p, q = g.q, ld = g.ld, dim = g.dim;
  T* t1 = reinterpret_cast<T*>(smem_raw);
  T* par = t1 + 2 * kPMax * kPMax;
  T* bufA = par + q * nch;
  T* bufB = bufA + q * nch;
  const int64_t P = blockIdx.x;
  if (npts[box0 + P] == 0) return;
  for (int t = threadIdx.x; t < 2 * p * p; t += blockDim.x) t1[t] = (T)tab[p * p + t];
  const int nchild = 1 << dim;
  const T* Lp = Lx + (box0 + P) * (int64_t)q * ld;
  for (int r0 = 0; r0 < ld; r0 += nch) {
    const int w = min(nch, ld - r0);
    for (int t = threadIdx.x; t < q * nch; t += blockDim.x) {
      int a = t / nch, r = t % nch;
      par[t] = r < w ? Lp[(int64_t)a * ld + r0 + r] : (T)0;
    }
    __syncthreads();
    for (int c = 0; c < nchild; ++c) {
      const int64_t cb = child0 + P * nchild + c;
      if (npts[cb] == 0) continue;
      const T* s = par;
      T* d = bufA;
      for (int ax = 0; ax < dim; ++ax) {
        int cax = (c >> (dim - 1 - ax)) & 1;
        apply_axis<T>(s, d, t1 + cax * p * p, p, q, dim, ax, nch, true);
        s = d;
        d = (d == bufA) ? bufB : bufA;
      }
      T* Lc = Lx + cb * (int64_t)q * ld;
      for (int t = threadIdx.x; t < q * nch; t += blockDim.x) {
        int a = t / nch, r = t % nch;
        if (r < w) Lc[(int64_t)a * ld + r0 + r] += s[t];
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// M2M / L2L with the box data of one column in registers (q = P^DIM <= 64)
// ---------------------------------------------------------------------------
// One warp per (parent box, 32-column chunk); lane l owns column r0 + l, so every load
// and store of a node row is one coalesced 128-byte access. The separable transfer
// (T1[c_0] x ... x T1[c_{DIM-1}]) is applied axis by axis in registers: for each line of
// P nodes along the axis, P temporaries, the P x P transfer matrix of that axis held in
// registers. M2M: W_P = sum_c (x_ax T1[c_ax])^T W_c (plain store); L2L:
// L_c += (x_ax T1[c_ax]) L_P. T1[cax] is [child node][parent node].
constexpr int kRegWarps = 4;

// cp.async of one 4- or 8-byte element (global -> shared), commit, wait
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, int P, int DIM, bool TRANSPOSED, typename Sink>
__device__ __forceinline__ void transfer_column(T (&x)[ipow_c(P, DIM)], const T* __restrict__ t1s, int c,
                                                Sink&& sink) {
  // forward: out[a] = sum_k T1[k][a] in[k]; transposed: out[a] = sum_k T1[a][k] in[k]. Axes
  // 0 .. DIM-2 are applied in place (P temporaries per line), the last axis streams its
  // outputs into the sink, so only the q inputs are live; every output sums k in order,
  // axis after axis, as the shared-memory kernel does. The matrices stay in shared memory
  // (every lane reads the same entry); the empty asm statements keep the compiler from
  // hoisting later reads over earlier work, which would raise the register count.
  constexpr int Q = ipow_c(P, DIM);
#pragma unroll
  for (int ax = 0; ax + 1 < DIM; ++ax) {
    asm volatile("" ::: "memory");
    const T* mm = t1s + ((c >> (DIM - 1 - ax)) & 1) * P * P;
    int stride = 1;
#pragma unroll
    for (int e = ax + 1; e < DIM; ++e) stride *= P;
#pragma unroll
    for (int o = 0; o < Q / P; ++o) {
      if (Q > 49) asm volatile("" ::: "memory");
      const int base = (o / stride) * stride * P + (o % stride);
      T tmp[P];
#pragma unroll
      for (int a = 0; a < P; ++a) {
        T acc = (T)0;
#pragma unroll
        for (int k = 0; k < P; ++k) acc += (TRANSPOSED ? mm[a * P + k] : mm[k * P + a]) * x[base + k * stride];
        tmp[a] = acc;
      }
#pragma unroll
      for (int a = 0; a < P; ++a) x[base + a * stride] = tmp[a];
    }
  }
  asm volatile("" ::: "memory");
  const T* mm = t1s + (c & 1) * P * P;  // the last axis (stride 1)
#pragma unroll
  for (int a = 0; a < P; ++a) {
    if (Q > 49) asm volatile("" ::: "memory");
    T m0[P];
#pragma unroll
    for (int k = 0; k < P; ++k) m0[k] = TRANSPOSED ? mm[a * P + k] : mm[k * P + a];
#pragma unroll
    for (int o = 0; o < Q / P; ++o) {
      T acc = (T)0;
#pragma unroll
      for (int k = 0; k < P; ++k) acc += m0[k] * x[o * P + k];
      sink(o * P + a, acc);
    }
  }
}

template <typename T, int P, int DIM, bool UP>
__global__ void __launch_bounds__(32 * kRegWarps) transfer_reg_kernel(int ld, const double* __restrict__ tab,
                                                                      const int64_t* __restrict__ cnt,
                                                                      int64_t box0, int64_t child0, int64_t nparent,
                                                                      T* __restrict__ X) {
  constexpr int Q = ipow_c(P, DIM), NC = 1 << DIM;
  __shared__ __align__(16) T t1s[2 * P * P];
  // per warp: the parent's accumulator (M2M) or the parent's values (L2L), [node][lane]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int t = threadIdx.x; t < 2 * P * P; t += blockDim.x) t1s[t] = (T)tab[P * P + t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  T* buf = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * Q * 32 + lane;
  const int nchunk = ld / 32;
  const int64_t item = (int64_t)blockIdx.x * kRegWarps + (threadIdx.x >> 5);
  if (item >= nparent * nchunk) return;
  const int64_t par = item / nchunk;
  const int r = (int)(item % nchunk) * 32 + lane;
  if (cnt[box0 + par] == 0) return;
  T* Xp = X + (box0 + par) * (int64_t)Q * ld + r;
  if (UP) {
    // children with sources, in order; each child's column is copied into one of two
    // shared stages with cp.async while the previous child is transformed, so the
    // transform reads its inputs from shared memory (no values held across global loads)
    int list[NC], nl = 0;
    for (int c = 0; c < NC; ++c)
      if (cnt[child0 + par * NC + c] != 0) list[nl++] = c;
    T* stage = buf + Q * 32 * kRegWarps;  // two per-warp stages after the accumulators
    auto issue = [&](int t) {
      const T* Xc = X + (child0 + par * NC + list[t]) * (int64_t)Q * ld + r;
      T* dst = stage + (t & 1) * Q * 32 * kRegWarps;
#pragma unroll 8
      for (int a = 0; a < Q; ++a) cp_async_elem(dst + a * 32, Xc + (int64_t)a * ld);
      cp_async_commit();
    };
#pragma unroll
    for (int a = 0; a < Q; ++a) buf[a * 32] = (T)0;
    if (nl > 0) issue(0);
    for (int t = 0; t < nl; ++t) {
      if (t + 1 < nl) {
        issue(t + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      const T* src = stage + (t & 1) * Q * 32 * kRegWarps;
      T x[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) x[a] = src[a * 32];
      transfer_column<T, P, DIM, false>(x, t1s, list[t], [&](int a, T v) { buf[a * 32] += v; });
    }
#pragma unroll
    for (int a = 0; a < Q; ++a, Xp += ld) *Xp = buf[a * 32];
  } else {
    // children with points, in order; each child's current column is copied into one of
    // two shared stages with cp.async while the previous child is transformed, the
    // transform adds into the stage, and the stage is written back with plain stores
    int list[NC], nl = 0;
    for (int c = 0; c < NC; ++c)
      if (cnt[child0 + par * NC + c] != 0) list[nl++] = c;
    T* stage = buf + Q * 32 * kRegWarps;
    auto child_col = [&](int t) { return X + (child0 + par * NC + list[t]) * (int64_t)Q * ld + r; };
    auto issue = [&](int t) {
      const T* Xc = child_col(t);
      T* dst = stage + (t & 1) * Q * 32 * kRegWarps;
#pragma unroll 8
      for (int a = 0; a < Q; ++a) cp_async_elem(dst + a * 32, Xc + (int64_t)a * ld);
      cp_async_commit();
    };
    if (nl > 0) issue(0);
#pragma unroll
    for (int a = 0; a < Q; ++a, Xp += ld) buf[a * 32] = *Xp;
    for (int t = 0; t < nl; ++t) {
      if (t + 1 < nl) {
        issue(t + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      T* st = stage + (t & 1) * Q * 32 * kRegWarps;
      T x[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) x[a] = buf[a * 32];
      transfer_column<T, P, DIM, true>(x, t1s, list[t], [&](int a, T v) { st[a * 32] += v; });
      T* Xc = child_col(t);
#pragma unroll 8
      for (int a = 0; a < Q; ++a) Xc[(int64_t)a * ld] = st[a * 32];
    }
  }
}

// launch the register kernel when (p, dim) has an instance; false otherwise
template <typename T, bool UP>
bool launch_transfer_reg(int p, int dim, int ld, const double* tab, const int64_t* cnt, int64_t box0,
                         int64_t child0, int64_t nparent, T* X, cudaStream_t s) {
  if (ld % 32 != 0) return false;
  if (sizeof(T) == 8 && ipow(p, dim) > 36) return false;  // two FP64 q-vectors in registers
  const int64_t items = nparent * (ld / 32);
  const unsigned grid = (unsigned)((items + kRegWarps - 1) / kRegWarps);
  // per warp: the accumulator (M2M) or the parent's values (L2L), plus two stages of a child's column
  const size_t smem = sizeof(T) * (size_t)kRegWarps * ipow(p, dim) * 32 * 3;  // <= 108 KB
#define HIKF_TRANSFER_CASE(PP, DD)                                                                        \
  if (p == PP && dim == DD) {                                                                             \
    if (cudaFuncSetAttribute(transfer_reg_kernel<T, PP, DD, UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem) != cudaSuccess)                                                   \
      return false;                                                                                       \
    transfer_reg_kernel<T, PP, DD, UP><<<grid, 32 * kRegWarps, smem, s>>>(ld, tab, cnt, box0, child0, nparent, X); \
    return true;                                                                                          \
  }
  HIKF_TRANSFER_CASE(2, 2)
  HIKF_TRANSFER_CASE(3, 2)
  HIKF_TRANSFER_CASE(4, 2)
  HIKF_TRANSFER_CASE(5, 2)
  HIKF_TRANSFER_CASE(6, 2)
  HIKF_TRANSFER_CASE(7, 2)
  HIKF_TRANSFER_CASE(8, 2)
  HIKF_TRANSFER_CASE(2, 3)
  HIKF_TRANSFER_CASE(3, 3)
  HIKF_TRANSFER_CASE(4, 3)
#undef HIKF_TRANSFER_CASE
  return false;
}

// ---------------------------------------------------------------------------
// M2L: L_B += sum_{B' in IL(B)} K_{lev, B'-B} W_B'   (tiled GEMM over the list)
// ---------------------------------------------------------------------------
constexpr int kM2L_BM = 64, kM2L_BN = 64, kM2L_BK = 16;

template <typename T>
__global__ void __launch_bounds__(kThreads) m2l_kernel(Geo g, int lev, const T* __restrict__ kop,
                                                       const int64_t* __restrict__ nsrc,
                                                       const int64_t* __restrict__ npts, int64_t box0,
                                                       const T* __restrict__ W, T* __restrict__ Lx) {
  __shared__ T As[kM2L_BK][kM2L_BM];
  __shared__ T Bs[kM2L_BK][kM2L_BN];
  __shared__ int il_box[216];
  __shared__ int il_off[216];
  __shared__ int il_n;
  const int q = g.q, ld = g.ld, dim = g.dim;
  const int64_t B = blockIdx.x;
  if (npts[box0 + B] == 0) return;
  const int a0 = blockIdx.y * kM2L_BM, r0 = blockIdx.z * kM2L_BN;
  if (r0 >= ld) return;
  // box coordinates from Morton index
  int64_t cb[3] = {0, 0, 0};
  for (int bit = 0; bit < lev; ++bit)
    for (int d = 0; d < dim; ++d) cb[d] |= ((B >> (bit * dim + (dim - 1 - d))) & 1) << bit;
  if (threadIdx.x == 0) il_n = 0;
  __syncthreads();
  // candidates: children of the parent's neighbours, offsets in [-3, 3]^dim relative to B
  const int ncand = ipow(6, dim);
  for (int t = threadIdx.x; t < ncand; t += blockDim.x) {
    int tt = t;
    int64_t cc[3] = {0, 0, 0};
    int offs[3] = {0, 0, 0};
    bool ok = true, sep = false;
    for (int d = dim - 1; d >= 0; --d) {
      int k = tt % 6;
      tt /= 6;
      cc[d] = 2 * (cb[d] >> 1) - 2 + k;
      offs[d] = (int)(cc[d] - cb[d]);
      if (cc[d] < 0 || cc[d] >= ((int64_t)1 << lev)) ok = false;
      if (offs[d] > 1 || offs[d] < -1) sep = true;
    }
    if (!ok || !sep) continue;
    int64_t key = 0;
    for (int bit = lev - 1; bit >= 0; --bit)
      for (int d = 0; d < dim; ++d) key = (key << 1) | ((cc[d] >> bit) & 1);
    if (nsrc[box0 + key] == 0) continue;
    int oi = 0;
    for (int d = 0; d < dim; ++d) oi = oi * 7 + (offs[d] + 3);
    int slot = atomicAdd(&il_n, 1);
    il_box[slot] = (int)key;
    il_off[slot] = oi;
  }
  __syncthreads();
  const int nil = il_n;
  if (nil == 0) return;
  // deterministic order of the list
  if (threadIdx.x == 0) {
    for (int i = 1; i < nil; ++i) {
      int kb = il_box[i], ko = il_off[i], j = i - 1;
      while (j >= 0 && il_box[j] > kb) {
        il_box[j + 1] = il_box[j];
        il_off[j + 1] = il_off[j];
        --j;
      }
      il_box[j + 1] = kb;
      il_off[j + 1] = ko;
    }
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 4 x 4 outputs each
  T acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
  const int noff = ipow(7, dim);
  const T* kl = kop + (int64_t)(lev - 2) * noff * q * q;
  const int kblocks = (q + kM2L_BK - 1) / kM2L_BK;
  for (int e = 0; e < nil; ++e) {
    const T* K = kl + (int64_t)il_off[e] * q * q;
    const T* Ws = W + (box0 + il_box[e]) * (int64_t)q * ld;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int c0 = kb * kM2L_BK;
      for (int t = threadIdx.x; t < kM2L_BK * kM2L_BM; t += blockDim.x) {
        int a = t / kM2L_BK, kk = t % kM2L_BK;
        As[kk][a] = (a0 + a < q && c0 + kk < q) ? K[(int64_t)(a0 + a) * q + c0 + kk] : (T)0;
      }
      for (int t = threadIdx.x; t < kM2L_BK * kM2L_BN; t += blockDim.x) {
        int kk = t / kM2L_BN, r = t % kM2L_BN;
        Bs[kk][r] = (c0 + kk < q && r0 + r < ld) ? Ws[(int64_t)(c0 + kk) * ld + r0 + r] : (T)0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kM2L_BK; ++kk) {
        T av[4], bv[4];
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
      }
      __syncthreads();
    }
  }
  T* Lb = Lx + (box0 + B) * (int64_t)q * ld;
  for (int i = 0; i < 4; ++i) {
    int a = a0 + ty * 4 + i;
    if (a >= q) continue;
    for (int j = 0; j < 4; ++j) {
      int r = r0 + tx + 16 * j;
      if (r < ld) Lb[(int64_t)a * ld + r] += acc[i][j];
    }
  }
}

// eight consecutive values from a 16-byte aligned address
__device__ __forceinline__ void load8(const float* __restrict__ p, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const double* __restrict__ p, double (&v)[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 a = reinterpret_cast<const double2*>(p)[k];
    v[2 * k] = a.x;
    v[2 * k + 1] = a.y;
  }
}

// ---------------------------------------------------------------------------
// L2P + P2P: C_Q rows of one leaf
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) l2p_p2p_kernel(Geo g, const double* __restrict__ pts,
                                                           const int64_t* __restrict__ leaf_start,
                                                           const int64_t* __restrict__ trowptr,
                                                           const int32_t* __restrict__ tcol,
                                                           const double* __restrict__ tval,
                                                           const double* __restrict__ tab,
                                                           const int64_t* __restrict__ nsrc, int64_t leaf_box0,
                                                           int nch, const T* __restrict__ Lx, int64_t row0,
                                                           int64_t row1, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = g.p, q = g.q, ld = g.ld, dim = g.dim, L = g.depth;
  T* tj = reinterpret_cast<T*>(smem_raw);
  T* w1 = tj + kPMax * kPMax;
  T* S = w1 + kPT * 3 * kPMax;
  T* Cs = S + kPT * q;                  // kPT x (nch + 1)
  T* tx = Cs + kPT * (nch + 1);         // kPT x 3 target coords relative to the leaf centre
  T* sx = tx + kPT * 3;                 // kPT x 3 staged source coords
  int64_t* se = reinterpret_cast<int64_t*>(sx + kPT * 3 + 2);  // kPT x 2 H^T row ranges (8-byte aligned)
  // kPT sources x kPT targets: kernel values. With one column chunk and q >= kPT they share
  // storage with S (kPT x q): within a chunk of points, L2P reads S before P2P starts and
  // S is formed again for the next chunk (the launch sizes shared memory the same way)
  const bool alias_kv = q >= kPT && nch >= ld;
  T* kvs = alias_kv ? S : reinterpret_cast<T*>(se + 2 * kPT);
  T* zv = reinterpret_cast<T*>(se + 2 * kPT) + (alias_kv ? 0 : kPT * kPT);  // the chunk's H^T values (kNzStage)
  int* zc = reinterpret_cast<int*>(zv + kNzStage);              // and their ray indices
  __shared__ int se_cnt[2];                                     // crossed sources per staging warp
  const int64_t b = blockIdx.x;
  // the leaf's points within the rows being formed; out holds row row0 first
  const int64_t p0 = cmax64(leaf_start[b], row0), p1 = cmin64(leaf_start[b + 1], row1);
  if (p1 <= p0) return;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) tj[t] = (T)tab[t];
  int64_t cb[3] = {0, 0, 0};
  for (int bit = 0; bit < L; ++bit)
    for (int d = 0; d < dim; ++d) cb[d] |= ((b >> (bit * dim + (dim - 1 - d))) & 1) << bit;
  const double wl = g.wl;
  double ctr[3];
  for (int d = 0; d < dim; ++d) ctr[d] = g.lo[d] + ((double)cb[d] + 0.5) * wl;
  const T theta = (T)g.theta, inv_len = (T)g.inv_len, inv_len2 = (T)g.inv_len2;
  const T* Lb = Lx + (leaf_box0 + b) * (int64_t)q * ld;
  const int nnb = ipow(3, dim);
  const int parts = kThreads / kPT;  // threads per target point
  __syncthreads();
  for (int64_t ps = p0; ps < p1; ps += kPT) {
    const int cnt = (int)cmin64(kPT, p1 - ps);
    if (L >= 2) leaf_weights<T>(g, pts, ps, cnt, b, tj, w1, S);
    for (int t = threadIdx.x; t < cnt * dim; t += blockDim.x) {
      int i = t / dim, d = t % dim;
      tx[i * 3 + d] = (T)(pts[(ps + i) * dim + d] - ctr[d]);
    }
    __syncthreads();
    for (int r0 = 0; r0 < ld; r0 += nch) {
      const int w = min(nch, ld - r0);
      // L2P: a PT-point x 8-column register tile per thread (8 points in FP32, so each entry
      // of L is read by kPT / 8 threads; 4 in FP64, for the registers); L rows read as
      // 16-byte vectors; every output sums over a in the same order whatever PT is
      {
        constexpr int PT = sizeof(T) == 4 ? 8 : 4;
        const int ncg = nch / 8, ntile = (kPT / PT) * ncg;
        for (int t = threadIdx.x; t < ntile; t += blockDim.x) {
          const int i0 = (t / ncg) * PT, c0 = (t % ncg) * 8;
          T acc[PT][8];
#pragma unroll
          for (int u = 0; u < PT; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = (T)0;
          if (L >= 2 && i0 < cnt && c0 < w) {
            const T* lrow = Lb + r0 + c0;
            for (int a = 0; a < q; ++a) {
              T lv[8];
              load8(lrow + (int64_t)a * ld, lv);
              T sv[PT];
#pragma unroll
              for (int u = 0; u < PT; ++u) sv[u] = i0 + u < cnt ? S[(i0 + u) * q + a] : (T)0;
#pragma unroll
              for (int u = 0; u < PT; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] += sv[u] * lv[v];
            }
          }
#pragma unroll
          for (int u = 0; u < PT; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) Cs[(i0 + u) * (nch + 1) + c0 + v] = acc[u][v];
        }
      }
      __syncthreads();
      // P2P over the touching leaves (exact kernel, sparse sources); the source
      // coordinates relative to this leaf's centre are staged once per chunk
      const int i = threadIdx.x % kPT, part = threadIdx.x / kPT;
      const int cw = (nch + parts - 1) / parts;
      const int rlo = part * cw, rhi = min(nch, rlo + cw);
      for (int nb = 0; nb < nnb; ++nb) {
        int64_t cn[3] = {0, 0, 0};
        int tt = nb;
        bool ok = true;
        for (int d = dim - 1; d >= 0; --d) {
          cn[d] = cb[d] + (tt % 3) - 1;
          tt /= 3;
          if (cn[d] < 0 || cn[d] >= ((int64_t)1 << L)) ok = false;
        }
        if (!ok) continue;
        int64_t key = 0;
        for (int bit = L - 1; bit >= 0; --bit)
          for (int d = 0; d < dim; ++d) key = (key << 1) | ((cn[d] >> bit) & 1);
        if (nsrc[leaf_box0 + key] == 0) continue;
        for (int64_t js = leaf_start[key]; js < leaf_start[key + 1]; js += kPT) {
          const int jc = (int)cmin64(kPT, leaf_start[key + 1] - js);
          // stage only the sources some ray crosses, in point order (most cells are
          // crossed by none); kPT = 64 sources are compacted by two warps' ballots
          if (threadIdx.x < kPT) {
            const int t = (int)threadIdx.x;
            int64_t e0 = 0, e1 = 0;
            if (t < jc) {
              e0 = trowptr[js + t];
              e1 = trowptr[js + t + 1];
            }
            const bool on = e1 > e0;
            const unsigned bal = __ballot_sync(0xffffffffu, on);
            const int below = __popc(bal & ((1u << (t & 31)) - 1u));
            if ((t & 31) == 0) se_cnt[t >> 5] = __popc(bal);
            __syncwarp();
            // warp 1 needs warp 0's count: publish it through shared memory first
            asm volatile("bar.sync 1, 64;" ::: "memory");
            const int slot = (t >> 5 ? se_cnt[0] : 0) + below;
            if (on) {
              se[2 * slot] = e0;
              se[2 * slot + 1] = e1;
              for (int d = 0; d < dim; ++d) sx[slot * 3 + d] = (T)(pts[(js + t) * dim + d] - ctr[d]);
            }
          }
          __syncthreads();
          const int ns = se_cnt[0] + se_cnt[1];
          // every (target, source) kernel value once, shared by the column parts
          for (int t = threadIdx.x; t < ns * kPT; t += blockDim.x) {
            const int j = t / kPT, ii = t % kPT;
            T v = (T)0;
            if (ii < cnt) {
              T r2 = (T)0;
              for (int d = 0; d < dim; ++d) {
                T dx = tx[ii * 3 + d] - sx[j * 3 + d];
                r2 += dx * dx;
              }
              v = kernel_value<T>(r2, g.pow, theta, inv_len, inv_len2, (T)g.shape, (T)g.kdiag);
            }
            kvs[j * kPT + ii] = v;
          }
          // the chunk's H^T entries are one contiguous range; stage it when it fits
          const int64_t eb = trowptr[js], ne = trowptr[js + jc] - eb;
          const bool staged = ne <= kNzStage;
          if (staged)
            for (int t = threadIdx.x; t < (int)ne; t += blockDim.x) {
              zc[t] = tcol[eb + t];
              zv[t] = (T)tval[eb + t];
            }
          __syncthreads();
          if (i < cnt) {
            for (int j = 0; j < ns; ++j) {
              const int64_t e0 = se[2 * j], e1 = se[2 * j + 1];
              const T kv = kvs[j * kPT + i];
              if (staged) {
                for (int e = (int)(e0 - eb); e < (int)(e1 - eb); ++e) {
                  const int r = zc[e] - r0;
                  if (r >= rlo && r < rhi) Cs[i * (nch + 1) + r] += kv * zv[e];
                }
              } else {
                for (int64_t e = e0; e < e1; ++e) {
                  int r = tcol[e] - r0;
                  if (r >= rlo && r < rhi) Cs[i * (nch + 1) + r] += kv * (T)tval[e];
                }
              }
            }
          }
          __syncthreads();
        }
      }
      for (int t = threadIdx.x; t < cnt * nch; t += blockDim.x) {
        int ii = t / nch, r = t % nch;
        if (r < w) out[(ps + ii - row0) * (int64_t)ld + r0 + r] = Cs[ii * (nch + 1) + r];
      }
      __syncthreads();
    }
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <typename T>
Status set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) HIKF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return Status::Ok();
}

}  // namespace

template <typename T>
Status h2_product(const Tree& t, const SparseH& h, const FmmParams& fp, T* out, int ldc, cudaStream_t s,
                  int64_t row0, int64_t row1) {
  Geo g;
  for (int d = 0; d < 3; ++d) g.lo[d] = t.lo[d];
  g.side = t.side;
  g.dim = t.dim;
  g.depth = t.depth;
  g.p = fp.order;
  g.q = ipow(fp.order, t.dim);
  g.ld = ldc;
  g.n = h.n;
  g.pow = fp.pow;
  g.theta = fp.theta;
  g.length = fp.length;
  g.shape = fp.shape;
  g.kdiag = fp.pow == HIKF_KERNEL_LOG ? fp.theta * std::log(fp.length / fp.shape) : 0.0;
  g.wl = t.side / (double)((int64_t)1 << t.depth);
  g.inv_len = 1.0 / fp.length;
  g.inv_len2 = 1.0 / (fp.length * fp.length);
  const int p = g.p, q = g.q, L = t.depth, dim = t.dim;
  const int64_t nbox = t.nbox_total;
  const int64_t m = t.m;
  if (row1 < 0) row1 = m;
  if (row0 < 0 || row1 > m || row0 >= row1) return make_status(HIKF_EINVAL, "H^2 product: empty or bad row range");

  HIKF_CUDA(cudaMemsetAsync(out, 0, sizeof(T) * (size_t)(row1 - row0) * ldc, s));
  // column chunk: keep q * nch * sizeof(T) * 3 within ~150 KB
  int nch = 128;
  while (nch > 32 && (size_t)q * nch * sizeof(T) * 3 > 150 * 1024) nch /= 2;
  nch = std::min(nch, ldc);

  double* tab = nullptr;
  int64_t *nsrc = nullptr, *npts = nullptr, *boff = nullptr;
  T *W = nullptr, *Lx = nullptr, *kop = nullptr;
  const size_t boxbytes = sizeof(T) * (size_t)q * ldc;
  HIKF_CUDA(hikf::pool_malloc((void**)&tab, sizeof(double) * 3 * kPMax * kPMax, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&nsrc, sizeof(int64_t) * nbox, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&npts, sizeof(int64_t) * nbox, s));
  HIKF_CUDA(hikf::pool_malloc((void**)&boff, sizeof(int64_t) * (L + 2), s));
  HIKF_CUDA(cudaMemcpyAsync(boff, t.box_offset, sizeof(int64_t) * (L + 2), cudaMemcpyHostToDevice, s));
  cheb_tables<<<1, 512, 0, s>>>(p, tab);
  HIKF_LAUNCH_CHECK("cheb_tables");
  box_sources<<<nblk(nbox, kThreads), kThreads, 0, s>>>(t.leaf_start, h.trowptr, boff, L, dim, nbox, row0, row1,
                                                         nsrc, npts);
  HIKF_LAUNCH_CHECK("box_sources");

  const int64_t leaf0 = t.box_offset[L];
  const size_t smem_pts = sizeof(T) * (kPMax * kPMax + kPT * 3 * kPMax + (size_t)kPT * q);
  if (L >= 2) {
    HIKF_CUDA(hikf::pool_malloc((void**)&W, boxbytes * nbox, s));
    HIKF_CUDA(hikf::pool_malloc((void**)&Lx, boxbytes * nbox, s));
    HIKF_CUDA(cudaMemsetAsync(W, 0, boxbytes * nbox, s));
    HIKF_CUDA(cudaMemsetAsync(Lx, 0, boxbytes * nbox, s));
    const int noff = ipow(7, dim);
    const int64_t ktotal = (int64_t)(L - 1) * noff * q * q;
    HIKF_CUDA(hikf::pool_malloc((void**)&kop, sizeof(T) * ktotal, s));
    m2l_table<T><<<nblk(ktotal, kThreads), kThreads, 0, s>>>(g, tab, kop, ktotal);
    HIKF_LAUNCH_CHECK("m2l_table");
    // P2M
    {
      size_t sm = smem_pts + sizeof(T) * kPT * nch + sizeof(int) * (2 * (size_t)nch + 1);
      HIKF_TRY(set_smem<T>((const void*)p2m_kernel<T>, sm));
      p2m_kernel<T><<<(unsigned)t.nleaf, kThreads, sm, s>>>(g, t.pts, t.leaf_start, h.trowptr, h.tcol, h.tval, tab,
                                                             nsrc, leaf0, nch, W);
      HIKF_LAUNCH_CHECK("p2m");
    }
    // M2M, levels L-1 .. 2
    {
      size_t sm = sizeof(T) * (2 * kPMax * kPMax + 3 * (size_t)q * nch);
      HIKF_TRY(set_smem<T>((const void*)m2m_kernel<T>, sm));
      for (int lev = L - 1; lev >= 2; --lev) {
        const int64_t npar = (int64_t)1 << (dim * lev);
        if (!launch_transfer_reg<T, true>(p, dim, ldc, tab, nsrc, t.box_offset[lev], t.box_offset[lev + 1], npar, W,
                                          s))
          m2m_kernel<T><<<(unsigned)npar, kThreads, sm, s>>>(g, lev, tab, nsrc, t.box_offset[lev],
                                                            t.box_offset[lev + 1], nch, W);
        HIKF_LAUNCH_CHECK("m2m");
      }
    }
    // M2L, all levels 2 .. L
    const bool tc = fp.tensor_m2l && sizeof(T) == 4 && m2l_tc_supported(q, ldc) && L - 1 <= 16;
    if (tc) {
      int* err = nullptr;
      HIKF_CUDA(hikf::pool_malloc((void**)&err, sizeof(int), s));
      HIKF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
      M2lTcAll ma;
      ma.dim = dim;
      ma.q = q;
      ma.ld = ldc;
      ma.sms = fp.sms;
      ma.nlev = L - 1;
      for (int lev = 2; lev <= L; ++lev) {
        ma.lev[lev - 2] = lev;
        ma.box0[lev - 2] = t.box_offset[lev];
        ma.nbox[lev - 2] = (int64_t)1 << (dim * lev);
      }
      ma.W = (const float*)W;
      ma.L = (float*)Lx;
      ma.kop = (const float*)kop;
      ma.nsrc = nsrc;
      ma.npts = npts;
      ma.err = err;
      ma.autotune = fp.autotune;
      Status st = m2l_tc_all(ma, s);
      int herr = 0;
      HIKF_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      HIKF_CUDA(cudaStreamSynchronize(s));
      HIKF_CUDA(cudaFreeAsync(err, s));
      HIKF_TRY(st);
      if (herr) return make_status(HIKF_ETIMEOUT, "a bounded wait in the tensor-core M2L timed out");
    } else {
      for (int lev = 2; lev <= L; ++lev) {
        dim3 grid((unsigned)((int64_t)1 << (dim * lev)), (unsigned)((q + kM2L_BM - 1) / kM2L_BM),
                  (unsigned)((ldc + kM2L_BN - 1) / kM2L_BN));
        m2l_kernel<T><<<grid, kThreads, 0, s>>>(g, lev, kop, nsrc, npts, t.box_offset[lev], W, Lx);
        HIKF_LAUNCH_CHECK("m2l");
      }
    }
    // L2L, levels 2 .. L-1 (parent level)
    {
      size_t sm = sizeof(T) * (2 * kPMax * kPMax + 3 * (size_t)q * nch);
      HIKF_TRY(set_smem<T>((const void*)l2l_kernel<T>, sm));
      for (int lev = 2; lev <= L - 1; ++lev) {
        const int64_t npar = (int64_t)1 << (dim * lev);
        if (!launch_transfer_reg<T, false>(p, dim, ldc, tab, npts, t.box_offset[lev], t.box_offset[lev + 1], npar,
                                           Lx, s))
          l2l_kernel<T><<<(unsigned)npar, kThreads, sm, s>>>(g, lev, tab, npts, t.box_offset[lev],
                                                            t.box_offset[lev + 1], nch, Lx);
        HIKF_LAUNCH_CHECK("l2l");
      }
    }
  }
  // L2P + P2P at the leaves
  {
    int nchp = ldc;
    // P2P tables: kernel values (kPT x kPT) and the staged H^T entries of a source chunk
    const size_t p2p_full = sizeof(T) * ((size_t)kPT * kPT + kNzStage) + sizeof(int) * kNzStage;
    while (nchp > 32 && smem_pts + p2p_full + sizeof(T) * (size_t)kPT * (nchp + 1) > 190 * 1024) nchp /= 2;
    nchp = std::max(8, nchp / 8 * 8);  // the L2P tile reads 8 columns at a time
    // the kernel-value table lives in S's storage when there is one column chunk (as in the kernel)
    const bool alias_kv = q >= kPT && nchp >= ldc;
    const size_t p2p = p2p_full - (alias_kv ? sizeof(T) * (size_t)kPT * kPT : 0);
    size_t sm = smem_pts + sizeof(T) * ((size_t)kPT * (nchp + 1) + kPT * 6 + 4) + sizeof(int64_t) * 2 * kPT + p2p;
    HIKF_TRY(set_smem<T>((const void*)l2p_p2p_kernel<T>, sm));
    l2p_p2p_kernel<T><<<(unsigned)t.nleaf, kThreads, sm, s>>>(g, t.pts, t.leaf_start, h.trowptr, h.tcol, h.tval,
                                                                tab, nsrc, leaf0, nchp, Lx, row0, row1, out);
    HIKF_LAUNCH_CHECK("l2p_p2p");
  }
  HIKF_CUDA(cudaFreeAsync(tab, s));
  HIKF_CUDA(cudaFreeAsync(nsrc, s));
  HIKF_CUDA(cudaFreeAsync(npts, s));
  HIKF_CUDA(cudaFreeAsync(boff, s));
  if (W) HIKF_CUDA(cudaFreeAsync(W, s));
  if (Lx) HIKF_CUDA(cudaFreeAsync(Lx, s));
  if (kop) HIKF_CUDA(cudaFreeAsync(kop, s));
  return Status::Ok();
}

template Status h2_product<float>(const Tree&, const SparseH&, const FmmParams&, float*, int, cudaStream_t, int64_t,
                                  int64_t);
template Status h2_product<double>(const Tree&, const SparseH&, const FmmParams&, double*, int, cudaStream_t, int64_t,
                                   int64_t);

}  // namespace hikf
