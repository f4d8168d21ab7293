// Differentiation of the two objectives the method is trained or evaluated
// with, on the GPU:
//
//   * the subspace loss L(P_hat) = ||(I - Q Q^T) B||_F^2 with Q = qf(P_hat)
//     (Sec. 3, the QR layer after the learned map; the residual energy whose minimisation is the
//     maximisation of the subspace energy, Appendix on optimality) and its
//     gradient through the thin-QR layer;
//   * the residual norm ||r_T|| after T unrolled PCG iterations with the
//     two-level preconditioner of Algorithm 1 built from a full-rank P
//     (A_c = P^T A P), x0 = 0, and its gradient with respect to P by reverse
//     mode through the iterations (forward states kept as per-iteration
//     checkpoints).
//
// Vectors of the PCG recurrences are FP64; the preconditioner pieces run in
// the preconditioner precision T (FP32 production, FP64 for checks).  All
// scalars of the recurrences stay on the device, so a call enqueues its work
// without host round trips until the loss is read back.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "stencil.cuh"

namespace {

constexpr int VB = 256;  // threads per block of the vector kernels

// ---------------------------------------------------------------------------
// FP64 vector kernels with device-side coefficients:
//   coef = mult * (ia >= 0 ? S[ia] : 1) / (ib >= 0 ? S[ib] : 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double coef_of(const double* S, int ia, int ib, double mult) {
  double c = mult;
  if (ia >= 0) c *= S[ia];
  if (ib >= 0) c /= S[ib];
  return c;
}

// Block partial sums of x . y (fixed order: deterministic).
__global__ void __launch_bounds__(VB) k_vdot_part(const double* __restrict__ x, const double* __restrict__ y,
                                                  int64_t n, double* __restrict__ part) {
  __shared__ double sm[VB / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * VB + threadIdx.x; i < n; i += (int64_t)gridDim.x * VB) s = fma(x[i], y[i], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < VB / 32 ? sm[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// S[out] = sum of nb partials in block order (one warp).
__global__ void k_vdot_fin(const double* __restrict__ part, int nb, double* S, int out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) s += part[b];
  s = warp_sum(s);
  if (threadIdx.x == 0) S[out] = s;
}

__global__ void k_vaxpy(double* __restrict__ y, const double* __restrict__ x, int64_t n, const double* S, int ia,
                        int ib, double mult) {
  const double c = coef_of(S, ia, ib, mult);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(c, x[i], y[i]);
}

// y = c x (x may alias y)
__global__ void k_vscale(double* y, const double* x, int64_t n, const double* S, int ia, int ib, double mult) {
  const double c = coef_of(S, ia, ib, mult);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = c * x[i];
}

// y = x + c y
__global__ void k_vxpay(double* __restrict__ y, const double* __restrict__ x, int64_t n, const double* S, int ia,
                        int ib, double mult) {
  const double c = coef_of(S, ia, ib, mult);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(c, y[i], x[i]);
}

// y = A x, or y += A x
template <int KIND>
__global__ void k_vspmv(StencilView<double> A, const double* __restrict__ x, double* __restrict__ y, int accumulate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return x[m]; });
    y[i] = accumulate ? y[i] + v : v;
  }
}

// ---------------------------------------------------------------------------
// Scalars of the unrolled recurrences, in one FP64 array S on the device.
// ---------------------------------------------------------------------------
struct ScalarIndex {
  int T;
  __host__ __device__ int gam(int t) const { return t; }                // gamma_t = r_t . z_t
  __host__ __device__ int del(int t) const { return (T + 1) + t; }      // delta_t = p_t . q_t
  __host__ __device__ int alp(int t) const { return 2 * (T + 1) + t; }  // alpha_t
  __host__ __device__ int bet(int t) const { return 3 * (T + 1) + t; }  // beta_t
  __host__ __device__ int gbar(int t) const { return 4 * (T + 1) + t; }  // adjoint of gamma_t
  __host__ __device__ int x0() const { return 5 * (T + 1); }            // scratch dot products
  __host__ __device__ int x1() const { return x0() + 1; }
  __host__ __device__ int x2() const { return x0() + 2; }               // adjoint of delta_t
  __host__ __device__ int loss() const { return x0() + 3; }
  __host__ __device__ int rr() const { return x0() + 4; }
  __host__ __device__ int count() const { return x0() + 5; }
};

enum ScalarOp { OP_INIT = 0, OP_ALPHA, OP_BETA, OP_LOSS, OP_REV_BETA, OP_REV_ALPHA };

// One step of the scalar part of the recurrences (one thread).
__global__ void k_scalar(double* S, ScalarIndex ix, int op, int t) {
  switch (op) {
    case OP_INIT:
      for (int i = 0; i < ix.count(); ++i) S[i] = 0.0;
      break;
    case OP_ALPHA:  // alpha_t = gamma_t / delta_t
      S[ix.alp(t)] = S[ix.gam(t)] / S[ix.del(t)];
      break;
    case OP_BETA:  // beta_t = gamma_{t+1} / gamma_t
      S[ix.bet(t)] = S[ix.gam(t + 1)] / S[ix.gam(t)];
      break;
    case OP_LOSS:
      S[ix.loss()] = sqrt(S[ix.rr()]);
      break;
    case OP_REV_BETA: {  // beta_t = gamma_{t+1} / gamma_t, with beta_bar in x0
      const double bb = S[ix.x0()], g = S[ix.gam(t)];
      S[ix.gbar(t + 1)] += bb / g;
      S[ix.gbar(t)] -= bb * S[ix.gam(t + 1)] / (g * g);
      break;
    }
    case OP_REV_ALPHA: {  // alpha_t = gamma_t / delta_t, alpha_bar = -(q_t . rbar_{t+1}) in x1
      const double ab = -S[ix.x1()], d = S[ix.del(t)];
      S[ix.gbar(t)] += ab / d;
      S[ix.x2()] = -ab * S[ix.gam(t)] / (d * d);
      break;
    }
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// Preconditioner pieces in precision T (node-tiled P, n_pad rows).
// ---------------------------------------------------------------------------
// zout = zin + w D^-1 (v - A zin); zin == null means zin = 0.
template <int KIND, typename T>
__global__ void k_jsweep(StencilView<T> A, T omega, const double* __restrict__ v, const T* __restrict__ zin,
                         T* __restrict__ zout) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    T az = T(0), zi = T(0);
    if (zin) {
      az = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return zin[m]; });
      zi = zin[i];
    }
    zout[i] = zi + omega * stencil_dinv<KIND>(A, i) * ((T)v[i] - az);
  }
}

// Transposed sweep operator: wout = (I - w D^-1 A)^T win = win - A (w D^-1 win).
template <int KIND, typename T>
__global__ void k_jsweep_t(StencilView<T> A, T omega, const T* __restrict__ win, T* __restrict__ wout) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const T az = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N),
                                     [&](int64_t m) { return omega * stencil_dinv<KIND>(A, m) * win[m]; });
    wout[i] = win[i] - az;
  }
}

// rho = v - A z
template <int KIND, typename T>
__global__ void k_resid(StencilView<T> A, const double* __restrict__ v, const T* __restrict__ z,
                        T* __restrict__ rho) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x)
    rho[i] = (T)v[i] - stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return z[m]; });
}

// Block partials of P^T x (k columns, x of length n_pad with zero padding):
// warp w owns columns w, w + 8, ..., each lane four nodes of every tile.
constexpr int RV_THREADS = 256;
constexpr int RV_MAXC = 16;  // columns per warp (k <= 128)

template <typename T>
__global__ void __launch_bounds__(RV_THREADS) k_restrict_vec(const T* __restrict__ P, int k, int64_t n_pad,
                                                            const T* __restrict__ x, double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T acc[RV_MAXC];
#pragma unroll
  for (int j = 0; j < RV_MAXC; ++j) acc[j] = T(0);
  const int64_t ntiles = n_pad / NLSP_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    T xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = x[t * NLSP_TILE + lane + 32 * u];
    // all of the warp's column loads of the tile first, then the products
    T pv[RV_MAXC][4];
#pragma unroll
    for (int j = 0; j < RV_MAXC; ++j) {
      const int col = warp + 8 * j;
      const T* src = P + (t * k + (col < k ? col : 0)) * NLSP_TILE;
#pragma unroll
      for (int u = 0; u < 4; ++u) pv[j][u] = col < k ? src[lane + 32 * u] : T(0);
    }
#pragma unroll
    for (int j = 0; j < RV_MAXC; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[j] += pv[j][u] * xv[u];
  }
  // warp sums in T (the accumulation precision; FP32 shuffles and adds are
  // cheap), stored as FP64 block partials
#pragma unroll
  for (int j = 0; j < RV_MAXC; ++j) {
    const int col = warp + 8 * j;
    const T s = warp_sum(acc[j]);
    if (lane == 0 && col < k) part[(int64_t)blockIdx.x * k + col] = (double)s;
  }
}

// c = sum of the nb block partials, e = A_c^-1 c (FP64; k <= 128).  Block j
// adds column j in a fixed order (the threads' strided sums, then a tree) and
// stores it in cbuf; the last block to finish forms e from cbuf.  Spreading
// the nb k FP64 additions over k blocks keeps them off one SM's FP64 pipe
// (GB300 runs FP64 at 1/64 of the FP32 rate).  c_out / e_out may be null.
constexpr int CC_THREADS = 256;

__global__ void __launch_bounds__(CC_THREADS) k_coarse_cols(const double* __restrict__ part, int nb, int k,
                                                            const double* __restrict__ Ainv, double* cbuf,
                                                            unsigned* counter, double* __restrict__ c_out,
                                                            double* __restrict__ e_out) {
  __shared__ double sm[CC_THREADS];
  __shared__ double c[128];
  __shared__ int flag;
  const int j = blockIdx.x, tid = threadIdx.x;
  double s = 0.0;
  for (int b = tid; b < nb; b += CC_THREADS) s += part[(int64_t)b * k + j];
  sm[tid] = s;
  __syncthreads();
  if (tid < 32) {
    double t = 0.0;
    for (int q = tid; q < CC_THREADS; q += 32) t += sm[q];
    t = warp_sum(t);
    if (tid == 0) {
      cbuf[j] = t;
      if (c_out) c_out[j] = t;
    }
  }
  if (!last_block_arrive(counter, &flag)) return;
  for (int q = tid; q < k; q += CC_THREADS) c[q] = __ldcg(cbuf + q);
  __syncthreads();
  // e = A_c^-1 c: thread (row, g) adds the columns g, g + G, ... of its row
  const int G = CC_THREADS / k;  // >= 2
  const int row = tid % k, g = tid / k;
  double t = 0.0;
  if (g < G)
    for (int jj = g; jj < k; jj += G) t = fma(Ainv[(int64_t)jj * k + row], c[jj], t);
  sm[tid] = t;
  __syncthreads();
  if (tid < k) {
    double e = 0.0;
    for (int q = 0; q < G; ++q) e += sm[q * k + tid];
    if (e_out) e_out[tid] = e;
  }
}

// z += P e on every node (one 128-thread block per tile at a time).
template <typename T>
__global__ void __launch_bounds__(NLSP_TILE) k_prolong_vec(const T* __restrict__ P, int k, int64_t n,
                                                          const double* __restrict__ e, T* __restrict__ z) {
  __shared__ T es[128];
  for (int j = threadIdx.x; j < k; j += NLSP_TILE) es[j] = (T)e[j];
  __syncthreads();
  const int64_t ntiles = (n + NLSP_TILE - 1) / NLSP_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * NLSP_TILE + threadIdx.x;
    T s0 = T(0), s1 = T(0);
    const T* src = P + t * k * NLSP_TILE + threadIdx.x;
    int j = 0;
#pragma unroll 8
    for (; j + 1 < k; j += 2) {  // sixteen loads in flight, two partial sums
      s0 += src[(int64_t)j * NLSP_TILE] * es[j];
      s1 += src[(int64_t)(j + 1) * NLSP_TILE] * es[j + 1];
    }
    if (j < k) s0 += src[(int64_t)j * NLSP_TILE] * es[j];
    if (i < n) z[i] += s0 + s1;
  }
}

template <typename T>
__global__ void k_to_f64(const T* __restrict__ z, int64_t n, double* __restrict__ out, int accumulate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = accumulate ? out[i] + (double)z[i] : (double)z[i];
}

template <typename T>
__global__ void k_from_f64(const double* __restrict__ x, int64_t n, int64_t n_pad, T* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = i < n ? (T)x[i] : T(0);
}

// Column-major FP64 (n x ncols, leading dimension ld) -> node-tiled T with
// zero padding rows.
template <typename T>
__global__ void k_to_tiled(const double* __restrict__ src, int64_t n, int64_t ld, int ncols, int64_t n_pad,
                           T* __restrict__ dst) {
  const int64_t total = n_pad * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = e / ((int64_t)ncols * NLSP_TILE);
    const int64_t rem = e - tile * ncols * NLSP_TILE;
    const int c = (int)(rem / NLSP_TILE);
    const int64_t i = tile * NLSP_TILE + (rem % NLSP_TILE);
    dst[e] = i < n ? (T)src[(int64_t)c * ld + i] : T(0);
  }
}

// A applied to each column of a node-tiled block (T precision).
template <int KIND, typename T>
__global__ void k_apply_tiled(StencilView<T> A, const T* __restrict__ X, int ncols, int64_t n_pad,
                              T* __restrict__ Y) {
  const int64_t total = n_pad * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tile = e / ((int64_t)ncols * NLSP_TILE);
    const int64_t rem = e - tile * ncols * NLSP_TILE;
    const int c = (int)(rem / NLSP_TILE);
    const int64_t i = tile * NLSP_TILE + (rem % NLSP_TILE);
    T v = T(0);
    if (i < A.n)
      v = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return X[tiled_index(m, c, ncols)]; });
    Y[e] = v;
  }
}

}  // namespace

namespace {

// W = sum_j (e_j cbar_j^T + cbar_j e_j^T)  (k x k, column-major, FP64), the
// coefficient of A P in the gradient.
__global__ void k_wsym(const double* __restrict__ E, const double* __restrict__ Cb, int J, int k,
                       double* __restrict__ W) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int d = e % k, c = e / k;
    double s = 0.0;
    for (int j = 0; j < J; ++j)
      s += E[(int64_t)j * k + d] * Cb[(int64_t)j * k + c] + Cb[(int64_t)j * k + d] * E[(int64_t)j * k + c];
    W[e] = s;
  }
}

// grad P (column-major FP64, n x k, leading dimension ld) =
//   sum_j (ybar_j e_j^T + rho_j cbar_j^T) - (A P) W
// One 128-thread block per tile at a time, 16 output columns per pass.
constexpr int PB_CH = 16;

template <typename T>
__global__ void __launch_bounds__(NLSP_TILE) k_pbar(const T* __restrict__ Yb, const T* __restrict__ RH,
                                                   const double* __restrict__ E, const double* __restrict__ Cb, int J,
                                                   const T* __restrict__ AP, const double* __restrict__ W, int k,
                                                   int64_t n, int64_t n_pad, double* __restrict__ out, int64_t ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);  // [k][k]
  T* Es = Ws + (size_t)k * k;              // [J][k]
  T* Cs = Es + (size_t)J * k;              // [J][k]
  for (int e = threadIdx.x; e < k * k; e += NLSP_TILE) Ws[e] = (T)W[e];
  for (int e = threadIdx.x; e < J * k; e += NLSP_TILE) {
    Es[e] = (T)E[e];
    Cs[e] = (T)Cb[e];
  }
  __syncthreads();
  const int64_t ntiles = n_pad / NLSP_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * NLSP_TILE + threadIdx.x;
    const T* ap = AP + t * k * NLSP_TILE + threadIdx.x;
    for (int c0 = 0; c0 < k; c0 += PB_CH) {
      T acc[PB_CH];
#pragma unroll
      for (int jj = 0; jj < PB_CH; ++jj) acc[jj] = T(0);
      for (int d = 0; d < k; ++d) {
        const T a = ap[(int64_t)d * NLSP_TILE];
#pragma unroll
        for (int jj = 0; jj < PB_CH; ++jj)
          if (c0 + jj < k) acc[jj] -= a * Ws[(int64_t)(c0 + jj) * k + d];
      }
      for (int j = 0; j < J; ++j) {
        const T y = Yb[(int64_t)j * n_pad + i], r = RH[(int64_t)j * n_pad + i];
#pragma unroll
        for (int jj = 0; jj < PB_CH; ++jj)
          if (c0 + jj < k) acc[jj] += y * Es[j * k + c0 + jj] + r * Cs[j * k + c0 + jj];
      }
      if (i < n) {
#pragma unroll
        for (int jj = 0; jj < PB_CH; ++jj)
          if (c0 + jj < k) out[(int64_t)(c0 + jj) * ld + i] = (double)acc[jj];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tall-skinny cross products X^T Y over node tiles (X: ncx columns, Y: ncy
// columns, node-tiled), block partials in FP64.  16 x 16 threads, each with
// an RBX x RBY register tile; chunks of 32 nodes staged in shared memory.
// ---------------------------------------------------------------------------
constexpr int TS_CW = 32;

template <typename T, int RBX, int RBY>
__global__ void __launch_bounds__(256) k_ts_cross(const T* __restrict__ X, int ncx, const T* __restrict__ Y, int ncy,
                                                 int64_t n_pad, double* __restrict__ part) {
  constexpr int TD = 16, LX = RBX * TD + 1, LY = RBY * TD + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);  // [CW][LX]
  T* ys = xs + TS_CW * LX;                 // [CW][LY]
  const int tx = threadIdx.x % TD, ty = threadIdx.x / TD;
  T acc[RBX][RBY];
#pragma unroll
  for (int a = 0; a < RBX; ++a)
#pragma unroll
    for (int b = 0; b < RBY; ++b) acc[a][b] = T(0);
  const int64_t ntiles = n_pad / NLSP_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int w0 = 0; w0 < NLSP_TILE; w0 += TS_CW) {
      __syncthreads();
      for (int e = threadIdx.x; e < TS_CW * RBX * TD; e += 256) {
        const int c = e / TS_CW, w = e % TS_CW;
        xs[w * LX + c] = c < ncx ? X[(t * ncx + c) * NLSP_TILE + w0 + w] : T(0);
      }
      for (int e = threadIdx.x; e < TS_CW * RBY * TD; e += 256) {
        const int c = e / TS_CW, w = e % TS_CW;
        ys[w * LY + c] = c < ncy ? Y[(t * ncy + c) * NLSP_TILE + w0 + w] : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int w = 0; w < TS_CW; ++w) {
        T xa[RBX], yb[RBY];
#pragma unroll
        for (int a = 0; a < RBX; ++a) xa[a] = xs[w * LX + ty * RBX + a];
#pragma unroll
        for (int b = 0; b < RBY; ++b) yb[b] = ys[w * LY + tx * RBY + b];
#pragma unroll
        for (int a = 0; a < RBX; ++a)
#pragma unroll
          for (int b = 0; b < RBY; ++b) acc[a][b] += xa[a] * yb[b];
      }
    }
  }
  double* out = part + (int64_t)blockIdx.x * ncx * ncy;
#pragma unroll
  for (int a = 0; a < RBX; ++a) {
    const int row = ty * RBX + a;
#pragma unroll
    for (int b = 0; b < RBY; ++b) {
      const int col = tx * RBY + b;
      if (row < ncx && col < ncy) out[(int64_t)col * ncx + row] = (double)acc[a][b];
    }
  }
}

// out[e] = sum over blocks of part[b][e], block order.
__global__ void k_sum_blocks(const double* __restrict__ part, int nb, int count, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * count + e];
    out[e] = s;
  }
}

// acc[0..KC) += sum over the nc input columns c of x[c] * m[c][j0 + j] for
// one node: x points at the node's entry of column 0 of a tile (columns
// NLSP_TILE apart), m is row-major with rows padded to ldm (a multiple of the
// 16-byte vector width, zeros past the last column).  Input loads are issued
// CU at a time ahead of their products; m is read as 16-byte broadcasts.
template <typename T, int KC, int CU>
__device__ __forceinline__ void tile_rows_times(const T* __restrict__ x, int nc, const T* m, int ldm, int j0,
                                                T (&acc)[KC]) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::N;
  for (int c0 = 0; c0 < nc; c0 += CU) {
    T sv[CU];
#pragma unroll
    for (int u = 0; u < CU; ++u) sv[u] = c0 + u < nc ? x[(int64_t)(c0 + u) * NLSP_TILE] : T(0);
#pragma unroll
    for (int u = 0; u < CU; ++u) {
      if (c0 + u >= nc) break;
      const T* mrow = m + (c0 + u) * ldm + j0;
#pragma unroll
      for (int j = 0; j < KC; j += VN) {
        if (j0 + j >= ldm) break;
        T mv[VN];
        *reinterpret_cast<V*>(mv) = *reinterpret_cast<const V*>(mrow + j);
#pragma unroll
        for (int q = 0; q < VN; ++q) acc[j + q] += sv[u] * mv[q];
      }
    }
  }
}

constexpr int TG_KC = 32;  // output columns per register pass of k_tile_gemm2
constexpr int TG_CU = 8;   // input loads in flight

__host__ __device__ constexpr int tg_ldm(int k) { return (k + 3) / 4 * 4; }

// Out (column-major FP64 n x k, ld) = In1 M1 + In2 M2 with In1 (nc1 columns)
// and In2 (nc2 columns) node-tiled, M1 (nc1 x k) and M2 (nc2 x k)
// column-major FP64.  One 128-thread block per tile at a time; M1 and M2 sit
// in shared memory as T, rows padded to tg_ldm(k).
template <typename T>
__global__ void __launch_bounds__(NLSP_TILE) k_tile_gemm2(const T* __restrict__ In1, int nc1,
                                                         const double* __restrict__ M1, const T* __restrict__ In2,
                                                         int nc2, const double* __restrict__ M2, int k, int64_t n,
                                                         int64_t n_pad, double* __restrict__ out, int64_t ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldm = tg_ldm(k);
  T* m1 = reinterpret_cast<T*>(smem_raw);  // [nc1][ldm] (row = input column)
  T* m2 = m1 + (size_t)nc1 * ldm;
  for (int e = threadIdx.x; e < nc1 * ldm; e += NLSP_TILE) {
    const int c = e / ldm, j = e % ldm;
    m1[e] = j < k ? (T)M1[(int64_t)j * nc1 + c] : T(0);
  }
  for (int e = threadIdx.x; e < nc2 * ldm; e += NLSP_TILE) {
    const int c = e / ldm, j = e % ldm;
    m2[e] = j < k ? (T)M2[(int64_t)j * nc2 + c] : T(0);
  }
  __syncthreads();
  const int64_t ntiles = n_pad / NLSP_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t i = t * NLSP_TILE + threadIdx.x;
    const T* x1 = In1 + t * nc1 * NLSP_TILE + threadIdx.x;
    const T* x2 = In2 + t * nc2 * NLSP_TILE + threadIdx.x;
    for (int c0 = 0; c0 < k; c0 += TG_KC) {
      T acc[TG_KC];
#pragma unroll
      for (int jj = 0; jj < TG_KC; ++jj) acc[jj] = T(0);
      tile_rows_times<T, TG_KC, TG_CU>(x1, nc1, m1, ldm, c0, acc);
      tile_rows_times<T, TG_KC, TG_CU>(x2, nc2, m2, ldm, c0, acc);
      if (i < n) {
#pragma unroll
        for (int jj = 0; jj < TG_KC; ++jj)
          if (c0 + jj < k) out[(int64_t)(c0 + jj) * ld + i] = (double)acc[jj];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Small dense FP64 algebra for the k x k / k x K factors (one block).
// ---------------------------------------------------------------------------
// Lower Cholesky factor of the SPD m x m matrix G (column-major): G = L L^T.
// *ok = 0 when a pivot is not positive.  Right-looking, one column a step.
__global__ void k_small_chol(const double* __restrict__ G, int m, double* __restrict__ L, int* ok) {
  extern __shared__ double a[];  // m x m working copy
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) a[e] = G[e];
  __shared__ int good;
  if (threadIdx.x == 0) good = 1;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double d = a[j * m + j];
      if (!(d > 0.0)) good = 0;
      a[j * m + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double piv = a[j * m + j];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) a[j * m + i] /= piv;
    __syncthreads();
    // trailing update of the lower triangle
    for (int e = threadIdx.x; e < (m - j - 1) * (m - j - 1); e += blockDim.x) {
      const int r = j + 1 + e % (m - j - 1), c = j + 1 + e / (m - j - 1);
      if (r >= c) a[c * m + r] -= a[j * m + r] * a[j * m + c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    L[e] = r >= c ? a[e] : 0.0;
  }
  if (threadIdx.x == 0) *ok = good;
}

// Inverse of the lower-triangular L (column-major): column c of L^-1 by
// forward substitution, one thread per column.
__global__ void k_small_trinv(const double* __restrict__ L, int m, double* __restrict__ Li) {
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    for (int r = 0; r < m; ++r) {
      double s = r == c ? 1.0 : 0.0;
      for (int q = c; q < r; ++q) s -= L[(int64_t)q * m + r] * Li[(int64_t)c * m + q];
      Li[(int64_t)c * m + r] = r < c ? 0.0 : s / L[(int64_t)r * m + r];
    }
  }
}

// C (m x p) = alpha op(A) op(B), op(A) m x q, op(B) q x p, column-major with
// leading dimensions = row counts of the stored matrices.
__global__ void k_small_mm(const double* __restrict__ A, int ta, const double* __restrict__ B, int tb,
                           double* __restrict__ C, int m, int p, int q, double alpha) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * p; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;
    double s = 0.0;
    for (int l = 0; l < q; ++l) {
      const double av = ta ? A[(int64_t)i * q + l] : A[(int64_t)l * m + i];
      const double bv = tb ? B[(int64_t)l * p + j] : B[(int64_t)j * q + l];
      s = fma(av, bv, s);
    }
    C[e] = alpha * s;
  }
}

// Nested (NLSS) weights on the rows of C = Q^T B (k x K, column-major):
// S[out] = sum_i w_i sum_j C_ij^2 with w_i = (k - i) / k (row i enters the
// partial sums of levels i + 1 .. k), and, when Cw is given,
// Cw = diag(w) C / S[0] with S[0] = ||B||^2.  One block of 256 threads,
// partials combined in a fixed order.
__global__ void __launch_bounds__(256) k_nlss_weights(const double* __restrict__ C, int k, int K, double* S, int out,
                                                      double* __restrict__ Cw) {
  __shared__ double red[256];
  const int count = k * K;
  const double inv_b = Cw ? 1.0 / S[0] : 0.0;
  double s = 0.0;
  for (int e = threadIdx.x; e < count; e += blockDim.x) {
    const int i = e % k;
    const double w = (double)(k - i) / (double)k;
    const double c = C[e];
    s = fma(w * c, c, s);
    if (Cw) Cw[e] = w * c * inv_b;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) S[out] = red[0];
}

// out = alpha * copyltu(M) for a k x k column-major M: the lower triangle
// (diagonal included) kept and mirrored onto the upper one.
__global__ void k_copyltu(const double* __restrict__ M, int k, double alpha, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e % k, j = e / k;
    out[e] = alpha * (i >= j ? M[e] : M[(int64_t)i * k + j]);
  }
}

// S[out] = sum of squares of x (count entries), one warp (small matrices).
__global__ void k_small_sumsq(const double* __restrict__ x, int count, double* S, int out) {
  double s = 0.0;
  for (int e = threadIdx.x; e < count; e += 32) s = fma(x[e], x[e], s);
  s = warp_sum(s);
  if (threadIdx.x == 0) S[out] = s;
}

}  // namespace

// ============================================================================
// Host side
// ============================================================================
namespace {

// Device workspace of one call, carved from the context's grow-only adjoint
// scratch slot (kept for the next call: an allocation and a free per call
// would cost more than a short call's kernels, and the free synchronises).
struct Arena {
  unsigned char* base = nullptr;
  size_t used = 0, cap = 0;
  nlsp_status reserve(nlsp_ctx* ctx, size_t bytes) {
    base = reinterpret_cast<unsigned char*>(ctx_slot(ctx, SLOT_ADJ, bytes));
    if (!base) return NLSP_ERR_OOM;
    cap = bytes;
    return NLSP_OK;
  }
  template <typename U>
  U* take(size_t count) {
    const size_t off = align_up(used, 256);
    used = off + sizeof(U) * count;
    return used <= cap ? reinterpret_cast<U*>(base + off) : nullptr;
  }
};

size_t arena_bytes(const std::vector<size_t>& parts) {
  size_t s = 0;
  for (size_t p : parts) s += align_up(p, 256) + 256;
  return s;
}

template <typename T>
const StencilView<T>& vview(const nlsp_op* A) {
  return *reinterpret_cast<const StencilView<T>*>(sizeof(T) == 8 ? (const void*)&A->v64 : (const void*)&A->v32);
}

int vgrid(const nlsp_ctx* ctx, int64_t n) { return grid_for(ctx, n, VB, 8); }

// Unrolled PCG (T iterations, x0 = 0) with the two-level preconditioner M
// built from P, its loss ||r_T|| and the gradient with respect to P.
template <int KIND, typename TP>
struct Unrolled {
  nlsp_ctx* ctx;
  const nlsp_op* A;
  nlsp_prec* M;
  int T, nu, k, nb, ntb;  // nb: partial-sum grids; ntb: tile-per-block grids
  int64_t n, n_pad;
  TP omega;
  ScalarIndex ix;
  double* S;
  double* part;        // dot / restriction partials
  double* R;           // r_0 .. r_T            (T + 1) x n
  double* Pv;          // p_0 .. p_{T-1}        T x n
  double* Q;           // q_0 .. q_{T-1}        T x n
  double* Z;           // z_0 .. z_{T-1}        T x n
  TP* RHO;             // rho of application j  T x n_pad
  double* E;           // e of application j    T x k
  TP* YB;              // ybar of application j T x n_pad
  double* CB;          // cbar of application j T x k
  double* cbuf;        // coarse right-hand side of the current application (k)
  unsigned* counter;   // arrival counter of the coarse step (zero between launches)
  TP* w0;              // preconditioner work vectors (n_pad)
  TP* w1;
  double* vtmp;        // FP64 scratch vectors
  double* rbar;
  double* pbar;
  double* zbar;
  double* qbar;
  TP* AP;              // A P, node-tiled
  double* W;           // k x k
  cudaStream_t s;
  int launches = 0;

  void dot(const double* x, const double* y, int out) {
    k_vdot_part<<<nb, VB, 0, s>>>(x, y, n, part);
    k_vdot_fin<<<1, 32, 0, s>>>(part, nb, S, out);
    launches += 2;
  }
  void scalar(int op, int t) {
    k_scalar<<<1, 1, 0, s>>>(S, ix, op, t);
    ++launches;
  }
  void axpy(double* y, const double* x, int ia, int ib, double mult) {
    k_vaxpy<<<vgrid(ctx, n), VB, 0, s>>>(y, x, n, S, ia, ib, mult);
    ++launches;
  }
  void scale(double* y, const double* x, int ia, int ib, double mult) {
    k_vscale<<<vgrid(ctx, n), VB, 0, s>>>(y, x, n, S, ia, ib, mult);
    ++launches;
  }
  void xpay(double* y, const double* x, int ia, int ib, double mult) {
    k_vxpay<<<vgrid(ctx, n), VB, 0, s>>>(y, x, n, S, ia, ib, mult);
    ++launches;
  }
  void spmv(const double* x, double* y, int accumulate) {
    k_vspmv<KIND><<<vgrid(ctx, n), VB, 0, s>>>(A->v64, x, y, accumulate);
    ++launches;
  }

  // out = B v (FP64).  With j >= 0 the residual rho and the coarse
  // correction e of the application are kept as checkpoint j.
  void apply(const double* v, double* out, int j) {
    const StencilView<TP>& AT = vview<TP>(A);
    const int g = vgrid(ctx, n);
    TP* cur = w0;
    TP* oth = w1;
    k_jsweep<KIND, TP><<<g, VB, 0, s>>>(AT, omega, v, nullptr, cur);
    for (int sw = 1; sw < nu; ++sw) {
      k_jsweep<KIND, TP><<<g, VB, 0, s>>>(AT, omega, v, cur, oth);
      std::swap(cur, oth);
    }
    TP* rho = j >= 0 ? RHO + (size_t)j * n_pad : oth;
    k_resid<KIND, TP><<<g, VB, 0, s>>>(AT, v, cur, rho);
    k_restrict_vec<TP><<<nb, RV_THREADS, 0, s>>>((const TP*)M->P, k, n_pad, rho, part);
    double* e = j >= 0 ? E + (size_t)j * k : vtmp + n;  // vtmp holds n + k doubles
    k_coarse_cols<<<k, CC_THREADS, 0, s>>>(part, nb, k, M->Ainv, cbuf, counter, nullptr, e);
    k_prolong_vec<TP><<<ntb, NLSP_TILE, 0, s>>>((const TP*)M->P, k, n, e, cur);
    for (int sw = 0; sw < nu; ++sw) {
      k_jsweep<KIND, TP><<<g, VB, 0, s>>>(AT, omega, v, cur, oth);
      std::swap(cur, oth);
    }
    k_to_f64<TP><<<g, VB, 0, s>>>(cur, n, out, 0);
    launches += 2 * nu + 5;
  }

  // Adjoint of application j with respect to P, given zbar: ybar_j =
  // (S_J^nu)^T zbar, cbar_j = A_c^-1 P^T ybar_j.
  void apply_adjoint_P(const double* zb, int j) {
    const StencilView<TP>& AT = vview<TP>(A);
    const int g = vgrid(ctx, n);
    TP* cur = w0;
    TP* oth = w1;
    k_from_f64<TP><<<vgrid(ctx, n_pad), VB, 0, s>>>(zb, n, n_pad, cur);
    for (int sw = 0; sw < nu; ++sw) {
      k_jsweep_t<KIND, TP><<<g, VB, 0, s>>>(AT, omega, cur, oth);
      std::swap(cur, oth);
    }
    TP* yb = YB + (size_t)j * n_pad;
    cudaMemcpyAsync(yb, cur, sizeof(TP) * n_pad, cudaMemcpyDeviceToDevice, s);
    k_restrict_vec<TP><<<nb, RV_THREADS, 0, s>>>((const TP*)M->P, k, n_pad, yb, part);
    k_coarse_cols<<<k, CC_THREADS, 0, s>>>(part, nb, k, M->Ainv, cbuf, counter, nullptr, CB + (size_t)j * k);
    launches += nu + 3;
  }

  double* r(int t) { return R + (size_t)t * n; }
  double* p(int t) { return Pv + (size_t)t * n; }
  double* q(int t) { return Q + (size_t)t * n; }
  double* z(int t) { return Z + (size_t)t * n; }

  void forward(const double* b) {
    scalar(OP_INIT, 0);
    cudaMemcpyAsync(r(0), b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    apply(r(0), z(0), 0);
    cudaMemcpyAsync(p(0), z(0), sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    dot(r(0), z(0), ix.gam(0));
    for (int t = 0; t < T; ++t) {
      spmv(p(t), q(t), 0);
      dot(p(t), q(t), ix.del(t));
      scalar(OP_ALPHA, t);
      cudaMemcpyAsync(r(t + 1), r(t), sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
      axpy(r(t + 1), q(t), ix.alp(t), -1, -1.0);
      if (t == T - 1) break;
      apply(r(t + 1), z(t + 1), t + 1);
      dot(r(t + 1), z(t + 1), ix.gam(t + 1));
      scalar(OP_BETA, t);
      cudaMemcpyAsync(p(t + 1), p(t), sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
      xpay(p(t + 1), z(t + 1), ix.bet(t), -1, 1.0);
    }
    dot(r(T), r(T), ix.rr());
    scalar(OP_LOSS, 0);
  }

  void reverse() {
    // rbar_T = r_T / ||r_T||
    scale(rbar, r(T), -1, ix.loss(), 1.0);
    for (int t = T - 1; t >= 0; --t) {
      if (t < T - 1) {
        // p_{t+1} = z_{t+1} + beta_t p_t
        cudaMemcpyAsync(zbar, pbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
        dot(pbar, p(t), ix.x0());  // beta_bar
        scale(pbar, pbar, ix.bet(t), -1, 1.0);
        scalar(OP_REV_BETA, t);
        // gamma_{t+1} = r_{t+1} . z_{t+1}
        axpy(rbar, z(t + 1), ix.gbar(t + 1), -1, 1.0);
        axpy(zbar, r(t + 1), ix.gbar(t + 1), -1, 1.0);
        // z_{t+1} = B r_{t+1}: P part, then rbar_{t+1} += B zbar (B symmetric)
        apply_adjoint_P(zbar, t + 1);
        apply(zbar, vtmp, -1);
        axpy(rbar, vtmp, -1, -1, 1.0);
      } else {
        cudaMemsetAsync(pbar, 0, sizeof(double) * n, s);
      }
      // r_{t+1} = r_t - alpha_t q_t  (rbar_t = rbar_{t+1})
      dot(q(t), rbar, ix.x1());
      scale(qbar, rbar, ix.alp(t), -1, -1.0);
      scalar(OP_REV_ALPHA, t);
      // delta_t = p_t . q_t, q_t = A p_t
      axpy(pbar, q(t), ix.x2(), -1, 1.0);
      axpy(qbar, p(t), ix.x2(), -1, 1.0);
      spmv(qbar, pbar, 1);
    }
    // p_0 = z_0, gamma_0 = r_0 . z_0, z_0 = B r_0 (r_0 = b is not a variable)
    cudaMemcpyAsync(zbar, pbar, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    axpy(zbar, r(0), ix.gbar(0), -1, 1.0);
    apply_adjoint_P(zbar, 0);
  }

  // grad = sum_j (ybar_j e_j^T + rho_j cbar_j^T) - (A P) W
  nlsp_status gradient(double* grad) {
    const StencilView<TP>& AT = vview<TP>(A);
    k_apply_tiled<KIND, TP><<<grid_for(ctx, n_pad * k, VB, 8), VB, 0, s>>>(AT, (const TP*)M->P, k, n_pad, AP);
    k_wsym<<<div_up((int64_t)k * k, 256), 256, 0, s>>>(E, CB, T, k, W);
    const size_t sm = sizeof(TP) * ((size_t)k * k + 2 * (size_t)T * k);
    auto fn = k_pbar<TP>;
    if (sm > 48 * 1024) NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    fn<<<ntb, NLSP_TILE, sm, s>>>(YB, RHO, E, CB, T, AP, W, k, n, n_pad, grad, n);
    launches += 3;
    NLSP_LAUNCH_CHECK();
    return NLSP_OK;
  }

  static nlsp_status run(nlsp_ctx* ctx, const nlsp_op* A, nlsp_prec* M, int nu, double omega, const double* b, int T,
                         double* loss, double* grad) {
    Unrolled u;
    u.ctx = ctx;
    u.A = A;
    u.M = M;
    u.T = T;
    u.nu = nu;
    u.k = M->k;
    u.n = A->n;
    u.n_pad = M->n_pad;
    u.omega = (TP)omega;
    u.ix.T = T;
    u.s = ctx->stream;
    u.nb = std::max(1, std::min<int>(2 * ctx->num_sms, (int)(u.n_pad / NLSP_TILE)));
    u.ntb = (int)std::max<int64_t>(1, std::min<int64_t>(u.n_pad / NLSP_TILE, (int64_t)16 * ctx->num_sms));
    const int64_t n = u.n, n_pad = u.n_pad, k = u.k;
    Arena ar;
    const std::vector<size_t> parts = {
        sizeof(double) * (size_t)u.ix.count(), sizeof(double) * (size_t)u.nb * k,
        sizeof(double) * (size_t)(T + 1) * n, sizeof(double) * (size_t)T * n * 3,
        sizeof(TP) * (size_t)T * n_pad * 2, sizeof(double) * (size_t)T * k * 2, sizeof(TP) * (size_t)n_pad * 2,
        sizeof(double) * (size_t)(n + k), sizeof(double) * (size_t)n * 4, sizeof(TP) * (size_t)n_pad * k,
        sizeof(double) * (size_t)k * k, sizeof(double) * (size_t)k, sizeof(unsigned) * 8};
    NLSP_TRY(ar.reserve(ctx, arena_bytes(parts) + 4096));
    u.S = ar.take<double>(u.ix.count());
    u.part = ar.take<double>((size_t)u.nb * k);
    u.cbuf = ar.take<double>((size_t)k);
    u.counter = ar.take<unsigned>(8);
    u.R = ar.take<double>((size_t)(T + 1) * n);
    u.Pv = ar.take<double>((size_t)T * n);
    u.Q = ar.take<double>((size_t)T * n);
    u.Z = ar.take<double>((size_t)T * n);
    u.RHO = ar.take<TP>((size_t)T * n_pad);
    u.YB = ar.take<TP>((size_t)T * n_pad);
    u.E = ar.take<double>((size_t)T * k);
    u.CB = ar.take<double>((size_t)T * k);
    u.w0 = ar.take<TP>(n_pad);
    u.w1 = ar.take<TP>(n_pad);
    u.vtmp = ar.take<double>(n + k);
    u.rbar = ar.take<double>(n);
    u.pbar = ar.take<double>(n);
    u.zbar = ar.take<double>(n);
    u.qbar = ar.take<double>(n);
    u.AP = ar.take<TP>((size_t)n_pad * k);
    u.W = ar.take<double>((size_t)k * k);
    if (!u.W) return NLSP_ERR_OOM;
    // padding rows of the work vectors stay zero (the restriction reads them)
    NLSP_CUDA(cudaMemsetAsync(u.RHO, 0, sizeof(TP) * (size_t)T * n_pad, u.s));
    NLSP_CUDA(cudaMemsetAsync(u.w0, 0, sizeof(TP) * n_pad, u.s));
    NLSP_CUDA(cudaMemsetAsync(u.counter, 0, sizeof(unsigned) * 8, u.s));
    NLSP_CUDA(cudaMemsetAsync(u.w1, 0, sizeof(TP) * n_pad, u.s));
    u.forward(b);
    NLSP_LAUNCH_CHECK();
    if (grad) {
      u.reverse();
      NLSP_LAUNCH_CHECK();
      NLSP_TRY(u.gradient(grad));
    }
    double h = 0.0;
    NLSP_CUDA(cudaMemcpyAsync(&h, u.S + u.ix.loss(), sizeof(double), cudaMemcpyDeviceToHost, u.s));
    NLSP_CUDA(cudaStreamSynchronize(u.s));
    count_launches(ctx, (unsigned long long)u.launches);
    *loss = h;
    return NLSP_OK;
  }
};

template <typename TP>
nlsp_status unrolled_dispatch(nlsp_ctx* ctx, const nlsp_op* A, nlsp_prec* M, int nu, double omega, const double* b,
                              int T, double* loss, double* grad) {
  switch (A->kind) {
    case ST_5PT: return Unrolled<ST_5PT, TP>::run(ctx, A, M, nu, omega, b, T, loss, grad);
    case ST_9PT: return Unrolled<ST_9PT, TP>::run(ctx, A, M, nu, omega, b, T, loss, grad);
    case ST_CSR: return Unrolled<ST_CSR, TP>::run(ctx, A, M, nu, omega, b, T, loss, grad);
    default: return Unrolled<ST_7PT, TP>::run(ctx, A, M, nu, omega, b, T, loss, grad);
  }
}

}  // namespace

extern "C" nlsp_status nlsp_unrolled_pcg(nlsp_ctx* ctx, const nlsp_op* A, const double* dev_P, int k, int nu,
                                         double omega, int precision, const double* dev_b, int T, double* loss,
                                         double* dev_grad) {
  if (!ctx || !A || !dev_P || !dev_b || !loss || k < 1 || k > 128 || nu < 1 || T < 1 || T > 1000 ||
      !(omega > 0.0 && omega < 2.0) || (precision != NLSP_FP64 && precision != NLSP_MIXED_FP32))
    return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  nlsp_setup_params p;
  memset(&p, 0, sizeof(p));
  p.k = k;
  p.nu1 = p.nu2 = nu;
  p.omega = omega;
  p.precision = precision;
  nlsp_prec* M = nullptr;
  NLSP_TRY(nlsp_prec_from_basis(ctx, A, &p, dev_P, k, &M));
  nlsp_status st = precision == NLSP_FP64 ? unrolled_dispatch<double>(ctx, A, M, nu, omega, dev_b, T, loss, dev_grad)
                                          : unrolled_dispatch<float>(ctx, A, M, nu, omega, dev_b, T, loss, dev_grad);
  nlsp_free_prec(M);
  return st;
}

// ---------------------------------------------------------------------------
// Subspace loss and its gradient.
//   G = P_hat^T P_hat = L L^T (so R = L^T in P_hat = Q R),  H = P_hat^T B,
//   C = Q^T B = L^-1 H,  loss = ||B||^2 - ||C||^2,
//   grad = -2 (I - Q Q^T) B C^T R^-T = -2 B X + 2 P_hat Z with
//   X = C^T L^-1 (K x k),  Z = L^-T C C^T L^-1 (k x k).
// The closed form is the thin-QR backward rule (P_hat_bar = (Q_bar + Q
// copyltu(M)) R^-T, M = R R_bar^T - Q_bar^T Q) with R_bar = 0 and
// Q_bar = -2 B C^T, for which M = 2 C C^T is already symmetric.
// ---------------------------------------------------------------------------
namespace {

template <typename TP>
nlsp_status launch_cross(nlsp_ctx* ctx, const TP* X, int ncx, const TP* Y, int ncy, int64_t n_pad, double* part,
                         int nb) {
  auto go = [&](auto fn, int rbx, int rby) -> nlsp_status {
    const size_t sm = sizeof(TP) * TS_CW * ((size_t)rbx * 16 + 1 + (size_t)rby * 16 + 1);
    if (sm > 48 * 1024) NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    fn<<<nb, 256, sm, ctx->stream>>>(X, ncx, Y, ncy, n_pad, part);
    NLSP_LAUNCH_CHECK();
    return NLSP_OK;
  };
  const int rbx = ncx <= 16 ? 1 : ncx <= 32 ? 2 : ncx <= 64 ? 4 : 8;
  const int rby = ncy <= 16 ? 1 : ncy <= 32 ? 2 : ncy <= 64 ? 4 : ncy <= 128 ? 8 : 16;
#define NLSP_CROSS(RX, RY) \
  if (rbx == RX && rby == RY) return go(k_ts_cross<TP, RX, RY>, RX, RY);
  NLSP_CROSS(1, 1) NLSP_CROSS(1, 2) NLSP_CROSS(1, 4) NLSP_CROSS(1, 8) NLSP_CROSS(1, 16)
  NLSP_CROSS(2, 2) NLSP_CROSS(2, 4) NLSP_CROSS(2, 8) NLSP_CROSS(2, 16)
  NLSP_CROSS(4, 4) NLSP_CROSS(4, 8) NLSP_CROSS(4, 16)
  NLSP_CROSS(8, 8) NLSP_CROSS(8, 16)
#undef NLSP_CROSS
  nlsp_record_message("subspace loss: unsupported column counts");
  return NLSP_ERR_INVALID;
}

// Subspace loss (NESTED = false) or the nested subspace loss NLSS (NESTED =
// true) and their gradients, from G = P_hat^T P_hat = L L^T (R = L^T),
// H = P_hat^T B and C = Q^T B = L^-1 H.
template <typename TP, bool NESTED>
nlsp_status subspace_impl(nlsp_ctx* ctx, int64_t n, int k, int K, const double* Ph, const double* B, double* loss,
                          double* grad) {
  cudaStream_t s = ctx->stream;
  const int64_t n_pad = pad_tile(n);
  const int nb = std::max(1, std::min<int>(2 * ctx->num_sms, (int)(n_pad / NLSP_TILE)));
  Arena ar;
  const std::vector<size_t> parts = {sizeof(TP) * (size_t)n_pad * k, sizeof(TP) * (size_t)n_pad * K,
                                     sizeof(double) * (size_t)nb * k * std::max(k, K), sizeof(double) * 16,
                                     sizeof(double) * (size_t)k * k * 6 + sizeof(double) * (size_t)k * K * 4,
                                     sizeof(double) * (size_t)nb, sizeof(int) * 4};
  NLSP_TRY(ar.reserve(ctx, arena_bytes(parts) + 4096));
  TP* Pt = ar.take<TP>((size_t)n_pad * k);
  TP* Bt = ar.take<TP>((size_t)n_pad * K);
  double* part = ar.take<double>((size_t)nb * k * std::max(k, K));
  double* S = ar.take<double>(16);
  double* G = ar.take<double>((size_t)k * k);
  double* Lf = ar.take<double>((size_t)k * k);
  double* Li = ar.take<double>((size_t)k * k);
  double* CC = ar.take<double>((size_t)k * k);
  double* Zt = ar.take<double>((size_t)k * k);
  double* Z = ar.take<double>((size_t)k * k);
  double* H = ar.take<double>((size_t)k * K);
  double* C = ar.take<double>((size_t)k * K);
  double* X = ar.take<double>((size_t)K * k);
  double* Cw = ar.take<double>((size_t)k * K);
  double* dpart = ar.take<double>(nb);
  int* ok = ar.take<int>(4);
  if (!ok) return NLSP_ERR_OOM;
  const int g = grid_for(ctx, n_pad * std::max(k, K), VB, 8);
  k_to_tiled<TP><<<g, VB, 0, s>>>(Ph, n, n, k, n_pad, Pt);
  k_to_tiled<TP><<<g, VB, 0, s>>>(B, n, n, K, n_pad, Bt);
  NLSP_LAUNCH_CHECK();
  NLSP_TRY(launch_cross<TP>(ctx, Pt, k, Pt, k, n_pad, part, nb));
  k_sum_blocks<<<div_up((int64_t)k * k, 256), 256, 0, s>>>(part, nb, k * k, G);
  NLSP_TRY(launch_cross<TP>(ctx, Pt, k, Bt, K, n_pad, part, nb));
  k_sum_blocks<<<div_up((int64_t)k * K, 256), 256, 0, s>>>(part, nb, k * K, H);
  // ||B||^2 from the FP64 input
  k_vdot_part<<<nb, VB, 0, s>>>(B, B, n * K, dpart);
  k_vdot_fin<<<1, 32, 0, s>>>(dpart, nb, S, 0);
  if (sizeof(double) * k * k > 48 * 1024)
    NLSP_CUDA(cudaFuncSetAttribute(k_small_chol, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(double) * k * k)));
  k_small_chol<<<1, 256, sizeof(double) * k * k, s>>>(G, k, Lf, ok);
  k_small_trinv<<<1, 128, 0, s>>>(Lf, k, Li);
  k_small_mm<<<div_up((int64_t)k * K, 128), 128, 0, s>>>(Li, 0, H, 0, C, k, K, k, 1.0);  // C = L^-1 H
  if (NESTED)
    k_nlss_weights<<<1, 256, 0, s>>>(C, k, K, S, 1, grad ? Cw : nullptr);  // sum_i w_i ||c_i||^2, diag(w) C / ||B||^2
  else
    k_small_sumsq<<<1, 32, 0, s>>>(C, k * K, S, 1);
  NLSP_LAUNCH_CHECK();
  int launches = 11;
  if (grad && !NESTED) {
    k_small_mm<<<div_up((int64_t)K * k, 128), 128, 0, s>>>(C, 1, Li, 0, X, K, k, k, -2.0);  // -2 C^T L^-1
    k_small_mm<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(C, 0, C, 1, CC, k, k, K, 1.0);   // C C^T
    k_small_mm<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(CC, 0, Li, 0, Zt, k, k, k, 1.0);  // C C^T L^-1
    k_small_mm<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(Li, 1, Zt, 0, Z, k, k, k, 2.0);  // 2 L^-T C C^T L^-1
  } else if (grad) {
    // NLSS: Q_bar = -(2 / ||B||^2) B C^T W, M = -Q_bar^T Q = (2 / ||B||^2) W C C^T (not
    // symmetric), P_hat_bar = (Q_bar + Q copyltu(M)) R^-T
    //                       = B (-2 Cw^T L^-1) + P_hat (L^-T copyltu(2 Cw C^T) L^-1)
    k_small_mm<<<div_up((int64_t)K * k, 128), 128, 0, s>>>(Cw, 1, Li, 0, X, K, k, k, -2.0);  // -2 Cw^T L^-1
    k_small_mm<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(Cw, 0, C, 1, CC, k, k, K, 1.0);   // Cw C^T
    k_copyltu<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(CC, k, 2.0, Zt);                    // M
    k_small_mm<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(Zt, 0, Li, 0, CC, k, k, k, 1.0);  // M L^-1
    k_small_mm<<<div_up((int64_t)k * k, 128), 128, 0, s>>>(Li, 1, CC, 0, Z, k, k, k, 1.0);  // L^-T M L^-1
    launches += 1;
  }
  if (grad) {
    const size_t sm = sizeof(TP) * (size_t)(K + k) * tg_ldm(k);
    auto fn = k_tile_gemm2<TP>;
    if (sm > 48 * 1024) NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int ntb = (int)std::min<int64_t>(n_pad / NLSP_TILE, (int64_t)16 * ctx->num_sms);
    fn<<<ntb, NLSP_TILE, sm, s>>>(Bt, K, X, Pt, k, Z, k, n, n_pad, grad, n);
    NLSP_LAUNCH_CHECK();
    launches += 5;
  }
  double h[2];
  int hok = 0;
  NLSP_CUDA(cudaMemcpyAsync(h, S, sizeof(h), cudaMemcpyDeviceToHost, s));
  NLSP_CUDA(cudaMemcpyAsync(&hok, ok, sizeof(int), cudaMemcpyDeviceToHost, s));
  NLSP_CUDA(cudaStreamSynchronize(s));
  count_launches(ctx, (unsigned long long)launches);
  if (!hok) {
    nlsp_record_message("subspace loss: P_hat^T P_hat is not positive definite (P_hat rank deficient)");
    return NLSP_ERR_NOT_SPD;
  }
  // subspace: ||B||^2 - ||C||^2; NLSS: (1/k) sum_l (1 - ||Q_{1:l}^T B||^2 / ||B||^2)
  *loss = NESTED ? 1.0 - h[1] / h[0] : h[0] - h[1];
  return NLSP_OK;
}

}  // namespace

extern "C" nlsp_status nlsp_subspace_loss(nlsp_ctx* ctx, int64_t n, int k, int K, int precision,
                                          const double* dev_Phat, const double* dev_B, double* loss,
                                          double* dev_grad) {
  if (!ctx || !dev_Phat || !dev_B || !loss || n < 1 || k < 1 || k > 128 || K < 1 || K > 256 || k > n ||
      (precision != NLSP_FP64 && precision != NLSP_MIXED_FP32))
    return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  return precision == NLSP_FP64 ? subspace_impl<double, false>(ctx, n, k, K, dev_Phat, dev_B, loss, dev_grad)
                                : subspace_impl<float, false>(ctx, n, k, K, dev_Phat, dev_B, loss, dev_grad);
}

extern "C" nlsp_status nlsp_nlss_loss(nlsp_ctx* ctx, int64_t n, int k, int K, int precision, const double* dev_Phat,
                                      const double* dev_S, double* loss, double* dev_grad) {
  if (!ctx || !dev_Phat || !dev_S || !loss || n < 1 || k < 1 || k > 128 || K < 1 || K > 256 || k > n ||
      (precision != NLSP_FP64 && precision != NLSP_MIXED_FP32))
    return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  return precision == NLSP_FP64 ? subspace_impl<double, true>(ctx, n, k, K, dev_Phat, dev_S, loss, dev_grad)
                                : subspace_impl<float, true>(ctx, n, k, K, dev_Phat, dev_S, loss, dev_grad);
}
