// Two-level preconditioner apply (Algorithm 1, "Apply preconditioner to
// residual b") and preconditioned CG (Sec. 4, two-grid solver evaluation).
//
// One PCG iteration t is five kernels (plus extra sweeps when nu > 2):
//   spmv    p_t = z_{t-1} + beta p_{t-1} (evaluated on the fly, also at the
//           stencil neighbours), q = A p_t, p^T q;     last block: alpha
//   pre     x += alpha p, r_t = r_{t-1} - alpha q, ||r_t||^2, and the first
//           two Jacobi sweeps from z = 0 (z1 = w D^-1 r is elementwise, so
//           z2 = z1 + w D^-1 (r - A z1) needs only neighbour values of r);
//           last block: convergence test
//   restrict  rho = r - A z, c = P^T rho;              last block: e_c = A_c^-1 c
//   prolong   z += P e_c
//   post    the post sweeps (FP32: two fused, the inner one recomputed at the
//           neighbours), r^T z (and r^T z_old for flexible CG);
//           last block: beta, loop condition
// Vectors that a kernel reads at stencil neighbours while another block of
// the same kernel writes them are double-buffered by iteration parity.
// Scalar reductions are deterministic: per-block partials summed in block
// order by the last block to arrive.  The loop runs as a CUDA graph whose
// while node is driven by the post kernel, so a solve needs no host round
// trip until it finishes.
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "stencil.cuh"

struct PcgState {
  double bnorm2, tol2bn, rz, pq, alpha, beta, rr, true_rr;
  int iter, done, status, maxit;
  int flexible, pad0;
};

// Vector bound to iteration parity: v[(t + shift) & 1].
template <typename V>
struct Pair {
  V* v[2];
  __device__ __forceinline__ V* at(int t) const { return v[t & 1]; }
};

namespace {

constexpr int TPB = 256;  // threads per block for node-parallel kernels

struct RedSlots {
  double* part;       // [4][max_blocks]
  unsigned* counter;  // [4]
  int max_blocks;
};

__device__ __forceinline__ int load_iter(const PcgState* st) { return st ? *((volatile const int*)&st->iter) : 0; }
__device__ __forceinline__ bool load_done(const PcgState* st) { return st && *((volatile const int*)&st->done); }

__device__ __forceinline__ void mark_breakdown(PcgState* st) {
  st->status = (int)NLSP_ERR_BREAKDOWN;
  st->done = 1;
}

// ----------------------------------------------------------------------------
// PCG start: r_0 = b, x = 0, p = q = 0, ||b||^2.
// ----------------------------------------------------------------------------
__global__ void k_pcg_init(int64_t n, const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r0,
                           double* __restrict__ p0, double* __restrict__ p1, double* __restrict__ q, PcgState* st,
                           double tol, int maxit, int flexible, RedSlots red) {
  __shared__ double sred[32];
  __shared__ int flag;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    r0[i] = bi;
    x[i] = 0.0;
    p0[i] = 0.0;
    p1[i] = 0.0;
    q[i] = 0.0;
    s += bi * bi;
  }
  s = block_sum(s, sred);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[0], &flag)) {
    const double bb = block_sum_partials(red.part, gridDim.x, 1, sred);
    if (threadIdx.x == 0) {
      st->bnorm2 = bb;
      st->tol2bn = tol * tol * bb;
      st->rz = 0.0;
      st->pq = 0.0;
      st->alpha = 0.0;
      st->beta = 0.0;
      st->rr = bb;
      st->true_rr = 0.0;
      st->iter = 0;
      st->maxit = maxit;
      st->flexible = flexible;
      st->status = (int)NLSP_OK;
      st->done = (bb == 0.0) ? 1 : (isfinite(bb) ? 0 : 1);
      if (!isfinite(bb)) st->status = (int)NLSP_ERR_BREAKDOWN;
    }
  }
}

// ----------------------------------------------------------------------------
// spmv: p_t = z_{t-1} + beta p_{t-1}; q = A p_t; p_t^T q.  FP64.
// ----------------------------------------------------------------------------
template <int KIND, typename T>
__global__ void __launch_bounds__(TPB) k_pcg_spmv(StencilView<double> A, Pair<const T> Z, Pair<double> Pv,
                                                  double* __restrict__ q, PcgState* st, RedSlots red) {
  __shared__ double sred[32];
  __shared__ int flag;
  if (load_done(st)) return;
  const int t = load_iter(st);  // number of completed A p products
  const double beta = st->beta;
  const T* __restrict__ z = Z.at(t);
  const double* __restrict__ pin = Pv.at(t);
  double* __restrict__ pout = Pv.at(t + 1);
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    auto pv = [&](int64_t m) { return (double)z[m] + beta * pin[m]; };
    const double pi = pv(i);
    const double qi = stencil_apply<KIND>(A, i, c, pv);
    pout[i] = pi;
    q[i] = qi;
    s += pi * qi;
  }
  s = block_sum(s, sred);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[0], &flag)) {
    const double pq = block_sum_partials(red.part, gridDim.x, 1, sred);
    if (threadIdx.x == 0) {
      st->pq = pq;
      st->iter = t + 1;
      if (!(pq > 0.0) || !isfinite(pq)) mark_breakdown(st);
      else st->alpha = st->rz / pq;
    }
  }
}

// ----------------------------------------------------------------------------
// pre: CG update of x and r (loop mode), ||r||^2, first two Jacobi sweeps.
//   INIT: start of the solve or a standalone apply: r is read, not updated.
// ----------------------------------------------------------------------------
template <int KIND, typename T, bool INIT>
__global__ void __launch_bounds__(TPB) k_pcg_pre(StencilView<T> A, T omega, int nu1, Pair<double> R,
                                                 const double* __restrict__ q, Pair<const double> Pv,
                                                 double* __restrict__ x, T* __restrict__ zout, PcgState* st,
                                                 RedSlots red) {
  __shared__ double sred[32];
  __shared__ int flag;
  if (load_done(st)) return;
  const int t = load_iter(st);
  const double alpha = INIT ? 0.0 : st->alpha;
  const double* __restrict__ rin = INIT ? R.at(t) : R.at(t - 1);
  double* __restrict__ rout = R.at(t);
  const double* __restrict__ p = Pv.at(t);
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    double ri;
    if (INIT) {
      ri = rin[i];
    } else {
      x[i] += alpha * p[i];
      ri = rin[i] - alpha * q[i];
      rout[i] = ri;
      s += ri * ri;
    }
    const T z1 = omega * stencil_dinv<KIND>(A, i) * (T)ri;
    T zf = z1;
    if (nu1 >= 2) {
      const NodeCoord c = node_coord<KIND>(i, A.N);
      auto z1at = [&](int64_t m) -> T {
        if (m == i) return z1;
        const double rm = INIT ? rin[m] : rin[m] - alpha * q[m];
        return omega * stencil_dinv<KIND>(A, m) * (T)rm;
      };
      const T az = stencil_apply<KIND>(A, i, c, z1at);
      zf = z1 + omega * stencil_dinv<KIND>(A, i) * ((T)ri - az);
    }
    zout[i] = zf;
  }
  if (!INIT && st) {
    s = block_sum(s, sred);
    if (threadIdx.x == 0) red.part[blockIdx.x] = s;
    if (last_block_arrive(&red.counter[1], &flag)) {
      const double rr = block_sum_partials(red.part, gridDim.x, 1, sred);
      if (threadIdx.x == 0) {
        st->rr = rr;
        if (!isfinite(rr)) mark_breakdown(st);
        else if (rr <= st->tol2bn) st->done = 1;  // converged: status stays NLSP_OK
      }
    }
  }
}

// One extra Jacobi sweep: zout = zin + w D^-1 (r - A zin).
template <int KIND, typename T>
__global__ void __launch_bounds__(TPB) k_sweep(StencilView<T> A, T omega, Pair<const double> R,
                                               const T* __restrict__ zin, T* __restrict__ zout, const PcgState* st) {
  if (load_done(st)) return;
  const double* __restrict__ r = R.at(load_iter(st));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    const T az = stencil_apply<KIND>(A, i, c, [&](int64_t m) { return zin[m]; });
    zout[i] = zin[i] + omega * stencil_dinv<KIND>(A, i) * ((T)r[i] - az);
  }
}

// ----------------------------------------------------------------------------
// restrict: rho = r - A z, c = P_r^T rho (per-block partials, FP64), and in the
// last block c = sum of partials, e_c = A_c^-1 c (FP64).
// Block = 8 warps; columns are split into NCH chunks of KC, each chunk handled
// by 8/NCH warps, each warp one node tile at a time with 4 nodes per lane
// (one 16-byte load of P per lane per column for FP32).
// ----------------------------------------------------------------------------
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  __device__ __forceinline__ static void load(const float* p, float v[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <> struct Vec4<double> {
  __device__ __forceinline__ static void load(const double* p, double v[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

template <int KIND, typename T, int KC, int NCH>
__global__ void __launch_bounds__(TPB) k_restrict(StencilView<T> A, Pair<const double> R, const T* __restrict__ z,
                                                  const T* __restrict__ P, int k, int r, const double* __restrict__ Ainv,
                                                  double* __restrict__ cpart, double* __restrict__ ec,
                                                  unsigned* counter, const PcgState* st) {
  constexpr int TPG = 8 / NCH;  // tiles per group
  __shared__ double sacc[8][KC];
  __shared__ double cfull[128];
  __shared__ int flag;
  if (load_done(st)) return;
  const double* __restrict__ rv = R.at(load_iter(st));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ch = warp / TPG, tw = warp % TPG;
  const int c0 = ch * KC;
  T acc[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) acc[j] = T(0);
  const int64_t ntiles = (A.n + NLSP_TILE - 1) / NLSP_TILE;
  const int64_t ngroups = (ntiles + TPG - 1) / TPG;
  for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
    const int64_t tt = g * TPG + tw;
    if (tt >= ntiles) continue;
    T rho[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = tt * NLSP_TILE + 4 * lane + u;
      rho[u] = T(0);
      if (i < A.n) {
        const NodeCoord c = node_coord<KIND>(i, A.N);
        rho[u] = (T)rv[i] - stencil_apply<KIND>(A, i, c, [&](int64_t m) { return z[m]; });
      }
    }
    const T* pt = P + (tt * k) * NLSP_TILE + 4 * lane;
#pragma unroll 8
    for (int j = 0; j < KC; ++j) {
      if (c0 + j < r) {
        T pv[4];
        Vec4<T>::load(pt + (int64_t)(c0 + j) * NLSP_TILE, pv);
        acc[j] += rho[0] * pv[0] + rho[1] * pv[1] + rho[2] * pv[2] + rho[3] * pv[3];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KC; ++j) {
    const double v = warp_sum((double)acc[j]);
    if (lane == 0) sacc[warp][j] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NCH * KC; e += blockDim.x) {
    const int chh = e / KC, j = e % KC;
    double s = 0.0;
    for (int w = 0; w < TPG; ++w) s += sacc[chh * TPG + w][j];
    const int col = chh * KC + j;
    if (col < r) cpart[(int64_t)blockIdx.x * k + col] = s;
  }
  if (last_block_arrive(counter, &flag)) {
    for (int col = threadIdx.x; col < r; col += blockDim.x) {
      double s = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) s += cpart[(int64_t)b * k + col];
      cfull[col] = s;
    }
    __syncthreads();
    for (int row = threadIdx.x; row < r; row += blockDim.x) {
      double s = 0.0;
      for (int col = 0; col < r; ++col) s += Ainv[(int64_t)col * r + row] * cfull[col];
      ec[row] = s;
    }
  }
}

// prolong: z += P_r e_c.  Warp per tile, 4 nodes per lane.
template <typename T>
__global__ void __launch_bounds__(TPB) k_prolong(int64_t n, const T* __restrict__ P, int k, int r,
                                                 const double* __restrict__ ec, T* __restrict__ z, const PcgState* st) {
  __shared__ T e[128];
  if (load_done(st)) return;
  for (int j = threadIdx.x; j < r; j += blockDim.x) e[j] = (T)ec[j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = (n + NLSP_TILE - 1) / NLSP_TILE;
  for (int64_t tt = (int64_t)blockIdx.x * 8 + warp; tt < ntiles; tt += (int64_t)gridDim.x * 8) {
    const T* pt = P + (tt * k) * NLSP_TILE + 4 * lane;
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 8
    for (int j = 0; j < r; ++j) {
      T pv[4];
      Vec4<T>::load(pt + (int64_t)j * NLSP_TILE, pv);
      const T ej = e[j];
      a0 += pv[0] * ej;
      a1 += pv[1] * ej;
      a2 += pv[2] * ej;
      a3 += pv[3] * ej;
    }
    const int64_t i0 = tt * NLSP_TILE + 4 * lane;
    if (i0 + 0 < n) z[i0 + 0] += a0;
    if (i0 + 1 < n) z[i0 + 1] += a1;
    if (i0 + 2 < n) z[i0 + 2] += a2;
    if (i0 + 3 < n) z[i0 + 3] += a3;
  }
}

// ----------------------------------------------------------------------------
// post: final post-smoothing sweep(s) into z_t, r^T z_t (and r^T z_{t-1}).
//   FUSE2: two sweeps in one pass, the first recomputed at the neighbours.
// ----------------------------------------------------------------------------
template <int KIND, typename T, bool FUSE2, bool INIT>
__global__ void __launch_bounds__(TPB) k_pcg_post(StencilView<T> A, T omega, Pair<const double> R,
                                                  const T* __restrict__ zin, Pair<T> Z, PcgState* st, RedSlots red,
                                                  cudaGraphConditionalHandle cond, int set_cond) {
  __shared__ double sred[32];
  __shared__ int flag;
  if (load_done(st)) {
    if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const int t = load_iter(st);
  const double* __restrict__ r = R.at(t);
  T* __restrict__ zout = Z.at(t);
  const T* __restrict__ zold = Z.at(t + 1);  // z_{t-1}
  const bool flex = st && !INIT && st->flexible;
  double s_rz = 0.0, s_ro = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    T zf;
    if (FUSE2) {
      auto z4at = [&](int64_t m, NodeCoord cm) -> T {
        const T az = stencil_apply<KIND>(A, m, cm, [&](int64_t mm) { return zin[mm]; });
        return zin[m] + omega * stencil_dinv<KIND>(A, m) * ((T)r[m] - az);
      };
      const T z4i = z4at(i, c);
      T az4 = stencil_diag<KIND>(A, i) * z4i;
      for_each_neighbour<KIND>(A, i, c, [&](int64_t m, NodeCoord cm, T a) { az4 += a * z4at(m, cm); });
      zf = z4i + omega * stencil_dinv<KIND>(A, i) * ((T)r[i] - az4);
    } else {
      const T az = stencil_apply<KIND>(A, i, c, [&](int64_t m) { return zin[m]; });
      zf = zin[i] + omega * stencil_dinv<KIND>(A, i) * ((T)r[i] - az);
    }
    zout[i] = zf;
    if (st) {
      s_rz += r[i] * (double)zf;
      if (flex) s_ro += r[i] * (double)zold[i];
    }
  }
  if (!st) return;
  s_rz = block_sum(s_rz, sred);
  if (flex) s_ro = block_sum(s_ro, sred);
  if (threadIdx.x == 0) {
    red.part[2 * red.max_blocks + blockIdx.x] = s_rz;
    red.part[3 * red.max_blocks + blockIdx.x] = s_ro;
  }
  if (last_block_arrive(&red.counter[2], &flag)) {
    const double rz = block_sum_partials(red.part + 2 * red.max_blocks, gridDim.x, 1, sred);
    const double ro = flex ? block_sum_partials(red.part + 3 * red.max_blocks, gridDim.x, 1, sred) : 0.0;
    if (threadIdx.x == 0) {
      if (!(rz > 0.0) || !isfinite(rz)) {
        mark_breakdown(st);
      } else {
        st->beta = INIT ? 0.0 : (rz - ro) / st->rz;
        st->rz = rz;
      }
      if (!st->done && st->iter >= st->maxit) {
        st->status = (int)NLSP_NOT_CONVERGED;
        st->done = 1;
      }
      if (set_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
    }
  }
}

// ||b - A x||^2 after the solve (FP64).
template <int KIND>
__global__ void __launch_bounds__(TPB) k_true_residual(StencilView<double> A, const double* __restrict__ b,
                                                       const double* __restrict__ x, PcgState* st, RedSlots red) {
  __shared__ double sred[32];
  __shared__ int flag;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    const double ri = b[i] - stencil_apply<KIND>(A, i, c, [&](int64_t m) { return x[m]; });
    s += ri * ri;
  }
  s = block_sum(s, sred);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[3], &flag)) {
    const double tr = block_sum_partials(red.part, gridDim.x, 1, sred);
    if (threadIdx.x == 0) st->true_rr = tr;
  }
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

}  // namespace

// ============================================================================
// Host side
// ============================================================================
struct PcgWork {
  int64_t n = 0;
  int tsize = 0;
  double* vec = nullptr;   // R[2], Pv[2], q, x  (n each)
  void* zbuf = nullptr;    // Z[2] in the preconditioner precision
  double* part = nullptr;  // [4][max_blocks]
  unsigned* counter = nullptr;
  int max_blocks = 0;
  PcgState* st = nullptr;  // the state the graph works on
  PcgState* st_all = nullptr;
  int st_cap = 0;
  PcgState* h_st = nullptr;  // pinned
  cudaStream_t cap = nullptr;  // capture stream (never the legacy default stream)
  cudaGraph_t g_while = nullptr, g_iter = nullptr;
  cudaGraphExec_t x_while = nullptr, x_iter = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int built_r = -1;
};

namespace {

void destroy_graphs(PcgWork* w) {
  if (w->x_while) cudaGraphExecDestroy(w->x_while);
  if (w->g_while) cudaGraphDestroy(w->g_while);
  if (w->x_iter) cudaGraphExecDestroy(w->x_iter);
  if (w->g_iter) cudaGraphDestroy(w->g_iter);
  w->x_while = nullptr;
  w->g_while = nullptr;
  w->x_iter = nullptr;
  w->g_iter = nullptr;
  w->built_r = -1;
}

void free_work(PcgWork* w) {
  if (!w) return;
  destroy_graphs(w);
  if (w->vec) cudaFree(w->vec);
  if (w->zbuf) cudaFree(w->zbuf);
  if (w->part) cudaFree(w->part);
  if (w->counter) cudaFree(w->counter);
  if (w->st_all) cudaFree(w->st_all);
  if (w->h_st) cudaFreeHost(w->h_st);
  if (w->cap) cudaStreamDestroy(w->cap);
  delete w;
}

nlsp_status ensure_work(nlsp_prec* M, int m) {
  nlsp_ctx* ctx = M->ctx;
  if (!M->pcg) {
    PcgWork* w = new PcgWork();
    w->n = M->n;
    w->tsize = M->precision == NLSP_FP64 ? 8 : 4;
    w->max_blocks = ctx->num_sms * 8;
    M->pcg = w;
    NLSP_CUDA(cudaMalloc(&w->vec, sizeof(double) * M->n * 6));
    NLSP_CUDA(cudaMalloc(&w->zbuf, (size_t)w->tsize * M->n * 2));
    NLSP_CUDA(cudaMalloc(&w->part, sizeof(double) * 4 * w->max_blocks));
    NLSP_CUDA(cudaMalloc(&w->counter, sizeof(unsigned) * 4));
    NLSP_CUDA(cudaMemsetAsync(w->counter, 0, sizeof(unsigned) * 4, ctx->stream));
    NLSP_CUDA(cudaMemsetAsync(w->zbuf, 0, (size_t)w->tsize * M->n * 2, ctx->stream));
    NLSP_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
  }
  PcgWork* w = M->pcg;
  if (w->st_cap < m + 1) {
    if (w->st_all) cudaFree(w->st_all);
    if (w->h_st) cudaFreeHost(w->h_st);
    w->st_all = nullptr;
    w->h_st = nullptr;
    w->st_cap = 0;
    NLSP_CUDA(cudaMalloc(&w->st_all, sizeof(PcgState) * (m + 1)));
    NLSP_CUDA(cudaMallocHost(&w->h_st, sizeof(PcgState) * (m + 1)));
    w->st_cap = m + 1;
    w->st = w->st_all + m;  // working state sits after the per-column copies
    destroy_graphs(w);      // the graphs hold the old state pointer
  }
  return NLSP_OK;
}

RedSlots red_of(PcgWork* w) { return RedSlots{w->part, w->counter, w->max_blocks}; }

int node_grid(const nlsp_ctx* ctx, int64_t n) { return grid_for(ctx, n, TPB, 8); }

// Enqueues one preconditioner application on stream s.
//  loop = false: z = B r with r = R.at(iter) (start of a solve, or standalone)
//  loop = true:  the PCG iteration body after the spmv kernel
template <int KIND, typename T>
nlsp_status enqueue_apply(const nlsp_prec* M, cudaStream_t s, bool loop, Pair<double> R, const double* q,
                          Pair<const double> Pv, double* x, Pair<T> Z, PcgState* st, RedSlots red,
                          cudaGraphConditionalHandle cond, int set_cond) {
  const nlsp_ctx* ctx = M->ctx;
  const StencilView<T>& A = *reinterpret_cast<const StencilView<T>*>(
      sizeof(T) == 8 ? (const void*)&M->A->v64 : (const void*)&M->A->v32);
  const T omega = (T)M->omega;
  const int g = node_grid(ctx, M->n);
  T* cur = (T*)M->w0;
  T* oth = (T*)M->w1;
  Pair<const double> Rc{{R.v[0], R.v[1]}};
  if (loop)
    k_pcg_pre<KIND, T, false><<<g, TPB, 0, s>>>(A, omega, M->nu1, R, q, Pv, x, cur, st, red);
  else
    k_pcg_pre<KIND, T, true><<<g, TPB, 0, s>>>(A, omega, M->nu1, R, q, Pv, x, cur, st, red);
  for (int sw = 2; sw < M->nu1; ++sw) {
    k_sweep<KIND, T><<<g, TPB, 0, s>>>(A, omega, Rc, cur, oth, st);
    std::swap(cur, oth);
  }
  // restriction + coarse solve
  const int r = M->r, k = M->k;
  const int64_t ntiles = (M->n + NLSP_TILE - 1) / NLSP_TILE;
  const int nch = r <= 32 ? 1 : (r <= 64 ? 2 : 4);
  const int64_t ngroups = (ntiles + (8 / nch) - 1) / (8 / nch);
  const int rg = (int)std::min<int64_t>(ngroups, M->rblocks);
  const T* P = (const T*)M->P;
  if (nch == 1)
    k_restrict<KIND, T, 32, 1><<<rg, TPB, 0, s>>>(A, Rc, cur, P, k, r, M->Ainv, M->cpart, M->ec, M->counter, st);
  else if (nch == 2)
    k_restrict<KIND, T, 32, 2><<<rg, TPB, 0, s>>>(A, Rc, cur, P, k, r, M->Ainv, M->cpart, M->ec, M->counter, st);
  else
    k_restrict<KIND, T, 32, 4><<<rg, TPB, 0, s>>>(A, Rc, cur, P, k, r, M->Ainv, M->cpart, M->ec, M->counter, st);
  const int pg = (int)std::max<int64_t>(1, std::min<int64_t>((ntiles + 7) / 8, (int64_t)ctx->num_sms * 8));
  k_prolong<T><<<pg, TPB, 0, s>>>(M->n, P, k, r, M->ec, cur, st);
  constexpr bool FUSE2 = sizeof(T) == 4;
  const int nfinal = (FUSE2 && M->nu2 >= 2) ? 2 : 1;
  for (int sw = nfinal; sw < M->nu2; ++sw) {
    k_sweep<KIND, T><<<g, TPB, 0, s>>>(A, omega, Rc, cur, oth, st);
    std::swap(cur, oth);
  }
  Pair<const double> Rp{{R.v[0], R.v[1]}};
  if (nfinal == 2) {
    if (loop) k_pcg_post<KIND, T, true, false><<<g, TPB, 0, s>>>(A, omega, Rp, cur, Z, st, red, cond, set_cond);
    else k_pcg_post<KIND, T, true, true><<<g, TPB, 0, s>>>(A, omega, Rp, cur, Z, st, red, cond, set_cond);
  } else {
    if (loop) k_pcg_post<KIND, T, false, false><<<g, TPB, 0, s>>>(A, omega, Rp, cur, Z, st, red, cond, set_cond);
    else k_pcg_post<KIND, T, false, true><<<g, TPB, 0, s>>>(A, omega, Rp, cur, Z, st, red, cond, set_cond);
  }
  NLSP_LAUNCH_CHECK();
  return NLSP_OK;
}

template <int KIND, typename T>
struct Solver {
  static Pair<double> Rpair(PcgWork* w) { return Pair<double>{{w->vec, w->vec + w->n}}; }
  static Pair<double> Ppair(PcgWork* w) { return Pair<double>{{w->vec + 2 * w->n, w->vec + 3 * w->n}}; }
  static double* q(PcgWork* w) { return w->vec + 4 * w->n; }
  static double* x(PcgWork* w) { return w->vec + 5 * w->n; }
  static Pair<T> Zpair(PcgWork* w) { return Pair<T>{{(T*)w->zbuf, (T*)w->zbuf + w->n}}; }

  // One PCG iteration body (spmv, pre, restrict, prolong, post).
  static nlsp_status enqueue_body(const nlsp_prec* M, cudaStream_t s, int set_cond) {
    PcgWork* w = M->pcg;
    const int g = node_grid(M->ctx, M->n);
    Pair<const T> Zc{{(const T*)w->zbuf, (const T*)w->zbuf + w->n}};
    k_pcg_spmv<KIND, T><<<g, TPB, 0, s>>>(M->A->v64, Zc, Ppair(w), q(w), w->st, red_of(w));
    NLSP_LAUNCH_CHECK();
    Pair<double> P2 = Ppair(w);
    Pair<const double> Pc{{P2.v[0], P2.v[1]}};
    return enqueue_apply<KIND, T>(M, s, true, Rpair(w), q(w), Pc, x(w), Zpair(w), w->st, red_of(w), w->cond,
                                  set_cond);
  }

  static nlsp_status build_graphs(nlsp_prec* M) {
    PcgWork* w = M->pcg;
    destroy_graphs(w);
    // while-loop graph: a single conditional node whose body is one iteration
    NLSP_CUDA(cudaGraphCreate(&w->g_while, 0));
    NLSP_CUDA(cudaGraphConditionalHandleCreate(&w->cond, w->g_while, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = w->cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    NLSP_CUDA(cudaGraphAddNode(&node, w->g_while, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    NLSP_CUDA(cudaStreamBeginCaptureToGraph(w->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    nlsp_status st = enqueue_body(M, w->cap, 1);
    cudaGraph_t dummy = nullptr;
    cudaError_t e = cudaStreamEndCapture(w->cap, &dummy);
    if (st != NLSP_OK) return st;
    NLSP_CUDA(e);
    NLSP_CUDA(cudaGraphInstantiate(&w->x_while, w->g_while, 0));
    // single-iteration graph for host-checked mode
    NLSP_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    st = enqueue_body(M, w->cap, 0);
    e = cudaStreamEndCapture(w->cap, &w->g_iter);
    if (st != NLSP_OK) return st;
    NLSP_CUDA(e);
    NLSP_CUDA(cudaGraphInstantiate(&w->x_iter, w->g_iter, 0));
    w->built_r = M->r;
    return NLSP_OK;
  }

  static nlsp_status solve(nlsp_prec* M, int m, const double* B, int64_t ldb, double* X, int64_t ldx,
                           const nlsp_solve_params* prm, nlsp_solve_info* infos) {
    nlsp_ctx* ctx = M->ctx;
    cudaStream_t s = ctx->stream;
    NLSP_TRY(ensure_work(M, m));
    PcgWork* w = M->pcg;
    if (!w->x_while || w->built_r != M->r) NLSP_TRY(build_graphs(M));
    const int flexible = prm->flexible < 0 ? (M->precision != NLSP_FP64) : (prm->flexible != 0);
    const int g = node_grid(ctx, M->n);
    for (int col = 0; col < m; ++col) {
      const double* b = B + col * ldb;
      Pair<double> R = Rpair(w), P2 = Ppair(w);
      k_pcg_init<<<g, TPB, 0, s>>>(M->n, b, x(w), R.v[0], P2.v[0], P2.v[1], q(w), w->st, prm->tol, prm->maxit,
                                   flexible, red_of(w));
      NLSP_LAUNCH_CHECK();
      Pair<const double> Pc{{P2.v[0], P2.v[1]}};
      NLSP_TRY((enqueue_apply<KIND, T>(M, s, false, R, q(w), Pc, x(w), Zpair(w), w->st, red_of(w), 0, 0)));
      if (prm->graph_mode == 1) {
        NLSP_CUDA(cudaGraphLaunch(w->x_while, s));
      } else {
        int done_iters = 0;
        while (done_iters < prm->maxit) {
          const int chunk = std::min(8, prm->maxit - done_iters);
          for (int c = 0; c < chunk; ++c) NLSP_CUDA(cudaGraphLaunch(w->x_iter, s));
          done_iters += chunk;
          NLSP_CUDA(cudaMemcpyAsync(w->h_st, w->st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
          NLSP_CUDA(cudaStreamSynchronize(s));
          if (w->h_st[0].done) break;
        }
      }
      k_true_residual<KIND><<<g, TPB, 0, s>>>(M->A->v64, b, x(w), w->st, red_of(w));
      NLSP_LAUNCH_CHECK();
      NLSP_CUDA(cudaMemcpyAsync(X + col * ldx, x(w), sizeof(double) * M->n, cudaMemcpyDeviceToDevice, s));
      NLSP_CUDA(cudaMemcpyAsync(w->st_all + col, w->st, sizeof(PcgState), cudaMemcpyDeviceToDevice, s));
    }
    NLSP_CUDA(cudaMemcpyAsync(w->h_st, w->st_all, sizeof(PcgState) * m, cudaMemcpyDeviceToHost, s));
    NLSP_CUDA(cudaStreamSynchronize(s));
    nlsp_status worst = NLSP_OK;
    for (int col = 0; col < m; ++col) {
      const PcgState& h = w->h_st[col];
      int stc = h.status;
      if (stc == NLSP_OK && !h.done) stc = NLSP_NOT_CONVERGED;
      if (infos) {
        infos[col].iterations = h.iter;
        infos[col].status = stc;
        infos[col].relres = h.bnorm2 > 0 ? sqrt(h.rr / h.bnorm2) : 0.0;
        infos[col].true_relres = h.bnorm2 > 0 ? sqrt(h.true_rr / h.bnorm2) : 0.0;
      }
      if (stc == NLSP_ERR_BREAKDOWN) worst = NLSP_ERR_BREAKDOWN;
      else if (stc == NLSP_NOT_CONVERGED && worst == NLSP_OK) worst = NLSP_NOT_CONVERGED;
    }
    return worst;
  }

  static nlsp_status apply(nlsp_prec* M, int m, const double* Rin, int64_t ldr, double* Z, int64_t ldz) {
    nlsp_ctx* ctx = M->ctx;
    cudaStream_t s = ctx->stream;
    NLSP_TRY(ensure_work(M, 1));
    PcgWork* w = M->pcg;
    T* zout = (T*)w->zbuf;
    for (int col = 0; col < m; ++col) {
      double* rc = const_cast<double*>(Rin + col * ldr);
      Pair<double> R{{rc, rc}};
      Pair<const double> Pc{{nullptr, nullptr}};
      Pair<T> Zp{{zout, zout}};
      NLSP_TRY((enqueue_apply<KIND, T>(M, s, false, R, nullptr, Pc, nullptr, Zp, nullptr, red_of(w), 0, 0)));
      k_to_double<T><<<node_grid(ctx, M->n), TPB, 0, s>>>(zout, Z + col * ldz, M->n);
      NLSP_LAUNCH_CHECK();
    }
    return NLSP_OK;
  }
};

template <typename F>
nlsp_status dispatch(const nlsp_prec* M, F f) {
  if (M->precision == NLSP_FP64) {
    switch (M->A->kind) {
      case ST_5PT: return f(Solver<ST_5PT, double>());
      case ST_9PT: return f(Solver<ST_9PT, double>());
      default: return f(Solver<ST_7PT, double>());
    }
  }
  switch (M->A->kind) {
    case ST_5PT: return f(Solver<ST_5PT, float>());
    case ST_9PT: return f(Solver<ST_9PT, float>());
    default: return f(Solver<ST_7PT, float>());
  }
}

}  // namespace

void nlsp_internal_invalidate_graphs(nlsp_prec* M) {
  if (M && M->pcg) destroy_graphs(M->pcg);
}

extern "C" nlsp_status nlsp_apply_prec(nlsp_ctx* ctx, const nlsp_prec* Mc, int m, const double* dev_R, int64_t ldr,
                                       double* dev_Z, int64_t ldz) {
  if (!ctx || !Mc || m < 0 || (m > 0 && (!dev_R || !dev_Z)) || ldr < Mc->n || ldz < Mc->n) return NLSP_ERR_INVALID;
  if (m == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  nlsp_prec* M = const_cast<nlsp_prec*>(Mc);
  return dispatch(M, [&](auto S) { return decltype(S)::apply(M, m, dev_R, ldr, dev_Z, ldz); });
}

extern "C" nlsp_status nlsp_solve(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* Mc, int m, const double* dev_B,
                                  int64_t ldb, double* dev_X, int64_t ldx, const nlsp_solve_params* params,
                                  nlsp_solve_info* infos) {
  if (!ctx || !A || !Mc || !params || Mc->A != A || m < 0 || ldb < A->n || ldx < A->n) return NLSP_ERR_INVALID;
  if (m > 0 && (!dev_B || !dev_X)) return NLSP_ERR_INVALID;
  if (!(params->tol >= 0.0) || params->maxit < 1 || (params->graph_mode != 0 && params->graph_mode != 1))
    return NLSP_ERR_INVALID;
  if (m == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  nlsp_prec* M = const_cast<nlsp_prec*>(Mc);
  return dispatch(M, [&](auto S) { return decltype(S)::solve(M, m, dev_B, ldb, dev_X, ldx, params, infos); });
}

extern "C" void nlsp_free_prec(nlsp_prec* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  cudaDeviceSynchronize();  // the context (and its stream) may already be gone
  free_work(M->pcg);
  void* bufs[] = {M->P, M->sigma, M->Ac, M->L, M->Ainv, M->cpart, M->ec, M->counter, M->status, M->w0, M->w1};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete M;
}
