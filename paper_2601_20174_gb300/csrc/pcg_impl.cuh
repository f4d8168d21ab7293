// Two-level preconditioner apply (Algorithm 1, "Apply preconditioner to
// residual b") and preconditioned CG (Sec. 4, two-grid solver evaluation).
//
// GB300 runs FP64 (including FP32<->FP64 conversions) at ~2 lanes/clk/SM,
// 1/62 of FP32, so the iteration is arranged to spend FP64 only on the outer
// recurrences and their dot products; everything inside the preconditioner
// is FP32 in the mixed path, where recomputing stencil values is cheaper than
// storing them.  One PCG iteration t:
//   spmv      p_t = z_{t-1} + beta p_{t-1} (evaluated on the fly, also at the
//             stencil neighbours), q = A p_t, p^T q;   last block: alpha
//   pre       x += alpha p, r -= alpha q, ||r||^2, rT = r in the
//             preconditioner precision;                last block: stop test
//   restrict  the nu1 <= 2 pre-sweeps from z = 0 recomputed from rT
//             (z1 = w D^-1 rT is elementwise, so z2 at a node needs rT only
//             at its stencil neighbours), rho = rT - A z2, c = P_r^T rho,
//             z2 stored;                                last block: e_c = A_c^-1 c
//   prolong   z += P_r e_c
//   post      the post sweeps (FP32: the last two fused, the inner one
//             recomputed at the neighbours), z_t stored in FP64, r^T z_t
//             (and r^T z_{t-1} for flexible CG); last block: beta, loop test
// The FP64 path (T = double) stores the pre-sweeps instead of recomputing.
// Vectors that a kernel reads at stencil neighbours while another block of
// the same kernel writes them are double-buffered by iteration parity.
// Scalar reductions are deterministic: per-block partials summed in block
// order by the last block to arrive.  The loop runs as a CUDA graph whose
// while node is driven by the post kernel, so a solve needs no host round
// trip until it finishes.
//
// This header holds the templated kernels and the host-side solver of every
// stencil kind; each pcg_<kind>_<precision>.cu instantiates one (kind,
// precision) pair and exports it as a PcgKindOps table, so the instantiations
// compile in parallel.  pcg.cu holds the C-ABI entry points.
#pragma once

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "convert.cuh"
#include "kernels.cuh"
#include "stencil.cuh"
#include "tma.cuh"

struct PcgState {
  double bnorm2, tol2bn, rz, pq, alpha, beta, rr, true_rr;
  int iter, done, status, maxit;
  int flexible, pad0;
};

// Vector bound to iteration parity: v[t & 1].
template <typename V>
struct Pair {
  V* v[2];
  __device__ __forceinline__ V* at(int t) const { return v[t & 1]; }
};

// Team plan of a batched solve (host only; defined in pcg.cu).
nlsp_status nlsp_internal_plan_teams(int count, const int64_t* n, const int* cap, int G, int tiles_per_cta,
                                     int* first, int* size, double* start);


namespace {

constexpr int TPB = 256;     // threads per block for node-parallel kernels
constexpr int NODE_BPS = 8;  // node-kernel blocks per SM: one node per thread up to full occupancy

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

// FP64 block sum with few FP64 instructions: partials go to shared memory and
// one warp adds them (the FP64 pipe is charged per warp instruction).  The
// result is valid in warp 0.  Fixed order => deterministic.
__device__ __forceinline__ double block_sum_lean(double v, double* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += sm[i];
    s = warp_sum(s);
  }
  __syncthreads();
  return s;
}

__device__ __forceinline__ double sum_partials_lean(const double* part, int count, double* sm) {
  double s = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) s += part[b];
  return block_sum_lean(s, sm);
}

// ----------------------------------------------------------------------------
// PCG start: r_0 = b, rT = b, x = 0, p = q = 0, ||b||^2.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TPB) k_pcg_init(int64_t n, const double* __restrict__ b, double* __restrict__ x,
                                                  double* __restrict__ r, T* __restrict__ rT, double* __restrict__ p0,
                                                  double* __restrict__ p1, double* __restrict__ q, PcgState* st,
                                                  double tol, int maxit, int flexible, RedSlots red) {
  __shared__ double sm[TPB];
  __shared__ int flag;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double bi = b[i];
    r[i] = bi;
    if (sizeof(T) == 4) rT[i] = (T)bi;
    x[i] = 0.0;
    p0[i] = 0.0;
    p1[i] = 0.0;
    q[i] = 0.0;
    s += bi * bi;
  }
  s = block_sum_lean(s, sm);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[0], &flag)) {
    const double bb = sum_partials_lean(red.part, gridDim.x, sm);
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
template <int KIND>
__global__ void __launch_bounds__(TPB) k_pcg_spmv(StencilView<double> A, Pair<const double> Z, Pair<double> Pv,
                                                  double* __restrict__ q, PcgState* st, RedSlots red) {
  __shared__ double sm[TPB];
  __shared__ int flag;
  if (load_done(st)) return;
  const int t = load_iter(st);  // number of completed A p products
  const double beta = st->beta;
  const double* __restrict__ z = Z.at(t);
  const double* __restrict__ pin = Pv.at(t);
  double* __restrict__ pout = Pv.at(t + 1);
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    auto pv = [&](int64_t m) { return fma(beta, pin[m], z[m]); };
    const double pi = pv(i);
    const double qi = stencil_apply<KIND>(A, i, c, pv);
    pout[i] = pi;
    q[i] = qi;
    s = fma(pi, qi, s);
  }
  s = block_sum_lean(s, sm);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[0], &flag)) {
    const double pq = sum_partials_lean(red.part, gridDim.x, sm);
    if (threadIdx.x == 0) {
      st->pq = pq;
      st->iter = t + 1;
      if (!(pq > 0.0) || !isfinite(pq)) mark_breakdown(st);
      else st->alpha = st->rz / pq;
    }
  }
}

// ----------------------------------------------------------------------------
// pre: x += alpha p, r -= alpha q, ||r||^2, rT = r (preconditioner precision).
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TPB) k_pcg_pre(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                 T* __restrict__ rT, const double* __restrict__ q,
                                                 Pair<const double> Pv, PcgState* st, RedSlots red) {
  __shared__ double sm[TPB];
  __shared__ int flag;
  if (load_done(st)) return;
  const int t = load_iter(st);
  const double alpha = st->alpha;
  const double* __restrict__ p = Pv.at(t);
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    if (sizeof(T) == 4) rT[i] = from_f64<T>(ri);
    s = fma(ri, ri, s);
  }
  s = block_sum_lean(s, sm);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[1], &flag)) {
    const double rr = sum_partials_lean(red.part, gridDim.x, sm);
    if (threadIdx.x == 0) {
      st->rr = rr;
      if (!isfinite(rr)) mark_breakdown(st);
      else if (rr <= st->tol2bn) st->done = 1;  // converged: status stays NLSP_OK
    }
  }
}

// ----------------------------------------------------------------------------
// Jacobi sweeps on A z = r (the residual in the preconditioner precision).
// ----------------------------------------------------------------------------
// z after `NU` (1 or 2) sweeps from z = 0, at node m with coordinates cm.
// rT is not __restrict__: the persistent solver rewrites it between phases of
// one launch, so its loads must not take the read-only (non-coherent) path.
template <int KIND, typename T, int NU>
__device__ __forceinline__ T presmooth_at(const StencilView<T>& A, T omega, const T* rT, int64_t m, NodeCoord cm) {
  const T z1m = omega * stencil_dinv<KIND>(A, m) * rT[m];
  if (NU == 1) return z1m;
  const T az = stencil_apply<KIND>(A, m, cm, [&](int64_t mm) {
    return mm == m ? z1m : omega * stencil_dinv<KIND>(A, mm) * rT[mm];
  });
  return z1m + omega * stencil_dinv<KIND>(A, m) * (rT[m] - az);
}

// zout = z after NU sweeps from zero (used when the pre-sweeps are stored).
template <int KIND, typename T, int NU>
__global__ void __launch_bounds__(TPB) k_presmooth(StencilView<T> A, T omega, const T* __restrict__ rT,
                                                   T* __restrict__ zout, const PcgState* st) {
  if (load_done(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
    zout[i] = presmooth_at<KIND, T, NU>(A, omega, rT, i, node_coord<KIND>(i, A.N));
}

// One sweep: zout = zin + w D^-1 (rT - A zin).
template <int KIND, typename T>
__global__ void __launch_bounds__(TPB) k_sweep(StencilView<T> A, T omega, const T* __restrict__ rT,
                                               const T* __restrict__ zin, T* __restrict__ zout, const PcgState* st) {
  if (load_done(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    const T az = stencil_apply<KIND>(A, i, c, [&](int64_t m) { return zin[m]; });
    zout[i] = zin[i] + omega * stencil_dinv<KIND>(A, i) * (rT[i] - az);
  }
}

// ----------------------------------------------------------------------------
// restrict: rho = rT - A z, c = P_r^T rho as per-block partials in T (the
// coarse solve is the prolongation's first step).
//   ZMODE 0: z read from zin;  ZMODE 1 / 2: z = 1 / 2 pre-sweeps recomputed
//   from rT and stored to zout.
// Block = 8 warps; columns are split into NCH chunks of 32, each chunk handled
// by 8/NCH warps, each warp one 128-node tile at a time with 4 nodes per lane
// (one 16-byte load of P per lane per column for FP32).
// ----------------------------------------------------------------------------
// Warp reduce-scatter of 32 per-lane values: afterwards lane l holds the sum
// over the warp of value l (31 shuffle-adds per lane instead of 5 per value).
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < off; ++j) {
      const T send = upper ? v[j] : v[j + off];
      const T keep = upper ? v[j + off] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// The two P-streaming kernels (restrict, prolong) run one CTA per SM over a
// contiguous range of node tiles.  Thread 0 keeps NSTAGE tiles (the first r
// columns of a tile are one contiguous block: r x 128 values) in flight with
// bulk asynchronous copies into a shared-memory ring, completion tracked by
// one mbarrier per stage; a CTA-wide barrier after each tile releases its
// stage for the next copy.  Thread (w, h) of a CTA of 128 * NCH threads owns
// node w of the tile and columns [32 h, 32 h + 32).
struct StreamArgs {
  int nstage;     // tiles in flight per CTA
  int max_nodes;  // capacity of the per-CTA residual buffer (restrict)
  int n_tm;       // persistent solver: tiles per CTA kept in tensor memory
  int n_sm;       // persistent solver: tiles per CTA kept in shared memory
};

// Waits for stage `s` of iteration `it`; on a timeout records it in *abort_s.
__device__ __forceinline__ void stream_wait(uint64_t* bar, int it, int nstage, int* abort_s) {
  if (!tma::mbar_wait(&bar[it % nstage], (unsigned)((it / nstage) & 1))) *abort_s = 1;
}

// After a timeout: waits (bounded) for every copy still in flight, so that
// no copy lands in shared memory after the CTA has moved on.
__device__ __forceinline__ void stream_drain(uint64_t* bar, int it, int nt, int nstage) {
  if (threadIdx.x == 0)
    for (int j = it; j < nt && j < it + nstage; ++j) tma::mbar_wait(&bar[j % nstage], (unsigned)((j / nstage) & 1));
}

__device__ __forceinline__ void report_timeout(PcgState* st, int* err) {
  if (threadIdx.x != 0) return;
  if (st) {
    st->status = (int)NLSP_ERR_TIMEOUT;
    st->done = 1;
  } else {
    atomicExch(err, (int)NLSP_ERR_TIMEOUT);
  }
}

template <int KIND, typename T, int NCH, int ZMODE>
__global__ void __launch_bounds__(128 * NCH) k_restrict(StencilView<T> A, T omega, const T* __restrict__ rT,
                                                        const T* __restrict__ zin, T* __restrict__ zout,
                                                        const T* __restrict__ P, int k, int r, StreamArgs sa,
                                                        T* __restrict__ cpart, PcgState* st, int* err) {
  constexpr int NT = 128 * NCH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[8];
  __shared__ T sacc[NT / 32][32];
  __shared__ int abort_s;
  if (load_done(st)) return;
  const int nstage = sa.nstage;
  const int ntiles = (int)((A.n + NLSP_TILE - 1) / NLSP_TILE);
  const int t0 = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
  const int nt = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x) - t0;
  const unsigned tile_bytes = (unsigned)r * NLSP_TILE * (unsigned)sizeof(T);
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* rho_s = buf + (size_t)nstage * r * NLSP_TILE;
  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int s = 0; s < nstage; ++s) tma::mbar_init(&bar[s], 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < nstage && s < nt; ++s) {
      tma::mbar_arrive_expect_tx(&bar[s], tile_bytes);
      tma::bulk_g2s(buf + (size_t)s * r * NLSP_TILE, P + (size_t)(t0 + s) * k * NLSP_TILE, tile_bytes, &bar[s]);
    }
  // phase 1 (overlaps the first copies): rho = rT - A z for the CTA's nodes,
  // four nodes per thread at a time as independent chains, so that their
  // loads are in flight together
  auto rho_at = [&](int e) {
    const int i = t0 * NLSP_TILE + e;
    T rho = T(0);
    if (i < A.n) {
      const NodeCoord c = node_coord<KIND>(i, A.N);
      if (ZMODE == 0) {
        rho = rT[i] - stencil_apply<KIND>(A, i, c, [&](int64_t m) { return zin[m]; });
      } else {
        const T zi = presmooth_at<KIND, T, ZMODE>(A, omega, rT, i, c);
        T az = stencil_diag<KIND>(A, i) * zi;
        for_each_neighbour<KIND>(A, i, c, [&](int64_t m, NodeCoord cm, T a) {
          az += a * presmooth_at<KIND, T, ZMODE>(A, omega, rT, m, cm);
        });
        rho = rT[i] - az;
        zout[i] = zi;
      }
    }
    return rho;
  };
  const int total = nt * NLSP_TILE;
  for (int e0 = threadIdx.x; e0 < total; e0 += 4 * NT) {
    T rv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) rv[u] = e0 + u * NT < total ? rho_at(e0 + u * NT) : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (e0 + u * NT < total) rho_s[e0 + u * NT] = rv[u];
  }
  __syncthreads();
  // phase 2: stream the tiles, acc[j] = sum over the CTA's nodes of rho * P
  const int w = threadIdx.x & (NLSP_TILE - 1), h = threadIdx.x >> 7;
  const int c0 = h * 32;
  T acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = T(0);
  for (int it = 0; it < nt; ++it) {
    stream_wait(bar, it, nstage, &abort_s);
    const T* tile = buf + (size_t)(it % nstage) * r * NLSP_TILE;
    const T rho = rho_s[it * NLSP_TILE + w];
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < r) acc[j] += rho * tile[(c0 + j) * NLSP_TILE + w];
    __syncthreads();
    if (abort_s) {
      stream_drain(bar, it, nt, nstage);
      report_timeout(st, err);
      break;
    }
    if (threadIdx.x == 0 && it + nstage < nt) {
      const int s = it % nstage;
      tma::mbar_arrive_expect_tx(&bar[s], tile_bytes);
      tma::bulk_g2s(buf + (size_t)s * r * NLSP_TILE, P + (size_t)(t0 + it + nstage) * k * NLSP_TILE, tile_bytes,
                    &bar[s]);
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  sacc[warp][lane] = warp_reduce_scatter32(acc, lane);  // column c0 + lane, summed over the warp
  __syncthreads();
  for (int col = threadIdx.x; col < r; col += NT) {
    const int hh = col >> 5, j = col & 31;
    T s = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) s += sacc[hh * 4 + q][j];
    cpart[(int64_t)blockIdx.x * k + col] = s;
  }
}

// prolong: e_c = A_c^-1 (sum of the restriction's nb per-block partials; A_c^-1
// in T, rounded once from the FP64 inverse of the FP64 Cholesky factor), then
// z += P_r e_c, streaming the tiles like restrict.  Every CTA forms e_c itself
// in the same fixed order while its first tiles are in flight.
template <typename T, int NCH>
__global__ void __launch_bounds__(128 * NCH) k_prolong(int64_t n, const T* __restrict__ P, int k, int r,
                                                       StreamArgs sa, const T* __restrict__ cpart, int nb,
                                                       const T* __restrict__ Ainv, T* __restrict__ z, PcgState* st,
                                                       int* err) {
  constexpr int NT = 128 * NCH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[8];
  __shared__ T zpart[2][NCH][NLSP_TILE];
  __shared__ T e[128];
  __shared__ T cfull[128];
  __shared__ T red[NT];
  __shared__ int abort_s;
  if (load_done(st)) return;
  const int nstage = sa.nstage;
  const int ntiles = (int)((n + NLSP_TILE - 1) / NLSP_TILE);
  const int t0 = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
  const int nt = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x) - t0;
  const unsigned tile_bytes = (unsigned)r * NLSP_TILE * (unsigned)sizeof(T);
  T* buf = reinterpret_cast<T*>(smem_raw);
  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int s = 0; s < nstage; ++s) tma::mbar_init(&bar[s], 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < nstage && s < nt; ++s) {
      tma::mbar_arrive_expect_tx(&bar[s], tile_bytes);
      tma::bulk_g2s(buf + (size_t)s * r * NLSP_TILE, P + (size_t)(t0 + s) * k * NLSP_TILE, tile_bytes, &bar[s]);
    }
  {
    // c: thread (col, sl) adds partials sl, sl + S, ... sixteen loads at a
    // time (all in flight together), then the S slices in order
    const int S = NT / r > 0 ? NT / r : 1;
    T part = T(0);
    if (threadIdx.x < S * r) {
      const int col = threadIdx.x % r, sl = threadIdx.x / r;
      for (int b0 = sl; b0 < nb; b0 += 16 * S) {
        T v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int b = b0 + u * S;
          v[u] = b < nb ? cpart[(int64_t)b * k + col] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) part += v[u];
      }
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int col = threadIdx.x; col < r; col += NT) {
      T c = T(0);
      for (int sl = 0; sl < S; ++sl) c += red[sl * r + col];
      cfull[col] = c;
    }
    __syncthreads();
    // e = A_c^-1 c: thread (row, g) adds the columns g, g + S, ... (r / S <=
    // 32 of them), sixteen loads at a time
    T v = T(0);
    if (threadIdx.x < S * r) {
      const int row = threadIdx.x % r, g = threadIdx.x / r;
      for (int c0 = g; c0 < r; c0 += 16 * S) {
        T a[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int col = c0 + u * S;
          a[u] = col < r ? Ainv[(int64_t)col * r + row] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int col = c0 + u * S;
          if (col < r) v += a[u] * cfull[col];
        }
      }
    }
    red[threadIdx.x] = v;
    __syncthreads();
    for (int row = threadIdx.x; row < r; row += NT) {
      T ev = T(0);
      for (int g = 0; g < S; ++g) ev += red[g * r + row];
      e[row] = ev;
    }
    __syncthreads();
  }
  const int w = threadIdx.x & (NLSP_TILE - 1), h = threadIdx.x >> 7;
  const int c0 = h * 32;
  for (int it = 0; it < nt; ++it) {
    // this tile's z is loaded before the wait for its P tile, so that the
    // read's latency runs under the copy
    const int64_t i = (int64_t)(t0 + it) * NLSP_TILE + w;
    const T zold = (h == 0 && i < n) ? z[i] : T(0);
    stream_wait(bar, it, nstage, &abort_s);
    const T* tile = buf + (size_t)(it % nstage) * r * NLSP_TILE;
    T a = T(0);
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < r) a += tile[(c0 + j) * NLSP_TILE + w] * e[c0 + j];
    zpart[it & 1][h][w] = a;
    __syncthreads();
    if (abort_s) {
      stream_drain(bar, it, nt, nstage);
      report_timeout(st, err);
      return;
    }
    if (threadIdx.x == 0 && it + nstage < nt) {
      const int s = it % nstage;
      tma::mbar_arrive_expect_tx(&bar[s], tile_bytes);
      tma::bulk_g2s(buf + (size_t)s * r * NLSP_TILE, P + (size_t)(t0 + it + nstage) * k * NLSP_TILE, tile_bytes,
                    &bar[s]);
    }
    if (h == 0) {
      T sum = zpart[it & 1][0][w];
#pragma unroll
      for (int q = 1; q < NCH; ++q) sum += zpart[it & 1][q][w];
      if (i < n) z[i] = zold + sum;
    }
  }
}

// ----------------------------------------------------------------------------
// post: final post-smoothing sweep(s), z_t stored in FP64, r^T z_t (and
// r^T z_{t-1}).  FUSE2: two sweeps in one pass, the first recomputed at the
// neighbours.  With st == nullptr (standalone apply) only z is written.
// ----------------------------------------------------------------------------
template <int KIND, typename T, bool FUSE2, bool INIT, bool SET_COND>
__global__ void __launch_bounds__(TPB) k_pcg_post(StencilView<T> A, T omega, const T* __restrict__ rT,
                                                  const double* __restrict__ r, const T* __restrict__ zin,
                                                  Pair<double> Z, PcgState* st, RedSlots red,
                                                  cudaGraphConditionalHandle cond) {
  __shared__ double sm[TPB];
  __shared__ int flag;
  if (load_done(st)) {
    if (SET_COND && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  const int t = load_iter(st);
  double* __restrict__ zout = Z.at(t);
  const double* __restrict__ zold = Z.at(t + 1);  // z_{t-1}
  const bool flex = st && !INIT && st->flexible;
  double s_rz = 0.0, s_ro = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    T zf;
    if (FUSE2) {
      auto z4at = [&](int64_t m, NodeCoord cm) -> T {
        const T az = stencil_apply<KIND>(A, m, cm, [&](int64_t mm) { return zin[mm]; });
        return zin[m] + omega * stencil_dinv<KIND>(A, m) * (rT[m] - az);
      };
      const T z4i = z4at(i, c);
      T az4 = stencil_diag<KIND>(A, i) * z4i;
      for_each_neighbour<KIND>(A, i, c, [&](int64_t m, NodeCoord cm, T a) { az4 += a * z4at(m, cm); });
      zf = z4i + omega * stencil_dinv<KIND>(A, i) * (rT[i] - az4);
    } else {
      const T az = stencil_apply<KIND>(A, i, c, [&](int64_t m) { return zin[m]; });
      zf = zin[i] + omega * stencil_dinv<KIND>(A, i) * (rT[i] - az);
    }
    const double zd = to_f64<T>(zf);
    zout[i] = zd;
    if (st) {
      const double ri = r[i];
      s_rz = fma(ri, zd, s_rz);
      if (flex) s_ro = fma(ri, zold[i], s_ro);
    }
  }
  if (!st) return;
  s_rz = block_sum_lean(s_rz, sm);
  if (flex) s_ro = block_sum_lean(s_ro, sm);
  if (threadIdx.x == 0) {
    red.part[2 * red.max_blocks + blockIdx.x] = s_rz;
    red.part[3 * red.max_blocks + blockIdx.x] = s_ro;
  }
  if (last_block_arrive(&red.counter[2], &flag)) {
    const double rz = sum_partials_lean(red.part + 2 * red.max_blocks, gridDim.x, sm);
    const double ro = flex ? sum_partials_lean(red.part + 3 * red.max_blocks, gridDim.x, sm) : 0.0;
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
      if (SET_COND) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
    }
  }
}

// ||b - A x||^2 after the solve (FP64).
template <int KIND>
__global__ void __launch_bounds__(TPB) k_true_residual(StencilView<double> A, const double* __restrict__ b,
                                                       const double* __restrict__ x, PcgState* st, RedSlots red) {
  __shared__ double sm[TPB];
  __shared__ int flag;
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const NodeCoord c = node_coord<KIND>(i, A.N);
    const double ri = b[i] - stencil_apply<KIND>(A, i, c, [&](int64_t m) { return x[m]; });
    s = fma(ri, ri, s);
  }
  s = block_sum_lean(s, sm);
  if (threadIdx.x == 0) red.part[blockIdx.x] = s;
  if (last_block_arrive(&red.counter[3], &flag)) {
    const double tr = sum_partials_lean(red.part, gridDim.x, sm);
    if (threadIdx.x == 0) st->true_rr = tr;
  }
}

template <typename T>
__global__ void k_convert(const double* __restrict__ a, T* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (T)a[i];
}

}  // namespace

// ============================================================================
// Persistent solver: the whole PCG solve of one right-hand side in one
// cooperative launch.  One CTA per SM owns a contiguous range of node tiles;
// the phases of an iteration are separated by a grid-wide barrier instead of
// kernel boundaries (a kernel boundary plus a last-block reduction costs
// several microseconds on GB300, a barrier about one).  Every CTA reduces the
// per-CTA partials of each dot product itself, in the same order, so all CTAs
// take the same control decisions.  Iteration t+1:
//   spmv     p = z + beta p, q = A p, p^T q            | barrier
//   pre      alpha; x += alpha p, r -= alpha q, rT, r^T r | barrier; stop test
//   [pre-sweeps stored, FP64 path / nu1 > 2]             | barrier each
//   restrict z2, rho = rT - A z2, c = P^T rho (TMA ring) | barrier
//   prolong  e_c = A_c^-1 sum(c); z += P e_c (TMA ring) | barrier
//   [post-sweeps stored]                                 | barrier each
//   post     last sweep(s), z in FP64, r^T z (r^T z_old)| barrier; beta
// ============================================================================
namespace {

constexpr int PT = 512;  // threads per CTA of the persistent solver

template <typename T>
struct PersistArgs {
  StencilView<double> A64;
  StencilView<T> AT;
  T omega;
  int nu1, nu2, flexible, maxit;
  double tol;
  const double* b;
  double* x;
  double* r;
  double* q;
  double* p0;
  double* p1;
  double* z0;
  double* z1;
  double* r1;  // second residual buffer (merged CG update + restriction)
  int merge;   // 1: the CG update runs inside the restriction phase (staged 2D, FP32)
  T* rT;    // residual in the preconditioner precision (== r for FP64)
  T* zw;    // preconditioner work vectors
  T* zw2;
  const T* P;
  int k, rr_;  // stored rank, active rank
  const T* Ainv;
  unsigned long long* xw;  // team exchange area (16-byte aligned, zero at launch): arrival counter (two
                           // words), partial slots [2][2][team rounded up to even] (FP64), rows c_rank of
                           // the coarse right-hand side [team][k]
  int* abort;              // set when a wait gave up
  unsigned* progress;  // launch-wide progress word (batched launches; null otherwise)
  PcgState* st;   // written by CTA 0 at the end
  StreamArgs sa;
  unsigned long long* ptimes;  // optional phase timers [PH_COUNT][2] (work, barrier wait) ns, CTA 0's view
};

enum { PH_SPMV = 0, PH_PRE, PH_SMOOTH, PH_RESTRICT, PH_PROLONG, PH_POST, PH_OTHER, PH_COUNT };
// Marks inside phases (time since the previous mark or barrier release,
// CTA 0 thread 0), stored after the phase timers.
enum {
  MK_SPMV_TOTALS = 0, MK_SPMV_NODES, MK_PRE_TOTALS, MK_PRE_NODES, MK_RES_RHO, MK_RES_RESIDENT, MK_RES_STREAM,
  MK_RES_REDUCE, MK_PRO_COARSE, MK_PRO_RESIDENT, MK_PRO_STREAM, MK_POST_NODES, MK_SPMV_ISSUE, MK_SPMV_FINISH,
  MK_RES_STAGE_A, MK_RES_STAGE_B, MK_POST_STAGE, MK_COUNT
};
constexpr int PTIMES_LEN = 2 * PH_COUNT + MK_COUNT;


// ---- team barriers ------------------------------------------------------------
// The CTAs of one instance (a team; all CTAs of the launch are co-resident)
// meet at barriers: thread 0 of each CTA releases the CTA's global writes
// (fence) and adds one to the team's arrival counter; barrier number gen is
// passed when the counter reaches gen * team.  Sums over the team go through
// per-rank partial slots written before a barrier and read after it; the slots
// are double buffered by the parity of the barrier number (a CTA rewrites a
// slot only after every rank has arrived at the next barrier, which each rank
// does only after reading the slot).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* ptr) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ptr) : "memory");
  return v;
}

// Bounded wait bookkeeping of one polling thread: gives up after 2 s (the
// count restarts while the launch-wide progress word moves: in batched
// launches a team member may be busy with earlier instances) or when the
// abort flag is set.  Returns false when the thread must stop waiting.
struct PollClock {
  unsigned long long t0;
  unsigned seen;
  bool started;
  __device__ __forceinline__ PollClock() : t0(0), seen(0), started(false) {}
  __device__ __forceinline__ bool keep_going(int* abort, const unsigned* progress) {
    if (*((volatile int*)abort)) return false;
    const unsigned long long t = tma::now_ns();
    if (!started) {
      started = true;
      t0 = t;
      seen = progress ? *((const volatile unsigned*)progress) : 0u;
      return true;
    }
    if (t - t0 <= tma::WAIT_LIMIT_NS) return true;
    if (progress) {
      const unsigned now_p = *((const volatile unsigned*)progress);
      if (now_p != seen) {
        seen = now_p;
        t0 = t;
        return true;
      }
    }
    atomicExch(abort, 1);
    return false;
  }
};

constexpr int XMAX_RANKS = 160;  // team size limit (the team sums read 5 ranks per lane)

// Barrier number `gen` of the team; false in every thread when the wait gave
// up (abort flag or time limit).
__device__ __forceinline__ bool team_barrier(unsigned* ctr, int* abort, const unsigned* progress, unsigned gen,
                                             int team, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    int ok = 1;
    PollClock clk;
    const unsigned target = gen * (unsigned)team;
    while (ld_acquire_u32(ctr) < target)
      if (!clk.keep_going(abort, progress)) {
        ok = 0;
        break;
      }
    if (ok && *((volatile int*)abort)) ok = 0;
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

constexpr int XBAR = 7;  // mbarrier of the partial-slot copies (the P ring uses the first ones)

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Sums the first nv of NV values over the CTA; result valid in thread 0.
// Per value every thread stores it and warp 0 adds the PT / 32 values of its
// lane column, then its 32 lane sums by a shuffle tree: one FP64 add per
// value, instead of a shuffle tree in every warp (GB300 executes FP64 at 1/64
// of the FP32 rate, charged per warp instruction).  Ends after a
// __syncthreads that every thread has passed with its values stored.
template <int NV>
__device__ __forceinline__ void cta_sums(const double (&val)[NV], double* sm_d, double (&out)[NV], int nv) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int v = 0; v < nv; ++v) {
    if (v > 0) __syncthreads();  // warp 0 has read the previous value
    sm_d[threadIdx.x] = val[v];
    __syncthreads();
    if (warp == 0) {
      double s = sm_d[lane];
#pragma unroll
      for (int w = 1; w < PT / 32; ++w) s += sm_d[w * 32 + lane];
      out[v] = warp_sum(s);
    }
  }
}

// Streams the CTA's P tiles through the ring: copy number j (running over the
// whole kernel) uses stage j % nstage with parity (j / nstage) & 1.
template <typename T>
__device__ __forceinline__ void ring_issue(uint64_t* bar, T* buf, const T* P, int k, int r, int nstage, unsigned j,
                                           int tile) {
  const unsigned bytes = (unsigned)r * NLSP_TILE * (unsigned)sizeof(T);
  const int s = (int)(j % (unsigned)nstage);
  // the stage was last read (or used as scratch) through the generic proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tma::mbar_arrive_expect_tx(&bar[s], bytes);
  tma::bulk_g2s(buf + (size_t)s * r * NLSP_TILE, P + (size_t)tile * k * NLSP_TILE, bytes, &bar[s]);
}

__device__ __forceinline__ bool ring_wait(uint64_t* bar, int nstage, unsigned j) {
  return tma::mbar_wait(&bar[j % (unsigned)nstage], (j / (unsigned)nstage) & 1u);
}

// Arguments of the restriction when it also performs the CG update
// (x += alpha p, r_next = r_cur - alpha q): its own nodes' results go to
// global memory, the updated residual of the own nodes and two stencil hops
// around them to shared memory for the pre-sweeps.
struct MergeArgs {
  double alpha;
  const double* rc;   // r_cur (read on own and halo nodes)
  double* rn;         // r_next (own nodes)
  const double* pd;   // p (own nodes)
  double s_rr;        // this thread's part of r_next^T r_next
};

// Node loop over [lo, hi) with stride PT, U nodes per thread at a time:
// f(m) (loads and arithmetic only) for all U nodes first, then store(m, v)
// for each, so the loads of the U nodes are in flight together (a store
// through a generic pointer would otherwise keep the next node's loads
// behind it).  store() runs in node order.
template <int U, typename F, typename S>
__device__ __forceinline__ void node_batches(int lo, int hi, F f, S store) {
  using V = decltype(f(lo));
  for (int m0 = lo + (int)threadIdx.x; m0 < hi; m0 += U * PT) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m0 + u * PT;
      if (m < hi) v[u] = f(m);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m0 + u * PT;
      if (m < hi) store(m, v[u]);
    }
  }
}

template <typename T>
struct RhoZ {
  T rho, z;
};

struct PostVals {
  double zd, ri, zo;
};

// CPG = columns of P per warp group (4 groups of 4 warps; r_pad = 4 CPG).
// The CTA's first n_tm tiles of P live in tensor memory (FP32 path), the next
// n_sm in shared memory, both loaded once per solve; only the rest is
// streamed through the TMA ring in every restriction and prolongation.
template <int KIND, typename T, int CPG>
__device__ __forceinline__ bool solve_instance(const PersistArgs<T>& a, const int cta, const int G,
                                               const unsigned tbase_all, uint64_t* mbar,
                                               unsigned char* smem_raw) {
  __shared__ double sm_d[PT];
  __shared__ T red_t[PT];
  __shared__ T sacc[PT / 32][32];
  __shared__ T cfull[128];
  __shared__ T e_s[128];
  __shared__ T zpart[2][4][NLSP_TILE];
  __shared__ double bc[4];  // totals, then scalars derived from them by one thread
  __shared__ __align__(16) double tot_s[2][XMAX_RANKS];  // copies of the team's partial slots
  __shared__ int ok_s, abort_s;

  constexpr bool FP32 = sizeof(T) == 4;
  constexpr int RPAD = 4 * CPG;
  const int tid = threadIdx.x;
  const int n = (int)a.AT.n, N = a.AT.N;
  const int ntiles = (n + NLSP_TILE - 1) / NLSP_TILE;
  const int t0 = (int)((int64_t)ntiles * cta / G);
  const int nt = (int)((int64_t)ntiles * (cta + 1) / G) - t0;
  const int i0 = t0 * NLSP_TILE, i1 = min((t0 + nt) * NLSP_TILE, n);
  const int nstage = a.sa.nstage, r = a.rr_, k = a.k;
  const int ntm = FP32 ? min(nt, a.sa.n_tm) : 0;    // tiles in tensor memory
  const int nsm = min(nt - ntm, a.sa.n_sm);         // tiles resident in shared memory
  const int nst = nt - ntm - nsm;                   // tiles streamed per phase
  const int tst = t0 + ntm + nsm;                   // first streamed tile
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* res = buf + (size_t)nstage * r * NLSP_TILE;
  T* rho_s = res + (size_t)a.sa.n_sm * r * NLSP_TILE;
  const T omega = a.omega;
  const int warp = tid >> 5, lane = tid & 31, q = warp & 3, g = warp >> 2, nd = 32 * q + lane;
  // staged smoothing (2D stencils, FP32): node ranges one and two stencil
  // hops (N + 1 nodes, diagonals included) around the own nodes, kept in the
  // ring buffer when they fit
  const int hop = N + 1;
  const int e1lo = max(0, i0 - hop), e1hi = min(n, i1 + hop);
  const int e2lo = max(0, i0 - 2 * hop), e2hi = min(n, i1 + 2 * hop);
  const int ring_elems = nstage * r * NLSP_TILE;
  const bool stage_pre = FP32 && (KIND == ST_5PT || KIND == ST_9PT) && i1 > i0 && (e2hi - e2lo) + (e1hi - e1lo) <= ring_elems;
  const bool stage_post = FP32 && (KIND == ST_5PT || KIND == ST_9PT) && i1 > i0 && (e1hi - e1lo) <= ring_elems;
  unsigned gen = 0, jc = 0;
  bool ok = true;
  double tol2bn = 0.0;

  // the ring's barriers are re-initialised for every instance (all copies of
  // the previous instance have been consumed)
  __syncthreads();
  if (tid == 0) {
    abort_s = 0;
    for (int s = 0; s < nstage; ++s) {
      tma::mbar_inval(&mbar[s]);
      tma::mbar_init(&mbar[s], 1);
    }
    tma::mbar_inval(&mbar[XBAR]);
    tma::mbar_init(&mbar[XBAR], 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  const unsigned tlane = (unsigned)(32 * q) << 16;
  const unsigned tbase = ntm > 0 ? tbase_all : 0u;
  // one-time loads of the resident tiles
  for (int ti = 0; ti < ntm; ++ti) {
    float v[CPG];
    const T* src = a.P + ((size_t)(t0 + ti) * k) * NLSP_TILE + nd;
#pragma unroll
    for (int j = 0; j < CPG; ++j) {
      const int col = g * CPG + j;
      v[j] = col < r ? (float)src[(size_t)col * NLSP_TILE] : 0.0f;
    }
    if (FP32) tmem::Io<CPG>::st(tbase + tlane + (unsigned)(ti * RPAD + g * CPG), v);
  }
  for (int ts = 0; ts < nsm; ++ts) {
    const T* src = a.P + ((size_t)(t0 + ntm + ts) * k) * NLSP_TILE;
    T* dst = res + (size_t)ts * r * NLSP_TILE;
    for (int e = tid; e < r * NLSP_TILE; e += PT) dst[e] = src[e];
  }
  __syncthreads();

  const bool timed0 = a.ptimes && cta == 0 && tid == 0;
  unsigned long long t_last = timed0 ? tma::now_ns() : 0ull, t_mark = t_last;
  // exchange area: arrival counter, partial slots [2][2][gs], c_rank rows
  const int gs = (G + 1) & ~1;  // slot length: whole 16-byte units for the bulk copies
  unsigned* const ctr = reinterpret_cast<unsigned*>(a.xw);
  double* const slots = reinterpret_cast<double*>(a.xw + 2);
  T* const cpart = reinterpret_cast<T*>(a.xw + 2 + (size_t)4 * gs);  // [team][k]
  unsigned tpar = 0;  // copies of partial slots so far (mbarrier phase)
  auto phase_time = [&](int phase, unsigned long long t_arr) {
    if (timed0) {
      const unsigned long long t_rel = tma::now_ns();
      a.ptimes[2 * phase] += t_arr - t_last;
      a.ptimes[2 * phase + 1] += t_rel - t_arr;
      t_last = t_mark = t_rel;
    }
  };
  // slot of sum v for barrier number g
  auto slot_of = [&](unsigned g, int v) { return slots + ((size_t)(g & 1u) * 2 + v) * gs; };
  // the CTA's partials of the sums carried by the next barrier
  auto put = [&](int nv, double v0, double v1) {
    const double in[2] = {v0, v1};
    double s[2] = {0.0, 0.0};
    cta_sums<2>(in, sm_d, s, nv);
    if (tid == 0) {
      slot_of(gen + 1, 0)[cta] = s[0];
      if (nv > 1) slot_of(gen + 1, 1)[cta] = s[1];
    }
  };
  auto bar = [&](int phase) -> bool {
    const unsigned long long t_arr = timed0 ? tma::now_ns() : 0ull;
    ++gen;
    ok = ok && team_barrier(ctr, a.abort, a.progress, gen, G, &ok_s);
    phase_time(phase, t_arr);
    return ok;
  };
  // Totals of the nv sums carried by the last barrier: tot_issue starts bulk
  // copies of the slots into shared memory (no registers held while other
  // work runs), tot_finish adds them in rank order (the same value in every
  // CTA).  False when the copy wait gave up.
  auto tot_issue = [&](int nv) {
    if (tid == 0) {
      fence_proxy_async_global();  // the slots were acquired through the generic proxy
      const unsigned bytes = (unsigned)(gs * sizeof(double));
      tma::mbar_arrive_expect_tx(&mbar[XBAR], bytes * nv);
      for (int v = 0; v < nv; ++v) tma::bulk_g2s(tot_s[v], slot_of(gen, v), bytes, &mbar[XBAR]);
    }
  };
  // derive(bc) runs in thread 0 once the totals are in bc[0 .. nv): scalar
  // FP64 work (alpha, beta: divisions) done once instead of by every thread,
  // since GB300 executes FP64 at 1/64 of the FP32 rate.
  auto tot_finish_d = [&](int nv, double* out, auto derive) -> bool {
    if (tid < 32) {
      const bool got = tma::mbar_wait(&mbar[XBAR], tpar & 1u);
      if (!got && tid == 0) {
        atomicExch(a.abort, 1);
        abort_s = 1;
      }
      for (int v = 0; v < nv; ++v) {
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < XMAX_RANKS / 32; ++u) {
          const int c = tid + 32 * u;
          if (c < G) s += tot_s[v][c];
        }
        s = warp_sum(s);
        if (tid == 0) bc[v] = s;
      }
      if (tid == 0) derive(bc);
    }
    ++tpar;
    __syncthreads();
    for (int v = 0; v < nv; ++v) out[v] = bc[v];
    const bool good = abort_s == 0;
    __syncthreads();
    if (!good) ok = false;
    return good;
  };
  auto tot_finish = [&](int nv, double* out) -> bool { return tot_finish_d(nv, out, [](double*) {}); };
  auto total1 = [&]() -> double {
    double o[1] = {0.0};
    tot_issue(1);
    tot_finish(1, o);
    return o[0];
  };
  auto mark = [&](int id) {
    if (timed0) {
      const unsigned long long t = tma::now_ns();
      a.ptimes[2 * PH_COUNT + id] += t - t_mark;
      t_mark = t;
    }
  };

  // ---- the two phases that read P ----------------------------------------
  // restrict: rho for the own nodes (z recomputed from rT when zm > 0), then
  // c_cta = P^T rho over the own tiles -> row cta of cpart.  Thread (g, q, lane)
  // accumulates columns [g CPG, g CPG + CPG) for node 32 q + lane of each tile.
  auto restrict_phase = [&](int zm, const T* zin, MergeArgs* mg) {
    const bool staged = zm > 0 && stage_pre;
    if (!staged)
      for (int s = 0; s < nstage && s < nst; ++s)
        if (tid == 0) ring_issue(mbar, buf, a.P, k, r, nstage, jc + s, tst + s);
    if (staged) {
      // z1 = w D^-1 rT on the own nodes and two grid rows around them, then
      // z2 = z1 + w D^-1 (rT - A z1) on one row around them, both in the ring
      // buffer; rho = rT - A z2 on the own nodes.  Same arithmetic as
      // presmooth_at, without recomputing z1 and z2 at every neighbour.
      T* rts = buf;                                   // merged: updated residual (E2)
      T* z1s = buf + (mg ? (e2hi - e2lo) : 0);
      T* z2s = z1s + (e2hi - e2lo);
      if (mg) {
        node_batches<4>(
            e2lo, e2hi, [&](int m) { return fma(-mg->alpha, __ldcg(a.q + m), __ldcg(mg->rc + m)); },
            [&](int m, double v) {
              const T vt = from_f64<T>(v);
              rts[m - e2lo] = vt;
              if (m >= i0 && m < i1) {
                mg->rn[m] = v;
                a.rT[m] = vt;
                a.x[m] = fma(mg->alpha, mg->pd[m], a.x[m]);
                mg->s_rr = fma(v, v, mg->s_rr);
              }
            });
        __syncthreads();
      }
      auto rt = [&](int m) -> T { return mg ? rts[m - e2lo] : a.rT[m]; };
      node_batches<4>(
          e2lo, e2hi, [&](int m) { return omega * stencil_dinv<KIND>(a.AT, m) * rt(m); },
          [&](int m, T v) { z1s[m - e2lo] = v; });
      __syncthreads();
      mark(MK_RES_STAGE_A);
      if (zm == 2) {
        node_batches<1>(
            e1lo, e1hi,
            [&](int m) {
              const T az = stencil_apply<KIND>(a.AT, m, node_coord<KIND>(m, a.AT.N),
                                               [&](int64_t mm) { return z1s[mm - e2lo]; });
              return z1s[m - e2lo] + omega * stencil_dinv<KIND>(a.AT, m) * (rt(m) - az);
            },
            [&](int m, T v) { z2s[m - e1lo] = v; });
        __syncthreads();
        mark(MK_RES_STAGE_B);
      }
      const T* zs = zm == 2 ? z2s : z1s;
      const int zlo = zm == 2 ? e1lo : e2lo;
      node_batches<1>(
          i0, i1,
          [&](int i) {
            const T az = stencil_apply<KIND>(a.AT, i, node_coord<KIND>(i, a.AT.N),
                                             [&](int64_t mm) { return zs[mm - zlo]; });
            return RhoZ<T>{rt(i) - az, zs[i - zlo]};
          },
          [&](int i, RhoZ<T> v) {
            rho_s[i - i0] = v.rho;
            a.zw[i] = v.z;
          });
      for (int e = (i1 - i0) + tid; e < nt * NLSP_TILE; e += PT) rho_s[e] = T(0);  // ragged last tile
      __syncthreads();  // the ring buffer is free again
      for (int s = 0; s < nstage && s < nst; ++s)
        if (tid == 0) ring_issue(mbar, buf, a.P, k, r, nstage, jc + s, tst + s);
    }
    for (int e = tid; e < (staged ? 0 : nt * NLSP_TILE); e += PT) {
      const int i = i0 + e;
      T rho = T(0);
      if (i < n) {
        const NodeCoord c = node_coord<KIND>(i, a.AT.N);
        if (zm == 0) {
          rho = a.rT[i] - stencil_apply<KIND>(a.AT, i, c, [&](int64_t m) { return zin[m]; });
        } else {
          T zi, az;
          if (zm == 1) {
            zi = presmooth_at<KIND, T, 1>(a.AT, omega, a.rT, i, c);
            az = stencil_diag<KIND>(a.AT, i) * zi;
            for_each_neighbour<KIND>(a.AT, i, c, [&](int64_t m, NodeCoord cm, T w) {
              az += w * presmooth_at<KIND, T, 1>(a.AT, omega, a.rT, m, cm);
            });
          } else {
            zi = presmooth_at<KIND, T, 2>(a.AT, omega, a.rT, i, c);
            az = stencil_diag<KIND>(a.AT, i) * zi;
            for_each_neighbour<KIND>(a.AT, i, c, [&](int64_t m, NodeCoord cm, T w) {
              az += w * presmooth_at<KIND, T, 2>(a.AT, omega, a.rT, m, cm);
            });
          }
          rho = a.rT[i] - az;
          a.zw[i] = zi;
        }
      }
      rho_s[e] = rho;
    }
    __syncthreads();
    mark(MK_RES_RHO);
    T acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = T(0);
    for (int ti = 0; ti < ntm; ++ti) {
      float v[CPG];
      tmem::Io<CPG>::ld(tbase + tlane + (unsigned)(ti * RPAD + g * CPG), v);
      const T rho = rho_s[ti * NLSP_TILE + nd];
#pragma unroll
      for (int j = 0; j < CPG; ++j) acc[j] += rho * (T)v[j];
    }
    for (int ts = 0; ts < nsm; ++ts) {
      const T* tile = res + (size_t)ts * r * NLSP_TILE;
      const T rho = rho_s[(ntm + ts) * NLSP_TILE + nd];
#pragma unroll
      for (int j = 0; j < CPG; ++j) {
        const int col = g * CPG + j;
        if (col < r) acc[j] += rho * tile[col * NLSP_TILE + nd];
      }
    }
    mark(MK_RES_RESIDENT);
    for (int it = 0; it < nst; ++it) {
      if (!ring_wait(mbar, nstage, jc + it)) abort_s = 1;
      const T* tile = buf + (size_t)((jc + it) % (unsigned)nstage) * r * NLSP_TILE;
      const T rho = rho_s[(ntm + nsm + it) * NLSP_TILE + nd];
#pragma unroll
      for (int j = 0; j < CPG; ++j) {
        const int col = g * CPG + j;
        if (col < r) acc[j] += rho * tile[col * NLSP_TILE + nd];
      }
      __syncthreads();
      if (abort_s) {
        stream_drain(mbar, (int)(jc + it), (int)(jc + nst), nstage);
        if (tid == 0) atomicExch(a.abort, 1);
        break;
      }
      if (tid == 0 && it + nstage < nst) ring_issue(mbar, buf, a.P, k, r, nstage, jc + it + nstage, tst + it + nstage);
    }
    jc += nst;
    mark(MK_RES_STREAM);
    sacc[warp][lane] = warp_reduce_scatter32(acc, lane);  // column g CPG + lane (lane < CPG)
    __syncthreads();
    for (int col = tid; col < r; col += PT) {
      const int gg = col / CPG, j = col % CPG;
      T s = T(0);
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) s += sacc[gg * 4 + qq][j];
      cpart[(size_t)cta * k + col] = s;
    }
    mark(MK_RES_REDUCE);
  };

  // prolong: e_c = A_c^-1 (sum of the CTAs' c), z += P e_c on the own tiles.
  // Resident tiles: warp group g takes tiles g, g + 4, ... and each thread
  // its node's whole row; streamed tiles: the (g, q, lane) split with a
  // shared-memory combine.
  auto prolong_phase = [&](T* z) {
    for (int s = 0; s < nstage && s < nst; ++s)
      if (tid == 0) ring_issue(mbar, buf, a.P, k, r, nstage, jc + s, tst + s);
    {
      // sum of the team's c_rank: thread (col, sl) adds ranks sl, sl + S, ...
      // in order, eight loads in flight
      const int S = PT / r > 0 ? PT / r : 1;
      T part = T(0);
      if (tid < S * r) {
        const int col = tid % r, sl = tid / r;
#pragma unroll 8
        for (int c = sl; c < G; c += S) part += __ldcg(cpart + (size_t)c * k + col);
      }
      red_t[tid] = part;
      __syncthreads();
      for (int col = tid; col < r; col += PT) {
        T s = T(0);
        for (int sl = 0; sl < S; ++sl) s += red_t[sl * r + col];
        cfull[col] = s;
      }
      __syncthreads();
      {  // e_c = A_c^-1 c: PT / RPAD column groups per row, then a combine
        constexpr int CG = PT / RPAD;
        const int row = tid % RPAD, cg = tid / RPAD;
        T s = T(0);
        if (row < r) {
#pragma unroll 4
          for (int col = cg; col < r; col += CG) s += a.Ainv[(int64_t)col * r + row] * cfull[col];
        }
        red_t[tid] = s;
        __syncthreads();
        if (tid < RPAD) {
          T e = T(0);
#pragma unroll
          for (int gg = 0; gg < CG; ++gg) e += red_t[gg * RPAD + tid];
          e_s[tid] = e;  // zero beyond r
        }
      }
      __syncthreads();
      mark(MK_PRO_COARSE);
    }
    for (int tl = g; tl < ntm + nsm; tl += 4) {
      T s = T(0);
      if (tl < ntm) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          float v[CPG];
          tmem::Io<CPG>::ld(tbase + tlane + (unsigned)(tl * RPAD + cc * CPG), v);
#pragma unroll
          for (int j = 0; j < CPG; ++j) s += (T)v[j] * e_s[cc * CPG + j];
        }
      } else {
        const T* tile = res + (size_t)(tl - ntm) * r * NLSP_TILE;
        for (int col = 0; col < r; ++col) s += tile[col * NLSP_TILE + nd] * e_s[col];
      }
      const int i = (t0 + tl) * NLSP_TILE + nd;
      if (i < n) z[i] += s;
    }
    mark(MK_PRO_RESIDENT);
    for (int it = 0; it < nst; ++it) {
      if (!ring_wait(mbar, nstage, jc + it)) abort_s = 1;
      const T* tile = buf + (size_t)((jc + it) % (unsigned)nstage) * r * NLSP_TILE;
      T s = T(0);
#pragma unroll
      for (int j = 0; j < CPG; ++j) {
        const int col = g * CPG + j;
        if (col < r) s += tile[col * NLSP_TILE + nd] * e_s[col];
      }
      zpart[it & 1][g][nd] = s;
      __syncthreads();
      if (abort_s) {
        stream_drain(mbar, (int)(jc + it), (int)(jc + nst), nstage);
        if (tid == 0) atomicExch(a.abort, 1);
        break;
      }
      if (tid == 0 && it + nstage < nst) ring_issue(mbar, buf, a.P, k, r, nstage, jc + it + nstage, tst + it + nstage);
      if (g == 0) {
        const T sum = zpart[it & 1][0][nd] + zpart[it & 1][1][nd] + zpart[it & 1][2][nd] + zpart[it & 1][3][nd];
        const int i = (tst + it) * NLSP_TILE + nd;
        if (i < n) z[i] += sum;
      }
    }
    jc += nst;
    mark(MK_PRO_STREAM);
  };

  auto sweep_phase = [&](const T* zin, T* zout) {
    for (int i = i0 + tid; i < i1; i += PT) {
      const NodeCoord c = node_coord<KIND>(i, a.AT.N);
      const T az = stencil_apply<KIND>(a.AT, i, c, [&](int64_t m) { return zin[m]; });
      zout[i] = zin[i] + omega * stencil_dinv<KIND>(a.AT, i) * (a.rT[i] - az);
    }
  };

  // The preconditioner on the current residual: z (FP64) -> zout64, with
  // r^T z and r^T zold64 accumulated into the RED_RZ / RED_RO partials.
  // The preconditioner on the current residual: z (FP64) -> zout64, with the
  // partials of r^T z (and r^T zold64) carried by its last barrier.  When
  // rr_out is given, the team's r^T r from the barrier before is added up
  // while the restriction runs; the application stops after the restriction
  // (returns 2) when that shows convergence or a non-finite residual.
  // Returns 0 when a wait gave up, 1 when done.
  const double* rpost = a.r;  // the residual the post-smoothing's r^T z uses
  // With mg (merged path) the restriction also performs the CG update and
  // its barrier carries r^T r, added up during the prolongation.
  auto apply = [&](double* zout64, const double* zold64, bool flex, double* rr_out, MergeArgs* mg) -> int {
    if (rr_out && !mg) tot_issue(1);
    T* cur = a.zw;
    T* oth = a.zw2;
    const bool fused_pre = FP32 && a.nu1 <= 2;
    if (!fused_pre) {
      for (int i = i0 + tid; i < i1; i += PT) {
        const NodeCoord c = node_coord<KIND>(i, a.AT.N);
        cur[i] = a.nu1 == 1 ? presmooth_at<KIND, T, 1>(a.AT, omega, a.rT, i, c)
                            : presmooth_at<KIND, T, 2>(a.AT, omega, a.rT, i, c);
      }
      if (!bar(PH_SMOOTH)) return 0;
      for (int sw = 2; sw < a.nu1; ++sw) {
        sweep_phase(cur, oth);
        T* tmp = cur; cur = oth; oth = tmp;
        if (!bar(PH_SMOOTH)) return 0;
      }
    }
    restrict_phase(fused_pre ? a.nu1 : 0, cur, mg);
    if (rr_out && !mg) {
      double o[1] = {0.0};
      if (!tot_finish(1, o)) return 0;
      *rr_out = o[0];
      if (!isfinite(o[0]) || o[0] <= tol2bn) return 2;
    }
    if (mg) put(1, mg->s_rr, 0.0);
    if (!bar(PH_RESTRICT)) return 0;
    if (mg) tot_issue(1);
    prolong_phase(cur);
    if (mg) {
      double o[1] = {0.0};
      if (!tot_finish(1, o)) return 0;
      *rr_out = o[0];
      if (!isfinite(o[0]) || o[0] <= tol2bn) return 2;
    }
    if (!bar(PH_PROLONG)) return 0;
    const int nfinal = (FP32 && a.nu2 >= 2) ? 2 : 1;
    for (int sw = nfinal; sw < a.nu2; ++sw) {
      sweep_phase(cur, oth);
      T* tmp = cur; cur = oth; oth = tmp;
      if (!bar(PH_SMOOTH)) return 0;
    }
    double s_rz = 0.0, s_ro = 0.0;
    const bool staged = nfinal == 2 && stage_post;
    if (staged) {
      // first post-sweep on the own nodes and one grid row around them into
      // the (idle) ring buffer, the second one below reads it
      T* z3s = buf;
      node_batches<1>(
          e1lo, e1hi,
          [&](int m) {
            const T az =
                stencil_apply<KIND>(a.AT, m, node_coord<KIND>(m, a.AT.N), [&](int64_t mm) { return cur[mm]; });
            return cur[m] + omega * stencil_dinv<KIND>(a.AT, m) * (a.rT[m] - az);
          },
          [&](int m, T v) { z3s[m - e1lo] = v; });
      __syncthreads();
      mark(MK_POST_STAGE);
      const T* z3c = buf;
      node_batches<1>(
          i0, i1,
          [&](int i) {
            const T az4 = stencil_apply<KIND>(a.AT, i, node_coord<KIND>(i, a.AT.N),
                                              [&](int64_t mm) { return z3c[mm - e1lo]; });
            const T zf = z3c[i - e1lo] + omega * stencil_dinv<KIND>(a.AT, i) * (a.rT[i] - az4);
            return PostVals{to_f64<T>(zf), rpost[i], flex ? zold64[i] : 0.0};
          },
          [&](int i, PostVals v) {
            zout64[i] = v.zd;
            s_rz = fma(v.ri, v.zd, s_rz);
            if (flex) s_ro = fma(v.ri, v.zo, s_ro);
          });
    }
    for (int i = i0 + tid; i < (staged ? 0 : i1); i += PT) {
      const NodeCoord c = node_coord<KIND>(i, a.AT.N);
      T zf;
      if (nfinal == 2) {
        auto z4at = [&](int64_t m, NodeCoord cm) -> T {
          const T az = stencil_apply<KIND>(a.AT, m, cm, [&](int64_t mm) { return cur[mm]; });
          return cur[m] + omega * stencil_dinv<KIND>(a.AT, m) * (a.rT[m] - az);
        };
        const T z4i = z4at(i, c);
        T az4 = stencil_diag<KIND>(a.AT, i) * z4i;
        for_each_neighbour<KIND>(a.AT, i, c, [&](int64_t m, NodeCoord cm, T w) { az4 += w * z4at(m, cm); });
        zf = z4i + omega * stencil_dinv<KIND>(a.AT, i) * (a.rT[i] - az4);
      } else {
        const T az = stencil_apply<KIND>(a.AT, i, c, [&](int64_t m) { return cur[m]; });
        zf = cur[i] + omega * stencil_dinv<KIND>(a.AT, i) * (a.rT[i] - az);
      }
      const double zd = to_f64<T>(zf);
      const double ri = rpost[i];
      zout64[i] = zd;
      s_rz = fma(ri, zd, s_rz);
      if (flex) s_ro = fma(ri, zold64[i], s_ro);
    }
    mark(MK_POST_NODES);
    put(2, s_rz, s_ro);
    return bar(PH_POST) ? 1 : 0;
  };

  // ---- start: r = b, x = 0, p = 0 ---------------------------------------
  int status = (int)NLSP_OK, iter = 0;
  double bb = 0.0, rz = 0.0, rr = 0.0, beta = 0.0;
  {
    double s = 0.0;
    for (int i = i0 + tid; i < i1; i += PT) {
      const double bi = a.b[i];
      a.r[i] = bi;
      if (FP32) a.rT[i] = (T)bi;
      a.x[i] = 0.0;
      a.p0[i] = 0.0;
      a.p1[i] = 0.0;
      a.q[i] = 0.0;  // q = A z + beta q_old starts from q_old = 0
      s = fma(bi, bi, s);
    }
    put(1, s, 0.0);
  }
  bool done = false;
  if (bar(PH_OTHER)) {
    bb = total1();
    tol2bn = a.tol * a.tol * bb;
    rr = bb;
    if (bb == 0.0) done = true;
    else if (!isfinite(bb)) { status = (int)NLSP_ERR_BREAKDOWN; done = true; }
  } else {
    done = true;
  }
  // initial preconditioner application z_0 = B r_0
  if (!done && apply(a.z0, a.z1, false, nullptr, nullptr) != 1) done = true;
  // ---- iterations --------------------------------------------------------
  while (!done && ok) {
    const int t = iter;
    if (a.progress && cta == 0 && tid == 0) atomicAdd(a.progress, 1u);
    const double* zc = (t & 1) ? a.z1 : a.z0;
    const double* pin = (t & 1) ? a.p1 : a.p0;
    double* pout = (t & 1) ? a.p0 : a.p1;
    {  // spmv in the form q = A z + beta q_old (= A p for p = z + beta p_old):
       // A z on the own nodes needs no beta, so it is computed while the
       // team's r^T z (and r^T z_old) are added up; then p, q and p^T q.
      tot_issue(2);
      double az[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int iu = i0 + tid + u * PT;
        az[u] = iu < i1 ? stencil_apply<KIND>(a.A64, iu, node_coord<KIND>(iu, a.A64.N),
                                              [&](int64_t m) { return __ldcg(zc + m); })
                        : 0.0;
      }
      mark(MK_SPMV_ISSUE);
      double tot[2] = {0.0, 0.0};
      if (!tot_finish_d(2, tot, [&](double* b) { b[2] = t > 0 ? (b[0] - (a.flexible ? b[1] : 0.0)) / rz : 0.0; }))
        break;
      mark(MK_SPMV_FINISH);
      const double rzn = tot[0];
      if (!(rzn > 0.0) || !isfinite(rzn)) { status = (int)NLSP_ERR_BREAKDOWN; break; }
      if (t > 0) {
        beta = bc[2];
        if (iter >= a.maxit) { status = (int)NLSP_NOT_CONVERGED; break; }
      }
      rz = rzn;
      mark(MK_SPMV_TOTALS);
      double s = 0.0;
      auto update = [&](int i, double azi) {
        const double pi = fma(beta, __ldcg(pin + i), __ldcg(zc + i));
        const double qi = fma(beta, a.q[i], azi);
        pout[i] = pi;
        a.q[i] = qi;
        s = fma(pi, qi, s);
      };
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int iu = i0 + tid + u * PT;
        if (iu < i1) update(iu, az[u]);
      }
      for (int i = i0 + tid + 4 * PT; i < i1; i += PT)
        update(i, stencil_apply<KIND>(a.A64, i, node_coord<KIND>(i, a.A64.N), [&](int64_t m) { return __ldcg(zc + m); }));
      mark(MK_SPMV_NODES);
      put(1, s, 0.0);
      if (!bar(PH_SPMV)) break;
    }
    iter = t + 1;
    if (a.merge) {
      // the CG update runs inside the restriction; r alternates between
      // two buffers so that halo nodes read the previous residual
      tot_issue(1);
      double tot[1] = {0.0};
      if (!tot_finish_d(1, tot, [&](double* b) { b[2] = rz / b[0]; })) break;
      const double pq = tot[0];
      if (!(pq > 0.0) || !isfinite(pq)) { status = (int)NLSP_ERR_BREAKDOWN; break; }
      MergeArgs mg;
      mg.alpha = bc[2];
      mg.rc = (t & 1) ? a.r1 : a.r;
      mg.rn = (t & 1) ? a.r : a.r1;
      mg.pd = pout;
      mg.s_rr = 0.0;
      mark(MK_PRE_TOTALS);
      rpost = mg.rn;
      double* zn = (iter & 1) ? a.z1 : a.z0;
      const double* zo = (iter & 1) ? a.z0 : a.z1;
      const int st_apply = apply(zn, zo, a.flexible != 0, &rr, &mg);
      if (st_apply == 0) break;
      if (st_apply == 2) {
        if (!isfinite(rr)) status = (int)NLSP_ERR_BREAKDOWN;
        break;
      }
      continue;
    }
    {  // pre: x, r update; the own nodes' data is loaded while p^T q is added up
      tot_issue(1);
      double pv[4], xv[4], qv[4], rv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int iu = i0 + tid + u * PT;
        const bool in = iu < i1;
        pv[u] = in ? pout[iu] : 0.0;
        xv[u] = in ? a.x[iu] : 0.0;
        qv[u] = in ? a.q[iu] : 0.0;
        rv[u] = in ? a.r[iu] : 0.0;
      }
      double tot[1] = {0.0};
      if (!tot_finish_d(1, tot, [&](double* b) { b[2] = rz / b[0]; })) break;
      const double pq = tot[0];
      if (!(pq > 0.0) || !isfinite(pq)) { status = (int)NLSP_ERR_BREAKDOWN; break; }
      const double alpha = bc[2];
      mark(MK_PRE_TOTALS);
      double s = 0.0;
      auto update = [&](int i, double pi, double xi, double qi, double ri) {
        const double rn = fma(-alpha, qi, ri);
        a.x[i] = fma(alpha, pi, xi);
        a.r[i] = rn;
        if (FP32) a.rT[i] = from_f64<T>(rn);
        s = fma(rn, rn, s);
      };
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int iu = i0 + tid + u * PT;
        if (iu < i1) update(iu, pv[u], xv[u], qv[u], rv[u]);
      }
      for (int i = i0 + tid + 4 * PT; i < i1; i += PT) update(i, pout[i], a.x[i], a.q[i], a.r[i]);
      mark(MK_PRE_NODES);
      put(1, s, 0.0);
      if (!bar(PH_PRE)) break;
    }
    double* zn = (iter & 1) ? a.z1 : a.z0;
    const double* zo = (iter & 1) ? a.z0 : a.z1;
    const int st_apply = apply(zn, zo, a.flexible != 0, &rr, nullptr);
    if (st_apply == 0) break;
    if (st_apply == 2) {
      if (!isfinite(rr)) status = (int)NLSP_ERR_BREAKDOWN;
      break;  // converged (or broke down)
    }
  }
  if (!ok) status = (int)NLSP_ERR_TIMEOUT;
  // ---- true residual ------------------------------------------------------
  double trr = 0.0;
  if (ok) {
    double s = 0.0;
    for (int i = i0 + tid; i < i1; i += PT) {
      const NodeCoord c = node_coord<KIND>(i, a.A64.N);
      const double ri = a.b[i] - stencil_apply<KIND>(a.A64, i, c, [&](int64_t m) { return __ldcg(a.x + m); });
      s = fma(ri, ri, s);
    }
    put(1, s, 0.0);
    if (bar(PH_OTHER)) trr = total1();
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (cta == 0 && tid == 0) {
    PcgState* st = a.st;
    st->bnorm2 = bb;
    st->tol2bn = tol2bn;
    st->rz = rz;
    st->rr = rr;
    st->true_rr = trr;
    st->iter = iter;
    st->status = ok ? status : (int)NLSP_ERR_TIMEOUT;
    st->done = 1;
    st->maxit = a.maxit;
    st->flexible = a.flexible;
  }
  const bool ring_ok = abort_s == 0;
  __syncthreads();
  return ring_ok;
}

// One task of a CTA: instance `inst`, as CTA `rank` of a team of `size`.
struct TeamTask {
  int inst, rank, size, pad;
};

// The persistent solver kernel.  Without a task table (task_begin == null)
// all CTAs of the launch solve instance `one` together.  Otherwise every CTA
// works through its own list of tasks tasks[task_begin[cta] ..
// task_begin[cta + 1]), which the host orders by planned start time (ties by
// instance): the CTAs of one team meet their shared instances in the same
// order, so no team waits on a CTA that waits on it.  A CTA whose copy ring
// failed (a TMA wait that gave up) leaves its remaining tasks; their teams'
// barrier waits then end at the time limit with a timeout status.  Tensor
// memory is allocated once per CTA for the whole launch.
template <int KIND, typename T, int CPG>
__global__ void __launch_bounds__(PT, 1) k_pcg_persistent(PersistArgs<T> one, const PersistArgs<T>* __restrict__ insts,
                                                         const int* __restrict__ task_begin,
                                                         const TeamTask* __restrict__ tasks, int use_tmem) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[8];
  __shared__ unsigned tbase_s;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0)
    for (int s = 0; s < 8; ++s) tma::mbar_init(&mbar[s], 1);
  if (use_tmem && warp == 0) tmem::alloc(&tbase_s, 512);
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const unsigned tbase = use_tmem ? tbase_s : 0u;
  // the instance's arguments are staged in shared memory (the single-
  // instance launch passes them as a kernel parameter)
  __shared__ __align__(16) PersistArgs<T> args_s;
  const bool table = task_begin != nullptr;
  const int tb = table ? task_begin[blockIdx.x] : 0, te = table ? task_begin[blockIdx.x + 1] : 1;
  for (int t = tb; t < te; ++t) {
    const TeamTask task = table ? tasks[t] : TeamTask{0, (int)blockIdx.x, (int)gridDim.x, 0};
    __syncthreads();  // the previous instance is done with args_s
    if (threadIdx.x == 0) args_s = table ? insts[task.inst] : one;
    __syncthreads();
    if (!solve_instance<KIND, T, CPG>(args_s, task.rank, task.size, tbase, mbar, smem_raw)) break;
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (use_tmem && warp == 0) tmem::dealloc(tbase, 512);
}

}  // namespace

// ============================================================================
// Host side
// ============================================================================
#include "pcg_cluster.cuh"

struct PcgWork {
  int64_t n = 0;
  int tsize = 0;
  double* vec = nullptr;   // x, r, q, Pv[2], Z[2]  (n each, FP64)
  void* rT = nullptr;      // residual in the preconditioner precision (FP32 path)
  double* part = nullptr;  // [4][max_blocks]
  unsigned* counter = nullptr;
  int max_blocks = 0;
  PcgState* st = nullptr;  // the state the graphs work on
  PcgState* st_all = nullptr;
  int st_cap = 0;
  PcgState* h_st = nullptr;  // pinned
  cudaStream_t cap = nullptr;  // capture stream (never the legacy default stream)
  cudaGraph_t g_while = nullptr, g_iter = nullptr;
  cudaGraphExec_t x_while = nullptr, x_iter = nullptr;
  cudaGraphConditionalHandle cond = 0;
  int built_r = -1;
  int body_launches = 0;  // kernels in one iteration body
  unsigned long long* ptimes = nullptr;  // phase timers of the persistent solver (NLSP_PHASE_TIMERS=1)
  unsigned long long* xw = nullptr;      // exchange words of the persistent solver
  size_t xw_cap = 0;
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
  if (w->rT) cudaFree(w->rT);
  if (w->part) cudaFree(w->part);
  if (w->counter) cudaFree(w->counter);
  if (w->ptimes) cudaFree(w->ptimes);
  if (w->xw) cudaFree(w->xw);
  if (w->st_all) cudaFree(w->st_all);
  if (w->h_st) cudaFreeHost(w->h_st);
  if (w->cap) cudaStreamDestroy(w->cap);
  delete w;
}

int node_grid(const nlsp_ctx* ctx, int64_t n) { return grid_for(ctx, n, TPB, NODE_BPS); }

nlsp_status ensure_work(nlsp_prec* M, int m) {
  nlsp_ctx* ctx = M->ctx;
  if (!M->pcg) {
    PcgWork* w = new PcgWork();
    w->n = M->n;
    w->tsize = M->precision == NLSP_FP64 ? 8 : 4;
    w->max_blocks = ctx->num_sms * NODE_BPS;
    M->pcg = w;
    NLSP_CUDA(cudaMalloc(&w->vec, sizeof(double) * M->n * 8));  // x r q p0 p1 z0 z1 r1
    NLSP_CUDA(cudaMemsetAsync(w->vec, 0, sizeof(double) * M->n * 8, ctx->stream));
    NLSP_CUDA(cudaMalloc(&w->rT, (size_t)w->tsize * M->n));
    NLSP_CUDA(cudaMalloc(&w->part, sizeof(double) * 4 * w->max_blocks));
    // [0..3]: last-block arrival counters of the graph kernels;
    // [4], [5]: grid-barrier counter and abort flag of the persistent solver
    NLSP_CUDA(cudaMalloc(&w->counter, sizeof(unsigned) * 8));
    NLSP_CUDA(cudaMemsetAsync(w->counter, 0, sizeof(unsigned) * 8, ctx->stream));
    NLSP_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    const char* pt = getenv("NLSP_PHASE_TIMERS");
    if (pt && pt[0] == '1') {
      NLSP_CUDA(cudaMalloc(&w->ptimes, sizeof(unsigned long long) * PTIMES_LEN));
      NLSP_CUDA(cudaMemsetAsync(w->ptimes, 0, sizeof(unsigned long long) * PTIMES_LEN, ctx->stream));
    }
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

template <typename T>
const StencilView<T>& view_T(const nlsp_op* A) {
  return *reinterpret_cast<const StencilView<T>*>(sizeof(T) == 8 ? (const void*)&A->v64 : (const void*)&A->v32);
}

// Launch plan of the P-streaming kernels: two CTAs per SM (more when a CTA's
// residual buffer would exceed 32 KB), as many tiles in flight as fit in
// ~100 KB of shared memory per CTA (at most 4).
struct StreamPlan {
  int grid, nch;
  StreamArgs sa;
  size_t smem_restrict, smem_prolong;
};

// Mutable workspace of one preconditioner application: the two smoothing
// work vectors, the restriction's per-block partials, its arrival counter,
// the coarse correction and the error word.
struct PrecWork {
  void* w0;
  void* w1;
  void* cpart;
  void* ec;
  unsigned* counter;
  int* err;
};

PrecWork prec_work_of(const nlsp_prec* M) { return PrecWork{M->w0, M->w1, M->cpart, M->ec, M->counter, M->status}; }

template <typename T>
StreamPlan stream_plan(const nlsp_prec* M) {
  StreamPlan pl;
  const int ntiles = (int)((M->n + NLSP_TILE - 1) / NLSP_TILE);
  pl.grid = std::max(std::min(ntiles, 2 * M->ctx->num_sms), div_up((int64_t)ntiles * NLSP_TILE, 8192));
  pl.grid = std::min(pl.grid, M->rblocks);
  pl.nch = (M->r + 31) / 32;
  const size_t tile = (size_t)M->r * NLSP_TILE * sizeof(T);
  pl.sa.max_nodes = div_up(ntiles, pl.grid) * NLSP_TILE;
  const size_t rho = (size_t)pl.sa.max_nodes * sizeof(T);
  const size_t budget = std::max<size_t>(100 * 1024, tile + rho);
  pl.sa.nstage = (int)std::max<size_t>(1, std::min<size_t>(4, (budget - std::min(budget - tile, rho)) / tile));
  pl.smem_restrict = (size_t)pl.sa.nstage * tile + rho;
  pl.smem_prolong = (size_t)pl.sa.nstage * tile;
  return pl;
}

// Raises a kernel's dynamic shared-memory limit to what the device allows
// beside its static shared memory.  Called before any stream capture.
template <typename F>
nlsp_status allow_max_smem(F fn) {
  cudaFuncAttributes fa;
  NLSP_CUDA(cudaFuncGetAttributes(&fa, fn));
  int dev = 0, optin = 0;
  NLSP_CUDA(cudaGetDevice(&dev));
  NLSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
  return NLSP_OK;
}

// Shared-memory limits are per device: the opt-in is raised once per
// instantiation and device (the device current at the call).
constexpr int PREP_MAX_DEVICES = 64;

template <int KIND, typename T>
nlsp_status prepare_stream_kernels() {
  static bool done_on[PREP_MAX_DEVICES];
  int dev = 0;
  NLSP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= PREP_MAX_DEVICES) return NLSP_ERR_INVALID;
  if (done_on[dev]) return NLSP_OK;
  NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 1, 0>)); NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 1, 1>));
  NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 1, 2>)); NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 2, 0>));
  NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 2, 1>)); NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 2, 2>));
  NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 3, 0>)); NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 3, 1>));
  NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 3, 2>)); NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 4, 0>));
  NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 4, 1>)); NLSP_TRY(allow_max_smem(k_restrict<KIND, T, 4, 2>));
  NLSP_TRY(allow_max_smem(k_prolong<T, 1>)); NLSP_TRY(allow_max_smem(k_prolong<T, 2>));
  NLSP_TRY(allow_max_smem(k_prolong<T, 3>)); NLSP_TRY(allow_max_smem(k_prolong<T, 4>));
  NLSP_TRY(allow_max_smem(k_pcg_persistent<KIND, T, 8>)); NLSP_TRY(allow_max_smem(k_pcg_persistent<KIND, T, 16>));
  NLSP_TRY(allow_max_smem(k_pcg_persistent<KIND, T, 32>));
  done_on[dev] = true;
  return NLSP_OK;
}

template <int KIND, typename T, int NCH>
nlsp_status launch_restrict_n(const nlsp_prec* M, const PrecWork& pw, cudaStream_t s, const StreamPlan& pl, int zm,
                              const T* rT, T* z, PcgState* st) {
  const StencilView<T>& A = view_T<T>(M->A);
  auto go = [&](auto fn) -> nlsp_status {
    fn<<<pl.grid, 128 * NCH, pl.smem_restrict, s>>>(A, (T)M->omega, rT, z, z, (const T*)M->P, M->k, M->r, pl.sa,
                                                    (T*)pw.cpart, st, pw.err);
    return NLSP_OK;
  };
  if (zm == 0) return go(k_restrict<KIND, T, NCH, 0>);
  if (zm == 1) return go(k_restrict<KIND, T, NCH, 1>);
  return go(k_restrict<KIND, T, NCH, 2>);
}

template <int KIND, typename T>
nlsp_status launch_restrict(const nlsp_prec* M, const PrecWork& pw, cudaStream_t s, const StreamPlan& pl, int zm,
                            const T* rT, T* z, PcgState* st) {
  switch (pl.nch) {
    case 1: return launch_restrict_n<KIND, T, 1>(M, pw, s, pl, zm, rT, z, st);
    case 2: return launch_restrict_n<KIND, T, 2>(M, pw, s, pl, zm, rT, z, st);
    case 3: return launch_restrict_n<KIND, T, 3>(M, pw, s, pl, zm, rT, z, st);
    default: return launch_restrict_n<KIND, T, 4>(M, pw, s, pl, zm, rT, z, st);
  }
}

template <typename T>
nlsp_status launch_prolong(const nlsp_prec* M, const PrecWork& pw, cudaStream_t s, const StreamPlan& pl, T* z,
                           PcgState* st) {
  auto go = [&](auto fn, int nt) -> nlsp_status {
    fn<<<pl.grid, nt, pl.smem_prolong, s>>>(M->n, (const T*)M->P, M->k, M->r, pl.sa, (const T*)pw.cpart, pl.grid,
                                            (const T*)M->AinvT, z, st, pw.err);
    return NLSP_OK;
  };
  switch (pl.nch) {
    case 1: return go(k_prolong<T, 1>, 128);
    case 2: return go(k_prolong<T, 2>, 256);
    case 3: return go(k_prolong<T, 3>, 384);
    default: return go(k_prolong<T, 4>, 512);
  }
}

// Enqueues the preconditioner application z = B r on stream s: rT holds r in
// the preconditioner precision; the result goes to Z.at(iter) in FP64, with
// r^T z (and flexible terms) reduced into st when st != nullptr.
// Returns the number of kernels enqueued in *nlaunch.
template <int KIND, typename T>
nlsp_status enqueue_prec(const nlsp_prec* M, const PrecWork& pw, cudaStream_t s, bool init, const T* rT,
                         const double* r, Pair<double> Z, PcgState* st, RedSlots red, cudaGraphConditionalHandle cond,
                         int set_cond, int* nlaunch) {
  const nlsp_ctx* ctx = M->ctx;
  const StencilView<T>& A = view_T<T>(M->A);
  const T omega = (T)M->omega;
  const int g = node_grid(ctx, M->n);
  T* cur = (T*)pw.w0;
  T* oth = (T*)pw.w1;
  int nl = 0;
  constexpr bool FP32 = sizeof(T) == 4;
  const StreamPlan pl = stream_plan<T>(M);
  // pre-smoothing (+ restriction)
  const bool fused_pre = FP32 && M->nu1 <= 2;
  if (!fused_pre) {
    if (M->nu1 == 1) k_presmooth<KIND, T, 1><<<g, TPB, 0, s>>>(A, omega, rT, cur, st);
    else k_presmooth<KIND, T, 2><<<g, TPB, 0, s>>>(A, omega, rT, cur, st);
    ++nl;
    for (int sw = 2; sw < M->nu1; ++sw, ++nl) {
      k_sweep<KIND, T><<<g, TPB, 0, s>>>(A, omega, rT, cur, oth, st);
      std::swap(cur, oth);
    }
  }
  NLSP_TRY((launch_restrict<KIND, T>(M, pw, s, pl, fused_pre ? M->nu1 : 0, rT, cur, st)));
  NLSP_TRY(launch_prolong<T>(M, pw, s, pl, cur, st));
  nl += 2;
  // post-smoothing
  const int nfinal = (FP32 && M->nu2 >= 2) ? 2 : 1;
  for (int sw = nfinal; sw < M->nu2; ++sw, ++nl) {
    k_sweep<KIND, T><<<g, TPB, 0, s>>>(A, omega, rT, cur, oth, st);
    std::swap(cur, oth);
  }
#define NLSP_POST(F2_, INIT_, SC_) \
  k_pcg_post<KIND, T, F2_, INIT_, SC_><<<g, TPB, 0, s>>>(A, omega, rT, r, cur, Z, st, red, cond)
  if (nfinal == 2) {
    if (init) NLSP_POST(true, true, false); else if (set_cond) NLSP_POST(true, false, true); else NLSP_POST(true, false, false);
  } else {
    if (init) NLSP_POST(false, true, false); else if (set_cond) NLSP_POST(false, false, true); else NLSP_POST(false, false, false);
  }
#undef NLSP_POST
  ++nl;
  NLSP_LAUNCH_CHECK();
  *nlaunch = nl;
  return NLSP_OK;
}


template <int KIND, typename T>
struct Solver {
  static double* x(PcgWork* w) { return w->vec; }
  static double* r(PcgWork* w) { return w->vec + w->n; }
  static double* r_(PcgWork* w) { return r(w); }
  static double* q(PcgWork* w) { return w->vec + 2 * w->n; }
  static Pair<double> Ppair(PcgWork* w) { return Pair<double>{{w->vec + 3 * w->n, w->vec + 4 * w->n}}; }
  static Pair<double> Zpair(PcgWork* w) { return Pair<double>{{w->vec + 5 * w->n, w->vec + 6 * w->n}}; }
  // residual in the preconditioner precision (the FP64 path uses r itself)
  static T* rT(PcgWork* w) { return sizeof(T) == 8 ? (T*)r(w) : (T*)w->rT; }

  // One PCG iteration (spmv, pre, then the preconditioner).
  static nlsp_status enqueue_body(const nlsp_prec* M, cudaStream_t s, int set_cond, int* nlaunch) {
    PcgWork* w = M->pcg;
    const int g = node_grid(M->ctx, M->n);
    Pair<double> Z = Zpair(w), P2 = Ppair(w);
    Pair<const double> Zc{{Z.v[0], Z.v[1]}}, Pc{{P2.v[0], P2.v[1]}};
    k_pcg_spmv<KIND><<<g, TPB, 0, s>>>(M->A->v64, Zc, P2, q(w), w->st, red_of(w));
    k_pcg_pre<T><<<g, TPB, 0, s>>>(M->n, x(w), r(w), rT(w), q(w), Pc, w->st, red_of(w));
    NLSP_LAUNCH_CHECK();
    int na = 0;
    nlsp_status st = enqueue_prec<KIND, T>(M, prec_work_of(M), s, false, rT(w), r(w), Z, w->st, red_of(w), w->cond,
                                           set_cond, &na);
    *nlaunch = 2 + na;
    return st;
  }

  // Keeps P resident in L2 while the iteration graphs run: the captured
  // kernel nodes inherit an access-policy window over P from the capture
  // stream (P is read twice per iteration).  The persisting-L2 limit is a
  // setting of this process's context only.
  static nlsp_status set_l2_window(nlsp_prec* M) {
    PcgWork* w = M->pcg;
    int dev = 0, max_persist = 0, max_window = 0;
    NLSP_CUDA(cudaGetDevice(&dev));
    NLSP_CUDA(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev));
    NLSP_CUDA(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev));
    if (max_persist <= 0 || max_window <= 0) return NLSP_OK;
    const size_t pbytes = (size_t)M->n_pad * M->k * sizeof(T);
    size_t limit = 0;
    NLSP_CUDA(cudaDeviceGetLimit(&limit, cudaLimitPersistingL2CacheSize));
    const size_t want = std::min<size_t>(pbytes, (size_t)max_persist);
    if (limit < want) NLSP_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
    cudaStreamAttrValue v;
    memset(&v, 0, sizeof(v));
    v.accessPolicyWindow.base_ptr = M->P;
    v.accessPolicyWindow.num_bytes = std::min<size_t>(pbytes, (size_t)max_window);
    v.accessPolicyWindow.hitRatio = (float)std::min(1.0, (double)want / (double)v.accessPolicyWindow.num_bytes);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    NLSP_CUDA(cudaStreamSetAttribute(w->cap, cudaStreamAttributeAccessPolicyWindow, &v));
    return NLSP_OK;
  }

  static nlsp_status build_graphs(nlsp_prec* M) {
    PcgWork* w = M->pcg;
    destroy_graphs(w);
    NLSP_TRY(set_l2_window(M));
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
    nlsp_status st = enqueue_body(M, w->cap, 1, &w->body_launches);
    cudaGraph_t dummy = nullptr;
    cudaError_t e = cudaStreamEndCapture(w->cap, &dummy);
    if (st != NLSP_OK) return st;
    NLSP_CUDA(e);
    NLSP_CUDA(cudaGraphInstantiate(&w->x_while, w->g_while, 0));
    // single-iteration graph for the host-checked mode
    NLSP_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
    int nb = 0;
    st = enqueue_body(M, w->cap, 0, &nb);
    e = cudaStreamEndCapture(w->cap, &w->g_iter);
    if (st != NLSP_OK) return st;
    NLSP_CUDA(e);
    NLSP_CUDA(cudaGraphInstantiate(&w->x_iter, w->g_iter, 0));
    w->built_r = M->r;
    return NLSP_OK;
  }

  static int cpg_for(int r) { return r <= 32 ? 8 : (r <= 64 ? 16 : 32); }
  static const void* persistent_fn(int cpg) {
    return cpg == 8 ? (const void*)k_pcg_persistent<KIND, T, 8>
         : cpg == 16 ? (const void*)k_pcg_persistent<KIND, T, 16>
                     : (const void*)k_pcg_persistent<KIND, T, 32>;
  }

  // Dynamic shared memory the persistent kernel may use beside its static
  // shared memory (one CTA per SM).
  static nlsp_status persistent_smem(int cpg, size_t* smem) {
    cudaFuncAttributes fa;
    NLSP_CUDA(cudaFuncGetAttributes(&fa, persistent_fn(cpg)));
    int dev = 0, optin = 0;
    NLSP_CUDA(cudaGetDevice(&dev));
    NLSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    *smem = (size_t)std::max<int64_t>(0, (int64_t)optin - (int64_t)fa.sharedSizeBytes - 1024);
    return NLSP_OK;
  }

  // Residency plan of one instance solved by `team` CTAs with `avail` bytes
  // of dynamic shared memory: the first tiles of each CTA in tensor memory
  // (FP32), the next ones resident in shared memory, the rest streamed
  // through a TMA ring.  *need = the dynamic shared memory the plan uses.
  static nlsp_status plan_instance(const nlsp_prec* M, int team, int cpg, bool tmem_ok, size_t avail,
                                   StreamArgs* sa, size_t* need) {
    const int ntiles = (int)((M->n + NLSP_TILE - 1) / NLSP_TILE);
    const size_t tile = (size_t)M->r * NLSP_TILE * sizeof(T);
    const int max_tiles = div_up(ntiles, team);
    const size_t rho = (size_t)max_tiles * NLSP_TILE * sizeof(T);
    const int64_t left = (int64_t)avail - (int64_t)rho;
    sa->max_nodes = max_tiles * NLSP_TILE;
    sa->n_tm = (sizeof(T) == 4 && tmem_ok) ? std::min(max_tiles, 512 / (4 * cpg)) : 0;
    const int rem = max_tiles - sa->n_tm;
    sa->nstage = rem > 0 ? 2 : 1;
    if (left < (int64_t)(sa->nstage * tile)) sa->nstage = 1;
    if (left < (int64_t)tile) {
      nlsp_record_message("persistent solver: one P tile does not fit in shared memory");
      return NLSP_ERR_INVALID;
    }
    sa->n_sm = rem > 0 ? (int)std::min<int64_t>(rem, (left - (int64_t)sa->nstage * tile) / (int64_t)tile) : 0;
    *need = (size_t)(sa->nstage + sa->n_sm) * tile + rho;
    return NLSP_OK;
  }

  // Whether the CG update can run inside the staged restriction: FP32, a 2D
  // stencil, fused pre-smoothing (nu <= 2) and, for the largest CTA share,
  // room in the ring buffer for the updated residual and both pre-sweeps
  // over the own nodes plus two stencil hops (N + 1 nodes each).  Off with
  // NLSP_MERGE_PRE=0.
  static int merge_ok(const nlsp_prec* M, const StreamArgs& sa) {
    const char* env = getenv("NLSP_MERGE_PRE");
    if (env && env[0] == '0') return 0;
    if (sizeof(T) != 4 || (KIND != ST_5PT && KIND != ST_9PT) || M->nu1 > 2) return 0;
    const int64_t hop = (int64_t)M->A->N + 1;
    const int64_t nodes = sa.max_nodes;
    const int64_t need = 2 * (nodes + 4 * hop) + (nodes + 2 * hop);
    return need <= (int64_t)sa.nstage * M->r * NLSP_TILE ? 1 : 0;
  }

  // Exchange words of one instance solved by `team` CTAs (zero at launch).
  static size_t xw_words(const nlsp_prec* M, int team) {
    return 2 + (size_t)4 * ((team + 1) & ~1) + ((size_t)team * M->k * sizeof(T) + 7) / 8;
  }

  // Kernel arguments of one instance: right-hand side b, iterate x (may be
  // the caller's output: it is set to zero first), state st, exchange words
  // xw and abort flag.
  static PersistArgs<T> instance_args(nlsp_prec* M, const double* b, double* x_, const nlsp_solve_params* prm,
                                      int flexible, PcgState* st_out, unsigned long long* xw, int* abort_flag,
                                      const StreamArgs& sa) {
    PcgWork* w = M->pcg;
    PersistArgs<T> a;
    a.A64 = M->A->v64;
    a.AT = view_T<T>(M->A);
    a.omega = (T)M->omega;
    a.nu1 = M->nu1;
    a.nu2 = M->nu2;
    a.flexible = flexible;
    a.maxit = prm->maxit;
    a.tol = prm->tol;
    a.b = b;
    a.x = x_;
    a.r = r_(w);
    a.q = q(w);
    Pair<double> P2 = Ppair(w), Z2 = Zpair(w);
    a.p0 = P2.v[0];
    a.p1 = P2.v[1];
    a.z0 = Z2.v[0];
    a.z1 = Z2.v[1];
    a.r1 = w->vec + 7 * w->n;
    a.merge = merge_ok(M, sa);
    a.rT = rT(w);
    a.zw = (T*)M->w0;
    a.zw2 = (T*)M->w1;
    a.P = (const T*)M->P;
    a.k = M->k;
    a.rr_ = M->r;
    a.Ainv = (const T*)M->AinvT;
    a.xw = xw;
    a.abort = abort_flag;
    a.progress = nullptr;
    a.st = st_out;
    a.sa = sa;
    a.ptimes = w->ptimes;
    return a;
  }

  // Cluster-resident solver for small systems (graph_mode 2): the smallest
  // power-of-two cluster of C <= 16 CTAs whose ranks' shared memory holds the
  // vectors and P rows of about n / C nodes, preferring C with at most ~96
  // nodes per rank (the FP64 work of a rank is what an iteration waits for).
  // Off with NLSP_CLUSTER=0.  Returns false when the system does not fit.
  struct ClusterPlan {
    int C, nl, nlp, ew, ainv;
    size_t smem;
  };

  // Cluster size and shared-memory layout of the cluster-resident solver, or
  // false when the system does not fit one cluster (the grid-wide persistent
  // kernel then runs).  A_c^-1 is copied into shared memory when it still fits.
  static bool cluster_plan(const nlsp_prec* M, ClusterPlan* pl) {
    const char* env = getenv("NLSP_CLUSTER");
    if (env && env[0] == '0') return false;
    if (M->n > 16 * 4096) return false;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void*)k_pcg_cluster<KIND, T>) != cudaSuccess) return false;
    const size_t avail = (size_t)optin - fa.sharedSizeBytes - 1024;
    const int ew = KIND == ST_CSR ? M->A->wmax : cluster_stencil_width<KIND>();
    if (ew < 0 || ew > 64) return false;
    int c = 1;
    while (c < CL_MAX && (M->n + c - 1) / c > 96) c *= 2;
    const char* csz = getenv("NLSP_CLUSTER_SIZE");  // a fixed cluster size (1, 2, 4, 8 or 16)
    if (csz && atoi(csz) >= 1 && atoi(csz) <= CL_MAX && (atoi(csz) & (atoi(csz) - 1)) == 0) c = atoi(csz);
    for (; c <= CL_MAX; c *= 2) {
      const int l = (int)((M->n + c - 1) / c);
      if (l > 32767) continue;  // node references keep the index within the owner in 16 bits
      const int lp = l | 1;
      for (int ainv = 1; ainv >= 0; --ainv) {
        const size_t need = cluster_smem<T>(l, lp, M->r, ew, ainv != 0);
        if (need <= avail) {
          *pl = ClusterPlan{c, l, lp, ew, ainv, need};
          return true;
        }
      }
    }
    return false;
  }

  static nlsp_status launch_cluster(nlsp_prec* M, const double* b, double* xout, const nlsp_solve_params* prm,
                                    int flexible, PcgState* st_out, const ClusterPlan& pl) {
    const int C = pl.C;
    const size_t smem = pl.smem;
    nlsp_ctx* ctx = M->ctx;
    auto fn = k_pcg_cluster<KIND, T>;
    NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    ClusterArgs a;
    a.n = M->n;
    a.nl = pl.nl;
    a.nlp = pl.nlp;
    a.k = M->k;
    a.r = M->r;
    a.nu1 = M->nu1;
    a.nu2 = M->nu2;
    a.flexible = flexible;
    a.maxit = prm->maxit;
    a.tol = prm->tol;
    a.b = b;
    a.x = xout;
    a.P = M->P;
    a.Ainv = M->AinvT;
    a.ew = pl.ew;
    a.ainv_smem = pl.ainv;
    a.rg = 1;
    while (a.rg < 32 && 2 * a.rg * M->r <= CT) a.rg *= 2;
    a.lc = 1;
    while (a.lc < CL_MAX && 2 * a.lc * M->r <= CT) a.lc *= 2;
    a.st = st_out;
    a.ptimes = M->pcg ? M->pcg->ptimes : nullptr;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(CT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    NLSP_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg));
    if (nclusters < 1) {
      nlsp_record_message("cluster solver: the cluster does not fit on the device");
      return NLSP_ERR_INVALID;
    }
    NLSP_CUDA(cudaLaunchKernelEx(&cfg, fn, M->A->v64, view_T<T>(M->A), (T)M->omega, a));
    count_launches(ctx, 1);
    return NLSP_OK;
  }

  // The persistent cooperative solver (graph_mode 2): one launch per column,
  // all CTAs on the one instance.
  static nlsp_status launch_persistent(nlsp_prec* M, const double* b, double* xout, const nlsp_solve_params* prm,
                                       int flexible, PcgState* st_out) {
    nlsp_ctx* ctx = M->ctx;
    PcgWork* w = M->pcg;
    cudaStream_t s = ctx->stream;
    const int G = std::min(ctx->num_sms, XMAX_RANKS);
    const int cpg = cpg_for(M->r);
    const void* fn = persistent_fn(cpg);
    size_t avail = 0, smem = 0;
    NLSP_TRY(persistent_smem(cpg, &avail));
    StreamArgs sa;
    NLSP_TRY(plan_instance(M, G, cpg, true, avail, &sa, &smem));
    const size_t words = xw_words(M, G);
    if (w->xw_cap < words) {
      if (w->xw) cudaFree(w->xw);
      w->xw = nullptr;
      w->xw_cap = 0;
      NLSP_CUDA(cudaMalloc(&w->xw, sizeof(unsigned long long) * words));
      w->xw_cap = words;
    }
    PersistArgs<T> a = instance_args(M, b, x(w), prm, flexible, st_out, w->xw, (int*)(w->counter + 5), sa);
    int per_sm = 0;
    NLSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PT, smem));
    if (per_sm < 1) {
      nlsp_record_message("persistent solver: one CTA per SM does not fit (shared memory or registers)");
      return NLSP_ERR_INVALID;
    }
    NLSP_CUDA(cudaMemsetAsync(w->xw, 0, sizeof(unsigned long long) * words, s));
    NLSP_CUDA(cudaMemsetAsync(w->counter + 4, 0, sizeof(unsigned) * 2, s));
    const PersistArgs<T>* no_insts = nullptr;
    const int* no_begin = nullptr;
    const TeamTask* no_tasks = nullptr;
    int use_tmem = sa.n_tm > 0 ? 1 : 0;
    void* args[] = {&a, &no_insts, &no_begin, &no_tasks, &use_tmem};
    NLSP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(PT), args, smem, s));
    count_launches(ctx, 1);
    NLSP_CUDA(cudaMemcpyAsync(xout, x(w), sizeof(double) * M->n, cudaMemcpyDeviceToDevice, s));
    return NLSP_OK;
  }

  static nlsp_status solve(nlsp_prec* M, int m, const double* B, int64_t ldb, double* X, int64_t ldx,
                           const nlsp_solve_params* prm, nlsp_solve_info* infos) {
    nlsp_ctx* ctx = M->ctx;
    cudaStream_t s = ctx->stream;
    NLSP_TRY(ensure_work(M, m));
    NLSP_TRY((prepare_stream_kernels<KIND, T>()));
    PcgWork* w = M->pcg;
    if (prm->graph_mode == 2) {
      const int flexible = prm->flexible < 0 ? (M->precision != NLSP_FP64) : (prm->flexible != 0);
      ClusterPlan pl{};
      const bool clus = cluster_plan(M, &pl);
      for (int col = 0; col < m; ++col) {
        if (clus)
          NLSP_TRY(launch_cluster(M, B + col * ldb, X + col * ldx, prm, flexible, w->st_all + col, pl));
        else
          NLSP_TRY(launch_persistent(M, B + col * ldb, X + col * ldx, prm, flexible, w->st_all + col));
      }
      NLSP_CUDA(cudaMemcpyAsync(w->h_st, w->st_all, sizeof(PcgState) * m, cudaMemcpyDeviceToHost, s));
      NLSP_CUDA(cudaStreamSynchronize(s));
      return summarize(w, m, infos, 0);
    }
    if (!w->x_while || w->built_r != M->r) NLSP_TRY(build_graphs(M));
    const int flexible = prm->flexible < 0 ? (M->precision != NLSP_FP64) : (prm->flexible != 0);
    const int g = node_grid(ctx, M->n);
    for (int col = 0; col < m; ++col) {
      const double* b = B + col * ldb;
      Pair<double> P2 = Ppair(w);
      k_pcg_init<T><<<g, TPB, 0, s>>>(M->n, b, x(w), r(w), rT(w), P2.v[0], P2.v[1], q(w), w->st, prm->tol,
                                      prm->maxit, flexible, red_of(w));
      NLSP_LAUNCH_CHECK();
      int na = 0;
      NLSP_TRY((enqueue_prec<KIND, T>(M, prec_work_of(M), s, true, rT(w), r(w), Zpair(w), w->st, red_of(w), 0, 0,
                                      &na)));
      count_launches(ctx, 2 + na);  // init, preconditioner, true residual
      if (prm->graph_mode == 1) {
        NLSP_CUDA(cudaGraphLaunch(w->x_while, s));
      } else {
        int done_iters = 0;
        while (done_iters < prm->maxit) {
          const int chunk = std::min(8, prm->maxit - done_iters);
          for (int c = 0; c < chunk; ++c) NLSP_CUDA(cudaGraphLaunch(w->x_iter, s));
          count_launches(ctx, (unsigned long long)chunk * w->body_launches);
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
    if (prm->graph_mode == 1)
      for (int col = 0; col < m; ++col)
        count_launches(ctx, (unsigned long long)std::max(w->h_st[col].iter, 1) * w->body_launches);
    return summarize(w, m, infos, 0);
  }

  // Batched persistent solve: instance i solves A_i x_i = b_i with its own
  // preconditioner Ms[i]; one cooperative launch runs every instance on a
  // team of CTAs planned by nlsp_internal_plan_teams.
  static nlsp_status solve_batched(nlsp_ctx* ctx, int count, nlsp_prec* const* Ms, const double* const* B,
                                   double* const* X, const nlsp_solve_params* prm, int tiles_per_cta,
                                   nlsp_solve_info* infos) {
    cudaStream_t s = ctx->stream;
    const int G = std::min(ctx->num_sms, XMAX_RANKS);
    NLSP_TRY((prepare_stream_kernels<KIND, T>()));
    int rmax = 1;
    std::vector<int64_t> nn(count);
    std::vector<int> cap(count, G);
    for (int i = 0; i < count; ++i) {
      NLSP_TRY(ensure_work(Ms[i], 1));
      rmax = std::max(rmax, Ms[i]->r);
      nn[i] = Ms[i]->n;
    }
    const int cpg = cpg_for(rmax);
    const void* fn = persistent_fn(cpg);
    size_t avail = 0;
    NLSP_TRY(persistent_smem(cpg, &avail));
    std::vector<int> first(count), size(count);
    std::vector<double> start(count);
    NLSP_TRY(nlsp_internal_plan_teams(count, nn.data(), cap.data(), G, tiles_per_cta, first.data(), size.data(),
                                      start.data()));
    // device table: instances, CTA task ranges, tasks, abort flags and the
    // progress word, states, exchange words
    std::vector<std::vector<TeamTask>> per(G);
    std::vector<std::pair<double, int>> key(count);
    for (int i = 0; i < count; ++i) key[i] = {start[i], i};
    std::sort(key.begin(), key.end());
    for (const auto& kv : key) {
      const int i = kv.second;
      for (int c = 0; c < size[i]; ++c) per[first[i] + c].push_back(TeamTask{i, c, size[i], 0});
    }
    int ntask = 0;
    for (int c = 0; c < G; ++c) ntask += (int)per[c].size();
    const size_t off_begin = align_up(sizeof(PersistArgs<T>) * count, 256);
    const size_t off_tasks = off_begin + align_up(sizeof(int) * (G + 1), 256);
    const size_t off_ctr = off_tasks + align_up(sizeof(TeamTask) * std::max(ntask, 1), 256);
    const size_t off_st = off_ctr + align_up(sizeof(unsigned) * (count + 1), 256);
    const size_t off_xw = off_st + align_up(sizeof(PcgState) * count, 256);
    std::vector<size_t> xw_at(count);
    size_t xw_total = 0;
    for (int i = 0; i < count; ++i) {
      xw_at[i] = xw_total;
      xw_total += align_up(xw_words(Ms[i], size[i]), 32);
    }
    const size_t bytes = off_xw + sizeof(unsigned long long) * xw_total;
    unsigned char* dev = (unsigned char*)ctx_slot(ctx, SLOT_BATCH, bytes);
    if (!dev) return NLSP_ERR_OOM;
    std::vector<unsigned char> host(off_xw, 0);
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
      StreamArgs sa;
      size_t need = 0;
      NLSP_TRY(plan_instance(Ms[i], size[i], cpg, true, avail, &sa, &need));
      smem = std::max(smem, need);
      PersistArgs<T> a = instance_args(Ms[i], B[i], X[i], prm,
                                       prm->flexible < 0 ? (Ms[i]->precision != NLSP_FP64) : (prm->flexible != 0),
                                       (PcgState*)(dev + off_st) + i,
                                       (unsigned long long*)(dev + off_xw) + xw_at[i], (int*)(dev + off_ctr) + i, sa);
      a.ptimes = nullptr;
      a.progress = (unsigned*)(dev + off_ctr) + count;
      memcpy(host.data() + sizeof(PersistArgs<T>) * i, &a, sizeof(a));
    }
    int* hb = (int*)(host.data() + off_begin);
    TeamTask* ht = (TeamTask*)(host.data() + off_tasks);
    for (int c = 0, t = 0; c < G; ++c) {
      hb[c] = t;
      for (const TeamTask& task : per[c]) ht[t++] = task;
      hb[c + 1] = t;
    }
    int per_sm = 0;
    NLSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PT, smem));
    if (per_sm < 1) {
      nlsp_record_message("batched solver: one CTA per SM does not fit (shared memory or registers)");
      return NLSP_ERR_INVALID;
    }
    NLSP_CUDA(cudaMemcpyAsync(dev, host.data(), off_xw, cudaMemcpyHostToDevice, s));
    NLSP_CUDA(cudaMemsetAsync(dev + off_xw, 0, sizeof(unsigned long long) * xw_total, s));
    PersistArgs<T> one;
    memset(&one, 0, sizeof(one));
    const PersistArgs<T>* d_insts = (const PersistArgs<T>*)dev;
    const int* d_begin = (const int*)(dev + off_begin);
    const TeamTask* d_tasks = (const TeamTask*)(dev + off_tasks);
    int use_tmem = sizeof(T) == 4 ? 1 : 0;
    void* args[] = {&one, &d_insts, &d_begin, &d_tasks, &use_tmem};
    NLSP_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(PT), args, smem, s));
    count_launches(ctx, 1);
    std::vector<PcgState> hs(count);
    NLSP_CUDA(cudaMemcpyAsync(hs.data(), dev + off_st, sizeof(PcgState) * count, cudaMemcpyDeviceToHost, s));
    NLSP_CUDA(cudaStreamSynchronize(s));
    return summarize_states(hs.data(), count, infos);
  }

  static nlsp_status summarize(PcgWork* w, int m, nlsp_solve_info* infos, int) {
    return summarize_states(w->h_st, m, infos);
  }

  static nlsp_status summarize_states(const PcgState* hs, int m, nlsp_solve_info* infos) {
    nlsp_status worst = NLSP_OK;
    for (int col = 0; col < m; ++col) {
      const PcgState& h = hs[col];
      int stc = h.status;
      if (stc == NLSP_OK && !h.done) stc = NLSP_NOT_CONVERGED;
      if (infos) {
        infos[col].iterations = h.iter;
        infos[col].status = stc;
        infos[col].relres = h.bnorm2 > 0 ? sqrt(h.rr / h.bnorm2) : 0.0;
        infos[col].true_relres = h.bnorm2 > 0 ? sqrt(h.true_rr / h.bnorm2) : 0.0;
      }
      if (stc == NLSP_ERR_BREAKDOWN || stc == NLSP_ERR_TIMEOUT) worst = (nlsp_status)stc;
      else if (stc == NLSP_NOT_CONVERGED && worst == NLSP_OK) worst = NLSP_NOT_CONVERGED;
    }
    return worst;
  }

  static nlsp_status apply(nlsp_prec* M, int m, const double* Rin, int64_t ldr, double* Zout, int64_t ldz) {
    nlsp_ctx* ctx = M->ctx;
    cudaStream_t s = ctx->stream;
    NLSP_TRY(ensure_work(M, 1));
    NLSP_TRY((prepare_stream_kernels<KIND, T>()));
    PcgWork* w = M->pcg;
    for (int col = 0; col < m; ++col) {
      const double* rc = Rin + col * ldr;
      const T* rt = (const T*)rc;
      if (sizeof(T) == 4) {
        k_convert<T><<<node_grid(ctx, M->n), TPB, 0, s>>>(rc, (T*)w->rT, M->n);
        rt = (const T*)w->rT;
        count_launches(ctx, 1);
      }
      double* zc = Zout + col * ldz;
      Pair<double> Zp{{zc, zc}};
      int na = 0;
      NLSP_TRY((enqueue_prec<KIND, T>(M, prec_work_of(M), s, true, rt, rc, Zp, nullptr, red_of(w), 0, 0, &na)));
      count_launches(ctx, na);
    }
    return NLSP_OK;
  }
};

// Back-to-back launches of one hot kernel on the current buffers (timing).
template <int KIND, typename T>
nlsp_status bench_launch(nlsp_prec* M, int which, int reps) {
  PcgWork* w = M->pcg;
  cudaStream_t s = M->ctx->stream;
  NLSP_TRY((prepare_stream_kernels<KIND, T>()));
  const StreamPlan pl = stream_plan<T>(M);
  T* z = (T*)M->w0;
  const T* rT = Solver<KIND, T>::rT(w);
  constexpr int ZM = sizeof(T) == 4 ? 2 : 0;
  for (int i = 0; i < reps; ++i) {
    if (which == 0) NLSP_TRY((launch_restrict<KIND, T>(M, prec_work_of(M), s, pl, ZM, rT, z, nullptr)));
    else NLSP_TRY(launch_prolong<T>(M, prec_work_of(M), s, pl, z, nullptr));
  }
  NLSP_LAUNCH_CHECK();
  count_launches(M->ctx, reps);
  return NLSP_OK;
}

// ----------------------------------------------------------------------------
// Layout of the no-allocation scratch array (the array itself, its address
// lookup and the entry point are in pcg.cu): residual in the preconditioner
// precision, two smoothing work vectors, the restriction partials (strided
// by the stored rank k), the coarse correction and the arrival counter.
// ----------------------------------------------------------------------------

constexpr int64_t NOALLOC_MAX_BLOCKS = 1024;
constexpr size_t NOALLOC_VEC_BYTES = (size_t)NLSP_NOALLOC_MAX_N * sizeof(double);
constexpr size_t NOALLOC_PART_BYTES = (size_t)NOALLOC_MAX_BLOCKS * NLSP_NOALLOC_MAX_RANK * sizeof(double);
constexpr size_t NOALLOC_BYTES = 3 * NOALLOC_VEC_BYTES + NOALLOC_PART_BYTES + NLSP_NOALLOC_MAX_RANK * sizeof(double) + 256;


template <int KIND, typename T>
nlsp_status apply_noalloc(const nlsp_prec* M, unsigned char* base, int m, const double* R, int64_t ldr, double* Z,
                          int64_t ldz) {
  cudaStream_t s = M->ctx->stream;
  NLSP_TRY((prepare_stream_kernels<KIND, T>()));
  const StreamPlan pl = stream_plan<T>(M);
  if (pl.grid > NOALLOC_MAX_BLOCKS) {
    nlsp_record_message("nlsp_apply_prec_noalloc: restriction grid exceeds the scratch capacity");
    return NLSP_ERR_INVALID;
  }
  T* rT = (T*)base;
  PrecWork pw;
  pw.w0 = base + NOALLOC_VEC_BYTES;
  pw.w1 = base + 2 * NOALLOC_VEC_BYTES;
  pw.cpart = base + 3 * NOALLOC_VEC_BYTES;
  pw.ec = base + 3 * NOALLOC_VEC_BYTES + NOALLOC_PART_BYTES;
  pw.counter = (unsigned*)(base + 3 * NOALLOC_VEC_BYTES + NOALLOC_PART_BYTES +
                           NLSP_NOALLOC_MAX_RANK * sizeof(double));
  pw.err = M->status;
  // the restriction's arrival counter must start at zero (the array keeps
  // whatever the last call left)
  NLSP_CUDA(cudaMemsetAsync(pw.counter, 0, 256, s));
  RedSlots none{nullptr, nullptr, 0};
  for (int col = 0; col < m; ++col) {
    const double* rc = R + col * ldr;
    const T* rt = (const T*)rc;
    if (sizeof(T) == 4) {
      k_convert<T><<<node_grid(M->ctx, M->n), TPB, 0, s>>>(rc, rT, M->n);
      rt = rT;
      count_launches(M->ctx, 1);
    }
    double* zc = Z + col * ldz;
    Pair<double> Zp{{zc, zc}};
    int na = 0;
    NLSP_TRY((enqueue_prec<KIND, T>(M, pw, s, true, rt, rc, Zp, nullptr, none, 0, 0, &na)));
    count_launches(M->ctx, na);
  }
  return NLSP_OK;
}

}  // namespace

// Entry points of one (stencil kind, precision) instantiation of the solver.
struct PcgKindOps {
  nlsp_status (*apply)(nlsp_prec* M, int m, const double* R, int64_t ldr, double* Z, int64_t ldz);
  nlsp_status (*solve)(nlsp_prec* M, int m, const double* B, int64_t ldb, double* X, int64_t ldx,
                       const nlsp_solve_params* prm, nlsp_solve_info* infos);
  nlsp_status (*solve_batched)(nlsp_ctx* ctx, int count, nlsp_prec* const* Ms, const double* const* B,
                               double* const* X, const nlsp_solve_params* prm, int tiles_per_cta,
                               nlsp_solve_info* infos);
  nlsp_status (*bench)(nlsp_prec* M, int which, int reps);
  nlsp_status (*apply_noalloc)(const nlsp_prec* M, unsigned char* base, int m, const double* R, int64_t ldr,
                               double* Z, int64_t ldz);
};

const PcgKindOps* nlsp_pcg_ops_5pt_f64();
const PcgKindOps* nlsp_pcg_ops_5pt_f32();
const PcgKindOps* nlsp_pcg_ops_9pt_f64();
const PcgKindOps* nlsp_pcg_ops_9pt_f32();
const PcgKindOps* nlsp_pcg_ops_7pt_f64();
const PcgKindOps* nlsp_pcg_ops_7pt_f32();
const PcgKindOps* nlsp_pcg_ops_csr_f64();
const PcgKindOps* nlsp_pcg_ops_csr_f32();

// Defines nlsp_pcg_ops_<NAME_>() for stencil kind KIND_ in precision T_.
#define NLSP_PCG_OPS(KIND_, T_, NAME_)                                                                  \
  const PcgKindOps* nlsp_pcg_ops_##NAME_() {                                                          \
    static const PcgKindOps ops = {Solver<KIND_, T_>::apply, Solver<KIND_, T_>::solve,                 \
                                   Solver<KIND_, T_>::solve_batched, bench_launch<KIND_, T_>,         \
                                   apply_noalloc<KIND_, T_>};                                         \
    return &ops;                                                                                      \
  }
