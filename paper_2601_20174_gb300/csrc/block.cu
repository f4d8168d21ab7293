// Block PCG: m <= 32 right-hand sides advance together (independent
// recurrences, one per column; Sec. 4 PCG with the two-level preconditioner
// of Algorithm 1), so each preconditioner application reads P once for all
// columns: the restriction is the dense product P^T rho (k x m) and the
// prolongation P E (n x m).
//
// Layout: block vectors are node-major with a row of 32 columns per node
// (element (i, c) at i * 32 + c), so a warp holds one node's row (lane =
// column) and every stencil neighbour is one coalesced row.  Columns beyond m
// are zero and never iterate.  The PCG recurrences and their dot products are
// FP64; the preconditioner runs in its own precision T (FP32 or FP64).
// Per-column scalars (alpha, beta, r^T z, convergence, iteration counts)
// stay on the device; the host relaunches a captured iteration graph in
// chunks and reads one "all columns done" word between chunks.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "stencil.cuh"
#include "tma.cuh"
#include "block_lp.cuh"

namespace {

constexpr int MB = 32;        // columns per node row
constexpr int BT = 256;       // threads per block (8 warps)
constexpr int BW = BT / 32;   // warps per block

// Per-column state of the block recurrences (device).
struct BlockState {
  double bb[MB], tol2bn[MB], rz[MB], rr[MB], alpha[MB], beta[MB], true_rr[MB];
  int iter[MB], done[MB], status[MB];
  int all_done, maxit, flexible, m;
  int t;    // iterations started (A p products formed)
  int err;  // a tensor-core completion wait gave up
};

// Sum of the warps' per-column partials of a block, written to part[block][c].
__device__ __forceinline__ void block_col_partial(double v, double (*sm)[MB], double* part) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  sm[w][lane] = v;
  __syncthreads();
  if (w == 0) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < BW; ++q) s += sm[q][lane];
    part[(int64_t)blockIdx.x * MB + lane] = s;
  }
}

// p = z + beta p (beta = 0 before the first iteration, p = 0 initially)
__global__ void __launch_bounds__(BT) k_b_dir(const double* __restrict__ z, double* __restrict__ p, int64_t n,
                                             const BlockState* st) {
  const int lane = threadIdx.x & 31;
  const double beta = st->beta[lane];
  for (int64_t e = (int64_t)blockIdx.x * BT + threadIdx.x; e < n * MB; e += (int64_t)gridDim.x * BT)
    p[e] = fma(beta, p[e], z[e]);
}

// q = A p, per-column partials of p^T q
template <int KIND>
__global__ void __launch_bounds__(BT) k_b_spmv(StencilView<double> A, const double* __restrict__ p,
                                              double* __restrict__ q, double* __restrict__ part) {
  __shared__ double sm[BW][MB];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  double s = 0.0;
  for (int64_t i = w0; i < A.n; i += ws) {
    const double qi = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return p[m * MB + lane]; });
    q[i * MB + lane] = qi;
    s = fma(p[i * MB + lane], qi, s);
  }
  block_col_partial(s, sm, part);
}

// x += alpha p, r -= alpha q, rT = r (precision T), z1 = w D^-1 rT (first
// pre-sweep from zero), per-column partials of r^T r
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_b_update(StencilView<T> A, T omega, double* __restrict__ x,
                                                double* __restrict__ r, const double* __restrict__ p,
                                                const double* __restrict__ q, T* __restrict__ rT,
                                                T* __restrict__ z1, const BlockState* st,
                                                double* __restrict__ part) {
  __shared__ double sm[BW][MB];
  const int lane = threadIdx.x & 31;
  const double alpha = st->alpha[lane];
  const int64_t w0 = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  double s = 0.0;
  for (int64_t i = w0; i < A.n; i += ws) {
    const int64_t e = i * MB + lane;
    x[e] = fma(alpha, p[e], x[e]);
    const double rn = fma(-alpha, q[e], r[e]);
    r[e] = rn;
    const T rt = (T)rn;
    rT[e] = rt;
    z1[e] = omega * stencil_dinv<KIND>(A, i) * rt;
    s = fma(rn, rn, s);
  }
  block_col_partial(s, sm, part);
}

// ---- four columns per thread: 8 threads per node row, vector loads -------
template <typename T>
struct V4 {
  T v[4];
};

template <typename T>
__device__ __forceinline__ V4<T> ld4(const T* p) {
  V4<T> r;
  if (sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    r.v[0] = (T)f.x; r.v[1] = (T)f.y; r.v[2] = (T)f.z; r.v[3] = (T)f.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    r.v[0] = (T)a.x; r.v[1] = (T)a.y; r.v[2] = (T)b.x; r.v[3] = (T)b.y;
  }
  return r;
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const V4<T>& r) {
  if (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4((float)r.v[0], (float)r.v[1], (float)r.v[2], (float)r.v[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2((double)r.v[0], (double)r.v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2((double)r.v[2], (double)r.v[3]);
  }
}

// (A x)_idx for four columns at once (same arithmetic as stencil_apply, per column)
template <int KIND, typename T, typename Get>
__device__ __forceinline__ V4<T> stencil_apply4(const StencilView<T>& A, int64_t idx, NodeCoord c, Get get) {
  const int N = A.N;
  V4<T> s;
  if (KIND == ST_CSR) {
    const V4<T> x0 = get(idx);
    const T d = A.diag[idx];
#pragma unroll
    for (int q = 0; q < 4; ++q) s.v[q] = d * x0.v[q];
    int64_t base;
    int wd;
    csr_row(A, idx, &base, &wd);
    for (int j = 0; j < wd; ++j) {
      const int64_t e = base + 32 * (int64_t)j;
      const T a = A.sval[e];
      const V4<T> x = get((int64_t)A.scol[e]);  // padding: (own row, 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) s.v[q] += a * x.v[q];
    }
  } else if (KIND == ST_9PT) {
    const bool w = c.i > 0, e = c.i < N - 1, so = c.j > 0, no = c.j < N - 1;
    const V4<T> x0 = get(idx);
    V4<T> ew, ns, d1, d2;
#pragma unroll
    for (int q = 0; q < 4; ++q) ew.v[q] = ns.v[q] = d1.v[q] = d2.v[q] = T(0);
    auto add = [&](V4<T>& acc, int64_t m) {
      const V4<T> x = get(m);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc.v[q] += x.v[q];
    };
    if (w) add(ew, idx - 1);
    if (e) add(ew, idx + 1);
    if (so) add(ns, idx - N);
    if (no) add(ns, idx + N);
    if (e && no) add(d1, idx + N + 1);
    if (w && so) add(d1, idx - N - 1);
    if (w && no) add(d2, idx + N - 1);
    if (e && so) add(d2, idx - N + 1);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      s.v[q] = A.c[0] * x0.v[q] + A.c[1] * ew.v[q] + A.c[2] * ns.v[q] + A.c[3] * d1.v[q] + A.c[4] * d2.v[q];
  } else {
    const V4<T> x0 = get(idx);
    const T d = A.diag[idx];
#pragma unroll
    for (int q = 0; q < 4; ++q) s.v[q] = d * x0.v[q];
    auto sub = [&](T wgt, int64_t m) {
      const V4<T> x = get(m);
#pragma unroll
      for (int q = 0; q < 4; ++q) s.v[q] -= wgt * x.v[q];
    };
    if (c.i > 0) sub(A.cx[idx - 1], idx - 1);
    if (c.i < N - 1) sub(A.cx[idx], idx + 1);
    if (c.j > 0) sub(A.cy[idx - N], idx - N);
    if (c.j < N - 1) sub(A.cy[idx], idx + N);
    if (KIND == ST_7PT) {
      const int64_t nn = (int64_t)N * N;
      if (c.l > 0) sub(A.cz[idx - nn], idx - nn);
      if (c.l < N - 1) sub(A.cz[idx], idx + nn);
    }
  }
  return s;
}

// Per-column block partials from four-column threads: thread (slot g, quad
// q) holds columns 4q .. 4q + 3 of its nodes.
__device__ __forceinline__ void block_col_partial4(const double (&v)[4], double (*sm)[MB], double* part) {
  const int g = threadIdx.x >> 3, q = threadIdx.x & 7;
#pragma unroll
  for (int j = 0; j < 4; ++j) sm[g][4 * q + j] = v[j];
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int gg = 0; gg < BT / 8; ++gg) s += sm[gg][threadIdx.x];
    part[(int64_t)blockIdx.x * MB + threadIdx.x] = s;
  }
}

constexpr int NPB = BT / 8;  // node rows per block step (8 threads per row)

// q = A p (FP64), four columns per thread, partials of p^T q
template <int KIND>
__global__ void __launch_bounds__(BT) k_b_spmv4(StencilView<double> A, const double* __restrict__ p,
                                               double* __restrict__ q, double* __restrict__ part) {
  __shared__ double sm[NPB][MB];
  const int qd = threadIdx.x & 7;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * NPB + (threadIdx.x >> 3); i < A.n; i += (int64_t)gridDim.x * NPB) {
    const V4<double> qi = stencil_apply4<KIND>(A, i, node_coord<KIND>(i, A.N),
                                               [&](int64_t m) { return ld4(p + m * MB + 4 * qd); });
    const int64_t e = i * MB + 4 * qd;
    const V4<double> pi = ld4(p + e);
    st4(q + e, qi);
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = fma(pi.v[j], qi.v[j], s[j]);
  }
  block_col_partial4(s, sm, part);
}

// zout = zin + w D^-1 (rT - A zin), four columns per thread
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_b_sweep4(StencilView<T> A, T omega, const T* __restrict__ rT,
                                                const T* __restrict__ zin, T* __restrict__ zout) {
  const int q = threadIdx.x & 7;
  for (int64_t i = (int64_t)blockIdx.x * NPB + (threadIdx.x >> 3); i < A.n; i += (int64_t)gridDim.x * NPB) {
    const V4<T> az = stencil_apply4<KIND>(A, i, node_coord<KIND>(i, A.N),
                                          [&](int64_t m) { return ld4(zin + m * MB + 4 * q); });
    const int64_t e = i * MB + 4 * q;
    const V4<T> z0 = ld4(zin + e), r0 = ld4(rT + e);
    const T di = omega * stencil_dinv<KIND>(A, i);
    V4<T> o;
#pragma unroll
    for (int j = 0; j < 4; ++j) o.v[j] = z0.v[j] + di * (r0.v[j] - az.v[j]);
    st4(zout + e, o);
  }
}

// Last post-sweep, four columns per thread: z (FP64) and the partials of
// r^T z and r^T z_old.
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_b_post4(StencilView<T> A, T omega, const T* __restrict__ rT,
                                               const T* __restrict__ zin, const double* __restrict__ r,
                                               double* __restrict__ zout, double* __restrict__ part) {
  __shared__ double sm[NPB][MB];
  const int q = threadIdx.x & 7;
  double s_rz[4] = {0.0, 0.0, 0.0, 0.0}, s_ro[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * NPB + (threadIdx.x >> 3); i < A.n; i += (int64_t)gridDim.x * NPB) {
    const V4<T> az = stencil_apply4<KIND>(A, i, node_coord<KIND>(i, A.N),
                                          [&](int64_t m) { return ld4(zin + m * MB + 4 * q); });
    const int64_t e = i * MB + 4 * q;
    const V4<T> z0 = ld4(zin + e), r0 = ld4(rT + e);
    const V4<double> ri = ld4(r + e), zo = ld4(zout + e);
    const T di = omega * stencil_dinv<KIND>(A, i);
    V4<double> zd;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      zd.v[j] = (double)(z0.v[j] + di * (r0.v[j] - az.v[j]));
      s_ro[j] = fma(ri.v[j], zo.v[j], s_ro[j]);
      s_rz[j] = fma(ri.v[j], zd.v[j], s_rz[j]);
    }
    st4(zout + e, zd);
  }
  block_col_partial4(s_rz, sm, part);
  __syncthreads();
  block_col_partial4(s_ro, sm, part + (int64_t)gridDim.x * MB);
}

// zout = zin + w D^-1 (rT - A zin)  (pre-sweeps 2..nu and post-sweeps)
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_b_sweep(StencilView<T> A, T omega, const T* __restrict__ rT,
                                               const T* __restrict__ zin, T* __restrict__ zout) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  for (int64_t i = w0; i < A.n; i += ws) {
    const T az = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return zin[m * MB + lane]; });
    const int64_t e = i * MB + lane;
    zout[e] = zin[e] + omega * stencil_dinv<KIND>(A, i) * (rT[e] - az);
  }
}

// Restriction of the residual after the pre-sweeps: per block, over its node
// tiles, C_b = P_t^T rho_t (k x 32) with rho = rT - A z.  The tile's rho
// (128 x 32) and its P rows, transposed to [node][k + 1], are staged in
// shared memory; thread (jb, cb) owns a 4 x 4 register tile of C.
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_b_restrict(StencilView<T> A, const T* __restrict__ rT,
                                                  const T* __restrict__ z, const T* __restrict__ P, int kst,
                                                  int k, int64_t ntiles, T* __restrict__ cpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kp = (k + 3) / 4 * 4 + 4;             // rows of whole 16-byte units, zero-padded
  T* ps = reinterpret_cast<T*>(smem_raw);         // [128][k + 4]
  T* rs = ps + (size_t)NLSP_TILE * kp;            // [128][36]
  const int jb = threadIdx.x >> 3, cb = threadIdx.x & 7;  // j = 4 jb .. (k <= 128), c = 4 cb ..
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    // rho rows of the tile's nodes (8 threads per node, four columns each)
    for (int wn = threadIdx.x >> 3; wn < NLSP_TILE; wn += BT / 8) {
      const int qd = threadIdx.x & 7;
      const int64_t i = t * NLSP_TILE + wn;
      V4<T> rho;
#pragma unroll
      for (int j = 0; j < 4; ++j) rho.v[j] = T(0);
      if (i < A.n) {
        const V4<T> az = stencil_apply4<KIND>(A, i, node_coord<KIND>(i, A.N),
                                              [&](int64_t m) { return ld4(z + m * MB + 4 * qd); });
        const V4<T> r0 = ld4(rT + i * MB + 4 * qd);
#pragma unroll
        for (int j = 0; j < 4; ++j) rho.v[j] = r0.v[j] - az.v[j];
      }
      st4(rs + wn * 36 + 4 * qd, rho);
    }
    // P tile transposed: ps[node][j], columns k .. kp - 1 zero
    const T* src = P + t * kst * NLSP_TILE;  // the first k of the tile's kst columns
    for (int e = threadIdx.x; e < kp * NLSP_TILE; e += BT) {
      const int j = e / NLSP_TILE, wn = e % NLSP_TILE;
      ps[wn * kp + j] = j < k ? src[e] : T(0);
    }
    __syncthreads();
    if (4 * jb < k) {
      for (int wn = 0; wn < NLSP_TILE; ++wn) {
        // k is a multiple of 4 here or the tail columns of ps are zero
        const V4<T> pa = ld4(ps + wn * kp + 4 * jb), rb = ld4(rs + wn * 36 + 4 * cb);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += pa.v[a] * rb.v[b];
      }
    }
  }
  if (4 * jb < k) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * jb + a < k) cpart[((int64_t)blockIdx.x * k + 4 * jb + a) * MB + 4 * cb + b] = acc[a][b];
  }
}

// C = sum of the restriction partials in block order (one thread per entry
// of the k x 32 block), FP64.
template <typename T>
__global__ void k_b_csum(const T* __restrict__ cpart, int nb, int k, double* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * MB) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += (double)cpart[(int64_t)b * k * MB + e];
  C[e] = s;
}

// E = A_c^-1 C (k x 32), one thread per entry.
template <typename T>
__global__ void k_b_coarse(const double* __restrict__ C, int k, const double* __restrict__ Ainv, T* __restrict__ E) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * MB) return;
  const int i = e / MB, c = e % MB;
  double s = 0.0;
  for (int j = 0; j < k; ++j) s = fma(Ainv[(int64_t)j * k + i], C[j * MB + c], s);
  E[e] = (T)s;
}

// z += P E: the block's two halves take one node tile each; a thread owns
// its node's whole row (32 columns).  P's tile rows are read once, coalesced
// along the nodes, sixteen loads in flight; E is read from shared memory as
// 16-byte vectors.
template <typename T>
__global__ void __launch_bounds__(BT) k_b_prolong(const T* __restrict__ P, int kst, int k, int64_t n,
                                                 const T* __restrict__ E, T* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* es = reinterpret_cast<T*>(smem_raw);  // [k][32]
  for (int e = threadIdx.x; e < k * MB; e += BT) es[e] = E[e];
  __syncthreads();
  const int node = threadIdx.x & (NLSP_TILE - 1), half = threadIdx.x >> 7;
  const int64_t ntiles = (n + NLSP_TILE - 1) / NLSP_TILE;
  for (int64_t t = 2 * (int64_t)blockIdx.x + half; t < ntiles; t += 2 * (int64_t)gridDim.x) {
    const int64_t i = t * NLSP_TILE + node;
    const T* pc = P + t * kst * NLSP_TILE + node;
    T acc[MB];
#pragma unroll
    for (int c = 0; c < MB; ++c) acc[c] = T(0);
#pragma unroll 16
    for (int j = 0; j < k; ++j) {
      const T pv = pc[(int64_t)j * NLSP_TILE];
      const T* ej = es + j * MB;
#pragma unroll
      for (int c4 = 0; c4 < MB / 4; ++c4) {
        const V4<T> e4 = ld4(ej + 4 * c4);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[4 * c4 + c] += pv * e4.v[c];
      }
    }
    if (i < n) {
      T* zr = z + i * MB;
#pragma unroll
      for (int c4 = 0; c4 < MB / 4; ++c4) {
        V4<T> zv = ld4(zr + 4 * c4);
#pragma unroll
        for (int c = 0; c < 4; ++c) zv.v[c] += acc[4 * c4 + c];
        st4(zr + 4 * c4, zv);
      }
    }
  }
}

// ---- tensor-core (tcgen05, kind::tf32) restriction and prolongation ------
// Operands live in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, (row / 8, k / 4) -> ((row / 8) *
// (kcols / 4) + k / 4) * 128 bytes, row r of a core matrix at r * 16.  One
// instruction is M = 128, N = 32, K = 8 (two core matrices along K); the
// accumulator is 32 TMEM columns over the 128 lanes.
namespace tc {

__host__ __device__ inline unsigned core_off(int row, int kk, int kcols) {
  return (unsigned)(((row >> 3) * (kcols >> 2) + (kk >> 2)) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}

__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFF) >> 4) | ((unsigned long long)(lbo >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void ld16(unsigned ta, float (&v)[16]) { tmem::Io<16>::ld(ta, v); }

// x = hi + lo with hi rounded to TF32 (round to nearest, ties away) and lo
// the remainder: the three-product split of Ootomo & Yokota (2022,
// "Recovering single precision accuracy from Tensor Cores while surpassing
// the FP32 theoretical peak performance") keeps FP32-level accuracy.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  unsigned h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

__device__ __forceinline__ void split4(const float4 v, float4& hi, float4& lo) {
  split_tf32(v.x, hi.x, lo.x);
  split_tf32(v.y, hi.y, lo.y);
  split_tf32(v.z, hi.z, lo.z);
  split_tf32(v.w, hi.w, lo.w);
}

// D [+]= A_hi B_hi + A_hi B_lo + A_lo B_hi, `ksteps` MMA steps of K = 8 from
// the operand start addresses (A: 128 rows, B: 32 rows, canonical K-major
// layouts with M/N-group strides a_sbo / b_sbo); one commit for all.
__device__ __forceinline__ void mma3_128x32(unsigned tmem_d, unsigned ah, unsigned al, unsigned a_sbo, unsigned bh,
                                            unsigned bl, unsigned b_sbo, int ksteps, bool accumulate,
                                            uint64_t* bar) {
  constexpr unsigned idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(MB >> 3) << 17) | ((128u >> 4) << 24);
  const unsigned as[3] = {al, ah, ah}, bs[3] = {bh, bl, bh};  // small terms first
  for (int pr = 0; pr < 3; ++pr)
    for (int ks = 0; ks < ksteps; ++ks) {
      const unsigned long long ad = sdesc(as[pr] + ks * 256, 128, a_sbo);
      const unsigned long long bd = sdesc(bs[pr] + ks * 256, 128, b_sbo);
      const unsigned acc = (accumulate || pr > 0 || ks > 0) ? 1u : 0u;
      asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                   "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                   "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                   : "memory");
    }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tma::smem_addr(bar))
               : "memory");
}

}  // namespace tc

constexpr int TCK = 64;  // K chunk of the tensor-core contractions (2 CTAs per SM fit)

// Restriction on tensor cores (FP32 preconditioner): per block, over its
// tiles, D[j][c] += sum over the tile's nodes of P[node][j] rho[node][c],
// accumulated in TMEM across tiles; A = P_t^T (rows j, zero beyond k), B =
// rho_t^T (rows c), K = the tile's nodes in two chunks of 64.  Each operand
// is split into TF32 hi + lo parts (three products).
template <int KIND>
__global__ void __launch_bounds__(BT, 2) k_b_restrict_tc(StencilView<float> A, const float* __restrict__ rT,
                                                        const float* __restrict__ z, const float* __restrict__ P,
                                                        int kst, int k, int64_t ntiles, float* __restrict__ cpart,
                                                        BlockState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sa = smem_raw;               // A_hi: 128 x 64 tf32 (32 KB)
  unsigned char* sal = sa + 128 * TCK * 4;    // A_lo
  unsigned char* sb = sal + 128 * TCK * 4;    // B_hi: 32 x 64 (8 KB)
  unsigned char* sbl = sb + 32 * TCK * 4;     // B_lo
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tbase_s;
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_barrier_init();
    bad = 0;
  }
  if (warp == 0) tmem::alloc(&tbase_s, 32);
  for (int e = tid; e < 128 * TCK; e += BT) {  // rows j >= k of A stay zero
    const int j = e / TCK, nd = e % TCK;
    if (j >= k) {
      *reinterpret_cast<float*>(sa + tc::core_off(j, nd, TCK)) = 0.0f;
      *reinterpret_cast<float*>(sal + tc::core_off(j, nd, TCK)) = 0.0f;
    }
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const unsigned td = tbase_s;
  const unsigned sbo = (TCK / 4) * 128;
  unsigned phase = 0;
  bool first = true;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int h = 0; h < NLSP_TILE / TCK; ++h) {
      // rho of the chunk's 64 nodes -> B (8 threads per node, four columns each)
      for (int wn = tid >> 3; wn < TCK; wn += BT / 8) {
        const int qd = tid & 7;
        const int64_t i = t * NLSP_TILE + h * TCK + wn;
        V4<float> rho;
#pragma unroll
        for (int j = 0; j < 4; ++j) rho.v[j] = 0.0f;
        if (i < A.n) {
          const V4<float> az = stencil_apply4<KIND>(A, i, node_coord<KIND>(i, A.N),
                                                    [&](int64_t m) { return ld4(z + m * MB + 4 * qd); });
          const V4<float> r0 = ld4(rT + i * MB + 4 * qd);
#pragma unroll
          for (int j = 0; j < 4; ++j) rho.v[j] = r0.v[j] - az.v[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float hi, lo;
          tc::split_tf32(rho.v[j], hi, lo);
          *reinterpret_cast<float*>(sb + tc::core_off(4 * qd + j, wn, TCK)) = hi;
          *reinterpret_cast<float*>(sbl + tc::core_off(4 * qd + j, wn, TCK)) = lo;
        }
      }
      // the chunk's P rows -> A (row j, K = node); 16-byte chunks of four nodes
      const float* src = P + t * kst * NLSP_TILE + h * TCK;
      for (int e = tid; e < k * (TCK / 4); e += BT) {
        const int j = e % k, q = e / k;  // j fastest across the threads (fewer bank conflicts)
        const float4 v = *reinterpret_cast<const float4*>(src + (int64_t)j * NLSP_TILE + 4 * q);
        float4 hi, lo;
        tc::split4(v, hi, lo);
        *reinterpret_cast<float4*>(sa + tc::core_off(j, 4 * q, TCK)) = hi;
        *reinterpret_cast<float4*>(sal + tc::core_off(j, 4 * q, TCK)) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0)
        tc::mma3_128x32(td, tma::smem_addr(sa), tma::smem_addr(sal), sbo, tma::smem_addr(sb), tma::smem_addr(sbl),
                        sbo, TCK / 8, !first, &bar);
      if (!tma::mbar_wait(&bar, phase)) bad = 1;  // the operands are reused by the next chunk
      phase ^= 1u;
      first = false;
      tmem::fence_after_sync();
      __syncthreads();
    }
  }
  // D -> partials (warps 0-3: columns 0-15, warps 4-7: columns 16-31)
  if (!first) {
    float v[16];
    tc::ld16(td + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(16 * (warp >> 2)), v);
    const int j = 32 * (warp & 3) + lane;
    if (j < k) {
#pragma unroll
      for (int c = 0; c < 16; ++c) cpart[((int64_t)blockIdx.x * k + j) * MB + 16 * (warp >> 2) + c] = v[c];
    }
  } else {
    for (int e = tid; e < k * MB; e += BT) cpart[(int64_t)blockIdx.x * k * MB + e] = 0.0f;
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (warp == 0) tmem::dealloc(td, 32);
  if (tid == 0 && bad) atomicExch(&st->err, 1);
}

// Prolongation on tensor cores (FP32): per tile, D[node][c] = sum_j
// P[node][j] E[j][c] with A = the P tile (rows = nodes, K = j, in chunks of
// 64) and B = E^T (rows c, all of K resident), then z += D.  Operands split
// into TF32 hi + lo parts (three products).
__global__ void __launch_bounds__(BT, 2) k_b_prolong_tc(const float* __restrict__ P, int kst, int k, int64_t n,
                                                       const float* __restrict__ E, float* __restrict__ z,
                                                       BlockState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kp = (k + 7) / 8 * 8;              // K padded to whole MMA steps
  const int kc = kp < TCK ? kp : TCK;          // chunk width
  unsigned char* sa = smem_raw;                // A_hi: 128 x kc
  unsigned char* sal = sa + 128 * kc * 4;      // A_lo
  unsigned char* sb = sal + 128 * kc * 4;      // B_hi: 32 x kp
  unsigned char* sbl = sb + 32 * kp * 4;       // B_lo
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned tbase_s;
  __shared__ int bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_barrier_init();
    bad = 0;
  }
  if (warp == 0) tmem::alloc(&tbase_s, 32);
  for (int e = tid; e < MB * kp; e += BT) {  // B = E^T, zero beyond k
    const int c = e % MB, j = e / MB;
    float hi = 0.0f, lo = 0.0f;
    if (j < k) tc::split_tf32(E[j * MB + c], hi, lo);
    *reinterpret_cast<float*>(sb + tc::core_off(c, j, kp)) = hi;
    *reinterpret_cast<float*>(sbl + tc::core_off(c, j, kp)) = lo;
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const unsigned td = tbase_s;
  const unsigned a_sbo = (unsigned)(kc / 4) * 128, b_sbo = (unsigned)(kp / 4) * 128;
  unsigned phase = 0;
  const int64_t ntiles = (n + NLSP_TILE - 1) / NLSP_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const float* src = P + t * kst * NLSP_TILE;
    for (int j0 = 0; j0 < kp; j0 += kc) {
      for (int e = tid; e < kc * NLSP_TILE; e += BT) {  // coalesced along the nodes
        const int jj = e / NLSP_TILE, nd = e % NLSP_TILE, j = j0 + jj;
        float hi = 0.0f, lo = 0.0f;
        if (j < k) tc::split_tf32(src[(int64_t)j * NLSP_TILE + nd], hi, lo);
        *reinterpret_cast<float*>(sa + tc::core_off(nd, jj, kc)) = hi;
        *reinterpret_cast<float*>(sal + tc::core_off(nd, jj, kc)) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        const unsigned boff = (unsigned)(j0 / 4) * 128;  // K offset of the chunk in B
        tc::mma3_128x32(td, tma::smem_addr(sa), tma::smem_addr(sal), a_sbo, tma::smem_addr(sb) + boff,
                        tma::smem_addr(sbl) + boff, b_sbo, kc / 8, j0 > 0, &bar);
      }
      if (!tma::mbar_wait(&bar, phase)) bad = 1;
      phase ^= 1u;
      tmem::fence_after_sync();
      __syncthreads();  // A is restaged by the next chunk
    }
    float v[16];
    tc::ld16(td + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(16 * (warp >> 2)), v);
    const int64_t i = t * NLSP_TILE + 32 * (warp & 3) + lane;
    if (i < n) {
      float* zr = z + i * MB + 16 * (warp >> 2);
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        V4<float> zv = ld4(zr + 4 * c4);
#pragma unroll
        for (int c = 0; c < 4; ++c) zv.v[c] += v[4 * c4 + c];
        st4(zr + 4 * c4, zv);
      }
    }
    tmem::fence_before_sync();
    __syncthreads();  // D is overwritten by the next tile
    tmem::fence_after_sync();
  }
  if (warp == 0) tmem::dealloc(td, 32);
  if (tid == 0 && bad) atomicExch(&st->err, 1);
}

// ---- reduced-precision restriction and prolongation (block_lp.cuh) -------
constexpr int LP_NS = 4;  // stages of the operand ring

// Restriction with TF32 / BF16 operands: per block, over its tiles' 64-node
// chunks, D[j][c] += sum_node R[j][node] rho[node][c] in TMEM, with R the
// repacked chunk of P (bulk-copied into a ring of LP_NS stages) and rho =
// rT - A z computed by the threads into one of two B buffers.  Thread 0
// issues the MMAs of a chunk once its copy has landed and commits them to the
// stage's and the B buffer's "free" barriers; it refills the stage of the
// previous chunk when that chunk's MMAs are done.  The block's r x 32 result
// goes to cpart (FP32).
template <int KIND, int OP, int NT>
__global__ void __launch_bounds__(NT) k_b_restrict_lp(StencilView<float> A, const float* __restrict__ rT,
                                                      const float* __restrict__ z,
                                                      const unsigned char* __restrict__ Rc, int k, int64_t ntiles,
                                                      float* __restrict__ cpart, int ns, BlockState* st) {
  using Sx = typename lp::Op<OP>::S;
  constexpr int ES = lp::Op<OP>::ES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rr = lp::rows_r(k);
  const unsigned a_bytes = 128u * lp::RCH * ES;           // one A stage (128 rows)
  const unsigned chunk_bytes = (unsigned)rr * lp::RCH * ES;  // rows that the copy fills
  const unsigned b_bytes = (unsigned)lp::MBC * lp::RCH * ES;
  unsigned char* sa = smem_raw;                            // ns <= LP_NS stages
  unsigned char* sb = smem_raw + (size_t)ns * a_bytes;     // 2 B buffers
  __shared__ __align__(8) uint64_t full[LP_NS], afree[LP_NS], bfree[2];
  __shared__ unsigned tbase_s;
  __shared__ int bad, nmma;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int nchunk = (int)(my_tiles * 2);
  auto chunk_src = [&](int c) {  // chunk c of this block: tile blockIdx.x + (c / 2) gridDim.x, half c % 2
    const int64_t t = blockIdx.x + (int64_t)(c >> 1) * gridDim.x;
    return Rc + (size_t)(t * 2 + (c & 1)) * chunk_bytes;
  };
  if (tid == 0) {
    for (int q = 0; q < LP_NS; ++q) {
      tma::mbar_init(&full[q], 1);
      tma::mbar_init(&afree[q], 1);
    }
    tma::mbar_init(&bfree[0], 1);
    tma::mbar_init(&bfree[1], 1);
    tma::fence_barrier_init();
    bad = 0;
    nmma = 0;
  }
  // rows rr .. 127 of every stage stay zero (the copies fill rows < rr)
  for (unsigned e = tid; e < (unsigned)ns * (a_bytes - chunk_bytes) / 16; e += NT) {
    const unsigned per = (a_bytes - chunk_bytes) / 16;
    *reinterpret_cast<uint4*>(sa + (size_t)(e / per) * a_bytes + chunk_bytes + (size_t)(e % per) * 16) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  if (warp == 0) tmem::alloc(&tbase_s, 32);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const unsigned td = tbase_s;
  if (tid == 0)
    for (int c = 0; c < ns && c < nchunk; ++c) {
      tma::mbar_arrive_expect_tx(&full[c], chunk_bytes);
      tma::bulk_g2s(sa + (size_t)c * a_bytes, chunk_src(c), chunk_bytes, &full[c]);
    }
  const unsigned a_sbo = (lp::RCH / lp::Op<OP>::EPC) * 128, b_sbo = a_sbo;
  const int ksteps = lp::RCH / lp::Op<OP>::KSTEP;
  int q = 0;
  for (; q < nchunk; ++q) {
    const int b = q & 1;
    if (q >= 2 && !tma::mbar_wait(&bfree[b], (unsigned)(((q - 2) >> 1) & 1))) bad = 1;
    __syncthreads();
    if (bad) break;
    // rho of the chunk's 64 nodes -> B buffer b (8 threads per node, four columns each)
    const int64_t t = blockIdx.x + (int64_t)(q >> 1) * gridDim.x;
    unsigned char* bb = sb + (size_t)b * b_bytes;
    // both node-quads of a thread are evaluated before either is stored, so
    // that their loads are in flight together
    constexpr int PER = lp::RCH / (NT / 8);
    static_assert(PER >= 1 && PER * (NT / 8) == lp::RCH, "a chunk splits evenly over the block");
    const int qd = tid & 7;
    V4<float> rho[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int wn = (tid >> 3) + u * (NT / 8);
      const int64_t i = t * NLSP_TILE + (q & 1) * lp::RCH + wn;
#pragma unroll
      for (int j = 0; j < 4; ++j) rho[u].v[j] = 0.0f;
      if (i < A.n) {
        const V4<float> az = stencil_apply4<KIND>(A, i, node_coord<KIND>(i, A.N),
                                                  [&](int64_t m) { return ld4(z + m * MB + 4 * qd); });
        const V4<float> r0 = ld4(rT + i * MB + 4 * qd);
#pragma unroll
        for (int j = 0; j < 4; ++j) rho[u].v[j] = r0.v[j] - az.v[j];
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int wn = (tid >> 3) + u * (NT / 8);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        *reinterpret_cast<Sx*>(bb + lp::off<OP>(4 * qd + j, wn, lp::RCH)) = lp::Op<OP>::cvt(rho[u].v[j]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      const int s = q % ns;
      if (!tma::mbar_wait(&full[s], (unsigned)((q / ns) & 1))) {
        bad = 1;
      } else {
        tmem::fence_after_sync();
        lp::mma_run<OP>(td, tma::smem_addr(sa + (size_t)s * a_bytes), a_sbo, tma::smem_addr(bb), b_sbo, ksteps, q > 0);
        lp::commit(&afree[s]);
        lp::commit(&bfree[b]);
        nmma = q + 1;
        // refill the stage of an earlier chunk once its MMAs are done: two
        // chunks back when the ring has room (its MMAs finished long ago, so
        // the wait does not hold up this thread's warp), else the previous one
        const int pc = q - (ns >= 3 ? 2 : 1);
        if (pc >= 0 && pc + ns < nchunk) {
          const int ps = pc % ns;
          if (!tma::mbar_wait(&afree[ps], (unsigned)((pc / ns) & 1))) {
            bad = 1;
          } else {
            tma::mbar_arrive_expect_tx(&full[ps], chunk_bytes);
            tma::bulk_g2s(sa + (size_t)ps * a_bytes, chunk_src(pc + ns), chunk_bytes, &full[ps]);
          }
        }
      }
    }
  }
  // every MMA issued so far is complete once the last one's commit arrived
  // (a commit tracks all earlier MMAs of the thread); copies still in
  // flight after a failure are drained (bounded) before leaving
  __syncthreads();
  const int issued = nmma;  // chunks whose MMAs were issued (all of them unless a wait gave up)
  if (issued > 0 && !tma::mbar_wait(&bfree[(issued - 1) & 1], (unsigned)(((issued - 1) >> 1) & 1))) bad = 1;
  __syncthreads();
  if (tid == 0 && bad) {
    // copies were issued for chunks below max(ns, issued + ns - lag) and
    // consumed below `issued`: wait (bounded) for the rest to land
    const int hi = min(nchunk, max(ns, issued + ns - (ns >= 3 ? 2 : 1)));
    for (int c = issued; c < hi; ++c) tma::mbar_wait(&full[c % ns], (unsigned)((c / ns) & 1));
    atomicExch(&st->err, 1);
  }
  tmem::fence_after_sync();
  if (!bad && issued > 0 && warp < 8) {  // warps 0-7 read the 128 lanes x 32 columns of D
    float v[16];
    tc::ld16(td + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(16 * (warp >> 2)), v);
    const int j = 32 * (warp & 3) + lane;
    if (j < k) {
#pragma unroll
      for (int c = 0; c < 16; ++c) cpart[((int64_t)blockIdx.x * k + j) * MB + 16 * (warp >> 2) + c] = v[c];
    }
  } else if (bad || issued == 0) {
    for (int e = tid; e < k * MB; e += NT) cpart[(int64_t)blockIdx.x * k * MB + e] = 0.0f;
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (warp == 0) tmem::dealloc(td, 32);
}

// Prolongation with TF32 / BF16 operands: per tile, D = Q_t E (128 nodes x
// 32 columns) with Q_t the repacked tile of P (bulk-copied into a ring of
// LP_NS stages) and B = E^T (32 x r, converted once per block), then
// z += D.  Two TMEM accumulators alternate, so thread 0 issues the MMAs of
// tile i + 1 before the block adds tile i's result to z.
template <int OP>
__global__ void __launch_bounds__(BT) k_b_prolong_lp(const unsigned char* __restrict__ Qc, int k, int64_t n,
                                                     const float* __restrict__ E, float* __restrict__ z,
                                                     int ns, BlockState* st) {
  using Sx = typename lp::Op<OP>::S;
  constexpr int ES = lp::Op<OP>::ES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int kq = lp::kcols_q(k);
  const unsigned tile_bytes = (unsigned)NLSP_TILE * kq * ES;
  unsigned char* sa = smem_raw;                             // ns <= LP_NS stages
  unsigned char* sbm = smem_raw + (size_t)ns * tile_bytes;   // E^T: 32 x kq
  __shared__ __align__(8) uint64_t full[LP_NS], afree[LP_NS], dfull[2];
  __shared__ unsigned tbase_s;
  __shared__ int bad, nmma;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (n + NLSP_TILE - 1) / NLSP_TILE;
  const int nt = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  auto tile_src = [&](int i) { return Qc + (size_t)(blockIdx.x + (int64_t)i * gridDim.x) * tile_bytes; };
  if (tid == 0) {
    for (int q = 0; q < LP_NS; ++q) {
      tma::mbar_init(&full[q], 1);
      tma::mbar_init(&afree[q], 1);
    }
    tma::mbar_init(&dfull[0], 1);
    tma::mbar_init(&dfull[1], 1);
    tma::fence_barrier_init();
    bad = 0;
    nmma = 0;
  }
  for (int e = tid; e < lp::MBC * kq; e += BT) {  // B = E^T, zero beyond k
    const int c = e % lp::MBC, j = e / lp::MBC;
    *reinterpret_cast<Sx*>(sbm + lp::off<OP>(c, j, kq)) = lp::Op<OP>::cvt(j < k ? E[j * MB + c] : 0.0f);
  }
  if (warp == 0) tmem::alloc(&tbase_s, 64);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const unsigned td = tbase_s;
  const unsigned a_sbo = (unsigned)(kq / lp::Op<OP>::EPC) * 128, b_sbo = a_sbo;
  const int ksteps = kq / lp::Op<OP>::KSTEP;
  // thread 0: MMAs of tile i into accumulator i % 2 once its copy landed,
  // then the refill of the stage of tile i - 1 (whose MMAs are done)
  auto issue = [&](int i) {
    const int s = i % ns;
    if (!tma::mbar_wait(&full[s], (unsigned)((i / ns) & 1))) {
      bad = 1;
      return;
    }
    tmem::fence_after_sync();
    lp::mma_run<OP>(td + (unsigned)(32 * (i & 1)), tma::smem_addr(sa + (size_t)s * tile_bytes), a_sbo,
                    tma::smem_addr(sbm), b_sbo, ksteps, false);
    lp::commit(&afree[s]);
    lp::commit(&dfull[i & 1]);
    nmma = i + 1;
    const int pi = i - 1;
    if (pi >= 0 && pi + ns < nt) {
      const int ps = pi % ns;
      if (!tma::mbar_wait(&afree[ps], (unsigned)((pi / ns) & 1))) {
        bad = 1;
        return;
      }
      tma::mbar_arrive_expect_tx(&full[ps], tile_bytes);
      tma::bulk_g2s(sa + (size_t)ps * tile_bytes, tile_src(pi + ns), tile_bytes, &full[ps]);
    }
  };
  if (tid == 0) {
    for (int i = 0; i < ns && i < nt; ++i) {
      tma::mbar_arrive_expect_tx(&full[i], tile_bytes);
      tma::bulk_g2s(sa + (size_t)i * tile_bytes, tile_src(i), tile_bytes, &full[i]);
    }
    if (nt > 0) issue(0);
  }
  for (int i = 0; i < nt; ++i) {
    __syncthreads();  // accumulator (i + 1) % 2 was drained by the previous iteration
    // the z rows this thread updates are loaded before the wait for the
    // accumulator (they do not depend on it)
    const int64_t node = (blockIdx.x + (int64_t)i * gridDim.x) * NLSP_TILE + 32 * (warp & 3) + lane;
    float* zr = z + node * MB + 16 * (warp >> 2);
    V4<float> zv[4];
    if (node < n) {
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) zv[c4] = ld4(zr + 4 * c4);
    }
    if (tid == 0 && !bad && i + 1 < nt) issue(i + 1);
    if (!tma::mbar_wait(&dfull[i & 1], (unsigned)((i >> 1) & 1))) bad = 1;
    __syncthreads();
    if (bad) break;
    tmem::fence_after_sync();
    float v[16];
    tc::ld16(td + (unsigned)(32 * (i & 1)) + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(16 * (warp >> 2)), v);
    if (node < n) {
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
#pragma unroll
        for (int c = 0; c < 4; ++c) zv[c4].v[c] += v[4 * c4 + c];
        st4(zr + 4 * c4, zv[c4]);
      }
    }
    tmem::fence_before_sync();
  }
  __syncthreads();
  if (tid == 0 && bad) {
    // drain: the last issued MMAs, then the copies issued beyond them
    const int issued = nmma;
    if (issued > 0) tma::mbar_wait(&afree[(issued - 1) % ns], (unsigned)(((issued - 1) / ns) & 1));
    const int hi = min(nt, max(ns, issued + ns - 1));
    for (int c = issued; c < hi; ++c) tma::mbar_wait(&full[c % ns], (unsigned)((c / ns) & 1));
    atomicExch(&st->err, 1);
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (warp == 0) tmem::dealloc(td, 64);
}

// Last post-sweep: z = zin + w D^-1 (rT - A zin) stored in FP64, with the
// per-column partials of r^T z and r^T z_old (flexible beta).
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_b_post(StencilView<T> A, T omega, const T* __restrict__ rT,
                                              const T* __restrict__ zin, const double* __restrict__ r,
                                              double* __restrict__ zout, double* __restrict__ part) {
  __shared__ double sm[BW][MB];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  double s_rz = 0.0, s_ro = 0.0;
  for (int64_t i = w0; i < A.n; i += ws) {
    const T az = stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return zin[m * MB + lane]; });
    const int64_t e = i * MB + lane;
    const double zd = (double)(zin[e] + omega * stencil_dinv<KIND>(A, i) * (rT[e] - az));
    const double ri = r[e];
    s_ro = fma(ri, zout[e], s_ro);  // the previous z
    zout[e] = zd;
    s_rz = fma(ri, zd, s_rz);
  }
  block_col_partial(s_rz, sm, part);
  __syncthreads();
  block_col_partial(s_ro, sm, part + (int64_t)gridDim.x * MB);
}

enum BlockStage { BS_INIT = 0, BS_PQ, BS_RR, BS_RZ };

// Per-column scalar step from the block partials (one warp, lane = column).
// 32 x 32 threads: group g adds blocks g, g + 32, ... of column c, then warp
// 0 adds the 32 group sums in order (deterministic).
__global__ void __launch_bounds__(1024) k_b_scalars(const double* __restrict__ part, int nb, BlockState* st,
                                                    int stage) {
  __shared__ double gs[2][32][MB];
  const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
  const bool two = stage == BS_RZ && st->flexible;
  double a0 = 0.0, a1 = 0.0;
  for (int b = g; b < nb; b += 32) {
    a0 += part[(int64_t)b * MB + c];
    if (two) a1 += part[(int64_t)(nb + b) * MB + c];
  }
  gs[0][g][c] = a0;
  gs[1][g][c] = a1;
  __syncthreads();
  if (g != 0) return;
  const int t = st->t;  // read before any lane may advance it
  __syncwarp();
  double s0 = 0.0, s1 = 0.0;
  for (int q = 0; q < 32; ++q) {
    s0 += gs[0][q][c];
    s1 += gs[1][q][c];
  }
  const bool active = c < st->m && !st->done[c];
  switch (stage) {
    case BS_INIT:  // s0 = b^T b
      st->bb[c] = s0;
      st->rr[c] = s0;
      st->tol2bn[c] = 0.0;
      st->iter[c] = 0;
      st->status[c] = (int)NLSP_OK;
      st->alpha[c] = 0.0;
      st->beta[c] = 0.0;
      st->done[c] = c >= st->m ? 1 : 0;
      if (c < st->m) {
        if (s0 == 0.0) st->done[c] = 1;
        else if (!isfinite(s0)) { st->status[c] = (int)NLSP_ERR_BREAKDOWN; st->done[c] = 1; }
      }
      break;
    case BS_PQ:  // s0 = p^T q; starts iteration t + 1
      if (c == 0) st->t = t + 1;
      if (active) {
        st->iter[c] = t + 1;
        if (!(s0 > 0.0) || !isfinite(s0)) {
          st->status[c] = (int)NLSP_ERR_BREAKDOWN;
          st->done[c] = 1;
          st->alpha[c] = 0.0;
        } else {
          st->alpha[c] = st->rz[c] / s0;
        }
      } else {
        st->alpha[c] = 0.0;
      }
      break;
    case BS_RR:  // s0 = r^T r after the update
      if (active) {
        st->rr[c] = s0;
        if (!isfinite(s0)) { st->status[c] = (int)NLSP_ERR_BREAKDOWN; st->done[c] = 1; }
        else if (s0 <= st->tol2bn[c]) st->done[c] = 1;
        else if (t >= st->maxit) { st->status[c] = (int)NLSP_NOT_CONVERGED; st->done[c] = 1; }
      }
      break;
    case BS_RZ:  // s0 = r^T z, s1 = r^T z_old
      if (active) {
        if (!(s0 > 0.0) || !isfinite(s0)) {
          st->status[c] = (int)NLSP_ERR_BREAKDOWN;
          st->done[c] = 1;
        } else {
          st->beta[c] = t == 0 ? 0.0 : (s0 - (st->flexible ? s1 : 0.0)) / st->rz[c];
          st->rz[c] = s0;
        }
      }
      if (!active) st->beta[c] = 0.0;
      break;
    default:
      break;
  }
  __syncwarp();
  const unsigned pend = __ballot_sync(0xffffffffu, c < st->m && !st->done[c]);
  if (c == 0) st->all_done = pend == 0u;
}

__global__ void k_b_set_tol(BlockState* st, double tol) {
  const int c = threadIdx.x;
  st->tol2bn[c] = tol * tol * st->bb[c];
}

// column-major (ld) <-> node rows of 32
__global__ void k_b_gather(const double* __restrict__ src, int64_t ld, int m, int64_t n, double* __restrict__ dst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * MB; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / MB;
    const int c = (int)(e % MB);
    dst[e] = c < m ? src[(int64_t)c * ld + i] : 0.0;
  }
}

__global__ void k_b_scatter(const double* __restrict__ src, int m, int64_t n, double* __restrict__ dst, int64_t ld) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * m; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n);
    const int64_t i = e % n;
    dst[(int64_t)c * ld + i] = src[i * MB + c];
  }
}

// true residual partials: ||b - A x||^2 per column
template <int KIND>
__global__ void __launch_bounds__(BT) k_b_true(StencilView<double> A, const double* __restrict__ b,
                                              const double* __restrict__ x, double* __restrict__ part) {
  __shared__ double sm[BW][MB];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  double s = 0.0;
  for (int64_t i = w0; i < A.n; i += ws) {
    const double ri =
        b[i * MB + lane] - stencil_apply<KIND>(A, i, node_coord<KIND>(i, A.N), [&](int64_t m) { return x[m * MB + lane]; });
    s = fma(ri, ri, s);
  }
  block_col_partial(s, sm, part);
}

__global__ void k_b_true_fin(const double* __restrict__ part, int nb, BlockState* st) {
  const int c = threadIdx.x;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * MB + c];
  st->true_rr[c] = s;
}

__global__ void k_b_dot_init(const double* __restrict__ b, int64_t n, double* __restrict__ part) {
  __shared__ double sm[BW][MB];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  double s = 0.0;
  for (int64_t i = w0; i < n; i += ws) s = fma(b[i * MB + lane], b[i * MB + lane], s);
  block_col_partial(s, sm, part);
}

}  // namespace

// ============================================================================
// Host side
// ============================================================================
namespace {

template <typename T>
const StencilView<T>& bview(const nlsp_op* A) {
  return *reinterpret_cast<const StencilView<T>*>(sizeof(T) == 8 ? (const void*)&A->v64 : (const void*)&A->v32);
}

#include "block_cg.cuh"

template <int KIND, typename T>
struct BlockSolver {
  // Breakdown-free block CG (block_cg.cuh) on the block workspace: every
  // iteration Q = A P, the Gram products and small solves for alpha and beta,
  // X and R updates, Z = M R through the block preconditioner kernels, and the
  // re-orthonormalised search block.  The host reads the state word after each
  // iteration (one small copy).
  template <typename Prec>
  static nlsp_status block_cg(nlsp_ctx* ctx, const nlsp_prec* M, int m, const double* B, int64_t ldb, double* X,
                              int64_t ldx, const nlsp_solve_params* prm, nlsp_solve_info* infos, double* b,
                              double* x, double* r, double* P, double* Q, double* z, T* rT, T* za, BlockState* bst,
                              Prec& precond_rest, int nb, int ge) {
    cudaStream_t s = ctx->stream;
    const nlsp_op* A = M->A;
    const int64_t n = A->n;
    const StencilView<T>& AT = bview<T>(A);
    const T omega = (T)M->omega;
    const int nw = nb * BW;  // warp partials of the Gram products (grid nb)
    const size_t nv = (size_t)n * MB;
    DevBuf wbuf;
    NLSP_TRY(wbuf.alloc(sizeof(double) * (nv + (size_t)nw * MB * MB + 6 * MB * MB) + sizeof(BcgState) + 1024));
    double* W = wbuf.as<double>();
    double* part = W + nv;
    double* G1 = part + (size_t)nw * MB * MB;
    double* G2 = G1 + MB * MB;
    double* Dfac = G2 + MB * MB;
    double* coef = Dfac + MB * MB;
    double* G3 = coef + MB * MB;
    BcgState* st = (BcgState*)(G3 + 2 * MB * MB);
    BcgState h;
    memset(&h, 0, sizeof(h));
    h.m = m;
    h.maxit = prm->maxit;
    NLSP_CUDA(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    int launches = 0;
    auto gram = [&](const double* Xa, const double* Yb, double* out) {
      k_bcg_gram<<<nb, BT, 0, s>>>(Xa, Yb, n, part);
      k_bcg_sum<<<MB, 256, 0, s>>>(part, nw, out);
      launches += 2;
    };
    // R = B, X = 0; column norms; Z = M R; P = orth(Z)
    k_b_gather<<<ge, BT, 0, s>>>(B, ldb, m, n, b);
    NLSP_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    NLSP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nv, s));
    NLSP_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * nv, s));
    gram(r, r, G3);
    k_bcg_state<<<1, 32, 0, s>>>(G3, st, 0, prm->tol);
    k_bcg_prep<KIND, T><<<nb, BT, 0, s>>>(AT, omega, r, rT, za, n);
    launches += 3 + precond_rest(s);
    gram(z, z, G1);
    k_bcg_small<<<1, 1024, 0, s>>>(BCG_ORTH, G1, nullptr, Dfac, coef, st);
    k_bcg_mm<<<nb, BT, 0, s>>>(P, nullptr, z, coef, n, 1.0, 0);
    launches += 2;
    NLSP_LAUNCH_CHECK();
    NLSP_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    NLSP_CUDA(cudaStreamSynchronize(s));
    int it = 0;
    while (!h.all_done && h.s > 0 && it < prm->maxit) {
      k_b_spmv4<KIND><<<nb, BT, 0, s>>>(A->v64, P, Q, part);       // Q = A P
      gram(P, Q, G1);                                                // D = P^T Q
      gram(P, r, G2);                                                // P^T R
      k_bcg_small<<<1, 1024, 0, s>>>(BCG_ALPHA, G1, G2, Dfac, coef, st);
      k_bcg_mm<<<nb, BT, 0, s>>>(x, nullptr, P, coef, n, 1.0, 1);  // X += P alpha
      k_bcg_mm<<<nb, BT, 0, s>>>(r, nullptr, Q, coef, n, -1.0, 1); // R -= Q alpha
      k_bcg_tick<<<1, 32, 0, s>>>(st);
      gram(r, r, G3);
      k_bcg_state<<<1, 32, 0, s>>>(G3, st, 1, prm->tol);
      launches += 6;
      ++it;
      NLSP_LAUNCH_CHECK();
      NLSP_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
      NLSP_CUDA(cudaStreamSynchronize(s));
      if (h.all_done || it >= prm->maxit) break;
      k_bcg_prep<KIND, T><<<nb, BT, 0, s>>>(AT, omega, r, rT, za, n);  // Z = M R
      launches += 1 + precond_rest(s);
      gram(Q, z, G1);                                                   // Q^T Z
      k_bcg_small<<<1, 1024, 0, s>>>(BCG_BETA, G1, nullptr, Dfac, coef, st);
      k_bcg_mm<<<nb, BT, 0, s>>>(W, z, P, coef, n, 1.0, 0);             // W = Z + P beta
      gram(W, W, G1);
      k_bcg_small<<<1, 1024, 0, s>>>(BCG_ORTH, G1, nullptr, Dfac, coef, st);
      k_bcg_mm<<<nb, BT, 0, s>>>(P, nullptr, W, coef, n, 1.0, 0);       // P = orth(W)
      launches += 5;
    }
    // true residuals b - A x (FP64) per column, then x out
    k_b_true<KIND><<<nb, BT, 0, s>>>(A->v64, b, x, part);
    k_b_scatter<<<ge, BT, 0, s>>>(x, m, n, X, ldx);
    launches += 2;
    NLSP_LAUNCH_CHECK();
    std::vector<double> hp((size_t)nb * MB);
    NLSP_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, s));
    NLSP_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    int herr = 0;
    NLSP_CUDA(cudaMemcpyAsync(&herr, &bst->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NLSP_CUDA(cudaStreamSynchronize(s));
    count_launches(ctx, (unsigned long long)launches);
    if (herr) {
      nlsp_record_message("block CG: a tensor-core completion wait gave up");
      return NLSP_ERR_TIMEOUT;
    }
    nlsp_status worst = NLSP_OK;
    for (int c = 0; c < m; ++c) {
      double tr = 0.0;
      for (int q = 0; q < nb; ++q) tr += hp[(size_t)q * MB + c];
      int stc = h.status[c];
      if (stc == NLSP_OK && !h.done[c]) stc = h.bad ? NLSP_ERR_BREAKDOWN : NLSP_NOT_CONVERGED;
      if (infos) {
        infos[c].iterations = h.iter[c];
        infos[c].status = stc;
        infos[c].relres = h.bb[c] > 0 ? sqrt(h.rr[c] / h.bb[c]) : 0.0;
        infos[c].true_relres = h.bb[c] > 0 ? sqrt(tr / h.bb[c]) : 0.0;
      }
      if (stc == NLSP_ERR_BREAKDOWN) worst = NLSP_ERR_BREAKDOWN;
      else if (stc == NLSP_NOT_CONVERGED && worst == NLSP_OK) worst = NLSP_NOT_CONVERGED;
    }
    return worst;
  }

  static nlsp_status run(nlsp_ctx* ctx, const nlsp_prec* M, int m, const double* B, int64_t ldb, double* X,
                         int64_t ldx, const nlsp_solve_params* prm, nlsp_solve_info* infos, bool krylov) {
    cudaStream_t s = ctx->stream;
    const nlsp_op* A = M->A;
    const int64_t n = A->n, n_pad = M->n_pad;
    const int k = M->r;  // active rank
    const int nu = M->nu1;
    const T omega = (T)M->omega;
    const StencilView<T>& AT = bview<T>(A);
    const int nb = std::max(1, std::min<int>(ctx->num_sms * 8, (int)((n + BW - 1) / BW)));
    const int64_t ntiles = n_pad / NLSP_TILE;
    const int nbr = (int)std::max<int64_t>(1, std::min<int64_t>(2 * ctx->num_sms, ntiles));
    const int flexible = prm->flexible < 0 ? (M->precision != NLSP_FP64) : (prm->flexible != 0);
    // workspace
    const size_t nv = (size_t)n * MB;
    // reduced-precision tensor-core contractions (NLSP_MIXED_TF32 / _BF16):
    // repacked operand copies of P, sized for the active rank
    const int lp_op = M->precision == NLSP_MIXED_BF16 ? lp::OP_BF16 : lp::OP_TF32;
    const bool use_lp = sizeof(T) == 4 && (M->precision == NLSP_MIXED_BF16 || M->precision == NLSP_MIXED_TF32);
    const int lp_es = lp_op == lp::OP_BF16 ? 2 : 4;
    const size_t lp_rchunk = (size_t)lp::rows_r(k) * lp::RCH * lp_es;
    const size_t lp_qtile = (size_t)NLSP_TILE * lp::kcols_q(k) * lp_es;
    const size_t lp_bytes = use_lp ? (size_t)ntiles * (2 * lp_rchunk + lp_qtile) + 512 : 0;
    const size_t bytes = sizeof(double) * nv * 6 + sizeof(T) * nv * 4 + sizeof(double) * (size_t)2 * nb * MB +
                         sizeof(T) * (size_t)nbr * k * MB + (sizeof(T) + sizeof(double)) * (size_t)k * MB +
                         sizeof(BlockState) + 8192 + lp_bytes;
    DevBuf buf;
    NLSP_TRY(buf.alloc(bytes));
    unsigned char* base = buf.as<unsigned char>();
    size_t off = 0;
    auto take = [&](size_t b) {
      unsigned char* q = base + off;
      off = align_up(off + b, 256);
      return q;
    };
    double* b = (double*)take(sizeof(double) * nv);
    double* x = (double*)take(sizeof(double) * nv);
    double* r = (double*)take(sizeof(double) * nv);
    double* p = (double*)take(sizeof(double) * nv);
    double* q = (double*)take(sizeof(double) * nv);
    double* z = (double*)take(sizeof(double) * nv);
    T* rT = (T*)take(sizeof(T) * nv);
    T* za = (T*)take(sizeof(T) * nv);
    T* zb = (T*)take(sizeof(T) * nv);
    T* E = (T*)take(sizeof(T) * (size_t)k * MB);
    double* Csum = (double*)take(sizeof(double) * (size_t)k * MB);
    double* part = (double*)take(sizeof(double) * (size_t)2 * nb * MB);
    T* cpart = (T*)take(sizeof(T) * (size_t)nbr * k * MB);
    BlockState* st = (BlockState*)take(sizeof(BlockState));
    unsigned char* lp_R = use_lp ? take((size_t)ntiles * 2 * lp_rchunk) : nullptr;
    unsigned char* lp_Q = use_lp ? take((size_t)ntiles * lp_qtile) : nullptr;
    (void)zb;
    // restriction / prolongation shared memory
    const size_t sm_r = sizeof(T) * ((size_t)NLSP_TILE * ((k + 3) / 4 * 4 + 4) + (size_t)NLSP_TILE * 36);
    const size_t sm_p = sizeof(T) * (size_t)k * MB;
    auto fr = k_b_restrict<KIND, T>;
    auto fp = k_b_prolong<T>;
    if (sm_r > 48 * 1024) NLSP_CUDA(cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_r));
    if (sm_p > 48 * 1024) NLSP_CUDA(cudaFuncSetAttribute(fp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_p));
    // FP32 preconditioner: the restriction on tensor cores (split TF32
    // inputs, FP32 accumulation); the prolongation too with NLSP_BLOCK_TC=2
    // (slower on GB300: its operand staging costs more than the CUDA-core
    // product), neither with NLSP_BLOCK_TC=0.
    const char* tc_env = getenv("NLSP_BLOCK_TC");
    const int tc_mode = tc_env ? (tc_env[0] - '0') : 1;
    const bool use_tc = sizeof(T) == 4 && tc_mode >= 1;
    const bool use_tc_prolong = sizeof(T) == 4 && tc_mode >= 2;
    const int kp8 = (k + 7) / 8 * 8;
    const size_t sm_rtc = (size_t)2 * (128 * TCK + 32 * TCK) * 4;
    const size_t sm_ptc = (size_t)2 * (128 * std::min(kp8, TCK) + 32 * kp8) * 4;
    if (use_tc) {
      NLSP_CUDA(cudaFuncSetAttribute(k_b_restrict_tc<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rtc));
      NLSP_CUDA(cudaFuncSetAttribute(k_b_prolong_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_ptc));
    }
    // reduced-precision kernels: restriction ring of LP_NS 128-row stages
    // plus two residual buffers; prolongation ring of as many tile stages as
    // fit (at most LP_NS) plus E^T
    // stage counts: at least two CTAs per SM where two stages fit (the
    // kernels are latency-bound per chunk, so resident CTAs matter more than
    // ring depth), else as many stages as one CTA holds
    int optin = 0;
    NLSP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    const size_t lp_achunk = (size_t)128 * lp::RCH * lp_es, lp_bbuf = (size_t)2 * lp::MBC * lp::RCH * lp_es;
    const size_t half = (size_t)optin / 2 - 2048;
    const int lp_nsr = (int)std::max<size_t>(2, std::min<size_t>(LP_NS, (half - lp_bbuf) / lp_achunk));
    const size_t sm_rlp = (size_t)lp_nsr * lp_achunk + lp_bbuf;
    const size_t lp_bt = (size_t)lp::MBC * lp::kcols_q(k) * lp_es;
    const size_t ns2 = (half - lp_bt) / lp_qtile;
    const int lp_ns = (int)(ns2 >= 2 ? std::min<size_t>(LP_NS, ns2)
                                     : std::max<size_t>(1, std::min<size_t>(LP_NS, ((size_t)optin - 4096 - lp_bt) / lp_qtile)));
    const size_t sm_plp = (size_t)lp_ns * lp_qtile + lp_bt;
    constexpr int LPT = 512;  // threads of the reduced-precision restriction (one node-quad each per chunk)
    auto fr_lp = lp_op == lp::OP_BF16 ? k_b_restrict_lp<KIND, lp::OP_BF16, LPT> : k_b_restrict_lp<KIND, lp::OP_TF32, LPT>;
    auto fp_lp = lp_op == lp::OP_BF16 ? k_b_prolong_lp<lp::OP_BF16> : k_b_prolong_lp<lp::OP_TF32>;
    if (use_lp) {
      NLSP_CUDA(cudaFuncSetAttribute(fr_lp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_rlp));
      NLSP_CUDA(cudaFuncSetAttribute(fp_lp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_plp));
      const int gp = grid_for(ctx, ntiles * NLSP_TILE * (int64_t)lp::kcols_q(k), BT, 8);
      if (lp_op == lp::OP_BF16)
        lp::k_pack<lp::OP_BF16><<<gp, BT, 0, s>>>((const float*)M->P, M->k, k, ntiles, lp_R, lp_Q);
      else
        lp::k_pack<lp::OP_TF32><<<gp, BT, 0, s>>>((const float*)M->P, M->k, k, ntiles, lp_R, lp_Q);
      NLSP_LAUNCH_CHECK();
    }
    // state
    BlockState h;
    memset(&h, 0, sizeof(h));
    h.maxit = prm->maxit;
    h.flexible = flexible;
    h.m = m;
    NLSP_CUDA(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    const int ge = grid_for(ctx, (int64_t)nv, BT, 8);
    k_b_gather<<<ge, BT, 0, s>>>(B, ldb, m, n, b);
    NLSP_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    NLSP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * nv, s));
    NLSP_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * nv, s));
    k_b_dot_init<<<nb, BT, 0, s>>>(b, n, part);
    k_b_scalars<<<1, 1024, 0, s>>>(part, nb, st, BS_INIT);
    k_b_set_tol<<<1, 32, 0, s>>>(st, prm->tol);
    NLSP_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * nv, s));
    NLSP_CUDA(cudaMemsetAsync(q, 0, sizeof(double) * nv, s));
    NLSP_LAUNCH_CHECK();
    int launches = use_lp ? 7 : 6;
    // z = B r.  In the iteration the update kernel forms x, r with alpha and
    // then rT and the first pre-sweep; for the initial application alpha = 0
    // leaves x and r as they are.
    // the preconditioner after the first pre-sweep (za holds it): the other
    // pre-sweeps, restriction, coarse solve, prolongation, post-sweeps; the
    // last one writes z in FP64 with the per-column r^T z partials
    auto precond_rest = [&](cudaStream_t ss) -> int {
      int nl = 0;
      T* cur = za;
      T* oth = zb;
      for (int sw = 1; sw < nu; ++sw, ++nl) {
        k_b_sweep4<KIND, T><<<nb, BT, 0, ss>>>(AT, omega, rT, cur, oth);
        std::swap(cur, oth);
      }
      if (use_lp)
        fr_lp<<<nbr, LPT, sm_rlp, ss>>>(*reinterpret_cast<const StencilView<float>*>(&AT), (const float*)rT,
                                       (const float*)cur, lp_R, k, ntiles, (float*)cpart, lp_nsr, st);
      else if (use_tc)
        k_b_restrict_tc<KIND><<<nbr, BT, sm_rtc, ss>>>(*reinterpret_cast<const StencilView<float>*>(&AT),
                                                       (const float*)rT, (const float*)cur, (const float*)M->P,
                                                       M->k, k, ntiles, (float*)cpart, st);
      else
        fr<<<nbr, BT, sm_r, ss>>>(AT, rT, cur, (const T*)M->P, M->k, k, ntiles, cpart);
      k_b_csum<T><<<div_up((int64_t)k * MB, 128), 128, 0, ss>>>(cpart, nbr, k, Csum);
      k_b_coarse<T><<<div_up((int64_t)k * MB, 128), 128, 0, ss>>>(Csum, k, M->Ainv, E);
      if (use_lp)
        fp_lp<<<nbr, BT, sm_plp, ss>>>(lp_Q, k, n, (const float*)E, (float*)cur, lp_ns, st);
      else if (use_tc_prolong)
        k_b_prolong_tc<<<nbr, BT, sm_ptc, ss>>>((const float*)M->P, M->k, k, n, (const float*)E, (float*)cur, st);
      else
        fp<<<nb, BT, sm_p, ss>>>((const T*)M->P, M->k, k, n, E, cur);
      nl += 4;
      for (int sw = 1; sw < nu; ++sw, ++nl) {
        k_b_sweep4<KIND, T><<<nb, BT, 0, ss>>>(AT, omega, rT, cur, oth);
        std::swap(cur, oth);
      }
      k_b_post4<KIND, T><<<nb, BT, 0, ss>>>(AT, omega, rT, cur, r, z, part);
      return nl + 1;
    };
    auto apply = [&](cudaStream_t ss, bool with_rr) -> int {
      int nl = 0;
      k_b_update<KIND, T><<<nb, BT, 0, ss>>>(AT, omega, x, r, p, q, rT, za, st, part);
      ++nl;
      if (with_rr) {  // r^T r of the updated residual: convergence, maxit
        k_b_scalars<<<1, 1024, 0, ss>>>(part, nb, st, BS_RR);
        ++nl;
      }
      nl += precond_rest(ss);
      k_b_scalars<<<1, 1024, 0, ss>>>(part, nb, st, BS_RZ);
      return nl + 1;
    };
    if (krylov) {
      const nlsp_status bst = block_cg(ctx, M, m, B, ldb, X, ldx, prm, infos, b, x, r, p, q, z, rT, za, st,
                                       precond_rest, nb, ge);
      NLSP_CUDA(cudaStreamSynchronize(s));
      return bst;
    }
    launches += apply(s, false);
    NLSP_LAUNCH_CHECK();
    // one iteration: p = z + beta p, q = A p, alpha, update, z = B r, beta
    auto body = [&](cudaStream_t ss) -> int {
      k_b_dir<<<ge, BT, 0, ss>>>(z, p, n, st);
      k_b_spmv4<KIND><<<nb, BT, 0, ss>>>(A->v64, p, q, part);
      k_b_scalars<<<1, 1024, 0, ss>>>(part, nb, st, BS_PQ);
      return 3 + apply(ss, true);
    };
    cudaStream_t cap;
    NLSP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
    };
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int nbody = 0;
    if (ce == cudaSuccess) {
      nbody = body(cap);
      ce = cudaStreamEndCapture(cap, &graph);
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
      cleanup();
      NLSP_CUDA(ce);
    }
    // relaunch in chunks of 8 iterations; iterations past a column's stop
    // leave it untouched (alpha = 0), so a chunk may overrun safely
    int hdone = 0, iters = 0;
    while (iters < prm->maxit) {
      const int chunk = std::min(8, prm->maxit - iters);
      for (int c = 0; c < chunk; ++c) {
        ce = cudaGraphLaunch(exec, s);
        if (ce != cudaSuccess) {
          cleanup();
          NLSP_CUDA(ce);
        }
      }
      launches += chunk * nbody;
      iters += chunk;
      ce = cudaMemcpyAsync(&hdone, &st->all_done, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        cleanup();
        NLSP_CUDA(ce);
      }
      if (hdone) break;
    }
    cleanup();
    k_b_true<KIND><<<nb, BT, 0, s>>>(A->v64, b, x, part);
    k_b_true_fin<<<1, 32, 0, s>>>(part, nb, st);
    k_b_scatter<<<ge, BT, 0, s>>>(x, m, n, X, ldx);
    NLSP_LAUNCH_CHECK();
    launches += 3;
    NLSP_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    NLSP_CUDA(cudaStreamSynchronize(s));
    count_launches(ctx, (unsigned long long)launches);
    if (h.err) {
      nlsp_record_message("block solve: a tensor-core completion wait gave up");
      return NLSP_ERR_TIMEOUT;
    }
    nlsp_status worst = NLSP_OK;
    for (int c = 0; c < m; ++c) {
      int stc = h.status[c];
      if (stc == NLSP_OK && !h.done[c]) stc = NLSP_NOT_CONVERGED;
      if (infos) {
        infos[c].iterations = h.iter[c];
        infos[c].status = stc;
        infos[c].relres = h.bb[c] > 0 ? sqrt(h.rr[c] / h.bb[c]) : 0.0;
        infos[c].true_relres = h.bb[c] > 0 ? sqrt(h.true_rr[c] / h.bb[c]) : 0.0;
      }
      if (stc == NLSP_ERR_BREAKDOWN) worst = NLSP_ERR_BREAKDOWN;
      else if (stc == NLSP_NOT_CONVERGED && worst == NLSP_OK) worst = NLSP_NOT_CONVERGED;
    }
    return worst;
  }
};

}  // namespace

namespace {

nlsp_status solve_block_any(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* M, int m, const double* dev_B,
                            int64_t ldb, double* dev_X, int64_t ldx, const nlsp_solve_params* params,
                            nlsp_solve_info* infos, bool krylov) {
  if (!ctx || !A || !M || !params || M->A != A || m < 0 || m > MB || ldb < A->n || ldx < A->n) return NLSP_ERR_INVALID;
  if (m > 0 && (!dev_B || !dev_X)) return NLSP_ERR_INVALID;
  if (!(params->tol >= 0.0) || params->maxit < 1 || M->r > 128) return NLSP_ERR_INVALID;
  if (m == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  if (M->precision == NLSP_FP64) {
    switch (A->kind) {
      case ST_5PT: return BlockSolver<ST_5PT, double>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
      case ST_9PT: return BlockSolver<ST_9PT, double>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
      case ST_CSR: return BlockSolver<ST_CSR, double>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
      default: return BlockSolver<ST_7PT, double>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
    }
  }
  switch (A->kind) {
    case ST_5PT: return BlockSolver<ST_5PT, float>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
    case ST_9PT: return BlockSolver<ST_9PT, float>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
    case ST_CSR: return BlockSolver<ST_CSR, float>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
    default: return BlockSolver<ST_7PT, float>::run(ctx, M, m, dev_B, ldb, dev_X, ldx, params, infos, krylov);
  }
}

}  // namespace

extern "C" nlsp_status nlsp_solve_block(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* M, int m,
                                        const double* dev_B, int64_t ldb, double* dev_X, int64_t ldx,
                                        const nlsp_solve_params* params, nlsp_solve_info* infos) {
  return solve_block_any(ctx, A, M, m, dev_B, ldb, dev_X, ldx, params, infos, false);
}

extern "C" nlsp_status nlsp_solve_block_cg(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* M, int m,
                                           const double* dev_B, int64_t ldb, double* dev_X, int64_t ldx,
                                           const nlsp_solve_params* params, nlsp_solve_info* infos) {
  return solve_block_any(ctx, A, M, m, dev_B, ldb, dev_X, ldx, params, infos, true);
}
