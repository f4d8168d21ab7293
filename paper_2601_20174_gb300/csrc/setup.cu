// Setup of the two-level preconditioner (Algorithm 1, setup):
//   S = (I - w D^-1 A)^s1 S0          sample smoothing (Sec. 3, Near-Nullspace Vectors)
//   P = U_k of S                      thin SVD (Sec. 3, SVD-Centric Construction) via the
//                                     Gram matrix S^T S: FP32 Jacobi eigensolver, then in
//                                     FP64 mode Ogita-Aishima refinement and CholeskyQR
//                                     (P = qf(.), Sec. 3)
//   A_c = P_r^T A P_r, A_c = L L^T    Galerkin operator and FP64 Cholesky
//
// GB300 notes: FP64 runs at 1/62 of the FP32 rate on this part, so every
// O(n K^2) and O(K^3) step of the mixed path is FP32 (with FP64 cross-block
// sums), and the FP64 path solves the K x K eigenproblem in FP32 first and
// refines it with FP64 matrix products instead of running FP64 Jacobi
// rotations on one SM.
#include <math.h>
#include <string.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "stencil.cuh"

namespace {

// ---------------------------------------------------------------------------
// Layout conversion between column-major FP64 (ld = n) and tiled T.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_colmajor_to_tiled(const double* __restrict__ src, int64_t n, int64_t ld, int ncols,
                                    int64_t n_pad, T* __restrict__ dst) {
  const int64_t total = n_pad * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / ((int64_t)ncols * NLSP_TILE);
    const int c = (int)((e / NLSP_TILE) % ncols);
    const int64_t i = t * NLSP_TILE + (e % NLSP_TILE);
    dst[e] = i < n ? (T)src[c * ld + i] : T(0);
  }
}

template <typename T>
__global__ void k_tiled_to_colmajor(const T* __restrict__ src, int64_t n, int ncols, int ncols_out,
                                    double* __restrict__ dst, int64_t ld) {
  const int64_t total = n * ncols_out;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n);
    const int64_t i = e - (int64_t)c * n;
    dst[c * ld + i] = (double)src[tiled_index(i, c, ncols)];
  }
}

// Random test vectors S0 ~ N(0, 1) drawn on the device, straight into the
// tiled layout: SplitMix64 (Steele, Lea, Flood 2014) counter streams and the
// Box-Muller transform, the same definition as the host-side input
// generator: element (i, c) is normal number c * n + i of stream `stream`
// under `seed`; normal 2j / 2j+1 use uniforms 2j, 2j+1 (top 53 bits) as
// sqrt(-2 log(1 - u1)) * (cos, sin)(2 pi u2).
__device__ __forceinline__ uint64_t splitmix_fin(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t splitmix_stream_base(uint64_t seed, uint64_t stream) {
  uint64_t v = seed ^ (stream * 0xD1B54A32D192ED03ull);
  v += 0x9E3779B97F4A7C15ull;
  v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
  v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
  return v ^ (v >> 31);
}

__device__ __forceinline__ double normal_draw(uint64_t base, uint64_t idx) {
  const uint64_t j = idx >> 1;
  const uint64_t a = splitmix_fin(base + (2 * j + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t b = splitmix_fin(base + (2 * j + 2) * 0x9E3779B97F4A7C15ull);
  const double u1 = (double)(a >> 11) * 0x1.0p-53, u2 = (double)(b >> 11) * 0x1.0p-53;
  const double rad = sqrt(-2.0 * log1p(-u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return rad * ((idx & 1) ? s : c);
}

// The same draw evaluated in FP32 (for FP32 sample blocks): 1 - u1 is formed
// exactly as an integer and rounded once, u2 keeps its top 24 bits, and the
// transform uses FP32 log / sincospi.  Agrees with normal_draw to a few FP32
// ulps of the radius plus 2^-24 of the angle.
__device__ __forceinline__ float normal_draw_f32(uint64_t base, uint64_t idx) {
  const uint64_t j = idx >> 1;
  const uint64_t a = splitmix_fin(base + (2 * j + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t b = splitmix_fin(base + (2 * j + 2) * 0x9E3779B97F4A7C15ull);
  const float om = __ull2float_rn((1ull << 53) - (a >> 11)) * 0x1.0p-53f;  // 1 - u1, in (0, 1]
  const float u2 = __uint2float_rn((unsigned)(b >> 40)) * 0x1.0p-24f;
  const float rad = sqrtf(-2.0f * logf(om));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return rad * ((idx & 1) ? s : c);
}

template <typename T>
__global__ void k_random_samples_tiled(uint64_t base, int64_t n, int ncols, int64_t n_pad, T* __restrict__ dst) {
  const int64_t total = n_pad * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / ((int64_t)ncols * NLSP_TILE);
    const int c = (int)((e / NLSP_TILE) % ncols);
    const int64_t i = t * NLSP_TILE + (e % NLSP_TILE);
    T v = T(0);
    if (i < n) {
      if constexpr (sizeof(T) == 4)
        v = normal_draw_f32(base, (uint64_t)c * n + i);
      else
        v = (T)normal_draw(base, (uint64_t)c * n + i);
    }
    dst[e] = v;
  }
}

__global__ void k_random_normal(uint64_t base, uint64_t offset, int64_t count, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = normal_draw(base, offset + e);
}

// One weighted-Jacobi sweep on A S = 0 for all K columns of a tiled block:
// S_out = S_in - w D^-1 A S_in.  Grid: x over the padded nodes, y over groups
// of CPT columns (the index arithmetic and the coefficients of a node are
// shared by its CPT columns); padding rows are written as zero.
template <int KIND, typename T, int CPT>
__global__ void __launch_bounds__(256) k_smooth_sweep(StencilView<T> A, T omega, int ncols, int n_pad,
                                                      const T* __restrict__ Sin, T* __restrict__ Sout) {
  const int cbase = blockIdx.y * CPT;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
    const int64_t e0 = tiled_index(i, cbase, ncols);
    if (i >= A.n) {
#pragma unroll
      for (int c = 0; c < CPT; ++c)
        if (cbase + c < ncols) Sout[e0 + (int64_t)c * NLSP_TILE] = T(0);
      continue;
    }
    const NodeCoord nc = node_coord<KIND>(i, A.N);
    const T wd = omega * stencil_dinv<KIND>(A, i);
    T as[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      as[c] = cbase + c < ncols ? stencil_diag<KIND>(A, i) * Sin[e0 + (int64_t)c * NLSP_TILE] : T(0);
    for_each_neighbour<KIND>(A, i, nc, [&](int64_t m, NodeCoord, T a) {
      const int64_t em = tiled_index(m, cbase, ncols);
#pragma unroll
      for (int c = 0; c < CPT; ++c)
        if (cbase + c < ncols) as[c] += a * Sin[em + (int64_t)c * NLSP_TILE];
    });
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (cbase + c < ncols) Sout[e0 + (int64_t)c * NLSP_TILE] = Sin[e0 + (int64_t)c * NLSP_TILE] - wd * as[c];
  }
}

// The same sweep on the 2D grids, streamed along grid rows: thread x of a
// block walks the rows j0 .. j0 + band - 1 of grid column x for one group of
// CPT sample columns, holding the rows below, at and above the current one
// in registers, so that every sample value is read from memory once per band
// (plus the two rows around it) instead of once more for each vertical
// neighbour.  East/west (and, for the 9-point stencil, diagonal) neighbours
// are read from lines the warp itself has just loaded.  Grid: x over
// SR_THREADS grid columns, y over bands, z over column groups; the first
// block of each column group also zeroes the padding rows.  The neighbours
// are visited in the order for_each_neighbour uses, so the sums are the same.
constexpr int SR_THREADS = 128;

template <int KIND, typename T, int CPT>
__global__ void __launch_bounds__(SR_THREADS) k_smooth_rows(StencilView<T> A, T omega, int ncols, int n_pad, int band,
                                                           const T* __restrict__ Sin, T* __restrict__ Sout) {
  static_assert(KIND == ST_5PT || KIND == ST_9PT, "row streaming needs a 2D grid");
  const int N = A.N;
  const int cbase = blockIdx.z * CPT;
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    for (int64_t i = A.n + threadIdx.x; i < n_pad; i += SR_THREADS) {
      const int64_t e0 = tiled_index(i, cbase, ncols);
#pragma unroll
      for (int c = 0; c < CPT; ++c)
        if (cbase + c < ncols) Sout[e0 + (int64_t)c * NLSP_TILE] = T(0);
    }
  }
  const int x = blockIdx.x * SR_THREADS + threadIdx.x;
  const int j0 = blockIdx.y * band;
  if (x >= N || j0 >= N) return;
  const int j1 = min(j0 + band, N);
  // the CPT columns of node i (0 past ncols)
  auto load = [&](int64_t i, T(&v)[CPT]) {
    const int64_t e = tiled_index(i, cbase, ncols);
#pragma unroll
    for (int c = 0; c < CPT; ++c) v[c] = cbase + c < ncols ? Sin[e + (int64_t)c * NLSP_TILE] : T(0);
  };
  T rs[CPT], rc[CPT], rn[CPT], t[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) rs[c] = rn[c] = T(0);
  if (j0 > 0) load((int64_t)(j0 - 1) * N + x, rs);
  load((int64_t)j0 * N + x, rc);
  T cys = T(0);  // 5-point: coupling of the current row to the row below
  if (KIND == ST_5PT && j0 > 0) cys = A.cy[(int64_t)(j0 - 1) * N + x];
  const bool w = x > 0, e = x < N - 1;
  for (int j = j0; j < j1; ++j) {
    const int64_t idx = (int64_t)j * N + x;
    const bool so = j > 0, no = j < N - 1;
    if (no) load(idx + N, rn);
    T as[CPT];
    T wd;
    auto add = [&](T a, const T(&v)[CPT]) {
#pragma unroll
      for (int c = 0; c < CPT; ++c) as[c] += a * v[c];
    };
    if constexpr (KIND == ST_9PT) {
      wd = omega * A.cdinv;
#pragma unroll
      for (int c = 0; c < CPT; ++c) as[c] = A.c[0] * rc[c];
      if (w) {
        load(idx - 1, t);
        add(A.c[1], t);
      }
      if (e) {
        load(idx + 1, t);
        add(A.c[1], t);
      }
      if (so) add(A.c[2], rs);
      if (no) add(A.c[2], rn);
      if (e && no) {
        load(idx + N + 1, t);
        add(A.c[3], t);
      }
      if (w && so) {
        load(idx - N - 1, t);
        add(A.c[3], t);
      }
      if (w && no) {
        load(idx + N - 1, t);
        add(A.c[4], t);
      }
      if (e && so) {
        load(idx - N + 1, t);
        add(A.c[4], t);
      }
    } else {
      wd = omega * A.dinv[idx];
      const T dg = A.diag[idx];
#pragma unroll
      for (int c = 0; c < CPT; ++c) as[c] = dg * rc[c];
      if (w) {
        const T a = -A.cx[idx - 1];
        load(idx - 1, t);
        add(a, t);
      }
      if (e) {
        const T a = -A.cx[idx];
        load(idx + 1, t);
        add(a, t);
      }
      if (so) add(-cys, rs);
      T cyn = T(0);
      if (no) {
        cyn = A.cy[idx];
        add(-cyn, rn);
      }
      cys = cyn;
    }
    const int64_t e0 = tiled_index(idx, cbase, ncols);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (cbase + c < ncols) Sout[e0 + (int64_t)c * NLSP_TILE] = rc[c] - wd * as[c];
      rs[c] = rc[c];
      rc[c] = rn[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Tall-skinny products over node tiles: partial[b] = sum over the tiles of
// block b of X_t^T Y_t (ncx x ncy block of the first ncx / ncy columns), with
// Y = X or Y = A X (evaluated on the fly from X's neighbour rows).  Thread
// (ty, tx) of a TD x TD block owns an RB x RB register tile of the output.
// The tile's node chunk is staged transposed in shared memory ([w][c]) so the
// inner loop reads contiguous float4/double2 rows.  FP32 inputs accumulate in
// FP32 within a block and leave as FP64 partials.
// ---------------------------------------------------------------------------
constexpr int GRAM_CW = 32;  // nodes per staged chunk

// The block's products are X_t[:, cx0 .. cx0 + ncx)^T Y_t[:, cy0 .. cy0 + ncy)
// with Y = A X, or (TWO) Y = X with a column range of its own (quadrants of
// a Gram matrix wider than KP); X^T X itself uses the pipelined path.
template <typename T, int RB, int TD, int KIND, bool WITH_A, bool TWO = false>
__global__ void __launch_bounds__(TD* TD) k_tsgemm(StencilView<T> A, const T* __restrict__ X, int ncols, int ncx,
                                                  int64_t n_pad, double* __restrict__ partial, int cx0, int cy0,
                                                  int ncy) {
  constexpr int KP = RB * TD;
  constexpr int LDS = KP + (sizeof(T) == 4 ? 4 : 2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);  // [CW][LDS]
  T* ys = (WITH_A || TWO) ? xs + GRAM_CW * LDS : xs;
  const int tx = threadIdx.x % TD, ty = threadIdx.x / TD;
  T acc[RB][RB];
#pragma unroll
  for (int a = 0; a < RB; ++a)
#pragma unroll
    for (int b = 0; b < RB; ++b) acc[a][b] = T(0);

  const int64_t ntiles = n_pad / NLSP_TILE;
  constexpr int nthreads = TD * TD;
  auto products = [&]() {
#pragma unroll 1
    for (int w = 0; w < GRAM_CW; ++w) {
      T xa[RB], yb[RB];
#pragma unroll
      for (int a = 0; a < RB; ++a) xa[a] = xs[w * LDS + ty * RB + a];
#pragma unroll
      for (int b = 0; b < RB; ++b) yb[b] = ys[w * LDS + tx * RB + b];
#pragma unroll
      for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) acc[a][b] += xa[a] * yb[b];
    }
  };
  if constexpr (!WITH_A && !TWO) {
    // Software pipeline over the block's chunks (CW nodes of one tile each):
    // the loads of chunk q + 1 are in flight while chunk q is multiplied.
    constexpr int PER = GRAM_CW * KP / nthreads;
    static_assert(PER * nthreads == GRAM_CW * KP, "chunk must split evenly over the block");
    constexpr int CPT = NLSP_TILE / GRAM_CW;  // chunks per tile
    // chunks are dealt round-robin over the blocks (a small system still
    // spreads over CPT blocks per tile)
    const int64_t all = ntiles * CPT;
    const int64_t nchunks = blockIdx.x < all ? (all - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    T pre[PER];
    auto load = [&](int64_t q) {
      const int64_t gq = blockIdx.x + q * gridDim.x;
      const int64_t t = gq / CPT;
      const int w0 = (int)(gq % CPT) * GRAM_CW;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * nthreads;
        const int c = e / GRAM_CW, w = e % GRAM_CW;
        pre[u] = c < ncx ? X[(t * ncols + c) * NLSP_TILE + w0 + w] : T(0);
      }
    };
    if (nchunks > 0) load(0);
    for (int64_t q = 0; q < nchunks; ++q) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * nthreads;
        xs[(e % GRAM_CW) * LDS + e / GRAM_CW] = pre[u];
      }
      __syncthreads();
      if (q + 1 < nchunks) load(q + 1);
      products();
    }
  } else {
    for (int64_t gq = blockIdx.x; gq < ntiles * (NLSP_TILE / GRAM_CW); gq += gridDim.x) {
      const int64_t t = gq / (NLSP_TILE / GRAM_CW);
      const int w0 = (int)(gq % (NLSP_TILE / GRAM_CW)) * GRAM_CW;
      {
        __syncthreads();
        // stage the X chunk and the Y chunk (A X, or X's other columns)
        // transposed: element (w, c)
        for (int e = threadIdx.x; e < GRAM_CW * KP; e += nthreads) {
          const int c = e / GRAM_CW, w = e % GRAM_CW;
          T xv = T(0), yv = T(0);
          const int64_t i = t * NLSP_TILE + w0 + w;
          if (c < ncx) xv = X[(t * ncols + cx0 + c) * NLSP_TILE + w0 + w];
          if (c < ncy) {
            if (TWO) {
              yv = X[(t * ncols + cy0 + c) * NLSP_TILE + w0 + w];
            } else if (i < A.n) {
              const NodeCoord nc = node_coord<KIND>(i, A.N);
              yv = stencil_apply<KIND>(A, i, nc, [&](int64_t m) { return X[tiled_index(m, cy0 + c, ncols)]; });
            }
          }
          xs[w * LDS + c] = xv;
          ys[w * LDS + c] = yv;
        }
        __syncthreads();
        products();
      }
    }
  }
  double* out = partial + (int64_t)blockIdx.x * ncx * ncy;
#pragma unroll
  for (int a = 0; a < RB; ++a) {
    const int row = ty * RB + a;
#pragma unroll
    for (int b = 0; b < RB; ++b) {
      const int col = tx * RB + b;
      if (row < ncx && col < ncy) out[(int64_t)col * ncx + row] = (double)acc[a][b];
    }
  }
}

// out = sum_b partial[b] in a fixed order (deterministic); a partial is a
// rows x cols block (column-major) that lands at (r0, c0) of out (leading
// dimension ld).  A block of 256 threads covers 32 entries, warp g adding
// partials b = g, g + 8, ... (four running sums), then the eight warp sums
// are added in warp order.
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ partial, int nblocks, int rows,
                                                      int cols, double* __restrict__ out, int ld, int r0, int c0) {
  __shared__ double red[8][33];
  const int mm = rows * cols;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (e < mm) {
    int b = g;
    for (; b + 24 < nblocks; b += 32) {
      s0 += partial[(int64_t)b * mm + e];
      s1 += partial[(int64_t)(b + 8) * mm + e];
      s2 += partial[(int64_t)(b + 16) * mm + e];
      s3 += partial[(int64_t)(b + 24) * mm + e];
    }
    for (; b < nblocks; b += 8) s0 += partial[(int64_t)b * mm + e];
  }
  red[g][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (g == 0 && e < mm) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    const int row = e % rows, col = e / rows;
    out[(int64_t)(c0 + col) * ld + r0 + row] = t;
  }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Round-robin ordering of the Jacobi pairs: in round r of an even order KP
// the KP / 2 pairs u = 0 .. KP/2 - 1 are disjoint and every pair of indices
// meets once in KP - 1 rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rr_pair(int KP, int r, int u, int* p, int* q) {
  if (u == 0) {
    *p = KP - 1;
    *q = r;
  } else {
    *p = (r + u) % (KP - 1);
    *q = (r - u + (KP - 1)) % (KP - 1);
  }
}

// ---------------------------------------------------------------------------
// Eigen-decomposition of the positive semi-definite Gram matrix for the FP32
// preconditioner, one CTA, FP32: pivoted Cholesky G = L L^T (the largest
// remaining diagonal first; it stops where the pivot is no longer positive),
// then one-sided (Hestenes) Jacobi on the columns of L: plane rotations from
// the right make them mutually orthogonal, L W = U Sigma with W orthogonal,
// so G = U Sigma^2 U^T: the normalised columns are eigenvectors and their
// squared norms the eigenvalues, and W is never formed.  L is the transposed
// triangular factor of a column-pivoted QR of the samples, the starting point
// of the preconditioned Jacobi SVD of Drmac and Veselic (SIAM J. Matrix Anal.
// Appl. 29, 2008).  A round rotates disjoint pairs of the round-robin
// ordering, one warp per pair with its lanes holding rows, so a round needs
// no per-element bookkeeping and no eigenvector accumulation.  Eigenpairs
// beyond the numerical rank come out as zeros; K <= 128.
// ---------------------------------------------------------------------------
constexpr int CE_THREADS = 512;
constexpr int CE_MAX_SWEEPS = 32;

// Rows of a column, padded to whole 32-row groups (one float4 per lane of an
// eight-lane pair group and group).
__host__ __device__ constexpr int chol_eig_ldx(int K) { return (K + 31) / 32 * 32; }

// Dynamic shared memory: two buffers of the trailing matrix (K x (K + 1)),
// later reused for the pair table; the factor L (K columns of
// chol_eig_ldx(K) rows); positions' original indices (two buffers); column
// norms.
__host__ __device__ constexpr size_t chol_eig_smem(int K) {
  return (size_t)2 * K * (K + 1) * 4 + (size_t)K * chol_eig_ldx(K) * 4 + (size_t)K * 12 + 64;
}

// NV = chol_eig_ldx(K) / 32 float4 per lane and column.
// complete != 0: the eigenvectors beyond the numerical rank are replaced by
// an orthonormal basis of the complement (unit vectors orthogonalised twice
// against the columns before them), so that V is a full orthonormal basis.
template <int NV>
__global__ void __launch_bounds__(CE_THREADS) k_chol_jacobi_eig(const double* __restrict__ G, int K, float tol,
                                                                int complete, double* __restrict__ evals,
                                                                double* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int LD = K + 1, LDX = 32 * NV;
  float* cur = reinterpret_cast<float*>(smem_raw);  // trailing matrix, lower triangle, by position
  float* nxt = cur + K * LD;
  float* X = nxt + K * LD;                          // X[c * LDX + i]: column c of L, row = original index
  int* oc = reinterpret_cast<int*>(X + K * LDX);    // original index of each position (two buffers)
  int* on = oc + K;
  float* lam = reinterpret_cast<float*>(on + K);
  uchar2* pairs = reinterpret_cast<uchar2*>(smem_raw);  // after the factorisation
  __shared__ int rotated[CE_MAX_SWEEPS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = CE_THREADS / 32;
  for (int e = tid; e < K * K; e += CE_THREADS) {
    const int i = e / K, m = e - i * K;
    if (m <= i) cur[i * LD + m] = (float)G[(int64_t)m * K + i];
  }
  for (int e = tid; e < K * LDX; e += CE_THREADS) X[e] = 0.0f;
  for (int i = tid; i < K; i += CE_THREADS) oc[i] = i;
  for (int i = tid; i < CE_MAX_SWEEPS; i += CE_THREADS) rotated[i] = 0;
  __syncthreads();
  // entry (x, y) of the symmetric trailing matrix from its lower triangle;
  // the index is selected, not the load, so lanes do not diverge
  auto sym = [&](const float* a, int x, int y) { return a[max(x, y) * LD + min(x, y)]; };

  // pivoted Cholesky; step j moves the pivot to position j (rows and columns
  // of the trailing matrix are read through the swap, the new trailing
  // matrix goes to the other buffer)
  int r = K;
  float d0 = 0.0f;
  for (int j = 0; j < K; ++j) {
    // every warp finds the pivot itself: largest diagonal, ties by position
    float best = -1.0f;
    int bi = j;
    for (int i = j + lane; i < K; i += 32) {
      const float v = cur[i * LD + i];
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    const int p = bi;
    const float d = best;
    if (j == 0) d0 = d;
    if (!(d > 0.0f) || !(d >= 1e-30f * d0)) {  // (NaN fails too) numerical rank reached
      r = j;
      break;
    }
    const float isd = rsqrtf(d), sd = d * isd, id = isd * isd;
    const int t = tid >> 2, sub = tid & 3;  // four threads per trailing row
    const int i = j + 1 + t;
    if (i < K) {
      const int si = i == p ? j : i;
      const int oi = oc[si];  // the row's original index
      const float lip = sym(cur, si, p);
      if (sub == 0) {
        on[i] = oi;
        X[j * LDX + oi] = lip * isd;
      }
      const float f = lip * id;
#pragma unroll 4
      for (int m = j + 1 + sub; m <= i; m += 4) {
        const int sm = m == p ? j : m;
        nxt[i * LD + m] = fmaf(-f, sym(cur, sm, p), sym(cur, si, sm));
      }
    }
    if (tid == 0) X[j * LDX + oc[p]] = sd;
    __syncthreads();
    float* tmp = cur;
    cur = nxt;
    nxt = tmp;
    int* ti = oc;
    oc = on;
    on = ti;
  }

  // one-sided Jacobi on the r columns of L.  Eight lanes rotate one pair
  // (lane g holds rows 4g..4g+3 of every 32-row group), four pairs per warp;
  // the round-robin pairs of every round are tabulated first.
  const int R = r + (r & 1), H = R / 2;
  for (int e = tid; e < (R - 1) * H; e += CE_THREADS) {
    int pp, qq;
    rr_pair(R, e / H, e % H, &pp, &qq);
    pairs[e] = make_uchar2((unsigned char)pp, (unsigned char)qq);
  }
  __syncthreads();
  const int g = lane & 7;
  const int u = warp * 4 + (lane >> 3);  // this group's pair (K <= 128: one pass)
  for (int sweep = 0; sweep < CE_MAX_SWEEPS && R >= 2; ++sweep) {
    for (int rd = 0; rd < R - 1; ++rd) {
      int p = R, q = R;
      if (u < H) {
        const uchar2 pq = pairs[rd * H + u];
        p = pq.x;
        q = pq.y;
      }
      const bool act = p < r && q < r;  // (the padding column of an odd rank stays)
      float4 vp[NV], vq[NV];
      float a = 0.0f, b = 0.0f, c = 0.0f;
      if (act) {
        const float4* xp = reinterpret_cast<const float4*>(X + p * LDX) + g;
        const float4* xq = reinterpret_cast<const float4*>(X + q * LDX) + g;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          vp[v] = xp[8 * v];
          vq[v] = xq[8 * v];
          a = fmaf(vp[v].x, vp[v].x, fmaf(vp[v].y, vp[v].y, fmaf(vp[v].z, vp[v].z, fmaf(vp[v].w, vp[v].w, a))));
          b = fmaf(vq[v].x, vq[v].x, fmaf(vq[v].y, vq[v].y, fmaf(vq[v].z, vq[v].z, fmaf(vq[v].w, vq[v].w, b))));
          c = fmaf(vp[v].x, vq[v].x, fmaf(vp[v].y, vq[v].y, fmaf(vp[v].z, vq[v].z, fmaf(vp[v].w, vq[v].w, c))));
        }
      }
      // butterfly within the eight-lane group: identical sums in its lanes
      for (int off = 1; off < 8; off <<= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
      }
      if (act && fabsf(c) * rsqrtf(a) * rsqrtf(b) > tol) {  // (a zero column gives NaN: no rotation)
        // the rotation zeroing the pair's inner product (Rutishauser's
        // formulas); |zeta| is capped so that zeta^2 stays finite
        const float zeta = __fdividef(b - a, 2.0f * c);
        const float z = fminf(fabsf(zeta), 1e18f);
        const float w = fmaf(z, z, 1.0f);
        const float tt = copysignf(__fdividef(1.0f, z + w * rsqrtf(w)), zeta);
        const float cs = rsqrtf(fmaf(tt, tt, 1.0f)), sn = cs * tt;
        float4* xp = reinterpret_cast<float4*>(X + p * LDX) + g;
        float4* xq = reinterpret_cast<float4*>(X + q * LDX) + g;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 P0 = vp[v], Q0 = vq[v];
          xp[8 * v] = make_float4(cs * P0.x - sn * Q0.x, cs * P0.y - sn * Q0.y, cs * P0.z - sn * Q0.z,
                                  cs * P0.w - sn * Q0.w);
          xq[8 * v] = make_float4(sn * P0.x + cs * Q0.x, sn * P0.y + cs * Q0.y, sn * P0.z + cs * Q0.z,
                                  sn * P0.w + cs * Q0.w);
        }
        if (g == 0) rotated[sweep] = 1;
      }
      __syncthreads();
    }
    if (!rotated[sweep]) break;  // written only in this sweep, read after its last barrier
  }

  // eigenvalues = squared column norms; columns normalised in place
  for (int c = warp; c < r; c += NW) {
    float s = 0.0f;
    for (int i = lane; i < K; i += 32) s = fmaf(X[c * LDX + i], X[c * LDX + i], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const float inv = s > 0.0f ? 1.0f / sqrtf(s) : 0.0f;
    for (int i = lane; i < K; i += 32) X[c * LDX + i] *= inv;
    if (lane == 0) lam[c] = s;
  }
  __syncthreads();
  if (complete && r < K) {
    // unit vectors e_m (the first m whose remainder is not too small), made
    // orthogonal to the columns before them by two classical Gram-Schmidt
    // passes; some e_m keeps at least 1/sqrt(K) of its length
    float* v = nxt;           // K (free after the factorisation)
    float* h = nxt + LDX;     // K
    __shared__ float nrm;
    const float accept = 0.3f * rsqrtf((float)K);
    for (int c = r; c < K; ++c) {
      for (int m = 0; m < K; ++m) {
        for (int i = tid; i < K; i += CE_THREADS) {
          float s = i == m ? 1.0f : 0.0f;
          for (int b = 0; b < c; ++b) s = fmaf(-X[b * LDX + i], X[b * LDX + m], s);
          v[i] = s;
        }
        __syncthreads();
        for (int b = warp; b < c; b += NW) {
          float s = 0.0f;
          for (int i = lane; i < K; i += 32) s = fmaf(X[b * LDX + i], v[i], s);
          for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
          if (lane == 0) h[b] = s;
        }
        __syncthreads();
        float vmine = 0.0f;  // entry tid of the remainder (K <= 128 < CE_THREADS)
        if (tid < K) {
          float s = v[tid];
          for (int b = 0; b < c; ++b) s = fmaf(-h[b], X[b * LDX + tid], s);
          vmine = s;
        }
        if (warp == 0) {
          float s = 0.0f;
          for (int i = lane; i < K; i += 32) {
            float w = v[i];
            for (int b = 0; b < c; ++b) w = fmaf(-h[b], X[b * LDX + i], w);
            s = fmaf(w, w, s);
          }
          for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
          if (lane == 0) nrm = sqrtf(s);
        }
        __syncthreads();
        const float nv = nrm;
        if (nv > accept) {
          if (tid < K) X[c * LDX + tid] = vmine / nv;
          __syncthreads();
          break;
        }
      }
      if (tid == 0) lam[c] = 0.0f;
    }
    __syncthreads();
  }
  // sort descending (ties by column); zero columns past the rank unless completed
  for (int c = warp; c < K; c += NW) {
    if (c < r) {
      const float lc = lam[c];
      int pos = 0;
      for (int b2 = lane; b2 < r; b2 += 32) pos += (lam[b2] > lc) || (lam[b2] == lc && b2 < c);
      for (int off = 16; off > 0; off >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, off);
      if (lane == 0) evals[pos] = (double)lc;
      for (int i = lane; i < K; i += 32) V[(int64_t)pos * K + i] = (double)X[c * LDX + i];
    } else {
      if (lane == 0) evals[c] = 0.0;
      for (int i = lane; i < K; i += 32) V[(int64_t)c * K + i] = complete ? (double)X[c * LDX + i] : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// Eigen-decomposition of the Gram matrix for 128 < K <= 256 on a cluster of
// two CTAs, FP32: one-sided (Hestenes) Jacobi on the columns of G itself.
// For the symmetric positive semi-definite G, G W = U Lambda with W
// orthogonal, so the normalised columns are eigenvectors and the column
// norms the eigenvalues.  The K x K columns (256 KB in FP32) do not fit one
// CTA: each rank keeps Kc = K / 2 of them in shared memory, a round's disjoint
// pairs alternate between the ranks (pair u on rank u % 2), and a column
// owned by the other rank is read and written through distributed shared
// memory; the cluster barrier ends every round.  Eight lanes rotate one
// pair as in k_chol_jacobi_eig.  NV = ceil(K / 32) float4 per lane and
// column.
// ---------------------------------------------------------------------------
constexpr int CJ_THREADS = 512;
constexpr int CJ_RANKS = 2;
constexpr int CJ_MAX_SWEEPS = 40;

__host__ __device__ constexpr size_t cluster_eig_smem(int K) {
  return (size_t)((K + CJ_RANKS - 1) / CJ_RANKS) * ((K + 31) / 32 * 32) * 4 + (size_t)K * 8 + 64;
}

template <int NV>
__global__ void __launch_bounds__(CJ_THREADS, 1) k_cluster_jacobi_eig(const double* __restrict__ G, int K, float tol,
                                                                      double* __restrict__ evals,
                                                                      double* __restrict__ V) {
  namespace cgx = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int LDX = 32 * NV;
  cgx::cluster_group cl = cgx::this_cluster();
  const int rank = (int)cl.block_rank();
  const int Kc = (K + CJ_RANKS - 1) / CJ_RANKS;
  float* X = reinterpret_cast<float*>(smem_raw);  // [Kc][LDX]: columns rank Kc ..
  float* lam = X + (size_t)Kc * LDX;              // [K]: this rank's entries (read by the others)
  float* lall = lam + K;                          // [K]: every rank's, gathered
  __shared__ int rotated[CJ_MAX_SWEEPS];
  __shared__ float* xr[CJ_RANKS];
  __shared__ float* lr[CJ_RANKS];
  __shared__ int* rr[CJ_RANKS];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int e = tid; e < Kc * LDX; e += CJ_THREADS) {
    const int c = e / LDX, i = e - c * LDX;
    const int gc = rank * Kc + c;
    X[e] = (gc < K && i < K) ? (float)G[(int64_t)gc * K + i] : 0.0f;
  }
  for (int i = tid; i < CJ_MAX_SWEEPS; i += CJ_THREADS) rotated[i] = 0;
  if (tid < CJ_RANKS) {
    xr[tid] = cl.map_shared_rank(X, tid);
    lr[tid] = cl.map_shared_rank(lam, tid);
    rr[tid] = cl.map_shared_rank(&rotated[0], tid);
  }
  cl.sync();
  auto col = [&](int c) { return xr[c / Kc] + (size_t)(c % Kc) * LDX; };
  const int R = K + (K & 1), H = R / 2;
  const int g = lane & 7;
  const int u = rank + CJ_RANKS * (tid >> 3);  // this group's pair (H <= 128: one pass)
  for (int sweep = 0; sweep < CJ_MAX_SWEEPS; ++sweep) {
    for (int rd = 0; rd < R - 1; ++rd) {
      int p = R, q = R;
      if (u < H) rr_pair(R, rd, u, &p, &q);
      const bool act = p < K && q < K;
      float4 vp[NV], vq[NV];
      float a = 0.0f, b = 0.0f, c = 0.0f;
      float4* xp = nullptr;
      float4* xq = nullptr;
      if (act) {
        xp = reinterpret_cast<float4*>(col(p)) + g;
        xq = reinterpret_cast<float4*>(col(q)) + g;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          vp[v] = xp[8 * v];
          vq[v] = xq[8 * v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          a = fmaf(vp[v].x, vp[v].x, fmaf(vp[v].y, vp[v].y, fmaf(vp[v].z, vp[v].z, fmaf(vp[v].w, vp[v].w, a))));
          b = fmaf(vq[v].x, vq[v].x, fmaf(vq[v].y, vq[v].y, fmaf(vq[v].z, vq[v].z, fmaf(vq[v].w, vq[v].w, b))));
          c = fmaf(vp[v].x, vq[v].x, fmaf(vp[v].y, vq[v].y, fmaf(vp[v].z, vq[v].z, fmaf(vp[v].w, vq[v].w, c))));
        }
      }
      for (int off = 1; off < 8; off <<= 1) {  // butterfly within the eight-lane group
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
      }
      if (act && fabsf(c) * rsqrtf(a) * rsqrtf(b) > tol) {  // (a zero column gives NaN: no rotation)
        const float zeta = __fdividef(b - a, 2.0f * c);
        const float z = fminf(fabsf(zeta), 1e18f);
        const float w = fmaf(z, z, 1.0f);
        const float tt = copysignf(__fdividef(1.0f, z + w * rsqrtf(w)), zeta);
        const float cs = rsqrtf(fmaf(tt, tt, 1.0f)), sn = cs * tt;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 P0 = vp[v], Q0 = vq[v];
          xp[8 * v] = make_float4(cs * P0.x - sn * Q0.x, cs * P0.y - sn * Q0.y, cs * P0.z - sn * Q0.z,
                                  cs * P0.w - sn * Q0.w);
          xq[8 * v] = make_float4(sn * P0.x + cs * Q0.x, sn * P0.y + cs * Q0.y, sn * P0.z + cs * Q0.z,
                                  sn * P0.w + cs * Q0.w);
        }
        if (g == 0) rotated[sweep] = 1;
      }
      cl.sync();
    }
    // any rotation on any rank (flags of this sweep are final after the barrier)
    int any = 0;
    for (int q2 = 0; q2 < CJ_RANKS; ++q2) any |= rr[q2][sweep];
    if (!any) break;  // the same decision on every rank
  }
  // eigenvalues = column norms (G W = U Lambda)
  const int warp = tid >> 5;
  for (int c = warp; c < Kc; c += CJ_THREADS / 32) {
    const int gc = rank * Kc + c;
    float s2 = 0.0f;
    for (int i = lane; i < K; i += 32) s2 = fmaf(X[(size_t)c * LDX + i], X[(size_t)c * LDX + i], s2);
    for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    if (lane == 0 && gc < K) lam[gc] = sqrtf(s2);
  }
  cl.sync();
  // every rank's eigenvalues, then the position and output of the own columns
  for (int c = tid; c < K; c += CJ_THREADS) lall[c] = lr[c / Kc][c];
  __syncthreads();
  for (int c = warp; c < Kc; c += CJ_THREADS / 32) {
    const int gc = rank * Kc + c;
    if (gc >= K) continue;
    const float lc = lall[gc];
    int pos = 0;
    for (int b2 = lane; b2 < K; b2 += 32) pos += (lall[b2] > lc) || (lall[b2] == lc && b2 < gc);
    for (int off = 16; off > 0; off >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, off);
    const float inv = lc > 0.0f ? 1.0f / lc : 0.0f;
    if (lane == 0) evals[pos] = (double)lc;
    for (int i = lane; i < K; i += 32) V[(int64_t)pos * K + i] = (double)(X[(size_t)c * LDX + i] * inv);
  }
  cl.sync();  // no rank leaves while another may still read its shared memory
}

// Ogita & Aishima, "Iterative refinement for symmetric eigenvalue
// decomposition" (Japan J. Indust. Appl. Math., 2018), one step, given
// XtX = X^T X and S = X^T G X:  R = I - XtX, lambda_i = S_ii / (1 - R_ii),
// E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) when the gap exceeds
// delta = 2 (||S - diag(lambda)|| + ||G|| ||R||), else R_ij / 2; E_ii = R_ii / 2.
// Writes E and lambda; the caller forms X <- X + X E.
// One block per column j of E (K <= 256 blocks): every block forms lambda,
// the two norms and max |lambda| itself (K^2 cheap reads), then divides only
// its column, so the K^2 FP64 divisions are spread over K SMs.
__global__ void k_oa_step(const double* __restrict__ XtX, const double* __restrict__ S, int K, double* __restrict__ E,
                          double* __restrict__ lam) {
  __shared__ double red[32];
  __shared__ double lm[256];
  __shared__ double mx;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < K; i += nt) {
    const double rii = 1.0 - XtX[(int64_t)i * K + i];
    lm[i] = S[(int64_t)i * K + i] / (1.0 - rii);
    if (blockIdx.x == 0) lam[i] = lm[i];
  }
  __syncthreads();
  double so = 0.0, rr = 0.0, lmax = 0.0;
  for (int e = tid; e < K * K; e += nt) {
    const int i = e % K, j = e / K;
    const double r = (i == j ? 1.0 : 0.0) - XtX[e];
    rr += r * r;
    if (i != j) so += S[e] * S[e];
  }
  for (int i = tid; i < K; i += nt) {
    const double d = S[(int64_t)i * K + i] - lm[i];
    so += d * d;
    lmax = fmax(lmax, fabs(lm[i]));
  }
  so = block_sum(so, red);
  rr = block_sum(rr, red);
  // max |lambda| over the block: warp maxima, then warp 0
  for (int off = 16; off > 0; off >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
  if ((tid & 31) == 0) red[tid >> 5] = lmax;
  __syncthreads();
  if (tid < 32) {
    double m = tid < (nt >> 5) ? red[tid] : 0.0;
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (tid == 0) mx = m;
  }
  __syncthreads();
  const double delta = 2.0 * (sqrt(so) + mx * sqrt(rr));
  const int j = blockIdx.x;
  for (int i = tid; i < K; i += nt) {
    const int64_t e = (int64_t)j * K + i;
    const double r = (i == j ? 1.0 : 0.0) - XtX[e];
    double v;
    if (i == j) v = 0.5 * r;
    else if (fabs(lm[j] - lm[i]) > delta) v = (S[e] + lm[j] * r) / (lm[j] - lm[i]);
    else v = 0.5 * r;
    E[e] = v;
  }
}

__global__ void k_add(double* __restrict__ X, const double* __restrict__ Y, int count) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x) X[e] += Y[e];
}

// Sorts eigenpairs descending: lam (K), X (K x K, columns) -> evals, V.  One
// warp per eigenpair (its rank counted by the lanes, then its column copied).
__global__ void k_sort_eig(const double* __restrict__ lam, const double* __restrict__ X, int K,
                           double* __restrict__ evals, double* __restrict__ V) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = threadIdx.x >> 5; a < K; a += nw) {
    const double la = lam[a];
    int pos = 0;
    for (int b = lane; b < K; b += 32) pos += (lam[b] > la) || (lam[b] == la && b < a);
    for (int off = 16; off > 0; off >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, off);
    if (lane == 0) evals[pos] = la;
    for (int row = lane; row < K; row += 32) V[(int64_t)pos * K + row] = X[(int64_t)a * K + row];
  }
}

// M = V[:, :k] diag(1 / sqrt(lambda)) as T (K x k, row-major: M[c * k + j]);
// sigma = sqrt(lambda).  Flags a non-positive lambda_j (j < k).
template <typename T>
__global__ void k_make_basis_coeffs(const double* __restrict__ evals, const double* __restrict__ V, int K, int k,
                                    T* __restrict__ M, double* __restrict__ sigma, int* status) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * k; e += gridDim.x * blockDim.x) {
    const int c = e / k, j = e % k;
    const double lj = evals[j];
    M[e] = lj > 0.0 ? (T)(V[(int64_t)j * K + c] / sqrt(lj)) : T(0);
  }
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      const double lj = evals[j];
      sigma[j] = lj > 0.0 ? sqrt(lj) : 0.0;
      if (j < k && !(lj > 0.0)) atomicExch(status, (int)NLSP_ERR_NOT_SPD);
    }
}

// Out_t = In_t * M for every node tile: In tiled with `ncin` columns, M is
// ncin x k (row-major), Out tiled with k columns.  One thread per node of a
// tile; outputs in register chunks of KC columns.  M sits in shared memory
// with its rows padded with zeros to ldm, a multiple of KC, so the product
// loop needs no column test; it is read as 16-byte broadcasts.  The input
// column loads are issued CU at a time ahead of their products.
// This launch forms output columns [jlo, jlo + jw) (M's columns staged for
// them only).
template <typename T, int KC, int CU>
__global__ void __launch_bounds__(NLSP_TILE) k_tile_times_small(const T* __restrict__ In, int ncin,
                                                               const T* __restrict__ Mg, int k, int64_t n_pad,
                                                               T* __restrict__ Out, int jlo, int jw) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::N;
  static_assert(KC % VN == 0, "KC must be a multiple of the vector width");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* M = reinterpret_cast<T*>(smem_raw);
  const int ldm = (jw + KC - 1) / KC * KC;
  for (int e = threadIdx.x; e < ncin * ldm; e += blockDim.x) {
    const int c = e / ldm, j = e % ldm;
    M[e] = j < jw ? Mg[c * k + jlo + j] : T(0);
  }
  __syncthreads();
  const int64_t ntiles = n_pad / NLSP_TILE;
  const int w = threadIdx.x;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const T* in = In + t * ncin * NLSP_TILE + w;
    T* out = Out + t * (int64_t)k * NLSP_TILE + w;
    for (int j0 = 0; j0 < jw; j0 += KC) {
      T acc[KC];
#pragma unroll
      for (int j = 0; j < KC; ++j) acc[j] = T(0);
      int c0 = 0;
      for (; c0 + CU <= ncin; c0 += CU) {
        T sv[CU];
#pragma unroll
        for (int u = 0; u < CU; ++u) sv[u] = in[(int64_t)(c0 + u) * NLSP_TILE];
#pragma unroll
        for (int u = 0; u < CU; ++u) {
          const T* mrow = M + (c0 + u) * ldm + j0;
#pragma unroll
          for (int j = 0; j < KC; j += VN) {
            T mv[VN];
            *reinterpret_cast<V*>(mv) = *reinterpret_cast<const V*>(mrow + j);
#pragma unroll
            for (int q = 0; q < VN; ++q) acc[j + q] += sv[u] * mv[q];
          }
        }
      }
      for (; c0 < ncin; ++c0) {
        const T s = in[(int64_t)c0 * NLSP_TILE];
        const T* mrow = M + c0 * ldm + j0;
#pragma unroll
        for (int j = 0; j < KC; j += VN) {
          T mv[VN];
          *reinterpret_cast<V*>(mv) = *reinterpret_cast<const V*>(mrow + j);
#pragma unroll
          for (int q = 0; q < VN; ++q) acc[j + q] += s * mv[q];
        }
      }
#pragma unroll
      for (int j = 0; j < KC; ++j)
        if (j0 + j < jw) out[(int64_t)(jlo + j0 + j) * NLSP_TILE] = acc[j];
    }
  }
}

// ---------------------------------------------------------------------------
// Dense FP64 Cholesky A = L L^T of an m x m SPD matrix in one CTA of 256
// threads (right-looking, shared memory, column-major), one barrier per
// column.  In the pass for column j every thread reads the pivot words of
// column j (1 / d and 1 / sqrt(d), d = a_jj), writes its share of column j
// scaled by 1 / sqrt(d) and updates the trailing lower triangle with the
// unscaled column, a_ci -= a_ji a_jc / d (a 16 x 16 thread grid over the
// (c, i >= c) pairs).  Thread 0's first element is a_{j+1,j+1}, so it forms
// the next pivot words right after updating it, into the other half of a
// double-buffered pair.  A non-positive or non-finite pivot sets
// NLSP_ERR_NOT_SPD and L is returned as zeros.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool chol_pivot(double d, double* piv, double* ljj) {
  if (!(d > 0.0) || !isfinite(d)) return false;
  const double rl = rsqrt(d);
  piv[0] = rl * rl;
  piv[1] = rl;
  *ljj = d * rl;
  return true;
}

__global__ void __launch_bounds__(256) k_cholesky(const double* __restrict__ Ain, int m, double* __restrict__ Lout,
                                                  int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* a = reinterpret_cast<double*>(smem_raw);  // column-major m x m
  __shared__ double piv[2][2];                       // [column parity] {1 / d, 1 / sqrt(d)}
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tx = tid % 16, ty = tid / 16;
  for (int e = tid; e < m * m; e += nt) a[e] = Ain[e];
  if (tid == 0) bad = 0;
  __syncthreads();
  if (tid == 0) {
    double l;
    if (chol_pivot(a[0], piv[0], &l)) Lout[0] = l;
    else bad = 1;
  }
  __syncthreads();
  for (int j = 0; j < m && !bad; ++j) {
    const double inv_d = piv[j & 1][0], inv_l = piv[j & 1][1];
    for (int i = j + 1 + tid; i < m; i += nt) Lout[(int64_t)j * m + i] = a[j * m + i] * inv_l;
    const int rem = m - j - 1;
    for (int cy = ty; cy < rem; cy += 16) {
      const int c = j + 1 + cy;
      const double t = a[j * m + c] * inv_d;
      for (int ix = cy + tx; ix < rem; ix += 16) {
        const int i = j + 1 + ix;
        const double v = a[c * m + i] - a[j * m + i] * t;
        a[c * m + i] = v;
        if (tid == 0 && ix == 0 && cy == 0) {  // v = a_{j+1, j+1}: next pivot
          double l;
          if (chol_pivot(v, piv[(j + 1) & 1], &l)) Lout[(int64_t)(j + 1) * m + j + 1] = l;
          else bad = 1;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && bad) atomicExch(status, (int)NLSP_ERR_NOT_SPD);
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, c = e / m;
    if (bad || i < c) Lout[e] = 0.0;
  }
}

// Column q of A^-1 = L^-T L^-1 e_q by one warp, in the column (axpy) form
// of both substitutions so that no step needs a reduction: forward,
// y_i /= L_ii then y_c -= L_ci y_i for c > i (starting at i = q, since
// (L^-1 e_q)_i = 0 for i < q); backward, x_i = y_i / L_ii then
// y_c -= L_ic x_i for c < i.  L is staged in shared memory with leading
// dimension m + 1, so its columns (forward) and rows (backward) are both
// read without bank conflicts; the reciprocal diagonal is formed once.
__global__ void __launch_bounds__(32) k_spd_inverse_cols(const double* __restrict__ L, int m,
                                                         double* __restrict__ Ainv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = m + 1;
  double* Ls = reinterpret_cast<double*>(smem_raw);  // L(i, c) at c * ld + i
  double* y = Ls + (size_t)m * ld;
  double* dinv = y + m;
  const int q = blockIdx.x, lane = threadIdx.x;
  for (int e = lane; e < m * m; e += 32) Ls[(e / m) * ld + (e % m)] = L[e];
  __syncwarp();
  for (int i = lane; i < m; i += 32) {
    dinv[i] = 1.0 / Ls[i * ld + i];
    y[i] = (i == q) ? 1.0 : 0.0;
  }
  __syncwarp();
  for (int i = q; i < m; ++i) {  // L y = e_q
    const double yi = y[i] * dinv[i];
    __syncwarp();
    if (lane == 0) y[i] = yi;
    for (int c = i + 1 + lane; c < m; c += 32) y[c] -= Ls[i * ld + c] * yi;
    __syncwarp();
  }
  for (int i = m - 1; i >= 0; --i) {  // L^T x = y  (x overwrites y)
    const double xi = y[i] * dinv[i];
    __syncwarp();
    if (lane == 0) y[i] = xi;
    for (int c = lane; c < i; c += 32) y[c] -= Ls[c * ld + i] * xi;
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) Ainv[(int64_t)q * m + i] = y[i];
}

// Dynamic shared memory of k_spd_inverse_cols for order m.
inline size_t spd_inverse_smem(int m) { return sizeof(double) * ((size_t)m * (m + 1) + 2 * (size_t)m); }

// C (m x n) = op(A) op(B), op(A) m x kk, op(B) kk x n, all FP64 column-major
// with leading dimensions; ta / tb select the transposes.  A 16 x 16 block
// grid over C.
__global__ void __launch_bounds__(256) k_gemm_small(const double* __restrict__ A, int lda, int ta,
                                                    const double* __restrict__ B, int ldb, int tb,
                                                    double* __restrict__ C, int ldc, int m, int n, int kk) {
  // one 16 x 16 tile of C per block; the inner dimension in strips of up to
  // 128 (one strip, i.e. one round of loads, for K <= 128), op(A) and op(B)
  // strips staged in shared memory with loads coalesced along the stored
  // dimension, then four interleaved FP64 FMA chains per output
  constexpr int LC = 128;
  __shared__ double As[LC][17];      // op(A)(i0 + ii, l0 + l) at As[l][ii]
  __shared__ double Bs[16][LC + 1];  // op(B)(l0 + l, j0 + jj) at Bs[jj][l]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (int l0 = 0; l0 < kk; l0 += LC) {
    const int lw = min(LC, kk - l0);
    for (int e = tid; e < 16 * LC; e += 256) {
      const int ii = ta ? e / LC : e % 16, la = ta ? e % LC : e / 16;
      const int ai = i0 + ii, al = l0 + la;
      As[la][ii] = (ai < m && la < lw) ? (ta ? A[(int64_t)ai * lda + al] : A[(int64_t)al * lda + ai]) : 0.0;
      const int jj = tb ? e % 16 : e / LC, lb = tb ? e / 16 : e % LC;
      const int bj = j0 + jj, bl = l0 + lb;
      Bs[jj][lb] = (bj < n && lb < lw) ? (tb ? B[(int64_t)bl * ldb + bj] : B[(int64_t)bj * ldb + bl]) : 0.0;
    }
    __syncthreads();
    for (int l = 0; l < lw; l += 4) {  // entries past lw are zero
      a0 = fma(As[l][tx], Bs[ty][l], a0);
      a1 = fma(As[l + 1][tx], Bs[ty][l + 1], a1);
      a2 = fma(As[l + 2][tx], Bs[ty][l + 2], a2);
      a3 = fma(As[l + 3][tx], Bs[ty][l + 3], a3);
    }
    __syncthreads();
  }
  if (i0 + tx < m && j0 + ty < n) C[(int64_t)(j0 + ty) * ldc + i0 + tx] = (a0 + a1) + (a2 + a3);
}

// Coefficients of the randomised basis: M = X V[:, :k] (K x k, row-major
// M[c * k + j], precision T) from X (K x l) and the eigenvectors V (l x l) of
// B B^T; sigma = sqrt of its l eigenvalues (zero beyond l, up to K).  Flags a
// non-positive eigenvalue among the first k.
template <typename T>
__global__ void k_randomized_coeffs(const double* __restrict__ X, const double* __restrict__ V,
                                    const double* __restrict__ evals, int K, int l, int k, T* __restrict__ M,
                                    double* __restrict__ sigma, int* status) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * k; e += gridDim.x * blockDim.x) {
    const int c = e / k, j = e % k;
    double s = 0.0;
    for (int q = 0; q < l; ++q) s += X[(int64_t)q * K + c] * V[(int64_t)j * l + q];
    M[e] = (T)s;
  }
  if (blockIdx.x == 0)
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
      const double lj = j < l ? evals[j] : 0.0;
      sigma[j] = lj > 0.0 ? sqrt(lj) : 0.0;
      if (j < k && !(lj > 0.0)) atomicExch(status, (int)NLSP_ERR_NOT_SPD);
    }
}

__global__ void k_symmetrize(double* __restrict__ M, int m) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e % m, j = e / m;
    if (i < j) {
      const double v = 0.5 * (M[e] + M[(int64_t)i * m + j]);
      M[e] = v;
      M[(int64_t)i * m + j] = v;
    }
  }
}

}  // namespace

// ============================================================================
// Host orchestration.  Temporaries live in the context's grow-only scratch
// slots: SA/SB the two tiled sample blocks, PART the per-block partial
// products, SMALL the K x K work of the eigensolver, PNEW the re-orthonormal
// basis.
// ============================================================================
namespace {

template <typename T>
const StencilView<T>& view_of(const nlsp_op* A);
template <>
const StencilView<double>& view_of<double>(const nlsp_op* A) { return A->v64; }
template <>
const StencilView<float>& view_of<float>(const nlsp_op* A) { return A->v32; }

nlsp_status set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return NLSP_OK;
}

template <typename T>
T* slot_as(nlsp_ctx* ctx, int s, size_t count) {
  return reinterpret_cast<T*>(ctx_slot(ctx, s, sizeof(T) * count));
}

// X_t^T Y_t summed over all tiles -> out (ncx x ncx FP64, column-major),
// Y = X or A X.
template <typename T, bool WITH_A>
nlsp_status tsgemm(nlsp_ctx* ctx, const nlsp_op* A, const T* X, int ncols, int ncx, int64_t n_pad, double* out,
                   int symmetrize) {
  cudaStream_t s = ctx->stream;
  const int64_t ntiles = n_pad / NLSP_TILE;
  int launches = 0;
  // One product of X's columns [cx0, cx0 + nx) with Y's columns [cy0, cy0 +
  // ny) (Y = X, or A X), summed into out at (cx0, cy0).  Up to four resident
  // blocks per SM, so that one block's staging loads overlap another's
  // products; never more blocks than node chunks.
#define NLSP_TSGEMM_LAUNCH(RB, TD, TWO_, CX0, CY0, NX, NY)                                                \
  do {                                                                                                   \
    constexpr int LDS_ = RB * TD + (sizeof(T) == 4 ? 4 : 2);                                             \
    const size_t sm = (size_t)GRAM_CW * LDS_ * sizeof(T) * ((WITH_A || TWO_) ? 2 : 1);                   \
    NLSP_DISPATCH_KIND(A->kind, KD, {                                                                    \
      auto fn = k_tsgemm<T, RB, TD, KD, WITH_A, TWO_>;                                                   \
      NLSP_TRY(set_smem((const void*)fn, sm));                                                           \
      int per_sm = 1;                                                                                    \
      NLSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TD * TD, sm));                \
      const int blocks = (int)std::min<int64_t>((int64_t)ctx->num_sms * std::min(std::max(per_sm, 1), 4), \
                                                std::max<int64_t>(ntiles * (NLSP_TILE / GRAM_CW), 1));    \
      double* partial = slot_as<double>(ctx, SLOT_PART, (size_t)blocks * (NX) * (NY));                   \
      if (!partial) return NLSP_ERR_OOM;                                                                 \
      fn<<<blocks, TD * TD, sm, s>>>(view_of<T>(A), X, ncols, NX, n_pad, partial, CX0, CY0, NY);         \
      NLSP_LAUNCH_CHECK();                                                                               \
      k_sum_partials<<<div_up((int64_t)(NX) * (NY), 32), 256, 0, s>>>(partial, blocks, NX, NY, out, ncx,  \
                                                                     CX0, CY0);                          \
      launches += 2;                                                                                     \
    });                                                                                                  \
  } while (0)
  if (ncx <= 32) NLSP_TSGEMM_LAUNCH(2, 16, false, 0, 0, ncx, ncx);
  else if (ncx <= 64) NLSP_TSGEMM_LAUNCH(4, 16, false, 0, 0, ncx, ncx);
  else if (ncx <= 128) NLSP_TSGEMM_LAUNCH(8, 16, false, 0, 0, ncx, ncx);
  else if (ncx <= 256) {
    // four quadrants of at most 128 x 128 (the off-diagonal ones computed
    // rather than mirrored, so that the A-product variant needs no symmetry)
    const int h = 128, rr = ncx - 128;
    NLSP_TSGEMM_LAUNCH(8, 16, !WITH_A, 0, 0, h, h);
    NLSP_TSGEMM_LAUNCH(8, 16, !WITH_A, 0, h, h, rr);
    NLSP_TSGEMM_LAUNCH(8, 16, !WITH_A, h, 0, rr, h);
    NLSP_TSGEMM_LAUNCH(8, 16, !WITH_A, h, h, rr, rr);
  } else {
    return NLSP_ERR_INVALID;
  }
#undef NLSP_TSGEMM_LAUNCH
  NLSP_LAUNCH_CHECK();
  if (symmetrize) {
    k_symmetrize<<<div_up((int64_t)ncx * ncx, 256), 256, 0, s>>>(out, ncx);
    NLSP_LAUNCH_CHECK();
    ++launches;
  }
  count_launches(ctx, launches);
  return NLSP_OK;
}

template <typename T>
nlsp_status tile_times_small(nlsp_ctx* ctx, const T* In, int ncin, const T* M, int k, int64_t n_pad, T* Out) {
  // register chunk: the smallest of 16 / 32 / 64 (FP64: 16 / 32) columns
  // that covers k, else the largest in several passes
  const int kc = k <= 16 ? 16 : (k <= 32 || sizeof(T) == 8) ? 32 : 64;
  const void* fn;
  if (kc == 16) fn = (const void*)k_tile_times_small<T, 16, 16>;
  else if (kc == 32) fn = (const void*)k_tile_times_small<T, 32, 16>;
  else fn = (const void*)k_tile_times_small<T, 64, 16>;
  // output columns per launch: all of them when M fits in shared memory,
  // else chunks of whole kc (a wide FP64 M: K = 256, k = 128 is 256 KB)
  const size_t limit = 200 * 1024;
  int width = (k + kc - 1) / kc * kc;
  while (width > kc && (size_t)ncin * width * sizeof(T) > limit) width -= kc;
  if ((size_t)ncin * width * sizeof(T) > limit) return NLSP_ERR_INVALID;
  NLSP_TRY(set_smem(fn, (size_t)ncin * width * sizeof(T)));
  const int64_t ntiles = n_pad / NLSP_TILE;
  const int g = (int)std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * 8);
  int launches = 0;
  for (int jlo = 0; jlo < k; jlo += width) {
    const int jw = std::min(width, k - jlo);
    const size_t sm = (size_t)ncin * ((jw + kc - 1) / kc * kc) * sizeof(T);
    if (kc == 16) k_tile_times_small<T, 16, 16><<<g, NLSP_TILE, sm, ctx->stream>>>(In, ncin, M, k, n_pad, Out, jlo, jw);
    else if (kc == 32)
      k_tile_times_small<T, 32, 16><<<g, NLSP_TILE, sm, ctx->stream>>>(In, ncin, M, k, n_pad, Out, jlo, jw);
    else k_tile_times_small<T, 64, 16><<<g, NLSP_TILE, sm, ctx->stream>>>(In, ncin, M, k, n_pad, Out, jlo, jw);
    NLSP_LAUNCH_CHECK();
    ++launches;
  }
  count_launches(ctx, launches);
  return NLSP_OK;
}

// Smooths the tiled sample block (ping-pong between a and tmp); *result is
// the buffer holding S.
template <typename T>
nlsp_status smooth_tiled(nlsp_ctx* ctx, const nlsp_op* A, int K, int s1, double omega, int64_t n_pad, T* a, T* tmp,
                         T** result) {
  T* src = a;
  T* dst = tmp;
  // columns per thread: 8 on large systems (67.8 us per sweep at 512^2, K =
  // 128, against 77.4 with 4), 4 where 8 would leave too few threads
  const bool wide = n_pad >= 65536;
  const int cpt = wide ? 8 : 4;
  const dim3 g((unsigned)div_up(n_pad, 256), (unsigned)div_up(K, cpt));
  // large 2D grids stream along rows in FP32 (62.8 against 69.7 us per sweep
  // at 512^2, K = 128; 587 against 662 at 1024^2, 9-point, K = 256); the
  // bands are as long as makes the grid one wave of resident blocks (equal
  // work, no partial last wave).  The FP64 sweep is bound by the FP64 pipe,
  // where the per-node kernel's lower register count keeps more warps busy
  // (349 against 394 us at 512^2, K = 128).
  const bool rows = wide && sizeof(T) == 4 && (A->kind == ST_5PT || A->kind == ST_9PT);
  dim3 gr(1, 1, 1);
  int band = 0;
  if (rows) {
    int per_sm = 0;
    NLSP_DISPATCH_KIND(A->kind, KD, {
      if constexpr ((KD == ST_5PT || KD == ST_9PT) && sizeof(T) == 4)
        NLSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smooth_rows<KD, T, 8>, SR_THREADS, 0));
    });
    const int strips = div_up(A->N, SR_THREADS) * div_up(K, 8);
    const int bands = std::max(1, std::max(per_sm, 1) * ctx->num_sms / strips);
    band = div_up(A->N, bands);
    gr = dim3((unsigned)div_up(A->N, SR_THREADS), (unsigned)div_up(A->N, band), (unsigned)div_up(K, 8));
  }
  for (int it = 0; it < s1; ++it) {
    NLSP_DISPATCH_KIND(A->kind, KD, {
      bool done = false;
      if constexpr ((KD == ST_5PT || KD == ST_9PT) && sizeof(T) == 4) {
        if (rows) {
          k_smooth_rows<KD, T, 8><<<gr, SR_THREADS, 0, ctx->stream>>>(view_of<T>(A), (T)omega, K, (int)n_pad, band,
                                                                       src, dst);
          done = true;
        }
      }
      if (!done && wide)
        k_smooth_sweep<KD, T, 8><<<g, 256, 0, ctx->stream>>>(view_of<T>(A), (T)omega, K, (int)n_pad, src, dst);
      else if (!done)
        k_smooth_sweep<KD, T, 4><<<g, 256, 0, ctx->stream>>>(view_of<T>(A), (T)omega, K, (int)n_pad, src, dst);
    });
    NLSP_LAUNCH_CHECK();
    std::swap(src, dst);
  }
  count_launches(ctx, s1);
  *result = src;
  return NLSP_OK;
}

nlsp_status check_setup_params(const nlsp_op* A, const nlsp_setup_params* p, bool need_K) {
  if (!A || !p) return NLSP_ERR_INVALID;
  if (p->precision < NLSP_FP64 || p->precision > NLSP_MIXED_TF32) return NLSP_ERR_INVALID;
  if (p->k < 1 || p->k > 128 || p->k > A->n) return NLSP_ERR_INVALID;
  if (need_K && (p->K < p->k || p->K > 256 || p->K > A->n || p->s1 < 0)) return NLSP_ERR_INVALID;
  if (p->nu1 < 1 || p->nu2 != p->nu1 || p->nu1 > 64) return NLSP_ERR_INVALID;
  if (!(p->omega > 0.0) || !(p->omega < 2.0)) return NLSP_ERR_INVALID;
  return NLSP_OK;
}

nlsp_prec* new_prec(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* p, int k, int K) {
  nlsp_prec* M = new nlsp_prec();
  memset(M, 0, sizeof(*M));
  M->ctx = ctx;
  M->device = ctx->device;
  M->A = A;
  M->precision = p->precision;
  M->n = A->n;
  M->n_pad = pad_tile(A->n);
  M->k = k;
  M->r = k;
  M->K = K;
  M->nu1 = p->nu1;
  M->nu2 = p->nu2;
  M->omega = p->omega;
  const int ntiles = (int)(M->n_pad / NLSP_TILE);
  M->rblocks = std::max(2 * ctx->num_sms, div_up((int64_t)ntiles * NLSP_TILE, 16384));
  return M;
}

// The preconditioner's own storage: one allocation carved into its arrays.
nlsp_status alloc_prec_storage(nlsp_prec* M) {
  const size_t tsz = M->precision == NLSP_FP64 ? sizeof(double) : sizeof(float);
  const size_t k = M->k;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t sizes[] = {up(tsz * M->n_pad * k), up(sizeof(double) * std::max(M->K, 1)), up(sizeof(double) * k * k),
                          up(sizeof(double) * k * k), up(sizeof(double) * k * k),
                          up(tsz * (size_t)M->rblocks * k), up(tsz * k),
                          up(sizeof(unsigned) * 8), up(sizeof(int)), up(tsz * M->n_pad), up(tsz * M->n_pad),
                          up(tsz * k * k)};
  size_t total = 0;
  for (size_t b : sizes) total += b;
  char* base = nullptr;
  NLSP_CUDA(cudaMalloc(&base, total));
  M->storage = base;
  void** dst[] = {&M->P, (void**)&M->sigma, (void**)&M->Ac, (void**)&M->L, (void**)&M->Ainv, &M->cpart,
                  &M->ec, (void**)&M->counter, (void**)&M->status, &M->w0, &M->w1, &M->AinvT};
  size_t off = 0;
  for (int i = 0; i < 12; ++i) {
    *dst[i] = base + off;
    off += sizes[i];
  }
  NLSP_CUDA(cudaMemsetAsync(M->sigma, 0, sizes[1], M->ctx->stream));
  NLSP_CUDA(cudaMemsetAsync(M->counter, 0, sizes[7], M->ctx->stream));
  NLSP_CUDA(cudaMemsetAsync(M->status, 0, sizes[8], M->ctx->stream));
  return NLSP_OK;
}

// Launches the pivoted-Cholesky / one-sided Jacobi eigensolver (K <= 128).
nlsp_status chol_jacobi_eig(cudaStream_t s, const double* G, int K, int complete, double* evals, double* V) {
  const size_t sm = chol_eig_smem(K);
  const int nv = chol_eig_ldx(K) / 32;
  const void* fn = nv == 1   ? (const void*)k_chol_jacobi_eig<1>
                   : nv == 2 ? (const void*)k_chol_jacobi_eig<2>
                   : nv == 3 ? (const void*)k_chol_jacobi_eig<3>
                             : (const void*)k_chol_jacobi_eig<4>;
  NLSP_TRY(set_smem(fn, sm));
  const float tol = 4e-6f;
  void* args[] = {(void*)&G, (void*)&K, (void*)&tol, (void*)&complete, (void*)&evals, (void*)&V};
  NLSP_CUDA(cudaLaunchKernel(fn, dim3(1), dim3(CE_THREADS), args, sm, s));
  return NLSP_OK;
}

// Launches the two-CTA cluster eigensolver (128 < K <= 256).
nlsp_status cluster_jacobi_eig(cudaStream_t s, const double* G, int K, double* evals, double* V) {
  const size_t sm = cluster_eig_smem(K);
  const int nv = (K + 31) / 32;
  const void* fn = nv == 5   ? (const void*)k_cluster_jacobi_eig<5>
                   : nv == 6 ? (const void*)k_cluster_jacobi_eig<6>
                   : nv == 7 ? (const void*)k_cluster_jacobi_eig<7>
                             : (const void*)k_cluster_jacobi_eig<8>;
  NLSP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CJ_RANKS);
  cfg.blockDim = dim3(CJ_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CJ_RANKS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const float tol = 4e-6f;
  void* args[] = {(void*)&G, (void*)&K, (void*)&tol, (void*)&evals, (void*)&V};
  NLSP_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
  return NLSP_OK;
}

// Eigen-decomposition of the FP64 Gram matrix G (K x K): descending evals and
// eigenvectors V (column-major).  refine = number of FP64 refinement steps.
// work: 6 K^2 + K doubles.
nlsp_status gram_eigen(nlsp_ctx* ctx, const double* G, int K, int refine, double* evals, double* V, double* work) {
  cudaStream_t s = ctx->stream;
  if (K <= 128) {  // FP32 pivoted Cholesky + one-sided Jacobi (a complete basis when it is refined)
    NLSP_TRY(chol_jacobi_eig(s, G, K, refine > 0, evals, V));
  } else if (K <= 256) {  // FP32 one-sided Jacobi on G over a cluster of two CTAs
    NLSP_TRY(cluster_jacobi_eig(s, G, K, evals, V));
  } else {
    return NLSP_ERR_INVALID;
  }
  count_launches(ctx, 1);
  if (refine == 0) return NLSP_OK;
  if (refine > 0) {
    double* XtX = work;
    double* GX = XtX + K * K;
    double* S = GX + K * K;
    double* E = S + K * K;
    double* XE = E + K * K;
    double* vcopy = XE + K * K;
    double* lam = vcopy + K * K;
    // K x K products C = op(A) B
    const dim3 gg((unsigned)div_up(K, 16), (unsigned)div_up(K, 16));
    auto mm = [&](const double* A_, int ta, const double* B_, double* C_) {
      k_gemm_small<<<gg, 256, 0, s>>>(A_, K, ta, B_, K, 0, C_, K, K, K, K);
    };
    for (int it = 0; it < refine; ++it) {
      mm(V, 1, V, XtX);
      mm(G, 0, V, GX);
      mm(V, 1, GX, S);
      k_oa_step<<<K, 256, 0, s>>>(XtX, S, K, E, lam);
      mm(V, 0, E, XE);
      k_add<<<div_up((int64_t)K * K, 256), 256, 0, s>>>(V, XE, K * K);
      NLSP_LAUNCH_CHECK();
    }
    // eigenvalues of the refined basis (Rayleigh quotients), then sort
    mm(V, 1, V, XtX);
    mm(G, 0, V, GX);
    mm(V, 1, GX, S);
    k_oa_step<<<K, 256, 0, s>>>(XtX, S, K, E, lam);
    NLSP_CUDA(cudaMemcpyAsync(vcopy, V, sizeof(double) * K * K, cudaMemcpyDeviceToDevice, s));
    k_sort_eig<<<1, 1024, 0, s>>>(lam, vcopy, K, evals, V);
    NLSP_LAUNCH_CHECK();
    count_launches(ctx, 6 * refine + 5);
  }
  return NLSP_OK;
}

// P (tiled T, k columns) from the tiled smoothed samples S (K columns).
// With a_weighted, the Gram matrix is S^T A S (the eigen-decomposition of
// Z^T Z for Z = A^{1/2} S), so that P = S V_k Sigma_k^-1 is A-orthonormal and
// A^{1/2} P spans the top-k left singular subspace of A^{1/2} S (Appendix,
// Galerkin Convergence).
template <typename T>
nlsp_status basis_from_samples(nlsp_ctx* ctx, nlsp_prec* M, const T* S, bool a_weighted) {
  cudaStream_t s = ctx->stream;
  const int K = M->K, k = M->k;
  const size_t nsmall = (size_t)K * K * 2 + K + (6 * (size_t)K * K + K) + (size_t)K * k + 8;
  double* G = slot_as<double>(ctx, SLOT_SMALL, nsmall);
  if (!G) return NLSP_ERR_OOM;
  double* V = G + K * K;
  double* evals = V + K * K;
  double* work = evals + K;
  T* Mc = reinterpret_cast<T*>(work + 6 * K * K + K);
  if (a_weighted)
    NLSP_TRY((tsgemm<T, true>(ctx, M->A, S, K, K, M->n_pad, G, 1)));
  else
    NLSP_TRY((tsgemm<T, false>(ctx, M->A, S, K, K, M->n_pad, G, 0)));
  const int refine = M->precision == NLSP_FP64 ? 2 : 0;
  NLSP_TRY(gram_eigen(ctx, G, K, refine, evals, V, work));
  k_make_basis_coeffs<T><<<div_up((int64_t)K * k, 256), 256, 0, s>>>(evals, V, K, k, Mc, M->sigma, M->status);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 1);
  NLSP_TRY(tile_times_small<T>(ctx, S, K, Mc, k, M->n_pad, (T*)M->P));
  return NLSP_OK;
}

// C = op(A) op(B) (FP64, column-major, see k_gemm_small).
nlsp_status gemm64(nlsp_ctx* ctx, int ta, int tb, int m, int n, int kk, const double* A, int lda, const double* B,
                   int ldb, double* C, int ldc) {
  if (m <= 0 || n <= 0 || kk < 0) return NLSP_ERR_INVALID;
  k_gemm_small<<<dim3((unsigned)div_up(m, 16), (unsigned)div_up(n, 16)), 256, 0, ctx->stream>>>(A, lda, ta, B, ldb, tb,
                                                                                                 C, ldc, m, n, kk);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 1);
  return NLSP_OK;
}

// X (K x l) <- X L^-T where L L^T = X^T W X (W = G, or the identity when G is
// null): the columns of X become orthonormal in the metric W.  work: 5 l^2 +
// K l doubles.  A rank-deficient X gives NLSP_ERR_NOT_SPD in M->status.
nlsp_status orthonormalize_small(nlsp_ctx* ctx, nlsp_prec* M, const double* G, int K, int l, double* X,
                                 double* work) {
  cudaStream_t s = ctx->stream;
  double* WX = work;                 // K x l
  double* H = WX + (size_t)K * l;    // l x l
  double* Lf = H + (size_t)l * l;
  double* Hinv = Lf + (size_t)l * l;
  double* Lit = Hinv + (size_t)l * l;  // X L^-T goes to WX
  const double* WXp = X;
  if (G) {
    NLSP_TRY(gemm64(ctx, 0, 0, K, l, K, G, K, X, K, WX, K));
    WXp = WX;
  }
  NLSP_TRY(gemm64(ctx, 1, 0, l, l, K, X, K, WXp, K, H, l));
  k_symmetrize<<<div_up((int64_t)l * l, 256), 256, 0, s>>>(H, l);
  NLSP_TRY(set_smem((const void*)k_cholesky, sizeof(double) * l * l));
  k_cholesky<<<1, 256, sizeof(double) * l * l, s>>>(H, l, Lf, M->status);
  NLSP_TRY(set_smem((const void*)k_spd_inverse_cols, spd_inverse_smem(l)));
  k_spd_inverse_cols<<<l, 32, spd_inverse_smem(l), s>>>(Lf, l, Hinv);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 3);
  NLSP_TRY(gemm64(ctx, 0, 0, l, l, l, Hinv, l, Lf, l, Lit, l));  // (L L^T)^-1 L = L^-T
  NLSP_TRY(gemm64(ctx, 0, 0, K, l, l, X, K, Lit, l, WX, K));
  NLSP_CUDA(cudaMemcpyAsync(X, WX, sizeof(double) * K * l, cudaMemcpyDeviceToDevice, s));
  return NLSP_OK;
}

// Randomised-SVD basis (Halko, Martinsson, Tropp, "Finding structure with
// randomness", SIAM Review 2011: the randomised range finder with power
// iterations, their Algorithm 4.4, then the SVD of the small projected
// matrix, their Algorithm 5.1) of the tiled smoothed samples S (n x K), with
// l = k + oversample columns of the Gaussian sketch Omega (K x l, FP64
// column-major) and q power iterations.  Every n-sized iterate lies in the
// column space of S, Y = S X with X K x l, so the algorithm runs in the
// K-dimensional coefficient space through the Gram matrix G = S^T S (one
// tall-skinny product, the n-proportional cost):
//   Q = S X is orthonormal      <=>  X^T G X = I  (X <- X L^-T)
//   S^T Q = G X                       (power step; orthonormalised as W)
//   Q <- S W, re-orthonormalised      (X <- W, X^T G X = I)
//   B = Q^T S = X^T G, B B^T = (G X)^T (G X), eigenvectors U_B (l x l)
//   P = Q U_B[:, :k] = S (X U_B[:, :k])  (one tile product)
// The singular values reported are those of B (the first l).
template <typename T>
nlsp_status randomized_from_samples(nlsp_ctx* ctx, nlsp_prec* M, const T* S, int l, int power_iters,
                                    const double* sketch) {
  cudaStream_t s = ctx->stream;
  const int K = M->K, k = M->k;
  const size_t nsmall = (size_t)K * K + 2 * (size_t)K * l + (size_t)l * l * 2 + l + (6 * (size_t)l * l + l) +
                        (5 * (size_t)l * l + (size_t)K * l) + (size_t)K * k + 16;
  double* G = slot_as<double>(ctx, SLOT_SMALL, nsmall);
  if (!G) return NLSP_ERR_OOM;
  double* X = G + (size_t)K * K;                // K x l
  double* Z = X + (size_t)K * l;                // K x l
  double* BB = Z + (size_t)K * l;               // l x l
  double* V = BB + (size_t)l * l;               // l x l
  double* evals = V + (size_t)l * l;            // l
  double* ework = evals + l;                    // eigen refinement work
  double* owork = ework + 6 * (size_t)l * l + l;  // orthonormalisation work
  T* Mc = reinterpret_cast<T*>(owork + 5 * (size_t)l * l + (size_t)K * l);
  NLSP_TRY((tsgemm<T, false>(ctx, M->A, S, K, K, M->n_pad, G, 1)));
  NLSP_CUDA(cudaMemcpyAsync(X, sketch, sizeof(double) * K * l, cudaMemcpyDeviceToDevice, s));
  NLSP_TRY(orthonormalize_small(ctx, M, G, K, l, X, owork));  // Q = qr(S Omega)
  for (int it = 0; it < power_iters; ++it) {
    NLSP_TRY(gemm64(ctx, 0, 0, K, l, K, G, K, X, K, Z, K));    // S^T Q
    NLSP_TRY(orthonormalize_small(ctx, M, nullptr, K, l, Z, owork));  // W = qr(S^T Q)
    NLSP_CUDA(cudaMemcpyAsync(X, Z, sizeof(double) * K * l, cudaMemcpyDeviceToDevice, s));
    NLSP_TRY(orthonormalize_small(ctx, M, G, K, l, X, owork));  // Q = qr(S W)
  }
  NLSP_TRY(gemm64(ctx, 0, 0, K, l, K, G, K, X, K, Z, K));      // B^T = G X
  NLSP_TRY(gemm64(ctx, 1, 0, l, l, K, Z, K, Z, K, BB, l));      // B B^T
  k_symmetrize<<<div_up((int64_t)l * l, 256), 256, 0, s>>>(BB, l);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 1);
  const int refine = M->precision == NLSP_FP64 ? 2 : 0;
  NLSP_TRY(gram_eigen(ctx, BB, l, refine, evals, V, ework));
  k_randomized_coeffs<T><<<div_up((int64_t)K * k, 256), 256, 0, s>>>(X, V, evals, K, l, k, Mc, M->sigma, M->status);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 1);
  NLSP_TRY(tile_times_small<T>(ctx, S, K, Mc, k, M->n_pad, (T*)M->P));
  return NLSP_OK;
}

// Transposes the column-major k x k FP64 matrix W into row-major T.
template <typename T>
__global__ void k_transpose_to(const double* __restrict__ W, int k, T* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int c = e / k, j = e % k;  // out[c][j] = W(c, j)
    out[e] = (T)W[(int64_t)j * k + c];
  }
}

// CholeskyQR re-orthonormalisation P <- P L^-T with P^T P = L L^T (the thin-Q
// factor qf of Sec. 3, up to column signs).
template <typename T>
nlsp_status cholesky_qr(nlsp_ctx* ctx, nlsp_prec* M) {
  cudaStream_t s = ctx->stream;
  const int k = M->k;
  double* Gp = slot_as<double>(ctx, SLOT_SMALL, (size_t)k * k * 5 + 8);
  if (!Gp) return NLSP_ERR_OOM;
  double* Lp = Gp + k * k;
  double* Linv = Lp + k * k;
  double* W = Linv + k * k;
  T* Mt = reinterpret_cast<T*>(W + k * k);
  T* Pnew = slot_as<T>(ctx, SLOT_PNEW, (size_t)M->n_pad * k);
  if (!Pnew) return NLSP_ERR_OOM;
  NLSP_TRY((tsgemm<T, false>(ctx, M->A, (const T*)M->P, k, k, M->n_pad, Gp, 1)));
  NLSP_TRY(set_smem((const void*)k_cholesky, sizeof(double) * k * k));
  k_cholesky<<<1, 256, sizeof(double) * k * k, s>>>(Gp, k, Lp, M->status);
  // With P^T P = L L^T:  (L L^T)^-1 L = L^-T, so P L^-T needs only the SPD
  // inverse kernel and one small product.
  NLSP_TRY(set_smem((const void*)k_spd_inverse_cols, spd_inverse_smem(k)));
  k_spd_inverse_cols<<<k, 32, spd_inverse_smem(k), s>>>(Lp, k, Linv);  // (L L^T)^-1
  k_gemm_small<<<dim3((unsigned)div_up(k, 16), (unsigned)div_up(k, 16)), 256, 0, s>>>(Linv, k, 0, Lp, k, 0, W, k, k,
                                                                                     k, k);  // L^-T
  k_transpose_to<T><<<div_up((int64_t)k * k, 256), 256, 0, s>>>(W, k, Mt);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 4);
  NLSP_TRY(tile_times_small<T>(ctx, (const T*)M->P, k, Mt, k, M->n_pad, Pnew));
  NLSP_CUDA(cudaMemcpyAsync(M->P, Pnew, sizeof(T) * M->n_pad * k, cudaMemcpyDeviceToDevice, s));
  return NLSP_OK;
}

// How the basis is taken from the smoothed samples: the exact thin SVD, the
// A-weighted spectral basis, or the randomised SVD (sketch columns l = k +
// oversample, q power iterations, the sketch Omega on the device or drawn).
struct BasisChoice {
  int mode;  // 0 exact, 1 A-weighted, 2 randomised
  int oversample, power_iters;
  const double* sketch;
  unsigned long long seed;
};

template <typename T>
nlsp_status build_impl(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* p, const double* S0,
                       nlsp_prec** out, BasisChoice bc) {
  const bool a_weighted = bc.mode == 1;
  nlsp_prec* M = new_prec(ctx, A, p, p->k, p->K);
  nlsp_status st = alloc_prec_storage(M);
  auto fail = [&](nlsp_status e) {
    nlsp_free_prec(M);
    return e;
  };
  if (st != NLSP_OK) return fail(st);
  cudaStream_t s = ctx->stream;
  const int K = p->K;
  T* sa = slot_as<T>(ctx, SLOT_SA, (size_t)M->n_pad * K);
  T* sb = slot_as<T>(ctx, SLOT_SB, (size_t)M->n_pad * K);
  if (!sa || !sb) return fail(NLSP_ERR_OOM);
  if (S0)
    k_colmajor_to_tiled<T><<<grid_for(ctx, M->n_pad * K, 256, 8), 256, 0, s>>>(S0, A->n, A->n, K, M->n_pad, sa);
  else
    k_random_samples_tiled<T><<<grid_for(ctx, M->n_pad * K, 256, 8), 256, 0, s>>>(
        splitmix_stream_base(p->seed, NLSP_STREAM_S0), A->n, K, M->n_pad, sa);
  if (cudaGetLastError() != cudaSuccess) return fail(NLSP_ERR_CUDA);
  count_launches(ctx, 1);
  T* S = nullptr;
  if ((st = smooth_tiled<T>(ctx, A, K, p->s1, p->omega, M->n_pad, sa, sb, &S)) != NLSP_OK) return fail(st);
  if (bc.mode == 2) {
    const int l = p->k + bc.oversample;
    const double* sketch = bc.sketch;
    if (!sketch) {  // Omega (K x l) from the counter-based generator: element (c, j) is normal j K + c
      double* d = slot_as<double>(ctx, SLOT_PNEW, (size_t)K * l);
      if (!d) return fail(NLSP_ERR_OOM);
      k_random_normal<<<grid_for(ctx, (int64_t)K * l, 256, 8), 256, 0, s>>>(
          splitmix_stream_base(bc.seed, NLSP_STREAM_SKETCH), 0, (int64_t)K * l, d);
      if (cudaGetLastError() != cudaSuccess) return fail(NLSP_ERR_CUDA);
      count_launches(ctx, 1);
      sketch = d;
    }
    if ((st = randomized_from_samples<T>(ctx, M, S, l, bc.power_iters, sketch)) != NLSP_OK) return fail(st);
  } else if ((st = basis_from_samples<T>(ctx, M, S, a_weighted)) != NLSP_OK) {
    return fail(st);
  }
  if (p->precision == NLSP_FP64 && !a_weighted)  // the A-weighted basis is A-orthonormal already
    if ((st = cholesky_qr<T>(ctx, M)) != NLSP_OK) return fail(st);
  if ((st = nlsp_internal_factor(ctx, M, M->k)) != NLSP_OK) return fail(st);
  *out = M;
  return NLSP_OK;
}

template <typename T>
nlsp_status from_basis_impl(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* p, const double* P, int k,
                            nlsp_prec** out) {
  nlsp_prec* M = new_prec(ctx, A, p, k, 0);
  nlsp_status st = alloc_prec_storage(M);
  if (st != NLSP_OK) {
    nlsp_free_prec(M);
    return st;
  }
  k_colmajor_to_tiled<T><<<grid_for(ctx, M->n_pad * k, 256, 8), 256, 0, ctx->stream>>>(P, A->n, A->n, k, M->n_pad,
                                                                                         (T*)M->P);
  if (cudaGetLastError() != cudaSuccess) {
    nlsp_free_prec(M);
    return NLSP_ERR_CUDA;
  }
  count_launches(ctx, 1);
  if ((st = nlsp_internal_factor(ctx, M, k)) != NLSP_OK) {
    nlsp_free_prec(M);
    return st;
  }
  *out = M;
  return NLSP_OK;
}

}  // namespace

// A_c = P_r^T A P_r (FP64 result), Cholesky and explicit inverse.  Reads the
// status word (synchronises).
nlsp_status nlsp_internal_factor(nlsp_ctx* ctx, nlsp_prec* M, int r) {
  cudaStream_t s = ctx->stream;
  if (M->precision == NLSP_FP64)
    NLSP_TRY((tsgemm<double, true>(ctx, M->A, (const double*)M->P, M->k, r, M->n_pad, M->Ac, 1)));
  else
    NLSP_TRY((tsgemm<float, true>(ctx, M->A, (const float*)M->P, M->k, r, M->n_pad, M->Ac, 1)));
  NLSP_TRY(set_smem((const void*)k_cholesky, sizeof(double) * r * r));
  k_cholesky<<<1, 256, sizeof(double) * r * r, s>>>(M->Ac, r, M->L, M->status);
  NLSP_LAUNCH_CHECK();
  NLSP_TRY(set_smem((const void*)k_spd_inverse_cols, spd_inverse_smem(r)));
  k_spd_inverse_cols<<<r, 32, spd_inverse_smem(r), s>>>(M->L, r, M->Ainv);
  k_symmetrize<<<div_up((int64_t)r * r, 256), 256, 0, s>>>(M->Ainv, r);
  if (M->precision == NLSP_FP64)
    NLSP_CUDA(cudaMemcpyAsync(M->AinvT, M->Ainv, sizeof(double) * r * r, cudaMemcpyDeviceToDevice, s));
  else
    k_transpose_to<float><<<div_up((int64_t)r * r, 256), 256, 0, s>>>(M->Ainv, r, (float*)M->AinvT);  // symmetric
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, M->precision == NLSP_FP64 ? 3 : 4);
  int hstat = 0;
  NLSP_CUDA(cudaMemcpyAsync(&hstat, M->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  NLSP_CUDA(cudaStreamSynchronize(s));
  if (hstat != 0) return (nlsp_status)hstat;
  M->r = r;
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_smooth_samples(nlsp_ctx* ctx, const nlsp_op* A, int K, int s1, double omega,
                                           int precision, const double* dev_S0, double* dev_S) {
  if (!ctx || !A || !dev_S0 || !dev_S || K < 1 || s1 < 0 || !(omega > 0.0) || !(omega < 2.0)) return NLSP_ERR_INVALID;
  if (precision != NLSP_FP64 && precision != NLSP_MIXED_FP32) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  const int64_t n_pad = pad_tile(A->n);
  cudaStream_t s = ctx->stream;
  const int g = grid_for(ctx, n_pad * K, 256, 8);
  auto run = [&](auto tag) -> nlsp_status {
    using T = decltype(tag);
    T* a = slot_as<T>(ctx, SLOT_SA, (size_t)n_pad * K);
    T* b = slot_as<T>(ctx, SLOT_SB, (size_t)n_pad * K);
    if (!a || !b) return NLSP_ERR_OOM;
    k_colmajor_to_tiled<T><<<g, 256, 0, s>>>(dev_S0, A->n, A->n, K, n_pad, a);
    T* r = nullptr;
    NLSP_TRY(smooth_tiled<T>(ctx, A, K, s1, omega, n_pad, a, b, &r));
    k_tiled_to_colmajor<T><<<g, 256, 0, s>>>(r, A->n, K, K, dev_S, A->n);
    NLSP_LAUNCH_CHECK();
    count_launches(ctx, 2);
    return NLSP_OK;
  };
  NLSP_TRY(precision == NLSP_FP64 ? run(double()) : run(float()));
  NLSP_CUDA(cudaStreamSynchronize(s));
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_random_normal(nlsp_ctx* ctx, unsigned long long seed, unsigned long long stream,
                                          unsigned long long offset, int64_t count, double* dev_out) {
  if (!ctx || count < 0 || (count > 0 && !dev_out)) return NLSP_ERR_INVALID;
  if (count == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  k_random_normal<<<grid_for(ctx, count, 256, 8), 256, 0, ctx->stream>>>(splitmix_stream_base(seed, stream), offset,
                                                                          count, dev_out);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 1);
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_build_prolongation(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* params,
                                               const double* dev_S0, nlsp_prec** M_out) {
  if (!ctx || !M_out) return NLSP_ERR_INVALID;
  *M_out = nullptr;
  NLSP_TRY(check_setup_params(A, params, true));
  NLSP_CUDA(cudaSetDevice(ctx->device));
  const BasisChoice bc{0, 0, 0, nullptr, 0};
  if (params->precision == NLSP_FP64) return build_impl<double>(ctx, A, params, dev_S0, M_out, bc);
  return build_impl<float>(ctx, A, params, dev_S0, M_out, bc);
}

extern "C" nlsp_status nlsp_build_prolongation_a_weighted(nlsp_ctx* ctx, const nlsp_op* A,
                                                          const nlsp_setup_params* params, const double* dev_S0,
                                                          nlsp_prec** M_out) {
  if (!ctx || !M_out) return NLSP_ERR_INVALID;
  *M_out = nullptr;
  NLSP_TRY(check_setup_params(A, params, true));
  if (params->K > 128) {  // the wider (K <= 256) eigensolver path serves the exact-SVD basis only
    nlsp_record_message("nlsp_build_prolongation_a_weighted: K <= 128");
    return NLSP_ERR_INVALID;
  }
  NLSP_CUDA(cudaSetDevice(ctx->device));
  const BasisChoice bc{1, 0, 0, nullptr, 0};
  if (params->precision == NLSP_FP64) return build_impl<double>(ctx, A, params, dev_S0, M_out, bc);
  return build_impl<float>(ctx, A, params, dev_S0, M_out, bc);
}

extern "C" nlsp_status nlsp_build_prolongation_randomized(nlsp_ctx* ctx, const nlsp_op* A,
                                                          const nlsp_setup_params* params, const double* dev_S0,
                                                          int oversample, int power_iters, const double* dev_sketch,
                                                          nlsp_prec** M_out) {
  if (!ctx || !M_out) return NLSP_ERR_INVALID;
  *M_out = nullptr;
  NLSP_TRY(check_setup_params(A, params, true));
  if (params->K > 128) {  // the wider (K <= 256) eigensolver path serves the exact-SVD basis only
    nlsp_record_message("nlsp_build_prolongation_randomized: K <= 128");
    return NLSP_ERR_INVALID;
  }
  if (oversample < 0 || params->k + oversample > params->K || power_iters < 0 || power_iters > 16) {
    nlsp_record_message("nlsp_build_prolongation_randomized: need 0 <= oversample, k + oversample <= K, "
                        "0 <= power_iters <= 16");
    return NLSP_ERR_INVALID;
  }
  NLSP_CUDA(cudaSetDevice(ctx->device));
  const BasisChoice bc{2, oversample, power_iters, dev_sketch, params->seed};
  if (params->precision == NLSP_FP64) return build_impl<double>(ctx, A, params, dev_S0, M_out, bc);
  return build_impl<float>(ctx, A, params, dev_S0, M_out, bc);
}

extern "C" nlsp_status nlsp_prec_from_basis(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* params,
                                            const double* dev_P, int k, nlsp_prec** M_out) {
  if (!ctx || !M_out || !dev_P || !params) return NLSP_ERR_INVALID;
  *M_out = nullptr;
  nlsp_setup_params p = *params;
  p.k = k;
  NLSP_TRY(check_setup_params(A, &p, false));
  NLSP_CUDA(cudaSetDevice(ctx->device));
  if (p.precision == NLSP_FP64) return from_basis_impl<double>(ctx, A, &p, dev_P, k, M_out);
  return from_basis_impl<float>(ctx, A, &p, dev_P, k, M_out);
}

extern "C" nlsp_status nlsp_factor_coarse(nlsp_ctx* ctx, const nlsp_op* A, nlsp_prec* M, int r) {
  if (!ctx || !M || A != M->A || r < 1 || r > M->k) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  return nlsp_internal_factor(ctx, M, r);
}

extern "C" nlsp_status nlsp_prec_dims(const nlsp_prec* M, int64_t* n, int* k, int* r, int* K, int* precision) {
  if (!M) return NLSP_ERR_INVALID;
  if (n) *n = M->n;
  if (k) *k = M->k;
  if (r) *r = M->r;
  if (K) *K = M->K;
  if (precision) *precision = M->precision;
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_prec_copy_basis(nlsp_ctx* ctx, const nlsp_prec* M, double* dev_P) {
  if (!ctx || !M || !dev_P) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  const int g = grid_for(ctx, M->n * M->k, 256, 8);
  if (M->precision == NLSP_FP64)
    k_tiled_to_colmajor<double><<<g, 256, 0, ctx->stream>>>((const double*)M->P, M->n, M->k, M->k, dev_P, M->n);
  else
    k_tiled_to_colmajor<float><<<g, 256, 0, ctx->stream>>>((const float*)M->P, M->n, M->k, M->k, dev_P, M->n);
  NLSP_LAUNCH_CHECK();
  count_launches(ctx, 1);
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_prec_copy_sigma(nlsp_ctx* ctx, const nlsp_prec* M, double* dev_sigma) {
  if (!ctx || !M || !dev_sigma) return NLSP_ERR_INVALID;
  if (M->K > 0)
    NLSP_CUDA(cudaMemcpyAsync(dev_sigma, M->sigma, sizeof(double) * M->K, cudaMemcpyDeviceToDevice, ctx->stream));
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_prec_copy_coarse(nlsp_ctx* ctx, const nlsp_prec* M, double* dev_Ac, double* dev_L) {
  if (!ctx || !M) return NLSP_ERR_INVALID;
  const size_t b = sizeof(double) * M->r * M->r;
  if (dev_Ac) NLSP_CUDA(cudaMemcpyAsync(dev_Ac, M->Ac, b, cudaMemcpyDeviceToDevice, ctx->stream));
  if (dev_L) NLSP_CUDA(cudaMemcpyAsync(dev_L, M->L, b, cudaMemcpyDeviceToDevice, ctx->stream));
  return NLSP_OK;
}
