// Breakdown-free block conjugate gradient (Ji & Li, "A breakdown-free block
// conjugate gradient method", BIT Numerical Mathematics 57, 2017; the block
// CG of O'Leary, "The block conjugate gradient algorithm and related
// methods", Linear Algebra Appl. 29, 1980, with the search block
// re-orthonormalised and rank-deflated every iteration), preconditioned by
// the two-level preconditioner of Algorithm 1.  Unlike nlsp_solve_block's
// independent recurrences, the m <= 32 columns share one search space:
//
//   R = B, Z = M R, P = orth(Z)                      (s <= m columns)
//   loop:  Q = A P,  D = P^T Q,  alpha = D^-1 P^T R
//          X += P alpha,  R -= Q alpha               (stop when every column
//                                                     has ||r_c|| <= tol ||b_c||)
//          Z = M R,  beta = -D^-1 Q^T Z
//          P = orth(Z + P beta)
//
// orth is a pivoted Cholesky QR: the Gram matrix W^T W is factored with
// diagonal pivoting until the largest remaining pivot falls below 1e-14 of
// the largest diagonal; the dropped directions are (numerically) in the span
// of the kept ones -- converged or dependent columns -- which is what keeps
// D = P^T A P positive definite.  All block quantities are FP64 (node-major
// rows of 32 columns); the preconditioner runs in its own precision through
// the block solver's kernels.  This header is included by block.cu after its
// kernels.
#pragma once

// (included inside block.cu's anonymous namespace)
constexpr double BCG_DROP = 1e-14;  // relative pivot below which orth drops a direction

struct BcgState {
  int s;              // columns of the current search block P
  int m;              // right-hand sides
  int t;              // iterations taken
  int maxit;
  int all_done;
  int bad;            // a factorisation failed (breakdown)
  double bb[MB], rr[MB], tol2bn[MB];
  int iter[MB], done[MB], status[MB];
};

// Gram partials of two node-major blocks: part[w][a][b] = sum over the nodes
// of warp w of X[i][a] Y[i][b] (lane b; X's row is broadcast by shuffles).
__global__ void __launch_bounds__(BT) k_bcg_gram(const double* __restrict__ X, const double* __restrict__ Y,
                                                 int64_t n, double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5), ws = (int64_t)gridDim.x * BW;
  double acc[MB];
#pragma unroll
  for (int a = 0; a < MB; ++a) acc[a] = 0.0;
  for (int64_t i = w; i < n; i += ws) {
    const double xa = X[i * MB + lane];
    const double yb = Y[i * MB + lane];
#pragma unroll
    for (int a = 0; a < MB; ++a) acc[a] = fma(__shfl_sync(0xffffffffu, xa, a), yb, acc[a]);
  }
  double* out = part + w * (MB * MB);
#pragma unroll
  for (int a = 0; a < MB; ++a) out[a * MB + lane] = acc[a];
}

// out[e] (e < 1024) = sum over the nw warp partials, in a fixed order: block
// of 256 threads per 32 entries, warp g adding partials g, g + 8, ... in four
// running sums, then the eight warp sums in warp order.
__global__ void __launch_bounds__(256) k_bcg_sum(const double* __restrict__ part, int nw, double* __restrict__ out) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int b = g;
  for (; b + 24 < nw; b += 32) {
    s0 += part[(int64_t)b * (MB * MB) + e];
    s1 += part[(int64_t)(b + 8) * (MB * MB) + e];
    s2 += part[(int64_t)(b + 16) * (MB * MB) + e];
    s3 += part[(int64_t)(b + 24) * (MB * MB) + e];
  }
  for (; b < nw; b += 8) s0 += part[(int64_t)b * (MB * MB) + e];
  red[g][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (g == 0) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    out[e] = t;
  }
}

// Out[i][c] = (Base ? Base[i][c] : keep ? Out[i][c] : 0) + sign * sum_a In[i][a] M[a][c]
// (M 32 x 32 row-major, FP64).  One warp per node row.
__global__ void __launch_bounds__(BT) k_bcg_mm(double* __restrict__ Out, const double* __restrict__ Base,
                                               const double* __restrict__ In, const double* __restrict__ Mg,
                                               int64_t n, double sign, int keep) {
  __shared__ double Ms[MB * MB];
  for (int e = threadIdx.x; e < MB * MB; e += BT) Ms[e] = Mg[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * BW) {
    const double xa = In[i * MB + lane];
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < MB; ++a) acc = fma(__shfl_sync(0xffffffffu, xa, a), Ms[a * MB + lane], acc);
    const double base = Base ? Base[i * MB + lane] : (keep ? Out[i * MB + lane] : 0.0);
    Out[i * MB + lane] = base + sign * acc;
  }
}

// rT = R in the preconditioner precision, za = omega D^-1 rT (the first
// pre-sweep from z = 0).
template <int KIND, typename T>
__global__ void __launch_bounds__(BT) k_bcg_prep(StencilView<T> A, T omega, const double* __restrict__ R,
                                                 T* __restrict__ rT, T* __restrict__ za, int64_t n) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * BW) {
    const T rt = (T)R[i * MB + lane];
    rT[i * MB + lane] = rt;
    za[i * MB + lane] = omega * stencil_dinv<KIND>(A, i) * rt;
  }
}

// ---- the small dense algebra, one CTA of 1024 threads ---------------------
// Cholesky of the leading s x s block of G (row-major, ld 32) in shared
// memory, right-looking; false on a non-positive or non-finite pivot.
__device__ bool bcg_cholesky(double (*L)[MB + 1], int s) {
  const int tid = threadIdx.x, r = tid >> 5, c = tid & 31;
  __shared__ int ok;
  if (tid == 0) ok = 1;
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (tid == 0) {
      const double d = L[j][j];
      if (!(d > 0.0) || !isfinite(d)) ok = 0;
      L[j][j] = ok ? sqrt(d) : 1.0;
    }
    __syncthreads();
    if (tid > j && tid < s) L[tid][j] /= L[j][j];
    __syncthreads();
    if (r > j && r < s && c > j && c <= r) L[r][c] -= L[r][j] * L[c][j];
    __syncthreads();
  }
  return ok != 0;
}

// Y (s x m, row-major in shared memory) <- L^-T L^-1 Y for the lower factor L.
__device__ void bcg_solve(double (*L)[MB + 1], double (*Y)[MB + 1], int s, int m) {
  const int tid = threadIdx.x, r = tid >> 5, c = tid & 31;
  for (int i = 0; i < s; ++i) {  // forward: L y = e
    if (tid < m) Y[i][tid] /= L[i][i];
    __syncthreads();
    if (r > i && r < s && c < m) Y[r][c] -= L[r][i] * Y[i][c];
    __syncthreads();
  }
  for (int i = s - 1; i >= 0; --i) {  // backward: L^T x = y
    if (tid < m) Y[i][tid] /= L[i][i];
    __syncthreads();
    if (r < i && c < m) Y[r][c] -= L[i][r] * Y[i][c];
    __syncthreads();
  }
}

enum { BCG_ALPHA = 0, BCG_BETA = 1, BCG_ORTH = 2 };

// ALPHA: D = G1 (P^T Q), coef = D^-1 G2 (P^T R), also keeps D's factor.
// BETA:  coef = -D^-1 G1 (Q^T Z) with the kept factor.
// ORTH:  pivoted Cholesky of G1 (W^T W, m x m); coef (32 x 32) maps W to the
//        orthonormal block P = W coef, whose first s' columns are kept.
// coef is written row-major 32 x 32 with zeros outside the used block.
__global__ void __launch_bounds__(1024) k_bcg_small(int mode, const double* __restrict__ G1,
                                                    const double* __restrict__ G2, double* __restrict__ Dfac,
                                                    double* __restrict__ coef, BcgState* st) {
  __shared__ double L[MB][MB + 1];
  __shared__ double Y[MB][MB + 1];
  __shared__ int perm[MB];
  __shared__ int sp;
  const int tid = threadIdx.x, r = tid >> 5, c = tid & 31;
  const int s = st->s, m = st->m;
  if (mode == BCG_ALPHA) {
    L[r][c] = (r < s && c < s) ? G1[r * MB + c] : 0.0;
    Y[r][c] = (r < s && c < m) ? G2[r * MB + c] : 0.0;
    __syncthreads();
    const bool ok = bcg_cholesky(L, s);
    Dfac[r * MB + c] = L[r][c];
    if (!ok) {
      coef[r * MB + c] = 0.0;
      if (tid == 0) st->bad = 1;
      return;
    }
    bcg_solve(L, Y, s, m);
    coef[r * MB + c] = (r < s && c < m) ? Y[r][c] : 0.0;
  } else if (mode == BCG_BETA) {
    L[r][c] = Dfac[r * MB + c];
    Y[r][c] = (r < s && c < m) ? G1[r * MB + c] : 0.0;
    __syncthreads();
    if (st->bad) {
      coef[r * MB + c] = 0.0;
      return;
    }
    bcg_solve(L, Y, s, m);
    coef[r * MB + c] = (r < s && c < m) ? -Y[r][c] : 0.0;
  } else {
    // pivoted Cholesky of the m x m Gram matrix, in place on a permuted copy
    L[r][c] = (r < m && c < m) ? G1[r * MB + c] : 0.0;
    if (tid < MB) perm[tid] = tid;
    __syncthreads();
    __shared__ double dmax0;
    if (tid == 0) {
      double d = 0.0;
      for (int q = 0; q < m; ++q) d = fmax(d, L[q][q]);
      dmax0 = d;
      sp = 0;
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      if (tid == 0) {  // pivot: the largest remaining diagonal, swapped into place j
        int q = j;
        for (int t = j + 1; t < m; ++t)
          if (L[t][t] > L[q][q]) q = t;
        const double d = L[q][q];
        sp = (d > BCG_DROP * dmax0 && isfinite(d)) ? j + 1 : -(j + 1);
        if (sp > 0 && q != j) {
          const int tp = perm[j]; perm[j] = perm[q]; perm[q] = tp;
          for (int t = 0; t < m; ++t) { const double v = L[j][t]; L[j][t] = L[q][t]; L[q][t] = v; }
          for (int t = 0; t < m; ++t) { const double v = L[t][j]; L[t][j] = L[t][q]; L[t][q] = v; }
        }
        if (sp > 0) L[j][j] = sqrt(L[j][j]);
      }
      __syncthreads();
      if (sp < 0) break;
      if (tid > j && tid < m) L[tid][j] /= L[j][j];
      __syncthreads();
      // the whole trailing block stays symmetric (a later pivot swap moves
      // entries across its diagonal)
      if (r > j && r < m && c > j && c < m) L[r][c] -= L[r][j] * L[c][j];
      __syncthreads();
    }
    const int sn = sp > 0 ? m : -sp - 1;  // columns kept
    // T = L^-T (upper, sn x sn) column by column: solve L^T t_j = e_j
    Y[r][c] = (r == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int i = sn - 1; i >= 0; --i) {  // back substitution, all columns at once
      if (tid < sn) Y[i][tid] /= L[i][i];
      __syncthreads();
      if (r < i && c < sn) Y[r][c] -= L[i][r] * Y[i][c];
      __syncthreads();
    }
    // coef[perm[a]][j] = T[a][j] for a, j < sn
    coef[r * MB + c] = 0.0;
    __syncthreads();
    if (r < sn && c < sn) coef[perm[r] * MB + c] = Y[r][c];
    if (tid == 0) st->s = sn;
  }
}

// Per-column convergence from the diagonal of R^T R (G, row-major 32 x 32);
// stage 0 records ||b_c||^2.  Sets all_done when every column is done (or a
// factorisation failed).
__global__ void k_bcg_state(const double* __restrict__ G, BcgState* st, int stage, double tol) {
  const int c = threadIdx.x;
  const double rr = G[c * MB + c];
  const int m = st->m;
  if (stage == 0) {
    st->bb[c] = rr;
    st->tol2bn[c] = tol * tol * rr;
    st->rr[c] = rr;
    st->iter[c] = 0;
    st->status[c] = (int)NLSP_OK;
    st->done[c] = c >= m || rr == 0.0;
    if (c < m && !isfinite(rr)) {
      st->status[c] = (int)NLSP_ERR_BREAKDOWN;
      st->done[c] = 1;
    }
  } else {
    const int t = st->t;
    if (c < m) {
      st->rr[c] = rr;
      if (!st->done[c]) {
        st->iter[c] = t;
        if (!isfinite(rr)) {
          st->status[c] = (int)NLSP_ERR_BREAKDOWN;
          st->done[c] = 1;
        } else if (rr <= st->tol2bn[c]) {
          st->done[c] = 1;
        } else if (t >= st->maxit) {
          st->status[c] = (int)NLSP_NOT_CONVERGED;
          st->done[c] = 1;
        }
      }
    }
  }
  __syncwarp();
  const unsigned pend = __ballot_sync(0xffffffffu, c < m && !st->done[c]);
  if (c == 0) st->all_done = (pend == 0u || st->bad || (stage != 0 && st->s == 0)) ? 1 : 0;
}

__global__ void k_bcg_tick(BcgState* st) {
  if (threadIdx.x == 0) st->t += 1;
}
