// Evaluation of A (Sec. 3, Eq. discretized_pde): matrix-free stencils on the
// structured grids (2D 5-point and 9-point, 3D 7-point, Dirichlet nodes
// eliminated) and the general sparse operator in row slices.  Every function evaluates in precision T and reads the vector in
// its own storage type X (so an FP32 preconditioner can read FP64 residuals).
#pragma once

#include "common.cuh"

struct NodeCoord {
  int i, j, l;
};

// Grid coordinates of node idx (n < 2^31: 32-bit unsigned division only).
template <int KIND>
__device__ __forceinline__ NodeCoord node_coord(int64_t idx, int N) {
  NodeCoord c;
  if (KIND == ST_CSR) {  // no grid: neighbours come from the row's entries
    c.i = c.j = c.l = 0;
    return c;
  }
  const unsigned u = (unsigned)idx, un = (unsigned)N;
  if (KIND == ST_7PT) {
    const unsigned nn = un * un;
    c.l = (int)(u / nn);
    const unsigned rem = u - (unsigned)c.l * nn;
    c.j = (int)(rem / un);
    c.i = (int)(rem - (unsigned)c.j * un);
  } else {
    c.j = (int)(u / un);
    c.i = (int)(u - (unsigned)c.j * un);
    c.l = 0;
  }
  return c;
}

// Entries of row idx of the general sparse operator: first entry at *base,
// the following ones 32 apart, *w of them (the row's slice width).
template <typename T>
__device__ __forceinline__ void csr_row(const StencilView<T>& A, int64_t idx, int64_t* base, int* w) {
  const int p = A.ppos[idx];
  const int sl = p >> 5;
  const int64_t s0 = A.soff[sl];
  *base = s0 + (p & 31);
  *w = (int)((A.soff[sl + 1] - s0) >> 5);
}

template <int KIND, typename T>
__device__ __forceinline__ T stencil_diag(const StencilView<T>& A, int64_t idx) {
  return KIND == ST_9PT ? A.c[0] : A.diag[idx];
}

template <int KIND, typename T>
__device__ __forceinline__ T stencil_dinv(const StencilView<T>& A, int64_t idx) {
  return KIND == ST_9PT ? A.cdinv : A.dinv[idx];
}

// (A x)_idx.  `get(m)` returns x at node m converted to T; it is only called
// for nodes inside the grid.
template <int KIND, typename T, typename Get>
__device__ __forceinline__ T stencil_apply(const StencilView<T>& A, int64_t idx, NodeCoord c, Get get) {
  const int N = A.N;
  if (KIND == ST_CSR) {
    T s = A.diag[idx] * get(idx);
    int64_t base;
    int w;
    csr_row(A, idx, &base, &w);
    for (int j = 0; j < w; ++j) {
      const int64_t e = base + 32 * (int64_t)j;
      s += A.sval[e] * get((int64_t)A.scol[e]);  // padding: (own row, 0)
    }
    return s;
  }
  if (KIND == ST_9PT) {
    T s = A.c[0] * get(idx);
    const bool w = c.i > 0, e = c.i < N - 1, so = c.j > 0, no = c.j < N - 1;
    T ew = T(0), ns = T(0), d1 = T(0), d2 = T(0);
    if (w) ew += get(idx - 1);
    if (e) ew += get(idx + 1);
    if (so) ns += get(idx - N);
    if (no) ns += get(idx + N);
    if (e && no) d1 += get(idx + N + 1);
    if (w && so) d1 += get(idx - N - 1);
    if (w && no) d2 += get(idx + N - 1);
    if (e && so) d2 += get(idx - N + 1);
    s += A.c[1] * ew + A.c[2] * ns + A.c[3] * d1 + A.c[4] * d2;
    return s;
  } else {
    T s = A.diag[idx] * get(idx);
    if (c.i > 0) s -= A.cx[idx - 1] * get(idx - 1);
    if (c.i < N - 1) s -= A.cx[idx] * get(idx + 1);
    if (c.j > 0) s -= A.cy[idx - N] * get(idx - N);
    if (c.j < N - 1) s -= A.cy[idx] * get(idx + N);
    if (KIND == ST_7PT) {
      const int64_t nn = (int64_t)N * N;
      if (c.l > 0) s -= A.cz[idx - nn] * get(idx - nn);
      if (c.l < N - 1) s -= A.cz[idx] * get(idx + nn);
    }
    return s;
  }
}

// Visits the off-diagonal neighbours m of node idx: f(m, coord_m, a_idx_m)
// with a_idx_m the (signed) matrix entry.
template <int KIND, typename T, typename F>
__device__ __forceinline__ void for_each_neighbour(const StencilView<T>& A, int64_t idx, NodeCoord c, F f) {
  const int N = A.N;
  if (KIND == ST_CSR) {
    int64_t base;
    int wd;
    csr_row(A, idx, &base, &wd);
    for (int j = 0; j < wd; ++j) {
      const int64_t e = base + 32 * (int64_t)j;
      const int64_t m = A.scol[e];
      if (m != idx) f(m, NodeCoord{0, 0, 0}, A.sval[e]);  // padding entries point at the own row
    }
    return;
  }
  const bool w = c.i > 0, e = c.i < N - 1, so = c.j > 0, no = c.j < N - 1;
  if (KIND == ST_9PT) {
    if (w) f(idx - 1, NodeCoord{c.i - 1, c.j, c.l}, A.c[1]);
    if (e) f(idx + 1, NodeCoord{c.i + 1, c.j, c.l}, A.c[1]);
    if (so) f(idx - N, NodeCoord{c.i, c.j - 1, c.l}, A.c[2]);
    if (no) f(idx + N, NodeCoord{c.i, c.j + 1, c.l}, A.c[2]);
    if (e && no) f(idx + N + 1, NodeCoord{c.i + 1, c.j + 1, c.l}, A.c[3]);
    if (w && so) f(idx - N - 1, NodeCoord{c.i - 1, c.j - 1, c.l}, A.c[3]);
    if (w && no) f(idx + N - 1, NodeCoord{c.i - 1, c.j + 1, c.l}, A.c[4]);
    if (e && so) f(idx - N + 1, NodeCoord{c.i + 1, c.j - 1, c.l}, A.c[4]);
  } else {
    if (w) f(idx - 1, NodeCoord{c.i - 1, c.j, c.l}, -A.cx[idx - 1]);
    if (e) f(idx + 1, NodeCoord{c.i + 1, c.j, c.l}, -A.cx[idx]);
    if (so) f(idx - N, NodeCoord{c.i, c.j - 1, c.l}, -A.cy[idx - N]);
    if (no) f(idx + N, NodeCoord{c.i, c.j + 1, c.l}, -A.cy[idx]);
    if (KIND == ST_7PT) {
      const int64_t nn = (int64_t)N * N;
      if (c.l > 0) f(idx - nn, NodeCoord{c.i, c.j, c.l - 1}, -A.cz[idx - nn]);
      if (c.l < N - 1) f(idx + nn, NodeCoord{c.i, c.j, c.l + 1}, -A.cz[idx]);
    }
  }
}
