// Shared definitions of the nlsp CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "nlsp.h"

// ----------------------------------------------------------------------------
// Error handling: every CUDA runtime call is checked; failures become
// NLSP_ERR_CUDA (NLSP_ERR_OOM for allocation failures) and are never thrown.
// ----------------------------------------------------------------------------
#define NLSP_CUDA(call)                                                            \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      nlsp_record_cuda_error(e_, #call, __FILE__, __LINE__);                       \
      return e_ == cudaErrorMemoryAllocation ? NLSP_ERR_OOM : NLSP_ERR_CUDA;       \
    }                                                                              \
  } while (0)

#define NLSP_TRY(expr)                                                             \
  do {                                                                             \
    nlsp_status s_ = (expr);                                                       \
    if (s_ < 0) return s_;                                                         \
  } while (0)

#define NLSP_LAUNCH_CHECK() NLSP_CUDA(cudaGetLastError())

void nlsp_record_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void nlsp_record_message(const char* msg);

// 16-byte vector of T (float4 / double2), for broadcast reads of small
// matrices held in shared memory.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int N = 2;
};

// ----------------------------------------------------------------------------
// Geometry and layouts
// ----------------------------------------------------------------------------
// Node tiles: P and the sample block S are stored as tiles of NLSP_TILE
// consecutive nodes, each tile holding all columns contiguously:
//   element (node i, column c) at ((i / W) * ncols + c) * W + (i % W).
// One tile of one column is 512 B (FP32) / 1 KB (FP64): one coalesced warp
// load of float4 / two of double2, and a whole tile (all columns) is a single
// contiguous block for bulk copies.  n is padded to a multiple of W with zero
// rows.
constexpr int NLSP_TILE = 128;

__host__ __device__ inline int64_t tiled_index(int64_t i, int c, int ncols) {
  return (((int64_t)((uint64_t)i >> 7)) * ncols + c) * NLSP_TILE + (int64_t)((uint64_t)i & 127u);
}
static_assert(NLSP_TILE == 128, "tiled_index assumes 128-node tiles");
inline int64_t pad_tile(int64_t n) { return (n + NLSP_TILE - 1) / NLSP_TILE * NLSP_TILE; }

enum StencilKind { ST_5PT = 0, ST_9PT = 1, ST_7PT = 2, ST_CSR = 3 };

// Row slices of the general sparse operator (sliced ELLPACK with sorting
// windows, "SELL-C-sigma"): within each window of NLSP_SIGMA consecutive rows
// the rows are ordered by decreasing length, and every 32 consecutive
// positions of that order form a slice whose off-diagonal entries are stored
// column by column: entry j of the row at position p sits at
// soff[p / 32] + 32 j + p % 32, so a warp on 32 consecutive positions reads
// each of its j-th entries as one coalesced 128-byte (index) / 256-byte (FP64
// value) access.  A slice is as wide as its longest row; shorter rows are
// padded with (own row, 0).  Sorting within windows keeps the padding small
// (rows of similar length share slices) while a window's rows stay close in
// memory.  ppos[i] is the position of row i, prow[p] the row at position p
// (-1 past the last row).
constexpr int NLSP_SLICE = 32;
constexpr int NLSP_SIGMA = 256;

// Matrix-free view of A in one precision.
//  5-point / 7-point: positive edge weights (h^-2 included) to the +x, +y, +z
//  neighbour, zero where that neighbour is a boundary node, the diagonal and
//  its inverse.  (A x)_i = d_i x_i - sum over neighbours of w_e x_nb.
//  9-point constant: signed entries c[0] centre, c[1] E/W, c[2] N/S,
//  c[3] NE/SW, c[4] NW/SE.
//  General sparse (CSR input): the diagonal, its inverse and the signed
//  off-diagonal entries in row slices (soff, scol, sval; see NLSP_SLICE):
//  (A x)_i = d_i x_i + sum_j a_ij x_j.
template <typename T>
struct StencilView {
  int N;
  int64_t n;
  const T* diag;
  const T* cx;
  const T* cy;
  const T* cz;
  const T* dinv;
  T c[5];
  T cdinv;  // 1 / c[0] for the 9-point stencil
  const int64_t* soff;  // slice offsets (n / 32 rounded up, plus one)
  const int* ppos;      // position of each row in the sliced order
  const int* scol;      // column of each sliced entry
  const T* sval;        // value of each sliced entry
};

// ----------------------------------------------------------------------------
// Library objects
// ----------------------------------------------------------------------------
// Grow-only device scratch slots owned by the context: setup and solve
// temporaries are carved from them, so repeated calls allocate nothing once
// the slots have grown to the working size.  Valid until the next call that
// uses the same slot on this context.
enum ScratchSlot { SLOT_SA = 0, SLOT_SB, SLOT_PART, SLOT_SMALL, SLOT_PNEW, SLOT_BATCH, SLOT_ADJ, SLOT_COUNT };

struct nlsp_ctx {
  int device;
  cudaStream_t stream;
  int num_sms;
  size_t l2_bytes;
  void* slot[SLOT_COUNT];
  size_t slot_bytes[SLOT_COUNT];
  unsigned long long launches;  // kernels this context has enqueued
  // batched-solve tuning (nlsp_tune_batched): signature of a set of instance
  // sizes -> fastest tiles per CTA measured for it
  unsigned long long tune_key[8];
  int tune_tpc[8];
  int tune_next;
};

// Returns slot `s` with at least `bytes` (grows it, synchronising the
// device when it has to reallocate).  nullptr on allocation failure.
void* ctx_slot(nlsp_ctx* ctx, int s, size_t bytes);
inline void count_launches(nlsp_ctx* ctx, unsigned long long k) { ctx->launches += k; }

struct nlsp_op {
  nlsp_ctx* ctx;
  int device;  // kept so that freeing never touches a destroyed context
  int dim, points, kind, N;
  int64_t n;
  double* a64;  // one allocation: diag, cx, cy, cz, dinv (n each); general
                // sparse: diag, dinv (n each), then the sliced entries
  float* a32;
  void* sidx;   // general sparse: slice offsets (int64), row positions and the
                // row at each position (int32), entry columns (int32)
  int64_t nnz;  // general sparse: stored entries of the CSR input
  int64_t sliced;  // general sparse: sliced off-diagonal entries (with padding)
  const int* prow;  // general sparse: row at each slice position (-1: none)
  int64_t npos;     // general sparse: slice positions (n rounded up to 32)
  int wmax;         // general sparse: most off-diagonal entries of a row
  double c9[5];
  StencilView<double> v64;
  StencilView<float> v32;
};

struct PcgWork;  // pcg.cu

struct nlsp_prec {
  nlsp_ctx* ctx;
  int device;
  const nlsp_op* A;
  int precision;
  int64_t n, n_pad;
  int k, r, K;
  int nu1, nu2;
  double omega;
  void* P;          // tiled [n_pad/W][k][W], float or double
  double* sigma;    // K singular values (descending)
  double* Ac;       // r x r column-major
  double* L;        // r x r lower Cholesky factor, column-major
  double* Ainv;     // r x r inverse of A_c (from the factor), FP64
  void* AinvT;      // A_c^-1 in the preconditioner precision (== Ainv in FP64)
  void* cpart;      // restriction partials [blocks][k], preconditioner precision
  void* ec;         // coarse correction (k), preconditioner precision
  unsigned* counter;
  int* status;      // device status word (Cholesky pivots)
  int rblocks;      // blocks of the restriction kernel
  // apply workspace (precision T, n_pad each)
  void* w0;
  void* w1;
  PcgWork* pcg;     // lazily built solver workspace and graphs
  void* storage;    // the single allocation holding the arrays above
};

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result valid in
// every thread.  Fixed order => deterministic.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* smem32) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) smem32[wid] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  T t = (threadIdx.x < nw) ? smem32[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) smem32[0] = t;
  __syncthreads();
  T r = smem32[0];
  __syncthreads();
  return r;
}

// "Last block done": every block publishes its partial, then one arrival
// counter decides which block is last; that block sees every partial
// (threadfence before and after the counter) and resets the counter.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter, int* smem_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    *smem_flag = (prev == gridDim.x - 1);
  }
  __syncthreads();
  bool last = *smem_flag != 0;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// Deterministic sum of `count` partials (stride `stride`) by one block.
__device__ __forceinline__ double block_sum_partials(const double* part, int count, int stride,
                                                     double* smem32) {
  double s = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x) s += part[(int64_t)b * stride];
  return block_sum(s, smem32);
}

template <typename T> __device__ __forceinline__ T ld_cg(const T* p) { return *p; }

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }
