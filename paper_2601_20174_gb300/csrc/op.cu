// Context management and the operator A (Sec. 3, Eq. discretized_pde;
// Algorithm 1 setup line D = diag(A)).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "stencil.cuh"
#include "kernels.cuh"

static thread_local char g_last_error[512];

void nlsp_record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file,
           line);
  if (getenv("NLSP_VERBOSE")) fprintf(stderr, "[nlsp] %s\n", g_last_error);
}

void nlsp_record_message(const char* msg) {
  snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
  if (getenv("NLSP_VERBOSE")) fprintf(stderr, "[nlsp] %s\n", g_last_error);
}

extern "C" const char* nlsp_last_error(void) { return g_last_error; }

extern "C" const char* nlsp_status_string(int status) {
  switch (status) {
    case NLSP_OK: return "NLSP_OK";
    case NLSP_NOT_CONVERGED: return "NLSP_NOT_CONVERGED";
    case NLSP_ERR_INVALID: return "NLSP_ERR_INVALID";
    case NLSP_ERR_CUDA: return "NLSP_ERR_CUDA";
    case NLSP_ERR_NOT_SPD: return "NLSP_ERR_NOT_SPD";
    case NLSP_ERR_BREAKDOWN: return "NLSP_ERR_BREAKDOWN";
    case NLSP_ERR_TIMEOUT: return "NLSP_ERR_TIMEOUT";
    case NLSP_ERR_OOM: return "NLSP_ERR_OOM";
    default: return "NLSP_UNKNOWN_STATUS";
  }
}

extern "C" nlsp_status nlsp_create(nlsp_ctx** ctx_out, int device, void* cuda_stream) {
  if (!ctx_out) return NLSP_ERR_INVALID;
  *ctx_out = nullptr;
  int count = 0;
  NLSP_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(device));
  nlsp_ctx* c = new nlsp_ctx();
  memset(c, 0, sizeof(*c));
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  int sms = 0, l2 = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  c->num_sms = sms > 0 ? sms : 1;
  c->l2_bytes = (size_t)l2;
  *ctx_out = c;
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_set_stream(nlsp_ctx* ctx, void* cuda_stream) {
  if (!ctx) return NLSP_ERR_INVALID;
  ctx->stream = (cudaStream_t)cuda_stream;
  return NLSP_OK;
}

extern "C" void nlsp_destroy(nlsp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (int s = 0; s < SLOT_COUNT; ++s)
    if (ctx->slot[s]) cudaFree(ctx->slot[s]);
  delete ctx;
}

void* ctx_slot(nlsp_ctx* ctx, int s, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (ctx->slot_bytes[s] >= bytes) return ctx->slot[s];
  if (ctx->slot[s]) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->slot[s]);
  }
  ctx->slot[s] = nullptr;
  ctx->slot_bytes[s] = 0;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    nlsp_record_cuda_error(e, "cudaMalloc (scratch)", __FILE__, __LINE__);
    return nullptr;
  }
  ctx->slot[s] = p;
  ctx->slot_bytes[s] = bytes;
  return p;
}

extern "C" unsigned long long nlsp_launch_count(const nlsp_ctx* ctx) { return ctx ? ctx->launches : 0ull; }

// ----------------------------------------------------------------------------
// Assembly kernels: cell kappa -> edge weights, diagonal and its inverse.
// ----------------------------------------------------------------------------
namespace {

// 2D: x-edge between node columns i and i+1 of node row j lies in cell column
// i+1 between cell rows j and j+1; y-edge between node rows j and j+1 of node
// column i lies in cell row j+1 between cell columns i and i+1.  Weight = mean
// of the two cells, scaled by h^-2.
__global__ void k_assemble_5pt(int N, const double* __restrict__ kap, double* diag, double* cx, double* cy,
                               double* dinv, int* bad) {
  const int64_t n = (int64_t)N * N;
  const int M = N + 1;
  const double h2 = (double)M * (double)M;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx - (int64_t)j * N);
    auto K = [&](int cj, int ci) { return kap[(int64_t)cj * M + ci]; };
    const double west = 0.5 * (K(j, i) + K(j + 1, i)) * h2;
    const double east = 0.5 * (K(j, i + 1) + K(j + 1, i + 1)) * h2;
    const double south = 0.5 * (K(j, i) + K(j, i + 1)) * h2;
    const double north = 0.5 * (K(j + 1, i) + K(j + 1, i + 1)) * h2;
    const double d = west + east + south + north;
    diag[idx] = d;
    cx[idx] = (i < N - 1) ? east : 0.0;
    cy[idx] = (j < N - 1) ? north : 0.0;
    dinv[idx] = 1.0 / d;
    if (!(d > 0.0) || !(west > 0.0) || !(east > 0.0) || !(south > 0.0) || !(north > 0.0) || !isfinite(d))
      atomicOr(bad, 1);
  }
}

// 3D: the x-edge between node columns i and i+1 at (j, l) lies in cell column
// i+1 and is surrounded by cells (j|j+1, l|l+1); similarly for y and z.
__global__ void k_assemble_7pt(int N, const double* __restrict__ kap, double* diag, double* cx, double* cy,
                               double* cz, double* dinv, int* bad) {
  const int64_t nn = (int64_t)N * N, n = nn * N;
  const int M = N + 1;
  const double h2 = (double)M * (double)M;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx / nn);
    const int rem = (int)(idx - (int64_t)l * nn);
    const int j = rem / N, i = rem - j * N;
    auto K = [&](int cl, int cj, int ci) { return kap[((int64_t)cl * M + cj) * M + ci]; };
    auto xedge = [&](int ci) { return 0.25 * (K(l, j, ci) + K(l, j + 1, ci) + K(l + 1, j, ci) + K(l + 1, j + 1, ci)) * h2; };
    auto yedge = [&](int cj) { return 0.25 * (K(l, cj, i) + K(l, cj, i + 1) + K(l + 1, cj, i) + K(l + 1, cj, i + 1)) * h2; };
    auto zedge = [&](int cl) { return 0.25 * (K(cl, j, i) + K(cl, j, i + 1) + K(cl, j + 1, i) + K(cl, j + 1, i + 1)) * h2; };
    const double xw = xedge(i), xe = xedge(i + 1), ys = yedge(j), yn = yedge(j + 1), zd = zedge(l),
                 zu = zedge(l + 1);
    const double d = xw + xe + ys + yn + zd + zu;
    diag[idx] = d;
    cx[idx] = (i < N - 1) ? xe : 0.0;
    cy[idx] = (j < N - 1) ? yn : 0.0;
    cz[idx] = (l < N - 1) ? zu : 0.0;
    dinv[idx] = 1.0 / d;
    if (!(xw > 0.0) || !(xe > 0.0) || !(ys > 0.0) || !(yn > 0.0) || !(zd > 0.0) || !(zu > 0.0) || !isfinite(d))
      atomicOr(bad, 1);
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

template <int KIND>
__global__ void k_apply_cols(StencilView<double> A, int m, const double* __restrict__ X, int64_t ldx,
                             double* __restrict__ Y, int64_t ldy) {
  const int col = blockIdx.y;
  const double* x = X + col * ldx;
  double* y = Y + col * ldy;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < A.n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    NodeCoord c = node_coord<KIND>(idx, A.N);
    y[idx] = stencil_apply<KIND>(A, idx, c, [&](int64_t m_) { return x[m_]; });
  }
}

// General sparse operator from CSR (rowptr int64, col int32, val FP64):
// per row the number of off-diagonal entries, the diagonal (sum of the row's
// diagonal entries) and its inverse.  bad: bit 0 column out of range, bit 1
// non-positive or non-finite diagonal, bit 2 row pointers not monotone or not
// spanning [0, nnz), bit 3 non-finite entry.
__global__ void k_csr_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, int* __restrict__ cnt, double* __restrict__ diag,
                           double* __restrict__ dinv, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    int flags = 0;
    if (b < 0 || e < b || e > nnz || (i == 0 && b != 0) || (i == n - 1 && e != nnz)) {
      atomicOr(bad, 4);
      cnt[i] = 0;
      diag[i] = 1.0;
      dinv[i] = 1.0;
      continue;
    }
    double d = 0.0;
    int c = 0;
    for (int64_t q = b; q < e; ++q) {
      const int j = col[q];
      const double v = val[q];
      if (j < 0 || (int64_t)j >= n) flags |= 1;
      if (!isfinite(v)) flags |= 8;
      if ((int64_t)j == i) d += v;
      else ++c;
    }
    if (!(d > 0.0) || !isfinite(d)) flags |= 2;
    cnt[i] = c;
    diag[i] = d;
    dinv[i] = 1.0 / d;
    if (flags) atomicOr(bad, flags);
  }
}

// Scatters each row's off-diagonal entries into its slice (entry j of the
// row at position p at soff[p / 32] + 32 j + p % 32) and pads the row to the
// slice width with (own row, 0).
__global__ void k_csr_fill(int64_t n, const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, const int64_t* __restrict__ soff,
                           const int* __restrict__ ppos, int* __restrict__ scol, double* __restrict__ sval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = ppos[i];
    const int64_t sl = p / NLSP_SLICE;
    const int64_t base = soff[sl] + p % NLSP_SLICE;
    const int w = (int)((soff[sl + 1] - soff[sl]) / NLSP_SLICE);
    int c = 0;
    for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int j = col[q];
      if ((int64_t)j == i) continue;
      scol[base + (int64_t)NLSP_SLICE * c] = j;
      sval[base + (int64_t)NLSP_SLICE * c] = val[q];
      ++c;
    }
    for (; c < w; ++c) {
      scol[base + (int64_t)NLSP_SLICE * c] = (int)i;
      sval[base + (int64_t)NLSP_SLICE * c] = 0.0;
    }
  }
}

// y = A x for the general sparse operator in position order: thread per
// slice position, so each warp's j-th entries are one coalesced access; the
// row's result goes to y[prow[p]] (rows of one sorting window stay within a
// few cache lines).  Column-batched over blockIdx.y like k_apply_cols.
__global__ void __launch_bounds__(256) k_csr_spmv(StencilView<double> A, const int* __restrict__ prow, int64_t npos,
                                                  const double* __restrict__ X, int64_t ldx, double* __restrict__ Y,
                                                  int64_t ldy) {
  const double* x = X + blockIdx.y * ldx;
  double* y = Y + blockIdx.y * ldy;
  const double* __restrict__ sval = A.sval;
  const int* __restrict__ scol = A.scol;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = prow[p];
    const int64_t sl = p >> 5;
    const int64_t s0 = A.soff[sl];
    const int64_t base = s0 + (p & 31);
    const int w = (int)((A.soff[sl + 1] - s0) >> 5);
    double s = 0.0;
    int j = 0;
    for (; j + 4 <= w; j += 4) {  // four entries' loads in flight
      const int64_t e = base + 32 * (int64_t)j;
      const int c0 = __ldg(scol + e), c1 = __ldg(scol + e + 32), c2 = __ldg(scol + e + 64), c3 = __ldg(scol + e + 96);
      const double v0 = __ldg(sval + e), v1 = __ldg(sval + e + 32), v2 = __ldg(sval + e + 64), v3 = __ldg(sval + e + 96);
      s = fma(v0, x[c0], s);
      s = fma(v1, x[c1], s);
      s = fma(v2, x[c2], s);
      s = fma(v3, x[c3], s);
    }
    for (; j < w; ++j) {
      const int64_t e = base + 32 * (int64_t)j;
      s = fma(__ldg(sval + e), x[__ldg(scol + e)], s);
    }
    if (i >= 0) y[i] = fma(A.diag[i], x[i], s);
  }
}

__global__ void k_diag_9pt(double d, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = d;
}

}  // namespace

int grid_for(const nlsp_ctx* ctx, int64_t work, int threads, int per_sm) {
  int64_t g = (work + threads - 1) / threads;
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

extern "C" nlsp_status nlsp_assemble_stencil(nlsp_ctx* ctx, int dim, const int64_t grid[3], int points,
                                             const double* dev_coeffs, int coeff_layout, nlsp_op** A_out) {
  if (!ctx || !grid || !dev_coeffs || !A_out) return NLSP_ERR_INVALID;
  *A_out = nullptr;
  int kind;
  if (dim == 2 && points == 5 && coeff_layout == NLSP_COEF_CELL_KAPPA) kind = ST_5PT;
  else if (dim == 2 && points == 9 && coeff_layout == NLSP_COEF_CONST_TENSOR) kind = ST_9PT;
  else if (dim == 3 && points == 7 && coeff_layout == NLSP_COEF_CELL_KAPPA) kind = ST_7PT;
  else return NLSP_ERR_INVALID;
  const int64_t N = grid[0];
  if (N < 1 || grid[1] != N || (dim == 3 ? grid[2] != N : (grid[2] != 1 && grid[2] != 0))) return NLSP_ERR_INVALID;
  const int64_t n = dim == 3 ? N * N * N : N * N;
  if (N > 65535 || n > ((int64_t)1 << 31) - 1) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));

  nlsp_op* op = new nlsp_op();
  memset(op, 0, sizeof(*op));
  op->ctx = ctx;
  op->device = ctx->device;
  op->dim = dim;
  op->points = points;
  op->kind = kind;
  op->N = (int)N;
  op->n = n;
  cudaStream_t s = ctx->stream;
  int* bad = nullptr;
  auto fail = [&](nlsp_status e) {
    if (bad) cudaFree(bad);
    nlsp_free_op(op);
    return e;
  };
  const double h2 = (double)(N + 1) * (double)(N + 1);
  if (kind == ST_9PT) {
    double t[3];
    if (cudaMemcpy(t, dev_coeffs, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(NLSP_ERR_CUDA);
    const double axx = t[0], ayy = t[1], axy = t[2];
    if (!(axx > 0.0) || !(ayy > 0.0) || !(axx * ayy > axy * axy)) return fail(NLSP_ERR_INVALID);
    op->c9[0] = 2.0 * (axx + ayy) * h2;
    op->c9[1] = -axx * h2;
    op->c9[2] = -ayy * h2;
    op->c9[3] = -0.5 * axy * h2;
    op->c9[4] = 0.5 * axy * h2;
  } else {
    if (cudaMalloc(&op->a64, sizeof(double) * 5 * n) != cudaSuccess) return fail(NLSP_ERR_OOM);
    if (cudaMalloc(&op->a32, sizeof(float) * 5 * n) != cudaSuccess) return fail(NLSP_ERR_OOM);
    if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) return fail(NLSP_ERR_OOM);
    if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
    if (cudaMemsetAsync(op->a64, 0, sizeof(double) * 5 * n, s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
    double* d = op->a64;
    const int g = grid_for(ctx, n, 256, 8);
    if (kind == ST_5PT)
      k_assemble_5pt<<<g, 256, 0, s>>>((int)N, dev_coeffs, d, d + n, d + 2 * n, d + 4 * n, bad);
    else
      k_assemble_7pt<<<g, 256, 0, s>>>((int)N, dev_coeffs, d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, bad);
    k_to_float<<<grid_for(ctx, 5 * n, 256, 8), 256, 0, s>>>(op->a64, op->a32, 5 * n);
    count_launches(ctx, 2);
    if (cudaGetLastError() != cudaSuccess) return fail(NLSP_ERR_CUDA);
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
    cudaFree(bad);
    bad = nullptr;
    if (hbad) return fail(NLSP_ERR_INVALID);
  }
  // views
  StencilView<double>& v = op->v64;
  StencilView<float>& w = op->v32;
  v.N = w.N = (int)N;
  v.n = w.n = n;
  if (op->a64) {
    v.diag = op->a64; v.cx = op->a64 + n; v.cy = op->a64 + 2 * n; v.cz = op->a64 + 3 * n; v.dinv = op->a64 + 4 * n;
    w.diag = op->a32; w.cx = op->a32 + n; w.cy = op->a32 + 2 * n; w.cz = op->a32 + 3 * n; w.dinv = op->a32 + 4 * n;
  }
  for (int q = 0; q < 5; ++q) {
    v.c[q] = op->c9[q];
    w.c[q] = (float)op->c9[q];
  }
  v.cdinv = kind == ST_9PT ? 1.0 / op->c9[0] : 0.0;
  w.cdinv = (float)v.cdinv;
  *A_out = op;
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_assemble_csr(nlsp_ctx* ctx, int64_t n, int64_t nnz, const int64_t* dev_rowptr,
                                         const int32_t* dev_col, const double* dev_val, nlsp_op** A_out) {
  if (!ctx || !A_out || !dev_rowptr || !dev_col || !dev_val) return NLSP_ERR_INVALID;
  *A_out = nullptr;
  if (n < 1 || n > ((int64_t)1 << 31) - 1 || nnz < n) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  nlsp_op* op = new nlsp_op();
  memset(op, 0, sizeof(*op));
  op->ctx = ctx;
  op->device = ctx->device;
  op->dim = 0;
  op->points = 0;
  op->kind = ST_CSR;
  op->N = 0;
  op->n = n;
  op->nnz = nnz;
  cudaStream_t s = ctx->stream;
  const int64_t nsl = (n + NLSP_SLICE - 1) / NLSP_SLICE;
  DevBuf tmp;  // row counts (n), error word
  auto fail = [&](nlsp_status e) {
    nlsp_free_op(op);
    return e;
  };
  nlsp_status st = tmp.alloc(sizeof(int) * (size_t)(n + 1));
  if (st != NLSP_OK) return fail(st);
  int* cnt = tmp.as<int>();
  int* bad = cnt + n;
  DevBuf dd;  // diagonal and inverse before the final allocation is sized
  if ((st = dd.alloc(sizeof(double) * 2 * (size_t)n)) != NLSP_OK) return fail(st);
  if (cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
  const int g = grid_for(ctx, n, 256, 8);
  k_csr_rows<<<g, 256, 0, s>>>(n, nnz, dev_rowptr, (const int*)dev_col, dev_val, cnt, dd.as<double>(),
                               dd.as<double>() + n, bad);
  count_launches(ctx, 1);
  if (cudaGetLastError() != cudaSuccess) return fail(NLSP_ERR_CUDA);
  std::vector<int> hc((size_t)n + 1);
  if (cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * (size_t)(n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return fail(NLSP_ERR_CUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
  const int hbad = hc[(size_t)n];
  if (hbad) {
    nlsp_record_message((hbad & 4) ? "nlsp_assemble_csr: row pointers are not monotone from 0 to nnz"
                        : (hbad & 1) ? "nlsp_assemble_csr: a column index is outside [0, n)"
                        : (hbad & 8) ? "nlsp_assemble_csr: a non-finite entry"
                                     : "nlsp_assemble_csr: a diagonal entry is missing, non-positive or non-finite");
    return fail(NLSP_ERR_INVALID);
  }
  // positions: rows of each window of NLSP_SIGMA ordered by decreasing
  // off-diagonal count (ties by row), then slice widths and offsets
  const int64_t npos = nsl * NLSP_SLICE;
  std::vector<int> prow((size_t)npos, -1), ppos((size_t)n);
  for (int64_t w0 = 0; w0 < n; w0 += NLSP_SIGMA) {
    const int64_t w1 = std::min<int64_t>(n, w0 + NLSP_SIGMA);
    for (int64_t i = w0; i < w1; ++i) prow[(size_t)i] = (int)i;
    std::stable_sort(prow.begin() + w0, prow.begin() + w1, [&](int a, int b) { return hc[(size_t)a] > hc[(size_t)b]; });
    for (int64_t q = w0; q < w1; ++q) ppos[(size_t)prow[(size_t)q]] = (int)q;
  }
  op->wmax = 0;
  for (int64_t i = 0; i < n; ++i) op->wmax = std::max(op->wmax, hc[(size_t)i]);
  std::vector<int64_t> soff((size_t)nsl + 1);
  soff[0] = 0;
  for (int64_t q = 0; q < nsl; ++q) {
    int wmax = 0;
    for (int64_t p = q * NLSP_SLICE; p < (q + 1) * NLSP_SLICE && p < n; ++p) wmax = std::max(wmax, hc[(size_t)prow[(size_t)p]]);
    soff[(size_t)q + 1] = soff[(size_t)q] + (int64_t)NLSP_SLICE * wmax;
  }
  const int64_t sliced = soff[(size_t)nsl];
  op->sliced = sliced;
  const size_t nval = (size_t)(2 * n + sliced);
  if (cudaMalloc(&op->a64, sizeof(double) * nval) != cudaSuccess) return fail(NLSP_ERR_OOM);
  if (cudaMalloc(&op->a32, sizeof(float) * nval) != cudaSuccess) return fail(NLSP_ERR_OOM);
  const size_t idx_bytes = sizeof(int64_t) * (size_t)(nsl + 1) + sizeof(int) * (size_t)(n + npos) +
                           sizeof(int) * (size_t)std::max<int64_t>(sliced, 1);
  if (cudaMalloc(&op->sidx, idx_bytes) != cudaSuccess) return fail(NLSP_ERR_OOM);
  int64_t* d_soff = (int64_t*)op->sidx;
  int* d_ppos = (int*)(d_soff + nsl + 1);
  int* d_prow = d_ppos + n;
  int* d_scol = d_prow + npos;
  op->prow = d_prow;
  op->npos = npos;
  if (cudaMemsetAsync(op->a64, 0, sizeof(double) * nval, s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
  if (cudaMemsetAsync(op->sidx, 0, idx_bytes, s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
  if (cudaMemcpyAsync(op->a64, dd.p, sizeof(double) * 2 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(NLSP_ERR_CUDA);
  if (cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * soff.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_ppos, ppos.data(), sizeof(int) * ppos.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_prow, prow.data(), sizeof(int) * prow.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(NLSP_ERR_CUDA);
  k_csr_fill<<<g, 256, 0, s>>>(n, dev_rowptr, (const int*)dev_col, dev_val, d_soff, d_ppos, d_scol, op->a64 + 2 * n);
  k_to_float<<<grid_for(ctx, (int64_t)nval, 256, 8), 256, 0, s>>>(op->a64, op->a32, (int64_t)nval);
  count_launches(ctx, 2);
  if (cudaGetLastError() != cudaSuccess) return fail(NLSP_ERR_CUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(NLSP_ERR_CUDA);
  StencilView<double>& v = op->v64;
  StencilView<float>& w = op->v32;
  v.N = w.N = 0;
  v.n = w.n = n;
  v.diag = op->a64;
  v.dinv = op->a64 + n;
  v.sval = op->a64 + 2 * n;
  w.diag = op->a32;
  w.dinv = op->a32 + n;
  w.sval = op->a32 + 2 * n;
  v.soff = w.soff = d_soff;
  v.ppos = w.ppos = d_ppos;
  v.scol = w.scol = d_scol;
  *A_out = op;
  return NLSP_OK;
}

extern "C" int64_t nlsp_op_size(const nlsp_op* A) { return A ? A->n : -1; }

extern "C" nlsp_status nlsp_op_apply(nlsp_ctx* ctx, const nlsp_op* A, int m, const double* dev_X, int64_t ldx,
                                     double* dev_Y, int64_t ldy) {
  if (!ctx || !A || m < 0 || (m > 0 && (!dev_X || !dev_Y)) || ldx < A->n || ldy < A->n || m > 65535)
    return NLSP_ERR_INVALID;
  if (m == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  dim3 g(grid_for(ctx, A->n, 256, 8), m);
  switch (A->kind) {
    case ST_5PT: k_apply_cols<ST_5PT><<<g, 256, 0, ctx->stream>>>(A->v64, m, dev_X, ldx, dev_Y, ldy); break;
    case ST_9PT: k_apply_cols<ST_9PT><<<g, 256, 0, ctx->stream>>>(A->v64, m, dev_X, ldx, dev_Y, ldy); break;
    case ST_CSR:
      k_csr_spmv<<<dim3(grid_for(ctx, A->npos, 256, 8), m), 256, 0, ctx->stream>>>(A->v64, A->prow, A->npos, dev_X,
                                                                                   ldx, dev_Y, ldy);
      break;
    default: k_apply_cols<ST_7PT><<<g, 256, 0, ctx->stream>>>(A->v64, m, dev_X, ldx, dev_Y, ldy); break;
  }
  count_launches(ctx, 1);
  NLSP_LAUNCH_CHECK();
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_op_diagonal(nlsp_ctx* ctx, const nlsp_op* A, double* dev_d) {
  if (!ctx || !A || !dev_d) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  if (A->kind == ST_9PT) {
    k_diag_9pt<<<grid_for(ctx, A->n, 256, 8), 256, 0, ctx->stream>>>(A->c9[0], dev_d, A->n);
    NLSP_LAUNCH_CHECK();
  } else {
    NLSP_CUDA(cudaMemcpyAsync(dev_d, A->a64, sizeof(double) * A->n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return NLSP_OK;
}

extern "C" void nlsp_free_op(nlsp_op* A) {
  if (!A) return;
  cudaSetDevice(A->device);
  if (A->a64) cudaFree(A->a64);
  if (A->a32) cudaFree(A->a32);
  if (A->sidx) cudaFree(A->sidx);
  delete A;
}
