// C-ABI entry points of the two-level preconditioner apply (Algorithm 1,
// "Apply preconditioner to residual b") and of preconditioned CG (Sec. 4,
// two-grid solver evaluation); the kernels and the host-side solver are in
// pcg_impl.cuh, instantiated per stencil kind and precision by the
// pcg_<kind>_<precision>.cu files.
#include "pcg_impl.cuh"

namespace {

// Self-test: counts the inputs where either conversion differs from the
// hardware one (bit patterns; any NaN matches any NaN).  x holds FP64 bit
// patterns; their low 32 bits serve as the FP32 inputs.
__global__ void k_check_conversions(const unsigned long long* __restrict__ x, int64_t n,
                                    unsigned long long* __restrict__ bad) {
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = __longlong_as_double((long long)x[i]);
    const float a = f64_to_f32_rn(d), b = (float)d;
    if (!(isnan(a) && isnan(b)) && __float_as_uint(a) != __float_as_uint(b)) ++cnt;
    const float f = __uint_as_float((unsigned)(x[i] & 0xFFFFFFFFull));
    const double c = f32_to_f64(f), e = (double)f;
    if (!(isnan(c) && isnan(e)) && __double_as_longlong(c) != __double_as_longlong(e)) ++cnt;
  }
  if (cnt) atomicAdd(bad, cnt);
}

}  // namespace

// Team plan of a batched solve (host only).  Instance i of n[i] nodes gets a
// team of size[i] consecutive CTAs starting at first[i]: ceil(tiles_i /
// tiles_per_cta) CTAs, between 1 and min(num_ctas, tiles_i, cap[i]).  The
// teams are placed greedily, largest estimated area (duration x size) first,
// each in the window of CTAs that frees earliest (ties: least idle time, then
// lowest CTA).  The duration model counts tile-iterations: sqrt(n_i)
// iterations (PCG iteration counts grow with the grid side), each costing the
// team's largest tile share plus 1.5 tiles of barrier time when the team has
// more than one CTA.  start[i] is the planned start in those units; each
// CTA later runs its tasks in (start, instance) order.
nlsp_status nlsp_internal_plan_teams(int count, const int64_t* n, const int* cap, int G, int tiles_per_cta,
                                     int* first, int* size, double* start) {
  if (count < 0 || G < 1 || tiles_per_cta < 0 || (count > 0 && (!n || !first || !size || !start)))
    return NLSP_ERR_INVALID;
  if (tiles_per_cta == 0) tiles_per_cta = 16;
  std::vector<double> dur(count);
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1) return NLSP_ERR_INVALID;
    const int64_t tiles = (n[i] + NLSP_TILE - 1) / NLSP_TILE;
    int64_t hi = std::min<int64_t>(G, tiles);
    if (cap) hi = std::min<int64_t>(hi, std::max(1, cap[i]));
    const int s = (int)std::max<int64_t>(1, std::min<int64_t>(hi, (tiles + tiles_per_cta - 1) / tiles_per_cta));
    size[i] = s;
    const double share = (double)((tiles + s - 1) / s);
    dur[i] = std::sqrt((double)n[i]) * (share + (s > 1 ? 1.5 : 0.0));
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return dur[a] * size[a] > dur[b] * size[b]; });
  std::vector<double> freeat(G, 0.0);
  for (int i : order) {
    const int s = size[i];
    int best_w = 0;
    double best_st = 0.0, best_idle = 0.0;
    for (int w = 0; w + s <= G; ++w) {
      double st = 0.0, idle = 0.0;
      for (int c = w; c < w + s; ++c) st = std::max(st, freeat[c]);
      for (int c = w; c < w + s; ++c) idle += st - freeat[c];
      if (w == 0 || st < best_st || (st == best_st && idle < best_idle)) {
        best_w = w;
        best_st = st;
        best_idle = idle;
      }
    }
    first[i] = best_w;
    start[i] = best_st;
    for (int c = best_w; c < best_w + s; ++c) freeat[c] = best_st + dur[i];
  }
  return NLSP_OK;
}

namespace {

// The instantiation that serves a preconditioner (its operator's stencil kind
// and its precision).
const PcgKindOps* pcg_ops(const nlsp_prec* M) {
  const bool f64 = M->precision == NLSP_FP64;
  switch (M->A->kind) {
    case ST_5PT: return f64 ? nlsp_pcg_ops_5pt_f64() : nlsp_pcg_ops_5pt_f32();
    case ST_9PT: return f64 ? nlsp_pcg_ops_9pt_f64() : nlsp_pcg_ops_9pt_f32();
    case ST_CSR: return f64 ? nlsp_pcg_ops_csr_f64() : nlsp_pcg_ops_csr_f32();
    default: return f64 ? nlsp_pcg_ops_7pt_f64() : nlsp_pcg_ops_7pt_f32();
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
  return pcg_ops(M)->apply(M, m, dev_R, ldr, dev_Z, ldz);
}

extern "C" nlsp_status nlsp_solve(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* Mc, int m, const double* dev_B,
                                  int64_t ldb, double* dev_X, int64_t ldx, const nlsp_solve_params* params,
                                  nlsp_solve_info* infos) {
  if (!ctx || !A || !Mc || !params || Mc->A != A || m < 0 || ldb < A->n || ldx < A->n) return NLSP_ERR_INVALID;
  if (m > 0 && (!dev_B || !dev_X)) return NLSP_ERR_INVALID;
  if (!(params->tol >= 0.0) || params->maxit < 1 || params->graph_mode < 0 || params->graph_mode > 2)
    return NLSP_ERR_INVALID;
  if (m == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  nlsp_prec* M = const_cast<nlsp_prec*>(Mc);
  return pcg_ops(M)->solve(M, m, dev_B, ldb, dev_X, ldx, params, infos);
}

extern "C" nlsp_status nlsp_plan_teams(int count, const int64_t* n, int num_ctas, int tiles_per_cta, int* first_cta,
                                       int* team_size, double* start) {
  return nlsp_internal_plan_teams(count, n, nullptr, num_ctas, tiles_per_cta, first_cta, team_size, start);
}

namespace {

// Signature of a batch: FNV-1a over the stencil kind, precision and every
// instance's node count and active rank, in instance order.
unsigned long long batch_signature(int count, nlsp_prec* const* M) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xFFull;
      h *= 1099511628211ull;
    }
  };
  mix((unsigned long long)count);
  mix((unsigned long long)M[0]->A->kind);
  mix((unsigned long long)M[0]->precision);
  for (int i = 0; i < count; ++i) {
    mix((unsigned long long)M[i]->n);
    mix((unsigned long long)M[i]->r);
  }
  return h;
}

int tuned_tiles(const nlsp_ctx* ctx, unsigned long long key) {
  for (int i = 0; i < 8; ++i)
    if (ctx->tune_tpc[i] > 0 && ctx->tune_key[i] == key) return ctx->tune_tpc[i];
  return 0;
}

void remember_tiles(nlsp_ctx* ctx, unsigned long long key, int tpc) {
  for (int i = 0; i < 8; ++i)
    if (ctx->tune_tpc[i] > 0 && ctx->tune_key[i] == key) {
      ctx->tune_tpc[i] = tpc;
      return;
    }
  const int slot = ctx->tune_next;
  ctx->tune_key[slot] = key;
  ctx->tune_tpc[slot] = tpc;
  ctx->tune_next = (slot + 1) % 8;
}

}  // namespace

extern "C" nlsp_status nlsp_solve_batched(nlsp_ctx* ctx, int count, nlsp_prec* const* M, const double* const* dev_b,
                                          double* const* dev_x, const nlsp_solve_params* params, int tiles_per_cta,
                                          nlsp_solve_info* infos) {
  if (!ctx || !params || count < 0 || tiles_per_cta < 0) return NLSP_ERR_INVALID;
  if (count == 0) return NLSP_OK;
  if (!M || !dev_b || !dev_x || !(params->tol >= 0.0) || params->maxit < 1) return NLSP_ERR_INVALID;
  std::vector<const nlsp_prec*> seen(M, M + count);
  for (int i = 0; i < count; ++i) {
    if (!M[i] || M[i]->ctx != ctx || !dev_b[i] || !dev_x[i] || dev_b[i] == dev_x[i]) return NLSP_ERR_INVALID;
    if (M[i]->precision != M[0]->precision || M[i]->A->kind != M[0]->A->kind) {
      nlsp_record_message("nlsp_solve_batched: every instance must share the stencil kind and the precision");
      return NLSP_ERR_INVALID;
    }
  }
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
    nlsp_record_message("nlsp_solve_batched: a preconditioner appears twice (instances need their own workspace)");
    return NLSP_ERR_INVALID;
  }
  NLSP_CUDA(cudaSetDevice(ctx->device));
  if (tiles_per_cta == 0) tiles_per_cta = tuned_tiles(ctx, batch_signature(count, M));  // 0: the plan's default
  return pcg_ops(M[0])->solve_batched(ctx, count, M, dev_b, dev_x, params, tiles_per_cta, infos);
}

extern "C" nlsp_status nlsp_tune_batched(nlsp_ctx* ctx, int count, nlsp_prec* const* M, const double* const* dev_b,
                                         double* const* dev_x, const nlsp_solve_params* params,
                                         const int* candidates, int ncand, int* best, double* ms_out) {
  if (!ctx || !params || count < 1 || !M || !candidates || ncand < 1 || !best) return NLSP_ERR_INVALID;
  for (int c = 0; c < ncand; ++c)
    if (candidates[c] < 1) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  cudaEvent_t e0, e1;
  NLSP_CUDA(cudaEventCreate(&e0));
  NLSP_CUDA(cudaEventCreate(&e1));
  double best_ms = 0.0;
  int best_t = 0;
  nlsp_status worst = NLSP_OK;
  for (int c = 0; c < ncand && worst >= 0; ++c) {
    nlsp_status st = nlsp_solve_batched(ctx, count, M, dev_b, dev_x, params, candidates[c], nullptr);  // warm
    if (st >= 0) {
      cudaEventRecord(e0, ctx->stream);
      st = nlsp_solve_batched(ctx, count, M, dev_b, dev_x, params, candidates[c], nullptr);
      cudaEventRecord(e1, ctx->stream);
    }
    if (st < 0) {
      worst = st;
      break;
    }
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      worst = NLSP_ERR_CUDA;
      break;
    }
    if (ms_out) ms_out[c] = ms;
    if (best_t == 0 || ms < best_ms) {
      best_ms = ms;
      best_t = candidates[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (worst < 0) return worst;
  *best = best_t;
  remember_tiles(ctx, batch_signature(count, M), best_t);
  return NLSP_OK;
}

extern "C" void nlsp_free_prec(nlsp_prec* M) {
  if (!M) return;
  cudaSetDevice(M->device);
  cudaDeviceSynchronize();  // the context (and its stream) may already be gone
  free_work(M->pcg);
  if (M->storage) cudaFree(M->storage);
  delete M;
}

extern "C" nlsp_status nlsp_prec_phase_times(nlsp_ctx* ctx, const nlsp_prec* M, double* out_ns, int count) {
  if (!ctx || !M || !out_ns || count < 0) return NLSP_ERR_INVALID;
  for (int i = 0; i < count; ++i) out_ns[i] = 0.0;
  if (!M->pcg || !M->pcg->ptimes) return NLSP_OK;
  unsigned long long h[PTIMES_LEN];
  NLSP_CUDA(cudaMemcpyAsync(h, M->pcg->ptimes, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  NLSP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < count && i < PTIMES_LEN; ++i) out_ns[i] = (double)h[i];
  NLSP_CUDA(cudaMemsetAsync(M->pcg->ptimes, 0, sizeof(h), ctx->stream));
  return NLSP_OK;
}

extern "C" nlsp_status nlsp_bench_kernel(nlsp_ctx* ctx, const nlsp_prec* Mc, int which, int reps) {
  if (!ctx || !Mc || reps < 0 || which < 0 || which > 1) return NLSP_ERR_INVALID;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  nlsp_prec* M = const_cast<nlsp_prec*>(Mc);
  NLSP_TRY(ensure_work(M, 1));
  return pcg_ops(M)->bench(M, which, reps);
}

// ============================================================================
// Preconditioner application without device allocation.
//
// For callers that must not allocate device memory while they run: code that
// enqueues work inside its own stream capture (cudaMalloc / cudaFree
// synchronise the device and are illegal during capture), and applications
// whose memory pool owns all of device memory under a fixed cap, where a
// stray cudaMalloc fails or fragments the pool.  The temporaries of
// nlsp_apply_prec (the residual in the preconditioner precision, the two
// smoothing work vectors, the restriction's per-block partials, its arrival
// counter and the coarse correction) live here in one file-scope device
// array instead, sized for n <= NLSP_NOALLOC_MAX_N and r <= NLSP_NOALLOC_MAX_RANK.
// Every GPU that loads the library holds this array until the process exits.
// ============================================================================
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of the array, per device

// Device address of the scratch array on `device` (which must be current).
// Host code cannot use the symbol itself: in host code it names a host-side
// stand-in, not device memory.
nlsp_status noalloc_scratch(int device, unsigned char** out) {
  if (device < 0 || device >= NOALLOC_MAX_DEVICES) return NLSP_ERR_INVALID;
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      nlsp_record_cuda_error(e, "cudaGetSymbolAddress (no-allocation scratch)", __FILE__, __LINE__);
      return NLSP_ERR_CUDA;
    }
    g_noalloc_addr[device] = p;
  }
  *out = (unsigned char*)g_noalloc_addr[device];
  return NLSP_OK;
}

}  // namespace

extern "C" nlsp_status nlsp_apply_prec_noalloc(nlsp_ctx* ctx, const nlsp_prec* M, int m, const double* dev_R,
                                               int64_t ldr, double* dev_Z, int64_t ldz) {
  if (!ctx || !M || m < 0 || (m > 0 && (!dev_R || !dev_Z)) || ldr < M->n || ldz < M->n) return NLSP_ERR_INVALID;
  // the restriction's per-block partials are strided by the stored rank k
  // (r <= k), so k is what the scratch must hold
  if (M->n > NLSP_NOALLOC_MAX_N || M->k > NLSP_NOALLOC_MAX_RANK) {
    nlsp_record_message("nlsp_apply_prec_noalloc: n or rank exceeds NLSP_NOALLOC_MAX_N / NLSP_NOALLOC_MAX_RANK");
    return NLSP_ERR_INVALID;
  }
  if (m == 0) return NLSP_OK;
  NLSP_CUDA(cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  NLSP_TRY(noalloc_scratch(ctx->device, &base));
  return pcg_ops(M)->apply_noalloc(M, base, m, dev_R, ldr, dev_Z, ldz);
}

// Self-test of the solver's integer-pipe FP64 <-> FP32 conversions against
// the hardware conversions (see f64_to_f32_rn / f32_to_f64).
extern "C" nlsp_status nlsp_check_conversions(nlsp_ctx* ctx, const unsigned long long* dev_bits, int64_t n,
                                              unsigned long long* mismatches) {
  if (!ctx || !mismatches || n < 0 || (n > 0 && !dev_bits)) return NLSP_ERR_INVALID;
  unsigned long long* d_bad = nullptr;
  NLSP_CUDA(cudaMallocAsync(&d_bad, sizeof(unsigned long long), ctx->stream));
  NLSP_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), ctx->stream));
  if (n > 0) {
    const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8);
    k_check_conversions<<<g, 256, 0, ctx->stream>>>(dev_bits, n, d_bad);
    NLSP_LAUNCH_CHECK();
    count_launches(ctx, 1);
  }
  unsigned long long h = 0;
  NLSP_CUDA(cudaMemcpyAsync(&h, d_bad, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  NLSP_CUDA(cudaFreeAsync(d_bad, ctx->stream));
  NLSP_CUDA(cudaStreamSynchronize(ctx->stream));
  *mismatches = h;
  return NLSP_OK;
}
