// Host-side helpers shared between the translation units.
#pragma once

#include "common.cuh"

// Grid size for `work` items at `threads` per block, capped at per_sm blocks
// per SM (grid-stride loops cover the rest).
int grid_for(const nlsp_ctx* ctx, int64_t work, int threads, int per_sm);

// Device buffer owned by a host scope.
struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  nlsp_status alloc(size_t bytes) {
    if (p) cudaFree(p);
    p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      nlsp_record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
      return e == cudaErrorMemoryAllocation ? NLSP_ERR_OOM : NLSP_ERR_CUDA;
    }
    return NLSP_OK;
  }
  template <typename T> T* as() const { return (T*)p; }
  void* release() {
    void* q = p;
    p = nullptr;
    return q;
  }
};

#define NLSP_DISPATCH_KIND(kind, KIND_CONST, ...)        \
  switch (kind) {                                        \
    case ST_5PT: {                                       \
      constexpr int KIND_CONST = ST_5PT;                 \
      __VA_ARGS__;                                       \
    } break;                                             \
    case ST_9PT: {                                       \
      constexpr int KIND_CONST = ST_9PT;                 \
      __VA_ARGS__;                                       \
    } break;                                             \
    case ST_CSR: {                                       \
      constexpr int KIND_CONST = ST_CSR;                 \
      __VA_ARGS__;                                       \
    } break;                                             \
    default: {                                           \
      constexpr int KIND_CONST = ST_7PT;                 \
      __VA_ARGS__;                                       \
    } break;                                             \
  }

// Setup building blocks implemented in setup.cu and used by pcg.cu.
nlsp_status nlsp_internal_factor(nlsp_ctx* ctx, nlsp_prec* M, int r);
