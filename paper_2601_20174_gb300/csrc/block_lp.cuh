// Reduced-precision tensor-core contractions of the block solver: the
// restriction P_r^T rho (r x 32) and the prolongation z += P_r E (n x 32) with
// TF32 or BF16 operands and FP32 accumulation in tensor memory (tcgen05.mma,
// kind::tf32 / kind::f16), for preconditioners built with NLSP_MIXED_TF32 /
// NLSP_MIXED_BF16.
//
// P is repacked once per block solve into two operand copies in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices,
// element (row, kk) of a `kcols`-wide operand at ((row / 8) (kcols / E) +
// kk / E) 128 + (row % 8) 16 + (kk % E) es for E = 16 / es elements of es
// bytes per core row):
//   R copy: per 64-node chunk of a tile, rows = the r columns of P (padded to
//           a multiple of 8), K = the chunk's nodes;
//   Q copy: per 128-node tile, rows = the nodes, K = the columns of P
//           (padded to a multiple of 16, zeros beyond r).
// Each chunk / tile is one contiguous block, so a single bulk asynchronous
// copy (cp.async.bulk + mbarrier) moves it from HBM into shared memory in the
// layout the MMA reads: no thread touches P.  A ring of stages keeps several
// copies in flight while the MMAs of earlier ones run; completion of each MMA
// group is tracked by tcgen05.commit on mbarriers, so the threads computing
// the next residual chunk (restriction) or adding the previous tile's result
// to z (prolongation) overlap the copies and the MMAs.  Every wait is bounded
// (2 s); a wait that gives up sets BlockState::err and the kernel returns
// after draining its copies.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace lp {

enum { OP_TF32 = 0, OP_BF16 = 1 };

template <int OP>
struct Op;
template <>
struct Op<OP_TF32> {
  using S = uint32_t;                // storage: the TF32-rounded FP32 bit pattern
  static constexpr int ES = 4;       // bytes per element
  static constexpr int EPC = 4;      // elements per 16-byte core row
  static constexpr int KSTEP = 8;    // K of one MMA instruction
  static constexpr unsigned FMT = 2; // a/b format code of kind::tf32
  __device__ __forceinline__ static S cvt(float x) {
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    return h;
  }
};
template <>
struct Op<OP_BF16> {
  using S = uint16_t;
  static constexpr int ES = 2;
  static constexpr int EPC = 8;
  static constexpr int KSTEP = 16;
  static constexpr unsigned FMT = 1;  // BF16 in kind::f16
  __device__ __forceinline__ static S cvt(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
};

// Byte offset of element (row, kk) in a canonical K-major operand kcols wide.
template <int OP>
__host__ __device__ __forceinline__ unsigned off(int row, int kk, int kcols) {
  constexpr int E = Op<OP>::EPC;
  return (unsigned)(((row >> 3) * (kcols / E) + kk / E) * 128 + (row & 7) * 16 + (kk % E) * Op<OP>::ES);
}

constexpr int RCH = 64;  // nodes per restriction chunk (K of the restriction MMAs)
constexpr int MBC = 32;  // columns of the block vectors (N of the MMAs)

__host__ __device__ inline int rows_r(int r) { return (r + 7) / 8 * 8; }     // R copy rows
__host__ __device__ inline int kcols_q(int r) { return (r + 15) / 16 * 16; }  // Q copy K width

// Instruction descriptor: FP32 accumulate, A and B of format FMT, K-major
// both, N = 32, M = 128.
template <int OP>
__device__ __forceinline__ constexpr unsigned idesc() {
  return (1u << 4) | (Op<OP>::FMT << 7) | (Op<OP>::FMT << 10) | ((unsigned)(MBC >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFF) >> 4) | ((unsigned long long)(128u >> 4) << 16) |
         ((unsigned long long)(sbo >> 4) << 32) | (1ull << 46);
}

// D [+]= A B^T over `ksteps` MMA instructions (A: 128 rows, B: 32 rows,
// consecutive K steps 256 bytes apart in both operands).
template <int OP>
__device__ __forceinline__ void mma_run(unsigned tmem_d, unsigned a, unsigned a_sbo, unsigned b, unsigned b_sbo,
                                        int ksteps, bool accumulate) {
  constexpr unsigned id = idesc<OP>();
  for (int ks = 0; ks < ksteps; ++ks) {
    const unsigned long long ad = sdesc(a + ks * 256, a_sbo);
    const unsigned long long bd = sdesc(b + ks * 256, b_sbo);
    const unsigned acc = (accumulate || ks > 0) ? 1u : 0u;
    if (OP == OP_TF32)
      asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                   "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                   "l"(ad), "l"(bd), "r"(id), "r"(acc)
                   : "memory");
    else
      asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                   "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                   "l"(ad), "l"(bd), "r"(id), "r"(acc)
                   : "memory");
  }
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tma::smem_addr(bar))
               : "memory");
}

// Repacks the tiled FP32 P (first r of kst columns) into the R and Q copies.
template <int OP>
__global__ void k_pack(const float* __restrict__ P, int kst, int r, int64_t ntiles, unsigned char* __restrict__ Rc,
                       unsigned char* __restrict__ Qc) {
  using S = typename Op<OP>::S;
  const int rr = rows_r(r), kq = kcols_q(r);
  const size_t rchunk = (size_t)rr * RCH * Op<OP>::ES, qtile = (size_t)NLSP_TILE * kq * Op<OP>::ES;
  const int64_t total = ntiles * NLSP_TILE * (int64_t)kq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(e % NLSP_TILE);
    const int j = (int)((e / NLSP_TILE) % kq);
    const int64_t t = e / ((int64_t)NLSP_TILE * kq);
    const float v = j < r ? P[(t * kst + j) * NLSP_TILE + w] : 0.0f;
    const S s = Op<OP>::cvt(v);
    *reinterpret_cast<S*>(Qc + t * qtile + off<OP>(w, j, kq)) = s;
    if (j < rr) {
      const int h = w / RCH;
      *reinterpret_cast<S*>(Rc + (t * 2 + h) * rchunk + off<OP>(j, w % RCH, RCH)) = s;
    }
  }
}

}  // namespace lp
