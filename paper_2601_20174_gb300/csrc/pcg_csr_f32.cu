// Solver instantiation: general sparse operator (CSR input, row slices), FP32 preconditioner.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_CSR, float, csr_f32)
