// Solver instantiation: general sparse operator (CSR input, row slices), FP64.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_CSR, double, csr_f64)
