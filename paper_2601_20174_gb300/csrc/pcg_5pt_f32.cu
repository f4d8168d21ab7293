// Solver instantiation: 5-point stencil, FP32 preconditioner.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_5PT, float, 5pt_f32)
