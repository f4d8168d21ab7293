// Solver instantiation: 7-point stencil, FP32 preconditioner.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_7PT, float, 7pt_f32)
