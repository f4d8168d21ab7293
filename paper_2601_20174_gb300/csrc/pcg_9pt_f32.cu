// Solver instantiation: 9-point stencil, FP32 preconditioner.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_9PT, float, 9pt_f32)
