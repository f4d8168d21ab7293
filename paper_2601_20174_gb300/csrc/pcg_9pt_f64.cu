// Solver instantiation: 9-point stencil, FP64.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_9PT, double, 9pt_f64)
