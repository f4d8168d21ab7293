// Solver instantiation: 5-point stencil, FP64.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_5PT, double, 5pt_f64)
