// Solver instantiation: 7-point stencil, FP64.
#include "pcg_impl.cuh"

NLSP_PCG_OPS(ST_7PT, double, 7pt_f64)
