// batch_dims_lo.cu -- the batched dimension kernels k_batch_dim<d> for
// d = 1..8 (compiled in a unit of their own, beside batch_dims_hi.cu, so
// that the build compiles them in parallel).
#include "batch_dim.cuh"
#include "kernels.h"

extern "C" const void* gv_batch_dim_kernel_lo(int d, int pif) { return gv::dim_kernel_in<1, 8>(d, pif); }
