// batch_dims_hi.cu -- the batched dimension kernels k_batch_dim<d> for
// d = 9..16 (see batch_dims_lo.cu).
#include "batch_dim.cuh"
#include "kernels.h"

extern "C" const void* gv_batch_dim_kernel_hi(int d, int pif) { return gv::dim_kernel_in<9, 16>(d, pif); }
