// inst_dgauss_24.cu -- sampling kernels for the two-peak Gaussian integrand with
// 24 random bits per axis.
#include "sample_kernel.cuh"

namespace gv {

bool entries_dgauss_y24(int prec, int d, KernelEntry* out) {
  if (d <= 4) return pick_precision_yb<DoubleGaussian, 4, 24>(prec, out);
  if (d <= 8) return pick_precision_yb<DoubleGaussian, 8, 24>(prec, out);
  if (d <= 16) return pick_precision_yb<DoubleGaussian, 16, 24>(prec, out);
  if (d <= 32) return pick_precision_yb<DoubleGaussian, 32, 24>(prec, out);
  return false;
}

}  // namespace gv
