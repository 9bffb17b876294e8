// inst_dgauss_53.cu -- sampling kernels for the two-peak Gaussian integrand with
// 53 random bits per axis.
#include "sample_kernel.cuh"

namespace gv {

bool entries_dgauss_y53(int prec, int d, KernelEntry* out) {
  if (d <= 4) return pick_precision_yb<DoubleGaussian, 4, 53>(prec, out);
  if (d <= 8) return pick_precision_yb<DoubleGaussian, 8, 53>(prec, out);
  if (d <= 16) return pick_precision_yb<DoubleGaussian, 16, 53>(prec, out);
  if (d <= 32) return pick_precision_yb<DoubleGaussian, 32, 53>(prec, out);
  return false;
}

}  // namespace gv
