// inst_genz_continuous_24.cu -- sampling kernels for the Genz continuous integrand with
// 24 random bits per axis.
#include "sample_kernel.cuh"

namespace gv {

bool entries_genz_continuous_y24(int prec, int d, KernelEntry* out) {
  if (d <= 4) return pick_precision_yb<GenzContinuous, 4, 24>(prec, out);
  if (d <= 8) return pick_precision_yb<GenzContinuous, 8, 24>(prec, out);
  if (d <= 16) return pick_precision_yb<GenzContinuous, 16, 24>(prec, out);
  if (d <= 32) return pick_precision_yb<GenzContinuous, 32, 24>(prec, out);
  return false;
}

}  // namespace gv
