// inst_genz_discontinuous_53.cu -- sampling kernels for the Genz discontinuous integrand with
// 53 random bits per axis.
#include "sample_kernel.cuh"

namespace gv {

bool entries_genz_discontinuous_y53(int prec, int d, KernelEntry* out) {
  if (d <= 4) return pick_precision_yb<GenzDiscontinuous, 4, 53>(prec, out);
  if (d <= 8) return pick_precision_yb<GenzDiscontinuous, 8, 53>(prec, out);
  if (d <= 16) return pick_precision_yb<GenzDiscontinuous, 16, 53>(prec, out);
  if (d <= 32) return pick_precision_yb<GenzDiscontinuous, 32, 53>(prec, out);
  return false;
}

}  // namespace gv
