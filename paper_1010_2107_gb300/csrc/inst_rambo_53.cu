// inst_rambo_53.cu -- sampling kernels for the RAMBO + Breit-Wigner integrand
// with 53 random bits per axis (d = 4 n; bounds 8, 16, 20 and 32 cover
// n = 2, 3-4, 5 and 6-8).
#include "sample_kernel.cuh"

namespace gv {

bool entries_rambo_y53(int prec, int d, KernelEntry* out) {
  if (d % 4 != 0 || d < 8) return false;
  if (d <= 8) return pick_precision_yb<RamboBW, 8, 53>(prec, out);
  if (d <= 16) return pick_precision_yb<RamboBW, 16, 53>(prec, out);
  if (d <= 20) return pick_precision_yb<RamboBW, 20, 53>(prec, out);
  if (d <= 32) return pick_precision_yb<RamboBW, 32, 53>(prec, out);
  return false;
}

}  // namespace gv
