// inst_rambo.cu -- sampling kernels for the RAMBO + Breit-Wigner integrand
// (d = 4 n; bounds 8, 16, 20 and 32 cover n = 2, 3-4, 5 and 6-8).
#include "sample_kernel.cuh"

namespace gv {

bool entries_rambo(int prec, int d, KernelEntry* out) {
  if (d % 4 != 0 || d < 8) return false;
  if (d <= 8) return pick_precision<RamboBW, 8>(prec, out);
  if (d <= 16) return pick_precision<RamboBW, 16>(prec, out);
  if (d <= 20) return pick_precision<RamboBW, 20>(prec, out);
  if (d <= 32) return pick_precision<RamboBW, 32>(prec, out);
  return false;
}

}  // namespace gv
