// inst_wmunu_24.cu -- sampling kernels for the u dbar -> W+ -> mu+ nu integrand
// (exactly five dimensions) with 24 random bits per axis.
#include "sample_kernel.cuh"

namespace gv {

bool entries_wmunu_y24(int prec, int d, KernelEntry* out) {
  if (d == 5) return pick_precision_yb<WMuNu, 5, 24>(prec, out);
  return false;
}

}  // namespace gv
