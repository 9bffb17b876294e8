// inst_wmunu_53.cu -- sampling kernels for the u dbar -> W+ -> mu+ nu integrand
// (exactly five dimensions) with 53 random bits per axis.
#include "sample_kernel.cuh"

namespace gv {

bool entries_wmunu_y53(int prec, int d, KernelEntry* out) {
  if (d == 5) return pick_precision_yb<WMuNu, 5, 53>(prec, out);
  return false;
}

}  // namespace gv
