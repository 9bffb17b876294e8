// inst_genz_product_peak.cu -- sampling kernels for the Genz product peak family.
#include "sample_kernel.cuh"

namespace gv {

bool entries_genz_product_peak(int prec, int d, KernelEntry* out) {
  return pick_pow2_bound<GenzProductPeak>(prec, d, out);
}

}  // namespace gv
