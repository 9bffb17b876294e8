// inst_genz_corner_peak.cu -- sampling kernels for the Genz corner peak family.
#include "sample_kernel.cuh"

namespace gv {

bool entries_genz_corner_peak(int prec, int d, KernelEntry* out) {
  return pick_pow2_bound<GenzCornerPeak>(prec, d, out);
}

}  // namespace gv
