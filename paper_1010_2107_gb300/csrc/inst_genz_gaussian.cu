// inst_genz_gaussian.cu -- sampling kernels for the Genz gaussian family.
#include "sample_kernel.cuh"

namespace gv {

bool entries_genz_gaussian(int prec, int d, KernelEntry* out) {
  return pick_pow2_bound<GenzGaussian>(prec, d, out);
}

}  // namespace gv
