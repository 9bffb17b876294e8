// inst_genz_oscillatory.cu -- sampling kernels for the Genz oscillatory family.
#include "sample_kernel.cuh"

namespace gv {

bool entries_genz_oscillatory(int prec, int d, KernelEntry* out) {
  return pick_pow2_bound<GenzOscillatory>(prec, d, out);
}

}  // namespace gv
