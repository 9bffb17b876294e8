// inst_dgauss.cu -- sampling kernels for the two-peak Gaussian.
#include "sample_kernel.cuh"

namespace gv {

bool entries_dgauss(int prec, int d, KernelEntry* out) {
  return pick_pow2_bound<DoubleGaussian>(prec, d, out);
}

}  // namespace gv
