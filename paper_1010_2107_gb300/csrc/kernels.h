// kernels.h -- host-side view of the device kernels: per-integrand kernel
// registry (filled by the inst_*.cu translation units) and the launchers of
// the reduction / finalisation kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "common.cuh"

namespace gv {

// One compiled sampling kernel and its companions for a (kind, precision, DM).
struct KernelEntry {
  const void* sample;                 // k_sample<T, DM, F, ACC, YB, false> (any d <= DM)
  const void* sample_spec;            // k_sample<..., true>: d == DM, 24-bit, power-of-two
                                      // divisions with g N <= 256; may be null
  const void* dump;                   // k_dump<T, DM, F>
  size_t (*smem)(int d, int N, int cap);  // dynamic shared memory of `sample`
                                          // with bucket capacity cap
  int dm;                             // compile-time dimension bound
  const void* grad;                   // k_grad<T, DM, F, YB> or null
  int grad_nt;                        // its gradient columns (F<T, DM>::NT)
  size_t (*grad_smem)(int d, int N);
};

// Per-kind registries (one per random-bit width); false when no
// instantiation covers (precision, d).
bool entries_genz_gaussian_y24(int prec, int d, KernelEntry* out);
bool entries_genz_gaussian_y53(int prec, int d, KernelEntry* out);
bool entries_genz_product_peak_y24(int prec, int d, KernelEntry* out);
bool entries_genz_product_peak_y53(int prec, int d, KernelEntry* out);
bool entries_genz_corner_peak_y24(int prec, int d, KernelEntry* out);
bool entries_genz_corner_peak_y53(int prec, int d, KernelEntry* out);
bool entries_genz_oscillatory_y24(int prec, int d, KernelEntry* out);
bool entries_genz_oscillatory_y53(int prec, int d, KernelEntry* out);
bool entries_dgauss_y24(int prec, int d, KernelEntry* out);
bool entries_dgauss_y53(int prec, int d, KernelEntry* out);
bool entries_rambo_y24(int prec, int d, KernelEntry* out);
bool entries_rambo_y53(int prec, int d, KernelEntry* out);

// Number of parameters the integrand `kind` takes in `d` dimensions (-1 for
// an unknown kind), and the constants its device code reads (`dv`, length
// kNumDerived) plus the output scale; false with a reason when invalid.
int expected_nparams(int kind, int d);
bool derive_params(int kind, int d, const double* p, double* dv, double* scale, std::string* why);

// Arguments of the per-sample dump kernel.
struct DumpArgs {
  SampleArgs S;
  const uint64_t* s;
  long long n;
  uint32_t* words;
  int32_t* bins;
  double* x;
  double* jac;
  double* f;
};

}  // namespace gv

extern "C" {
cudaError_t gv_launch_reduce(const gv::FinArgs* F, cudaStream_t s);
cudaError_t gv_launch_finalize(const gv::FinArgs* F, cudaStream_t s);
cudaError_t gv_launch_colsum(const double* part, int ncols, int nrows, double* out, cudaStream_t s);
cudaError_t gv_launch_control(gv::GState* st, int ops, double acc, cudaStream_t s);
cudaError_t gv_launch_uniform_grid(double* edges, int d, int N, cudaStream_t s);
cudaError_t gv_launch_tables(const double* edges, int d, int N, double2* t64, float2* t32,
                             cudaStream_t s);
}
