// kernels.h -- host-side view of the device kernels: per-integrand kernel
// registry (filled by the inst_*.cu translation units) and the launchers of
// the reduction / finalisation kernels.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stddef.h>

#include <string>
#endif

#include "common.cuh"

namespace gv {

#ifndef __CUDACC_RTC__  // host side only (run-time compiled kernels see the argument blocks)

// One compiled sampling kernel and its companions for a (kind, precision, DM).
struct KernelEntry {
  const void* sample;                 // k_sample<T, DM, F, ACC, YB, false> (any d <= DM)
  const void* sample_spec;            // k_sample<..., true>: d == DM, 24-bit, power-of-two
                                      // divisions with g N <= 256; may be null
  const void* dump;                   // k_dump<T, DM, F>
  size_t (*smem)(int d, int N, int cap);  // dynamic shared memory of `sample`
                                          // with bucket capacity cap
  size_t (*smem_nobins)(int d, int N);    // ... of a pass without the histogram
  int dm;                             // compile-time dimension bound
  int spec_ppt_min;                   // `sample_spec` evaluates this many points per
                                      // thread at a time: tiles are multiples of it
  const void* grad;                   // k_grad<T, DM, F, YB> or null
  const void* grad_spec;              // k_grad<T, DM, F, 24, true> (specialised shape) or null
  int grad_nt;                        // its gradient columns (F<T, DM>::NT)
  size_t (*grad_smem)(int d, int N);
  const void* spring;                 // k_spring<T, DM, F, YB, false>
  const void* spring_spec;            // k_spring<T, DM, F, 24, true> or null
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
bool entries_genz_continuous_y24(int prec, int d, KernelEntry* out);
bool entries_genz_continuous_y53(int prec, int d, KernelEntry* out);
bool entries_genz_discontinuous_y24(int prec, int d, KernelEntry* out);
bool entries_genz_discontinuous_y53(int prec, int d, KernelEntry* out);
bool entries_wmunu_y24(int prec, int d, KernelEntry* out);
bool entries_wmunu_y53(int prec, int d, KernelEntry* out);
bool entries_rambo_y24(int prec, int d, KernelEntry* out);
bool entries_rambo_y53(int prec, int d, KernelEntry* out);

// Number of parameters the integrand `kind` takes in `d` dimensions (-1 for
// an unknown kind), and the constants its device code reads (`dv`, length
// kNumDerived) plus the output scale; false with a reason when invalid.
int expected_nparams(int kind, int d);
bool derive_params(int kind, int d, const double* p, double* dv, double* scale, std::string* why);

// Kernels of a run-time compiled integrand (rtc.cu) with exact dimension
// d: the specialised sampling and SPRING kernels when `spec` (the shape
// allows them), else the general ones, plus the dump kernel.  Returns
// VEGAS_OK, VEGAS_EINVAL (the source does not compile: *why holds the
// compiler's log) or VEGAS_ECUDA (no run-time compiler, or the module does
// not load).
int rtc_user_entry(const char* source, int prec, int ybits, int d, bool spec, KernelEntry* out, std::string* why);
// The same compile without loading (no device needed); the result is cached.
int rtc_user_compile(const char* source, int prec, int ybits, int d, bool spec, std::string* why);

// Histogram tile of a sampling kernel: ppt points per thread between two
// gathers, bucket capacity cap per (axis, bin), and the CTAs per SM that
// leaves resident.
struct TileShape {
  int ppt, cap, occ;
};

// Choice of the tile for `threads` threads over N bins.  A tile of
// threads x ppt points fills a cell with m = threads ppt / N points on
// average; the capacity runs from m + 4 sqrt(m) + 2 (a Poisson tail: claims
// past it are rare and spill to float atomics) down to m + 2 sqrt(m) + 1,
// in steps of 4, until the CTAs per SM reach occ_cap (the bound without
// shared memory).  Larger tiles amortise the gather and its barriers, so
// the largest ppt in {4, 2, 1} that keeps at least 16 warps per SM (or the
// most the kernel can have) wins; ppt_req > 0 forces the tile and then halves
// the capacity until it fits.  A kernel that evaluates ppt_min points per
// thread at a time (1 or 2) gets tiles that are multiples of it.
// occ_of(cap, ppt) returns the CTAs per SM (0: does not fit).  With
// `small_cap` the smallest capacity of the range that reaches the best
// occupancy is taken (less to gather, more claims spilling past the
// buckets), else the largest.  `dense` lowers the range's floor to
// m + sqrt(m) + 1 (a few percent of the claims spill), for kernels whose
// shared memory is what holds the CTAs per SM down.
template <class OccOf>
inline TileShape choose_tile(int threads, int N, int ppt_req, int ppt_min, int occ_cap, OccOf occ_of,
                             bool small_cap = false, bool dense = false) {
  auto ceil4 = [](double v) { return ((int)v + 1 + 3) & ~3; };
  TileShape best{0, 0, 0};
  const int wanted = occ_cap * threads / 32 < 16 ? occ_cap * threads / 32 : 16;
  const int cands[3] = {4, 2, 1};
  if (ppt_req > 0) ppt_req = (ppt_req + ppt_min - 1) / ppt_min * ppt_min;
  for (int i = 0; i < 3; ++i) {
    if (ppt_req <= 0 && cands[i] < ppt_min) continue;
    const int ppt = ppt_req > 0 ? ppt_req : cands[i];
    const double m = (double)threads * ppt / N;
    int hi = ceil4(m + 4.0 * __builtin_sqrt(m) + 2.0), lo = ceil4(m + (dense ? 1.0 : 2.0) * __builtin_sqrt(m) + 1.0);
    hi = hi > 64 ? 64 : hi;
    lo = lo > hi ? hi : lo;
    TileShape t{ppt, hi, 0};
    for (int cap = hi; cap >= lo; cap -= 4) {
      const int o = occ_of(cap, ppt);
      if (o > t.occ || (small_cap && o == t.occ && o > 0)) t = TileShape{ppt, cap, o};
      if (o >= occ_cap && !small_cap) break;
    }
    if (ppt_req > 0) {  // forced tile: shrink the capacity until it fits
      for (int cap = lo; t.occ < 1 && cap > 4;) {
        cap = (cap / 2) & ~3;  // capacities stay multiples of 4 (vector gather)
        cap = cap < 4 ? 4 : cap;
        const int o = occ_of(cap, ppt);
        if (o > 0) t = TileShape{ppt, cap, o};
      }
      return t;
    }
    if (t.occ * threads / 32 >= wanted) return t;
    if (t.occ > best.occ) best = t;
  }
  if (best.occ > 0) return best;
  // nothing fits at the smallest tile's capacities: halve below them
  for (int cap = 8; cap >= 4; cap /= 2) {
    const int o = occ_of(cap, ppt_min);
    if (o > 0) return TileShape{ppt_min, cap, o};
  }
  return TileShape{ppt_min, 4, 0};
}

// Lanes per hypercube (stratified sampling): the smallest power of two L
// <= min(32, nc) that gives at least four rounds of `ctas` CTAs of
// `threads` threads over the G hypercubes (load balance).  Larger L would
// shorten the last round, but it also packs more points of one hypercube
// into a histogram tile, which crowds its (axis, bin) buckets.
inline int choose_lanes(uint64_t G, uint64_t nc, int threads, int64_t ctas) {
  int L = 1;
  while (L < 32 && (uint64_t)(2 * L) <= nc && G * (uint64_t)L < 4 * (uint64_t)ctas * (uint64_t)threads) L *= 2;
  return L;
}

#endif  // __CUDACC_RTC__

// Arguments of the SPRING trial kernel: trials trial0 .. trial0 + n - 1 in
// chunks of `chunk` trials; the kept points of chunk k go, in trial order, to
// stage_x[(k chunk + i) d + a] and stage_t[k chunk + i], their number to
// counts[k]; counters: [0] bound overflows, [1] non-positive weights.
struct SpringArgs {
  SampleArgs S;
  const uint64_t* prefix;   // [G + 1] exclusive prefix sums of the integer cube weights
  const double* mt;         // [G] cube bounds q_c / scale (FP64, formed by the table kernel)
  const float* mt32;        // [G] the same rounded to FP32 (the FP32 kernels' keep decision)
  const uint32_t* guide;    // [2^gk + 1] guide table of the cube search (Chen and Asau):
                            // guide[j] = the last cube c with prefix[c] <= floor(j Q / 2^gk)
  uint32_t gk;              // log2 of the number of guide intervals
  const double* meta;       // {Q, scale} written by the table kernel
  double out_scale;         // integrand output scale: weights in the integrand's units
  uint32_t trial0, n, chunk, nchunks;
  double* stage_x;
  uint64_t* stage_t;
  uint32_t* counts;
  unsigned long long* counters;
};

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

#ifndef __CUDACC_RTC__
extern "C" {
cudaError_t gv_prepare_aux_kernels(void);
// Raise (never lower) a kernel's dynamic shared-memory limit to `bytes`.
cudaError_t gv_raise_smem_limit(const void* fn, size_t bytes);
// Every device (gv_dev_malloc) and pinned host (gv_host_malloc) allocation
// of the library: cudaMalloc / cudaMallocHost behind a counter and the
// failure injection of vegas_fail_alloc_after.
cudaError_t gv_dev_malloc(void** p, size_t bytes);
cudaError_t gv_host_malloc(void** p, size_t bytes);
// The batched dimension kernels k_batch_dim<d, pif> (batch_dims_lo.cu:
// d = 1..8, batch_dims_hi.cu: d = 9..16); null outside the range.
const void* gv_batch_dim_kernel_lo(int d, int pif);
const void* gv_batch_dim_kernel_hi(int d, int pif);
cudaError_t gv_launch_finish(const gv::FinArgs* F, cudaStream_t s);
cudaError_t gv_launch_colsum(const double* part, int ncols, int nrows, double* out, cudaStream_t s);
cudaError_t gv_launch_control(gv::GState* st, int ops, double acc, uint32_t it, cudaStream_t s);
cudaError_t gv_launch_uniform_grid(double* edges, int d, int N, cudaStream_t s);
cudaError_t gv_launch_tables(const double* edges, int d, int N, double2* t64, float2* t32,
                             cudaStream_t s);
}
#endif  // __CUDACC_RTC__

#ifndef __CUDACC_RTC__
template <class T>
inline cudaError_t gv_malloc(T** p, size_t bytes) {
  return gv_dev_malloc(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t gv_malloc_host(T** p, size_t bytes) {
  return gv_host_malloc(reinterpret_cast<void**>(p), bytes);
}
#endif
