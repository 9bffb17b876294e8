// common.cuh -- device-side building blocks of the sm_103a VEGAS / BASES path:
// Philox4x32-10 in registers, compensated FP32 sums, precision-generic math,
// and the argument blocks of the kernels.
#pragma once

#ifdef __CUDACC_RTC__
// Run-time compilation (user integrands, see rtc.cu): no host headers, so
// the fixed-width types are spelled out (LP64, as on the host side).
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long int64_t;
typedef unsigned long uint64_t;
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "../../include/gvegas.h"

namespace gv {

constexpr int kMaxDim = GVEGAS_MAXDIM;
constexpr int kMaxBins = GVEGAS_MAXBINS;
constexpr int kMaxHist = GVEGAS_MAXHIST;
constexpr int kNumDerived = 3 * kMaxDim + 24;  // derived integrand constants
constexpr int kTotCols = 8;                     // per-CTA totals columns

// Columns of the per-CTA totals block.
enum { TOT_SW = 0, TOT_SW2 = 1, TOT_SI = 2, TOT_SV = 3, TOT_NONFINITE = 4 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): the counter-based
// generator that replaces the per-thread xorshift state of Appendix A.
// Stateless: any thread can produce the words of any sample.
// ---------------------------------------------------------------------------
// The 64-bit product a b as (lo, hi) through one widening multiply (the
// batched kernels' bin and fraction).  The Philox rounds keep a low and a
// high multiply, which measured faster there (dgauss8 passes 2-3 %).
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t& lo, uint32_t& hi) {
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Round keys of Philox4x32-10 for key (k0, k1): ks[2 r], ks[2 r + 1] are
// the two key words of round r (Weyl increments 0x9E3779B9, 0xBB67AE85).
// Kernels receive them precomputed in their arguments, so every round reads
// its key from the constant bank instead of adding it on the fly.
constexpr int kPhiloxKeyWords = 20;
__host__ __device__ inline void philox_key_schedule(uint32_t k0, uint32_t k1, uint32_t* ks) {
  for (int r = 0; r < 10; ++r) {
    ks[2 * r] = k0;
    ks[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&ks)[kPhiloxKeyWords]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ ks[2 * r], lo1, hi0 ^ c.w ^ ks[2 * r + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t pick(const uint4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// Error-free transformation (Knuth TwoSum) and compensated pairs.
// ---------------------------------------------------------------------------
struct fpair {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void comp_add(fpair& p, float v) {
  float s, e;
  two_sum(p.hi, v, s, e);
  p.hi = s;
  p.lo = __fadd_rn(p.lo, e);
}

__device__ __forceinline__ void comp_merge(fpair& p, const fpair& q) {
  float s, e;
  two_sum(p.hi, q.hi, s, e);
  p.hi = s;
  p.lo = __fadd_rn(__fadd_rn(p.lo, q.lo), e);
}

__device__ __forceinline__ double comp_value(const fpair& p) {
  return (double)p.hi + (double)p.lo;
}

// ---------------------------------------------------------------------------
// Precision-generic math.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double vexp(double x) { return exp(x); }
__device__ __forceinline__ float vexp(float x) { return expf(x); }
__device__ __forceinline__ double vlog(double x) { return log(x); }
__device__ __forceinline__ float vlog(float x) { return logf(x); }
__device__ __forceinline__ double vsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float vsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double vatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float vatan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double vcos(double x) { return cos(x); }
__device__ __forceinline__ float vcos(float x) { return cosf(x); }
__device__ __forceinline__ double vsin(double x) { return sin(x); }
__device__ __forceinline__ float vsin(float x) { return sinf(x); }
__device__ __forceinline__ void vsincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void vsincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ double vpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float vpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double vcopysign(double x, double y) { return copysign(x, y); }
__device__ __forceinline__ float vcopysign(float x, float y) { return copysignf(x, y); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ bool vfinite(double x) { return isfinite(x); }
__device__ __forceinline__ bool vfinite(float x) { return isfinite(x); }

// Quick FP32 forms for the FP32 integrands: the special-function unit's
// approximations (__logf, __expf, __sincosf, __fdividef, sqrt.approx),
// a few parts in 2^22 on the ranges used; arguments of the trigonometric
// forms are kept in [-pi, pi] by their callers.  The FP64 overloads are the
// correctly rounded library functions, so FP64 kernels are unchanged.
__device__ __forceinline__ float qlog(float x) { return __logf(x); }
__device__ __forceinline__ double qlog(double x) { return log(x); }
// ln x with a small relative error also near x = 1, where __logf's
// absolute error would dominate a small result: 2 atanh(s),
// s = (x - 1)/(x + 1), by its odd series through s^9 on [0.75, 1.25]
// (|s| <= 1/7, truncation below 1e-8 relative), __logf elsewhere.
__device__ __forceinline__ float qlog_rel(float x) {
  const float s = __fdividef(x - 1.0f, x + 1.0f), s2 = s * s;
  const float series =
      2.0f * s * fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 1.0f / 9.0f, 1.0f / 7.0f), 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
  return (x > 0.75f && x < 1.25f) ? series : __logf(x);
}
__device__ __forceinline__ double qlog_rel(double x) { return log(x); }
__device__ __forceinline__ float qexp(float x) { return __expf(x); }
__device__ __forceinline__ double qexp(double x) { return exp(x); }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qsqrt(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float qsin(float x) { return __sinf(x); }
__device__ __forceinline__ double qsin(double x) { return sin(x); }
__device__ __forceinline__ float qcos(float x) { return __cosf(x); }
__device__ __forceinline__ double qcos(double x) { return cos(x); }
// sin and cos of 2 pi u for u in [0, 1): evaluated at 2 pi (u - 1/2) in
// [-pi, pi) and negated
__device__ __forceinline__ void qsincos2pi(float u, float* s, float* c) {
  float sn, cs;
  __sincosf(6.28318530717958648f * (u - 0.5f), &sn, &cs);
  *s = -sn;
  *c = -cs;
}
__device__ __forceinline__ void qsincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }

// A compile-time flag as a type (selects a code path of a generic lambda).
template <bool V> struct BoolTag {
  static constexpr bool value = V;
};

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// ---------------------------------------------------------------------------
// Device-resident iteration state (one per context).
// ---------------------------------------------------------------------------
struct GState {
  uint32_t it;          // Philox iteration counter: iterations run so far
  int done;             // set when the ACC test stops the current call
  int live;             // latched per pass by the sampling kernel: 1 if it ran
  int nhist;            // iterations in the combination window
  int stopped;
  long long nonfinite;  // non-finite weights in the window
  long long samples;    // points in the window
  double acc;           // relative accuracy target of the current call
  double I, sigma, chi2;
  double last_I, last_var, last_sw, last_sw2;
  long long last_nonfinite;
  // snapshot of the first BASES phase
  double ph1_I, ph1_sigma, ph1_chi2;
  int ph1_iters, ph1_stopped;
  long long ph1_nonfinite, ph1_samples;
  unsigned arrive[kMaxDim + 1];  // block arrivals per group of k_finish (reset by the last)
  double hist[kMaxHist][2];
};

// Threads per block of k_finish.
constexpr int kFinishThreads = 256;

// Device-side control operations captured into the iteration graphs.
enum { CTL_RESET_WINDOW = 1, CTL_SET_ACC = 2, CTL_SNAPSHOT = 4, CTL_SET_ITER = 8 };

// Arguments of the sampling kernel (steps 2-4).
struct SampleArgs {
  int d, N, g, ybits;
  int lanes;               // lanes per hypercube (stratified mode), power of two <= 32
  int cap;                 // bucket capacity per (axis, bin) and tile
  int ppt;                 // points per thread per tile (>= 1)
  int strat;
  int nobins;              // 1: no per-bin histogram (a pass whose grid is not refined)
  uint32_t key0, key1, instance;
  uint32_t ks[kPhiloxKeyWords];  // Philox round keys of (key0, key1)
  int it_override;         // >= 0: use this iteration index
  uint64_t ncall;
  uint32_t nc;             // points per hypercube
  uint32_t ncubes;         // number of hypercubes
  uint32_t cube_mul;       // odd multiplier permuting the cube order (power-of-two
                           // cube counts; 1 otherwise)
  int g_pow2, g_log2;
  int t32;                 // 24-bit bins fit 32-bit integers (g N <= 256)
  float inv_gb_f;          // 1 / (g 2^ybits)
  double inv_gb_d;
  double inv_nc, inv_nc1;  // 1 / nc, 1 / (nc - 1)
  int nparts;              // number of CTAs == partial rows
  const void* tab;         // [d][N] (e_k, Delta_k) in the kernel precision
  const double* dparams;   // derived integrand constants
  GState* st;              // the sampling kernel latches st->live
  void* part_bins;         // [2 d N][nparts]: double, or float (hi, lo) pairs (FP32 forms)
  double* part_tot;        // [kTotCols][nparts]
  void* cubes;             // [ncubes]: double (sum w, sum w^2), or float (hi, lo, hi, lo)
  double* cube_max;        // [ncubes] running max(0, largest w) (integration phase), or null
};

// Arguments of the reduction and finalisation kernels (steps 4-6).
struct FinArgs {
  int d, N, nparts, strat, refine, record;
  int nobins;              // the pass kept no per-bin histogram: totals only, no refinement
  int pair32;              // part_bins hold float (hi, lo) pairs
  uint64_t ncall;
  uint64_t ncubes;
  const double* scale;     // integrand output scale (RAMBO units), in device memory so
                           // that captured graphs follow vegas_set_params
  double alpha;
  const void* part_bins;
  const double* part_tot;
  double* bins;            // [2][d][N] reduced, scaled
  double* tot;             // [kTotCols] reduced, scaled
  double* edges;           // [d][N+1]
  double2* tab64;          // [d][N]
  float2* tab32;           // [d][N]
  GState* st;
};

}  // namespace gv
