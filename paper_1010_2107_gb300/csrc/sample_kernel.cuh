// sample_kernel.cuh -- steps 2-4 of Sec. 2.1 fused in one persistent kernel:
// Philox words in registers -> integer-exact grid bins -> x = g(y), J ->
// integrand -> w = f J -> privatised shared-memory bin histograms, per-thread
// totals and (stratified mode) per-hypercube sums.  Nothing per point is
// written to global memory; each CTA writes one row of partial sums.
//
// Template parameters: T (double or float: map and integrand precision),
// DM (compile-time bound on ndim), F (integrand), ACC (0: FP64 sums,
// 1: FP32 point values into FP64 sums, 2: compensated FP32 sums with FP64
// flushes).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "integrands.cuh"
#include "kernels.h"

namespace gv {

template <int ACC> struct AccTraits;
template <> struct AccTraits<0> { using H = double; };   // histogram cell type
template <> struct AccTraits<1> { using H = double; };
template <> struct AccTraits<2> { using H = float; };

// Per-thread running sums in the accumulation precision.
template <int ACC> struct Run {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ void add(float v) { s += (double)v; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void shfl_merge(int off, int width) {
    s += __shfl_xor_sync(0xffffffffu, s, off, width);
  }
  __device__ __forceinline__ void reset() { s = 0.0; }
};
template <> struct Run<2> {
  fpair p{0.f, 0.f};
  __device__ __forceinline__ void add(float v) { comp_add(p, v); }
  __device__ __forceinline__ double value() const { return comp_value(p); }
  __device__ __forceinline__ void shfl_merge(int off, int width) {
    fpair q;
    q.hi = __shfl_xor_sync(0xffffffffu, p.hi, off, width);
    q.lo = __shfl_xor_sync(0xffffffffu, p.lo, off, width);
    comp_merge(p, q);
  }
  __device__ __forceinline__ void reset() { p.hi = p.lo = 0.f; }
};

// Point generation for one sample: bins kb[a], point x[a] and the Jacobian.
// `cd` holds the hypercube digits c_a (zero without stratification).
template <typename T, int DM>
__device__ __forceinline__ T make_point(const SampleArgs& A, uint32_t it, uint32_t s,
                                        const int (&cd)[DM],
                                        const typename Vec2<T>::type* tab,
                                        T (&x)[DM], int (&kb)[DM], uint32_t* words_out) {
  const int d = A.d, N = A.N;
  const T Nf = T(N);
  T J = T(1);
  uint4 w4 = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int a = 0; a < DM; ++a) {
    if (a < d) {
      uint64_t m;
      int b;
      if (A.ybits == 24) {
        if ((a & 3) == 0) w4 = philox4x32_10(make_uint4(s, (uint32_t)(a >> 2), it, A.instance), A.key0, A.key1);
        const uint32_t u = pick(w4, a & 3);
        if (words_out) words_out[a] = u;
        m = u >> 8;
        b = 24;
      } else {
        if (((2 * a) & 3) == 0)
          w4 = philox4x32_10(make_uint4(s, (uint32_t)((2 * a) >> 2), it, A.instance), A.key0, A.key1);
        const uint32_t uh = pick(w4, (2 * a) & 3), ul = pick(w4, (2 * a + 1) & 3);
        if (words_out) {
          words_out[2 * a] = uh;
          words_out[2 * a + 1] = ul;
        }
        m = ((uint64_t)(uh >> 5) << 26) | (uint64_t)(ul >> 6);
        b = 53;
      }
      int k;
      T fr;
      if (!A.strat) {
        if (b == 24) {
          const uint32_t t = (uint32_t)m * (uint32_t)N;  // < 2^32 for N <= 256
          k = (int)(t >> 24);
          fr = T(t & 0xFFFFFFu) * T(1.0 / 16777216.0);
        } else {
          const uint64_t t = m * (uint64_t)N;
          k = (int)(t >> 53);
          fr = T(t & ((1ull << 53) - 1)) * T(1.0 / 9007199254740992.0);
        }
      } else {
        const uint64_t Y = ((uint64_t)cd[a] << b) | m;
        const uint64_t t = Y * (uint64_t)N;
        const uint32_t top = (uint32_t)(t >> b);  // floor(g y N) < g N
        if (A.g_pow2) {
          k = (int)(top >> A.g_log2);
          const uint64_t r = t & ((1ull << (b + A.g_log2)) - 1);
          fr = T(r) * T(1.0 / (double)(1ull << (b + A.g_log2)) );
        } else {
          k = (int)(top / (uint32_t)A.g);
          const uint64_t r = t - ((uint64_t)k * (uint64_t)A.g << b);
          fr = T(r) / T((double)A.g * (double)(1ull << b));
        }
      }
      const typename Vec2<T>::type e = tab[a * N + k];
      x[a] = vfma(fr, e.y, e.x);
      J *= Nf * e.y;
      kb[a] = k;
    }
  }
  return J;
}

template <typename T, int DM, template <typename, int> class F, int ACC>
__global__ void __launch_bounds__(256) k_sample(const SampleArgs A) {
  using H = typename AccTraits<ACC>::H;
  using T2 = typename Vec2<T>::type;
  if (A.st->done) return;  // the ACC test stopped this call (device-side)
  const uint32_t it = A.it_override >= 0 ? (uint32_t)A.it_override : A.st->it;
  const int d = A.d, N = A.N, dN = d * N;

  extern __shared__ __align__(16) unsigned char smem[];
  T2* tab = reinterpret_cast<T2*>(smem);
  T* P = reinterpret_cast<T*>(tab + dN);
  double* hd = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(P + kNumDerived) + 15) & ~uintptr_t(15));  // FP64 histogram [2][d][N]
  H* hs = reinterpret_cast<H*>(ACC == 2 ? (void*)(hd + 2 * dN) : (void*)hd);  // histogram atomics target

  const int tid = threadIdx.x;
  // Coalesced, vectorised grid-table load (one 8- or 16-byte cell per bin).
  const T2* gtab = reinterpret_cast<const T2*>(A.tab);
  for (int i = tid; i < dN; i += blockDim.x) tab[i] = gtab[i];
  for (int i = tid; i < kNumDerived; i += blockDim.x) P[i] = (T)A.dparams[i];
  for (int i = tid; i < 2 * dN; i += blockDim.x) {
    hd[i] = 0.0;
    if (ACC == 2) hs[i] = H(0);
  }
  __syncthreads();

  Run<ACC> sw, sw2;      // point totals
  double sI = 0.0, sV = 0.0;  // stratified: sum of cube means, cube-mean variances
  int nonfinite = 0;
  int cd[DM];
#pragma unroll
  for (int a = 0; a < DM; ++a) cd[a] = 0;

  auto accumulate_bins = [&](const int (&kb)[DM], H w) {
    const H w2 = w * w;
#pragma unroll
    for (int a = 0; a < DM; ++a)
      if (a < d) {
        atomicAdd(&hs[a * N + kb[a]], (H)w);
        atomicAdd(&hs[dN + a * N + kb[a]], (H)w2);
      }
  };
  auto flush = [&]() {  // compensated mode: FP32 histogram -> FP64 histogram
    __syncthreads();
    for (int i = tid; i < 2 * dN; i += blockDim.x) {
      hd[i] += (double)hs[i];
      hs[i] = H(0);
    }
    __syncthreads();
  };
  // w = f J in the kernel precision, widened to the histogram type H
  // (squares are then formed in H: FP64 unless ACC == 2).
  auto eval_point = [&](uint32_t s, int (&kb)[DM]) -> H {
    T x[DM];
    const T J = make_point<T, DM>(A, it, s, cd, tab, x, kb, nullptr);
    const T f = F<T, DM>::eval(x, d, P);
    T w = f * J;
    if (!vfinite(w)) {
      ++nonfinite;
      w = T(0);
    }
    return (H)w;
  };

  if (!A.strat) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x;
    const uint64_t rounds = first < A.ncall ? (A.ncall - first + stride - 1) / stride : 0;
    for (uint64_t r = 0; r < rounds; ++r) {
      const uint64_t s = first + tid + r * stride;
      if (s < A.ncall) {
        int kb[DM];
        const H w = eval_point((uint32_t)s, kb);
        sw.add(w);
        sw2.add(w * w);
        accumulate_bins(kb, w);
      }
      if (ACC == 2 && ((r + 1) % (uint64_t)A.flush_rounds == 0)) flush();
    }
  } else {
    // Groups of L lanes share a hypercube; lane j of a group takes the
    // cube's points j, j + L, ...; the group then reduces its sums with a
    // fixed xor-butterfly (deterministic).
    const int L = A.lanes;
    const int lane = tid & 31;
    const int gl = lane & (L - 1);
    const uint64_t groups_per_cta = blockDim.x / L;
    const uint64_t gstride = (uint64_t)gridDim.x * groups_per_cta;
    const uint64_t gfirst = (uint64_t)blockIdx.x * groups_per_cta;
    const uint64_t rounds = gfirst < A.ncubes ? (A.ncubes - gfirst + gstride - 1) / gstride : 0;
    for (uint64_t r = 0; r < rounds; ++r) {
      const uint64_t c = gfirst + tid / L + r * gstride;
      const bool live = c < A.ncubes;  // uniform within a group
      Run<ACC> c1, c2;
      if (live) {
        uint64_t rest = c;
#pragma unroll
        for (int a = 0; a < DM; ++a)
          if (a < d) {
            if (A.g_pow2) {
              cd[a] = (int)(rest & (uint64_t)(A.g - 1));
              rest >>= A.g_log2;
            } else {
              cd[a] = (int)(rest % (uint64_t)A.g);
              rest /= (uint64_t)A.g;
            }
          }
        const uint64_t s0 = c * A.nc;
        for (uint64_t j = gl; j < A.nc; j += L) {
          int kb[DM];
          const H w = eval_point((uint32_t)(s0 + j), kb);
          c1.add(w);
          c2.add(w * w);
          accumulate_bins(kb, w);
        }
      }
      for (int off = L >> 1; off > 0; off >>= 1) {
        c1.shfl_merge(off, L);
        c2.shfl_merge(off, L);
      }
      if (live && gl == 0) {
        const double C1 = c1.value(), C2 = c2.value();
        const double nc = (double)A.nc;
        const double m = C1 / nc;
        double v = (C2 / nc - m * m) / (nc - 1.0);
        if (v < 0.0) v = 0.0;
        sI += m;
        sV += v;
        sw.add(C1);
        sw2.add(C2);
        if (A.cubes) {
          A.cubes[2 * c] = C1;
          A.cubes[2 * c + 1] = C2;
        }
      }
      if (ACC == 2 && ((r + 1) % (uint64_t)A.flush_rounds == 0)) flush();
    }
  }
  if (ACC == 2) flush();
  __syncthreads();

  // Partial row of this CTA: histograms, then totals (fixed-order reduction).
  const int np = A.nparts, row = blockIdx.x;
  for (int i = tid; i < 2 * dN; i += blockDim.x) A.part_bins[(size_t)i * np + row] = hd[i];

  double t[5] = {sw.value(), sw2.value(), sI, sV, (double)nonfinite};
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t[q] += __shfl_xor_sync(0xffffffffu, t[q], off);
  __shared__ double wsum[32][5];
  const int warp = tid >> 5, nw = blockDim.x >> 5;
  if ((tid & 31) == 0)
#pragma unroll
    for (int q = 0; q < 5; ++q) wsum[warp][q] = t[q];
  __syncthreads();
  if (tid < 5) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += wsum[w][tid];
    A.part_tot[(size_t)tid * np + row] = acc;
  }
}

// Shared memory of k_sample for a given shape.
template <typename T, int ACC>
inline size_t sample_smem_bytes(int d, int N) {
  size_t b = (size_t)d * N * sizeof(typename Vec2<T>::type) + kNumDerived * sizeof(T);
  b = (b + 15) & ~size_t(15);
  b += 2 * (size_t)d * N * sizeof(double);
  if (ACC == 2) b += 2 * (size_t)d * N * sizeof(float);
  return b + 16;
}

}  // namespace gv

namespace gv {

// Steps 2-3 for a list of sample indices (parity checks and debugging):
// the Philox words, bins, point, Jacobian and integrand value of each.
template <typename T, int DM, template <typename, int> class F>
__global__ void __launch_bounds__(256) k_dump(const DumpArgs D) {
  __shared__ T P[kNumDerived];
  for (int i = threadIdx.x; i < kNumDerived; i += blockDim.x) P[i] = (T)D.S.dparams[i];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D.n) return;
  const SampleArgs& A = D.S;
  const uint32_t it = A.it_override >= 0 ? (uint32_t)A.it_override : A.st->it;
  const uint64_t s = D.s[i];
  int cd[DM];
  uint64_t rest = A.strat ? s / A.nc : 0;
#pragma unroll
  for (int a = 0; a < DM; ++a) {
    cd[a] = 0;
    if (a < A.d && A.strat) {
      cd[a] = (int)(rest % (uint64_t)A.g);
      rest /= (uint64_t)A.g;
    }
  }
  T x[DM];
  int kb[DM];
  uint32_t wl[2 * DM];
  const T J = make_point<T, DM>(A, it, (uint32_t)s, cd,
                                reinterpret_cast<const typename Vec2<T>::type*>(A.tab), x, kb, wl);
  const T f = F<T, DM>::eval(x, A.d, P);
  const int W = A.ybits == 24 ? A.d : 2 * A.d;
  if (D.words)
    for (int j = 0; j < W; ++j) D.words[i * W + j] = wl[j];
#pragma unroll
  for (int a = 0; a < DM; ++a)
    if (a < A.d) {
      if (D.bins) D.bins[i * A.d + a] = kb[a];
      if (D.x) D.x[i * A.d + a] = (double)x[a];
    }
  if (D.jac) D.jac[i] = (double)J;
  if (D.f) D.f[i] = (double)f;
}

template <typename T, int DM, template <typename, int> class F, int ACC>
inline KernelEntry make_entry() {
  KernelEntry e;
  e.sample = (const void*)&k_sample<T, DM, F, ACC>;
  e.dump = (const void*)&k_dump<T, DM, F>;
  e.smem = &sample_smem_bytes<T, ACC>;
  e.dm = DM;
  return e;
}

template <template <typename, int> class F, int DM>
inline bool pick_precision(int prec, KernelEntry* out) {
  switch (prec) {
    case VG_FP64: *out = make_entry<double, DM, F, 0>(); return true;
    case VG_FP32_ACC64: *out = make_entry<float, DM, F, 1>(); return true;
    case VG_FP32_ACCCOMP: *out = make_entry<float, DM, F, 2>(); return true;
    default: return false;
  }
}

// Smallest instantiated bound from {4, 8, 16, 32} that covers d.
template <template <typename, int> class F>
inline bool pick_pow2_bound(int prec, int d, KernelEntry* out) {
  if (d <= 4) return pick_precision<F, 4>(prec, out);
  if (d <= 8) return pick_precision<F, 8>(prec, out);
  if (d <= 16) return pick_precision<F, 16>(prec, out);
  if (d <= 32) return pick_precision<F, 32>(prec, out);
  return false;
}

}  // namespace gv
