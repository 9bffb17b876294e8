// sample_kernel.cuh -- steps 2-4 of Sec. 2.1 fused in one persistent kernel:
// Philox words in registers -> integer-exact grid bins -> x = g(y), J ->
// integrand -> w = f J -> privatised shared-memory bin histograms, per-thread
// totals and (stratified mode) per-hypercube sums.  Nothing per point is
// written to global memory; each CTA writes one row of partial sums.
//
// Template parameters: T (double or float: map and integrand precision),
// DM (compile-time bound on ndim), F (integrand), ACC (0: FP64 sums,
// 1: FP32 point values into FP64 sums, 2: compensated FP32 sums), YB (24 or
// 53 random bits per axis).
#pragma once

#ifdef __CUDACC_RTC__
// run-time compilation sees no C++ library: the two traits used here
namespace std {
template <class A, class B> struct is_same { static constexpr bool value = false; };
template <class A> struct is_same<A, A> { static constexpr bool value = true; };
template <bool C, class A, class B> struct conditional { using type = A; };
template <class A, class B> struct conditional<false, A, B> { using type = B; };
}  // namespace std
#else
#include <type_traits>
#endif

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
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void shfl_merge(int off, int width) {
    s += __shfl_xor_sync(0xffffffffu, s, off, width);
  }
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
};

// FP32 in-bin fraction from the top 23 of 24 fraction bits v: the float
// 1 + (v >> 1) 2^-23 minus one, exact (two instructions, no conversion unit).
__device__ __forceinline__ float frac23(uint32_t v24) {
  return __uint_as_float(0x3F800000u | (v24 >> 1)) - 1.0f;
}

// Grid bin k and position in the bin (as a fraction) of axis a from its
// random bits m (YB bits) and hypercube digit c: g y = c + m / 2^YB,
// k = floor(y N), frac = y N - k, in integer arithmetic.  The FP32 kernels
// keep the top 23 bits of the fraction (an error below 2^-24 of a bin).
template <typename T, int YB, bool SPEC>
__device__ __forceinline__ void bin_frac(const SampleArgs& A, uint64_t m, int c, int& k, T& fr) {
  const uint32_t N = (uint32_t)A.N;
  constexpr bool F32 = std::is_same<T, float>::value;
  if (SPEC) {  // 24 bits, power-of-two divisions, g N <= 256 (checked on the host)
    const uint32_t t = (((uint32_t)c << 24) | (uint32_t)m) * N;
    const int sh = 24 + A.g_log2;
    k = (int)(t >> sh);
    const uint32_t r = t & ((1u << sh) - 1u);
    if (F32)
      fr = T(frac23(r >> A.g_log2));
    else
      fr = T((double)r * A.inv_gb_d);
    return;
  }
  if (YB == 24 && A.t32) {
    const uint32_t t = (((uint32_t)c << 24) | (uint32_t)m) * N;  // g 2^24 y N < 2^32
    uint32_t r;
    if (A.g_pow2) {
      const int sh = 24 + A.g_log2;
      k = (int)(t >> sh);
      r = t & ((1u << sh) - 1u);
      if (F32) {
        fr = T(frac23(r >> A.g_log2));
        return;
      }
    } else {
      k = (int)((t >> 24) / (uint32_t)A.g);
      r = t - (uint32_t)k * ((uint32_t)A.g << 24);
    }
    if (F32)
      fr = T((float)r * A.inv_gb_f);
    else
      fr = T((double)r * A.inv_gb_d);
    return;
  }
  const uint64_t t = (((uint64_t)c << YB) | m) * (uint64_t)N;
  uint64_t r;
  if (A.g_pow2) {
    const int sh = YB + A.g_log2;
    k = (int)(t >> sh);
    r = t & ((1ull << sh) - 1ull);
    if (F32) {
      fr = T(frac23((uint32_t)(r >> (sh - 24))));
      return;
    }
  } else {
    k = (int)((uint32_t)(t >> YB) / (uint32_t)A.g);
    r = t - (((uint64_t)k * (uint64_t)A.g) << YB);
  }
  if (F32)
    fr = T((float)r * A.inv_gb_f);
  else
    fr = T((double)r * A.inv_gb_d);
}

// Point generation for one sample: bins kb[a], point x[a] and the Jacobian.
// `cd` holds the hypercube digits c_a (zero without stratification).
template <typename T, int DM, int YB, bool SPEC = false>
__device__ __forceinline__ T make_point(const SampleArgs& A, uint32_t it, uint32_t s,
                                        const int (&cd)[DM],
                                        const typename Vec2<T>::type* tab,
                                        T (&x)[DM], int (&kb)[DM], uint32_t* words_out) {
  const int d = SPEC ? DM : A.d, N = A.N;
  const T Nf = T(N);
  T J = T(1);
  uint4 w4 = make_uint4(0, 0, 0, 0);
  constexpr bool FAST = SPEC && YB == 24 && std::is_same<T, float>::value;
  const int sh = 24 + A.g_log2;  // SPEC: y g N 2^24 < 2^32, bin k = t >> sh
#pragma unroll
  for (int a = 0; a < DM; ++a) {
    if (a < d) {
      uint64_t m;
      if (YB == 24) {
        if ((a & 3) == 0) w4 = philox4x32_10(make_uint4(s, (uint32_t)(a >> 2), it, A.instance), A.ks);
        const uint32_t u = pick(w4, a & 3);
        if (words_out) words_out[a] = u;
        if constexpr (FAST) {
          // t = ((c << 24) | (u >> 8)) N, then k = t >> sh and the top 23
          // bits of t mod 2^sh as the fraction: the same bits as bin_frac
          // and frac23, with funnel shifts doing the packing
          const uint32_t t = __funnelshift_r(u, (uint32_t)cd[a], 8) * (uint32_t)N;
          const int k = (int)(t >> sh);
          const float fr = __uint_as_float(__funnelshift_r(t << (32 - sh), 0x7Fu, 9)) - 1.0f;
          const typename Vec2<T>::type e = tab[a * N + k];
          x[a] = vfma(fr, e.y, e.x);
          J *= Nf * e.y;
          kb[a] = k;
          continue;
        }
        m = u >> 8;
      } else {
        if (((2 * a) & 3) == 0)
          w4 = philox4x32_10(make_uint4(s, (uint32_t)((2 * a) >> 2), it, A.instance), A.ks);
        const uint32_t uh = pick(w4, (2 * a) & 3), ul = pick(w4, (2 * a + 1) & 3);
        if (words_out) {
          words_out[2 * a] = uh;
          words_out[2 * a + 1] = ul;
        }
        m = ((uint64_t)(uh >> 5) << 26) | (uint64_t)(ul >> 6);
      }
      int k;
      T fr;
      bin_frac<T, YB, SPEC>(A, m, cd[a], k, fr);
      const typename Vec2<T>::type e = tab[a * N + k];
      x[a] = vfma(fr, e.y, e.x);
      J *= Nf * e.y;
      kb[a] = k;
    }
  }
  return J;
}

// Sampling kernels that keep two points per thread in flight: FP32,
// specialised shape, at most 8 dimensions.
template <typename T, int DM, bool SPEC>
constexpr bool kPairPoints = SPEC && std::is_same<T, float>::value && DM <= 8;

// Points per thread between compensated folds of the CTA histogram (ACC 2):
// the plain FP32 cells add the bucket sums of at most this many points per
// thread before they are folded into the pairs.
constexpr int kFoldPoints = 8;

// Bucketed tile histogram of one CTA (shared memory).  Shared-memory float
// atomics are compare-and-swap loops on this GPU while 32-bit integer
// atomics are native, so a point claims a slot of each of its (axis, bin)
// buckets with one integer atomicAdd and stores w there (scatter); at the end
// of a tile one thread per cell sums its bucket into the CTA's cells, w and
// w^2 (gather).  Buckets are cell-major rows of S = cap + V slots (V values
// per 16 bytes), so the gather reads and clears four slots per vector load
// and store; slots past a bucket's fill are zero (cleared after every read),
// so the reads need no masking.  A claim past the capacity stores into the
// spare slot `cap` (never read) and the point, which remembers the largest
// claim it made, then adds those values to the cells with float atomics,
// off the common path.  Layout from the base: counters [d N] (int), buckets
// [d N][S] (H), cells [2][d N] (H), and for ACC 2 compensated pairs [2][d N].
template <int ACC>
struct TileHist {
  using H = typename AccTraits<ACC>::H;
  static constexpr bool COMP = ACC == 2;
  static constexpr int V = 16 / (int)sizeof(H);  // slots per 16-byte vector
  using HV = typename std::conditional<sizeof(H) == 4, float4, double2>::type;
  // cap slots and a spare vector, padded to an odd number of 16-byte
  // vectors: the rows of consecutive cells then start in all eight vector
  // positions of the 32 banks (conflict-free vector reads in the gather)
  static __host__ __device__ int stride(int cap) {
    int s = cap + V;
    while ((s / V) % 2 == 0) s += V;
    return s;
  }
  static __host__ __device__ size_t a16(size_t b) { return (b + 15) & ~size_t(15); }
  static __host__ __device__ size_t off_bucket(int dN) { return a16((size_t)dN * sizeof(int)); }
  static __host__ __device__ size_t off_cta(int dN, int cap) {
    return a16(off_bucket(dN) + (size_t)stride(cap) * dN * sizeof(H));
  }
  static __host__ __device__ size_t off_comp(int dN, int cap) { return a16(off_cta(dN, cap) + 2 * (size_t)dN * sizeof(H)); }
  static __host__ __device__ size_t bytes(int dN, int cap) {
    return off_comp(dN, cap) + (COMP ? 2 * (size_t)dN * sizeof(fpair) : 0);
  }

  int* cnt;
  H* bucket;  // [d N][S]
  H* cta;
  fpair* cmp;
  int N, dN, cap, S, tile, fold_every;

  // dN cells in use of a layout sized for `cells` >= dN; cap: a multiple of
  // 4; ppt: points per thread per tile
  __device__ __forceinline__ void bind(unsigned char* base, int dN_, int N_, int cap_, int ppt, int cells) {
    dN = dN_;
    N = N_;
    cap = cap_;
    S = stride(cap_);
    tile = 0;
    fold_every = max(1, kFoldPoints / ppt);
    cnt = reinterpret_cast<int*>(base);
    bucket = reinterpret_cast<H*>(base + off_bucket(cells));
    cta = reinterpret_cast<H*>(base + off_cta(cells, cap));
    cmp = reinterpret_cast<fpair*>(base + off_comp(cells, cap));
  }
  // Clear the bucket slots of `cells` cells: once per launch, since every
  // gather leaves the slots it read cleared (the caller synchronises).
  __device__ __forceinline__ void zero_buckets(int tid, int nthr, int cells) {
    HV* b = reinterpret_cast<HV*>(bucket);
    const HV z{};
    for (int i = tid; i < cells * S / V; i += nthr) b[i] = z;
  }
  // Clear counters and cells (the caller synchronises before the first
  // scatter).
  __device__ __forceinline__ void zero(int tid, int nthr) {
    for (int i = tid; i < dN; i += nthr) cnt[i] = 0;
    for (int i = tid; i < 2 * dN; i += nthr) {
      cta[i] = H(0);
      if (COMP) cmp[i] = fpair{0.f, 0.f};
    }
  }
  // The claims of a group of axes are issued together, then their stores
  // (a store may alias a later claim's counter as far as the compiler
  // knows: claim-store pairs in sequence would expose every claim's
  // latency).
  template <int DM>
  __device__ __forceinline__ void scatter(const int (&kb)[DM], int d, H w) {
    constexpr int G = DM <= 20 ? DM : 8;  // axes per group (all up to 20 axes: measured best)
    int pos[DM];
    int top = 0;
#pragma unroll
    for (int a0 = 0; a0 < DM; a0 += G) {
#pragma unroll
      for (int a = a0; a < a0 + G && a < DM; ++a)
        if (a < d) pos[a] = atomicAdd(&cnt[a * N + kb[a]], 1);
#pragma unroll
      for (int a = a0; a < a0 + G && a < DM; ++a)
        if (a < d) {
          bucket[(a * N + kb[a]) * S + min(pos[a], cap)] = w;
          top = max(top, pos[a]);
        }
    }
    if (__builtin_expect(top >= cap, 0)) {
      // spare-slot claims: add to the cells directly (nothing reads them
      // before the gather's barrier)
#pragma unroll
      for (int a = 0; a < DM; ++a)
        if (a < d && pos[a] >= cap) {
          const int cell = a * N + kb[a];
          atomicAdd(&cta[cell], w);
          atomicAdd(&cta[dN + cell], w * w);
        }
    }
  }
  // End of a tile (all threads of the CTA); ACC 2 folds the FP32 cells into
  // the compensated pairs every kFoldPoints points per thread.
  __device__ __forceinline__ void gather(int tid, int nthr) {
    __syncthreads();
    const bool fold = COMP && (++tile == fold_every);
    if (fold) tile = 0;
    const HV z{};
    for (int cell = tid; cell < dN; cell += nthr) {
      const int nq = (min(cnt[cell], cap) + V - 1) / V;  // vectors holding the fill
      HV* row = reinterpret_cast<HV*>(bucket + (size_t)cell * S);
      H s1 = H(0), s2 = H(0);
      // FP32: two-lane sums with the paired FP32 instructions (one add and
      // one fused square-add per two slots)
      float2 a1 = make_float2(0.f, 0.f), a2 = make_float2(0.f, 0.f);
      // four vectors per step: the loads issue together, then the clears
      for (int q = 0; q < nq; q += 4) {
        HV v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = q + u < nq ? row[q + u] : z;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (q + u < nq) row[q + u] = z;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if constexpr (V == 4) {
            const float2 lo = make_float2(v[u].x, v[u].y), hi = make_float2(v[u].z, v[u].w);
            a1 = __fadd2_rn(a1, __fadd2_rn(lo, hi));
            a2 = __ffma2_rn(lo, lo, a2);
            a2 = __ffma2_rn(hi, hi, a2);
          } else {
            s1 += v[u].x + v[u].y;
            s2 += v[u].x * v[u].x + v[u].y * v[u].y;
          }
        }
      }
      if constexpr (V == 4) {
        s1 = a1.x + a1.y;
        s2 = a2.x + a2.y;
      }
      H c1 = cta[cell] + s1, c2 = cta[dN + cell] + s2;
      if (fold) {
        comp_add(cmp[cell], (float)c1);
        comp_add(cmp[dN + cell], (float)c2);
        c1 = c2 = H(0);
      }
      cta[cell] = c1;
      cta[dN + cell] = c2;
      cnt[cell] = 0;
    }
    __syncthreads();
  }
  // Final value of cell i in [0, 2 d N) (after a gather): a compensated pair
  // (ACC 2) or a double.
  __device__ __forceinline__ fpair pair(int i) const {
    fpair p = cmp[i];
    comp_add(p, (float)cta[i]);
    return p;
  }
  __device__ __forceinline__ double value(int i) const { return (double)cta[i]; }
};

// Shared memory layout of k_sample (byte offsets): grid table, integrand
// constants, then the tile histogram.
template <typename T, int ACC>
struct SmemLayout {
  static __host__ __device__ size_t a16(size_t b) { return (b + 15) & ~size_t(15); }
  static __host__ __device__ size_t params(int dN) { return (size_t)dN * sizeof(typename Vec2<T>::type); }
  static __host__ __device__ size_t hist(int dN) { return a16(params(dN) + kNumDerived * sizeof(T)); }
  static __host__ __device__ size_t total(int dN, int cap) { return hist(dN) + TileHist<ACC>::bytes(dN, cap); }
};

// Warp all-reduce of a compensated pair (fixed xor order).
__device__ __forceinline__ fpair warp_sum(fpair p) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fpair q;
    q.hi = __shfl_xor_sync(0xffffffffu, p.hi, off);
    q.lo = __shfl_xor_sync(0xffffffffu, p.lo, off);
    comp_merge(p, q);
  }
  return p;
}

// Threads per CTA a sampling kernel may be launched with: the specialised
// kernels up to 512 (larger tiles for many cells), the general ones 256
// (their register budget).
template <bool SPEC>
constexpr int kSampleMaxThreads = SPEC ? 512 : 256;

template <typename T, int DM, template <typename, int> class F, int ACC, int YB, bool SPEC>
__global__ void __launch_bounds__(kSampleMaxThreads<SPEC>) k_sample(const SampleArgs A) {
  using H = typename AccTraits<ACC>::H;
  using T2 = typename Vec2<T>::type;
  using L = SmemLayout<T, ACC>;
  constexpr bool COMP = ACC == 2;  // FP32 throughout, no FP64 in the loop
  // the ACC test stopped this call (device-side): no pass, and k_finish
  // then skips it too (it reads `live`, nothing else here writes it)
  const int stop = A.st->done;
  if (blockIdx.x == 0 && threadIdx.x == 0) A.st->live = !stop;
  if (stop) return;
  const uint32_t it = A.it_override >= 0 ? (uint32_t)A.it_override : A.st->it;
  // SPEC: d equals the compile-time bound DM, 24-bit words and power-of-two
  // hypercube divisions with g N <= 256: every per-axis guard folds away.
  const int d = SPEC ? DM : A.d, N = A.N, dN = d * N, cap = A.cap;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

  extern __shared__ __align__(16) unsigned char smem[];
  T2* tab = reinterpret_cast<T2*>(smem);
  T* P = reinterpret_cast<T*>(smem + L::params(dN));
  TileHist<ACC> hist;
  hist.bind(smem + L::hist(dN), dN, N, cap, A.ppt, dN);

  // Coalesced, vectorised grid-table load (one 8- or 16-byte cell per bin).
  const T2* gtab = reinterpret_cast<const T2*>(A.tab);
  for (int i = tid; i < dN; i += blockDim.x) tab[i] = gtab[i];
  for (int i = tid; i < kNumDerived; i += blockDim.x) P[i] = (T)A.dparams[i];
  // Per-bin sums feed only the grid refinement (step 5); a pass that does
  // not refine (the integration phase of BASES, a frozen-grid VEGAS call)
  // keeps its estimate, cube sums and maxima and skips the histogram.
  const bool bins = !A.nobins;
  if (bins) {
    hist.zero_buckets(tid, blockDim.x, dN);
    hist.zero(tid, blockDim.x);
  }
  __syncthreads();

  int nonfinite = 0;
  int cd[DM];
#pragma unroll
  for (int a = 0; a < DM; ++a) cd[a] = 0;

  // w = f J in the kernel precision, widened to the histogram type H
  // (squares are then formed in H: FP64 unless ACC == 2).
  auto eval_point = [&](uint32_t s, int (&kb)[DM], bool valid = true) -> H {
    T x[DM];
    const T J = make_point<T, DM, YB, SPEC>(A, it, s, cd, tab, x, kb, nullptr);
    const T f = F<T, DM>::eval(x, d, P);
    T w = f * J;
    if (!vfinite(w)) {
      nonfinite += valid;
      w = T(0);
    }
    return (H)w;
  };
  // Two points per thread in flight (specialised FP32 kernels of low
  // dimension, whose registers allow it): their independent instruction
  // streams interleave, and the tile then holds an even number of points
  // per thread.  Sums take the two in order, as one point at a time would.
  constexpr bool PAIR = kPairPoints<T, DM, SPEC>;

  // Totals: sum w, sum w^2, sum of cube means, sum of cube-mean variances;
  // FP64 (ACC 0/1) or compensated FP32 pairs (ACC 2).
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  fpair tp[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  // The pass loop, compiled twice: with the per-bin histogram and without
  // it (a uniform choice per launch; no test inside the loops).
  auto pass = [&](auto with_bins) {
    constexpr bool B = decltype(with_bins)::value;
    auto scatter = [&](const int (&kb)[DM], H w) {
      if constexpr (B) hist.template scatter<DM>(kb, d, w);
    };
    auto gather = [&]() {
      if constexpr (B) hist.gather(tid, blockDim.x);
    };
    if (!A.strat) {
      Run<ACC> sw, sw2;
      H pmax = H(0);  // largest weight (integration-phase maximum of the one cube)
      const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
      const uint64_t first = (uint64_t)blockIdx.x * blockDim.x;
      const uint64_t rounds = first < A.ncall ? (A.ncall - first + stride - 1) / stride : 0;
      uint64_t s = first + tid;
      int pend = 0;  // points per thread since the last gather (uniform in the CTA)
      if constexpr (PAIR) {
        for (uint64_t r = 0; r < rounds; r += 2, s += 2 * stride) {
          const bool v0 = s < A.ncall, v1 = s + stride < A.ncall;
          int kb0[DM], kb1[DM];
          const H w0 = eval_point((uint32_t)s, kb0, v0);
          const H w1 = eval_point((uint32_t)(s + stride), kb1, v1);
          if (v0) {
            sw.add(w0);
            sw2.add(w0 * w0);
            pmax = max(pmax, w0);
            scatter(kb0, w0);
          }
          if (v1) {
            sw.add(w1);
            sw2.add(w1 * w1);
            pmax = max(pmax, w1);
            scatter(kb1, w1);
          }
          if ((pend += 2) >= A.ppt) {
            gather();
            pend = 0;
          }
        }
      } else {
        for (uint64_t r = 0; r < rounds; ++r, s += stride) {
          if (s < A.ncall) {
            int kb[DM];
            const H w = eval_point((uint32_t)s, kb);
            sw.add(w);
            sw2.add(w * w);
            pmax = max(pmax, w);
            scatter(kb, w);
          }
          if (++pend == A.ppt) {
            gather();
            pend = 0;
          }
        }
      }
      if (pend) gather();
      if (A.cube_max) {  // non-negative doubles order as their bit patterns
  #pragma unroll
        for (int off = 16; off > 0; off >>= 1) pmax = max(pmax, __shfl_xor_sync(0xffffffffu, pmax, off));
        if (lane == 0 && pmax > H(0))
          atomicMax(reinterpret_cast<unsigned long long*>(A.cube_max),
                    (unsigned long long)__double_as_longlong((double)pmax));
      }
      if constexpr (COMP) {
        tp[0] = sw.p;
        tp[1] = sw2.p;
      } else {
        t[0] = sw.value();
        t[1] = sw2.value();
      }
    } else {
      // Groups of Lw lanes share a hypercube; lane j of a group takes the
      // cube's points j, j + Lw, ... in lock-step with the rest of the CTA
      // (one tile per step); the group then reduces its sums with a fixed
      // xor-butterfly (deterministic).  Group i takes cube
      // (i * cube_mul) mod ncubes, so that the groups of a CTA sit in
      // unrelated cubes and spread over the bins.
      const int Lw = A.lanes;
      const int gl = tid & (Lw - 1);
      const uint32_t groups_per_cta = blockDim.x / Lw;
      const uint32_t gstride = gridDim.x * groups_per_cta;
      const uint32_t gfirst = blockIdx.x * groups_per_cta;
      const uint32_t rounds = gfirst < A.ncubes ? (A.ncubes - gfirst + gstride - 1) / gstride : 0;
      const uint32_t cmask = A.ncubes - 1u;
      const uint32_t per_lane = (A.nc + Lw - 1) / Lw;
      uint32_t gi = gfirst + tid / Lw;
      int pend = 0;  // points per thread since the last gather (uniform in the CTA)
      for (uint32_t r = 0; r < rounds; ++r, gi += gstride) {
        const bool live = gi < A.ncubes;  // uniform within a group
        const uint32_t c = A.cube_mul == 1u ? gi : (gi * A.cube_mul) & cmask;
        if (live) {
          uint32_t rest = c;
  #pragma unroll
          for (int a = 0; a < DM; ++a)
            if (a < d) {
              if (A.g_pow2) {
                cd[a] = (int)(rest & (uint32_t)(A.g - 1));
                rest >>= A.g_log2;
              } else {
                cd[a] = (int)(rest % (uint32_t)A.g);
                rest /= (uint32_t)A.g;
              }
            }
        }
        const uint32_t s0 = c * A.nc;
        // a lane's chain of points in one cube is short: plain sums in H,
        // compensated merges across the group; pmax: the largest weight (for
        // the per-cube maxima of the integration phase)
        H p1 = H(0), p2 = H(0), pmax = H(0);
        if constexpr (PAIR) {
          for (uint32_t i = 0; i < per_lane; i += 2) {
            const uint32_t j0 = gl + i * Lw, j1 = j0 + Lw;
            const bool v0 = live && j0 < A.nc, v1 = live && j1 < A.nc;
            int kb0[DM], kb1[DM];
            const H w0 = eval_point(s0 + j0, kb0, v0);
            const H w1 = eval_point(s0 + j1, kb1, v1);
            if (v0) {
              p1 += w0;
              p2 += w0 * w0;
              pmax = max(pmax, w0);
              scatter(kb0, w0);
            }
            if (v1) {
              p1 += w1;
              p2 += w1 * w1;
              pmax = max(pmax, w1);
              scatter(kb1, w1);
            }
            if ((pend += 2) >= A.ppt) {
              gather();
              pend = 0;
            }
          }
        } else {
          for (uint32_t i = 0; i < per_lane; ++i) {
            const uint32_t j = gl + i * Lw;
            if (live && j < A.nc) {
              int kb[DM];
              const H w = eval_point(s0 + j, kb);
              p1 += w;
              p2 += w * w;
              pmax = max(pmax, w);
              scatter(kb, w);
            }
            if (++pend == A.ppt) {
              gather();
              pend = 0;
            }
          }
        }
        if (A.cube_max) {  // integration phase: per-cube maxima (one group per cube)
          for (int off = Lw >> 1; off > 0; off >>= 1) pmax = max(pmax, __shfl_xor_sync(0xffffffffu, pmax, off, Lw));
          if (live && gl == 0) A.cube_max[c] = fmax(A.cube_max[c], (double)pmax);
        }
        if constexpr (COMP) {
          fpair c1{p1, 0.f}, c2{p2, 0.f};
          for (int off = Lw >> 1; off > 0; off >>= 1) {
            fpair o1, o2;
            o1.hi = __shfl_xor_sync(0xffffffffu, c1.hi, off, Lw);
            o1.lo = __shfl_xor_sync(0xffffffffu, c1.lo, off, Lw);
            o2.hi = __shfl_xor_sync(0xffffffffu, c2.hi, off, Lw);
            o2.lo = __shfl_xor_sync(0xffffffffu, c2.lo, off, Lw);
            comp_merge(c1, o1);
            comp_merge(c2, o2);
          }
          if (live && gl == 0) {
            // cube mean m = C1 / nc and variance (C2 / nc - m^2) / (nc - 1),
            // in FP32 with the square formed exactly (FMA) and the pairs kept
            const float inv = (float)A.inv_nc, inv1 = (float)A.inv_nc1;
            const float mh = c1.hi * inv, ml = c1.lo * inv;
            const float sq = mh * mh;
            const float sqe = fmaf(mh, mh, -sq) + 2.0f * mh * ml;
            const float e2h = c2.hi * inv, e2l = c2.lo * inv;
            float v = ((e2h - sq) + (e2l - sqe)) * inv1;
            if (!(v > 0.f)) v = 0.f;
            comp_merge(tp[0], c1);
            comp_merge(tp[1], c2);
            comp_add(tp[2], mh);
            comp_add(tp[2], ml);
            comp_add(tp[3], v);
            if (A.cubes)
              reinterpret_cast<float4*>(A.cubes)[c] = make_float4(c1.hi, c1.lo, c2.hi, c2.lo);
          }
        } else {
          double c1 = p1, c2 = p2;
          for (int off = Lw >> 1; off > 0; off >>= 1) {
            c1 += __shfl_xor_sync(0xffffffffu, c1, off, Lw);
            c2 += __shfl_xor_sync(0xffffffffu, c2, off, Lw);
          }
          if (live && gl == 0) {
            const double m = c1 * A.inv_nc;
            double v = (c2 * A.inv_nc - m * m) * A.inv_nc1;
            if (v < 0.0) v = 0.0;
            t[0] += c1;
            t[1] += c2;
            t[2] += m;
            t[3] += v;
            if (A.cubes) {
              reinterpret_cast<double*>(A.cubes)[2 * (size_t)c] = c1;
              reinterpret_cast<double*>(A.cubes)[2 * (size_t)c + 1] = c2;
            }
          }
        }
      }
      if (pend) gather();
    }
  };
  if (bins)
    pass(BoolTag<true>{});
  else
    pass(BoolTag<false>{});
  __syncthreads();

  // Partial row of this CTA: histogram cells (FP64, or compensated FP32
  // pairs) including the overflow cells, then the totals.
  const int np = A.nparts, row = blockIdx.x;
  for (int i = tid; bins && i < 2 * dN; i += blockDim.x) {
    if constexpr (COMP) {
      const fpair p = hist.pair(i);
      reinterpret_cast<float2*>(A.part_bins)[(size_t)i * np + row] = make_float2(p.hi, p.lo);
    } else {
      reinterpret_cast<double*>(A.part_bins)[(size_t)i * np + row] = hist.value(i);
    }
  }

  __shared__ double wsum[32][5];
  __shared__ fpair wpair[32][4];
  if constexpr (COMP) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const fpair v = warp_sum(tp[q]);
      if (lane == 0) wpair[warp][q] = v;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = t[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) wsum[warp][q] = v;
    }
  }
  int nf = nonfinite;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, off);
  if (lane == 0) wsum[warp][4] = (double)nf;
  __syncthreads();
  if (tid < 5) {
    double acc = 0.0;
    if (COMP && tid < 4) {
      fpair p{0.f, 0.f};
      for (int w = 0; w < nw; ++w) comp_merge(p, wpair[w][tid]);
      acc = comp_value(p);
    } else {
      for (int w = 0; w < nw; ++w) acc += wsum[w][tid];
    }
    A.part_tot[(size_t)tid * np + row] = acc;
  }
}

template <typename T, int ACC>
__host__ __device__ inline size_t sample_smem_bytes(int d, int N, int cap) {
  return SmemLayout<T, ACC>::total(d * N, cap);
}
template <typename T, int ACC>
__host__ __device__ inline size_t sample_smem_nobins(int d, int N) {
  return SmemLayout<T, ACC>::hist(d * N);
}

// Steps 2-3 for a list of sample indices (parity checks and debugging):
// the Philox words, bins, point, Jacobian and integrand value of each.
// SPRING trials (event generation on the frozen grid of the BASES
// integration phase; the reading is that of the oracle): trial t draws
// Philox words from counter (t, word group, 0xFFFFFFFF, instance); words
// 0..W-1 place the point as the sampling step does, words W and W+1 pick
// the cube through the integer prefix sums, the next word (two for 53-bit
// words) gives v, and the trial is kept iff w > 0 and (w exceeds the cube's
// bound, or v times the bound is below w), the comparison in FP64 (in FP32
// for the FP32 form with 24-bit words, whose weight is FP32).  Each
// chunk of trials is compacted in trial order (warp ballots, then warps in
// order).  One thread per trial and round; 256 threads.
constexpr uint32_t kSpringIt = 0xFFFFFFFFu;

template <typename T, int DM, template <typename, int> class F, int YB, bool SPEC>
__global__ void __launch_bounds__(256) k_spring(const SpringArgs R) {
  using T2 = typename Vec2<T>::type;
  const SampleArgs& A = R.S;
  const int d = SPEC ? DM : A.d, N = A.N, dN = d * N;
  extern __shared__ __align__(16) unsigned char smem[];
  T2* tab = reinterpret_cast<T2*>(smem);
  T* P = reinterpret_cast<T*>(smem + (size_t)dN * sizeof(T2));
  // kept trials per warp, double-buffered by round: one barrier per round
  // (a buffer is rewritten two rounds later, after every thread has passed
  // the next round's barrier)
  __shared__ uint32_t wcount[2][8];
  uint32_t parity = 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const T2* gtab = reinterpret_cast<const T2*>(A.tab);
  for (int i = tid; i < dN; i += blockDim.x) tab[i] = gtab[i];
  for (int i = tid; i < kNumDerived; i += blockDim.x) P[i] = (T)A.dparams[i];
  __syncthreads();
  const uint64_t Qi = R.prefix[A.ncubes];  // Q, the total integer weight
  const uint32_t G = A.ncubes;
  const int W = YB == 24 ? d : 2 * d;
  // words W .. W+2 (24-bit) or W+3 (53-bit) from the blocks of W >> 2 on:
  // the second block only when they run past the first
  const int o = W & 3;
  const bool two_blocks = o + (YB == 24 ? 3 : 4) > 4;
  unsigned long long ov = 0, np = 0;
  for (uint32_t chunk = blockIdx.x; chunk < R.nchunks; chunk += gridDim.x) {
    uint32_t chunk_count = 0;  // the same in every thread
    const uint32_t base = chunk * R.chunk;
    for (uint32_t r = 0; r < R.chunk; r += blockDim.x) {
      const uint32_t rel = base + r + tid;
      bool keep = false;
      T x[DM];
      if (rel < R.n) {
        const uint32_t t = R.trial0 + rel;
        // words W .. W+3 (cube and acceptance): at most two Philox blocks
        uint32_t wx[8];
        const int g0 = W >> 2;
        const uint4 b0 = philox4x32_10(make_uint4(t, (uint32_t)g0, kSpringIt, A.instance), A.ks);
        const uint4 b1 = two_blocks ? philox4x32_10(make_uint4(t, (uint32_t)(g0 + 1), kSpringIt, A.instance), A.ks)
                                    : make_uint4(0u, 0u, 0u, 0u);
        wx[0] = b0.x; wx[1] = b0.y; wx[2] = b0.z; wx[3] = b0.w;
        wx[4] = b1.x; wx[5] = b1.y; wx[6] = b1.z; wx[7] = b1.w;
        const uint64_t U = ((uint64_t)wx[o] << 32) | (uint64_t)wx[o + 1];
        const uint64_t u = __umul64hi(U, Qi);
        // the cube c with prefix[c] <= u < prefix[c + 1] (the last of equal
        // prefixes).  u lies in guide interval j = floor(U 2^gk / 2^64), whose
        // ends floor(j Q / 2^gk) and floor((j + 1) Q / 2^gk) bound it, so c
        // lies in [guide[j], guide[j + 1]]: a bisection over those cubes only
        const uint32_t j = R.gk ? (uint32_t)(U >> (64 - R.gk)) : 0u;
        uint32_t lo = __ldg(R.guide + j), hi = __ldg(R.guide + j + 1) + 1u;
        while (hi - lo > 1) {
          const uint32_t mid = lo + ((hi - lo) >> 1);
          if (__ldg(R.prefix + mid) <= u)
            lo = mid;
          else
            hi = mid;
        }
        const uint32_t c = lo;
        int cd[DM];
        uint32_t rest = c;
#pragma unroll
        for (int a = 0; a < DM; ++a) {
          cd[a] = 0;
          if (a < d) {
            if (A.g_pow2) {
              cd[a] = (int)(rest & (uint32_t)(A.g - 1));
              rest >>= A.g_log2;
            } else {
              cd[a] = (int)(rest % (uint32_t)A.g);
              rest /= (uint32_t)A.g;
            }
          }
        }
        int kb[DM];  // bins: not needed here
        const T J = make_point<T, DM, YB, SPEC>(A, kSpringIt, t, cd, tab, x, kb, nullptr);
        if constexpr (std::is_same<T, float>::value && YB == 24) {
          // FP32 form: the weight is FP32 already, so the decision is taken
          // in FP32 too (v is exact in 24 bits; the bound is rounded once);
          // it departs from the FP64 one only within FP32 rounding of w
          float w = F<T, DM>::eval(x, d, P) * J;
          if (R.out_scale != 1.0) w *= (float)R.out_scale;
          const float v = (float)(wx[o + 2] >> 8) * (1.0f / 16777216.0f);
          const float Mt = __ldg(R.mt32 + c);
          if (!(w > 0.f)) {
            ++np;
          } else if (w > Mt) {
            ++ov;
            keep = true;
          } else {
            keep = v * Mt < w;
          }
        } else {
          double w = (double)(F<T, DM>::eval(x, d, P) * J);
          if (R.out_scale != 1.0) w *= R.out_scale;
          const double v = YB == 24 ? (double)(wx[o + 2] >> 8) * (1.0 / 16777216.0)
                                    : ((double)(wx[o + 2] >> 5) * 67108864.0 + (double)(wx[o + 3] >> 6)) *
                                          (1.0 / 9007199254740992.0);
          const double Mt = __ldg(R.mt + c);
          if (!(w > 0.0)) {
            ++np;
          } else if (w > Mt) {
            ++ov;
            keep = true;
          } else {
            keep = v * Mt < w;
          }
        }
      }
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      if (lane == 0) wcount[parity][warp] = __popc(bal);
      __syncthreads();
      uint32_t off = chunk_count, tot = 0;
      for (int k = 0; k < nw; ++k) {
        if (k < warp) off += wcount[parity][k];
        tot += wcount[parity][k];
      }
      parity ^= 1u;
      if (keep) {
        const uint32_t pos = base + off + __popc(bal & ((1u << lane) - 1u));
#pragma unroll
        for (int a = 0; a < DM; ++a)
          if (a < d) R.stage_x[(size_t)pos * d + a] = (double)x[a];
        R.stage_t[pos] = (uint64_t)R.trial0 + rel;
      }
      chunk_count += tot;
    }
    if (tid == 0) R.counts[chunk] = chunk_count;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ov += __shfl_xor_sync(0xffffffffu, ov, off);
    np += __shfl_xor_sync(0xffffffffu, np, off);
  }
  if (lane == 0) {
    if (ov) atomicAdd(R.counters, ov);
    if (np) atomicAdd(R.counters + 1, np);
  }
}

template <typename T, int DM, template <typename, int> class F, int YB>
__global__ void __launch_bounds__(256) k_dump(const DumpArgs D) {
  __shared__ __align__(16) T P[kNumDerived];  // paired loads read 8-byte pairs
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
  const T J = make_point<T, DM, YB>(A, it, (uint32_t)s, cd,
                                    reinterpret_cast<const typename Vec2<T>::type*>(A.tab), x, kb, wl);
  const T f = F<T, DM>::eval(x, A.d, P);
  const int W = YB == 24 ? A.d : 2 * A.d;
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

// ---------------------------------------------------------------------------
// Adjoint pass: the gradient of the iteration estimate with respect to the
// integrand parameters on a frozen grid, with the random numbers of one
// iteration (common random numbers):  dI/dtheta = (1/NCALL) sum_s J_s
// df/dtheta(x_s).  Each CTA writes one partial row per column: the NT
// gradient sums, then sum w and sum w^2 (FP64, or compensated FP32 pairs
// converted once per CTA).
// ---------------------------------------------------------------------------
template <template <typename, int> class F> struct HasGrad { static constexpr bool value = false; };
template <> struct HasGrad<GenzGaussian> { static constexpr bool value = true; };
template <> struct HasGrad<DoubleGaussian> { static constexpr bool value = true; };
template <> struct HasGrad<RamboBW> { static constexpr bool value = true; };

template <typename T, int DM, template <typename, int> class F, int YB, bool SPEC = false>
__global__ void __launch_bounds__(256) k_grad(const SampleArgs A, double* part) {
  using T2 = typename Vec2<T>::type;
  constexpr int NT = F<T, DM>::NT;
  constexpr int NC = NT + 2;
  constexpr bool F32 = std::is_same<T, float>::value;
  // SPEC: d equals DM, 24-bit words, power-of-two divisions (as k_sample)
  const int d = SPEC ? DM : A.d, N = A.N, dN = d * N;
  const uint32_t it = (uint32_t)A.it_override;
  extern __shared__ __align__(16) unsigned char smem[];
  T2* tab = reinterpret_cast<T2*>(smem);
  T* P = reinterpret_cast<T*>(smem + (size_t)dN * sizeof(T2));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const T2* gtab = reinterpret_cast<const T2*>(A.tab);
  for (int i = tid; i < dN; i += blockDim.x) tab[i] = gtab[i];
  for (int i = tid; i < kNumDerived; i += blockDim.x) P[i] = (T)A.dparams[i];
  __syncthreads();

  double accd[NC];
  fpair accf[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    accd[q] = 0.0;
    accf[q] = fpair{0.f, 0.f};
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + tid; s < A.ncall; s += stride) {
    int cd[DM];
    uint32_t rest = A.strat ? (uint32_t)(s / A.nc) : 0u;
#pragma unroll
    for (int a = 0; a < DM; ++a) {
      cd[a] = 0;
      if (a < d && A.strat) {
        if (SPEC) {
          cd[a] = (int)(rest & (uint32_t)(A.g - 1));
          rest >>= A.g_log2;
        } else {
          cd[a] = (int)(rest % (uint32_t)A.g);
          rest /= (uint32_t)A.g;
        }
      }
    }
    T x[DM];
    int kb[DM];
    const T J = make_point<T, DM, YB, SPEC>(A, it, (uint32_t)s, cd, tab, x, kb, nullptr);
    T g[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) g[q] = T(0);
    const T f = F<T, DM>::grad(x, d, P, g);
    const T w = f * J;
    if (!vfinite(w)) continue;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const T v = q < NT ? g[q] * J : (q == NT ? w : w * w);
      if (!vfinite(v)) continue;
      if (F32)
        comp_add(accf[q], (float)v);
      else
        accd[q] += (double)v;
    }
  }
  __shared__ double red[8][NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    double v;
    if (F32) {
      fpair p = accf[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        fpair o;
        o.hi = __shfl_xor_sync(0xffffffffu, p.hi, off);
        o.lo = __shfl_xor_sync(0xffffffffu, p.lo, off);
        comp_merge(p, o);
      }
      v = comp_value(p);
    } else {
      v = accd[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    }
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  for (int q = tid; q < NC; q += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += red[w][q];
    part[(size_t)q * gridDim.x + blockIdx.x] = v;
  }
}

#ifndef __CUDACC_RTC__  // host-side registry builders

template <typename T>
inline size_t grad_smem_bytes(int d, int N) {
  return (size_t)d * N * sizeof(typename Vec2<T>::type) + kNumDerived * sizeof(T);
}

template <typename T, int DM, template <typename, int> class F, int YB>
inline void grad_entry(KernelEntry& e) {
  if constexpr (HasGrad<F>::value && (DM <= 20)) {
    e.grad = (const void*)&k_grad<T, DM, F, YB>;
    if constexpr (YB == 24)
      e.grad_spec = (const void*)&k_grad<T, DM, F, 24, true>;
    else
      e.grad_spec = nullptr;
    e.grad_nt = F<T, DM>::NT;
    e.grad_smem = &grad_smem_bytes<T>;
  } else {
    e.grad = nullptr;
    e.grad_spec = nullptr;
    e.grad_nt = 0;
    e.grad_smem = nullptr;
  }
}

template <typename T, int DM, template <typename, int> class F, int ACC, int YB>
inline const void* spec_kernel() {
  if constexpr (YB == 24 && ACC != 1)
    return (const void*)&k_sample<T, DM, F, ACC, 24, true>;
  else
    return nullptr;
}

template <typename T, int DM, template <typename, int> class F, int ACC, int YB>
inline KernelEntry make_entry() {
  KernelEntry e;
  e.sample = (const void*)&k_sample<T, DM, F, ACC, YB, false>;
  e.sample_spec = spec_kernel<T, DM, F, ACC, YB>();
  grad_entry<T, DM, F, YB>(e);
  e.dump = (const void*)&k_dump<T, DM, F, YB>;
  e.spring = (const void*)&k_spring<T, DM, F, YB, false>;
  if constexpr (YB == 24)
    e.spring_spec = (const void*)&k_spring<T, DM, F, 24, true>;
  else
    e.spring_spec = nullptr;
  e.smem = &sample_smem_bytes<T, ACC>;
  e.smem_nobins = &sample_smem_nobins<T, ACC>;
  e.dm = DM;
  e.spec_ppt_min = kPairPoints<T, DM, true> ? 2 : 1;
  return e;
}

template <template <typename, int> class F, int DM, int YB>
inline bool pick_precision_yb(int prec, KernelEntry* out) {
  switch (prec) {
    case VG_FP64: *out = make_entry<double, DM, F, 0, YB>(); return true;
    case VG_FP32_ACC64: *out = make_entry<float, DM, F, 1, YB>(); return true;
    case VG_FP32_ACCCOMP: *out = make_entry<float, DM, F, 2, YB>(); return true;
    default: return false;
  }
}

template <template <typename, int> class F, int DM>
inline bool pick_precision(int prec, int ybits, KernelEntry* out) {
  return ybits == 24 ? pick_precision_yb<F, DM, 24>(prec, out) : pick_precision_yb<F, DM, 53>(prec, out);
}

// Smallest instantiated bound from {4, 8, 16, 32} that covers d.
template <template <typename, int> class F>
inline bool pick_pow2_bound(int prec, int ybits, int d, KernelEntry* out) {
  if (d <= 4) return pick_precision<F, 4>(prec, ybits, out);
  if (d <= 8) return pick_precision<F, 8>(prec, ybits, out);
  if (d <= 16) return pick_precision<F, 16>(prec, ybits, out);
  if (d <= 32) return pick_precision<F, 32>(prec, ybits, out);
  return false;
}

#endif  // __CUDACC_RTC__

}  // namespace gv
