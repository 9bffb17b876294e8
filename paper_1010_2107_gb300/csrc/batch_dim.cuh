// batch_dim.cuh -- the batched sampling pass of the FP32 form with 24-bit
// words (steps 2-4 of Sec. 2.1 for many instances at once), one kernel per
// exact dimension d = 1..16.
//
// The batch's items (threads * rounds points of one instance) are grouped
// by the instance's dimension, and each dimension runs its own persistent
// kernel k_batch_dim<D> over its own item queue; the kernels of one
// iteration run concurrently (forked streams in the iteration's graph), so
// their tails overlap.  With D a compile-time constant every loop over axes
// is unrolled exactly (no guard, no predicated-off axis), and the shared
// memory a CTA needs (the grid table and histogram of D axes) is sized for
// D, so instances of few dimensions keep many CTAs resident.
//
// A point is evaluated axis by axis: the Philox block of four words, then
// for each axis its integer-exact bin and in-bin fraction (one 64-bit
// product), x = g(y), the Jacobian factor and the integrand family's
// running accumulator (every family of the batch is a sum or a product over
// axes), with the bins kept as packed bytes.  No array of x values or bins
// is live, so a thread keeps two points in flight (PIF = 2: independent
// instruction streams) within a modest register budget.  The Philox round
// keys are read from the kernel arguments (constant bank).
//
// Histogram: the bucketed tile scheme of k_sample (a native 32-bit shared
// atomic claims a slot of each (axis, bin) bucket, the value is stored
// there, and after the tile's barrier one thread per cell sums its bucket).
// The scatter has no branch per axis: a claim past the capacity stores into
// a junk word (never read) and sets a bit of the point's overflow mask;
// after the point's axes, the rare overflowed ones go to their cells with
// float atomics.  The cells hold FP32 (S1, S2) tile sums, folded every 16
// tiles into a second FP32 level kept in the item's own output row (global
// memory, written by the one thread that owns the cell), so an item's cell
// carries at most 16 + tiles/16 roundings of FP32 (1.4e-6 relative for 128
// tiles); the row ends as the exact (hi, lo) pair of the two levels and the
// finalisation merges rows compensated.  Per-thread sums of w and w^2 are
// plain FP32 over 16 points, then merged into compensated pairs.
#pragma once

#include "batch_types.cuh"
#include "sample_kernel.cuh"

namespace gv {

// Streaming form of one integrand family: init, one update per axis (x, the
// axis constants c = (P[a], P[kMaxDim + a])), value at the end.  The
// arithmetic of each family is that of its eval in integrands.cuh, axis by
// axis in order.
template <int KIND>
struct Stream {
  float a0, a1;
  __device__ __forceinline__ void init(const float* sc) {
    a1 = 0.f;
    if (KIND == VG_GENZ_PRODUCT_PEAK) a0 = 1.f;
    else if (KIND == VG_GENZ_CORNER_PEAK) a0 = 1.f;
    else if (KIND == VG_GENZ_OSCILLATORY) a0 = sc[0];  // 2 pi u1
    else a0 = 0.f;
  }
  __device__ __forceinline__ void axis(int a, float x, float2 c, const float* sc) {
    if (KIND == VG_GENZ_GAUSSIAN) {
      const float t = x - c.y;
      a0 = fmaf(c.x * t, t, a0);
    } else if (KIND == VG_GENZ_PRODUCT_PEAK) {
      const float t = x - c.y;
      a0 *= fmaf(t, t, c.x);
    } else if (KIND == VG_GENZ_CORNER_PEAK || KIND == VG_GENZ_OSCILLATORY) {
      a0 = fmaf(c.x, x, a0);
    } else if (KIND == VG_GENZ_CONTINUOUS) {
      a0 = fmaf(c.x, fabsf(x - c.y), a0);
    } else if (KIND == VG_GENZ_DISCONTINUOUS) {
      a0 = fmaf(c.x, x, a0);
      if (a < 2 && x > sc[a]) a1 = 1.f;  // outside x_1 <= u_1, x_2 <= u_2
    } else {  // VG_DOUBLE_GAUSSIAN: c1 = sc[0], c2 = sc[1]
      const float t1 = x - sc[0], t2 = x - sc[1];
      a0 = fmaf(t1, t1, a0);
      a1 = fmaf(t2, t2, a1);
    }
  }
  __device__ __forceinline__ float value(const float* sc) const {
    if (KIND == VG_GENZ_GAUSSIAN || KIND == VG_GENZ_CONTINUOUS) return __expf(-a0);
    if (KIND == VG_GENZ_PRODUCT_PEAK) return __fdividef(1.f, a0);
    if (KIND == VG_GENZ_CORNER_PEAK) return __expf(sc[0] * __logf(a0));  // -(d+1) ln t
    if (KIND == VG_GENZ_OSCILLATORY) return qcos_any(a0);
    if (KIND == VG_GENZ_DISCONTINUOUS) return a1 != 0.f ? 0.f : __expf(a0);
    return sc[3] * (__expf(-a0 * sc[2]) + __expf(-a1 * sc[2]));  // K/2 (e1 + e2)
  }
};

// Scalar constants a family reads (sc[0..4]): corner peak -(d+1),
// oscillatory 2 pi u1, discontinuous u1, u2, two-peak Gaussian c1, c2,
// 1/w^2, K/2.
__host__ __device__ inline int stream_scalar_base(int kind) {
  return (kind == VG_GENZ_CORNER_PEAK || kind == VG_GENZ_OSCILLATORY || kind == VG_GENZ_DISCONTINUOUS ||
          kind == VG_DOUBLE_GAUSSIAN)
             ? kScalar
             : -1;
}

// Shared memory of k_batch_dim<D> with bucket capacity cap (cells = D N):
// grid table, axis constants, scalars, the cells' claim counters, the
// bucket rows, a junk word, then the cells' (S1, S2) tile sums.  A bucket
// row is S words, S the smallest value >= cap with S/2 odd: the gather
// reads a row as 8-byte pairs, and with S/2 odd the rows of 16 consecutive
// cells start on 16 different bank pairs (conflict-free reads).  Claims past
// the capacity store into the junk word (never read).
struct DimSmem {
  static __host__ __device__ size_t a16(size_t b) { return (b + 15) & ~size_t(15); }
  static __host__ __device__ int stride(int cap) {
    int r = (cap + 1) & ~1;
    return (r / 2) % 2 == 0 ? r + 2 : r;
  }
  static __host__ __device__ size_t off_pc(int cells) { return a16((size_t)cells * sizeof(float2)); }
  static __host__ __device__ size_t off_sc(int cells, int d) { return off_pc(cells) + a16((size_t)d * sizeof(float2)); }
  static __host__ __device__ size_t off_cnt(int cells, int d) { return a16(off_sc(cells, d) + 8 * sizeof(float)); }
  static __host__ __device__ size_t off_rows(int cells, int d) { return a16(off_cnt(cells, d) + (size_t)cells * sizeof(int)); }
  static __host__ __device__ size_t off_cells(int cells, int d, int cap) {
    return a16(off_rows(cells, d) + (size_t)cells * stride(cap) * sizeof(float) + sizeof(float));  // rows, junk
  }
  static __host__ __device__ size_t bytes(int cells, int d, int cap) {
    return off_cells(cells, d, cap) + (size_t)cells * sizeof(float2);  // (S1, S2) tile sums
  }
};

constexpr int kFoldTiles = 16;  // tiles between folds of the FP32 cells
constexpr int kSumPoints = 16;  // points per thread between compensated merges

// One point: Philox words, bins (packed bytes into kb), x, J and the family
// accumulator; returns w = f J.  The Jacobian is the product of the bin
// widths, scaled by N^4 after each full block of four axes (npw.x) and by
// N^(D mod 4) after a last partial one (npw.y): J = prod_a N Delta_a
// without a multiply per axis, and no partial product falls out of FP32
// range.
template <int D, int KIND>
__device__ __forceinline__ float dim_point(const BatchArgs& B, uint32_t s, uint32_t it, uint32_t inst, int N,
                                           float2 npw, const float2* tab, const float2* pc, const float* sc,
                                           uint32_t (&kb)[(D + 3) / 4]) {
  float J = 1.f;
  Stream<KIND> st;
  st.init(sc);
#pragma unroll
  for (int b = 0; b < (D + 3) / 4; ++b) {
    kb[b] = 0u;
    const uint4 w4 = philox4x32_10(make_uint4(s, (uint32_t)b, it, inst), B.ks);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = 4 * b + j;
      if (a < D) {  // compile-time
        const uint32_t u = pick(w4, j);
        // 24-bit y, no strata: (y 2^32) N as one 64-bit product, whose high
        // word is the bin k = floor(y N) and whose low word holds the 24
        // fraction bits (shifted up by 8); the fraction's top 23 bits under
        // the exponent of 1.0f by one funnel shift: the bits of bin_frac /
        // frac23
        uint32_t lo, k;
        mul_wide(u & 0xFFFFFF00u, (uint32_t)N, lo, k);
        const float fr = __uint_as_float(__funnelshift_r(lo, 0x7Fu, 9)) - 1.0f;
        const float2 e = tab[a * N + (int)k];
        const float x = fmaf(fr, e.y, e.x);
        J *= e.y;
        kb[b] |= k << (8 * j);
        st.axis(a, x, pc[a], sc);
      }
    }
    J *= 4 * b + 4 <= D ? npw.x : npw.y;
  }
  return st.value(sc) * J;
}

// Bucket scatter of one point's weight into its D cells (cnt: the claim
// counters; rows: the bucket rows; cc: the cells' (S1, S2) tile sums).
// The claims of the point's axes are issued together, then their stores:
// a store may alias a later claim's counter as far as the compiler knows,
// so claim-store pairs in sequence would expose every claim's latency.
template <int D>
__device__ __forceinline__ void dim_scatter(int* cnt, float* rows, float* junk, float2* cc, int N, int S, int cap,
                                            const uint32_t (&kb)[(D + 3) / 4], float w) {
  constexpr int G = D;  // axes per group of claims: all (measured best)
  uint32_t ovf = 0u;
#pragma unroll
  for (int a0 = 0; a0 < D; a0 += G) {
    int cell[G], pos[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int a = a0 + g;
      if (a < D) {
        cell[g] = a * N + (int)__byte_perm(kb[a >> 2], 0u, 0x4440u | (unsigned)(a & 3));
        pos[g] = atomicAdd(&cnt[cell[g]], 1);
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int a = a0 + g;
      if (a < D) {
        const bool over = pos[g] >= cap;
        *(over ? junk : rows + cell[g] * S + pos[g]) = w;
        if (over) ovf |= 1u << a;
      }
    }
  }
  if (ovf) {  // claims past the capacity (rare): straight to the cells
#pragma unroll
    for (int a = 0; a < D; ++a)
      if ((ovf >> a) & 1u) {
        const int cell = a * N + (int)__byte_perm(kb[a >> 2], 0u, 0x4440u | (unsigned)(a & 3));
        atomicAdd(&cc[cell].x, w);
        atomicAdd(&cc[cell].y, w * w);
      }
  }
}

// End of a tile (all threads): each cell's bucket into its FP32 (S1, S2)
// tile sums (paired instructions) and the counter reset; when `fold`, the
// tile sums move into the second level, the .x words of the cell's two
// entries in the item row (S1 at cell, S2 at dN + cell), which only this
// thread touches until the row is finished.  Only the filled slots are
// read: whole pairs, then a last odd slot (the slots are never cleared:
// shared-memory stores are the scarce resource).
__device__ __forceinline__ void dim_gather(int* cnt, const float* rows, float2* cc, float2* row, int dN, int S,
                                           int cap, bool fold) {
  __syncthreads();
  for (int cell = threadIdx.x; cell < dN; cell += blockDim.x) {
    const int n = min(cnt[cell], cap);
    const float2* r2 = reinterpret_cast<const float2*>(rows + cell * S);
    float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
    const int np = n >> 1;
    for (int q = 0; q < np; ++q) {
      const float2 v = r2[q];
      s1 = __fadd2_rn(s1, v);
      s2 = __ffma2_rn(v, v, s2);
    }
    if (n & 1) {
      const float v = rows[cell * S + n - 1];
      s1.x += v;
      s2.x = fmaf(v, v, s2.x);
    }
    float2 c = cc[cell];
    c.x += s1.x + s1.y;
    c.y += s2.x + s2.y;
    if (fold) {
      row[cell].x += c.x;
      row[dN + cell].x += c.y;
      c = make_float2(0.f, 0.f);
    }
    cc[cell] = c;
    cnt[cell] = 0;
  }
  __syncthreads();
}

// The points of one work item, family KIND: PIF points per thread per step
// (the step is one histogram tile), sums and scatter in point order.
template <int D, int PIF, int KIND>
__device__ __forceinline__ void dim_item(const BatchArgs& B, const BatchItem& W, uint32_t it, uint32_t inst, int N,
                                         float2 npw, const float2* tab, const float2* pc, const float* sc, int* cnt,
                                         float* rows, float* junk, float2* cc, float2* row, int S, int cap, fpair& sw,
                                         fpair& sw2, int& nonfinite) {
  const int tid = threadIdx.x, T = blockDim.x, dN = D * N;
  const uint32_t rounds = (W.count + T - 1) / T;
  float p1 = 0.f, p2 = 0.f;  // plain FP32 sums since the last compensated merge
  int since = 0, tiles = 0;
  for (uint32_t r = 0; r < rounds; r += PIF) {
    uint32_t kb[PIF][(D + 3) / 4];
    float w[PIF];
    bool v[PIF];
#pragma unroll
    for (int q = 0; q < PIF; ++q) {
      const uint32_t j = (r + q) * T + tid;
      v[q] = j < W.count;  // (r + q < rounds follows)
      w[q] = dim_point<D, KIND>(B, W.s0 + j, it, inst, N, npw, tab, pc, sc, kb[q]);
      if (!isfinite(w[q])) {
        nonfinite += v[q];
        w[q] = 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < PIF; ++q)
      if (v[q]) {
        p1 += w[q];
        p2 = fmaf(w[q], w[q], p2);
        dim_scatter<D>(cnt, rows, junk, cc, N, S, cap, kb[q], w[q]);
      }
    if ((since += PIF) >= kSumPoints) {
      comp_add(sw, p1);
      comp_add(sw2, p2);
      p1 = p2 = 0.f;
      since = 0;
    }
    dim_gather(cnt, rows, cc, row, dN, S, cap, ++tiles % kFoldTiles == 0);
  }
  comp_add(sw, p1);
  comp_add(sw2, p2);
}

// Register budget per dimension: the widest kernels are held to about three
// CTAs of 256 threads per SM by their shared memory, the narrower ones can
// keep more resident.
template <int D>
constexpr int kDimMinBlocks = D > 12 ? 3 : (D > 8 ? 4 : (D > 4 ? 5 : 6));

template <int D, int PIF>
__global__ void __launch_bounds__(256, kDimMinBlocks<D>) k_batch_dim(const BatchArgs B, const BatchRange R) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = B.N, cells = D * N, cap = R.cap, S = DimSmem::stride(cap);
  float2* tab = reinterpret_cast<float2*>(smem);
  float2* pc = reinterpret_cast<float2*>(smem + DimSmem::off_pc(cells));
  float* sc = reinterpret_cast<float*>(smem + DimSmem::off_sc(cells, D));
  int* cnt = reinterpret_cast<int*>(smem + DimSmem::off_cnt(cells, D));
  float* rows = reinterpret_cast<float*>(smem + DimSmem::off_rows(cells, D));
  float* junk = rows + (size_t)cells * S;
  float2* cc = reinterpret_cast<float2*>(smem + DimSmem::off_cells(cells, D, cap));
  __shared__ int s_item;
  __shared__ fpair red_p[8][2];
  __shared__ int red_n[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  // counters start at zero and every gather leaves them so; the bucket
  // slots need no clearing (a gather reads only the filled ones)
  for (int i = tid; i < cells; i += blockDim.x) cnt[i] = 0;
  int cur = -1;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(R.head, 1);
    __syncthreads();
    const int k = s_item;
    __syncthreads();
    if (k >= R.count) break;
    const BatchItem W = B.items[R.first + k];
    const BatchInst I = B.inst[W.inst];
    if (W.inst != cur) {  // the instance's grid cells and constants
      const float2* gtab = reinterpret_cast<const float2*>(B.tab) + I.tab_off;
      for (int i = tid; i < cells; i += blockDim.x) tab[i] = gtab[i];
      const double* dp = B.dparams + (size_t)W.inst * kNumDerived;
      for (int i = tid; i < D; i += blockDim.x) pc[i] = make_float2((float)dp[i], (float)dp[kMaxDim + i]);
      const int base = stream_scalar_base(I.kind);
      if (tid < 8) sc[tid] = base >= 0 ? (float)dp[base + tid] : 0.f;
      cur = W.inst;
    }
    // the item's row: its cells' .x words hold the folded level until the
    // row is finished (each by the thread that owns the cell); cleared as
    // whole pairs, so that every 32-byte sector is written in full and L2
    // need not fetch it from memory
    float2* row = reinterpret_cast<float2*>(B.rows) + W.row;
    for (int i = tid; i < cells; i += blockDim.x) {
      cc[i] = make_float2(0.f, 0.f);
      row[i] = make_float2(0.f, 0.f);
      row[cells + i] = make_float2(0.f, 0.f);
    }
    // N^4 and N^(D mod 4) for the Jacobian
    const float Nf = (float)N, N2 = Nf * Nf;
    constexpr int rem = D & 3;
    const float2 npw = make_float2(N2 * N2, rem == 1 ? Nf : (rem == 2 ? N2 : N2 * Nf));
    __syncthreads();
    const uint32_t it = B.st[W.inst].it;
    fpair sw{0.f, 0.f}, sw2{0.f, 0.f};
    int nonfinite = 0;
#define GV_DIM_ITEM(K) \
  dim_item<D, PIF, K>(B, W, it, I.instance, N, npw, tab, pc, sc, cnt, rows, junk, cc, row, S, cap, sw, sw2, nonfinite)
    switch (I.kind) {
      case VG_GENZ_GAUSSIAN: GV_DIM_ITEM(VG_GENZ_GAUSSIAN); break;
      case VG_GENZ_PRODUCT_PEAK: GV_DIM_ITEM(VG_GENZ_PRODUCT_PEAK); break;
      case VG_GENZ_CORNER_PEAK: GV_DIM_ITEM(VG_GENZ_CORNER_PEAK); break;
      case VG_GENZ_OSCILLATORY: GV_DIM_ITEM(VG_GENZ_OSCILLATORY); break;
      case VG_GENZ_CONTINUOUS: GV_DIM_ITEM(VG_GENZ_CONTINUOUS); break;
      case VG_GENZ_DISCONTINUOUS: GV_DIM_ITEM(VG_GENZ_DISCONTINUOUS); break;
      default: GV_DIM_ITEM(VG_DOUBLE_GAUSSIAN); break;
    }
#undef GV_DIM_ITEM
    // the item's row, S1 cells then S2 cells, each the exact pair of its
    // two FP32 levels
    for (int i = tid; i < cells; i += blockDim.x) {
      const float2 c = cc[i];
      float hi, lo;
      two_sum(row[i].x, c.x, hi, lo);
      row[i] = make_float2(hi, lo);
      two_sum(row[cells + i].x, c.y, hi, lo);
      row[cells + i] = make_float2(hi, lo);
    }
    const fpair a = warp_sum(sw), b = warp_sum(sw2);
    int nf = nonfinite;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, off);
    if (lane == 0) {
      red_p[warp][0] = a;
      red_p[warp][1] = b;
      red_n[warp] = nf;
    }
    __syncthreads();
    if (tid < 2) {
      fpair p{0.f, 0.f};
      for (int w = 0; w < nw; ++w) comp_merge(p, red_p[w][tid]);
      row[2 * cells + tid] = make_float2(p.hi, p.lo);
    } else if (tid == 2) {
      int c = 0;
      for (int w = 0; w < nw; ++w) c += red_n[w];
      row[2 * cells + 2] = make_float2((float)c, 0.f);
    }
    __syncthreads();
  }
}

#ifndef __CUDACC_RTC__
// The dimension kernels of one translation unit: k_batch_dim<d, pif>, or
// null outside its range of d.
template <int D0, int D1>
inline const void* dim_kernel_in(int d, int pif) {
  if constexpr (D0 > D1) {
    return nullptr;
  } else {
    if (d == D0) return pif == 1 ? (const void*)&k_batch_dim<D0, 1> : (const void*)&k_batch_dim<D0, 2>;
    return dim_kernel_in<D0 + 1, D1>(d, pif);
  }
}
#endif

}  // namespace gv
