// refine.cuh -- step 5 (grid optimisation, Lepage 1978) and the step-6
// combination of iterations as device functions shared by the single-context
// and the batched finalisation kernels.  All FP64.
#pragma once

#include "common.cuh"

namespace gv {

// Error-free sum of two doubles (Knuth TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The first n threads of a block (n a multiple of 32) working as one team
// with a barrier of its own (named barrier 1), so that a step needing few
// threads leaves the other warps idle: scalar FP64 is slow on this GPU and
// even idle lanes of a warp that issues an FP64 instruction cost its pipe.
struct Team {
  int n;
  __device__ __forceinline__ void sync() const { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }
};

// Compensated all-reduce over the team (every thread gets the sum).  A
// thread's values are summed in a fixed tree (xor butterfly within a warp,
// then the warps in order), each step with TwoSum, so the result is
// deterministic and its error is that of a twice-as-precise sum.  `buf`:
// shared scratch of 2 x (warps) doubles; all team threads must call.
__device__ inline double block_sum(double v, double* buf, Team t) {
  double s = v, c = 0.0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double os = __shfl_xor_sync(0xffffffffu, s, off), oc = __shfl_xor_sync(0xffffffffu, c, off);
    double t, e;
    two_sum_d(s, os, t, e);
    s = t;
    c = c + oc + e;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = t.n >> 5;
  t.sync();  // buf may still be read from an earlier call
  if (lane == 0) {
    buf[2 * warp] = s;
    buf[2 * warp + 1] = c;
  }
  t.sync();
  double S = buf[0], C = buf[1];
  for (int w = 1; w < nw; ++w) {
    double t, e;
    two_sum_d(S, buf[2 * w], t, e);
    S = t;
    C = C + buf[2 * w + 1] + e;
  }
  return S + C;
}

// Inclusive prefix sums of x[0..n) into out[0..n) by the team (Hillis-Steele
// doubling over shared memory).
__device__ inline void block_prefix(const double* x, double* out, double* tmp, int n, Team t) {
  const int tid = threadIdx.x;
  for (int k = tid; k < n; k += t.n) out[k] = x[k];
  t.sync();
  for (int off = 1; off < n; off <<= 1) {
    for (int k = tid; k < n; k += t.n) tmp[k] = k >= off ? out[k] + out[k - off] : out[k];
    t.sync();
    for (int k = tid; k < n; k += t.n) out[k] = tmp[k];
    t.sync();
  }
}

// One axis, one team of threads: smooth the per-bin sums of w^2 over
// neighbours, compress them with r_k = ((1 - d_k/D) / ln(D/d_k))^alpha, and
// move the edges so that every new bin holds an equal share of sum r, with r
// spread uniformly inside each old bin.  dd: S2 of the axis (N values);
// e: its N+1 edges (updated in place); t64 / t32: its (e_k, Delta_k) cells.
// An axis whose smoothed sum is zero or not finite is left unchanged.
// The sums D and R are compensated block reductions, and new edge j is
// found by each thread on its own from the prefix sums C_k = r_0 + ... +
// r_{k-1}: old bin k_j is the first k with C_{k+1} >= tau_j = j R / N (or
// the last bin), and the new edge sits at the fraction (tau_j - C_k) / r_k
// of it.  This is the sequential rebinning walk of Lepage written without
// its loop-carried dependence; FP64 scalar arithmetic is slow on this GPU,
// so the serial chains are kept short.
__device__ inline void refine_axis_core(const double* dd, double* ea, double2* t64, float2* t32, int N,
                                        double alpha, Team t) {
  __shared__ double dsm[kMaxBins], r[kMaxBins], e[kMaxBins + 1], enew[kMaxBins + 1], C[kMaxBins + 1],
      tmp[kMaxBins], buf[64];
  const int tid = threadIdx.x;
  for (int k = tid; k <= N; k += t.n) e[k] = ea[k];
  double part = 0.0;
  for (int k = tid; k < N; k += t.n) {
    double v;
    if (N == 2)
      v = (dd[0] + dd[1]) / 2.0;
    else if (k == 0)
      v = (dd[0] + dd[1]) / 2.0;
    else if (k == N - 1)
      v = (dd[N - 2] + dd[N - 1]) / 2.0;
    else
      v = (dd[k - 1] + dd[k] + dd[k + 1]) / 3.0;
    dsm[k] = v;
    part += v;
  }
  const double D = block_sum(part, buf, t);
  if (!(D > 0.0) || !isfinite(D)) return;  // uniform across the team
  part = 0.0;
  for (int k = tid; k < N; k += t.n) {
    const double x = dsm[k];
    double rk = x <= 0.0 ? 0.0 : 1.0;
    if (x > 0.0 && x < D) {
      // y^alpha; the default alpha = 3/2 as y sqrt(y) (a few FP64
      // instructions instead of a general power)
      const double y = (1.0 - x / D) / log(D / x);
      rk = alpha == 1.5 ? y * sqrt(y) : pow(y, alpha);
    }
    r[k] = rk;
    part += rk;
  }
  const double R = block_sum(part, buf, t);
  // C[k + 1] = r_0 + ... + r_k, C[0] = 0
  block_prefix(r, C + 1, tmp, N, t);
  if (tid == 0) {
    C[0] = 0.0;
    enew[0] = 0.0;
    enew[N] = 1.0;
  }
  t.sync();
  for (int j = 1 + tid; j < N; j += t.n) {
    const double tau = (double)j * R / (double)N;
    // first k in [0, N-1) with C[k + 1] >= tau, else N - 1 (C is nondecreasing)
    int lo = 0, hi = N - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (C[mid + 1] >= tau)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int k = lo;
    enew[j] = e[k] + (tau - C[k]) / r[k] * (e[k + 1] - e[k]);
  }
  t.sync();
  for (int k = tid; k <= N; k += t.n) ea[k] = enew[k];
  for (int k = tid; k < N; k += t.n) {
    const double lo = enew[k], w = enew[k + 1] - enew[k];
    t64[k] = make_double2(lo, w);
    t32[k] = make_float2((float)lo, (float)w);
  }
}

// Inverse-variance combination of h iteration estimates (Lepage):
// weighted mean, its standard error and chi^2 per degree of freedom; any
// zero-variance estimate makes the result the mean of those, with sigma 0.
// Compensated xor-butterfly sum of the lanes' (s, c) pairs.
__device__ inline double warp_sum_comp(double s, double c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double os = __shfl_xor_sync(0xffffffffu, s, off), oc = __shfl_xor_sync(0xffffffffu, c, off);
    double t, e;
    two_sum_d(s, os, t, e);
    s = t;
    c = c + oc + e;
  }
  return s + c;
}

// Called by a full warp: lane j takes estimates j, j + 32, ... (divisions in
// parallel, a compensated running sum per lane), then a compensated xor
// butterfly merges the lanes; every lane returns the same result.
__device__ inline void combine_history(const double (*hist)[2], int h, double* Ib, double* sg, double* chi) {
  const int lane = threadIdx.x & 31;
  double zs = 0.0, zc = 0.0, ws = 0.0, wc = 0.0, qs = 0.0, qc = 0.0;
  int nz = 0;
  for (int j = lane; j < h; j += 32) {
    const double I = hist[j][0], v = hist[j][1];
    double t, e;
    if (!(v > 0.0)) {
      two_sum_d(zs, I, t, e);
      zs = t;
      zc += e;
      ++nz;
    } else {
      const double iv = 1.0 / v;
      two_sum_d(ws, iv, t, e);
      ws = t;
      wc += e;
      two_sum_d(qs, I * iv, t, e);
      qs = t;
      qc += e;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, off);
  const double Z = warp_sum_comp(zs, zc);
  const double W = warp_sum_comp(ws, wc);
  const double Q = warp_sum_comp(qs, qc);
  double I = 0.0, s = 0.0, x2 = 0.0;
  if (nz > 0) {
    I = Z / (double)nz;
  } else if (h > 0) {
    I = Q / W;
    s = 1.0 / sqrt(W);
    if (h > 1) {
      double cs = 0.0, cc = 0.0;
      for (int j = lane; j < h; j += 32) {
        const double dv = hist[j][0] - I;
        double t, e;
        two_sum_d(cs, dv * dv / hist[j][1], t, e);
        cs = t;
        cc += e;
      }
      x2 = warp_sum_comp(cs, cc) / (double)(h - 1);
    }
  }
  *Ib = I;
  *sg = s;
  *chi = x2;
}

}  // namespace gv
