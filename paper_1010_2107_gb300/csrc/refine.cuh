// refine.cuh -- step 5 (grid optimisation, Lepage 1978) and the step-6
// combination of iterations as device functions shared by the single-context
// and the batched finalisation kernels.  All FP64.
#pragma once

#include "common.cuh"

namespace gv {

// Neumaier compensated accumulation (same scheme as the CPU oracle).
struct KSum {
  double s = 0.0, c = 0.0;
  __device__ void add(double v) {
    const double t = s + v;
    if (fabs(s) >= fabs(v))
      c += (s - t) + v;
    else
      c += (v - t) + s;
    s = t;
  }
  __device__ double value() const { return s + c; }
};

// One axis, one thread block: smooth the per-bin sums of w^2 over
// neighbours, compress them with r_k = ((1 - d_k/D) / ln(D/d_k))^alpha, and
// move the edges so that every new bin holds an equal share of sum r, with r
// spread uniformly inside each old bin.  dd: S2 of the axis (N values);
// e: its N+1 edges (updated in place); t64 / t32: its (e_k, Delta_k) cells.
// An axis whose smoothed sum is zero or not finite is left unchanged.
__device__ inline void refine_axis_core(const double* dd, double* ea, double2* t64, float2* t32, int N,
                                        double alpha) {
  __shared__ double dsm[kMaxBins], r[kMaxBins], e[kMaxBins + 1], enew[kMaxBins + 1];
  __shared__ int skip;
  __shared__ double D;
  const int tid = threadIdx.x;
  for (int k = tid; k <= N; k += blockDim.x) e[k] = ea[k];
  for (int k = tid; k < N; k += blockDim.x) {
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
  }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += dsm[k];
    D = s;
    skip = !(s > 0.0) || !isfinite(s);
  }
  __syncthreads();
  if (skip) return;
  for (int k = tid; k < N; k += blockDim.x) {
    const double x = dsm[k];
    r[k] = x <= 0.0 ? 0.0 : (x >= D ? 1.0 : pow((1.0 - x / D) / log(D / x), alpha));
  }
  __syncthreads();
  if (tid == 0) {
    double R = 0.0;
    for (int k = 0; k < N; ++k) R += r[k];
    enew[0] = 0.0;
    enew[N] = 1.0;
    int k = 0;
    double acc = 0.0;
    for (int j = 1; j < N; ++j) {
      const double tau = (double)j * R / (double)N;
      while (k < N - 1 && acc + r[k] < tau) {
        acc += r[k];
        ++k;
      }
      enew[j] = e[k] + (tau - acc) / r[k] * (e[k + 1] - e[k]);
    }
  }
  __syncthreads();
  for (int k = tid; k <= N; k += blockDim.x) ea[k] = enew[k];
  for (int k = tid; k < N; k += blockDim.x) {
    const double lo = enew[k], w = enew[k + 1] - enew[k];
    t64[k] = make_double2(lo, w);
    t32[k] = make_float2((float)lo, (float)w);
  }
}

// Inverse-variance combination of h iteration estimates (Lepage):
// weighted mean, its standard error and chi^2 per degree of freedom; any
// zero-variance estimate makes the result the mean of those, with sigma 0.
__device__ inline void combine_history(const double (*hist)[2], int h, double* Ib, double* sg, double* chi) {
  int nzero = 0;
  KSum z;
  for (int j = 0; j < h; ++j)
    if (!(hist[j][1] > 0.0)) {
      z.add(hist[j][0]);
      ++nzero;
    }
  *Ib = 0.0;
  *sg = 0.0;
  *chi = 0.0;
  if (nzero > 0) {
    *Ib = z.value() / (double)nzero;
  } else if (h > 0) {
    KSum sw, swi;
    for (int j = 0; j < h; ++j) {
      sw.add(1.0 / hist[j][1]);
      swi.add(hist[j][0] / hist[j][1]);
    }
    *Ib = swi.value() / sw.value();
    *sg = 1.0 / sqrt(sw.value());
    if (h > 1) {
      KSum c2;
      for (int j = 0; j < h; ++j) {
        const double dv = hist[j][0] - *Ib;
        c2.add(dv * dv / hist[j][1]);
      }
      *chi = c2.value() / (double)(h - 1);
    }
  }
}

}  // namespace gv
