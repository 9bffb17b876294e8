// finalize.cu -- steps 4-6 of Sec. 2.1 after the sampling pass, all on the
// GPU in FP64 (the paper ran them on the host, Sec. 2.2), in one launch:
//   k_finish    fixed-order reduction of the per-CTA partial rows into the
//               per-bin sums S1, S2 and the iteration totals (one warp per
//               column; lanes stride the rows, then an xor butterfly); the
//               last block of each axis then runs the grid optimisation
//               (Lepage 1978: smoothing, log-compression with exponent
//               alpha, rebinning to equal weight) and the last block of the
//               totals the iteration estimate, the inverse-variance
//               combination, chi^2 and the ACC test.
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "kernels.h"
#include "refine.cuh"

namespace gv {

// Fixed-order sum of one column of per-CTA partials by one warp (lanes
// stride the rows, eight loads in flight, then an xor butterfly); compensated
// FP32 pairs or doubles.  Returns the sum on every lane.
__device__ double column_sum(const FinArgs& F, int col, int lane) {
  const int dN = F.d * F.N, np = F.nparts;
  if (col < 2 * dN && F.pair32) {
    const float2* p = reinterpret_cast<const float2*>(F.part_bins) + (size_t)col * np;
    fpair acc{0.f, 0.f};
    int r = lane;
    for (; r + 7 * 32 < np; r += 8 * 32) {
      float2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldcg(p + r + 32 * j);
#pragma unroll
      for (int j = 0; j < 8; ++j) comp_merge(acc, fpair{v[j].x, v[j].y});
    }
    for (; r < np; r += 32) {
      const float2 v = __ldcg(p + r);
      comp_merge(acc, fpair{v.x, v.y});
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      fpair o;
      o.hi = __shfl_xor_sync(0xffffffffu, acc.hi, off);
      o.lo = __shfl_xor_sync(0xffffffffu, acc.lo, off);
      comp_merge(acc, o);
    }
    return comp_value(acc);
  }
  const double* src = col < 2 * dN ? reinterpret_cast<const double*>(F.part_bins) + (size_t)col * np
                                   : F.part_tot + (size_t)(col - 2 * dN) * np;
  double acc = 0.0;
  int r = lane;
  for (; r + 7 * 32 < np; r += 8 * 32) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __ldcg(src + r + 32 * j);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j];
  }
  for (; r < np; r += 32) acc += __ldcg(src + r);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  return acc;
}

// Refinement of axis a from its S2 column sums, which other blocks of this
// launch wrote: read past L1 into shared memory first.  One thread per bin
// (whole warps) takes part; the other warps leave.
__device__ void refine_axis(const FinArgs& F, int a) {
  __shared__ double s2[kMaxBins];
  const int N = F.N;
  const Team t{min((int)blockDim.x, (N + 31) / 32 * 32)};
  if ((int)threadIdx.x >= t.n) return;
  const double* src = F.bins + (size_t)F.d * N + (size_t)a * N;
  for (int k = threadIdx.x; k < N; k += t.n) s2[k] = __ldcg(src + k);
  t.sync();
  refine_axis_core(s2, F.edges + (size_t)a * (N + 1), F.tab64 + (size_t)a * N, F.tab32 + (size_t)a * N, N,
                   F.alpha, t);
}

// Step 6 for the pass, by one full warp (lane 0 writes the state).
__device__ void record_iteration(const FinArgs& F) {
  GState* st = F.st;
  const double* t = F.tot;
  const int lane = threadIdx.x & 31;
  double I, var;
  if (F.strat) {
    const double G = (double)F.ncubes;
    I = t[TOT_SI] / G;
    var = t[TOT_SV] / (G * G);
  } else {
    const double n = (double)F.ncall;
    I = t[TOT_SW] / n;
    var = (t[TOT_SW2] / n - I * I) / (n - 1.0);
    if (var < 0.0) var = 0.0;
  }
  if (lane == 0) {
    st->last_I = I;
    st->last_var = var;
    st->last_sw = t[TOT_SW];
    st->last_sw2 = t[TOT_SW2];
    st->last_nonfinite = (long long)t[TOT_NONFINITE];
  }
  if (!F.record) return;
  int h = st->nhist;
  if (h < kMaxHist) {
    if (lane == 0) {
      st->hist[h][0] = I;
      st->hist[h][1] = var;
      st->nhist = h + 1;
    }
    ++h;
  }
  __syncwarp();
  if (lane == 0) {
    st->nonfinite += (long long)t[TOT_NONFINITE];
    st->samples += (long long)F.ncall;
    st->it += 1;
  }
  // Inverse-variance combination over the window (Lepage).
  double Ib, sg, chi;
  combine_history(st->hist, h, &Ib, &sg, &chi);
  if (lane == 0) {
    st->I = Ib;
    st->sigma = sg;
    st->chi2 = chi;
    if (st->acc > 0.0 && sg < st->acc * fabs(Ib)) {
      st->done = 1;
      st->stopped = 1;
    }
  }
}

// Steps 4-6 after a sampling pass in one launch.  Blocks come in groups:
// group a < d reduces the 2N columns (S1, S2) of axis a, one warp per
// column, and the last of its blocks to finish (an arrival counter, after
// a memory fence) refines axis a; the final group reduces the iteration
// totals and records the iteration.  No block waits for another: the last
// arrival does the dependent work.  `live` was latched by the sampling
// kernel of this pass and the ACC test below writes only `done`.
__global__ void __launch_bounds__(kFinishThreads) k_finish(const FinArgs F) {
  GState* st = F.st;
  if (!st->live) return;
  const int wpb = kFinishThreads / 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = F.N, dN = F.d * N;
  const int bpa = (2 * N + wpb - 1) / wpb;  // blocks per axis
  const int b = blockIdx.x;
  // without per-bin sums only the totals block is launched
  const int group = (!F.nobins && b < F.d * bpa) ? b / bpa : F.d;
  if (group < F.d) {
    const int a = group, i = (b - a * bpa) * wpb + warp;  // column of the axis, 0 .. 2N
    if (i < 2 * N) {
      const int col = i < N ? a * N + i : dN + a * N + (i - N);
      const double v = column_sum(F, col, lane);
      const double sc = *F.scale;
      if (lane == 0) F.bins[col] = v * (i < N ? sc : sc * sc);
    }
  } else if (warp < kTotCols) {
    const int q = warp;
    if (q < 5) {
      const double v = column_sum(F, 2 * dN + q, lane);
      const double s1 = *F.scale;
      const double sc = (q == TOT_SW || q == TOT_SI) ? s1 : (q == TOT_NONFINITE ? 1.0 : s1 * s1);
      if (lane == 0) F.tot[q] = v * sc;
    }
  }
  // arrival: the group's last block continues
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int n = group < F.d ? bpa : 1;
    last = atomicAdd(&st->arrive[group], 1u) == (unsigned)(n - 1);
    if (last) st->arrive[group] = 0;  // ready for the next pass
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (group < F.d) {
    if (F.refine && !F.nobins) refine_axis(F, group);
  } else if (threadIdx.x < 32) {
    record_iteration(F);
  }
}

// Column sums of a [ncols][nrows] partial block (one warp per column,
// lanes stride the rows, fixed xor butterfly).
__global__ void __launch_bounds__(256) k_colsum(const double* part, int ncols, int nrows, double* out) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= ncols) return;
  double acc = 0.0;
  for (int r = lane; r < nrows; r += 32) acc += part[(size_t)col * nrows + r];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) out[col] = acc;
}

// Window / stop-flag bookkeeping between passes (one thread); CTL_SET_ITER
// sets the Philox iteration counter.
__global__ void k_control(GState* st, int ops, double acc, uint32_t it) {
  if (ops & CTL_SET_ITER) st->it = it;
  if (ops & CTL_SNAPSHOT) {
    st->ph1_I = st->I;
    st->ph1_sigma = st->sigma;
    st->ph1_chi2 = st->chi2;
    st->ph1_iters = st->nhist;
    st->ph1_stopped = st->stopped;
    st->ph1_nonfinite = st->nonfinite;
    st->ph1_samples = st->samples;
  }
  if (ops & CTL_RESET_WINDOW) {
    st->nhist = 0;
    st->nonfinite = 0;
    st->samples = 0;
    st->I = st->sigma = st->chi2 = 0.0;
  }
  if (ops & CTL_SET_ACC) {
    st->acc = acc;
    st->done = 0;
    st->stopped = 0;
  }
}

// Uniform grid e_a[k] = k / N (step 1).
__global__ void k_uniform_grid(double* edges, int d, int N) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d * (N + 1)) return;
  edges[i] = (double)(i % (N + 1)) / (double)N;
}

// Pure table rebuild (after vegas_set_grid): tab64 / tab32 from edges.
__global__ void k_tables(const double* edges, int d, int N, double2* tab64, float2* tab32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d * N) return;
  const int a = i / N, k = i % N;
  const double lo = edges[(size_t)a * (N + 1) + k], w = edges[(size_t)a * (N + 1) + k + 1] - lo;
  tab64[i] = make_double2(lo, w);
  tab32[i] = make_float2((float)lo, (float)w);
}

}  // namespace gv

extern "C" {

// The sampling kernels run with most of the unified L1 / shared memory as
// shared memory; the small kernels between them ask for the same split, so
// that an SM need not change its partition (and drain) at every boundary.
cudaError_t gv_prepare_aux_kernels(void) {
  const void* fns[] = {(const void*)gv::k_finish, (const void*)gv::k_colsum,
                       (const void*)gv::k_control, (const void*)gv::k_uniform_grid, (const void*)gv::k_tables};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Dynamic shared-memory limit of a kernel on the current device, raised to
// at least `bytes` and never lowered.  Contexts, batches and the
// no-allocation pass share compiled kernels with different tile shapes;
// captured graphs and later launches of each keep needing the size it
// asked for, so the limit only grows (mutex: any host thread may call).
cudaError_t gv_raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[std::make_pair(dev, fn)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t gv_launch_finish(const gv::FinArgs* F, cudaStream_t s) {
  const int wpb = gv::kFinishThreads / 32;
  const int blocks = F->nobins ? 1 : F->d * ((2 * F->N + wpb - 1) / wpb) + 1;
  gv::k_finish<<<blocks, gv::kFinishThreads, 0, s>>>(*F);
  return cudaGetLastError();
}

cudaError_t gv_launch_colsum(const double* part, int ncols, int nrows, double* out, cudaStream_t s) {
  gv::k_colsum<<<(ncols + 7) / 8, 256, 0, s>>>(part, ncols, nrows, out);
  return cudaGetLastError();
}

cudaError_t gv_launch_control(gv::GState* st, int ops, double acc, uint32_t it, cudaStream_t s) {
  gv::k_control<<<1, 1, 0, s>>>(st, ops, acc, it);
  return cudaGetLastError();
}

cudaError_t gv_launch_uniform_grid(double* edges, int d, int N, cudaStream_t s) {
  const int n = d * (N + 1);
  gv::k_uniform_grid<<<(n + 255) / 256, 256, 0, s>>>(edges, d, N);
  return cudaGetLastError();
}

cudaError_t gv_launch_tables(const double* edges, int d, int N, double2* t64, float2* t32,
                             cudaStream_t s) {
  const int n = d * N;
  gv::k_tables<<<(n + 255) / 256, 256, 0, s>>>(edges, d, N, t64, t32);
  return cudaGetLastError();
}
}
