// finalize.cu -- steps 4-6 of Sec. 2.1 after the sampling pass, all on the
// GPU in FP64 (the paper ran them on the host, Sec. 2.2):
//   k_reduce    fixed-order reduction of the per-CTA partial rows into the
//               per-bin sums S1, S2 and the iteration totals (one warp per
//               column; lanes stride the rows, then an xor butterfly);
//   k_finalize  per axis: grid optimisation (Lepage 1978: smoothing,
//               log-compression with exponent alpha, rebinning to equal
//               weight); one more block: the iteration estimate, the
//               inverse-variance combination, chi^2 and the ACC test.
#include "common.cuh"
#include "kernels.h"
#include "refine.cuh"

namespace gv {

__global__ void __launch_bounds__(256) k_reduce(const FinArgs F) {
  GState* st = F.st;
  const int stop = st->done;  // nobody writes `done` while k_reduce runs
  if (blockIdx.x == 0 && threadIdx.x == 0) st->live = !stop;
  if (stop) return;  // the ACC test stopped this call; no sampling pass ran
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int dN = F.d * F.N;
  const int np = F.nparts;
  const double* src;
  double sc;
  double* dst;
  if (col < 2 * dN && F.pair32) {
    // compensated FP32 pairs: fixed-order compensated sum, one conversion
    const float2* p = reinterpret_cast<const float2*>(F.part_bins) + (size_t)col * np;
    fpair acc{0.f, 0.f};
    int r = lane;
    // eight loads in flight per lane, merged in row order
    for (; r + 7 * 32 < np; r += 8 * 32) {
      float2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = p[r + 32 * j];
#pragma unroll
      for (int j = 0; j < 8; ++j) comp_merge(acc, fpair{v[j].x, v[j].y});
    }
    for (; r < np; r += 32) {
      const float2 v = p[r];
      comp_merge(acc, fpair{v.x, v.y});
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      fpair o;
      o.hi = __shfl_xor_sync(0xffffffffu, acc.hi, off);
      o.lo = __shfl_xor_sync(0xffffffffu, acc.lo, off);
      comp_merge(acc, o);
    }
    if (lane == 0) F.bins[col] = comp_value(acc) * (col < dN ? F.scale : F.scale * F.scale);
    return;
  }
  if (col < 2 * dN) {
    src = reinterpret_cast<const double*>(F.part_bins) + (size_t)col * np;
    sc = col < dN ? F.scale : F.scale * F.scale;
    dst = F.bins + col;
  } else if (col < 2 * dN + 5) {
    const int q = col - 2 * dN;
    src = F.part_tot + (size_t)q * np;
    sc = (q == TOT_SW || q == TOT_SI) ? F.scale
         : (q == TOT_NONFINITE ? 1.0 : F.scale * F.scale);
    dst = F.tot + q;
  } else {
    return;
  }
  double acc = 0.0;
  int r = lane;
  for (; r + 7 * 32 < np; r += 8 * 32) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = src[r + 32 * j];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc += v[j];
  }
  for (; r < np; r += 32) acc += src[r];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) *dst = acc * sc;
}

__device__ void refine_axis(const FinArgs& F, int a) {
  const int N = F.N;
  refine_axis_core(F.bins + (size_t)F.d * N + (size_t)a * N, F.edges + (size_t)a * (N + 1),
                   F.tab64 + (size_t)a * N, F.tab32 + (size_t)a * N, N, F.alpha);
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

__global__ void __launch_bounds__(256) k_finalize(const FinArgs F) {
  // `live` was latched by k_reduce of this pass; the ACC test below writes
  // only `done`, so every block sees the same decision.
  if (!F.st->live) return;
  if ((int)blockIdx.x < F.d) {
    if (F.refine) refine_axis(F, blockIdx.x);
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

// Window / stop-flag bookkeeping between passes (one thread).
__global__ void k_control(GState* st, int ops, double acc) {
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
  const void* fns[] = {(const void*)gv::k_reduce, (const void*)gv::k_finalize, (const void*)gv::k_colsum,
                       (const void*)gv::k_control, (const void*)gv::k_uniform_grid, (const void*)gv::k_tables};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t gv_launch_reduce(const gv::FinArgs* F, cudaStream_t s) {
  const int cols = 2 * F->d * F->N + 5;
  const int wpb = 8;
  gv::k_reduce<<<(cols + wpb - 1) / wpb, 32 * wpb, 0, s>>>(*F);
  return cudaGetLastError();
}

cudaError_t gv_launch_finalize(const gv::FinArgs* F, cudaStream_t s) {
  gv::k_finalize<<<F->d + 1, 64, 0, s>>>(*F);
  return cudaGetLastError();
}

cudaError_t gv_launch_colsum(const double* part, int ncols, int nrows, double* out, cudaStream_t s) {
  gv::k_colsum<<<(ncols + 7) / 8, 256, 0, s>>>(part, ncols, nrows, out);
  return cudaGetLastError();
}

cudaError_t gv_launch_control(gv::GState* st, int ops, double acc, cudaStream_t s) {
  gv::k_control<<<1, 1, 0, s>>>(st, ops, acc);
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
