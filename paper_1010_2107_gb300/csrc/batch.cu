// batch.cu -- many independent VEGAS integrations in one persistent kernel
// per iteration (the batched form of the iteration loop of Sec. 2.1).
//
// Instances may differ in dimension (up to 16), integrand, parameters and
// NCALL.  Work is cut into items of `threads * rounds` points of one
// instance; persistent CTAs pull items from a device counter (no waiting:
// a CTA that finds the counter past the last item exits), evaluate them with
// the same point generation and bucketed histograms as k_sample, and write
// one partial row per item.  A finalisation kernel then reduces each
// instance's rows in a fixed order, refines each axis of each instance and
// records each instance's estimate.  A whole call is one CUDA graph.
//
// Philox: instance i draws with counter word 3 = its `instance` id, so an
// instance in a batch sees exactly the points of a standalone context with
// the same id.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "batch_types.cuh"
#include "kernels.h"
#include "refine.cuh"
#include "sample_kernel.cuh"

namespace gv {

// Integrand dispatch for the batch (the family is uniform over an item).
template <typename T, int DM>
__device__ __forceinline__ T batch_eval(int kind, const T (&x)[DM], int d, const T* P) {
  switch (kind) {
    case VG_GENZ_GAUSSIAN: return GenzGaussian<T, DM>::eval(x, d, P);
    case VG_GENZ_PRODUCT_PEAK: return GenzProductPeak<T, DM>::eval(x, d, P);
    case VG_GENZ_CORNER_PEAK: return GenzCornerPeak<T, DM>::eval(x, d, P);
    case VG_GENZ_OSCILLATORY: return GenzOscillatory<T, DM>::eval(x, d, P);
    case VG_GENZ_CONTINUOUS: return GenzContinuous<T, DM>::eval(x, d, P);
    case VG_GENZ_DISCONTINUOUS: return GenzDiscontinuous<T, DM>::eval(x, d, P);
    default: return DoubleGaussian<T, DM>::eval(x, d, P);
  }
}

// The points of one work item (all threads of the CTA); DMC bounds the
// instance's dimension.
template <typename T, int ACC, int YB, int DMC>
__device__ __forceinline__ void batch_item_points(const BatchArgs& B, const SampleArgs& A, const BatchItem& W,
                                                  int kind, uint32_t it, int d,
                                                  const typename Vec2<T>::type* tab, const T* P,
                                                  TileHist<ACC>& hist, Run<ACC>& sw, Run<ACC>& sw2,
                                                  int& nonfinite) {
  using H = typename AccTraits<ACC>::H;
  int cd[DMC];
#pragma unroll
  for (int a = 0; a < DMC; ++a) cd[a] = 0;
  const int tid = threadIdx.x;
  const uint32_t rounds = (W.count + blockDim.x - 1) / blockDim.x;
  for (uint32_t r = 0; r < rounds; ++r) {
    const uint32_t j = r * blockDim.x + tid;
    if (j < W.count) {
      T x[DMC];
      int kb[DMC];
      const T J = make_point<T, DMC, YB>(A, it, W.s0 + j, cd, tab, x, kb, nullptr);
      T w = batch_eval<T, DMC>(kind, x, d, P) * J;
      if (!vfinite(w)) {
        ++nonfinite;
        w = T(0);
      }
      const H wh = (H)w;
      sw.add(wh);
      sw2.add(wh * wh);
      hist.template scatter<DMC>(kb, d, wh);
    }
    if ((r + 1) % (uint32_t)B.ppt == 0 || r + 1 == rounds) hist.gather(tid, blockDim.x);
  }
}

template <typename T, int ACC>
struct BatchSmem {
  static __host__ __device__ size_t a16(size_t b) { return (b + 15) & ~size_t(15); }
  static __host__ __device__ size_t params(int md, int N) { return (size_t)md * N * sizeof(typename Vec2<T>::type); }
  static __host__ __device__ size_t hist(int md, int N) { return a16(params(md, N) + kNumDerived * sizeof(T)); }
  static __host__ __device__ size_t total(int md, int N, int cap) {
    return hist(md, N) + TileHist<ACC>::bytes(md * N, cap);
  }
};

template <typename T, int ACC, int YB>
__global__ void __launch_bounds__(256) k_batch_sample(const BatchArgs B) {
  using H = typename AccTraits<ACC>::H;
  using T2 = typename Vec2<T>::type;
  using L = BatchSmem<T, ACC>;
  constexpr int DM = kBatchDM;
  constexpr bool COMP = ACC == 2;
  extern __shared__ __align__(16) unsigned char smem[];
  T2* tab = reinterpret_cast<T2*>(smem);
  T* P = reinterpret_cast<T*>(smem + L::params(B.maxd, B.N));
  __shared__ int s_item;
  __shared__ double red_d[8][3];
  __shared__ fpair red_p[8][2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int N = B.N;
  int cur = -1;
  TileHist<ACC> hist;
  SampleArgs A{};
  A.N = N;
  A.g = 1;
  A.ybits = YB;
  A.strat = 0;
  A.t32 = 1;
  A.g_pow2 = 1;
  A.g_log2 = 0;
  A.key0 = B.key0;
  A.key1 = B.key1;
#pragma unroll
  for (int i = 0; i < kPhiloxKeyWords; ++i) A.ks[i] = B.ks[i];
  A.inv_gb_d = 1.0 / (double)(1ull << YB);
  A.inv_gb_f = (float)A.inv_gb_d;
  // one layout for every instance (sized for the widest); the bucket
  // slots are cleared once and every gather leaves them cleared
  const int MD = B.maxd;
  hist.bind(smem + L::hist(MD, N), MD * N, N, B.cap, B.ppt, MD * N);
  hist.zero_buckets(tid, blockDim.x, MD * N);

  for (;;) {
    if (tid == 0) s_item = atomicAdd(B.head, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= B.nitems) break;
    const BatchItem W = B.items[item];
    const BatchInst I = B.inst[W.inst];
    const int d = I.d, dN = d * N;
    if (W.inst != cur) {  // stage the instance's grid cells and constants
      const T2* gtab = reinterpret_cast<const T2*>(B.tab) + I.tab_off;
      for (int i = tid; i < dN; i += blockDim.x) tab[i] = gtab[i];
      const double* dp = B.dparams + (size_t)W.inst * kNumDerived;
      for (int i = tid; i < kNumDerived; i += blockDim.x) P[i] = (T)dp[i];
      cur = W.inst;
    }
    hist.bind(smem + L::hist(MD, N), dN, N, B.cap, B.ppt, MD * N);
    hist.zero(tid, blockDim.x);
    __syncthreads();
    A.d = d;
    A.instance = I.instance;
    const uint32_t it = B.st[W.inst].it;
    Run<ACC> sw, sw2;
    int nonfinite = 0;
    batch_item_points<T, ACC, YB, DM>(B, A, W, I.kind, it, d, tab, P, hist, sw, sw2, nonfinite);
    // the item's partial row: cells, then sum w, sum w^2, non-finite count
    for (int i = tid; i < 2 * dN; i += blockDim.x) {
      if constexpr (COMP) {
        const fpair p = hist.pair(i);
        reinterpret_cast<float2*>(B.rows)[W.row + i] = make_float2(p.hi, p.lo);
      } else {
        reinterpret_cast<double*>(B.rows)[W.row + i] = hist.value(i);
      }
    }
    int nf = nonfinite;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, off);
    if constexpr (COMP) {
      const fpair a = warp_sum(sw.p), b = warp_sum(sw2.p);
      if (lane == 0) {
        red_p[warp][0] = a;
        red_p[warp][1] = b;
        red_d[warp][2] = (double)nf;
      }
    } else {
      double a = sw.value(), b = sw2.value();
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
      }
      if (lane == 0) {
        red_d[warp][0] = a;
        red_d[warp][1] = b;
        red_d[warp][2] = (double)nf;
      }
    }
    __syncthreads();
    if (tid < kRowTail) {
      if constexpr (COMP) {
        if (tid < 2) {
          fpair p{0.f, 0.f};
          for (int w = 0; w < nw; ++w) comp_merge(p, red_p[w][tid]);
          reinterpret_cast<float2*>(B.rows)[W.row + 2 * dN + tid] = make_float2(p.hi, p.lo);
        } else {
          double c = 0.0;
          for (int w = 0; w < nw; ++w) c += red_d[w][2];
          reinterpret_cast<float2*>(B.rows)[W.row + 2 * dN + 2] = make_float2((float)c, 0.f);
        }
      } else {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += red_d[w][tid];
        reinterpret_cast<double*>(B.rows)[W.row + 2 * dN + tid] = v;
      }
    }
    __syncthreads();
  }
}

// Sums of the entries off[0..K) over an instance's item rows, each in item
// order.  The rows of an instance's items are consecutive, 2 d N + kRowTail
// entries apart, so the addresses need no lookup: eight rows' loads are
// issued ahead of their merges, which keep the sequential order.
template <int K>
__device__ inline void row_sums(const BatchArgs& B, const BatchInst& I, const int (&off)[K], double (&out)[K]) {
  constexpr int U = 8;
  const int n = I.nitems;
  const size_t stride = 2 * (size_t)I.d * B.N + kRowTail, base = B.items[I.first_item].row;
  if (B.pair32) {
    const float2* rows = reinterpret_cast<const float2*>(B.rows) + base;
    fpair acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = fpair{0.f, 0.f};
    int k = 0;
    for (; k + U <= n; k += U) {
      float2 v[U][K];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < K; ++j) v[u][j] = rows[(size_t)(k + u) * stride + off[j]];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int j = 0; j < K; ++j) comp_merge(acc[j], fpair{v[u][j].x, v[u][j].y});
    }
    for (; k < n; ++k)
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const float2 v = rows[(size_t)k * stride + off[j]];
        comp_merge(acc[j], fpair{v.x, v.y});
      }
#pragma unroll
    for (int j = 0; j < K; ++j) out[j] = comp_value(acc[j]);
    return;
  }
  const double* rows = reinterpret_cast<const double*>(B.rows) + base;
  double acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0.0;
  int k = 0;
  for (; k + U <= n; k += U) {
    double v[U][K];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < K; ++j) v[u][j] = rows[(size_t)(k + u) * stride + off[j]];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += v[u][j];
  }
  for (; k < n; ++k)
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] += rows[(size_t)k * stride + off[j]];
#pragma unroll
  for (int j = 0; j < K; ++j) out[j] = acc[j];
}

// Blocks [0, naxes): reduce one axis of one instance (2 N cells) and refine
// it; blocks [naxes, naxes + n): estimate, history and combination of one
// instance.
__global__ void __launch_bounds__(128) k_batch_finalize(const BatchArgs B) {
  __shared__ double s2[kMaxBins];
  const int b = blockIdx.x;
  if (b < B.naxes) {
    const int2 ia = B.axis_map[b];
    const BatchInst I = B.inst[ia.x];
    const int N = B.N, a = ia.y, dN = I.d * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const int off[2] = {a * N + k, dN + a * N + k};
      double S[2];
      row_sums<2>(B, I, off, S);
      B.bins[I.bins_off + a * N + k] = S[0];
      B.bins[I.bins_off + dN + a * N + k] = S[1];
      s2[k] = S[1];
    }
    __syncthreads();
    const Team t{min((int)blockDim.x, (N + 31) / 32 * 32)};  // one thread per bin, whole warps
    if (B.refine && (int)threadIdx.x < t.n)
      refine_axis_core(s2, B.edges + I.edge_off + (size_t)a * (N + 1), B.tab64 + I.tab_off + (size_t)a * N,
                       B.tab32 + I.tab_off + (size_t)a * N, N, I.alpha, t);
    return;
  }
  const int i = b - B.naxes;
  if (i >= B.n || threadIdx.x >= 32) return;  // one warp per instance; lane 0 writes
  const bool w0 = threadIdx.x == 0;
  const BatchInst I = B.inst[i];
  const int dN = I.d * B.N;
  const int off[3] = {2 * dN, 2 * dN + 1, 2 * dN + 2};
  double tot[3];
  row_sums<3>(B, I, off, tot);
  const double sw = tot[0], sw2 = tot[1], nf = tot[2];
  const double n = (double)I.ncall;
  const double Ij = sw / n;
  double var = (sw2 / n - Ij * Ij) / (n - 1.0);
  if (var < 0.0) var = 0.0;
  BatchState* st = B.st + i;
  if (w0) {
    st->last_I = Ij;
    st->last_var = var;
  }
  if (!B.record) return;
  int h = st->nhist;
  if (h < kBatchHist) {
    if (w0) {
      st->hist[h][0] = Ij;
      st->hist[h][1] = var;
      st->nhist = h + 1;
    }
    ++h;
  }
  __syncwarp();
  if (w0) {
    st->nonfinite += (long long)nf;
    st->samples += (long long)I.ncall;
    st->it += 1;
  }
  double Ib, sg, chi;
  combine_history(st->hist, h, &Ib, &sg, &chi);
  if (w0) {
    st->I = Ib;
    st->sigma = sg;
    st->chi2 = chi;
  }
}

// Whole-batch reset in one launch: block i clears instance i's state and
// writes its uniform grid and both cell tables; block 0 also clears the
// work-queue head.
__global__ void k_batch_reset(BatchState* st, const BatchInst* inst, int n, int N, double* edges,
                              double2* tab64, float2* tab32, int* head) {
  const int i = blockIdx.x;
  if (i >= n) return;
  if (threadIdx.x == 0) {
    st[i].nhist = 0;
    st[i].nonfinite = 0;
    st[i].samples = 0;
    st[i].I = st[i].sigma = st[i].chi2 = 0.0;
    st[i].it = 0;
    if (i == 0) *head = 0;
  }
  const BatchInst I = inst[i];
  for (int j = threadIdx.x; j < I.d * (N + 1); j += blockDim.x)
    edges[I.edge_off + j] = (double)(j % (N + 1)) / (double)N;
  for (int j = threadIdx.x; j < I.d * N; j += blockDim.x) {
    const int k = j % N;
    const double lo = (double)k / (double)N, w = (double)(k + 1) / (double)N - lo;
    tab64[I.tab_off + j] = make_double2(lo, w);
    tab32[I.tab_off + j] = make_float2((float)lo, (float)w);
  }
}

}  // namespace gv

#include "batch_dim.cuh"

using gv::BatchArgs;
using gv::BatchInst;
using gv::BatchItem;
using gv::BatchState;

namespace {

thread_local std::string g_batch_err;

}  // namespace

struct vegas_batch {
  int n = 0, N = 50, prec = VG_FP32_ACCCOMP, ybits = 24;
  int maxd = 1;  // widest instance
  uint64_t seed = 1;
  std::vector<vegas_config> cfg;
  std::vector<int> kind, d;
  std::vector<std::vector<double>> params;
  std::vector<double> derived;  // [n][kNumDerived]
  int sm_count = 0;
  // launch shape
  int threads = 256, rounds = 32, ctas = 0, cap = 16, ppt = 1, occ = 0;
  int ppt_req = 0;         // points per thread per tile asked for (0: automatic)
  bool small_cap = false;  // tile capacity policy (gv::choose_tile)
  bool dense_cap = false;  // the dense floor of that policy (per-dimension kernels)
  // FP32 form with 24-bit words: one kernel per exact dimension d = 1..16,
  // each with its item range, tile and launch shape, run concurrently on
  // the auxiliary streams (forked from and joined to `stream`)
  bool by_dim = false;
  struct Dim {
    int first = 0, count = 0, cap = 4, ctas = 0, occ = 0;
    size_t smem = 0;
    const void* fn = nullptr;
  } dims[gv::kBatchDM];
  static constexpr int kAux = 4;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t fork = nullptr, join[kAux] = {};
  size_t smem = 0;
  const void* kernel = nullptr;
  // host copies of the tables
  std::vector<BatchInst> inst;
  std::vector<BatchItem> items;
  std::vector<int2> axis_map;
  size_t row_entries = 0, rows_cap = 0;
  // device buffers
  BatchInst* d_inst = nullptr;
  BatchItem* d_items = nullptr;
  size_t items_cap = 0;
  int2* d_axis = nullptr;
  double *d_edges = nullptr, *d_derived = nullptr, *d_bins = nullptr;
  double2* d_tab64 = nullptr;
  float2* d_tab32 = nullptr;
  void* d_rows = nullptr;
  BatchState* d_st = nullptr;
  int* d_head = nullptr;
  BatchState* h_st = nullptr;
  double* h_derived = nullptr;  // pinned staging of vegas_batch_set_params
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  std::string err;

  vegas_status fail(vegas_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    char buf[512];
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    g_batch_err = err;
    return s;
  }
};

namespace {

#define BK(b, call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return (b)->fail(e_ == cudaErrorMemoryAllocation ? VEGAS_ENOMEM : VEGAS_ECUDA,   \
                       "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

vegas_status bfail(const char* msg) {
  g_batch_err = msg;
  return VEGAS_EINVAL;
}

void drop_graphs(vegas_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

template <typename T, int ACC, int YB>
const void* batch_kernel() {
  return (const void*)&gv::k_batch_sample<T, ACC, YB>;
}

// The general kernel: FP64, or FP32 with 53-bit words (the FP32 form with
// 24-bit words runs the per-dimension kernels instead).
const void* pick_batch_kernel(int prec, int ybits) {
  if (prec == VG_FP64) return ybits == 24 ? batch_kernel<double, 0, 24>() : batch_kernel<double, 0, 53>();
  return batch_kernel<float, 2, 53>();
}

size_t batch_smem(int prec, int md, int N, int cap) {
  return prec == VG_FP64 ? gv::BatchSmem<double, 0>::total(md, N, cap) : gv::BatchSmem<float, 2>::total(md, N, cap);
}

// Items of `threads * rounds` points, instances in decreasing NCALL order so
// that the small items come last (grouped by dimension first, widest first,
// when the dimension kernels run); rows laid out in item order.
vegas_status build_items(vegas_batch* b) {
  const uint64_t tile = (uint64_t)b->threads * b->rounds;
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    if (b->by_dim && b->d[x] != b->d[y]) return b->d[x] > b->d[y];
    return b->cfg[x].ncall > b->cfg[y].ncall;
  });
  b->items.clear();
  for (auto& c : b->dims) c.first = c.count = 0;
  size_t row = 0;
  for (int i : order) {
    BatchInst& I = b->inst[i];
    if (b->by_dim) {
      auto& c = b->dims[I.d - 1];
      if (c.count == 0) c.first = (int)b->items.size();
    }
    // an instance's items are consecutive and so are their rows, each
    // 2 d N + kRowTail entries long: k_batch_finalize addresses them by
    // that stride from the first item's row
    I.first_item = (int)b->items.size();
    const uint64_t n = (uint64_t)b->cfg[i].ncall;
    for (uint64_t s0 = 0; s0 < n; s0 += tile) {
      BatchItem it;
      it.inst = i;
      it.s0 = (uint32_t)s0;
      it.count = (uint32_t)std::min<uint64_t>(tile, n - s0);
      it.row = (uint32_t)row;
      row += 2 * (size_t)I.d * b->N + gv::kRowTail;
      b->items.push_back(it);
    }
    I.nitems = (int)b->items.size() - I.first_item;
    if (b->by_dim) b->dims[I.d - 1].count += I.nitems;
  }
  for (auto& c : b->dims) c.ctas = std::min(c.count, b->sm_count * std::max(c.occ, 1));
  if (row > 0xFFFFFFFFull) return b->fail(VEGAS_EINVAL, "batch too large for the partial-row index");
  const size_t esz = b->prec == VG_FP64 ? sizeof(double) : sizeof(float2);
  if (row > b->rows_cap) {
    cudaFree(b->d_rows);
    b->d_rows = nullptr;
    b->rows_cap = 0;
    BK(b, gv_dev_malloc(&b->d_rows, row * esz));
    b->rows_cap = row;
  }
  b->row_entries = row;
  if (b->items.size() > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    BK(b, gv_malloc(&b->d_items, b->items.size() * sizeof(BatchItem)));
    b->items_cap = b->items.size();
  }
  BK(b, cudaMemcpyAsync(b->d_items, b->items.data(), b->items.size() * sizeof(BatchItem),
                        cudaMemcpyHostToDevice, b->stream));
  BK(b, cudaMemcpyAsync(b->d_inst, b->inst.data(), b->n * sizeof(BatchInst), cudaMemcpyHostToDevice,
                        b->stream));
  BK(b, cudaStreamSynchronize(b->stream));
  drop_graphs(b);
  return VEGAS_OK;
}

// Dimension kernels: for each dimension present its kernel (points in
// flight = the tile's points per thread), bucket capacity and CTAs per SM.
vegas_status configure_dims(vegas_batch* b) {
  const int pif = b->ppt_req == 1 ? 1 : 2;
  b->ppt = pif;
  bool present[gv::kBatchDM] = {};
  for (int i = 0; i < b->n; ++i) present[b->d[i] - 1] = true;
  int widest = 0;
  for (int d = 1; d <= gv::kBatchDM; ++d) {
    auto& c = b->dims[d - 1];
    c.occ = 0;
    if (!present[d - 1]) continue;
    widest = d;
    const int cells = d * b->N;
    c.fn = d <= 8 ? gv_batch_dim_kernel_lo(d, pif) : gv_batch_dim_kernel_hi(d, pif);
    BK(b, cudaFuncSetAttribute(c.fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
    cudaError_t e = cudaSuccess;
    auto occ_of = [&](int cap, int) -> int {
      const size_t smem = gv::DimSmem::bytes(cells, d, cap);
      int o = 0;
      if (e != cudaSuccess || smem > 227 * 1024) return 0;
      e = gv_raise_smem_limit(c.fn, smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, c.fn, b->threads, smem);
      return e == cudaSuccess ? o : 0;
    };
    int occ_cap = 0;
    BK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cap, c.fn, b->threads, 0));
    const gv::TileShape t = gv::choose_tile(b->threads, b->N, pif, pif, occ_cap, occ_of, b->small_cap, b->dense_cap);
    BK(b, e);
    if (t.occ < 1) return b->fail(VEGAS_EINVAL, "batch kernel for %d axes does not fit: %d threads", d, b->threads);
    c.cap = gv::DimSmem::stride(t.cap);  // the row holds this many slots
    c.occ = t.occ;
    c.smem = gv::DimSmem::bytes(cells, d, c.cap);
    BK(b, gv_raise_smem_limit(c.fn, c.smem));
  }
  b->cap = widest ? b->dims[widest - 1].cap : 0;
  b->occ = widest ? b->dims[widest - 1].occ : 0;
  b->ctas = b->sm_count * b->occ;
  return build_items(b);
}

vegas_status configure(vegas_batch* b) {
  if (b->by_dim) return configure_dims(b);
  b->kernel = pick_batch_kernel(b->prec, b->ybits);
  BK(b, cudaFuncSetAttribute(b->kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared));
  cudaError_t e = cudaSuccess;
  auto occ_of = [&](int cap, int) -> int {
    const size_t smem = batch_smem(b->prec, b->maxd, b->N, cap);
    int o = 0;
    if (e != cudaSuccess || smem > 227 * 1024) return 0;
    e = gv_raise_smem_limit(b->kernel, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, b->kernel, b->threads, smem);
    return e == cudaSuccess ? o : 0;
  };
  int occ_cap = 0;
  BK(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cap, b->kernel, b->threads, 0));
  const gv::TileShape t = gv::choose_tile(b->threads, b->N, b->ppt_req, 1, occ_cap, occ_of, b->small_cap);
  BK(b, e);
  if (t.occ < 1) return b->fail(VEGAS_EINVAL, "batch kernel does not fit: %d threads", b->threads);
  b->smem = batch_smem(b->prec, b->maxd, b->N, t.cap);
  BK(b, gv_raise_smem_limit(b->kernel, b->smem));
  b->cap = t.cap;
  b->ppt = t.ppt;
  b->occ = t.occ;
  const int occ = t.occ;
  b->ctas = b->sm_count * occ;
  return build_items(b);
}

BatchArgs batch_args(const vegas_batch* b, int refine, int record) {
  BatchArgs A{};
  A.n = b->n;
  A.nitems = (int)b->items.size();
  A.N = b->N;
  A.cap = b->cap;
  A.ppt = b->ppt;
  A.maxd = b->maxd;
  A.key0 = (uint32_t)b->seed;
  A.key1 = (uint32_t)(b->seed >> 32);
  gv::philox_key_schedule(A.key0, A.key1, A.ks);
  A.inst = b->d_inst;
  A.items = b->d_items;
  A.tab = b->prec == VG_FP64 ? (const void*)b->d_tab64 : (const void*)b->d_tab32;
  A.dparams = b->d_derived;
  A.head = b->d_head;
  A.rows = b->d_rows;
  A.st = b->d_st;
  A.edges = b->d_edges;
  A.tab64 = b->d_tab64;
  A.tab32 = b->d_tab32;
  A.bins = b->d_bins;
  A.axis_map = b->d_axis;
  A.naxes = (int)b->axis_map.size();
  A.refine = refine;
  A.record = record;
  A.pair32 = b->prec != VG_FP64;
  return A;
}

vegas_status launch_sample(vegas_batch* b, BatchArgs& A) {
  BK(b, cudaMemsetAsync(b->d_head, 0, (1 + gv::kBatchDM) * sizeof(int), b->stream));
  if (b->by_dim) {
    // fork: the dimension kernels on the auxiliary streams (the widest, with
    // the longest items, first), then join them back
    BK(b, cudaEventRecord(b->fork, b->stream));
    int k = 0;
    for (int d = gv::kBatchDM; d >= 1; --d) {
      const auto& c = b->dims[d - 1];
      if (c.count == 0) continue;
      cudaStream_t s = b->aux[k % vegas_batch::kAux];
      if (k < vegas_batch::kAux) BK(b, cudaStreamWaitEvent(s, b->fork, 0));
      gv::BatchRange R{c.first, c.count, b->d_head + d, c.cap};
      void* args[] = {&A, &R};
      BK(b, cudaLaunchKernel(c.fn, dim3(c.ctas), dim3(b->threads), args, c.smem, s));
      ++k;
    }
    for (int i = 0; i < std::min(k, vegas_batch::kAux); ++i) {
      BK(b, cudaEventRecord(b->join[i], b->aux[i]));
      BK(b, cudaStreamWaitEvent(b->stream, b->join[i], 0));
    }
    return VEGAS_OK;
  }
  void* args[] = {&A};
  BK(b, cudaLaunchKernel(b->kernel, dim3(b->ctas), dim3(b->threads), args, b->smem, b->stream));
  return VEGAS_OK;
}

vegas_status launch_iteration(vegas_batch* b, int refine, int record) {
  BatchArgs A = batch_args(b, refine, record);
  vegas_status st = launch_sample(b, A);
  if (st) return st;
  const int blocks = A.naxes + A.n;
  gv::k_batch_finalize<<<blocks, 128, 0, b->stream>>>(A);
  BK(b, cudaGetLastError());
  return VEGAS_OK;
}

vegas_status read_states(vegas_batch* b) {
  BK(b, cudaMemcpyAsync(b->h_st, b->d_st, sizeof(BatchState) * b->n, cudaMemcpyDeviceToHost, b->stream));
  BK(b, cudaStreamSynchronize(b->stream));
  return VEGAS_OK;
}

}  // namespace

extern "C" {

const char* vegas_batch_last_error(const vegas_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void vegas_batch_destroy(vegas_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  cudaFree(b->d_inst);
  cudaFree(b->d_items);
  cudaFree(b->d_axis);
  cudaFree(b->d_edges);
  cudaFree(b->d_derived);
  cudaFree(b->d_bins);
  cudaFree(b->d_tab64);
  cudaFree(b->d_tab32);
  cudaFree(b->d_rows);
  cudaFree(b->d_st);
  cudaFree(b->d_head);
  if (b->h_st) cudaFreeHost(b->h_st);
  if (b->h_derived) cudaFreeHost(b->h_derived);
  for (int i = 0; i < vegas_batch::kAux; ++i) {
    if (b->aux[i]) cudaStreamDestroy(b->aux[i]);
    if (b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

vegas_status vegas_batch_create(int n, const vegas_config* cfgs, const vegas_integrand* fns, vegas_batch** out) {
  if (!out) return bfail("out is NULL");
  *out = nullptr;
  if (n < 1 || !cfgs || !fns) return bfail("need n >= 1 configs and integrands");
  const vegas_config& c0 = cfgs[0];
  const int prec = c0.precision;
  if (prec != VG_FP64 && prec != VG_FP32_ACCCOMP) return bfail("batch precision must be VG_FP64 or VG_FP32_ACCCOMP");
  const int ybits = c0.ybits ? c0.ybits : (prec == VG_FP64 ? 53 : 24);
  if (ybits != 24 && ybits != 53) return bfail("ybits must be 24 or 53");
  if (c0.nbins < 2 || c0.nbins > GVEGAS_MAXBINS) return bfail("nbins out of range");
  for (int i = 0; i < n; ++i) {
    const vegas_config& c = cfgs[i];
    const int cy = c.ybits ? c.ybits : (c.precision == VG_FP64 ? 53 : 24);
    if (c.precision != prec || cy != ybits || c.nbins != c0.nbins || c.seed != c0.seed)
      return bfail("batch instances must share precision, ybits, nbins and seed");
    if (c.nstrat > 1) return bfail("batch instances are not stratified");
    if (c.ndim < 1 || c.ndim > gv::kBatchDM) return bfail("batch instances need 1 <= ndim <= 16");
    if (c.ncall < 2 || c.ncall > ((int64_t)1 << 32) - 1) return bfail("ncall outside 2..2^32-1");
    if (!(c.alpha >= 0.0)) return bfail("alpha must be >= 0");
    if (fns[i].ndim != c.ndim) return bfail("integrand ndim differs from config ndim");
    if (fns[i].kind == VG_RAMBO_BW || fns[i].kind == VG_W_MUNU)
      return bfail("RAMBO and W -> mu nu integrands are not batched");
    const int np = gv::expected_nparams(fns[i].kind, c.ndim);
    if (np < 0 || fns[i].nparams != np || (np > 0 && !fns[i].params))
      return bfail("integrand parameter count does not match its kind");
  }
  vegas_batch* b = new vegas_batch();
  auto bail = [&](vegas_status s) {
    g_batch_err = b->err;
    vegas_batch_destroy(b);
    return s;
  };
  b->n = n;
  b->N = c0.nbins;
  b->prec = prec;
  b->ybits = ybits;
  b->seed = c0.seed;
  b->by_dim = prec == VG_FP32_ACCCOMP && ybits == 24;
  b->cfg.assign(cfgs, cfgs + n);
  b->derived.assign((size_t)n * gv::kNumDerived, 0.0);
  b->inst.resize(n);
  int cells = 0, edges = 0;
  for (int i = 0; i < n; ++i) {
    const int d = cfgs[i].ndim;
    b->kind.push_back(fns[i].kind);
    b->d.push_back(d);
    b->maxd = std::max(b->maxd, d);
    b->params.emplace_back(fns[i].params, fns[i].params + fns[i].nparams);
    double scale = 1.0;
    std::string why;
    if (!gv::derive_params(fns[i].kind, d, b->params.back().data(), &b->derived[(size_t)i * gv::kNumDerived],
                           &scale, &why)) {
      b->fail(VEGAS_EINVAL, "instance %d: %s", i, why.c_str());
      return bail(VEGAS_EINVAL);
    }
    BatchInst& I = b->inst[i];
    I.kind = fns[i].kind;
    I.d = d;
    I.ncall = (uint64_t)cfgs[i].ncall;
    I.instance = cfgs[i].instance;
    I.tab_off = cells;
    I.edge_off = edges;
    I.bins_off = 2 * cells;
    I.alpha = cfgs[i].alpha;
    cells += d * b->N;
    edges += d * (b->N + 1);
    for (int a = 0; a < d; ++a) b->axis_map.push_back(make_int2(i, a));
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    b->fail(VEGAS_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    return bail(VEGAS_ECUDA);
  }
  // one shared-memory split for every kernel of the iteration (no SM
  // repartitioning between them)
  e = gv_prepare_aux_kernels();
  for (const void* f : {(const void*)gv::k_batch_finalize, (const void*)gv::k_batch_reset})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) {
    b->fail(VEGAS_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    return bail(VEGAS_ECUDA);
  }
  if (c0.stream) {
    b->stream = (cudaStream_t)c0.stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      b->fail(VEGAS_ECUDA, "stream: %s", cudaGetErrorString(e));
      return bail(VEGAS_ECUDA);
    }
    b->own_stream = true;
  }
  if (b->by_dim) {  // the streams and events of the dimension kernels' fork and join
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < vegas_batch::kAux && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&b->aux[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
      b->fail(VEGAS_ECUDA, "streams: %s", cudaGetErrorString(e));
      return bail(VEGAS_ECUDA);
    }
  }
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (gv_dev_malloc(p, bytes) == cudaSuccess) return true;
    b->fail(VEGAS_ENOMEM, "cudaMalloc(%zu) failed", bytes);
    return false;
  };
  if (!alloc((void**)&b->d_inst, sizeof(BatchInst) * n) || !alloc((void**)&b->d_axis, sizeof(int2) * b->axis_map.size()) ||
      !alloc((void**)&b->d_edges, sizeof(double) * edges) || !alloc((void**)&b->d_derived, sizeof(double) * b->derived.size()) ||
      !alloc((void**)&b->d_bins, sizeof(double) * 2 * cells) || !alloc((void**)&b->d_tab64, sizeof(double2) * cells) ||
      !alloc((void**)&b->d_tab32, sizeof(float2) * cells) || !alloc((void**)&b->d_st, sizeof(BatchState) * n) ||
      !alloc((void**)&b->d_head, (1 + gv::kBatchDM) * sizeof(int)))
    return bail(VEGAS_ENOMEM);
  if (gv_malloc_host(&b->h_st, sizeof(BatchState) * n) != cudaSuccess) {
    b->fail(VEGAS_ENOMEM, "cudaMallocHost failed");
    return bail(VEGAS_ENOMEM);
  }
  memset(b->h_st, 0, sizeof(BatchState) * n);
  std::vector<double> e0(edges);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < b->d[i]; ++a)
      for (int k = 0; k <= b->N; ++k) e0[b->inst[i].edge_off + a * (b->N + 1) + k] = (double)k / (double)b->N;
  e = cudaMemcpy(b->d_edges, e0.data(), sizeof(double) * edges, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_derived, b->derived.data(), sizeof(double) * b->derived.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_axis, b->axis_map.data(), sizeof(int2) * b->axis_map.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_st, b->h_st, sizeof(BatchState) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_bins, 0, sizeof(double) * 2 * cells);
  if (e != cudaSuccess) {
    b->fail(VEGAS_ECUDA, "batch upload: %s", cudaGetErrorString(e));
    return bail(VEGAS_ECUDA);
  }
  // the (e_k, Delta_k) cells of every instance: one table kernel per axis run
  for (int i = 0; i < n; ++i) {
    e = gv_launch_tables(b->d_edges + b->inst[i].edge_off, b->d[i], b->N, b->d_tab64 + b->inst[i].tab_off,
                         b->d_tab32 + b->inst[i].tab_off, b->stream);
    if (e != cudaSuccess) {
      b->fail(VEGAS_ECUDA, "batch tables: %s", cudaGetErrorString(e));
      return bail(VEGAS_ECUDA);
    }
  }
  vegas_status st = configure(b);
  if (st) return bail(st);
  *out = b;
  return VEGAS_OK;
}

vegas_status vegas_batch_iterate(vegas_batch* b, int n_iter, int refine, vegas_result* out) {
  if (!b) return bfail("batch is NULL");
  if (n_iter < 0 || n_iter > gv::kBatchHist) return b->fail(VEGAS_EINVAL, "n_iter outside 0..%d", gv::kBatchHist);
  if (n_iter > 0) {
    auto key = std::make_pair(n_iter, refine ? 1 : 0);
    auto itg = b->graphs.find(key);
    cudaGraphExec_t ge = nullptr;
    if (itg != b->graphs.end()) {
      ge = itg->second;
    } else {
      cudaGraph_t g = nullptr;
      BK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      vegas_status st = VEGAS_OK;
      for (int i = 0; i < n_iter && !st; ++i) st = launch_iteration(b, refine ? 1 : 0, 1);
      cudaError_t e = cudaStreamEndCapture(b->stream, &g);
      if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return b->fail(VEGAS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return b->fail(VEGAS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
      b->graphs[key] = ge;
    }
    BK(b, cudaGraphLaunch(ge, b->stream));
  }
  if (out) {
    vegas_status st = read_states(b);
    if (st) return st;
    for (int i = 0; i < b->n; ++i) {
      const BatchState& s = b->h_st[i];
      out[i].I = s.I;
      out[i].sigma = s.sigma;
      out[i].chi2_dof = s.chi2;
      out[i].iters_done = s.nhist;
      out[i].stopped = 0;
      out[i].nonfinite = s.nonfinite;
      out[i].samples = s.samples;
    }
  }
  return VEGAS_OK;
}

vegas_status vegas_batch_reset(vegas_batch* b) {
  if (!b) return bfail("batch is NULL");
  gv::k_batch_reset<<<b->n, 128, 0, b->stream>>>(b->d_st, b->d_inst, b->n, b->N, b->d_edges, b->d_tab64,
                                                   b->d_tab32, b->d_head);
  BK(b, cudaGetLastError());
  return VEGAS_OK;
}

vegas_status vegas_batch_get_grid(vegas_batch* b, int i, double* edges, double* bin_sums) {
  if (!b) return bfail("batch is NULL");
  if (i < 0 || i >= b->n) return b->fail(VEGAS_EINVAL, "instance %d out of range", i);
  const BatchInst& I = b->inst[i];
  if (edges)
    BK(b, cudaMemcpyAsync(edges, b->d_edges + I.edge_off, sizeof(double) * I.d * (b->N + 1), cudaMemcpyDeviceToHost,
                          b->stream));
  if (bin_sums)
    BK(b, cudaMemcpyAsync(bin_sums, b->d_bins + I.bins_off, sizeof(double) * 2 * I.d * b->N, cudaMemcpyDeviceToHost,
                          b->stream));
  BK(b, cudaStreamSynchronize(b->stream));
  return VEGAS_OK;
}

vegas_status vegas_batch_get_history(vegas_batch* b, int i, double* hist, int max_iters, int* n_out) {
  if (!b) return bfail("batch is NULL");
  if (i < 0 || i >= b->n) return b->fail(VEGAS_EINVAL, "instance %d out of range", i);
  vegas_status st = read_states(b);
  if (st) return st;
  const int n = std::min(b->h_st[i].nhist, std::max(0, max_iters));
  if (n_out) *n_out = b->h_st[i].nhist;
  if (hist && n > 0) memcpy(hist, b->h_st[i].hist, sizeof(double) * 2 * n);
  return VEGAS_OK;
}

vegas_status vegas_batch_set_params(vegas_batch* b, int first, int count, const double* params, int stride) {
  if (!b) return bfail("batch is NULL");
  if (first < 0 || count < 1 || first > b->n - count || !params)
    return b->fail(VEGAS_EINVAL, "instances %d..%d outside the batch of %d, or params NULL", first, first + count - 1,
                   b->n);
  constexpr int K = gv::kNumDerived;
  std::vector<double> dv((size_t)count * K, 0.0);
  for (int j = 0; j < count; ++j) {
    const int i = first + j;
    const int np = (int)b->params[i].size();
    if (np > stride) return b->fail(VEGAS_EINVAL, "stride %d below the %d parameters of instance %d", stride, np, i);
    double scale = 1.0;
    std::string why;
    if (!gv::derive_params(b->kind[i], b->d[i], params + (size_t)j * stride, &dv[(size_t)j * K], &scale, &why))
      return b->fail(VEGAS_EINVAL, "instance %d: %s", i, why.c_str());
  }
  if (!b->h_derived && gv_malloc_host(&b->h_derived, b->derived.size() * sizeof(double)) != cudaSuccess) {
    b->h_derived = nullptr;
    return b->fail(VEGAS_ENOMEM, "cudaMallocHost failed (parameter staging)");
  }
  BK(b, cudaStreamSynchronize(b->stream));  // the staging's previous upload has left it
  for (int j = 0; j < count; ++j) {
    const double* p = params + (size_t)j * stride;
    b->params[first + j].assign(p, p + b->params[first + j].size());
  }
  std::copy(dv.begin(), dv.end(), b->derived.begin() + (size_t)first * K);
  std::copy(dv.begin(), dv.end(), b->h_derived + (size_t)first * K);
  BK(b, cudaMemcpyAsync(b->d_derived + (size_t)first * K, b->h_derived + (size_t)first * K, dv.size() * sizeof(double),
                        cudaMemcpyHostToDevice, b->stream));
  return VEGAS_OK;
}

vegas_status vegas_batch_set_launch(vegas_batch* b, int threads, int rounds) {
  if (!b) return bfail("batch is NULL");
  if (threads < 64 || threads > 256 || threads % 32 || rounds < 1 || rounds > 4096)
    return b->fail(VEGAS_EINVAL, "threads must be 64..256 (multiple of 32), rounds 1..4096");
  BK(b, cudaStreamSynchronize(b->stream));
  b->threads = threads;
  b->rounds = rounds;
  return configure(b);
}

vegas_status vegas_batch_set_tile(vegas_batch* b, int points_per_thread) {
  if (!b) return bfail("batch is NULL");
  const int hi = b->by_dim ? 2 : 4;
  if (points_per_thread < 0 || points_per_thread > hi)
    return b->fail(VEGAS_EINVAL, "points_per_thread must be in 0..%d (0: automatic)", hi);
  BK(b, cudaStreamSynchronize(b->stream));
  const int p0 = b->ppt_req;
  b->ppt_req = points_per_thread;
  vegas_status st = configure(b);
  if (st) {
    b->ppt_req = p0;
    configure(b);
  }
  return st;
}

vegas_status vegas_batch_get_tile(vegas_batch* b, int* points_per_thread, int* cap) {
  if (!b) return bfail("batch is NULL");
  if (points_per_thread) *points_per_thread = b->ppt;
  if (cap) *cap = b->cap;
  return VEGAS_OK;
}

vegas_status vegas_batch_get_launch(vegas_batch* b, int* threads, int* rounds, int* ctas, int* items) {
  if (!b) return bfail("batch is NULL");
  if (threads) *threads = b->threads;
  if (rounds) *rounds = b->rounds;
  if (ctas) *ctas = b->ctas;
  if (items) *items = (int)b->items.size();
  return VEGAS_OK;
}

vegas_status vegas_batch_profile(vegas_batch* b, int n_pass, double* ms) {
  if (!b) return bfail("batch is NULL");
  if (n_pass < 1 || !ms) return b->fail(VEGAS_EINVAL, "need n_pass >= 1 and ms[2]");
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) BK(b, cudaEventCreate(&ev[i]));
  double acc[2] = {0.0, 0.0};
  vegas_status st = VEGAS_OK;
  for (int p = 0; p < n_pass && !st; ++p) {
    BatchArgs A = batch_args(b, 0, 0);
    cudaEventRecord(ev[0], b->stream);
    st = launch_sample(b, A);
    cudaEventRecord(ev[1], b->stream);
    if (!st) {
      gv::k_batch_finalize<<<A.naxes + A.n, 128, 0, b->stream>>>(A);
      if (cudaGetLastError() != cudaSuccess) st = b->fail(VEGAS_ECUDA, "finalize launch failed");
    }
    cudaEventRecord(ev[2], b->stream);
    cudaEventSynchronize(ev[2]);
    float t0 = 0.f, t1 = 0.f;
    cudaEventElapsedTime(&t0, ev[0], ev[1]);
    cudaEventElapsedTime(&t1, ev[1], ev[2]);
    acc[0] += t0;
    acc[1] += t1;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  if (st) return st;
  ms[0] = acc[0] / n_pass;
  ms[1] = acc[1] / n_pass;
  return VEGAS_OK;
}

vegas_status vegas_batch_autotune(vegas_batch* b, int* threads, int* rounds, double* ms) {
  if (!b) return bfail("batch is NULL");
  static const int kThreads[] = {128, 256};
  static const int kRounds[] = {8, 16, 32, 64, 128};
  struct Cand {
    int t, r, p, pol;
    double ms;
  };
  std::vector<Cand> cands;
  // one warm-up pass, then the mean of n passes, for shape (t, r), tile p
  // (the per-dimension kernels: points in flight) and capacity policy pol
  // (0: the largest capacity of the range, 1: the smallest, 2: the dense
  // floor, per-dimension kernels only)
  auto time_shape = [&](int t, int r, int p, int pol, int n, double* out) -> vegas_status {
    b->small_cap = pol >= 1;
    b->dense_cap = pol == 2;
    b->ppt_req = p;
    vegas_status st = vegas_batch_set_launch(b, t, r);
    double m[2];
    if (!st) st = vegas_batch_profile(b, 1, m);
    if (!st) st = vegas_batch_profile(b, n, m);
    if (!st) *out = m[0];
    return st;
  };
  const std::vector<int> tiles = b->by_dim ? std::vector<int>{1, 2} : std::vector<int>{0};
  for (int t : kThreads)
    for (int r : kRounds)
      for (int p : tiles) {
        int cap_large = -1;  // a repeated tile is not timed twice
        for (int pol = 0; pol < (b->by_dim ? 3 : 2); ++pol) {
          double m = 0.0;
          vegas_status st = time_shape(t, r, p, pol, 3, &m);
          if (st) return st;
          if (pol == 1 && b->cap == cap_large) continue;
          if (pol == 0) cap_large = b->cap;
          cands.push_back({t, r, p, pol, m});
        }
      }
  // the three fastest again in interleaved rounds, keeping each one's best
  std::sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& c) { return a.ms < c.ms; });
  cands.resize(std::min<size_t>(cands.size(), 3));
  for (int k = 0; k < 3; ++k)
    for (Cand& c : cands) {
      double m = 0.0;
      vegas_status st = time_shape(c.t, c.r, c.p, c.pol, 3, &m);
      if (st) return st;
      c.ms = k == 0 ? m : std::min(c.ms, m);
    }
  const Cand best = *std::min_element(cands.begin(), cands.end(),
                                      [](const Cand& a, const Cand& c) { return a.ms < c.ms; });
  b->small_cap = best.pol >= 1;
  b->dense_cap = best.pol == 2;
  b->ppt_req = best.p;
  vegas_status st = vegas_batch_set_launch(b, best.t, best.r);
  if (st) return st;
  if (threads) *threads = best.t;
  if (rounds) *rounds = best.r;
  if (ms) *ms = best.ms;
  return VEGAS_OK;
}

}  // extern "C"
