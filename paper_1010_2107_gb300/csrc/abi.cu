// abi.cu -- host side of the C ABI declared in include/gvegas.h: context
// lifetime, derived integrand constants, launch geometry, the per-iteration
// kernel sequence (captured once into a CUDA graph per call shape) and the
// result read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"
#include "integrands.cuh"
#include "kernels.h"

using gv::GState;

static_assert(GVEGAS_MAXUSERPARAMS == gv::kNumDerived, "user parameters fill the derived-constant block");

namespace {

thread_local std::string g_thread_err;

std::string vformat(const char* fmt, va_list ap) {
  char buf[512];
  va_list ap2;
  va_copy(ap2, ap);
  const int n = vsnprintf(buf, sizeof buf, fmt, ap);
  if (n < (int)sizeof buf) {
    va_end(ap2);
    return std::string(buf);
  }
  std::string big((size_t)n + 1, '\0');
  vsnprintf(&big[0], big.size(), fmt, ap2);
  va_end(ap2);
  big.resize((size_t)n);
  return big;
}

// Allocation wrappers.  g_alloc_left: allocations still allowed before an
// injected failure (-1: none armed); the failing call returns
// cudaErrorMemoryAllocation without calling the allocator and disarms.
std::atomic<long long> g_alloc_left{-1};
std::atomic<unsigned long long> g_alloc_count{0};

bool injected_failure() {
  long long left = g_alloc_left.load();
  while (left >= 0)
    if (g_alloc_left.compare_exchange_weak(left, left - 1)) return left == 0;
  return false;
}

}  // namespace

extern "C" cudaError_t gv_dev_malloc(void** p, size_t bytes) {
  g_alloc_count.fetch_add(1);
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

extern "C" cudaError_t gv_host_malloc(void** p, size_t bytes) {
  g_alloc_count.fetch_add(1);
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

extern "C" void vegas_fail_alloc_after(int64_t n) { g_alloc_left.store(n < 0 ? -1 : (long long)n); }

extern "C" uint64_t vegas_alloc_count(void) { return (uint64_t)g_alloc_count.load(); }

struct vegas_ctx {
  vegas_config cfg{};
  int kind = 0;
  std::vector<double> params;            // integrand parameters as given
  double derived[gv::kNumDerived] = {};  // device constants (see integrands.cuh)
  double scale = 1.0;                    // output scale applied in k_reduce
  int prec = VG_FP64;
  int ybits = 53;
  int g = 1;
  uint64_t ncubes = 1, nc = 0;
  int strat = 0;
  gv::KernelEntry ke{};
  int sm_count = 0;
  // launch geometry
  int threads = 256, ctas_per_sm_req = 0, ctas = 0, lanes = 1, lanes_req = 0, occ = 0;
  int cap = 16;  // histogram bucket capacity (see sample_kernel.cuh)
  int ctas_nb = 0;      // CTAs of a pass without the per-bin histogram
  size_t smem_nb = 0;   // and its dynamic shared memory
  int ppt = 1, ppt_req = 0, ppt_min = 1;  // points per thread per histogram tile
  bool small_cap = false;                 // tile capacity policy (gv::choose_tile)
  size_t smem = 0;
  // device buffers
  double* d_edges = nullptr;
  double2* d_tab64 = nullptr;
  float2* d_tab32 = nullptr;
  double* d_derived = nullptr;
  double* d_part_bins = nullptr;
  double* d_part_tot = nullptr;
  int part_rows = 0;
  double* d_bins = nullptr;
  double* d_tot = nullptr;
  double* d_cubes = nullptr;
  double* d_cube_max = nullptr;  // [G] max(0, largest w) per cube, integration phase
  bool have_max = false;         // a bases_integrate has recorded the maxima
  // SPRING buffers (grown on demand)
  uint64_t* d_q = nullptr;
  uint64_t* d_prefix = nullptr;
  double* d_mt = nullptr;          // [G] cube bounds q_c / scale
  float* d_mt32 = nullptr;         // [G] the same in FP32
  uint32_t* d_guide = nullptr;     // guide table of the cube search
  double* d_bmax = nullptr;        // per-block maxima and sums of the table kernels
  unsigned long long* d_bsum = nullptr;
  double* d_meta = nullptr;        // {Q, scale, status}
  double* d_stage_x = nullptr;     // [n][d]
  uint64_t* d_stage_t = nullptr;   // [n]
  double* d_out_x = nullptr;
  uint64_t* d_out_t = nullptr;
  uint32_t* d_counts = nullptr;
  unsigned long long* d_counters = nullptr;
  uint32_t spring_cap = 0, spring_chunks_cap = 0;
  cudaEvent_t spring_timer[2] = {nullptr, nullptr};  // set by spring_profile around the trial kernel
  double* d_gpart = nullptr;  // adjoint partials [grad_nt + 2][grad_ctas] then totals
  int grad_ctas = 0;
  size_t grad_smem = 0;
  GState* d_st = nullptr;
  // host staging (pinned)
  GState* h_st = nullptr;
  double* h_stage = nullptr;
  size_t h_stage_len = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // graph cache, keyed by (shape, n1, n2, refine, acc1, acc2)
  std::map<std::tuple<int, int, int, int, double, double>, cudaGraphExec_t> graphs;
  int hist_upper = 0;  // upper bound of the window length (host shadow)
  std::string err;

  vegas_status fail(vegas_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    err = vformat(fmt, ap);
    va_end(ap);
    g_thread_err = err;
    return st;
  }
};

namespace {

vegas_status thread_fail(vegas_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  g_thread_err = vformat(fmt, ap);
  va_end(ap);
  return st;
}

#define CK(ctx, call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return (ctx)->fail(e_ == cudaErrorMemoryAllocation ? VEGAS_ENOMEM : VEGAS_ECUDA, \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,    \
                         __LINE__);                                                    \
  } while (0)

bool lookup_kernel(int kind, int prec, int ybits, int d, gv::KernelEntry* e) {
  const bool y24 = ybits == 24;
  switch (kind) {
    case VG_GENZ_GAUSSIAN:
      return y24 ? gv::entries_genz_gaussian_y24(prec, d, e) : gv::entries_genz_gaussian_y53(prec, d, e);
    case VG_GENZ_PRODUCT_PEAK:
      return y24 ? gv::entries_genz_product_peak_y24(prec, d, e) : gv::entries_genz_product_peak_y53(prec, d, e);
    case VG_GENZ_CORNER_PEAK:
      return y24 ? gv::entries_genz_corner_peak_y24(prec, d, e) : gv::entries_genz_corner_peak_y53(prec, d, e);
    case VG_GENZ_OSCILLATORY:
      return y24 ? gv::entries_genz_oscillatory_y24(prec, d, e) : gv::entries_genz_oscillatory_y53(prec, d, e);
    case VG_DOUBLE_GAUSSIAN:
      return y24 ? gv::entries_dgauss_y24(prec, d, e) : gv::entries_dgauss_y53(prec, d, e);
    case VG_RAMBO_BW:
      return y24 ? gv::entries_rambo_y24(prec, d, e) : gv::entries_rambo_y53(prec, d, e);
    case VG_W_MUNU:
      return y24 ? gv::entries_wmunu_y24(prec, d, e) : gv::entries_wmunu_y53(prec, d, e);
    case VG_GENZ_CONTINUOUS:
      return y24 ? gv::entries_genz_continuous_y24(prec, d, e) : gv::entries_genz_continuous_y53(prec, d, e);
    case VG_GENZ_DISCONTINUOUS:
      return y24 ? gv::entries_genz_discontinuous_y24(prec, d, e)
                 : gv::entries_genz_discontinuous_y53(prec, d, e);
    default: return false;
  }
}

void destroy_graphs(vegas_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// Launch geometry: a persistent grid of CTAs per SM as occupancy allows
// (or as requested), capped by the work available.
// SPRING table, in four small kernels over blocks of kSpan cubes (every
// FP64 operation of a cube is the oracle's, in the oracle's order; the
// integer sums are exact in any order):
//   k_spring_max      per-block maxima of M_c = cmax_c * out_scale;
//   k_spring_weights  M = the largest M_c, scale = 2^24 / M,
//                     q_c = ceil(M_c scale), the bound mt_c = q_c / scale,
//                     per-block sums of q;
//   k_spring_scan     (one block) exclusive scan of the block sums,
//                     P[G] = Q, meta = {Q, scale, status} (status 1: no
//                     positive maximum);
//   k_spring_prefix   exclusive prefix sums P[0..G) in 64-bit integers;
//   k_spring_guide    the guide table (Chen and Asau): for each of the 2^gk
//                     equal intervals of [0, Q), guide[j] = the last cube c
//                     with P[c] <= floor(j Q / 2^gk); guide[2^gk] = G - 1.
constexpr int kSpanThreads = 256, kSpanPer = 4;
constexpr uint32_t kSpan = kSpanThreads * kSpanPer;  // cubes per block

__device__ double block_max_d(double m, double* sm) {
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  double M = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = fmax(M, sm[w]);
  return M;
}

__global__ void __launch_bounds__(kSpanThreads) k_spring_max(const double* cmax, uint32_t G, double out_scale,
                                                             double* bmax) {
  __shared__ double sm[32];
  const uint32_t lo = blockIdx.x * kSpan, hi = min(lo + kSpan, G);
  double m = 0.0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) m = fmax(m, cmax[i] * out_scale);
  m = block_max_d(m, sm);
  if (threadIdx.x == 0) bmax[blockIdx.x] = m;
}

// The largest of the block maxima (any order: max is exact).
__device__ double spring_global_max(const double* bmax, uint32_t nb, double* sm) {
  double m = 0.0;
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, bmax[i]);
  return block_max_d(m, sm);
}

__global__ void __launch_bounds__(kSpanThreads) k_spring_weights(const double* cmax, uint32_t G, double out_scale,
                                                                 const double* bmax, uint32_t nb, uint64_t* q,
                                                                 double* mt, float* mt32, unsigned long long* bsum) {
  __shared__ double sm[32];
  __shared__ unsigned long long ss[32];
  const double M = spring_global_max(bmax, nb, sm);
  if (!(M > 0.0) || !isfinite(M)) return;  // k_spring_scan reports it
  const double scale = 16777216.0 / M;
  const uint32_t lo = blockIdx.x * kSpan, hi = min(lo + kSpan, G);
  unsigned long long sum = 0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double v = cmax[i] * out_scale;
    const uint64_t qi = v > 0.0 ? (uint64_t)ceil(v * scale) : 0ull;
    q[i] = qi;
    const double b = (double)qi / scale;  // the cube's bound in the integrand's units
    mt[i] = b;
    mt32[i] = (float)b;
    sum += qi;
  }
  for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
  if ((threadIdx.x & 31) == 0) ss[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ss[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_spring_scan(const double* bmax, uint32_t nb, unsigned long long* bsum,
                                                      uint32_t G, uint64_t* prefix, double* meta) {
  __shared__ double sm[32];
  __shared__ unsigned long long ssum[1024];
  const double M = spring_global_max(bmax, nb, sm);
  const int tid = threadIdx.x, nt = blockDim.x;
  if (!(M > 0.0) || !isfinite(M)) {
    if (tid == 0) {
      meta[0] = 0.0;
      meta[1] = 0.0;
      meta[2] = 1.0;
    }
    return;
  }
  // exclusive scan of bsum[0..nb) in place: contiguous runs per thread
  const uint32_t per = (nb + nt - 1) / nt, lo = min((uint32_t)tid * per, nb), hi = min(lo + per, nb);
  unsigned long long sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += bsum[i];
  ssum[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    unsigned long long run = 0;
    for (int k = 0; k < nt; ++k) {
      const unsigned long long v = ssum[k];
      ssum[k] = run;
      run += v;
    }
    prefix[G] = run;
    meta[0] = (double)run;
    meta[1] = 16777216.0 / M;
    meta[2] = 0.0;
  }
  __syncthreads();
  unsigned long long run = ssum[tid];
  for (uint32_t i = lo; i < hi; ++i) {
    const unsigned long long v = bsum[i];
    bsum[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kSpanThreads) k_spring_prefix(const uint64_t* q, uint32_t G,
                                                                const unsigned long long* boff, uint64_t* prefix,
                                                                const double* meta) {
  __shared__ unsigned long long sw[32];
  if (meta[2] != 0.0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lo = blockIdx.x * kSpan + (uint32_t)tid * kSpanPer;
  uint64_t v[kSpanPer];
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < kSpanPer; ++k) {
    v[k] = lo + k < G ? q[lo + k] : 0ull;
    s += v[k];
  }
  // exclusive scan of the thread sums: within the warp, then over the warps
  unsigned long long inc = s;
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += o;
  }
  if (lane == 31) sw[warp] = inc;
  __syncthreads();
  unsigned long long run = boff[blockIdx.x] + inc - s;
  for (int w = 0; w < warp; ++w) run += sw[w];
#pragma unroll
  for (int k = 0; k < kSpanPer; ++k) {
    const uint32_t i = lo + k;
    if (i < G) prefix[i] = run;
    run += v[k];
  }
}

// One guide entry per thread: the interval start b_j = floor(j Q / 2^gk)
// from the 128-bit product, then the last cube with P[c] <= b_j by
// bisection (P[0] = 0 <= b_j always).
__global__ void __launch_bounds__(256) k_spring_guide(const uint64_t* prefix, uint32_t G, uint32_t gk,
                                                      uint32_t* guide, const double* meta) {
  if (meta[2] != 0.0) return;
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > (1u << gk)) return;
  const uint64_t Q = prefix[G];
  const uint64_t plo = (uint64_t)j * Q, phi = __umul64hi((uint64_t)j, Q);
  const uint64_t b = gk ? ((phi << (64 - gk)) | (plo >> gk)) : plo;
  uint32_t lo = 0, hi = G;
  while (hi - lo > 1) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (prefix[mid] <= b)
      lo = mid;
    else
      hi = mid;
  }
  guide[j] = lo;
}

// SPRING compaction: block k copies chunk k's kept points behind those of
// chunks 0 .. k-1 (trial order).
__global__ void k_spring_compact(const uint32_t* counts, uint32_t chunk, int d, const double* sx, const uint64_t* st,
                                 double* ox, uint64_t* ot) {
  __shared__ unsigned long long part[32];
  const uint32_t k = blockIdx.x;
  unsigned long long o = 0;
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) o += counts[i];
  for (int off = 16; off > 0; off >>= 1) o += __shfl_xor_sync(0xffffffffu, o, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = o;
  __syncthreads();
  unsigned long long off = 0;
  for (uint32_t w = 0; w < blockDim.x / 32; ++w) off += part[w];
  const uint32_t n = counts[k];
  const size_t src = (size_t)k * chunk;
  for (uint32_t i = threadIdx.x; i < n * (uint32_t)d; i += blockDim.x) ox[off * d + i] = sx[src * d + i];
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) ot[off + i] = st[src + i];
}

vegas_status configure_launch(vegas_ctx* c) {
  const int d = c->cfg.ndim, N = c->cfg.nbins;
  // Histogram tile (gv::choose_tile): points per thread between gathers and
  // bucket capacity, against the CTAs per SM each leaves resident.
  cudaError_t e = cudaSuccess;
  auto occ_of = [&](int cap, int) -> int {
    const size_t smem = c->ke.smem(d, N, cap);
    int o = 0;
    if (e != cudaSuccess || smem > 227 * 1024) return 0;
    e = gv_raise_smem_limit(c->ke.sample, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, c->ke.sample, c->threads, smem);
    return e == cudaSuccess ? o : 0;
  };
  int occ_cap = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cap, c->ke.sample, c->threads, 0);
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
  const gv::TileShape t = gv::choose_tile(c->threads, N, c->ppt_req, c->ppt_min, occ_cap, occ_of, c->small_cap);
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
  if (t.occ < 1) return c->fail(VEGAS_EINVAL, "sampling kernel does not fit: %d threads, %d points per thread",
                                c->threads, t.ppt);
  // the limit covers the chosen size (it only grows: see gv_raise_smem_limit)
  c->smem = c->ke.smem(d, N, t.cap);
  e = gv_raise_smem_limit(c->ke.sample, c->smem);
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
  c->cap = t.cap;
  c->ppt = t.ppt;
  const int occ = t.occ;
  c->occ = occ;
  const int per_sm = c->ctas_per_sm_req > 0 ? std::min(c->ctas_per_sm_req, occ) : occ;
  const int64_t cap_ctas = (int64_t)c->sm_count * per_sm;
  uint64_t units;
  if (c->strat) {
    // lanes per hypercube: the best balance of rounds and chain length
    int L = gv::choose_lanes(c->ncubes, c->nc, c->threads, cap_ctas);
    if (c->lanes_req > 0) L = std::min<int>(c->lanes_req, (int)std::min<uint64_t>(32, c->nc));
    int Lp = 1;
    while (2 * Lp <= L) Lp *= 2;
    c->lanes = Lp;
    units = c->ncubes * (uint64_t)Lp;
  } else {
    c->lanes = 1;
    units = (uint64_t)c->cfg.ncall;
  }
  int64_t ctas = (int64_t)((units + c->threads - 1) / c->threads);
  c->ctas = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, cap_ctas));
  // passes without the per-bin histogram (no refinement) need only the
  // grid table and constants in shared memory: more CTAs may be resident
  c->smem_nb = c->ke.smem_nobins(d, N);
  int occ_nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_nb, c->ke.sample, c->threads, c->smem_nb);
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
  occ_nb = std::max(occ_nb, per_sm);
  if (c->ctas_per_sm_req > 0) occ_nb = std::min(occ_nb, std::max(c->ctas_per_sm_req, per_sm));
  c->ctas_nb = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)c->sm_count * occ_nb));
  const int rows = std::max(c->ctas, c->ctas_nb);
  if (rows > c->part_rows) {
    if (c->d_part_bins) cudaFree(c->d_part_bins);
    if (c->d_part_tot) cudaFree(c->d_part_tot);
    c->d_part_bins = nullptr;
    c->d_part_tot = nullptr;
    c->part_rows = 0;
    CK(c, gv_malloc(&c->d_part_bins, sizeof(double) * 2 * (size_t)d * N * rows));
    CK(c, gv_malloc(&c->d_part_tot, sizeof(double) * gv::kTotCols * (size_t)rows));
    c->part_rows = rows;
  }
  destroy_graphs(c);
  return VEGAS_OK;
}

gv::SampleArgs sample_args(const vegas_ctx* c, int it_override, bool nobins = false) {
  gv::SampleArgs A{};
  A.nobins = nobins;
  A.d = c->cfg.ndim;
  A.N = c->cfg.nbins;
  A.g = c->g;
  A.ybits = c->ybits;
  A.lanes = c->lanes;
  A.cap = c->cap;
  A.ppt = c->ppt;
  A.strat = c->strat;
  A.key0 = (uint32_t)c->cfg.seed;
  A.key1 = (uint32_t)(c->cfg.seed >> 32);
  gv::philox_key_schedule(A.key0, A.key1, A.ks);
  A.instance = c->cfg.instance;
  A.it_override = it_override;
  A.ncall = (uint64_t)c->cfg.ncall;
  A.nc = (uint32_t)c->nc;
  A.ncubes = (uint32_t)c->ncubes;
  const bool cubes_pow2 = (c->ncubes & (c->ncubes - 1)) == 0;
  A.cube_mul = (c->strat && cubes_pow2 && c->ncubes > 1) ? 0x9E3779B1u : 1u;
  A.g_pow2 = (c->g & (c->g - 1)) == 0;
  A.g_log2 = 0;
  while ((1 << A.g_log2) < c->g) ++A.g_log2;
  A.t32 = (int64_t)c->g * c->cfg.nbins <= 256;
  const double gb = (double)c->g * std::ldexp(1.0, c->ybits);
  A.inv_gb_d = 1.0 / gb;
  A.inv_gb_f = (float)(1.0 / gb);
  A.inv_nc = c->nc > 0 ? 1.0 / (double)c->nc : 0.0;
  A.inv_nc1 = c->nc > 1 ? 1.0 / (double)(c->nc - 1) : 0.0;
  A.nparts = nobins ? c->ctas_nb : c->ctas;
  A.tab = c->prec == VG_FP64 ? (const void*)c->d_tab64 : (const void*)c->d_tab32;
  A.dparams = c->d_derived;
  A.st = c->d_st;
  A.part_bins = c->d_part_bins;
  A.part_tot = c->d_part_tot;
  A.cubes = c->d_cubes;
  return A;
}

gv::FinArgs fin_args(const vegas_ctx* c, int refine, int record, bool nobins = false) {
  gv::FinArgs F{};
  F.d = c->cfg.ndim;
  F.N = c->cfg.nbins;
  F.nobins = nobins;
  F.nparts = nobins ? c->ctas_nb : c->ctas;
  F.strat = c->strat;
  F.refine = refine;
  F.record = record;
  F.pair32 = c->prec == VG_FP32_ACCCOMP;
  F.ncall = (uint64_t)c->cfg.ncall;
  F.ncubes = c->ncubes;
  F.scale = c->d_derived + gv::kNumDerived;
  F.alpha = c->cfg.alpha;
  F.part_bins = c->d_part_bins;
  F.part_tot = c->d_part_tot;
  F.bins = c->d_bins;
  F.tot = c->d_tot;
  F.edges = c->d_edges;
  F.tab64 = c->d_tab64;
  F.tab32 = c->d_tab32;
  F.st = c->d_st;
  return F;
}

// One pass of steps 2-6 on the context stream.  A pass that does not
// refine the grid skips the per-bin histogram, whose sums only step 5
// reads (`nobins`), unless the caller wants them.
vegas_status launch_pass(vegas_ctx* c, int it_override, int refine, int record, bool record_max = false,
                         bool nobins = false) {
  if (refine) nobins = false;
  gv::SampleArgs A = sample_args(c, it_override, nobins);
  if (record_max) A.cube_max = c->d_cube_max;
  void* args[] = {&A};
  CK(c, cudaLaunchKernel(c->ke.sample, dim3(nobins ? c->ctas_nb : c->ctas), dim3(c->threads), args,
                         nobins ? c->smem_nb : c->smem, c->stream));
  gv::FinArgs F = fin_args(c, refine, record, nobins);
  CK(c, gv_launch_finish(&F, c->stream));
  return VEGAS_OK;
}

// Graph of one call.  shape 0 (vegas_iterate): set the ACC target, then n1
// passes (refining if `refine`).  shape 1 (bases_integrate): reset the
// window, n1 refining passes at acc1, snapshot phase 1, reset, n2 frozen-grid
// passes at acc2.  Each call shape is captured once and replayed.
vegas_status get_graph(vegas_ctx* c, int shape, int n1, int n2, int refine, double acc1, double acc2,
                       cudaGraphExec_t* out) {
  auto key = std::make_tuple(shape, n1, n2, refine, acc1, acc2);
  auto itg = c->graphs.find(key);
  if (itg != c->graphs.end()) {
    *out = itg->second;
    return VEGAS_OK;
  }
  cudaGraph_t g = nullptr;
  CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  vegas_status st = VEGAS_OK;
  auto ctl = [&](int ops, double acc) {
    if (st) return;
    cudaError_t e = gv_launch_control(c->d_st, ops, acc, 0u, c->stream);
    if (e != cudaSuccess) st = c->fail(VEGAS_ECUDA, "control: %s", cudaGetErrorString(e));
  };
  if (shape == 0) {
    ctl(gv::CTL_SET_ACC, acc1);
    for (int i = 0; i < n1 && !st; ++i) st = launch_pass(c, -1, refine, 1, false, !refine);
  } else {
    ctl(gv::CTL_RESET_WINDOW | gv::CTL_SET_ACC, acc1);
    for (int i = 0; i < n1 && !st; ++i) st = launch_pass(c, -1, 1, 1);
    ctl(gv::CTL_SNAPSHOT | gv::CTL_RESET_WINDOW | gv::CTL_SET_ACC, acc2);
    // the integration phase records the per-cube maxima that SPRING uses
    if (!st && cudaMemsetAsync(c->d_cube_max, 0, sizeof(double) * c->ncubes, c->stream) != cudaSuccess)
      st = c->fail(VEGAS_ECUDA, "cube maxima reset");
    for (int i = 0; i < n2 && !st; ++i) st = launch_pass(c, -1, 0, 1, true, true);
  }
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (st != VEGAS_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  if (c->graphs.size() >= 64) destroy_graphs(c);
  c->graphs[key] = ge;
  *out = ge;
  return VEGAS_OK;
}

vegas_status read_state(vegas_ctx* c) {
  CK(c, cudaMemcpyAsync(c->h_st, c->d_st, offsetof(GState, hist), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return VEGAS_OK;
}

void fill_result(const vegas_ctx* c, vegas_result* r) {
  const GState* s = c->h_st;
  r->I = s->I;
  r->sigma = s->sigma;
  r->chi2_dof = s->chi2;
  r->iters_done = s->nhist;
  r->stopped = s->stopped;
  r->nonfinite = s->nonfinite;
  r->samples = s->samples;
}

vegas_status stage(vegas_ctx* c, size_t n) {
  if (n <= c->h_stage_len) return VEGAS_OK;
  CK(c, cudaStreamSynchronize(c->stream));  // no copy may still read the old buffer
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->h_stage_len = 0;
  CK(c, gv_malloc_host(&c->h_stage, n * sizeof(double)));
  c->h_stage_len = n;
  return VEGAS_OK;
}

vegas_status upload_grid(vegas_ctx* c, const double* edges) {
  const int d = c->cfg.ndim, N = c->cfg.nbins;
  const size_t n = (size_t)d * (N + 1);
  vegas_status st = stage(c, n);
  if (st) return st;
  CK(c, cudaStreamSynchronize(c->stream));  // staging buffer may still be in use
  memcpy(c->h_stage, edges, n * sizeof(double));
  CK(c, cudaMemcpyAsync(c->d_edges, c->h_stage, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(c, gv_launch_tables(c->d_edges, d, N, c->d_tab64, c->d_tab32, c->stream));
  return VEGAS_OK;  // stream-ordered; the next host write to the stage synchronises first
}

vegas_status upload_derived(vegas_ctx* c) {
  vegas_status st = stage(c, gv::kNumDerived + 1);
  if (st) return st;
  CK(c, cudaStreamSynchronize(c->stream));
  memcpy(c->h_stage, c->derived, sizeof c->derived);
  c->h_stage[gv::kNumDerived] = c->scale;  // the output scale follows the constants
  CK(c, cudaMemcpyAsync(c->d_derived, c->h_stage, sizeof c->derived + sizeof(double), cudaMemcpyHostToDevice,
                        c->stream));
  return VEGAS_OK;  // stream-ordered; the next host write to the stage synchronises first
}

bool valid_grid(const double* e, int d, int N) {
  for (int a = 0; a < d; ++a) {
    const double* r = e + (size_t)a * (N + 1);
    if (r[0] != 0.0 || r[N] != 1.0) return false;
    for (int k = 0; k < N; ++k)
      if (!(r[k + 1] > r[k])) return false;
  }
  return true;
}

// Checks on a configuration shared by every constructor: sizes, precision,
// random bits (ybits, resolved), and the stratification g^d | ncall.
vegas_status check_config(const vegas_config* cfg, int* ybits_out, int* g_out, uint64_t* G_out) {
  const int d = cfg->ndim, N = cfg->nbins;
  if (d < 1 || d > GVEGAS_MAXDIM) return thread_fail(VEGAS_EINVAL, "ndim %d outside 1..%d", d, GVEGAS_MAXDIM);
  if (N < 2 || N > GVEGAS_MAXBINS) return thread_fail(VEGAS_EINVAL, "nbins %d outside 2..%d", N, GVEGAS_MAXBINS);
  if (cfg->ncall < 2 || cfg->ncall > (int64_t)1 << 32)
    return thread_fail(VEGAS_EINVAL, "ncall %lld outside 2..2^32", (long long)cfg->ncall);
  if (cfg->precision < VG_FP64 || cfg->precision > VG_FP32_ACCCOMP)
    return thread_fail(VEGAS_EINVAL, "unknown precision %d", cfg->precision);
  const int ybits = cfg->ybits ? cfg->ybits : (cfg->precision == VG_FP64 ? 53 : 24);
  if (ybits != 24 && ybits != 53) return thread_fail(VEGAS_EINVAL, "ybits must be 24 or 53");
  if (!(cfg->alpha >= 0.0) || !std::isfinite(cfg->alpha)) return thread_fail(VEGAS_EINVAL, "alpha must be >= 0");
  const int g = cfg->nstrat < 1 ? 1 : cfg->nstrat;
  uint64_t G = 1;
  for (int a = 0; a < d; ++a) {
    G *= (uint64_t)g;
    if (G > (uint64_t)cfg->ncall) return thread_fail(VEGAS_EINVAL, "nstrat^ndim exceeds ncall");
  }
  if ((uint64_t)cfg->ncall % G != 0) return thread_fail(VEGAS_EINVAL, "ncall must be a multiple of nstrat^ndim");
  if (G > 1 && (uint64_t)cfg->ncall / G < 2) return thread_fail(VEGAS_EINVAL, "need >= 2 points per hypercube");
  if ((int64_t)g * N >= (ybits == 53 ? 2048 : (1 << 30)))
    return thread_fail(VEGAS_EINVAL, "nstrat * nbins too large for %d-bit sampling", ybits);
  *ybits_out = ybits;
  *g_out = g;
  *G_out = G;
  return VEGAS_OK;
}

vegas_ctx* new_context(const vegas_config* cfg, int ybits, int g, uint64_t G) {
  vegas_ctx* c = new vegas_ctx();
  c->cfg = *cfg;
  c->cfg.ybits = ybits;
  c->prec = cfg->precision;
  c->ybits = ybits;
  c->g = g;
  c->ncubes = G;
  c->nc = (uint64_t)cfg->ncall / G;
  c->strat = G > 1;
  return c;
}

// The specialised sampling kernel applies: d equal to the compile-time bound
// dm, 24-bit words, a power-of-two number of divisions with g N <= 256.
bool spec_shape(int d, int dm, int ybits, int g, int N) {
  return d == dm && ybits == 24 && (g & (g - 1)) == 0 && (int64_t)g * N <= 256;
}

// Second half of every constructor, for a context whose integrand, kernel
// entry and constants are set: device buffers, launch shape, uniform grid.
vegas_status finish_create(vegas_ctx* c, vegas_ctx** out) {
  const vegas_config* cfg = &c->cfg;
  const int d = cfg->ndim, N = cfg->nbins;
  const uint64_t G = c->ncubes;
  // the specialised kernel when the shape allows it (see kernels.h)
  if (c->ke.sample_spec && spec_shape(d, c->ke.dm, c->ybits, c->g, N)) {
    c->ke.sample = c->ke.sample_spec;
    c->ppt_min = c->ke.spec_ppt_min;
    if (c->ke.grad_spec) c->ke.grad = c->ke.grad_spec;
  }
  auto bail = [&](vegas_status st) {
    g_thread_err = c->err;
    vegas_destroy(c);
    return st;
  };
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(c->fail(VEGAS_ECUDA, "no CUDA device: %s", cudaGetErrorString(e)));
  e = gv_prepare_aux_kernels();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(c->ke.sample, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return bail(c->fail(VEGAS_ECUDA, "kernel attributes: %s", cudaGetErrorString(e)));
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(c->fail(VEGAS_ECUDA, "stream: %s", cudaGetErrorString(e)));
    c->own_stream = true;
  }
  auto alloc = [&](void** p, size_t bytes) -> vegas_status {
    cudaError_t ae = gv_dev_malloc(p, bytes);
    if (ae != cudaSuccess)
      return c->fail(VEGAS_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(ae));
    return VEGAS_OK;
  };
  vegas_status st = VEGAS_OK;
  if (!st) st = alloc((void**)&c->d_edges, sizeof(double) * d * (N + 1));
  if (!st) st = alloc((void**)&c->d_tab64, sizeof(double2) * d * N);
  if (!st) st = alloc((void**)&c->d_tab32, sizeof(float2) * d * N);
  if (!st) st = alloc((void**)&c->d_derived, sizeof c->derived + sizeof(double));  // + the output scale
  if (!st) st = alloc((void**)&c->d_bins, sizeof(double) * 2 * d * N);
  if (!st) st = alloc((void**)&c->d_tot, sizeof(double) * gv::kTotCols);
  if (!st && c->strat) st = alloc((void**)&c->d_cubes, sizeof(double) * 2 * G);
  if (!st) st = alloc((void**)&c->d_cube_max, sizeof(double) * G);
  if (!st) st = alloc((void**)&c->d_st, sizeof(GState));
  if (st) return bail(st);
  if (gv_malloc_host(&c->h_st, sizeof(GState)) != cudaSuccess)
    return bail(c->fail(VEGAS_ENOMEM, "cudaMallocHost(GState)"));
  memset(c->h_st, 0, sizeof(GState));
  c->h_st->acc = cfg->acc;
  if (cudaMemcpyAsync(c->d_st, c->h_st, sizeof(GState), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->d_bins, 0, sizeof(double) * 2 * d * N, c->stream) != cudaSuccess)
    return bail(c->fail(VEGAS_ECUDA, "state initialisation failed"));
  if ((st = configure_launch(c))) return bail(st);
  if (c->ke.grad) {  // adjoint pass (vegas_grad): launch shape and partial rows
    c->grad_smem = c->ke.grad_smem(d, N);
    int occg = 0;
    e = gv_raise_smem_limit(c->ke.grad, c->grad_smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occg, c->ke.grad, 256, c->grad_smem);
    if (e != cudaSuccess) return bail(c->fail(VEGAS_ECUDA, "adjoint launch: %s", cudaGetErrorString(e)));
    const int64_t want = (cfg->ncall + 255) / 256;
    c->grad_ctas = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->sm_count * std::max(occg, 1)));
    if ((st = alloc((void**)&c->d_gpart, sizeof(double) * (size_t)(c->ke.grad_nt + 2) * (c->grad_ctas + 1))))
      return bail(st);
  }
  std::vector<double> e0((size_t)d * (N + 1));
  for (int a = 0; a < d; ++a)
    for (int k = 0; k <= N; ++k) e0[(size_t)a * (N + 1) + k] = (double)k / (double)N;
  if ((st = upload_grid(c, e0.data()))) return bail(st);
  if ((st = upload_derived(c))) return bail(st);
  *out = c;
  return VEGAS_OK;
}

}  // namespace

extern "C" {

const char* vegas_last_error(const vegas_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_thread_err.c_str();
}

void vegas_destroy(vegas_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  destroy_graphs(c);
  cudaFree(c->d_edges);
  cudaFree(c->d_tab64);
  cudaFree(c->d_tab32);
  cudaFree(c->d_derived);
  cudaFree(c->d_part_bins);
  cudaFree(c->d_part_tot);
  cudaFree(c->d_bins);
  cudaFree(c->d_tot);
  cudaFree(c->d_cubes);
  cudaFree(c->d_cube_max);
  for (void* p : {(void*)c->d_q, (void*)c->d_mt, (void*)c->d_mt32, (void*)c->d_guide, (void*)c->d_bmax, (void*)c->d_bsum, (void*)c->d_prefix, (void*)c->d_meta, (void*)c->d_stage_x, (void*)c->d_stage_t,
                  (void*)c->d_out_x, (void*)c->d_out_t, (void*)c->d_counts, (void*)c->d_counters})
    cudaFree(p);
  cudaFree(c->d_gpart);
  cudaFree(c->d_st);
  if (c->h_st) cudaFreeHost(c->h_st);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

vegas_status vegas_create(const vegas_config* cfg, const vegas_integrand* fn, vegas_ctx** out) {
  if (!out) return thread_fail(VEGAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || !fn) return thread_fail(VEGAS_EINVAL, "config or integrand is NULL");
  int ybits = 0, g = 1;
  uint64_t G = 1;
  vegas_status cs = check_config(cfg, &ybits, &g, &G);
  if (cs) return cs;
  const int d = cfg->ndim;
  if (fn->ndim != d) return thread_fail(VEGAS_EINVAL, "integrand ndim %d != config ndim %d", fn->ndim, d);
  const int np = gv::expected_nparams(fn->kind, d);
  if (np < 0) return thread_fail(VEGAS_EINVAL, "unknown integrand kind %d", fn->kind);
  if (fn->nparams != np || (np > 0 && !fn->params))
    return thread_fail(VEGAS_EINVAL, "integrand kind %d needs %d parameters, got %d", fn->kind, np, fn->nparams);
  vegas_ctx* c = new_context(cfg, ybits, g, G);
  c->kind = fn->kind;
  c->params.assign(fn->params, fn->params + np);
  std::string why;
  if (!gv::derive_params(fn->kind, d, c->params.data(), c->derived, &c->scale, &why)) {
    delete c;
    return thread_fail(VEGAS_EINVAL, "%s", why.c_str());
  }
  if (!lookup_kernel(fn->kind, c->prec, ybits, d, &c->ke)) {
    delete c;
    return thread_fail(VEGAS_EINVAL, "no kernel for kind %d, ndim %d", fn->kind, d);
  }
  return finish_create(c, out);
}

vegas_status vegas_create_user(const vegas_config* cfg, const char* source, const double* params, int nparams,
                               vegas_ctx** out) {
  if (!out) return thread_fail(VEGAS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg || !source) return thread_fail(VEGAS_EINVAL, "config or source is NULL");
  int ybits = 0, g = 1;
  uint64_t G = 1;
  vegas_status cs = check_config(cfg, &ybits, &g, &G);
  if (cs) return cs;
  if (nparams < 0 || nparams > GVEGAS_MAXUSERPARAMS || (nparams > 0 && !params))
    return thread_fail(VEGAS_EINVAL, "user integrand takes 0..%d parameters, got %d", GVEGAS_MAXUSERPARAMS, nparams);
  vegas_ctx* c = new_context(cfg, ybits, g, G);
  c->kind = VG_USER;
  c->params.assign(params, params + nparams);
  std::copy(c->params.begin(), c->params.end(), c->derived);
  c->scale = 1.0;
  std::string why;
  const int d = cfg->ndim;
  const int rs = gv::rtc_user_entry(source, c->prec, ybits, d, spec_shape(d, d, ybits, g, cfg->nbins), &c->ke, &why);
  if (rs != VEGAS_OK) {
    delete c;
    return thread_fail((vegas_status)rs, "%s", why.c_str());
  }
  return finish_create(c, out);
}

vegas_status vegas_user_compile(const vegas_config* cfg, const char* source) {
  if (!cfg || !source) return thread_fail(VEGAS_EINVAL, "config or source is NULL");
  int ybits = 0, g = 1;
  uint64_t G = 1;
  vegas_status cs = check_config(cfg, &ybits, &g, &G);
  if (cs) return cs;
  const int d = cfg->ndim;
  std::string why;
  const int rs = gv::rtc_user_compile(source, cfg->precision, ybits, d, spec_shape(d, d, ybits, g, cfg->nbins), &why);
  if (rs != VEGAS_OK) return thread_fail((vegas_status)rs, "%s", why.c_str());
  return VEGAS_OK;
}

vegas_status vegas_iterate(vegas_ctx* c, int n_iter, int refine, vegas_result* out) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (n_iter < 0) return c->fail(VEGAS_EINVAL, "n_iter < 0");
  if (n_iter > 0) {
    if (c->hist_upper + n_iter > gv::kMaxHist)
      return c->fail(VEGAS_EINVAL, "window would exceed %d iterations; call vegas_reset_results", gv::kMaxHist);
    cudaGraphExec_t ge;
    vegas_status st = get_graph(c, 0, n_iter, 0, refine ? 1 : 0, c->cfg.acc, 0.0, &ge);
    if (st) return st;
    CK(c, cudaGraphLaunch(ge, c->stream));
    c->hist_upper += n_iter;
  }
  if (out) {
    vegas_status st = read_state(c);
    if (st) return st;
    fill_result(c, out);
  }
  return VEGAS_OK;
}

vegas_status vegas_reset_results(vegas_ctx* c) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  CK(c, gv_launch_control(c->d_st, gv::CTL_RESET_WINDOW | gv::CTL_SET_ACC, c->cfg.acc, 0u, c->stream));
  c->hist_upper = 0;
  return VEGAS_OK;
}

vegas_status vegas_reset_grid(vegas_ctx* c) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  const int d = c->cfg.ndim, N = c->cfg.nbins;
  CK(c, gv_launch_uniform_grid(c->d_edges, d, N, c->stream));
  CK(c, gv_launch_tables(c->d_edges, d, N, c->d_tab64, c->d_tab32, c->stream));
  return VEGAS_OK;
}

vegas_status bases_integrate(vegas_ctx* c, int itmx1, double acc1, int itmx2, double acc2,
                             vegas_result* out, vegas_result* phase1) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (itmx1 < 0 || itmx2 < 1 || itmx1 > gv::kMaxHist || itmx2 > gv::kMaxHist)
    return c->fail(VEGAS_EINVAL, "need 0 <= itmx1 <= %d and 1 <= itmx2 <= %d", gv::kMaxHist, gv::kMaxHist);
  cudaGraphExec_t ge;
  vegas_status st = get_graph(c, 1, itmx1, itmx2, 1, acc1, acc2, &ge);
  if (st) return st;
  CK(c, cudaGraphLaunch(ge, c->stream));
  c->hist_upper = itmx2;
  c->have_max = true;
  if (out || phase1) {
    if ((st = read_state(c))) return st;
    if (out) fill_result(c, out);
    if (phase1) {
      const GState* h = c->h_st;
      phase1->I = h->ph1_I;
      phase1->sigma = h->ph1_sigma;
      phase1->chi2_dof = h->ph1_chi2;
      phase1->iters_done = h->ph1_iters;
      phase1->stopped = h->ph1_stopped;
      phase1->nonfinite = h->ph1_nonfinite;
      phase1->samples = h->ph1_samples;
    }
  }
  return VEGAS_OK;
}

vegas_status vegas_get_grid(vegas_ctx* c, double* edges, double* bin_sums) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  const int d = c->cfg.ndim, N = c->cfg.nbins;
  const size_t ne = (size_t)d * (N + 1), nb = 2 * (size_t)d * N;
  vegas_status st = stage(c, ne + nb);
  if (st) return st;
  if (edges) CK(c, cudaMemcpyAsync(c->h_stage, c->d_edges, ne * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (bin_sums)
    CK(c, cudaMemcpyAsync(c->h_stage + ne, c->d_bins, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (edges) memcpy(edges, c->h_stage, ne * sizeof(double));
  if (bin_sums) memcpy(bin_sums, c->h_stage + ne, nb * sizeof(double));
  return VEGAS_OK;
}

vegas_status vegas_set_grid(vegas_ctx* c, const double* edges) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (!edges || !valid_grid(edges, c->cfg.ndim, c->cfg.nbins))
    return c->fail(VEGAS_EINVAL, "edges must start at 0, end at 1 and increase strictly");
  return upload_grid(c, edges);
}

vegas_status vegas_get_history(vegas_ctx* c, double* hist, int max_iters, int* n_out) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  vegas_status st = read_state(c);
  if (st) return st;
  const int n = std::min(c->h_st->nhist, std::max(max_iters, 0));
  if (n_out) *n_out = c->h_st->nhist;
  if (n > 0 && hist) {
    if ((st = stage(c, 2 * (size_t)n))) return st;
    CK(c, cudaMemcpyAsync(c->h_stage, &c->d_st->hist[0][0], 2 * n * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    memcpy(hist, c->h_stage, 2 * n * sizeof(double));
  }
  return VEGAS_OK;
}

vegas_status vegas_get_cube_sums(vegas_ctx* c, double* sums) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (!c->strat) return c->fail(VEGAS_ESTATE, "context is not stratified");
  if (!sums) return c->fail(VEGAS_EINVAL, "sums is NULL");
  const size_t n = 2 * (size_t)c->ncubes;
  vegas_status st = stage(c, n);
  if (st) return st;
  CK(c, cudaMemcpyAsync(c->h_stage, c->d_cubes, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const double s1 = c->scale, s2 = c->scale * c->scale;
  const bool pairs = c->prec == VG_FP32_ACCCOMP;  // (hi, lo, hi, lo) floats per cube
  const float* fp = reinterpret_cast<const float*>(c->h_stage);
  for (size_t i = 0; i < c->ncubes; ++i) {
    if (pairs) {
      sums[2 * i] = ((double)fp[4 * i] + (double)fp[4 * i + 1]) * s1;
      sums[2 * i + 1] = ((double)fp[4 * i + 2] + (double)fp[4 * i + 3]) * s2;
    } else {
      sums[2 * i] = c->h_stage[2 * i] * s1;
      sums[2 * i + 1] = c->h_stage[2 * i + 1] * s2;
    }
  }
  return VEGAS_OK;
}

vegas_status vegas_get_cube_max(vegas_ctx* c, double* cmax) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (!cmax) return c->fail(VEGAS_EINVAL, "cmax is NULL");
  if (!c->have_max) return c->fail(VEGAS_ESTATE, "no integration phase has run (bases_integrate)");
  const size_t n = (size_t)c->ncubes;
  vegas_status st = stage(c, n);
  if (st) return st;
  CK(c, cudaMemcpyAsync(c->h_stage, c->d_cube_max, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < n; ++i) cmax[i] = c->h_stage[i] * c->scale;
  return VEGAS_OK;
}

vegas_status spring_generate(vegas_ctx* c, uint64_t trial0, uint32_t n_trials, double* x_out, uint64_t* trial_out,
                             uint32_t* n_events, uint32_t* n_overflow, uint32_t* n_nonpos) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (!n_events) return c->fail(VEGAS_EINVAL, "n_events is NULL");
  if (!c->have_max) return c->fail(VEGAS_ESTATE, "no integration phase has run (bases_integrate)");
  if (trial0 + (uint64_t)n_trials > 0x100000000ull) return c->fail(VEGAS_EINVAL, "trial indices must stay below 2^32");
  if (c->ncubes > 0xFFFFFFFFull) return c->fail(VEGAS_EINVAL, "too many hypercubes");
  *n_events = 0;
  if (n_overflow) *n_overflow = 0;
  if (n_nonpos) *n_nonpos = 0;
  if (n_trials == 0) return VEGAS_OK;
  const int d = c->cfg.ndim, N = c->cfg.nbins;
  const uint32_t chunk = 4096, nchunks = (n_trials + chunk - 1) / chunk;
  const bool spec = c->ke.sample == c->ke.sample_spec && c->ke.spring_spec;
  const void* fn = spec ? c->ke.spring_spec : c->ke.spring;
  auto grow = [&](void** p, size_t bytes) -> vegas_status {
    cudaFree(*p);
    *p = nullptr;
    if (gv_dev_malloc(p, bytes) != cudaSuccess) return c->fail(VEGAS_ENOMEM, "cudaMalloc(%zu)", bytes);
    return VEGAS_OK;
  };
  vegas_status st = VEGAS_OK;
  uint32_t gk = 0;  // 2^gk guide intervals: about one per cube, at most 2^22 (16 MB)
  while (gk < 22 && (1ull << gk) < c->ncubes) ++gk;
  if (!c->d_q) {
    if (!st) st = grow((void**)&c->d_q, sizeof(uint64_t) * c->ncubes);
    if (!st) st = grow((void**)&c->d_mt, sizeof(double) * c->ncubes);
    if (!st) st = grow((void**)&c->d_mt32, sizeof(float) * c->ncubes);
    if (!st) st = grow((void**)&c->d_guide, sizeof(uint32_t) * ((1ull << gk) + 1));
    const size_t nb = (c->ncubes + kSpan - 1) / kSpan;
    if (!st) st = grow((void**)&c->d_bmax, sizeof(double) * nb);
    if (!st) st = grow((void**)&c->d_bsum, sizeof(unsigned long long) * nb);
    if (!st) st = grow((void**)&c->d_prefix, sizeof(uint64_t) * (c->ncubes + 1));
    if (!st) st = grow((void**)&c->d_meta, sizeof(double) * 3);
    if (!st) st = grow((void**)&c->d_counters, sizeof(unsigned long long) * 2);
  }
  if (!st && n_trials > c->spring_cap) {
    if (!st) st = grow((void**)&c->d_stage_x, sizeof(double) * d * (size_t)n_trials);
    if (!st) st = grow((void**)&c->d_out_x, sizeof(double) * d * (size_t)n_trials);
    if (!st) st = grow((void**)&c->d_stage_t, sizeof(uint64_t) * (size_t)n_trials);
    if (!st) st = grow((void**)&c->d_out_t, sizeof(uint64_t) * (size_t)n_trials);
    if (!st) st = grow((void**)&c->d_counts, sizeof(uint32_t) * nchunks);
    if (!st) {
      c->spring_cap = n_trials;
      c->spring_chunks_cap = nchunks;
    }
  }
  if (st) {
    c->spring_cap = 0;
    return st;
  }
  // integer cube table from the recorded maxima (in the integrand's units)
  {
    const uint32_t G = (uint32_t)c->ncubes, nb = (G + kSpan - 1) / kSpan;
    k_spring_max<<<nb, kSpanThreads, 0, c->stream>>>(c->d_cube_max, G, c->scale, c->d_bmax);
    k_spring_weights<<<nb, kSpanThreads, 0, c->stream>>>(c->d_cube_max, G, c->scale, c->d_bmax, nb, c->d_q,
                                                         c->d_mt, c->d_mt32, c->d_bsum);
    k_spring_scan<<<1, 1024, 0, c->stream>>>(c->d_bmax, nb, c->d_bsum, G, c->d_prefix, c->d_meta);
    k_spring_prefix<<<nb, kSpanThreads, 0, c->stream>>>(c->d_q, G, c->d_bsum, c->d_prefix, c->d_meta);
    k_spring_guide<<<(uint32_t)(((1ull << gk) + 256) / 256), 256, 0, c->stream>>>(c->d_prefix, G, gk, c->d_guide,
                                                                                  c->d_meta);
  }
  CK(c, cudaGetLastError());
  CK(c, cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * 2, c->stream));
  gv::SpringArgs R{};
  R.S = sample_args(c, 0);
  R.prefix = c->d_prefix;
  R.mt = c->d_mt;
  R.mt32 = c->d_mt32;
  R.guide = c->d_guide;
  R.gk = gk;
  R.meta = c->d_meta;
  R.out_scale = c->scale;
  R.trial0 = (uint32_t)trial0;
  R.n = n_trials;
  R.chunk = chunk;
  R.nchunks = nchunks;
  R.stage_x = c->d_stage_x;
  R.stage_t = c->d_stage_t;
  R.counts = c->d_counts;
  R.counters = c->d_counters;
  const bool f64 = c->prec == VG_FP64;
  const size_t smem = (size_t)d * N * (f64 ? sizeof(double2) : sizeof(float2)) +
                      gv::kNumDerived * (f64 ? sizeof(double) : sizeof(float));
  int occ = 0;
  CK(c, gv_raise_smem_limit(fn, smem));
  CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, smem));
  if (occ < 1) return c->fail(VEGAS_EINVAL, "SPRING kernel does not fit");
  const uint32_t blocks = std::min<uint32_t>(nchunks, (uint32_t)(c->sm_count * occ));
  void* args[] = {&R};
  if (c->spring_timer[0]) CK(c, cudaEventRecord(c->spring_timer[0], c->stream));
  CK(c, cudaLaunchKernel(fn, dim3(blocks), dim3(256), args, smem, c->stream));
  if (c->spring_timer[1]) CK(c, cudaEventRecord(c->spring_timer[1], c->stream));
  k_spring_compact<<<nchunks, 256, 0, c->stream>>>(c->d_counts, chunk, d, c->d_stage_x, c->d_stage_t, c->d_out_x,
                                                  c->d_out_t);
  CK(c, cudaGetLastError());
  // status, counts and counters back to the host
  std::vector<uint32_t> counts(nchunks);
  double meta[3];
  unsigned long long ctr[2];
  CK(c, cudaMemcpyAsync(meta, c->d_meta, sizeof meta, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(counts.data(), c->d_counts, sizeof(uint32_t) * nchunks, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(ctr, c->d_counters, sizeof ctr, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (meta[2] != 0.0) return c->fail(VEGAS_ESTATE, "every recorded cube maximum is zero");
  uint64_t total = 0;
  for (uint32_t k : counts) total += k;
  *n_events = (uint32_t)total;
  if (n_overflow) *n_overflow = (uint32_t)ctr[0];
  if (n_nonpos) *n_nonpos = (uint32_t)ctr[1];
  if (x_out && total)
    CK(c, cudaMemcpyAsync(x_out, c->d_out_x, sizeof(double) * d * total, cudaMemcpyDeviceToHost, c->stream));
  if (trial_out && total)
    CK(c, cudaMemcpyAsync(trial_out, c->d_out_t, sizeof(uint64_t) * total, cudaMemcpyDeviceToHost, c->stream));
  if ((x_out || trial_out) && total) CK(c, cudaStreamSynchronize(c->stream));
  return VEGAS_OK;
}

vegas_status spring_profile(vegas_ctx* c, uint32_t n_trials, int reps, double* ms) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (reps < 1 || !ms) return c->fail(VEGAS_EINVAL, "need reps >= 1 and ms");
  uint32_t k = 0;
  vegas_status st = spring_generate(c, 0, n_trials, nullptr, nullptr, &k, nullptr, nullptr);  // buffers, warm-up
  if (st) return st;
  cudaEvent_t a, b;
  CK(c, cudaEventCreate(&a));
  CK(c, cudaEventCreate(&b));
  double acc = 0.0;
  for (int r = 0; r < reps && !st; ++r) {
    c->spring_timer[0] = a;
    c->spring_timer[1] = b;
    st = spring_generate(c, 0, n_trials, nullptr, nullptr, &k, nullptr, nullptr);
    float t = 0.f;
    if (!st && cudaEventElapsedTime(&t, a, b) != cudaSuccess) st = c->fail(VEGAS_ECUDA, "event timing");
    acc += t;
  }
  c->spring_timer[0] = c->spring_timer[1] = nullptr;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st) return st;
  *ms = acc / reps;
  return VEGAS_OK;
}

vegas_status vegas_get_iteration(vegas_ctx* c, uint32_t* it) {
  if (!c || !it) return thread_fail(VEGAS_EINVAL, "NULL argument");
  vegas_status st = read_state(c);
  if (st) return st;
  *it = c->h_st->it;
  return VEGAS_OK;
}

vegas_status vegas_set_iteration(vegas_ctx* c, uint32_t it) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  CK(c, gv_launch_control(c->d_st, gv::CTL_SET_ITER, 0.0, it, c->stream));
  return VEGAS_OK;
}

vegas_status vegas_set_params(vegas_ctx* c, const double* params, int nparams) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (!params || nparams != (int)c->params.size())
    return c->fail(VEGAS_EINVAL, "expected %d parameters", (int)c->params.size());
  std::vector<double> p(params, params + nparams);
  double dv[gv::kNumDerived] = {}, sc = 1.0;
  std::string why;
  if (c->kind == VG_USER)  // the user's parameters are the device constants
    std::copy(p.begin(), p.end(), dv);
  else if (!gv::derive_params(c->kind, c->cfg.ndim, p.data(), dv, &sc, &why))
    return c->fail(VEGAS_EINVAL, "%s", why.c_str());
  c->params = p;
  memcpy(c->derived, dv, sizeof dv);
  c->scale = sc;
  // constants and scale live in device memory: the captured graphs read
  // them at run time and stay valid
  return upload_derived(c);
}

vegas_status vegas_eval(vegas_ctx* c, uint32_t it, double* I, double* var) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (it > 0x7FFFFFFFu) return c->fail(VEGAS_EINVAL, "iteration index must be < 2^31");
  int zero = 0;
  CK(c, cudaMemcpyAsync(&c->d_st->done, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  vegas_status st = launch_pass(c, (int)it, 0, 0);
  if (st) return st;
  if ((st = read_state(c))) return st;
  if (I) *I = c->h_st->last_I;
  if (var) *var = c->h_st->last_var;
  return VEGAS_OK;
}

vegas_status vegas_sample_dump(vegas_ctx* c, uint32_t it, const uint64_t* s, int64_t n, uint32_t* words,
                               int32_t* bins, double* x, double* jac, double* f) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (n < 0 || (n > 0 && !s)) return c->fail(VEGAS_EINVAL, "bad sample list");
  if (n == 0) return VEGAS_OK;
  if (it > 0x7FFFFFFFu) return c->fail(VEGAS_EINVAL, "iteration index must be < 2^31");
  for (int64_t i = 0; i < n; ++i)
    if (s[i] >= (uint64_t)c->cfg.ncall) return c->fail(VEGAS_EINVAL, "sample index %llu >= ncall", (unsigned long long)s[i]);
  const int d = c->cfg.ndim, W = c->ybits == 24 ? d : 2 * d;
  uint64_t* ds = nullptr;
  uint32_t* dw = nullptr;
  int32_t* db = nullptr;
  double *dx = nullptr, *dj = nullptr, *df = nullptr;
  vegas_status st = VEGAS_OK;
  auto A = [&](void** p, size_t b) {
    if (!st && gv_dev_malloc(p, b) != cudaSuccess) st = c->fail(VEGAS_ENOMEM, "cudaMalloc(%zu)", b);
  };
  A((void**)&ds, n * sizeof(uint64_t));
  if (words) A((void**)&dw, n * W * sizeof(uint32_t));
  if (bins) A((void**)&db, n * d * sizeof(int32_t));
  if (x) A((void**)&dx, n * d * sizeof(double));
  if (jac) A((void**)&dj, n * sizeof(double));
  if (f) A((void**)&df, n * sizeof(double));
  cudaError_t e = cudaSuccess;
  if (!st) {
    gv::DumpArgs D{};
    D.S = sample_args(c, (int)it);
    D.s = ds;
    D.n = n;
    D.words = dw;
    D.bins = db;
    D.x = dx;
    D.jac = dj;
    D.f = df;
    void* args[] = {&D};
    e = cudaMemcpyAsync(ds, s, n * sizeof(uint64_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaLaunchKernel(c->ke.dump, dim3((unsigned)((n + 255) / 256)), dim3(256), args, 0, c->stream);
    if (e == cudaSuccess && words) e = cudaMemcpyAsync(words, dw, n * W * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && bins) e = cudaMemcpyAsync(bins, db, n * d * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && x) e = cudaMemcpyAsync(x, dx, n * d * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && jac) e = cudaMemcpyAsync(jac, dj, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(f, df, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = c->fail(VEGAS_ECUDA, "sample dump: %s", cudaGetErrorString(e));
  }
  cudaFree(ds);
  cudaFree(dw);
  cudaFree(db);
  cudaFree(dx);
  cudaFree(dj);
  cudaFree(df);
  if (!st && f) {
    for (int64_t i = 0; i < n; ++i) f[i] *= c->scale;
    if (jac) {
      // jac is reported as the Jacobian itself; f carries the integrand scale
    }
  }
  return st;
}

vegas_status vegas_set_launch(vegas_ctx* c, int threads, int ctas_per_sm) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  cudaFuncAttributes fa{};
  CK(c, cudaFuncGetAttributes(&fa, c->ke.sample));
  if (threads < 64 || threads > fa.maxThreadsPerBlock || threads % 32 != 0)
    return c->fail(VEGAS_EINVAL, "threads must be a multiple of 32 in 64..%d", fa.maxThreadsPerBlock);
  if (ctas_per_sm < 0) return c->fail(VEGAS_EINVAL, "ctas_per_sm < 0");
  CK(c, cudaStreamSynchronize(c->stream));
  const int t0 = c->threads, p0 = c->ctas_per_sm_req;
  c->threads = threads;
  c->ctas_per_sm_req = ctas_per_sm;
  vegas_status st = configure_launch(c);
  if (st) {
    c->threads = t0;
    c->ctas_per_sm_req = p0;
    configure_launch(c);
  }
  return st;
}

vegas_status vegas_set_tile(vegas_ctx* c, int points_per_thread) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (points_per_thread < 0 || points_per_thread > 8)
    return c->fail(VEGAS_EINVAL, "points_per_thread must be in 0..8 (0: automatic)");
  CK(c, cudaStreamSynchronize(c->stream));
  const int p0 = c->ppt_req;
  c->ppt_req = points_per_thread;
  vegas_status st = configure_launch(c);
  if (st) {
    c->ppt_req = p0;
    configure_launch(c);
  }
  return st;
}

vegas_status vegas_autotune(vegas_ctx* c, int* threads, int* points_per_thread, double* ms) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  static const int kThreads[] = {128, 256, 384, 512};
  static const int kTiles[] = {0, 1, 2, 4};
  struct Cand {
    int t, p;
    bool small;
    double ms;
  };
  std::vector<Cand> cands;
  // one pass of warm-up, then the mean of n passes, for shape (t, p) and
  // capacity policy `small`
  auto time_shape = [&](int t, int p, bool small, int n, double* out) -> vegas_status {
    c->small_cap = small;
    if (vegas_set_launch(c, t, 0) != VEGAS_OK || vegas_set_tile(c, p) != VEGAS_OK) return VEGAS_EINVAL;
    double m[3];
    vegas_status st = vegas_profile_pass(c, 1, m);
    if (!st) st = vegas_profile_pass(c, n, m);
    if (!st) *out = m[2];
    return st == VEGAS_OK ? VEGAS_OK : VEGAS_ECUDA;
  };
  // screening: every shape the kernel takes (the others are skipped)
  for (int t : kThreads)
    for (int p : kTiles) {
      int cap_large = -1;  // the tile of the largest-capacity policy (a repeat is not timed twice)
      for (bool small : {false, true}) {
        double m = 0.0;
        const vegas_status st = time_shape(t, p, small, 3, &m);
        if (st == VEGAS_ECUDA) return c->err.empty() ? c->fail(st, "autotune: pass failed") : st;
        if (st != VEGAS_OK || (small && c->cap == cap_large)) continue;
        if (!small) cap_large = c->cap;
        cands.push_back({t, p, small, m});
      }
    }
  if (cands.empty()) return c->fail(VEGAS_EINVAL, "autotune: no launch shape fits");
  // the three fastest again, in interleaved rounds, keeping each one's best
  // round (shapes a few percent apart are within one screening's noise)
  std::sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) { return a.ms < b.ms; });
  cands.resize(std::min<size_t>(cands.size(), 3));
  for (int r = 0; r < 3; ++r)
    for (Cand& k : cands) {
      double m = 0.0;
      if (time_shape(k.t, k.p, k.small, 5, &m) != VEGAS_OK) return c->fail(VEGAS_ECUDA, "autotune: pass failed");
      k.ms = r == 0 ? m : std::min(k.ms, m);
    }
  const Cand best = *std::min_element(cands.begin(), cands.end(),
                                      [](const Cand& a, const Cand& b) { return a.ms < b.ms; });
  c->small_cap = best.small;
  vegas_status st = vegas_set_launch(c, best.t, 0);
  if (!st) st = vegas_set_tile(c, best.p);
  if (st) return st;
  if (threads) *threads = best.t;
  if (points_per_thread) *points_per_thread = c->ppt;
  if (ms) *ms = best.ms;
  return VEGAS_OK;
}

vegas_status vegas_get_tile(vegas_ctx* c, int* points_per_thread, int* cap) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (points_per_thread) *points_per_thread = c->ppt;
  if (cap) *cap = c->cap;
  return VEGAS_OK;
}

vegas_status vegas_get_launch(vegas_ctx* c, int* threads, int* ctas, int* ctas_per_sm) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (threads) *threads = c->threads;
  if (ctas) *ctas = c->ctas;
  if (ctas_per_sm) *ctas_per_sm = c->occ;
  return VEGAS_OK;
}

vegas_status vegas_grad(vegas_ctx* c, uint32_t it, double* grad, double* I) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (!grad) return c->fail(VEGAS_EINVAL, "grad is NULL");
  if (it > 0x7FFFFFFFu) return c->fail(VEGAS_EINVAL, "iteration index must be < 2^31");
  const int nt = vegas_ntheta(c);
  if (!c->ke.grad || nt == 0 || nt > c->ke.grad_nt)
    return c->fail(VEGAS_EINVAL, "no adjoint kernel for integrand kind %d with ndim %d", c->kind, c->cfg.ndim);
  if (c->kind == VG_RAMBO_BW && c->params[VG_RB_OBS] != 0.0)
    return c->fail(VEGAS_EINVAL, "the RAMBO gradient is defined for the full integrand (observable 0)");
  const int ncol = c->ke.grad_nt + 2;
  gv::SampleArgs A = sample_args(c, (int)it);
  double* part = c->d_gpart;
  double* out = c->d_gpart + (size_t)ncol * c->grad_ctas;
  void* args[] = {&A, &part};
  CK(c, cudaLaunchKernel(c->ke.grad, dim3(c->grad_ctas), dim3(256), args, c->grad_smem, c->stream));
  CK(c, gv_launch_colsum(part, ncol, c->grad_ctas, out, c->stream));
  vegas_status st = stage(c, ncol);
  if (st) return st;
  CK(c, cudaMemcpyAsync(c->h_stage, out, ncol * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  const double k = c->scale / (double)c->cfg.ncall;
  const int d = c->cfg.ndim, DM = c->ke.dm;
  for (int t = 0; t < nt; ++t) {
    // the Genz Gaussian kernel stores du at [0, d) and da at [DM, DM + d)
    const int src = (c->kind == VG_GENZ_GAUSSIAN && t >= d) ? DM + (t - d) : t;
    grad[t] = c->h_stage[src] * k;
  }
  if (I) *I = c->h_stage[c->ke.grad_nt] * k;
  return VEGAS_OK;
}

}  // extern "C"

namespace {
vegas_status profile_passes(vegas_ctx* c, int n_pass, bool nobins, double* ms);
}  // namespace

extern "C" {

vegas_status vegas_profile_pass(vegas_ctx* c, int n_pass, double* ms) { return profile_passes(c, n_pass, false, ms); }

vegas_status vegas_profile_frozen_pass(vegas_ctx* c, int n_pass, double* ms) {
  return profile_passes(c, n_pass, true, ms);
}

}  // extern "C"

namespace {

vegas_status profile_passes(vegas_ctx* c, int n_pass, bool nobins, double* ms) {
  if (!c) return thread_fail(VEGAS_EINVAL, "ctx is NULL");
  if (n_pass < 1 || !ms) return c->fail(VEGAS_EINVAL, "need n_pass >= 1 and ms[3]");
  CK(c, cudaStreamSynchronize(c->stream));
  vegas_status st = read_state(c);
  if (st) return st;
  const uint32_t it = c->h_st->it;
  int zero = 0;
  CK(c, cudaMemcpyAsync(&c->d_st->done, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i) CK(c, cudaEventCreate(&ev[i]));
  double acc[3] = {0, 0, 0};
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < n_pass && e == cudaSuccess; ++p) {
    gv::SampleArgs A = sample_args(c, (int)(it & 0x7FFFFFFFu), nobins);
    void* args[] = {&A};
    gv::FinArgs F = fin_args(c, 0, 0, nobins);
    e = cudaEventRecord(ev[0], c->stream);
    if (!e)
      e = cudaLaunchKernel(c->ke.sample, dim3(nobins ? c->ctas_nb : c->ctas), dim3(c->threads), args,
                           nobins ? c->smem_nb : c->smem, c->stream);
    if (!e) e = cudaEventRecord(ev[1], c->stream);
    if (!e) e = gv_launch_finish(&F, c->stream);
    if (!e) e = cudaEventRecord(ev[2], c->stream);
    if (!e) e = cudaEventSynchronize(ev[2]);
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
    if (!e) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (!e) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
    if (!e) e = cudaEventElapsedTime(&t2, ev[0], ev[2]);
    acc[0] += t0;
    acc[1] += t1;
    acc[2] += t2;
  }
  for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return c->fail(VEGAS_ECUDA, "profile: %s", cudaGetErrorString(e));
  for (int k = 0; k < 3; ++k) ms[k] = acc[k] / n_pass;
  return VEGAS_OK;
}

}  // namespace

extern "C" {

int vegas_ntheta(const vegas_ctx* c) {
  if (!c) return 0;
  switch (c->kind) {
    case VG_GENZ_GAUSSIAN: return 2 * c->cfg.ndim;
    case VG_DOUBLE_GAUSSIAN: return 3;
    case VG_RAMBO_BW: return 3;
    default: return 0;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// One evaluation pass without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// runtime's memory pool with a fixed budget, or a latency-critical loop where
// an allocation (which may synchronise the device or fail under
// fragmentation) is not allowed after start-up.  vegas_eval_noalloc serves
// them: the caller passes the grid and the output in its own device memory,
// and every intermediate the pass needs (grid tables, integrand constants,
// pass state, per-CTA partial sums) lives in the file-scope array below.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;  // 8 MiB, held by every GPU
                                                    // that loads this library
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kNoAllocMaxDevices] = {};
int g_noalloc_sms[kNoAllocMaxDevices] = {};

struct DerivedBlock {
  double v[gv::kNumDerived + 1];  // the constants, then the output scale
};

__global__ void k_noalloc_params(DerivedBlock b, double* dst) {
  for (int i = threadIdx.x; i <= gv::kNumDerived; i += blockDim.x) dst[i] = b.v[i];
}

__global__ void k_noalloc_result(const GState* st, double* out) {
  out[0] = st->last_I;
  out[1] = st->last_var;
  out[2] = st->last_sw;
  out[3] = st->last_sw2;
  out[4] = (double)st->last_nonfinite;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" vegas_status vegas_eval_noalloc(const vegas_config* cfg, const vegas_integrand* fn,
                                           const double* edges, uint32_t it, double* out) {
  if (!cfg || !fn || !edges || !out) return thread_fail(VEGAS_EINVAL, "NULL argument");
  const int d = cfg->ndim, N = cfg->nbins;
  if (d < 1 || d > GVEGAS_MAXDIM) return thread_fail(VEGAS_EINVAL, "ndim %d outside 1..%d", d, GVEGAS_MAXDIM);
  if (N < 2 || N > GVEGAS_MAXBINS) return thread_fail(VEGAS_EINVAL, "nbins %d outside 2..%d", N, GVEGAS_MAXBINS);
  if (cfg->ncall < 2 || cfg->ncall > (int64_t)1 << 32)
    return thread_fail(VEGAS_EINVAL, "ncall %lld outside 2..2^32", (long long)cfg->ncall);
  if (cfg->precision < VG_FP64 || cfg->precision > VG_FP32_ACCCOMP)
    return thread_fail(VEGAS_EINVAL, "unknown precision %d", cfg->precision);
  if (it > 0x7FFFFFFFu) return thread_fail(VEGAS_EINVAL, "iteration index must be < 2^31");
  const int ybits = cfg->ybits ? cfg->ybits : (cfg->precision == VG_FP64 ? 53 : 24);
  if (ybits != 24 && ybits != 53) return thread_fail(VEGAS_EINVAL, "ybits must be 24 or 53");
  if (fn->ndim != d) return thread_fail(VEGAS_EINVAL, "integrand ndim %d != config ndim %d", fn->ndim, d);
  const int np = gv::expected_nparams(fn->kind, d);
  if (np < 0) return thread_fail(VEGAS_EINVAL, "unknown integrand kind %d", fn->kind);
  if (fn->nparams != np || (np > 0 && !fn->params))
    return thread_fail(VEGAS_EINVAL, "integrand kind %d needs %d parameters, got %d", fn->kind, np, fn->nparams);
  const int g = cfg->nstrat < 1 ? 1 : cfg->nstrat;
  uint64_t G = 1;
  for (int a = 0; a < d; ++a) {
    G *= (uint64_t)g;
    if (G > (uint64_t)cfg->ncall) return thread_fail(VEGAS_EINVAL, "nstrat^ndim exceeds ncall");
  }
  if ((uint64_t)cfg->ncall % G != 0) return thread_fail(VEGAS_EINVAL, "ncall must be a multiple of nstrat^ndim");
  if (G > 1 && (uint64_t)cfg->ncall / G < 2) return thread_fail(VEGAS_EINVAL, "need >= 2 points per hypercube");
  if ((int64_t)g * N >= (ybits == 53 ? 2048 : (1 << 30)))
    return thread_fail(VEGAS_EINVAL, "nstrat * nbins too large for %d-bit sampling", ybits);

  DerivedBlock db;
  double scale = 1.0;
  char why_buf[128] = {0};
  {
    std::string why;
    if (!gv::derive_params(fn->kind, d, fn->params, db.v, &scale, &why)) {
      snprintf(why_buf, sizeof why_buf, "%s", why.c_str());
      return thread_fail(VEGAS_EINVAL, "%s", why_buf);
    }
    db.v[gv::kNumDerived] = scale;
  }
  gv::KernelEntry ke{};
  if (!lookup_kernel(fn->kind, cfg->precision, ybits, d, &ke))
    return thread_fail(VEGAS_EINVAL, "no kernel for kind %d, ndim %d", fn->kind, d);
  int ppt_min = 1;
  if (ke.sample_spec && d == ke.dm && ybits == 24 && (g & (g - 1)) == 0 && (int64_t)g * N <= 256) {
    ke.sample = ke.sample_spec;
    ppt_min = ke.spec_ppt_min;
  }

  // Per-device set-up on the first call for the current device: the device
  // address of the scratch array (its host-side name is only a stand-in).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return thread_fail(VEGAS_EINVAL, "device index %d too large", dev);
  unsigned char* scratch;
  int sms;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      int n = 0;
      e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "device attribute: %s", cudaGetErrorString(e));
      g_noalloc_sms[dev] = n;
      g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_noalloc_ptr[dev];
    sms = g_noalloc_sms[dev];
  }

  // Launch shape (as for a context) with the CTA count bounded by the rows
  // of partial sums that fit in the scratch array.
  const int threads = 256;
  auto occ_of = [&](int cap, int) -> int {
    const size_t sm = ke.smem(d, N, cap);
    int o = 0;
    if (e != cudaSuccess || sm > 227 * 1024) return 0;
    e = gv_raise_smem_limit(ke.sample, sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, ke.sample, threads, sm);
    return e == cudaSuccess ? o : 0;
  };
  int occ_cap = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cap, ke.sample, threads, 0);
  const gv::TileShape t = e == cudaSuccess ? gv::choose_tile(threads, N, 0, ppt_min, occ_cap, occ_of) : gv::TileShape{1, 4, 0};
  if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
  if (t.occ < 1) return thread_fail(VEGAS_EINVAL, "sampling kernel does not fit in shared memory");
  const int ppt = t.ppt, cap = t.cap, occ = t.occ;
  const size_t smem = ke.smem(d, N, cap);
  e = gv_raise_smem_limit(ke.sample, smem);
  if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "launch configuration: %s", cudaGetErrorString(e));
  const int dN = d * N;
  const size_t off_st = 0;
  const size_t off_dp = align256(off_st + sizeof(GState));
  const size_t off_t64 = align256(off_dp + sizeof(double) * (gv::kNumDerived + 1));
  const size_t off_t32 = align256(off_t64 + sizeof(double2) * dN);
  const size_t off_tot = align256(off_t32 + sizeof(float2) * dN);
  const size_t off_rows = align256(off_tot + sizeof(double) * gv::kTotCols);
  const size_t row_bytes = sizeof(double) * (2 * (size_t)dN + gv::kTotCols);
  const int64_t max_rows = off_rows < kNoAllocScratchBytes ? (int64_t)((kNoAllocScratchBytes - off_rows - 512) / row_bytes) : 0;
  if (max_rows < 1)
    return thread_fail(VEGAS_EINVAL, "ndim * nbins = %d too large for the %zu-byte no-allocation scratch", dN,
                       kNoAllocScratchBytes);
  const uint64_t nc = (uint64_t)cfg->ncall / G;
  const int strat = G > 1;
  const int64_t cap_ctas = (int64_t)sms * occ;
  int L = 1;
  uint64_t units = (uint64_t)cfg->ncall;
  if (strat) {
    L = gv::choose_lanes(G, nc, threads, std::min<int64_t>(cap_ctas, max_rows));
    units = G * (uint64_t)L;
  }
  const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)((units + threads - 1) / threads), cap_ctas, max_rows}));
  double* part_tot = reinterpret_cast<double*>(scratch + off_rows);
  double* part_bins = reinterpret_cast<double*>(scratch + align256(off_rows + sizeof(double) * gv::kTotCols * ctas));
  GState* st = reinterpret_cast<GState*>(scratch + off_st);

  cudaStream_t s = (cudaStream_t)cfg->stream;
  // Contents left by the previous call: the pass state must start cleared
  // (its stop flag gates the kernels); tables, partial rows and totals are
  // overwritten in full below.
  e = cudaMemsetAsync(st, 0, offsetof(GState, hist), s);
  if (e == cudaSuccess) {
    k_noalloc_params<<<1, 128, 0, s>>>(db, reinterpret_cast<double*>(scratch + off_dp));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = gv_launch_tables(edges, d, N, reinterpret_cast<double2*>(scratch + off_t64),
                         reinterpret_cast<float2*>(scratch + off_t32), s);
  if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "no-allocation set-up: %s", cudaGetErrorString(e));

  gv::SampleArgs A{};
  A.d = d;
  A.N = N;
  A.g = g;
  A.ybits = ybits;
  A.lanes = L;
  A.cap = cap;
  A.ppt = ppt;
  A.strat = strat;
  A.key0 = (uint32_t)cfg->seed;
  A.key1 = (uint32_t)(cfg->seed >> 32);
  gv::philox_key_schedule(A.key0, A.key1, A.ks);
  A.instance = cfg->instance;
  A.it_override = (int)it;
  A.ncall = (uint64_t)cfg->ncall;
  A.nc = (uint32_t)nc;
  A.ncubes = (uint32_t)G;
  A.cube_mul = (strat && (G & (G - 1)) == 0 && G > 1) ? 0x9E3779B1u : 1u;
  A.g_pow2 = (g & (g - 1)) == 0;
  A.g_log2 = 0;
  while ((1 << A.g_log2) < g) ++A.g_log2;
  A.t32 = (int64_t)g * N <= 256;
  const double gb = (double)g * std::ldexp(1.0, ybits);
  A.inv_gb_d = 1.0 / gb;
  A.inv_gb_f = (float)(1.0 / gb);
  A.inv_nc = 1.0 / (double)nc;
  A.inv_nc1 = nc > 1 ? 1.0 / (double)(nc - 1) : 0.0;
  A.nparts = ctas;
  A.tab = cfg->precision == VG_FP64 ? (const void*)(scratch + off_t64) : (const void*)(scratch + off_t32);
  A.dparams = reinterpret_cast<const double*>(scratch + off_dp);
  A.st = st;
  A.part_bins = part_bins;
  A.part_tot = part_tot;
  A.cubes = nullptr;
  void* args[] = {&A};
  e = cudaLaunchKernel(ke.sample, dim3(ctas), dim3(threads), args, smem, s);
  gv::FinArgs F{};
  F.d = d;
  F.N = N;
  F.nparts = ctas;
  F.strat = strat;
  F.refine = 0;
  F.record = 0;
  F.pair32 = cfg->precision == VG_FP32_ACCCOMP;
  F.ncall = (uint64_t)cfg->ncall;
  F.ncubes = G;
  F.scale = reinterpret_cast<double*>(scratch + off_dp) + gv::kNumDerived;
  F.alpha = cfg->alpha;
  F.part_bins = part_bins;
  F.part_tot = part_tot;
  F.bins = out;
  F.tot = reinterpret_cast<double*>(scratch + off_tot);
  F.edges = nullptr;
  F.tab64 = reinterpret_cast<double2*>(scratch + off_t64);
  F.tab32 = reinterpret_cast<float2*>(scratch + off_t32);
  F.st = st;
  if (e == cudaSuccess) e = gv_launch_finish(&F, s);
  if (e == cudaSuccess) {
    k_noalloc_result<<<1, 1, 0, s>>>(st, out + 2 * (size_t)dN);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return thread_fail(VEGAS_ECUDA, "no-allocation pass: %s", cudaGetErrorString(e));
  return VEGAS_OK;
}
