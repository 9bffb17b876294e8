// microbench.cu -- measured issue rates of the instruction classes the
// sampling kernel is built from (FP32 FMA, 32x32->64 integer multiplies,
// FP64 FMA, special-function unit, integer->float conversion, Philox blocks)
// and of the shared-memory histogram update strategies.  These are the
// denominators of the ALU roofline and the evidence for the histogram design.
#include <cuda_runtime.h>

#include "common.cuh"

namespace gv {
namespace mb {

constexpr int kIters = 4096;

__global__ void k_ffma(float* out, float a) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3f + i;
  for (int r = 0; r < kIters; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, 0.5f);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 123.456f) out[0] = s;
}

__global__ void k_imad_wide(uint32_t* out, uint32_t a) {
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x + 977u * i;
  for (int r = 0; r < kIters; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = __umulhi(x[i], a) ^ (x[i] * a);
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s ^= x[i];
  if (s == 0x12345678u) out[0] = s;
}

__global__ void k_dfma(double* out, double a) {
  double x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int r = 0; r < kIters / 16; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = fma(x[i], a, 0.5);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += x[i];
  if (s == 123.456) out[0] = s;
}

__global__ void k_mufu(float* out, float a) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-6f + 1e-3f * i;
  for (int r = 0; r < kIters / 4; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = exp2f(x[i] * a);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 123.456f) out[0] = s;
}

__global__ void k_i2f(float* out, uint32_t a) {
  uint32_t u[8];
  float s[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    u[i] = threadIdx.x * 7u + i;
    s[i] = 0.f;
  }
  for (int r = 0; r < kIters / 4; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      s[i] += (float)u[i];
      u[i] += a;
    }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += s[i];
  if (t == 123.456f) out[0] = t;
}

__global__ void k_philox(uint32_t* out, uint32_t k0) {
  uint32_t acc = 0;
  for (int r = 0; r < kIters / 64; ++r) {
    const uint4 v = philox4x32_10(make_uint4(threadIdx.x + blockIdx.x * blockDim.x, r, 7u, 0u), k0, 3u);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x12345678u) out[0] = acc;
}

// Philox with the 32x32->64 products written as 64-bit multiplies.
__device__ __forceinline__ uint4 philox_wide(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
  }
  return c;
}

__global__ void k_philox_wide(uint32_t* out, uint32_t k0) {
  uint32_t acc = 0;
  for (int r = 0; r < kIters / 64; ++r) {
    const uint4 v = philox_wide(make_uint4(threadIdx.x + blockIdx.x * blockDim.x, r, 7u, 0u), k0, 3u);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x12345678u) out[0] = acc;
}

__global__ void k_shfl(float* out) {
  float x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = threadIdx.x + i;
  for (int r = 0; r < kIters / 8; ++r)
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = __shfl_xor_sync(0xffffffffu, x[i], (r + i) & 31) + 1.0f;
  if (x[0] + x[1] + x[2] + x[3] == 123.456f) out[0] = x[0];
}

// Warp bin ownership: 8 axes, 50 bins; lane l owns bins l and l + 32 of every
// axis; each round every lane's value visits all 32 lanes by xor shuffles and
// is added by its owner into registers (no atomics).  Counts axis-updates.
__global__ void k_owner(float* out) {
  const uint32_t lane = threadIdx.x & 31;
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.f;
  uint32_t x = 2463534242u ^ (threadIdx.x * 747796405u + blockIdx.x * 2891336453u);
  for (int r = 0; r < kIters / 256; ++r) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    uint32_t w0 = 0, w1 = 0;  // 8 bins of 8 bits
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      w0 |= __umulhi(x * (2654435761u + 2u * a), 50u) << (8 * a);
      w1 |= __umulhi(x * (2246822519u + 2u * a), 50u) << (8 * a);
    }
    const float w = (float)(x >> 8) * 1e-7f;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      const uint32_t b0 = __shfl_xor_sync(0xffffffffu, w0, k);
      const uint32_t b1 = __shfl_xor_sync(0xffffffffu, w1, k);
      const float v = __shfl_xor_sync(0xffffffffu, w, k);
      const float v2 = v * v;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const uint32_t b = ((a < 4 ? b0 : b1) >> (8 * (a & 3))) & 0xFFu;
        if (b == lane) {
          acc[a][0] += v;
          acc[a][1] += v2;
        }
        if (b == lane + 32u) {
          acc[a][2] += v;
          acc[a][3] += v2;
        }
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) s += acc[a][q];
  if (s == 123.456f) out[0] = s;
}

// Shared-memory histogram updates: 50 bins, bins from a per-thread
// xorshift.  mode 0: one histogram per CTA, float atomicAdd; 1: one
// histogram per warp, float atomicAdd; 2: per CTA, 32-bit integer
// atomicAdd; 3: per CTA, double atomicAdd.
template <int MODE>
__global__ void k_hist(float* out) {
  __shared__ float hf[8 * 64];
  __shared__ int hi[64];
  __shared__ double hd[64];
  __shared__ unsigned long long hu[8 * 64];
  __shared__ int hw[8 * 64];
  for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x) {
    hu[i] = 0ull;
    hw[i] = 0;
  }
  for (int i = threadIdx.x; i < 8 * 64; i += blockDim.x) hf[i] = 0.f;
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    hi[i] = 0;
    hd[i] = 0.0;
  }
  __syncthreads();
  uint32_t x = 2463534242u ^ (threadIdx.x * 747796405u + blockIdx.x * 2891336453u);
  float* h = MODE == 1 ? hf + 64 * (threadIdx.x >> 5) : hf;
  for (int r = 0; r < kIters / 8; ++r) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    const uint32_t b = __umulhi(x, 50u);
    if (MODE == 0 || MODE == 1) atomicAdd(&h[b], 1.0f);
    if (MODE == 2) atomicAdd(&hi[b], 1);
    if (MODE == 3) atomicAdd(&hd[b], 1.0);
    if (MODE == 4) atomicAdd(&hi[b + 64 * 0], 1);
    if (MODE == 5) atomicAdd(&hu[b], 1ull);
    if (MODE == 6) atomicAdd(&hu[64 * (threadIdx.x >> 5) + b], 1ull);
    if (MODE == 7) atomicAdd(&hw[64 * (threadIdx.x >> 5) + b], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) out[blockIdx.x] = hf[0] + (float)hi[0] + (float)hd[0] + (float)hu[0] + (float)hw[0];
}

}  // namespace mb
}  // namespace gv

extern "C" vegas_status vegas_microbench(int op, double* rate) {
  using namespace gv::mb;
  if (!rate) return VEGAS_EINVAL;
  *rate = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VEGAS_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VEGAS_ECUDA;
  const int threads = 256, blocks = sms * 8;
  const double nthreads = (double)threads * blocks;
  void* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks) != cudaSuccess) return VEGAS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double ops = 0.0;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {  // first run warms up
    cudaEventRecord(e0);
    switch (op) {
      case 0: k_ffma<<<blocks, threads>>>((float*)buf, 0.999f); ops = nthreads * kIters * 8; break;
      case 1: k_imad_wide<<<blocks, threads>>>((uint32_t*)buf, 0xD2511F53u); ops = nthreads * kIters * 8; break;
      case 2: k_dfma<<<blocks, threads>>>((double*)buf, 0.999); ops = nthreads * (kIters / 16) * 4; break;
      case 3: k_mufu<<<blocks, threads>>>((float*)buf, 0.999f); ops = nthreads * (kIters / 4) * 8; break;
      case 4: k_i2f<<<blocks, threads>>>((float*)buf, 3u); ops = nthreads * (kIters / 4) * 8; break;
      case 5: k_philox<<<blocks, threads>>>((uint32_t*)buf, 11u); ops = nthreads * (kIters / 64); break;
      case 6: k_hist<0><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      case 7: k_hist<1><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      case 8: k_hist<2><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      case 9: k_hist<3><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      case 10: k_philox_wide<<<blocks, threads>>>((uint32_t*)buf, 11u); ops = nthreads * (kIters / 64); break;
      case 11: k_shfl<<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8) * 4; break;
      case 12: k_owner<<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 256) * 8; break;
      case 13: k_hist<5><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      case 14: k_hist<6><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      case 15: k_hist<7><<<blocks, threads>>>((float*)buf); ops = nthreads * (kIters / 8); break;
      default:
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(buf);
        return VEGAS_EINVAL;
    }
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
  }
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return VEGAS_ECUDA;
  *rate = ops / (ms * 1e-3);
  return VEGAS_OK;
}
