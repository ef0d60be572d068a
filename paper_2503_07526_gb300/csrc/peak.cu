// Measured FP32 throughput of the GPU the library runs on.
//
// The roofline of the pair kernel is its FP32 rate, and no vendor or driver
// figure for it is at hand, so it is measured here: every thread of a grid
// that fills every SM runs eight independent chains of dependent FMAs (scalar
// fma.rn.f32, or paired fma.rn.f32x2 on register pairs), long enough that
// launch overhead is negligible; the rate is the FMAs' flops (2 per FMA per
// lane) over the kernel time taken with CUDA events.
#include <cstdint>

#include "common.cuh"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;   // independent FMA chains per thread
constexpr int kPeakUnroll = 16;  // FMAs per chain per loop iteration

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void unpack2(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

template <bool PAIRED>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int64_t iters, float *out) {
  const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 63);
  float sum = 0.f;
  if constexpr (PAIRED) {
    uint64_t a[kPeakChains];
    const uint64_t b = pack2(0.9999999f, 0.9999998f), c = pack2(1e-7f, 2e-7f);
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q) a[q] = pack2(seed + q, seed - q);
    for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
      for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
        for (int q = 0; q < kPeakChains; ++q)
          asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[q]) : "l"(b), "l"(c));
      }
    }
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q) {
      float lo, hi;
      unpack2(a[q], lo, hi);
      sum += lo + hi;
    }
  } else {
    float a[kPeakChains];
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q) a[q] = seed + q;
    for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
      for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
        for (int q = 0; q < kPeakChains; ++q)
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[q]) : "f"(0.9999999f), "f"(1e-7f));
      }
    }
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q) sum += a[q];
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = sum;  // keeps the chains live
}

}  // namespace

extern "C" {

int md_fp32_peak(int32_t paired, int64_t iters, int32_t reps, void *cuda_stream, double *flops_per_launch,
                 double *ms_per_launch, int32_t *sm_count) {
  otf::clear_error();
  if (iters < 1 || reps < 1 || !flops_per_launch || !ms_per_launch || !sm_count) {
    otf::set_error("md_fp32_peak: iters and reps must be positive and every output non-null");
    return MD_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0;
  OTF_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop{};
  OTF_CUDA(cudaGetDeviceProperties(&prop, dev));
  int per_sm = 0;
  if (paired)
    OTF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<true>, kPeakThreads, 0));
  else
    OTF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<false>, kPeakThreads, 0));
  const int blocks = prop.multiProcessorCount * (per_sm > 0 ? per_sm : 1);
  float *out = nullptr;
  OTF_CUDA(cudaMalloc(&out, (size_t)blocks * kPeakThreads * sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MD_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    otf::set_error("md_fp32_peak: cudaEventCreate failed");
    rc = MD_ECUDA;
  }
  for (int k = 0; k <= reps && rc == MD_OK; ++k) {  // launch 0 is a warm-up
    if (k == 1) cudaEventRecord(e0, s);
    if (paired)
      k_fma_peak<true><<<blocks, kPeakThreads, 0, s>>>(iters, out);
    else
      k_fma_peak<false><<<blocks, kPeakThreads, 0, s>>>(iters, out);
    if (cudaGetLastError() != cudaSuccess) {
      otf::set_error("md_fp32_peak: launch failed");
      rc = MD_ECUDA;
    }
  }
  float ms = 0.f;
  if (rc == MD_OK) {
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      otf::set_error("md_fp32_peak: timing failed");
      rc = MD_ECUDA;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(out);
  if (rc) return rc;
  const double fma_per_thread = (double)iters * kPeakUnroll * kPeakChains * (paired ? 2.0 : 1.0);
  *flops_per_launch = 2.0 * fma_per_thread * blocks * kPeakThreads;
  *ms_per_launch = ms / reps;
  *sm_count = prop.multiProcessorCount;
  return MD_OK;
}

}  // extern "C"
