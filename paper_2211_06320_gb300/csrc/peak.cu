// FMA-pipe throughput microbenchmark (fpe_bench.h): the measured denominator
// of the FP64 roofline the evaluation kernels are compared against.
#include <cuda_runtime.h>

#include "fpe_bench.h"
#include "fpe_internal.h"

namespace fpe {

constexpr int kPeakIters = 2048;
constexpr int kPeakChains = 8;

template <class T>
__global__ void k_fma_peak(T *sink, T a, T b) {
  T acc[kPeakChains];
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) acc[i] = (T)(threadIdx.x * 1e-3 + i);
  for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) acc[i] = fma(acc[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kPeakChains; ++i) s += acc[i];
  if (s == (T)12345.678) sink[threadIdx.x] = s;  // never true; keeps the chains live
}

// bf16 mma.sync (m16n8k16, fp32 accumulation) issue rate: the instruction the
// tensor-core window sums use.  Eight independent accumulators per warp,
// operands in registers.
constexpr int kMmaIters = 4096;
__global__ void k_mma_peak(float *sink) {
  uint32_t a[4], b[2];
  for (int i = 0; i < 4; ++i) a[i] = 0x3f803f80u + (uint32_t)((threadIdx.x + i) & 7);
  for (int i = 0; i < 2; ++i) b[i] = 0x40003f80u + (uint32_t)((threadIdx.x * 3 + i) & 7);
  float d[8][4];
  for (int j = 0; j < 8; ++j)
    for (int i = 0; i < 4; ++i) d[j][i] = 0.0f;
  for (int it = 0; it < kMmaIters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(d[j][0]), "+f"(d[j][1]), "+f"(d[j][2]), "+f"(d[j][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0.0f;
  for (int j = 0; j < 8; ++j)
    for (int i = 0; i < 4; ++i) s += d[j][i];
  if (s == 12345.678f) sink[threadIdx.x] = s;  // never true; keeps the accumulators live
}

}  // namespace fpe

extern "C" fpe_status fpe_measure_mma_peak(int reps, double *flop_per_s) {
  using namespace fpe;
  if (reps < 1 || !flop_per_s) {
    set_error("fpe_measure_mma_peak: reps >= 1 and a non-NULL output");
    return FPE_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 2;
  void *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, threads * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r <= reps; ++r) {
    cudaEventRecord(e0, 0);
    k_mma_peak<<<blocks, threads>>>((float *)sink);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "k_mma_peak");
  // 16 x 8 x 16 multiply-adds per mma, 2 flop each
  *flop_per_s = (double)blocks * (threads / 32) * kMmaIters * 8 * (2.0 * 16 * 8 * 16) / (best * 1e-3);
  return FPE_OK;
}

extern "C" fpe_status fpe_measure_fma_peak(int precision, int reps, double *fma_per_s) {
  using namespace fpe;
  if ((precision != 64 && precision != 32) || reps < 1 || !fma_per_s) {
    set_error("fpe_measure_fma_peak: precision must be 32 or 64, reps >= 1, output non-NULL");
    return FPE_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 4;
  void *sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, threads * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int r = 0; r <= reps; ++r) {
    cudaEventRecord(e0, 0);
    if (precision == 64)
      k_fma_peak<double><<<blocks, threads>>>((double *)sink, 1.0000001, 1e-9);
    else
      k_fma_peak<float><<<blocks, threads>>>((float *)sink, 1.0001f, 1e-6f);
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (r > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "k_fma_peak");
  *fma_per_s = (double)blocks * threads * kPeakIters * kPeakChains / (best * 1e-3);
  return FPE_OK;
}
