// fmm_device_peaks: measured arithmetic throughput of the current device, the
// denominators of the compute rooflines of the near field and M2L (FP32 FMA,
// packed FP32x2 FMA, FP64 FMA, MUFU rsqrt).  Each probe runs many
// independent dependency chains per thread over a grid of several waves, so
// the measured rate is the pipe's issue limit rather than its latency.
#include "common.cuh"

namespace fmm {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) ffma_probe(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 12345.678f) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(kThreads) ffma2_probe(float* out, int iters, float b, float c) {
  unsigned long long a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) {
    const float x = (float)(threadIdx.x + k) * 1e-3f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(x), "f"(x + 1.f));
  }
  unsigned long long bb, cc;
  asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
  asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c), "f"(c));
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++)
#pragma unroll
      for (int k = 0; k < kChains; k++) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; k++) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a[k]));
    s += x + y;
  }
  if (s == 12345.678f) out[0] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_probe(float* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 12345.678) out[0] = (float)s;
}

__global__ void __launch_bounds__(kThreads) rsqrt_probe(float* out, int iters, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int r = 0; r < 16; r++)
#pragma unroll
      for (int k = 0; k < kChains; k++) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[k]));
        a[k] = y + c;  // stays near 1; one FADD per rsqrt keeps the chain dependent
      }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 12345.678f) out[0] = s;
}

template <class K>
double time_ms(K launch, cudaStream_t st) {
  cudaEvent_t a, b;
  FMM_CUDA_TRY(cudaEventCreate(&a));
  FMM_CUDA_TRY(cudaEventCreate(&b));
  launch();  // warm-up
  FMM_CUDA_TRY(cudaEventRecord(a, st));
  launch();
  FMM_CUDA_TRY(cudaEventRecord(b, st));
  FMM_CUDA_TRY(cudaEventSynchronize(b));
  float ms = 0.f;
  FMM_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)ms;
}

}  // namespace
}  // namespace fmm

extern "C" int fmm_device_peaks(double* out, void* stream) {
  using namespace fmm;
  try {
    require(out != nullptr, "out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    FMM_CUDA_TRY(cudaGetDevice(&dev));
    FMM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    FMM_CUDA_TRY(cudaMalloc(&sink, sizeof(float)));
    const int blocks = nsm * 8;  // eight 256-thread blocks per SM: full occupancy, one wave
    const double threads = (double)blocks * kThreads;
    const double per_iter = 16.0 * kChains;
    int iters = 4096;
    double ms = time_ms([&] { ffma_probe<<<blocks, kThreads, 0, st>>>(sink, iters, 0.999999f, 1e-6f); }, st);
    out[0] = threads * iters * per_iter * 2.0 / (ms * 1e-3) / 1e12;
    ms = time_ms([&] { ffma2_probe<<<blocks, kThreads, 0, st>>>(sink, iters, 0.999999f, 1e-6f); }, st);
    out[1] = threads * iters * per_iter * 4.0 / (ms * 1e-3) / 1e12;
    const int iters64 = 256;
    ms = time_ms([&] { dfma_probe<<<blocks, kThreads, 0, st>>>(sink, iters64, 0.999999, 1e-6); }, st);
    out[2] = threads * iters64 * per_iter * 2.0 / (ms * 1e-3) / 1e12;
    const int iters_r = 1024;
    ms = time_ms([&] { rsqrt_probe<<<blocks, kThreads, 0, st>>>(sink, iters_r, 1e-3f); }, st);
    out[3] = threads * iters_r * per_iter / (ms * 1e-3) / 1e9;
    FMM_LAUNCH_CHECK();
    cudaFree(sink);
    return FMM_OK;
  } catch (const Fail& e) {
    return e.code;
  } catch (...) {
    set_error("unexpected C++ exception");
    return FMM_ERR_CUDA;
  }
}
