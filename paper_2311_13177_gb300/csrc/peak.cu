// Device diagnostics: the FP32 FMA throughput (the ALU ceiling the
// interpolation and spread kernels are compared with; they stay far left of
// the FP32 ridge) and a check of the bounded mbarrier wait that every staged
// kernel relies on to report, rather than hang on, a copy that never lands.
#include "prop_internal.cuh"
#include "tma.cuh"

namespace {

// Waits on an mbarrier that nobody arrives at: the bounded wait must give up
// after `limit` cycles and the kernel return normally.
__global__ void bounded_wait_probe_kernel(int* expired, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    prop::mbar_init(&bar, 1);
    prop::fence_mbar_init();
  }
  __syncthreads();
  const bool done = prop::mbar_wait_bounded(&bar, 0u, limit);
  if (threadIdx.x == 0) *expired = done ? 0 : 1;
}

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kUnroll = 16;     // FMAs per chain per loop trip
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float* out, int trips, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (float)(threadIdx.x + i);
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live; never true
}

}  // namespace

extern "C" PROP_API prop_status prop_fp32_fma_peak(int device, double* tflops) {
  using namespace prop;
  if (!tflops) return fail(PROP_ERR_INVALID_ARG, "prop_fp32_fma_peak: tflops is null");
  DeviceGuard g(device);
  if (!g.ok) return fail(PROP_ERR_INVALID_ARG, "prop_fp32_fma_peak: bad device");
  int sms = 0;
  PROP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int blocks = sms * 8;
  const int trips = 4096;
  float* out = nullptr;
  PROP_CUDA(cudaMalloc(&out, sizeof(float) * (size_t)blocks * kPeakThreads));
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      fma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, trips, 0.99999f, 1e-6f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;  // first launch is warm-up
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "prop_fp32_fma_peak");
  const double flops = 2.0 * (double)blocks * kPeakThreads * trips * kUnroll * kChains;
  *tflops = flops / (best_ms * 1e-3) / 1e12;
  return PROP_OK;
}

extern "C" PROP_API prop_status prop_check_bounded_wait(int device, long long limit_cycles, int* expired,
                                                        double* ms) {
  using namespace prop;
  if (!expired) return fail(PROP_ERR_INVALID_ARG, "prop_check_bounded_wait: expired is null");
  if (limit_cycles <= 0 || limit_cycles > kWaitLimitCycles)
    return fail(PROP_ERR_INVALID_ARG, "prop_check_bounded_wait: limit_cycles must be in (0, 4e9]");
  DeviceGuard g(device);
  if (!g.ok) return fail(PROP_ERR_INVALID_ARG, "prop_check_bounded_wait: bad device");
  int* flag = nullptr;
  PROP_CUDA(cudaMalloc(&flag, sizeof(int)));
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0xff, sizeof(int), s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    bounded_wait_probe_kernel<<<1, 32, 0, s>>>(flag, limit_cycles);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(flag);
  if (e != cudaSuccess) return cuda_fail(e, "prop_check_bounded_wait");
  *expired = h;
  if (ms) *ms = t;
  return PROP_OK;
}
