// Diagnostics of the library on the current GPU.
//
// elf_measure_fp32_peak: the FP32 FMA throughput of the current GPU, measured.
//
// The tile kernel of Eqs. 1-12 is bound by FP32 arithmetic, so its roofline needs the
// CUDA-core peak of the GPU it runs on.  This kernel gives every thread kChains
// independent FMA chains x <- x * m + c (enough independent work per warp to cover the
// FMA latency) and launches a few waves of full blocks on every SM; the throughput is
// 2 FLOP per FMA over the launch's CUDA-event duration.  m and c keep every chain
// bounded and normal (|x| stays near c / (1 - m)), and the result is stored only under a
// condition the compiler cannot decide, so no FMA can be removed.
//
// launch_wait_timeout (elf_selftest_wait_timeout): one warp waits on an mbarrier phase that nothing
// completes (it expects 16 bytes that are never sent), with the bounded wait of the tile kernels'
// exchanges and a caller's poll limit; the wait runs out, sets the error flag and the kernel returns.
#include <cuda_runtime.h>

#include <string>

#include "../../include/elfpie.h"
#include "dsmem.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__device__ float g_peak_sink;

__global__ void __launch_bounds__(kThreads) fma_peak_kernel(float m, float c, int iters, float never) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == never) g_peak_sink = s;
}

}  // namespace

namespace elf {
int noalloc_set_error(int code, const char* msg);

namespace {
__global__ void __launch_bounds__(32) wait_timeout_kernel(int* err, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init_expect(&bar, 16);
  __syncthreads();
  mbar_wait_or_flag(&bar, err, (long)limit);
}
}  // namespace

cudaError_t launch_wait_timeout(int* err, long long limit, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(err, limit);
  return cudaGetLastError();
}
}  // namespace elf

extern "C" int elf_measure_fp32_peak(int iters, int repeats, void* cuda_stream, double* tflops, double* best_ms) {
  if (!tflops || iters < 1 || repeats < 1) return elf::noalloc_set_error(ELF_EINVAL, "bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return elf::noalloc_set_error(ELF_ECUDA, cudaGetErrorString(e));
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return elf::noalloc_set_error(ELF_ECUDA, cudaGetErrorString(e));
  }
  const dim3 grid(sms * kBlocksPerSm), block(kThreads);
  float best = 1e30f;
  for (int r = -1; r < repeats && e == cudaSuccess; ++r) {  // r = -1: warm-up launch
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess) {
      fma_peak_kernel<<<grid, block, 0, s>>>(0.99999994f, 1e-7f, iters, -1.0f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && r >= 0 && ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return elf::noalloc_set_error(ELF_ECUDA, cudaGetErrorString(e));
  const double flop = 2.0 * kChains * (double)iters * (double)grid.x * kThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (best_ms) *best_ms = best;
  return ELF_OK;
}
