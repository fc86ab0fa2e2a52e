// elf_estimate_weights_noalloc: the alpha = beta estimate of Eqs. 16-17 for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted,
// for example a host process whose device memory is owned by another allocator
// or a fixed budget, or code that prepares work while a framework forbids new
// allocations.  The regular path (elf_set_measurements) computes the same
// estimate but needs a handle, whose creation allocates.
//
// The estimator's only scratch is one FP64 partial sum per (image, 16-row
// chunk).  Here it lives in the file-scope array below, which every GPU that
// loads this library keeps until the process exits.  Host code cannot use the
// array's name as a device address (in host code it names a host-side stand-in),
// so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current, and caches it.  The cached
// address belongs to the device's primary context: after cudaDeviceReset on that
// device the module is loaded again elsewhere and the cached address is stale, so
// this entry point must not be called on a device after it has been reset.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/elfpie.h"
#include "internal.cuh"

namespace {

__device__ __align__(256) double g_weight_partials[ELF_NOALLOC_WEIGHT_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {};

}  // namespace

namespace elf {
int noalloc_set_error(int code, const char* msg);
}

extern "C" int elf_estimate_weights_noalloc(const float* I, int n_led, int n_lowres, int fidelity, double* weights,
                                            void* cuda_stream) {
  if (!I || !weights) return elf::noalloc_set_error(ELF_EINVAL, "null I or weights");
  if (n_led < 1 || n_lowres < 3 || n_lowres > 4096 || (fidelity != 0 && fidelity != 1))
    return elf::noalloc_set_error(ELF_EINVAL, "n_led must be >= 1, n_lowres in [3, 4096], fidelity 0 or 1");
  // one partial per (image, 16-row chunk of the interior), counted in 64 bits: every image needs at least
  // one, so n_led alone already bounds the count from below
  const long long parts = n_led > ELF_NOALLOC_WEIGHT_MAX_PARTIALS
                              ? (long long)n_led
                              : (long long)n_led * (long long)((n_lowres - 2 + 15) / 16);
  if (parts > ELF_NOALLOC_WEIGHT_MAX_PARTIALS)
    return elf::noalloc_set_error(
        ELF_EINVAL, ("problem too large for the static scratch: needs " + std::to_string(parts) +
                     " partials (n_led * ceil((n_lowres - 2) / 16)), the maximum is " +
                     std::to_string(ELF_NOALLOC_WEIGHT_MAX_PARTIALS))
                        .c_str());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return elf::noalloc_set_error(ELF_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return elf::noalloc_set_error(ELF_EINVAL, "device ordinal out of range");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_weight_partials);
      if (e != cudaSuccess) return elf::noalloc_set_error(ELF_ECUDA, cudaGetErrorString(e));
      g_scratch[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch[dev];
  }
  // Every partial is overwritten by this call before it is read, so nothing needs
  // clearing; overlapping calls on the GPU share the array and race.
  e = elf::launch_alpha(I, n_led, n_lowres, fidelity == 1, scratch, weights, -1.0, -1.0,
                        static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return elf::noalloc_set_error(ELF_ECUDA, cudaGetErrorString(e));
  return ELF_OK;
}
