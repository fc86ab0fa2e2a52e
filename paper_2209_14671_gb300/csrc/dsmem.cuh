// Distributed-shared-memory exchanges between the CTAs of a thread-block cluster (tile_kernel.cu): st.async stores into another CTA's shared memory, each counted in bytes on an
// mbarrier of the receiving CTA, which waits for the byte count it expects.  The sender never waits
// for its stores (no release fence); every wait is bounded and sets an error flag when it runs out.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace elf {

// The two halves of a cluster barrier (no memory ordering: used only to know that every CTA
// of the cluster is running); every thread of every CTA executes both.
template <int CS>
__device__ __forceinline__ void cluster_arrive() {
  if constexpr (CS > 1) asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
template <int CS>
__device__ __forceinline__ void cluster_wait() {
  if constexpr (CS > 1) asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t mapa_u32(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_async_f2(uint32_t raddr, float2 v, uint32_t rmbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "f"(v.x), "f"(v.y), "r"(rmbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init_expect(uint64_t* bar, uint32_t bytes) {
  const uint32_t a = smem_u32(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

constexpr long kTileSpinLimit = 1L << 18;  // about 1 s of polls on GB300 (3.8 us per poll, measured)

// Wait (acquire, cluster scope) for phase 0 of bar; after `limit` polls flag the error and go on.
__device__ __forceinline__ void mbar_wait_or_flag(uint64_t* bar, int* err, long limit = kTileSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], 0;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a)
        : "memory");
    if (ok) return;
  }
  atomicExch(err, 1);
}


}  // namespace elf
