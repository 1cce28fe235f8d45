// dsmem.cuh — point-to-point exchange between the CTAs of a thread-block cluster:
// st.async writes into a peer CTA's shared memory and completes its bytes on the
// peer's mbarrier (transaction count), so a receiver waits only for the data it needs
// instead of a cluster-wide barrier; cp.async prefetch into shared memory.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace pxa {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t map_rank(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_async_f64(uint32_t raddr, double v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
               ::"r"(raddr), "d"(v), "r"(rbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arm(uint64_t* bar, int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; "
      "selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait: gives up after the context's wait limit (status[1] x 1024 cycles; 0 means
// 2^31 cycles, about 1 s) or as soon as another CTA has reported an error, setting
// PXA_ERR_TIMEOUT so that the host sees it. `status` points to the context's two-int
// status block (status word, wait limit).
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try(bar, parity)) return;
  const int units = ((volatile int*)status)[1];
  const long long limit = units > 0 ? (long long)units << 10 : (1LL << 31);
  const long long t0 = clock64();
  for (int it = 1;; ++it) {
    if (mbar_try(bar, parity)) return;
    if ((it & 255) == 0) {
      if (*(volatile int*)status != 0) return;
      if (clock64() - t0 > limit) {
        set_status(status, PXA_ERR_TIMEOUT);
        return;
      }
    }
  }
}

// Bounded wait that ignores the status word: lets a copy still in flight land before a
// CTA that gave up on an earlier wait leaves.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it)
    if (mbar_try(bar, parity)) return;
}

// One bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// memory into this CTA's shared memory, completing its bytes on `bar` (armed by the caller
// with mbar_arm for the same byte count).
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem)),
      "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace pxa
