// TMA tensor copies and mbarrier primitives (inline PTX), and the host-side
// cache of 3-D tensor maps, shared by the fine-grid kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace thermo {

// ---- TMA / mbarrier primitives (inline PTX)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// default stage wait: 2^31 clock64 cycles, about one second at the GB300's clocks
constexpr long long kStageWait = 1LL << 31;
// Wait for the phase of parity `parity` of *bar to complete, giving up after
// `limit` clock64 cycles (limit 0: one non-blocking test).  false: gave up.
__device__ __forceinline__ bool mbar_wait_limited(uint64_t* bar, unsigned parity, long long limit) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 < limit)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Ring of `ns` stages in which group q (q >= q0) lands on stage (q - q0) % ns
// in phase (q - q0) / ns.  Before the issuing thread exits, wait (default
// limit) for the last ns groups issued, q0 .. qhi, so that no bulk copy into
// the CTA's shared memory is still in flight when the CTA retires (after a
// stage wait gave up, the consumers skip their waits).  Groups already
// waited on return at once.
__device__ __forceinline__ void mbar_drain(uint64_t* bars, int ns, int q0, int qhi) {
  for (int q = (qhi - ns + 1 > q0 ? qhi - ns + 1 : q0); q <= qhi; ++q)
    mbar_wait_limited(bars + (q - q0) % ns, (unsigned)(((q - q0) / ns) & 1), kStageWait);
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}


// 3-D map of a padded array: dims (d0 elements, d1 rows, d2 planes), dense
// rows of d0 elements, box (b0, b1, 1), zero fill outside (cached per buffer
// and box; thread-safe).
cudaError_t get_map(CUtensorMap* out, const void* base, CUtensorMapDataType dt, int esize, long long d0,
                    long long d1, long long d2, int b0, int b1);

}  // namespace thermo
