// wf_tma.cuh -- bulk asynchronous copies (TMA) between global and shared memory, completed on
// mbarriers, for the persistent spectral passes.
//
// A pass keeps STG tile buffers in shared memory.  One thread issues the tensor copy of a tile
// into a free buffer and arms that buffer's mbarrier with the tile's byte count; every thread
// waits on the barrier's phase before transforming the tile; after the transform all threads
// fence their shared-memory writes towards the async proxy, synchronise, and one thread issues the
// tensor store of the tile and commits it as a bulk group.  Before a buffer is refilled, that
// thread waits until the store's reads of it are done.  No registers are spent on staging, and
// the load of the next tile runs under the transform of the current one.
//
// Every wait is bounded: a barrier that does not complete within kMbarSpinLimit polls reports a
// timeout, which the pass turns into an error word for the host and an early exit.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "wf_common.cuh"

namespace wf {

// polls of an mbarrier before a wait is reported as timed out (~seconds: far beyond any copy)
constexpr unsigned kMbarSpinLimit = 1u << 26;

WF_D unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

WF_D void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the async proxy (the copy engine)
WF_D void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one arrival that also expects `bytes` of transaction count (the copies issued next)
WF_D void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// wait for the phase with the given parity to complete; false after kMbarSpinLimit polls
WF_D bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (unsigned i = 0; i < kMbarSpinLimit; ++i) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// order this thread's generic-proxy shared-memory writes before later async-proxy reads
WF_D void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// tiled 4D tensor copies (coordinates in elements of the map, innermost first)
WF_D void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
WF_D void tma_store_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3, const void* src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
               : "memory");
}
// contiguous copies (16-byte aligned addresses, size a multiple of 16)
WF_D void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
WF_D void bulk_store(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
WF_D void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until at most N committed bulk groups still read shared memory / are still in flight
template <int N> WF_D void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
template <int N> WF_D void bulk_wait() { asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory"); }
// per-thread asynchronous 16-byte copies global -> shared (completed by commit / wait groups)
WF_D void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
WF_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N> WF_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

WF_D void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---- host side -----------------------------------------------------------------------------
// A 4D tensor map over `nb` packed half spectra [nb][N][N][N/2] of complex storage elements,
// addressed in real components (dimension 0 = 2 N/2 floats or doubles), with box
// {2 nl, b1, b2, 1}: nl consecutive kz columns by b1 rows along the second-fastest axis by b2
// along the slowest spatial axis.  Returns false if the driver refuses the map.
bool make_spectrum_map(CUtensorMap* map, void* base, int n, int nb, bool fp64, int nl, int b1, int b2);

}  // namespace wf
