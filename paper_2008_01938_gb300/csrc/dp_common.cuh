// dp_common.cuh -- device helpers shared by the MCM and S-DP kernels:
// inline PTX for mbarriers, 1-D bulk (TMA) copies, proxy fences, acquire /
// release accesses to global flags, and bounded spin-waits.
//
// Every wait in this library is bounded: it gives up after `limit` SM clock
// cycles, records DP_ETIMEOUT in the caller's status word and lets the kernel
// return, so a missing producer never hangs the GPU.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dpgpu.h"

namespace dpk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------
// mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async proxy (bulk copies).
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase of parity `parity` to complete; false on timeout.
// After a few quick polls the waiting warp sleeps between polls, so blocks
// that wait for data do not take issue slots from blocks that compute.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  uint32_t polls = 0, backoff = 32;
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
    if (++polls > 4) {
      __nanosleep(backoff);
      backoff = backoff < 512 ? backoff * 2 : 512;
    }
  }
  return true;
}

// mbar_wait with the sleep between polls capped at cap_ns, for waits on the
// critical path (a long sleep delays the wake-up after the data lands).
__device__ __forceinline__ bool mbar_wait_cap(uint64_t* bar, uint32_t parity, long long limit, uint32_t cap_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  uint32_t polls = 0, backoff = 16;
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
    if (++polls > 4) {
      __nanosleep(backoff);
      backoff = backoff < cap_ns ? backoff * 2 : cap_ns;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// 1-D bulk copy global -> shared (TMA), completion counted on an mbarrier.
// dst, src 16-byte aligned; bytes a multiple of 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Orders this thread's earlier generic-proxy view of global memory before its
// later async-proxy (bulk copy) reads.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---------------------------------------------------------------------------
// global flags
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t ld_acquire(const int32_t* p) {
  int32_t v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int32_t* p, int32_t v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_release_add(int32_t* p, int32_t v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acquire_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Records the first device-side error in *status (later errors are dropped).
__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  atomicCAS(status, 0, code);
}

// Spins until *flag >= target (relaxed polling with a short sleep -- a waiting
// finisher is usually on the critical path -- then one acquire fence).
// Returns false (and records DP_ETIMEOUT) if `limit` cycles pass first or if
// another block already recorded an error.
__device__ __forceinline__ bool wait_flag_geq(const int32_t* flag, int32_t target, long long limit,
                                              int32_t* status) {
  if (ld_acquire(flag) >= target) return true;
  const long long t0 = clock64();
  uint32_t backoff = 32;
  while (true) {
    if (ld_relaxed(flag) >= target) {
      fence_acquire_gpu();
      return true;
    }
    if (clock64() - t0 > limit) {
      set_status(status, DP_ETIMEOUT);
      return false;
    }
    if (*reinterpret_cast<volatile const int32_t*>(status) != 0) return false;
    __nanosleep(backoff);
    backoff = backoff < 64 ? backoff * 2 : 64;
  }
}

// wait_flag_geq with the sleep between polls capped at CAP ns and acquire
// loads for the polls (int32 MCM instances: every flag wait there is,
// directly or through the tasks that follow, on the chain of
// tile-diagonals).
template <uint32_t CAP>
__device__ __forceinline__ bool wait_flag_geq_cap(const int32_t* flag, int32_t target, long long limit,
                                                  int32_t* status) {
  if (ld_acquire(flag) >= target) return true;
  const long long t0 = clock64();
  uint32_t backoff = CAP < 32 ? CAP : 32;
  while (true) {
    if (ld_acquire(flag) >= target) return true;  // acquire polls: no fence after the flip
    if (clock64() - t0 > limit) {
      set_status(status, DP_ETIMEOUT);
      return false;
    }
    if (*reinterpret_cast<volatile const int32_t*>(status) != 0) return false;
    __nanosleep(backoff);
    backoff = backoff < CAP ? backoff * 2 : CAP;
  }
}

// Waits until f[x] >= target[x] for every x < N (int32 MCM instances).  The
// first test issues all N acquire loads at once, so the words already set
// cost one round trip together rather than one each; any still short are
// then polled one at a time with wait_flag_geq_cap.  A target of 0 is met at
// once.  Every word is read by an acquire load, so no fence follows.
template <uint32_t CAP, int N>
__device__ __forceinline__ bool wait_flags_geq_cap(const int32_t* const (&f)[N], const int32_t (&target)[N],
                                                   long long limit, int32_t* status) {
  int32_t v[N];
#pragma unroll
  for (int x = 0; x < N; ++x) v[x] = ld_acquire(f[x]);
  bool all = true;
#pragma unroll
  for (int x = 0; x < N; ++x) all = all && v[x] >= target[x];
  if (!all) {
#pragma unroll
    for (int x = 0; x < N; ++x)
      if (v[x] < target[x] && !wait_flag_geq_cap<CAP>(f[x], target[x], limit, status)) return false;
  }
  return true;
}

}  // namespace dpk
