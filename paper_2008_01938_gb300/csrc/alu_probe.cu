// alu_probe.cu -- measured integer throughput of the GPU the library runs on:
// the denominator of the MCM kernel's INT32-ALU roofline.
//
// Each probe keeps every SM full (eight 256-thread blocks, 16 warps per
// sub-partition) of independent dependency chains of one kind of integer
// instruction, and counts SM clock cycles around the loop with clock64().
// Lanes per clock per SM = (threads resident on an SM x instructions per
// thread) / (cycles of the slowest block on it), so the figure does not
// depend on the clock the SM happened to run at; CUDA events around the
// launch give the clock itself (cycles / time).
//
// The probes:
//   0  three-input add            a = a + b + c
//   1  integer multiply-add       a = a * m + b
//   2  three-way unsigned minimum a = min(a, b, c)   (__vimin3_u32)
//   3  two-input add                a = a + b
//      The compiler issues two-input adds to both integer pipes (the ALU pipe
//      and, as multiply-adds by one, the FMA pipe), so this probe keeps both
//      busy: it is the combined INT32 rate, the roofline's peak.
//   4  probes 0 and 1 interleaved, half the chains each: three-input adds on
//      the ALU pipe beside multiply-adds on the FMA pipe, the two kinds of
//      instruction of the solver's split evaluations
//   5  the MCM bulk loop: the split evaluations of one 32 x 32 tile against
//      one k-segment, 4 x 2 cells per thread, operands read from shared
//      memory exactly as the solver's bulk tasks read them (packed keys, a
//      multiply-add and a fused add-and-minimum per candidate, the chunk
//      merge into 64-bit keys); reported as split evaluations per clock per
//      SM.  This is the
//      ceiling of the solver's inner loop when nothing waits.
#include <cuda_runtime.h>

#include <cstdint>

#include "api_internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kChains = 8;   // independent accumulators per thread
constexpr int kUnroll = 16;  // chain steps per loop trip

struct ProbeOut {
  unsigned long long cycles_max;  // slowest block of the launch
  unsigned long long sink;        // keeps the results alive
};

template <int OP>
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    int32_rate_kernel(ProbeOut* out, uint32_t seed, int trips) {
  uint32_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * (i + 1u);
  const uint32_t m = seed | 1u;
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 1
  for (int it = 0; it < trips; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        const uint32_t b = a[(i + 1) % kChains], c = a[(i + 3) % kChains];
        if constexpr (OP == 0) a[i] = a[i] + b + c;
        if constexpr (OP == 1) a[i] = a[i] * m + b;
        if constexpr (OP == 2) a[i] = __vimin3_u32(a[i], b, c);
        if constexpr (OP == 3) a[i] = a[i] + b;
        if constexpr (OP == 4) a[i] = (i & 1) ? a[i] * m + b : a[i] + b + c;
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) x ^= a[i];
  if (threadIdx.x == 0) atomicMax(&out->cycles_max, (unsigned long long)(t1 - t0));
  if (x == 0x12345678u) atomicAdd(&out->sink, 1ull);
}

// The solver's bulk loop (one compute group's share of a 32-split segment
// with chunks of 32 aligned splits), on a panel staged once in shared memory,
// at the solver's occupancy (three blocks of 256 computing threads per SM).
constexpr int kBulkBlocksPerSm = 3;
__global__ void __launch_bounds__(kProbeThreads, kBulkBlocksPerSm)
    bulk_rate_kernel(ProbeOut* out, uint32_t seed, int trips) {
  constexpr int T = 32;
  __shared__ __align__(16) uint32_t A[T * T], B[T * T], PK[T];
  for (int x = threadIdx.x; x < T * T; x += blockDim.x) {
    A[x] = (seed * (x + 7u)) & 0x7FFFFFE0u;
    B[x] = (seed * (x + 3u)) & 0x3FFFFFE0u;
  }
  if (threadIdx.x < T) PK[threadIdx.x] = ((threadIdx.x % 31u) + 1u) << 5;
  const int tg = threadIdx.x & 127, ty = tg >> 4, tx = tg & 15;
  uint32_t P[4][2];
  unsigned long long best[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      P[r][c] = ((seed >> (2 * r + c)) & 1023u) | 1u;  // eight different multipliers, as in a tile
      best[r][c] = ~0ull;
    }
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 1
  for (int it = 0; it < trips; ++it) {
    uint32_t acc[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = 0xFFFFFFFFu;
#pragma unroll
    for (int kk = 0; kk < T; kk += 2) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(A + kk * T + 4 * ty);
      const uint2 b0 = *reinterpret_cast<const uint2*>(B + kk * T + 2 * tx);
      const uint4 a1 = *reinterpret_cast<const uint4*>(A + (kk + 1) * T + 4 * ty);
      const uint2 b1 = *reinterpret_cast<const uint2*>(B + (kk + 1) * T + 2 * tx);
      const uint32_t pk0 = PK[kk], pk1 = PK[kk + 1];
      const uint32_t av0[4] = {a0.x, a0.y, a0.z, a0.w}, av1[4] = {a1.x, a1.y, a1.z, a1.w};
      const uint32_t bv0[2] = {b0.x, b0.y}, bv1[2] = {b1.x, b1.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          acc[r][c] = __viaddmin_u32(P[r][c] * pk0 + av0[r], bv0[c], acc[r][c]);
          acc[r][c] = __viaddmin_u32(P[r][c] * pk1 + av1[r], bv1[c], acc[r][c]);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const unsigned long long v = acc[r][c] >> 5;
        const unsigned long long k = (unsigned)(it & 1023) * T + (acc[r][c] & 31u);
        best[r][c] = best[r][c] < ((v << 32) | k) ? best[r][c] : ((v << 32) | k);
      }
    // a different panel word each trip, so nothing is loop-invariant
    if (threadIdx.x == 0) PK[it & 31] += 32u;
    __syncthreads();
  }
  const long long t1 = clock64();
  unsigned long long x = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) x ^= best[r][c];
  if (threadIdx.x == 0) atomicMax(&out->cycles_max, (unsigned long long)(t1 - t0));
  if (x == 0x123456789ull) atomicAdd(&out->sink, 1ull);
}

// The int64 solver's bulk loop (seg_i64): 64-bit packed (value, k) entries
// on a shared-memory panel, a 64-bit multiply-add of the weight and a 64-bit
// minimum per split, 4 x 2 cells per thread, two resident blocks per SM as
// in the int64 solver.
constexpr int kBulk64BlocksPerSm = 2;
__global__ void __launch_bounds__(kProbeThreads, kBulk64BlocksPerSm)
    bulk64_rate_kernel(ProbeOut* out, uint32_t seed, int trips) {
  constexpr int T = 32;
  __shared__ __align__(16) unsigned long long A[T * T], B[T * T];
  __shared__ uint32_t PK[T];
  for (int x = threadIdx.x; x < T * T; x += blockDim.x) {
    A[x] = ((unsigned long long)((seed * (x + 7u)) & 0x7FFFFFu) << 16) | (unsigned)(x & 1023);
    B[x] = ((unsigned long long)((seed * (x + 3u)) & 0x3FFFFFu) << 16);
  }
  if (threadIdx.x < T) PK[threadIdx.x] = (threadIdx.x % 31u) + 1u;
  const int tg = threadIdx.x & 127, ty = tg >> 4, tx = tg & 15;
  uint32_t P[4][2];
  unsigned long long best[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      P[r][c] = (((seed >> (2 * r + c)) & 1023u) | 1u) << 16;
      best[r][c] = ~0ull;
    }
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 1
  for (int it = 0; it < trips; ++it) {
#pragma unroll 4
    for (int kk = 0; kk < T; ++kk) {
      const ulonglong2 a01 = *reinterpret_cast<const ulonglong2*>(A + kk * T + 4 * ty);
      const ulonglong2 a23 = *reinterpret_cast<const ulonglong2*>(A + kk * T + 4 * ty + 2);
      const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(B + kk * T + 2 * tx);
      const uint32_t pk = PK[kk];
      const unsigned long long av[4] = {a01.x, a01.y, a23.x, a23.y};
      const unsigned long long bv[2] = {b.x, b.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const unsigned long long cand = (unsigned long long)P[r][c] * pk + av[r] + bv[c];
          best[r][c] = best[r][c] < cand ? best[r][c] : cand;
        }
    }
    // a different panel word each trip, so nothing is loop-invariant
    if (threadIdx.x == 0) PK[it & 31] += 1u;
    __syncthreads();
  }
  const long long t1 = clock64();
  unsigned long long x = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) x ^= best[r][c];
  if (threadIdx.x == 0) atomicMax(&out->cycles_max, (unsigned long long)(t1 - t0));
  if (x == 0x123456789ull) atomicAdd(&out->sink, 1ull);
}

}  // namespace

using namespace dph;

extern "C" dp_status dp_measure_int32_rates(double* out, int32_t nout, void* stream) {
  if (!out || nout < 9) return fail(DP_EINVAL, "dp_measure_int32_rates: out must hold 9 values");
  const int nprobes = nout >= 10 ? 7 : 6;  // probe 6 (the int64 bulk loop) when out has room for it
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  int occ[7] = {0, 0, 0, 0, 0, 0, 0};
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], int32_rate_kernel<0>, kProbeThreads, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], int32_rate_kernel<1>, kProbeThreads, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], int32_rate_kernel<2>, kProbeThreads, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[3], int32_rate_kernel<3>, kProbeThreads, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[4], int32_rate_kernel<4>, kProbeThreads, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[5], bulk_rate_kernel, kProbeThreads, 0)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[6], bulk64_rate_kernel, kProbeThreads, 0)) != cudaSuccess)
    return fail_cuda(e, "dp_measure_int32_rates: occupancy");
  ProbeOut* d = nullptr;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(ProbeOut), st)) != cudaSuccess)
    return fail_cuda(e, "dp_measure_int32_rates: allocation");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaFreeAsync(d, st);
    return fail_cuda(e, "dp_measure_int32_rates: events");
  }
  double clk_sum = 0.0;
  for (int op = 0; op < nprobes && rc == DP_OK; ++op) {
    // every block resident at once: one block per (SM, slot), no second wave
    const int want = op == 5 ? kBulkBlocksPerSm : op == 6 ? kBulk64BlocksPerSm : kProbeBlocksPerSm;
    const int bps = occ[op] < want ? occ[op] : want;
    const int grid = ds->sms * (bps > 0 ? bps : 1);
    const int trips = op >= 5 ? 1024 : 2048;
    for (int rep = 0; rep < 2 && rc == DP_OK; ++rep) {  // the first launch warms up
      cudaMemsetAsync(d, 0, sizeof(ProbeOut), st);
      cudaEventRecord(e0, st);
      switch (op) {
        case 0: int32_rate_kernel<0><<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
        case 1: int32_rate_kernel<1><<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
        case 2: int32_rate_kernel<2><<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
        case 3: int32_rate_kernel<3><<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
        case 4: int32_rate_kernel<4><<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
        case 5: bulk_rate_kernel<<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
        default: bulk64_rate_kernel<<<grid, kProbeThreads, 0, st>>>(d, 0x2545F491u, trips); break;
      }
      cudaEventRecord(e1, st);
      if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
        rc = fail_cuda(e, "dp_measure_int32_rates: probe");
        break;
      }
      ProbeOut h{};
      float ms = 0.f;
      if ((e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        rc = fail_cuda(e, "dp_measure_int32_rates: read-back");
        break;
      }
      if (rep == 0 || h.cycles_max == 0) continue;
      const double threads_per_sm = (double)bps * kProbeThreads;
      // instructions (probes 0-4) or split evaluations (probes 5, 6) per thread
      const double per_thread = op >= 5 ? (double)trips * 32.0 * 8.0 : (double)trips * kUnroll * kChains;
      out[op == 6 ? 9 : op] = threads_per_sm * per_thread / (double)h.cycles_max;
      clk_sum += (double)h.cycles_max / (ms * 1e3);  // MHz (the slowest block spans about the launch)
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(d, st);
  if (rc != DP_OK) return rc;
  out[6] = (double)ds->sms;
  out[7] = clk_sum / nprobes;
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, ds->device);
  out[8] = clk_khz / 1e3;
  return DP_OK;
}
