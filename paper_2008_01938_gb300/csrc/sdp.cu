// sdp.cu -- sm_103a kernels for the simplified DP problem (paper Definition 1,
// Eq. (1)).  One thread block per instance; see sdp_kernels.cuh.
#include <cstdint>

#include "dp_common.cuh"
#include "sdp_kernels.cuh"

namespace dpk {

namespace {

template <int OP>
__device__ __forceinline__ uint32_t combine(uint32_t x, uint32_t y) {
  if constexpr (OP == 0) return x < y ? x : y;
  return x + y;  // wraps modulo 2^32
}

// RING: keep the last values in a shared-memory ring; otherwise read the table.
// KREG: offsets held in registers (k <= kSdpMaxKRegs).
template <int OP, bool RING, bool KREG>
__global__ void __launch_bounds__(1024) sdp_kernel(const SdpLaunchArgs args) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int b = blockIdx.x;
  SdpInstDev in = args.insts ? args.insts[b] : args.one;
  uint32_t* st = args.st_off ? args.st_all + args.st_off[b] : in.st;
  const int64_t n = in.n;
  const int k = in.k;
  const int tid = threadIdx.x;
  const int ring_log2 = args.ring_log2;
  const uint32_t mask = (1u << ring_log2) - 1u;
  uint32_t* ring = sm;
  int32_t* offs = reinterpret_cast<int32_t*>(sm + (RING ? (1u << ring_log2) : 0u));

  for (int j = tid; j < k; j += blockDim.x) offs[j] = args.insts ? in.a[j] : args.one_offs[j];
  __syncthreads();
  const int32_t a1 = offs[0];
  const int32_t ak = offs[k - 1];
  if (n <= a1) return;
  int32_t ro[kSdpMaxKRegs];
  if constexpr (KREG) {
#pragma unroll
    for (int j = 0; j < kSdpMaxKRegs; ++j) ro[j] = j < k ? offs[j] : offs[0];
  }
  if constexpr (RING) {
    for (int x = tid; x < a1; x += blockDim.x) ring[x & mask] = st[x];
    __syncthreads();
  }
  const int W = ak < (int)blockDim.x ? ak : (int)blockDim.x;
  for (int64_t base = a1; base < n; base += W) {
    const int64_t i = base + tid;
    if (tid < W && i < n) {
      uint32_t v;
      if constexpr (KREG) {
        if constexpr (RING) {
          v = ring[(uint32_t)(i - ro[0]) & mask];
#pragma unroll
          for (int j = 1; j < kSdpMaxKRegs; ++j)
            if (j < k) v = combine<OP>(v, ring[(uint32_t)(i - ro[j]) & mask]);
        } else {
          v = st[i - ro[0]];
#pragma unroll
          for (int j = 1; j < kSdpMaxKRegs; ++j)
            if (j < k) v = combine<OP>(v, st[i - ro[j]]);
        }
      } else {
        if constexpr (RING) {
          v = ring[(uint32_t)(i - offs[0]) & mask];
          for (int j = 1; j < k; ++j) v = combine<OP>(v, ring[(uint32_t)(i - offs[j]) & mask]);
        } else {
          v = st[i - offs[0]];
          for (int j = 1; j < k; ++j) v = combine<OP>(v, st[i - offs[j]]);
        }
      }
      if constexpr (RING) ring[(uint32_t)i & mask] = v;
      st[i] = v;
    }
    __syncthreads();
  }
}

template <int OP, bool RING, bool KREG>
cudaError_t launch_variant(const SdpLaunchArgs& a, size_t smem, cudaStream_t stream) {
  auto kern = sdp_kernel<OP, RING, KREG>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.ninst, a.threads, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t sdp_smem_bytes(int ring_log2, int kmax) {
  return (ring_log2 > 0 ? ((size_t)1 << ring_log2) * 4 : 0) + (size_t)kmax * 4;
}

cudaError_t launch_sdp(const SdpLaunchArgs& a, cudaStream_t stream) {
  if (a.ninst <= 0) return cudaSuccess;
  const bool ring = a.ring_log2 > 0;
  // kmax: largest k in the launch (the host passes it through one.k for both paths)
  const int kmax = a.one.k;
  const bool kreg = kmax <= kSdpMaxKRegs;
  const size_t smem = sdp_smem_bytes(a.ring_log2, kmax);
  if (a.op == 0) {
    if (ring) return kreg ? launch_variant<0, true, true>(a, smem, stream) : launch_variant<0, true, false>(a, smem, stream);
    return kreg ? launch_variant<0, false, true>(a, smem, stream) : launch_variant<0, false, false>(a, smem, stream);
  }
  if (ring) return kreg ? launch_variant<1, true, true>(a, smem, stream) : launch_variant<1, true, false>(a, smem, stream);
  return kreg ? launch_variant<1, false, true>(a, smem, stream) : launch_variant<1, false, false>(a, smem, stream);
}

}  // namespace dpk
