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

// RING = 0: read the table in global memory (window too large for shared memory).
// RING = 1: a ring of R = 2^ring_log2 words indexed modulo R.
// RING = 2: the same ring stored twice (word x at x and at x + R), so that the
//           read of ST[i - a_j] is ring[(i mod R) + R - a_j] with no wrap:
//           an add, a load and the operator per offset.
// KREG: offsets held in registers (k <= kSdpMaxKRegs); KFULL: k == kSdpMaxKRegs
// (no per-offset predicate).
template <int OP, int RING, bool KREG, bool KFULL>
__global__ void __launch_bounds__(1024) sdp_kernel(const SdpLaunchArgs args) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int b = blockIdx.x;
  SdpInstDev in = args.insts ? args.insts[b] : args.one;
  uint32_t* st = args.st_off ? args.st_all + args.st_off[b] : in.st;
  const int64_t n = in.n;
  const int k = in.k;
  const int tid = threadIdx.x;
  const int ring_log2 = args.ring_log2;
  const uint32_t R = RING ? (1u << ring_log2) : 0u;
  const uint32_t mask = R - 1u;
  uint32_t* ring = sm;
  int32_t* offs = reinterpret_cast<int32_t*>(sm + (RING == 2 ? 2 * R : R));

  for (int j = tid; j < k; j += blockDim.x) offs[j] = args.insts ? in.a[j] : args.one_offs[j];
  __syncthreads();
  const int32_t a1 = offs[0];
  const int32_t ak = offs[k - 1];
  if (n <= a1) return;
  // per-offset read displacement: -a_j (table), R - a_j (mirrored ring)
  int32_t ro[kSdpMaxKRegs];
  if constexpr (KREG) {
#pragma unroll
    for (int j = 0; j < kSdpMaxKRegs; ++j) {
      const int32_t a = j < k ? offs[j] : offs[0];
      ro[j] = RING == 2 ? (int32_t)R - a : a;
    }
  }
  if constexpr (RING != 0) {
    for (int x = tid; x < a1; x += blockDim.x) {
      const uint32_t v = st[x];
      ring[(uint32_t)x & mask] = v;
      if constexpr (RING == 2) ring[((uint32_t)x & mask) + R] = v;
    }
    __syncthreads();
  }
  const int W = ak < (int)blockDim.x ? ak : (int)blockDim.x;
  uint32_t pos = ((uint32_t)a1 + (uint32_t)tid) & mask;  // (i mod R) for the ring modes
  for (int64_t base = a1; base < n; base += W) {
    const int64_t i = base + tid;
    if (tid < W && i < n) {
      uint32_t v;
      if constexpr (RING == 2) {
        const uint32_t* rp = ring + pos;
        if constexpr (KREG) {
          v = rp[ro[0]];
#pragma unroll
          for (int j = 1; j < kSdpMaxKRegs; ++j)
            if (KFULL || j < k) v = combine<OP>(v, rp[ro[j]]);
        } else {
          v = rp[(int32_t)R - offs[0]];
          for (int j = 1; j < k; ++j) v = combine<OP>(v, rp[(int32_t)R - offs[j]]);
        }
        ring[pos] = v;
        ring[pos + R] = v;
      } else if constexpr (RING == 1) {
        if constexpr (KREG) {
          v = ring[(pos - (uint32_t)ro[0]) & mask];
#pragma unroll
          for (int j = 1; j < kSdpMaxKRegs; ++j)
            if (KFULL || j < k) v = combine<OP>(v, ring[(pos - (uint32_t)ro[j]) & mask]);
        } else {
          v = ring[(pos - (uint32_t)offs[0]) & mask];
          for (int j = 1; j < k; ++j) v = combine<OP>(v, ring[(pos - (uint32_t)offs[j]) & mask]);
        }
        ring[pos] = v;
      } else {
        if constexpr (KREG) {
          v = st[i - ro[0]];
#pragma unroll
          for (int j = 1; j < kSdpMaxKRegs; ++j)
            if (KFULL || j < k) v = combine<OP>(v, st[i - ro[j]]);
        } else {
          v = st[i - offs[0]];
          for (int j = 1; j < k; ++j) v = combine<OP>(v, st[i - offs[j]]);
        }
      }
      st[i] = v;
    }
    pos = (pos + (uint32_t)W) & mask;
    __syncthreads();
  }
}

template <int OP, int RING, bool KREG, bool KFULL>
cudaError_t launch_variant(const SdpLaunchArgs& a, size_t smem, cudaStream_t stream) {
  auto kern = sdp_kernel<OP, RING, KREG, KFULL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.ninst, a.threads, smem, stream>>>(a);
  return cudaGetLastError();
}

template <int OP, int RING>
cudaError_t launch_k(const SdpLaunchArgs& a, int kmax, bool all_full, size_t smem, cudaStream_t stream) {
  if (kmax > kSdpMaxKRegs) return launch_variant<OP, RING, false, false>(a, smem, stream);
  if (all_full) return launch_variant<OP, RING, true, true>(a, smem, stream);
  return launch_variant<OP, RING, true, false>(a, smem, stream);
}

template <int OP>
cudaError_t launch_op(const SdpLaunchArgs& a, int kmax, bool all_full, size_t smem, cudaStream_t stream) {
  const int mode = sdp_ring_mode(a.ring_log2);
  if (mode == 2) return launch_k<OP, 2>(a, kmax, all_full, smem, stream);
  if (mode == 1) return launch_k<OP, 1>(a, kmax, all_full, smem, stream);
  return launch_k<OP, 0>(a, kmax, all_full, smem, stream);
}

}  // namespace

int sdp_ring_mode(int ring_log2) {
  if (ring_log2 <= 0) return 0;
  return ring_log2 <= kSdpMirrorMaxLog2 ? 2 : 1;
}

size_t sdp_smem_bytes(int ring_log2, int kmax) {
  const int mode = sdp_ring_mode(ring_log2);
  const size_t ring = mode == 0 ? 0 : ((size_t)1 << ring_log2) * 4 * (mode == 2 ? 2 : 1);
  return ring + (size_t)kmax * 4;
}

cudaError_t launch_sdp(const SdpLaunchArgs& a, cudaStream_t stream) {
  if (a.ninst <= 0) return cudaSuccess;
  // kmax: largest k in the launch (the host passes it through one.k for both
  // paths); kfull: every instance has exactly kSdpMaxKRegs offsets
  const int kmax = a.one.k;
  const bool kfull = a.kfull != 0;
  const size_t smem = sdp_smem_bytes(a.ring_log2, kmax);
  if (a.op == 0) return launch_op<0>(a, kmax, kfull, smem, stream);
  return launch_op<1>(a, kmax, kfull, smem, stream);
}

}  // namespace dpk
