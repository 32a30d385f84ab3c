// sdp_kernels.cuh -- launch-side declarations of the S-DP kernels.
//
// Problem (paper Definition 1, Eq. (1)):  ST[i] = (x)_{j=1..k} ST[i - a_j]
// for i >= a_1, with a_1 > ... > a_k > 0 and ST[0 .. a_1-1] preset;
// (x) = min or + modulo 2^32 on uint32.
//
// Parallel width.  Every offset is at least a_k, so cells i .. i + a_k - 1
// depend only on cells below i: one step fills W = min(a_k, threads) cells at
// once (the paper's pipeline of Fig. 2 advances one head position per step;
// here a whole block of cells per step).  Only the last a_1 values are ever
// read, so they live in a shared-memory ring of R >= a_1 + W words (R a power
// of two, stored twice when it fits so that no read wraps); each step reads
// the ring, writes the new cells to the ring and, coalesced, to the table in
// global memory.  Consecutive threads handle
// consecutive cells, so for any offset the ring reads of a warp are 32
// consecutive words: bank-conflict free.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpk {

constexpr int kSdpMaxKRegs = 32;       // offsets kept in registers up to this k
constexpr int kSdpMaxK = 1024;         // offsets per instance (shared-memory copy)
constexpr int kSdpRingMaxLog2 = 15;    // ring of at most 32768 words (128 KiB)
constexpr int kSdpMirrorMaxLog2 = 14;  // mirrored ring (two copies) up to 2 x 16384 words

struct SdpInstDev {
  uint32_t* st;        // table (set by the launcher, or st_all + st_off[b])
  int64_t n;           // table length
  const int32_t* a;    // offsets on the device (batched path)
  int32_t k;
  int32_t a_off;       // offset of this instance's offsets in a shared array
};

struct SdpLaunchArgs {
  const SdpInstDev* insts;   // batched: device array; single: nullptr (use `one`)
  SdpInstDev one;
  int32_t ninst;
  int32_t op;                // 0 = min, 1 = add mod 2^32
  int32_t ring_log2;         // 0: no ring (read the table in global memory)
  int32_t threads;
  int32_t kfull;             // 1: every instance has exactly kSdpMaxKRegs offsets
  int32_t pad_;
  uint32_t* st_all;          // batched tables
  const int64_t* st_off;
  int32_t* status;
  int32_t one_offs[kSdpMaxK];  // single path: offsets by value
};

int sdp_ring_mode(int ring_log2);     // 0: table in global memory, 1: ring, 2: mirrored ring
size_t sdp_smem_bytes(int ring_log2, int kmax);
cudaError_t launch_sdp(const SdpLaunchArgs& a, cudaStream_t st);

}  // namespace dpk
