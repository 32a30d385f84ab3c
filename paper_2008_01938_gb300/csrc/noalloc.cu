// noalloc.cu -- mcm_solve_noalloc: the int32-cost MCM solve of mcm_solve
// without any memory allocation.
//
// mcm_solve takes its workspace (packed panels, flags, accumulators, dims)
// from the stream-ordered allocator and its work queue from a per-size plan
// cache in fresh device memory.  Some callers cannot allocate at the moment
// they solve: a process that has handed all free HBM to its own allocator
// (a cudaMallocAsync there fails or forces the pool to grow), or a
// latency-critical loop that must not enter the allocator at all.  This entry
// point serves them: its scratch is one file-scope __device__ array of fixed
// size, which exists from the moment this translation unit's module is
// loaded, and everything a solve needs inside it -- the work queue included
// -- is written by a set-up kernel at the start of each call.
//
// The kernels that solve are the ones mcm_solve runs (prologue and
// persistent main kernel); only the way their arguments are laid out
// differs.  The paper has no counterpart to this entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "api_internal.h"
#include "dp_common.cuh"
#include "mcm_kernels.cuh"

namespace {

using dpk::kTile;
using dpk::McmInstDev;
using dpk::McmTask;

constexpr int32_t kMaxN = 1024;                            // largest chain the scratch holds
constexpr int kMaxNt = kMaxN / kTile;                      // 32 tiles per side (one warp lane per tile row)
constexpr int64_t kMaxTiles = (int64_t)kMaxNt * (kMaxNt + 1) / 2;
// a tile on tile-diagonal D < kMaxNt has fewer than kMaxNt / 2 bulk levels
constexpr int kMaxParts = (kMaxNt / 2 + dpk::kLevelsPerPart - 1) / dpk::kLevelsPerPart;
constexpr int64_t kMaxTasks = kMaxTiles * (1 + kMaxParts);  // a finisher and its bulk parts per tile
constexpr int kMaxDevices = 64;

constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

// Scratch layout (byte offsets; every region starts on a 256-byte boundary).
constexpr int64_t kAF = 0;                                            // row panels, int32 packed
constexpr int64_t kBF = kAF + align256(kMaxTiles * kTile * kTile * 4);  // column panels
constexpr int64_t kFlags = kBF + align256(kMaxTiles * kTile * kTile * 4);
constexpr int64_t kCounters = kFlags + align256(kMaxTiles * 4);
constexpr int64_t kQueue = kCounters + align256(kMaxTiles * 4);
constexpr int64_t kAcc = kQueue + 256;                                // one 32x32 u64 slot per tile
constexpr int64_t kPP = kAcc + align256(kMaxTiles * kTile * kTile * 8);
constexpr int64_t kPK = kPP + align256(((int64_t)kMaxNt * kTile + 32) * 4);
constexpr int64_t kInsts = kPK + align256((int64_t)kMaxNt * kTile * 4);
constexpr int64_t kTasks = kInsts + 256;
constexpr int64_t kAccSlot = kTasks + align256(kMaxTasks * (int64_t)sizeof(McmTask));
constexpr int64_t kScratchBytes = kAccSlot + align256(kMaxTiles * 4);  // 8,691,968 bytes

static_assert(sizeof(McmInstDev) <= 256, "chain record must fit its region");
static_assert(sizeof(McmTask) == 16, "task layout");
static_assert(kMaxNt == 32, "the queue builder maps one warp lane to each tile row");

__device__ __align__(256) uint8_t g_mcm_scratch[kScratchBytes];

// The work split of a tile on tile-diagonal D (see kLevelsPerPart): bulk
// part q covers levels [rmin + q*kLevelsPerPart, r1(q)], r1(q) = min(that +
// kLevelsPerPart - 1, fin_lo - 1); the finisher keeps [fin_lo, D - 1].
struct TileSplit {
  int rmin, fin_lo, nparts;
};

__host__ __device__ inline TileSplit tile_split(int D) {
  TileSplit t{1, 0, 0};
  if (D < 2) return t;
  t.rmin = (D + 1) / 2;
  t.fin_lo = D - 1;
  if (t.fin_lo - t.rmin < dpk::kMinBulkLevels) t.fin_lo = t.rmin;
  t.nparts = (t.fin_lo - t.rmin + dpk::kLevelsPerPart - 1) / dpk::kLevelsPerPart;
  return t;
}

__host__ __device__ inline int part_r1(const TileSplit& t, int q) {
  const int r1 = t.rmin + q * dpk::kLevelsPerPart + dpk::kLevelsPerPart - 1;
  return r1 < t.fin_lo - 1 ? r1 : t.fin_lo - 1;
}

// Queue length for a chain of nt tiles per side.
int64_t queue_length(int nt) {
  int64_t q = 0;
  for (int D = 0; D < nt; ++D) q += (int64_t)(nt - D) * (1 + tile_split(D).nparts);
  return q;
}

// Bucket (tile-diagonal at which a task becomes ready) of bulk part q.
__device__ __forceinline__ int part_bucket(const TileSplit& t, int q) { return part_r1(t, q) + 1; }

// Writes everything a solve expects in the scratch before it starts:
//   * the work queue, in the order the host queue builder uses (by bucket;
//     inside a bucket the finishers of tile-diagonal b by tile row, then the
//     bulk parts by (tile row, tile column));
//   * the chain record, the per-tile accumulator slot table (slot = tile
//     index, -1 for a tile without bulk parts);
//   * the state that must start at zero: tile flags, bulk counters and the
//     queue counter; and the accumulators, which start at all ones (+inf).
// Block 0 (1024 threads: warp = bucket, lane = tile row) builds the queue;
// the other blocks fill the accumulators.
__global__ void __launch_bounds__(1024) mcm_noalloc_setup_kernel(uint8_t* scratch, int32_t n, int32_t nt,
                                                                 int32_t ntasks, int32_t* status) {
  const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
  if (blockIdx.x > 0) {
    ulonglong2* acc = reinterpret_cast<ulonglong2*>(scratch + kAcc);
    const int64_t total = ntiles * kTile * kTile / 2;
    const ulonglong2 ones = make_ulonglong2(~0ull, ~0ull);
    for (int64_t x = (int64_t)(blockIdx.x - 1) * blockDim.x + threadIdx.x; x < total;
         x += (int64_t)(gridDim.x - 1) * blockDim.x)
      acc[x] = ones;
    return;
  }
  __shared__ int s_tot[32], s_base[32];
  McmTask* tasks = reinterpret_cast<McmTask*>(scratch + kTasks);
  int32_t* flags = reinterpret_cast<int32_t*>(scratch + kFlags);
  int32_t* counters = reinterpret_cast<int32_t*>(scratch + kCounters);
  int32_t* accslot = reinterpret_cast<int32_t*>(scratch + kAccSlot);
  const int tid = threadIdx.x, b = tid >> 5, lane = tid & 31;

  // per-tile tables and the zero-initialised state
  for (int idx = tid; idx < nt * nt; idx += blockDim.x) {
    const int I = idx / nt, J = idx % nt;
    if (J < I) continue;
    const int64_t tix = (int64_t)I * nt - (int64_t)I * (I - 1) / 2 + (J - I);
    flags[tix] = 0;
    counters[tix] = 0;
    accslot[tix] = tile_split(J - I).nparts > 0 ? (int32_t)tix : -1;
  }
  if (tid < 4) reinterpret_cast<int32_t*>(scratch + kQueue)[tid] = 0;
  if (tid == 0) {
    McmInstDev in{};
    in.n = n;
    in.nt = nt;
    *reinterpret_cast<McmInstDev*>(scratch + kInsts) = in;  // p, m, s, shift: set by the prologue
  }

  // Bucket b holds the finishers of tile-diagonal b and every bulk part whose
  // last level is b - 1.  Lane D marks whether tile-diagonal D has such a part.
  bool has = false;
  if (b < nt && lane < nt) {
    const TileSplit t = tile_split(lane);
    for (int q = 0; q < t.nparts; ++q) has |= part_bucket(t, q) == b;
  }
  const uint32_t mask = __ballot_sync(0xffffffffu, has);
  // this lane's tile row I = lane: parts of tile-diagonals D in mask with I + D < nt
  const int I = lane;
  const uint32_t lim = (b < nt && I < nt) ? mask & ((2u << (nt - 1 - I)) - 1u) : 0u;
  const int cnt = __popc(lim);
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_tot[b] = (b < nt ? nt - b : 0) + incl;
  __syncthreads();
  if (b == 0) {
    const int v = s_tot[lane];
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    s_base[lane] = x - v;
    if (lane == 31 && x != ntasks) dpk::set_status(status, DP_ECUDA);  // host and device counts disagree
  }
  __syncthreads();
  if (b >= nt) return;
  if (I < nt - b) {  // finisher of tile (I, I + b)
    const TileSplit t = tile_split(b);
    McmTask f{};
    f.inst = 0;
    f.I = (int16_t)I;
    f.J = (int16_t)(I + b);
    f.kind = 0;
    f.r_lo = (int16_t)(b < 2 ? 1 : t.fin_lo);
    f.r_hi = (int16_t)(b < 2 ? 0 : b - 1);
    f.nparts = (int16_t)t.nparts;
    tasks[s_base[b] + I] = f;
  }
  int pos = s_base[b] + (nt - b) + (incl - cnt);
  for (uint32_t bits = lim; bits; bits &= bits - 1) {
    const int D = __ffs(bits) - 1;
    const TileSplit t = tile_split(D);
    for (int q = 0; q < t.nparts; ++q) {
      if (part_bucket(t, q) != b) continue;
      McmTask pt{};
      pt.inst = 0;
      pt.I = (int16_t)I;
      pt.J = (int16_t)(I + D);
      pt.r_lo = (int16_t)(t.rmin + q * dpk::kLevelsPerPart);
      pt.r_hi = (int16_t)part_r1(t, q);
      pt.kind = 1;
      tasks[pos++] = pt;
    }
  }
}

// Per-device set-up, done once by the first call on each device.
struct NoAllocDev {
  bool ready = false;
  uint8_t* scratch = nullptr;
  int sms = 0;
  int occ = 0;
};
NoAllocDev g_dev[kMaxDevices];
std::mutex g_mu;

dp_status setup(NoAllocDev* out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dph::fail_cuda(e, "mcm_solve_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return dph::fail(DP_EINVAL, "mcm_solve_noalloc: device ordinal %d outside [0, %d)", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  NoAllocDev& d = g_dev[dev];
  if (!d.ready) {
    // the address of this device's copy of the scratch array (this device is current)
    void* ptr = nullptr;
    if ((e = cudaGetSymbolAddress(&ptr, g_mcm_scratch)) != cudaSuccess)
      return dph::fail_cuda(e, "mcm_solve_noalloc: cudaGetSymbolAddress(scratch)");
    if ((e = dpk::mcm_configure(false)) != cudaSuccess)
      return dph::fail_cuda(e, "mcm_solve_noalloc: configure MCM kernel");
    if ((e = dpk::mcm_preload(false)) != cudaSuccess) return dph::fail_cuda(e, "mcm_solve_noalloc: load kernels");
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, mcm_noalloc_setup_kernel)) != cudaSuccess)
      return dph::fail_cuda(e, "mcm_solve_noalloc: load set-up kernel");
    int sms = 0, occ = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return dph::fail_cuda(e, "mcm_solve_noalloc: SM count");
    if ((e = dpk::mcm_occupancy(false, &occ)) != cudaSuccess)
      return dph::fail_cuda(e, "mcm_solve_noalloc: occupancy");
    d.scratch = static_cast<uint8_t*>(ptr);
    d.sms = sms;
    d.occ = occ < 1 ? 1 : occ;
    d.ready = true;
  }
  *out = d;
  return DP_OK;
}

}  // namespace

extern "C" dp_status mcm_solve_noalloc(const int32_t* p, int32_t n, int32_t* m, int16_t* s, int32_t* status_dev,
                                       void* stream) {
  if (!p || !m || !s || !status_dev) return dph::fail(DP_EINVAL, "mcm_solve_noalloc: NULL pointer argument");
  if (n < 1 || n > kMaxN)
    return dph::fail(DP_EINVAL, "mcm_solve_noalloc: n = %d outside [1, %d] (the size of its static scratch)", n,
                     kMaxN);
  NoAllocDev d;
  dp_status rc = setup(&d);
  if (rc != DP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nt = (n + kTile - 1) / kTile;
  const int64_t ntiles = (int64_t)nt * (nt + 1) / 2;
  const int64_t ntasks = queue_length(nt);
  uint8_t* w = d.scratch;

  const int fill_blocks = (int)std::min<int64_t>(d.sms, (ntiles * kTile * kTile / 2 + 1023) / 1024);
  mcm_noalloc_setup_kernel<<<1 + fill_blocks, 1024, 0, st>>>(w, n, nt, (int32_t)ntasks, status_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dph::fail_cuda(e, "mcm_solve_noalloc: launch set-up kernel");

  dpk::McmLaunchArgs a{};
  a.insts = reinterpret_cast<McmInstDev*>(w + kInsts);
  a.tasks = reinterpret_cast<const McmTask*>(w + kTasks);
  a.ninst = 1;
  a.ntasks = (int32_t)ntasks;
  a.af = w + kAF;
  a.bf = w + kBF;
  a.flags = reinterpret_cast<int32_t*>(w + kFlags);
  a.counters = reinterpret_cast<int32_t*>(w + kCounters);
  a.accslot = reinterpret_cast<const int32_t*>(w + kAccSlot);
  a.acc = reinterpret_cast<unsigned long long*>(w + kAcc);
  a.pp = reinterpret_cast<int32_t*>(w + kPP);
  a.pk = reinterpret_cast<uint32_t*>(w + kPK);
  a.queue = reinterpret_cast<int32_t*>(w + kQueue);
  a.status = status_dev;
  a.spin_limit = dph::spin_limit();
  a.drop_task = -1;
  a.p_all = p;
  a.p_off = nullptr;
  a.tab_off = nullptr;
  a.m_all = m;
  a.s_all = s;
  if ((e = dpk::launch_mcm_prologue(a, false, st)) != cudaSuccess)
    return dph::fail_cuda(e, "mcm_solve_noalloc: launch prologue");
  const int grid = (int)std::max<int64_t>(2, std::min<int64_t>((int64_t)d.sms * d.occ, ntasks));
  if ((e = dpk::launch_mcm_main(a, false, grid, st)) != cudaSuccess)
    return dph::fail_cuda(e, "mcm_solve_noalloc: launch MCM kernel");
  return DP_OK;
}
