// mcm.cu -- sm_103a kernels for the matrix-chain multiplication table
// (paper Section IV-A, Eq. (2)).  See mcm_kernels.cuh for the decomposition
// and the packed cost encodings.
#include <cstdint>
#include <type_traits>

#include "dp_common.cuh"
#include "mcm_kernels.cuh"

namespace dpk {

namespace {

constexpr int T = kTile;
constexpr uint32_t kFinPollNs = 64;   // finisher mbarrier waits (int32): longest sleep between polls
constexpr uint32_t kFlagPollNs = 32;  // flag and counter waits (int32): longest sleep between polls

// Flag wait of the int32 instances (shorter polling), or the common one.
template <bool I64>
__device__ __forceinline__ bool wait_flag(const int32_t* flag, int32_t target, long long limit, int32_t* status) {
  if constexpr (I64)
    return wait_flag_geq(flag, target, limit, status);
  else
    return wait_flag_geq_cap<kFlagPollNs>(flag, target, limit, status);
}
constexpr int kDiagRows = 2 * T;  // cell diagonals e = lj - li in [-31, 31] (dI = e + 31), one spare row

template <bool I64>
struct Cost {
  using E = typename std::conditional<I64, unsigned long long, uint32_t>::type;
  static constexpr int KB = I64 ? 16 : 32;  // k bits in the 64-bit (value, k) key
};

__device__ __forceinline__ int64_t tile_index(const McmInstDev& in, int I, int J) {
  return in.tile_base + (int64_t)I * in.nt - (int64_t)I * (I - 1) / 2 + (J - I);
}

// Shared-memory carve-up (byte offsets); identical for all blocks.
//
// In-tile wavefront arrays (finisher of an off-diagonal tile) start at STA and
// reuse the bulk-copy stages (every copy of the task has landed before they
// are written); where they need more room than the stages, the finisher
// buffers that follow are moved up.  Row indices of the U^T / L tables:
//   int32: row = t + 32 for t in [-32, 63] (96 rows, constant offsets per step)
//   int64: row = t & 63 (64 rows; saves the shared memory that keeps two
//          int64 blocks resident per SM)
// Rows outside t = 0 .. 30 hold zeros.
template <bool I64>
struct Smem {
  static constexpr int ES = I64 ? 8 : 4;
  static constexpr int TILE = T * T * ES;
  static constexpr bool kPadRows = !I64;
  // int32: the cell-value arrays Xr / Xc live outside the stage area, so
  // their entries for cells that do not exist are set to all ones once per
  // block and stay so (every existing cell is written before it is read).
  static constexpr bool kXOut = !I64;
  static constexpr int kRows = kPadRows ? 96 : 64;
  static constexpr int kRowOff = kPadRows ? 32 : 0;
  static constexpr int UPW = I64 ? 34 : 36;                       // U^T pitch: 16-byte rows, conflict-free
  static constexpr int BARS = 0;                                 // 9 mbarriers + task slot
  static constexpr int STA = 128;                                // [group][stage] row panels
  static constexpr int STB = STA + 4 * TILE;                     // [group][stage] column panels
  static constexpr int STPK = STB + 4 * TILE;                    // [group][stage] 32 x u32 dims
  static constexpr int STEND = STPK + 4 * 128;
  static constexpr int XBYTES = kDiagRows * T * ES;
  static constexpr int WUP = STA;                                // Up[row(t)][li] = m[IT+li][IT+t]
  static constexpr int WLP = WUP + ((kRows * UPW * ES + 127) / 128) * 128;  // Lp[row(u)][lj] = m[JT+u+1][JT+lj]
  static constexpr int WPKI = WLP + kRows * T * ES;               // PKIp[row(t)] = p[IT+t+1]
  static constexpr int WPKJ = WPKI + kRows * 4;                  // PKJp[row(u)] = p[JT+u+1]
  static constexpr int WXIN = (WPKJ + kRows * 4 + 127) / 128 * 128;  // Xr, Xc when inside the stage area
  static constexpr int WEND = kXOut ? WXIN : WXIN + 2 * XBYTES;
  static constexpr int FINU = ((STEND > WEND ? STEND : WEND) + 127) / 128 * 128;  // row panel of (I,I)
  static constexpr int FINL = FINU + TILE;                       // column panel of diagonal tile (J,J)
  static constexpr int FINBROW = FINL + TILE;                    // boundary row (one tile row)
  static constexpr int FINPP = FINBROW + 256;                    // p[32I .. 32I+31]
  static constexpr int FINPKI = FINPP + 128;                     // p[32I+1 ..] << S
  static constexpr int FINPKJ = FINPKI + 128;                    // p[32J+1 ..] << S
  static constexpr int FINACC = FINPKJ + 128;                    // bulk-task partial minima
  static constexpr int BEST = FINACC + T * T * 8;                // running (value, k) keys
  static constexpr int WXR = kXOut ? BEST + T * T * 8 : WXIN;    // Xr[e+31][li]: final value of cell (li, li+e)
  static constexpr int WXC = WXR + XBYTES;                       // Xc[e+31][lj]: final value of cell (lj-e, lj)
  static constexpr int TOTAL = kXOut ? WXC + XBYTES : BEST + T * T * 8;
  static constexpr int XV = STA;                                 // diagonal tiles: the tile's values
  __host__ __device__ static constexpr int row(int t) { return kPadRows ? t + kRowOff : (t & 63); }
  static_assert(WXR % 16 == 0 && WUP % 16 == 0 && (UPW * ES) % 16 == 0, "16-byte vector rows");
};

__device__ __forceinline__ void bar_compute() {  // the 256 compute threads only
  asm volatile("bar.sync 1, %0;" ::"n"(kComputeThreads) : "memory");
}

// Barrier over the 256 compute threads that also ANDs a predicate, so a
// decision taken after per-thread bounded waits is the same in every thread
// (every later named barrier is then reached by all 256 or by none).
__device__ __forceinline__ bool bar_compute_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kComputeThreads)
      : "memory");
  return r != 0;
}

template <typename E>
__device__ __forceinline__ E umin(E a, E b) { return a < b ? a : b; }

// ---------------------------------------------------------------------------
// In-tile solve of an off-diagonal tile (I, J).
// X is the tile; its in-tile splits are
//   column splits k = IT + t, li <= t <= 30:  U[li][t] + X[t+1][lj] + w
//   row splits    k = JT + u,  0 <= u < lj:   X[li][u] + L[u][lj] + w
// with U = the diagonal tile (I, I), L = rows shifted by one of (J, J) and
// w = p[IT+li] p[k+1] p[JT+lj+1]; the boundary split k = IT + 31 and the
// external splits are known before the solve starts.
//
// Cell (li, lj) lies on cell diagonal e = lj - li in [-31, 31] and depends
// only on cells of lower diagonals, so the tile is solved in the paper's
// diagonal order (Figs. 5-7), one diagonal per step: in step e every cell
// pulls the candidate of its row split and of its column split whose operand
// lies on diagonal e (exactly one of each), and the cells of diagonal e + 1,
// whose last operands were on diagonal e, become final.  Warp w owns rows
// 4w .. 4w+3 and lane = column.
//
// Each thread keeps one running minimum per cell (values only).  The operands
// that do not depend on the tile move predictably from step to step and are
// loaded ahead of the barrier: the row split of cell (li, lj) at step e uses
// L[li + e][lj], the thread's 4 rows use 4 consecutive rows of L, so a
// 4-entry register window gains one new row per step; U[li][lj - e - 1] and
// p[IT + lj - e] come from one 16-byte load and one word per step.  The cell
// values themselves are exchanged through two diagonal-major arrays written
// once, when a cell becomes final: Xr (indexed by row, the row-split operand)
// and Xc (indexed by column, the column-split operand).
//
// Out-of-range operands are read from zero rows (U, L, dims) and from
// all-ones entries (cells that do not exist), so no candidate needs a
// predicate: a missing cell yields an all-ones candidate, and a candidate
// whose operand exists but whose split is outside the cell's range only
// arises after the cell was finalised (its running minimum is then dead).
// The smallest minimising split is recovered after the tile is published, by
// scanning the splits of each cell in increasing k.
// ---------------------------------------------------------------------------
template <typename E>
struct Vec4 {
  E v[4];
};

template <typename E>
__device__ __forceinline__ Vec4<E> lds4(const E* p) {  // 4 consecutive elements, 16-byte aligned
  Vec4<E> r;
  if constexpr (sizeof(E) == 4) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    r.v[0] = q.x, r.v[1] = q.y, r.v[2] = q.z, r.v[3] = q.w;
  } else {
    const ulonglong2 q0 = *reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 q1 = *reinterpret_cast<const ulonglong2*>(p + 2);
    r.v[0] = q0.x, r.v[1] = q0.y, r.v[2] = q1.x, r.v[3] = q1.y;
  }
  return r;
}

// a[r] for a runtime r in 0..3 (any r: only its low two bits are used) as
// a two-level tree of predicated selects (a C conditional chain here is
// compiled to divergent branches, which cost several times more inside the
// wavefront step).
template <typename E>
__device__ __forceinline__ E sel4(int r, E a0, E a1, E a2, E a3) {
  if constexpr (sizeof(E) == 4) {
    uint32_t v;
    asm("{\n\t.reg .pred p0, p1;\n\t.reg .b32 lo, hi, b;\n\t"
        "and.b32 b, %5, 1;\n\tsetp.ne.u32 p0, b, 0;\n\tand.b32 b, %5, 2;\n\tsetp.ne.u32 p1, b, 0;\n\t"
        "selp.b32 lo, %2, %1, p0;\n\tselp.b32 hi, %4, %3, p0;\n\tselp.b32 %0, hi, lo, p1;\n\t}"
        : "=r"(v)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(r));
    return v;
  } else {
    unsigned long long v;
    asm("{\n\t.reg .pred p0, p1;\n\t.reg .b64 lo, hi;\n\t.reg .b32 b;\n\t"
        "and.b32 b, %5, 1;\n\tsetp.ne.u32 p0, b, 0;\n\tand.b32 b, %5, 2;\n\tsetp.ne.u32 p1, b, 0;\n\t"
        "selp.b64 lo, %2, %1, p0;\n\tselp.b64 hi, %4, %3, p0;\n\tselp.b64 %0, hi, lo, p1;\n\t}"
        : "=l"(v)
        : "l"(a0), "l"(a1), "l"(a2), "l"(a3), "r"(r));
    return v;
  }
}

// a[r] where p0 and p1 are bits 0 and 1 of r, already computed.
template <typename E>
__device__ __forceinline__ E sel4p(bool p0, bool p1, E a0, E a1, E a2, E a3) {
  const E lo = p0 ? a1 : a0, hi = p0 ? a3 : a2;
  return p1 ? hi : lo;
}

// Shared-memory store of v at 32-bit shared address addr when p holds.
template <typename E>
__device__ __forceinline__ void sts_if(bool p, uint32_t addr, E v) {
  if constexpr (sizeof(E) == 4)
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.u32 [%1], %2;\n\t}" ::"r"((uint32_t)p),
                 "r"(addr), "r"(v)
                 : "memory");
  else
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t@q st.shared.u64 [%1], %2;\n\t}" ::"r"((uint32_t)p),
                 "r"(addr), "l"(v)
                 : "memory");
}

// ---------------------------------------------------------------------------
// Bulk segment reductions (one compute group, 128 threads, 4 x 2 cells each).
// ---------------------------------------------------------------------------

// int32 costs, chunks of 2^LOGC aligned splits.
template <int LOGC>
__device__ __forceinline__ void seg_i32(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                        const uint32_t* __restrict__ PK, const uint32_t (&P)[4][2],
                                        unsigned long long (&best)[4][2], int ty, int tx, int S, int KT) {
  constexpr int C = 1 << LOGC;
#pragma unroll 1
  for (int c0 = 0; c0 < T; c0 += C) {
    uint32_t acc[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = 0xFFFFFFFFu;
    // One split evaluation is a multiply-add on the FMA pipe (weight plus the
    // row-panel key) and a fused add-and-minimum (__viaddmin_u32, one ALU-pipe
    // instruction) that adds the column-panel key and folds the candidate
    // into the running minimum: two instructions, one on each integer pipe.
#pragma unroll
    for (int kk = 0; kk < C; kk += 2) {
      const uint4 a0 = *reinterpret_cast<const uint4*>(A + (c0 + kk) * T + 4 * ty);
      const uint2 b0 = *reinterpret_cast<const uint2*>(B + (c0 + kk) * T + 2 * tx);
      const uint4 a1 = *reinterpret_cast<const uint4*>(A + (c0 + kk + 1) * T + 4 * ty);
      const uint2 b1 = *reinterpret_cast<const uint2*>(B + (c0 + kk + 1) * T + 2 * tx);
      const uint32_t pk0 = PK[c0 + kk], pk1 = PK[c0 + kk + 1];
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
        const unsigned long long v = acc[r][c] >> S;
        const unsigned long long k = (unsigned)(KT + c0) + (acc[r][c] & (C - 1));
        best[r][c] = umin(best[r][c], (v << 32) | k);
      }
  }
}

// int64 costs: entries already carry the split index in their low 16 bits.
__device__ __forceinline__ void seg_i64(const unsigned long long* __restrict__ A,
                                        const unsigned long long* __restrict__ B,
                                        const uint32_t* __restrict__ PK, const uint32_t (&P)[4][2],
                                        unsigned long long (&best)[4][2], int ty, int tx) {
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
      for (int c = 0; c < 2; ++c)
        best[r][c] = umin(best[r][c], (unsigned long long)P[r][c] * pk + av[r] + bv[c]);
  }
}

// Walks the external segments of a task in the order both roles agree on.
template <typename F>
__device__ __forceinline__ void for_each_segment(const McmTask& t, F&& body) {
  int q = 0;
  for (int r = t.r_lo; r <= t.r_hi; ++r) {
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int K = h == 0 ? t.I + r : t.J - r;
      if (h == 1 && K == t.I + r) continue;
      if (K < t.I + 1 || K > t.J - 1) continue;
      body(K, q);
      ++q;
    }
  }
}

template <bool I64, bool W>
__global__ void __launch_bounds__(kMcmThreads, I64 ? 2 : 3) mcm_main_kernel(const McmLaunchArgs a) {
  using E = typename Cost<I64>::E;
  constexpr int KB = Cost<I64>::KB;
  using SM = Smem<I64>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t* bar_full = reinterpret_cast<uint64_t*>(smem + SM::BARS);      // [g*2+st]
  uint64_t* bar_empty = bar_full + 4;                                      // [g*2+st]
  uint64_t* bar_fin = bar_full + 8;
  volatile int32_t* task_slot = reinterpret_cast<volatile int32_t*>(smem + SM::BARS + 80);
  E* stA = reinterpret_cast<E*>(smem + SM::STA);
  E* stB = reinterpret_cast<E*>(smem + SM::STB);
  uint32_t* stPK = reinterpret_cast<uint32_t*>(smem + SM::STPK);
  E* finU = reinterpret_cast<E*>(smem + SM::FINU);
  E* finL = reinterpret_cast<E*>(smem + SM::FINL);
  E* finBrow = reinterpret_cast<E*>(smem + SM::FINBROW);
  int32_t* finPP = reinterpret_cast<int32_t*>(smem + SM::FINPP);
  uint32_t* finPKI = reinterpret_cast<uint32_t*>(smem + SM::FINPKI);
  uint32_t* finPKJ = reinterpret_cast<uint32_t*>(smem + SM::FINPKJ);
  unsigned long long* finAcc = reinterpret_cast<unsigned long long*>(smem + SM::FINACC);
  unsigned long long* bestS = reinterpret_cast<unsigned long long*>(smem + SM::BEST);
  E* Xv = reinterpret_cast<E*>(smem + SM::XV);  // in-tile solve only (stage area)

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const long long limit = a.spin_limit;
  int32_t* status = a.status;

  if constexpr (SM::kXOut) {
    E* x = reinterpret_cast<E*>(smem + SM::WXR);
    for (int i = tid; i < 2 * kDiagRows * T; i += blockDim.x) x[i] = ~(E)0;
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) {
      mbar_init(&bar_full[i], 1);
      mbar_init(&bar_empty[i], kGroupThreads);
    }
    mbar_init(bar_fin, 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Per-role running counters (each role walks the same segment sequence).
  uint32_t use_cnt[2] = {0u, 0u};   // producer: stage uses issued per group; consumer: own group
  uint32_t fin_cnt = 0;             // finisher-barrier uses

  while (true) {
    if (tid == 0) {
      int32_t t = -1;
      if (*reinterpret_cast<volatile int32_t*>(status) == 0) t = atomicAdd(a.queue, 1);
      *task_slot = t;
    }
    __syncthreads();
    const int32_t tix = *task_slot;
    if (tix < 0 || tix >= a.ntasks) break;
    if (tix == a.drop_task) {  // injected fault: the task's flag is never published
      __syncthreads();
      continue;
    }
    const McmTask task = a.tasks[tix];
    const McmInstDev inst = a.insts[task.inst];
    const int I = task.I, J = task.J, D = J - I;
    const int IT = I * T, JT = J * T;
    const int64_t tidx = tile_index(inst, I, J);
    const bool finisher = task.kind == 0;
    const int S = inst.shift;
    const int32_t accslot = a.accslot[tidx];

    if (warp == kComputeThreads / 32) {
      // ===================== producer warp (lane 0) =====================
      if (lane == 0) {
        // the stage area was written and read through the generic proxy by the
        // previous task's in-tile solve; order that before this task's copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bool ok = true;
        bool issued[2][kStages] = {{false, false}, {false, false}};
        bool fin_issued = false;
        uint32_t last_parity[2][kStages] = {{0u, 0u}, {0u, 0u}};
        for_each_segment(task, [&](int K, int q) {
          const int g = q & 1;
          const uint32_t u = use_cnt[g]++;
          const int st = u % kStages;
          const uint32_t round = u / kStages;
          if (!ok) return;
          if constexpr (I64) {
            ok = wait_flag<I64>(a.flags + tile_index(inst, I, K), 1, limit, status) &&
                 wait_flag<I64>(a.flags + tile_index(inst, K, J), 1, limit, status) &&
                 wait_flag<I64>(a.flags + tile_index(inst, K + 1, J), 1, limit, status);
          } else {  // the three tiles' flags in one round trip when they are set
            const int32_t* const fl[3] = {a.flags + tile_index(inst, I, K), a.flags + tile_index(inst, K, J),
                                          a.flags + tile_index(inst, K + 1, J)};
            const int32_t tg[3] = {1, 1, 1};
            ok = wait_flags_geq_cap<kFlagPollNs, 3>(fl, tg, limit, status);
          }
          if (!ok) return;
          fence_proxy_async_global();
          if (!mbar_wait(&bar_empty[g * kStages + st], (round & 1u) ^ 1u, limit)) {
            set_status(status, DP_ETIMEOUT);
            ok = false;
            return;
          }
          uint64_t* fb = &bar_full[g * kStages + st];
          mbar_arrive_expect_tx(fb, 2 * SM::TILE + 128);
          bulk_g2s(stA + (g * kStages + st) * T * T,
                   static_cast<const E*>(a.af) + tile_index(inst, I, K) * T * T, SM::TILE, fb);
          bulk_g2s(stB + (g * kStages + st) * T * T,
                   static_cast<const E*>(a.bf) + tile_index(inst, K, J) * T * T, SM::TILE, fb);
          bulk_g2s(stPK + (g * kStages + st) * 32, a.pk + inst.pk_base + (int64_t)K * T, 128, fb);
          issued[g][st] = true;
          last_parity[g][st] = round & 1u;
        });
        if (finisher && ok) {
          if constexpr (I64) {
            if (D >= 1)
              ok = wait_flag<I64>(a.flags + tile_index(inst, I, I), 1, limit, status) &&
                   wait_flag<I64>(a.flags + tile_index(inst, J, J), 1, limit, status) &&
                   wait_flag<I64>(a.flags + tile_index(inst, I + 1, J), 1, limit, status);
            if (ok && task.nparts > 0) ok = wait_flag<I64>(a.counters + tidx, task.nparts, limit, status);
          } else {
            // tiles (I, I), (J, J), (I+1, J) and the bulk-task counter in one
            // round trip when they are ready; a diagonal tile has no
            // neighbours, so its own flag stands in with target 0
            const bool nb = D >= 1;
            const int32_t* const fl[4] = {a.flags + (nb ? tile_index(inst, I, I) : tidx),
                                          a.flags + (nb ? tile_index(inst, J, J) : tidx),
                                          a.flags + (nb ? tile_index(inst, I + 1, J) : tidx), a.counters + tidx};
            const int32_t tg[4] = {nb ? 1 : 0, nb ? 1 : 0, nb ? 1 : 0, task.nparts > 0 ? (int32_t)task.nparts : 0};
            ok = wait_flags_geq_cap<kFlagPollNs, 4>(fl, tg, limit, status);
          }
          if (ok) {
            fence_proxy_async_global();
            uint32_t bytes = 3 * 128;
            if (D >= 1) bytes += 2 * SM::TILE + T * (uint32_t)sizeof(E);
            if (task.nparts > 0) bytes += T * T * 8;
            mbar_arrive_expect_tx(bar_fin, bytes);
            bulk_g2s(finPP, a.pp + inst.pp_base + IT, 128, bar_fin);
            bulk_g2s(finPKI, a.pk + inst.pk_base + IT, 128, bar_fin);
            bulk_g2s(finPKJ, a.pk + inst.pk_base + JT, 128, bar_fin);
            if (D >= 1) {
              bulk_g2s(finU, static_cast<const E*>(a.af) + tile_index(inst, I, I) * T * T, SM::TILE, bar_fin);
              bulk_g2s(finL, static_cast<const E*>(a.bf) + tile_index(inst, J, J) * T * T, SM::TILE, bar_fin);
              bulk_g2s(finBrow, static_cast<const E*>(a.bf) + tidx * T * T + (T - 1) * T, T * sizeof(E), bar_fin);
            }
            if (task.nparts > 0) bulk_g2s(finAcc, a.acc + (int64_t)accslot * T * T, T * T * 8, bar_fin);
            fin_issued = true;
          } else {
            // keep the finisher barrier's phase sequence intact for the consumers
            mbar_arrive(bar_fin);
          }
        } else if (finisher) {
          mbar_arrive(bar_fin);
        }
        // No bulk copy may still be in flight when the task ends.
        for (int g = 0; g < 2; ++g)
          for (int st = 0; st < kStages; ++st)
            if (issued[g][st]) mbar_wait(&bar_full[g * kStages + st], last_parity[g][st], limit * 4);
        if (fin_issued) mbar_wait(bar_fin, fin_cnt & 1u, limit * 4);
      }
    } else {
      // ===================== compute threads (2 groups) =====================
      const int g = warp >> 2;
      const int tg = tid & (kGroupThreads - 1);
      const int ty = tg >> 4, tx = tg & 15;
      unsigned long long best[4][2];
      uint32_t P[4][2];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t pi = (uint32_t)a.pp[inst.pp_base + IT + 4 * ty + r];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          P[r][c] = pi * (uint32_t)a.pp[inst.pp_base + JT + 2 * tx + c + 1];
          best[r][c] = ~0ull;
        }
      }
      bool ok = true;
      for_each_segment(task, [&](int K, int q) {
        if ((q & 1) != g) return;
        const uint32_t u = use_cnt[g]++;
        const int st = u % kStages;
        const uint32_t round = u / kStages;
        if (!ok) return;
        bool got;
        if constexpr (I64) {
          got = mbar_wait(&bar_full[g * kStages + st], round & 1u, limit);
        } else {  // a finisher's segments are on the critical path: poll more often
          got = finisher ? mbar_wait_cap(&bar_full[g * kStages + st], round & 1u, limit, kFinPollNs)
                         : mbar_wait(&bar_full[g * kStages + st], round & 1u, limit);
        }
        if (!got) {
          set_status(status, DP_ETIMEOUT);
          ok = false;
          return;
        }
        const E* A = stA + (g * kStages + st) * T * T;
        const E* B = stB + (g * kStages + st) * T * T;
        const uint32_t* PK = stPK + (g * kStages + st) * 32;
        if constexpr (I64) {
          seg_i64(A, B, PK, P, best, ty, tx);
        } else {
          const int logc = S < 5 ? S : 5;
          switch (logc) {
            case 5: seg_i32<5>(A, B, PK, P, best, ty, tx, S, K * T); break;
            case 4: seg_i32<4>(A, B, PK, P, best, ty, tx, S, K * T); break;
            case 3: seg_i32<3>(A, B, PK, P, best, ty, tx, S, K * T); break;
            case 2: seg_i32<2>(A, B, PK, P, best, ty, tx, S, K * T); break;
            default: seg_i32<1>(A, B, PK, P, best, ty, tx, S, K * T); break;
          }
        }
        mbar_arrive(&bar_empty[g * kStages + st]);
      });

      // merge the two groups' minima: group 1 publishes, group 0 combines
      if (g == 1) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 2; ++c) bestS[(4 * ty + r) * T + 2 * tx + c] = best[r][c];
      }
      bar_compute();
      if (g == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int cell = (4 * ty + r) * T + 2 * tx + c;
            const unsigned long long v = umin(best[r][c], bestS[cell]);
            if (finisher)
              bestS[cell] = v;
            else if (v != ~0ull)
              atomicMin(a.acc + (int64_t)accslot * T * T + cell, v);
          }
      }

      if (finisher) {
        bar_compute();
        // ------------------ in-tile wavefront (finisher) ------------------
        // layout: warp w owns rows 4w..4w+3, lane = column
        const int w = warp;
        // interval DP: the weights of the thread's 4 cells, loaded while the copies land
        E wt[4] = {0, 0, 0, 0};
        if constexpr (W) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int64_t i = IT + 4 * w + r, j = JT + lane;
            if (i < j && j < inst.n) wt[r] = static_cast<const E*>(inst.w)[i * inst.n + j];
          }
        }
        const uint32_t fpar = fin_cnt & 1u;
        bool fin_ok;
        if constexpr (I64)
          fin_ok = mbar_wait(bar_fin, fpar, limit);
        else
          fin_ok = mbar_wait_cap(bar_fin, fpar, limit, kFinPollNs);
        if (!fin_ok) set_status(status, DP_ETIMEOUT);
        const bool go = bar_compute_and(fin_ok && *reinterpret_cast<volatile int32_t*>(status) == 0);
        const int shiftv = I64 ? 16 : S;
        const int n = inst.n;
        unsigned long long cb[4];
        E pi[4];
        const E pj1 = (E)(finPKJ[lane] >> shiftv);  // p[JT + lane + 1]
        if (go) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int li = 4 * w + r;
            pi[r] = (E)finPP[li];
            cb[r] = bestS[li * T + lane];
            if (task.nparts > 0) cb[r] = umin(cb[r], finAcc[li * T + lane]);
          }
          if (D >= 1) {
            E* Up = reinterpret_cast<E*>(smem + SM::WUP);
            E* Lp = reinterpret_cast<E*>(smem + SM::WLP);
            E* Xr = reinterpret_cast<E*>(smem + SM::WXR);
            E* Xc = reinterpret_cast<E*>(smem + SM::WXC);
            uint32_t* PKIp = reinterpret_cast<uint32_t*>(smem + SM::WPKI);
            uint32_t* PKJp = reinterpret_cast<uint32_t*>(smem + SM::WPKJ);
            constexpr E kInf = ~(E)0;
            // boundary split k = IT + 31: U[li][31] + m[IT+32][j] + w
            const E brow = finBrow[lane] >> shiftv;
            const E pI32 = (E)(finPKI[T - 1] >> shiftv);
            E m[4], wv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int li = 4 * w + r;
              bestS[li * T + lane] = cb[r];  // external minimum: (value, smallest k)
              wv[r] = pi[r] * pj1;
              const E bnd = (finU[(T - 1) * T + li] >> shiftv) + brow + wv[r] * pI32;
              m[r] = umin((E)(cb[r] >> KB), bnd);
            }
            if constexpr (!I64) {
              // 16-byte vectors: 8 per row, 3 per thread (all row pitches are 16-byte multiples)
              for (int v = tid; v < SM::kRows * T / 4; v += kComputeThreads) {
                const int q = v >> 3, x = (v & 7) * 4, t = q - SM::kRowOff;
                uint4 uu = make_uint4(0u, 0u, 0u, 0u), ll = make_uint4(0u, 0u, 0u, 0u);
                if (t >= 0 && t <= T - 2) {
                  const uint4 fu = *reinterpret_cast<const uint4*>(finU + t * T + x);
                  const uint4 fl = *reinterpret_cast<const uint4*>(finL + t * T + x);
                  uu = make_uint4(fu.x >> S, fu.y >> S, fu.z >> S, fu.w >> S);
                  ll = make_uint4(fl.x >> S, fl.y >> S, fl.z >> S, fl.w >> S);
                }
                *reinterpret_cast<uint4*>(Up + q * SM::UPW + x) = uu;
                *reinterpret_cast<uint4*>(Lp + q * T + x) = ll;
              }
            } else {
              for (int idx = tid; idx < SM::kRows * T; idx += kComputeThreads) {
                const int q = idx >> 5, x = idx & 31, t = q - SM::kRowOff;
                const bool in = t >= 0 && t <= T - 2;
                Up[q * SM::UPW + x] = in ? (finU[t * T + x] >> shiftv) : (E)0;
                Lp[idx] = in ? (finL[t * T + x] >> shiftv) : (E)0;
              }
            }
            if constexpr (!SM::kXOut) {
              for (int idx = tid; idx < kDiagRows * T; idx += kComputeThreads) {
                Xr[idx] = kInf;
                Xc[idx] = kInf;
              }
            }
            if (tid < SM::kRows) {
              const int t = tid - SM::kRowOff;
              const bool in = t >= 0 && t <= T - 2;
              PKIp[tid] = in ? (finPKI[t] >> shiftv) : 0u;
              PKJp[tid] = in ? (finPKJ[t] >> shiftv) : 0u;
            }
            const uint32_t sXr = smem_u32(Xr), sXc = smem_u32(Xc);
            const int e_last = T - 2 - 4 * w;  // the warp's last cell, (4w, 31), is final after this step
            const int c0 = lane - 4 * w - 1;   // at step e the lane's cell in row 4w + c0 - e becomes final
            bar_compute();
            if (w == 7 && lane == 0) {  // cell (31, 0), the only cell of diagonal -31
              Xr[T - 1] = m[3] + wt[3];
              Xc[0] = m[3] + wt[3];
            }
            // Operands of the first step.  Window slot (u & 3) holds L[u][lane]
            // and p[JT + u + 1] for u = 4w + e .. 4w + e + 3; with e = 1 mod 4
            // at the start of each group of 4 steps, the slots are compile-time
            // indices.
            E R[4];
            uint32_t P[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int u = 4 * w - (T - 1) + r;
              R[(1 + r) & 3] = Lp[SM::row(u) * T + lane];
              P[(1 + r) & 3] = PKJp[SM::row(u)];
            }
            Vec4<E> u4 = lds4(Up + SM::row(lane + T - 2) * SM::UPW + 4 * w);  // t = lane - 1 - e
            E pkc = (E)PKIp[SM::row(lane + T - 2)];
            bar_compute();
            if constexpr (!I64) {
              // int32: the 62 steps are unrolled, so every shared-memory
              // operand is a constant offset from a per-thread base. The
              // operands of step e + 1 (independent of the tile values) are
              // loaded at the start of step e, so the barrier after the step
              // does not wait for them, and each candidate is a multiply-add
              // plus a fused add-and-minimum. The row of the cell made final
              // is chosen with predicates computed once: bit 0 of c0 - e
              // flips every step, bit 1 repeats every four steps.
              const E* Lb = Lp + SM::row(4 * w) * T + lane;                 // + u * T: L row u = 4w + e + r
              const uint32_t* PJb = PKJp + SM::row(4 * w);                  // + u
              const E* Ub = Up + SM::row(lane - 1) * SM::UPW + 4 * w;       // - (e + 1) * UPW: t = lane - 2 - e
              const uint32_t* PIb = PKIp + SM::row(lane - 1);               // - (e + 1)
              const E* Xcb = Xc + (T - 1) * T + lane;                       // + e * T: X[lane - e][lane]
              const E* Xrb = Xr + (T - 1) * T + 4 * w;                      // + e * T: X[li][li + e]
              const uint32_t sXcw = sXc + (uint32_t)((T * T + lane) * 4);      // + e * T * 4
              const uint32_t sXrw = sXr + (uint32_t)((T * T + lane - 1) * 4);  // + e * (T - 1) * 4
              const bool b0e = (c0 & 1) != 0;  // bit 0 of c0 - e for even e
              bool b1[4];                      // bit 1 of c0 - e for e = k mod 4
#pragma unroll
              for (int k = 0; k < 4; ++k) b1[k] = ((c0 - k) & 2) != 0;
#pragma unroll
              for (int e = -(T - 1); e <= T - 2; ++e) {
                const int s4 = (e + T - 1) & 3;
                if (e <= e_last) {
                  const E Rn = Lb[(e + 4) * T];
                  const uint32_t Pn = PJb[e + 4];
                  const Vec4<E> u4n = lds4(Ub - (e + 1) * SM::UPW);
                  const E pkcn = (E)PIb[-(e + 1)];
                  const E xc = Xcb[e * T];             // column operand X[lane - e][lane]
                  const Vec4<E> x4 = lds4(Xrb + e * T);  // row operands X[li][li + e]
#pragma unroll
                  for (int r = 0; r < 4; ++r) {
                    const int q = (1 + s4 + r) & 3;
                    m[r] = __viaddmin_u32(u4.v[r] + wv[r] * pkc, xc, m[r]);
                    m[r] = __viaddmin_u32(R[q] + wv[r] * (E)P[q], x4.v[r], m[r]);
                  }
                  // the lane's cell on diagonal e + 1 (row 4w + c0 - e) is final now
                  const bool p0 = (e & 1) ? !b0e : b0e;
                  const bool p1 = b1[(e + 32) & 3];
                  E v = sel4p(p0, p1, m[0], m[1], m[2], m[3]);
                  if constexpr (W) v += sel4p(p0, p1, wt[0], wt[1], wt[2], wt[3]);
                  const bool own = (unsigned)(c0 - e) <= 3u;
                  sts_if(own, sXrw + (uint32_t)(e * (T - 1) * 4), v);
                  sts_if(own, sXcw + (uint32_t)(e * T * 4), v);
                  R[(1 + s4) & 3] = Rn;
                  P[(1 + s4) & 3] = Pn;
                  u4 = u4n;
                  pkc = pkcn;
                }
                bar_compute();
              }
            } else {
#pragma unroll 1
            for (int eb = -(T - 1); eb <= T - 2; eb += 4) {
#pragma unroll
              for (int s4 = 0; s4 < 4; ++s4) {
                const int e = eb + s4;
                if (e <= T - 2) {
                  if (e <= e_last) {
                    const int dI = e + T - 1;
                    const E xc = Xc[dI * T + lane];             // column operand X[lane - e][lane]
                    const Vec4<E> x4 = lds4(Xr + dI * T + 4 * w);  // row operands X[li][li + e]
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                      const int q = (1 + s4 + r) & 3;
                      const E cc = u4.v[r] + xc + wv[r] * pkc;
                      const E cr = x4.v[r] + R[q] + wv[r] * (E)P[q];
                      if constexpr (I64)
                        m[r] = umin(m[r], umin(cc, cr));
                      else
                        m[r] = __vimin3_u32(m[r], cc, cr);
                    }
                    // the lane's cell on diagonal e + 1 is final now
                    const int rr = c0 - e;
                    const bool own = (unsigned)rr <= 3u;
                    E v = sel4(rr, m[0], m[1], m[2], m[3]);
                    if constexpr (W) v += sel4(rr, wt[0], wt[1], wt[2], wt[3]);
                    sts_if(own, sXr + (uint32_t)(((dI + 1) * T + 4 * w + rr) * (int)sizeof(E)), v);
                    sts_if(own, sXc + (uint32_t)(((dI + 1) * T + lane) * (int)sizeof(E)), v);
                    // operands of step e + 1 (independent of the tile values)
                    const int un = 4 * w + e + 4;
                    R[(1 + s4) & 3] = Lp[SM::row(un) * T + lane];
                    P[(1 + s4) & 3] = PKJp[SM::row(un)];
                    const int tn = lane - 2 - e;
                    u4 = lds4(Up + SM::row(tn) * SM::UPW + 4 * w);
                    pkc = (E)PKIp[SM::row(tn)];
                  }
                  bar_compute();
                }
              }
            }
            }
            // ---------------- panels needed by other tiles, then publish ----------------
            const int64_t nn = n;
            E vals[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) vals[r] = Xc[(lane - 4 * w - r + T - 1) * T + lane];
            {
              E* af = static_cast<E*>(a.af) + tidx * T * T;
              E pa[4];
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                if constexpr (I64)
                  pa[r] = ((E)vals[r] << 16) | (E)(JT + lane);
                else
                  pa[r] = (vals[r] << S) | (E)(lane & ((1 << (S < 5 ? S : 5)) - 1));
              }
              if constexpr (I64) {
                *reinterpret_cast<ulonglong2*>(af + lane * T + 4 * w) = make_ulonglong2(pa[0], pa[1]);
                *reinterpret_cast<ulonglong2*>(af + lane * T + 4 * w + 2) = make_ulonglong2(pa[2], pa[3]);
              } else {
                *reinterpret_cast<uint4*>(af + lane * T + 4 * w) = make_uint4(pa[0], pa[1], pa[2], pa[3]);
              }
              E* bf = static_cast<E*>(a.bf);
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int li = 4 * w + r;
                const E pb = vals[r] << shiftv;
                if (li >= 1)
                  bf[tidx * T * T + (li - 1) * T + lane] = pb;
                else if (I >= 1)
                  bf[tile_index(inst, I - 1, J) * T * T + (T - 1) * T + lane] = pb;
              }
            }
            bar_compute();
            // release: the panel stores of every compute thread, ordered before
            // this store by the barrier, are visible to whoever acquires the flag
            if (tid == 0) st_release(a.flags + tidx, 1);
            // ---------------- the tables themselves (not read by other tiles) ----------------
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int li = 4 * w + r;
              const int64_t i = IT + li, j = JT + lane;
              if (i < nn && j < nn) {
                if constexpr (I64)
                  static_cast<int64_t*>(inst.m)[i * nn + j] = (int64_t)vals[r];
                else
                  static_cast<int32_t*>(inst.m)[i * nn + j] = (int32_t)vals[r];
              }
              const int64_t i2 = JT + li, j2 = IT + lane;  // mirror tile (J, I)
              if (i2 < nn && j2 < nn) {
                if constexpr (I64)
                  static_cast<int64_t*>(inst.m)[i2 * nn + j2] = 0;
                else
                  static_cast<int32_t*>(inst.m)[i2 * nn + j2] = 0;
                inst.s[i2 * nn + j2] = -1;
              }
            }
            // ---------------- split table (off the critical path) ----------------
            // The smallest k reaching the final value, scanning in increasing
            // k: column splits IT+li .. IT+30, the boundary IT+31, the
            // external splits (smallest one kept with the external minimum),
            // row splits JT .. j-1.
            const unsigned long long kmask = (1ull << KB) - 1ull;
#pragma unroll 1
            for (int r = 0; r < 4; ++r) {
              // int32: warp w scans rows w, w + 8, w + 16 and w + 24, a mix of
              // long and short column scans, so that the warps finish together
              // (the value, weight and multiplier of the row are read again);
              // int64: the warp's own rows 4w .. 4w + 3
              const int li = I64 ? 4 * w + r : w + 8 * r;
              const int64_t i = IT + li, j = JT + lane;
              if (i >= nn || j >= nn) continue;
              // (register arrays are read through sel4: a runtime index would move them to local memory)
              E v;   // the minimum, less the cell's own weight
              E wr;  // the row's multiplier p[i] p[j+1]
              if constexpr (I64) {
                v = sel4(r, vals[0], vals[1], vals[2], vals[3]);
                if constexpr (W) v -= sel4(r, wt[0], wt[1], wt[2], wt[3]);
                wr = sel4(r, wv[0], wv[1], wv[2], wv[3]);
              } else {
                v = Xc[(lane - li + T - 1) * T + lane];
                if constexpr (W) v -= static_cast<const E*>(inst.w)[i * inst.n + j];
                wr = (E)finPP[li] * pj1;
              }
              int k = -1;
              if constexpr (!I64) {
                // int32: four splits per round with independent loads, the
                // smallest matching one kept; a lane stops after the first
                // round with a match
                for (int t0 = li; t0 <= T - 2 && k < 0; t0 += 4) {
                  E c4[4];
#pragma unroll
                  for (int d = 0; d < 4; ++d) {
                    const int t = t0 + d <= T - 2 ? t0 + d : T - 2;
                    c4[d] = Up[SM::row(t) * SM::UPW + li] + Xc[(lane - t - 1 + T - 1) * T + lane] + wr * (E)PKIp[SM::row(t)];
                  }
#pragma unroll
                  for (int d = 3; d >= 0; --d)
                    if (t0 + d <= T - 2 && c4[d] == v) k = IT + t0 + d;
                }
              } else {
              for (int t = li; t <= T - 2; ++t) {
                if (Up[SM::row(t) * SM::UPW + li] + Xc[(lane - t - 1 + T - 1) * T + lane] + wr * (E)PKIp[SM::row(t)] ==
                    v) {
                  k = IT + t;
                  break;
                }
              }
              }
              if (k < 0 && (finU[(T - 1) * T + li] >> shiftv) + brow + wr * pI32 == v) k = IT + T - 1;
              if (k < 0) {
                const unsigned long long ek = bestS[li * T + lane];
                if ((E)(ek >> KB) == v) k = (int)(ek & kmask);
              }
              if (k < 0) {
                if constexpr (!I64) {
                  for (int u0 = 0; u0 < lane && k < 0; u0 += 4) {
                    E c4[4];
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                      const int u = u0 + d <= T - 2 ? u0 + d : T - 2;
                      c4[d] = Xr[(u - li + T - 1) * T + li] + Lp[SM::row(u) * T + lane] + wr * (E)PKJp[SM::row(u)];
                    }
#pragma unroll
                    for (int d = 3; d >= 0; --d)
                      if (u0 + d < lane && c4[d] == v) k = JT + u0 + d;
                  }
                } else {
                for (int u = 0; u < lane; ++u) {
                  if (Xr[(u - li + T - 1) * T + li] + Lp[SM::row(u) * T + lane] + wr * (E)PKJp[SM::row(u)] == v) {
                    k = JT + u;
                    break;
                  }
                }
                }
              }
              inst.s[i * nn + j] = (int16_t)k;
            }
          } else {
            // diagonal tile: ordinary MCM on the 32-matrix sub-chain
            const E pj1d = (E)(finPKI[lane] >> shiftv);
            bool keyed = false;
            if constexpr (!I64) {
              if (S == 5) {
                // int32 with a 5-bit shift: a cell's running minimum is one
                // 32-bit key (value << 5) + (k - IT), whose unsigned minimum
                // keeps the smallest split on ties, as the 64-bit keys below
                // do; final values are stored shifted in Xv, and a candidate
                // whose operands are not both final is not taken (a select,
                // no branch)
                uint32_t* Xs = reinterpret_cast<uint32_t*>(Xv);
                uint32_t key[4], pij[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                  key[r] = 0xFFFFFFFFu;
                  pij[r] = pi[r] * pj1d;
                }
#pragma unroll 1
                for (int e = 0; e <= T - 2; ++e) {
#pragma unroll
                  for (int r = 0; r < 4; ++r) {
                    const int li = 4 * w + r;
                    if (lane - li == e) Xs[li * T + lane] = e == 0 ? 0u : (key[r] & ~31u) + (wt[r] << 5);
                  }
                  bar_compute();
#pragma unroll
                  for (int r = 0; r < 4; ++r) {
                    const int li = 4 * w + r;
                    const int f = lane - li;
                    // split k1 = li + e: left operand on diagonal e, right on f - e - 1
                    const bool v1 = f > e && f - e - 1 <= e;
                    const int k1 = v1 ? li + e : 0;
                    const uint32_t c1 = Xs[li * T + k1] + pij[r] * finPKI[k1] + (uint32_t)k1;
                    const uint32_t n1 = __viaddmin_u32(c1, Xs[(k1 + 1) * T + lane], key[r]);
                    // split k2 = lane - 1 - e: right operand on diagonal e, left on f - 1 - e
                    const bool v2 = f > e && f - 1 - e < e;
                    const int k2 = v2 ? lane - 1 - e : 0;
                    const uint32_t c2 = Xs[li * T + k2] + pij[r] * finPKI[k2] + (uint32_t)k2;
                    const uint32_t n2 = __viaddmin_u32(c2, Xs[(k2 + 1) * T + lane], v1 ? n1 : key[r]);
                    key[r] = v2 ? n2 : (v1 ? n1 : key[r]);
                  }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
                  cb[r] = key[r] == 0xFFFFFFFFu ? ~0ull
                                                : ((unsigned long long)(key[r] >> 5) << KB) | (unsigned)(IT + (key[r] & 31u));
                keyed = true;
              }
            }
#pragma unroll 1
            for (int e = 0; e <= T - 2 && !keyed; ++e) {
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int li = 4 * w + r;
                if (lane - li == e) Xv[li * T + lane] = e == 0 ? (E)0 : (E)(cb[r] >> KB) + wt[r];
              }
              bar_compute();
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int li = 4 * w + r;
                const int f = lane - li;
                if (f > e) {
                  if (f - e - 1 <= e) {  // split k = li + e: left operand on diagonal e
                    const E cand = Xv[li * T + li + e] + Xv[(li + e + 1) * T + lane] +
                                   pi[r] * (E)(finPKI[li + e] >> shiftv) * pj1d;
                    cb[r] = umin(cb[r], ((unsigned long long)cand << KB) | (unsigned)(IT + li + e));
                  }
                  if (f - 1 - e < e) {  // split k = lane - 1 - e: right operand on diagonal e
                    const E cand = Xv[li * T + lane - 1 - e] + Xv[(lane - e) * T + lane] +
                                   pi[r] * (E)(finPKI[lane - 1 - e] >> shiftv) * pj1d;
                    cb[r] = umin(cb[r], ((unsigned long long)cand << KB) | (unsigned)(IT + lane - 1 - e));
                  }
                }
              }
            }
          // ------------------ outputs ------------------
          const int64_t nn = n;
          const unsigned long long kmask = (1ull << KB) - 1ull;
          E vals[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int li = 4 * w + r;
            const int64_t i = IT + li, j = JT + lane;
            const bool upper = D >= 1 || li < lane;
            const E v = upper ? (E)(cb[r] >> KB) + wt[r] : (E)0;
            const int kk = upper ? (int)(cb[r] & kmask) : -1;
            vals[r] = v;
            if (i < nn && j < nn) {
              if constexpr (I64)
                static_cast<int64_t*>(inst.m)[i * nn + j] = (int64_t)v;
              else
                static_cast<int32_t*>(inst.m)[i * nn + j] = (int32_t)v;
              inst.s[i * nn + j] = (int16_t)kk;
            }
            if (D >= 1) {  // mirror tile (J, I) in the lower triangle
              const int64_t i2 = JT + li, j2 = IT + lane;
              if (i2 < nn && j2 < nn) {
                if constexpr (I64)
                  static_cast<int64_t*>(inst.m)[i2 * nn + j2] = 0;
                else
                  static_cast<int32_t*>(inst.m)[i2 * nn + j2] = 0;
                inst.s[i2 * nn + j2] = -1;
              }
            }
          }
          // packed row panel: af[tile][k = lane][row]
          E* af = static_cast<E*>(a.af) + tidx * T * T;
          E pa[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if constexpr (I64)
              pa[r] = ((E)vals[r] << 16) | (E)(JT + lane);
            else
              pa[r] = (vals[r] << S) | (E)(lane & ((1 << (S < 5 ? S : 5)) - 1));
          }
          if constexpr (I64) {
            *reinterpret_cast<ulonglong2*>(af + lane * T + 4 * w) = make_ulonglong2(pa[0], pa[1]);
            *reinterpret_cast<ulonglong2*>(af + lane * T + 4 * w + 2) = make_ulonglong2(pa[2], pa[3]);
          } else {
            *reinterpret_cast<uint4*>(af + lane * T + 4 * w) = make_uint4(pa[0], pa[1], pa[2], pa[3]);
          }
          // packed column panel, rows shifted by one: bf[tile(X, J)][row r] = m[32X + r + 1][.]
          E* bf = static_cast<E*>(a.bf);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int li = 4 * w + r;
            const E pb = vals[r] << shiftv;
            if (li >= 1)
              bf[tidx * T * T + (li - 1) * T + lane] = pb;
            else if (I >= 1)
              bf[tile_index(inst, I - 1, J) * T * T + (T - 1) * T + lane] = pb;
          }
          }
        }
      }
    }
    if (finisher) ++fin_cnt;
    __syncthreads();
    if (tid == 0 && *reinterpret_cast<volatile int32_t*>(status) == 0) {
      // release (cumulative over the block's merges and stores before the barrier)
      if (!finisher)
        red_release_add(a.counters + tidx, 1);
      else if (D == 0)  // off-diagonal tiles publish right after their values
        st_release(a.flags + tidx, 1);
    }
  }
}

// Interval DP, before the prologue: the largest weight above the diagonal of
// each chain (blockIdx.y), merged into McmInstDev::wmax; a negative weight
// there is DP_EINVAL.  Entries on and below the diagonal are not read.
// Weights are int32 (the cost type the interval DP is built for).
__global__ void __launch_bounds__(256) mcm_weight_max_kernel(const McmLaunchArgs a) {
  using SW = int32_t;
  __shared__ unsigned long long s_max[8];
  const int b = blockIdx.y;
  McmInstDev* inst = a.insts + b;
  const int n = inst->n;
  const SW* w = static_cast<const SW*>(a.w_all) + (a.tab_off ? a.tab_off[b] : 0);
  unsigned long long mx = 0;
  bool neg = false;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const SW* row = w + (int64_t)i * n;
    for (int j = i + 1 + (int)threadIdx.x; j < n; j += blockDim.x) {
      const SW v = row[j];
      neg |= v < 0;
      mx = v > 0 && (unsigned long long)v > mx ? (unsigned long long)v : mx;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = x > mx ? x : mx;
  }
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  neg = __syncthreads_or(neg);
  if (threadIdx.x == 0) {
    for (int x = 1; x < (int)(blockDim.x >> 5); ++x) mx = s_max[x] > mx ? s_max[x] : mx;
    if (neg) set_status(a.status, DP_EINVAL);
    if (mx > 0) atomicMax(&inst->wmax, mx);
  }
}

// One block per chain: validates dims, derives the cost bound and the packing
// shift, writes the padded / shifted dim arrays and the chain's pointers.
template <bool I64, bool W>
__global__ void __launch_bounds__(256) mcm_prologue_kernel(const McmLaunchArgs a) {
  __shared__ int32_t s_max[8], s_min[8];
  __shared__ int32_t s_shift;
  const int b = blockIdx.x;
  McmInstDev* inst = a.insts + b;
  const int n = inst->n;
  const int32_t* p = a.p_off ? a.p_all + a.p_off[b] : a.p_all;
  int32_t mx = 0, mn = 0x7fffffff;
  for (int x = threadIdx.x; x <= n; x += blockDim.x) {
    const int32_t v = p[x];
    mx = v > mx ? v : mx;
    mn = v < mn ? v : mn;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_max[threadIdx.x >> 5] = mx;
    s_min[threadIdx.x >> 5] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mx = max(mx, s_max[w]);
      mn = min(mn, s_min[w]);
    }
    int shift = -1;
    // interval DP: dims may be 0 (no rank-1 term); the weight adds at most
    // wmax per product, and n - 1 products make up a cell
    const unsigned long long wm = W ? inst->wmax : 0ull;
    if (mn < (W ? 0 : 1)) {
      set_status(a.status, DP_EINVAL);
    } else if (mx >= 65536 || wm >= (1ull << 47)) {
      set_status(a.status, DP_EOVERFLOW);
    } else {
      const unsigned long long m3 = (unsigned long long)mx * mx * mx;         // < 2^48
      const unsigned long long bound = (unsigned long long)(n - 1) * (m3 + wm);  // < 2^64
      if (I64) {
        if (bound >= (1ull << 47)) set_status(a.status, DP_EOVERFLOW);
        else shift = 16;
      } else {
        if (bound >= (1ull << 31)) {
          set_status(a.status, DP_EOVERFLOW);
        } else {
          shift = 1;
          while (shift < 5 && ((bound + 1) << (shift + 1)) <= (1ull << 32)) ++shift;
        }
      }
    }
    s_shift = shift;
    inst->shift = shift;
    inst->p = p;
    const int64_t to = a.tab_off ? a.tab_off[b] : 0;
    inst->m = static_cast<uint8_t*>(a.m_all) + to * (I64 ? 8 : 4);
    inst->s = a.s_all + to;
    if (W) inst->w = static_cast<const uint8_t*>(a.w_all) + to * (I64 ? 8 : 4);
  }
  __syncthreads();
  const int shift = s_shift;
  if (shift < 0) return;
  const int ext = inst->nt * T;
  for (int x = threadIdx.x; x < ext + 32; x += blockDim.x) {
    a.pp[inst->pp_base + x] = x <= n ? p[x] : 1;
    if (x < ext) a.pk[inst->pk_base + x] = (uint32_t)(x + 1 <= n ? p[x + 1] : 1) << shift;
  }
}

}  // namespace

size_t mcm_smem_bytes(bool i64) { return i64 ? Smem<true>::TOTAL : Smem<false>::TOTAL; }

cudaError_t mcm_configure(bool i64) {
  cudaError_t e;
  if (i64)
    return cudaFuncSetAttribute(mcm_main_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Smem<true>::TOTAL);
  if ((e = cudaFuncSetAttribute(mcm_main_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Smem<false>::TOTAL)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(mcm_main_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Smem<false>::TOTAL);
}

// Both instances of a cost type have the same launch bounds and shared
// memory, hence the same occupancy.
cudaError_t mcm_occupancy(bool i64, int* blocks_per_sm) {
  if (i64)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcm_main_kernel<true, false>, kMcmThreads,
                                                         Smem<true>::TOTAL);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcm_main_kernel<false, false>, kMcmThreads,
                                                       Smem<false>::TOTAL);
}

cudaError_t mcm_preload(bool i64) {
  cudaFuncAttributes fa;
  cudaError_t e;
  if (i64) {
    if ((e = cudaFuncGetAttributes(&fa, mcm_prologue_kernel<true, false>)) != cudaSuccess) return e;
    return cudaFuncGetAttributes(&fa, mcm_main_kernel<true, false>);
  }
  if ((e = cudaFuncGetAttributes(&fa, mcm_prologue_kernel<false, false>)) != cudaSuccess) return e;
  return cudaFuncGetAttributes(&fa, mcm_main_kernel<false, false>);
}

// The interval DP is built for int32 costs only (see launch_mcm_weight_max
// in mcm_kernels.cuh): with int64 costs and weights these return
// cudaErrorNotSupported and launch nothing.
cudaError_t launch_mcm_weight_max(const McmLaunchArgs& a, bool i64, int sms, cudaStream_t st) {
  if (a.ninst <= 0 || !a.w_all) return cudaSuccess;
  if (i64) return cudaErrorNotSupported;
  const dim3 grid((unsigned)(sms > 0 ? 4 * sms : 256), (unsigned)a.ninst);
  mcm_weight_max_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mcm_prologue(const McmLaunchArgs& a, bool i64, cudaStream_t st) {
  if (a.ninst <= 0) return cudaSuccess;
  const bool w = a.w_all != nullptr;
  if (i64) {
    if (w) return cudaErrorNotSupported;
    mcm_prologue_kernel<true, false><<<a.ninst, 256, 0, st>>>(a);
  } else {
    if (w) mcm_prologue_kernel<false, true><<<a.ninst, 256, 0, st>>>(a);
    else mcm_prologue_kernel<false, false><<<a.ninst, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_mcm_main(const McmLaunchArgs& a, bool i64, int grid, cudaStream_t st) {
  if (a.ntasks <= 0) return cudaSuccess;
  const bool w = a.w_all != nullptr;
  if (i64) {
    if (w) return cudaErrorNotSupported;
    mcm_main_kernel<true, false><<<grid, kMcmThreads, Smem<true>::TOTAL, st>>>(a);
  } else {
    if (w) mcm_main_kernel<false, true><<<grid, kMcmThreads, Smem<false>::TOTAL, st>>>(a);
    else mcm_main_kernel<false, false><<<grid, kMcmThreads, Smem<false>::TOTAL, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dpk
