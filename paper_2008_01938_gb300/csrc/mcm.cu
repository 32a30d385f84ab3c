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
constexpr int kUP = 36;  // pitch of U^T in shared memory (bank-conflict free for the block solve)
constexpr int kLP = 40;  // pitch of L
constexpr int kXP = 33;  // pitch of X and of the running minima

template <bool I64>
struct Cost {
  using E = typename std::conditional<I64, unsigned long long, uint32_t>::type;
  static constexpr int KB = I64 ? 16 : 32;  // k bits in the 64-bit (value, k) key
};

__device__ __forceinline__ int64_t tile_index(const McmInstDev& in, int I, int J) {
  return in.tile_base + (int64_t)I * in.nt - (int64_t)I * (I - 1) / 2 + (J - I);
}

// Shared-memory carve-up (byte offsets); identical for all blocks.  During a
// finisher's in-tile solve the bulk-copy stages are idle (every copy of the
// task has landed), so the solve's working arrays are carved from them.
template <bool I64>
struct Smem {
  static constexpr int ES = I64 ? 8 : 4;
  static constexpr int TILE = T * T * ES;
  static constexpr int BARS = 0;                                 // 9 mbarriers + task slot
  static constexpr int STA = 128;                                // [group][stage] row panels
  static constexpr int STB = STA + 4 * TILE;                     // [group][stage] column panels
  static constexpr int STPK = STB + 4 * TILE;                    // [group][stage] 32 x u32 dims
  static constexpr int FINU = STPK + 4 * 128;                    // row panel of diagonal tile (I,I)
  static constexpr int FINL = FINU + TILE;                       // column panel of diagonal tile (J,J)
  static constexpr int FINBROW = FINL + TILE;                    // boundary row (one tile row)
  static constexpr int FINPP = FINBROW + 256;                    // p[32I .. 32I+31]
  static constexpr int FINPKI = FINPP + 128;                     // p[32I+1 ..] << S
  static constexpr int FINPKJ = FINPKI + 128;                    // p[32J+1 ..] << S
  static constexpr int FINACC = FINPKJ + 128;                    // bulk-task partial minima
  static constexpr int BEST = FINACC + T * T * 8;                // running (value, k) keys
  static constexpr int TOTAL = BEST + T * T * 8;
  // in-tile solve arrays, inside the stage area (pitch 32 everywhere: the
  // access patterns of the pipelined solve are bank-conflict free with it)
  static constexpr int UP = kUP, LP = kLP, XP = kXP;
  static constexpr int UT = STA;                                 // U^T[t][li] = m[IT+li][IT+t]
  static constexpr int LM = UT + ((T * UP * ES + 127) / 128) * 128;  // L[u][lj] = m[JT+u+1][JT+lj]
  static constexpr int XV = LM + ((T * LP * ES + 127) / 128) * 128;  // final values of the tile
  static constexpr int ACCV = XV + ((T * XP * ES + 127) / 128) * 128;  // running minima of older splits
  static constexpr int PV = ACCV + ((T * XP * ES + 127) / 128) * 128;  // p[IT+li], p[IT+t+1], p[JT+u+1]
  static_assert(PV + 3 * T * ES <= STPK, "in-tile arrays must fit in the stage area");
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
// w = p[IT+li] p[k+1] p[JT+lj+1].
// The tile is cut into 4 x 4 blocks of 8 x 8; block (bi, bj) depends on the
// blocks below it in its column and left of it in its row.  Blocks are solved
// one block-diagonal E = bj - bi at a time (7 steps), one warp per block:
//   * the warp first folds in the splits whose operand lies in the two
//     neighbour blocks finished in the previous step (8x8x8 products);
//   * then it runs the paper's diagonal-order wavefront over the block's 15
//     cell diagonals with warp shuffles only (lane = column c + 8 g, cells of
//     rows g and g + 4);
//   * warps without a block in this step fold the previous step's blocks into
//     the blocks two or more diagonals ahead.
// Only values are carried; the split index is recovered after the tile is
// published.
// ---------------------------------------------------------------------------

// Column splits of the lane's two cells (rows R + g, R + g + 4, column C + c)
// whose second operand lies in block row si (rows 8si .. 8si+7).  Pointers
// are rebased so that the loop indexes with lane constants only:
//   xs = Xv + (8si)*XP + C, us = Ut + (8si-1)*UP + R, ps = pI1 + 8si - 1.
template <typename E>
__device__ __forceinline__ void blk_col_product(const E* __restrict__ xs, const E* __restrict__ us,
                                                const E* __restrict__ ps, int g, int c, E w0, E w1, E& m0, E& m1) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const E x = xs[q * kXP + c];
    const E pk = ps[q];
    m0 = umin(m0, us[q * kUP + g] + x + w0 * pk);
    m1 = umin(m1, us[q * kUP + g + 4] + x + w1 * pk);
  }
}

// Row splits of the lane's two cells whose first operand lies in block
// column sj (columns 8sj .. 8sj+7):
//   xr = Xv + R*XP + 8sj, ls = Lm + (8sj)*LP + C, ps = pJ1 + 8sj.
template <typename E>
__device__ __forceinline__ void blk_row_product(const E* __restrict__ xr, const E* __restrict__ ls,
                                                const E* __restrict__ ps, int g, int c, E w0, E w1, E& m0, E& m1) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const E l = ls[q * kLP + c];
    const E pk = ps[q];
    m0 = umin(m0, xr[g * kXP + q] + l + w0 * pk);
    m1 = umin(m1, xr[(g + 4) * kXP + q] + l + w1 * pk);
  }
}

// Wavefront over one 8x8 block (origin R0, C0) by one warp; v0 / v1 hold the
// minima of all splits outside the block for the lane's two cells on entry
// and the final values on exit (also stored to X).  Rebased pointers:
//   xb = Xv + R0*XP + C0, ub = Ut + (R0-1)*UP + R0 (so ub[a*UP + r] = U[R0+r][R0+a-1]),
//   lb = Lm + C0*LP + C0, pi1 = pI1 + R0 - 1, pj1 = pJ1 + C0.
template <typename E>
__device__ __forceinline__ void blk_solve8(E* __restrict__ xb, const E* __restrict__ ub, const E* __restrict__ lb,
                                           const E* __restrict__ pi1, const E* __restrict__ pj1, int g, int c, E w0,
                                           E w1, E& v0, E& v1) {
  const int r0 = g, r1 = g + 4;
#pragma unroll
  for (int e = -7; e <= 7; ++e) {
    const E xe = (c - r0 == e) ? v0 : v1;  // this lane's cell on diagonal e, if any
    const int a = c - e;                   // column split from row a of the block
    const int ac = a < 1 ? 1 : (a > 7 ? 7 : a);
    const E xa = __shfl_sync(0xffffffffu, xe, (ac & 3) * 8 + c);
    const int b0 = r0 + e, b1 = r1 + e;    // row splits from columns b0, b1
    const int b0c = b0 < 0 ? 0 : (b0 > 7 ? 7 : b0), b1c = b1 < 0 ? 0 : (b1 > 7 ? 7 : b1);
    const E xb0 = __shfl_sync(0xffffffffu, xe, g * 8 + b0c);
    const E xb1 = __shfl_sync(0xffffffffu, xe, g * 8 + b1c);
    const E pkt = pi1[ac];
    const E ca0 = ub[ac * kUP + r0] + xa + w0 * pkt;
    const E ca1 = ub[ac * kUP + r1] + xa + w1 * pkt;
    const E cb0 = xb0 + lb[b0c * kLP + c] + w0 * pj1[b0c];
    const E cb1 = xb1 + lb[b1c * kLP + c] + w1 * pj1[b1c];
    if (c - r0 > e) {
      if (a <= 7) v0 = umin(v0, ca0);
      if (b0 >= 0) v0 = umin(v0, cb0);
    }
    if (c - r1 > e) {
      if (a <= 7) v1 = umin(v1, ca1);
      if (b1 >= 0) v1 = umin(v1, cb1);
    }
  }
  xb[r0 * kXP + c] = v0;
  xb[r1 * kXP + c] = v1;
}

// Folds into block (ti, tj) the splits whose operand lies in block (si, tj)
// below it (hc) and / or block (ti, sj) left of it (hr); m0 / m1 in/out.
template <typename E>
__device__ __forceinline__ void blk_fold(const E* __restrict__ Xv, const E* __restrict__ Ut, const E* __restrict__ Lm,
                                         const E* __restrict__ pI1, const E* __restrict__ pJ1, int ti, int tj, int si,
                                         int sj, bool hc, bool hr, int g, int c, E w0, E w1, E& m0, E& m1) {
  const int R = 8 * ti, C = 8 * tj;
  if (hc) blk_col_product(Xv + 8 * si * kXP + C, Ut + (8 * si - 1) * kUP + R, pI1 + 8 * si - 1, g, c, w0, w1, m0, m1);
  if (hr) blk_row_product(Xv + R * kXP + 8 * sj, Lm + 8 * sj * kLP + C, pJ1 + 8 * sj, g, c, w0, w1, m0, m1);
}

// The whole in-tile solve (all 8 compute warps; ends with Xv final).
template <typename E>
__device__ __forceinline__ void tile_solve_blocks(E* __restrict__ Xv, E* __restrict__ acc, const E* __restrict__ Ut,
                                                  const E* __restrict__ Lm, const E* __restrict__ pI,
                                                  const E* __restrict__ pI1, const E* __restrict__ pJ1, int warp,
                                                  int lane) {
  const int g = lane >> 3, c = lane & 7;
#pragma unroll 1
  for (int s = 0; s < 7; ++s) {
    const int E_ = s - 3;
    const int nb = 4 - (E_ < 0 ? -E_ : E_);
    const int bi0 = E_ < 0 ? -E_ : 0;
    if (warp < nb) {
      const int bi = bi0 + warp, bj = bi + E_;
      const int R = 8 * bi, C = 8 * bj;
      const E pj = pJ1[C + c];
      const E w0 = pI[R + g] * pj, w1 = pI[R + g + 4] * pj;
      E v0 = acc[(R + g) * kXP + C + c];
      E v1 = acc[(R + g + 4) * kXP + C + c];
      // splits from the two neighbour blocks finished in the previous step
      blk_fold(Xv, Ut, Lm, pI1, pJ1, bi, bj, bi + 1, bj - 1, bi < 3, bj > 0, g, c, w0, w1, v0, v1);
      blk_solve8(Xv + R * kXP + C, Ut + (R - 1) * kUP + R, Lm + C * kLP + C, pI1 + R - 1, pJ1 + C, g, c, w0, w1, v0,
                 v1);
    } else if (s >= 1) {
      // fold the blocks of diagonal E_-1 into the blocks on diagonals >= E_+1
      const int idle = warp - nb, nidle = 8 - nb;
      const int Es = E_ - 1;
      int k = 0, next = idle;
#pragma unroll 1
      for (int blk = 0; blk < 16; ++blk) {
        const int ti = blk >> 2, tj = blk & 3;
        if (tj - ti < E_ + 1) continue;
        const int si = tj - Es, sj = ti + Es;
        const bool hc = si > ti && si <= 3, hr = sj >= 0 && sj < tj;
        if (!hc && !hr) continue;
        if (k++ != next) continue;
        next += nidle;
        const int R = 8 * ti, C = 8 * tj;
        const E pj = pJ1[C + c];
        const E w0 = pI[R + g] * pj, w1 = pI[R + g + 4] * pj;
        E m0 = acc[(R + g) * kXP + C + c];
        E m1 = acc[(R + g + 4) * kXP + C + c];
        blk_fold(Xv, Ut, Lm, pI1, pJ1, ti, tj, si, sj, hc, hr, g, c, w0, w1, m0, m1);
        acc[(R + g) * kXP + C + c] = m0;
        acc[(R + g + 4) * kXP + C + c] = m1;
      }
    }
    bar_compute();
  }
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
#pragma unroll
    for (int kk = 0; kk < C; ++kk) {
      const uint4 a = *reinterpret_cast<const uint4*>(A + (c0 + kk) * T + 4 * ty);
      const uint2 b = *reinterpret_cast<const uint2*>(B + (c0 + kk) * T + 2 * tx);
      const uint32_t pk = PK[c0 + kk];
      const uint32_t av[4] = {a.x, a.y, a.z, a.w};
      const uint32_t bv[2] = {b.x, b.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[r][c] = umin(acc[r][c], P[r][c] * pk + av[r] + bv[c]);
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

template <bool I64>
__global__ void __launch_bounds__(kMcmThreads, 3) mcm_main_kernel(const McmLaunchArgs a) {
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
          ok = wait_flag_geq(a.flags + tile_index(inst, I, K), 1, limit, status) &&
               wait_flag_geq(a.flags + tile_index(inst, K, J), 1, limit, status) &&
               wait_flag_geq(a.flags + tile_index(inst, K + 1, J), 1, limit, status);
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
          if (D >= 1)
            ok = wait_flag_geq(a.flags + tile_index(inst, I, I), 1, limit, status) &&
                 wait_flag_geq(a.flags + tile_index(inst, J, J), 1, limit, status) &&
                 wait_flag_geq(a.flags + tile_index(inst, I + 1, J), 1, limit, status);
          if (ok && task.nparts > 0) ok = wait_flag_geq(a.counters + tidx, task.nparts, limit, status);
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
        if (!mbar_wait(&bar_full[g * kStages + st], round & 1u, limit)) {
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
        const uint32_t fpar = fin_cnt & 1u;
        const bool fin_ok = mbar_wait(bar_fin, fpar, limit);
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
            E* Ut = reinterpret_cast<E*>(smem + SM::UT);
            E* Lm = reinterpret_cast<E*>(smem + SM::LM);
            E* accv = reinterpret_cast<E*>(smem + SM::ACCV);
            E* pv = reinterpret_cast<E*>(smem + SM::PV);
            for (int idx = tid; idx < T * T; idx += kComputeThreads) {
              const int t = idx >> 5, x = idx & 31;
              Ut[t * SM::UP + x] = finU[idx] >> shiftv;
              Lm[t * SM::LP + x] = finL[idx] >> shiftv;
            }
            if (tid < T) {
              pv[tid] = (E)finPP[tid];
              pv[T + tid] = (E)(finPKI[tid] >> shiftv);
              pv[2 * T + tid] = (E)(finPKJ[tid] >> shiftv);
            }
            // boundary split k = IT + 31: U[li][31] + m[IT+32][j] + w
            const E brow = finBrow[lane] >> shiftv;
            const E pI32 = (E)(finPKI[T - 1] >> shiftv);
            E bnd[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int li = 4 * w + r;
              bestS[li * T + lane] = cb[r];  // external minimum: (value, smallest k)
              bnd[r] = (finU[(T - 1) * T + li] >> shiftv) + brow + pi[r] * pI32 * pj1;
              accv[li * SM::XP + lane] = umin((E)(cb[r] >> KB), bnd[r]);
            }
            bar_compute();
            {
              tile_solve_blocks<E>(Xv, accv, Ut, Lm, pv, pv + T, pv + 2 * T, warp, lane);
            }
            // ---------------- outputs needed by other tiles, then publish ----------------
            const int64_t nn = n;
            E vals[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) vals[r] = Xv[(4 * w + r) * SM::XP + lane];
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
            if (tid == 0) {
              __threadfence();
              st_release(a.flags + tidx, 1);
            }
            // provisional split: k of the external minimum (-1 if none); the split
            // pass replaces it by the smallest k over all splits reaching the value
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int li = 4 * w + r;
              const int64_t i = IT + li, j = JT + lane;
              const unsigned long long ek = bestS[li * T + lane];
              const int kx = (ek >> KB) == (~0ull >> KB) ? -1 : (int)(ek & ((1ull << KB) - 1ull));
              if (i < nn && j < nn) inst.s[i * nn + j] = (int16_t)kx;
            }
          } else {
            // diagonal tile: ordinary MCM on the 32-matrix sub-chain
            const E pj1d = (E)(finPKI[lane] >> shiftv);
#pragma unroll 1
            for (int e = 0; e <= T - 2; ++e) {
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const int li = 4 * w + r;
                if (lane - li == e) Xv[li * T + lane] = e == 0 ? (E)0 : (E)(cb[r] >> KB);
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
            const E v = upper ? (E)(cb[r] >> KB) : (E)0;
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
      __threadfence();
      if (!finisher)
        red_release_add(a.counters + tidx, 1);
      else if (D == 0)  // off-diagonal tiles publish right after their values
        st_release(a.flags + tidx, 1);
    }
  }
}

// One block per chain: validates dims, derives the cost bound and the packing
// shift, writes the padded / shifted dim arrays and the chain's pointers.
template <bool I64>
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
    if (mn < 1) {
      set_status(a.status, DP_EINVAL);
    } else if (mx >= 65536) {
      set_status(a.status, DP_EOVERFLOW);
    } else {
      const unsigned long long m3 = (unsigned long long)mx * mx * mx;      // < 2^48
      const unsigned long long bound = (unsigned long long)(n - 1) * m3;   // < 2^63
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

// Split pass for off-diagonal tiles: replaces the provisional split (k of
// the smallest external candidate) by the smallest k over ALL splits whose
// candidate equals the final m[i][j], scanning in increasing k: column splits
// k = IT+li .. IT+30, the boundary split IT+31, the external split, the row
// splits JT .. j-1.  Reads only the final table and the dims.
template <bool I64>
__global__ void __launch_bounds__(256) mcm_splits_kernel(const McmLaunchArgs a) {
  using E = typename Cost<I64>::E;
  __shared__ E Us[T][T + 1];   // Us[li][t]  = m[IT+li][IT+t]
  __shared__ E Xs[T + 1][T + 1];  // Xs[r][lj] = m[IT+r][JT+lj], r = 0..32 (row 32: boundary row)
  __shared__ E Ls[T][T + 1];   // Ls[u][lj] = m[JT+u+1][JT+lj]
  __shared__ E pI[T + 1], pJ[T + 1];  // p[IT + x], p[JT + x + 1]
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  // after a device-reported error the tables (and provisional splits) were
  // never written: touch nothing
  if (*reinterpret_cast<volatile int32_t*>(a.status) != 0) return;
  for (int t = blockIdx.x; t < a.ntasks; t += gridDim.x) {
    const McmTask task = a.tasks[t];
    const int I = task.I, J = task.J;
    if (task.kind != 0 || J == I) continue;  // diagonal tiles compute exact splits themselves
    const McmInstDev in = a.insts[task.inst];
    const int64_t n = in.n;
    const int IT = I * T, JT = J * T;
    const E* m = static_cast<const E*>(in.m);
    __syncthreads();
    for (int idx = tid; idx < T * T; idx += blockDim.x) {
      const int r = idx >> 5, x = idx & 31;
      const int64_t gi = IT + r;
      Us[r][x] = (gi < n && IT + x < n) ? m[gi * n + IT + x] : (E)0;
      Xs[r][x] = (gi < n && JT + x < n) ? m[gi * n + JT + x] : (E)0;
      const int64_t gl = JT + r + 1;
      Ls[r][x] = (gl < n && JT + x < n) ? m[gl * n + JT + x] : (E)0;
    }
    if (tid < T) {
      const int64_t gb = IT + T;
      Xs[T][tid] = (gb < n && JT + tid < n) ? m[gb * n + JT + tid] : (E)0;
    }
    if (tid <= T) {
      pI[tid] = (IT + tid <= n) ? (E)in.p[IT + tid] : (E)1;
      pJ[tid] = (JT + tid + 1 <= n) ? (E)in.p[JT + tid + 1] : (E)1;
    }
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
      const int li = 4 * w + r;
      const int64_t i = IT + li, j = JT + lane;
      if (i >= n || j >= n) continue;
      const E v = Xs[li][lane];
      const E pij = pI[li] * pJ[lane];  // p[i] * p[j+1]
      int k = -1;
      for (int tt = li; tt <= T - 1 && k < 0; ++tt)  // column splits and (tt = 31) the boundary split
        if (Us[li][tt] + Xs[tt + 1][lane] + pij * pI[tt + 1] == v) k = IT + tt;
      if (k < 0) {
        const int kx = in.s[i * n + j];  // external splits lie in [IT + 32, JT - 1]
        if (kx >= IT + T && kx < JT && m[i * n + kx] + m[(int64_t)(kx + 1) * n + j] + pij * (E)in.p[kx + 1] == v)
          k = kx;
      }
      for (int u = 0; u < lane && k < 0; ++u)
        if (Xs[li][u] + Ls[u][lane] + pij * pJ[u] == v) k = JT + u;
      in.s[i * n + j] = (int16_t)k;
    }
  }
}

}  // namespace

size_t mcm_smem_bytes(bool i64) { return i64 ? Smem<true>::TOTAL : Smem<false>::TOTAL; }

cudaError_t mcm_configure(bool i64) {
  if (i64)
    return cudaFuncSetAttribute(mcm_main_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Smem<true>::TOTAL);
  return cudaFuncSetAttribute(mcm_main_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Smem<false>::TOTAL);
}

cudaError_t mcm_occupancy(bool i64, int* blocks_per_sm) {
  if (i64)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcm_main_kernel<true>, kMcmThreads,
                                                         Smem<true>::TOTAL);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, mcm_main_kernel<false>, kMcmThreads,
                                                       Smem<false>::TOTAL);
}

cudaError_t mcm_preload(bool i64) {
  cudaFuncAttributes fa;
  cudaError_t e;
  if (i64) {
    if ((e = cudaFuncGetAttributes(&fa, mcm_prologue_kernel<true>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, mcm_main_kernel<true>)) != cudaSuccess) return e;
    return cudaFuncGetAttributes(&fa, mcm_splits_kernel<true>);
  }
  if ((e = cudaFuncGetAttributes(&fa, mcm_prologue_kernel<false>)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&fa, mcm_main_kernel<false>)) != cudaSuccess) return e;
  return cudaFuncGetAttributes(&fa, mcm_splits_kernel<false>);
}

cudaError_t launch_mcm_prologue(const McmLaunchArgs& a, bool i64, cudaStream_t st) {
  if (a.ninst <= 0) return cudaSuccess;
  if (i64)
    mcm_prologue_kernel<true><<<a.ninst, 256, 0, st>>>(a);
  else
    mcm_prologue_kernel<false><<<a.ninst, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mcm_splits(const McmLaunchArgs& a, bool i64, int grid, cudaStream_t st) {
  if (a.ntasks <= 0) return cudaSuccess;
  if (i64)
    mcm_splits_kernel<true><<<grid, 256, 0, st>>>(a);
  else
    mcm_splits_kernel<false><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mcm_main(const McmLaunchArgs& a, bool i64, int grid, cudaStream_t st) {
  if (a.ntasks <= 0) return cudaSuccess;
  if (i64)
    mcm_main_kernel<true><<<grid, kMcmThreads, Smem<true>::TOTAL, st>>>(a);
  else
    mcm_main_kernel<false><<<grid, kMcmThreads, Smem<false>::TOTAL, st>>>(a);
  return cudaGetLastError();
}

}  // namespace dpk
