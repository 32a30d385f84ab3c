// sdp_minjump.cu -- S-DP with (x) = min on one instance, cut into chunks that
// run side by side.
//
// Unrolling Eq. (1) with (x) = min down to the preset gives, for every N,
//     ST[N] = min_{s in C_N} ST[s],   C_N a subset of [0, a_1),
// where C_N = {N} for N < a_1 and C_N = union_j C_{N - a_j} otherwise
// (min is idempotent, so only which preset cells reach N matters, not how
// often).  The recurrence is shift-invariant, so the same holds for the table
// read from any position M on: ST[N + M] = min_{s in C_N} ST[M + s].  With
// M = t this gives the whole a_1-wide window at N from the first 2 a_1 - 1
// table values:
//     ST[N + t] = min_{s in C_N} ST[s + t],   0 <= t < a_1,              (W)
// and with M = N' it gives the composition rule
//     C_{N + N'} = union_{s in C_N} C_{N' + s}.
// Read C_N as a polynomial with Boolean coefficients, R_N(x) = sum_{s in C_N}
// x^s.  Then R_{N+1} = x R_N with x^{a_1} replaced by sum_j x^{a_1 - a_j}, so
// R_N is x^N reduced modulo chi(x) = x^{a_1} + sum_j x^{a_1 - a_j} over the
// Boolean semiring (OR for +, AND for x), and the composition rule is the
// product R_{N+N'} = R_N R_{N'} mod chi: a sumset of two bitsets followed by
// the reduction.  This is Kitamasa's method for linear recurrences, which
// needs only a commutative semiring; with bitsets a product costs about
// a_1^2 / 32 word operations.
//
// The path (a_k >= 32 and a_1 <= 8192; the reduction below relies on the
// first, the window kernel's run buffer on the second):
//   1. ST[a_1 .. 2 a_1 - 2] by the plain recurrence (the S-DP kernel);
//   2. C_L for the chunk length L = L0 2^s (L0 < a_1, so C_L0 = {L0}) by s
//      squarings, then C_{qL} for q < P by a doubling tree
//      (C_q = C_m C_{q-m} for q in (m, 2m], one launch per level, one block
//      per product);
//   3. a sparse table of range minima over ST[0 .. 2 a_1 - 2], and every
//      chunk's window by (W): the minimum, over the maximal runs [u, v] of
//      C_{qL}, of the range minimum of ST[t + u .. t + v];
//   4. the chunks [qL, (q+1)L), one block each, side by side, by the S-DP
//      kernel, each from its window.
// Every step is exact (minima and bit operations), so the table is
// bit-identical to the one the plain recurrence gives.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "api_internal.h"
#include "sdp_kernels.cuh"

namespace dpk {
namespace {

constexpr int kMjMaxA = 8192;                // a_1 limit of this path
constexpr int kMjMaxWords = kMjMaxA / 32;    // words of a set C (bits 0 .. a_1-1)
constexpr int kMjProdWords = 2 * kMjMaxWords;  // words of a product (bits 0 .. 2 a_1 - 2)
constexpr int kMjMaxRuns = kMjMaxA / 2 + 1;  // maximal runs of a set of a_1 bits

// Bits [p, p + 32) of the bitset w (words 0 .. nw-1, zero outside; p may be
// negative).
__device__ __forceinline__ uint32_t bits32(const uint32_t* w, int nw, int p) {
  const int q = p >> 5, r = p & 31;
  const uint32_t lo = (q >= 0 && q < nw) ? w[q] : 0u;
  const uint32_t hi = (q + 1 >= 0 && q + 1 < nw) ? w[q + 1] : 0u;
  return r == 0 ? lo : __funnelshift_r(lo, hi, r);
}

struct MjMulArgs {
  const uint32_t* x;  // item b: x + b * xs
  int64_t xs;
  const uint32_t* y;  // item b: y + b * ys
  int64_t ys;
  uint32_t* dst;      // item b: dst + b * ds (the reduced product, words 0 .. Aw-1)
  uint32_t* prod;     // item b: prod + b * kMjProdWords, zero between launches
  int32_t* counters;  // item b: blocks of the item done, zero between launches
  int64_t ds;
  const int32_t* offs;
  int32_t k;
  int32_t A;
};

// Exclusive prefix sum of v over the block (up to 1024 threads); *total gets
// the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int32_t* warp_sums, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < nwarps ? warp_sums[lane] : 0;
    int s = w;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane < nwarps) warp_sums[lane] = s - w;
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const int r = warp_sums[warp] + incl - v;
  __syncthreads();  // warp_sums may be reused by the caller
  return r;
}

// Lists the maximal runs of set bits of the A-bit set c (words 0 .. Aw-1,
// Aw <= blockDim.x) in run_u / run_v, in increasing order: the i-th run
// starts at the i-th set bit whose lower neighbour is clear and ends at the
// i-th set bit whose upper neighbour is clear.  Returns the number of runs.
__device__ int list_runs(const uint32_t* c, int A, int32_t* run_u, int32_t* run_v, int32_t* warp_sums,
                         int32_t* counts) {
  const int Aw = (A + 31) >> 5;
  const int tid = threadIdx.x;
  const uint32_t top_mask = (A & 31) ? (1u << (A & 31)) - 1u : 0xFFFFFFFFu;  // bits of the last word below A
  auto word = [&](int i) -> uint32_t {
    if (i < 0 || i >= Aw) return 0u;
    const uint32_t v = c[i];
    return i == Aw - 1 ? (v & top_mask) : v;
  };
  const uint32_t w = tid < Aw ? word(tid) : 0u;
  const uint32_t prevw = tid < Aw ? word(tid - 1) : 0u, nextw = tid < Aw ? word(tid + 1) : 0u;
  uint32_t starts = w & ~((w << 1) | (prevw >> 31));
  uint32_t ends = w & ~((w >> 1) | (nextw << 31));
  int rs = block_exclusive_scan(__popc(starts), warp_sums, &counts[0]);
  int re = block_exclusive_scan(__popc(ends), warp_sums, &counts[1]);
  while (starts) {
    run_u[rs++] = 32 * tid + __ffs(starts) - 1;
    starts &= starts - 1u;
  }
  while (ends) {
    run_v[re++] = 32 * tid + __ffs(ends) - 1;
    ends &= ends - 1u;
  }
  __syncthreads();
  return counts[0];
}

// One product modulo chi per item b = blockIdx.y: dst_b = (x_b y_b) mod chi,
// computed by gridDim.x blocks.
//  * If x or y is the full set [0, A), so is the product.  (With C_N full,
//    C_{N+M} = U_M, the union of C_{M+s} over 0 <= s < a_1; U_0 is the union
//    of the singletons {s}, the full set, and U_{M+1} contains U_M because
//    C_{M+a_1} contains C_M, a_1 being one of the offsets.)  Block 0 writes
//    it and no other work is done.
//  * Otherwise block sl takes the runs of x that START in its slice of x's
//    words (a run may extend into later slices) and ORs its part of the
//    sumset into the item's product in global memory: a run [u, v] of x
//    contributes y dilated by [u, v], the union of y << d for u <= d <= v.
//    A run of at most 32 bits is done bit by bit (thread i owns product word
//    i and ORs in bits [32 i - d, 32 i - d + 32) of y); a longer run by
//    doubling, E |= E << m for m = 1, 2, 4, ..., then shifted by u.
//  * The last block of the item to finish (a counter per item) reduces the
//    product: degrees d >= A are replaced, from the top down, by the degrees
//    d - a_j.  With a_k >= 32 a block of floor(a_k / 32) words never feeds
//    itself (every target lies at least a_k bits below the bit it comes from,
//    so below the block's lowest word), so a whole block of words is folded
//    at once: snapshot its degrees >= A, OR each of them shifted down by every
//    a_j into the lower words, then clear them.  It then clears the product
//    and the counter for the next launch.
constexpr int kMjThreads = 512;   // >= kMjProdWords: thread x owns product word x
constexpr int kMjSlices = 32;     // blocks per product
constexpr int kMjSliceRuns = 8 * 32 / 2 + 2;  // runs that can start in a slice of <= 8 words
__global__ void __launch_bounds__(kMjThreads) mj_mul_kernel(const MjMulArgs a) {
  __shared__ uint32_t xw[kMjMaxWords], ys[kMjMaxWords];
  __shared__ uint32_t z[kMjProdWords], e[kMjProdWords];
  __shared__ int32_t run_u[kMjSliceRuns], run_v[kMjSliceRuns];
  __shared__ int32_t warp_sums[32], nruns, popx, popy, last;
  const int b = blockIdx.y, sl = blockIdx.x, S = gridDim.x;
  const int A = a.A, Aw = (A + 31) >> 5, Pw = 2 * Aw;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t top_mask = (A & 31) ? (1u << (A & 31)) - 1u : 0xFFFFFFFFu;  // bits of the last word below A
  const uint32_t* x = a.x + b * a.xs;
  const uint32_t* y = a.y + b * a.ys;
  uint32_t* dst = a.dst + b * a.ds;
  if (tid == 0) popx = popy = nruns = 0;
  __syncthreads();
  int px = 0, py = 0;
  if (tid < Aw) {
    xw[tid] = x[tid] & (tid == Aw - 1 ? top_mask : 0xFFFFFFFFu);
    ys[tid] = y[tid] & (tid == Aw - 1 ? top_mask : 0xFFFFFFFFu);
    px = __popc(xw[tid]);
    py = __popc(ys[tid]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    px += __shfl_xor_sync(0xffffffffu, px, o);
    py += __shfl_xor_sync(0xffffffffu, py, o);
  }
  if (lane == 0 && (px | py)) {
    atomicAdd(&popx, px);
    atomicAdd(&popy, py);
  }
  __syncthreads();
  if (popx == A || popy == A) {
    if (sl == 0 && tid < Aw) dst[tid] = tid == Aw - 1 ? top_mask : 0xFFFFFFFFu;
    return;  // every block of the item leaves here: the counter is not used
  }
  // runs starting in this slice's words [w0, w1)
  const int w0 = (int)((int64_t)sl * Aw / S), w1 = (int)((int64_t)(sl + 1) * Aw / S);
  uint32_t starts = 0u;
  if (tid < w1 - w0) {
    const int i = w0 + tid;
    starts = xw[i] & ~((xw[i] << 1) | (i > 0 ? xw[i - 1] >> 31 : 0u));
  }
  int r = block_exclusive_scan(__popc(starts), warp_sums, &nruns);
  while (starts) {
    const int u = 32 * (w0 + tid) + __ffs(starts) - 1;
    starts &= starts - 1u;
    // the run's end: the bit before the first clear bit at or above u
    int w = u >> 5;
    uint32_t rest = ~(xw[w] >> (u & 31));  // clear bits from u up (bits beyond the word read as clear)
    int v;
    if ((u & 31) != 0 && rest == (0xFFFFFFFFu << (32 - (u & 31)))) rest = 0u;  // word w set from u to its top
    if (rest) {
      v = u + __ffs(rest) - 2;
    } else {
      ++w;
      while (w < Aw && xw[w] == 0xFFFFFFFFu) ++w;
      v = w < Aw ? 32 * w + __ffs(~xw[w]) - 2 : 32 * Aw - 1;
    }
    run_u[r] = u;
    run_v[r] = v < A - 1 ? v : A - 1;
    ++r;
  }
  __syncthreads();
  const int R = nruns;
  uint32_t acc = 0u;
  for (int i = 0; i < R; ++i) {
    const int u = run_u[i], len = run_v[i] - u + 1;
    if (len <= 32) {
      if (tid < Pw)
        for (int d = u; d < u + len; ++d) acc |= bits32(ys, Aw, 32 * tid - d);
      continue;
    }
    if (tid < Pw) e[tid] = tid < Aw ? ys[tid] : 0u;
    __syncthreads();
    int m = 1;
    for (; 2 * m <= len; m *= 2) {  // e = y dilated by [0, 2m)
      const uint32_t val = tid < Pw ? (e[tid] | bits32(e, Pw, 32 * tid - m)) : 0u;
      __syncthreads();
      if (tid < Pw) e[tid] = val;
      __syncthreads();
    }
    if (m < len) {  // [0, m) and [len - m, len) cover [0, len)
      const uint32_t val = tid < Pw ? (e[tid] | bits32(e, Pw, 32 * tid - (len - m))) : 0u;
      __syncthreads();
      if (tid < Pw) e[tid] = val;
      __syncthreads();
    }
    if (tid < Pw) acc |= bits32(e, Pw, 32 * tid - u);
    __syncthreads();
  }
  uint32_t* prod = a.prod + (int64_t)b * kMjProdWords;
  if (tid < Pw && acc) atomicOr(prod + tid, acc);
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(a.counters + b, 1) == S - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tid < Pw) {
    z[tid] = __ldcg(prod + tid);
    prod[tid] = 0u;
  }
  if (tid == 0) a.counters[b] = 0;
  __syncthreads();
  // reduction modulo chi
  uint32_t* blk = e;  // reused
  const int Wb = a.offs[a.k - 1] >> 5;  // >= 1 on this path
  const int wlo = A >> 5;               // lowest word holding a degree >= A
  const uint32_t hi_mask = ~top_mask | ((A & 31) ? 0u : 0xFFFFFFFFu);  // degrees >= A in word wlo
  for (int top = Pw - 1; top >= wlo; top -= Wb) {
    const int bot = top - Wb + 1 > wlo ? top - Wb + 1 : wlo;
    const int nwords = top - bot + 1;
    if (tid < nwords) {
      const int w = bot + tid;
      blk[tid] = w == wlo ? (z[w] & hi_mask) : z[w];
    }
    __syncthreads();
    for (int p = tid; p < nwords * a.k; p += blockDim.x) {
      const int wi = p % nwords, j = p / nwords;
      const uint32_t bits = blk[wi];
      if (!bits) continue;
      // bit c of word w (degree 32 w + c >= A >= a_j) goes to degree 32 w + c - a_j
      const int tb = 32 * (bot + wi) - a.offs[j];
      const int tq = tb >> 5, tr = tb & 31;  // tq >= -1; word -1 would only receive bits below A, which are 0
      if (tq >= 0) atomicOr(&z[tq], bits << tr);
      if (tr) atomicOr(&z[tq + 1], bits >> (32 - tr));
    }
    __syncthreads();
    if (tid < nwords) {
      const int w = bot + tid;
      z[w] = w == wlo ? (z[w] & ~hi_mask) : 0u;
    }
    __syncthreads();
  }
  if (tid < Aw) dst[tid] = z[tid];
}

// Range minima over ST[0 .. m-1]: sp[l][i] = min ST[i .. i + 2^l - 1] for
// i + 2^l <= m.  Block b fills i in [1024 b, 1024 b + 1024) for every level:
// it stages ST[1024 b .. 1024 b + 1024 + 2^(levels-1)) and doubles in place.
constexpr int kRmqTile = 1024;
__global__ void __launch_bounds__(1024) mj_rmq_kernel(const uint32_t* st, int m, uint32_t* sp, int levels) {
  extern __shared__ uint32_t buf[];
  const int i0 = blockIdx.x * kRmqTile;
  const int span = min(m - i0, kRmqTile + (1 << (levels - 1)));
  for (int i = threadIdx.x; i < span; i += blockDim.x) buf[i] = st[i0 + i];
  __syncthreads();
  for (int i = threadIdx.x; i < kRmqTile && i0 + i < m; i += blockDim.x) sp[i0 + i] = buf[i];
  for (int l = 1; l < levels; ++l) {
    const int h = 1 << (l - 1);
    // buf[i] = min(buf[i], buf[i + h]) for i + 2h <= span, read before written
    const int cnt = span - 2 * h + 1;
    uint32_t vals[(kRmqTile + (1 << 13)) / 1024 + 1];
#pragma unroll
    for (int r = 0; r < (int)(sizeof(vals) / sizeof(vals[0])); ++r) {
      const int i = threadIdx.x + r * blockDim.x;
      vals[r] = i < cnt ? min(buf[i], buf[i + h]) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < (int)(sizeof(vals) / sizeof(vals[0])); ++r) {
      const int i = threadIdx.x + r * blockDim.x;
      if (i < cnt) buf[i] = vals[r];
    }
    __syncthreads();
    uint32_t* row = sp + (int64_t)l * m;
    for (int i = threadIdx.x; i < kRmqTile && i < cnt; i += blockDim.x) row[i0 + i] = buf[i];
  }
}

// Windows by (W), one block per item q = blockIdx.x + 1: the maximal runs of
// C = sets + q Aw are listed, then output t is the minimum over the runs
// [u, v] of min ST[t + u .. t + v], two reads of the range-minimum table.
__global__ void __launch_bounds__(1024) mj_window_kernel(const uint32_t* sets, int A, const uint32_t* sp, int m,
                                                         uint32_t* st, int64_t n, int64_t L) {
  __shared__ int32_t run_u[kMjMaxRuns], run_v[kMjMaxRuns];
  __shared__ int32_t warp_sums[32], counts[2];
  const int q = blockIdx.x + 1;
  const int Aw = (A + 31) >> 5;
  const int R = list_runs(sets + (int64_t)q * Aw, A, run_u, run_v, warp_sums, counts);
  const int64_t pos = (int64_t)q * L;
  for (int t = threadIdx.x; t < A; t += blockDim.x) {
    if (pos + t >= n) break;
    uint32_t v = 0xFFFFFFFFu;
    for (int i = 0; i < R; ++i) {
      const int lo = t + run_u[i], hi = t + run_v[i];
      const int l = 31 - __clz(hi - lo + 1);
      const uint32_t* row = sp + (int64_t)l * m;
      v = __vimin3_u32(v, row[lo], row[hi - (1 << l) + 1]);
    }
    st[pos + t] = v;
  }
}

// Device-side set-up: the offsets, the chunk records, the record of the
// first 2 A - 1 cells, and C_L0 = {L0}.
struct MjSetup {
  int32_t offs[kSdpMaxK];
  int32_t k;
  int32_t A;
  int32_t P;
  int32_t L0;
  int64_t L;
  int64_t n;
  uint32_t* st;
  int32_t* d_offs;
  uint32_t* set1;  // C_L0, Aw words
  SdpInstDev* insts;
  SdpInstDev* pre;
};

__global__ void __launch_bounds__(256) mj_setup_kernel(const MjSetup s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int Aw = (s.A + 31) >> 5;
  if (i < s.k) s.d_offs[i] = s.offs[i];
  if (i < Aw) s.set1[i] = (s.L0 >> 5) == i ? (1u << (s.L0 & 31)) : 0u;
  if (i == 0) {
    SdpInstDev in{};
    in.st = s.st;
    in.n = 2 * (int64_t)s.A - 1 < s.n ? 2 * (int64_t)s.A - 1 : s.n;
    in.a = s.d_offs;
    in.k = s.k;
    *s.pre = in;
  }
  if (i < s.P) {
    SdpInstDev in{};
    in.st = s.st + i * s.L;
    in.n = s.n - i * s.L < s.L ? s.n - i * s.L : s.L;
    in.a = s.d_offs;
    in.k = s.k;
    s.insts[i] = in;
  }
}

}  // namespace
}  // namespace dpk

namespace dph {

namespace {
// Plain-kernel time model, microseconds: about 220 + W (k + 2) / 32 clocks
// per step of W = min(a_k, 1024) cells at 2 GHz (measured at k = 32).
double mj_plain_us(int64_t cells, int32_t ak, int32_t k) {
  if (cells <= 0) return 0.0;
  const double W = std::min<int32_t>(ak, 1024);
  return std::ceil((double)cells / W) * (220.0 + W * (k + 2) / 32.0) / 2.0e3;
}

struct MjPlan {
  int P = 0;
  int64_t L = 0;
  int32_t L0 = 0;
  int s = 0;
};

// About `chunks` chunks of length L = L0 2^s with L0 < A (so that C_L0 is the
// monomial x^L0); P = 0 when chunks of at least 2 A cells are impossible.
MjPlan mj_plan_for(int64_t n, int32_t A, int chunks) {
  MjPlan p;
  if (chunks < 2 || A < 2) return p;
  const int64_t Lt = (n + chunks - 1) / chunks;
  if (Lt < 2 * (int64_t)A) return p;
  int s = 0;
  while (((Lt + ((int64_t)1 << s) - 1) >> s) > A - 1) ++s;
  p.s = s;
  p.L0 = (int32_t)((Lt + ((int64_t)1 << s) - 1) >> s);
  p.L = (int64_t)p.L0 << s;
  p.P = (int)((n + p.L - 1) / p.L);
  if (p.P < 2) p.P = 0;
  return p;
}

int mj_levels(int64_t qmax) {
  int l = 0;
  for (int64_t m = 1; m + 1 <= qmax; m *= 2) ++l;
  return l;
}

// Overhead model of the jump, microseconds: about 8 us per product level
// (one launch) and 30 us for the set-up, the range-minimum table and the
// windows.
double mj_jump_us(int64_t n, int32_t A, int32_t ak, int32_t k, const MjPlan& p) {
  const int levels = p.s + mj_levels(p.P - 1);
  return mj_plain_us(std::min<int64_t>(p.L, n) - A, ak, k) + mj_plain_us(A, ak, k) + 8.0 * levels + 30.0;
}

dp_status mj_launch_records(const dpk::SdpInstDev* insts, int count, int32_t k, int32_t threads, int32_t ring_log2,
                            int32_t* status, cudaStream_t stream) {
  if (count <= 0) return DP_OK;
  dpk::SdpLaunchArgs args{};
  args.insts = insts;
  args.one.k = k;
  args.kfull = k == dpk::kSdpMaxKRegs;
  args.ninst = count;
  args.op = DP_OP_MIN;
  args.threads = threads;
  args.ring_log2 = ring_log2;
  args.status = status;
  const cudaError_t e = dpk::launch_sdp(args, stream);
  return e == cudaSuccess ? DP_OK : fail_cuda(e, "sdp min jump: launch of the chunk kernel");
}
}  // namespace

bool sdp_min_jump_eligible(int64_t n, const int32_t* a, int32_t k) {
  const int32_t A = a[0], ak = a[k - 1];
  if (A < 2 || A > dpk::kMjMaxA || ak < 32 || n < 8 * (int64_t)A) return false;
  int32_t tl = 0, rl = 0;
  sdp_shape(A, ak, &tl, &rl);
  return rl > 0;  // the chunks keep the window on chip
}

int sdp_min_jump_plan(int64_t n, const int32_t* a, int32_t k, int sms, int64_t out[5]) {
  const int chunks = sdp_min_jump_chunks(n, a, k, sms);
  for (int i = 0; i < 5; ++i) out[i] = 0;
  if (chunks < 2) return 0;
  const MjPlan p = mj_plan_for(n, a[0], chunks);
  out[0] = p.P;
  out[1] = p.L;
  out[2] = p.L0;
  out[3] = p.s;
  out[4] = chunks;
  return chunks;
}

int sdp_min_jump_chunks(int64_t n, const int32_t* a, int32_t k, int sms) {
  if (!sdp_min_jump_eligible(n, a, k)) return 0;
  const int32_t A = a[0], ak = a[k - 1];
  double best = 0.8 * mj_plain_us(n - A, ak, k);  // the jump must win clearly
  int bestP = 0;
  for (int c = 2; c <= sms; ++c) {
    const MjPlan p = mj_plan_for(n, A, c);
    if (p.P < 2) break;
    const double t = mj_jump_us(n, A, ak, k, p);
    if (t < best) {
      best = t;
      bestP = c;
    }
  }
  return bestP;
}

dp_status sdp_min_jump(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, int chunks, int32_t* status,
                       cudaStream_t st) {
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  if (!sdp_min_jump_eligible(n, a, k))
    return fail(DP_EINVAL, "sdp min jump: needs a_k >= 32, a_1 <= %d and n >= 8 a_1", dpk::kMjMaxA);
  const int32_t A = a[0];
  const MjPlan pl = mj_plan_for(n, A, chunks);
  if (pl.P < 2)
    return fail(DP_EINVAL, "sdp min jump: %d chunks of at least %d cells do not fit n = %lld", chunks, 2 * A,
                (long long)n);
  int32_t threads = 0, ring_log2 = 0;
  sdp_shape(A, a[k - 1], &threads, &ring_log2);
  const int P = pl.P;
  const int Aw = (A + 31) / 32;
  const int m = 2 * A - 1;
  int levels = 1;
  while ((1 << levels) <= m) ++levels;  // rows l with 2^l <= m
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += al(std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_offs = take((size_t)k * 4);
  const size_t o_sets = take((size_t)P * Aw * 4);                       // C_{qL}, q = 0 .. P-1 (q = 0 unused)
  const size_t o_sp = take((size_t)levels * m * 4);                     // range-minimum table
  int64_t nb = 1;                                                       // widest batch of the product tree
  for (int64_t mm = 1; mm + 1 <= P - 1; mm *= 2) nb = std::max<int64_t>(nb, std::min<int64_t>(2 * mm, P - 1) - mm);
  const size_t o_prod = take((size_t)nb * dpk::kMjProdWords * 4);       // sumsets of one level
  const size_t o_cnt = take((size_t)nb * 4);                            // finished blocks per product
  const size_t o_insts = take((size_t)P * sizeof(dpk::SdpInstDev));
  const size_t o_pre = take(sizeof(dpk::SdpInstDev));
  uint8_t* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), off, st);
  if (e != cudaSuccess) return fail_cuda(e, "sdp min jump: workspace");
  int32_t* d_offs = reinterpret_cast<int32_t*>(ws + o_offs);
  uint32_t* sets = reinterpret_cast<uint32_t*>(ws + o_sets);
  uint32_t* sp = reinterpret_cast<uint32_t*>(ws + o_sp);
  uint32_t* prod = reinterpret_cast<uint32_t*>(ws + o_prod);
  int32_t* counters = reinterpret_cast<int32_t*>(ws + o_cnt);
  auto* insts = reinterpret_cast<dpk::SdpInstDev*>(ws + o_insts);
  auto* pre = reinterpret_cast<dpk::SdpInstDev*>(ws + o_pre);

  const bool prof = profiling();
  if (prof) profile_mark(1, st, false);
  auto done = [&](dp_status r) {
    if (prof) profile_mark(1, st, true);
    const cudaError_t fe = cudaFreeAsync(ws, st);
    if (r == DP_OK && fe != cudaSuccess) return fail_cuda(fe, "sdp min jump: workspace release");
    return r;
  };

  dpk::MjSetup su{};
  for (int j = 0; j < k; ++j) su.offs[j] = a[j];
  su.k = k;
  su.A = A;
  su.P = P;
  su.L0 = pl.L0;
  su.L = pl.L;
  su.n = n;
  su.st = ST;
  su.d_offs = d_offs;
  su.set1 = sets + Aw;
  su.insts = insts;
  su.pre = pre;
  const int64_t su_n = std::max<int64_t>({(int64_t)k, (int64_t)Aw, (int64_t)P, 1});
  dpk::mj_setup_kernel<<<(unsigned)((su_n + 255) / 256), 256, 0, st>>>(su);
  // the product buffers and counters start at zero; every product leaves them so
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemsetAsync(ws + o_prod, 0, o_cnt + nb * 4 - o_prod, st)) != cudaSuccess)
    return done(fail_cuda(e, "sdp min jump: set-up"));
  // 1. ST[A .. 2A - 2]
  if ((rc = mj_launch_records(pre, 1, k, threads, ring_log2, status, st)) != DP_OK) return done(rc);
  // dst + i ds = (x + i xs)(y + i ys) mod chi for i < cnt
  auto mulmod = [&](const uint32_t* x, int64_t xs, const uint32_t* y, int64_t ys, uint32_t* dst, int64_t ds_,
                    int64_t cnt) {
    dpk::MjMulArgs ma{};
    ma.x = x;
    ma.xs = xs;
    ma.y = y;
    ma.ys = ys;
    ma.dst = dst;
    ma.ds = ds_;
    ma.prod = prod;
    ma.counters = counters;
    ma.offs = d_offs;
    ma.k = k;
    ma.A = A;
    const int slices = std::min(dpk::kMjSlices, Aw);
    dpk::mj_mul_kernel<<<dim3((unsigned)slices, (unsigned)cnt), dpk::kMjThreads, 0, st>>>(ma);
    return cudaGetLastError();
  };
  // 2. C_L = C_L0 squared s times; C_q = C_m C_{q-m} for q in (m, 2m], q <= P - 1
  for (int i = 0; i < pl.s; ++i)
    if ((e = mulmod(sets + Aw, 0, sets + Aw, 0, sets + Aw, 0, 1)) != cudaSuccess)
      return done(fail_cuda(e, "sdp min jump: squaring"));
  for (int64_t mm = 1; mm + 1 <= P - 1; mm *= 2) {
    const int64_t cnt = std::min<int64_t>(2 * mm, P - 1) - mm;
    if ((e = mulmod(sets + mm * Aw, 0, sets + Aw, Aw, sets + (mm + 1) * Aw, Aw, cnt)) != cudaSuccess)
      return done(fail_cuda(e, "sdp min jump: product tree"));
  }
  // 3. range minima over ST[0 .. 2A - 2], then the windows at q L, q = 1 .. P-1
  dpk::mj_rmq_kernel<<<(unsigned)((m + dpk::kRmqTile - 1) / dpk::kRmqTile), 1024,
                       (size_t)std::min(m, dpk::kRmqTile + (1 << (levels - 1))) * 4, st>>>(ST, m, sp, levels);
  if ((e = cudaGetLastError()) != cudaSuccess) return done(fail_cuda(e, "sdp min jump: range minima"));
  dpk::mj_window_kernel<<<(unsigned)(P - 1), 1024, 0, st>>>(sets, A, sp, m, ST, n, pl.L);
  if ((e = cudaGetLastError()) != cudaSuccess) return done(fail_cuda(e, "sdp min jump: windows"));
  // 4. the chunks, side by side
  if ((rc = mj_launch_records(insts, P, k, threads, ring_log2, status, st)) != DP_OK) return done(rc);
  return done(DP_OK);
}

}  // namespace dph
