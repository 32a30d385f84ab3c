// sdp_jump.cu -- S-DP with (x) = + modulo 2^32 on one instance, cut into
// chunks that run side by side.
//
// With (x) = +, Eq. (1) is a linear recurrence with constant coefficients
// over Z/2^32.  Its characteristic polynomial
//     chi(x) = x^{a_1} - sum_j x^{a_1 - a_j}
// is monic, so x^N mod chi = sum_{s < a_1} r_s x^s exists over Z/2^32 for
// every N, and the linear map x^m -> ST[m] vanishes on x^m chi(x) for every
// m (that is the recurrence).  Hence, for every N and t,
//     ST[N + t] = sum_{s < a_1} r_s ST[s + t],                          (J)
// the jump of Fiduccia's method for linear recurrences (C. M. Fiduccia, "An
// efficient formula for linear recurrences", SIAM J. Comput. 14, 1985): the
// whole a_1-wide window at N follows from the first 2 a_1 - 1 table values.
// The paper runs the recurrence one block of cells at a time (Section III);
// this path gives every chunk of the table its own starting window, so that
// the chunks run at once on separate SMs:
//   1. ST[a_1 .. 2 a_1 - 2] by the plain recurrence (the S-DP kernel);
//   2. beside it, g, the impulse response of the recurrence (g[0] = 1,
//      g[m] = sum_j g[m - a_j]) up to m = Gm, by the same kernel;
//   3. R_1 = x^L mod chi for the chunk length L = L0 2^s (L0 <= Gm) by s
//      squarings of x^L0 mod chi, which g gives directly
//      (jump_start_kernel); R_j = x^{jL} for j <= P2 and Q_i = x^{i P2 L}
//      for i < P1 by doubling trees, R_q = R_m R_{q-m} for q in (m, 2m], a
//      level per set of launches;
//   4. the windows at (i P2 + j) L by (J): the "major" ones (j = 0) from the
//      preset via Q_i, each extended by a_1 - 1 values with the plain
//      kernel, then the others from their major window via R_j: batched
//      Hankel products;
//   5. the chunks [pL, (p+1)L), one block each, side by side, by the S-DP
//      kernel, each from its window.
// Reduction of a product c (degree <= 2 a_1 - 2) modulo chi: let h[d] be the
// multiple of x^{d - a_1} chi taken away at degree d, from the top down.
// Then h[d] = c[d] + sum_j h[d + a_j], whose solution is h[d] = sum_m g[m]
// c[d + m], and the remainder is r[e] = c[e] + sum_j h[e + a_j] over the j
// with a_1 <= e + a_j <= 2 a_1 - 2.
// Every product and sum wraps modulo 2^32, which is exact in Z/2^32, so the
// table is bit-identical to the one the plain recurrence gives.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "api_internal.h"
#include "sdp_kernels.cuh"

namespace dpk {
namespace {

// ---------------------------------------------------------------------------
// Batched Toeplitz product over Z/2^32:
//   CONV: out[b][t] (+)= sum_s u[b][s] z[b][t - s + zoff]
//   CORR: out[b][t] (+)= sum_s u[b][s] z[b][t + s + zoff]
// for t < tout, s < S, z read as 0 outside [0, zlen).  A block computes
// kTB consecutive outputs over pieces of kSB splits: pieces blockIdx.y,
// blockIdx.y + gridDim.y, ...  (with gridDim.y > 1 the outputs are added
// with atomics into a zeroed buffer); blockIdx.z is the batch item.  A
// thread keeps kTo consecutive outputs and, per inner step of kTs splits,
// the kTo + kTs - 1 z values they need in registers: 256 multiply-adds for
// 12 shared-memory vector loads.  The staged z window is padded by 4 words
// every 16, so that the 16-byte loads of a quarter-warp (threads 16 words
// apart) fall into distinct banks.
// ---------------------------------------------------------------------------
constexpr int kTT = 256;                // threads per block
constexpr int kTo = 16;                 // outputs per thread
constexpr int kTs = 16;                 // splits per inner step
constexpr int kTB = kTT * kTo;          // outputs per block
constexpr int kSB = 128;                // splits per piece
constexpr int kZW = kTB + kSB + 32;     // staged z words
__host__ __device__ constexpr int zpad(int i) { return i + 4 * (i >> 4); }
constexpr int kZS = zpad(kZW) + 4;      // padded staging words

// Batch item b is (v, b_hi, b_lo): v = b / nvi (0 when nvi <= 0), then
// (b_hi, b_lo) = (r / nlo, r % nlo) for r = b - v nvi; each operand moves by
// its lo stride per b_lo, its hi stride per b_hi and its v stride per v.
struct ToepArgs {
  const uint32_t* u;
  int64_t ustride, ustride_hi;
  int64_t S;
  const uint32_t* z;
  int64_t zstride, zstride_hi;
  int64_t zlen;
  int64_t zoff;
  int64_t zlim;  // z word i of item b is read only where (its offset from z) + i < zlim
  uint32_t* out;
  int64_t ostride, ostride_hi;
  int64_t tout;
  int64_t olim;  // out word t of item b is written only where (its offset from out) + t < olim
  int64_t nlo;
  uint32_t* zero;    // zero[0 .. zero_len) is cleared by the grid, for a later launch
  int64_t zero_len;
  int64_t nvi;       // items per variant (<= 0: one variant)
  int64_t ustride_v, zstride_v, ostride_v;
};

template <bool CONV>
__global__ void __launch_bounds__(kTT) toeplitz_kernel(const ToepArgs a) {
  __shared__ __align__(16) uint32_t us[kSB];
  __shared__ __align__(16) uint32_t zs[kZS];
  const int tid = threadIdx.x;
  if (a.zero_len > 0) {
    const int64_t nthreads = (int64_t)gridDim.x * gridDim.y * gridDim.z * kTT;
    const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    for (int64_t i = blk * kTT + tid; i < a.zero_len; i += nthreads) a.zero[i] = 0u;
  }
  const int64_t T0 = (int64_t)blockIdx.x * kTB;
  const int64_t bv = a.nvi > 0 ? (int64_t)blockIdx.z / a.nvi : 0;
  const int64_t br = (int64_t)blockIdx.z - bv * (a.nvi > 0 ? a.nvi : 0);
  const int64_t b_hi = br / a.nlo, b_lo = br % a.nlo;
  if (T0 >= a.tout) return;
  const int64_t Tw = T0 + (int64_t)(tid >> 5) * (32 * kTo);  // the warp's first output
  const int64_t zo = bv * a.zstride_v + b_hi * a.zstride_hi + b_lo * a.zstride;
  const uint32_t* zb = a.z + zo;
  const int64_t zlen = a.zlen < a.zlim - zo ? a.zlen : a.zlim - zo;
  const uint32_t* ub = a.u + bv * a.ustride_v + b_hi * a.ustride_hi + b_lo * a.ustride;
  uint32_t acc[kTo];
#pragma unroll
  for (int q = 0; q < kTo; ++q) acc[q] = 0u;
  // pieces blockIdx.y, blockIdx.y + gridDim.y, ... of kSB splits each
  for (int64_t S0 = (int64_t)blockIdx.y * kSB; S0 < a.S; S0 += (int64_t)gridDim.y * kSB) {
    // z index of output t = T0 + i and split s = S0 + j: c + i - j (CONV) or
    // c + i + j (CORR); the piece's range of z indices:
    const int64_t c = CONV ? T0 - S0 + a.zoff : T0 + S0 + a.zoff;
    const int64_t zmin = CONV ? c - (kSB - 1) : c;
    const int64_t zmax = CONV ? c + (kTB - 1) : c + (kTB - 1) + (kSB - 1);
    if (zmax < 0 || zmin >= zlen) continue;  // every product of the piece is zero (same for the whole block)
    // zs[i] holds z[zbase + i]; thread tid at inner step j reads the 32 words
    // from start(tid, j), a multiple of 16
    const int64_t zbase = CONV ? c - kSB - 15 : c;
    __syncthreads();  // the previous piece's reads are done
    for (int i = tid; i < kZW; i += kTT) {
      const int64_t zi = zbase + i;
      zs[zpad(i)] = (zi >= 0 && zi < zlen) ? zb[zi] : 0u;
    }
    for (int i = tid; i < kSB; i += kTT) us[i] = S0 + i < a.S ? ub[S0 + i] : 0u;
    __syncthreads();
#pragma unroll 1
    for (int j = 0; j < kSB; j += kTs) {
      // the warp's z indices at this step; all outside [0, zlen): nothing to add
      const int64_t wlo = CONV ? Tw - (S0 + j) - (kTs - 1) + a.zoff : Tw + S0 + j + a.zoff;
      const int64_t whi = wlo + (32 * kTo - 1) + (kTs - 1);
      if (whi < 0 || wlo >= zlen) continue;
      uint32_t ur[kTs], zr[32];
#pragma unroll
      for (int v = 0; v < kTs / 4; ++v) {
        const uint4 x = *reinterpret_cast<const uint4*>(us + j + 4 * v);
        ur[4 * v] = x.x;
        ur[4 * v + 1] = x.y;
        ur[4 * v + 2] = x.z;
        ur[4 * v + 3] = x.w;
      }
      const int start = CONV ? kTo * tid - j + kSB : kTo * tid + j;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const uint4 x = *reinterpret_cast<const uint4*>(zs + zpad(start + 4 * v));
        zr[4 * v] = x.x;
        zr[4 * v + 1] = x.y;
        zr[4 * v + 2] = x.z;
        zr[4 * v + 3] = x.w;
      }
      // CONV: z index c + kTo*tid + q - (j + r) = zbase + start + 15 + q - r
      // CORR: z index c + kTo*tid + q + (j + r) = zbase + start + q + r
#pragma unroll
      for (int r = 0; r < kTs; ++r)
#pragma unroll
        for (int q = 0; q < kTo; ++q) acc[q] += ur[r] * zr[CONV ? 15 + q - r : q + r];
    }
  }
  // every output of the block is written (zero where no piece contributed);
  // with the split range divided between blocks (gridDim.y > 1) the pieces'
  // sums are added into a zeroed buffer
  const int64_t oo = bv * a.ostride_v + b_hi * a.ostride_hi + b_lo * a.ostride;
  uint32_t* ob = a.out + oo;
  const bool split = gridDim.y > 1;
#pragma unroll
  for (int q = 0; q < kTo; ++q) {
    const int64_t t = T0 + (int64_t)kTo * tid + q;
    if (t < a.tout && oo + t < a.olim) {
      if (split)
        atomicAdd(ob + t, acc[q]);
      else
        ob[t] = acc[q];
    }
  }
}

// Transposed Karatsuba for a batch of middle products out[t] = sum_{s < 2h}
// u[s] z[t + s], t < 2h (rows (hi, lo): u by lo, z by hi): with u = u0 | u1
// and z viewed from 0, h and 2h,
//   out[t]     = P0[t] + P1[t],  out[h + t] = P0[t] + P2[t]   (t < h),
//   P0 = M(u0 + u1, z[h..]),  P1 = M(u0, z[..] - z[h..]),  P2 = M(u1, z[2h..] - z[h..]),
// three middle products of half the size (three quarters of the
// multiply-adds); exact over Z/2^32. This kernel lays out the operands of
// the three as variants v = 0, 1, 2 of one batch: ku[v][lo][s] (s < h) and
// kz[v][hi][i] (i < 2h - 1, rows of 2h words), with z read as 0 outside
// [0, zlen) and where (its offset from z) + i >= zlim.
__global__ void __launch_bounds__(256) kara_prep_kernel(const uint32_t* u, int64_t us, int64_t nlo, const uint32_t* z,
                                                        int64_t zs_hi, int64_t zlen, int64_t zlim, int64_t nhi,
                                                        int64_t h, uint32_t* ku, uint32_t* kz) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (b < nlo && x < h) {
    const uint32_t u0 = u[b * us + x], u1 = u[b * us + h + x];
    ku[b * h + x] = u0 + u1;
    ku[(nlo + b) * h + x] = u0;
    ku[(2 * nlo + b) * h + x] = u1;
  }
  if (b < nhi && x < 2 * h - 1) {
    const int64_t zo = b * zs_hi;
    auto Z = [&](int64_t i) { return (i < zlen && zo + i < zlim) ? z[zo + i] : 0u; };
    const uint32_t mid = Z(h + x);
    kz[b * 2 * h + x] = mid;
    kz[(nhi + b) * 2 * h + x] = Z(x) - mid;
    kz[(2 * nhi + b) * 2 * h + x] = Z(2 * h + x) - mid;
  }
}

// out[r][t] = P0[r][t] + P1[r][t], out[r][h + t] = P0[r][t] + P2[r][t] for
// t < h, rows r of 2h words; the products in kout[v][r][t] (the last step of
// the transposed Karatsuba above).
__global__ void __launch_bounds__(256) kara_combine_kernel(uint32_t* out, const uint32_t* kout, int64_t rows,
                                                           int64_t h) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = blockIdx.y;
  if (t >= h) return;
  const uint32_t p0 = kout[r * h + t];
  out[r * 2 * h + t] = p0 + kout[(rows + r) * h + t];
  out[r * 2 * h + h + t] = p0 + kout[(2 * rows + r) * h + t];
}

// r[b][e] = c[b][e] + sum_j h[b][e + a_j - A] over the j with A <= e + a_j <=
// 2A - 2, for e < A: the remainder of the reduction modulo chi.  The
// product c is not read again (its upper half was read by the previous
// launch), so each thread clears c[b][e] and c[b][e + A] for the next
// product, which adds into a zeroed buffer.
__global__ void __launch_bounds__(256) fold_kernel(uint32_t* c, int64_t cstride, const uint32_t* h,
                                                   int64_t hstride, uint32_t* r, int64_t rstride,
                                                   const int32_t* offs, int k, int A) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (e >= A) return;
  uint32_t v = c[b * cstride + e];
  c[b * cstride + e] = 0u;
  if (e + A < cstride) c[b * cstride + e + A] = 0u;
  const uint32_t* hb = h + b * hstride;
  for (int j = 0; j < k; ++j) {
    const int d = e + offs[j];
    if (d >= A && d <= 2 * A - 2) v += hb[d - A];
  }
  r[b * rstride + e] = v;
}

struct JumpSetup {
  int32_t offs[kSdpMaxK];
  int32_t k;
  int32_t A;
  int32_t P;    // chunks
  int32_t P1e;  // major windows, counting the preset's
  int64_t L;    // chunk length
  int64_t ML;   // distance between major windows (P2 L)
  int64_t n;
  uint32_t* st;
  int32_t* d_offs;
  int64_t hlen;     // A + Gm words: the impulse response g[m] at A - 1 + m
  uint32_t* hbuf;
  SdpInstDev* insts;      // P chunk records
  SdpInstDev* ext_insts;  // P1e - 1 records extending major windows 1 .. P1e-1
  SdpInstDev* pre_insts;  // 2 records: ST up to 2A - 2, and the impulse response
};

// Device-side set-up: the offsets, the impulse-response preset (a single 1
// at position A - 1), the chunk records, the records that extend each major
// window by A - 1 values, and the two records of the first launch.
__global__ void __launch_bounds__(256) jump_setup_kernel(const JumpSetup s) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < s.k) s.d_offs[i] = s.offs[i];
  if (i < s.A) s.hbuf[i] = i == s.A - 1 ? 1u : 0u;
  if (i < 2) {
    SdpInstDev in{};
    in.st = i == 0 ? s.st : s.hbuf;
    in.n = i == 0 ? 2 * (int64_t)s.A - 1 : s.hlen;
    in.a = s.d_offs;
    in.k = s.k;
    s.pre_insts[i] = in;
  }
  if (i < s.P) {
    SdpInstDev in{};
    in.st = s.st + i * s.L;
    in.n = s.n - i * s.L < s.L ? s.n - i * s.L : s.L;
    in.a = s.d_offs;
    in.k = s.k;
    s.insts[i] = in;
  }
  if (i + 1 < s.P1e) {
    const int64_t pos = (i + 1) * s.ML;
    SdpInstDev in{};
    in.st = s.st + pos;
    in.n = s.n - pos < 2 * (int64_t)s.A - 1 ? s.n - pos : 2 * (int64_t)s.A - 1;
    in.a = s.d_offs;
    in.k = s.k;
    s.ext_insts[i] = in;
  }
}

// R1 = x^L0 mod chi.  For L0 < A the monomial.  Otherwise, from the
// impulse response g (g[m] = h[A - 1 + m], computed up to m = L0): reversing
// x^L0 = Q chi + R1 shows that the reversed quotient is the power series
// 1 / (1 - sum_j x^{a_j}) = sum_m g[m] x^m cut after degree L0 - A, and then
// R1[A - 1 - t] = g[M + t] - sum over a_j <= t of g[M + t - a_j], M = L0 - A + 1.
__global__ void __launch_bounds__(256) jump_start_kernel(uint32_t* R1, const uint32_t* h, const int32_t* offs,
                                                         int k, int A, int64_t L0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A) return;
  if (L0 < A) {
    R1[t] = t == L0 ? 1u : 0u;
    return;
  }
  const uint32_t* g = h + (A - 1);
  const int64_t M = L0 - A + 1;
  uint32_t v = g[M + t];
  for (int j = 0; j < k; ++j)
    if (offs[j] <= t) v -= g[M + t - offs[j]];
  R1[A - 1 - t] = v;
}

cudaError_t toeplitz(bool conv, const ToepArgs& a, int64_t batch, int sblocks, cudaStream_t st) {
  const dim3 grid((unsigned)((a.tout + kTB - 1) / kTB), (unsigned)sblocks, (unsigned)batch);
  if (conv)
    toeplitz_kernel<true><<<grid, kTT, 0, st>>>(a);
  else
    toeplitz_kernel<false><<<grid, kTT, 0, st>>>(a);
  return cudaGetLastError();
}

// split-range pieces for a product of `batch` items with `tblocks` output
// blocks each: as many as keep the launch within one wave of five blocks per
// SM, the most that are resident at once (registers and shared memory both
// allow five).
int split_count(int64_t S, int64_t tblocks, int64_t batch, int sms) {
  const int64_t most = (S + kSB - 1) / kSB;
  const int64_t want = (5 * (int64_t)sms) / (tblocks * batch);
  return (int)std::max<int64_t>(1, std::min(most, want));
}

}  // namespace
}  // namespace dpk

namespace dph {

namespace {
// Approximate device times, in microseconds, for the choice between the
// plain path and the jump path.  The plain kernel takes about 220 + W (k +
// 2) / 32 clocks per step of W = min(a_k, 1024) cells (measured at k = 32:
// 1299 clocks per step).  A Toeplitz product runs at about 14 T
// multiply-adds/s (measured); a product modulo chi costs about 1.7 a_1^2 of
// them in three launches, a window a_1^2, and the three launches of one
// product level on small batches about 35 us (measured: 16, 13 and 5 us).
double plain_us(int64_t cells, int32_t ak, int32_t k) {
  if (cells <= 0) return 0.0;
  const double W = std::min<int32_t>(ak, 1024);
  const double step_us = (220.0 + W * (k + 2) / 32.0) / 2.0e3;
  return std::ceil((double)cells / W) * step_us;
}

int ceil_log2(int64_t x) {
  int l = 0;
  while (((int64_t)1 << l) < x) ++l;
  return l;
}

// Chunks of length L = L0 2^s, P of them, in P1 groups of P2: the windows
// at multiples of P2 L ("major") come from the preset, the others from the
// nearest major window.  x^L0 mod chi is read off the impulse response,
// computed up to Gm >= L0 (a monomial when L0 < A).
struct JumpPlan {
  int P = 0;
  int P1 = 0, P2 = 0, P1e = 0;
  int64_t L = 0;
  int64_t L0 = 0;  // <= Gm: x^L0 mod chi comes from the impulse response
  int64_t Gm = 0;  // the impulse response is computed for m <= Gm (at least A - 1)
  int s = 0;
};

// The plan for about `chunks` chunks with the impulse response up to Gm;
// P = 0 when chunks of at least 2 A cells are impossible.
JumpPlan plan_for(int64_t n, int32_t A, int chunks, int64_t Gm) {
  JumpPlan p;
  if (chunks < 2 || A < 2) return p;
  const int64_t Lt = (n + chunks - 1) / chunks;
  if (Lt < 2 * (int64_t)A) return p;
  Gm = std::max<int64_t>(Gm, A - 1);
  int s = 0;
  while (((Lt + ((int64_t)1 << s) - 1) >> s) > Gm) ++s;
  p.s = s;
  p.Gm = Gm;
  p.L0 = (Lt + ((int64_t)1 << s) - 1) >> s;
  p.L = (int64_t)p.L0 << s;
  p.P = (int)((n + p.L - 1) / p.L);
  if (p.P < 2) {
    p.P = 0;
    return p;
  }
  p.P2 = std::max(1, (int)std::lround(std::sqrt((double)p.P)));
  p.P1 = (p.P + p.P2 - 1) / p.P2;
  p.P1e = (int)((n + (int64_t)p.P2 * p.L - 1) / ((int64_t)p.P2 * p.L));
  return p;
}

double jump_us(int64_t n, int32_t A, int32_t ak, int32_t k, const JumpPlan& p) {
  const double A2 = (double)A * A;
  const int products = p.s + (p.P2 - 1) + std::max(p.P1e - 2, 0);
  const int levels = p.s + ceil_log2(p.P2) + ceil_log2(std::max(p.P1e - 1, 1)) + 4;
  const double mads = products * 1.7 * A2 + (p.P - 1) * A2;
  return plain_us(std::min<int64_t>(p.L, n) - A, ak, k) + plain_us(A, ak, k) +
         std::max(plain_us(A, ak, k), plain_us(p.Gm + 1, ak, k)) + mads / 14.0e6 + levels * 35.0;
}

dp_status launch_records(const dpk::SdpInstDev* insts, int count, int32_t k, int32_t threads, int32_t ring_log2,
                         int32_t* status, cudaStream_t stream) {
  if (count <= 0) return DP_OK;
  dpk::SdpLaunchArgs args{};
  args.insts = insts;
  args.one.k = k;
  args.kfull = k == dpk::kSdpMaxKRegs;
  args.ninst = count;
  args.op = DP_OP_ADD_MOD32;
  args.threads = threads;
  args.ring_log2 = ring_log2;
  args.status = status;
  const cudaError_t e = dpk::launch_sdp(args, stream);
  return e == cudaSuccess ? DP_OK : fail_cuda(e, "sdp jump: launch of the chunk kernel");
}
// How far to compute the impulse response for `chunks` chunks: every
// doubling of its reach saves one squaring and costs a longer plain run.
int64_t jump_reach(int64_t n, int32_t A, int32_t ak, int32_t k, int chunks) {
  int64_t best_gm = A - 1;
  double best = -1.0;
  for (int64_t gm : {(int64_t)A - 1, 2 * (int64_t)A, 4 * (int64_t)A, 8 * (int64_t)A, 16 * (int64_t)A}) {
    const JumpPlan p = plan_for(n, A, chunks, gm);
    if (p.P < 2) return A - 1;
    const double t = jump_us(n, A, ak, k, p);
    if (best < 0.0 || t < best) {
      best = t;
      best_gm = gm;
    }
  }
  return best_gm;
}
}  // namespace

int sdp_jump_chunks(int64_t n, const int32_t* a, int32_t k, int sms) {
  const int32_t A = a[0], ak = a[k - 1];
  if (A < 2 || n < 8 * (int64_t)A) return 0;
  int32_t tl = 0, rl = 0;
  sdp_shape(A, ak, &tl, &rl);
  if (rl <= 0) return 0;  // the chunks need the window on chip
  double best = 0.8 * plain_us(n - A, ak, k);  // the jump must win clearly
  int bestP = 0;
  for (int c = 2; c <= sms; ++c) {
    const JumpPlan p = plan_for(n, A, c, jump_reach(n, A, ak, k, c));
    if (p.P < 2) break;
    const double t = jump_us(n, A, ak, k, p);
    if (t < best) {
      best = t;
      bestP = c;
    }
  }
  return bestP;
}

int sdp_jump_plan(int64_t n, const int32_t* a, int32_t k, int sms, int64_t out[8]) {
  const int chunks = sdp_jump_chunks(n, a, k, sms);
  for (int i = 0; i < 8; ++i) out[i] = 0;
  if (chunks < 2) return 0;
  const JumpPlan p = plan_for(n, a[0], chunks, jump_reach(n, a[0], a[k - 1], k, chunks));
  out[0] = p.P;
  out[1] = p.L;
  out[2] = p.L0;
  out[3] = p.s;
  out[4] = p.Gm;
  out[5] = p.P2;
  out[6] = p.P1e;
  out[7] = chunks;
  return chunks;
}

dp_status sdp_add_jump(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, int chunks, int32_t* status,
                       cudaStream_t st) {
  using dpk::ToepArgs;
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  const int32_t A = a[0];
  if (A < 2) return fail(DP_EINVAL, "sdp jump: a_1 = %d, the table is constant", A);
  const JumpPlan pl = plan_for(n, A, chunks, jump_reach(n, A, a[k - 1], k, chunks));
  if (pl.P < 2)
    return fail(DP_EINVAL, "sdp jump: %d chunks of at least %d cells do not fit n = %lld", chunks, 2 * A,
                (long long)n);
  int32_t threads = 0, ring_log2 = 0;
  sdp_shape(A, a[k - 1], &threads, &ring_log2);
  if (ring_log2 <= 0) return fail(DP_EINVAL, "sdp jump: window a_1 = %d too wide for the on-chip ring", A);
  const int P = pl.P, P2 = pl.P2, P1e = pl.P1e;
  const int64_t ML = (int64_t)P2 * pl.L;
  // largest batch of a tree level: R_2 .. R_P2 and Q_2 .. Q_{P1e-1}
  auto widest = [](int64_t qmax) {
    int64_t w = 1;
    for (int64_t m = 1; m + 1 <= qmax; m *= 2) w = std::max<int64_t>(w, std::min<int64_t>(2 * m, qmax) - m);
    return w;
  };
  const int64_t nb = std::max(widest(P2), widest(P1e - 1));
  const int64_t PS = 2 * (int64_t)A;  // product stride (2A - 1 coefficients)
  const int64_t HS = A;               // stride of the top-down multiples (A - 1 of them)
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += al(std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_offs = take((size_t)k * 4);
  const int64_t hlen = A + pl.Gm;  // the impulse response g[m] at A - 1 + m, m <= Gm
  const size_t o_h = take((size_t)hlen * 4);
  const size_t o_R = take((size_t)(P2 + 1) * A * 4);                  // R_0 .. R_P2 (R_0 unused)
  const size_t o_Q = take((size_t)std::max(P1e, 2) * A * 4);          // Q_0 .. Q_{P1e-1} (Q_0 unused)
  const size_t o_prod = take((size_t)nb * PS * 4);
  const size_t o_hf = take((size_t)nb * HS * 4);
  const int64_t nwin = std::max<int64_t>((int64_t)P1e * P2, 2);     // window scratch rows
  const size_t o_win = take((size_t)nwin * A * 4);
  // the windows' middle products by one transposed Karatsuba step (A even,
  // and each half still a full output block of the Toeplitz kernel)
  const int64_t kh = A / 2;
  const bool kara = A % 2 == 0 && kh >= dpk::kTB;
  const int64_t knlo = std::max<int64_t>({(int64_t)P1e, (int64_t)P2, 1});
  const size_t o_ku = take(kara ? (size_t)3 * knlo * kh * 4 : 0);
  const size_t o_kz = take(kara ? (size_t)3 * P1e * 2 * kh * 4 : 0);
  const size_t o_kout = take(kara ? (size_t)3 * nwin * kh * 4 : 0);
  const size_t o_insts = take((size_t)P * sizeof(dpk::SdpInstDev));
  const size_t o_ext = take((size_t)std::max(P1e - 1, 1) * sizeof(dpk::SdpInstDev));
  const size_t o_pre = take(2 * sizeof(dpk::SdpInstDev));
  uint8_t* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), off, st);
  if (e != cudaSuccess) return fail_cuda(e, "sdp jump: workspace");
  int32_t* d_offs = reinterpret_cast<int32_t*>(ws + o_offs);
  uint32_t* hbuf = reinterpret_cast<uint32_t*>(ws + o_h);
  uint32_t* R = reinterpret_cast<uint32_t*>(ws + o_R);
  uint32_t* Q = reinterpret_cast<uint32_t*>(ws + o_Q);
  uint32_t* prod = reinterpret_cast<uint32_t*>(ws + o_prod);
  uint32_t* hf = reinterpret_cast<uint32_t*>(ws + o_hf);
  uint32_t* win = reinterpret_cast<uint32_t*>(ws + o_win);
  uint32_t* ku = reinterpret_cast<uint32_t*>(ws + o_ku);
  uint32_t* kz = reinterpret_cast<uint32_t*>(ws + o_kz);
  uint32_t* kout = reinterpret_cast<uint32_t*>(ws + o_kout);
  auto* insts = reinterpret_cast<dpk::SdpInstDev*>(ws + o_insts);
  auto* ext_insts = reinterpret_cast<dpk::SdpInstDev*>(ws + o_ext);
  auto* pre_insts = reinterpret_cast<dpk::SdpInstDev*>(ws + o_pre);
  const uint32_t* g = hbuf + (A - 1);  // g[m] = hbuf[A - 1 + m]

  const bool prof = profiling();
  if (prof) profile_mark(1, st, false);
  auto done = [&](dp_status r) {
    if (prof) profile_mark(1, st, true);
    const cudaError_t fe = cudaFreeAsync(ws, st);
    if (r == DP_OK && fe != cudaSuccess) return fail_cuda(fe, "sdp jump: workspace release");
    return r;
  };

  dpk::JumpSetup su{};
  for (int j = 0; j < k; ++j) su.offs[j] = a[j];
  su.k = k;
  su.A = A;
  su.P = P;
  su.P1e = P1e;
  su.L = pl.L;
  su.ML = ML;
  su.n = n;
  su.st = ST;
  su.d_offs = d_offs;
  su.hbuf = hbuf;
  su.hlen = hlen;
  su.insts = insts;
  su.ext_insts = ext_insts;
  su.pre_insts = pre_insts;
  const int64_t su_n = std::max<int64_t>({(int64_t)k, (int64_t)A, (int64_t)P, (int64_t)P1e, 2});
  dpk::jump_setup_kernel<<<(unsigned)((su_n + 255) / 256), 256, 0, st>>>(su);
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaMemsetAsync(prod, 0, (size_t)nb * PS * 4, st)) != cudaSuccess)
    return done(fail_cuda(e, "sdp jump: set-up"));
  // 1. ST[A .. 2A - 2] and 2. the impulse response g[0 .. Gm], side by side;
  // then R_1 starts as x^L0 mod chi
  if ((rc = launch_records(pre_insts, 2, k, threads, ring_log2, status, st)) != DP_OK) return done(rc);
  dpk::jump_start_kernel<<<(unsigned)((A + 255) / 256), 256, 0, st>>>(R + A, hbuf, d_offs, k, A, pl.L0);
  if ((e = cudaGetLastError()) != cudaSuccess) return done(fail_cuda(e, "sdp jump: start"));

  // dst + i A = (x + i xs) (y + i ys) mod chi, for i < cnt
  auto mulmod = [&](const uint32_t* x, int64_t xs, const uint32_t* y, int64_t ys, uint32_t* dst, int64_t cnt) {
    // prod is all zero here (set-up, then every fold clears what it read);
    // the product launch clears hf for the reduction that follows it
    const int64_t tb_prod = (2 * (int64_t)A - 1 + dpk::kTB - 1) / dpk::kTB;
    const int sp = dpk::split_count(A, tb_prod, cnt, ds->sms);
    ToepArgs ta{};
    ta.zero = hf;
    ta.zero_len = cnt * HS;
    ta.u = x;
    ta.ustride = xs;
    ta.S = A;
    ta.z = y;
    ta.zstride = ys;
    ta.zlen = A;
    ta.zlim = INT64_MAX;
    ta.out = prod;
    ta.ostride = PS;
    ta.tout = 2 * (int64_t)A - 1;
    ta.olim = INT64_MAX;
    ta.nlo = cnt;
    if ((e = dpk::toeplitz(true, ta, cnt, sp, st)) != cudaSuccess) return e;
    const int64_t tb_h = (A - 1 + dpk::kTB - 1) / dpk::kTB;
    const int sh = dpk::split_count(A - 1, tb_h, cnt, ds->sms);
    ToepArgs th{};
    th.u = g;
    th.S = A - 1;
    th.z = prod;
    th.zstride = PS;
    th.zlen = 2 * (int64_t)A - 1;
    th.zoff = A;
    th.zlim = INT64_MAX;
    th.out = hf;
    th.ostride = HS;
    th.tout = A - 1;
    th.olim = INT64_MAX;
    th.nlo = cnt;
    if ((e = dpk::toeplitz(false, th, cnt, sh, st)) != cudaSuccess) return e;
    dpk::fold_kernel<<<dim3((unsigned)((A + 255) / 256), (unsigned)cnt), 256, 0, st>>>(prod, PS, hf, HS, dst, A,
                                                                                       d_offs, k, A);
    return cudaGetLastError();
  };
  // X[q] = X[m] X[q - m] for q in (m, 2m], m = 1, 2, 4, ..., up to X[qmax]
  auto tree = [&](uint32_t* X, int64_t qmax) {
    for (int64_t m = 1; m + 1 <= qmax; m *= 2) {
      const int64_t cnt = std::min<int64_t>(2 * m, qmax) - m;
      if ((e = mulmod(X + m * A, 0, X + A, A, X + (m + 1) * A, cnt)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // Hankel products into the window scratch (rows win + (hi nlo + lo) A):
  // row (hi, lo), t < A = sum_s U_(hi, lo)[s] ST[hi zs_hi + s + t]
  auto windows = [&](const uint32_t* U, int64_t us, int64_t us_hi, int64_t zs_hi, int64_t nhi, int64_t nlo) {
    if (nhi * nlo <= 0) return cudaSuccess;
    if (kara && us_hi == 0) {
      // the three half-size products as one launch of 3 rows items; the
      // split count divides the pieces evenly
      const int64_t rows = nhi * nlo;
      const int64_t pieces = (kh + dpk::kSB - 1) / dpk::kSB;
      const int64_t want = std::max<int64_t>(1, (5 * (int64_t)ds->sms) / (3 * rows));
      int64_t sp = 1;
      for (int64_t d = 1; d <= pieces && d <= want; ++d)
        if (pieces % d == 0) sp = d;
      if (sp > 1 && (e = cudaMemsetAsync(kout, 0, (size_t)3 * rows * kh * 4, st)) != cudaSuccess) return e;
      dpk::kara_prep_kernel<<<dim3((unsigned)((2 * kh + 255) / 256), (unsigned)std::max(nlo, nhi)), 256, 0, st>>>(
          U, us, nlo, ST, zs_hi, 2 * (int64_t)A - 1, n, nhi, kh, ku, kz);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      ToepArgs tk{};
      tk.u = ku;
      tk.ustride = kh;
      tk.ustride_v = nlo * kh;
      tk.S = kh;
      tk.z = kz;
      tk.zstride_hi = 2 * kh;
      tk.zstride_v = nhi * 2 * kh;
      tk.zlen = 2 * kh - 1;
      tk.zlim = INT64_MAX;
      tk.out = kout;
      tk.ostride = kh;
      tk.ostride_hi = nlo * kh;
      tk.ostride_v = rows * kh;
      tk.tout = kh;
      tk.olim = INT64_MAX;
      tk.nlo = nlo;
      tk.nvi = rows;
      if ((e = dpk::toeplitz(false, tk, 3 * rows, (int)sp, st)) != cudaSuccess) return e;
      dpk::kara_combine_kernel<<<dim3((unsigned)((kh + 255) / 256), (unsigned)rows), 256, 0, st>>>(win, kout, rows,
                                                                                                   kh);
      return cudaGetLastError();
    }
    const int64_t tb = (A + dpk::kTB - 1) / dpk::kTB;
    const int sp = dpk::split_count(A, tb, nhi * nlo, ds->sms);
    if ((e = cudaMemsetAsync(win, 0, (size_t)nhi * nlo * A * 4, st)) != cudaSuccess) return e;
    ToepArgs tw{};
    tw.u = U;
    tw.ustride = us;
    tw.ustride_hi = us_hi;
    tw.S = A;
    tw.z = ST;
    tw.zstride_hi = zs_hi;
    tw.zlen = 2 * (int64_t)A - 1;
    tw.zlim = n;
    tw.out = win;
    tw.ostride = A;
    tw.ostride_hi = nlo * (int64_t)A;
    tw.tout = A;
    tw.olim = INT64_MAX;
    tw.nlo = nlo;
    // with one piece the kernel stores instead of adding: same result on the zeroed rows
    return dpk::toeplitz(false, tw, nhi * nlo, sp, st);
  };
  // copies `rows` scratch rows, from row r0, to ST + pos0 + r * pitch,
  // clipped at n
  auto place = [&](int64_t r0, int64_t pos0, int64_t pitch, int64_t rows) {
    int64_t full = 0;
    while (full < rows && pos0 + full * pitch + A <= n) ++full;
    if (full > 0 &&
        (e = cudaMemcpy2DAsync(ST + pos0, (size_t)pitch * 4, win + r0 * A, (size_t)A * 4, (size_t)A * 4, (size_t)full,
                               cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
    const int64_t pos = pos0 + full * pitch;
    if (full < rows && pos < n &&
        (e = cudaMemcpyAsync(ST + pos, win + (r0 + full) * A, (size_t)(n - pos) * 4, cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
      return e;
    return cudaSuccess;
  };

  // 3. R_1 = (x^L0)^(2^s); R_2 .. R_P2; Q_i = R_P2^i for i < P1e
  for (int i = 0; i < pl.s; ++i)
    if ((e = mulmod(R + A, 0, R + A, 0, R + A, 1)) != cudaSuccess) return done(fail_cuda(e, "sdp jump: squaring"));
  if ((e = tree(R, P2)) != cudaSuccess) return done(fail_cuda(e, "sdp jump: product tree"));
  if (P1e > 1) {
    if ((e = cudaMemcpyAsync(Q + A, R + (int64_t)P2 * A, (size_t)A * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
        (e = tree(Q, P1e - 1)) != cudaSuccess)
      return done(fail_cuda(e, "sdp jump: product tree of the major windows"));
  }
  // 4. major windows at i P2 L (1 <= i < P1e), from the preset; each
  // extended by A - 1 values; then the windows between them, from the
  // nearest major window: ST[(i P2 + j) L + t] = sum_s R_j[s] ST[i P2 L + s + t]
  if ((e = windows(Q + A, A, 0, 0, 1, P1e - 1)) != cudaSuccess || (e = place(0, ML, ML, P1e - 1)) != cudaSuccess)
    return done(fail_cuda(e, "sdp jump: major windows"));
  if ((rc = launch_records(ext_insts, P1e - 1, k, threads, ring_log2, status, st)) != DP_OK) return done(rc);
  if (P2 > 1) {
    if ((e = windows(R + A, A, 0, ML, P1e, P2 - 1)) != cudaSuccess) return done(fail_cuda(e, "sdp jump: windows"));
    for (int64_t i = 0; i < P1e; ++i)
      if ((e = place(i * (P2 - 1), i * ML + pl.L, pl.L, P2 - 1)) != cudaSuccess)
        return done(fail_cuda(e, "sdp jump: windows"));
  }
  // 5. the chunks, side by side
  if ((rc = launch_records(insts, P, k, threads, ring_log2, status, st)) != DP_OK) return done(rc);
  return done(DP_OK);
}

}  // namespace dph
