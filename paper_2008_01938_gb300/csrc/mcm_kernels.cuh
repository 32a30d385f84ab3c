// mcm_kernels.cuh -- launch-side declarations of the MCM kernels.
//
// Problem (paper Section IV-A, Eq. (2); recurrence from Cormen et al., which
// the paper cites): for i < j
//     m[i][j] = min_{i <= k < j} m[i][k] + m[k+1][j] + p[i] * p[k+1] * p[j+1]
// and s[i][j] = the smallest minimising k.  The interval-DP instances add a
// per-cell weight w[i][j] to every candidate of cell (i, j) (Eq. (2) with a
// more general f), which they do once, when the cell's minimum is final.
//
// GPU decomposition.  The n x n table is cut into 32 x 32 tiles (I, J), J >= I.
// Tile (I, J) lies on tile-diagonal D = J - I.  For a cell of tile (I, J) the
// splits k fall into
//   * external segments K = I+1 .. J-1 (k in [32K, 32K+32)): the row panel is
//     tile (I, K), the column panel rows 32K+1 .. 32K+32 of tile column J;
//     segment K becomes computable once tile-diagonal r(K) = max(K-I, J-K) is
//     complete, so most of a tile's work is ready long before its neighbours;
//   * the boundary split k = 32I + 31 (needs row 32(I+1) of tile (I+1, J));
//   * the in-tile splits k in [i, 32I+30] and [32J, j-1], which depend on the
//     tile's own cells and are resolved by a wavefront over the tile's 63
//     anti-diagonals (the paper's diagonal computation order, Figs. 5-7,
//     applied inside one tile).
// Work items ("tasks") are (tile, range of r levels).  A bulk task reduces a
// group of external segments and merges its (value, k) minima into the tile's
// partial accumulator with 64-bit atomicMin (deterministic: the packed
// comparison is lexicographic on (value, k)).  The finisher task of a tile
// waits for those, reduces the last segments, adds the boundary split, runs
// the in-tile wavefront, writes the outputs and publishes the tile's flag.
// Tasks are popped from one queue in order of the tile-diagonal at which they
// become ready (finishers of diagonal D after every task they wait for), so a
// block only ever waits for tasks popped before its own: the queue makes
// progress whatever the number of resident blocks.
//
// Cost encodings (exact integer arithmetic throughout):
//   int32 costs: every candidate is at most (n-1)*max(p)^3 =: bound < 2^31
//     (interval DP: (n-1)*(max(p)^3 + max(w))).
//     The packed row-panel entry is (m << S) | (k mod 2^S) and the column
//     panel entry m << S, with S the largest value <= 5 such that
//     (bound + 1) << S <= 2^32.  Then  A + B + (p_i p_j1) (p_k1 << S)
//     = (candidate << S) | (k mod 2^S), so an unsigned min over a chunk of
//     2^min(S,5) aligned splits yields the minimum and its smallest k at once.
//   int64 costs (bound < 2^47): entries are (m << 16) | k and m << 16, so one
//     unsigned 64-bit min yields (value, smallest k) directly.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dpk {

constexpr int kTile = 32;
constexpr int kGroupThreads = 128;                     // one compute group
constexpr int kComputeThreads = 2 * kGroupThreads;     // two groups
constexpr int kMcmThreads = kComputeThreads + 32;      // + producer warp
constexpr int kStages = 2;                             // bulk-copy stages per group

// Work split of a tile on tile-diagonal D >= 2: its external levels
// r = (D+1)/2 .. D-1 go to bulk tasks of kLevelsPerPart levels each, except
// the last level, which the finisher keeps; a tile with fewer than
// kMinBulkLevels bulk levels is not split at all.
constexpr int kLevelsPerPart = 8;
constexpr int kMinBulkLevels = 2;
// int32 plans cut a tile's bulk levels from the top: the part that ends at
// the last bulk level D-2 -- the part the finisher is likeliest to wait for,
// since it becomes ready only when tile-diagonal D-2 is complete -- holds
// kLastPartLevels levels, and kLevelsPerPart-level parts cover the levels
// below it.
constexpr int kLastPartLevels = 4;
// Queue position of the other int32 parts: not before they become ready, and
// not earlier than kDeferBuckets tile-diagonals before their finisher. Work
// that is not needed soon then waits behind the tasks of the chain in the
// middle diagonals (where blocks are scarce) and fills the blocks that the
// last diagonals leave idle.
constexpr int kDeferBuckets = 3;

struct McmInstDev {
  const int32_t* p;   // dims p[0..n] (set by the prologue)
  void* m;            // output cost table (set by the prologue)
  int16_t* s;         // output split table (set by the prologue)
  int32_t n;          // matrices
  int32_t nt;         // tiles per side
  int32_t shift;      // packing shift S (set by the prologue)
  int32_t pad_;
  int64_t tile_base;  // first index of this chain's tiles in the per-tile arrays
  int64_t pp_base;    // offset of this chain's padded dims in McmLaunchArgs::pp
  int64_t pk_base;    // offset of this chain's shifted dims in McmLaunchArgs::pk
  const void* w;      // interval DP: per-cell weight table, like m (set by the prologue)
  unsigned long long wmax;  // interval DP: largest weight above the diagonal (weight pass)
};

// kind 0: finisher of tile (I, J) for r levels [r_lo, r_hi], waits for
// `nparts` bulk tasks.  kind 1: bulk task for r levels [r_lo, r_hi].
struct McmTask {
  int32_t inst;
  int16_t I, J;
  int16_t r_lo, r_hi;
  int16_t kind, nparts;
};

struct McmLaunchArgs {
  McmInstDev* insts;
  const McmTask* tasks;
  int32_t ninst;
  int32_t ntasks;
  void* af;                      // packed row panels, tile-major, k-major inside a tile
  void* bf;                      // packed column panels (rows shifted by one), tile-major
  int32_t* flags;                // per tile: 1 once the tile is final
  int32_t* counters;             // per tile: bulk tasks merged so far
  const int32_t* accslot;        // per tile: partial-accumulator slot or -1
  unsigned long long* acc;       // per slot: 32*32 packed (value, k) minima
  int32_t* pp;                   // padded dims
  uint32_t* pk;                  // pk[x] = p[x+1] << S
  int32_t* queue;                // task counter
  int32_t* status;               // device status word
  long long spin_limit;          // clock cycles a wait may take before DP_ETIMEOUT
  int32_t drop_task;             // fault injection: this queue entry is popped but never run (-1: none)
  int32_t pad_;
  const int32_t* p_all;          // prologue inputs
  const int64_t* p_off;          // nullptr: single chain at p_all
  const int64_t* tab_off;        // nullptr: single chain at m_all / s_all
  void* m_all;
  int16_t* s_all;
  // Interval DP (nullptr: plain MCM): per-cell weights laid out like m_all
  // (chain b's n x n table at offset tab_off[b]); w[i][j], i < j, is added to
  // the minimum of cell (i, j), and p may then hold zeros.
  const void* w_all;
};

size_t mcm_smem_bytes(bool i64);
cudaError_t mcm_configure(bool i64);
cudaError_t mcm_occupancy(bool i64, int* blocks_per_sm);
// With a.w_all set, the prologue and main kernel are the interval-DP
// instances, and launch_mcm_weight_max must run first (it fills
// McmInstDev::wmax, from which the prologue derives the cost bound).  The
// interval-DP instances exist for int32 costs only: the int64 one faulted on
// the GPU for a reason that was not found, so it is not built, and these
// calls return cudaErrorNotSupported for i64 with weights.
cudaError_t launch_mcm_weight_max(const McmLaunchArgs& a, bool i64, int sms, cudaStream_t st);
cudaError_t launch_mcm_prologue(const McmLaunchArgs& a, bool i64, cudaStream_t st);
cudaError_t launch_mcm_main(const McmLaunchArgs& a, bool i64, int grid, cudaStream_t st);
// Loads the prologue, main and split-pass kernels into the current context
// (with lazy module loading a kernel is otherwise loaded at its first launch).
cudaError_t mcm_preload(bool i64);

}  // namespace dpk
