/*
 * dpgpu.h -- C ABI of the GB300 (sm_103a) solvers for the two dynamic programs
 * of Matsumae & Miyazaki, "Solving Dynamic Programming Problem by Pipeline
 * Implementation on GPU":
 *
 *   - the matrix-chain multiplication (MCM) table of Section IV-A (the paper
 *     takes the problem from Cormen et al.; its Eq. (2) writes each cell as a
 *     min over splits of f(left, right)):
 *         m[i][j] = min_{i <= k < j}  m[i][k] + m[k+1][j] + p[i]*p[k+1]*p[j+1]
 *     with the split table s[i][j] = the smallest minimising k;
 *   - the simplified DP problem (S-DP) of Definition 1, Eq. (1):
 *         ST[i] = (x)_{1 <= j <= k} ST[i - a_j],  a_1 > ... > a_k > 0,
 *     ST[0 .. a_1-1] preset, (x) = min or + modulo 2^32.
 *
 * Conventions shared by every entry point
 *   - Indices are 0-based.  The chain is A_0..A_{n-1}; A_i is p[i] x p[i+1].
 *   - MCM tables are n*n row-major (leading dimension n).  On and below the
 *     diagonal m = 0 and s = -1.
 *   - Pointers named *_dev or documented as "device" are CUDA device pointers
 *     owned by the caller; the library never frees them.  Host pointers are
 *     read before the call returns unless stated otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous unless stated.
 *   - Return value: errors the host can see at call time (bad arguments,
 *     allocation or launch failure).  Errors found on the device (invalid
 *     dims, overflow, a bounded wait that timed out) are written to
 *     `status_dev` (an int32 device word, nullable; the library keeps its own
 *     per-device word when it is NULL) and read back by dp_sync_status().
 *   - No C++ exception crosses this boundary.  dp_last_error() gives a
 *     thread-local message for the last failing call.
 *   - Results are exact: integer arithmetic only, bit-identical to a
 *     sequential solve.
 */
#ifndef DPGPU_H
#define DPGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DP_OK = 0,
  DP_EINVAL = 1,     /* invalid argument (n, dims < 1, offsets not strictly decreasing, ...) */
  DP_ENOMEM = 2,     /* device or host allocation failed */
  DP_ECUDA = 3,      /* a CUDA runtime call failed */
  DP_EOVERFLOW = 4,  /* the cost bound does not fit the chosen cost type */
  DP_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
  DP_EBUSY = 6,      /* serving: request not admissible right now */
  DP_EPENDING = 7    /* serving: result not ready yet */
} dp_status;

typedef enum { DP_COST_I32 = 0, DP_COST_I64 = 1 } dp_cost;
typedef enum { DP_OP_MIN = 0, DP_OP_ADD_MOD32 = 1 } dp_op;

/* ------------------------------------------------------------------------- */
/* Library information and status                                             */
/* ------------------------------------------------------------------------- */

/* Thread-local text of the last error reported by this thread (never NULL). */
const char *dp_last_error(void);

/* Version string of the library build. */
const char *dp_version(void);

/* Waits for `stream`, then reads and clears the device status word
 * (`status_dev`, or the library's own word for the current device when NULL).
 * Returns that status (DP_OK when the device saw no error), or DP_ECUDA if
 * the stream itself failed. */
dp_status dp_sync_status(void *stream, int32_t *status_dev);

/* Kernel timing.  Between dp_profile_begin() and dp_profile_end(), every
 * launch of a solver kernel (not the small set-up kernels) made by this
 * process is bracketed by two CUDA events recorded on the launching stream.
 * dp_profile_end() waits for them and returns the summed device time in
 * milliseconds and the number of launches for the MCM kernel (mcm_*) and the
 * S-DP kernel (sdp_*).  Do not profile while capturing a CUDA graph. */
dp_status dp_profile_begin(void);
dp_status dp_profile_end(double *mcm_ms, int64_t *mcm_launches, double *sdp_ms, int64_t *sdp_launches);

/* Measured integer throughput of the current device, the denominator of the
 * MCM kernel's INT32-ALU roofline (the paper has no counterpart: it is a
 * measurement utility).  Every SM is kept full of independent dependency
 * chains of one instruction kind; SM clock cycles are counted around the loop
 * on the device, so the lane figures do not depend on the clock.  Fills
 * out[0..8] (host doubles, nout >= 9, else DP_EINVAL), and out[9] when
 * nout >= 10:
 *   out[0]  three-input integer add (ALU pipe), lanes per clock per SM
 *   out[1]  integer multiply-add (FMA pipe), lanes per clock per SM
 *   out[2]  three-way unsigned minimum (ALU pipe), lanes per clock per SM
 *   out[3]  two-input integer add, lanes per clock per SM: the compiler
 *           spreads these over both integer pipes, so this is the combined
 *           INT32 rate (the roofline's peak)
 *   out[4]  three-input adds and multiply-adds interleaved 1:1, lanes per
 *           clock per SM (the solver's two kinds of split-evaluation
 *           instruction)
 *   out[5]  the MCM solver's bulk loop (packed keys on a shared-memory panel,
 *           nothing waiting), split evaluations per clock per SM
 *   out[6]  SM count of the device (cudaDevAttrMultiProcessorCount)
 *   out[7]  SM clock seen during the probes, MHz (cycles / event time)
 *   out[8]  the device's reported maximum SM clock, MHz
 *   out[9]  the int64 solver's bulk loop (64-bit packed keys, two resident
 *           blocks per SM as in the int64 solver), split evaluations per
 *           clock per SM
 * Runs twelve short launches (fourteen with out[9]) on `stream`, about 30 ms
 * in all, and waits for them; a 16-byte stream-ordered allocation holds the
 * cycle counts. */
dp_status dp_measure_int32_rates(double *out, int32_t nout, void *stream);

/* ------------------------------------------------------------------------- */
/* MCM (Section IV-A, Eq. (2))                                                */
/* ------------------------------------------------------------------------- */

/* Solves one chain.
 *   p       device int32[n+1], every p[t] >= 1 (checked on the device:
 *           DP_EINVAL in *status_dev otherwise).
 *   n       number of matrices, 1 <= n <= 32767 (s is int16).
 *   ct      DP_COST_I32: m is int32[n*n]; needs (n-1)*max(p)^3 < 2^31.
 *           DP_COST_I64: m is int64[n*n]; needs (n-1)*max(p)^3 < 2^47.
 *           (n-1)*max(p)^3 bounds every candidate cost m[i][k]+m[k+1][j]+w;
 *           exceeding it gives DP_EOVERFLOW in *status_dev.)
 *   m, s    device outputs, n*n each, row-major (ld = n); fully written.
 * Scratch (about 2*n^2 cost elements plus per-tile state) is allocated
 * stream-ordered from the current device's memory pool and released
 * stream-ordered before the call returns. */
dp_status mcm_solve(const int32_t *p, int32_t n, dp_cost ct, void *m, int16_t *s,
                    int32_t *status_dev, void *stream);

/* Interval DP with a user weight: the triangular-table DP of Section IV with
 * Eq. (2)'s f taken more generally (the paper presents MCM as one instance of
 * its technique).  For i < j
 *     m[i][j] = min_{i <= k < j} m[i][k] + m[k+1][j] + p[i]*p[k+1]*p[j+1] + w[i][j]
 * and s[i][j] = the smallest minimising k; m = 0 and s = -1 on and below the
 * diagonal.  w = 0 gives mcm_solve; p = 0 gives the split form of Knuth's
 * optimal binary search tree (cells = gaps 0..n-1 between keys, w[i][j] = the
 * weight of keys i+1..j and gaps i..j, root key = s + 1) and optimal merging.
 *   p       device int32[n+1], 0 <= p[t] < 65536 (DP_EINVAL / DP_EOVERFLOW in
 *           *status_dev otherwise).
 *   w       device int32[n*n], row-major (ld = n), the same layout as m;
 *           only entries with i < j are read, each >= 0 (DP_EINVAL in
 *           *status_dev otherwise).
 *   ct      DP_COST_I32 only (m int32, (n-1)*(max(p)^3 + max(w)) < 2^31,
 *           DP_EOVERFLOW in *status_dev otherwise); DP_COST_I64 returns
 *           DP_EINVAL.
 *   n, m, s, status_dev, stream: as for mcm_solve.
 * A device pass over w (one extra launch) finds max(w) before the solve.
 * NULL p, w, m or s return DP_EINVAL. */
dp_status interval_dp_solve(const int32_t *p, const void *w, int32_t n, dp_cost ct, void *m, int16_t *s,
                            int32_t *status_dev, void *stream);

/* mcm_solve for int32 costs that allocates no memory.  The paper has no
 * counterpart: it exists for callers that cannot allocate when they solve --
 * a process whose free device memory belongs to its own allocator (where a
 * stream-ordered allocation would fail or grow the pool), or a
 * latency-critical loop that must not enter an allocator.
 *   p, n, m, s  as for mcm_solve with ct = DP_COST_I32; m is int32[n*n].
 *   n           1 <= n <= 1024: the scratch is a fixed file-scope device
 *               array of 8,691,968 bytes per device; a larger n returns
 *               DP_EINVAL without touching the device.
 *   status_dev  required (NULL is DP_EINVAL): caller-owned device int32 that
 *               is zero on entry; device-side errors land there, read them
 *               with dp_sync_status(stream, status_dev).
 * The first call on a device does the set-up for that device (loads the
 * module that holds the scratch, takes the scratch's address on that device
 * with cudaGetSymbolAddress, sets kernel attributes); make it before any
 * stream capture.  Every call then starts with a set-up kernel that writes
 * all of the scratch a solve reads before writing it: the tile flags, bulk
 * counters and queue counter, which must start at zero, the accumulators
 * (all ones) and the work queue.  So the scratch needs no initial contents
 * and a failed call leaves nothing that the next one depends on.
 * One device has one scratch: calls that overlap in time on the same device
 * (two streams, or two host threads whose calls are not ordered on one
 * stream) race on it and corrupt each other's results. */
dp_status mcm_solve_noalloc(const int32_t *p, int32_t n, int32_t *m, int16_t *s, int32_t *status_dev,
                            void *stream);

/* The optimal parenthesisation encoded by a split table (the textbook's
 * PRINT-OPTIMAL-PARENS, which the paper's MCM recurrence follows), on the
 * device.
 *   s       device int16[n*n] as written by mcm_solve (split of (i, j) at
 *           s[i*n + j]).
 *   steps   device int32[3*(n-1)], filled with the n-1 products in post-order:
 *           entry t is (i, k, j) = multiply the product of matrices i..k by
 *           that of k+1..j; both operands are single matrices or results of
 *           earlier entries, and the last entry is (0, k, n-1).
 * Nothing is written for n = 1 (steps may then be NULL).  The tree is
 * expanded one level per pass of one block, so the time grows with the tree's
 * depth (at most n-1 levels).  A split outside [i, j) is reported as
 * DP_EINVAL in *status_dev (NULL: the library's status word, read by
 * dp_sync_status).  A small stream-ordered scratch allocation holds the
 * levels; NULL s or steps (n > 1) or n outside [1, 32767] return DP_EINVAL. */
dp_status mcm_traceback(const int16_t *s, int32_t n, int32_t *steps, int32_t *status_dev, void *stream);

/* Same computation with HOST buffers (p: n+1 int32, m: n*n cost elements,
 * s: n*n int16, row-major), waiting for completion before it returns.
 * Page-locked m and s (cudaHostAlloc, cudaHostRegister without the read-only
 * flag) that the current device can address, each inside one allocation, are
 * written by the kernel in place: the tables reach host memory while the
 * solve runs and no copy follows it.  A page-locked p is read in place.  Any
 * other buffer is staged through device memory with a copy before (p) or
 * after (m, s) the solve.  The caller owns all three buffers; their sizes are
 * not checked beyond the allocation test above. */
dp_status mcm_solve_host(const int32_t *p_host, int32_t n, dp_cost ct, void *m_host,
                         int16_t *s_host, void *stream);

/* Batched MCM: many chains of uneven length in one persistent launch.
 * mcm_plan_create reads n_host[0..batch-1] (host), validates the sizes,
 * builds the diagonal-ordered work queue and allocates the plan's device
 * workspace.  The plan is bound to the current device and to ct. */
dp_status mcm_plan_create(int32_t batch, const int32_t *n_host, dp_cost ct, void **plan);

/* Runs a plan.  All arrays are device pointers:
 *   p_all   concatenated dims; chain b owns p_all[p_off[b] .. p_off[b]+n_b].
 *   p_off   int64[batch]: start of chain b in p_all.
 *   tab_off int64[batch]: element offset of chain b's n_b*n_b table inside
 *           m_all (cost type of the plan) and s_all (int16).
 * Enqueues only memsets and one kernel launch on `stream` (no host sync, no
 * allocation), so it may be captured into a CUDA graph.  One plan must not
 * run on two streams at once (its workspace is shared). */
dp_status mcm_solve_batched(void *plan, const int32_t *p_all, const int64_t *p_off,
                            const int64_t *tab_off, void *m_all, int16_t *s_all,
                            int32_t *status_dev, void *stream);

/* Autotuner for a plan: runs the plan on the caller's own buffers (as for
 * mcm_solve_batched) under each candidate configuration -- external levels
 * per bulk task in {4, 8, 16} and 1 .. (occupancy limit) resident blocks per
 * SM -- twice each, timed with events on `stream`, and keeps the fastest.
 * Every configuration computes the same tables (the arithmetic is exact), and
 * the call ends with one more solve under the chosen configuration, so the
 * tables hold the solution on return.  It synchronises the stream, may
 * reallocate the plan's workspace, and must not be called while capturing a
 * graph; capture mcm_solve_batched afterwards. */
dp_status mcm_plan_autotune(void *plan, const int32_t *p_all, const int64_t *p_off,
                            const int64_t *tab_off, void *m_all, int16_t *s_all,
                            int32_t *status_dev, void *stream);

/* The configuration a plan currently uses (defaults until autotuned):
 * levels per bulk task, and resident blocks per SM (0 = the occupancy limit). */
dp_status mcm_plan_config(const void *plan, int32_t *levels_per_part, int32_t *blocks_per_sm);

dp_status mcm_plan_destroy(void *plan);

/* ------------------------------------------------------------------------- */
/* S-DP (Definition 1, Eq. (1))                                               */
/* ------------------------------------------------------------------------- */

/* Fills ST[a_1 .. n-1] in place.
 *   ST      device uint32[n]; ST[0 .. a[0]-1] must hold the preset values.
 *   n       table length (n <= a[0] is a no-op returning DP_OK).
 *   a       HOST int32[k], strictly decreasing, a[k-1] >= 1 (any a[0]: windows of
 *           up to 32768 words are kept in shared memory, larger ones are read
 *           from the table in global memory).
 *   op      DP_OP_MIN or DP_OP_ADD_MOD32.
 * Both operators are commutative and associative, so the result does not
 * depend on the order in which the k terms are combined.
 * With DP_OP_ADD_MOD32 and a table long enough (a cost model decides), the
 * table is cut into chunks that run side by side, each starting from a
 * window obtained by products modulo the recurrence's characteristic
 * polynomial.  That path enqueues a few dozen launches and takes a
 * workspace of a few MB from the stream-ordered allocator (released on the
 * same stream).  Its result is bit-identical. */
dp_status sdp_solve(uint32_t *ST, int64_t n, const int32_t *a, int32_t k, dp_op op,
                    int32_t *status_dev, void *stream);

/* Same with a HOST table: copies ST[0..a[0]-1] in, solves, copies ST out. */
dp_status sdp_solve_host(uint32_t *ST_host, int64_t n, const int32_t *a, int32_t k, dp_op op,
                         void *stream);

/* Batched S-DP: independent instances, one thread block each, one launch.
 * sdp_plan_create reads, on the host: n_host[b] (table lengths), k_host[b]
 * (offset counts) and the offsets concatenated in a_host (instance b's k_b
 * offsets follow those of instance b-1), validates them and copies the
 * offsets to the plan's device memory. */
dp_status sdp_plan_create(int32_t batch, const int64_t *n_host, const int32_t *k_host,
                          const int32_t *a_host, dp_op op, void **plan);

/* Runs a plan on device tables: instance b's table starts at element
 * st_off[b] (device int64[batch]) of ST_all.  Graph-capturable. */
dp_status sdp_solve_batched(void *plan, uint32_t *ST_all, const int64_t *st_off,
                            int32_t *status_dev, void *stream);

dp_status sdp_plan_destroy(void *plan);

/* ------------------------------------------------------------------------- */
/* Serving: continuous batching of MCM / S-DP requests                        */
/* ------------------------------------------------------------------------- */

typedef struct {
  int64_t hbm_cap_bytes;     /* admission cap on device tables held by the server */
  int32_t max_inflight;      /* maximum requests admitted but not released */
  int32_t num_streams;       /* launch streams used in rotation (>= 1) */
  int32_t max_batch;         /* maximum requests grouped into one launch */
  int32_t device;            /* CUDA device ordinal */
} dp_serve_config;

typedef enum { DP_REQ_MCM = 0, DP_REQ_SDP = 1 } dp_req_kind;

typedef struct {
  int32_t kind;              /* dp_req_kind */
  int32_t cost;              /* MCM: dp_cost */
  int64_t n;                 /* MCM: matrices; S-DP: table length */
  const int32_t *dims;       /* MCM: HOST int32[n+1] (copied at submit) */
  const int32_t *offsets;    /* S-DP: HOST int32[k] (copied at submit) */
  int32_t k;                 /* S-DP: number of offsets */
  int32_t op;                /* S-DP: dp_op */
  const uint32_t *preset;    /* S-DP: HOST uint32[offsets[0]] (copied at submit) */
} dp_request;

typedef struct {
  int32_t status;            /* dp_status of the solve */
  int32_t kind;
  int64_t n;
  const void *m_dev;         /* MCM: device table (cost type of the request), server-owned */
  const int16_t *s_dev;      /* MCM: device split table, server-owned */
  const uint32_t *st_dev;    /* S-DP: device table, server-owned */
  double t_submit;           /* seconds (server clock) when submitted */
  double t_start;            /* when its launch was enqueued */
  double t_done;             /* when completion was observed */
} dp_result;

/* Creates a server (starts its scheduler thread).  */
dp_status serve_create(const dp_serve_config *cfg, void **srv);
/* Admits a request (copies its host inputs) or returns DP_EBUSY when the
 * in-flight count or the HBM cap would be exceeded; *ticket identifies it. */
dp_status serve_submit(void *srv, const dp_request *req, uint64_t *ticket);
/* DP_EPENDING until the request finished; then fills *out.  Result pointers
 * stay valid until serve_release(ticket). */
dp_status serve_poll(void *srv, uint64_t ticket, dp_result *out);
/* Frees a finished request's device tables (returns its HBM to admission).
 * The free is ordered on the server's own stream only: work the caller has
 * enqueued that still reads the tables (a copy on another stream) must have
 * completed before this call -- synchronise first, or use
 * serve_release_stream. */
dp_status serve_release(void *srv, uint64_t ticket);
/* serve_release for a caller that still has reads of the tables enqueued on
 * `stream` (cudaStream_t as void*, NULL = legacy default stream): an event is
 * recorded on that stream, and the tables' memory is freed only after it (and
 * after the events of every other release of requests that share the same
 * allocation).  Returns at once; DP_ECUDA if the event cannot be recorded. */
dp_status serve_release_stream(void *srv, uint64_t ticket, void *stream);
/* Current server time in seconds (the clock used by dp_result). */
double serve_now(void *srv);
/* Stops the scheduler after the queued work drains and frees everything. */
dp_status serve_destroy(void *srv);

#ifdef __cplusplus
}
#endif

#endif /* DPGPU_H */
