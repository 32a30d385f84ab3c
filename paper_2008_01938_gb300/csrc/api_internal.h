// api_internal.h -- host-side helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <memory>
#include <vector>

#include "dpgpu.h"
#include "mcm_kernels.cuh"
#include "sdp_kernels.cuh"

namespace dph {

// Records a thread-local error message and returns `code`.
dp_status fail(dp_status code, const char* fmt, ...);
dp_status fail_cuda(cudaError_t e, const char* what);

struct DevState {
  int device = -1;
  int sms = 0;
  int occ[2] = {0, 0};        // MCM blocks per SM, int32 / int64 costs
  int32_t* status = nullptr;  // library-owned status word
};

// Per-device state for the current device (created on first use).
dp_status current_dev(DevState** out);

long long spin_limit();     // bounded-wait budget in clock cycles

// Kernel timing (dp_profile_begin / dp_profile_end): when enabled, the
// launchers bracket each solver kernel with events on its stream.
bool profiling();
void profile_mark(int which, cudaStream_t st, bool after);  // which: 0 = MCM, 1 = S-DP

// ---------------------------------------------------------------------------
// MCM plans
// ---------------------------------------------------------------------------
struct McmStatic {
  bool i64 = false;
  int device = -1;
  std::vector<int32_t> ns;
  std::vector<dpk::McmInstDev> insts;   // static fields only
  std::vector<dpk::McmTask> tasks;
  std::vector<int32_t> accslot;
  int64_t ntiles = 0, nslots = 0, pp_total = 0, pk_total = 0;
  double split_evals = 0;
  // device copies (immutable after creation)
  dpk::McmTask* d_tasks = nullptr;
  int32_t* d_accslot = nullptr;
  dpk::McmInstDev* d_insts = nullptr;
  bool owns_device = true;               // false: device pointers borrowed from a workspace
  ~McmStatic();
};

struct McmLayout {
  size_t af = 0, bf = 0, flags = 0, counters = 0, queue = 0, acc = 0, pp = 0, pk = 0, insts = 0;
  size_t zero_begin = 0, zero_bytes = 0, total = 0;
};

// Builds the work queue on the host; with upload=true also copies the queue,
// slot table and chain records to fresh device memory owned by the result.
// levels_per_part: external levels per bulk task (0 = the default).
dp_status mcm_build_static(const std::vector<int32_t>& ns, bool i64, std::shared_ptr<McmStatic>* out,
                           bool upload = true, int levels_per_part = 0);
McmLayout mcm_layout(const McmStatic& sp);
// Enqueues memsets + prologue + main kernel for a static plan on `ws`.
// w_all != nullptr: the interval DP with per-cell weights laid out like m_all
// (a weight pass is enqueued before the prologue).
dp_status mcm_enqueue(const McmStatic& sp, const McmLayout& L, void* ws, const int32_t* p_all,
                      const int64_t* p_off, const int64_t* tab_off, void* m_all, int16_t* s_all,
                      int32_t* status, cudaStream_t st, long long limit_override = 0,
                      int32_t drop_task = -1, int blocks_per_sm = 0, const void* w_all = nullptr);

// ---------------------------------------------------------------------------
// S-DP
// ---------------------------------------------------------------------------
dp_status sdp_validate(int64_t n, const int32_t* a, int32_t k, int op);
void sdp_shape(int32_t a1, int32_t ak, int* threads, int* ring_log2);
// (x) = + on one instance, by chunks that start from jumped windows
// (sdp_jump.cu): the number of chunks the cost model picks (0: solve step by
// step), and the solve with a given number of chunks.
int sdp_jump_chunks(int64_t n, const int32_t* a, int32_t k, int sms);
// The plan behind it (host arithmetic only): P, L, L0, squarings, reach of
// the impulse response, chunks per major window, major windows, chunks asked.
int sdp_jump_plan(int64_t n, const int32_t* a, int32_t k, int sms, int64_t out[8]);
dp_status sdp_add_jump(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, int chunks, int32_t* status,
                       cudaStream_t st);
// (x) = min on one instance, by chunks whose windows come from Boolean
// products modulo the characteristic polynomial (sdp_minjump.cu): whether the
// path applies (a_k >= 32, a_1 <= 8192, a long enough table, the window on
// chip), the number of chunks the cost model picks (0: solve step by step),
// and the solve with a given number of chunks.
bool sdp_min_jump_eligible(int64_t n, const int32_t* a, int32_t k);
int sdp_min_jump_chunks(int64_t n, const int32_t* a, int32_t k, int sms);
// The plan behind it (host arithmetic only): P, L, L0, squarings, chunks asked.
int sdp_min_jump_plan(int64_t n, const int32_t* a, int32_t k, int sms, int64_t out[5]);
dp_status sdp_min_jump(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, int chunks, int32_t* status,
                       cudaStream_t st);

}  // namespace dph
