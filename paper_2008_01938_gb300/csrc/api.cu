// api.cu -- host side of the C ABI declared in include/dpgpu.h: argument
// validation, the diagonal-ordered MCM work queue, workspaces and launches.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "api_internal.h"

namespace dph {

namespace {
thread_local std::string t_err = "no error";
std::mutex g_mu;
std::map<int, DevState> g_dev;

constexpr int T = dpk::kTile;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace

dp_status fail(dp_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

dp_status fail_cuda(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? DP_ENOMEM : DP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

long long spin_limit() {
  const char* s = getenv("DPGPU_SPIN_LIMIT");
  if (s && *s) {
    const long long v = atoll(s);
    if (v > 0) return v;
  }
  return 1ll << 32;  // about two seconds of SM clock
}

namespace {
std::atomic<bool> g_prof{false};
std::mutex g_prof_mu;
struct ProfPair {
  int which;
  cudaEvent_t a, b;
};
std::vector<ProfPair> g_prof_ev;
}  // namespace

bool profiling() { return g_prof.load(std::memory_order_relaxed); }

void profile_mark(int which, cudaStream_t st, bool after) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!after) {
    ProfPair p{which, nullptr, nullptr};
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    cudaEventRecord(p.a, st);
    g_prof_ev.push_back(p);
  } else {
    for (auto it = g_prof_ev.rbegin(); it != g_prof_ev.rend(); ++it) {
      if (it->which == which) {
        cudaEventRecord(it->b, st);
        break;
      }
    }
  }
}

dp_status current_dev(DevState** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev.find(dev);
  if (it != g_dev.end()) {
    *out = &it->second;
    return DP_OK;
  }
  DevState ds;
  ds.device = dev;
  if ((e = cudaDeviceGetAttribute(&ds.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail_cuda(e, "cudaDeviceGetAttribute");
  for (int c = 0; c < 2; ++c) {
    if ((e = dpk::mcm_configure(c == 1)) != cudaSuccess) return fail_cuda(e, "configure MCM kernel");
    if ((e = dpk::mcm_occupancy(c == 1, &ds.occ[c])) != cudaSuccess) return fail_cuda(e, "MCM occupancy");
    if (ds.occ[c] < 1) ds.occ[c] = 1;
  }
  if ((e = cudaMalloc(&ds.status, 256)) != cudaSuccess) return fail_cuda(e, "cudaMalloc(status)");
  if ((e = cudaMemset(ds.status, 0, 256)) != cudaSuccess) return fail_cuda(e, "cudaMemset(status)");
  // keep freed stream-ordered allocations cached in the pool
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  auto res = g_dev.emplace(dev, ds);
  *out = &res.first->second;
  return DP_OK;
}

// ---------------------------------------------------------------------------
// MCM: static plan (task queue) construction
// ---------------------------------------------------------------------------

McmStatic::~McmStatic() {
  if (device >= 0 && owns_device) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    cudaFree(d_tasks);
    cudaFree(d_accslot);
    cudaFree(d_insts);
    if (cur >= 0 && cur != device) cudaSetDevice(cur);
  }
}

namespace {
using dpk::kMinBulkLevels;

// Queue order: by bucket, a tile-diagonal no earlier than the one at which the
// task becomes ready (every task therefore waits only for tasks queued before
// it); within a bucket, finishers (the critical path) before bulk tasks, and
// bulk tasks by the tile-diagonal of the finisher that needs them.
struct SortKey {
  int32_t bucket, kind, need, inst, I, J;
  bool operator<(const SortKey& o) const {
    return std::tie(bucket, kind, need, inst, I, J) < std::tie(o.bucket, o.kind, o.need, o.inst, o.I, o.J);
  }
};
}  // namespace

dp_status mcm_build_static(const std::vector<int32_t>& ns, bool i64, std::shared_ptr<McmStatic>* out, bool upload,
                           int levels_per_part) {
  const int kLevelsPerPart = levels_per_part > 0 ? levels_per_part : dpk::kLevelsPerPart;
  auto sp = std::make_shared<McmStatic>();
  sp->i64 = i64;
  sp->ns = ns;
  int64_t tile_base = 0, pp_base = 0, pk_base = 0;
  for (size_t b = 0; b < ns.size(); ++b) {
    const int32_t n = ns[b];
    if (n < 1 || n > 32767) return fail(DP_EINVAL, "chain %zu: n = %d outside [1, 32767]", b, n);
    dpk::McmInstDev in{};
    in.n = n;
    in.nt = (n + T - 1) / T;
    in.tile_base = tile_base;
    in.pp_base = pp_base;
    in.pk_base = pk_base;
    sp->insts.push_back(in);
    tile_base += (int64_t)in.nt * (in.nt + 1) / 2;
    pp_base += (int64_t)in.nt * T + 32;
    pk_base += (int64_t)in.nt * T;
    sp->split_evals += ((double)n * n * n - n) / 6.0;
  }
  sp->ntiles = tile_base;
  sp->pp_total = pp_base;
  sp->pk_total = pk_base;
  sp->accslot.assign((size_t)tile_base, -1);

  std::vector<std::pair<SortKey, dpk::McmTask>> items;
  for (size_t b = 0; b < ns.size(); ++b) {
    const dpk::McmInstDev& in = sp->insts[b];
    const int nt = in.nt;
    for (int I = 0; I < nt; ++I) {
      for (int J = I; J < nt; ++J) {
        const int D = J - I;
        const int64_t tix = in.tile_base + (int64_t)I * nt - (int64_t)I * (I - 1) / 2 + (J - I);
        dpk::McmTask fin{};
        fin.inst = (int32_t)b;
        fin.I = (int16_t)I;
        fin.J = (int16_t)J;
        fin.kind = 0;
        fin.r_lo = 1;
        fin.r_hi = 0;  // empty range
        if (D >= 2) {
          const int rmin = (D + 1) / 2, rmax = D - 1;
          int fin_lo = rmax;  // the finisher keeps the last level (both neighbours)
          if (fin_lo - rmin < kMinBulkLevels) fin_lo = rmin;
          int nparts = 0;
          auto add_part = [&](int r0, int r1) {
            dpk::McmTask part{};
            part.inst = (int32_t)b;
            part.I = (int16_t)I;
            part.J = (int16_t)J;
            part.r_lo = (int16_t)r0;
            part.r_hi = (int16_t)r1;
            part.kind = 1;
            // ready at bucket r1 + 1; int32 parts other than the last one are
            // deferred to kDeferBuckets diagonals before their finisher (int64
            // plans keep the readiness order)
            const bool last = r1 == fin_lo - 1;
            const int bucket = (i64 || last) ? r1 + 1 : std::max(r1 + 1, D - dpk::kDeferBuckets);
            items.push_back({SortKey{bucket, 1, i64 ? 0 : D, (int32_t)b, I, J}, part});
            ++nparts;
          };
          if (i64) {
            for (int r0 = rmin; r0 < fin_lo; r0 += kLevelsPerPart)
              add_part(r0, std::min(r0 + kLevelsPerPart - 1, fin_lo - 1));
          } else if (fin_lo > rmin) {
            int r1 = fin_lo - 1;
            int r0 = std::max(rmin, r1 - dpk::kLastPartLevels + 1);
            add_part(r0, r1);
            for (r1 = r0 - 1; r1 >= rmin; r1 = r0 - 1) {
              r0 = std::max(rmin, r1 - kLevelsPerPart + 1);
              add_part(r0, r1);
            }
          }
          if (nparts > 0) sp->accslot[(size_t)tix] = (int32_t)sp->nslots++;
          fin.r_lo = (int16_t)fin_lo;
          fin.r_hi = (int16_t)rmax;
          fin.nparts = (int16_t)nparts;
        }
        items.push_back({SortKey{D, 0, 0, (int32_t)b, I, J}, fin});
      }
    }
  }
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<SortKey, dpk::McmTask>& x, const std::pair<SortKey, dpk::McmTask>& y) {
                     return x.first < y.first;
                   });
  sp->tasks.reserve(items.size());
  for (auto& it : items) sp->tasks.push_back(it.second);

  if (!upload) {
    *out = sp;
    return DP_OK;
  }
  cudaError_t e;
  if ((e = cudaGetDevice(&sp->device)) != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  const size_t tb = sp->tasks.size() * sizeof(dpk::McmTask);
  const size_t ab = sp->accslot.size() * sizeof(int32_t);
  const size_t ib = sp->insts.size() * sizeof(dpk::McmInstDev);
  if ((e = cudaMalloc(&sp->d_tasks, std::max<size_t>(tb, 16))) != cudaSuccess) return fail_cuda(e, "cudaMalloc(tasks)");
  if ((e = cudaMalloc(&sp->d_accslot, std::max<size_t>(ab, 16))) != cudaSuccess) return fail_cuda(e, "cudaMalloc(accslot)");
  if ((e = cudaMalloc(&sp->d_insts, std::max<size_t>(ib, 16))) != cudaSuccess) return fail_cuda(e, "cudaMalloc(insts)");
  if (tb && (e = cudaMemcpy(sp->d_tasks, sp->tasks.data(), tb, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail_cuda(e, "upload tasks");
  if (ab && (e = cudaMemcpy(sp->d_accslot, sp->accslot.data(), ab, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail_cuda(e, "upload accslot");
  if (ib && (e = cudaMemcpy(sp->d_insts, sp->insts.data(), ib, cudaMemcpyHostToDevice)) != cudaSuccess)
    return fail_cuda(e, "upload instances");
  *out = sp;
  return DP_OK;
}

McmLayout mcm_layout(const McmStatic& sp) {
  McmLayout L;
  const size_t es = sp.i64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 16), 256);
    return o;
  };
  L.af = take((size_t)sp.ntiles * T * T * es);
  L.bf = take((size_t)sp.ntiles * T * T * es);
  L.zero_begin = off;
  L.flags = take((size_t)sp.ntiles * 4);
  L.counters = take((size_t)sp.ntiles * 4);
  L.queue = take(16);
  L.zero_bytes = off - L.zero_begin;
  L.acc = take((size_t)sp.nslots * T * T * 8);
  L.pp = take((size_t)sp.pp_total * 4);
  L.pk = take((size_t)sp.pk_total * 4);
  L.insts = take(sp.insts.size() * sizeof(dpk::McmInstDev));
  L.total = off;
  return L;
}

dp_status mcm_enqueue(const McmStatic& sp, const McmLayout& L, void* ws, const int32_t* p_all,
                      const int64_t* p_off, const int64_t* tab_off, void* m_all, int16_t* s_all,
                      int32_t* status, cudaStream_t st, long long limit_override, int32_t drop_task,
                      int blocks_per_sm, const void* w_all) {
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  uint8_t* w = static_cast<uint8_t*>(ws);
  cudaError_t e;
  if ((e = cudaMemsetAsync(w + L.zero_begin, 0, L.zero_bytes, st)) != cudaSuccess) return fail_cuda(e, "memset flags");
  if (sp.nslots > 0 && (e = cudaMemsetAsync(w + L.acc, 0xFF, (size_t)sp.nslots * T * T * 8, st)) != cudaSuccess)
    return fail_cuda(e, "memset accumulators");
  if ((e = cudaMemcpyAsync(w + L.insts, sp.d_insts, sp.insts.size() * sizeof(dpk::McmInstDev),
                           cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return fail_cuda(e, "copy instances");
  dpk::McmLaunchArgs a{};
  a.insts = reinterpret_cast<dpk::McmInstDev*>(w + L.insts);
  a.tasks = sp.d_tasks;
  a.ninst = (int32_t)sp.insts.size();
  a.ntasks = (int32_t)sp.tasks.size();
  a.af = w + L.af;
  a.bf = w + L.bf;
  a.flags = reinterpret_cast<int32_t*>(w + L.flags);
  a.counters = reinterpret_cast<int32_t*>(w + L.counters);
  a.accslot = sp.d_accslot;
  a.acc = reinterpret_cast<unsigned long long*>(w + L.acc);
  a.pp = reinterpret_cast<int32_t*>(w + L.pp);
  a.pk = reinterpret_cast<uint32_t*>(w + L.pk);
  a.queue = reinterpret_cast<int32_t*>(w + L.queue);
  a.status = status ? status : ds->status;
  a.spin_limit = limit_override > 0 ? limit_override : spin_limit();
  a.drop_task = drop_task;
  a.p_all = p_all;
  a.p_off = p_off;
  a.tab_off = tab_off;
  a.m_all = m_all;
  a.s_all = s_all;
  a.w_all = w_all;
  if (w_all && (e = dpk::launch_mcm_weight_max(a, sp.i64, ds->sms, st)) != cudaSuccess)
    return fail_cuda(e, "launch weight pass");
  if ((e = dpk::launch_mcm_prologue(a, sp.i64, st)) != cudaSuccess) return fail_cuda(e, "launch MCM prologue");
  const int c = sp.i64 ? 1 : 0;
  const int bps = blocks_per_sm > 0 ? std::min(blocks_per_sm, ds->occ[c]) : ds->occ[c];
  const int grid = (int)std::max<int64_t>(2, std::min<int64_t>((int64_t)ds->sms * bps, (int64_t)sp.tasks.size()));
  const bool prof = profiling();
  if (prof) profile_mark(0, st, false);
  if ((e = dpk::launch_mcm_main(a, sp.i64, std::max(grid, 1), st)) != cudaSuccess)
    return fail_cuda(e, "launch MCM kernel");
  if (prof) profile_mark(0, st, true);
  return DP_OK;
}

// ---------------------------------------------------------------------------
// S-DP helpers
// ---------------------------------------------------------------------------
dp_status sdp_validate(int64_t n, const int32_t* a, int32_t k, int op) {
  if (op != DP_OP_MIN && op != DP_OP_ADD_MOD32) return fail(DP_EINVAL, "op must be DP_OP_MIN or DP_OP_ADD_MOD32");
  if (k < 1 || k > dpk::kSdpMaxK) return fail(DP_EINVAL, "k = %d outside [1, %d]", k, dpk::kSdpMaxK);
  if (!a) return fail(DP_EINVAL, "offsets pointer is NULL");
  if (n < 0) return fail(DP_EINVAL, "n = %lld < 0", (long long)n);
  for (int j = 0; j < k; ++j) {
    if (a[j] < 1) return fail(DP_EINVAL, "offset a[%d] = %d < 1", j, a[j]);
    if (j > 0 && a[j] >= a[j - 1])
      return fail(DP_EINVAL, "offsets must be strictly decreasing (a[%d] = %d >= a[%d] = %d)", j, a[j], j - 1,
                  a[j - 1]);
  }
  return DP_OK;
}

void sdp_shape(int32_t a1, int32_t ak, int* threads, int* ring_log2) {
  int th = ak >= 1024 ? 1024 : ((ak + 31) / 32) * 32;
  if (th < 32) th = 32;
  const int W = std::min(ak, th);
  int lg = 0;
  while ((1ll << lg) < (long long)a1 + W) ++lg;
  *threads = th;
  *ring_log2 = lg <= dpk::kSdpRingMaxLog2 ? std::max(lg, 1) : 0;
}

}  // namespace dph

using namespace dph;

// ===========================================================================
// C ABI
// ===========================================================================
namespace {
std::mutex g_cache_mu;
// per (device, n, cost) static plans for single-chain solves
std::list<std::tuple<int, int32_t, bool, std::shared_ptr<McmStatic>>> g_single_cache;

dp_status single_plan(int32_t n, bool i64, std::shared_ptr<McmStatic>* out) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto it = g_single_cache.begin(); it != g_single_cache.end(); ++it) {
    if (std::get<0>(*it) == dev && std::get<1>(*it) == n && std::get<2>(*it) == i64) {
      *out = std::get<3>(*it);
      g_single_cache.splice(g_single_cache.begin(), g_single_cache, it);
      return DP_OK;
    }
  }
  std::shared_ptr<McmStatic> sp;
  dp_status rc = mcm_build_static(std::vector<int32_t>{n}, i64, &sp);
  if (rc != DP_OK) return rc;
  g_single_cache.emplace_front(dev, n, i64, sp);
  if (g_single_cache.size() > 32) g_single_cache.pop_back();
  *out = sp;
  return DP_OK;
}

struct McmPlan {
  std::shared_ptr<McmStatic> sp;
  McmLayout L;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int device = -1;
  std::vector<int32_t> ns;
  bool i64 = false;
  int levels_per_part = dpk::kLevelsPerPart;  // queue granularity (chosen by mcm_plan_autotune)
  int blocks_per_sm = 0;                      // resident blocks per SM, 0 = occupancy limit
};

struct SdpPlan {
  int device = -1;
  int32_t batch = 0;
  int op = 0;
  int threads = 32, ring_log2 = 0, kmax = 1;
  bool kfull = false;
  dpk::SdpInstDev* d_insts = nullptr;
  int32_t* d_offs = nullptr;
};

// Device address of the host range [ptr, ptr + bytes) if the current device
// can access it in place: page-locked memory (cudaHostAlloc, cudaHostRegister)
// mapped for this device, the whole range inside one allocation, and
// writable by the device when `writable`.  nullptr otherwise (pageable
// memory, a range that leaves its allocation, or a query the driver does not
// answer), in which case the caller stages the data through device memory.
using PointerAttributeFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
PointerAttributeFn pointer_attribute_fn() {
  static const PointerAttributeFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PointerAttributeFn>(f);
  }();
  return fn;
}

void* host_range_device_address(const void* ptr, size_t bytes, bool writable) {
  if (!ptr || bytes == 0) return nullptr;
  const PointerAttributeFn attr = pointer_attribute_fn();
  if (!attr) return nullptr;
  const uint8_t* first = static_cast<const uint8_t*>(ptr);
  const uint8_t* last = first + (bytes - 1);
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, first) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (pa.type != cudaMemoryTypeHost || !pa.devicePointer) return nullptr;
  unsigned long long id0 = 0, id1 = 0;
  unsigned int access = 0;
  if (attr(&id0, CU_POINTER_ATTRIBUTE_BUFFER_ID, reinterpret_cast<CUdeviceptr>(first)) != CUDA_SUCCESS ||
      attr(&id1, CU_POINTER_ATTRIBUTE_BUFFER_ID, reinterpret_cast<CUdeviceptr>(last)) != CUDA_SUCCESS ||
      attr(&access, CU_POINTER_ATTRIBUTE_ACCESS_FLAGS, reinterpret_cast<CUdeviceptr>(first)) != CUDA_SUCCESS)
    return nullptr;
  if (id0 == 0 || id0 != id1) return nullptr;
  const unsigned int need = writable ? CU_POINTER_ATTRIBUTE_ACCESS_FLAG_READWRITE : CU_POINTER_ATTRIBUTE_ACCESS_FLAG_READ;
  if ((access & need) != need) return nullptr;
  return pa.devicePointer;
}

dp_status mcm_solve_impl(const int32_t* p, int32_t n, dp_cost ct, void* m, int16_t* s, int32_t* status_dev,
                         cudaStream_t st, long long limit_override, int32_t drop_task, const void* w = nullptr) {
  const char* who = w ? "interval_dp_solve" : "mcm_solve";
  if (!p || !m || !s) return fail(DP_EINVAL, "%s: NULL pointer argument", who);
  if (n < 1 || n > 32767) return fail(DP_EINVAL, "%s: n = %d outside [1, 32767]", who, n);
  if (ct != DP_COST_I32 && ct != DP_COST_I64) return fail(DP_EINVAL, "%s: unknown cost type %d", who, (int)ct);
  const bool i64 = ct == DP_COST_I64;
  if (w && i64) return fail(DP_EINVAL, "interval_dp_solve: only DP_COST_I32 is available");
  std::shared_ptr<McmStatic> sp;
  dp_status rc = single_plan(n, i64, &sp);
  if (rc != DP_OK) return rc;
  const McmLayout L = mcm_layout(*sp);
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, L.total, st);
  if (e != cudaSuccess) return fail_cuda(e, w ? "interval_dp_solve: workspace allocation" : "mcm_solve: workspace allocation");
  rc = mcm_enqueue(*sp, L, ws, p, nullptr, nullptr, m, s, status_dev, st, limit_override, drop_task, 0, w);
  e = cudaFreeAsync(ws, st);
  if (rc != DP_OK) return rc;
  if (e != cudaSuccess) return fail_cuda(e, w ? "interval_dp_solve: workspace release" : "mcm_solve: workspace release");
  return DP_OK;
}
}  // namespace

extern "C" {

const char* dp_last_error(void) { return t_err.c_str(); }

const char* dp_version(void) { return "dpgpu 0.1 (sm_103a)"; }

dp_status dp_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& p : g_prof_ev) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_prof_ev.clear();
  g_prof.store(true);
  return DP_OK;
}

dp_status dp_profile_end(double* mcm_ms, int64_t* mcm_launches, double* sdp_ms, int64_t* sdp_launches) {
  g_prof.store(false);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  double ms[2] = {0, 0};
  int64_t cnt[2] = {0, 0};
  dp_status rc = DP_OK;
  for (auto& p : g_prof_ev) {
    float t = 0;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
    if (e != cudaSuccess && rc == DP_OK) rc = fail_cuda(e, "dp_profile_end");
    ms[p.which] += t;
    cnt[p.which] += 1;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_prof_ev.clear();
  if (mcm_ms) *mcm_ms = ms[0];
  if (mcm_launches) *mcm_launches = cnt[0];
  if (sdp_ms) *sdp_ms = ms[1];
  if (sdp_launches) *sdp_launches = cnt[1];
  return rc;
}

dp_status dp_sync_status(void* stream, int32_t* status_dev) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(e, "dp_sync_status: stream");
  int32_t* word = status_dev;
  if (!word) {
    DevState* ds = nullptr;
    dp_status rc = current_dev(&ds);
    if (rc != DP_OK) return rc;
    word = ds->status;
  }
  int32_t h = 0;
  if ((e = cudaMemcpy(&h, word, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return fail_cuda(e, "read status");
  if (h != 0) {
    if ((e = cudaMemset(word, 0, 4)) != cudaSuccess) return fail_cuda(e, "clear status");
    const char* what = h == DP_EINVAL      ? "invalid input found on the device (a dimension < 1?)"
                       : h == DP_EOVERFLOW ? "cost bound does not fit the cost type"
                       : h == DP_ETIMEOUT  ? "a bounded device-side wait timed out"
                                           : "device error";
    return fail((dp_status)h, "device status %d: %s", h, what);
  }
  return DP_OK;
}

dp_status mcm_solve(const int32_t* p, int32_t n, dp_cost ct, void* m, int16_t* s, int32_t* status_dev,
                    void* stream) {
  return mcm_solve_impl(p, n, ct, m, s, status_dev, static_cast<cudaStream_t>(stream), 0, -1);
}

dp_status interval_dp_solve(const int32_t* p, const void* w, int32_t n, dp_cost ct, void* m, int16_t* s,
                            int32_t* status_dev, void* stream) {
  if (!w) return fail(DP_EINVAL, "interval_dp_solve: NULL pointer argument");
  return mcm_solve_impl(p, n, ct, m, s, status_dev, static_cast<cudaStream_t>(stream), 0, -1, w);
}

// Fault-injection hook for tests: like mcm_solve, but queue entry `drop_task`
// is popped and skipped, so the tiles waiting for it hit their bounded waits
// (`spin_limit` clock cycles) and the status word reports DP_ETIMEOUT.
dp_status dp_test_mcm_drop_task(const int32_t* p, int32_t n, dp_cost ct, void* m, int16_t* s,
                                int32_t* status_dev, void* stream, int32_t drop_task, long long limit) {
  return mcm_solve_impl(p, n, ct, m, s, status_dev, static_cast<cudaStream_t>(stream), limit, drop_task);
}

dp_status mcm_solve_host(const int32_t* p_host, int32_t n, dp_cost ct, void* m_host, int16_t* s_host,
                         void* stream) {
  if (!p_host || !m_host || !s_host) return fail(DP_EINVAL, "mcm_solve_host: NULL pointer argument");
  if (n < 1 || n > 32767) return fail(DP_EINVAL, "mcm_solve_host: n = %d outside [1, 32767]", n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t es = ct == DP_COST_I64 ? 8 : 4;
  const size_t nn = (size_t)n * n;
  // Page-locked tables the device may write are the kernel's outputs
  // themselves: the results reach host memory while the solve runs, and no
  // copy follows it.  Page-locked dims are read in place.
  void* m_dev = host_range_device_address(m_host, nn * es, true);
  void* s_dev = m_dev ? host_range_device_address(s_host, nn * 2, true) : nullptr;
  const bool direct = m_dev && s_dev;
  const int32_t* p_dev = static_cast<const int32_t*>(host_range_device_address(p_host, (size_t)(n + 1) * 4, false));
  uint8_t* buf = nullptr;
  const size_t pb = p_dev ? 0 : align_up((size_t)(n + 1) * 4, 256);
  const size_t mb = direct ? 0 : align_up(nn * es, 256), sb = direct ? 0 : align_up(nn * 2, 256);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), pb + mb + sb + 256, st);
  if (e != cudaSuccess) return fail_cuda(e, "mcm_solve_host: allocation");
  int32_t* d_status = reinterpret_cast<int32_t*>(buf + pb + mb + sb);
  dp_status rc = DP_OK;
  if ((e = cudaMemsetAsync(d_status, 0, 4, st)) != cudaSuccess ||
      (!p_dev && (e = cudaMemcpyAsync(buf, p_host, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)) {
    rc = fail_cuda(e, "mcm_solve_host: upload");
  }
  if (rc == DP_OK)
    rc = mcm_solve_impl(p_dev ? p_dev : reinterpret_cast<int32_t*>(buf), n, ct, direct ? m_dev : buf + pb,
                        direct ? static_cast<int16_t*>(s_dev) : reinterpret_cast<int16_t*>(buf + pb + mb), d_status,
                        st, 0, -1);
  if (rc == DP_OK && !direct) {
    if ((e = cudaMemcpyAsync(m_host, buf + pb, nn * es, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s_host, buf + pb + mb, nn * 2, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      rc = fail_cuda(e, "mcm_solve_host: download");
  }
  if (rc == DP_OK) rc = dp_sync_status(stream, d_status);
  cudaFreeAsync(buf, st);
  if (rc == DP_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = fail_cuda(e, "mcm_solve_host: sync");
  return rc;
}

// Test hook (host only): the MCM work queue of a plan over chains of ns[0..m)
// matrices, in pop order, 6 words per task: chain, I, J, kind (0 finisher,
// 1 bulk part), first and last external level. Returns the number of tasks
// (at most cap are written), or -1.
int32_t dp_test_mcm_queue(const int32_t* ns, int32_t m, int32_t i64, int32_t* out, int32_t cap) {
  if (!ns || m < 1) return -1;
  std::shared_ptr<McmStatic> sp;
  if (mcm_build_static(std::vector<int32_t>(ns, ns + m), i64 != 0, &sp, false) != DP_OK) return -1;
  const int64_t nt = (int64_t)sp->tasks.size();
  for (int64_t x = 0; x < nt && x < cap && out; ++x) {
    const dpk::McmTask& t = sp->tasks[(size_t)x];
    int32_t* o = out + 6 * x;
    o[0] = t.inst, o[1] = t.I, o[2] = t.J, o[3] = t.kind, o[4] = t.r_lo, o[5] = t.r_hi;
  }
  return nt > INT32_MAX ? -1 : (int32_t)nt;
}

// Test hooks for the (x) = + jump path: the number of chunks sdp_solve would
// use, and the path itself with a given number of chunks.
int32_t dp_test_sdp_jump_chunks(int64_t n, const int32_t* a, int32_t k) {
  DevState* ds = nullptr;
  if (!a || k < 1 || current_dev(&ds) != DP_OK) return -1;
  return sdp_jump_chunks(n, a, k, ds->sms);
}

// Test hooks for the (x) = min jump path: the number of chunks sdp_solve
// would use, and the path itself with a given number of chunks.
int32_t dp_test_sdp_min_jump_chunks(int64_t n, const int32_t* a, int32_t k) {
  DevState* ds = nullptr;
  if (!a || k < 1 || current_dev(&ds) != DP_OK) return -1;
  return sdp_min_jump_chunks(n, a, k, ds->sms);
}

// Test hook without a device: the min jump plan sdp_solve would take for
// `sms` SMs (out: P, L, L0, squarings, chunks).
int32_t dp_test_sdp_min_jump_plan(int64_t n, const int32_t* a, int32_t k, int32_t sms, int64_t* out) {
  if (!a || !out || k < 1 || k > dpk::kSdpMaxK || sms < 2) return -1;
  for (int j = 0; j < k; ++j)
    if (a[j] < 1 || (j > 0 && a[j] >= a[j - 1])) return -1;
  return sdp_min_jump_plan(n, a, k, sms, out);
}

dp_status dp_test_sdp_min_jump(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, int32_t chunks,
                               int32_t* status_dev, void* stream) {
  if (!ST) return fail(DP_EINVAL, "dp_test_sdp_min_jump: ST is NULL");
  dp_status rc = sdp_validate(n, a, k, DP_OP_MIN);
  if (rc != DP_OK) return rc;
  DevState* ds = nullptr;
  if ((rc = current_dev(&ds)) != DP_OK) return rc;
  return sdp_min_jump(ST, n, a, k, chunks, status_dev ? status_dev : ds->status, static_cast<cudaStream_t>(stream));
}

// Test hook without a device: the jump plan sdp_solve would take for `sms`
// SMs (out: P, L, L0, squarings, reach of g, P2, major windows, chunks).
int32_t dp_test_sdp_jump_plan(int64_t n, const int32_t* a, int32_t k, int32_t sms, int64_t* out) {
  if (!a || !out || k < 1 || k > dpk::kSdpMaxK || sms < 2) return -1;
  for (int j = 0; j < k; ++j)
    if (a[j] < 1 || (j > 0 && a[j] >= a[j - 1])) return -1;
  return sdp_jump_plan(n, a, k, sms, out);
}

dp_status dp_test_sdp_jump(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, int32_t chunks,
                           int32_t* status_dev, void* stream) {
  if (!ST) return fail(DP_EINVAL, "dp_test_sdp_jump: ST is NULL");
  dp_status rc = sdp_validate(n, a, k, DP_OP_ADD_MOD32);
  if (rc != DP_OK) return rc;
  DevState* ds = nullptr;
  if ((rc = current_dev(&ds)) != DP_OK) return rc;
  return sdp_add_jump(ST, n, a, k, chunks, status_dev ? status_dev : ds->status, static_cast<cudaStream_t>(stream));
}

// Test hook: the device address mcm_solve_host would use for a host range
// (nullptr: the range goes through a device copy).
void* dp_test_host_range_device_address(const void* ptr, size_t bytes, int writable) {
  return host_range_device_address(ptr, bytes, writable != 0);
}

dp_status mcm_plan_create(int32_t batch, const int32_t* n_host, dp_cost ct, void** plan) {
  if (!plan || (batch > 0 && !n_host) || batch < 0) return fail(DP_EINVAL, "mcm_plan_create: bad arguments");
  if (ct != DP_COST_I32 && ct != DP_COST_I64) return fail(DP_EINVAL, "mcm_plan_create: unknown cost type");
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  auto* pl = new McmPlan();
  pl->ns.assign(n_host, n_host + batch);
  pl->i64 = ct == DP_COST_I64;
  rc = mcm_build_static(pl->ns, pl->i64, &pl->sp);
  if (rc != DP_OK) {
    delete pl;
    return rc;
  }
  pl->L = mcm_layout(*pl->sp);
  pl->device = ds->device;
  cudaError_t e = cudaMalloc(&pl->ws, pl->L.total);
  if (e != cudaSuccess) {
    delete pl;
    return fail_cuda(e, "mcm_plan_create: workspace");
  }
  pl->ws_bytes = pl->L.total;
  *plan = pl;
  return DP_OK;
}

dp_status mcm_solve_batched(void* plan, const int32_t* p_all, const int64_t* p_off, const int64_t* tab_off,
                            void* m_all, int16_t* s_all, int32_t* status_dev, void* stream) {
  auto* pl = static_cast<McmPlan*>(plan);
  if (!pl || !p_all || !p_off || !tab_off || !m_all || !s_all)
    return fail(DP_EINVAL, "mcm_solve_batched: NULL argument");
  return mcm_enqueue(*pl->sp, pl->L, pl->ws, p_all, p_off, tab_off, m_all, s_all, status_dev,
                     static_cast<cudaStream_t>(stream), 0, -1, pl->blocks_per_sm);
}

dp_status mcm_plan_autotune(void* plan, const int32_t* p_all, const int64_t* p_off, const int64_t* tab_off,
                            void* m_all, int16_t* s_all, int32_t* status_dev, void* stream) {
  auto* pl = static_cast<McmPlan*>(plan);
  if (!pl || !p_all || !p_off || !tab_off || !m_all || !s_all)
    return fail(DP_EINVAL, "mcm_plan_autotune: NULL argument");
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int occ = ds->occ[pl->i64 ? 1 : 0];
  cudaEvent_t e0, e1;
  cudaError_t e;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
    return fail_cuda(e, "mcm_plan_autotune: events");
  float best_ms = -1.0f;
  int best_lpp = pl->levels_per_part, best_bps = pl->blocks_per_sm;
  std::shared_ptr<McmStatic> best_sp = pl->sp;
  for (int lpp : {4, 8, 16}) {
    std::shared_ptr<McmStatic> sp;
    if (lpp == pl->levels_per_part) {
      sp = pl->sp;
    } else if ((rc = mcm_build_static(pl->ns, pl->i64, &sp, true, lpp)) != DP_OK) {
      break;
    }
    const McmLayout L = mcm_layout(*sp);
    if (L.total > pl->ws_bytes) {  // a finer queue needs more partial-minimum slots
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
        rc = fail_cuda(e, "mcm_plan_autotune: sync");
        break;
      }
      cudaFree(pl->ws);
      pl->ws = nullptr;
      pl->ws_bytes = 0;
      if ((e = cudaMalloc(&pl->ws, L.total)) != cudaSuccess) {
        rc = fail_cuda(e, "mcm_plan_autotune: workspace");
        break;
      }
      pl->ws_bytes = L.total;
    }
    for (int bps = 1; bps <= occ; ++bps) {
      float t = 0.0f, tmin = -1.0f;
      for (int rep = 0; rep < 2 && rc == DP_OK; ++rep) {
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) rc = fail_cuda(e, "mcm_plan_autotune: event");
        if (rc == DP_OK)
          rc = mcm_enqueue(*sp, L, pl->ws, p_all, p_off, tab_off, m_all, s_all, status_dev, st, 0, -1, bps);
        if (rc == DP_OK && (e = cudaEventRecord(e1, st)) != cudaSuccess) rc = fail_cuda(e, "mcm_plan_autotune: event");
        if (rc == DP_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = fail_cuda(e, "mcm_plan_autotune: sync");
        if (rc == DP_OK && (e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess)
          rc = fail_cuda(e, "mcm_plan_autotune: timing");
        if (rc == DP_OK && (tmin < 0.0f || t < tmin)) tmin = t;
      }
      if (rc != DP_OK) break;
      if (best_ms < 0.0f || tmin < best_ms) {
        best_ms = tmin;
        best_lpp = lpp;
        best_bps = bps;
        best_sp = sp;
      }
    }
    if (rc != DP_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DP_OK) return rc;
  pl->sp = best_sp;
  pl->L = mcm_layout(*best_sp);
  pl->levels_per_part = best_lpp;
  pl->blocks_per_sm = best_bps;
  // leave the tables solved with the chosen configuration
  return mcm_enqueue(*pl->sp, pl->L, pl->ws, p_all, p_off, tab_off, m_all, s_all, status_dev, st, 0, -1,
                     pl->blocks_per_sm);
}

dp_status mcm_plan_config(const void* plan, int32_t* levels_per_part, int32_t* blocks_per_sm) {
  const auto* pl = static_cast<const McmPlan*>(plan);
  if (!pl) return fail(DP_EINVAL, "mcm_plan_config: NULL plan");
  if (levels_per_part) *levels_per_part = pl->levels_per_part;
  if (blocks_per_sm) *blocks_per_sm = pl->blocks_per_sm;
  return DP_OK;
}

dp_status mcm_plan_destroy(void* plan) {
  auto* pl = static_cast<McmPlan*>(plan);
  if (!pl) return DP_OK;
  cudaFree(pl->ws);
  delete pl;
  return DP_OK;
}

// Number of queue entries of a batched plan (for tests and benchmarks).
int64_t dp_mcm_plan_tasks(void* plan) {
  auto* pl = static_cast<McmPlan*>(plan);
  return pl ? (int64_t)pl->sp->tasks.size() : -1;
}

dp_status sdp_solve(uint32_t* ST, int64_t n, const int32_t* a, int32_t k, dp_op op, int32_t* status_dev,
                    void* stream) {
  if (!ST) return fail(DP_EINVAL, "sdp_solve: ST is NULL");
  dp_status rc = sdp_validate(n, a, k, op);
  if (rc != DP_OK) return rc;
  if (n <= a[0]) return DP_OK;
  DevState* ds = nullptr;
  if ((rc = current_dev(&ds)) != DP_OK) return rc;
  if (op == DP_OP_ADD_MOD32) {
    // long tables: chunks from jumped windows, side by side (sdp_jump.cu)
    const int chunks = sdp_jump_chunks(n, a, k, ds->sms);
    if (chunks >= 2)
      return sdp_add_jump(ST, n, a, k, chunks, status_dev ? status_dev : ds->status,
                          static_cast<cudaStream_t>(stream));
  } else {
    // the same for min, with Boolean products (sdp_minjump.cu)
    const int chunks = sdp_min_jump_chunks(n, a, k, ds->sms);
    if (chunks >= 2)
      return sdp_min_jump(ST, n, a, k, chunks, status_dev ? status_dev : ds->status,
                          static_cast<cudaStream_t>(stream));
  }
  dpk::SdpLaunchArgs args{};
  args.insts = nullptr;
  args.one.st = ST;
  args.one.n = n;
  args.one.a = nullptr;
  args.one.k = k;
  args.kfull = k == dpk::kSdpMaxKRegs;
  args.ninst = 1;
  args.op = (int32_t)op;
  sdp_shape(a[0], a[k - 1], &args.threads, &args.ring_log2);
  args.status = status_dev ? status_dev : ds->status;
  for (int j = 0; j < k; ++j) args.one_offs[j] = a[j];
  const bool prof = profiling();
  if (prof) profile_mark(1, static_cast<cudaStream_t>(stream), false);
  cudaError_t e = dpk::launch_sdp(args, static_cast<cudaStream_t>(stream));
  if (prof) profile_mark(1, static_cast<cudaStream_t>(stream), true);
  if (e != cudaSuccess) return fail_cuda(e, "sdp_solve: launch");
  return DP_OK;
}

dp_status sdp_solve_host(uint32_t* ST_host, int64_t n, const int32_t* a, int32_t k, dp_op op, void* stream) {
  if (!ST_host) return fail(DP_EINVAL, "sdp_solve_host: ST is NULL");
  dp_status rc = sdp_validate(n, a, k, op);
  if (rc != DP_OK) return rc;
  if (n <= a[0]) return DP_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // A page-locked table the device may write is solved in place when the
  // window fits the shared-memory ring: the kernel then reads the table only
  // for the preset and writes every other cell once, so nothing is copied.
  // (A wider window is read from the table at every step and is staged in
  // device memory instead.)
  int threads = 0, ring_log2 = 0;
  sdp_shape(a[0], a[k - 1], &threads, &ring_log2);
  if (void* in_place = ring_log2 > 0 ? host_range_device_address(ST_host, (size_t)n * 4, true) : nullptr) {
    rc = sdp_solve(static_cast<uint32_t*>(in_place), n, a, k, op, nullptr, stream);
    if (rc == DP_OK) rc = dp_sync_status(stream, nullptr);
    if (rc == DP_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = fail_cuda(e, "sdp_solve_host: sync");
    return rc;
  }
  uint32_t* d = nullptr;
  e = cudaMallocAsync(reinterpret_cast<void**>(&d), (size_t)n * 4, st);
  if (e != cudaSuccess) return fail_cuda(e, "sdp_solve_host: allocation");
  if ((e = cudaMemcpyAsync(d, ST_host, (size_t)a[0] * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    rc = fail_cuda(e, "sdp_solve_host: upload");
  if (rc == DP_OK) rc = sdp_solve(d, n, a, k, op, nullptr, stream);
  if (rc == DP_OK && (e = cudaMemcpyAsync(ST_host, d, (size_t)n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    rc = fail_cuda(e, "sdp_solve_host: download");
  if (rc == DP_OK) rc = dp_sync_status(stream, nullptr);
  cudaFreeAsync(d, st);
  if (rc == DP_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = fail_cuda(e, "sdp_solve_host: sync");
  return rc;
}

dp_status sdp_plan_create(int32_t batch, const int64_t* n_host, const int32_t* k_host, const int32_t* a_host,
                          dp_op op, void** plan) {
  if (!plan || batch < 0 || (batch > 0 && (!n_host || !k_host || !a_host)))
    return fail(DP_EINVAL, "sdp_plan_create: bad arguments");
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  std::vector<dpk::SdpInstDev> insts((size_t)batch);
  int64_t aoff = 0;
  int kmax = 1, threads = 32, ring_log2 = 1;
  bool ring_ok = true, kfull = batch > 0;
  for (int b = 0; b < batch; ++b) {
    const int32_t* a = a_host + aoff;
    kfull = kfull && k_host[b] == dpk::kSdpMaxKRegs;
    if ((rc = sdp_validate(n_host[b], a, k_host[b], op)) != DP_OK) return fail(rc, "instance %d: %s", b, t_err.c_str());
    insts[b].n = n_host[b];
    insts[b].k = k_host[b];
    insts[b].a_off = (int32_t)aoff;
    kmax = std::max(kmax, (int)k_host[b]);
    int th, lg;
    sdp_shape(a[0], a[k_host[b] - 1], &th, &lg);
    threads = std::max(threads, th);
    aoff += k_host[b];
  }
  // one block shape for the launch: recompute the ring for the widest step
  for (int b = 0; b < batch; ++b) {
    const int32_t* a = a_host + insts[b].a_off;
    const int W = std::min(a[insts[b].k - 1], threads);
    int lg = 0;
    while ((1ll << lg) < (long long)a[0] + W) ++lg;
    if (lg > dpk::kSdpRingMaxLog2) ring_ok = false;
    ring_log2 = std::max(ring_log2, lg);
  }
  auto* pl = new SdpPlan();
  pl->device = ds->device;
  pl->batch = batch;
  pl->op = (int)op;
  pl->threads = threads;
  pl->ring_log2 = ring_ok ? ring_log2 : 0;
  pl->kmax = kmax;
  pl->kfull = kfull;
  cudaError_t e;
  if ((e = cudaMalloc(&pl->d_offs, std::max<int64_t>(aoff, 4) * 4)) != cudaSuccess ||
      (e = cudaMalloc(&pl->d_insts, std::max<size_t>(insts.size(), 1) * sizeof(dpk::SdpInstDev))) != cudaSuccess) {
    cudaFree(pl->d_offs);
    delete pl;
    return fail_cuda(e, "sdp_plan_create: allocation");
  }
  for (auto& in : insts) in.a = pl->d_offs + in.a_off;
  if ((aoff && (e = cudaMemcpy(pl->d_offs, a_host, aoff * 4, cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (batch && (e = cudaMemcpy(pl->d_insts, insts.data(), insts.size() * sizeof(dpk::SdpInstDev),
                                cudaMemcpyHostToDevice)) != cudaSuccess)) {
    cudaFree(pl->d_offs);
    cudaFree(pl->d_insts);
    delete pl;
    return fail_cuda(e, "sdp_plan_create: upload");
  }
  *plan = pl;
  return DP_OK;
}

dp_status sdp_solve_batched(void* plan, uint32_t* ST_all, const int64_t* st_off, int32_t* status_dev,
                            void* stream) {
  auto* pl = static_cast<SdpPlan*>(plan);
  if (!pl || !ST_all || !st_off) return fail(DP_EINVAL, "sdp_solve_batched: NULL argument");
  if (pl->batch == 0) return DP_OK;
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  dpk::SdpLaunchArgs args{};
  args.insts = pl->d_insts;
  args.one.k = pl->kmax;
  args.kfull = pl->kfull;
  args.ninst = pl->batch;
  args.op = pl->op;
  args.threads = pl->threads;
  args.ring_log2 = pl->ring_log2;
  args.st_all = ST_all;
  args.st_off = st_off;
  args.status = status_dev ? status_dev : ds->status;
  const bool prof = profiling();
  if (prof) profile_mark(1, static_cast<cudaStream_t>(stream), false);
  cudaError_t e = dpk::launch_sdp(args, static_cast<cudaStream_t>(stream));
  if (prof) profile_mark(1, static_cast<cudaStream_t>(stream), true);
  if (e != cudaSuccess) return fail_cuda(e, "sdp_solve_batched: launch");
  return DP_OK;
}

dp_status sdp_plan_destroy(void* plan) {
  auto* pl = static_cast<SdpPlan*>(plan);
  if (!pl) return DP_OK;
  cudaFree(pl->d_offs);
  cudaFree(pl->d_insts);
  delete pl;
  return DP_OK;
}

}  // extern "C"
