// serve.cu -- continuous-batching request server for MCM and S-DP solves.
//
// A scheduler thread owns the device work.  Each tick it
//   1. retires finished launches (event query), marking their requests done;
//   2. takes the admitted-but-not-started requests (up to max_batch), groups
//      them by kind (and cost type / operator) and enqueues one batched launch
//      per group on the stream of a small pool with the fewest launches in
//      flight, without waiting for the launches already on the GPU -- so
//      requests that arrive while others run start as soon as the scheduler
//      sees them and their work overlaps on the device.
// Admission (serve_submit) is by footprint: a request is refused with DP_EBUSY
// when the in-flight count or the bytes of device tables it would add exceed
// the configured caps; released requests return their bytes.
// Every batched launch computes exactly the same per-instance result as a
// solve on its own (the kernels never mix data between instances), so a
// result does not depend on which requests shared its launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <string>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

using namespace dph;

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct DeviceBlock {  // one output allocation shared by the requests of a launch
  void* ptr = nullptr;
  int refs = 0;
  std::vector<cudaEvent_t> readers;  // recorded on the streams of releases that named one
};

// Frees a block when its last request is released: on the server's first
// stream, after every event recorded by a release on the caller's stream, so
// that reads of the tables the caller enqueued before releasing complete
// before the memory can be handed to another launch.
void free_block(cudaStream_t st, DeviceBlock* b) {
  for (cudaEvent_t ev : b->readers) {
    cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
  }
  b->readers.clear();
  cudaFreeAsync(b->ptr, st);
}

struct Req {
  uint64_t ticket = 0;
  int kind = 0, cost = 0, op = 0;
  int64_t n = 0;
  std::vector<int32_t> dims, offs;
  std::vector<uint32_t> preset;
  int64_t footprint = 0;
  enum { QUEUED, RUNNING, DONE } state = QUEUED;
  int32_t status = DP_OK;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::shared_ptr<DeviceBlock> block;
  const void* m_dev = nullptr;
  const int16_t* s_dev = nullptr;
  const uint32_t* st_dev = nullptr;
};

struct Launch {
  cudaEvent_t ev = nullptr;
  int stream = 0;
  std::vector<Req*> reqs;
  void* pinned = nullptr;      // staging + status readback
  size_t pinned_bytes = 0;
  int32_t* status_host = nullptr;
  std::shared_ptr<McmStatic> sp;  // keeps the host queue alive until done
};

struct Server {
  dp_serve_config cfg{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Req*> queued;
  std::unordered_map<uint64_t, Req*> all;
  std::list<Launch*> running;
  int64_t resident = 0;
  int inflight = 0;
  uint64_t next_ticket = 1;
  std::vector<cudaStream_t> streams;
  int rr = 0;
  std::chrono::steady_clock::time_point t0;
  std::vector<std::pair<void*, size_t>> pinned_pool;  // free pinned buffers

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  void* get_pinned(size_t bytes, size_t* got) {
    for (size_t i = 0; i < pinned_pool.size(); ++i) {
      if (pinned_pool[i].second >= bytes) {
        void* p = pinned_pool[i].first;
        *got = pinned_pool[i].second;
        pinned_pool.erase(pinned_pool.begin() + i);
        return p;
      }
    }
    const size_t sz = std::max<size_t>(align_up(bytes, 1 << 16), 1 << 20);
    void* p = nullptr;
    if (cudaHostAlloc(&p, sz, cudaHostAllocDefault) != cudaSuccess) return nullptr;
    *got = sz;
    return p;
  }
  void put_pinned(void* p, size_t sz) { pinned_pool.emplace_back(p, sz); }
};

int64_t mcm_footprint(int64_t n, int cost) {
  const int64_t es = cost == DP_COST_I64 ? 8 : 4;
  // tables (m + s) plus the solve's workspace: two packed panels per cell and
  // the partial accumulators (8 bytes per cell of a split tile, at most n^2/2)
  return n * n * (es + 2) + n * n * es * 2 + n * n * 4 + (1 << 20);
}

int64_t sdp_footprint(int64_t n) { return n * 4 + (1 << 16); }

// ---- launch builders (called by the scheduler thread with the lock released) ----

dp_status launch_mcm_group(Server* S, const std::vector<Req*>& reqs, bool i64, Launch* L) {
  std::vector<int32_t> ns;
  for (Req* r : reqs) ns.push_back((int32_t)r->n);
  std::shared_ptr<McmStatic> sp;
  dp_status rc = mcm_build_static(ns, i64, &sp, /*upload=*/false);
  if (rc != DP_OK) return rc;
  sp->owns_device = false;
  const McmLayout lay = mcm_layout(*sp);
  const size_t es = i64 ? 8 : 4;
  // outputs: m tables then s tables, same element offsets
  std::vector<int64_t> tab_off(reqs.size()), p_off(reqs.size());
  int64_t cells = 0, dims = 0;
  for (size_t b = 0; b < reqs.size(); ++b) {
    tab_off[b] = cells;
    cells += reqs[b]->n * reqs[b]->n;
    cells = (int64_t)align_up((size_t)cells, 64);
    p_off[b] = dims;
    dims += reqs[b]->n + 1;
  }
  const size_t m_bytes = align_up((size_t)cells * es, 256), s_bytes = align_up((size_t)cells * 2, 256);
  // inputs staged in pinned memory: dims | p_off | tab_off | tasks | accslot | insts
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = align_up(off + std::max<size_t>(b, 16), 256); return o; };
  const size_t o_dims = take((size_t)dims * 4), o_poff = take(reqs.size() * 8), o_toff = take(reqs.size() * 8);
  const size_t o_tasks = take(sp->tasks.size() * sizeof(dpk::McmTask));
  const size_t o_acc = take(sp->accslot.size() * 4);
  const size_t o_insts = take(sp->insts.size() * sizeof(dpk::McmInstDev));
  const size_t in_bytes = off;
  const size_t o_status = take(16);
  size_t got = 0;
  uint8_t* hp = static_cast<uint8_t*>(S->get_pinned(off, &got));
  if (!hp) return fail(DP_ENOMEM, "serve: pinned staging allocation failed");
  L->pinned = hp;
  L->pinned_bytes = got;
  L->status_host = reinterpret_cast<int32_t*>(hp + o_status);
  *L->status_host = 0;
  for (size_t b = 0; b < reqs.size(); ++b)
    memcpy(hp + o_dims + p_off[b] * 4, reqs[b]->dims.data(), (reqs[b]->n + 1) * 4);
  memcpy(hp + o_poff, p_off.data(), reqs.size() * 8);
  memcpy(hp + o_toff, tab_off.data(), reqs.size() * 8);
  memcpy(hp + o_tasks, sp->tasks.data(), sp->tasks.size() * sizeof(dpk::McmTask));
  memcpy(hp + o_acc, sp->accslot.data(), sp->accslot.size() * 4);
  memcpy(hp + o_insts, sp->insts.data(), sp->insts.size() * sizeof(dpk::McmInstDev));

  cudaStream_t st = S->streams[L->stream];
  auto block = std::make_shared<DeviceBlock>();
  cudaError_t e = cudaMallocAsync(&block->ptr, m_bytes + s_bytes, st);
  if (e != cudaSuccess) return fail_cuda(e, "serve: table allocation");
  uint8_t* ws = nullptr;
  e = cudaMallocAsync(reinterpret_cast<void**>(&ws), in_bytes + 256 + lay.total, st);
  if (e != cudaSuccess) return fail_cuda(e, "serve: workspace allocation");
  uint8_t* scratch = ws + in_bytes + 256;
  int32_t* d_status = reinterpret_cast<int32_t*>(ws + in_bytes);
  sp->d_tasks = reinterpret_cast<dpk::McmTask*>(ws + o_tasks);
  sp->d_accslot = reinterpret_cast<int32_t*>(ws + o_acc);
  sp->d_insts = reinterpret_cast<dpk::McmInstDev*>(ws + o_insts);

  if ((e = cudaMemcpyAsync(ws, hp, in_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail_cuda(e, "serve: upload");
  if ((e = cudaMemsetAsync(d_status, 0, 4, st)) != cudaSuccess) return fail_cuda(e, "serve: status");
  uint8_t* m_all = static_cast<uint8_t*>(block->ptr);
  int16_t* s_all = reinterpret_cast<int16_t*>(m_all + m_bytes);
  // one resident block per SM: the S-DP blocks of concurrent launches then
  // still fit beside the MCM ones
  rc = mcm_enqueue(*sp, lay, scratch, reinterpret_cast<int32_t*>(ws + o_dims),
                   reinterpret_cast<int64_t*>(ws + o_poff), reinterpret_cast<int64_t*>(ws + o_toff), m_all, s_all,
                   d_status, st, 0, -1, 1);
  if (rc != DP_OK) return rc;
  if ((e = cudaMemcpyAsync(L->status_host, d_status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail_cuda(e, "serve: status readback");
  cudaFreeAsync(ws, st);
  for (size_t b = 0; b < reqs.size(); ++b) {
    reqs[b]->block = block;
    reqs[b]->m_dev = m_all + tab_off[b] * es;
    reqs[b]->s_dev = s_all + tab_off[b];
  }
  block->refs = (int)reqs.size();
  L->sp = sp;
  return DP_OK;
}

// A group of S-DP requests with one operator.  Requests long enough for the
// chunked paths of sdp_solve (sdp_jump.cu for +, sdp_minjump.cu for min; the
// same cost models decide) run through those, spread over the SMs; the
// others share one launch of the S-DP kernel, one block each.  Everything is
// enqueued on the launch's stream, so one event covers the group.
dp_status launch_sdp_group(Server* S, const std::vector<Req*>& reqs, int op, Launch* L) {
  int threads = 32, kmax = 1, ring_log2 = 1;
  DevState* ds = nullptr;
  dp_status rc0 = current_dev(&ds);
  if (rc0 != DP_OK) return rc0;
  std::vector<int> chunks(reqs.size(), 0);
  std::vector<size_t> bat;  // requests of the shared launch
  for (size_t b = 0; b < reqs.size(); ++b) {
    const Req* r = reqs[b];
    const int k = (int)r->offs.size();
    if (r->n > r->offs[0])
      chunks[b] = op == DP_OP_MIN ? sdp_min_jump_chunks(r->n, r->offs.data(), k, ds->sms)
                                  : sdp_jump_chunks(r->n, r->offs.data(), k, ds->sms);
    if (chunks[b] < 2) bat.push_back(b);
  }
  bool ring_ok = true, kfull = !bat.empty();
  std::vector<int64_t> st_off(reqs.size());
  int64_t cells = 0, noffs = 0;
  for (size_t b = 0; b < reqs.size(); ++b) {
    const Req* r = reqs[b];
    st_off[b] = cells;
    cells = (int64_t)align_up((size_t)(cells + std::max<int64_t>(r->n, r->offs[0])), 64);
    noffs += (int64_t)r->offs.size();
  }
  for (size_t b : bat) {
    const Req* r = reqs[b];
    kmax = std::max(kmax, (int)r->offs.size());
    kfull = kfull && (int)r->offs.size() == dpk::kSdpMaxKRegs;
    int th, lg;
    sdp_shape(r->offs[0], r->offs.back(), &th, &lg);
    threads = std::max(threads, th);
  }
  for (size_t b : bat) {
    const Req* r = reqs[b];
    const int W = std::min<int>(r->offs.back(), threads);
    int lg = 0;
    while ((1ll << lg) < (long long)r->offs[0] + W) ++lg;
    if (lg > dpk::kSdpRingMaxLog2) ring_ok = false;
    ring_log2 = std::max(ring_log2, lg);
  }
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off = align_up(off + std::max<size_t>(b, 16), 256); return o; };
  const size_t o_offs = take((size_t)noffs * 4), o_insts = take(std::max<size_t>(bat.size(), 1) * sizeof(dpk::SdpInstDev));
  const size_t o_stoff = take(std::max<size_t>(bat.size(), 1) * 8);
  std::vector<size_t> o_pre(reqs.size());
  for (size_t b = 0; b < reqs.size(); ++b) o_pre[b] = take(reqs[b]->offs[0] * 4);
  const size_t in_bytes = off;
  const size_t o_status = take(16);
  size_t got = 0;
  uint8_t* hp = static_cast<uint8_t*>(S->get_pinned(off, &got));
  if (!hp) return fail(DP_ENOMEM, "serve: pinned staging allocation failed");
  L->pinned = hp;
  L->pinned_bytes = got;
  L->status_host = reinterpret_cast<int32_t*>(hp + o_status);
  *L->status_host = 0;

  cudaStream_t st = S->streams[L->stream];
  auto block = std::make_shared<DeviceBlock>();
  cudaError_t e = cudaMallocAsync(&block->ptr, std::max<int64_t>(cells, 16) * 4, st);
  if (e != cudaSuccess) return fail_cuda(e, "serve: table allocation");
  uint8_t* ws = nullptr;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(&ws), in_bytes + 256, st)) != cudaSuccess)
    return fail_cuda(e, "serve: workspace allocation");
  std::vector<dpk::SdpInstDev> insts(bat.size());
  std::vector<int64_t> bat_off(bat.size());
  std::vector<int64_t> a_at(reqs.size());
  int64_t ao = 0;
  for (size_t b = 0; b < reqs.size(); ++b) {
    memcpy(hp + o_offs + ao * 4, reqs[b]->offs.data(), reqs[b]->offs.size() * 4);
    a_at[b] = ao;
    ao += (int64_t)reqs[b]->offs.size();
    memcpy(hp + o_pre[b], reqs[b]->preset.data(), reqs[b]->offs[0] * 4);
  }
  for (size_t i = 0; i < bat.size(); ++i) {
    const size_t b = bat[i];
    insts[i].st = nullptr;
    insts[i].n = reqs[b]->n;
    insts[i].k = (int32_t)reqs[b]->offs.size();
    insts[i].a = reinterpret_cast<const int32_t*>(ws + o_offs) + a_at[b];
    insts[i].a_off = (int32_t)a_at[b];
    bat_off[i] = st_off[b];
  }
  memcpy(hp + o_insts, insts.data(), insts.size() * sizeof(dpk::SdpInstDev));
  memcpy(hp + o_stoff, bat_off.data(), bat_off.size() * 8);
  if ((e = cudaMemcpyAsync(ws, hp, in_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return fail_cuda(e, "serve: upload");
  int32_t* d_status = reinterpret_cast<int32_t*>(ws + in_bytes);
  if ((e = cudaMemsetAsync(d_status, 0, 4, st)) != cudaSuccess) return fail_cuda(e, "serve: status");
  uint32_t* st_all = static_cast<uint32_t*>(block->ptr);
  for (size_t b = 0; b < reqs.size(); ++b) {
    const int64_t cnt = std::min<int64_t>(reqs[b]->offs[0], reqs[b]->n);
    if (cnt > 0 && (e = cudaMemcpyAsync(st_all + st_off[b], ws + o_pre[b], cnt * 4, cudaMemcpyDeviceToDevice, st)) !=
                       cudaSuccess)
      return fail_cuda(e, "serve: preset copy");
  }
  if (!bat.empty()) {
    dpk::SdpLaunchArgs args{};
    args.insts = reinterpret_cast<const dpk::SdpInstDev*>(ws + o_insts);
    args.one.k = kmax;
    args.kfull = kfull;
    args.ninst = (int32_t)bat.size();
    args.op = op;
    args.threads = threads;
    args.ring_log2 = ring_ok ? ring_log2 : 0;
    args.st_all = st_all;
    args.st_off = reinterpret_cast<const int64_t*>(ws + o_stoff);
    args.status = d_status;
    if ((e = dpk::launch_sdp(args, st)) != cudaSuccess) return fail_cuda(e, "serve: S-DP launch");
  }
  for (size_t b = 0; b < reqs.size(); ++b) {
    if (chunks[b] < 2) continue;
    const Req* r = reqs[b];
    const dp_status rc = op == DP_OP_MIN
                             ? sdp_min_jump(st_all + st_off[b], r->n, r->offs.data(), (int32_t)r->offs.size(), chunks[b],
                                            d_status, st)
                             : sdp_add_jump(st_all + st_off[b], r->n, r->offs.data(), (int32_t)r->offs.size(), chunks[b],
                                            d_status, st);
    if (rc != DP_OK) return rc;
  }
  if ((e = cudaMemcpyAsync(L->status_host, d_status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return fail_cuda(e, "serve: status readback");
  cudaFreeAsync(ws, st);
  for (size_t b = 0; b < reqs.size(); ++b) {
    reqs[b]->block = block;
    reqs[b]->st_dev = st_all + st_off[b];
  }
  block->refs = (int)reqs.size();
  return DP_OK;
}

void scheduler(Server* S) {
  cudaSetDevice(S->cfg.device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    // 1. retire finished launches
    for (auto it = S->running.begin(); it != S->running.end();) {
      Launch* L = *it;
      const cudaError_t q = cudaEventQuery(L->ev);
      if (q == cudaErrorNotReady) {
        ++it;
        continue;
      }
      const double t = S->now();
      const int32_t dev_status = q == cudaSuccess ? *L->status_host : (int32_t)DP_ECUDA;
      for (Req* r : L->reqs) {
        r->state = Req::DONE;
        r->status = dev_status;
        r->t_done = t;
      }
      cudaEventDestroy(L->ev);
      S->put_pinned(L->pinned, L->pinned_bytes);
      delete L;
      it = S->running.erase(it);
    }
    if (S->stop && S->queued.empty() && S->running.empty()) break;
    // 2. start queued requests
    if (!S->queued.empty()) {
      std::vector<Req*> take;
      while (!S->queued.empty() && (int)take.size() < std::max(1, S->cfg.max_batch)) {
        take.push_back(S->queued.front());
        S->queued.pop_front();
      }
      const double t = S->now();
      for (Req* r : take) {
        r->state = Req::RUNNING;
        r->t_start = t;
      }
      lk.unlock();
      // group by kind and cost type / operator
      std::vector<Req*> groups[4];
      for (Req* r : take) {
        const int g = r->kind == DP_REQ_MCM ? (r->cost == DP_COST_I64 ? 1 : 0) : (r->op == DP_OP_MIN ? 2 : 3);
        groups[g].push_back(r);
      }
      std::vector<Launch*> made;
      // launches in flight per stream (only this thread changes `running`)
      std::vector<int> busy(S->streams.size(), 0);
      for (const Launch* R : S->running) ++busy[R->stream];
      for (int g = 0; g < 4; ++g) {
        if (groups[g].empty()) continue;
        Launch* L = new Launch();
        L->reqs = groups[g];
        // the stream with the fewest launches in flight (ties: round robin),
        // so that a short launch queues behind a long one only when every
        // stream is busy
        const int ns = (int)S->streams.size();
        int pick = S->rr;
        for (int i = 1; i < ns; ++i) {
          const int c = (S->rr + i) % ns;
          if (busy[c] < busy[pick]) pick = c;
        }
        L->stream = pick;
        ++busy[pick];
        S->rr = (pick + 1) % ns;
        dp_status rc = g < 2 ? launch_mcm_group(S, groups[g], g == 1, L)
                             : launch_sdp_group(S, groups[g], g == 2 ? DP_OP_MIN : DP_OP_ADD_MOD32, L);
        if (rc == DP_OK && cudaEventCreateWithFlags(&L->ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventRecord(L->ev, S->streams[L->stream]) == cudaSuccess) {
          made.push_back(L);
        } else {
          // the launch could not be enqueued: fail its requests now
          cudaStreamSynchronize(S->streams[L->stream]);
          std::lock_guard<std::mutex> g2(S->mu);
          for (Req* r : L->reqs) {
            r->state = Req::DONE;
            r->status = rc != DP_OK ? rc : DP_ECUDA;
            r->t_done = S->now();
          }
          if (L->pinned) S->put_pinned(L->pinned, L->pinned_bytes);
          if (L->ev) cudaEventDestroy(L->ev);
          delete L;
        }
      }
      lk.lock();
      for (Launch* L : made) S->running.push_back(L);
      continue;
    }
    // 3. idle: wait for a submission, or poll completions shortly
    if (S->running.empty())
      S->cv.wait(lk, [&] { return S->stop || !S->queued.empty(); });
    else
      S->cv.wait_for(lk, std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

dp_status serve_create(const dp_serve_config* cfg, void** srv) {
  if (!cfg || !srv) return fail(DP_EINVAL, "serve_create: NULL argument");
  if (cfg->num_streams < 1 || cfg->max_inflight < 1 || cfg->hbm_cap_bytes <= 0)
    return fail(DP_EINVAL, "serve_create: num_streams, max_inflight and hbm_cap_bytes must be positive");
  cudaError_t e = cudaSetDevice(cfg->device);
  if (e != cudaSuccess) return fail_cuda(e, "serve_create: cudaSetDevice");
  DevState* ds = nullptr;
  dp_status rc = current_dev(&ds);
  if (rc != DP_OK) return rc;
  auto* S = new Server();
  S->cfg = *cfg;
  S->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < cfg->num_streams; ++i) {
    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
      for (auto s : S->streams) cudaStreamDestroy(s);
      delete S;
      return fail_cuda(e, "serve_create: stream");
    }
    S->streams.push_back(st);
  }
  S->th = std::thread(scheduler, S);
  *srv = S;
  return DP_OK;
}

dp_status serve_submit(void* srv, const dp_request* req, uint64_t* ticket) {
  auto* S = static_cast<Server*>(srv);
  if (!S || !req || !ticket) return fail(DP_EINVAL, "serve_submit: NULL argument");
  auto r = std::make_unique<Req>();
  r->kind = req->kind;
  r->n = req->n;
  if (req->kind == DP_REQ_MCM) {
    if (req->n < 1 || req->n > 32767 || !req->dims) return fail(DP_EINVAL, "serve_submit: bad MCM request");
    if (req->cost != DP_COST_I32 && req->cost != DP_COST_I64) return fail(DP_EINVAL, "serve_submit: bad cost type");
    r->cost = req->cost;
    r->dims.assign(req->dims, req->dims + req->n + 1);
    for (int32_t d : r->dims)
      if (d < 1) return fail(DP_EINVAL, "serve_submit: dimension < 1");
    r->footprint = mcm_footprint(req->n, req->cost);
  } else if (req->kind == DP_REQ_SDP) {
    dp_status rc = sdp_validate(req->n, req->offsets, req->k, req->op);
    if (rc != DP_OK) return rc;
    if (!req->preset) return fail(DP_EINVAL, "serve_submit: preset is NULL");
    r->op = req->op;
    r->offs.assign(req->offsets, req->offsets + req->k);
    r->preset.assign(req->preset, req->preset + req->offsets[0]);
    r->footprint = sdp_footprint(std::max<int64_t>(req->n, req->offsets[0]));
  } else {
    return fail(DP_EINVAL, "serve_submit: unknown request kind %d", req->kind);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return fail(DP_EINVAL, "serve_submit: server is shutting down");
  if (S->inflight + 1 > S->cfg.max_inflight || S->resident + r->footprint > S->cfg.hbm_cap_bytes)
    return fail(DP_EBUSY, "serve_submit: at capacity (%d in flight, %lld bytes resident)", S->inflight,
                (long long)S->resident);
  r->ticket = S->next_ticket++;
  r->t_submit = S->now();
  S->inflight += 1;
  S->resident += r->footprint;
  *ticket = r->ticket;
  Req* raw = r.release();
  S->all.emplace(raw->ticket, raw);
  S->queued.push_back(raw);
  S->cv.notify_one();
  return DP_OK;
}

dp_status serve_poll(void* srv, uint64_t ticket, dp_result* out) {
  auto* S = static_cast<Server*>(srv);
  if (!S || !out) return fail(DP_EINVAL, "serve_poll: NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(DP_EINVAL, "serve_poll: unknown ticket %llu", (unsigned long long)ticket);
  Req* r = it->second;
  if (r->state != Req::DONE) return DP_EPENDING;
  out->status = r->status;
  out->kind = r->kind;
  out->n = r->n;
  out->m_dev = r->m_dev;
  out->s_dev = r->s_dev;
  out->st_dev = r->st_dev;
  out->t_submit = r->t_submit;
  out->t_start = r->t_start;
  out->t_done = r->t_done;
  return DP_OK;
}

namespace {
dp_status release_impl(Server* S, uint64_t ticket, bool after_stream, cudaStream_t reader) {
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(DP_EINVAL, "serve_release: unknown ticket %llu", (unsigned long long)ticket);
  Req* r = it->second;
  if (r->state != Req::DONE) return fail(DP_EPENDING, "serve_release: request still running");
  if (r->block) {
    if (after_stream) {
      cudaEvent_t ev = nullptr;
      cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess && (e = cudaEventRecord(ev, reader)) != cudaSuccess) cudaEventDestroy(ev);
      if (e != cudaSuccess) return fail_cuda(e, "serve_release_stream: event on the caller's stream");
      r->block->readers.push_back(ev);
    }
    if (--r->block->refs == 0) free_block(S->streams[0], r->block.get());
  }
  S->resident -= r->footprint;
  S->inflight -= 1;
  S->all.erase(it);
  delete r;
  return DP_OK;
}
}  // namespace

dp_status serve_release(void* srv, uint64_t ticket) {
  auto* S = static_cast<Server*>(srv);
  if (!S) return fail(DP_EINVAL, "serve_release: NULL server");
  return release_impl(S, ticket, false, nullptr);
}

dp_status serve_release_stream(void* srv, uint64_t ticket, void* stream) {
  auto* S = static_cast<Server*>(srv);
  if (!S) return fail(DP_EINVAL, "serve_release_stream: NULL server");
  return release_impl(S, ticket, true, static_cast<cudaStream_t>(stream));
}

double serve_now(void* srv) {
  auto* S = static_cast<Server*>(srv);
  return S ? S->now() : 0.0;
}

dp_status serve_destroy(void* srv) {
  auto* S = static_cast<Server*>(srv);
  if (!S) return DP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  S->th.join();
  for (auto& kv : S->all) {
    Req* r = kv.second;
    if (r->block && --r->block->refs == 0) free_block(S->streams[0], r->block.get());
    delete r;
  }
  for (auto s : S->streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (auto& p : S->pinned_pool) cudaFreeHost(p.first);
  delete S;
  return DP_OK;
}

}  // extern "C"
