// vd_serve.cu -- a server of dJFA steps for many resident simulations, with
// continuous batching.
//
// Simulations live on the device for their whole life (maps, seeds, table in
// one allocation each), admitted while an HBM budget allows.  Step requests
// queue in arrival order; two launch lanes (each its own stream, plan slot and
// completion event) take turns: whenever a lane is free, it takes every queued
// request whose simulation has no step in flight (at most one per simulation,
// up to max_batch) and launches that subset as one batched step.  Requests that
// arrive while a lane runs are admitted by the other lane as soon as it frees,
// so consecutive batches overlap on the device.  A simulation's result does not
// depend on the mix: each runs the same per-pixel code on its own state, and
// its moves are drawn from its own SplitMix64 stream (stream id = its slot).
#include <chrono>
#include <deque>
#include <thread>

#include "vd_batch_engine.cuh"

namespace {

struct Request {
  int64_t ticket;
  int sim;
  double t_arrive;
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  vdb::PlanSlot slot;
  bool busy = false;
  std::vector<Request> reqs;
};

}  // namespace

struct vd_server {
  int device = 0;
  int max_sims = 0;
  int64_t budget = 0, used = 0;
  int32_t d_max = 0, vn_waves = 2, metric = 0, max_disp = 0;
  uint64_t rng_seed = 0;
  // 8 rows a thread: saturation 8.6k -> 9.2k steps/s at 1000 simulations,
  // p50 / p99 at 2k and 5k requests a second about unchanged
  int rows_per_thread = 8;
  int max_batch = 1 << 30;
  std::vector<vdb::SimDesc> sims;
  std::vector<char> live, in_flight;
  std::vector<void*> mem;
  std::vector<int64_t> bytes;
  vdb::SimDesc* d_sims = nullptr;
  vdb::Barrier* bar = nullptr;  // unused by the per-round kernels; kept valid for BatchArgs
  cudaStream_t admin = nullptr;
  vdb::PlanSlot admin_slot;
  Lane lanes[2];
  std::deque<Request> pending;
  std::vector<int64_t> done_ticket;
  std::vector<double> done_latency;
  std::vector<int32_t> done_sim;
  int64_t next_ticket = 0;
  int64_t launches = 0;
  int64_t steps_done = 0;
  std::chrono::steady_clock::time_point t0;
};

namespace {

double now_s(const vd_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

int64_t sim_bytes(int w, int h, int n) {
  const int64_t pitch = (w + 31) / 32 * 32;
  // maps, seeds, the pass table, the position table and the seed entries of
  // the wide position-tagged layouts (8 bytes each, after an 8-byte alignment)
  return 2 * pitch * h * 4 + static_cast<int64_t>(n) * 8 + (static_cast<int64_t>(n) + 1) * (8 + 4 + 8) + 8 + 256;
}

void server_free(vd_server* s) {
  for (Lane& l : s->lanes) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    l.slot.release();
    if (l.done) cudaEventDestroy(l.done);
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  if (s->admin) cudaStreamSynchronize(s->admin);
  s->admin_slot.release();
  if (s->admin) cudaStreamDestroy(s->admin);
  for (void* p : s->mem) cudaFree(p);
  cudaFree(s->d_sims);
  cudaFree(s->bar);
}

// Reaps finished lanes; returns the number of requests completed.
int reap(vd_server* s, int* completed) {
  *completed = 0;
  for (Lane& l : s->lanes) {
    if (!l.busy) continue;
    const cudaError_t q = cudaEventQuery(l.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return vd_cuda_check(q, "server lane");
    const double t = now_s(s);
    for (const Request& r : l.reqs) {
      s->in_flight[r.sim] = 0;
      s->done_ticket.push_back(r.ticket);
      s->done_latency.push_back(t - r.t_arrive);
      s->done_sim.push_back(r.sim);
    }
    *completed += static_cast<int>(l.reqs.size());
    s->steps_done += static_cast<int64_t>(l.reqs.size());
    l.reqs.clear();
    l.busy = false;
  }
  return VD_OK;
}

// Fills free lanes with queued requests whose simulations are idle.
int admit(vd_server* s) {
  for (Lane& l : s->lanes) {
    if (l.busy || s->pending.empty()) continue;
    std::vector<int> act;
    std::deque<Request> keep;
    while (!s->pending.empty()) {
      Request r = s->pending.front();
      s->pending.pop_front();
      if (s->in_flight[r.sim] || static_cast<int>(act.size()) >= s->max_batch) {
        keep.push_back(r);
        continue;
      }
      s->in_flight[r.sim] = 1;
      act.push_back(r.sim);
      l.reqs.push_back(r);
    }
    s->pending.swap(keep);
    if (act.empty()) continue;
    vdb::HostPlan p = vdb::make_plan(s->sims, act, 0, s->rows_per_thread);
    vdb::BatchArgs A = vdb::make_args(s->rows_per_thread, s->bar, 0, 0, 1);
    A.sched = 0;
    A.mark = 1;
    A.move = 1;
    A.max_disp = s->max_disp;
    A.rng_seed = s->rng_seed;
    int rc = vdb::plan_upload(l.slot, p, s->d_sims, l.stream, &A);
    if (!rc) rc = vdb::launch_rounds(p, A, s->metric, l.stream, &s->launches);
    if (!rc) rc = vd_cuda_check(cudaEventRecord(l.done, l.stream), "event");
    if (rc) return rc;
    l.busy = true;
  }
  return VD_OK;
}

}  // namespace

#define VD_CHECK_SERVER(s) \
  if (!(s)) return vd_fail(VD_EINVAL, "null server")

extern "C" vd_server* vd_server_create(int32_t max_sims, int64_t hbm_budget_bytes, int32_t d_max, int32_t vn_waves,
                                       int32_t metric, int32_t max_disp, uint64_t rng_seed) {
  if (max_sims < 1 || hbm_budget_bytes < 1 || d_max < 0 || vn_waves < 0 || max_disp < 0 || max_disp > VD_MAX_SIDE ||
      (metric != VD_METRIC_EUCLID && metric != VD_METRIC_MANHATTAN)) {
    vd_fail(VD_EINVAL, "bad server parameters");
    return nullptr;
  }
  vd_server* s = new vd_server();
  cudaGetDevice(&s->device);
  s->max_sims = max_sims;
  s->budget = hbm_budget_bytes;
  s->d_max = d_max;
  s->vn_waves = vn_waves;
  s->metric = metric;
  s->max_disp = max_disp;
  s->rng_seed = rng_seed;
  s->sims.resize(max_sims);
  std::memset(s->sims.data(), 0, sizeof(vdb::SimDesc) * max_sims);
  s->live.assign(max_sims, 0);
  s->in_flight.assign(max_sims, 0);
  s->mem.assign(max_sims, nullptr);
  s->bytes.assign(max_sims, 0);
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&s->d_sims), sizeof(vdb::SimDesc) * max_sims);
  if (e == cudaSuccess) e = cudaMemset(s->d_sims, 0, sizeof(vdb::SimDesc) * max_sims);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s->bar), sizeof(vdb::Barrier));
  if (e == cudaSuccess) e = cudaMemset(s->bar, 0, sizeof(vdb::Barrier));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking);
  for (Lane& l : s->lanes) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    vd_cuda_check(e, "server creation");
    server_free(s);
    delete s;
    return nullptr;
  }
  return s;
}

extern "C" int vd_server_destroy(vd_server* s) {
  if (!s) return VD_OK;
  server_free(s);
  delete s;
  return VD_OK;
}

extern "C" int32_t vd_server_add_sim(vd_server* s, int32_t w, int32_t h, int32_t n, const int32_t* xy) {
  VD_CHECK_SERVER(s);
  if (w < 1 || w > VD_MAX_SIDE || h < 1 || h > VD_MAX_SIDE || n < 1 || !xy)
    return vd_fail(VD_EINVAL, "bad simulation %dx%d with %d seeds", w, h, n);
  for (int k = 0; k < n; ++k)
    if (xy[2 * k] < 0 || xy[2 * k] >= w || xy[2 * k + 1] < 0 || xy[2 * k + 1] >= h)
      return vd_fail(VD_EINVAL, "seed %d outside the %dx%d grid", k, w, h);
  int slot = -1;
  for (int i = 0; i < s->max_sims && slot < 0; ++i)
    if (!s->live[i]) slot = i;
  if (slot < 0) return vd_fail(VD_EBUSY, "all %d simulation slots are live", s->max_sims);
  const int64_t need = sim_bytes(w, h, n);
  if (s->used + need > s->budget)
    return vd_fail(VD_EBUSY, "admission refused: %lld bytes over the HBM budget (%lld of %lld in use)",
                   static_cast<long long>(s->used + need - s->budget), static_cast<long long>(s->used),
                   static_cast<long long>(s->budget));
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return vd_fail(VD_ENOMEM, "device allocation of %lld bytes failed", static_cast<long long>(need));
  }
  vdb::SimDesc d;
  std::memset(&d, 0, sizeof(d));
  d.w = w;
  d.h = h;
  d.n = n;
  d.pitch = (w + 31) / 32 * 32;
  const size_t map_elems = static_cast<size_t>(d.pitch) * h;
  char* base = static_cast<char*>(mem);
  d.map[0] = reinterpret_cast<int32_t*>(base);
  d.map[1] = d.map[0] + map_elems;
  d.seeds = reinterpret_cast<int2*>(d.map[1] + map_elems);
  d.table = d.seeds + n;
  d.ptable = reinterpret_cast<uint32_t*>(d.table + (n + 1));
  {
    const uintptr_t end = reinterpret_cast<uintptr_t>(d.ptable + (n + 1));
    d.pkf = reinterpret_cast<uint2*>((end + 7) & ~static_cast<uintptr_t>(7));
  }
  d.cur = 0;
  d.step = 0;
  d.n_pass[0] = vdi::fill_schedule(vdi::djfa_first_step(w, h, n, s->d_max), s->vn_waves, 0, d.ks[0], d.nbs[0],
                                   vdb::kMaxPasses);
  d.n_pass[1] = vdi::fill_schedule(vdi::jfa_first_step(w, h), 0, 0, d.ks[1], d.nbs[1], vdb::kMaxPasses);
  vdb::set_clamp(d, 0, s->metric, -1);
  vdb::set_clamp(d, 1, s->metric, -1);
  cudaStream_t st = s->admin;
  int rc = vd_cuda_check(cudaMemcpyAsync(d.seeds, xy, sizeof(int2) * n, cudaMemcpyHostToDevice, st), "copy seeds");
  if (!rc) rc = vdi::launch_build_table(d.seeds, n, d.table, d.ptable, st);
  if (!rc) rc = vdi::launch_fill(d.map[0], 2 * static_cast<int64_t>(map_elems), -1, st);
  if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(s->d_sims + slot, &d, sizeof(d), cudaMemcpyHostToDevice, st), "descriptor");
  // frame 0: a full JFA frame for the new simulation alone
  std::vector<vdb::SimDesc> one(s->sims);
  one[slot] = d;
  vdb::HostPlan p = vdb::make_plan(one, std::vector<int>{slot}, 1, s->rows_per_thread);
  vdb::BatchArgs A = vdb::make_args(s->rows_per_thread, s->bar, 0, 0, 1);
  A.sched = 1;
  if (!rc) rc = vdb::plan_upload(s->admin_slot, p, s->d_sims, st, &A);
  if (!rc) rc = vdb::launch_rounds(p, A, s->metric, st, &s->launches);
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(st), "admit");
  if (rc) {
    cudaFree(mem);
    return rc;
  }
  s->sims[slot] = d;
  s->live[slot] = 1;
  s->mem[slot] = mem;
  s->bytes[slot] = need;
  s->used += need;
  return slot;
}

extern "C" int vd_server_remove_sim(vd_server* s, int32_t sim) {
  VD_CHECK_SERVER(s);
  if (sim < 0 || sim >= s->max_sims || !s->live[sim]) return vd_fail(VD_ENOTFOUND, "no live simulation %d", sim);
  if (s->in_flight[sim]) return vd_fail(VD_EBUSY, "simulation %d has a step in flight", sim);
  for (const Request& r : s->pending)
    if (r.sim == sim) return vd_fail(VD_EBUSY, "simulation %d has queued requests", sim);
  cudaFree(s->mem[sim]);
  s->mem[sim] = nullptr;
  s->live[sim] = 0;
  s->used -= s->bytes[sim];
  s->bytes[sim] = 0;
  return VD_OK;
}

extern "C" int64_t vd_server_submit(vd_server* s, int32_t sim, double t_arrive) {
  VD_CHECK_SERVER(s);
  if (sim < 0 || sim >= s->max_sims || !s->live[sim]) return vd_fail(VD_ENOTFOUND, "no live simulation %d", sim);
  Request r;
  r.ticket = s->next_ticket++;
  r.sim = sim;
  r.t_arrive = t_arrive < 0 ? now_s(s) : t_arrive;
  s->pending.push_back(r);
  return r.ticket;
}

extern "C" int vd_server_progress(vd_server* s) {
  VD_CHECK_SERVER(s);
  int completed = 0;
  int rc = reap(s, &completed);
  if (!rc) rc = admit(s);
  return rc ? rc : completed;
}

extern "C" int vd_server_drain(vd_server* s) {
  VD_CHECK_SERVER(s);
  for (;;) {
    const int rc = vd_server_progress(s);
    if (rc < 0) return rc;
    const bool busy = s->lanes[0].busy || s->lanes[1].busy;
    if (!busy && s->pending.empty()) return VD_OK;
    if (busy) std::this_thread::yield();
  }
}

extern "C" int32_t vd_server_completions(vd_server* s, int64_t* tickets, double* latency_s, int32_t* sims,
                                         int32_t cap) {
  VD_CHECK_SERVER(s);
  const int32_t n = static_cast<int32_t>(std::min<size_t>(cap < 0 ? 0 : cap, s->done_ticket.size()));
  for (int32_t i = 0; i < n; ++i) {
    if (tickets) tickets[i] = s->done_ticket[i];
    if (latency_s) latency_s[i] = s->done_latency[i];
    if (sims) sims[i] = s->done_sim[i];
  }
  s->done_ticket.erase(s->done_ticket.begin(), s->done_ticket.begin() + n);
  s->done_latency.erase(s->done_latency.begin(), s->done_latency.begin() + n);
  s->done_sim.erase(s->done_sim.begin(), s->done_sim.begin() + n);
  return n;
}

extern "C" double vd_server_now(const vd_server* s) { return s ? now_s(s) : -1.0; }

extern "C" int vd_server_run_trace(vd_server* s, const double* arrival_s, const int32_t* sims, int64_t n,
                                   double* latency_s) {
  VD_CHECK_SERVER(s);
  if (n < 0 || (n > 0 && (!arrival_s || !sims || !latency_s))) return vd_fail(VD_EINVAL, "bad trace");
  for (int64_t i = 0; i < n; ++i)
    if (sims[i] < 0 || sims[i] >= s->max_sims || !s->live[sims[i]])
      return vd_fail(VD_ENOTFOUND, "trace entry %lld names no live simulation", static_cast<long long>(i));
  int rc = vd_server_drain(s);
  if (rc) return rc;
  vd_server_completions(s, nullptr, nullptr, nullptr, static_cast<int32_t>(s->done_ticket.size()));
  const int64_t first = s->next_ticket;
  const double start = now_s(s);
  int64_t next = 0, done = 0;
  std::vector<int64_t> tk(1024);
  std::vector<double> lat(1024);
  while (done < n) {
    const double t = now_s(s) - start;
    while (next < n && arrival_s[next] <= t) {
      vd_server_submit(s, sims[next], start + arrival_s[next]);
      ++next;
    }
    rc = vd_server_progress(s);
    if (rc < 0) return rc;
    for (;;) {
      const int32_t m = vd_server_completions(s, tk.data(), lat.data(), nullptr, static_cast<int32_t>(tk.size()));
      for (int32_t i = 0; i < m; ++i) latency_s[tk[i] - first] = lat[i];
      done += m;
      if (m < static_cast<int32_t>(tk.size())) break;
    }
  }
  return VD_OK;
}

extern "C" int vd_server_get_labels(vd_server* s, int32_t sim, int32_t* labels, int on_device) {
  VD_CHECK_SERVER(s);
  if (sim < 0 || sim >= s->max_sims || !s->live[sim]) return vd_fail(VD_ENOTFOUND, "no live simulation %d", sim);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  if (s->in_flight[sim]) {
    const int rc = vd_server_drain(s);
    if (rc) return rc;
  }
  // cur and step are advanced on the device; read this simulation's record
  vdb::SimDesc d;
  int rc = vd_cuda_check(cudaMemcpyAsync(&d, s->d_sims + sim, sizeof(d), cudaMemcpyDeviceToHost, s->admin), "descriptor");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(s->admin), "synchronize");
  if (rc) return rc;
  rc = vd_cuda_check(cudaMemcpy2DAsync(labels, sizeof(int32_t) * d.w, d.map[d.cur], sizeof(int32_t) * d.pitch,
                                       sizeof(int32_t) * d.w, d.h,
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->admin),
                     "copy labels out");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(s->admin), "synchronize");
  return rc;
}

extern "C" int vd_server_stats(const vd_server* s, int64_t* used_bytes, int64_t* budget_bytes, int32_t* live_sims,
                               int64_t* pending, int64_t* steps_done, int64_t* launches) {
  VD_CHECK_SERVER(s);
  int32_t live = 0;
  for (char c : s->live) live += c;
  if (used_bytes) *used_bytes = s->used;
  if (budget_bytes) *budget_bytes = s->budget;
  if (live_sims) *live_sims = live;
  if (pending) *pending = static_cast<int64_t>(s->pending.size());
  if (steps_done) *steps_done = s->steps_done;
  if (launches) *launches = s->launches;
  return VD_OK;
}

extern "C" int vd_server_set_max_batch(vd_server* s, int32_t max_batch) {
  VD_CHECK_SERVER(s);
  if (max_batch < 1) return vd_fail(VD_EINVAL, "max_batch %d < 1", max_batch);
  s->max_batch = max_batch;
  return VD_OK;
}
