// vd_batch.cu -- many independent simulations stepped together.
//
// A batch owns one device arena with the label maps (two Jacobi buffers each,
// 128-byte row pitch, padding held at -1), seeds and pass tables of every
// simulation, plus a small descriptor per simulation.  A timestep of any
// subset of simulations is planned on the host (which simulations, their seed
// blocks, and per pass round the tiles of every simulation that still has a
// pass to run) and executed either as one launch per phase / pass round
// (captured in a CUDA graph when the plan repeats), or as ONE persistent
// cooperative launch whose phases are separated by a grid barrier with a
// bounded wait (a wait that runs out sets an error word and every block
// returns; the host reports VD_ETIMEOUT).
//
// Every simulation computes exactly what vd_djfa_step / vd_jfa compute for it
// alone: the same kernels' per-thread code (vdk::pass_quad) on the same data.
#include "vd_batch_engine.cuh"


// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct vd_batch {
  int device = 0;
  int n_sims = 0;
  cudaStream_t stream = nullptr;
  std::vector<vdb::SimDesc> sims;  // host mirror (cur and step are device-owned after the first step)
  vdb::SimDesc* d_sims = nullptr;
  int32_t* arena = nullptr;
  size_t arena_bytes = 0;
  int2* seeds = nullptr;
  int2* tables = nullptr;
  uint32_t* ptables = nullptr;
  uint2* pkfs = nullptr;  // seed entries of the wide position-tagged layouts, n + 1 per simulation
  int2* dxy_stage = nullptr;
  int64_t total_seeds = 0;
  int64_t total_pixels = 0;
  vdb::Barrier* bar = nullptr;
  int* h_err = nullptr;  // pinned mirror of bar->err
  unsigned long long* flag = nullptr;  // device counter for input validation
  vdb::PlanSlot plan;
  // configuration
  bool configured = false;
  int32_t d_max = 0, vn_waves = 2, extra = 0, metric = 0;
  // options
  int mode = 0;  // 0 = launch per phase/round, 1 = persistent
  int rows_per_thread = 1;
  int blocks_per_sm = 0;  // persistent: 0 = occupancy maximum
  int use_graphs = 1;
  long long timeout_ns = 2000000000LL;
  int test_skip_arrive = 0;
  int clamp = -1;  // clamped 32-bit keys: -1 auto, 0 never, 1 whenever usable
  int persistent_byte = 1;  // persistent launch: byte-offset keys where the auto rules pick them
  int persistent_min_blocks = 4;  // persistent launch: register budget for 4 (64 registers) or 5 (48) blocks per SM
  int packed = -1;  // launch per round: dJFA frames' last passes on position-tagged words (-1 auto, 0 never)
  int64_t launches = 0;
  // cached full-batch dJFA plan + graph
  int full_plan_valid = 0;
  cudaGraphExec_t full_graph = nullptr;
  int full_graph_given = -1;
  int64_t full_graph_launches = 0;  // kernel launches one replay of it makes
  int32_t last_max_disp = -1;
  uint64_t last_rng_seed = 0;
  int sm_count = 0;
};

namespace {

using vdb::HostPlan;

void drop_graph(vd_batch* b);

// Uploads a plan into the batch's plan buffer.  A cached full-step graph
// reads that buffer, so any upload invalidates it; the pinned staging buffer
// is reused, so the previous upload must have run.
int upload_plan(vd_batch* b, const HostPlan& p, vdb::BatchArgs* A) {
  drop_graph(b);
  const int rc = vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
  if (rc) return rc;
  return vdb::plan_upload(b->plan, p, b->d_sims, b->stream, A);
}

int launch_plan(vd_batch* b, const HostPlan& p, vdb::BatchArgs& A) {
  cudaStream_t st = b->stream;
  if (b->mode == 1) {
    int rc = vd_cuda_check(cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned int), st), "barrier reset");
    if (rc) return rc;
    const bool m5 = b->persistent_min_blocks == 5;
    const void* fn =
        b->metric == VD_METRIC_MANHATTAN
            ? (m5 ? reinterpret_cast<const void*>(&vdb::k_batch_persistent<vdk::kManhattan, 5>)
                  : reinterpret_cast<const void*>(&vdb::k_batch_persistent<vdk::kManhattan, 4>))
            : (m5 ? reinterpret_cast<const void*>(&vdb::k_batch_persistent<vdk::kEuclid, 5>)
                  : reinterpret_cast<const void*>(&vdb::k_batch_persistent<vdk::kEuclid, 4>));
    int per_sm = 0;
    rc = vd_cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, vdb::kThreads, 0), "occupancy");
    if (rc) return rc;
    if (b->blocks_per_sm > 0 && b->blocks_per_sm < per_sm) per_sm = b->blocks_per_sm;
    if (per_sm < 1) return vd_fail(VD_ECUDA, "persistent kernel does not fit on an SM");
    dim3 grid(b->sm_count * per_sm), block(vdb::kThreads);
    void* args[] = {&A};
    rc = vd_cuda_check(cudaLaunchCooperativeKernel(fn, grid, block, args, 0, st), "cooperative launch");
    if (rc) return rc;
    ++b->launches;
    return VD_OK;
  }
  return vdb::launch_rounds(p, A, b->metric, st, &b->launches);
}

vdb::BatchArgs base_args(const vd_batch* b) {
  return vdb::make_args(b->rows_per_thread, b->bar, b->timeout_ns, b->test_skip_arrive, b->persistent_byte);
}

void drop_graph(vd_batch* b) {
  if (b->full_graph) cudaGraphExecDestroy(b->full_graph);
  b->full_graph = nullptr;
  b->full_graph_given = -1;
}

void batch_free(vd_batch* b) {
  drop_graph(b);
  cudaFree(b->d_sims);
  cudaFree(b->arena);
  cudaFree(b->seeds);
  cudaFree(b->tables);
  cudaFree(b->ptables);
  cudaFree(b->pkfs);
  cudaFree(b->dxy_stage);
  cudaFree(b->bar);
  cudaFree(b->flag);
  b->plan.release();
  cudaFreeHost(b->h_err);
}

int upload_sims(vd_batch* b) {
  return vd_cuda_check(cudaMemcpyAsync(b->d_sims, b->sims.data(), sizeof(vdb::SimDesc) * b->n_sims,
                                       cudaMemcpyHostToDevice, b->stream),
                       "upload descriptors");
}

// cur and step live on the device once steps run; pull them before the host
// mirror is written back.
int pull_state(vd_batch* b) {
  std::vector<vdb::SimDesc> dev(b->n_sims);
  int rc = vd_cuda_check(cudaMemcpyAsync(dev.data(), b->d_sims, sizeof(vdb::SimDesc) * b->n_sims,
                                         cudaMemcpyDeviceToHost, b->stream), "download descriptors");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
  if (rc) return rc;
  for (int i = 0; i < b->n_sims; ++i) {
    b->sims[i].cur = dev[i].cur;
    b->sims[i].step = dev[i].step;
  }
  return VD_OK;
}

}  // namespace

#define VD_CHECK_BATCH(b) \
  if (!(b)) return vd_fail(VD_EINVAL, "null batch")

extern "C" vd_batch* vd_batch_create(int32_t n_sims, const int32_t* w, const int32_t* h, const int32_t* n_seeds) {
  if (n_sims < 1 || !w || !h || !n_seeds) {
    vd_fail(VD_EINVAL, "bad batch description");
    return nullptr;
  }
  for (int i = 0; i < n_sims; ++i) {
    if (w[i] < 1 || w[i] > VD_MAX_SIDE || h[i] < 1 || h[i] > VD_MAX_SIDE || n_seeds[i] < 1) {
      vd_fail(VD_EINVAL, "simulation %d: grid %dx%d, %d seeds", i, w[i], h[i], n_seeds[i]);
      return nullptr;
    }
  }
  vd_batch* b = new vd_batch();
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  b->n_sims = n_sims;
  b->sims.resize(n_sims);
  size_t map_elems = 0;
  int64_t seeds = 0;
  for (int i = 0; i < n_sims; ++i) {
    vdb::SimDesc& s = b->sims[i];
    std::memset(&s, 0, sizeof(s));
    s.w = w[i];
    s.h = h[i];
    s.n = n_seeds[i];
    s.pitch = (w[i] + 31) / 32 * 32;
    s.seed_off = static_cast<int>(seeds);
    map_elems += 2 * static_cast<size_t>(s.pitch) * s.h;
    seeds += s.n;
    b->total_pixels += static_cast<int64_t>(s.w) * s.h;
  }
  b->total_seeds = seeds;
  if (seeds > INT32_MAX / 2) {
    vd_fail(VD_EINVAL, "too many seeds in one batch");
    delete b;
    return nullptr;
  }
  b->arena_bytes = map_elems * sizeof(int32_t);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->arena), b->arena_bytes);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->seeds), sizeof(int2) * seeds);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->tables), sizeof(int2) * (seeds + n_sims));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->ptables), sizeof(uint32_t) * (seeds + n_sims));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->pkfs), sizeof(uint2) * (seeds + n_sims));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->dxy_stage), sizeof(int2) * seeds);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_sims), sizeof(vdb::SimDesc) * n_sims);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->bar), sizeof(vdb::Barrier));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->flag), sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->h_err), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->arena, 0xFF, b->arena_bytes);
  if (e == cudaSuccess) e = cudaMemset(b->seeds, 0, sizeof(int2) * seeds);
  if (e == cudaSuccess) e = cudaMemset(b->bar, 0, sizeof(vdb::Barrier));
  if (e != cudaSuccess) {
    vd_cuda_check(e, "batch allocation");
    cudaGetLastError();
    batch_free(b);
    delete b;
    return nullptr;
  }
  size_t off = 0;
  int64_t toff = 0;
  for (int i = 0; i < n_sims; ++i) {
    vdb::SimDesc& s = b->sims[i];
    const size_t m = static_cast<size_t>(s.pitch) * s.h;
    s.map[0] = b->arena + off;
    s.map[1] = b->arena + off + m;
    off += 2 * m;
    s.seeds = b->seeds + s.seed_off;
    s.table = b->tables + toff;
    s.ptable = b->ptables + toff;
    s.pkf = b->pkfs + toff;
    s.pk_m = 0;
    s.pk_first[0] = 0;
    toff += s.n + 1;
    // JFA schedule (index 1); the dJFA one is filled by vd_batch_configure
    s.n_pass[1] = vdi::fill_schedule(vdi::jfa_first_step(s.w, s.h), 0, 0, s.ks[1], s.nbs[1], vdb::kMaxPasses);
    vdb::set_clamp(s, 1, VD_METRIC_EUCLID, b->clamp, b->packed);
  }
  int rc = upload_sims(b);
  for (int i = 0; !rc && i < n_sims; ++i)
    rc = vdi::launch_build_table(b->sims[i].seeds, b->sims[i].n, b->sims[i].table, b->sims[i].ptable, b->stream);
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(b->stream), "create");
  if (rc) {
    batch_free(b);
    delete b;
    return nullptr;
  }
  return b;
}

extern "C" int vd_batch_destroy(vd_batch* b) {
  if (!b) return VD_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
  return VD_OK;
}

extern "C" int vd_batch_set_stream(vd_batch* b, void* stream) {
  VD_CHECK_BATCH(b);
  b->stream = static_cast<cudaStream_t>(stream);
  drop_graph(b);
  return VD_OK;
}

extern "C" int vd_batch_synchronize(vd_batch* b) {
  VD_CHECK_BATCH(b);
  int rc = vd_cuda_check(cudaMemcpyAsync(b->h_err, &b->bar->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
                         "read barrier status");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
  if (rc) return rc;
  if (*b->h_err != 0) {
    cudaMemsetAsync(&b->bar->err, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    return vd_fail(VD_ETIMEOUT,
                   "a grid barrier wait ran out in a persistent batched step; the maps of that step are undefined");
  }
  return VD_OK;
}

extern "C" int vd_batch_get_shape(const vd_batch* b, int32_t sim, int32_t* w, int32_t* h, int32_t* n_seeds,
                                  int32_t* seed_offset) {
  VD_CHECK_BATCH(b);
  if (sim < 0 || sim >= b->n_sims) return vd_fail(VD_EINVAL, "simulation %d of %d", sim, b->n_sims);
  const vdb::SimDesc& s = b->sims[sim];
  if (w) *w = s.w;
  if (h) *h = s.h;
  if (n_seeds) *n_seeds = s.n;
  if (seed_offset) *seed_offset = s.seed_off;
  return VD_OK;
}

extern "C" int vd_batch_set_seeds(vd_batch* b, const int32_t* xy, int on_device) {
  VD_CHECK_BATCH(b);
  if (!xy) return vd_fail(VD_EINVAL, "null seeds");
  int rc;
  if (!on_device) {
    for (int i = 0; i < b->n_sims; ++i) {
      const vdb::SimDesc& s = b->sims[i];
      for (int k = 0; k < s.n; ++k) {
        const int32_t x = xy[2 * (s.seed_off + k)], y = xy[2 * (s.seed_off + k) + 1];
        if (x < 0 || x >= s.w || y < 0 || y >= s.h)
          return vd_fail(VD_EINVAL, "simulation %d seed %d at (%d, %d) outside %dx%d", i, k, x, y, s.w, s.h);
      }
    }
    rc = vd_cuda_check(cudaMemcpyAsync(b->seeds, xy, sizeof(int2) * b->total_seeds, cudaMemcpyHostToDevice,
                                       b->stream), "copy seeds");
  } else {
    // validate per simulation in the staging buffer before adopting
    rc = vd_cuda_check(cudaMemcpyAsync(b->dxy_stage, xy, sizeof(int2) * b->total_seeds, cudaMemcpyDeviceToDevice,
                                       b->stream), "copy seeds");
    if (!rc) rc = vd_cuda_check(cudaMemsetAsync(b->flag, 0, sizeof(unsigned long long), b->stream), "memset");
    if (rc) return rc;
    for (int i = 0; i < b->n_sims; ++i) {
      const vdb::SimDesc& s = b->sims[i];
      vdk::k_check_seeds<<<(s.n + 255) / 256, 256, 0, b->stream>>>(b->dxy_stage + s.seed_off, s.n, s.w, s.h, b->flag);
      ++b->launches;
    }
    rc = vd_cuda_check(cudaGetLastError(), "check seeds");
    unsigned long long bad = 0;
    if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(&bad, b->flag, sizeof(bad), cudaMemcpyDeviceToHost, b->stream),
                                "copy flag");
    if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
    if (rc) return rc;
    if (bad) return vd_fail(VD_EINVAL, "%llu device seeds outside their grids", bad);
    rc = vd_cuda_check(cudaMemcpyAsync(b->seeds, b->dxy_stage, sizeof(int2) * b->total_seeds,
                                       cudaMemcpyDeviceToDevice, b->stream), "copy seeds");
  }
  if (rc) return rc;
  for (int i = 0; !rc && i < b->n_sims; ++i) {
    rc = vdi::launch_build_table(b->sims[i].seeds, b->sims[i].n, b->sims[i].table, b->sims[i].ptable, b->stream);
    ++b->launches;
  }
  return rc;
}

extern "C" int vd_batch_get_seeds(vd_batch* b, int32_t sim, int32_t* xy, int on_device) {
  VD_CHECK_BATCH(b);
  if (sim < 0 || sim >= b->n_sims) return vd_fail(VD_EINVAL, "simulation %d of %d", sim, b->n_sims);
  if (!xy) return vd_fail(VD_EINVAL, "null output");
  const vdb::SimDesc& s = b->sims[sim];
  int rc = vd_cuda_check(cudaMemcpyAsync(xy, s.seeds, sizeof(int2) * s.n,
                                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream),
                         "copy seeds out");
  if (rc || on_device) return rc;
  return vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
}

extern "C" int vd_batch_get_labels(vd_batch* b, int32_t sim, int32_t* labels, int on_device) {
  VD_CHECK_BATCH(b);
  if (sim < 0 || sim >= b->n_sims) return vd_fail(VD_EINVAL, "simulation %d of %d", sim, b->n_sims);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  int rc = vd_batch_synchronize(b);
  if (rc) return rc;
  rc = pull_state(b);
  if (rc) return rc;
  const vdb::SimDesc& s = b->sims[sim];
  rc = vd_cuda_check(cudaMemcpy2DAsync(labels, sizeof(int32_t) * s.w, s.map[s.cur], sizeof(int32_t) * s.pitch,
                                       sizeof(int32_t) * s.w, s.h,
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream),
                     "copy labels out");
  if (rc) return rc;
  return vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
}

extern "C" int vd_batch_configure(vd_batch* b, int32_t d_max, int32_t vn_waves, int32_t extra, int32_t metric) {
  VD_CHECK_BATCH(b);
  if (metric != VD_METRIC_EUCLID && metric != VD_METRIC_MANHATTAN) return vd_fail(VD_EINVAL, "metric %d", metric);
  if (d_max < 0 || vn_waves < 0 || extra < 0 || extra > 2) return vd_fail(VD_EINVAL, "bad dJFA parameters");
  int rc = pull_state(b);
  if (rc) return rc;
  for (vdb::SimDesc& s : b->sims) {
    s.n_pass[0] = vdi::fill_schedule(vdi::djfa_first_step(s.w, s.h, s.n, d_max), vn_waves, extra, s.ks[0], s.nbs[0],
                                     vdb::kMaxPasses);
    vdb::set_clamp(s, 0, metric, b->clamp, b->packed);
  }
  b->d_max = d_max;
  b->vn_waves = vn_waves;
  b->extra = extra;
  b->metric = metric;
  b->configured = true;
  drop_graph(b);
  return upload_sims(b);
}

static std::vector<int> all_sims(const vd_batch* b) {
  std::vector<int> a(b->n_sims);
  for (int i = 0; i < b->n_sims; ++i) a[i] = i;
  return a;
}

extern "C" int vd_batch_jfa(vd_batch* b, int32_t metric) {
  VD_CHECK_BATCH(b);
  if (metric != VD_METRIC_EUCLID && metric != VD_METRIC_MANHATTAN) return vd_fail(VD_EINVAL, "metric %d", metric);
  int rc = vd_batch_synchronize(b);
  if (!rc) rc = pull_state(b);
  if (rc) return rc;
  for (vdb::SimDesc& s : b->sims) vdb::set_clamp(s, 1, metric, b->clamp, b->packed);
  rc = upload_sims(b);
  if (rc) return rc;
  // frame 0 of every simulation: empty both buffers' current map, stamp, JFA passes
  for (const vdb::SimDesc& s : b->sims) {
    rc = vdi::launch_fill(s.map[s.cur], static_cast<int64_t>(s.pitch) * s.h, -1, b->stream);
    ++b->launches;
    if (rc) return rc;
  }
  const int saved_metric = b->metric, saved_mode = b->mode;
  b->metric = metric;
  b->mode = 0;
  HostPlan p = vdb::make_plan(b->sims, all_sims(b), 1, b->rows_per_thread);
  vdb::BatchArgs A = base_args(b);
  A.sched = 1;
  A.mark = 0;
  A.move = 0;
  rc = upload_plan(b, p, &A);
  if (!rc) rc = launch_plan(b, p, A);
  b->metric = saved_metric;
  b->mode = saved_mode;
  drop_graph(b);
  return rc;
}

static int batch_step(vd_batch* b, const std::vector<int>& act, bool given, int32_t max_disp, uint64_t rng_seed,
                      bool full) {
  if (!b->configured) return vd_fail(VD_EINVAL, "vd_batch_configure has not been called");
  vdb::BatchArgs A = base_args(b);
  A.sched = 0;
  A.mark = 1;
  A.move = 1;
  A.dxy = given ? b->dxy_stage : nullptr;
  A.max_disp = max_disp;
  A.rng_seed = rng_seed;
  HostPlan p = vdb::make_plan(b->sims, act, 0, b->rows_per_thread);
  const bool graphable = full && b->use_graphs && b->mode == 0 && b->stream != nullptr;
  if (graphable && b->full_graph && b->full_graph_given == static_cast<int>(given)) {
    // the plan and the arguments baked into the graph are unchanged except the
    // RNG parameters, which are per-launch: only replay when they match
    int rc = vd_cuda_check(cudaGraphLaunch(b->full_graph, b->stream), "graph launch");
    if (rc) return rc;
    b->launches += b->full_graph_launches;
    return VD_OK;
  }
  int rc = upload_plan(b, p, &A);
  if (rc) return rc;
  if (!graphable) return launch_plan(b, p, A);
  cudaGraph_t g = nullptr;
  rc = vd_cuda_check(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (rc) return rc;
  const int64_t l0 = b->launches;
  const int lrc = launch_plan(b, p, A);
  const cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
  const int64_t captured = b->launches - l0;
  b->launches = l0;
  if (lrc) {
    if (g) cudaGraphDestroy(g);
    return lrc;
  }
  rc = vd_cuda_check(ee, "end capture");
  if (rc) return rc;
  cudaGraphExec_t ex = nullptr;
  rc = vd_cuda_check(cudaGraphInstantiate(&ex, g, 0), "graph instantiate");
  cudaGraphDestroy(g);
  if (rc) return rc;
  drop_graph(b);
  b->full_graph = ex;
  b->full_graph_given = static_cast<int>(given);
  b->full_graph_launches = captured;
  rc = vd_cuda_check(cudaGraphLaunch(ex, b->stream), "graph launch");
  if (rc) return rc;
  b->launches += captured;
  return VD_OK;
}

extern "C" int vd_batch_step(vd_batch* b, const int32_t* dxy, int dxy_on_device, int32_t max_disp, uint64_t rng_seed) {
  VD_CHECK_BATCH(b);
  if (dxy) {
    const int rc = vd_cuda_check(cudaMemcpyAsync(b->dxy_stage, dxy, sizeof(int2) * b->total_seeds,
                                                 dxy_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                                 b->stream), "copy moves");
    if (rc) return rc;
  } else if (max_disp < 0 || max_disp > VD_MAX_SIDE) {
    return vd_fail(VD_EINVAL, "max_disp %d outside [0, %d]", max_disp, VD_MAX_SIDE);
  }
  // a cached graph bakes in max_disp and rng_seed: drop it when they change
  if (b->full_graph && !dxy && (b->last_max_disp != max_disp || b->last_rng_seed != rng_seed)) drop_graph(b);
  b->last_max_disp = max_disp;
  b->last_rng_seed = rng_seed;
  return batch_step(b, all_sims(b), dxy != nullptr, max_disp, rng_seed, true);
}

extern "C" int vd_batch_step_subset(vd_batch* b, const int32_t* sims, int32_t n, int32_t max_disp, uint64_t rng_seed) {
  VD_CHECK_BATCH(b);
  if (n < 0 || (n > 0 && !sims)) return vd_fail(VD_EINVAL, "bad subset");
  if (max_disp < 0 || max_disp > VD_MAX_SIDE) return vd_fail(VD_EINVAL, "max_disp %d outside [0, %d]", max_disp, VD_MAX_SIDE);
  std::vector<int> act;
  std::vector<char> seen(b->n_sims, 0);
  for (int i = 0; i < n; ++i) {
    if (sims[i] < 0 || sims[i] >= b->n_sims) return vd_fail(VD_EINVAL, "simulation %d of %d", sims[i], b->n_sims);
    if (seen[sims[i]]) return vd_fail(VD_EINVAL, "simulation %d listed twice in one step", sims[i]);
    seen[sims[i]] = 1;
    act.push_back(sims[i]);
  }
  if (act.empty()) return VD_OK;
  return batch_step(b, act, false, max_disp, rng_seed, false);
}

extern "C" int vd_batch_set_option(vd_batch* b, int32_t option, int64_t value) {
  VD_CHECK_BATCH(b);
  switch (option) {
    case VD_BOPT_MODE:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "mode must be 0 (per round) or 1 (persistent)");
      b->mode = static_cast<int>(value);
      break;
    case VD_BOPT_ROWS_PER_THREAD:
      if (value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
        return vd_fail(VD_EINVAL, "rows per thread must be 1, 2, 4, 8 or 16");
      b->rows_per_thread = static_cast<int>(value);
      break;
    case VD_BOPT_BLOCKS_PER_SM:
      if (value < 0 || value > 8) return vd_fail(VD_EINVAL, "blocks per SM outside [0, 8]");
      b->blocks_per_sm = static_cast<int>(value);
      break;
    case VD_BOPT_USE_GRAPHS:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "use_graphs must be 0 or 1");
      b->use_graphs = static_cast<int>(value);
      break;
    case VD_BOPT_BARRIER_TIMEOUT_US:
      if (value < 1000 || value > 60000000) return vd_fail(VD_EINVAL, "barrier timeout outside [1 ms, 60 s]");
      b->timeout_ns = value * 1000;
      break;
    case VD_BOPT_TEST_SKIP_ARRIVE:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "test flag must be 0 or 1");
      b->test_skip_arrive = static_cast<int>(value);
      break;
    case VD_BOPT_CLAMPED_KEYS:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "clamped keys must be -1, 0 or 1");
      b->clamp = static_cast<int>(value);
      // takes effect at the next vd_batch_configure / vd_batch_jfa
      break;
    case VD_BOPT_PERSISTENT_BYTE_KEYS:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "persistent byte keys must be 0 or 1");
      b->persistent_byte = static_cast<int>(value);
      break;
    case VD_BOPT_PERSISTENT_MIN_BLOCKS:
      if (value != 4 && value != 5) return vd_fail(VD_EINVAL, "persistent blocks per SM must be 4 or 5");
      b->persistent_min_blocks = static_cast<int>(value);
      break;
    case VD_BOPT_PACKED_MAP:
      if (value != -1 && value != 0) return vd_fail(VD_EINVAL, "packed map must be -1 (auto) or 0 (never)");
      b->packed = static_cast<int>(value);
      // takes effect at the next vd_batch_configure
      break;
    default:
      return vd_fail(VD_EINVAL, "unknown batch option %d", option);
  }
  drop_graph(b);
  return VD_OK;
}

extern "C" int vd_batch_get_option(const vd_batch* b, int32_t option, int64_t* value) {
  VD_CHECK_BATCH(b);
  if (!value) return vd_fail(VD_EINVAL, "null output");
  switch (option) {
    case VD_BOPT_MODE: *value = b->mode; break;
    case VD_BOPT_ROWS_PER_THREAD: *value = b->rows_per_thread; break;
    case VD_BOPT_BLOCKS_PER_SM: *value = b->blocks_per_sm; break;
    case VD_BOPT_USE_GRAPHS: *value = b->use_graphs; break;
    case VD_BOPT_BARRIER_TIMEOUT_US: *value = b->timeout_ns / 1000; break;
    case VD_BOPT_TEST_SKIP_ARRIVE: *value = b->test_skip_arrive; break;
    case VD_BOPT_CLAMPED_KEYS: *value = b->clamp; break;
    case VD_BOPT_PERSISTENT_BYTE_KEYS: *value = b->persistent_byte; break;
    case VD_BOPT_PERSISTENT_MIN_BLOCKS: *value = b->persistent_min_blocks; break;
    case VD_BOPT_PACKED_MAP: *value = b->packed; break;
    default: return vd_fail(VD_EINVAL, "unknown batch option %d", option);
  }
  return VD_OK;
}

extern "C" int64_t vd_batch_launch_count(const vd_batch* b) { return b ? b->launches : -1; }

extern "C" int vd_batch_work(const vd_batch* b, int64_t* pixels, int64_t* pixel_passes_per_step, int64_t* seeds) {
  VD_CHECK_BATCH(b);
  int64_t pp = 0;
  for (const vdb::SimDesc& s : b->sims) pp += static_cast<int64_t>(s.w) * s.h * (b->configured ? s.n_pass[0] : 0);
  if (pixels) *pixels = b->total_pixels;
  if (pixel_passes_per_step) *pixel_passes_per_step = pp;
  if (seeds) *seeds = b->total_seeds;
  return VD_OK;
}

namespace {

// A full copy of the batch's device state (maps, seeds, tables, descriptors).
struct Snapshot {
  int32_t* arena = nullptr;
  int2* seeds = nullptr;
  int2* tables = nullptr;
  uint32_t* ptables = nullptr;
  vdb::SimDesc* sims = nullptr;
  void release() {
    cudaFree(arena);
    cudaFree(seeds);
    cudaFree(tables);
    cudaFree(sims);
  }
};

int snapshot_copy(vd_batch* b, Snapshot& sn, bool save) {
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  cudaStream_t st = b->stream;
  int32_t* a_dst = save ? sn.arena : b->arena;
  const int32_t* a_src = save ? b->arena : sn.arena;
  int rc = vd_cuda_check(cudaMemcpyAsync(a_dst, a_src, b->arena_bytes, k, st), "snapshot maps");
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(save ? sn.seeds : b->seeds, save ? b->seeds : sn.seeds,
                                       sizeof(int2) * b->total_seeds, k, st), "snapshot seeds");
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(save ? sn.tables : b->tables, save ? b->tables : sn.tables,
                                       sizeof(int2) * (b->total_seeds + b->n_sims), k, st), "snapshot tables");
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(save ? sn.ptables : b->ptables, save ? b->ptables : sn.ptables,
                                       sizeof(uint32_t) * (b->total_seeds + b->n_sims), k, st), "snapshot positions");
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(save ? sn.sims : b->d_sims, save ? b->d_sims : sn.sims,
                                       sizeof(vdb::SimDesc) * b->n_sims, k, st), "snapshot descriptors");
  return rc;
}

}  // namespace

extern "C" int vd_batch_autotune(vd_batch* b, int32_t steps, int32_t max_disp, uint64_t rng_seed, int32_t* best,
                                 double* ms_per_step, int32_t cap) {
  VD_CHECK_BATCH(b);
  if (!b->configured) return vd_fail(VD_EINVAL, "vd_batch_configure has not been called");
  if (steps < 1 || steps > 1000) return vd_fail(VD_EINVAL, "steps outside [1, 1000]");
  struct Cand {
    int mode, rpt, bps, pbyte, minb;
  };
  // per-round launches with tiles of 256 x 4 r pixels (r rows per thread), and
  // the persistent launch at the occupancy maximum or capped at 3 or 2 blocks
  // per SM (fewer co-resident blocks: fewer arrivals at each grid barrier);
  // then per-round launches with 8 and 16 rows a thread (a thread's tile
  // look-up and descriptor reads shared by more pixels)
  const Cand cands[] = {{0, 1, 0, 1, 4}, {0, 2, 0, 1, 4}, {0, 4, 0, 1, 4}, {1, 1, 0, 1, 4}, {1, 2, 0, 1, 4},
                        {1, 4, 0, 1, 4}, {1, 1, 3, 1, 4}, {1, 2, 3, 1, 4}, {1, 1, 2, 1, 4}, {1, 2, 2, 1, 4},
                        {1, 1, 0, 0, 4}, {1, 2, 0, 0, 4}, {1, 1, 0, 1, 5}, {1, 2, 0, 1, 5}, {1, 4, 0, 1, 5},
                        {0, 8, 0, 1, 4}, {0, 16, 0, 1, 4}};
  const int nc = static_cast<int>(sizeof(cands) / sizeof(cands[0]));
  int rc = vd_batch_synchronize(b);
  if (rc) return rc;
  Snapshot sn;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&sn.arena), b->arena_bytes);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sn.seeds), sizeof(int2) * b->total_seeds);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sn.tables), sizeof(int2) * (b->total_seeds + b->n_sims));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sn.ptables), sizeof(uint32_t) * (b->total_seeds + b->n_sims));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sn.sims), sizeof(vdb::SimDesc) * b->n_sims);
  if (e != cudaSuccess) {
    sn.release();
    return vd_cuda_check(e, "autotune snapshot");
  }
  const int mode0 = b->mode, rpt0 = b->rows_per_thread, bps0 = b->blocks_per_sm, pb0 = b->persistent_byte;
  const int mb0 = b->persistent_min_blocks;
  rc = snapshot_copy(b, sn, true);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc) rc = vd_cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = vd_cuda_check(cudaEventCreate(&e1), "event");
  int best_i = -1;
  double best_ms = 1e30;
  for (int c = 0; !rc && c < nc; ++c) {
    b->mode = cands[c].mode;
    b->rows_per_thread = cands[c].rpt;
    b->blocks_per_sm = cands[c].bps;
    b->persistent_byte = cands[c].pbyte;
    b->persistent_min_blocks = cands[c].minb;
    drop_graph(b);
    rc = snapshot_copy(b, sn, false);
    if (!rc) rc = vd_batch_step(b, nullptr, 0, max_disp, rng_seed);  // warm-up (plan, graph)
    if (!rc) rc = vd_cuda_check(cudaEventRecord(e0, b->stream), "event");
    for (int s = 0; !rc && s < steps; ++s) rc = vd_batch_step(b, nullptr, 0, max_disp, rng_seed);
    if (!rc) rc = vd_cuda_check(cudaEventRecord(e1, b->stream), "event");
    if (!rc) rc = vd_batch_synchronize(b);
    float t = 0.f;
    if (!rc) rc = vd_cuda_check(cudaEventElapsedTime(&t, e0, e1), "elapsed");
    if (rc) break;
    const double per = static_cast<double>(t) / steps;
    if (ms_per_step && c < cap) ms_per_step[c] = per;
    if (per < best_ms) {
      best_ms = per;
      best_i = c;
    }
  }
  // put the state back exactly as it was, and keep the fastest configuration
  const int rrc = snapshot_copy(b, sn, false);
  if (!rc) rc = rrc;
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(b->stream), "synchronize");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  sn.release();
  if (best_i >= 0 && !rc) {
    b->mode = cands[best_i].mode;
    b->rows_per_thread = cands[best_i].rpt;
    b->blocks_per_sm = cands[best_i].bps;
    b->persistent_byte = cands[best_i].pbyte;
    b->persistent_min_blocks = cands[best_i].minb;
  } else {
    b->mode = mode0;
    b->rows_per_thread = rpt0;
    b->blocks_per_sm = bps0;
    b->persistent_byte = pb0;
    b->persistent_min_blocks = mb0;
  }
  drop_graph(b);
  if (best) *best = best_i;
  if (rc) return rc;
  return nc;
}
