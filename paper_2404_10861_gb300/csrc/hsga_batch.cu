// hsga_batch.cu -- many independent runs advanced together.
//
// A batch holds runs of uneven size and configuration (grid shape, agents
// per island, policy, mutation rates, seed, generation budget).  One "tick"
// advances every active run by one synchronous generation: a single launch
// per agents-per-lane class covers all of them, so small runs that could not
// fill the GPU alone share it.  The work list is a flat array of (run, first
// island) items of up to kGroup islands each; each run's parameters, planes
// and start tick live in a device descriptor, and the current tick lives in
// device memory so that a CUDA graph of many ticks can be captured once per
// active set and replayed.  Runs are admitted and retired between calls,
// which is what the serving loop builds on.  The launch shape (threads per
// block, resident blocks) is chosen by timing real ticks (launch shape never
// changes results).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "hsga.h"
#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {
namespace {

struct BatchRun {  // device descriptor of one run
  RunParams p;
  uint32_t *trait[2];
  uint64_t *surf[2];
  uint32_t start_tick;  // the run is at generation 0 at this tick
  uint32_t pad;
};

struct WorkItem {
  uint32_t run, isl0;
};

template <int AP>
__global__ void __launch_bounds__(512)
    batch_step_kernel(const BatchRun *__restrict__ runs, const WorkItem *__restrict__ items,
                      uint32_t n_items, const uint32_t *__restrict__ tick_base,
                      uint32_t tick_off) {
  const uint32_t tick = *tick_base + tick_off;
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t nwarps = gridDim.x * wpb;
  for (uint32_t i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n_items; i += nwarps) {
    const WorkItem w = items[i];
    const BatchRun &R = runs[w.run];
    const RunParams &p = R.p;  // read in place (a copy would live in local memory)
    const uint32_t G = tick - R.start_tick;
    const uint32_t par = tick & 1u;
    const uint32_t *tin = R.trait[par];
    const uint64_t *sin = R.surf[par];
    uint32_t *tout = R.trait[par ^ 1u];
    uint64_t *sout = R.surf[par ^ 1u];
    const Deposit dep = deposit_for(p, G);
    // 32-bit test, every-generation case first (a 64-bit modulo per work item otherwise)
    const bool do_mig = p.interval == 1u || (p.interval != 0u && G % p.interval == 0u);
    if (w.isl0 + kGroup <= p.islands) {
      PhiloxHead head[AP];
      replication_heads<AP>(p, G, head);
      if (dep.two)
        full_group<AP, true, false, 0, kInterleave, false, true>(p, dep, G, do_mig, w.isl0, tin,
                                                                 sin, tout, sout, head);
      else if (p.tournament == 2)
        full_group<AP, true, true, 0, kInterleave, false>(p, dep, G, do_mig, w.isl0, tin, sin,
                                                          tout, sout, head);
      else
        full_group<AP, true, false, 0, kInterleave, false>(p, dep, G, do_mig, w.isl0, tin, sin,
                                                           tout, sout, head);
    } else {
      partial_group<AP, true, false, false>(p, dep, G, do_mig, w.isl0, tin, sin, tout, sout);
    }
  }
}

__global__ void advance_tick_kernel(uint32_t *tick, uint32_t by) { *tick += by; }
__global__ void set_tick_kernel(uint32_t *tick, uint32_t v) { *tick = v; }

struct HostRun {
  hsga_config cfg;
  RunParams p;
  uint64_t budget = 0;
  uint64_t start_tick = 0;
  uint32_t *trait[2] = {nullptr, nullptr};
  uint64_t *surf[2] = {nullptr, nullptr};
  uint64_t agents = 0;
  bool live = false;
};

struct LaunchShape {
  int threads = 256;
  int blocks[2] = {0, 0};  // per agents-per-lane class
};

constexpr uint64_t kMaxTick = 0xFFFFFFFFull - 64;
constexpr uint32_t kGraphTicks = 64;

}  // namespace
}  // namespace hsga

using namespace hsga;

struct hsga_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;  // graphs cannot be captured on the legacy default stream
  AllocHooks alloc{};
  std::vector<HostRun> runs;
  BatchRun *d_runs = nullptr;
  size_t d_runs_cap = 0;
  bool runs_dirty = true;
  WorkItem *d_items[2] = {nullptr, nullptr};
  size_t items_cap[2] = {0, 0};
  uint32_t n_items[2] = {0, 0};
  std::vector<WorkItem> h_items[2];
  bool items_dirty = true;
  // runs in the work lists are ordered by finishing tick, latest first, so
  // the runs still active at any later tick are a prefix of each list:
  // (finishing tick, items up to and including that run)
  std::vector<std::pair<uint64_t, uint32_t>> prefix[2];
  uint32_t *d_tick = nullptr;
  uint64_t tick = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  LaunchShape shape;
  std::map<int, LaunchShape> tuned;  // by log4 of the item count
  int sms = 0;
  uint64_t launches = 0, replications = 0, phases = 0;
};

namespace {

bool active_at(const HostRun &r, uint64_t t) {
  return r.live && r.start_tick <= t && t < r.start_tick + r.budget;
}

void drop_graph(hsga_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_valid = false;
}

cudaError_t upload_runs(hsga_batch *b) {
  if (!b->runs_dirty) return cudaSuccess;
  const size_t n = std::max<size_t>(b->runs.size(), 1);
  if (n > b->d_runs_cap) {
    device_free(b->alloc, b->d_runs, b->stream);
    size_t cap = std::max<size_t>(n, 2 * b->d_runs_cap);
    b->d_runs = (BatchRun *)device_alloc(b->alloc, sizeof(BatchRun) * cap, b->stream);
    if (!b->d_runs) {
      b->d_runs_cap = 0;
      return cudaErrorMemoryAllocation;
    }
    b->d_runs_cap = cap;
  }
  std::vector<BatchRun> h(b->runs.size());
  for (size_t i = 0; i < b->runs.size(); ++i) {
    memset(&h[i], 0, sizeof(BatchRun));
    h[i].p = b->runs[i].p;
    for (int j = 0; j < 2; ++j) {
      h[i].trait[j] = b->runs[i].trait[j];
      h[i].surf[j] = b->runs[i].surf[j];
    }
    h[i].start_tick = (uint32_t)b->runs[i].start_tick;
  }
  cudaError_t e = cudaSuccess;
  if (!h.empty())
    e = cudaMemcpyAsync(b->d_runs, h.data(), sizeof(BatchRun) * h.size(),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // h is a local
  b->runs_dirty = false;
  drop_graph(b);
  return e;
}

// Work lists of the runs active at the current tick, one per agents-per-lane
// class (n <= 32, n > 32), each ordered by finishing tick, latest first.
cudaError_t rebuild_items(hsga_batch *b) {
  std::vector<uint32_t> order;
  for (size_t r = 0; r < b->runs.size(); ++r)
    if (active_at(b->runs[r], b->tick)) order.push_back((uint32_t)r);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    return b->runs[x].start_tick + b->runs[x].budget > b->runs[y].start_tick + b->runs[y].budget;
  });
  for (int c = 0; c < 2; ++c) {
    b->h_items[c].clear();
    b->prefix[c].clear();
  }
  for (uint32_t r : order) {
    const HostRun &R = b->runs[r];
    const int c = R.p.n <= 32 ? 0 : 1;
    for (uint32_t i0 = 0; i0 < R.p.islands; i0 += kGroup)
      b->h_items[c].push_back(WorkItem{r, i0});
    b->prefix[c].push_back({R.start_tick + R.budget, (uint32_t)b->h_items[c].size()});
  }
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
    const size_t n = b->h_items[c].size();
    if (n > b->items_cap[c]) {
      device_free(b->alloc, b->d_items[c], b->stream);
      const size_t cap = std::max(n, 2 * b->items_cap[c]);
      b->d_items[c] = (WorkItem *)device_alloc(b->alloc, sizeof(WorkItem) * cap, b->stream);
      if (!b->d_items[c]) {
        b->items_cap[c] = 0;
        return cudaErrorMemoryAllocation;
      }
      b->items_cap[c] = cap;
    }
    if (n)
      e = cudaMemcpyAsync(b->d_items[c], b->h_items[c].data(), sizeof(WorkItem) * n,
                          cudaMemcpyHostToDevice, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  b->items_dirty = false;
  b->n_items[0] = b->n_items[1] = 0xFFFFFFFFu;  // force a prefix update
  return e;
}

// Items of the runs still active at the current tick (a prefix of each list).
void select_active_prefix(hsga_batch *b) {
  for (int c = 0; c < 2; ++c) {
    uint32_t n = 0;
    for (const auto &pe : b->prefix[c]) {
      if (pe.first > b->tick) n = pe.second;
      else break;
    }
    if (n != b->n_items[c]) {
      b->n_items[c] = n;
      drop_graph(b);
    }
  }
}

void launch_tick(hsga_batch *b, const LaunchShape &s, uint32_t off) {
  if (b->n_items[0])
    batch_step_kernel<1><<<s.blocks[0], s.threads, 0, b->stream>>>(b->d_runs, b->d_items[0],
                                                                   b->n_items[0], b->d_tick, off);
  if (b->n_items[1])
    batch_step_kernel<2><<<s.blocks[1], s.threads, 0, b->stream>>>(b->d_runs, b->d_items[1],
                                                                   b->n_items[1], b->d_tick, off);
}

int launches_per_tick(const hsga_batch *b) {
  return (b->n_items[0] ? 1 : 0) + (b->n_items[1] ? 1 : 0);
}

LaunchShape shape_for(hsga_batch *b, int threads, bool persistent) {
  LaunchShape s;
  s.threads = threads;
  const int wpb = threads / 32;
  for (int c = 0; c < 2; ++c) {
    const uint32_t n = b->n_items[c];
    const uint64_t need = (n + wpb - 1) / wpb;
    int per_sm = 1;
    if (persistent) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, c == 0 ? (const void *)batch_step_kernel<1> : (const void *)batch_step_kernel<2>,
          threads, 0);
      per_sm = std::max(per_sm, 1);
      s.blocks[c] = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)per_sm * b->sms));
    } else {
      s.blocks[c] = (int)std::max<uint64_t>(1, need);
    }
  }
  return s;
}

// Launch-shape autotuner: each candidate advances the batch by a few real
// ticks (results do not depend on the shape) and the fastest is kept per
// work-list size class.
cudaError_t autotune(hsga_batch *b, uint64_t *ticks_left) {
  const uint32_t total = b->n_items[0] + b->n_items[1];
  int bucket = 0;
  for (uint32_t x = total; x > 3; x >>= 2) ++bucket;
  auto it = b->tuned.find(bucket);
  if (it != b->tuned.end()) {
    b->shape = shape_for(b, it->second.threads, true);
    return cudaSuccess;
  }
  const int cand_threads[3] = {128, 256, 512};
  const uint32_t per_cand = 4;
  float best = 1e30f;
  LaunchShape best_shape = shape_for(b, 256, true);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int tried = 0;
  for (int t : cand_threads) {
    if (*ticks_left < per_cand) break;
    const LaunchShape s = shape_for(b, t, true);
    cudaEventRecord(e0, b->stream);
    for (uint32_t k = 0; k < per_cand; ++k) launch_tick(b, s, k);
    advance_tick_kernel<<<1, 1, 0, b->stream>>>(b->d_tick, per_cand);
    cudaEventRecord(e1, b->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return e;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    b->tick += per_cand;
    *ticks_left -= per_cand;
    b->launches += per_cand * launches_per_tick(b) + 1;
    ++tried;
    if (ms < best) {
      best = ms;
      best_shape = s;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->shape = best_shape;
  if (tried == 3) b->tuned[bucket] = best_shape;  // keep only complete comparisons
  return cudaGetLastError();
}

cudaError_t run_ticks(hsga_batch *b, uint64_t L) {
  cudaError_t e = cudaSuccess;
  if (L >= kGraphTicks) {
    if (!b->graph_valid) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      for (uint32_t k = 0; k < kGraphTicks; ++k) launch_tick(b, b->shape, k);
      advance_tick_kernel<<<1, 1, 0, b->stream>>>(b->d_tick, kGraphTicks);
      e = cudaStreamEndCapture(b->stream, &g);
      if (e != cudaSuccess) return e;
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
      b->graph_valid = true;
    }
    while (L >= kGraphTicks && e == cudaSuccess) {
      e = cudaGraphLaunch(b->graph, b->stream);
      L -= kGraphTicks;
      b->tick += kGraphTicks;
      b->launches += (uint64_t)kGraphTicks * launches_per_tick(b) + 1;
    }
  }
  if (e == cudaSuccess && L > 0) {
    for (uint32_t k = 0; k < L; ++k) launch_tick(b, b->shape, k);
    advance_tick_kernel<<<1, 1, 0, b->stream>>>(b->d_tick, (uint32_t)L);
    b->tick += L;
    b->launches += L * launches_per_tick(b) + 1;
    e = cudaGetLastError();
  }
  return e;
}

int free_run(hsga_batch *b, HostRun &R) {
  for (int j = 0; j < 2; ++j) {
    device_free(b->alloc, R.trait[j], b->stream);
    device_free(b->alloc, R.surf[j], b->stream);
    R.trait[j] = nullptr;
    R.surf[j] = nullptr;
  }
  R.live = false;
  b->runs_dirty = true;
  b->items_dirty = true;
  return HSGA_OK;
}

// generation reached by run R at the batch's current tick, and its plane
uint64_t run_generation(const hsga_batch *b, const HostRun &R) {
  const uint64_t t = std::min(b->tick, R.start_tick + R.budget);
  return t - R.start_tick;
}

}  // namespace

extern "C" {

int hsga_batch_create(void *cuda_stream, hsga_batch **out) {
  if (!out) return HSGA_ERR_INVALID_ARG;
  *out = nullptr;
  hsga_batch *b = new (std::nothrow) hsga_batch();
  if (!b) return HSGA_ERR_OOM;
  b->stream = (cudaStream_t)cuda_stream;
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return HSGA_ERR_CUDA;
    }
    b->own_stream = true;
  }
  b->alloc = current_allocator();
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  b->d_tick = (uint32_t *)device_alloc(b->alloc, sizeof(uint32_t), b->stream);
  if (!b->d_tick) {
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return HSGA_ERR_OOM;
  }
  set_tick_kernel<<<1, 1, 0, b->stream>>>(b->d_tick, 0);
  if (cudaGetLastError() != cudaSuccess) {
    device_free(b->alloc, b->d_tick, b->stream);
    delete b;
    return HSGA_ERR_CUDA;
  }
  *out = b;
  return HSGA_OK;
}

int hsga_batch_add(hsga_batch *b, const hsga_config *cfg, uint64_t generations,
                   uint32_t *run_id) {
  if (!b || !run_id) return HSGA_ERR_INVALID_ARG;
  const int v = validate_config(cfg);
  if (v != HSGA_OK) return v;
  if (cfg->migration_mode != HSGA_MIGRATION_SYNC || cfg->fitness != HSGA_FITNESS_TRAIT ||
      cfg->surface_words > 1)
    return HSGA_ERR_UNSUPPORTED;
  if (b->tick + generations > kMaxTick) return HSGA_ERR_INVALID_ARG;
  HostRun R;
  R.cfg = *cfg;
  R.p = params_from_config(cfg);
  R.budget = generations;
  R.start_tick = b->tick;
  R.agents = (uint64_t)R.p.islands * R.p.n;
  bool ok = true;
  for (int j = 0; j < 2; ++j) {
    R.trait[j] = (uint32_t *)device_alloc(b->alloc, sizeof(uint32_t) * R.agents, b->stream);
    R.surf[j] = (uint64_t *)device_alloc(b->alloc, sizeof(uint64_t) * R.agents, b->stream);
    ok = ok && R.trait[j] && R.surf[j];
  }
  R.live = true;
  if (!ok) {
    free_run(b, R);
    return HSGA_ERR_OOM;
  }
  // founders in the plane the run starts from
  const int par = (int)(b->tick & 1);
  cudaError_t e = cudaMemsetAsync(R.trait[par], 0, sizeof(uint32_t) * R.agents, b->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(R.surf[par], 0, sizeof(uint64_t) * R.agents, b->stream);
  if (e != cudaSuccess) {
    free_run(b, R);
    return HSGA_ERR_CUDA;
  }
  b->runs.push_back(R);
  b->runs_dirty = true;
  b->items_dirty = true;
  *run_id = (uint32_t)(b->runs.size() - 1);
  return HSGA_OK;
}

int hsga_batch_run(hsga_batch *b, uint64_t ticks) {
  if (!b) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(b->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  cudaError_t e = upload_runs(b);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? HSGA_ERR_OOM : HSGA_ERR_CUDA;
  uint64_t left = ticks;
  while (left > 0) {
    uint64_t phase_end = b->tick + left;
    bool any = false;
    for (const HostRun &R : b->runs)
      if (active_at(R, b->tick)) {
        any = true;
        phase_end = std::min(phase_end, R.start_tick + R.budget);
      }
    if (!any) break;
    if (b->items_dirty) {
      e = rebuild_items(b);
      if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? HSGA_ERR_OOM : HSGA_ERR_CUDA;
    }
    select_active_prefix(b);
    b->phases++;
    for (const HostRun &R : b->runs)
      if (active_at(R, b->tick))
        b->replications += R.agents * (phase_end - b->tick);
    uint64_t L = phase_end - b->tick;
    left -= L;
    e = autotune(b, &L);
    if (e == cudaSuccess) e = run_ticks(b, L);
    if (e != cudaSuccess) return HSGA_ERR_CUDA;
  }
  return HSGA_OK;
}

int hsga_batch_info(const hsga_batch *b, uint32_t run, hsga_batch_run_info *out) {
  if (!b || !out || run >= b->runs.size()) return HSGA_ERR_INVALID_ARG;
  const HostRun &R = b->runs[run];
  memset(out, 0, sizeof(*out));
  out->generation = run_generation(b, R);
  out->budget = R.budget;
  out->agents = R.agents;
  out->done = out->generation >= R.budget ? 1u : 0u;
  out->live = R.live ? 1u : 0u;
  return HSGA_OK;
}

int hsga_batch_get_population(hsga_batch *b, uint32_t run, uint32_t *trait, uint64_t *surf) {
  if (!b || !trait || run >= b->runs.size() || !b->runs[run].live) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(b->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  const HostRun &R = b->runs[run];
  const int par = (int)((R.start_tick + run_generation(b, R)) & 1);
  cudaError_t e = cudaMemcpyAsync(trait, R.trait[par], sizeof(uint32_t) * R.agents,
                                  cudaMemcpyDefault, b->stream);
  if (e == cudaSuccess && surf)
    e = cudaMemcpyAsync(surf, R.surf[par], sizeof(uint64_t) * R.agents, cudaMemcpyDefault,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? HSGA_OK : HSGA_ERR_CUDA;
}

int hsga_batch_sample(hsga_batch *b, uint32_t run, uint32_t k, uint32_t *out_words,
                      uint32_t *out_island_slot) {
  if (!b || run >= b->runs.size() || !b->runs[run].live || (k > 0 && !out_words))
    return HSGA_ERR_INVALID_ARG;
  const HostRun &R = b->runs[run];
  if (k > R.p.islands) return HSGA_ERR_INVALID_ARG;
  if (k == 0) return HSGA_OK;
  if (stream_capturing(b->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  const uint64_t G = run_generation(b, R);
  const int par = (int)((R.start_tick + G) & 1);
  const size_t scratch_bytes = sample_scratch_bytes(R.p, k);
  uint32_t *scratch = scratch_bytes
                          ? (uint32_t *)device_alloc(b->alloc, scratch_bytes, b->stream)
                          : nullptr;
  uint32_t *staging = (uint32_t *)device_alloc(b->alloc, sizeof(uint32_t) * 6 * k, b->stream);
  if ((scratch_bytes && !scratch) || !staging) {
    device_free(b->alloc, scratch, b->stream);
    device_free(b->alloc, staging, b->stream);
    return HSGA_ERR_OOM;
  }
  cudaError_t e = launch_sample(R.p, (uint32_t)G, k, R.trait[par], R.surf[par], staging,
                                staging + 4 * (size_t)k, scratch, b->stream);
  b->launches++;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_words, staging, sizeof(uint32_t) * 4 * k, cudaMemcpyDefault,
                        b->stream);
  if (e == cudaSuccess && out_island_slot)
    e = cudaMemcpyAsync(out_island_slot, staging + 4 * (size_t)k, sizeof(uint32_t) * 2 * k,
                        cudaMemcpyDefault, b->stream);
  device_free(b->alloc, scratch, b->stream);
  device_free(b->alloc, staging, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? HSGA_OK : HSGA_ERR_CUDA;
}

int hsga_batch_remove(hsga_batch *b, uint32_t run) {
  if (!b || run >= b->runs.size() || !b->runs[run].live) return HSGA_ERR_INVALID_ARG;
  return free_run(b, b->runs[run]);
}

int hsga_batch_get_stats(const hsga_batch *b, hsga_batch_stats *out) {
  if (!b || !out) return HSGA_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->tick = b->tick;
  out->replications = b->replications;
  out->kernel_launches = b->launches;
  out->phases = b->phases;
  out->threads_per_block = (uint32_t)b->shape.threads;
  out->blocks = (uint32_t)(b->shape.blocks[0] + b->shape.blocks[1]);
  for (const HostRun &R : b->runs) {
    if (R.live) {
      out->live_runs++;
      out->device_bytes += R.agents * 24;
    }
    if (active_at(R, b->tick)) out->active_runs++;
  }
  return HSGA_OK;
}

int hsga_run_footprint(const hsga_config *cfg, uint64_t *bytes) {
  if (!bytes) return HSGA_ERR_INVALID_ARG;
  const int v = validate_config(cfg);
  if (v != HSGA_OK) return v;
  const uint64_t agents = (uint64_t)cfg->rows * cfg->cols * cfg->agents_per_island;
  *bytes = agents * 24 + sizeof(BatchRun) + sizeof(WorkItem) * ((uint64_t)cfg->rows * cfg->cols / kGroup + 1);
  return HSGA_OK;
}

int hsga_batch_synchronize(hsga_batch *b) {
  if (!b) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(b->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? HSGA_OK : HSGA_ERR_CUDA;
}

void hsga_batch_destroy(hsga_batch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (HostRun &R : b->runs)
    if (R.live) free_run(b, R);
  device_free(b->alloc, b->d_runs, b->stream);
  for (int c = 0; c < 2; ++c) device_free(b->alloc, b->d_items[c], b->stream);
  device_free(b->alloc, b->d_tick, b->stream);
  cudaStreamSynchronize(b->stream);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
