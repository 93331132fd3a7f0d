// hsga_capi.cu -- C-ABI runtime: grid lifetime, device memory, dispatch of
// the generation kernels, checkpointing, and the host-side site / lookup
// functions.  Declarations and contracts: include/hsga.h.
#include <cmath>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "hsga.h"
#include "hsga_internal.h"

using namespace hsga;

namespace {

struct Allocator {
  hsga_alloc_fn alloc = nullptr;
  hsga_free_fn free_fn = nullptr;
  void *ctx = nullptr;
};
Allocator g_allocator;

constexpr uint64_t kCheckpointMagic = 0x3130485341475348ull;  // "HSGAH01"
constexpr uint64_t kMaxGeneration = 0xFFFFFFFFull - 64;        // Philox counter word

}  // namespace

struct hsga_grid {
  hsga_config cfg;
  RunParams p;
  Allocator alloc;
  cudaStream_t stream = nullptr;
  uint64_t agents = 0;
  uint64_t swords = 0;     // surface words in a population: agents x K
  bool wide = false;       // K > 1
  uint64_t *wrec = nullptr;  // wide migrant records: islands x (K + 1)
  uint32_t *trait[2] = {nullptr, nullptr};
  uint64_t *surf[2] = {nullptr, nullptr};
  int cur = 0;
  uint4 *rec = nullptr;      // migrant records, 64 B per island (two stamped 4-word slots)
  int *err = nullptr;        // device error word
  uint32_t *sample_scratch = nullptr;
  size_t sample_scratch_bytes = 0;
  // fossil sampling: k genomes every `fossil_every` generations
  uint64_t fossil_every = 0;
  uint32_t fossil_k = 0, fossil_cap = 0, fossil_count = 0;
  uint64_t fossil_dropped = 0;
  uint32_t *fossil_words = nullptr;  // fossil_cap x 4
  uint32_t *fossil_where = nullptr;  // fossil_cap x 2
  // free-running migration: per-genome counters, last stamp seen per
  // (island, direction), optional take log
  bool async = false;     // either free-running mode
  bool buffered = false;  // per-neighbour buffers
  uint32_t *tcount = nullptr;
  uint32_t *seen = nullptr;
  // buffered mode, per island and direction: the channel's genome in flight
  // (4 self-stamped words), its acknowledgement, the receive buffer and the
  // lane state {posts, taken, waiting, 0}
  uint64_t *mail = nullptr;
  uint32_t *ack = nullptr;
  uint4 *inbuf = nullptr;
  uint4 *chst = nullptr;
  uint32_t *alog = nullptr;
  uint32_t alog_gens = 0;
  uint32_t octet_slice = 1;  // free-running: generations per octet visit
  uint64_t alog_G0 = 0;
  uint64_t G = 0;
  bool premigrated = false;
  bool resident = false;
  ResidentPlan plan;
  bool broken = false;
  uint64_t replications = 0;
  uint64_t launches = 0;
};

namespace {

void *dev_alloc(const Allocator &a, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (a.alloc) return a.alloc(bytes, (void *)s, a.ctx);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(const Allocator &a, void *ptr, cudaStream_t s) {
  if (!ptr) return;
  if (a.free_fn) a.free_fn(ptr, (void *)s, a.ctx);
  else cudaFreeAsync(ptr, s);
}

bool is_device_ptr(const void *ptr) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HSGA_OK : HSGA_ERR_CUDA; }

bool power_of_two(uint32_t x) { return x && !(x & (x - 1)); }

int validate(const hsga_config *c) {
  if (!c) return HSGA_ERR_INVALID_ARG;
  if (c->rows == 0 || c->cols == 0) return HSGA_ERR_INVALID_ARG;
  if ((uint64_t)c->rows * c->cols >= 0xFFFFFFF0ull) return HSGA_ERR_INVALID_ARG;
  if (c->agents_per_island == 0 || c->agents_per_island > 64) return HSGA_ERR_INVALID_ARG;
  // agent offsets are 32-bit in the kernels
  if ((uint64_t)c->rows * c->cols * c->agents_per_island >= 0xFFFFFFFFull)
    return HSGA_ERR_INVALID_ARG;
  if (c->tournament_size == 0 || c->tournament_size > 64) return HSGA_ERR_INVALID_ARG;
  if (c->surface_policy > HSGA_HYBRID) return HSGA_ERR_INVALID_ARG;
  const uint32_t b = c->differentia_bits;
  if (!(b == 1 || b == 2 || b == 4 || b == 8 || b == 16)) return HSGA_ERR_INVALID_ARG;
  const uint32_t K = c->surface_words;
  if (!(K <= 2 || K == 4)) return HSGA_ERR_INVALID_ARG;
  const uint32_t S = 64 * (K > 1 ? K : 1) / b, W = c->sites_per_level;
  if (c->surface_policy == HSGA_TILTED || c->surface_policy == HSGA_STRETCHED) {
    if (!(W == 1 || W == 2 || W == 4) || S / W < 2) return HSGA_ERR_INVALID_ARG;
  }
  if (c->surface_policy == HSGA_HYBRID) {  // two halves of S/2 sites each
    if (!(W == 1 || W == 2 || W == 4) || (S / 2) / W < 2) return HSGA_ERR_INVALID_ARG;
  }
  if (!(c->p_beneficial >= 0.0 && c->p_beneficial <= 1.0)) return HSGA_ERR_INVALID_ARG;
  if (!(c->p_deleterious >= 0.0 && c->p_deleterious <= 1.0)) return HSGA_ERR_INVALID_ARG;
  if (c->p_beneficial + c->p_deleterious > 1.0) return HSGA_ERR_INVALID_ARG;
  if (c->kernel > HSGA_KERNEL_RESIDENT_GRID || c->reserved != 0) return HSGA_ERR_INVALID_ARG;
  if (c->fitness > HSGA_FITNESS_FLOAT) return HSGA_ERR_INVALID_ARG;
  if (K > 1) {  // wide surfaces: the synchronous warp-per-island path
    if (c->surface_policy == HSGA_NONE || c->agents_per_island > 32) return HSGA_ERR_INVALID_ARG;
    if (c->migration_mode != HSGA_MIGRATION_SYNC) return HSGA_ERR_UNSUPPORTED;
    if (c->kernel != HSGA_KERNEL_AUTO && c->kernel != HSGA_KERNEL_STREAMED)
      return HSGA_ERR_UNSUPPORTED;
  }
  if (c->fitness == HSGA_FITNESS_FLOAT) {
    if (!(c->mutation_sigma > 0.0 && c->mutation_sigma < 1e30)) return HSGA_ERR_INVALID_ARG;
    if (c->agents_per_island > 32) return HSGA_ERR_INVALID_ARG;
    if (c->migration_mode == HSGA_MIGRATION_SYNC && c->kernel != HSGA_KERNEL_AUTO &&
        c->kernel != HSGA_KERNEL_STREAMED)
      return HSGA_ERR_UNSUPPORTED;
  }
  if (c->migration_mode > HSGA_MIGRATION_BUFFERED) return HSGA_ERR_INVALID_ARG;
  if (c->migration_mode != HSGA_MIGRATION_SYNC &&
      (c->agents_per_island > 32 || c->deposit_interval > 1))
    return HSGA_ERR_INVALID_ARG;
  return HSGA_OK;
}

uint64_t threshold(double p) { return (uint64_t)(p * 4294967296.0); }

RunParams make_params(const hsga_config *c) {
  RunParams p{};
  p.rows = c->rows;
  p.cols = c->cols;
  p.n = c->agents_per_island;
  p.islands = c->rows * c->cols;
  p.tournament = c->tournament_size;
  p.k0 = (uint32_t)c->seed;
  p.k1 = (uint32_t)(c->seed >> 32);
  p.policy = c->surface_policy;
  p.bits = c->differentia_bits;
  p.words = c->surface_words > 1 ? c->surface_words : 1;
  p.S = 64 * p.words / p.bits;
  p.W = (c->surface_policy == HSGA_TILTED || c->surface_policy == HSGA_STRETCHED ||
         c->surface_policy == HSGA_HYBRID)
            ? c->sites_per_level
            : 2;
  p.coarsen = c->deposit_interval > 1 ? c->deposit_interval : 1;
  p.interval = c->migration_interval;
  const uint64_t thr_ben = threshold(c->p_beneficial);
  const uint64_t thr_bd = thr_ben + threshold(c->p_deleterious);  // <= 2^32 (validated)
  p.ben32 = (uint32_t)thr_ben;
  p.ben_all = thr_ben >= (1ull << 32) ? 1u : 0u;
  p.bd32 = (uint32_t)thr_bd;
  p.bd_all = thr_bd >= (1ull << 32) ? 1u : 0u;
  p.has_del = thr_bd > thr_ben ? 1u : 0u;
  p.vmask = (1ull << p.bits) - 1;
  p.levels = p.S / p.W;
  p.levels_half = (p.S / 2) / p.W;
  p.flt = c->fitness == HSGA_FITNESS_FLOAT ? 1u : 0u;
  p.gscale = p.flt ? (float)(c->mutation_sigma / sqrt(24.0 + 1.0 / 12.0) / 16777216.0) : 0.0f;
  p.cols_div = make_fastdiv(p.cols);
  set_round_keys(p);
  return p;
}

int fetch_device_error(hsga_grid *g) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  if (h == kDevErrWaitTimeout) {
    g->broken = true;
    return HSGA_ERR_WAIT_TIMEOUT;
  }
  if (h != 0) {
    g->broken = true;
    return HSGA_ERR_DEVICE;
  }
  return HSGA_OK;
}

void free_grid(hsga_grid *g) {
  if (!g) return;
  for (int i = 0; i < 2; ++i) {
    dev_free(g->alloc, g->trait[i], g->stream);
    dev_free(g->alloc, g->surf[i], g->stream);
  }
  dev_free(g->alloc, g->rec, g->stream);
  dev_free(g->alloc, g->wrec, g->stream);
  dev_free(g->alloc, g->err, g->stream);
  dev_free(g->alloc, g->sample_scratch, g->stream);
  dev_free(g->alloc, g->fossil_words, g->stream);
  dev_free(g->alloc, g->fossil_where, g->stream);
  dev_free(g->alloc, g->tcount, g->stream);
  dev_free(g->alloc, g->seen, g->stream);
  dev_free(g->alloc, g->mail, g->stream);
  dev_free(g->alloc, g->ack, g->stream);
  dev_free(g->alloc, g->inbuf, g->stream);
  dev_free(g->alloc, g->chst, g->stream);
  dev_free(g->alloc, g->alog, g->stream);
  cudaStreamSynchronize(g->stream);
  delete g;
}

// Copy count elements of `bytes_each` between host/device `src` and device `dst`.
cudaError_t copy_in(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
}

__global__ void fill_u32_kernel(uint32_t *dst, uint32_t value, uint64_t count) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x)
    dst[i] = value;
}

cudaError_t fill_u32(uint32_t *dst, uint32_t value, uint64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint64_t blocks = (count + 255) / 256;
  fill_u32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(dst, value, count);
  return cudaGetLastError();
}

// Empties the buffered mode's channels: nothing in flight, nothing waiting,
// post numbers restart at 1.
cudaError_t reset_channels(hsga_grid *g) {
  if (!g->buffered) return cudaSuccess;
  const size_t C = 4 * (size_t)g->p.islands;
  cudaError_t e = cudaMemsetAsync(g->mail, 0, sizeof(uint64_t) * 4 * C, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->ack, 0, sizeof(uint32_t) * C, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->chst, 0, sizeof(uint4) * C, g->stream);
  return e;
}

int reset_sync_state(hsga_grid *g) {
  // records of an earlier run must not carry an expected stamp
  cudaError_t e = cudaMemsetAsync(g->rec, 0, sizeof(uint4) * 4 * (size_t)g->p.islands, g->stream);
  if (e == cudaSuccess) e = reset_channels(g);
  if (e == cudaSuccess && g->seen)
    e = cudaMemsetAsync(g->seen, 0, sizeof(uint32_t) * 4 * (size_t)g->p.islands, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->err, 0, sizeof(int), g->stream);
  g->broken = false;
  g->premigrated = false;
  return cuda_status(e);
}

}  // namespace

extern "C" {

int hsga_version(void) { return 100; }

const char *hsga_status_string(int s) {
  switch (s) {
    case HSGA_OK: return "ok";
    case HSGA_ERR_INVALID_ARG: return "invalid argument";
    case HSGA_ERR_OOM: return "device allocation failed";
    case HSGA_ERR_CUDA: return "CUDA runtime error";
    case HSGA_ERR_DEVICE: return "kernel reported an inconsistent state";
    case HSGA_ERR_WAIT_TIMEOUT: return "bounded device wait timed out";
    case HSGA_ERR_UNSUPPORTED: return "unsupported";
    case HSGA_ERR_NOT_CAPTURABLE: return "call waits for a stream under graph capture";
    default: return "unknown status";
  }
}

int hsga_set_allocator(hsga_alloc_fn alloc, hsga_free_fn free_fn, void *ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return HSGA_ERR_INVALID_ARG;
  g_allocator.alloc = alloc;
  g_allocator.free_fn = free_fn;
  g_allocator.ctx = ctx;
  return HSGA_OK;
}

int hsga_init_grid(const hsga_config *cfg, void *cuda_stream, hsga_grid **out) {
  if (!out) return HSGA_ERR_INVALID_ARG;
  *out = nullptr;
  int v = validate(cfg);
  if (v != HSGA_OK) return v;
  hsga_grid *g = new (std::nothrow) hsga_grid();
  if (!g) return HSGA_ERR_OOM;
  g->cfg = *cfg;
  g->p = make_params(cfg);
  g->alloc = g_allocator;
  g->stream = (cudaStream_t)cuda_stream;
  g->agents = (uint64_t)g->p.islands * g->p.n;
  g->swords = g->agents * g->p.words;
  g->wide = g->p.words > 1;
  const bool tracked = cfg->surface_policy != HSGA_NONE;
  for (int i = 0; i < 2; ++i) {
    g->trait[i] = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * g->agents, g->stream);
    g->surf[i] = tracked ? (uint64_t *)dev_alloc(g->alloc, sizeof(uint64_t) * g->swords, g->stream)
                         : nullptr;
  }
  g->rec = (uint4 *)dev_alloc(g->alloc, sizeof(uint4) * 4 * (size_t)g->p.islands, g->stream);
  g->async = cfg->migration_mode != HSGA_MIGRATION_SYNC;
  g->buffered = cfg->migration_mode == HSGA_MIGRATION_BUFFERED;
  if (g->async) {
    const size_t C = 4 * (size_t)g->p.islands;
    g->tcount = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * g->agents, g->stream);
    g->seen = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * C, g->stream);
    bool ok = g->tcount && g->seen;
    if (g->buffered) {
      g->mail = (uint64_t *)dev_alloc(g->alloc, sizeof(uint64_t) * 4 * C, g->stream);
      g->ack = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * C, g->stream);
      g->inbuf = (uint4 *)dev_alloc(g->alloc, sizeof(uint4) * 4 * C, g->stream);
      g->chst = (uint4 *)dev_alloc(g->alloc, sizeof(uint4) * C, g->stream);
      ok = ok && g->mail && g->ack && g->inbuf && g->chst;
    }
    if (!ok) {
      free_grid(g);
      return HSGA_ERR_OOM;
    }
    if (cudaMemsetAsync(g->tcount, 0, sizeof(uint32_t) * g->agents, g->stream) != cudaSuccess) {
      free_grid(g);
      return HSGA_ERR_CUDA;
    }
  }
  if (g->wide) {
    g->wrec = (uint64_t *)dev_alloc(g->alloc, sizeof(uint64_t) * (g->p.words + 1) *
                                                  (size_t)g->p.islands, g->stream);
    if (!g->wrec) {
      free_grid(g);
      return HSGA_ERR_OOM;
    }
  }
  g->err = (int *)dev_alloc(g->alloc, sizeof(int), g->stream);
  bool ok = g->trait[0] && g->trait[1] && g->rec && g->err &&
            (!tracked || (g->surf[0] && g->surf[1]));
  if (!ok) {
    free_grid(g);
    return HSGA_ERR_OOM;
  }
  cudaError_t e = cudaMemsetAsync(g->trait[0], 0, sizeof(uint32_t) * g->agents, g->stream);
  if (e == cudaSuccess && tracked)
    e = cudaMemsetAsync(g->surf[0], 0, sizeof(uint64_t) * g->swords, g->stream);
  if (e != cudaSuccess || reset_sync_state(g) != HSGA_OK) {
    free_grid(g);
    return HSGA_ERR_CUDA;
  }
  g->resident = false;
  if (cfg->kernel != HSGA_KERNEL_STREAMED && !g->async && !g->p.flt && !g->wide) {
    g->resident = resident_plan(g->p, &g->plan, cfg->kernel == HSGA_KERNEL_RESIDENT_GRID);
    if (!g->resident && cfg->kernel >= HSGA_KERNEL_RESIDENT) {
      free_grid(g);
      return HSGA_ERR_UNSUPPORTED;
    }
  }
  *out = g;
  return HSGA_OK;
}

int hsga_set_population(hsga_grid *g, const uint32_t *trait, const uint64_t *surf,
                        uint64_t generation) {
  if (!g || !trait || generation > kMaxGeneration) return HSGA_ERR_INVALID_ARG;
  const bool tracked = g->surf[0] != nullptr;
  if (tracked && !surf) return HSGA_ERR_INVALID_ARG;
  if ((!is_device_ptr(trait) || (tracked && !is_device_ptr(surf))) && stream_capturing(g->stream))
    return HSGA_ERR_NOT_CAPTURABLE;
  g->cur = 0;
  cudaError_t e = copy_in(g->trait[0], trait, sizeof(uint32_t) * g->agents, g->stream);
  if (e == cudaSuccess && tracked)
    e = copy_in(g->surf[0], surf, sizeof(uint64_t) * g->swords, g->stream);
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  g->G = generation;
  if (g->async && fill_u32(g->tcount, (uint32_t)generation, g->agents, g->stream) != cudaSuccess)
    return HSGA_ERR_CUDA;
  int r = reset_sync_state(g);
  if (r != HSGA_OK) return r;
  // host sources may be reused on return
  if (!is_device_ptr(trait) || (tracked && !is_device_ptr(surf)))
    return cuda_status(cudaStreamSynchronize(g->stream));
  return HSGA_OK;
}

int hsga_get_population(hsga_grid *g, uint32_t *trait, uint64_t *surf) {
  if (!g || !trait) return HSGA_ERR_INVALID_ARG;
  const bool tracked = g->surf[0] != nullptr;
  if ((!is_device_ptr(trait) || (surf && !is_device_ptr(surf))) && stream_capturing(g->stream))
    return HSGA_ERR_NOT_CAPTURABLE;
  cudaError_t e = cudaMemcpyAsync(trait, g->trait[g->cur], sizeof(uint32_t) * g->agents,
                                  cudaMemcpyDefault, g->stream);
  if (e == cudaSuccess && surf) {
    if (tracked)
      e = cudaMemcpyAsync(surf, g->surf[g->cur], sizeof(uint64_t) * g->swords, cudaMemcpyDefault,
                          g->stream);
    else
      e = is_device_ptr(surf) ? cudaMemsetAsync(surf, 0, sizeof(uint64_t) * g->swords, g->stream)
                              : (memset(surf, 0, sizeof(uint64_t) * g->swords), cudaSuccess);
  }
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  if (!is_device_ptr(trait) || (surf && !is_device_ptr(surf)))
    return cuda_status(cudaStreamSynchronize(g->stream));
  return HSGA_OK;
}

namespace {

int ensure_sample_scratch(hsga_grid *g, uint32_t k) {
  const size_t scratch = sample_scratch_bytes(g->p, k);
  if (scratch > g->sample_scratch_bytes) {
    dev_free(g->alloc, g->sample_scratch, g->stream);
    g->sample_scratch = (uint32_t *)dev_alloc(g->alloc, scratch, g->stream);
    g->sample_scratch_bytes = g->sample_scratch ? scratch : 0;
    if (!g->sample_scratch) return HSGA_ERR_OOM;
  }
  return HSGA_OK;
}

int advance(hsga_grid *g, uint64_t n);

// One fossil sample at the current generation into the fossil buffer.
int take_fossils(hsga_grid *g) {
  if (g->fossil_count + g->fossil_k > g->fossil_cap) {
    g->fossil_dropped += g->fossil_k;
    return HSGA_OK;
  }
  const int r = ensure_sample_scratch(g, g->fossil_k);
  if (r != HSGA_OK) return r;
  cudaError_t e = launch_sample(g->p, (uint32_t)g->G, g->fossil_k, g->trait[g->cur],
                                g->surf[g->cur], g->fossil_words + 4 * (size_t)g->fossil_count,
                                g->fossil_where + 2 * (size_t)g->fossil_count, g->sample_scratch,
                                g->stream, g->tcount);
  g->launches++;
  g->fossil_count += g->fossil_k;
  return cuda_status(e);
}

}  // namespace

int hsga_run_generations(hsga_grid *g, uint64_t n) {
  if (!g) return HSGA_ERR_INVALID_ARG;
  if (g->broken) return HSGA_ERR_DEVICE;
  if (n == 0) return HSGA_OK;
  if (g->G + n > kMaxGeneration) return HSGA_ERR_INVALID_ARG;
  if (!g->fossil_every) return advance(g, n);
  // stop at every multiple of the fossil interval to sample
  uint64_t left = n;
  while (left > 0) {
    const uint64_t to_next = g->fossil_every - (g->G % g->fossil_every);
    const uint64_t step = left < to_next ? left : to_next;
    int r = advance(g, step);
    if (r != HSGA_OK) return r;
    left -= step;
    if (g->G % g->fossil_every == 0) {
      r = take_fossils(g);
      if (r != HSGA_OK) return r;
    }
  }
  return HSGA_OK;
}

namespace {
int advance(hsga_grid *g, uint64_t n) {
  cudaError_t e = cudaSuccess;
  if (g->buffered) {
    const uint64_t slice = 1u << 16;
    for (uint64_t done = 0; done < n && e == cudaSuccess;) {
      const uint32_t m = (uint32_t)((n - done) < slice ? (n - done) : slice);
      e = launch_step_buffered(g->p, (uint32_t)(g->G + done), m, g->octet_slice, g->trait[g->cur],
                               g->surf[g->cur], g->tcount, g->mail, g->ack, g->inbuf, g->chst,
                               g->alog, (uint32_t)g->alog_G0, g->alog_gens, g->stream);
      g->launches++;
      done += m;
    }
  } else if (g->async) {
    const uint64_t slice = 1u << 16;
    for (uint64_t done = 0; done < n && e == cudaSuccess;) {
      const uint32_t m = (uint32_t)((n - done) < slice ? (n - done) : slice);
      e = launch_step_async(g->p, (uint32_t)(g->G + done), m, g->octet_slice, g->trait[g->cur],
                            g->surf[g->cur],
                            g->tcount, reinterpret_cast<uint64_t *>(g->rec), g->seen, g->alog,
                            (uint32_t)g->alog_G0, g->alog_gens, g->stream);
      g->launches++;
      done += m;
    }
  } else if (g->resident) {
    // Launch in slices so a single launch stays short.
    const uint64_t slice = 1u << 16;
    uint64_t done = 0;
    while (done < n && e == cudaSuccess) {
      const uint32_t m = (uint32_t)((n - done) < slice ? (n - done) : slice);
      e = launch_step_resident(g->p, g->plan, (uint32_t)(g->G + done), m,
                               g->premigrated && done == 0, g->trait[g->cur], g->surf[g->cur],
                               reinterpret_cast<uint64_t *>(g->rec), g->err, g->stream);
      g->launches++;
      done += m;
    }
  } else if (g->wide) {
    // surfaces of several words: explicit a1 + a2, then one warp per island
    for (uint64_t k = 0; k < n && e == cudaSuccess; ++k) {
      const uint64_t G = g->G + k;
      if (migrates(g->p, G) && !(g->premigrated && k == 0)) {
        e = launch_migrate_wide(g->p, (uint32_t)G, g->trait[g->cur], g->surf[g->cur], g->wrec,
                                g->stream);
        g->launches += 2;
      }
      if (e == cudaSuccess)
        e = launch_step_wide(g->p, (uint32_t)G, g->trait[g->cur], g->surf[g->cur],
                             g->trait[1 - g->cur], g->surf[1 - g->cur], g->stream);
      g->cur = 1 - g->cur;
      g->launches++;
    }
  } else if (g->p.flt) {
    // float fitness, synchronous: explicit a1 + a2, then one warp per island
    for (uint64_t k = 0; k < n && e == cudaSuccess; ++k) {
      const uint64_t G = g->G + k;
      if (migrates(g->p, G) && !(g->premigrated && k == 0)) {
        e = launch_migrate(g->p, (uint32_t)G, g->trait[g->cur], g->surf[g->cur], g->rec,
                           g->stream);
        g->launches += 2;
      }
      if (e == cudaSuccess)
        e = launch_step_float(g->p, (uint32_t)G, g->trait[g->cur], g->surf[g->cur],
                              g->trait[1 - g->cur], g->surf[1 - g->cur], g->stream);
      g->cur = 1 - g->cur;
      g->launches++;
    }
  } else {
    for (uint64_t k = 0; k < n && e == cudaSuccess; ++k) {
      const uint64_t G = g->G + k;
      const bool do_mig = migrates(g->p, G) && !(g->premigrated && k == 0);
      e = launch_step_streamed(g->p, (uint32_t)G, do_mig, g->trait[g->cur], g->surf[g->cur],
                               g->trait[1 - g->cur], g->surf[1 - g->cur], g->err, g->stream);
      g->cur = 1 - g->cur;
      g->launches++;
    }
  }
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  g->G += n;
  g->premigrated = false;
  g->replications += n * g->agents;
  return HSGA_OK;
}
}  // namespace

int hsga_set_fossil_sampling(hsga_grid *g, uint64_t every, uint32_t k, uint32_t capacity) {
  if (!g) return HSGA_ERR_INVALID_ARG;
  if (g->wide && every) return HSGA_ERR_UNSUPPORTED;
  if (every && (k == 0 || k > g->p.islands || capacity < k)) return HSGA_ERR_INVALID_ARG;
  dev_free(g->alloc, g->fossil_words, g->stream);
  dev_free(g->alloc, g->fossil_where, g->stream);
  g->fossil_words = g->fossil_where = nullptr;
  g->fossil_every = 0;
  g->fossil_k = g->fossil_cap = g->fossil_count = 0;
  g->fossil_dropped = 0;
  if (!every) return HSGA_OK;
  g->fossil_words = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * 4 * (size_t)capacity,
                                          g->stream);
  g->fossil_where = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * 2 * (size_t)capacity,
                                          g->stream);
  if (!g->fossil_words || !g->fossil_where) {
    dev_free(g->alloc, g->fossil_words, g->stream);
    dev_free(g->alloc, g->fossil_where, g->stream);
    g->fossil_words = g->fossil_where = nullptr;
    return HSGA_ERR_OOM;
  }
  g->fossil_every = every;
  g->fossil_k = k;
  g->fossil_cap = capacity;
  return HSGA_OK;
}

int hsga_get_fossils(hsga_grid *g, uint32_t *out_words, uint32_t *out_island_slot,
                     uint32_t max_records, uint32_t *count) {
  if (!g || !count) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  *count = g->fossil_count;
  const uint32_t m = g->fossil_count < max_records ? g->fossil_count : max_records;
  if (m == 0) return HSGA_OK;
  if (!out_words) return HSGA_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(out_words, g->fossil_words, sizeof(uint32_t) * 4 * (size_t)m,
                                  cudaMemcpyDefault, g->stream);
  if (e == cudaSuccess && out_island_slot)
    e = cudaMemcpyAsync(out_island_slot, g->fossil_where, sizeof(uint32_t) * 2 * (size_t)m,
                        cudaMemcpyDefault, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  return cuda_status(e);
}

int hsga_get_counters(hsga_grid *g, uint32_t *T_out) {
  if (!g || !T_out) return HSGA_ERR_INVALID_ARG;
  cudaError_t e;
  const bool dev = is_device_ptr(T_out);
  if (!dev && stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  if (g->async) {
    e = cudaMemcpyAsync(T_out, g->tcount, sizeof(uint32_t) * g->agents, cudaMemcpyDefault,
                        g->stream);
  } else if (dev) {
    e = fill_u32(T_out, (uint32_t)g->G, g->agents, g->stream);
  } else {
    for (uint64_t i = 0; i < g->agents; ++i) T_out[i] = (uint32_t)g->G;
    e = cudaSuccess;
  }
  if (e == cudaSuccess && !dev) e = cudaStreamSynchronize(g->stream);
  return cuda_status(e);
}

int hsga_set_async_log(hsga_grid *g, uint32_t generations) {
  if (!g) return HSGA_ERR_INVALID_ARG;
  if (!g->async) return HSGA_ERR_UNSUPPORTED;
  dev_free(g->alloc, g->alog, g->stream);
  g->alog = nullptr;
  g->alog_gens = 0;
  if (!generations) return HSGA_OK;
  const size_t bytes = sizeof(uint32_t) * 4 * (size_t)g->p.islands * generations;
  g->alog = (uint32_t *)dev_alloc(g->alloc, bytes, g->stream);
  if (!g->alog) return HSGA_ERR_OOM;
  cudaError_t e = cudaMemsetAsync(g->alog, 0, bytes, g->stream);
  // a fresh window: nothing published before it can be taken
  if (e == cudaSuccess)
    e = cudaMemsetAsync(g->rec, 0, sizeof(uint4) * 4 * (size_t)g->p.islands, g->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(g->seen, 0, sizeof(uint32_t) * 4 * (size_t)g->p.islands, g->stream);
  if (e == cudaSuccess) e = reset_channels(g);
  g->alog_gens = generations;
  g->alog_G0 = g->G;
  return cuda_status(e);
}

int hsga_set_octet_slice(hsga_grid *g, uint32_t generations) {
  if (!g) return HSGA_ERR_INVALID_ARG;
  if (!g->async) return HSGA_ERR_UNSUPPORTED;
  if (generations == 0 || generations > (1u << 16)) return HSGA_ERR_INVALID_ARG;
  g->octet_slice = generations;
  return HSGA_OK;
}

int hsga_get_async_log(hsga_grid *g, uint32_t *out) {
  if (!g || !out) return HSGA_ERR_INVALID_ARG;
  if (!g->alog) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  cudaError_t e = cudaMemcpyAsync(out, g->alog,
                                  sizeof(uint32_t) * 4 * (size_t)g->p.islands * g->alog_gens,
                                  cudaMemcpyDefault, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  return cuda_status(e);
}

int hsga_get_migration_buffers(hsga_grid *g, uint32_t *chan_out, uint32_t *inbuf_out) {
  if (!g || !chan_out) return HSGA_ERR_INVALID_ARG;
  if (!g->buffered) return HSGA_ERR_UNSUPPORTED;
  if (stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  const size_t C = 4 * (size_t)g->p.islands;
  // {posts, taken, waiting, 0} per channel -> 3 words per channel
  cudaError_t e = cudaMemcpy2DAsync(chan_out, 3 * sizeof(uint32_t), g->chst, sizeof(uint4),
                                    3 * sizeof(uint32_t), C, cudaMemcpyDefault, g->stream);
  if (e == cudaSuccess && inbuf_out)
    e = cudaMemcpyAsync(inbuf_out, g->inbuf, sizeof(uint4) * 4 * C, cudaMemcpyDefault,
                        g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  return cuda_status(e);
}

int hsga_migrate(hsga_grid *g) {
  if (!g) return HSGA_ERR_INVALID_ARG;
  if (g->broken) return HSGA_ERR_DEVICE;
  if (g->async) return HSGA_ERR_UNSUPPORTED;
  if (g->premigrated) return HSGA_ERR_INVALID_ARG;
  cudaError_t e = g->wide ? launch_migrate_wide(g->p, (uint32_t)g->G, g->trait[g->cur],
                                                g->surf[g->cur], g->wrec, g->stream)
                          : launch_migrate(g->p, (uint32_t)g->G, g->trait[g->cur],
                                           g->surf[g->cur], g->rec, g->stream);
  g->launches += 2;
  // the explicit records share the buffer with the resident kernel's stamped
  // records: clear them so no stale word can carry an expected stamp
  if (e == cudaSuccess && g->resident)
    e = cudaMemsetAsync(g->rec, 0, sizeof(uint4) * 4 * (size_t)g->p.islands, g->stream);
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  g->premigrated = true;
  return HSGA_OK;
}

int hsga_sample_surfaces(hsga_grid *g, uint32_t k, uint32_t *out_words,
                         uint32_t *out_island_slot) {
  if (!g || (k > 0 && !out_words)) return HSGA_ERR_INVALID_ARG;
  if (k > g->p.islands) return HSGA_ERR_INVALID_ARG;
  if (k == 0) return HSGA_OK;
  if (stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  const int sr = ensure_sample_scratch(g, k);
  if (sr != HSGA_OK) return sr;
  if (g->wide) {
    // pick (island, slot) as for one-word surfaces, then gather wide records
    const size_t rw = 2 + 2 * (size_t)g->p.words;
    uint32_t *staging = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * (6 + rw) * (size_t)k,
                                              g->stream);
    if (!staging) return HSGA_ERR_OOM;
    uint32_t *pick = staging + 4 * (size_t)k, *wide = staging + 6 * (size_t)k;
    cudaError_t e = launch_sample(g->p, (uint32_t)g->G, k, g->trait[g->cur], nullptr, staging,
                                  pick, g->sample_scratch, g->stream, nullptr);
    if (e == cudaSuccess)
      e = launch_gather_wide(g->p, (uint32_t)g->G, k, g->trait[g->cur], g->surf[g->cur], pick,
                             wide, g->stream);
    g->launches += 2;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_words, wide, sizeof(uint32_t) * rw * k, cudaMemcpyDefault,
                          g->stream);
    if (e == cudaSuccess && out_island_slot)
      e = cudaMemcpyAsync(out_island_slot, pick, sizeof(uint32_t) * 2 * k, cudaMemcpyDefault,
                          g->stream);
    dev_free(g->alloc, staging, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    return cuda_status(e);
  }
  // the kernels store 16-byte records and 8-byte pairs: misaligned device
  // outputs go through the staging buffer like host outputs
  const bool dev_words = is_device_ptr(out_words) && ((uintptr_t)out_words % 16) == 0;
  const bool dev_is = out_island_slot == nullptr ||
                      (is_device_ptr(out_island_slot) && ((uintptr_t)out_island_slot % 8) == 0);
  uint32_t *dw = out_words, *di = out_island_slot;
  uint32_t *staging = nullptr;
  if (!dev_words || !dev_is) {
    staging = (uint32_t *)dev_alloc(g->alloc, sizeof(uint32_t) * 6 * (size_t)k, g->stream);
    if (!staging) return HSGA_ERR_OOM;
    if (!dev_words) dw = staging;
    if (!dev_is) di = staging + 4 * (size_t)k;
  }
  cudaError_t e = launch_sample(g->p, (uint32_t)g->G, k, g->trait[g->cur], g->surf[g->cur], dw,
                                di, g->sample_scratch, g->stream, g->tcount);
  g->launches++;
  if (e == cudaSuccess && !dev_words)
    e = cudaMemcpyAsync(out_words, dw, sizeof(uint32_t) * 4 * (size_t)k, cudaMemcpyDefault,
                        g->stream);
  if (e == cudaSuccess && !dev_is)
    e = cudaMemcpyAsync(out_island_slot, di, sizeof(uint32_t) * 2 * (size_t)k, cudaMemcpyDefault,
                        g->stream);
  if (staging) {
    dev_free(g->alloc, staging, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  }
  return cuda_status(e);
}

int hsga_synchronize(hsga_grid *g) {
  if (!g) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  e = cudaGetLastError();
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  return fetch_device_error(g);
}

int hsga_get_stats(const hsga_grid *g, hsga_stats *out) {
  if (!g || !out) return HSGA_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->generation = g->G;
  out->replications = g->replications;
  out->kernel_launches = g->launches;
  out->kernel = !g->resident ? HSGA_KERNEL_STREAMED
                : (g->plan.mode == kBlockSync ? HSGA_KERNEL_RESIDENT : HSGA_KERNEL_RESIDENT_GRID);
  if (g->resident) {
    out->islands_per_warp = (uint32_t)g->plan.ipw;
    out->warps_per_block = (uint32_t)g->plan.warps_per_block;
    out->blocks = (uint32_t)g->plan.blocks;
  }
  out->fossils = g->fossil_count;
  out->fossils_dropped = g->fossil_dropped;
  return HSGA_OK;
}

// Checkpoint layout: magic, config, G, then traits and surfaces.
int hsga_save(hsga_grid *g, void *buf, size_t *len) {
  if (!g || !len) return HSGA_ERR_INVALID_ARG;
  if (buf && stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  if (g->async) return HSGA_ERR_UNSUPPORTED;
  const size_t need = sizeof(uint64_t) * 2 + sizeof(hsga_config) + g->agents * 4 + g->swords * 8;
  if (!buf) {
    *len = need;
    return HSGA_OK;
  }
  if (*len < need) return HSGA_ERR_INVALID_ARG;
  char *p = (char *)buf;
  memcpy(p, &kCheckpointMagic, 8);
  memcpy(p + 8, &g->cfg, sizeof(hsga_config));
  memcpy(p + 8 + sizeof(hsga_config), &g->G, 8);
  uint32_t *t = (uint32_t *)(p + 16 + sizeof(hsga_config));
  uint64_t *s = (uint64_t *)(t + g->agents);
  // surfaces may be unaligned for uint64 in the caller's buffer: stage via get_population
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (g->swords ? g->swords : 1));
  if (!tmp) return HSGA_ERR_OOM;
  int r = hsga_get_population(g, t, tmp);
  if (r == HSGA_OK) memcpy(s, tmp, sizeof(uint64_t) * g->swords);
  free(tmp);
  if (r == HSGA_OK) *len = need;
  return r;
}

int hsga_load(hsga_grid *g, const void *buf, size_t len) {
  if (!g || !buf) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing(g->stream)) return HSGA_ERR_NOT_CAPTURABLE;
  if (g->async) return HSGA_ERR_UNSUPPORTED;
  const size_t need = sizeof(uint64_t) * 2 + sizeof(hsga_config) + g->agents * 4 + g->swords * 8;
  if (len < need) return HSGA_ERR_INVALID_ARG;
  const char *p = (const char *)buf;
  uint64_t magic = 0, G = 0;
  memcpy(&magic, p, 8);
  if (magic != kCheckpointMagic) return HSGA_ERR_INVALID_ARG;
  if (memcmp(p + 8, &g->cfg, sizeof(hsga_config)) != 0) return HSGA_ERR_INVALID_ARG;
  memcpy(&G, p + 8 + sizeof(hsga_config), 8);
  const uint32_t *t = (const uint32_t *)(p + 16 + sizeof(hsga_config));
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (g->swords ? g->swords : 1));
  uint32_t *tt = (uint32_t *)malloc(sizeof(uint32_t) * (g->agents ? g->agents : 1));
  if (!tmp || !tt) {
    free(tmp);
    free(tt);
    return HSGA_ERR_OOM;
  }
  memcpy(tt, t, sizeof(uint32_t) * g->agents);
  memcpy(tmp, t + g->agents, sizeof(uint64_t) * g->swords);
  int r = hsga_set_population(g, tt, tmp, G);
  free(tmp);
  free(tt);
  return r;
}

void hsga_destroy(hsga_grid *g) { free_grid(g); }

uint32_t hsga_site(uint32_t policy, uint32_t S, uint32_t W, uint64_t T) {
  if (policy > HSGA_HYBRID || !power_of_two(S) || S < 2) return S;
  if ((policy == HSGA_TILTED || policy == HSGA_STRETCHED) && (!power_of_two(W) || S / W < 2))
    return S;
  if (policy == HSGA_HYBRID && S < 4) return S;
  return site_of(policy, S, W, T);
}

// Closed-form timestamp lookup (see hsga.h for the site functions it inverts).
int hsga_lookup(uint32_t policy, uint32_t S, uint32_t W, uint64_t N, int64_t *out) {
  if (!out || !power_of_two(S) || S < 2 || S > 256 || policy > HSGA_HYBRID)
    return HSGA_ERR_INVALID_ARG;
  if (policy == HSGA_HYBRID) {  // steady half, then tilted half
    if (S < 4) return HSGA_ERR_INVALID_ARG;
    const int r = hsga_lookup(HSGA_STEADY, S / 2, W, N, out);
    return r != HSGA_OK ? r : hsga_lookup(HSGA_TILTED, S / 2, W, N, out + S / 2);
  }
  for (uint32_t i = 0; i < S; ++i) out[i] = -1;
  if (N == 0 || policy == HSGA_NONE) return HSGA_OK;
  if (policy == HSGA_TRIVIAL) {
    for (uint32_t p = 0; p < S; ++p)
      if (N > p) out[p] = (int64_t)(p + S * ((N - 1 - p) / S));
    return HSGA_OK;
  }
  if (policy == HSGA_STEADY) {
    // After N depositions the current epoch is e = e(N-1).  Epoch-e items are
    // times m 2^e - 1 (1 <= m <= S) at site (m 2^e mod S+1) - 1; those with
    // m <= N / 2^e are in place, the other sites still hold the epoch-(e-1)
    // item that maps there.  Inverting the site map needs 2^-e mod S+1, and
    // 2^(2s) = 1 mod S+1 because 2^s = -1.
    const uint32_t s = bitlen64(S) - 1;
    const uint64_t M = (uint64_t)S + 1;
    const uint32_t e = (N <= S) ? 0u : bitlen64(N - 1) - s;
    if (e == 0) {
      for (uint32_t p = 0; p < S && p < N; ++p) out[p] = p;
      return HSGA_OK;
    }
    auto inv_pow2 = [&](uint32_t k) {  // 2^-k mod M
      const uint32_t r = (2 * s - (k % (2 * s))) % (2 * s);
      uint64_t v = 1;
      for (uint32_t i = 0; i < r; ++i) v = (v * 2) % M;
      return v;
    };
    const uint64_t ie = inv_pow2(e), ie1 = inv_pow2(e - 1);
    const uint64_t cap = N >> e;
    for (uint32_t p = 0; p < S; ++p) {
      const uint64_t m = ((uint64_t)(p + 1) * ie) % M;
      if (m >= 1 && m <= cap) {
        out[p] = (int64_t)((m << e) - 1);
      } else {
        const uint64_t m1 = ((uint64_t)(p + 1) * ie1) % M;
        out[p] = (int64_t)((m1 << (e - 1)) - 1);
      }
    }
    return HSGA_OK;
  }
  // tilted / stretched
  if (!power_of_two(W) || S / W < 2) return HSGA_ERR_INVALID_ARG;
  const uint32_t L = S / W;
  for (uint32_t lvl = 0; lvl < L; ++lvl) {
    const bool capped = lvl == L - 1;
    // depositions so far with ctz(t + 1) == lvl (or >= lvl for the capped
    // level); none at lvl >= 64 for a 64-bit count
    uint64_t c;
    if (capped)
      c = lvl >= 64 ? 0 : (N >> lvl);
    else if (lvl >= 63)
      c = lvl == 63 && N >= (1ull << 63) ? 1 : 0;
    else
      c = (N + (1ull << lvl)) >> (lvl + 1);
    for (uint32_t r = 0; r < W; ++r) {
      uint64_t idx;
      if (policy == HSGA_TILTED) {
        if (c <= r) continue;
        idx = r + (uint64_t)W * ((c - 1 - r) / W);
      } else {
        if (c <= r) continue;
        idx = r;
      }
      out[lvl * W + r] = capped ? (int64_t)(((idx + 1) << (L - 1)) - 1)
                                : (int64_t)(((2 * idx + 1) << lvl) - 1);
    }
  }
  return HSGA_OK;
}

int hsga_wait_probe(const uint64_t *record_dev, uint32_t seq, uint64_t limit_ns,
                    uint64_t *waited_ns, void *cuda_stream) {
  if (!record_dev || limit_ns > 1000000000ull || !is_device_ptr(record_dev) ||
      ((uintptr_t)record_dev % 8) != 0)
    return HSGA_ERR_INVALID_ARG;
  if (stream_capturing((cudaStream_t)cuda_stream)) return HSGA_ERR_NOT_CAPTURABLE;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  AllocHooks al = current_allocator();
  void *scratch = device_alloc(al, 32, st);  // error word + two results
  if (!scratch) return HSGA_ERR_OOM;
  int *err = (int *)scratch;
  uint64_t *out = (uint64_t *)((char *)scratch + 16);
  uint64_t host[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(scratch, 0, 32, st);
  if (e == cudaSuccess) e = launch_wait_probe(record_dev, seq, limit_ns, err, out, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, out, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  device_free(al, scratch, st);
  if (e != cudaSuccess) return HSGA_ERR_CUDA;
  if (waited_ns) *waited_ns = host[1];
  return host[0] ? HSGA_OK : HSGA_ERR_WAIT_TIMEOUT;
}

int hsga_philox_device(uint64_t seed, uint32_t c0, uint32_t count, uint32_t c1, uint32_t c2,
                       uint32_t c3, uint32_t *out_dev, void *cuda_stream) {
  if (count > 0 && (!out_dev || ((uintptr_t)out_dev % 16) != 0)) return HSGA_ERR_INVALID_ARG;
  if ((uint64_t)c0 + count > (1ull << 32)) return HSGA_ERR_INVALID_ARG;
  return cuda_status(
      launch_philox_sweep(seed, c0, count, c1, c2, c3, out_dev, (cudaStream_t)cuda_stream));
}

int hsga_philox_throughput(uint64_t seed, uint32_t threads, uint32_t blocks_per_thread,
                           uint32_t c2, uint32_t c3, uint32_t *out_dev, void *cuda_stream) {
  if (threads > 0 && !out_dev) return HSGA_ERR_INVALID_ARG;
  if (threads > (1u << 30)) return HSGA_ERR_INVALID_ARG;
  return cuda_status(launch_philox_throughput(seed, threads, blocks_per_thread, c2, c3, out_dev,
                                              (cudaStream_t)cuda_stream));
}

int hsga_sites_device(uint32_t policy, uint32_t S, uint32_t W, uint64_t T0, uint64_t count,
                      uint32_t *out_dev, void *cuda_stream) {
  if (count > 0 && !out_dev) return HSGA_ERR_INVALID_ARG;
  if (policy > HSGA_HYBRID || !power_of_two(S) || S < 2 || S > 256) return HSGA_ERR_INVALID_ARG;
  if (policy == HSGA_HYBRID && S < 4) return HSGA_ERR_INVALID_ARG;
  if ((policy == HSGA_TILTED || policy == HSGA_STRETCHED) && (!power_of_two(W) || S / W < 2))
    return HSGA_ERR_INVALID_ARG;
  if (T0 + count >= 0xFFFFFFFFull) return HSGA_ERR_INVALID_ARG;
  return cuda_status(launch_sites(policy, S, W, T0, count, out_dev, (cudaStream_t)cuda_stream));
}

}  // extern "C"

// Configuration checks and kernel parameters, shared with the
// allocation-free entry point (hsga_noalloc.cu).
namespace hsga {
int validate_config(const hsga_config *c) { return validate(c); }
RunParams params_from_config(const hsga_config *c) { return make_params(c); }
}  // namespace hsga

// Device memory through the registered hooks, for the batch engine
// (hsga_batch.cu).
namespace hsga {
AllocHooks current_allocator() {
  return AllocHooks{g_allocator.alloc, g_allocator.free_fn, g_allocator.ctx};
}
void *device_alloc(const AllocHooks &h, size_t bytes, cudaStream_t s) {
  return dev_alloc(Allocator{h.alloc, h.free_fn, h.ctx}, bytes, s);
}
void device_free(const AllocHooks &h, void *ptr, cudaStream_t s) {
  dev_free(Allocator{h.alloc, h.free_fn, h.ctx}, ptr, s);
}
bool device_pointer(const void *ptr) { return is_device_ptr(ptr); }
bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}
}  // namespace hsga
