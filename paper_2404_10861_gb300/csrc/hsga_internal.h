// hsga_internal.h -- kernel launch interface between the C-ABI runtime
// (hsga_capi.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "hsga_device.cuh"

namespace hsga {

constexpr int kStreamThreads = 256;     // streamed kernel block: 8 warps
constexpr int kStreamBlocksPerSM = 3;   // 24 resident warps per SM (<= 80 registers)
constexpr int kStagedThreads = 256;     // staged streamed kernel (n = 32) block: 8 warps
// 16 resident warps per SM (<= 128 registers) with two groups in flight per
// warp: measured fastest at 16.8M agents (75.3 us per generation; 24 warps:
// 78.7 us; 3-5 stages: 76.3-81.2 us).
constexpr int kStagedBlocksPerSM = 2;
constexpr uint32_t kStagedStages = 2;   // groups in flight per warp
constexpr int kResidentThreads = 128;   // resident kernel block: 4 warps
constexpr uint32_t kSampleSmemMax = 12288;  // largest k sampled by the shared-memory kernel
constexpr uint64_t kWaitNs = 1000000000ull; // bounded device wait: 1 s

// How the resident kernel exchanges emigrant records: polled stamped records
// in global memory; the whole grid in one block (shared memory, block
// barriers); or tiles of islands per block (shared memory inside a tile,
// polled records across tiles).
enum ResidentMode { kPolled = 0, kBlockSync = 1, kTiled = 2 };
constexpr bool kResidentTiles = true;   // multi-block grids use kTiled when a tile shape fits

struct ResidentPlan {
  int ap = 0;      // agents per lane (1: n <= 32, 2: n <= 64)
  int ipw = 0;     // islands per warp
  int blocks = 0;  // cooperative grid
  int warps_per_block = kResidentThreads / 32;
  int mode = kPolled;
  uint32_t tile = 0;  // kTiled: log2(tile rows) | log2(tile columns) << 8
};

// err: the grid's device error word (bounded waits report timeouts there).
cudaError_t launch_step_streamed(const RunParams &p, uint32_t G, bool do_mig,
                                 const uint32_t *tin, const uint64_t *sin, uint32_t *tout,
                                 uint64_t *sout, int *err, cudaStream_t stream);

// The same generation for 32-agent islands with the parents staged in shared
// memory by bulk asynchronous copies (hsga_staged.cu); waits report
// timeouts in err.
cudaError_t launch_step_staged(const RunParams &p, uint32_t G, bool do_mig, const uint32_t *tin,
                               const uint64_t *sin, uint32_t *tout, uint64_t *sout, int *err,
                               cudaStream_t stream);

// Chooses the resident tile (smallest islands-per-warp whose cooperative
// grid is co-resident).  Returns false when the grid does not fit on chip.
bool resident_plan(const RunParams &p, ResidentPlan *out, bool grid_only = false);

cudaError_t launch_step_resident(const RunParams &p, const ResidentPlan &plan, uint32_t G0,
                                 uint32_t ngen, bool premigrated, uint32_t *t, uint64_t *s,
                                 uint64_t *rec, int *err, cudaStream_t stream);

cudaError_t launch_migrate(const RunParams &p, uint32_t G, uint32_t *t, uint64_t *s,
                           uint4 *rec, cudaStream_t stream);

size_t sample_scratch_bytes(const RunParams &p, uint32_t k);

// T: per-genome deposition counters (free-running grids) written as word 3,
// or NULL to write G.
cudaError_t launch_sample(const RunParams &p, uint32_t G, uint32_t k, const uint32_t *t,
                          const uint64_t *s, uint32_t *out_words, uint32_t *out_is,
                          uint32_t *scratch, cudaStream_t stream, const uint32_t *T = nullptr);

// Wide surfaces (hsga_wide.cu): the field(s) a synchronous generation
// writes (word < 0: none).
struct WideDeposit {
  int word1;
  uint32_t shift1;
  int word2;
  uint32_t shift2;
};
WideDeposit wide_deposit_for(const RunParams &p, uint64_t G);
cudaError_t launch_migrate_wide(const RunParams &p, uint32_t G, uint32_t *t, uint64_t *s,
                                uint64_t *rec, cudaStream_t stream);
cudaError_t launch_step_wide(const RunParams &p, uint32_t G, const uint32_t *tin,
                             const uint64_t *sin, uint32_t *tout, uint64_t *sout,
                             cudaStream_t stream);
cudaError_t launch_gather_wide(const RunParams &p, uint32_t G, uint32_t k, const uint32_t *t,
                               const uint64_t *s, const uint32_t *where, uint32_t *out,
                               cudaStream_t stream);
cudaError_t launch_step_float(const RunParams &p, uint32_t G, const uint32_t *tin,
                              const uint64_t *sin, uint32_t *tout, uint64_t *sout,
                              cudaStream_t stream);
// Free-running generations (hsga_async.cu).  slice: generations each warp
// advances an island octet by per visit (1: the whole grid one generation at
// a time).
cudaError_t launch_step_buffered(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t slice,
                                 uint32_t *t, uint64_t *s, uint32_t *T, uint64_t *mail,
                                 uint32_t *ack, uint4 *inbuf, uint4 *chst, uint32_t *log,
                                 uint32_t log_G0, uint32_t log_gens, cudaStream_t stream);
cudaError_t launch_step_async(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t slice,
                              uint32_t *t, uint64_t *s, uint32_t *T, uint64_t *rec,
                              uint32_t *seen, uint32_t *log, uint32_t log_G0, uint32_t log_gens,
                              cudaStream_t stream);

// Device memory through the registered allocator hooks (hsga_capi.cu).
struct AllocHooks {
  hsga_alloc_fn alloc;
  hsga_free_fn free_fn;
  void *ctx;
};
AllocHooks current_allocator();
void *device_alloc(const AllocHooks &h, size_t bytes, cudaStream_t s);
void device_free(const AllocHooks &h, void *ptr, cudaStream_t s);
bool device_pointer(const void *ptr);

// Whether `s` is being captured into a CUDA graph (calls that wait for their
// stream return HSGA_ERR_NOT_CAPTURABLE then; defined in hsga_capi.cu).
bool stream_capturing(cudaStream_t s);

// Configuration checks and kernel parameters (defined in hsga_capi.cu).
int validate_config(const hsga_config *c);
RunParams params_from_config(const hsga_config *c);

cudaError_t launch_wait_probe(const uint64_t *record, uint32_t seq, uint64_t limit_ns, int *err,
                              uint64_t *out, cudaStream_t stream);
cudaError_t launch_philox_sweep(uint64_t seed, uint32_t c0, uint32_t count, uint32_t c1,
                                uint32_t c2, uint32_t c3, uint32_t *out, cudaStream_t stream);
cudaError_t launch_philox_throughput(uint64_t seed, uint32_t threads, uint32_t m, uint32_t c2,
                                     uint32_t c3, uint32_t *out, cudaStream_t stream);
cudaError_t launch_sites(uint32_t policy, uint32_t S, uint32_t W, uint64_t T0, uint64_t count,
                         uint32_t *out, cudaStream_t stream);

}  // namespace hsga
