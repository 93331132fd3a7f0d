// hsga_noalloc.cu -- hsga_run_generations_noalloc: the resident generation
// kernel on caller-owned device planes, with its scratch memory (stamped
// migrant records, error word) in a fixed-size array that the
// library image itself carries, so the call never allocates device memory.
//
// Who needs it: code that owns all device memory and forbids allocation
// behind its back -- a host process running under a fixed memory budget or a
// pre-reserved pool, a plugin inside another framework's allocator, or a
// caller that has simply already spent the device.  Such callers cannot use
// hsga_init_grid, which allocates the population planes and the scratch.
//
// The scratch array is a file-scope __device__ variable: every device that
// loads the library holds it (kNoAllocScratchBytes, about 512 KiB) until the
// process exits.  Its host-side name is only a stand-in for the device
// address, so the address is looked up once per device with
// cudaGetSymbolAddress (on the first call on that device, with that device
// current) and passed to the kernel.  That first call should therefore come
// before any stream capture.  The address is kept for the life of the
// process, so calling the entry point after a device reset is not supported.
// All calls share the one array and it keeps the last call's contents: each
// call clears the records and the error word it relies on, and calls whose
// work overlaps on the GPU race on it.  Every call waits for its stream and
// reads the kernels' error word back before it returns.
#include <cuda_runtime.h>

#include <mutex>

#include "hsga.h"
#include "hsga_internal.h"

namespace hsga {
namespace {

constexpr uint32_t kNoAllocMaxIslands = 8192;
constexpr size_t kRecBytes = sizeof(uint64_t) * 8 * kNoAllocMaxIslands;  // 512 KiB
constexpr size_t kNoAllocScratchBytes = kRecBytes + 256;                  // + error word
constexpr uint64_t kNoAllocMaxGeneration = 0xFFFFFFFFull - 64;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return HSGA_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return HSGA_ERR_CUDA;
    }
    g_scratch_addr[dev] = (unsigned char *)ptr;
  }
  *out = g_scratch_addr[dev];
  return HSGA_OK;
}

// Device memory (or managed memory) that belongs to device `dev`, the
// current device: the kernel runs there, with no peer mapping set up.
bool on_device(const void *ptr, int dev) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) return false;
  return attr.device == dev;
}

}  // namespace
}  // namespace hsga

using namespace hsga;

extern "C" int hsga_run_generations_noalloc(const hsga_config *cfg, uint64_t generation,
                                            uint64_t n_generations, uint32_t *trait,
                                            uint64_t *surf, void *cuda_stream) {
  const int v = validate_config(cfg);
  if (v != HSGA_OK) return v;
  if (cfg->migration_mode != HSGA_MIGRATION_SYNC || cfg->fitness != HSGA_FITNESS_TRAIT ||
      cfg->surface_words > 1)
    return HSGA_ERR_UNSUPPORTED;
  const RunParams p = params_from_config(cfg);
  const bool tracked = cfg->surface_policy != HSGA_NONE;
  if (p.islands > kNoAllocMaxIslands) return HSGA_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HSGA_ERR_CUDA;
  }
  if (!trait || !on_device(trait, dev)) return HSGA_ERR_INVALID_ARG;
  if (tracked && (!surf || !on_device(surf, dev))) return HSGA_ERR_INVALID_ARG;
  // written so that no sum can wrap around
  if (generation > kNoAllocMaxGeneration || n_generations > kNoAllocMaxGeneration - generation)
    return HSGA_ERR_INVALID_ARG;
  if (n_generations == 0) return HSGA_OK;
  ResidentPlan plan;
  if (!resident_plan(p, &plan)) return HSGA_ERR_UNSUPPORTED;
  unsigned char *scratch = nullptr;
  int r = scratch_address(&scratch);
  if (r != HSGA_OK) return r;
  uint64_t *rec = (uint64_t *)scratch;
  int *err = (int *)(scratch + kRecBytes);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // the previous call's records and error word must not leak into this one
  cudaError_t e = cudaMemsetAsync(rec, 0, sizeof(uint64_t) * 8 * p.islands, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), stream);
  const uint64_t slice = 1u << 16;
  for (uint64_t done = 0; done < n_generations && e == cudaSuccess;) {
    const uint32_t m =
        (uint32_t)((n_generations - done) < slice ? (n_generations - done) : slice);
    e = launch_step_resident(p, plan, (uint32_t)(generation + done), m, false, trait,
                             tracked ? surf : nullptr, rec, err, stream);
    done += m;
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HSGA_ERR_CUDA;
  }
  if (h == kDevErrWaitTimeout) return HSGA_ERR_WAIT_TIMEOUT;
  return h ? HSGA_ERR_DEVICE : HSGA_OK;
}
