// hsga_stage.cuh -- staging of island groups in shared memory by bulk
// asynchronous copies, shared by the single-run staged generation kernel
// (hsga_staged.cu) and the batch engine's staged kernel (hsga_batch.cu).
//
// A warp owns a ring of kStagedStages stages; a stage holds one group of six
// 32-agent islands: 768 bytes of traits, then 1,536 bytes of surfaces, each
// contiguous in the island-major planes, copied by one lane with
// cp.async.bulk and completing on the stage's mbarrier.  The helpers below
// are the barrier and copy primitives, the landing of a group's immigrants
// into a stage, and one child's replication from a stage.
#pragma once

#include <cuda_runtime.h>

#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {


constexpr uint32_t kStagedWarps = kStagedThreads / 32;
constexpr uint32_t kStageAgents = kGroup * 32;
constexpr uint32_t kTraitBytes = kStageAgents * 4;  // 768
constexpr uint32_t kSurfBytes = kStageAgents * 8;   // 1536
constexpr uint32_t kMaxPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Makes the barrier initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (and, after a warp
// barrier, its warp's) before later bulk copies into the same memory.
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) that completes `bytes` of the barrier's transaction count.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (uint32_t i = 1; i < kMaxPolls; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63u) == 0 && now_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// a2 for a staged group: lane 5p+r (r < 4) holds the immigrant of island p
// from direction r when it arrives; the landing plan of island p (lane 5p+4,
// byte 3-d: slot of direction d, 0xFF: none) says where.  The lane stores it
// unless a later direction lands on the same slot.
template <bool TRACKED>
__device__ __forceinline__ void land_staged(const GroupMigration &gm, uint32_t lane,
                                            uint32_t *tr, uint64_t *sr) {
  const uint32_t pi = lane / 5u, role = lane - 5u * pi;
  const uint32_t plan = __shfl_sync(kFull, gm.plan, min(5u * pi + 4u, 31u));
  if (lane < 5u * kGroup && role < 4u) {
    const uint32_t sh = 8u * (3u - role);
    const uint32_t slot = (plan >> sh) & 0xFFu;
    // bytes of later directions (below byte 3-role) kept, the rest all ones
    const uint32_t later = plan | ~((1u << sh) - 1u);
    const uint32_t x = later ^ (slot * 0x01010101u);
    const bool overwritten = ((x - 0x01010101u) & ~x & 0x80808080u) != 0u;
    if (slot != 0xFFu && !overwritten) {
      tr[pi * 32u + slot] = gm.it;
      if constexpr (TRACKED) sr[pi * 32u + slot] = gm.is;
    }
  }
}

// a3-a6 of child `lane` of one staged island (parents tr[0..31], sr[0..31]).
// RK: the run's round keys are in the parameter block (single-run kernels);
// otherwise they are derived from the key.
template <bool TRACKED, bool T2, bool TWO, bool DEL, bool RK = true>
__device__ __forceinline__ void replicate_staged(const RunParams &p, const Deposit &dep,
                                                 uint32_t lane, uint32_t isl, uint32_t G,
                                                 const Words4 &w, const uint32_t *tr,
                                                 const uint64_t *sr, uint32_t &ct,
                                                 uint64_t &cs) {
  uint32_t best = w.x >> 27;
  uint32_t fbest = tr[best];
  if (T2 || p.tournament >= 2) {
    const uint32_t c = w.y >> 27;
    const uint32_t fc = tr[c];
    const bool take = fc > fbest;
    best = take ? c : best;
    fbest = take ? fc : fbest;
  }
  if constexpr (!T2) {
    for (uint32_t c0 = 2; c0 < p.tournament; c0 += 4) {
      const Words4 e = philox_p<RK>(p, lane, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
      const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (c0 + r < p.tournament) {
          const uint32_t c = ew[r] >> 27;
          const uint32_t fc = tr[c];
          if (fc > fbest) {
            best = c;
            fbest = fc;
          }
        }
      }
    }
  }
  ct = mutate<DEL>(p, fbest, w.z);
  if constexpr (TRACKED) cs = deposit_into<TWO>(dep, sr[best], w.w);
  else cs = 0;
}

constexpr uint32_t kStageBytes = kTraitBytes + kSurfBytes;  // 2304 per group
constexpr uint32_t kStages = kStagedStages;
constexpr size_t kRingBytes = (size_t)kStagedWarps * kStages * kStageBytes;

// Shared memory requested per block: the ring, padded so that one block
// more than kStagedBlocksPerSM does not fit on an SM.  Otherwise the next
// generation's launch, scheduled early by programmatic dependent launch,
// parks a block in the free slot that competes with the running blocks for
// issue slots until it may start (107 us per generation at 16.8M agents
// with a free slot, 75.3 us without).
inline size_t staged_smem_bytes() {
  static size_t bytes = 0;
  if (bytes == 0) {
    int dev = 0, per_sm = 0, per_block = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    size_t pad = (size_t)per_sm / (kStagedBlocksPerSM + 1) + 128;
    pad = pad > (size_t)reserved ? pad - (size_t)reserved : pad;
    size_t b = kRingBytes > pad ? kRingBytes : pad;
    if (per_block > 0 && b > (size_t)per_block - 1024) b = kRingBytes;  // no room to pad
    bytes = (b + 127) & ~(size_t)127;
  }
  return bytes;
}

}  // namespace hsga
