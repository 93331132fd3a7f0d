// hsga_staged.cu -- streamed generation kernel for 32-agent islands with the
// parents staged in shared memory by bulk asynchronous copies.
//
// One launch advances one synchronous generation of the whole grid (steps
// a1-a6 of the paper's cycle, section "Asynchronous Island-model Genetic
// Algorithm": migration, then evaluation, tournament selection, mutation and
// the surface update).  A persistent grid of warps walks the islands in
// groups of six (the group of the island-group helpers: six islands' five
// migration blocks fill 30 lanes of one warp-wide Philox evaluation).  Each
// warp owns a ring of kStagedStages stages in shared memory; one lane copies
// a whole group's parents into a stage with cp.async.bulk (768 bytes of
// traits and 1,536 bytes of surfaces, both contiguous in the island-major
// planes), completing on that stage's mbarrier, up to kStagedStages groups
// ahead of the one being replicated.  The bytes in flight therefore cost no registers, and the
// tournament reads the parents from shared memory: two 4-byte loads for the
// candidates' fitness and one 8-byte load for the winner's surface per
// child, where a register-resident island needs its own loads plus four
// shuffles.  Immigrants are gathered from the neighbours' parent planes as
// in the register kernel and land with one shared-memory store each (the
// latest of N, E, S, W wins a shared slot).  Children go straight to the
// child planes with streaming stores.
//
// The replication blocks' counter words other than the island (child slot =
// lane, generation, purpose) are fixed for a launch, so each lane evaluates
// round 1's island-independent part once per launch (philox_head).
//
// Consecutive generations overlap at the launch boundary (programmatic
// dependent launch): a launch lets the next one be scheduled as soon as it
// starts, and the next one initialises its barriers and generator heads,
// then waits (griddepcontrol.wait) for this launch to complete and its
// writes to be visible before it touches either population plane.
//
// Waits on a stage are bounded (1 s of %globaltimer): on expiry the warp
// records HSGA_ERR_WAIT_TIMEOUT in the grid's error word, waits (bounded
// again) for its own copies still in flight, and leaves.
#include <cuda_runtime.h>

#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {
namespace {

constexpr uint32_t kWarpsPerBlock = kStagedThreads / 32;
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
template <bool TRACKED, bool T2, bool TWO, bool DEL>
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
      const Words4 e = philox_rk(p, lane, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
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
constexpr size_t kRingBytes = (size_t)kWarpsPerBlock * kStages * kStageBytes;

template <bool TRACKED, bool T2, bool TWO, bool DEL, bool MIG>
__global__ void __launch_bounds__(kStagedThreads, kStagedBlocksPerSM)
    step_staged_kernel(RunParams p, Deposit dep, uint32_t G, const uint32_t *__restrict__ tin,
                       const uint64_t *__restrict__ sin, uint32_t *__restrict__ tout,
                       uint64_t *__restrict__ sout, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char s_ring[];  // the ring (kRingBytes), padded
  __shared__ __align__(8) uint64_t s_bar[kWarpsPerBlock][kStages];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint32_t warp = blockIdx.x * kWarpsPerBlock + wib;
  const uint32_t nwarps = gridDim.x * kWarpsPerBlock;
  const uint32_t nfull = p.islands / kGroup;
  unsigned char *ring = s_ring + (size_t)wib * kStages * kStageBytes;
  uint64_t *bar = s_bar[wib];
  constexpr uint32_t kTx = kTraitBytes + (TRACKED ? kSurfBytes : 0u);

  // stage st holds a group's traits (768 B) then its surfaces (1,536 B)
  auto issue = [&](uint32_t grp, uint32_t st) {  // one lane
    unsigned char *dst = ring + st * kStageBytes;
    proxy_fence();
    mbar_expect_tx(&bar[st], kTx);
    bulk_load(dst, tin + (size_t)grp * kStageAgents, kTraitBytes, &bar[st]);
    if constexpr (TRACKED)
      bulk_load(dst + kTraitBytes, sin + (size_t)grp * kStageAgents, kSurfBytes, &bar[st]);
  };

  // the next launch may be scheduled now; it waits below for this one
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (lane == 0) {
#pragma unroll
    for (uint32_t st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
    mbar_init_fence();
  }
  const PhiloxHead head = philox_head(p.k0, p.k1, lane, G, kPurposeReplicate);
  // the previous launch (which wrote this launch's parents and read the
  // plane this one writes) has completed and its writes are visible
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (lane == 0) {
#pragma unroll
    for (uint32_t st = 0; st < kStages; ++st)
      if (warp + st * nwarps < nfull) issue(warp + st * nwarps, st);
  }
  __syncwarp();

  uint32_t st = 0, phase = 0;  // ring position of the k-th group and its phase parity
  for (uint32_t grp = warp; grp < nfull; grp += nwarps) {
    const uint32_t isl0 = grp * kGroup;
    GroupMigration gm;
    if constexpr (MIG) group_migration<TRACKED, true, 32>(p, isl0, G, tin, sin, gm);
    Words4 w[kGroup];
#pragma unroll
    for (uint32_t i = 0; i < kGroup; ++i) w[i] = philox_tail<true>(p, head, isl0 + i);
    if (!__all_sync(kFull, mbar_wait(&bar[st], phase))) {
      // give up: record the timeout, wait (bounded) for this warp's copies
      // still in flight (the groups issued into the ring from this one on),
      // leave
      if (lane == 0) {
        atomicCAS(err, 0, kDevErrWaitTimeout);
        uint32_t s2 = st, ph2 = phase;
        for (uint32_t j = 0; j < kStages && grp + j * nwarps < nfull; ++j) {
          mbar_wait(&bar[s2], ph2);
          if (++s2 == kStages) {
            s2 = 0;
            ph2 ^= 1u;
          }
        }
      }
      __syncwarp();
      return;
    }
    uint32_t *tr = (uint32_t *)(ring + st * kStageBytes);
    uint64_t *sr = (uint64_t *)(ring + st * kStageBytes + kTraitBytes);
    if constexpr (MIG) {
      land_staged<TRACKED>(gm, lane, tr, sr);
      __syncwarp();
    }
    uint32_t *to = tout + (size_t)isl0 * 32u + lane;
    uint64_t *so = TRACKED ? sout + (size_t)isl0 * 32u + lane : sout;
#pragma unroll
    for (uint32_t i = 0; i < kGroup; ++i) {
      uint32_t ct;
      uint64_t cs;
      replicate_staged<TRACKED, T2, TWO, DEL>(p, dep, lane, isl0 + i, G, w[i], tr + 32u * i,
                                              sr + (TRACKED ? 32u * i : 0u), ct, cs);
      __stcs(to + 32u * i, ct);
      if constexpr (TRACKED) __stcs(so + 32u * i, cs);
    }
    __syncwarp();  // every lane is done with this stage before it is refilled
    if (lane == 0 && grp + kStages * nwarps < nfull) issue(grp + kStages * nwarps, st);
    if (++st == kStages) {
      st = 0;
      phase ^= 1u;
    }
  }
  // the last, partial group (fewer than six islands) on the register path
  if (p.islands % kGroup != 0u && warp == nfull % nwarps)
    partial_group<1, TRACKED, T2>(p, dep, G, MIG, nfull * kGroup, tin, sin, tout, sout);
}

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

template <bool TRACKED, bool T2, bool TWO, bool DEL, bool MIG>
int staged_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = staged_smem_bytes();
    cudaFuncSetAttribute(step_staged_kernel<TRACKED, T2, TWO, DEL, MIG>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, step_staged_kernel<TRACKED, T2, TWO, DEL, MIG>, kStagedThreads, smem);
    if (per_sm > kStagedBlocksPerSM) per_sm = kStagedBlocksPerSM;
    blocks = sms * (per_sm > 0 ? per_sm : 1);
  }
  return blocks;
}

template <bool TRACKED, bool T2, bool TWO, bool DEL, bool MIG>
void launch_staged_t(const RunParams &p, const Deposit &dep, uint32_t G, const uint32_t *tin,
                     const uint64_t *sin, uint32_t *tout, uint64_t *sout, int *err,
                     cudaStream_t stream) {
  const uint32_t groups = (p.islands + kGroup - 1) / kGroup;
  const uint32_t need = (groups + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int b = staged_blocks<TRACKED, T2, TWO, DEL, MIG>();
  if ((uint32_t)b > need) b = (int)need;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)b);
  cfg.blockDim = dim3(kStagedThreads);
  cfg.dynamicSmemBytes = staged_smem_bytes();
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, step_staged_kernel<TRACKED, T2, TWO, DEL, MIG>, p, dep, G, tin, sin,
                     tout, sout, err);
}

template <bool TRACKED, bool T2>
void launch_staged_m(const RunParams &p, const Deposit &dep, uint32_t G, bool mig,
                     const uint32_t *tin, const uint64_t *sin, uint32_t *tout, uint64_t *sout,
                     int *err, cudaStream_t stream) {
#define HSGA_STAGED(TWO_, DEL_)                                                            \
  if (mig)                                                                                 \
    launch_staged_t<TRACKED, T2, TWO_, DEL_, true>(p, dep, G, tin, sin, tout, sout, err,   \
                                                   stream);                                \
  else                                                                                     \
    launch_staged_t<TRACKED, T2, TWO_, DEL_, false>(p, dep, G, tin, sin, tout, sout, err,  \
                                                    stream);
  if (TRACKED && dep.two) {
    HSGA_STAGED(true, true)
  } else if (p.has_del) {
    HSGA_STAGED(false, true)
  } else {
    HSGA_STAGED(false, false)
  }
#undef HSGA_STAGED
}

}  // namespace

cudaError_t launch_step_staged(const RunParams &p, uint32_t G, bool do_mig, const uint32_t *tin,
                               const uint64_t *sin, uint32_t *tout, uint64_t *sout, int *err,
                               cudaStream_t stream) {
  if (p.n != 32) return cudaErrorInvalidValue;
  const Deposit dep = deposit_for(p, G);
  const bool tracked = p.policy != HSGA_NONE;
  const bool t2 = p.tournament == 2;
  if (tracked) {
    if (t2) launch_staged_m<true, true>(p, dep, G, do_mig, tin, sin, tout, sout, err, stream);
    else launch_staged_m<true, false>(p, dep, G, do_mig, tin, sin, tout, sout, err, stream);
  } else {
    if (t2) launch_staged_m<false, true>(p, dep, G, do_mig, tin, sin, tout, sout, err, stream);
    else launch_staged_m<false, false>(p, dep, G, do_mig, tin, sin, tout, sout, err, stream);
  }
  return cudaGetLastError();
}

}  // namespace hsga
