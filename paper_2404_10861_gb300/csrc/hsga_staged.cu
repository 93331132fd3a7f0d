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

#include "hsga_stage.cuh"

namespace hsga {
namespace {

template <bool TRACKED, bool T2, bool TWO, bool DEL, bool MIG>
__global__ void __launch_bounds__(kStagedThreads, kStagedBlocksPerSM)
    step_staged_kernel(RunParams p, Deposit dep, uint32_t G, const uint32_t *__restrict__ tin,
                       const uint64_t *__restrict__ sin, uint32_t *__restrict__ tout,
                       uint64_t *__restrict__ sout, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char s_ring[];  // the ring (kRingBytes), padded
  __shared__ __align__(8) uint64_t s_bar[kStagedWarps][kStages];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint32_t warp = blockIdx.x * kStagedWarps + wib;
  const uint32_t nwarps = gridDim.x * kStagedWarps;
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
  const uint32_t need = (groups + kStagedWarps - 1) / kStagedWarps;
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
