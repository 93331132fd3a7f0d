// hsga_staged.cu -- streamed generation kernel for 32-agent islands with the
// parents staged in shared memory by bulk asynchronous copies.
//
// One launch advances one synchronous generation of the whole grid (steps
// a1-a6 of the paper's cycle, section "Asynchronous Island-model Genetic
// Algorithm": migration, then evaluation, tournament selection, mutation and
// the surface update).  A persistent grid of warps walks the islands in
// groups of six (the group of the island-group helpers: six islands' five
// migration blocks fill 30 lanes of one warp-wide Philox evaluation).  Each
// warp owns a two-stage ring in shared memory; one lane copies a whole
// group's parents into a stage with cp.async.bulk (768 bytes of traits and
// 1,536 bytes of surfaces, both contiguous in the island-major planes),
// completing on that stage's mbarrier, two groups ahead of the one being
// replicated.  The bytes in flight therefore cost no registers, and the
// tournament reads the parents from shared memory: two 4-byte loads for the
// candidates' fitness and one 8-byte load for the winner's surface per
// child, where a register-resident island needs its own loads plus four
// shuffles.  Immigrants are gathered from the neighbours' parent planes as
// in the register kernel and land with one shared-memory store each (the
// latest of N, E, S, W wins a shared slot).  Children go straight to the
// child planes with streaming stores.
//
// The counter words of the replication blocks other than the island are
// fixed for a launch (child slot = lane, generation, purpose), and so are
// those of the migration blocks (slot word by the lane's role, generation,
// purpose): each lane evaluates the island-independent part of rounds 1-3
// once per launch (philox_head3), leaving 16 of the 20 multiplies per block.
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

// a1 + a2 draws of a group (the register kernel's group_migration with the
// migration blocks' deep heads and branch-free neighbour indices): lane
// 5p+r (r < 4) draws the emigrant block of island isl0+p's neighbour in
// direction r and gathers that emigrant from the parent planes when it is
// aimed at isl0+p; lane 5p+4 draws isl0+p's placement block and builds its
// landing plan (byte 3-d: slot of the direction-d immigrant, 0xFF: none).
template <bool TRACKED>
__device__ __forceinline__ void group_migration_staged(const RunParams &p, const PhiloxHead3 &mh,
                                                       uint32_t lane, uint32_t isl0,
                                                       const uint32_t *__restrict__ tin,
                                                       const uint64_t *__restrict__ sin,
                                                       GroupMigration &gm) {
  const uint32_t pi = lane / 5u, role = lane - pi * 5u;
  const bool valid = lane < 5u * kGroup;
  const uint32_t isl = isl0 + (valid ? pi : 0u);
  uint32_t r = fastdiv(p.cols_div, isl), c = isl - r * p.cols;
  const uint32_t up = (r == 0u ? p.rows : r) - 1u, down = (r + 1u == p.rows) ? 0u : r + 1u;
  const uint32_t left = (c == 0u ? p.cols : c) - 1u, right = (c + 1u == p.cols) ? 0u : c + 1u;
  r = role == 0u ? up : (role == 2u ? down : r);
  c = role == 1u ? right : (role == 3u ? left : c);
  const uint32_t src = r * p.cols + c;  // role 4: the island itself
  const Words4 m = philox_tail3<true>(p, mh, src);
  const bool arrive = valid && role < 4u && (m.y >> 30) == ((role + 2u) & 3u);
  gm.it = 0;
  gm.is = 0;
  if (arrive) {
    const uint32_t a = src * 32u + (m.x >> 27);
    gm.it = __ldg(tin + a);
    if constexpr (TRACKED) gm.is = __ldg(sin + a);
  }
  const uint32_t arrivals = __ballot_sync(kFull, arrive);
  const uint32_t bits = (arrivals >> (5u * pi)) & 0xFu;
  // slots (< 32) in byte d, 0xFF in the bytes of directions with no arrival
  // (the multiply spreads bit d of `miss` to bit 8d without carries), then the
  // byte order reversed
  const uint32_t miss = ~bits & 0xFu;
  const uint32_t fwd = (m.x >> 27) | ((m.y >> 27) << 8) | ((m.z >> 27) << 16) |
                       ((m.w >> 27) << 24) | (((miss * 0x00204081u) & 0x01010101u) * 0xFFu);
  gm.plan = (role == 4u && valid) ? __byte_perm(fwd, 0u, 0x0123u) : 0xFFFFFFFFu;
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

template <bool TRACKED, bool T2, bool TWO, bool DEL, bool MIG>
__global__ void __launch_bounds__(kStagedThreads, kStagedBlocksPerSM)
    step_staged_kernel(RunParams p, Deposit dep, uint32_t G, const uint32_t *__restrict__ tin,
                       const uint64_t *__restrict__ sin, uint32_t *__restrict__ tout,
                       uint64_t *__restrict__ sout, int *__restrict__ err) {
  __shared__ __align__(128) uint32_t s_trait[kWarpsPerBlock][2][kStageAgents];
  __shared__ __align__(128) uint64_t s_surf[kWarpsPerBlock][2][TRACKED ? kStageAgents : 2];
  __shared__ __align__(8) uint64_t s_bar[kWarpsPerBlock][2];
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  const uint32_t warp = blockIdx.x * kWarpsPerBlock + wib;
  const uint32_t nwarps = gridDim.x * kWarpsPerBlock;
  const uint32_t nfull = p.islands / kGroup;
  uint64_t *bar = s_bar[wib];
  constexpr uint32_t kTx = kTraitBytes + (TRACKED ? kSurfBytes : 0u);

  auto issue = [&](uint32_t grp, uint32_t st) {  // one lane
    proxy_fence();
    mbar_expect_tx(&bar[st], kTx);
    bulk_load(s_trait[wib][st], tin + (size_t)grp * kStageAgents, kTraitBytes, &bar[st]);
    if constexpr (TRACKED)
      bulk_load(s_surf[wib][st], sin + (size_t)grp * kStageAgents, kSurfBytes, &bar[st]);
  };

  // the next launch may be scheduled now; it waits below for this one
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  const PhiloxHead3 head = philox_head3(p.k0, p.k1, lane, G, kPurposeReplicate);
  const PhiloxHead3 mhead = philox_head3(p.k0, p.k1, lane % 5u == 4u ? kSlotImmigrant
                                                                     : kSlotEmigrant,
                                         G, kPurposeMigration);
  // the previous launch (which wrote this launch's parents and read the
  // plane this one writes) has completed and its writes are visible
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (lane == 0) {
    if (warp < nfull) issue(warp, 0);
    if (warp + nwarps < nfull) issue(warp + nwarps, 1);
  }
  __syncwarp();

  uint32_t k = 0;
  for (uint32_t grp = warp; grp < nfull; grp += nwarps, ++k) {
    const uint32_t st = k & 1u, parity = (k >> 1) & 1u;
    const uint32_t isl0 = grp * kGroup;
    GroupMigration gm;
    if constexpr (MIG) group_migration_staged<TRACKED>(p, mhead, lane, isl0, tin, sin, gm);
    Words4 w[kGroup];
#pragma unroll
    for (uint32_t i = 0; i < kGroup; ++i) w[i] = philox_tail3<true>(p, head, isl0 + i);
    if (!__all_sync(kFull, mbar_wait(&bar[st], parity))) {
      // give up: record the timeout, wait (bounded) for this warp's copies
      // still in flight, leave
      if (lane == 0) {
        atomicCAS(err, 0, kDevErrWaitTimeout);
        mbar_wait(&bar[st], parity);
        if (grp + nwarps < nfull) mbar_wait(&bar[st ^ 1u], ((k + 1) >> 1) & 1u);
      }
      __syncwarp();
      return;
    }
    uint32_t *tr = s_trait[wib][st];
    uint64_t *sr = s_surf[wib][st];
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
    if (lane == 0 && grp + 2u * nwarps < nfull) issue(grp + 2u * nwarps, st);
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, step_staged_kernel<TRACKED, T2, TWO, DEL, MIG>, kStagedThreads, 0);
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
  cfg.dynamicSmemBytes = 0;
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
