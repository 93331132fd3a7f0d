// hsga_async.cu -- free-running (asynchronous) generation kernel.
//
// The paper's islands run without a global clock, each taking whatever its
// neighbours last sent (section "Asynchronous Island-model Genetic
// Algorithm").  Here one warp owns one island (lane = agent, n <= 32) and
// runs its generations without ever waiting: at every migrating generation
// it publishes its emigrant (slot and direction from the counter-based RNG,
// as in synchronous mode) into its single outgoing record, then looks at
// each neighbour's latest record and takes it if that record is new and was
// aimed at this island.  Records are guarded by a sequence stamp (a
// seqlock): the writer marks the stamp odd, writes the 16-byte genome, then
// publishes an even stamp ((G+1) << 3 | dir << 1) with a release store; a
// reader accepts the genome only if the stamp it acquired before reading is
// even, newer than the last one it saw from that neighbour, and unchanged
// after the read.  A record overwritten before a neighbour saw it is simply
// lost (the paper's dropped messages).  Genomes carry their own deposition
// counter T: an immigrant keeps its T, a child deposits at site(T_parent)
// and carries T_parent + 1.
//
// Which records each island took depends on timing, so a run is not
// reproducible; optionally every take is logged (the source generation per
// island, generation and direction) and the oracle replays the log exactly.
#include <cuda_runtime.h>

#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {
namespace {

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

template <bool TRACKED, bool T2, bool TWO>
__global__ void __launch_bounds__(kResidentThreads)
    step_async_kernel(RunParams p, uint32_t G0, uint32_t ngen, uint32_t *__restrict__ tplane,
                      uint64_t *__restrict__ splane, uint32_t *__restrict__ Tplane,
                      uint4 *__restrict__ rec, uint32_t *__restrict__ stamp,
                      uint32_t *__restrict__ seen_io, uint32_t *__restrict__ log,
                      uint32_t log_G0, uint32_t log_gens) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t isl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (isl >= p.islands) return;  // whole warps only; no block barriers are used
  const uint32_t n = p.n;
  const uint32_t base = isl * n;
  uint32_t pt[1] = {0}, pT[1] = {0};
  uint64_t ps[1] = {0};
  if (lane < n) {
    pt[0] = tplane[base + lane];
    if constexpr (TRACKED) ps[0] = splane[base + lane];
    pT[0] = Tplane[base + lane];
  }
  uint32_t seen = lane < 4 ? seen_io[isl * 4 + lane] : 0u;
  for (uint32_t g = 0; g < ngen; ++g) {
    const uint32_t G = G0 + g;
    Words4 w[1];
    replication_words<1>(p, isl, G, w);
    const bool logging = log && G >= log_G0 && G - log_G0 < log_gens;
    if (migrates(p, G)) {
      // lane 0: the emigrant block, lane 1: the placement block
      const Words4 m =
          philox_rk(p, lane == 1 ? kSlotImmigrant : kSlotEmigrant, isl, G, kPurposeMigration);
      const uint32_t eslot = uindex(__shfl_sync(kFull, m.x, 0), n);
      const uint32_t dir = __shfl_sync(kFull, m.y, 0) >> 30;
      const uint32_t te = __shfl_sync(kFull, pt[0], eslot);
      const uint64_t se = shfl64(ps[0], eslot);
      const uint32_t Te = __shfl_sync(kFull, pT[0], eslot);
      // a1: publish under the stamp
      if (lane == 0) {
        st_relaxed_u32(stamp + isl, ((G + 1u) << 3) | 1u);
        fence_acq_rel();
        rec[isl] = make_uint4(te, (uint32_t)se, (uint32_t)(se >> 32), Te);
        st_release_u32(stamp + isl, ((G + 1u) << 3) | (dir << 1));
      }
      // a2: each neighbour's latest record, if new and aimed here
      bool take = false;
      uint32_t it = 0, iT = 0, from = 0;
      uint64_t is = 0;
      if (lane < 4) {
        const uint32_t nb = neighbour(p, isl, lane);
        const uint32_t s1 = ld_acquire_u32(stamp + nb);
        if (!(s1 & 1u) && (s1 >> 3) > seen) {
          seen = s1 >> 3;
          if (((s1 >> 1) & 3u) == ((lane + 2u) & 3u)) {
            const uint4 r = __ldcg(rec + nb);
            fence_acq_rel();
            if (ld_relaxed_u32(stamp + nb) == s1) {
              take = true;
              it = r.x;
              is = ((uint64_t)r.z << 32) | r.y;
              iT = r.w;
              from = s1 >> 3;
            }
          }
        }
        if (logging) log[((size_t)isl * log_gens + (G - log_G0)) * 4 + lane] = from;
      }
      const uint32_t arrivals = __ballot_sync(kFull, take);
      const uint32_t place[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
      for (uint32_t dd = 0; dd < 4; ++dd) {
        if (arrivals & (1u << dd)) {
          const uint32_t slot = uindex(__shfl_sync(kFull, place[dd], 1), n);
          const uint32_t vt = __shfl_sync(kFull, it, dd);
          const uint64_t vs = shfl64(is, dd);
          const uint32_t vT = __shfl_sync(kFull, iT, dd);
          if (lane == slot) {
            pt[0] = vt;
            ps[0] = vs;
            pT[0] = vT;
          }
        }
      }
    } else if (logging && lane < 4) {
      log[((size_t)isl * log_gens + (G - log_G0)) * 4 + lane] = 0;
    }
    // a3-a5: tournament and mutation on the traits
    uint32_t best = uindex(w[0].x, n);
    uint32_t fbest = fetch32<1>(pt, best);
    if (T2 || p.tournament >= 2) {
      const uint32_t c = uindex(w[0].y, n);
      const uint32_t fc = fetch32<1>(pt, c);
      const bool pick = fc > fbest;
      best = pick ? c : best;
      fbest = pick ? fc : fbest;
    }
    if constexpr (!T2) {
      for (uint32_t c0 = 2; c0 < p.tournament; c0 += 4) {
        const Words4 e = philox_rk(p, lane, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
        const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (c0 + r < p.tournament) {
            const uint32_t c = uindex(ew[r], n);
            const uint32_t fc = fetch32<1>(pt, c);
            if (fc > fbest) {
              best = c;
              fbest = fc;
            }
          }
        }
      }
    }
    const uint32_t child_t = mutate(p, fbest, w[0].z);
    // a6: deposit at the site of the parent's own counter
    const uint32_t Tp = fetch32<1>(pT, best);
    uint64_t child_s = 0;
    if constexpr (TRACKED) {
      const Deposit dep = deposit_unpack(deposit_pack(p, Tp), (uint32_t)p.vmask);
      child_s = deposit_into<TWO>(dep, fetch64<1>(ps, best), w[0].w);
    }
    pt[0] = child_t;
    ps[0] = child_s;
    pT[0] = Tp + 1u;
  }
  if (lane < n) {
    tplane[base + lane] = pt[0];
    if constexpr (TRACKED) splane[base + lane] = ps[0];
    Tplane[base + lane] = pT[0];
  }
  if (lane < 4) seen_io[isl * 4 + lane] = seen;
}

using AsyncFn = void (*)(RunParams, uint32_t, uint32_t, uint32_t *, uint64_t *, uint32_t *,
                         uint4 *, uint32_t *, uint32_t *, uint32_t *, uint32_t, uint32_t);

AsyncFn pick_async(bool tracked, bool t2, bool two) {
  if (!tracked) return t2 ? step_async_kernel<false, true, false> : step_async_kernel<false, false, false>;
  if (two) return t2 ? step_async_kernel<true, true, true> : step_async_kernel<true, false, true>;
  return t2 ? step_async_kernel<true, true, false> : step_async_kernel<true, false, false>;
}

}  // namespace

cudaError_t launch_step_async(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t *t,
                              uint64_t *s, uint32_t *T, uint4 *rec, uint32_t *stamp,
                              uint32_t *seen, uint32_t *log, uint32_t log_G0, uint32_t log_gens,
                              cudaStream_t stream) {
  AsyncFn fn = pick_async(p.policy != HSGA_NONE, p.tournament == 2, p.policy == HSGA_HYBRID);
  const uint32_t wpb = kResidentThreads / 32;
  const uint32_t blocks = (p.islands + wpb - 1) / wpb;
  fn<<<blocks, kResidentThreads, 0, stream>>>(p, G0, ngen, t, s, T, rec, stamp, seen, log,
                                               log_G0, log_gens);
  return cudaGetLastError();
}

}  // namespace hsga
