// hsga_island.cuh -- warp-level island operations shared by the streamed and
// the resident generation kernels: one warp holds one island, lane l holds
// agents l and l+32 (AP = agents per lane), and selection reads the parents
// through warp shuffles (no shared memory, no block barriers).
#pragma once

#include "hsga_device.cuh"

namespace hsga {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int AP>
__device__ __forceinline__ uint32_t fetch32(const uint32_t (&v)[AP], uint32_t idx) {
  if constexpr (AP == 1) {
    return __shfl_sync(kFull, v[0], idx);
  } else {
    const uint32_t a = __shfl_sync(kFull, v[0], idx & 31u);
    const uint32_t b = __shfl_sync(kFull, v[1], idx & 31u);
    return (idx >> 5) ? b : a;
  }
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, uint32_t lane) {
  const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, lane);
  const uint32_t hi = __shfl_sync(kFull, (uint32_t)(v >> 32), lane);
  return ((uint64_t)hi << 32) | lo;
}

template <int AP>
__device__ __forceinline__ uint64_t fetch64(const uint64_t (&v)[AP], uint32_t idx) {
  if constexpr (AP == 1) {
    return shfl64(v[0], idx);
  } else {
    const uint64_t a = shfl64(v[0], idx & 31u);
    const uint64_t b = shfl64(v[1], idx & 31u);
    return (idx >> 5) ? b : a;
  }
}

// Replication words of child j (lane-owned): Philox(seed; j, island, G, 1).
template <int AP>
__device__ __forceinline__ void replication_words(const RunParams &p, uint32_t isl, uint32_t G,
                                                  Words4 (&w)[AP]) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int a = 0; a < AP; ++a)
    w[a] = philox_rk(p, lane + 32u * a, isl, G, kPurposeReplicate);
}

// a3-a6 for one island: parents (pt, ps) -> children (ct, cs).  Every lane
// runs the same shuffles; children of lanes at or beyond n are garbage and
// are never stored.  Candidate indices are always < n, so only loaded
// parents are ever read.  T2: the tournament size is exactly 2.
template <int AP, bool TRACKED, bool T2 = false>
__device__ __forceinline__ void replicate(const RunParams &p, const Deposit &dep, uint32_t isl,
                                          uint32_t G, const Words4 (&w)[AP],
                                          const uint32_t (&pt)[AP], const uint64_t (&ps)[AP],
                                          uint32_t (&ct)[AP], uint64_t (&cs)[AP]) {
  const uint32_t n = p.n;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    // a3 + a4: fitness is the trait; tournament with replacement, the first
    // drawn candidate keeps ties.
    uint32_t best = uindex(w[a].x, n);
    uint32_t fbest = fetch32<AP>(pt, best);
    if (T2 || p.tournament >= 2) {
      const uint32_t c = uindex(w[a].y, n);
      const uint32_t fc = fetch32<AP>(pt, c);
      const bool take = fc > fbest;
      best = take ? c : best;
      fbest = take ? fc : fbest;
    }
    if constexpr (!T2) {
      for (uint32_t c0 = 2; c0 < p.tournament; c0 += 4) {
        const uint32_t j = (threadIdx.x & 31u) + 32u * a;
        const Words4 e = philox_rk(p, j, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
        const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (c0 + r < p.tournament) {
            const uint32_t c = uindex(ew[r], n);
            const uint32_t fc = fetch32<AP>(pt, c);
            if (fc > fbest) {
              best = c;
              fbest = fc;
            }
          }
        }
      }
    }
    // a5: mutation of the winner's trait.
    ct[a] = mutate(p, fbest, w[a].z);
    // a6: the child inherits the winner's surface plus one new differentia.
    if constexpr (TRACKED) cs[a] = deposit_into(dep, fetch64<AP>(ps, best), w[a].w);
    else cs[a] = 0;
  }
}

// a2: overwrite slot `slot` with the immigrant (vt, vs) held by lane `src`.
template <int AP, bool TRACKED>
__device__ __forceinline__ void land(uint32_t slot, uint32_t src, uint32_t it, uint64_t is,
                                     uint32_t (&pt)[AP], uint64_t (&ps)[AP]) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t vt = __shfl_sync(kFull, it, src);
  uint64_t vs = 0;
  if constexpr (TRACKED) vs = shfl64(is, src);
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    if (lane + 32u * a == slot) {
      pt[a] = vt;
      if constexpr (TRACKED) ps[a] = vs;
    }
  }
}

}  // namespace hsga
