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

// Heads of the replication blocks Philox(seed; j, *, G, 1) of this lane's
// children j = lane + 32a, for a whole launch at generation G.
template <int AP>
__device__ __forceinline__ void replication_heads(const RunParams &p, uint32_t G,
                                                  PhiloxHead (&h)[AP]) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int a = 0; a < AP; ++a) h[a] = philox_head(p.k0, p.k1, lane + 32u * a, G, kPurposeReplicate);
}

// Replication words of child j (lane-owned): Philox(seed; j, island, G, 1).
template <int AP, bool RK = true>
__device__ __forceinline__ void replication_words(const RunParams &p, uint32_t isl, uint32_t G,
                                                  Words4 (&w)[AP]) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int a = 0; a < AP; ++a)
    w[a] = philox_p<RK>(p, lane + 32u * a, isl, G, kPurposeReplicate);
}

// floor(w n / 2^32); NN: n when known at compile time (32: a shift), else 0.
template <int NN>
__device__ __forceinline__ uint32_t uindex_nn(uint32_t w, uint32_t n) {
  if constexpr (NN == 32) return w >> 27;
  else return uindex(w, n);
}

// a3-a6 for one island: parents (pt, ps) -> children (ct, cs).  Every lane
// runs the same shuffles; children of lanes at or beyond n are garbage and
// are never stored.  Candidate indices are always < n, so only loaded
// parents are ever read.  T2: the tournament size is exactly 2.
template <int AP, bool TRACKED, bool T2 = false, bool RK = true, bool TWO = false,
          bool DEL = true, int NN = 0>
__device__ __forceinline__ void replicate(const RunParams &p, const Deposit &dep, uint32_t isl,
                                          uint32_t G, const Words4 (&w)[AP],
                                          const uint32_t (&pt)[AP], const uint64_t (&ps)[AP],
                                          uint32_t (&ct)[AP], uint64_t (&cs)[AP]) {
  const uint32_t n = p.n;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    // a3 + a4: fitness is the trait; tournament with replacement, the first
    // drawn candidate keeps ties.
    uint32_t best = uindex_nn<NN>(w[a].x, n);
    uint32_t fbest = fetch32<AP>(pt, best);
    if (T2 || p.tournament >= 2) {
      const uint32_t c = uindex_nn<NN>(w[a].y, n);
      const uint32_t fc = fetch32<AP>(pt, c);
      const bool take = fc > fbest;
      best = take ? c : best;
      fbest = take ? fc : fbest;
    }
    if constexpr (!T2) {
      for (uint32_t c0 = 2; c0 < p.tournament; c0 += 4) {
        const uint32_t j = (threadIdx.x & 31u) + 32u * a;
        const Words4 e = philox_p<RK>(p, j, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
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
    ct[a] = mutate<DEL>(p, fbest, w[a].z);
    // a6: the child inherits the winner's surface plus one new differentia.
    if constexpr (TRACKED) cs[a] = deposit_into<TWO>(dep, fetch64<AP>(ps, best), w[a].w);
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

// --------------------------------------------- island groups (streaming) ---
// A warp advances groups of kGroup consecutive islands.  The group's
// migration draws take one warp-wide Philox evaluation: lane 5p+r (r < 4)
// evaluates the emigrant block of the neighbour in direction r of island
// isl0+p and gathers that emigrant's genome from the parent planes when it is
// aimed at isl0+p; lane 5p+4 evaluates the placement block of isl0+p and
// turns it into a landing plan: byte 3-d holds the slot where the direction-d
// immigrant lands, or 0xFF when it does not arrive.  Later arrivals overwrite
// earlier ones, and the reversed byte order makes the lowest matching byte
// the latest direction, so slots shared by several arrivals need no pass.
constexpr uint32_t kGroup = 6;  // 6 islands x 5 blocks = 30 of 32 lanes

struct GroupMigration {
  uint32_t plan;  // lane 5p+4: landing plan of island isl0+p
  uint32_t it;    // lane 5p+r: the direction-r immigrant's genome
  uint64_t is;
};

template <bool TRACKED, bool RK = true, int NN = 0>
__device__ __forceinline__ void group_migration(const RunParams &p, uint32_t isl0, uint32_t G,
                                                const uint32_t *__restrict__ tin,
                                                const uint64_t *__restrict__ sin,
                                                GroupMigration &gm) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t pi = lane / 5u, role = lane - pi * 5u;
  const uint32_t isl = isl0 + pi;
  const bool valid = lane < 5u * kGroup && isl < p.islands;
  const uint32_t src = valid ? (role == 4 ? isl : neighbour(p, isl, role)) : 0u;
  const Words4 m =
      philox_p<RK>(p, role == 4 ? kSlotImmigrant : kSlotEmigrant, src, G, kPurposeMigration);
  const bool arrive = valid && role < 4 && (m.y >> 30) == ((role + 2u) & 3u);
  gm.it = 0;
  gm.is = 0;
  if (arrive) {
    const uint32_t a = src * (NN ? (uint32_t)NN : p.n) + uindex_nn<NN>(m.x, p.n);
    gm.it = __ldg(tin + a);
    if constexpr (TRACKED) gm.is = __ldg(sin + a);
  }
  const uint32_t arrivals = __ballot_sync(kFull, arrive);
  const uint32_t bits = (arrivals >> (5u * pi)) & 0xFu;
  // slots (< 64) in byte d, 0xFF in the bytes of directions with no arrival
  // (the multiply spreads bit d of `miss` to bit 8d without carries), then the
  // byte order reversed
  const uint32_t miss = ~bits & 0xFu;
  const uint32_t fwd = uindex_nn<NN>(m.x, p.n) | (uindex_nn<NN>(m.y, p.n) << 8) |
                       (uindex_nn<NN>(m.z, p.n) << 16) | (uindex_nn<NN>(m.w, p.n) << 24) |
                       (((miss * 0x00204081u) & 0x01010101u) * 0xFFu);
  gm.plan = (role == 4 && valid) ? __byte_perm(fwd, 0u, 0x0123u) : 0xFFFFFFFFu;
}

// a2 for island isl0+k: each lane looks its slots up in the landing plan
// (a zero-byte test on plan ^ slot) and pulls the immigrant from the lane that
// gathered it.
template <int AP, bool TRACKED>
__device__ __forceinline__ void group_land(const GroupMigration &gm, uint32_t k,
                                           uint32_t (&pt)[AP], uint64_t (&ps)[AP]) {
  const uint32_t plan = __shfl_sync(kFull, gm.plan, 5u * k + 4u);
  if (plan == 0xFFFFFFFFu) return;
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    const uint32_t x = plan ^ ((lane + 32u * a) * 0x01010101u);
    // the lowest set bit of z marks the lowest zero byte of x exactly (a
    // borrow only runs upward from a zero byte); byte 3-d is direction d, so
    // bit 31-8d isolated has 8d leading zeros
    const uint32_t z = (x - 0x01010101u) & ~x & 0x80808080u;
    const uint32_t d = (uint32_t)__clz(z & (0u - z)) >> 3;
    const uint32_t src = z ? 5u * k + d : lane;
    const uint32_t vt = __shfl_sync(kFull, gm.it, src);
    if (z) pt[a] = vt;
    if constexpr (TRACKED) {
      const uint64_t vs = shfl64(gm.is, src);
      if (z) ps[a] = vs;
    }
  }
}

// NN: agents per island known at compile time (32), or 0 for a runtime n.
template <int AP, bool TRACKED, int NN = 0>
__device__ __forceinline__ void load_island(const RunParams &p, uint32_t isl,
                                            const uint32_t *__restrict__ tin,
                                            const uint64_t *__restrict__ sin, uint32_t (&t)[AP],
                                            uint64_t (&s)[AP]) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = NN ? (uint32_t)NN : p.n;
  const uint32_t base = isl * n;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    const uint32_t j = lane + 32u * a;
    t[a] = 0;
    s[a] = 0;
    if (NN == 32 || j < n) {
      t[a] = __ldcs(tin + base + j);
      if constexpr (TRACKED) s[a] = __ldcs(sin + base + j);
    }
  }
}

template <int AP, bool TRACKED, int NN = 0>
__device__ __forceinline__ void store_island(const RunParams &p, uint32_t isl,
                                             uint32_t *__restrict__ tout,
                                             uint64_t *__restrict__ sout,
                                             const uint32_t (&t)[AP], const uint64_t (&s)[AP]) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = NN ? (uint32_t)NN : p.n;
  const uint32_t base = isl * n;
#pragma unroll
  for (int a = 0; a < AP; ++a) {
    const uint32_t j = lane + 32u * a;
    if (NN == 32 || j < n) {
      __stcs(tout + base + j, t[a]);
      if constexpr (TRACKED) __stcs(sout + base + j, s[a]);
    }
  }
}

// One full group: all six islands' genomes are requested up front (deep
// memory-level parallelism), then the islands are processed ILV at a time so
// that each lane runs ILV independent Philox chains (instruction-level
// parallelism hides the multiply-xor dependency chain of the rounds).
constexpr int kInterleave = 2;

// MIG: 1 or 0 when the launch is known to migrate or not (the migration draws
// then share a basic block with the first islands' replication draws, and the
// scheduler interleaves the chains); -1 reads do_mig at run time.
template <int AP, bool TRACKED, bool T2, int NN, int ILV = kInterleave, bool RK = true,
          bool TWO = false, bool DEL = true, int MIG = -1>
__device__ __forceinline__ void full_group(const RunParams &p, const Deposit &dep, uint32_t G,
                                           bool do_mig, uint32_t isl0,
                                           const uint32_t *__restrict__ tin,
                                           const uint64_t *__restrict__ sin,
                                           uint32_t *__restrict__ tout,
                                           uint64_t *__restrict__ sout,
                                           const PhiloxHead (&head)[AP]) {
  static_assert(kGroup % ILV == 0, "interleave width must divide the group");
  if constexpr (MIG >= 0) do_mig = MIG == 1;
  uint32_t pt[kGroup][AP];
  uint64_t ps[kGroup][AP];
#pragma unroll
  for (uint32_t k = 0; k < kGroup; ++k)
    load_island<AP, TRACKED, NN>(p, isl0 + k, tin, sin, pt[k], ps[k]);
  GroupMigration gm;
  if (do_mig) group_migration<TRACKED, RK, NN>(p, isl0, G, tin, sin, gm);
#pragma unroll
  for (uint32_t k = 0; k < kGroup; k += ILV) {
    Words4 w[ILV][AP];
#pragma unroll
    for (int i = 0; i < ILV; ++i)
#pragma unroll
      for (int a = 0; a < AP; ++a) w[i][a] = philox_tail<RK>(p, head[a], isl0 + k + i);
    if (do_mig) {
#pragma unroll
      for (int i = 0; i < ILV; ++i) group_land<AP, TRACKED>(gm, k + i, pt[k + i], ps[k + i]);
    }
    uint32_t ct[ILV][AP];
    uint64_t cs[ILV][AP];
#pragma unroll
    for (int i = 0; i < ILV; ++i)
      replicate<AP, TRACKED, T2, RK, TWO, DEL, NN>(p, dep, isl0 + k + i, G, w[i], pt[k + i],
                                                   ps[k + i], ct[i], cs[i]);
#pragma unroll
    for (int i = 0; i < ILV; ++i)
      store_island<AP, TRACKED, NN>(p, isl0 + k + i, tout, sout, ct[i], cs[i]);
  }
}

// The last, partial group: islands one at a time.
template <int AP, bool TRACKED, bool T2, bool RK = true>
__device__ __noinline__ void partial_group(const RunParams &p, const Deposit &dep, uint32_t G,
                                           bool do_mig, uint32_t isl0,
                                           const uint32_t *__restrict__ tin,
                                           const uint64_t *__restrict__ sin,
                                           uint32_t *__restrict__ tout,
                                           uint64_t *__restrict__ sout) {
  GroupMigration gm;
  if (do_mig) group_migration<TRACKED, RK>(p, isl0, G, tin, sin, gm);
  for (uint32_t k = 0; isl0 + k < p.islands; ++k) {
    uint32_t pt[AP], ct[AP];
    uint64_t ps[AP], cs[AP];
    load_island<AP, TRACKED>(p, isl0 + k, tin, sin, pt, ps);
    Words4 w[AP];
    replication_words<AP, RK>(p, isl0 + k, G, w);
    if (do_mig) group_land<AP, TRACKED>(gm, k, pt, ps);
    if (dep.two) replicate<AP, TRACKED, T2, RK, true>(p, dep, isl0 + k, G, w, pt, ps, ct, cs);
    else replicate<AP, TRACKED, T2, RK, false>(p, dep, isl0 + k, G, w, pt, ps, ct, cs);
    store_island<AP, TRACKED>(p, isl0 + k, tout, sout, ct, cs);
  }
}

}  // namespace hsga
