// hsga_async.cu -- free-running (asynchronous) generation kernel.
//
// The paper's islands run without a global clock, each taking whatever its
// neighbours last sent (section "Asynchronous Island-model Genetic
// Algorithm").  Here a warp owns a few islands (lane = agent, n <= 32) and
// runs their generations without ever waiting: at every migrating generation
// it publishes each island's emigrant (slot and direction from the
// counter-based RNG, as in synchronous mode) into that island's single
// outgoing record, then looks at each neighbour's latest record and takes it
// if that record is new and was aimed at this island.  A record is four
// 64-bit words, each holding one 32-bit word of the genome (trait, surface
// low, surface high, counter T) under the same 32-bit stamp
// ((G+1) << 3 | dir << 1).  A 64-bit relaxed access is single-copy atomic,
// so a reader that sees one stamp in all four words holds one whole record
// (exactly one record carries each stamp); a reader that sees mixed stamps
// caught a record being rewritten and ignores it.  No fence is needed on
// either side.  A record is taken if its stamp is newer than the last one
// the reader saw from that neighbour; a record overwritten before a
// neighbour saw it is simply lost (the paper's dropped messages).  Genomes carry their own deposition
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

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// a3-a6 of one island (lane = child slot) when genomes carry their own
// deposition counters: the child deposits at site(T_parent) and carries
// T_parent + 1.  t, s, T: this lane's genome, replaced by its child.  FLT:
// binary32 fitness with Gaussian mutation amounts.  h: the head of the
// replication block Philox(key; lane, *, G, 1), shared by all islands.
template <bool TRACKED, bool T2, bool TWO, bool FLT = false, int NN = 0>
__device__ __forceinline__ void counter_step(const RunParams &p, const PhiloxHead &h,
                                             uint32_t lane, uint32_t isl, uint32_t G,
                                             uint32_t &t, uint64_t &s, uint32_t &T) {
  const uint32_t n = NN ? (uint32_t)NN : p.n;
  uint32_t pt[1] = {t}, pT[1] = {T};
  uint64_t ps[1] = {s};
  const Words4 w = philox_tail<true>(p, h, isl);
  uint32_t best = uindex_nn<NN>(w.x, n);
  uint32_t fbest = fetch32<1>(pt, best);
  if (T2 || p.tournament >= 2) {
    const uint32_t c = uindex_nn<NN>(w.y, n);
    const uint32_t fc = fetch32<1>(pt, c);
    const bool pick = fitter<FLT>(fc, fbest);
    best = pick ? c : best;
    fbest = pick ? fc : fbest;
  }
  if constexpr (!T2) {
    for (uint32_t c0 = 2; c0 < p.tournament; c0 += 4) {
      const Words4 e = philox_rk(p, lane, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
      const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (c0 + q < p.tournament) {
          const uint32_t c = uindex_nn<NN>(ew[q], n);
          const uint32_t fc = fetch32<1>(pt, c);
          if (fitter<FLT>(fc, fbest)) {
            best = c;
            fbest = fc;
          }
        }
      }
    }
  }
  uint32_t child_t;
  if constexpr (FLT)
    child_t = mutate_float(p, fbest, w.z, lane, isl, G);
  else
    child_t = mutate(p, fbest, w.z);
  const uint32_t Tp = fetch32<1>(pT, best);
  uint64_t child_s = 0;
  if constexpr (TRACKED) child_s = deposit_lane<TWO>(p, Tp, fetch64<1>(ps, best), w.w);
  t = child_t;
  s = child_s;
  T = Tp + 1u;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t pick4(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                          uint32_t i) {
  return i == 0 ? a : i == 1 ? b : i == 2 ? c : d;
}

// ------------------------------------------------------------- octets ---
// A warp serves IPW consecutive islands (an "octet") at a time: lane j holds
// agent j of each island, and lane 4k + d serves island k in direction d for
// migration.  A launch keeps every warp resident and gives each a strided
// set of octets; each generation a warp advances all of its octets by one
// generation, so the whole grid progresses together (as the paper's
// processing elements do) however many islands there are.  A warp with a
// single octet keeps it in registers for the whole launch; otherwise octets
// are loaded and stored in place every generation.
template <int IPW>
struct Octet {
  uint32_t first;
  bool live[IPW];
  uint32_t t[IPW], T[IPW];
  uint64_t s[IPW];
};

// NN: agents per island known at compile time (32: the octet's planes are
// one contiguous run of 32 IPW genomes, addressed from one base), or 0.
template <bool TRACKED, int IPW, int NN = 0>
__device__ __forceinline__ void load_octet(const RunParams &p, Octet<IPW> &o, uint32_t first,
                                           uint32_t lane, const uint32_t *tplane,
                                           const uint64_t *splane, const uint32_t *Tplane) {
  o.first = first;
  const uint32_t n = NN ? (uint32_t)NN : p.n;
  const size_t base = (size_t)first * n + lane;
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    const uint32_t isl = first + k;
    o.live[k] = isl < p.islands;
    o.t[k] = o.T[k] = 0;
    o.s[k] = 0;
    if (o.live[k] && (NN == 32 || lane < n)) {
      o.t[k] = tplane[base + k * n];
      if constexpr (TRACKED) o.s[k] = splane[base + k * n];
      o.T[k] = Tplane[base + k * n];
    }
  }
}

template <bool TRACKED, int IPW, int NN = 0>
__device__ __forceinline__ void store_octet(const RunParams &p, const Octet<IPW> &o,
                                            uint32_t lane, uint32_t *tplane, uint64_t *splane,
                                            uint32_t *Tplane) {
  const uint32_t n = NN ? (uint32_t)NN : p.n;
  const size_t base = (size_t)o.first * n + lane;
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    if (o.live[k] && (NN == 32 || lane < n)) {
      tplane[base + k * n] = o.t[k];
      if constexpr (TRACKED) splane[base + k * n] = o.s[k];
      Tplane[base + k * n] = o.T[k];
    }
  }
}

// a3-a6 for every island of the octet.  Islands past the end of the grid
// (last octet only) hold zeros that are never stored or published, so they
// are stepped too: with no branch per island the islands' Philox chains
// share one basic block and the scheduler interleaves them.
template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT, int NN = 0>
__device__ __forceinline__ void octet_step(const RunParams &p, Octet<IPW> &o, uint32_t lane,
                                           uint32_t G) {
  const PhiloxHead h = philox_head(p.k0, p.k1, lane, G, kPurposeReplicate);
#pragma unroll
  for (int k = 0; k < IPW; ++k)
    counter_step<TRACKED, T2, TWO, FLT, NN>(p, h, lane, o.first + k, G, o.t[k], o.s[k],
                                            o.T[k]);
}

// Whether generation G migrates, in 32-bit arithmetic with the every-
// generation case first (free-running generations stay below 2^32).  The
// buffered kernel evaluates it once per generation per warp (208 -> 203 us
// per generation at 16.8M agents, against a 64-bit modulo in every octet's
// generation); the latest-emigrant kernel per octet.
__device__ __forceinline__ bool migrates32(const RunParams &p, uint32_t G) {
  return p.interval == 1u || (p.interval != 0u && G % p.interval == 0u);
}

// Octets owned by this warp: warp, warp + nwarps, ...
__device__ __forceinline__ uint32_t owned_octets(uint32_t warp, uint32_t nwarps,
                                                 uint32_t octets) {
  return warp < octets ? (octets - warp + nwarps - 1) / nwarps : 0u;
}

// ------------------------------------------------- latest-emigrant mode ---
// Migration draws of several octet generations in one Philox pass: lane
// 2 IPW e + b holds, for batch element e (the next octets of this warp, or
// the next generations of one octet) with first island first_e at
// generation G_e, the emigrant block of island first_e + b (b < IPW) or the
// placement block of island first_e + b - IPW.
template <int IPW>
constexpr uint32_t kMigBatch = 32u / (2u * IPW);

template <int IPW>
__device__ __forceinline__ Words4 migration_blocks(const RunParams &p, uint32_t lane,
                                                   uint32_t first_e, uint32_t G_e) {
  const uint32_t b = lane % (2u * IPW);
  return philox_rk(p, b >= (uint32_t)IPW ? kSlotImmigrant : kSlotEmigrant,
                   first_e + b % (uint32_t)IPW, G_e, kPurposeMigration);
}

// One generation of one octet: lane 4k + j publishes word j of island k's
// emigrant record, and lane 4k + d reads the record of island k's neighbour
// in direction d (`seen`: the newest stamp it has seen from it).  m: this
// generation's migration blocks from migration_blocks, at lanes msrc + b.
template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT, int NN = 0>
__device__ __forceinline__ void async_generation(const RunParams &p, Octet<IPW> &o,
                                                 uint32_t &seen, uint32_t lane, uint32_t G,
                                                 const Words4 &m, uint32_t msrc,
                                                 uint64_t *rec, uint32_t *log,
                                                 uint32_t log_G0, uint32_t log_gens) {
  const uint32_t n = NN ? (uint32_t)NN : p.n, first = o.first;
  const uint32_t rk = lane >> 2, rd = lane & 3u;
  const bool reader = lane < 4u * IPW && first + rk < p.islands;
  const uint32_t risl = first + rk;
  const bool logging = log && G >= log_G0 && G - log_G0 < log_gens;
  if (migrates32(p, G)) {
    // a1: lane 4k + j gathers word j of island k's emigrant and publishes it
    uint32_t word = 0, dir = 0;
#pragma unroll
    for (int k = 0; k < IPW; ++k) {
      const uint32_t eslot = uindex_nn<NN>(__shfl_sync(kFull, m.x, msrc + k), n);
      const uint32_t dk = __shfl_sync(kFull, m.y, msrc + k) >> 30;
      const uint32_t vt = __shfl_sync(kFull, o.t[k], eslot);
      const uint64_t vs = shfl64(o.s[k], eslot);
      const uint32_t vT = __shfl_sync(kFull, o.T[k], eslot);
      if (rk == (uint32_t)k) {
        word = pick4(vt, (uint32_t)vs, (uint32_t)(vs >> 32), vT, rd);
        dir = dk;
      }
    }
    if (reader) {
      const uint32_t st = ((G + 1u) << 3) | (dir << 1);
      st_relaxed_u64(rec + 4 * (size_t)risl + rd, ((uint64_t)st << 32) | word);
    }
    // a2: each reader lane looks at its neighbour's latest record
    bool take = false;
    uint32_t s1 = 0, r[4] = {0, 0, 0, 0};
    if (reader) {
      const uint32_t rnb = neighbour(p, risl, rd);
      uint64_t v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = ld_relaxed_u64(rec + 4 * (size_t)rnb + j);
      s1 = (uint32_t)(v[0] >> 32);
      const bool whole = (uint32_t)(v[1] >> 32) == s1 && (uint32_t)(v[2] >> 32) == s1 &&
                         (uint32_t)(v[3] >> 32) == s1;
      if (whole && (s1 >> 3) > seen) {
        seen = s1 >> 3;
        take = ((s1 >> 1) & 3u) == ((rd + 2u) & 3u);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) r[j] = (uint32_t)v[j];
    }
    if (reader && logging)
      log[((size_t)risl * log_gens + (G - log_G0)) * 4 + rd] = take ? (s1 >> 3) : 0u;
    const uint64_t is = ((uint64_t)r[2] << 32) | r[1];
    const uint32_t arrivals = __ballot_sync(kFull, take);
#pragma unroll
    for (int k = 0; k < IPW; ++k) {
      const uint32_t bits = (arrivals >> (4 * k)) & 0xFu;
      if (!bits) continue;
#pragma unroll
      for (uint32_t dd = 0; dd < 4; ++dd) {
        if (bits & (1u << dd)) {
          const uint32_t slot = uindex_nn<NN>(
              __shfl_sync(kFull, pick4(m.x, m.y, m.z, m.w, dd), msrc + IPW + k), n);
          const uint32_t src = 4u * k + dd;
          const uint32_t vt = __shfl_sync(kFull, r[0], src);
          const uint64_t vs = shfl64(is, src);
          const uint32_t vT = __shfl_sync(kFull, r[3], src);
          if (lane == slot) {
            o.t[k] = vt;
            o.s[k] = vs;
            o.T[k] = vT;
          }
        }
      }
    }
  } else if (reader && logging) {
    log[((size_t)risl * log_gens + (G - log_G0)) * 4 + rd] = 0;
  }
  octet_step<TRACKED, T2, TWO, IPW, FLT, NN>(p, o, lane, G);
}

// Residency bounds (blocks per SM) chosen by measurement at 16.8M agents:
// more resident warps outweigh the few spilled registers.
constexpr int kAsyncBlocksPerSM = 8;
constexpr int kBufferedBlocksPerSM = 8;

// SLICED: octets advance `slice` generations per visit (otherwise one, with
// the loop the compiler schedules best: 152.5 against 163.0 us per
// generation at 16.8M agents when the one-generation case runs the general
// loop).
template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT, int NN = 0, bool SLICED = false>
__global__ void __launch_bounds__(kResidentThreads, kAsyncBlocksPerSM)
    step_async_kernel(RunParams p, uint32_t G0, uint32_t ngen, uint32_t slice,
                      uint32_t *__restrict__ tplane,
                      uint64_t *__restrict__ splane, uint32_t *__restrict__ Tplane,
                      uint64_t *__restrict__ rec, uint32_t *__restrict__ seen_io,
                      uint32_t *__restrict__ log, uint32_t log_G0, uint32_t log_gens) {
  static_assert(4 * IPW <= 32, "one lane per island and record word or direction");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  const uint32_t octets = (p.islands + IPW - 1) / IPW;
  const uint32_t owned = owned_octets(warp, nwarps, octets);
  if (owned == 0) return;  // whole warps only; no block barriers are used
  const uint32_t rk = lane >> 2, rd = lane & 3u;
  Octet<IPW> o;
  uint32_t seen = 0;
  if constexpr (SLICED) {
    // each octet visit advances the octet by up to `slice` generations
    for (uint32_t g0 = 0; g0 < ngen; g0 += slice) {
      const uint32_t gl = min(slice, ngen - g0);
      for (uint32_t j = 0; j < owned; ++j) {
        const uint32_t first = (warp + j * nwarps) * IPW;
        const bool reader = lane < 4u * IPW && first + rk < p.islands;
        if (owned > 1 || g0 == 0) {
          load_octet<TRACKED, IPW, NN>(p, o, first, lane, tplane, splane, Tplane);
          seen = reader ? seen_io[(first + rk) * 4 + rd] : 0u;
        }
        Words4 m{0u, 0u, 0u, 0u};
        for (uint32_t g = g0; g < g0 + gl; ++g) {
          // migration draws batched over the next generations of this octet
          const uint32_t q = (g - g0) % kMigBatch<IPW>;
          if (q == 0 && p.interval != 0u)
            m = migration_blocks<IPW>(p, lane, first, G0 + g + lane / (2u * IPW));
          async_generation<TRACKED, T2, TWO, IPW, FLT, NN>(p, o, seen, lane, G0 + g, m,
                                                           q * 2u * IPW, rec, log, log_G0,
                                                           log_gens);
        }
        if (owned > 1 || g0 + gl == ngen) {
          store_octet<TRACKED, IPW, NN>(p, o, lane, tplane, splane, Tplane);
          if (reader) seen_io[(first + rk) * 4 + rd] = seen;
        }
      }
    }
  } else {
    // migration draws batched over this warp's next octets (or, for a warp
    // with a single octet, over its next generations)
    const bool batch_octets = owned > 1;
    Words4 m{0u, 0u, 0u, 0u};
    for (uint32_t g = 0; g < ngen; ++g) {
      for (uint32_t j = 0; j < owned; ++j) {
        const uint32_t first = (warp + j * nwarps) * IPW;
        const bool reader = lane < 4u * IPW && first + rk < p.islands;
        if (owned > 1 || g == 0) {
          load_octet<TRACKED, IPW, NN>(p, o, first, lane, tplane, splane, Tplane);
          seen = reader ? seen_io[(first + rk) * 4 + rd] : 0u;
        }
        const uint32_t q = (batch_octets ? j : g) % kMigBatch<IPW>;
        if (q == 0 && p.interval != 0u) {
          const uint32_t e = lane / (2u * IPW);
          m = batch_octets
                  ? migration_blocks<IPW>(p, lane, (warp + (j + e) * nwarps) * IPW, G0 + g)
                  : migration_blocks<IPW>(p, lane, first, G0 + g + e);
        }
        async_generation<TRACKED, T2, TWO, IPW, FLT, NN>(p, o, seen, lane, G0 + g, m,
                                                         q * 2u * IPW, rec, log, log_G0,
                                                         log_gens);
        if (owned > 1 || g + 1 == ngen) {
          store_octet<TRACKED, IPW, NN>(p, o, lane, tplane, splane, Tplane);
          if (reader) seen_io[(first + rk) * 4 + rd] = seen;
        }
      }
    }
  }
}

// ----------------------------------------------- per-neighbour buffers ---
// The paper's per-neighbour buffers (one genome to send, four received)
// with completion flags.  Lane 4k + d serves island k of the octet in
// direction d.  Each migrating generation it
//   receive: takes the genome on the channel from that neighbour if it is the
//            next post (post numbers count from 1 per channel), appends it to
//            its receive buffer and acknowledges it;
//   place:   when the buffer holds four, they replace members at slots from
//            Philox(key; kSlotImmigrant, island, G, 1 + d), in direction
//            order N, E, S, W and buffer order, later over earlier;
//   send:    if its previous post was acknowledged, posts a copy of the member
//            at the slot from word d of Philox(key; kSlotEmigrant, island, G,
//            0), taken after placement.
// A channel's genome in flight is four 64-bit words, each carrying one
// genome word under the post number: a 64-bit relaxed access is single-copy
// atomic, so a reader that sees the expected post number in all four words
// holds the whole genome, and a sender rewrites the channel only after its
// receiver acknowledged the previous post.  No waits, no fences; within a
// generation every channel store follows a warp vote on every channel load.  The lane
// state {posts, taken, waiting} and the first three buffered genomes live in
// global memory between octet visits; the fourth is placed as it arrives.
struct LaneChannel {
  uint32_t posts, taken, waiting;
};

// Emigrant draws of several generations of one octet in one Philox pass
// (octet slices): lane IPW e + k holds the emigrant block of island
// first + k at generation G + e.
template <int IPW>
constexpr uint32_t kSendBatch = 32u / IPW;

template <int IPW>
__device__ __forceinline__ Words4 emigrant_blocks(const RunParams &p, uint32_t lane,
                                                  uint32_t first, uint32_t G) {
  return philox_rk(p, kSlotEmigrant, first + lane % (uint32_t)IPW, G + lane / (uint32_t)IPW,
                   kPurposeMigration);
}

// BATCHED: the emigrant blocks come from emigrant_blocks (wb, this
// generation's at lanes wsrc + k); otherwise each lane draws its island's
// block itself (one block per generation, fewer registers held across
// octets: 193 against 208 us per generation at 16.8M agents).
template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT, int NN = 0, bool BATCHED = false>
__device__ __forceinline__ void buffered_generation(const RunParams &p, Octet<IPW> &o,
                                                    LaneChannel &ch, uint32_t lane, uint32_t G,
                                                    bool mig, const Words4 &wb, uint32_t wsrc,
                                                    uint64_t *mail, uint32_t *ack,
                                                    uint4 *inbuf, uint32_t *log,
                                                    uint32_t log_G0, uint32_t log_gens) {
  const uint32_t n = NN ? (uint32_t)NN : p.n;
  const uint32_t rk = lane >> 2, rd = lane & 3u;
  const uint32_t me = o.first + rk;
  const bool mine = lane < 4u * IPW && me < p.islands;
  const size_t c = 4 * (size_t)me + rd;  // own channel toward d, own receive buffer from d
  const bool logging = log && G >= log_G0 && G - log_G0 < log_gens;
  uint32_t entry = 0;
  if (mig) {
    const size_t inc = mine ? 4 * (size_t)neighbour(p, me, rd) + ((rd + 2u) & 3u) : 0;
    uint64_t v[4] = {0, 0, 0, 0};
    uint32_t a = 0;
    if (mine) {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = ld_relaxed_u64(mail + 4 * inc + j);
      a = ld_relaxed_u32(ack + c);
    }
    // receive.  The warp votes on every word it loaded (the acknowledgement
    // never exceeds the posts, so that term only ties the vote to it) before
    // any lane writes a channel or an acknowledgement: each island
    // generation then reads before it writes, which is what makes the logged
    // exchanges causally ordered.
    const uint32_t seq = (uint32_t)(v[0] >> 32);
    const bool take = mine && seq == ch.taken + 1u && (uint32_t)(v[1] >> 32) == seq &&
                      (uint32_t)(v[2] >> 32) == seq && (uint32_t)(v[3] >> 32) == seq &&
                      a <= ch.posts;
    const uint32_t takes = __ballot_sync(kFull, take);
    const uint32_t sends = __ballot_sync(kFull, mine && a == ch.posts);
    const bool got = (takes >> lane) & 1u;
    const uint4 arrived =
        make_uint4((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2], (uint32_t)v[3]);
    if (got) {
      if (ch.waiting < 3u) inbuf[4 * c + ch.waiting] = arrived;
      ++ch.waiting;
      ch.taken = seq;
      st_relaxed_u32(ack + inc, seq);
      entry = seq << 1;
    }
    // place full buffers (a buffer fills only as its fourth genome arrives)
    const uint32_t full = __ballot_sync(kFull, mine && ch.waiting == 4u);
    if (full) {
      Words4 pv{0, 0, 0, 0};
      uint4 b0 = make_uint4(0, 0, 0, 0), b1 = b0, b2 = b0;
      if (mine && ch.waiting == 4u) {
        pv = philox_rk(p, kSlotImmigrant, me, G, 1u + rd);
        b0 = inbuf[4 * c];
        b1 = inbuf[4 * c + 1];
        b2 = inbuf[4 * c + 2];
        ch.waiting = 0;
      }
#pragma unroll
      for (int k = 0; k < IPW; ++k) {
        uint32_t bits = (full >> (4 * k)) & 0xFu;
        while (bits) {
          const uint32_t src = 4u * k + (uint32_t)(__ffs(bits) - 1);
          bits &= bits - 1u;
#pragma unroll
          for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t slot =
                uindex_nn<NN>(__shfl_sync(kFull, pick4(pv.x, pv.y, pv.z, pv.w, j), src), n);
            const uint4 bj = j == 0 ? b0 : j == 1 ? b1 : j == 2 ? b2 : arrived;
            const uint32_t gt = __shfl_sync(kFull, bj.x, src);
            const uint32_t glo = __shfl_sync(kFull, bj.y, src);
            const uint32_t ghi = __shfl_sync(kFull, bj.z, src);
            const uint32_t gT = __shfl_sync(kFull, bj.w, src);
            if (lane == slot) {
              o.t[k] = gt;
              o.s[k] = ((uint64_t)ghi << 32) | glo;
              o.T[k] = gT;
            }
          }
        }
      }
    }
    // send on every channel whose previous post was acknowledged
    const bool send = (sends >> lane) & 1u;
    if (sends) {
      uint32_t slot;
      if constexpr (BATCHED) {
        // word d of island k's emigrant block, from lane wsrc + k
        const uint32_t src = wsrc + (rk & (uint32_t)(IPW - 1));
        const uint32_t wx = __shfl_sync(kFull, wb.x, src), wy = __shfl_sync(kFull, wb.y, src);
        const uint32_t wz = __shfl_sync(kFull, wb.z, src), ww = __shfl_sync(kFull, wb.w, src);
        slot = uindex_nn<NN>(pick4(wx, wy, wz, ww, rd), n);
      } else {
        const Words4 w = philox_rk(p, kSlotEmigrant, me, G, kPurposeMigration);
        slot = uindex_nn<NN>(pick4(w.x, w.y, w.z, w.w, rd), n);
      }
      uint32_t et = 0, eT = 0;
      uint64_t es = 0;
#pragma unroll
      for (int k = 0; k < IPW; ++k) {
        const uint32_t vt = __shfl_sync(kFull, o.t[k], slot);
        const uint64_t vs = shfl64(o.s[k], slot);
        const uint32_t vT = __shfl_sync(kFull, o.T[k], slot);
        if (rk == (uint32_t)k) {
          et = vt;
          es = vs;
          eT = vT;
        }
      }
      if (send) {
        ++ch.posts;
        const uint64_t stamp = (uint64_t)ch.posts << 32;
        st_relaxed_u64(mail + 4 * c, stamp | et);
        st_relaxed_u64(mail + 4 * c + 1, stamp | (uint32_t)es);
        st_relaxed_u64(mail + 4 * c + 2, stamp | (uint32_t)(es >> 32));
        st_relaxed_u64(mail + 4 * c + 3, stamp | eT);
        entry |= 1u;
      }
    }
  }
  if (mine && logging) log[((size_t)me * log_gens + (G - log_G0)) * 4 + rd] = entry;
  octet_step<TRACKED, T2, TWO, IPW, FLT, NN>(p, o, lane, G);
}

template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT, int NN = 0, bool SLICED = false>
__global__ void __launch_bounds__(kResidentThreads, kBufferedBlocksPerSM)
    step_buffered_kernel(RunParams p, uint32_t G0, uint32_t ngen, uint32_t slice,
                         uint32_t *__restrict__ tplane,
                         uint64_t *__restrict__ splane, uint32_t *__restrict__ Tplane,
                         uint64_t *__restrict__ mail, uint32_t *__restrict__ ack,
                         uint4 *__restrict__ inbuf, uint4 *__restrict__ chst,
                         uint32_t *__restrict__ log, uint32_t log_G0, uint32_t log_gens) {
  static_assert(4 * IPW <= 32, "one lane per island and direction");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  const uint32_t octets = (p.islands + IPW - 1) / IPW;
  const uint32_t owned = owned_octets(warp, nwarps, octets);
  if (owned == 0) return;  // whole warps only; no block barriers are used
  const uint32_t rk = lane >> 2, rd = lane & 3u;
  Octet<IPW> o;
  LaneChannel ch{0, 0, 0};
  if constexpr (SLICED) {
    // each octet visit advances the octet by up to `slice` generations
    for (uint32_t g0 = 0; g0 < ngen; g0 += slice) {
      const uint32_t gl = min(slice, ngen - g0);
      for (uint32_t j = 0; j < owned; ++j) {
        const uint32_t first = (warp + j * nwarps) * IPW;
        const bool mine = lane < 4u * IPW && first + rk < p.islands;
        const size_t c = 4 * (size_t)(first + rk) + rd;
        if (owned > 1 || g0 == 0) {
          load_octet<TRACKED, IPW, NN>(p, o, first, lane, tplane, splane, Tplane);
          if (mine) {
            const uint4 st = chst[c];
            ch = LaneChannel{st.x, st.y, st.z};
          }
        }
        Words4 wb{0u, 0u, 0u, 0u};
        for (uint32_t g = g0; g < g0 + gl; ++g) {
          // emigrant draws batched over the next generations of this octet
          const uint32_t q = (g - g0) % kSendBatch<IPW>;
          if (q == 0 && p.interval != 0u) wb = emigrant_blocks<IPW>(p, lane, first, G0 + g);
          buffered_generation<TRACKED, T2, TWO, IPW, FLT, NN, true>(
              p, o, ch, lane, G0 + g, migrates32(p, G0 + g), wb, q * IPW, mail, ack, inbuf, log,
              log_G0, log_gens);
        }
        if (owned > 1 || g0 + gl == ngen) {
          store_octet<TRACKED, IPW, NN>(p, o, lane, tplane, splane, Tplane);
          if (mine) chst[c] = make_uint4(ch.posts, ch.taken, ch.waiting, 0u);
        }
      }
    }
  } else {
    for (uint32_t g = 0; g < ngen; ++g) {
      const bool mig = migrates32(p, G0 + g);
      for (uint32_t j = 0; j < owned; ++j) {
        const uint32_t first = (warp + j * nwarps) * IPW;
        const bool mine = lane < 4u * IPW && first + rk < p.islands;
        const size_t c = 4 * (size_t)(first + rk) + rd;
        if (owned > 1 || g == 0) {
          load_octet<TRACKED, IPW, NN>(p, o, first, lane, tplane, splane, Tplane);
          if (mine) {
            const uint4 st = chst[c];
            ch = LaneChannel{st.x, st.y, st.z};
          }
        }
        buffered_generation<TRACKED, T2, TWO, IPW, FLT, NN>(p, o, ch, lane, G0 + g, mig,
                                                            Words4{0u, 0u, 0u, 0u}, 0u, mail,
                                                            ack, inbuf, log, log_G0, log_gens);
        if (owned > 1 || g + 1 == ngen) {
          store_octet<TRACKED, IPW, NN>(p, o, lane, tplane, splane, Tplane);
          if (mine) chst[c] = make_uint4(ch.posts, ch.taken, ch.waiting, 0u);
        }
      }
    }
  }
}

// Islands per warp, chosen by measurement at 16.8M agents: four-island
// octets at 8 blocks per SM beat eight-island octets at 6 in both modes.
constexpr int kAsyncIslandsPerWarp = 4;
constexpr int kBufferedIslandsPerWarp = 4;

using AsyncFn = void (*)(RunParams, uint32_t, uint32_t, uint32_t, uint32_t *, uint64_t *, uint32_t *,
                         uint64_t *, uint32_t *, uint32_t *, uint32_t, uint32_t);

template <bool S>
AsyncFn pick_async_t(bool tracked, bool t2, bool two, bool flt, bool n32) {
  constexpr int I = kAsyncIslandsPerWarp;
  if (n32 && tracked && !two && !flt)  // 32-agent islands, the paper's shape
    return t2 ? step_async_kernel<true, true, false, I, false, 32, S>
              : step_async_kernel<true, false, false, I, false, 32, S>;
  if (flt) {  // general tournament path only
    if (!tracked) return step_async_kernel<false, false, false, I, true, 0, S>;
    return two ? step_async_kernel<true, false, true, I, true, 0, S>
               : step_async_kernel<true, false, false, I, true, 0, S>;
  }
  if (!tracked)
    return t2 ? step_async_kernel<false, true, false, I, false, 0, S>
              : step_async_kernel<false, false, false, I, false, 0, S>;
  if (two)
    return t2 ? step_async_kernel<true, true, true, I, false, 0, S>
              : step_async_kernel<true, false, true, I, false, 0, S>;
  return t2 ? step_async_kernel<true, true, false, I, false, 0, S>
            : step_async_kernel<true, false, false, I, false, 0, S>;
}

AsyncFn pick_async(bool tracked, bool t2, bool two, bool flt, bool n32, bool sliced) {
  return sliced ? pick_async_t<true>(tracked, t2, two, flt, n32)
                : pick_async_t<false>(tracked, t2, two, flt, n32);
}

using BufferedFn = void (*)(RunParams, uint32_t, uint32_t, uint32_t, uint32_t *, uint64_t *, uint32_t *,
                            uint64_t *, uint32_t *, uint4 *, uint4 *, uint32_t *, uint32_t,
                            uint32_t);

template <bool S>
BufferedFn pick_buffered_t(bool tracked, bool t2, bool two, bool flt, bool n32) {
  constexpr int I = kBufferedIslandsPerWarp;
  if (n32 && tracked && !two && !flt)  // 32-agent islands, the paper's shape
    return t2 ? step_buffered_kernel<true, true, false, I, false, 32, S>
              : step_buffered_kernel<true, false, false, I, false, 32, S>;
  if (flt) {  // general tournament path only
    if (!tracked) return step_buffered_kernel<false, false, false, I, true, 0, S>;
    return two ? step_buffered_kernel<true, false, true, I, true, 0, S>
               : step_buffered_kernel<true, false, false, I, true, 0, S>;
  }
  if (!tracked)
    return t2 ? step_buffered_kernel<false, true, false, I, false, 0, S>
              : step_buffered_kernel<false, false, false, I, false, 0, S>;
  if (two)
    return t2 ? step_buffered_kernel<true, true, true, I, false, 0, S>
              : step_buffered_kernel<true, false, true, I, false, 0, S>;
  return t2 ? step_buffered_kernel<true, true, false, I, false, 0, S>
            : step_buffered_kernel<true, false, false, I, false, 0, S>;
}

BufferedFn pick_buffered(bool tracked, bool t2, bool two, bool flt, bool n32, bool sliced) {
  return sliced ? pick_buffered_t<true>(tracked, t2, two, flt, n32)
                : pick_buffered_t<false>(tracked, t2, two, flt, n32);
}

// Synchronous generation with float fitness (after the explicit a1 + a2
// kernels): one warp per island, IPW islands per warp, every genome's
// counter equal to G.
template <bool TRACKED, bool TWO, int IPW>
__global__ void __launch_bounds__(kResidentThreads)
    step_float_kernel(RunParams p, uint32_t G, const uint32_t *__restrict__ tin,
                      const uint64_t *__restrict__ sin, uint32_t *__restrict__ tout,
                      uint64_t *__restrict__ sout) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t first = warp * IPW;
  if (first >= p.islands) return;
  const uint32_t n = p.n;
  uint32_t t[IPW], T[IPW];
  uint64_t s[IPW];
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    const uint32_t isl = first + k;
    t[k] = 0;
    s[k] = 0;
    T[k] = G;
    if (isl < p.islands && lane < n) {
      t[k] = tin[isl * n + lane];
      if constexpr (TRACKED) s[k] = sin[isl * n + lane];
    }
  }
  const PhiloxHead h = philox_head(p.k0, p.k1, lane, G, kPurposeReplicate);
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    const uint32_t isl = first + k;
    if (isl >= p.islands) break;
    counter_step<TRACKED, false, TWO, true>(p, h, lane, isl, G, t[k], s[k], T[k]);
    if (lane < n) {
      tout[isl * n + lane] = t[k];
      if constexpr (TRACKED) sout[isl * n + lane] = s[k];
    }
  }
}

constexpr int kFloatIslandsPerWarp = 4;

// Blocks for a free-running launch: one warp per octet, but never more
// blocks than the device keeps resident at once, so that every island
// advances in the same pass over the grid (warps then own several octets).
uint32_t resident_blocks(const void *fn, uint32_t islands, uint32_t ipw, int max_per_sm) {
  const uint32_t wpb = kResidentThreads / 32;
  const uint32_t octets = (islands + ipw - 1) / ipw;
  const uint32_t need = (octets + wpb - 1) / wpb;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kResidentThreads, 0);
  if (per_sm > max_per_sm) per_sm = max_per_sm;
  const uint32_t cap = (uint32_t)(sms > 0 ? sms : 1) * (uint32_t)(per_sm > 0 ? per_sm : 1);
  return need < cap ? need : cap;
}

}  // namespace

cudaError_t launch_step_float(const RunParams &p, uint32_t G, const uint32_t *tin,
                              const uint64_t *sin, uint32_t *tout, uint64_t *sout,
                              cudaStream_t stream) {
  constexpr int I = kFloatIslandsPerWarp;
  const bool tracked = p.policy != HSGA_NONE, two = p.policy == HSGA_HYBRID;
  const uint32_t wpb = kResidentThreads / 32;
  const uint32_t warps = (p.islands + I - 1) / I;
  const uint32_t blocks = (warps + wpb - 1) / wpb;
  if (!tracked)
    step_float_kernel<false, false, I><<<blocks, kResidentThreads, 0, stream>>>(p, G, tin, sin,
                                                                                tout, sout);
  else if (two)
    step_float_kernel<true, true, I><<<blocks, kResidentThreads, 0, stream>>>(p, G, tin, sin,
                                                                              tout, sout);
  else
    step_float_kernel<true, false, I><<<blocks, kResidentThreads, 0, stream>>>(p, G, tin, sin,
                                                                               tout, sout);
  return cudaGetLastError();
}

cudaError_t launch_step_buffered(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t slice,
                                 uint32_t *t, uint64_t *s, uint32_t *T, uint64_t *mail,
                                 uint32_t *ack, uint4 *inbuf, uint4 *chst, uint32_t *log,
                                 uint32_t log_G0, uint32_t log_gens, cudaStream_t stream) {
  BufferedFn fn = pick_buffered(p.policy != HSGA_NONE, p.tournament == 2,
                                p.policy == HSGA_HYBRID, p.flt, p.n == 32, slice > 1);
  const uint32_t blocks = resident_blocks((const void *)fn, p.islands, kBufferedIslandsPerWarp,
                                          kBufferedBlocksPerSM);
  fn<<<blocks, kResidentThreads, 0, stream>>>(p, G0, ngen, slice > 0 ? slice : 1, t, s, T,
                                               mail, ack, inbuf, chst, log, log_G0, log_gens);
  return cudaGetLastError();
}

cudaError_t launch_step_async(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t slice,
                              uint32_t *t, uint64_t *s, uint32_t *T, uint64_t *rec,
                              uint32_t *seen, uint32_t *log, uint32_t log_G0, uint32_t log_gens,
                              cudaStream_t stream) {
  AsyncFn fn = pick_async(p.policy != HSGA_NONE, p.tournament == 2, p.policy == HSGA_HYBRID,
                          p.flt, p.n == 32, slice > 1);
  const uint32_t blocks = resident_blocks((const void *)fn, p.islands, kAsyncIslandsPerWarp,
                                          kAsyncBlocksPerSM);
  fn<<<blocks, kResidentThreads, 0, stream>>>(p, G0, ngen, slice > 0 ? slice : 1, t, s, T, rec,
                                               seen, log, log_G0, log_gens);
  return cudaGetLastError();
}

}  // namespace hsga
