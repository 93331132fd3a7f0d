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
// binary32 fitness with Gaussian mutation amounts.
template <bool TRACKED, bool T2, bool TWO, bool FLT = false>
__device__ __forceinline__ void counter_step(const RunParams &p, uint32_t lane, uint32_t isl,
                                             uint32_t G, uint32_t &t, uint64_t &s,
                                             uint32_t &T) {
  const uint32_t n = p.n;
  uint32_t pt[1] = {t}, pT[1] = {T};
  uint64_t ps[1] = {s};
  const Words4 w = philox_rk(p, lane, isl, G, kPurposeReplicate);
  uint32_t best = uindex(w.x, n);
  uint32_t fbest = fetch32<1>(pt, best);
  if (T2 || p.tournament >= 2) {
    const uint32_t c = uindex(w.y, n);
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
          const uint32_t c = uindex(ew[q], n);
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
  if constexpr (TRACKED) {
    const Deposit dep = deposit_unpack(deposit_pack(p, Tp), (uint32_t)p.vmask);
    child_s = deposit_into<TWO>(dep, fetch64<1>(ps, best), w.w);
  }
  t = child_t;
  s = child_s;
  T = Tp + 1u;
}

// IPW islands per warp: lane 4k + j writes word j of island k's record, and
// lane 4k + d reads the record of island k's neighbour in direction d.
template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT>
__global__ void __launch_bounds__(kResidentThreads)
    step_async_kernel(RunParams p, uint32_t G0, uint32_t ngen, uint32_t *__restrict__ tplane,
                      uint64_t *__restrict__ splane, uint32_t *__restrict__ Tplane,
                      uint64_t *__restrict__ rec, uint32_t *__restrict__ seen_io, uint32_t *__restrict__ log,
                      uint32_t log_G0, uint32_t log_gens) {
  static_assert(4 * IPW <= 32, "one lane per island and record word or direction");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t first = warp * IPW;
  if (first >= p.islands) return;  // whole warps only; no block barriers are used
  const uint32_t n = p.n;
  uint32_t isl[IPW];
  bool live[IPW];
  uint32_t pt[IPW][1], pT[IPW][1];
  uint64_t ps[IPW][1];
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    isl[k] = first + k;
    live[k] = isl[k] < p.islands;
    pt[k][0] = pT[k][0] = 0;
    ps[k][0] = 0;
    if (live[k] && lane < n) {
      pt[k][0] = tplane[isl[k] * n + lane];
      if constexpr (TRACKED) ps[k][0] = splane[isl[k] * n + lane];
      pT[k][0] = Tplane[isl[k] * n + lane];
    }
  }
  // reader lane r = 4k + d: island k, direction d
  const uint32_t rk = lane >> 2, rd = lane & 3u;
  const bool reader = lane < 4u * IPW && first + rk < p.islands;
  const uint32_t risl = first + rk;
  uint32_t seen = reader ? seen_io[risl * 4 + rd] : 0u;
  const uint32_t rnb = reader ? neighbour(p, risl, rd) : 0u;
  // block lane b: b < IPW the emigrant block of island b, IPW <= b < 2 IPW
  // the placement block of island b - IPW
  const uint32_t bk = lane < (uint32_t)IPW ? lane : (lane < 2u * IPW ? lane - IPW : 0u);
  for (uint32_t g = 0; g < ngen; ++g) {
    const uint32_t G = G0 + g;
    const bool logging = log && G >= log_G0 && G - log_G0 < log_gens;
    if (migrates(p, G)) {
      const Words4 m = philox_rk(p, lane >= (uint32_t)IPW ? kSlotImmigrant : kSlotEmigrant,
                                 first + bk, G, kPurposeMigration);
      // a1: lane 4k + j gathers word j of island k's emigrant and publishes it
      uint32_t word = 0, dir = 0;
#pragma unroll
      for (int k = 0; k < IPW; ++k) {
        const uint32_t eslot = uindex(__shfl_sync(kFull, m.x, k), n);
        const uint32_t dk = __shfl_sync(kFull, m.y, k) >> 30;
        const uint32_t vt = __shfl_sync(kFull, pt[k][0], eslot);
        const uint64_t vs = shfl64(ps[k][0], eslot);
        const uint32_t vT = __shfl_sync(kFull, pT[k][0], eslot);
        if (rk == (uint32_t)k) {
          word = rd == 0 ? vt : rd == 1 ? (uint32_t)vs : rd == 2 ? (uint32_t)(vs >> 32) : vT;
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
      const uint32_t it = r[0], iT = r[3];
      const uint64_t is = ((uint64_t)r[2] << 32) | r[1];
      const uint32_t arrivals = __ballot_sync(kFull, take);
      const uint32_t place[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
      for (int k = 0; k < IPW; ++k) {
        const uint32_t bits = (arrivals >> (4 * k)) & 0xFu;
        if (!bits) continue;
#pragma unroll
        for (uint32_t dd = 0; dd < 4; ++dd) {
          if (bits & (1u << dd)) {
            const uint32_t slot = uindex(__shfl_sync(kFull, place[dd], IPW + k), n);
            const uint32_t src = 4u * k + dd;
            const uint32_t vt = __shfl_sync(kFull, it, src);
            const uint64_t vs = shfl64(is, src);
            const uint32_t vT = __shfl_sync(kFull, iT, src);
            if (lane == slot) {
              pt[k][0] = vt;
              ps[k][0] = vs;
              pT[k][0] = vT;
            }
          }
        }
      }
    } else if (reader && logging) {
      log[((size_t)risl * log_gens + (G - log_G0)) * 4 + rd] = 0;
    }
    // a3-a6 for every owned island, with per-genome counters
#pragma unroll
    for (int k = 0; k < IPW; ++k)
      if (live[k])
        counter_step<TRACKED, T2, TWO, FLT>(p, lane, isl[k], G, pt[k][0], ps[k][0], pT[k][0]);
  }
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    if (live[k] && lane < n) {
      tplane[isl[k] * n + lane] = pt[k][0];
      if constexpr (TRACKED) splane[isl[k] * n + lane] = ps[k][0];
      Tplane[isl[k] * n + lane] = pT[k][0];
    }
  }
  if (reader) seen_io[risl * 4 + rd] = seen;
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

// Buffered free-running migration: the paper's per-neighbour buffers (one
// genome to send, four received) with completion flags.  Lane 4k + d of a
// warp serves island first + k in direction d.  Each migrating generation it
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
// receiver acknowledged the previous post.  No waits, no fences.  The lane
// state {posts, taken, waiting} and the first three buffered genomes persist
// in global memory between launches; the fourth is placed as it arrives.
template <bool TRACKED, bool T2, bool TWO, int IPW, bool FLT>
__global__ void __launch_bounds__(kResidentThreads)
    step_buffered_kernel(RunParams p, uint32_t G0, uint32_t ngen, uint32_t *__restrict__ tplane,
                         uint64_t *__restrict__ splane, uint32_t *__restrict__ Tplane,
                         uint64_t *__restrict__ mail, uint32_t *__restrict__ ack,
                         uint4 *__restrict__ inbuf, uint4 *__restrict__ chst,
                         uint32_t *__restrict__ log, uint32_t log_G0, uint32_t log_gens) {
  static_assert(4 * IPW <= 32, "one lane per island and direction");
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint32_t first = warp * IPW;
  if (first >= p.islands) return;  // whole warps only; no block barriers are used
  const uint32_t n = p.n;
  bool live[IPW];
  uint32_t pt[IPW][1], pT[IPW][1];
  uint64_t ps[IPW][1];
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    const uint32_t isl = first + k;
    live[k] = isl < p.islands;
    pt[k][0] = pT[k][0] = 0;
    ps[k][0] = 0;
    if (live[k] && lane < n) {
      pt[k][0] = tplane[isl * n + lane];
      if constexpr (TRACKED) ps[k][0] = splane[isl * n + lane];
      pT[k][0] = Tplane[isl * n + lane];
    }
  }
  const uint32_t rk = lane >> 2, rd = lane & 3u;
  const bool mine = lane < 4u * IPW && first + rk < p.islands;
  const uint32_t me = first + rk;
  const size_t c = 4 * (size_t)me + rd;  // own channel toward d, own receive buffer from d
  const size_t inc = mine ? 4 * (size_t)neighbour(p, me, rd) + ((rd + 2u) & 3u) : 0;
  uint32_t posts = 0, taken = 0, waiting = 0;
  if (mine) {
    const uint4 st = chst[c];
    posts = st.x;
    taken = st.y;
    waiting = st.z;
  }
  for (uint32_t g = 0; g < ngen; ++g) {
    const uint32_t G = G0 + g;
    const bool logging = log && G >= log_G0 && G - log_G0 < log_gens;
    uint32_t entry = 0;
    if (migrates(p, G)) {
      uint64_t v[4] = {0, 0, 0, 0};
      uint32_t a = 0;
      if (mine) {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = ld_relaxed_u64(mail + 4 * inc + j);
        a = ld_relaxed_u32(ack + c);
      }
      // receive
      const uint32_t seq = (uint32_t)(v[0] >> 32);
      const bool got = mine && seq == taken + 1u && (uint32_t)(v[1] >> 32) == seq &&
                       (uint32_t)(v[2] >> 32) == seq && (uint32_t)(v[3] >> 32) == seq;
      const uint4 arrived = make_uint4((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2],
                                       (uint32_t)v[3]);
      if (got) {
        if (waiting < 3u) inbuf[4 * c + waiting] = arrived;
        ++waiting;
        taken = seq;
        st_relaxed_u32(ack + inc, seq);
        entry = seq << 1;
      }
      // place full buffers (a buffer fills only as its fourth genome arrives)
      const uint32_t full = __ballot_sync(kFull, mine && waiting == 4u);
      if (full) {
        Words4 pv{0, 0, 0, 0};
        uint4 b0 = make_uint4(0, 0, 0, 0), b1 = b0, b2 = b0;
        if (mine && waiting == 4u) {
          pv = philox_rk(p, kSlotImmigrant, me, G, 1u + rd);
          b0 = inbuf[4 * c];
          b1 = inbuf[4 * c + 1];
          b2 = inbuf[4 * c + 2];
          waiting = 0;
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
                  uindex(__shfl_sync(kFull, pick4(pv.x, pv.y, pv.z, pv.w, j), src), n);
              const uint4 bj = j == 0 ? b0 : j == 1 ? b1 : j == 2 ? b2 : arrived;
              const uint32_t gt = __shfl_sync(kFull, bj.x, src);
              const uint32_t glo = __shfl_sync(kFull, bj.y, src);
              const uint32_t ghi = __shfl_sync(kFull, bj.z, src);
              const uint32_t gT = __shfl_sync(kFull, bj.w, src);
              if (lane == slot) {
                pt[k][0] = gt;
                ps[k][0] = ((uint64_t)ghi << 32) | glo;
                pT[k][0] = gT;
              }
            }
          }
        }
      }
      // send on every channel whose previous post was acknowledged
      const bool send = mine && a == posts;
      if (__any_sync(kFull, send)) {
        const Words4 w = philox_rk(p, kSlotEmigrant, me, G, kPurposeMigration);
        const uint32_t slot = uindex(pick4(w.x, w.y, w.z, w.w, rd), n);
        uint32_t et = 0, eT = 0;
        uint64_t es = 0;
#pragma unroll
        for (int k = 0; k < IPW; ++k) {
          const uint32_t vt = __shfl_sync(kFull, pt[k][0], slot);
          const uint64_t vs = shfl64(ps[k][0], slot);
          const uint32_t vT = __shfl_sync(kFull, pT[k][0], slot);
          if (rk == (uint32_t)k) {
            et = vt;
            es = vs;
            eT = vT;
          }
        }
        if (send) {
          ++posts;
          const uint64_t stamp = (uint64_t)posts << 32;
          st_relaxed_u64(mail + 4 * c, stamp | et);
          st_relaxed_u64(mail + 4 * c + 1, stamp | (uint32_t)es);
          st_relaxed_u64(mail + 4 * c + 2, stamp | (uint32_t)(es >> 32));
          st_relaxed_u64(mail + 4 * c + 3, stamp | eT);
          entry |= 1u;
        }
      }
    }
    if (mine && logging) log[((size_t)me * log_gens + (G - log_G0)) * 4 + rd] = entry;
    // a3-a6 for every owned island, with per-genome counters
#pragma unroll
    for (int k = 0; k < IPW; ++k)
      if (live[k])
        counter_step<TRACKED, T2, TWO, FLT>(p, lane, first + k, G, pt[k][0], ps[k][0], pT[k][0]);
  }
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    const uint32_t isl = first + k;
    if (live[k] && lane < n) {
      tplane[isl * n + lane] = pt[k][0];
      if constexpr (TRACKED) splane[isl * n + lane] = ps[k][0];
      Tplane[isl * n + lane] = pT[k][0];
    }
  }
  if (mine) chst[c] = make_uint4(posts, taken, waiting, 0u);
}

constexpr int kAsyncIslandsPerWarp = 8;

using AsyncFn = void (*)(RunParams, uint32_t, uint32_t, uint32_t *, uint64_t *, uint32_t *,
                         uint64_t *, uint32_t *, uint32_t *, uint32_t, uint32_t);

AsyncFn pick_async(bool tracked, bool t2, bool two, bool flt) {
  constexpr int I = kAsyncIslandsPerWarp;
  if (flt) {  // general tournament path only
    if (!tracked) return step_async_kernel<false, false, false, I, true>;
    return two ? step_async_kernel<true, false, true, I, true>
               : step_async_kernel<true, false, false, I, true>;
  }
  if (!tracked)
    return t2 ? step_async_kernel<false, true, false, I, false>
              : step_async_kernel<false, false, false, I, false>;
  if (two)
    return t2 ? step_async_kernel<true, true, true, I, false>
              : step_async_kernel<true, false, true, I, false>;
  return t2 ? step_async_kernel<true, true, false, I, false>
            : step_async_kernel<true, false, false, I, false>;
}

using BufferedFn = void (*)(RunParams, uint32_t, uint32_t, uint32_t *, uint64_t *, uint32_t *,
                            uint64_t *, uint32_t *, uint4 *, uint4 *, uint32_t *, uint32_t,
                            uint32_t);

BufferedFn pick_buffered(bool tracked, bool t2, bool two, bool flt) {
  constexpr int I = kAsyncIslandsPerWarp;
  if (flt) {  // general tournament path only
    if (!tracked) return step_buffered_kernel<false, false, false, I, true>;
    return two ? step_buffered_kernel<true, false, true, I, true>
               : step_buffered_kernel<true, false, false, I, true>;
  }
  if (!tracked)
    return t2 ? step_buffered_kernel<false, true, false, I, false>
              : step_buffered_kernel<false, false, false, I, false>;
  if (two)
    return t2 ? step_buffered_kernel<true, true, true, I, false>
              : step_buffered_kernel<true, false, true, I, false>;
  return t2 ? step_buffered_kernel<true, true, false, I, false>
            : step_buffered_kernel<true, false, false, I, false>;
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
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    const uint32_t isl = first + k;
    if (isl >= p.islands) break;
    counter_step<TRACKED, false, TWO, true>(p, lane, isl, G, t[k], s[k], T[k]);
    if (lane < n) {
      tout[isl * n + lane] = t[k];
      if constexpr (TRACKED) sout[isl * n + lane] = s[k];
    }
  }
}

constexpr int kFloatIslandsPerWarp = 4;

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

cudaError_t launch_step_buffered(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t *t,
                                 uint64_t *s, uint32_t *T, uint64_t *mail, uint32_t *ack,
                                 uint4 *inbuf, uint4 *chst, uint32_t *log, uint32_t log_G0,
                                 uint32_t log_gens, cudaStream_t stream) {
  BufferedFn fn =
      pick_buffered(p.policy != HSGA_NONE, p.tournament == 2, p.policy == HSGA_HYBRID, p.flt);
  const uint32_t wpb = kResidentThreads / 32;
  const uint32_t warps = (p.islands + kAsyncIslandsPerWarp - 1) / kAsyncIslandsPerWarp;
  const uint32_t blocks = (warps + wpb - 1) / wpb;
  fn<<<blocks, kResidentThreads, 0, stream>>>(p, G0, ngen, t, s, T, mail, ack, inbuf, chst, log,
                                               log_G0, log_gens);
  return cudaGetLastError();
}

cudaError_t launch_step_async(const RunParams &p, uint32_t G0, uint32_t ngen, uint32_t *t,
                              uint64_t *s, uint32_t *T, uint64_t *rec, uint32_t *seen,
                              uint32_t *log, uint32_t log_G0, uint32_t log_gens,
                              cudaStream_t stream) {
  AsyncFn fn =
      pick_async(p.policy != HSGA_NONE, p.tournament == 2, p.policy == HSGA_HYBRID, p.flt);
  const uint32_t wpb = kResidentThreads / 32;
  const uint32_t warps = (p.islands + kAsyncIslandsPerWarp - 1) / kAsyncIslandsPerWarp;
  const uint32_t blocks = (warps + wpb - 1) / wpb;
  fn<<<blocks, kResidentThreads, 0, stream>>>(p, G0, ngen, t, s, T, rec, seen, log, log_G0,
                                               log_gens);
  return cudaGetLastError();
}

}  // namespace hsga
