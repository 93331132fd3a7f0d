// hsga_resident.cu -- persistent resident generation kernel.
//
// One cooperative launch advances many synchronous generations.  Each warp
// owns IPW islands and keeps their genomes in registers for the whole launch
// (lane l: agents l and l+32).  There is no grid-wide barrier: islands only
// depend on their four neighbours' emigrants.  Multi-block grids are cut
// into tiles of islands, one tile per block (the smallest tiles that fit:
// 2x2 on a 64x64 grid); inside a tile the emigrants go through shared
// memory and one block barrier per migration.  Across tiles (and, where no
// tile shape fits, between all islands) each island publishes its emigrant
// as a record of four 64-bit words (trait, surface low, surface high,
// direction), each word carrying the migration's sequence number in its
// high half, into a slot double-buffered by migration parity; a receiver
// polls the four words of each neighbour's record until all carry the
// sequence number it expects.  A 64-bit relaxed access is single-copy
// atomic, so no fence or separate flag is needed: seeing the number in all
// four words means seeing the whole record.  An island can run at most one
// migration ahead of a neighbour, which is why two record buffers suffice: a
// record of migration m is only overwritten at m+2, after the writer has read
// the reader's m+1 record, which the reader publishes only after its poll of
// the m record has returned (the warp votes on the polled values before any
// later store).
//
// Every wait is bounded (1 s of %globaltimer); on expiry the warp records a
// timeout in the grid's error word and leaves (in a tile: at the block's
// next barrier, with the rest of the block), which lets its neighbours time
// out in turn.  The cooperative launch guarantees that every island's
// warp is resident, so waits only expire on an inconsistent state.
#include <cuda_runtime.h>

#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {

constexpr uint32_t kChunk = 16;  // generations whose per-island RNG blocks are batched

// Whether generation G migrates, and its migration number G / interval, in
// 32-bit arithmetic with the every-generation case first: a 64-bit modulo
// and a division per generation made up about half of the kernel's
// instructions on the 64x64-island grid.
__device__ __forceinline__ bool migration_of(const RunParams &p, uint32_t G, uint32_t *m_idx) {
  if (p.interval == 1u) {
    *m_idx = G;
    return true;
  }
  if (p.interval == 0u) return false;
  const uint32_t q = G / p.interval;
  *m_idx = q;
  return q * p.interval == G;
}

__device__ __forceinline__ uint64_t ld_relaxed64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until all four words of a record carry sequence number seq
// in their high halves; the record's low halves go to *out.  Gives up after
// limit_ns of the global timer or kMaxSpins polls, whichever comes first, or
// as soon as another warp has reported an error.  Returns false when it gave
// up.
constexpr uint32_t kMaxSpins = 1u << 22;

__device__ __forceinline__ bool record_ready(const uint64_t *r, uint32_t seq, uint4 *out) {
  const uint64_t w0 = ld_relaxed64(r), w1 = ld_relaxed64(r + 1);
  const uint64_t w2 = ld_relaxed64(r + 2), w3 = ld_relaxed64(r + 3);
  if ((uint32_t)(w0 >> 32) != seq || (uint32_t)(w1 >> 32) != seq ||
      (uint32_t)(w2 >> 32) != seq || (uint32_t)(w3 >> 32) != seq)
    return false;
  *out = make_uint4((uint32_t)w0, (uint32_t)w1, (uint32_t)w2, (uint32_t)w3);
  return true;
}

// Polls the first word alone until it carries seq, then reads the whole
// record: a quarter of the polling loads of reading all four words each time
// (2.93 against 3.34 us per generation on the 64x64-island grid, where 16k
// lanes poll at once and their traffic delays the records they wait for).
__device__ bool wait_record(const uint64_t *r, uint32_t seq, const int *err, uint4 *out,
                            uint64_t limit_ns = kWaitNs) {
  const uint64_t t0 = global_ns();
  for (uint32_t spin = 1; spin < kMaxSpins; ++spin) {
    if ((uint32_t)(ld_relaxed64(r) >> 32) == seq && record_ready(r, seq, out)) return true;
    if ((spin & 255u) == 0) {
      if (*(volatile const int *)err != 0) return false;
      if (global_ns() - t0 > limit_ns) return false;
    }
  }
  return false;
}

// kTiled: the whole warp waits for the records of its island's neighbours
// in other tiles at once.  Lane 4d + j (< 16) polls word j of the record of
// direction d (if `polled`: that neighbour lies in another tile), so every
// poll fetches whole records in one round trip; the wait ends when every
// polled word carries seq.  Lane 4d + j's word is returned in *word.
// Bounded like wait_record; returns false (on every lane) when it gave up.
__device__ bool wait_records_warp(const uint64_t *r, bool polled, uint32_t seq, const int *err,
                                  uint32_t *word, uint64_t limit_ns = kWaitNs) {
  const uint64_t t0 = global_ns();
  for (uint32_t spin = 1; spin < kMaxSpins; ++spin) {
    bool ready = true;
    if (polled) {
      const uint64_t v = ld_relaxed64(r);
      ready = (uint32_t)(v >> 32) == seq;
      *word = (uint32_t)v;
    }
    if (__all_sync(kFull, ready)) return true;
    if ((spin & 255u) == 0) {
      const bool stop = *(volatile const int *)err != 0 || global_ns() - t0 > limit_ns;
      if (__any_sync(kFull, stop)) return false;
    }
  }
  return false;
}

// Both forms of the wait on a caller's record (hsga_wait_probe), in turn:
// lane 0 alone runs wait_record, then the whole warp runs wait_records_warp
// with lanes 0..3 polling words 0..3.  out[0] = 1 if both saw the record
// carry seq, 0 if either gave up; out[1] = nanoseconds spent in all.
__global__ void wait_probe_kernel(const uint64_t *record, uint32_t seq, uint64_t limit_ns,
                                  int *err, uint64_t *out) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t t0 = global_ns();
  bool ok = true;
  if (lane == 0) {
    uint4 r;
    ok = wait_record(record, seq, err, &r, limit_ns);
  }
  ok = __shfl_sync(kFull, ok, 0);
  uint32_t word = 0;
  const bool ok_warp =
      wait_records_warp(record + (lane & 3u), lane < 4, seq, err, &word, limit_ns);
  if (lane == 0) {
    out[0] = (ok && ok_warp) ? 1u : 0u;
    out[1] = global_ns() - t0;
  }
}

// Three ways of exchanging the emigrant records (MODE):
//  kPolled:    every island polls its four neighbours' records in global
//              memory (warps numbered in row-major island order).
//  kBlockSync: the whole grid lives in one thread block (at most 32 warps);
//              records go to shared memory and one __syncthreads per
//              migration replaces the polling (the record buffer of
//              migration m is rewritten at m+2, after the barrier of m+1,
//              which every reader of m has passed).
//  kTiled:     each block holds a 2^ltr x 2^ltc tile of islands, one per
//              warp; neighbours inside the tile are read from shared memory
//              after one block barrier per migration, and only neighbours in
//              other tiles are polled in global memory (islands on the tile's
//              edge publish there as well).  The barrier also spreads a
//              failed wait to the whole block, so that every warp leaves at
//              the same barrier.
template <int AP, int IPW, bool TRACKED, int MODE>
__global__ void __launch_bounds__(MODE == kPolled ? kResidentThreads : 1024)
    step_resident_kernel(RunParams p, uint32_t G0, uint32_t ngen, int premigrated,
                         uint32_t tile, uint32_t *__restrict__ tplane,
                         uint64_t *__restrict__ splane, uint64_t *__restrict__ rec,
                         int *__restrict__ err) {
  constexpr bool BLOCKSYNC = MODE == kBlockSync;
  constexpr bool TILED = MODE == kTiled;
  static_assert(!TILED || IPW == 1, "tiled exchange: one island per warp");
  __shared__ uint4 srec[MODE == kPolled ? 1 : 2 * 32 * IPW];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  uint32_t isl[IPW];
  uint32_t pt[IPW][AP];
  uint64_t ps[IPW][AP];
  // kTiled: this warp's island, and per direction (lane d < 4) where its
  // neighbour's record is read: shared-memory slot, or global record.
  uint32_t nb_island = 0, nb_slot = 0;
  bool nb_inside = true, publish_global = !BLOCKSYNC;
  const uint64_t *poll_word = nullptr;  // kTiled, lane 4d + j: word j of direction d's record
  bool polls = false;
  if constexpr (TILED) {
    const uint32_t ltr = tile & 0xFFu, ltc = tile >> 8;
    const uint32_t tiles_c = (p.cols + (1u << ltc) - 1) >> ltc;
    const uint32_t tr = blockIdx.x / tiles_c, tc = blockIdx.x - tr * tiles_c;
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t r = (tr << ltr) + (w >> ltc), c = (tc << ltc) + (w & ((1u << ltc) - 1));
    const bool active = r < p.rows && c < p.cols;
    isl[0] = active ? r * p.cols + c : p.islands;
    if (active && lane < 4) {
      nb_island = neighbour(p, isl[0], lane);
      const uint32_t nr = nb_island / p.cols, nc = nb_island - nr * p.cols;
      nb_inside = (nr >> ltr) == tr && (nc >> ltc) == tc;
      nb_slot = ((nr & ((1u << ltr) - 1)) << ltc) | (nc & ((1u << ltc) - 1));
    }
    publish_global = __any_sync(kFull, !nb_inside);
    // lane 4d + j polls word j of direction d's record (both buffers: +buf offset)
    const uint32_t d = (lane >> 2) & 3u;
    const uint32_t nb_d = __shfl_sync(kFull, nb_island, d);
    const bool inside_d = __shfl_sync(kFull, nb_inside, d);
    polls = lane < 16 && !inside_d;
    poll_word = rec + (size_t)nb_d * 4 + (lane & 3u);
  }
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
    if constexpr (!TILED) isl[k] = warp * IPW + k;
#pragma unroll
    for (int a = 0; a < AP; ++a) {
      const uint32_t j = lane + 32u * a;
      pt[k][a] = 0;
      ps[k][a] = 0;
      if (isl[k] < p.islands && j < p.n) {
        pt[k][a] = tplane[(size_t)isl[k] * p.n + j];
        if constexpr (TRACKED) ps[k][a] = splane[(size_t)isl[k] * p.n + j];
      }
    }
  }
  const bool any_mig = p.interval != 0;
  bool failed = false;  // leave now (block-uniform in kTiled)
  bool wfail = false;   // kTiled: this warp's wait gave up; the block learns at its barrier

  for (uint32_t g0 = 0; g0 < ngen && !failed; g0 += kChunk) {
    // Batched per-chunk draws: lane o (< 16) holds the emigrant block of
    // generation G0+g0+o, lane 16+o its placement block; every lane holds
    // the packed deposit of generation G0+g0+(lane & 15).
    const uint32_t Gl = G0 + g0 + (lane & (kChunk - 1));
    const uint32_t dpack = deposit_pack(p, Gl);
    Words4 mig[IPW];
#pragma unroll
    for (int k = 0; k < IPW; ++k) {
      mig[k] = Words4{0, 0, 0, 0};
      if (any_mig && isl[k] < p.islands)
        mig[k] = philox_rk(p, lane < kChunk ? kSlotEmigrant : kSlotImmigrant, isl[k], Gl,
                        kPurposeMigration);
    }
    const uint32_t steps = min(kChunk, ngen - g0);
    for (uint32_t o = 0; o < steps; ++o) {
      const uint32_t G = G0 + g0 + o;
      const uint32_t dp = __shfl_sync(kFull, dpack, o);
      const Deposit dep = deposit_unpack(dp, (uint32_t)p.vmask);
      uint32_t m_idx = 0;
      const bool do_mig = migration_of(p, G, &m_idx) && !(premigrated && g0 + o == 0);
      uint32_t buf = 0, seq = 0;
      if (do_mig) {
        buf = m_idx & 1u;
        seq = m_idx + 1u;
        // a1: publish every owned island's emigrant before reading any.
#pragma unroll
        for (int k = 0; k < IPW; ++k) {
          if (isl[k] >= p.islands || wfail) continue;
          const uint32_t eslot = uindex(__shfl_sync(kFull, mig[k].x, o), p.n);
          const uint32_t dir = __shfl_sync(kFull, mig[k].y, o) >> 30;
          if (lane == (eslot & 31u)) {
            uint32_t tv = pt[k][0];
            uint64_t sv = ps[k][0];
            if constexpr (AP == 2) {
              if (eslot >> 5) {
                tv = pt[k][1];
                sv = ps[k][1];
              }
            }
            if constexpr (BLOCKSYNC) {
              srec[buf * 32 * IPW + isl[k]] =
                  make_uint4(tv, (uint32_t)sv, (uint32_t)(sv >> 32), dir);
            } else if (TILED) {
              srec[buf * 32 + (threadIdx.x >> 5)] =
                  make_uint4(tv, (uint32_t)sv, (uint32_t)(sv >> 32), dir);
            }
            if (publish_global) {
              uint64_t *r = rec + ((size_t)buf * p.islands + isl[k]) * 4;
              const uint64_t stamp = (uint64_t)seq << 32;
              st_relaxed64(r, stamp | tv);
              st_relaxed64(r + 1, stamp | (uint32_t)sv);
              st_relaxed64(r + 2, stamp | (uint32_t)(sv >> 32));
              st_relaxed64(r + 3, stamp | dir);
            }
          }
        }
        if constexpr (BLOCKSYNC) __syncthreads();
        if constexpr (TILED) {
          // every warp of the tile arrives here once per migration, also
          // after a failed wait, so the block leaves together
          if (__syncthreads_or(wfail ? 1 : 0)) {
            failed = true;
            break;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < IPW; ++k) {
        if (isl[k] >= p.islands) continue;
        Words4 w[AP];
        replication_words<AP>(p, isl[k], G, w);
        if (do_mig) {
          // a2: lanes 0..3 take the neighbour records in directions N, E, S, W.
          bool ok = true, arrive = false;
          uint32_t it = 0;
          uint64_t is = 0;
          if constexpr (TILED) {
            // records from other tiles: one warp-wide wait, then lane d
            // gathers the four words of direction d
            uint32_t word = 0;
            ok = wait_records_warp(poll_word + (size_t)buf * p.islands * 4, polls, seq, err,
                                   &word);
            const uint32_t src = (lane & 3u) << 2;
            const uint32_t g0 = __shfl_sync(kFull, word, src);
            const uint32_t g1 = __shfl_sync(kFull, word, src + 1);
            const uint32_t g2 = __shfl_sync(kFull, word, src + 2);
            const uint32_t g3 = __shfl_sync(kFull, word, src + 3);
            if (lane < 4 && ok) {
              uint4 r = make_uint4(g0, g1, g2, g3);
              if (nb_inside) r = srec[buf * 32 + nb_slot];
              arrive = r.w == ((lane + 2u) & 3u);
              it = r.x;
              is = ((uint64_t)r.z << 32) | r.y;
            }
          } else if (lane < 4) {
            const uint32_t nb = neighbour(p, isl[k], lane);
            uint4 r;
            if constexpr (BLOCKSYNC) {
              r = srec[buf * 32 * IPW + nb];
            } else {
              ok = wait_record(rec + ((size_t)buf * p.islands + nb) * 4, seq, err, &r);
            }
            if (ok) {
              arrive = r.w == ((lane + 2u) & 3u);
              it = r.x;
              is = ((uint64_t)r.z << 32) | r.y;
            }
          }
          if constexpr (MODE == kPolled) {
            if (__any_sync(kFull, !ok)) {
              if (lane == 0) atomicCAS(err, 0, kDevErrWaitTimeout);
              failed = true;
              break;
            }
          }
          if constexpr (TILED) {
            // the warp stops work and goes on to the next barrier, where
            // the block leaves together
            if (__any_sync(kFull, !ok)) {
              if (lane == 0) atomicCAS(err, 0, kDevErrWaitTimeout);
              wfail = true;
            }
            if (wfail) continue;
          }
          const uint32_t arrivals = __ballot_sync(kFull, arrive);
          const uint32_t place[4] = {mig[k].x, mig[k].y, mig[k].z, mig[k].w};
#pragma unroll
          for (uint32_t dd = 0; dd < 4; ++dd) {
            if (arrivals & (1u << dd)) {
              const uint32_t slot = uindex(__shfl_sync(kFull, place[dd], kChunk + o), p.n);
              land<AP, TRACKED>(slot, dd, it, is, pt[k], ps[k]);
            }
          }
        }
        uint32_t ct[AP];
        uint64_t cs[AP];
        if (dep.two) replicate<AP, TRACKED, false, true, true>(p, dep, isl[k], G, w, pt[k], ps[k],
                                                               ct, cs);
        else replicate<AP, TRACKED>(p, dep, isl[k], G, w, pt[k], ps[k], ct, cs);
#pragma unroll
        for (int a = 0; a < AP; ++a) {
          pt[k][a] = ct[a];
          ps[k][a] = cs[a];
        }
      }
      if (failed) break;
    }
  }
  if (failed || wfail) return;
#pragma unroll
  for (int k = 0; k < IPW; ++k) {
#pragma unroll
    for (int a = 0; a < AP; ++a) {
      const uint32_t j = lane + 32u * a;
      if (isl[k] < p.islands && j < p.n) {
        tplane[(size_t)isl[k] * p.n + j] = pt[k][a];
        if constexpr (TRACKED) splane[(size_t)isl[k] * p.n + j] = ps[k][a];
      }
    }
  }
}

// ------------------------------------------------------------- launch ---
using ResidentFn = void (*)(RunParams, uint32_t, uint32_t, int, uint32_t, uint32_t *,
                            uint64_t *, uint64_t *, int *);

static ResidentFn pick(int ap, int ipw, bool tracked, int mode) {
#define HSGA_PICK_MODE(AP_, IPW_, MODE_)                                              \
  if (mode == MODE_)                                                                  \
    return tracked ? step_resident_kernel<AP_, IPW_, true, MODE_>                     \
                   : step_resident_kernel<AP_, IPW_, false, MODE_>;
#define HSGA_PICK(AP_, IPW_)                                                          \
  if (ap == AP_ && ipw == IPW_) {                                                     \
    HSGA_PICK_MODE(AP_, IPW_, kPolled)                                                \
    HSGA_PICK_MODE(AP_, IPW_, kBlockSync)                                             \
  }
  if (ipw == 1 && mode == kTiled) {
    if (ap == 1) HSGA_PICK_MODE(1, 1, kTiled)
    if (ap == 2) HSGA_PICK_MODE(2, 1, kTiled)
  }
  HSGA_PICK(1, 1)
  HSGA_PICK(1, 2)
  HSGA_PICK(1, 4)
  HSGA_PICK(2, 1)
  HSGA_PICK(2, 2)
#undef HSGA_PICK
#undef HSGA_PICK_MODE
  return nullptr;
}

// Tile shape of the kTiled exchange: the smallest tiles (4 islands, then 8,
// 16, 32) whose blocks are all resident at once, and among tiles of that
// size the fewest globally polled neighbour edges per island.  Small tiles
// spread the grid over the most SMs with the cheapest block barriers:
// measured per generation, 2x2 tiles against 4x8 tiles took 1.24 against
// 1.79 us on an 8x8-island grid, 1.40 against 1.85 on 32x64, 1.74 against
// 1.82 on 64x64 (all polled: 1.38, 2.54, 2.65).  Returns false if none fits.
static bool pick_tile(const RunParams &p, int ap, bool tracked, int sms, ResidentPlan *out) {
  ResidentFn fn = pick(ap, 1, tracked, kTiled);
  if (!fn) return false;
  for (uint32_t lw = 2; lw <= 5; ++lw) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 << lw, 0) != cudaSuccess)
      return false;
    double best = 1e30;
    for (uint32_t ltr = 0; ltr <= lw; ++ltr) {
      const uint32_t ltc = lw - ltr;
      const uint64_t tr = 1u << ltr, tc = 1u << ltc;
      const uint64_t tiles = ((p.rows + tr - 1) / tr) * ((p.cols + tc - 1) / tc);
      if (per_sm < 1 || tiles > (uint64_t)per_sm * sms) continue;
      // edges that leave a tile: N and S unless the tile spans every row,
      // E and W unless it spans every column
      const double ext = (p.rows > tr ? 2.0 * tc : 0.0) + (p.cols > tc ? 2.0 * tr : 0.0);
      const double cost = ext / (double)(tr * tc);
      if (cost < best - 1e-12) {
        best = cost;
        out->blocks = (int)tiles;
        out->warps_per_block = 1 << lw;
        out->tile = ltr | (ltc << 8);
      }
    }
    if (best < 1e30) return true;
  }
  return false;
}

bool resident_plan(const RunParams &p, ResidentPlan *out, bool grid_only) {
  int dev = 0, sms = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  const int ap = p.n <= 32 ? 1 : 2;
  const bool tracked = p.policy != HSGA_NONE;
  const int ipws[3] = {1, 2, 4};
  // small grids: one thread block, shared-memory records, block barriers
  for (int ipw : ipws) {
    if (grid_only) break;
    ResidentFn fn = pick(ap, ipw, tracked, kBlockSync);
    if (!fn) continue;
    const uint64_t warps = ((uint64_t)p.islands + ipw - 1) / ipw;
    if (warps > 32) continue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)warps * 32, 0) !=
        cudaSuccess)
      return false;
    if (per_sm >= 1) {
      out->ap = ap;
      out->ipw = ipw;
      out->blocks = 1;
      out->warps_per_block = (int)warps;
      out->mode = kBlockSync;
      out->tile = 0;
      return true;
    }
  }
  if (!coop) return false;
  if (kResidentTiles) {
    ResidentPlan t;
    if (pick_tile(p, ap, tracked, sms, &t)) {
      out->ap = ap;
      out->ipw = 1;
      out->blocks = t.blocks;
      out->warps_per_block = t.warps_per_block;
      out->mode = kTiled;
      out->tile = t.tile;
      return true;
    }
  }
  const int wpb = kResidentThreads / 32;
  for (int ipw : ipws) {
    ResidentFn fn = pick(ap, ipw, tracked, kPolled);
    if (!fn) continue;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kResidentThreads, 0) !=
        cudaSuccess)
      return false;
    const uint64_t warps = ((uint64_t)p.islands + ipw - 1) / ipw;
    const uint64_t blocks = (warps + wpb - 1) / wpb;
    if (per_sm > 0 && blocks <= (uint64_t)per_sm * sms) {
      out->ap = ap;
      out->ipw = ipw;
      out->blocks = (int)blocks;
      out->warps_per_block = wpb;
      out->mode = kPolled;
      out->tile = 0;
      return true;
    }
  }
  return false;
}

cudaError_t launch_step_resident(const RunParams &p, const ResidentPlan &plan, uint32_t G0,
                                 uint32_t ngen, bool premigrated, uint32_t *t, uint64_t *s,
                                 uint64_t *rec, int *err, cudaStream_t stream) {
  ResidentFn fn = pick(plan.ap, plan.ipw, p.policy != HSGA_NONE, plan.mode);
  if (!fn) return cudaErrorInvalidValue;
  RunParams pp = p;
  int prem = premigrated ? 1 : 0;
  uint32_t tile = plan.tile;
  if (plan.mode == kBlockSync) {
    fn<<<1, plan.warps_per_block * 32, 0, stream>>>(pp, G0, ngen, prem, tile, t, s, rec, err);
    return cudaGetLastError();
  }
  void *args[] = {&pp, &G0, &ngen, &prem, &tile, &t, &s, &rec, &err};
  return cudaLaunchCooperativeKernel((const void *)fn, dim3(plan.blocks),
                                     dim3(plan.warps_per_block * 32), args, 0, stream);
}

cudaError_t launch_wait_probe(const uint64_t *record, uint32_t seq, uint64_t limit_ns, int *err,
                              uint64_t *out, cudaStream_t stream) {
  wait_probe_kernel<<<1, 32, 0, stream>>>(record, seq, limit_ns, err, out);
  return cudaGetLastError();
}

}  // namespace hsga
