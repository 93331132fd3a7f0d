// hsga_kernels.cu -- streamed generation kernel, explicit migration,
// end-state sampling and the site-function kernel.
//
// Streamed kernel: one launch advances one synchronous generation of the
// whole grid; the population ping-pongs between two structure-of-arrays
// planes in HBM (uint32 traits, uint64 surfaces: 12 bytes per agent,
// coalesced 128 B / 256 B per island).  The kernel boundary is the
// generation barrier.  Migration needs no exchange buffer: the receiver
// recomputes each neighbour's emigrant choice from the counter-based RNG and
// gathers that genome straight from the neighbour's parent plane.
#include <cuda_runtime.h>

#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {

// ------------------------------------------------------ streamed step ---
// The group helpers (migration draws, landing plans, island loads/stores)
// live in hsga_island.cuh.
// Islands whose Philox chains the streamed kernel interleaves: the whole
// group (measured at 16.8M agents: 85.9 us per generation against 86.3 with
// two at a time; 80 registers, 8 bytes spilled).  The batch kernel, which
// derives the round keys in registers, keeps two.
constexpr int kStreamInterleave = kGroup;

// MIG: whether this generation migrates (a compile-time flag, so that the
// full groups carry no run-time branch around the migration draws).
template <int AP, bool TRACKED, bool T2, int NN, bool MIG>
__global__ void __launch_bounds__(kStreamThreads, AP == 1 ? kStreamBlocksPerSM : 1)
    step_streamed_kernel(RunParams p, Deposit dep, uint32_t G,
                         const uint32_t *__restrict__ tin, const uint64_t *__restrict__ sin,
                         uint32_t *__restrict__ tout, uint64_t *__restrict__ sout) {
  constexpr int M = MIG ? 1 : 0;
  constexpr int IL = kStreamInterleave;
  const uint32_t wpb = blockDim.x >> 5;
  const uint32_t nwarps = gridDim.x * wpb;
  const uint32_t ngroups = (p.islands + kGroup - 1) / kGroup;
  PhiloxHead head[AP];
  replication_heads<AP>(p, G, head);
  for (uint32_t grp = blockIdx.x * wpb + (threadIdx.x >> 5); grp < ngroups; grp += nwarps) {
    const uint32_t isl0 = grp * kGroup;
    if (isl0 + kGroup <= p.islands) {
      if (dep.two)
        full_group<AP, TRACKED, T2, NN, IL, true, true, true, M>(
            p, dep, G, MIG, isl0, tin, sin, tout, sout, head);
      else if (p.has_del)
        full_group<AP, TRACKED, T2, NN, IL, true, false, true, M>(
            p, dep, G, MIG, isl0, tin, sin, tout, sout, head);
      else
        full_group<AP, TRACKED, T2, NN, IL, true, false, false, M>(
            p, dep, G, MIG, isl0, tin, sin, tout, sout, head);
    }
    else
      partial_group<AP, TRACKED, T2>(p, dep, G, MIG, isl0, tin, sin, tout, sout);
  }
}

template <int AP, bool TRACKED, bool T2, int NN, bool MIG>
static int streamed_blocks() {
  static int blocks = 0;
  if (blocks == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, step_streamed_kernel<AP, TRACKED, T2, NN, MIG>, kStreamThreads, 0);
    blocks = sms * (per_sm > 0 ? per_sm : 1);
  }
  return blocks;
}

template <int AP, bool TRACKED, bool T2, int NN>
static void launch_streamed_t(const RunParams &p, const Deposit &dep, uint32_t G, bool do_mig,
                              const uint32_t *tin, const uint64_t *sin, uint32_t *tout,
                              uint64_t *sout, cudaStream_t stream) {
  const uint32_t groups = (p.islands + kGroup - 1) / kGroup;
  const uint32_t need = (groups + kStreamThreads / 32 - 1) / (kStreamThreads / 32);
  int b = do_mig ? streamed_blocks<AP, TRACKED, T2, NN, true>()
                 : streamed_blocks<AP, TRACKED, T2, NN, false>();
  if ((uint32_t)b > need) b = (int)need;
  if (do_mig)
    step_streamed_kernel<AP, TRACKED, T2, NN, true>
        <<<b, kStreamThreads, 0, stream>>>(p, dep, G, tin, sin, tout, sout);
  else
    step_streamed_kernel<AP, TRACKED, T2, NN, false>
        <<<b, kStreamThreads, 0, stream>>>(p, dep, G, tin, sin, tout, sout);
}

cudaError_t launch_step_streamed(const RunParams &p, uint32_t G, bool do_mig,
                                 const uint32_t *tin, const uint64_t *sin, uint32_t *tout,
                                 uint64_t *sout, int *err, cudaStream_t stream) {
  // 32-agent islands (the paper's shape): parents staged in shared memory
  if (p.n == 32) return launch_step_staged(p, G, do_mig, tin, sin, tout, sout, err, stream);
  const Deposit dep = deposit_for(p, G);
  const bool tracked = p.policy != HSGA_NONE;
  const bool t2 = p.tournament == 2;
  (void)err;  // the register kernel has no waits
#define HSGA_LAUNCH(AP_, TR_, T2_, NN_) \
  launch_streamed_t<AP_, TR_, T2_, NN_>(p, dep, G, do_mig, tin, sin, tout, sout, stream)
#define HSGA_LAUNCH_T(AP_, NN_)                         \
  if (tracked) {                                        \
    if (t2) HSGA_LAUNCH(AP_, true, true, NN_);          \
    else HSGA_LAUNCH(AP_, true, false, NN_);            \
  } else {                                              \
    if (t2) HSGA_LAUNCH(AP_, false, true, NN_);         \
    else HSGA_LAUNCH(AP_, false, false, NN_);           \
  }
  if (p.n == 32) {
    HSGA_LAUNCH_T(1, 32)
  } else if (p.n < 32) {
    HSGA_LAUNCH_T(1, 0)
  } else {
    HSGA_LAUNCH_T(2, 0)
  }
#undef HSGA_LAUNCH_T
#undef HSGA_LAUNCH
  return cudaGetLastError();
}

// --------------------------------------------------- explicit a1 + a2 ---
// Emigrants are written to per-island 16-byte records (one 128-bit store:
// trait, surface low, surface high, direction) before any immigrant lands;
// a second launch lands them in place.
__global__ void emigrate_kernel(RunParams p, uint32_t G, const uint32_t *__restrict__ t,
                                const uint64_t *__restrict__ s, uint4 *__restrict__ rec) {
  const uint32_t isl = blockIdx.x * blockDim.x + threadIdx.x;
  if (isl >= p.islands) return;
  const Words4 m = philox_rk(p, kSlotEmigrant, isl, G, kPurposeMigration);
  const size_t a = (size_t)isl * p.n + uindex(m.x, p.n);
  const uint64_t sv = s ? s[a] : 0ull;
  rec[isl] = make_uint4(t[a], (uint32_t)sv, (uint32_t)(sv >> 32), m.y >> 30);
}

__global__ void immigrate_kernel(RunParams p, uint32_t G, uint32_t *__restrict__ t,
                                 uint64_t *__restrict__ s, const uint4 *__restrict__ rec) {
  const uint32_t isl = blockIdx.x * blockDim.x + threadIdx.x;
  if (isl >= p.islands) return;
  const Words4 v = philox_rk(p, kSlotImmigrant, isl, G, kPurposeMigration);
  const uint32_t place[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (uint32_t d = 0; d < 4; ++d) {
    const uint4 r = rec[neighbour(p, isl, d)];
    if (r.w != ((d + 2u) & 3u)) continue;
    const size_t a = (size_t)isl * p.n + uindex(place[d], p.n);
    t[a] = r.x;
    if (s) s[a] = ((uint64_t)r.z << 32) | r.y;
  }
}

cudaError_t launch_migrate(const RunParams &p, uint32_t G, uint32_t *t, uint64_t *s,
                           uint4 *rec, cudaStream_t stream) {
  const uint32_t blocks = (p.islands + 255) / 256;
  emigrate_kernel<<<blocks, 256, 0, stream>>>(p, G, t, s, rec);
  immigrate_kernel<<<blocks, 256, 0, stream>>>(p, G, t, s, rec);
  return cudaGetLastError();
}

// ------------------------------------------------------------ a7 sample ---
// Partial Fisher-Yates over the islands, k draws r_j = j + floor(w_j (I-j) /
// 2^32), evaluated in parallel.  After all swaps, position j holds the value
// that position r_j held just before step j (no later step touches position
// j).  That value is r_j unless an earlier step i < j also drew r_i = r_j, in
// which case it is f(i) for the last such i, where f(i) is the value position
// i held at the start of step i: f(i) = i unless an earlier step i' < i drew
// r_i' = i, then f(i) = f(last such i').  "Last earlier step with draw p" is
// a predecessor query on the (draw, step) pairs sorted once in shared memory.
__device__ __forceinline__ int last_before(const unsigned long long *sorted, uint32_t K2,
                                           uint32_t value, uint32_t j) {
  // greatest i < j with draw value, or -1: lower_bound of (value, j) minus one
  const unsigned long long key = ((unsigned long long)value << 32) | j;
  uint32_t lo = 0, hi = K2;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (sorted[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  if (lo == 0) return -1;
  const unsigned long long prev = sorted[lo - 1];
  return (uint32_t)(prev >> 32) == value ? (int)(uint32_t)prev : -1;
}

__global__ void __launch_bounds__(1024)
    sample_smem_kernel(RunParams p, uint32_t G, uint32_t k, uint32_t K2,
                       const uint32_t *__restrict__ t, const uint64_t *__restrict__ s,
                       uint32_t *__restrict__ out_words, uint32_t *__restrict__ out_is,
                       const uint32_t *__restrict__ T) {
  extern __shared__ unsigned long long smem[];
  unsigned long long *pairs = smem;                        // K2
  uint32_t *draw = (uint32_t *)(smem + K2);                // k
  int *val = (int *)(draw + k);                            // k
  __shared__ int changed;
  const uint32_t I = p.islands;
  for (uint32_t j = threadIdx.x; j < K2; j += blockDim.x) {
    if (j < k) {
      const Words4 w = philox_rk(p, j, 0xFFFFFFFFu, G, kPurposeSampleDraw);
      const uint32_t r = j + uindex(w.x, I - j);
      draw[j] = r;
      pairs[j] = ((unsigned long long)r << 32) | j;
    } else {
      pairs[j] = ~0ull;
    }
  }
  __syncthreads();
  // bitonic sort of the (draw, step) pairs, ascending
  for (uint32_t size = 2; size <= K2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t i = threadIdx.x; i < K2 / 2; i += blockDim.x) {
        // 2 stride floor(i / stride) + i mod stride, stride a power of two
        const uint32_t lo = ((i & ~(stride - 1u)) << 1) | (i & (stride - 1u));
        const uint32_t hi = lo + stride;
        const bool up = ((lo & size) == 0);
        const unsigned long long a = pairs[lo], b = pairs[hi];
        if ((a > b) == up) {
          pairs[lo] = b;
          pairs[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  // f(i): -(link+2) marks "equal to f(link)", values >= 0 are resolved
  for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
    const int link = last_before(pairs, K2, i, i);
    val[i] = link < 0 ? (int)i : -(link + 2);
  }
  __syncthreads();
  for (uint32_t round = 0; round < k + 1; ++round) {
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
      const int v = val[i];
      if (v < 0) {  // follow one link; links point to smaller steps, so u != v
        val[i] = val[-v - 2];
        changed = 1;
      }
    }
    __syncthreads();
    if (!changed) break;
    __syncthreads();
  }
  for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
    const int last = last_before(pairs, K2, draw[j], j);
    const uint32_t island = last < 0 ? draw[j] : (uint32_t)val[last];
    const Words4 w = philox_rk(p, kSlotSample, island, G, kPurposeMigration);
    const uint32_t slot = uindex(w.x, p.n);
    const size_t a = (size_t)island * p.n + slot;
    const uint64_t sv = s ? s[a] : 0ull;
    reinterpret_cast<uint4 *>(out_words)[j] =
        make_uint4(t[a], (uint32_t)sv, (uint32_t)(sv >> 32), T ? T[a] : G);
    if (out_is) reinterpret_cast<uint2 *>(out_is)[j] = make_uint2(island, slot);
  }
}

// Large k: the shuffle itself, step by step, on a scratch permutation.
__global__ void iota_kernel(uint32_t *perm, uint32_t I) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < I; i += gridDim.x * blockDim.x)
    perm[i] = i;
}

__global__ void shuffle_serial_kernel(RunParams p, uint32_t G, uint32_t k, uint32_t *perm) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (uint32_t j = 0; j < k; ++j) {
    const Words4 w = philox_rk(p, j, 0xFFFFFFFFu, G, kPurposeSampleDraw);
    const uint32_t r = j + uindex(w.x, p.islands - j);
    const uint32_t a = perm[j], b = perm[r];
    perm[j] = b;
    perm[r] = a;
  }
}

__global__ void gather_samples_kernel(RunParams p, uint32_t G, uint32_t k, const uint32_t *perm,
                                      const uint32_t *__restrict__ t,
                                      const uint64_t *__restrict__ s, uint32_t *out_words,
                                      uint32_t *out_is, const uint32_t *__restrict__ T) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const uint32_t island = perm[j];
  const Words4 w = philox_rk(p, kSlotSample, island, G, kPurposeMigration);
  const uint32_t slot = uindex(w.x, p.n);
  const size_t a = (size_t)island * p.n + slot;
  const uint64_t sv = s ? s[a] : 0ull;
  reinterpret_cast<uint4 *>(out_words)[j] =
      make_uint4(t[a], (uint32_t)sv, (uint32_t)(sv >> 32), T ? T[a] : G);
  if (out_is) reinterpret_cast<uint2 *>(out_is)[j] = make_uint2(island, slot);
}

size_t sample_scratch_bytes(const RunParams &p, uint32_t k) {
  return k <= kSampleSmemMax ? 0 : (size_t)p.islands * sizeof(uint32_t);
}

cudaError_t launch_sample(const RunParams &p, uint32_t G, uint32_t k, const uint32_t *t,
                          const uint64_t *s, uint32_t *out_words, uint32_t *out_is,
                          uint32_t *scratch, cudaStream_t stream, const uint32_t *T) {
  if (k == 0) return cudaSuccess;
  if (k <= kSampleSmemMax) {
    uint32_t K2 = 1;
    while (K2 < k) K2 <<= 1;
    const size_t smem = (size_t)K2 * 8 + (size_t)k * 8;
    cudaError_t e = cudaFuncSetAttribute(sample_smem_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sample_smem_kernel<<<1, 1024, smem, stream>>>(p, G, k, K2, t, s, out_words, out_is, T);
    return cudaGetLastError();
  }
  iota_kernel<<<1024, 256, 0, stream>>>(scratch, p.islands);
  shuffle_serial_kernel<<<1, 32, 0, stream>>>(p, G, k, scratch);
  gather_samples_kernel<<<(k + 255) / 256, 256, 0, stream>>>(p, G, k, scratch, t, s, out_words,
                                                             out_is, T);
  return cudaGetLastError();
}

// ------------------------------------------------------------ philox ---
__global__ void philox_sweep_kernel(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t count,
                                    uint32_t c1, uint32_t c2, uint32_t c3,
                                    uint4 *__restrict__ out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += gridDim.x * blockDim.x) {
    const Words4 w = philox(k0, k1, c0 + i, c1, c2, c3);
    out[i] = make_uint4(w.x, w.y, w.z, w.w);
  }
}

cudaError_t launch_philox_sweep(uint64_t seed, uint32_t c0, uint32_t count, uint32_t c1,
                                uint32_t c2, uint32_t c3, uint32_t *out, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  uint32_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  philox_sweep_kernel<<<blocks, 256, 0, stream>>>((uint32_t)seed, (uint32_t)(seed >> 32), c0,
                                                  count, c1, c2, c3, (uint4 *)out);
  return cudaGetLastError();
}

// ---------------------------------------------------- Philox throughput ---
// Thread t draws the blocks for counters (i, t, c2, c3), i < m, in the form
// the generation kernels use (round keys in the parameter block), four
// independent chains at a time, and stores the xor of every word it drew
// (so that no draw can be optimised away).
__global__ void __launch_bounds__(256)
    philox_throughput_kernel(RunParams p, uint32_t threads, uint32_t m, uint32_t c2,
                             uint32_t c3, uint32_t *__restrict__ out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= threads) return;
  uint32_t acc = 0;
  uint32_t i = 0;
  for (; i + 4 <= m; i += 4) {
    const Words4 a = philox_rk(p, i, t, c2, c3);
    const Words4 b = philox_rk(p, i + 1, t, c2, c3);
    const Words4 c = philox_rk(p, i + 2, t, c2, c3);
    const Words4 d = philox_rk(p, i + 3, t, c2, c3);
    acc ^= (a.x ^ a.y ^ a.z ^ a.w) ^ (b.x ^ b.y ^ b.z ^ b.w) ^ (c.x ^ c.y ^ c.z ^ c.w) ^
           (d.x ^ d.y ^ d.z ^ d.w);
  }
  for (; i < m; ++i) {
    const Words4 a = philox_rk(p, i, t, c2, c3);
    acc ^= a.x ^ a.y ^ a.z ^ a.w;
  }
  out[t] = acc;
}

cudaError_t launch_philox_throughput(uint64_t seed, uint32_t threads, uint32_t m, uint32_t c2,
                                     uint32_t c3, uint32_t *out, cudaStream_t stream) {
  if (threads == 0) return cudaSuccess;
  RunParams p{};
  p.k0 = (uint32_t)seed;
  p.k1 = (uint32_t)(seed >> 32);
  set_round_keys(p);
  const uint32_t blocks = (threads + 255) / 256;
  philox_throughput_kernel<<<blocks, 256, 0, stream>>>(p, threads, m, c2, c3, out);
  return cudaGetLastError();
}

// ------------------------------------------------------- site function ---
__global__ void sites_kernel(uint32_t policy, uint32_t S, uint32_t W, uint64_t T0,
                             uint64_t count, uint32_t *out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = site_of(policy, S, W, T0 + i);
}

cudaError_t launch_sites(uint32_t policy, uint32_t S, uint32_t W, uint64_t T0, uint64_t count,
                         uint32_t *out, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (count + 255) / 256;
  const uint64_t cap = (uint64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  sites_kernel<<<(unsigned)blocks, 256, 0, stream>>>(policy, S, W, T0, count, out);
  return cudaGetLastError();
}

}  // namespace hsga
