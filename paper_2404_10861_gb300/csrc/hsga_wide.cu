// hsga_wide.cu -- synchronous generations with surfaces of 2 or 4 64-bit
// words (128- or 256-bit fields; the paper draws a 256-bit field, section
// "Surface-based Hereditary Stratigraphy Algorithms", and names more and
// wider differentiae as the remedy for reconstruction precision, "Results ›
// Clade Reconstruction Trial").
//
// Surfaces are agent-major: word w of agent a at surf[a K + w]; site s
// occupies bits [s b mod 64, s b mod 64 + b) of word floor(s b / 64).  One
// warp serves one island (lane = agent, n <= 32).  The migration step is the
// explicit a1 + a2 pair with (K + 1)-word records: trait | direction << 32,
// then the surface words.
#include <cuda_runtime.h>

#include "hsga_internal.h"
#include "hsga_island.cuh"

namespace hsga {
namespace {

template <int K>
__global__ void emigrate_wide_kernel(RunParams p, uint32_t G, const uint32_t *__restrict__ t,
                                     const uint64_t *__restrict__ s,
                                     uint64_t *__restrict__ rec) {
  const uint32_t isl = blockIdx.x * blockDim.x + threadIdx.x;
  if (isl >= p.islands) return;
  const Words4 m = philox_rk(p, kSlotEmigrant, isl, G, kPurposeMigration);
  const size_t a = (size_t)isl * p.n + uindex(m.x, p.n);
  uint64_t *r = rec + (size_t)isl * (K + 1);
  r[0] = (uint64_t)t[a] | ((uint64_t)(m.y >> 30) << 32);
#pragma unroll
  for (int w = 0; w < K; ++w) r[1 + w] = s[a * K + w];
}

template <int K>
__global__ void immigrate_wide_kernel(RunParams p, uint32_t G, uint32_t *__restrict__ t,
                                      uint64_t *__restrict__ s,
                                      const uint64_t *__restrict__ rec) {
  const uint32_t isl = blockIdx.x * blockDim.x + threadIdx.x;
  if (isl >= p.islands) return;
  const Words4 v = philox_rk(p, kSlotImmigrant, isl, G, kPurposeMigration);
  const uint32_t place[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (uint32_t d = 0; d < 4; ++d) {
    const uint64_t *r = rec + (size_t)neighbour(p, isl, d) * (K + 1);
    if ((uint32_t)(r[0] >> 32) != ((d + 2u) & 3u)) continue;
    const size_t a = (size_t)isl * p.n + uindex(place[d], p.n);
    t[a] = (uint32_t)r[0];
#pragma unroll
    for (int w = 0; w < K; ++w) s[a * K + w] = r[1 + w];
  }
}

// Writes the b-bit value into the field at (word, shift) of a K-word
// surface held in registers (word < 0: nothing to write).
template <int K>
__device__ __forceinline__ void put_field(uint64_t (&s)[K], int word, uint32_t shift,
                                          uint64_t vmask, uint32_t value) {
#pragma unroll
  for (int w = 0; w < K; ++w)
    if (w == word) s[w] = (s[w] & ~(vmask << shift)) | (((uint64_t)value & vmask) << shift);
}

// a3-a6 of one island per warp; every child of generation G deposits at the
// same field(s) (T = G, or G / k under temporal coarsening).
template <int K, bool FLT, bool TWO>
__global__ void __launch_bounds__(kResidentThreads)
    step_wide_kernel(RunParams p, WideDeposit dep, uint32_t G, const uint32_t *__restrict__ tin,
                     const uint64_t *__restrict__ sin, uint32_t *__restrict__ tout,
                     uint64_t *__restrict__ sout) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t isl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (isl >= p.islands) return;
  const uint32_t n = p.n;
  uint32_t t = 0;
  uint64_t s[K];
#pragma unroll
  for (int w = 0; w < K; ++w) s[w] = 0;
  if (lane < n) {
    const size_t a = (size_t)isl * n + lane;
    t = tin[a];
#pragma unroll
    for (int w = 0; w < K; ++w) s[w] = sin[a * K + w];
  }
  const Words4 w4 = philox_rk(p, lane, isl, G, kPurposeReplicate);
  uint32_t best = uindex(w4.x, n);
  uint32_t fbest = __shfl_sync(kFull, t, best);
  if (p.tournament >= 2) {
    const uint32_t c = uindex(w4.y, n);
    const uint32_t fc = __shfl_sync(kFull, t, c);
    if (fitter<FLT>(fc, fbest)) {
      best = c;
      fbest = fc;
    }
  }
  for (uint32_t c0 = 2; c0 < p.tournament; c0 += 4) {
    const Words4 e = philox_rk(p, lane, isl, G, kPurposeReplicate + 1 + (c0 - 2) / 4);
    const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (c0 + q < p.tournament) {
        const uint32_t c = uindex(ew[q], n);
        const uint32_t fc = __shfl_sync(kFull, t, c);
        if (fitter<FLT>(fc, fbest)) {
          best = c;
          fbest = fc;
        }
      }
    }
  }
  uint32_t child_t;
  if constexpr (FLT)
    child_t = mutate_float(p, fbest, w4.z, lane, isl, G);
  else
    child_t = mutate(p, fbest, w4.z);
  uint64_t cs[K];
#pragma unroll
  for (int w = 0; w < K; ++w) cs[w] = shfl64(s[w], best);
  put_field<K>(cs, dep.word1, dep.shift1, p.vmask, w4.w);
  if constexpr (TWO) put_field<K>(cs, dep.word2, dep.shift2, p.vmask, w4.w >> 16);
  if (lane < n) {
    const size_t a = (size_t)isl * n + lane;
    tout[a] = child_t;
#pragma unroll
    for (int w = 0; w < K; ++w) sout[a * K + w] = cs[w];
  }
}

// Sample records of 2 + 2K words (trait, surface words as (low, high)
// pairs, T = G) from (island, slot) pairs.
__global__ void gather_wide_kernel(uint32_t k, uint32_t n, uint32_t K, uint32_t G,
                                   const uint32_t *__restrict__ t,
                                   const uint64_t *__restrict__ s,
                                   const uint32_t *__restrict__ where,
                                   uint32_t *__restrict__ out) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const size_t a = (size_t)where[2 * j] * n + where[2 * j + 1];
  uint32_t *o = out + (size_t)j * (2 + 2 * K);
  o[0] = t[a];
  for (uint32_t w = 0; w < K; ++w) {
    o[1 + 2 * w] = (uint32_t)s[a * K + w];
    o[2 + 2 * w] = (uint32_t)(s[a * K + w] >> 32);
  }
  o[1 + 2 * K] = G;
}

template <int K>
void launch_migrate_wide_t(const RunParams &p, uint32_t G, uint32_t *t, uint64_t *s,
                           uint64_t *rec, cudaStream_t stream) {
  const uint32_t blocks = (p.islands + 255) / 256;
  emigrate_wide_kernel<K><<<blocks, 256, 0, stream>>>(p, G, t, s, rec);
  immigrate_wide_kernel<K><<<blocks, 256, 0, stream>>>(p, G, t, s, rec);
}

template <int K, bool FLT>
void launch_step_wide_t(const RunParams &p, const WideDeposit &dep, uint32_t G,
                        const uint32_t *tin, const uint64_t *sin, uint32_t *tout,
                        uint64_t *sout, cudaStream_t stream) {
  const uint32_t wpb = kResidentThreads / 32;
  const uint32_t blocks = (p.islands + wpb - 1) / wpb;
  if (p.policy == HSGA_HYBRID)
    step_wide_kernel<K, FLT, true>
        <<<blocks, kResidentThreads, 0, stream>>>(p, dep, G, tin, sin, tout, sout);
  else
    step_wide_kernel<K, FLT, false>
        <<<blocks, kResidentThreads, 0, stream>>>(p, dep, G, tin, sin, tout, sout);
}

}  // namespace

WideDeposit wide_deposit_for(const RunParams &p, uint64_t G) {
  WideDeposit d{-1, 0, -1, 0};
  const uint32_t k = p.coarsen;
  if (k > 1 && (G % k) != 0) return d;
  const uint64_t T = k > 1 ? G / k : G;
  const uint32_t a = site_of(p.policy, p.S, p.W, T);
  if (a < p.S) {
    d.word1 = (int)(a * p.bits / 64);
    d.shift1 = a * p.bits % 64;
  }
  if (p.policy == HSGA_HYBRID) {
    const uint32_t half = p.S / 2;
    const uint32_t b = site_of(HSGA_TILTED, half, p.W, T);
    if (b < half) {
      d.word2 = (int)((half + b) * p.bits / 64);
      d.shift2 = (half + b) * p.bits % 64;
    }
  }
  return d;
}

cudaError_t launch_migrate_wide(const RunParams &p, uint32_t G, uint32_t *t, uint64_t *s,
                                uint64_t *rec, cudaStream_t stream) {
  if (p.words == 2)
    launch_migrate_wide_t<2>(p, G, t, s, rec, stream);
  else
    launch_migrate_wide_t<4>(p, G, t, s, rec, stream);
  return cudaGetLastError();
}

cudaError_t launch_step_wide(const RunParams &p, uint32_t G, const uint32_t *tin,
                             const uint64_t *sin, uint32_t *tout, uint64_t *sout,
                             cudaStream_t stream) {
  const WideDeposit dep = wide_deposit_for(p, G);
  if (p.words == 2)
    p.flt ? launch_step_wide_t<2, true>(p, dep, G, tin, sin, tout, sout, stream)
          : launch_step_wide_t<2, false>(p, dep, G, tin, sin, tout, sout, stream);
  else
    p.flt ? launch_step_wide_t<4, true>(p, dep, G, tin, sin, tout, sout, stream)
          : launch_step_wide_t<4, false>(p, dep, G, tin, sin, tout, sout, stream);
  return cudaGetLastError();
}

cudaError_t launch_gather_wide(const RunParams &p, uint32_t G, uint32_t k, const uint32_t *t,
                               const uint64_t *s, const uint32_t *where, uint32_t *out,
                               cudaStream_t stream) {
  gather_wide_kernel<<<(k + 255) / 256, 256, 0, stream>>>(k, p.n, p.words, G, t, s, where, out);
  return cudaGetLastError();
}

}  // namespace hsga
