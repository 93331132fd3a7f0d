// hsga_device.cuh -- device primitives of the island-model GA hot path
// (arXiv 2404.10861): Philox4x32-10, uniform indices, surface site
// functions, torus neighbours and the per-launch parameter block.
#pragma once

#include <stdint.h>

#include "hsga.h"

namespace hsga {

// ---------------------------------------------------------------- RNG ---
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies whose high halves are xor'd into the other two words
// with the round key; the key advances by the Weyl constants each round.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Counter purposes (word 3) and reserved slot values (word 0).
constexpr uint32_t kPurposeMigration = 0;  // with kSlot* in word 0
constexpr uint32_t kPurposeReplicate = 1;  // first tournament block
constexpr uint32_t kPurposeSampleDraw = 3; // with island word 0xFFFFFFFF
constexpr uint32_t kPurposeGauss = 256;    // float fitness: mutation amount
constexpr uint32_t kSlotEmigrant = 0xFFFFFFFFu;
constexpr uint32_t kSlotImmigrant = 0xFFFFFFFEu;
constexpr uint32_t kSlotSample = 0xFFFFFFFDu;

struct Words4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ Words4 philox(uint32_t k0, uint32_t k1, uint32_t c0,
                                                  uint32_t c1, uint32_t c2, uint32_t c3) {
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
#else
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c0, p1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return Words4{c0, c1, c2, c3};
}

// floor(w * m / 2^32): uniform index in [0, m) from one word.
__host__ __device__ __forceinline__ uint32_t uindex(uint32_t w, uint32_t m) {
#ifdef __CUDA_ARCH__
  return __umulhi(w, m);
#else
  return (uint32_t)(((uint64_t)w * m) >> 32);
#endif
}

// ------------------------------------------------------------ surface ---
__host__ __device__ __forceinline__ uint32_t bitlen64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return 64u - (uint32_t)__clzll((long long)x);
#else
  return x ? 64u - (uint32_t)__builtin_clzll(x) : 0u;
#endif
}

__host__ __device__ __forceinline__ uint32_t ctz64(uint64_t x) {  // x > 0
#ifdef __CUDA_ARCH__
  return (uint32_t)__ffsll((long long)x) - 1u;
#else
  return (uint32_t)__builtin_ctzll(x);
#endif
}

// Site of deposition T; S = discard.  See hsga.h for the readings.
__host__ __device__ __forceinline__ uint32_t site_of(uint32_t policy, uint32_t S, uint32_t W,
                                                     uint64_t T) {
  if (policy == HSGA_HYBRID) {  // its steady half (sites [0, S/2))
    S >>= 1;
    policy = HSGA_STEADY;
    const uint64_t t1 = T + 1;
    const uint32_t s = bitlen64(S) - 1;
    const uint32_t e = (t1 <= S) ? 0u : bitlen64(T) - s;
    if (ctz64(t1) < e) return 2 * S;
    return (uint32_t)(t1 % ((uint64_t)S + 1)) - 1u;
  }
  const uint64_t t1 = T + 1;
  switch (policy) {
    case HSGA_TRIVIAL:
      return (uint32_t)(T & (S - 1));
    case HSGA_STEADY: {
      const uint32_t s = bitlen64(S) - 1;
      const uint32_t e = (t1 <= S) ? 0u : bitlen64(T) - s;
      if (ctz64(t1) < e) return S;
      return (uint32_t)(t1 % ((uint64_t)S + 1)) - 1u;
    }
    case HSGA_TILTED:
    case HSGA_STRETCHED: {
      const uint32_t L = S / W;
      const uint32_t h = ctz64(t1);
      uint32_t level;
      uint64_t j;
      if (h < L - 1) {
        level = h;
        j = t1 >> (h + 1);
      } else {
        level = L - 1;
        j = (t1 >> (L - 1)) - 1;
      }
      if (policy == HSGA_TILTED) return level * W + (uint32_t)(j & (W - 1));
      return j < W ? level * W + (uint32_t)j : S;
    }
    default:
      return S;
  }
}

// ------------------------------------------------------------- params ---
// Unsigned division by a run-invariant divisor with one multiply-high
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, section 4): for 1 <= d < 2^32 with
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, the quotient of any
// 32-bit n is (t + ((n - t) >> min(l,1))) >> max(l-1,0), t = mulhi(m, n).
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ uint32_t fastdiv(const FastDiv &f, uint32_t n) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(f.m, n);
#else
  const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// Everything a generation kernel needs that is fixed for a run.
struct RunParams {
  uint32_t rows, cols, n, islands;
  uint32_t tournament;
  uint32_t k0, k1;         // Philox key = seed
  uint32_t policy, S, W, bits;
  uint32_t interval;
  uint32_t coarsen;        // annotate every coarsen-th generation (>= 1)
  // a5 thresholds floor(p 2^32) in [0, 2^32]: w2 < thr is (w2 < thr32) || thr_all
  uint32_t ben32, ben_all;  // beneficial: w2 < floor(p_ben 2^32)
  uint32_t bd32, bd_all;    // deleterious: otherwise w2 < floor(p_ben 2^32) + floor(p_del 2^32)
  uint32_t has_del;         // floor(p_del 2^32) > 0
  uint64_t vmask;          // (1 << bits) - 1
  uint32_t words;          // surface width K in 64-bit words (S = 64 K / bits)
  uint32_t levels, levels_half;  // S / W and (S / 2) / W (tilted, stretched, hybrid half)
  uint32_t flt;            // binary32 fitness with Gaussian mutation amounts
  float gscale;            // float(sigma / sqrt(24 + 1/12) / 2^24)
  FastDiv cols_div;        // island -> (row, column)
  uint32_t rk0[10], rk1[10];  // Philox round keys k + r * (W0, W1)
};

inline void set_round_keys(RunParams &p) {
  uint32_t a = p.k0, b = p.k1;
  for (int r = 0; r < 10; ++r) {
    p.rk0[r] = a;
    p.rk1[r] = b;
    a += kPhiloxW0;
    b += kPhiloxW1;
  }
}

// Philox4x32-10 with the run's precomputed round keys (same values as
// philox(p.k0, p.k1, ...)); the keys stay in the kernel's parameter space.
__device__ __forceinline__ Words4 philox_rk(const RunParams &p, uint32_t c0, uint32_t c1,
                                            uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)c0 * kPhiloxM0;  // one 32x32->64 multiply each
    const uint64_t p1 = (uint64_t)c2 * kPhiloxM1;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ p.rk0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ p.rk1[r];
    c0 = n0;
    c1 = (uint32_t)p1;
    c2 = n2;
    c3 = (uint32_t)p0;
  }
  return Words4{c0, c1, c2, c3};
}

// Per-generation deposit parameters: a whole synchronous generation shares
// T, hence the site.  A b-bit field never straddles the two 32-bit halves
// of the surface (b divides 32), so each insert is one bit-select per half:
// half = (half & clear) | ((value << shift) & ~clear), with clear = all ones
// for a half not written (or a discarded deposition).  The hybrid policy has
// a second field (its tilted half) whose value is bits 16.. of w3.
struct Deposit {
  uint32_t clear_lo, clear_hi, shift;     // first field
  uint32_t two;                           // a second field is written
  uint32_t clear2_lo, clear2_hi, shift2;  // second field
};

// Packed form: bits 0-5 bit offset of the first field, bit 6 "first field
// written", bits 8-13 / 14 the same for the second field.
constexpr uint32_t kPackOn = 0x40u;

__host__ __device__ __forceinline__ uint32_t deposit_pack(const RunParams &p, uint64_t G) {
  if (p.policy == HSGA_NONE) return 0u;
  const uint32_t k = p.coarsen;
  if (k > 1 && (G % k) != 0) return 0u;
  const uint64_t T = k > 1 ? G / k : G;
  uint32_t pack = 0u;
  const uint32_t a = site_of(p.policy, p.S, p.W, T);
  if (a < p.S) pack |= (a * p.bits) | kPackOn;
  if (p.policy == HSGA_HYBRID) {
    const uint32_t half = p.S / 2;
    const uint32_t b = site_of(HSGA_TILTED, half, p.W, T);
    if (b < half) pack |= (((half + b) * p.bits) | kPackOn) << 8;
  }
  return pack;
}

__host__ __device__ __forceinline__ Deposit deposit_unpack(uint32_t pack, uint32_t vmask) {
  Deposit d;
  const uint32_t bit = pack & 63u, bit2 = (pack >> 8) & 63u;
  const uint32_t field = (pack & kPackOn) ? (vmask << (bit & 31u)) : 0u;
  const uint32_t field2 = ((pack >> 8) & kPackOn) ? (vmask << (bit2 & 31u)) : 0u;
  d.shift = bit & 31u;
  d.clear_lo = (bit >> 5) ? 0xFFFFFFFFu : ~field;
  d.clear_hi = (bit >> 5) ? ~field : 0xFFFFFFFFu;
  d.two = field2 != 0u;
  d.shift2 = bit2 & 31u;
  d.clear2_lo = (bit2 >> 5) ? 0xFFFFFFFFu : ~field2;
  d.clear2_hi = (bit2 >> 5) ? ~field2 : 0xFFFFFFFFu;
  return d;
}

__host__ __device__ __forceinline__ Deposit deposit_for(const RunParams &p, uint64_t G) {
  return deposit_unpack(deposit_pack(p, G), (uint32_t)p.vmask);
}

// TWO: the caller has checked that a second field is written (the check is
// hoisted out of the per-agent code).
template <bool TWO>
__device__ __forceinline__ uint64_t deposit_into(const Deposit &d, uint64_t s, uint32_t w3) {
  const uint32_t v = w3 << d.shift;
  uint32_t lo = ((uint32_t)s & d.clear_lo) | (v & ~d.clear_lo);
  uint32_t hi = ((uint32_t)(s >> 32) & d.clear_hi) | (v & ~d.clear_hi);
  if constexpr (TWO) {
    const uint32_t v2 = (w3 >> 16) << d.shift2;
    lo = (lo & d.clear2_lo) | (v2 & ~d.clear2_lo);
    hi = (hi & d.clear2_hi) | (v2 & ~d.clear2_hi);
  }
  return ((uint64_t)hi << 32) | lo;
}

// Philox with counter words 0, 2 and 3 fixed (the child slot per lane, the
// generation and the purpose per launch): round 1's two products and three
// of its four outputs do not depend on word 1 (the island), so they are
// computed once and each island costs one xor plus rounds 2-10.
struct PhiloxHead {
  uint32_t x0;   // high(M1 c2) ^ round-1 key 0 (xored with the island later)
  uint32_t c1;   // low(M1 c2)
  uint32_t c2;   // high(M0 c0) ^ c3 ^ round-1 key 1
  uint32_t c3;   // low(M0 c0)
};

__device__ __forceinline__ PhiloxHead philox_head(uint32_t k0, uint32_t k1, uint32_t c0,
                                                  uint32_t c2, uint32_t c3) {
  const uint64_t p0 = (uint64_t)c0 * kPhiloxM0;
  const uint64_t p1 = (uint64_t)c2 * kPhiloxM1;
  return PhiloxHead{(uint32_t)(p1 >> 32) ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c3 ^ k1,
                    (uint32_t)p0};
}

// Rounds 2-10 after a precomputed head; RK as below.
template <bool RK>
__device__ __forceinline__ Words4 philox_tail(const RunParams &p, const PhiloxHead &h,
                                              uint32_t c1_in) {
  uint32_t c0 = h.x0 ^ c1_in, c1 = h.c1, c2 = h.c2, c3 = h.c3;
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    const uint32_t k0 = RK ? p.rk0[r] : p.k0 + (uint32_t)r * kPhiloxW0;
    const uint32_t k1 = RK ? p.rk1[r] : p.k1 + (uint32_t)r * kPhiloxW1;
    const uint64_t p0 = (uint64_t)c0 * kPhiloxM0;
    const uint64_t p1 = (uint64_t)c2 * kPhiloxM1;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c0 = n0;
    c1 = (uint32_t)p1;
    c2 = n2;
    c3 = (uint32_t)p0;
  }
  return Words4{c0, c1, c2, c3};
}

// RK: the run's round keys are precomputed in the parameter block (single-run
// kernels); otherwise they are derived from the key in registers.
template <bool RK>
__device__ __forceinline__ Words4 philox_p(const RunParams &p, uint32_t c0, uint32_t c1,
                                           uint32_t c2, uint32_t c3) {
  if constexpr (RK) return philox_rk(p, c0, c1, c2, c3);
  else return philox(p.k0, p.k1, c0, c1, c2, c3);
}

// Neighbour of island `isl` in direction d (0 N, 1 E, 2 S, 3 W).
__host__ __device__ __forceinline__ uint32_t neighbour(const RunParams &p, uint32_t isl,
                                                       uint32_t d) {
  uint32_t r = fastdiv(p.cols_div, isl), c = isl - r * p.cols;
  if (d == 0) r = (r == 0) ? p.rows - 1 : r - 1;
  else if (d == 2) r = (r + 1 == p.rows) ? 0 : r + 1;
  else if (d == 1) c = (c + 1 == p.cols) ? 0 : c + 1;
  else c = (c == 0) ? p.cols - 1 : c - 1;
  return r * p.cols + c;
}

__host__ __device__ __forceinline__ bool migrates(const RunParams &p, uint64_t G) {
  return p.interval != 0 && (G % p.interval) == 0;
}

// a5: saturating +1 / -1 from the mutation word (thresholds are ordered,
// floor(p_ben 2^32) <= floor(p_ben 2^32) + floor(p_del 2^32)).  DEL = false:
// the caller has checked that p_del is 0 (no deleterious branch).
template <bool DEL = true>
__device__ __forceinline__ uint32_t mutate(const RunParams &p, uint32_t trait, uint32_t w2) {
  const uint32_t ben = (uint32_t)(w2 < p.ben32) | p.ben_all;
  const uint32_t inc = ben & (uint32_t)(trait != 0xFFFFFFFFu);
  if constexpr (!DEL) return trait + inc;
  const uint32_t bd = (uint32_t)(w2 < p.bd32) | p.bd_all;
  const uint32_t dec = bd & (ben ^ 1u) & (uint32_t)(trait != 0u);
  return trait + inc - dec;
}

// Site of deposition T for one genome's own 32-bit counter (free-running
// modes, T + 1 < 2^32): the functions of site_of in 32-bit arithmetic, with
// the level counts precomputed; the steady policy defers to site_of.
__device__ __forceinline__ uint32_t level_site32(bool tilted, uint32_t t1, uint32_t L, uint32_t W,
                                                 uint32_t S) {
  const uint32_t h = (uint32_t)__ffs((int)t1) - 1u;  // t1 > 0
  uint32_t level, j;
  // t1 >> k for k up to 63 (0 from 32 on): a clamped funnel shift
  if (h + 1u < L) {
    level = h;
    j = __funnelshift_rc(t1, 0u, h + 1u);
  } else {
    level = L - 1u;
    j = __funnelshift_rc(t1, 0u, L - 1u) - 1u;
  }
  if (tilted) return level * W + (j & (W - 1u));
  return j < W ? level * W + j : S;
}

__device__ __forceinline__ uint32_t site_of32(const RunParams &p, uint32_t T) {
  if (p.policy == HSGA_TILTED || p.policy == HSGA_STRETCHED)
    return level_site32(p.policy == HSGA_TILTED, T + 1u, p.levels, p.W, p.S);
  return site_of(p.policy, p.S, p.W, T);
}

// Writes the b-bit differentia v into site `site` (< S) of a 64-bit surface.
__device__ __forceinline__ uint64_t put_site(uint64_t s, uint32_t site, uint32_t bits,
                                             uint64_t vmask, uint32_t v) {
  // b divides 32, so the field lies within one 32-bit half of the surface
  const uint32_t at = site * bits;
  const uint32_t sh = at & 31u;
  const uint32_t m = (uint32_t)vmask << sh;
  const uint32_t val = (v << sh) & m;
  uint32_t lo = (uint32_t)s, hi = (uint32_t)(s >> 32);
  if (at & 32u) hi = (hi & ~m) | val;
  else lo = (lo & ~m) | val;
  return ((uint64_t)hi << 32) | lo;
}

// a6 for one genome with its own counter T: the site(s) of deposition T
// (T / k when the coarsening interval k divides T, none otherwise), written
// with word 3 of the child's block (bits 16.. for the hybrid tilted half).
template <bool TWO>
__device__ __forceinline__ uint64_t deposit_lane(const RunParams &p, uint32_t T, uint64_t s,
                                                 uint32_t w3) {
  if (p.coarsen > 1) {
    if (T % p.coarsen) return s;
    T /= p.coarsen;
  }
  const uint32_t a = site_of32(p, T);
  if (a < p.S) s = put_site(s, a, p.bits, p.vmask, w3);
  if constexpr (TWO) {
    const uint32_t half = p.S >> 1;
    const uint32_t b = level_site32(true, T + 1u, p.levels_half, p.W, half);
    if (b < half) s = put_site(s, half + b, p.bits, p.vmask, w3 >> 16);
  }
  return s;
}

// Float fitness (hsga.h, HSGA_FITNESS_FLOAT): a later candidate wins only if
// strictly fitter as a binary32 value.
template <bool FLT>
__device__ __forceinline__ bool fitter(uint32_t a, uint32_t b) {
  if constexpr (FLT) return __uint_as_float(a) > __uint_as_float(b);
  return a > b;
}

// Sign-restricted Gaussian mutation of a binary32 fitness: the amount is
// |float(g) * gscale| with g = (B - 48) 2^24 + (q3 >> 8) - 2^23, B the
// popcount of q0..q2 (Binomial(96, 1/2)) and (q0..q3) = Philox(key; j, island,
// G, kPurposeGauss): the de Moivre-Laplace approximation to a normal of
// variance 24 + 1/12, smoothed by a 24-bit uniform.  The round-to-nearest
// intrinsics keep every float step a single correctly rounded operation.
__device__ __forceinline__ uint32_t mutate_float(const RunParams &p, uint32_t trait,
                                                 uint32_t w2, uint32_t j, uint32_t isl,
                                                 uint32_t G) {
  const bool ben = (w2 < p.ben32) || p.ben_all;
  const bool del = !ben && ((w2 < p.bd32) || p.bd_all);
  if (!ben && !del) return trait;
  const Words4 q = philox_rk(p, j, isl, G, kPurposeGauss);
  const int B = __popc(q.x) + __popc(q.y) + __popc(q.z);
  const int g = (B - 48) * (1 << 24) + (int)(q.w >> 8) - (1 << 23);
  const float amount = fabsf(__fmul_rn(__int2float_rn(g), p.gscale));
  const float f = __uint_as_float(trait);
  return __float_as_uint(ben ? __fadd_rn(f, amount) : __fsub_rn(f, amount));
}

// Device error word values (first error wins).
constexpr int kDevErrWaitTimeout = 1;
constexpr int kDevErrState = 2;

}  // namespace hsga
