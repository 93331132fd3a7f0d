/*
 * hsga_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * tracking-enabled island-model genetic algorithm of Moreno, Yang, Dolson &
 * Zaman, "Trackable Agent-based Evolution Models at Wafer Scale" (arXiv
 * 2404.10861).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load this library.  It shares
 * no source, header, table or helper with the CUDA path; neither includes the
 * other.
 *
 * What it computes, step by step, in the paper's order (section "Asynchronous
 * Island-model Genetic Algorithm"): migration first, then fitness evaluation,
 * tournament selection, mutation, and the hereditary-stratigraphy annotation
 * update.  Synchronous-migration reading, with every random number drawn from
 * a counter-based generator so that a run is a pure function of the seed:
 *
 *   a1 emigrate  : per island one emigrant slot and one direction (N,E,S,W)
 *                  from Philox(key; 0xFFFFFFFF, island, G, 0); the genome is
 *                  copied, not moved (emigration buffers are refilled with
 *                  copies of random members).
 *   a2 immigrate : for d = N,E,S,W in that order, an emigrant of the
 *                  neighbour in direction d that targets this island replaces
 *                  the member at slot floor(v_d * n / 2^32), with (v_0..v_3) =
 *                  Philox(key; 0xFFFFFFFE, island, G, 0); later arrivals
 *                  overwrite earlier ones.  All emigrants are chosen before any
 *                  immigrant lands.
 *   a3 evaluate  : fitness is the stored uint32 trait (the paper's trivial
 *                  fitness function: the genome stores its own fitness).
 *   a4 select    : child slot j draws its tournament from Philox(key; j,
 *                  island, G, 1): candidates floor(w0*n/2^32),
 *                  floor(w1*n/2^32) drawn with replacement; a later candidate
 *                  replaces the current best only if strictly fitter.
 *                  Candidates beyond the second come from purposes 2, 3, ...
 *                  four per block.
 *   a5 mutate    : w2 < floor(p_ben 2^32) -> trait + 1 (saturating);
 *                  else w2 < floor(p_ben 2^32) + floor(p_del 2^32) -> trait - 1
 *                  (saturating).
 *   a6 deposit   : site = site_fn(policy, S, W, T); unless the policy discards
 *                  this deposition, surface bits [site*b, site*b + b) take the
 *                  low b bits of w3.  T, the deposition counter, is then one
 *                  larger; in synchronous mode T equals the generation G.  With
 *                  temporal coarsening k, only generations divisible by k
 *                  deposit, as deposition G / k.  The hybrid policy writes a
 *                  second differentia (bits 16.. of w3) into its tilted half.
 *   a7 sample    : one genome per island at slot floor(w0*n/2^32) of
 *                  Philox(key; 0xFFFFFFFD, island, G, 0), then k islands
 *                  without replacement by a partial Fisher-Yates shuffle whose
 *                  j-th draw is word 0 of Philox(key; j, 0xFFFFFFFF, G, 3).
 *
 * Random numbers: Philox4x32-10 of Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11), written here from that
 * paper's definition.  The key is (seed_lo, seed_hi).  The same round and key
 * schedule is instantiated at 64-bit words (Philox4x64-10) only so that a test
 * can pin the round structure against numpy.random.Philox.
 *
 * Surface site selection: the paper leaves the indexing formulas to later
 * work (section "Surface-based Hereditary Stratigraphy Algorithms"); it fixes
 * only their properties: a fixed-size buffer written in place, implicit
 * pruning by overwrite, timestamps recoverable from (site, T) alone, "steady"
 * spreading retained time points evenly over history and "tilted" favouring
 * recent ones.  The functions below are this project's own O(1) readings of
 * those properties; the retention property tests pin them.  Parity with the
 * paper's (unpublished here) site sequences is unpinned.
 *
 * Timestamp lookup is written as its definition: the last deposition time
 * below T whose site is p, found by replaying the site function (brute force).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4xW-10 (Salmon et al. 2011, section 4): each round multiplies words
 * 0 and 2 by the round multipliers, takes the high halves xor'd with words
 * 1 and 3 and the round key, the low halves pass through; the key is bumped
 * by the Weyl constants after every round.  One macro serves both widths so
 * the 64-bit instance checks the structure of the 32-bit one. */
#define ORC_PHILOX_DEFINE(NAME, UINT, WIDE, BITS, M0, M1, W0, W1)              \
  void NAME(UINT k0, UINT k1, const UINT ctr[4], UINT out[4]) {               \
    UINT c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];                  \
    for (int round = 0; round < 10; ++round) {                                \
      WIDE p0 = (WIDE)(M0) * (WIDE)c0;                                        \
      WIDE p1 = (WIDE)(M1) * (WIDE)c2;                                        \
      UINT hi0 = (UINT)(p0 >> BITS), lo0 = (UINT)p0;                          \
      UINT hi1 = (UINT)(p1 >> BITS), lo1 = (UINT)p1;                          \
      UINT n0 = hi1 ^ c1 ^ k0;                                                \
      UINT n1 = lo1;                                                          \
      UINT n2 = hi0 ^ c3 ^ k1;                                                \
      UINT n3 = lo0;                                                          \
      c0 = n0; c1 = n1; c2 = n2; c3 = n3;                                     \
      k0 = (UINT)(k0 + (W0));                                                 \
      k1 = (UINT)(k1 + (W1));                                                 \
    }                                                                         \
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;                       \
  }

ORC_PHILOX_DEFINE(orc_philox4x32_10, uint32_t, uint64_t, 32,
                  0xD2511F53u, 0xCD9E8D57u, 0x9E3779B9u, 0xBB67AE85u)
ORC_PHILOX_DEFINE(orc_philox4x64_10, uint64_t, unsigned __int128, 64,
                  0xD2E7470EE14C6C93ull, 0xCA5A826395121157ull,
                  0x9E3779B97F4A7C15ull, 0xBB67AE8584CAA73Bull)

/* Philox4x32-10 blocks for counters (c0 + i, c1, c2, c3), i < count, key
 * (seed_lo, seed_hi): out[4 i + j] = word j (a bulk form of the generator,
 * for sweeps in tests). */
void orc_philox_sweep(uint64_t seed, uint32_t c0, uint32_t count, uint32_t c1,
                      uint32_t c2, uint32_t c3, uint32_t *out) {
  for (uint32_t i = 0; i < count; ++i) {
    uint32_t ctr[4] = {c0 + i, c1, c2, c3};
    orc_philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, out + 4 * (size_t)i);
  }
}

/* floor(w * m / 2^32): a uniform index in [0, m) from one 32-bit word. */
static uint32_t orc_index(uint32_t w, uint64_t m) {
  return (uint32_t)(((uint64_t)w * m) >> 32);
}

static void orc_draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                     uint32_t c3, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  orc_philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, out);
}

/* ------------------------------------------------------------------ */
/* Surface site selection (readings; see header). */

enum { ORC_STEADY = 0, ORC_TILTED = 1, ORC_STRETCHED = 2, ORC_TRIVIAL = 3,
       ORC_NONE = 4, ORC_HYBRID = 5 };

static unsigned orc_bitlen(uint64_t x) {
  unsigned n = 0;
  while (x) { ++n; x >>= 1; }
  return n;
}

static unsigned orc_ctz(uint64_t x) { /* x > 0 */
  unsigned n = 0;
  while (!(x & 1)) { ++n; x >>= 1; }
  return n;
}

/* Returns the site in [0, S) written by deposition number T, or S when the
 * policy discards that deposition.  S is a power of two; W divides S.  For
 * the hybrid policy this is the site of its steady half (sites [0, S/2));
 * see orc_hybrid_second_site for its tilted half. */
uint32_t orc_site(uint32_t policy, uint32_t S, uint32_t W, uint64_t T) {
  if (policy == ORC_HYBRID) {
    uint32_t a = orc_site(ORC_STEADY, S / 2, W, T);
    return a < S / 2 ? a : S;
  }
  if (policy == ORC_TRIVIAL) return (uint32_t)(T % S);
  if (policy == ORC_STEADY) {
    /* Epoch e: zero while the first S depositions fill the buffer, then
     * bitlen(T) - log2(S).  Deposition T is kept only if 2^e divides T+1;
     * writing T+1 = m*2^e (1 <= m <= S), its site is (T+1 mod S+1) - 1, a
     * bijection of m because 2 is invertible modulo the odd S+1.  Each new
     * epoch overwrites exactly the odd-m survivors of the previous one, so
     * the kept times are the multiples of 2^e: evenly spread. */
    unsigned s = orc_bitlen(S) - 1;
    unsigned e = (T + 1 <= S) ? 0 : orc_bitlen(T) - s;
    if (orc_ctz(T + 1) < e) return S;
    return (uint32_t)((T + 1) % ((uint64_t)S + 1)) - 1;
  }
  if (policy == ORC_TILTED || policy == ORC_STRETCHED) {
    /* Levels: deposition T belongs to level h = ctz(T+1) (capped at L-1,
     * L = S/W), and is the j-th deposition of that level.  Tilted keeps the
     * most recent W of every level in a per-level ring; stretched keeps the
     * first W of every level. */
    uint32_t L = S / W;
    unsigned h = orc_ctz(T + 1);
    uint32_t level;
    uint64_t j;
    if (h < L - 1) {
      level = h;
      j = (T + 1) >> (h + 1);
    } else {
      level = L - 1;
      j = ((T + 1) >> (L - 1)) - 1;
    }
    if (policy == ORC_TILTED) return level * W + (uint32_t)(j % W);
    return j < W ? level * W + (uint32_t)j : S;
  }
  return S; /* ORC_NONE: no surface */
}

/* Hybrid policy (the paper's suggestion to give half of the annotation space
 * to each strategy): every deposition writes two differentiae, one into the
 * steady half (sites [0, S/2)) and one into the tilted half (sites
 * [S/2, S)), each half curated by its policy over S/2 sites.  Site of the
 * tilted half, or S when discarded. */
uint32_t orc_hybrid_second_site(uint32_t S, uint32_t W, uint64_t T) {
  uint32_t b = orc_site(ORC_TILTED, S / 2, W, T);
  return b < S / 2 ? S / 2 + b : S;
}

/* Definition of the timestamp lookup: for every site, the largest deposition
 * time t < T that wrote it, or -1 if none did.  Brute-force replay. */
void orc_lookup(uint32_t policy, uint32_t S, uint32_t W, uint64_t T,
                int64_t *times_out) {
  for (uint32_t p = 0; p < S; ++p) times_out[p] = -1;
  for (uint64_t t = 0; t < T; ++t) {
    uint32_t site = orc_site(policy, S, W, t);
    if (site < S) times_out[site] = (int64_t)t;
    if (policy == ORC_HYBRID) {
      uint32_t second = orc_hybrid_second_site(S, W, t);
      if (second < S) times_out[second] = (int64_t)t;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Genetic algorithm. */

typedef struct orc_cfg {
  uint32_t rows, cols, n, tournament;
  uint32_t policy, bits, W, interval;
  double p_ben, p_del;
  uint64_t seed;
  uint32_t coarsen; /* annotate every coarsen-th generation (0 or 1: every one) */
  uint32_t fitness; /* ORC_FITNESS_TRAIT or ORC_FITNESS_FLOAT */
  double sigma;     /* ORC_FITNESS_FLOAT: standard deviation of the mutation amount */
  uint32_t words;   /* surface width in 64-bit words (0 or 1: one) */
  uint32_t pad;
} orc_cfg;

/* Surfaces of K = words 64-bit words per genome (agent-major: word w of
 * agent a at surf[a K + w]) hold S = 64 K / bits sites; site s occupies bits
 * [s b mod 64, s b mod 64 + b) of word floor(s b / 64) (b divides 64, so no
 * field straddles two words).  K = 4 with 1-bit differentiae is the 256-bit
 * field the paper draws ("Surface-based Hereditary Stratigraphy
 * Algorithms"); wider differentiae and more sites are its suggested
 * remedies for reconstruction precision ("Results › Clade Reconstruction
 * Trial"). */
static uint32_t orc_words(const orc_cfg *cfg) { return cfg->words > 1 ? cfg->words : 1; }

static uint32_t orc_sites(const orc_cfg *cfg) { return 64u * orc_words(cfg) / cfg->bits; }

static void orc_put_field(uint64_t *surface, uint32_t site, uint32_t bits, uint64_t value) {
  uint64_t mask = (bits == 64) ? ~0ull : ((1ull << bits) - 1);
  uint32_t word = site * bits / 64, shift = site * bits % 64;
  surface[word] = (surface[word] & ~(mask << shift)) | ((value & mask) << shift);
}

/* Fitness models ("Methods › Genome Model" and "Results › On-hardware
 * Trial").  TRAIT: the first genome word is an unsigned integer fitness and
 * mutation adds or removes one (saturating).  FLOAT: the first word is an
 * IEEE binary32 fitness (the paper's 128-bit layout) and mutation adds
 * (beneficial) or subtracts (deleterious) the absolute value of a normally
 * distributed amount -- the paper's Gaussian mutation with sign restrictions.
 * The normal variate is the de Moivre-Laplace approximation: with (q0..q3) =
 * Philox(key; j, island, G, ORC_PURPOSE_GAUSS), B = popcount(q0) +
 * popcount(q1) + popcount(q2) ~ Binomial(96, 1/2) (mean 48, variance 24) is
 * smoothed by U = bits 8..31 of q3 / 2^24 (uniform, variance 1/12):
 *   g = (B - 48) 2^24 + (q3 >> 8) - 2^23          (exact, in int32)
 *   amount = |float(g) * c|,  c = float(sigma / sqrt(24 + 1/12) / 2^24),
 * so amount / sigma is |N(0, 1)| to within the approximation.  Every float
 * step is one correctly rounded IEEE operation (int-to-float, multiply,
 * add), evaluated without contraction, so any IEEE machine gets the same
 * bits.  Tournament candidates compare as floats; a later candidate wins only
 * if strictly fitter (the paper breaks ties at random; the first of several
 * equally fit candidates drawn uniformly at random is itself uniformly
 * random among them). */
enum { ORC_FITNESS_TRAIT = 0, ORC_FITNESS_FLOAT = 1 };
#define ORC_PURPOSE_GAUSS 256u

static float orc_f32(uint32_t w) {
  float f;
  memcpy(&f, &w, sizeof f);
  return f;
}

static uint32_t orc_u32(float f) {
  uint32_t w;
  memcpy(&w, &f, sizeof w);
  return w;
}

static uint32_t orc_popcount(uint32_t x) {
  uint32_t c = 0;
  for (; x; x >>= 1) c += x & 1u;
  return c;
}

/* a3 + a4: is the genome with first word a strictly fitter than b's? */
static int orc_fitter(const orc_cfg *cfg, uint32_t a, uint32_t b) {
  if (cfg->fitness == ORC_FITNESS_FLOAT) return orc_f32(a) > orc_f32(b);
  return a > b;
}

static uint64_t orc_threshold(double p);

/* a5: mutation of child j of `island` at generation G whose parent's first
 * word is `trait`; w2 is word 2 of the child's replication block. */
static uint32_t orc_mutate(const orc_cfg *cfg, uint32_t trait, uint32_t w2,
                           uint32_t j, uint32_t island, uint64_t G) {
  uint64_t thr_b = orc_threshold(cfg->p_ben), thr_d = orc_threshold(cfg->p_del);
  int ben = (uint64_t)w2 < thr_b;
  int del = !ben && (uint64_t)w2 < thr_b + thr_d;
  if (cfg->fitness != ORC_FITNESS_FLOAT) {
    if (ben && trait != 0xFFFFFFFFu) return trait + 1;
    if (del && trait != 0) return trait - 1;
    return trait;
  }
  if (!ben && !del) return trait;
  uint32_t q[4];
  orc_draw(cfg->seed, j, island, (uint32_t)G, ORC_PURPOSE_GAUSS, q);
  int32_t B = (int32_t)(orc_popcount(q[0]) + orc_popcount(q[1]) + orc_popcount(q[2]));
  int32_t g = (B - 48) * (1 << 24) + (int32_t)(q[3] >> 8) - (1 << 23);
  float c = (float)(cfg->sigma / sqrt(24.0 + 1.0 / 12.0) / 16777216.0);
  float amount = fabsf((float)g * c);
  float f = orc_f32(trait);
  f = ben ? f + amount : f - amount;
  return orc_u32(f);
}

enum { ORC_N = 0, ORC_E = 1, ORC_S = 2, ORC_W = 3 };

/* Neighbour of global island g on the rows x cols torus in direction d. */
uint32_t orc_neighbour(const orc_cfg *cfg, uint32_t g, uint32_t d) {
  uint32_t r = g / cfg->cols, c = g % cfg->cols;
  switch (d) {
    case ORC_N: r = (r + cfg->rows - 1) % cfg->rows; break;
    case ORC_S: r = (r + 1) % cfg->rows; break;
    case ORC_E: c = (c + 1) % cfg->cols; break;
    default:    c = (c + cfg->cols - 1) % cfg->cols; break;
  }
  return r * cfg->cols + c;
}

/* An emigrant record: the copied genome, its direction and, for pedigree
 * tracking, the global agent index it was copied from: trait, dir, src_lo,
 * src_hi, then the surface words as (low, high) 32-bit pairs. */
static size_t orc_rec_words(const orc_cfg *cfg) { return 4 + 2 * (size_t)orc_words(cfg); }

/* a1: emigrant records of the local islands (global ids gid[0..n_local)).
 * Population arrays are local: island l holds agents [l*n, l*n + n). */
void orc_emigrate(const orc_cfg *cfg, uint32_t n_local, const uint32_t *gid,
                  const uint32_t *trait, const uint64_t *surf, uint64_t G,
                  uint32_t *rec) {
  for (uint32_t l = 0; l < n_local; ++l) {
    uint32_t w[4];
    orc_draw(cfg->seed, 0xFFFFFFFFu, gid[l], (uint32_t)G, 0, w);
    uint32_t slot = orc_index(w[0], cfg->n);
    uint32_t dir = w[1] >> 30;
    uint64_t src = (uint64_t)gid[l] * cfg->n + slot;
    uint32_t K = orc_words(cfg);
    uint32_t *r = rec + (size_t)l * orc_rec_words(cfg);
    size_t a = (size_t)l * cfg->n + slot;
    r[0] = trait[a];
    r[1] = dir;
    r[2] = (uint32_t)src;
    r[3] = (uint32_t)(src >> 32);
    for (uint32_t w2 = 0; w2 < K; ++w2) {
      r[4 + 2 * w2] = (uint32_t)surf[a * K + w2];
      r[5 + 2 * w2] = (uint32_t)(surf[a * K + w2] >> 32);
    }
  }
}

/* a2: in place on the active local islands.  nbr[l*4 + d] is the local index
 * of the neighbour of l in direction d; its record is rec[that].  src (may be
 * NULL) holds, per agent, the global agent index it descends from in the
 * pre-migration population; immigrants overwrite it with theirs. */
void orc_immigrate(const orc_cfg *cfg, uint32_t n_local, const uint32_t *gid,
                   const int32_t *nbr, const uint8_t *active, uint32_t *trait,
                   uint64_t *surf, const uint32_t *rec, uint64_t G,
                   uint64_t *src) {
  for (uint32_t l = 0; l < n_local; ++l) {
    if (active && !active[l]) continue;
    uint32_t v[4];
    orc_draw(cfg->seed, 0xFFFFFFFEu, gid[l], (uint32_t)G, 0, v);
    for (uint32_t d = 0; d < 4; ++d) {
      int32_t nb = nbr[(size_t)l * 4 + d];
      const uint32_t *r = rec + (size_t)nb * orc_rec_words(cfg);
      uint32_t toward_me = (d + 2) % 4; /* the neighbour must aim back at l */
      if (r[1] != toward_me) continue;
      uint32_t slot = orc_index(v[d], cfg->n);
      size_t a = (size_t)l * cfg->n + slot;
      uint32_t K = orc_words(cfg);
      trait[a] = r[0];
      for (uint32_t w2 = 0; w2 < K; ++w2)
        surf[a * K + w2] = (uint64_t)r[4 + 2 * w2] | ((uint64_t)r[5 + 2 * w2] << 32);
      if (src) src[a] = (uint64_t)r[2] | ((uint64_t)r[3] << 32);
    }
  }
}

static uint64_t orc_threshold(double p) {
  /* floor(p * 2^32); p in [0, 1]; multiplying by a power of two is exact. */
  return (uint64_t)(p * 4294967296.0);
}

/* a3-a6 for the active local islands: parents (post-migration) in
 * trait_in/surf_in, children to trait_out/surf_out.  T is the deposition
 * counter the children's new differentia is stamped with.  parent_out (may
 * be NULL) receives per child the pre-migration global agent index of its
 * parent, using src (or the parent's own index when src is NULL). */
void orc_select(const orc_cfg *cfg, uint32_t n_local, const uint32_t *gid,
                const uint8_t *active, const uint32_t *trait_in,
                const uint64_t *surf_in, const uint64_t *src, uint64_t G,
                uint64_t T, uint32_t *trait_out, uint64_t *surf_out,
                uint64_t *parent_out) {
  uint32_t n = cfg->n, K = orc_words(cfg);
  uint32_t S = orc_sites(cfg);
  /* Temporal coarsening (the paper's suggestion to update annotations only
   * every k-th generation): generation T deposits only when k divides it,
   * as deposition number T / k. */
  uint32_t k = cfg->coarsen > 1 ? cfg->coarsen : 1;
  int annotate = (T % k) == 0;
  uint64_t Td = T / k;
  uint32_t site = annotate ? orc_site(cfg->policy, S, cfg->W, Td) : S;
  uint32_t site2 = (annotate && cfg->policy == ORC_HYBRID)
                       ? orc_hybrid_second_site(S, cfg->W, Td) : S;
  for (uint32_t l = 0; l < n_local; ++l) {
    if (active && !active[l]) continue;
    const uint32_t *fit = trait_in + (size_t)l * n; /* a3: fitness = trait */
    for (uint32_t j = 0; j < n; ++j) {
      uint32_t w[4];
      orc_draw(cfg->seed, j, gid[l], (uint32_t)G, 1, w);
      /* a4: tournament of `tournament` candidates, with replacement. */
      uint32_t best = orc_index(w[0], n);
      for (uint32_t c = 1; c < cfg->tournament; ++c) {
        uint32_t word;
        if (c == 1) {
          word = w[1];
        } else {
          uint32_t extra[4];
          orc_draw(cfg->seed, j, gid[l], (uint32_t)G, 2 + (c - 2) / 4, extra);
          word = extra[(c - 2) % 4];
        }
        uint32_t cand = orc_index(word, n);
        if (orc_fitter(cfg, fit[cand], fit[best])) best = cand;
      }
      size_t pa = (size_t)l * n + best;
      size_t ca = (size_t)l * n + j;
      uint64_t *surface = surf_out + ca * K;
      memcpy(surface, surf_in + pa * K, sizeof(uint64_t) * K);
      /* a5: mutation of the trait. */
      uint32_t trait = orc_mutate(cfg, trait_in[pa], w[2], j, gid[l], G);
      /* a6: deposit the new differentia (the hybrid policy's second one is
       * taken from bits 16.. of the same word). */
      if (cfg->policy != ORC_NONE && site < S)
        orc_put_field(surface, site, cfg->bits, w[3]);
      if (cfg->policy != ORC_NONE && site2 < S)
        orc_put_field(surface, site2, cfg->bits, w[3] >> 16);
      trait_out[ca] = trait;
      if (parent_out)
        parent_out[ca] = src ? src[pa] : (uint64_t)gid[l] * n + best;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Whole-torus driver. */

static void orc_torus_tables(const orc_cfg *cfg, uint32_t *gid, int32_t *nbr) {
  uint32_t I = cfg->rows * cfg->cols;
  for (uint32_t g = 0; g < I; ++g) {
    gid[g] = g;
    for (uint32_t d = 0; d < 4; ++d)
      nbr[(size_t)g * 4 + d] = (int32_t)orc_neighbour(cfg, g, d);
  }
}

static int orc_migrates(const orc_cfg *cfg, uint64_t G) {
  return cfg->interval > 0 && G % cfg->interval == 0;
}

/* Runs n_gens generations from generation G0 (sync mode: T = G).  When
 * premigrated is nonzero the migration of generation G0 is taken as already
 * done (see orc_migrate_grid).  parents (may be NULL) receives
 * n_gens * rows*cols*n parent indices, generation-major.  Returns 0, or -1 on
 * allocation failure. */
int orc_run_grid(const orc_cfg *cfg, uint32_t *trait, uint64_t *surf,
                 uint64_t G0, uint64_t n_gens, int premigrated,
                 uint64_t *parents) {
  uint32_t I = cfg->rows * cfg->cols;
  size_t A = (size_t)I * cfg->n, K = orc_words(cfg);
  uint32_t *gid = malloc(sizeof(uint32_t) * I);
  int32_t *nbr = malloc(sizeof(int32_t) * I * 4);
  uint32_t *rec = malloc(sizeof(uint32_t) * orc_rec_words(cfg) * I);
  uint32_t *t2 = malloc(sizeof(uint32_t) * A);
  uint64_t *s2 = malloc(sizeof(uint64_t) * A * K);
  uint64_t *src = parents ? malloc(sizeof(uint64_t) * A) : NULL;
  if (!gid || !nbr || !rec || !t2 || !s2 || (parents && !src)) {
    free(gid); free(nbr); free(rec); free(t2); free(s2); free(src);
    return -1;
  }
  orc_torus_tables(cfg, gid, nbr);
  for (uint64_t k = 0; k < n_gens; ++k) {
    uint64_t G = G0 + k;
    if (src)
      for (size_t a = 0; a < A; ++a) src[a] = a;
    if (orc_migrates(cfg, G) && !(premigrated && k == 0)) {
      orc_emigrate(cfg, I, gid, trait, surf, G, rec);
      orc_immigrate(cfg, I, gid, nbr, NULL, trait, surf, rec, G, src);
    }
    orc_select(cfg, I, gid, NULL, trait, surf, src, G, G, t2, s2,
               parents ? parents + (size_t)k * A : NULL);
    memcpy(trait, t2, sizeof(uint32_t) * A);
    memcpy(surf, s2, sizeof(uint64_t) * A * K);
  }
  free(gid); free(nbr); free(rec); free(t2); free(s2); free(src);
  return 0;
}

/* Explicit a1+a2 of generation G, in place, on the whole torus. */
int orc_migrate_grid(const orc_cfg *cfg, uint32_t *trait, uint64_t *surf,
                     uint64_t G) {
  uint32_t I = cfg->rows * cfg->cols;
  uint32_t *gid = malloc(sizeof(uint32_t) * I);
  int32_t *nbr = malloc(sizeof(int32_t) * I * 4);
  uint32_t *rec = malloc(sizeof(uint32_t) * orc_rec_words(cfg) * I);
  if (!gid || !nbr || !rec) { free(gid); free(nbr); free(rec); return -1; }
  orc_torus_tables(cfg, gid, nbr);
  orc_emigrate(cfg, I, gid, trait, surf, G, rec);
  orc_immigrate(cfg, I, gid, nbr, NULL, trait, surf, rec, G, NULL);
  free(gid); free(nbr); free(rec);
  return 0;
}

/* State at generation G0 + n_gens of one island (row r, column c) of a
 * full-size torus, from a uniform founder state at G0 (every agent: trait0,
 * surface0), computed on its dependency cone only: a (2n_gens+1)^2 box around
 * the island; generation k advances the islands within Chebyshev radius
 * n_gens-k-1 of the centre, whose four neighbours lie inside the radius-
 * (n_gens-k) region known at that generation.  Requires 2*n_gens+1 <= rows
 * and <= cols (no wrap-around onto itself).  Writes the island's n agents. */
int orc_run_cone(const orc_cfg *cfg, uint32_t r, uint32_t c, uint32_t trait0,
                 uint64_t surf0, uint64_t G0, uint32_t n_gens,
                 uint32_t *trait_out, uint64_t *surf_out) {
  uint32_t R = n_gens, D = 2 * R + 1, I = D * D, n = cfg->n;
  if (D > cfg->rows || D > cfg->cols) return -2;
  size_t A = (size_t)I * n, K = orc_words(cfg);
  uint32_t *gid = malloc(sizeof(uint32_t) * I);
  int32_t *nbr = malloc(sizeof(int32_t) * I * 4);
  uint8_t *active = malloc(I);
  uint32_t *rec = malloc(sizeof(uint32_t) * orc_rec_words(cfg) * I);
  uint32_t *t1 = malloc(sizeof(uint32_t) * A), *t2 = malloc(sizeof(uint32_t) * A);
  uint64_t *s1 = malloc(sizeof(uint64_t) * A * K), *s2 = malloc(sizeof(uint64_t) * A * K);
  if (!gid || !nbr || !active || !rec || !t1 || !t2 || !s1 || !s2) {
    free(gid); free(nbr); free(active); free(rec);
    free(t1); free(t2); free(s1); free(s2);
    return -1;
  }
  for (uint32_t y = 0; y < D; ++y)
    for (uint32_t x = 0; x < D; ++x) {
      uint32_t l = y * D + x;
      uint32_t gr = (r + cfg->rows - R + y) % cfg->rows;
      uint32_t gc = (c + cfg->cols - R + x) % cfg->cols;
      gid[l] = gr * cfg->cols + gc;
      nbr[l * 4 + ORC_N] = y > 0 ? (int32_t)(l - D) : -1;
      nbr[l * 4 + ORC_S] = y + 1 < D ? (int32_t)(l + D) : -1;
      nbr[l * 4 + ORC_E] = x + 1 < D ? (int32_t)(l + 1) : -1;
      nbr[l * 4 + ORC_W] = x > 0 ? (int32_t)(l - 1) : -1;
    }
  for (size_t a = 0; a < A; ++a) {
    t1[a] = trait0;
    for (size_t w2 = 0; w2 < K; ++w2) s1[a * K + w2] = w2 == 0 ? surf0 : 0;
  }
  for (uint32_t k = 0; k < n_gens; ++k) {
    uint64_t G = G0 + k;
    uint32_t radius = R - k - 1;
    for (uint32_t y = 0; y < D; ++y)
      for (uint32_t x = 0; x < D; ++x) {
        uint32_t dy = y > R ? y - R : R - y, dx = x > R ? x - R : R - x;
        active[y * D + x] = (dy <= radius && dx <= radius);
      }
    memcpy(t2, t1, sizeof(uint32_t) * A);
    memcpy(s2, s1, sizeof(uint64_t) * A * K);
    if (orc_migrates(cfg, G)) {
      /* Records of every island are computed; only those within the known
       * region are read by the active islands. */
      orc_emigrate(cfg, I, gid, t1, s1, G, rec);
      orc_immigrate(cfg, I, gid, nbr, active, t1, s1, rec, G, NULL);
    }
    orc_select(cfg, I, gid, active, t1, s1, NULL, G, G, t2, s2, NULL);
    uint32_t *tt = t1; t1 = t2; t2 = tt;
    uint64_t *ss = s1; s1 = s2; s2 = ss;
  }
  size_t centre = (size_t)(R * D + R) * n;
  memcpy(trait_out, t1 + centre, sizeof(uint32_t) * n);
  memcpy(surf_out, s1 + centre * K, sizeof(uint64_t) * n * K);
  free(gid); free(nbr); free(active); free(rec);
  free(t1); free(t2); free(s1); free(s2);
  return 0;
}

/* a7: sample k genomes at generation G (one candidate per island, then k
 * distinct islands by partial Fisher-Yates).  out_words gets 2 + 2K words
 * per sample (trait, the surface words as (low, high) pairs, T=G: four words
 * for a one-word surface); out_island_slot (may be NULL) gets (island,
 * slot).  Returns -2 if k exceeds the island count. */
int orc_sample_grid(const orc_cfg *cfg, const uint32_t *trait,
                    const uint64_t *surf, uint64_t G, uint32_t k,
                    uint32_t *out_words, uint32_t *out_island_slot) {
  uint32_t I = cfg->rows * cfg->cols;
  if (k > I) return -2;
  uint32_t *perm = malloc(sizeof(uint32_t) * (I ? I : 1));
  if (!perm) return -1;
  for (uint32_t i = 0; i < I; ++i) perm[i] = i;
  for (uint32_t j = 0; j < k; ++j) {
    uint32_t w[4];
    orc_draw(cfg->seed, j, 0xFFFFFFFFu, (uint32_t)G, 3, w);
    uint32_t pick = j + orc_index(w[0], I - j);
    uint32_t tmp = perm[j]; perm[j] = perm[pick]; perm[pick] = tmp;
  }
  for (uint32_t j = 0; j < k; ++j) {
    uint32_t island = perm[j];
    uint32_t w[4];
    orc_draw(cfg->seed, 0xFFFFFFFDu, island, (uint32_t)G, 0, w);
    uint32_t slot = orc_index(w[0], cfg->n);
    size_t a = (size_t)island * cfg->n + slot;
    uint32_t K = orc_words(cfg);
    uint32_t *o = out_words + (size_t)j * (2 + 2 * K);
    o[0] = trait[a];
    for (uint32_t w2 = 0; w2 < K; ++w2) {
      o[1 + 2 * w2] = (uint32_t)surf[a * K + w2];
      o[2 + 2 * w2] = (uint32_t)(surf[a * K + w2] >> 32);
    }
    o[1 + 2 * K] = (uint32_t)G;
    if (out_island_slot) {
      out_island_slot[2 * j] = island;
      out_island_slot[2 * j + 1] = slot;
    }
  }
  free(perm);
  return 0;
}

/* ------------------------------------------------------------------ */
/* One generation (a3-a6) of island i when genomes carry their own
 * deposition counters (free-running modes): each child deposits at
 * site_fn(T_parent) and carries T_parent + 1 (the paper's per-genome
 * generation counter, "Methods › Genome Model"); the Philox draws are those
 * of the synchronous step.  Updates island i of trait, surf and tcount in
 * place.  Returns 0 or -1 on allocation failure. */
int orc_island_step(const orc_cfg *cfg, uint32_t i, uint64_t G, uint32_t *trait,
                    uint64_t *surf, uint32_t *tcount) {
  uint32_t n = cfg->n, K = orc_words(cfg);
  uint32_t S = orc_sites(cfg);
  uint32_t *ct = malloc(sizeof(uint32_t) * n), *cT = malloc(sizeof(uint32_t) * n);
  uint64_t *cs = malloc(sizeof(uint64_t) * n * K);
  if (!ct || !cT || !cs) {
    free(ct); free(cT); free(cs);
    return -1;
  }
  const uint32_t *fit = trait + (size_t)i * n;
  for (uint32_t j = 0; j < n; ++j) {
    uint32_t w[4];
    orc_draw(cfg->seed, j, i, (uint32_t)G, 1, w);
    uint32_t best = orc_index(w[0], n);
    for (uint32_t c = 1; c < cfg->tournament; ++c) {
      uint32_t word;
      if (c == 1) {
        word = w[1];
      } else {
        uint32_t extra[4];
        orc_draw(cfg->seed, j, i, (uint32_t)G, 2 + (c - 2) / 4, extra);
        word = extra[(c - 2) % 4];
      }
      uint32_t cand = orc_index(word, n);
      if (orc_fitter(cfg, fit[cand], fit[best])) best = cand;
    }
    size_t pa = (size_t)i * n + best;
    uint32_t tr = orc_mutate(cfg, trait[pa], w[2], j, i, G);
    uint64_t *su = cs + (size_t)j * K;
    memcpy(su, surf + pa * K, sizeof(uint64_t) * K);
    uint32_t T = tcount[pa];
    if (cfg->policy != ORC_NONE) {
      uint32_t site = orc_site(cfg->policy, S, cfg->W, T);
      if (site < S) orc_put_field(su, site, cfg->bits, w[3]);
      if (cfg->policy == ORC_HYBRID) {
        uint32_t site2 = orc_hybrid_second_site(S, cfg->W, T);
        if (site2 < S) orc_put_field(su, site2, cfg->bits, w[3] >> 16);
      }
    }
    ct[j] = tr;
    cT[j] = T + 1;
  }
  memcpy(trait + (size_t)i * n, ct, sizeof(uint32_t) * n);
  memcpy(surf + (size_t)i * n * K, cs, sizeof(uint64_t) * n * K);
  memcpy(tcount + (size_t)i * n, cT, sizeof(uint32_t) * n);
  free(ct); free(cT); free(cs);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Free-running (asynchronous) migration, replayed from a schedule.
 *
 * The paper's WSE islands run without a global clock: each keeps one
 * outgoing emigrant buffer per neighbour and takes whatever its neighbours
 * last sent ("Methods › Asynchronous Island-model Genetic Algorithm").  Here
 * every island publishes one emigrant per generation (slot and direction
 * from Philox(key; 0xFFFFFFFF, island, G, 0), as in synchronous mode), and
 * at each of its generations may take, from each neighbour, the latest
 * emigrant that neighbour aimed at it.  Which neighbour generation each
 * accepted emigrant came from is a property of the run's timing, so it is an
 * input: sched[(island * n_gens + g) * 4 + d] = 1 + the neighbour's
 * generation whose emigrant island `island` took from direction d at its own
 * generation g (relative to G0), or 0 for none.  Genomes carry their own
 * deposition counter T (the paper's per-genome generation counter): an
 * immigrant keeps its T, and a child deposits at site_fn(T_parent) and
 * carries T_parent + 1.  Given the schedule the run is deterministic.
 *
 * trait, surf, tcount: the population at G0 (updated in place).  Returns 0,
 * -1 on allocation failure, -3 if the schedule names an emigrant that was not
 * aimed at the island or cannot be ordered causally. */
int orc_run_async(const orc_cfg *cfg, uint32_t *trait, uint64_t *surf,
                  uint32_t *tcount, uint64_t G0, uint32_t n_gens,
                  const uint32_t *sched) {
  if (orc_words(cfg) != 1) return -2;
  uint32_t I = cfg->rows * cfg->cols, n = cfg->n;
  /* emigrant records by island and generation: trait, lo, hi, T, dir */
  uint32_t *hist = malloc(sizeof(uint32_t) * 5 * (size_t)I * (n_gens + 1));
  uint32_t *done = calloc(I, sizeof(uint32_t));
  if (!hist || !done) {
    free(hist); free(done);
    return -1;
  }
  /* the emigrant each island publishes at the start of its generation g */
#define ORC_PUBLISH(I_, G_)                                                    \
  do {                                                                         \
    uint32_t w_[4];                                                            \
    orc_draw(cfg->seed, 0xFFFFFFFFu, (I_), (uint32_t)(G0 + (G_)), 0, w_);      \
    size_t a_ = (size_t)(I_) * n + orc_index(w_[0], n);                        \
    uint32_t *h_ = hist + 5 * ((size_t)(I_) * (n_gens + 1) + (G_));            \
    h_[0] = trait[a_];                                                         \
    h_[1] = (uint32_t)surf[a_];                                                \
    h_[2] = (uint32_t)(surf[a_] >> 32);                                        \
    h_[3] = tcount[a_];                                                        \
    h_[4] = w_[1] >> 30;                                                       \
  } while (0)
  for (uint32_t i = 0; i < I; ++i) ORC_PUBLISH(i, 0);
  int status = 0;
  uint64_t remaining = (uint64_t)I * n_gens;
  while (remaining > 0 && status == 0) {
    int progress = 0;
    for (uint32_t i = 0; i < I && status == 0; ++i) {
      uint32_t g = done[i];
      if (g >= n_gens) continue;
      uint64_t G = G0 + g;
      const uint32_t *req = sched + ((size_t)i * n_gens + g) * 4;
      int ready = 1;
      for (uint32_t d = 0; d < 4; ++d) {
        if (!req[d]) continue;
        uint32_t nb = orc_neighbour(cfg, i, d);
        if (req[d] - 1 > n_gens || done[nb] < req[d] - 1) ready = 0;
      }
      if (!ready) continue;
      /* a2: take the scheduled emigrants, directions N, E, S, W */
      if (orc_migrates(cfg, G)) {
        uint32_t v[4];
        orc_draw(cfg->seed, 0xFFFFFFFEu, i, (uint32_t)G, 0, v);
        for (uint32_t d = 0; d < 4; ++d) {
          if (!req[d]) continue;
          uint32_t nb = orc_neighbour(cfg, i, d);
          const uint32_t *h = hist + 5 * ((size_t)nb * (n_gens + 1) + (req[d] - 1));
          if (h[4] != (d + 2) % 4) { status = -3; break; }
          size_t a = (size_t)i * n + orc_index(v[d], n);
          trait[a] = h[0];
          surf[a] = (uint64_t)h[1] | ((uint64_t)h[2] << 32);
          tcount[a] = h[3];
        }
      } else {
        for (uint32_t d = 0; d < 4; ++d)
          if (req[d]) status = -3;
      }
      if (status) break;
      /* a3-a6 with per-genome counters */
      if (orc_island_step(cfg, i, G, trait, surf, tcount)) { status = -1; break; }
      done[i] = g + 1;
      ORC_PUBLISH(i, g + 1);
      --remaining;
      progress = 1;
    }
    if (!progress && status == 0) status = -3;
  }
#undef ORC_PUBLISH
  free(hist); free(done);
  return status;
}

/* ------------------------------------------------------------------ */
/* Buffered free-running migration (the WSE's per-neighbour buffers),
 * replayed from a log.
 *
 * Section "Asynchronous Island-model Genetic Algorithm": every island keeps,
 * per cardinal neighbour, an emigration buffer of one genome and an
 * immigration buffer of four; each has a completion flag set when its
 * asynchronous send or receive finishes, and the main cycle first copies
 * every completed immigration buffer into the population over randomly
 * chosen members (then re-opens the receive), then refills every completed
 * emigration buffer with a randomly sampled member (then re-opens the send),
 * then evaluates, selects and mutates.  Reading used here, per island and
 * direction d (N, E, S, W), at each migrating generation G of the island:
 *
 *   receive : the channel from the neighbour in direction d holds at most one
 *             genome in flight, numbered by its post count.  If the island
 *             takes it (a property of timing, hence logged), it must be the
 *             one after the last it took from that channel; it is appended to
 *             the immigration buffer and acknowledged (the sender's
 *             send-complete flag).
 *   place   : for d = N, E, S, W in that order, an immigration buffer holding
 *             four genomes is copied into the population, genome j over the
 *             member at slot floor(v_j n / 2^32) of (v_0..v_3) =
 *             Philox(key; 0xFFFFFFFE, island, G, 1 + d), later over earlier,
 *             and emptied.
 *   send    : if the genome last posted toward d has been acknowledged
 *             (always true before the first post), the island may (logged)
 *             post a copy of the member at slot floor(w_d n / 2^32) of
 *             (w_0..w_3) = Philox(key; 0xFFFFFFFF, island, G, 0), taken after
 *             placement.
 *   a3-a6   : as orc_island_step (per-genome counters).
 *
 * The log has one word per island, generation (relative to G0) and
 * direction: (post number taken from direction d, or 0) << 1 | (1 if the
 * island posted toward d).  All channels and buffers start empty at G0.  The
 * replay runs island generations in any order that respects the log's
 * causality (a take needs its post, a post needs the acknowledgement of the
 * previous one) and checks the protocol: takes on a channel are numbered
 * 1, 2, 3, ... and a post is never logged before its acknowledgement.
 *
 * trait, surf, tcount: the population at G0 (updated in place).  chan (may
 * be NULL) receives per island and direction {posts made toward d, last post
 * number taken from d, genomes waiting in the immigration buffer}; inbuf
 * (may be NULL) the waiting genomes, 4 x {trait, lo, hi, T} per island and
 * direction.  Returns 0, -1 on allocation failure, -3 if the log breaks the
 * protocol or cannot be ordered causally. */
int orc_run_buffered(const orc_cfg *cfg, uint32_t *trait, uint64_t *surf,
                     uint32_t *tcount, uint64_t G0, uint32_t n_gens,
                     const uint32_t *log, uint32_t *chan, uint32_t *inbuf) {
  if (orc_words(cfg) != 1) return -2;
  uint32_t I = cfg->rows * cfg->cols, n = cfg->n;
  size_t C = (size_t)I * 4;
  uint32_t *mail = calloc(C * 4, sizeof(uint32_t));      /* genome in flight */
  uint32_t *posts = calloc(C, sizeof(uint32_t));         /* by (island, d) */
  uint32_t *taken = calloc(C, sizeof(uint32_t));         /* from (island, d) */
  uint32_t *count = calloc(C, sizeof(uint32_t));
  uint32_t *buf = calloc(C * 16, sizeof(uint32_t));
  uint32_t *done = calloc(I, sizeof(uint32_t));
  if (!mail || !posts || !taken || !count || !buf || !done) {
    free(mail); free(posts); free(taken); free(count); free(buf); free(done);
    return -1;
  }
  int status = 0;
  uint64_t remaining = (uint64_t)I * n_gens;
  while (remaining > 0 && status == 0) {
    int progress = 0;
    for (uint32_t i = 0; i < I && status == 0; ++i) {
      uint32_t g = done[i];
      if (g >= n_gens) continue;
      uint64_t G = G0 + g;
      const uint32_t *e = log + ((size_t)i * n_gens + g) * 4;
      int mig = orc_migrates(cfg, G);
      uint32_t nb[4], back[4];
      for (uint32_t d = 0; d < 4; ++d) {
        nb[d] = orc_neighbour(cfg, i, d);
        back[d] = (d + 2) % 4;
        if (!mig && e[d]) status = -3;
      }
      if (status) break;
      /* causality: each take needs its post, each post the acknowledgement
       * of the previous one (possibly by this very generation's take, when
       * the island is its own neighbour) */
      int ready = 1;
      for (uint32_t d = 0; d < 4; ++d) {
        uint32_t k = e[d] >> 1;
        if (k && posts[(size_t)nb[d] * 4 + back[d]] < k) ready = 0;
        if (e[d] & 1u) {
          uint32_t r = nb[d], rd = back[d];
          uint32_t ack = taken[(size_t)r * 4 + rd];
          if (r == i && (e[rd] >> 1)) ack = e[rd] >> 1;
          if (ack < posts[(size_t)i * 4 + d]) ready = 0;
        }
      }
      if (!ready) continue;
      if (mig) {
        /* receive */
        for (uint32_t d = 0; d < 4 && status == 0; ++d) {
          uint32_t k = e[d] >> 1;
          if (!k) continue;
          size_t c = (size_t)nb[d] * 4 + back[d], me = (size_t)i * 4 + d;
          if (k != taken[me] + 1 || posts[c] != k || count[me] >= 4) {
            status = -3;
            break;
          }
          memcpy(buf + (me * 4 + count[me]) * 4, mail + c * 4, 4 * sizeof(uint32_t));
          count[me] += 1;
          taken[me] = k;
        }
        if (status) break;
        /* place */
        for (uint32_t d = 0; d < 4; ++d) {
          size_t me = (size_t)i * 4 + d;
          if (count[me] < 4) continue;
          uint32_t v[4];
          orc_draw(cfg->seed, 0xFFFFFFFEu, i, (uint32_t)G, 1 + d, v);
          for (uint32_t j = 0; j < 4; ++j) {
            const uint32_t *h = buf + (me * 4 + j) * 4;
            size_t a = (size_t)i * n + orc_index(v[j], n);
            trait[a] = h[0];
            surf[a] = (uint64_t)h[1] | ((uint64_t)h[2] << 32);
            tcount[a] = h[3];
          }
          count[me] = 0;
        }
        /* send */
        uint32_t w[4];
        orc_draw(cfg->seed, 0xFFFFFFFFu, i, (uint32_t)G, 0, w);
        for (uint32_t d = 0; d < 4; ++d) {
          if (!(e[d] & 1u)) continue;
          size_t me = (size_t)i * 4 + d;
          size_t a = (size_t)i * n + orc_index(w[d], n);
          mail[me * 4 + 0] = trait[a];
          mail[me * 4 + 1] = (uint32_t)surf[a];
          mail[me * 4 + 2] = (uint32_t)(surf[a] >> 32);
          mail[me * 4 + 3] = tcount[a];
          posts[me] += 1;
        }
      }
      if (orc_island_step(cfg, i, G, trait, surf, tcount)) { status = -1; break; }
      done[i] = g + 1;
      --remaining;
      progress = 1;
    }
    if (!progress && status == 0) status = -3;
  }
  if (status == 0 && chan)
    for (size_t c = 0; c < C; ++c) {
      chan[3 * c] = posts[c];
      chan[3 * c + 1] = taken[c];
      chan[3 * c + 2] = count[c];
    }
  if (status == 0 && inbuf) memcpy(inbuf, buf, C * 16 * sizeof(uint32_t));
  free(mail); free(posts); free(taken); free(count); free(buf); free(done);
  return status;
}
