/*
 * hsga.h -- C-ABI of the GB300 (sm_103a) hot path of the tracking-enabled
 * island-model genetic algorithm of Moreno, Yang, Dolson & Zaman,
 * "Trackable Agent-based Evolution Models at Wafer Scale" (arXiv 2404.10861).
 *
 * The library advances a rows x cols toroidal grid of islands, each holding
 * n agents, one generation at a time.  Every generation follows the paper's
 * cycle (section "Asynchronous Island-model Genetic Algorithm") in
 * synchronous-migration form:
 *   a1 emigrate   one random member of every island is copied toward a
 *                 uniformly random von-Neumann neighbour;
 *   a2 immigrate  arriving copies replace random members (directions N, E,
 *                 S, W applied in that order);
 *   a3 evaluate   fitness is the stored uint32 trait;
 *   a4 select     tournament selection, ties to the first-drawn candidate;
 *   a5 mutate     trait +1 with probability p_beneficial, else -1 with
 *                 probability p_deleterious (both saturating);
 *   a6 deposit    the hereditary-stratigraphy annotation update: a new
 *                 random differentia of b bits is written into the 64-bit
 *                 surface at the site the curation policy picks from
 *                 (S, T) (sections "Distributed Phylogenetic Tracking" and
 *                 "Surface-based Hereditary Stratigraphy Algorithms");
 *   a7 sample     end-state genomes, one per island, then k islands without
 *                 replacement (section "On-hardware Trial").
 * All random numbers come from Philox4x32-10 keyed by the 64-bit seed, with
 * counters (slot, island, generation, purpose), so a run is a pure function
 * of its configuration.
 *
 * Conventions for every call:
 *   - Return value: HSGA_OK (0) or a negative hsga_status; nothing is thrown
 *     across the ABI.  hsga_status_string() names a status.
 *   - Calls that touch the device are stream-ordered on the grid's stream and
 *     asynchronous with respect to the host unless stated otherwise.
 *   - Pointers marked "host or device" may be either; the library asks the
 *     CUDA runtime which one it is and copies accordingly.  The caller owns
 *     every buffer it passes; the library owns the grid and its buffers
 *     until hsga_destroy().
 *   - rows * cols * agents_per_island must stay below 2^32 - 1 (agent
 *     offsets are 32-bit on the device).
 *   - Genome record (the paper's 128-bit layout, section "Genome Model"):
 *     4 x uint32 = [trait, surface bits 0..31, surface bits 32..63, T].
 *     Differentia of site p occupies surface bits [p*b, p*b + b).
 */
#ifndef HSGA_H
#define HSGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hsga_status {
  HSGA_OK = 0,
  HSGA_ERR_INVALID_ARG = -1,  /* a null pointer, a size or a field out of range */
  HSGA_ERR_OOM = -2,          /* device allocation failed */
  HSGA_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  HSGA_ERR_DEVICE = -4,       /* a kernel reported an inconsistent state */
  HSGA_ERR_WAIT_TIMEOUT = -5, /* a bounded device-side wait ran out */
  HSGA_ERR_UNSUPPORTED = -6,  /* valid request the library does not support */
  HSGA_ERR_NOT_CAPTURABLE = -7 /* a call that waits for its stream, made while that
                                  stream is being captured into a CUDA graph; the
                                  call returns before touching the stream, so the
                                  capture stays valid */
} hsga_status;

/* Surface curation policies.  The paper defines steady (retained time points
 * spread evenly over history) and tilted (recent time points preferred) and
 * fixes their properties, not their formulas; this library's O(1) site
 * functions are its own readings of those properties:
 *   steady    epoch e = max(0, bitlen(T) - log2 S); keep T only when 2^e
 *             divides T+1, at site ((T+1) mod (S+1)) - 1;
 *   tilted    level h = min(ctz(T+1), L-1), L = S/W; a per-level ring keeps
 *             the last W depositions of every level;
 *   stretched same levels, keeps the first W depositions of every level;
 *   trivial   site = T mod S (the paper's benchmark control);
 *   none      no surface (the paper's untracked 32-bit genome);
 *   hybrid    half of the sites steady and half tilted, each over S/2 sites
 *             (the paper's suggestion of splitting annotation space between
 *             the two): every deposition writes two differentiae, the second
 *             from bits 16.. of the random word. */
typedef enum hsga_policy {
  HSGA_STEADY = 0,
  HSGA_TILTED = 1,
  HSGA_STRETCHED = 2,
  HSGA_TRIVIAL = 3,
  HSGA_NONE = 4,
  HSGA_HYBRID = 5
} hsga_policy;

/* Which kernel advances generations. */
typedef enum hsga_kernel {
  HSGA_KERNEL_AUTO = 0,      /* resident when the grid fits on chip, else streamed */
  HSGA_KERNEL_STREAMED = 1,  /* one launch per generation, population in HBM */
  HSGA_KERNEL_RESIDENT = 2,  /* persistent launch, genomes in registers; grids of at
                                most 32 warps run in one block (block barriers), larger
                                ones as a cooperative grid (stamped neighbour records) */
  HSGA_KERNEL_RESIDENT_GRID = 3  /* resident, always the cooperative multi-block form */
} hsga_kernel;

/* Migration modes.  Synchronous: every island takes its neighbours' emigrants
 * of the same generation (bit-reproducible).  The two free-running modes are
 * the WSE's own regime (section "Asynchronous Island-model Genetic
 * Algorithm"): islands never wait for one another, results depend on timing,
 * genomes carry their own deposition counters, and agents_per_island <= 32,
 * deposit_interval <= 1.
 *   ASYNC: each island publishes one emigrant per migrating generation, aimed
 *     at a random neighbour, and takes a neighbour's latest emigrant if it is
 *     new and aimed at it (records overwritten unseen are lost).
 *   BUFFERED: the paper's per-neighbour buffers.  Per island and direction a
 *     one-genome send channel and a four-genome receive buffer: at each
 *     migrating generation an island takes the next genome waiting on each
 *     incoming channel (acknowledging it), copies every full receive buffer
 *     into the population over random members (directions N, E, S, W; slots
 *     from Philox(key; 0xFFFFFFFE, island, G, 1 + d)), then sends a copy of a
 *     random member (slot from word d of Philox(key; 0xFFFFFFFF, island, G,
 *     0)) on every channel whose previous genome was acknowledged.  No genome
 *     is lost; a slow receiver holds its sender back.
 * Free-running grids do not support hsga_migrate, checkpoints, batches or the
 * allocation-free entry point. */
typedef enum hsga_migration_mode {
  HSGA_MIGRATION_SYNC = 0,
  HSGA_MIGRATION_ASYNC = 1,
  HSGA_MIGRATION_BUFFERED = 2
} hsga_migration_mode;

/* Fitness models (sections "Genome Model" and "On-hardware Trial").
 *   TRAIT: the genome's first word is an unsigned integer fitness; mutations
 *     add or remove one (saturating).
 *   FLOAT: the first word is an IEEE binary32 fitness (the paper's 128-bit
 *     layout); a beneficial mutation adds, a deleterious one subtracts, the
 *     absolute value of a normally distributed amount of standard deviation
 *     mutation_sigma (the paper's Gaussian mutation with sign restrictions).
 *     The normal variate is the de Moivre-Laplace approximation from child
 *     j's block (q0..q3) = Philox(key; j, island, G, 256):
 *       g = (popc(q0) + popc(q1) + popc(q2) - 48) 2^24 + (q3 >> 8) - 2^23,
 *       amount = |float(g) * c|, c = float(sigma / sqrt(24 + 1/12) / 2^24),
 *     each float step one correctly rounded operation, so results are
 *     bit-reproducible.  Candidates compare as floats.  Requires
 *     agents_per_island <= 32 and the streamed kernel (or AUTO) in
 *     synchronous mode; not available in batches or the allocation-free
 *     entry point. */
typedef enum hsga_fitness {
  HSGA_FITNESS_TRAIT = 0,
  HSGA_FITNESS_FLOAT = 1
} hsga_fitness;

/* Surface width (sections "Surface-based Hereditary Stratigraphy
 * Algorithms", whose figure shows a 256-bit field, and "Results › Clade
 * Reconstruction Trial", which names more and wider differentiae as the
 * remedy for reconstruction precision).  A surface is K = surface_words
 * 64-bit words holding S = 64 K / differentia_bits sites; site s occupies
 * bits [s b mod 64, s b mod 64 + b) of word floor(s b / 64).  Population
 * arrays hold K words per agent, agent-major (word w of agent a at
 * surf[a K + w]); sample records are 2 + 2K words (trait, the surface words
 * as (low, high) 32-bit pairs, T), i.e. four words when K = 1.  K > 1 needs
 * synchronous migration, a surface policy, agents_per_island <= 32 and the
 * AUTO or STREAMED kernel (a warp-per-island path); fossil sampling,
 * batches and the allocation-free entry point need K = 1. */
/* Run configuration (plain data, caller-owned; copied by hsga_init_grid). */
typedef struct hsga_config {
  uint32_t rows, cols;          /* toroidal island grid, each >= 1 */
  uint32_t agents_per_island;   /* n, 1..64 (the paper's runs use 32) */
  uint32_t tournament_size;     /* 1..64 (the paper uses 5) */
  uint32_t surface_policy;      /* hsga_policy */
  uint32_t differentia_bits;    /* b in {1,2,4,8,16}; S = 64 K / b sites */
  uint32_t sites_per_level;     /* W for tilted / stretched: 1, 2 or 4, S/W >= 2 */
  uint32_t migration_interval;  /* migrate when G % interval == 0; 0 = never */
  double p_beneficial;          /* in [0,1]; p_beneficial + p_deleterious <= 1 */
  double p_deleterious;
  uint64_t seed;                /* Philox key (low word, high word) */
  uint32_t kernel;              /* hsga_kernel */
  uint32_t deposit_interval;    /* temporal coarsening k: only generations G with
                                   k | G deposit, as deposition G / k (0 or 1:
                                   every generation) */
  uint32_t migration_mode;      /* hsga_migration_mode */
  uint32_t fitness;             /* hsga_fitness */
  double mutation_sigma;        /* FLOAT: standard deviation of mutation amounts, > 0 */
  uint32_t surface_words;       /* K: surface width in 64-bit words, 1 (0), 2 or 4 */
  uint32_t reserved;            /* must be 0 */
} hsga_config;

typedef struct hsga_stats {
  uint64_t generation;          /* G: generations elapsed (= deposition count T) */
  uint64_t replications;        /* agents x generations advanced by this grid */
  uint64_t kernel_launches;     /* kernels this grid launched */
  uint32_t kernel;              /* hsga_kernel that advances generations */
  uint32_t islands_per_warp;    /* resident kernel tile shape (0 if streamed) */
  uint32_t warps_per_block;
  uint32_t blocks;
  uint32_t fossils;             /* fossil records held */
  uint64_t fossils_dropped;     /* fossil records not taken: buffer full */
} hsga_stats;

typedef struct hsga_grid hsga_grid;

/* Device allocator hooks (optional).  alloc returns device memory of at
 * least `bytes` bytes usable on `stream`, or NULL; free releases it.  Set
 * before hsga_init_grid; grids keep the hooks they were created with.
 * Passing NULL for both restores the default (cudaMallocAsync/cudaFreeAsync
 * on the grid's stream). */
typedef void *(*hsga_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*hsga_free_fn)(void *ptr, void *stream, void *ctx);
int hsga_set_allocator(hsga_alloc_fn alloc, hsga_free_fn free_fn, void *ctx);

/* Creates a grid at generation 0 holding the founding population (every
 * trait 0, every surface empty) on the current CUDA device.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * Paper: the generational cycle and its startup (section "Asynchronous
 * Island-model Genetic Algorithm"). */
int hsga_init_grid(const hsga_config *cfg, void *cuda_stream, hsga_grid **out);

/* Replaces the population and sets the generation counter.
 * trait: rows*cols*n uint32 (host or device); surf: rows*cols*n uint64
 * (host or device); agent a of island i is entry i*n + a.
 * generation: the new G (< 2^32 - 1).  A pending explicit migration is
 * cleared.  Host buffers may be reused when the call returns. */
int hsga_set_population(hsga_grid *g, const uint32_t *trait,
                        const uint64_t *surf, uint64_t generation);

/* Copies the population out (same layout as hsga_set_population; host or
 * device).  Synchronous when either destination is host memory. */
int hsga_get_population(hsga_grid *g, uint32_t *trait, uint64_t *surf);

/* Advances n_generations full cycles (steps a1-a6 each).
 * Paper: the main update loop repeated to a generation-count halt. */
int hsga_run_generations(hsga_grid *g, uint64_t n_generations);

/* Applies steps a1+a2 (emigrate, immigrate) of the current generation now,
 * in place; the next hsga_run_generations skips that generation's migration.
 * A second call before advancing returns HSGA_ERR_INVALID_ARG.
 * Paper: migration is handled first in every cycle. */
int hsga_migrate(hsga_grid *g);

/* Step a7: k end-state genomes.  Each island offers the member at slot
 * floor(w0*n/2^32) of Philox(seed; 0xFFFFFFFD, island, G, 0); k distinct
 * islands are chosen by a partial Fisher-Yates shuffle whose j-th draw is
 * word 0 of Philox(seed; j, 0xFFFFFFFF, G, 3).
 * out_words: k*4 uint32 genome records (host or device);
 * out_island_slot: k*2 uint32 (island, slot) or NULL (host or device).
 * k = 0 is a no-op; k > rows*cols is HSGA_ERR_INVALID_ARG.  Synchronous when
 * an output is host memory.
 * Paper: one genome sampled per PE, then subsamples of 10k (section
 * "On-hardware Trial"). */
int hsga_sample_surfaces(hsga_grid *g, uint32_t k, uint32_t *out_words,
                         uint32_t *out_island_slot);

/* Fossil sampling (section "Distributed Phylogenetic Tracking": sampling
 * genomes during the run keeps lineages that later go extinct in the
 * reconstruction).  After every generation G that `every` divides,
 * hsga_run_generations takes step a7 (k genomes, same draws and record
 * layout as hsga_sample_surfaces at that G; word 3 holds G) into a device
 * buffer of `capacity` records; once full, further samples are counted in
 * hsga_stats.fossils_dropped.  every = 0 turns sampling off and frees the
 * buffer; any call clears the records held.  k <= rows*cols,
 * capacity >= k. */
int hsga_set_fossil_sampling(hsga_grid *g, uint64_t every, uint32_t k, uint32_t capacity);

/* Copies up to max_records fossil records (in sampling order) to out_words
 * (4 words each) and out_island_slot (2 words each, may be NULL), host or
 * device; *count receives the number of records held.  Synchronous. */
int hsga_get_fossils(hsga_grid *g, uint32_t *out_words, uint32_t *out_island_slot,
                     uint32_t max_records, uint32_t *count);

/* Per-genome deposition counters T (rows*cols*n uint32, host or device).  In
 * synchronous mode every genome's T is the generation.  Synchronous when the
 * destination is host memory. */
int hsga_get_counters(hsga_grid *g, uint32_t *T_out);

/* Free-running grids: logs, for the next `generations` generations from the
 * current one, what each island exchanged; entry ((island * generations + g)
 * * 4 + d) describes direction d at generation G_now + g.  ASYNC: 1 + the
 * absolute generation of the emigrant taken from direction d, or 0.
 * BUFFERED: (number of the post taken from direction d, counted from 1 on
 * each channel, or 0) << 1 | (1 if the island sent toward d).  Starts a fresh
 * free-running window (no record published earlier is taken; buffered
 * channels and receive buffers are emptied), so the CPU oracle can replay the
 * window exactly.  generations = 0 stops logging. */
int hsga_set_async_log(hsga_grid *g, uint32_t generations);

/* Copies the log (islands * generations * 4 uint32; host or device).
 * Synchronous. */
int hsga_get_async_log(hsga_grid *g, uint32_t *out);

/* Free-running grids: generations (1..65536) by which a warp advances each
 * island octet (four consecutive islands) it owns before it moves to its
 * next one; the octet's genomes stay in registers meanwhile, so a grid too
 * large to stay on chip streams through device memory once per `generations`
 * generations instead of every generation.  At any moment the islands being
 * advanced form a band of consecutive islands; migrants from neighbours
 * outside the band are the latest those neighbours published, as free-
 * running migration allows ("Methods › Asynchronous Island-model Genetic
 * Algorithm": islands run without a global clock), and logged runs replay
 * exactly.  1 (the default) advances every octet one generation at a time,
 * the whole grid together.  HSGA_ERR_UNSUPPORTED for synchronous grids.
 * Host function; applies to later hsga_run_generations calls. */
int hsga_set_octet_slice(hsga_grid *g, uint32_t generations);

/* BUFFERED grids: channel state.  chan_out (islands * 4 * 3 uint32) receives
 * per island and direction {posts sent toward d, number of the last post
 * taken from d, genomes waiting in the receive buffer of d}; inbuf_out (may be
 * NULL; islands * 4 * 4 * 4 uint32) the receive buffers, 4 genomes
 * {trait, surface low, surface high, T} per island and direction, of which
 * the first `waiting` are meaningful.  Counts restart at every
 * hsga_set_async_log.  Host or device; synchronous.  HSGA_ERR_UNSUPPORTED for
 * other modes. */
int hsga_get_migration_buffers(hsga_grid *g, uint32_t *chan_out, uint32_t *inbuf_out);

/* Waits for the grid's stream and returns the first error a kernel reported
 * (HSGA_ERR_WAIT_TIMEOUT, HSGA_ERR_DEVICE) or a pending CUDA error. */
int hsga_synchronize(hsga_grid *g);

/* Host-side counters (no device access). */
int hsga_get_stats(const hsga_grid *g, hsga_stats *out);

/* Checkpoint.  hsga_save with buf == NULL stores the required size in *len;
 * otherwise writes config, generation and population into buf (host memory,
 * *len bytes available) and stores the bytes written.  hsga_load restores a
 * checkpoint taken from a grid of identical configuration; continuing from it
 * is bit-identical to an uninterrupted run.  Both are synchronous. */
int hsga_save(hsga_grid *g, void *buf, size_t *len);
int hsga_load(hsga_grid *g, const void *buf, size_t len);

/* Frees the grid and its device buffers (after waiting for its stream). */
void hsga_destroy(hsga_grid *g);

/* Site written by deposition number T (T < 2^32 - 1) under `policy` with S
 * sites (power of two, 2..256) and W sites per level; returns S when the
 * policy discards that deposition.  Host function. */
uint32_t hsga_site(uint32_t policy, uint32_t S, uint32_t W, uint64_t T);

/* Timestamp lookup: deposition time held by every site after T depositions,
 * from (site, T) alone (section "Distributed Phylogenetic Tracking": no
 * stored timestamps).  times_out: S int64 (host), -1 for a site never
 * written.  Closed form, O(S).  Host function.  With temporal coarsening k,
 * G generations make T = ceil(G / k) depositions and deposition t happened
 * at generation t k.  For the hybrid policy hsga_site returns the site of
 * its steady half; hsga_lookup covers both halves. */
int hsga_lookup(uint32_t policy, uint32_t S, uint32_t W, uint64_t T,
                int64_t *times_out);

/* Site function on the device for T = T0 .. T0+count-1 (T0+count < 2^32):
 * out_dev[i] = hsga_site(policy, S, W, T0 + i).  out_dev: device uint32.
 * Stream-ordered on cuda_stream.  The paper's per-operation surface
 * microbenchmark (section "Surface Algorithm Benchmark on Conventional
 * CPU"). */
int hsga_sites_device(uint32_t policy, uint32_t S, uint32_t W, uint64_t T0,
                      uint64_t count, uint32_t *out_dev, void *cuda_stream);

/* The bounded waits the resident kernel applies to its neighbours' migrant
 * records, run on a caller's record: waits until all four 64-bit words of
 * record_dev carry seq in their high 32 bits, giving up after limit_ns
 * (<= 1 s) of the GPU's global timer or 2^22 polls -- first in the form one
 * thread runs (islands polling each neighbour), then in the form a whole
 * warp runs (tiles of islands polling their neighbouring tiles; four lanes,
 * one word each).  Returns HSGA_OK when both saw the record arrive,
 * HSGA_ERR_WAIT_TIMEOUT when either gave up (the context stays usable);
 * *waited_ns (may be NULL) receives the time spent in both.  record_dev: device, 4 uint64, 8-byte aligned.  Synchronous on
 * cuda_stream.  For checking that an unmet wait ends with a status instead of
 * hanging. */
int hsga_wait_probe(const uint64_t *record_dev, uint32_t seq, uint64_t limit_ns,
                    uint64_t *waited_ns, void *cuda_stream);

/* The counter-based generator every kernel draws from (Philox4x32-10 of
 * Salmon et al., SC'11, key = (seed low, seed high)): out_dev[4 i + j] = word
 * j of the block for counter (c0 + i, c1, c2, c3), i < count (c0 + count <=
 * 2^32).  out_dev: device uint32.  Stream-ordered on cuda_stream.  For
 * checking the generator against an independent implementation; the paper
 * does not name its generator. */
int hsga_philox_device(uint64_t seed, uint32_t c0, uint32_t count, uint32_t c1, uint32_t c2,
                       uint32_t c3, uint32_t *out_dev, void *cuda_stream);

/* Throughput of the same generator in the form the generation kernels
 * evaluate it (round keys held in the kernel's parameter block), for the
 * path's integer-issue ceiling: every replication (steps a4-a6) draws one
 * block, so no kernel of the path can replicate faster than this kernel
 * draws blocks.  Thread t < threads evaluates the blocks for counters
 * (i, t, c2, c3), i < blocks_per_thread, and stores the xor of all their
 * words in out_dev[t] (device uint32; threads <= 2^30, else
 * HSGA_ERR_INVALID_ARG).  Stream-ordered on cuda_stream. */
int hsga_philox_throughput(uint64_t seed, uint32_t threads, uint32_t blocks_per_thread,
                           uint32_t c2, uint32_t c3, uint32_t *out_dev, void *cuda_stream);

/* Phylogeny reconstruction on the GPU from k sampled surfaces (of
 * surface_words 64-bit words each, agent-major; 0 means 1) that all
 * elapsed `generations` generations (synchronous mode, or free-running
 * genomes of one counter), section "Distributed Phylogenetic Tracking": each
 * genome's retained differentiae in ascending deposition time form a path in
 * a trie; the trie with unifurcations collapsed (the root kept) is the tree.
 * Nodes: 0 is the root (time -1); an internal node's time is the generation
 * of the last differentia its genomes share; leaves (time = generations)
 * follow the internal nodes, one per sample.  Outputs (host or device, all
 * the same kind): parent_out / time_out (capacity >= 2k + 1 entries;
 * parent of the root = -1), leaf_of_sample (k entries: the leaf node of
 * sample i), *n_nodes (host).  surf: k * surface_words uint64, host or
 * device.  Node numbering
 * other than the root's is unspecified.  deposit_interval as in hsga_config.
 * Allocates scratch through the registered allocator; synchronous on
 * cuda_stream.  HSGA_ERR_INVALID_ARG for k = 0, k > 2^28, policy NONE, a bad
 * width or capacity. */
int hsga_reconstruct(const uint64_t *surf, uint32_t k, uint32_t surface_words, uint32_t policy,
                     uint32_t differentia_bits, uint32_t W, uint64_t generations,
                     uint32_t deposit_interval,
                     int64_t *parent_out, int64_t *time_out, uint32_t *leaf_of_sample,
                     uint32_t capacity, uint32_t *n_nodes, void *cuda_stream);

/* ------------------------------------------------------------ batches ---
 * Many independent runs (uneven grids, agents per island, policies,
 * mutation rates, seeds and generation budgets) advanced together: each
 * "tick" advances every active run by one generation in one launch per
 * agents-per-lane class (n <= 32, n > 32), ticks are replayed from CUDA
 * graphs, and the launch shape is picked by timing real ticks.  Every run
 * is bit-identical to the same configuration run alone on a grid.  Runs can
 * be added and removed between calls (continuous batching); a run added at
 * tick t starts from founders at generation 0 and is active for its budget
 * of ticks.  Paper: many replicate runs of the island-model GA (section
 * "On-hardware Trial": replicates per treatment and array size). */
typedef struct hsga_batch hsga_batch;

typedef struct hsga_batch_run_info {
  uint64_t generation;  /* generations the run has completed */
  uint64_t budget;      /* generations it was admitted for */
  uint64_t agents;
  uint32_t done;        /* generation == budget */
  uint32_t live;        /* planes still held (not removed) */
} hsga_batch_run_info;

typedef struct hsga_batch_stats {
  uint64_t tick;             /* ticks elapsed */
  uint64_t replications;     /* agent replications advanced */
  uint64_t kernel_launches;
  uint64_t phases;           /* distinct active sets run */
  uint64_t device_bytes;     /* population planes held */
  uint32_t live_runs, active_runs;
  uint32_t threads_per_block, blocks;  /* current launch shape */
} hsga_batch_stats;

/* Creates an empty batch at tick 0.  cuda_stream: a cudaStream_t; NULL makes
 * the batch create (and later destroy) its own non-blocking stream, because
 * graphs cannot be captured on the legacy default stream. */
int hsga_batch_create(void *cuda_stream, hsga_batch **out);

/* Admits a run (founders at generation 0) for `generations` generations;
 * allocates its two population planes (24 bytes per agent) through the
 * registered allocator.  *run_id receives its index. */
int hsga_batch_add(hsga_batch *b, const hsga_config *cfg, uint64_t generations,
                   uint32_t *run_id);

/* Advances the batch by up to `ticks` ticks (stops early once no run is
 * active; each run stops at its own budget).  Stream-ordered. */
int hsga_batch_run(hsga_batch *b, uint64_t ticks);

int hsga_batch_info(const hsga_batch *b, uint32_t run, hsga_batch_run_info *out);

/* Population of a live run at its current generation (layout as
 * hsga_get_population; host or device destinations).  Synchronous. */
int hsga_batch_get_population(hsga_batch *b, uint32_t run, uint32_t *trait, uint64_t *surf);

/* Step a7 on a live run at its current generation (same draws and layout as
 * hsga_sample_surfaces).  Synchronous. */
int hsga_batch_sample(hsga_batch *b, uint32_t run, uint32_t k, uint32_t *out_words,
                      uint32_t *out_island_slot);

/* Frees a run's planes (its id stays allocated; further queries fail). */
int hsga_batch_remove(hsga_batch *b, uint32_t run);

int hsga_batch_get_stats(const hsga_batch *b, hsga_batch_stats *out);

/* Device bytes a run of this configuration holds in a batch (admission by
 * memory footprint).  Host function. */
int hsga_run_footprint(const hsga_config *cfg, uint64_t *bytes);

/* Waits for the batch's stream (all ticks issued so far). */
int hsga_batch_synchronize(hsga_batch *b);

void hsga_batch_destroy(hsga_batch *b);

/* Allocation-free variant of hsga_run_generations for callers that must not
 * allocate device memory (a process under a fixed memory budget, a plugin
 * living inside another framework's allocator): it advances n_generations
 * synchronous generations (steps a1-a6 each, bit-identical to a grid run
 * with the same configuration) in place on the caller's device planes, with
 * the resident kernel, and performs no device allocation of any kind.  The
 * paper has no counterpart; it is an interface convenience of this library.
 *   cfg: run configuration (cfg->kernel is ignored); rows*cols <= 8192
 *        islands, else HSGA_ERR_INVALID_ARG.
 *   generation: G of the population on entry (the result is at G + n);
 *        G + n must stay below 2^32 - 64, else HSGA_ERR_INVALID_ARG.
 *   trait, surf: device planes on the current device, layout as
 *        hsga_set_population; surf may be NULL only for HSGA_NONE.  Host
 *        pointers and planes on another device are HSGA_ERR_INVALID_ARG.
 * Scratch (stamped migrant records and an error word: ~512 KiB) is one
 * array built into the library and held on every device that loads it until
 * exit.  The first call on a device looks its address up
 * (cudaGetSymbolAddress), so make that first call before any stream capture;
 * the address is kept until exit, so calls after a device reset are not
 * supported.  All calls share the array: calls whose work overlaps on the
 * GPU race.  The work is stream-ordered on cuda_stream; the call then waits
 * for that stream and reads the kernels' error word back to the host before
 * it returns their status (HSGA_ERR_WAIT_TIMEOUT / HSGA_ERR_DEVICE on a
 * device-side error). */
int hsga_run_generations_noalloc(const hsga_config *cfg, uint64_t generation,
                                 uint64_t n_generations, uint32_t *trait,
                                 uint64_t *surf, void *cuda_stream);

const char *hsga_status_string(int status);

/* ABI version (major * 100 + minor). */
int hsga_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HSGA_H */
