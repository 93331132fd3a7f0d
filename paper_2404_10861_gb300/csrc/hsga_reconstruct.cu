// hsga_reconstruct.cu -- phylogeny reconstruction from sampled surfaces on
// the GPU.
//
// Section "Distributed Phylogenetic Tracking" (and "Results › On-hardware
// Trial", which reconstructs from 10,000-genome samples): each genome's
// retained differentiae, read in ascending deposition time, are a path in a
// trie; genomes share a path exactly as long as they share ancestry (up to
// differentia collisions), and the trie with its unifurcations collapsed is
// the reconstructed tree.  Node times: the root -1, a node reached after d
// differentiae the time of the d-th retained deposition, a leaf the
// generation count T.
//
// GPU formulation (all samples elapsed the same T, so they retain the same
// deposition times):
//   1. keys:  each surface's differentiae permuted into time order, oldest in
//             the most significant bits (of a key as wide as the surface), so
//             that numeric order is path order;
//   2. sort:  least-significant-digit radix sort of (key, sample) over the
//             key's significant bits (8-bit digits; stable block scatter
//             ranked with warp match);
//   3. lcp:   L[j] = number of leading differentiae shared by sorted keys j
//             and j + 1;
//   4. tree:  the collapsed trie's internal nodes are exactly the maximal
//             runs ("lcp intervals") of L >= l that contain an L == l, for
//             each l >= 1 -- the same correspondence that turns a suffix array
//             with its lcp array into a suffix tree.  An interval's parent is
//             the interval holding the larger of the two lcps just outside
//             it; a leaf hangs from the interval holding the larger of its
//             two neighbouring lcps; value 0 (or nothing) is the root.  The
//             nearest smaller values this needs come from a 32-ary tree of
//             minima, and each interval is named by its leftmost position
//             (pointer jumping along equal values).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "hsga.h"
#include "hsga_internal.h"

namespace hsga {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

constexpr int kMaxWords = 4;

struct KeyPlan {
  uint32_t fields;     // retained differentiae m
  uint32_t bits;       // differentia width b
  uint32_t words;      // surface (and key) width K in 64-bit words
  uint32_t src[64 * kMaxWords];  // bit offset of field j (time order) in the surface
};

// A key of K words: field j (time order) at key bits [j b, (j + 1) b)
// counted from the most significant bit of word 0.
struct KeyWords {
  uint64_t *w[kMaxWords];
};

__global__ void make_keys_kernel(KeyPlan kp, const uint64_t *__restrict__ surf, uint32_t k,
                                 KeyWords key, uint32_t *__restrict__ val) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  const uint64_t mask = (kp.bits == 64) ? ~0ull : ((1ull << kp.bits) - 1);
  uint64_t out[kMaxWords] = {0, 0, 0, 0};
  for (uint32_t j = 0; j < kp.fields; ++j) {
    const uint32_t src = kp.src[j];
    const uint64_t v = (surf[(size_t)i * kp.words + src / 64] >> (src % 64)) & mask;
    const uint32_t g = j * kp.bits;  // global key bit from the top
    out[g / 64] |= v << (64u - g % 64 - kp.bits);
  }
  for (uint32_t w = 0; w < kp.words; ++w) key.w[w][i] = out[w];
  val[i] = i;
}

// ------------------------------------------------------------ radix sort ---
__global__ void digit_histogram_kernel(const uint64_t *__restrict__ key, uint32_t k,
                                       uint32_t shift, uint32_t nblocks,
                                       uint32_t *__restrict__ hist) {
  // key: the key word that holds this pass's digit
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t e = base + r * kSortThreads + threadIdx.x;
    if (e < k) atomicAdd(&cnt[(uint32_t)(key[e] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix sum of n uint32 in place, one block of 1024 threads
// (each thread scans a contiguous chunk).
__global__ void exclusive_scan_kernel(uint32_t *__restrict__ a, uint32_t n,
                                      uint32_t *__restrict__ total) {
  __shared__ uint32_t part[1024];
  const uint32_t t = threadIdx.x;
  const uint32_t chunk = (n + 1023) / 1024;
  const uint32_t lo = min(n, t * chunk), hi = min(n, lo + chunk);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; ++i) s += a[i];
  part[t] = s;
  __syncthreads();
  for (uint32_t off = 1; off < 1024; off <<= 1) {
    const uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - s;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  if (t == 1023 && total) *total = part[1023];
}

// Stable scatter of one digit pass: elements keep their order within a
// digit.  A tile is processed in rounds of 256 elements; within a round the
// rank of an element among equal digits is (earlier rounds) + (earlier
// warps of this round) + (earlier lanes of its warp, from __match_any_sync).
__global__ void digit_scatter_kernel(KeyWords key_in, const uint32_t *__restrict__ val_in,
                                     uint32_t k, uint32_t words, uint32_t dword, uint32_t shift,
                                     uint32_t nblocks, const uint32_t *__restrict__ offsets,
                                     KeyWords key_out, uint32_t *__restrict__ val_out) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t running[256];
  __shared__ uint32_t wc[kWarps][256];
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  running[t] = offsets[t * nblocks + blockIdx.x];
  const uint32_t base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    for (int w = 0; w < kWarps; ++w) wc[w][t] = 0;
    __syncthreads();
    const uint32_t e = base + r * kSortThreads + t;
    const bool live = e < k;
    const uint32_t active = __ballot_sync(0xFFFFFFFFu, live);
    uint64_t kv[kMaxWords] = {0, 0, 0, 0};
    uint32_t vv = 0, d = 0, rank = 0;
    if (live) {
      for (uint32_t w = 0; w < words; ++w) kv[w] = key_in.w[w][e];
      vv = val_in[e];
      d = (uint32_t)(key_in.w[dword][e] >> shift) & 0xFFu;
      const uint32_t peers = __match_any_sync(active, d);
      rank = __popc(peers & ((1u << lane) - 1u));
      if (rank == 0) wc[warp][d] = __popc(peers);
    }
    __syncthreads();
    {  // thread t owns digit t: exclusive prefix over warps, then advance
      uint32_t run = running[t];
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wc[w][t];
        wc[w][t] = run;
        run += c;
      }
      running[t] = run;
    }
    __syncthreads();
    if (live) {
      const uint32_t pos = wc[warp][d] + rank;
      for (uint32_t w = 0; w < words; ++w) key_out.w[w][pos] = kv[w];
      val_out[pos] = vv;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------- lcp ---
__global__ void lcp_kernel(KeyWords key, uint32_t k, uint32_t words, uint32_t fields,
                           uint32_t bits, int32_t *__restrict__ L) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j + 1 >= k) return;
  uint32_t same = fields;
  for (uint32_t w = 0; w < words; ++w) {
    const uint64_t x = key.w[w][j] ^ key.w[w][j + 1];
    if (x) {
      same = (w * 64 + (uint32_t)__clzll((long long)x)) / bits;
      break;
    }
  }
  L[j] = (int32_t)min(same, fields);
}

// ------------------------------------------------- nearest smaller values ---
// Levels of a 32-ary tree of minima over L (level 0 = L itself).
struct MinTree {
  int32_t *lvl[8];
  uint32_t len[8];
  int levels;
};

__global__ void min_level_kernel(const int32_t *__restrict__ in, uint32_t n,
                                 int32_t *__restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t m = (n + 31) / 32;
  if (i >= m) return;
  int32_t v = INT32_MAX;
  for (uint32_t q = i * 32; q < min(n, i * 32 + 32); ++q) v = min(v, in[q]);
  out[i] = v;
}

// Nearest index q < j (dir < 0) or q > j (dir > 0) with L[q] < x, or -1.
__device__ int32_t nearest_below(const MinTree &mt, uint32_t j, int32_t x, int dir) {
  int level = 0;
  int64_t cur = j;  // exclusive bound at the current level
  int64_t found = -1;
  while (true) {
    const int32_t *a = mt.lvl[level];
    const int64_t n = mt.len[level];
    if (dir < 0) {
      const int64_t start = (cur / 32) * 32;
      for (int64_t q = cur - 1; q >= start; --q)
        if (a[q] < x) { found = q; break; }
      if (found >= 0 || start == 0 || level + 1 >= mt.levels) break;
      cur = start / 32;
    } else {
      const int64_t end = n < (cur / 32) * 32 + 32 ? n : (cur / 32) * 32 + 32;
      for (int64_t q = cur + 1; q < end; ++q)
        if (a[q] < x) { found = q; break; }
      if (found >= 0 || end >= n || level + 1 >= mt.levels) break;
      cur = end / 32 - 1;
      // the next level is searched strictly after index cur (this block)
    }
    ++level;
  }
  if (found < 0) return -1;
  while (level > 0) {  // descend into the block that holds the minimum
    --level;
    const int32_t *a = mt.lvl[level];
    const int64_t n = mt.len[level];
    const int64_t lo = found * 32, hi = n < lo + 32 ? n : lo + 32;
    int64_t pick = -1;
    if (dir < 0) {
      for (int64_t q = hi - 1; q >= lo; --q)
        if (a[q] < x) { pick = q; break; }
    } else {
      for (int64_t q = lo; q < hi; ++q)
        if (a[q] < x) { pick = q; break; }
    }
    found = pick;
  }
  return (int32_t)found;
}

// For each lcp position: PS (previous strictly smaller), NS (next strictly
// smaller) and the interval link (previous position with an equal value
// and only larger ones between, else itself).
__global__ void smaller_values_kernel(MinTree mt, uint32_t n, int32_t *__restrict__ ps,
                                      int32_t *__restrict__ ns, int32_t *__restrict__ link) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int32_t v = mt.lvl[0][j];
  ps[j] = nearest_below(mt, j, v, -1);
  ns[j] = nearest_below(mt, j, v, +1);
  const int32_t pse = nearest_below(mt, j, v + 1, -1);  // previous smaller-or-equal
  link[j] = (pse >= 0 && mt.lvl[0][pse] == v) ? pse : (int32_t)j;
}

__global__ void jump_kernel(const int32_t *__restrict__ in, uint32_t n,
                            int32_t *__restrict__ out) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = in[in[j]];
}

__global__ void rep_flags_kernel(const int32_t *__restrict__ L, const int32_t *__restrict__ rep,
                                 uint32_t n, uint32_t *__restrict__ flag) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) flag[j] = (rep[j] == (int32_t)j && L[j] >= 1) ? 1u : 0u;
}

// Node ids: 0 the root, 1 + id[j] the interval named by position j, then the
// leaves in sorted order.
__global__ void internal_nodes_kernel(const int32_t *__restrict__ L,
                                      const int32_t *__restrict__ rep,
                                      const int32_t *__restrict__ ps,
                                      const int32_t *__restrict__ ns,
                                      const uint32_t *__restrict__ id, uint32_t n,
                                      const int64_t *__restrict__ times,
                                      int64_t *__restrict__ parent, int64_t *__restrict__ time) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || rep[j] != (int32_t)j || L[j] < 1) return;
  const uint32_t node = 1 + id[j];
  const int32_t a = ps[j], b = ns[j];
  const int32_t La = a >= 0 ? L[a] : -1, Lb = b >= 0 ? L[b] : -1;
  int64_t par = 0;
  if (La > 0 || Lb > 0) par = 1 + id[rep[La >= Lb ? a : b]];
  parent[node] = par;
  time[node] = times[L[j] - 1];
}

__global__ void leaves_kernel(const int32_t *__restrict__ L, const int32_t *__restrict__ rep,
                              const uint32_t *__restrict__ id, const uint32_t *__restrict__ val,
                              uint32_t k, uint32_t internal, int64_t T,
                              int64_t *__restrict__ parent, int64_t *__restrict__ time,
                              uint32_t *__restrict__ leaf_of_sample) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= k) return;
  const int32_t La = p >= 1 ? L[p - 1] : -1, Lb = p + 1 < k ? L[p] : -1;
  int64_t par = 0;
  if (La > 0 || Lb > 0) par = 1 + id[rep[La >= Lb ? p - 1 : p]];
  const uint32_t node = 1 + internal + p;
  parent[node] = par;
  time[node] = T;
  leaf_of_sample[val[p]] = node;
}

__global__ void root_kernel(int64_t *__restrict__ parent, int64_t *__restrict__ time) {
  parent[0] = -1;
  time[0] = -1;
}

inline uint32_t blocks_for(uint64_t n, uint32_t threads) {
  return (uint32_t)((n + threads - 1) / threads);
}

}  // namespace
}  // namespace hsga

using namespace hsga;

int hsga_reconstruct(const uint64_t *surf, uint32_t k, uint32_t surface_words, uint32_t policy,
                     uint32_t differentia_bits, uint32_t W, uint64_t generations,
                     uint32_t deposit_interval,
                     int64_t *parent_out, int64_t *time_out, uint32_t *leaf_of_sample,
                     uint32_t capacity, uint32_t *n_nodes, void *cuda_stream) {
  const uint32_t b = differentia_bits;
  if (!surf || !parent_out || !time_out || !leaf_of_sample || !n_nodes) return HSGA_ERR_INVALID_ARG;
  const uint32_t K = surface_words > 1 ? surface_words : 1;
  if (k == 0 || k > (1u << 28) || !(b == 1 || b == 2 || b == 4 || b == 8 || b == 16))
    return HSGA_ERR_INVALID_ARG;
  if (!(K == 1 || K == 2 || K == 4)) return HSGA_ERR_INVALID_ARG;
  if (policy > HSGA_HYBRID || policy == HSGA_NONE) return HSGA_ERR_INVALID_ARG;
  const uint64_t need_nodes = 2ull * k + 1;
  if (capacity < need_nodes) return HSGA_ERR_INVALID_ARG;
  if (stream_capturing((cudaStream_t)cuda_stream)) return HSGA_ERR_NOT_CAPTURABLE;
  // retained deposition times in ascending order (the same for every sample)
  const uint32_t S = 64 * K / b;
  const uint64_t kk = deposit_interval > 1 ? deposit_interval : 1;
  const uint64_t T = (generations + kk - 1) / kk;
  std::vector<int64_t> dep(S);
  if (hsga_lookup(policy, S, W, T, dep.data()) != HSGA_OK) return HSGA_ERR_INVALID_ARG;
  std::vector<uint32_t> order;
  for (uint32_t s = 0; s < S; ++s)
    if (dep[s] >= 0) order.push_back(s);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t x, uint32_t y) { return dep[x] < dep[y]; });
  KeyPlan kp{};
  kp.fields = (uint32_t)order.size();
  kp.bits = b;
  kp.words = K;
  std::vector<int64_t> times(kp.fields > 0 ? kp.fields : 1, -1);
  for (uint32_t j = 0; j < kp.fields; ++j) {
    kp.src[j] = order[j] * b;
    times[j] = dep[order[j]] * (int64_t)kk;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  AllocHooks al = current_allocator();
  const uint32_t nblocks = blocks_for(k, kSortTile);
  const uint32_t n = k - 1;  // lcp positions
  // scratch
  std::vector<void *> held;
  auto alloc = [&](size_t bytes) {
    void *p = device_alloc(al, bytes < 256 ? 256 : bytes, st);
    held.push_back(p);
    return p;
  };
  KeyWords key[2] = {};
  for (int h = 0; h < 2; ++h)
    for (uint32_t w = 0; w < K; ++w) key[h].w[w] = (uint64_t *)alloc(8ull * k);
  uint32_t *val[2] = {(uint32_t *)alloc(4ull * k), (uint32_t *)alloc(4ull * k)};
  uint32_t *hist = (uint32_t *)alloc(4ull * 256 * nblocks);
  uint64_t *dsurf = (uint64_t *)alloc(8ull * k * K);
  int64_t *dtimes = (int64_t *)alloc(8ull * times.size());
  int32_t *L = (int32_t *)alloc(4ull * (n + 1));
  int32_t *ps = (int32_t *)alloc(4ull * (n + 1));
  int32_t *ns = (int32_t *)alloc(4ull * (n + 1));
  int32_t *link[2] = {(int32_t *)alloc(4ull * (n + 1)), (int32_t *)alloc(4ull * (n + 1))};
  uint32_t *id = (uint32_t *)alloc(4ull * (n + 1));
  uint32_t *total = (uint32_t *)alloc(4);
  const bool dev_out = device_pointer(parent_out);
  int64_t *dparent = dev_out ? parent_out : (int64_t *)alloc(8 * need_nodes);
  int64_t *dtime = dev_out ? time_out : (int64_t *)alloc(8 * need_nodes);
  uint32_t *dleaf = dev_out ? leaf_of_sample : (uint32_t *)alloc(4ull * k);
  MinTree mt{};
  {
    uint32_t len = n;
    mt.lvl[0] = L;
    mt.len[0] = len;
    mt.levels = 1;
    while (len > 32 && mt.levels < 8) {
      len = (len + 31) / 32;
      mt.lvl[mt.levels] = (int32_t *)alloc(4ull * len);
      mt.len[mt.levels] = len;
      ++mt.levels;
    }
  }
  int status = HSGA_OK;
  for (void *p : held)
    if (!p) status = HSGA_ERR_OOM;
  cudaError_t e = cudaSuccess;
  uint32_t internal = 0;
  if (status == HSGA_OK) {
    e = cudaMemcpyAsync(dsurf, surf, 8ull * k * K, cudaMemcpyDefault, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dtimes, times.data(), 8 * times.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      make_keys_kernel<<<blocks_for(k, 256), 256, 0, st>>>(kp, dsurf, k, key[0], val[0]);
      // sort over the significant bits only (the top fields * bits, rounded
      // up to whole 8-bit digits, which then never straddle two key words)
      const uint32_t passes = (kp.fields * b + 7) / 8;
      int cur = 0;
      for (uint32_t ps_i = 0; ps_i < passes; ++ps_i) {
        const uint32_t top = 8 * (passes - 1 - ps_i);  // digit's first bit from the top
        const uint32_t dword = top / 64, shift = 64 - top % 64 - 8;
        digit_histogram_kernel<<<nblocks, kSortThreads, 0, st>>>(key[cur].w[dword], k, shift,
                                                                 nblocks, hist);
        exclusive_scan_kernel<<<1, 1024, 0, st>>>(hist, 256 * nblocks, nullptr);
        digit_scatter_kernel<<<nblocks, kSortThreads, 0, st>>>(key[cur], val[cur], k, K, dword,
                                                               shift, nblocks, hist,
                                                               key[1 - cur], val[1 - cur]);
        cur = 1 - cur;
      }
      root_kernel<<<1, 1, 0, st>>>(dparent, dtime);
      if (n > 0) {
        lcp_kernel<<<blocks_for(n, 256), 256, 0, st>>>(key[cur], k, K, kp.fields, b, L);
        for (int l = 1; l < mt.levels; ++l)
          min_level_kernel<<<blocks_for(mt.len[l], 256), 256, 0, st>>>(mt.lvl[l - 1],
                                                                       mt.len[l - 1], mt.lvl[l]);
        smaller_values_kernel<<<blocks_for(n, 256), 256, 0, st>>>(mt, n, ps, ns, link[0]);
        int lc = 0;
        for (uint32_t span = 1; span < n; span <<= 1) {
          jump_kernel<<<blocks_for(n, 256), 256, 0, st>>>(link[lc], n, link[1 - lc]);
          lc = 1 - lc;
        }
        rep_flags_kernel<<<blocks_for(n, 256), 256, 0, st>>>(L, link[lc], n, id);
        exclusive_scan_kernel<<<1, 1024, 0, st>>>(id, n, total);
        e = cudaMemcpyAsync(&internal, total, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
          internal_nodes_kernel<<<blocks_for(n, 256), 256, 0, st>>>(L, link[lc], ps, ns, id, n,
                                                                    dtimes, dparent, dtime);
          leaves_kernel<<<blocks_for(k, 256), 256, 0, st>>>(L, link[lc], id, val[cur], k,
                                                            internal, (int64_t)generations,
                                                            dparent, dtime, dleaf);
        }
      } else {
        leaves_kernel<<<1, 32, 0, st>>>(L, link[0], id, val[cur], k, 0, (int64_t)generations,
                                        dparent, dtime, dleaf);
      }
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    const uint32_t nodes = 1 + internal + k;
    if (e == cudaSuccess && !dev_out) {
      e = cudaMemcpyAsync(parent_out, dparent, 8ull * nodes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(time_out, dtime, 8ull * nodes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(leaf_of_sample, dleaf, 4ull * k, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = HSGA_ERR_CUDA;
    *n_nodes = nodes;
  }
  for (void *p : held)
    if (p) device_free(al, p, st);
  cudaStreamSynchronize(st);
  return status;
}
