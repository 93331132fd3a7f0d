"""Post-hoc phylogenetic analysis for the oracle: pedigree MRCA, surface MRCA
bounds, trie reconstruction and phylometrics.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Concepts from arXiv 2404.10861, section "Distributed Phylogenetic Tracking":
every generation along a lineage appends one differentia; the first
mismatching differentia between two genomes bounds their common ancestry
from above, and a trie over the differentia sequences is the reconstruction.
The trie here is this project's own simple version (the paper's
agglomerative-trie algorithm lives in another paper):

* all sampled genomes share the deposition count T (synchronous mode), so
  they share the list of retained deposition times, given by the oracle's
  timestamp lookup;
* a genome is its differentiae in ascending deposition time; a trie node is
  (time, value); the root sits at time -1 and leaves at time T;
* unifurcations are collapsed; branch lengths are differences in time.

Genomes of free-running runs carry their own deposition counts, so their
retained times differ; for those, two genomes are compared on the times both
retain (ascending), and the last match before the first mismatch bounds
their common ancestry as before (the pairwise form of the same method).

Phylometrics (the on-hardware trial compares sum branch length and mean
evolutionary distinctiveness between purifying-only and adaptive treatments):

* sum branch length: total edge length;
* mean pairwise distance: mean path length over leaf pairs;
* Sackin: sum over leaves of the number of internal nodes on the root path;
* Colless, generalised to polytomies: sum over internal nodes of
  (largest - smallest child leaf count);
* evolutionary distinctiveness (fair proportion): per leaf, the sum over the
  edges on its root path of edge length / leaves below the edge.
"""
from __future__ import annotations

import numpy as np

from . import lookup


# ------------------------------------------------------------ pedigree ---

def lineage(parents: np.ndarray, agent: int) -> np.ndarray:
    """Ancestor indices a_g for g = 0..G of ``agent`` at generation G
    (a_G = agent; a_g = parents[g][a_{g+1}])."""
    G = parents.shape[0]
    out = np.zeros(G + 1, dtype=np.int64)
    out[G] = agent
    for g in range(G - 1, -1, -1):
        out[g] = int(parents[g, out[g + 1]])
    return out


def true_mrca_generation(parents: np.ndarray, x: int, y: int) -> int:
    """Largest g at which the lineages of x and y share one agent at the start
    of generation g, or 0 when they never do (different founders).  Every
    differentia deposited before that generation is shared; every one from it
    on was drawn independently by each lineage."""
    lx, ly = lineage(parents, x), lineage(parents, y)
    same = np.nonzero(lx == ly)[0]
    return int(same.max()) if len(same) else 0


# ------------------------------------------------------------- surfaces ---

def differentiae(surf: np.ndarray, bits: int, words: int = 1) -> np.ndarray:
    """(k, S) matrix of differentia values in site order, S = 64 words / bits;
    surf holds k genomes of `words` 64-bit words (agent-major), site s in bits
    [s b mod 64, s b mod 64 + b) of word floor(s b / 64)."""
    surf = np.asarray(surf, dtype=np.uint64).reshape(-1, words)
    S = 64 * words // bits
    site = np.arange(S)
    word = site * bits // 64
    shifts = (site * bits % 64).astype(np.uint64)
    mask = np.uint64((1 << bits) - 1)
    return ((surf[:, word] >> shifts[None, :]) & mask).astype(np.int64)


def retained_order(policy: int, S: int, W: int, T: int, coarsen: int = 1):
    """Sites holding a differentia after T generations, in ascending
    deposition time, and those times in generations.  With temporal
    coarsening k the generations 0, k, 2k, ... deposit, so after T
    generations ceil(T / k) depositions exist and deposition t is generation
    t k."""
    k = max(1, coarsen)
    times = lookup(policy, S, W, -(-T // k)) * k
    times[times < 0] = -1
    sites = np.nonzero(times >= 0)[0]
    order = sites[np.argsort(times[sites], kind="stable")]
    return order, times[order]


def retained_times(policy: int, S: int, W: int, T: int, coarsen: int = 1) -> np.ndarray:
    """Per site, the generation whose differentia it holds after T
    generations (-1 if empty)."""
    key = (policy, S, W, T, coarsen)
    if key not in _RETAINED:
        k = max(1, coarsen)
        times = lookup(policy, S, W, -(-T // k)) * k
        times[times < 0] = -1
        if len(_RETAINED) > 4096:
            _RETAINED.clear()
        _RETAINED[key] = times
    return _RETAINED[key].copy()


_RETAINED: dict = {}


def mrca_bounds_mixed(sa: int, Ta: int, sb: int, Tb: int, policy: int, bits: int, W: int,
                      coarsen: int = 1):
    """Two surfaces with their own generation counts: (t_prev, t_star) over
    the generations both still retain, in ascending order -- t_star the first
    at which their differentiae differ (None if none does), t_prev the last
    common retained generation before it (-1 if none).  Common ancestry ends
    at or before t_star."""
    S = 64 // bits
    d = differentiae(np.array([sa, sb], dtype=np.uint64), bits)
    va = {int(t): int(d[0, i]) for i, t in enumerate(retained_times(policy, S, W, Ta, coarsen))
          if t >= 0}
    vb = {int(t): int(d[1, i]) for i, t in enumerate(retained_times(policy, S, W, Tb, coarsen))
          if t >= 0}
    prev = -1
    for t in sorted(set(va) & set(vb)):
        if va[t] != vb[t]:
            return prev, t
        prev = t
    return prev, None


def mean_pairwise_distance_mixed(surf, T, policy: int, bits: int, W: int, pairs: int,
                                 rng, coarsen: int = 1) -> float:
    """Mean over `pairs` random pairs of (Ta - m) + (Tb - m), m = t_prev of
    mrca_bounds_mixed: the path length through the estimated common
    ancestor, as in the trie (whose branching node sits at t_prev)."""
    surf = np.asarray(surf, dtype=np.uint64)
    T = np.asarray(T, dtype=np.int64)
    total = 0
    for _ in range(pairs):
        a, b = rng.choice(len(surf), size=2, replace=False)
        m, _ = mrca_bounds_mixed(int(surf[a]), int(T[a]), int(surf[b]), int(T[b]), policy,
                                 bits, W, coarsen)
        total += int(T[a]) + int(T[b]) - 2 * m
    return total / pairs


def mrca_bounds(da: np.ndarray, db: np.ndarray, times: np.ndarray):
    """For two genomes' differentiae (already in time order) with deposition
    times ``times``: (t_prev, t_star) where t_star is the first mismatching
    retained time (None if all match) and t_prev the last retained time before
    it (-1 if none).  Common ancestry ends at or before t_star."""
    mism = np.nonzero(da != db)[0]
    if len(mism) == 0:
        return (int(times[-1]) if len(times) else -1), None
    i = int(mism[0])
    return (int(times[i - 1]) if i > 0 else -1), int(times[i])


# ------------------------------------------------------- reconstruction ---

class Tree:
    """Rooted tree: parent index per node (-1 for the root), node times, and
    which nodes are leaves (one per sampled genome, in sample order)."""

    def __init__(self, parent, time, leaf_of_sample):
        self.parent = np.asarray(parent, dtype=np.int64)
        self.time = np.asarray(time, dtype=np.int64)
        self.leaf_of_sample = np.asarray(leaf_of_sample, dtype=np.int64)

    @property
    def n_nodes(self):
        return len(self.parent)

    def children(self):
        ch = [[] for _ in range(self.n_nodes)]
        for v, p in enumerate(self.parent):
            if p >= 0:
                ch[p].append(v)
        return ch


def reconstruct(surf: np.ndarray, policy: int, bits: int, W: int, T: int,
                coarsen: int = 1, words: int = 1) -> Tree:
    """Trie reconstruction from sampled surfaces (of `words` 64-bit words
    each) that all elapsed T generations."""
    S = 64 * words // bits
    order, times = retained_order(policy, S, W, T, coarsen)
    D = differentiae(surf, bits, words)[:, order]
    parent, time = [-1], [-1]
    kids = [dict()]  # per node: value -> child node
    leaf_of_sample = []
    for row in D:
        node = 0
        for t, v in zip(times, row):
            nxt = kids[node].get(int(v))
            if nxt is None:
                nxt = len(parent)
                parent.append(node)
                time.append(int(t))
                kids.append(dict())
                kids[node][int(v)] = nxt
            node = nxt
        leaf = len(parent)
        parent.append(node)
        time.append(int(T))
        kids.append(dict())
        leaf_of_sample.append(leaf)
    return collapse(Tree(parent, time, leaf_of_sample))


def collapse(tree: Tree) -> Tree:
    """Remove internal non-root nodes with exactly one child (their edges
    merge; total length is unchanged)."""
    ch = tree.children()
    leaves = set(int(x) for x in tree.leaf_of_sample)
    keep = [v for v in range(tree.n_nodes)
            if v == 0 or v in leaves or len(ch[v]) != 1]
    new_id = {v: i for i, v in enumerate(keep)}

    def kept_ancestor(v):
        p = tree.parent[v]
        while p != 0 and p not in new_id:
            p = tree.parent[p]
        return p

    parent = [-1 if v == 0 else new_id[kept_ancestor(v)] for v in keep]
    time = [int(tree.time[v]) for v in keep]
    return Tree(parent, time, [new_id[int(x)] for x in tree.leaf_of_sample])


# --------------------------------------------------------- phylometrics ---

def _leaf_counts(tree: Tree):
    ch = tree.children()
    leaves = set(int(x) for x in tree.leaf_of_sample)
    count = np.zeros(tree.n_nodes, dtype=np.int64)
    # parents always precede children in construction order
    for v in range(tree.n_nodes - 1, -1, -1):
        count[v] += 1 if v in leaves else 0
        if tree.parent[v] >= 0:
            count[tree.parent[v]] += count[v]
    return count, ch, leaves


def sum_branch_length(tree: Tree) -> float:
    p = tree.parent
    m = p >= 0
    return float((tree.time[m] - tree.time[p[m]]).sum())


def mean_pairwise_distance(tree: Tree) -> float:
    """Each edge lies on the path of every pair split by it:
    sum = sum_edges length * k (N - k), over N (N - 1) / 2 pairs."""
    count, _, _ = _leaf_counts(tree)
    N = len(tree.leaf_of_sample)
    if N < 2:
        return 0.0
    p = tree.parent
    m = p >= 0
    length = tree.time[m] - tree.time[p[m]]
    k = count[m]
    return float((length * k * (N - k)).sum() / (N * (N - 1) / 2))


def pairwise_distance(tree: Tree, a: int, b: int) -> int:
    """Path length between the leaves of samples a and b (brute force)."""
    def path(v):
        out = [v]
        while tree.parent[out[-1]] >= 0:
            out.append(int(tree.parent[out[-1]]))
        return out
    pa = path(int(tree.leaf_of_sample[a]))
    pb = set(path(int(tree.leaf_of_sample[b])))
    lca = next(v for v in pa if v in pb)
    ta = tree.time[tree.leaf_of_sample[a]]
    tb = tree.time[tree.leaf_of_sample[b]]
    return int(ta + tb - 2 * tree.time[lca])


def sackin(tree: Tree) -> int:
    _, ch, leaves = _leaf_counts(tree)
    total = 0
    for leaf in tree.leaf_of_sample:
        v = int(tree.parent[leaf])
        while v >= 0:
            total += 1
            v = int(tree.parent[v])
    return total


def colless(tree: Tree) -> int:
    count, ch, leaves = _leaf_counts(tree)
    total = 0
    for v in range(tree.n_nodes):
        if ch[v]:
            c = [int(count[u]) for u in ch[v]]
            total += max(c) - min(c)
    return total


def evolutionary_distinctiveness(tree: Tree) -> np.ndarray:
    count, _, _ = _leaf_counts(tree)
    out = np.zeros(len(tree.leaf_of_sample))
    for i, leaf in enumerate(tree.leaf_of_sample):
        v = int(leaf)
        while tree.parent[v] >= 0:
            p = int(tree.parent[v])
            out[i] += (tree.time[v] - tree.time[p]) / count[v]
            v = p
    return out


def phylometrics(tree: Tree) -> dict:
    ed = evolutionary_distinctiveness(tree)
    return {"sum_branch_length": sum_branch_length(tree),
            "mean_pairwise_distance": mean_pairwise_distance(tree),
            "mean_evolutionary_distinctiveness": float(ed.mean()) if len(ed) else 0.0,
            "sackin": sackin(tree),
            "colless": colless(tree)}
