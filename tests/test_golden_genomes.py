"""The paper's printed example genomes (Supplemental Material, "Example
genomes sampled after validation experiment completion"; fixture in
tests/golden/example_genomes.txt) against the readings they bear on:

* free-running genomes carry their own generation counters (here 121, 117
  and 101 after one run), which is why the free-running kernels and the
  oracle's replay keep a counter per genome and deposit at the genome's own
  count;
* genomes of one founding lineage share more surface bits than genomes of
  different lineages (47 of 64 against 28 and 31 here); the oracle's
  surfaces show the same ordering for relatives and non-relatives.
"""
import os

import numpy as np

from paper_2404_10861_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "example_genomes.txt")


def load():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, *hexes = line.split()
        out[name] = bytes(int(h, 16) for h in hexes)
    return out


def agree(a: bytes, b: bytes) -> int:
    x = int.from_bytes(a, "little") ^ int.from_bytes(b, "little")
    return 64 - bin(x).count("1")


def test_printed_genomes_carry_their_own_counters():
    g = load()
    assert all(len(v) == 12 for v in g.values())
    counters = [int.from_bytes(g[k][2:4], "little") for k in ("genome0", "genome1", "genome2")]
    assert counters == [121, 117, 101]
    assert len(set(counters)) == 3          # one run, three different counts


def test_printed_lineage_shares_more_surface_bits():
    g = load()
    same = agree(g["genome0"][4:], g["genome1"][4:])
    cross = [agree(g["genome0"][4:], g["genome2"][4:]), agree(g["genome1"][4:], g["genome2"][4:])]
    assert g["genome0"][:2] == g["genome1"][:2] != g["genome2"][:2]
    assert (same, cross) == (47, [28, 31])
    assert same > max(cross)


def test_oracle_relatives_share_more_surface_bits(orc):
    """The same ordering in the oracle: from founders with independent random
    surfaces, after 121 generations genomes of one island (close relatives,
    descended from one founder) agree on more surface bits than genomes of
    islands that never exchanged migrants (unrelated: they agree by chance,
    on about half)."""
    c = orc.Config(rows=8, cols=8, n=16, tournament=2, policy=orc.TILTED, bits=1, W=2,
                   interval=0, seed=41)
    trait, surf = inputs.random_population(c.agents, seed=41, trait_max=0)
    _, surf, _ = orc.run(c, trait, surf, generations=121)
    s = surf.reshape(c.islands, c.n)
    pop = np.vectorize(lambda v: bin(int(v)).count("1"))
    within = np.mean([64 - pop(s[i, 0] ^ s[i, 1:]).mean() for i in range(c.islands)])
    across = np.mean([64 - pop(s[i, 0] ^ s[(i + 27) % c.islands, 0]) for i in range(c.islands)])
    assert within > across + 8
