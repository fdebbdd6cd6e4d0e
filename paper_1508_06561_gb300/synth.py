"""Seeded synthetic workloads shaped like the paper's database search.

The paper searches UniProt-SwissProt (547,085 sequences, Sec. III.B.5); that
dataset is not available here, so every workload is synthetic: residues drawn
i.i.d. over the 20 amino acids at background frequencies, lengths lognormal.
This module only draws random inputs.  It holds none of the method's
arithmetic and is the one module that both the GPU path's tests/benchmark and
the CPU oracle consume.

Codes follow the 24-letter BLOSUM62 order ``ARNDCQEGHILKMFPSTWYVBZX*``; the
generators only emit the 20 amino acids (codes 0..19).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LETTERS = "ARNDCQEGHILKMFPSTWYVBZX*"

# Amino-acid background composition of Robinson & Robinson, PNAS 88:8880
# (1991), in the order A R N D C Q E G H I L K M F P S T W Y V.
_ROBINSON = np.array([
    0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377, 0.02199, 0.05142,
    0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120, 0.05841, 0.01330, 0.03216, 0.06441])
BACKGROUND = _ROBINSON / _ROBINSON.sum()


def residues(rng: np.random.Generator, n: int) -> np.ndarray:
    """n residue codes (uint8, 0..19) drawn i.i.d. at background frequencies."""
    cdf = np.cumsum(BACKGROUND)
    cdf[-1] = 1.0
    out = np.empty(n, dtype=np.uint8)
    step = 1 << 24
    for s in range(0, n, step):
        m = min(step, n - s)
        out[s:s + m] = np.searchsorted(cdf, rng.random(m), side="right")
    return out


def lognormal_lengths(rng, n, median, sigma, lo, hi) -> np.ndarray:
    x = np.exp(np.log(median) + sigma * rng.standard_normal(n))
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def offsets_from_lengths(lengths) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


@dataclass
class Database:
    codes: np.ndarray          # uint8 [R]
    offsets: np.ndarray        # int64 [N+1]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def residues(self) -> int:
        return int(self.offsets[-1])

    def seq(self, i) -> np.ndarray:
        return self.codes[self.offsets[i]:self.offsets[i + 1]]

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)


def db_from_lengths(rng, lengths, name="") -> Database:
    lengths = np.asarray(lengths, dtype=np.int64)
    off = offsets_from_lengths(lengths)
    return Database(residues(rng, int(off[-1])), off, name)


# ---------------------------------------------------------------------------
# The five workloads.  Sizes follow the paper's database (Sec. III.B.5):
# ~570k sequences, ~205M residues, lognormal lengths with median 300.
# ---------------------------------------------------------------------------

def plain_small(seed: int = 0):
    """Plain single query: 64-residue query, 2,000 targets, lengths lognormal
    (median 300, sigma 0.6) clamped to [30, 2000]; top-10."""
    rng = np.random.default_rng(seed)
    lengths = lognormal_lengths(rng, 2000, 300, 0.6, 30, 2000)
    db = db_from_lengths(rng, lengths, "plain-q64-2k")
    q = residues(rng, 64)
    return db, q, 10


def swissprot_like(seed: int = 2, n: int = 570_000, sigma: float = 0.6) -> Database:
    """~570k targets / ~205M residues: lognormal lengths (median 300) clamped
    to [30, 35000], with a real long tail: 1e-4 of the sequences are redrawn
    log-uniform in [5000, 35000] and one is exactly 35,000 long."""
    rng = np.random.default_rng(seed)
    lengths = lognormal_lengths(rng, n, 300, sigma, 30, 35_000)
    ntail = max(1, int(round(n * 1e-4)))
    pos = rng.choice(n, size=ntail, replace=False)
    lengths[pos] = np.rint(np.exp(rng.uniform(np.log(5000), np.log(35_000), ntail))).astype(np.int64)
    lengths[pos[0]] = 35_000
    return db_from_lengths(rng, lengths, "swissprot-like-%dk" % (n // 1000))


def plain_large(seed_db: int = 2, seed_q: int = 2, n: int = 570_000):
    """Plain single query at database scale: a 256-residue query against the
    ~205M-residue SwissProt-like database; top-100."""
    db = swissprot_like(seed_db, n)
    q = residues(np.random.default_rng(1_000_003 + seed_q), 256)
    return db, q, 100


def mutate_homolog(rng, core: np.ndarray, identity: float, indel_rate: float = 1 / 40) -> np.ndarray:
    """A distant homolog of `core`: each position kept with probability
    `identity`, else substituted by a different background residue; indels
    at `indel_rate` per residue (half insertions, half deletions), lengths
    uniform in [1, 10]."""
    out = []
    i = 0
    n = len(core)
    while i < n:
        if rng.random() < indel_rate:
            ln = int(rng.integers(1, 11))
            if rng.random() < 0.5:
                out.extend(residues(rng, ln).tolist())
            else:
                i += ln
                continue
        if i >= n:
            break
        a = int(core[i])
        if rng.random() >= identity:
            while True:
                b = int(residues(rng, 1)[0])
                if b != a:
                    break
            a = b
        out.append(a)
        i += 1
    if not out:
        out = residues(rng, 1).tolist()
    return np.array(out, dtype=np.uint8)


def batched_homologs(seed: int = 3, n: int = 570_000, nq: int = 64, nplant: int = 500):
    """64 queries (lengths uniform in [30, 1000]) against the SwissProt-like
    database in which `nplant` sequences are replaced by planted distant
    homologs (query copies at 20-40% identity with indels), each embedded at
    a random offset in background flanks.  Returns (db, queries, planted)
    where planted maps database index -> query index."""
    rng = np.random.default_rng(seed)
    queries = [residues(rng, int(rng.integers(30, 1001))) for _ in range(nq)]
    base = swissprot_like(2, n)
    lengths = base.lengths().copy()
    slots = np.sort(rng.choice(n, size=nplant, replace=False))
    planted = {}
    seqs = {}
    for j, d in enumerate(slots):
        qi = j % nq
        core = mutate_homolog(rng, queries[qi], float(rng.uniform(0.2, 0.4)))
        total = max(len(core), int(lognormal_lengths(rng, 1, 300, 0.6, 30, 35_000)[0]))
        left = int(rng.integers(0, total - len(core) + 1))
        s = np.concatenate([residues(rng, left), core, residues(rng, total - len(core) - left)])
        seqs[int(d)] = s
        planted[int(d)] = qi
        lengths[d] = len(s)
    off = offsets_from_lengths(lengths)
    codes = np.empty(int(off[-1]), dtype=np.uint8)
    # copy the unchanged sequences in one gather, then write the planted ones
    keep = np.ones(n, dtype=bool)
    keep[slots] = False
    mask = np.repeat(keep, lengths)
    shift = np.repeat(base.offsets[:-1] - off[:-1], lengths)
    pos = np.nonzero(mask)[0]
    codes[pos] = base.codes[pos + shift[pos]]
    for d, s in seqs.items():
        codes[off[d]:off[d + 1]] = s
    db = Database(codes, off, "swissprot-like-570k+%d-homologs" % nplant)
    return db, queries, planted


def bimodal(seed: int = 4):
    """Load-balance stress: 100k targets, 90% with lengths uniform in
    [50, 150] and 10% uniform in [5000, 35000] (~209M residues); 16 queries
    of lengths 6x50, 5x500, 5x2000; top-50."""
    rng = np.random.default_rng(seed)
    n = 100_000
    long_ = rng.random(n) < 0.1
    lengths = np.where(long_, rng.integers(5000, 35_001, n), rng.integers(50, 151, n)).astype(np.int64)
    db = db_from_lengths(rng, lengths, "bimodal-100k")
    queries = [residues(rng, L) for L in [50] * 6 + [500] * 5 + [2000] * 5]
    return db, queries, 50


def serving_stream(seed: int = 5, n: int = 10_000, rate: float = 200.0):
    """Poisson arrivals at `rate` requests/s; query lengths lognormal
    (median 250, sigma 0.6) clamped to [20, 2000]; one seed per request.
    Returns (arrival_times_s, queries, seeds)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps)
    lens = lognormal_lengths(rng, n, 250, 0.6, 20, 2000)
    queries = [residues(rng, int(L)) for L in lens]
    seeds = rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64)
    return t, queries, seeds


def random_symmetric_matrix(rng, lo: int = -4, hi: int = 11) -> np.ndarray:
    """A random symmetric 24x24 int8 matrix with entries in [lo, hi]."""
    a = rng.integers(lo, hi + 1, size=(24, 24))
    a = np.triu(a) + np.triu(a, 1).T
    return a.astype(np.int8)
