"""Seeded synthetic inputs for protein database search.

This module holds input data and input generators only: the BLOSUM62 table,
the background amino-acid frequencies residues are drawn from, the length
distributions of queries and database sequences, and the named workloads.
It contains none of the alignment arithmetic; both the CPU oracle and the
CUDA path consume what it produces.

Stand-in for the paper's data (Section 4.1): 20 Swiss-Prot queries of
lengths 144..5478 searched against UniProtKB/Swiss-Prot 2021_04
(565,928 sequences, 204,173,280 residues, longest 35,213), BLOSUM62 with
gap penalties 10(2).  None of those sequences is reproduced here; every
residue is drawn i.i.d. from background frequencies with a seeded PRNG.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Residue order of the NCBI-distributed BLOSUM62 table (Henikoff & Henikoff
# 1992): the 20 standard amino acids, then B (D/N), Z (E/Q), X (any), '*'.
ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"
N_STANDARD = 20

_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0 -2 -1  0 -4
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3 -1  0 -1 -4
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3  3  0 -1 -4
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3  4  1 -1 -4
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1 -3 -3 -2 -4
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2  0  3 -1 -4
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3 -1 -2 -1 -4
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3  0  0 -1 -4
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3 -3 -3 -1 -4
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1 -4 -3 -1 -4
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2  0  1 -1 -4
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1 -3 -1 -1 -4
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1 -3 -3 -1 -4
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2 -2 -1 -2 -4
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2  0  0  0 -4
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0 -1 -1  0 -4
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3 -4 -3 -2 -4
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1 -3 -2 -1 -4
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4 -3 -2 -1 -4
-2 -1  3  4 -3  0  1 -1  0 -3 -4  0 -3 -3 -2  0 -1 -4 -3 -3  4  1 -1 -4
-1  0  0  1 -3  3  4 -2  0 -3 -3  1 -1 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -1 -1 -1 -2 -1 -1 -1 -1 -1 -1 -1 -1 -1 -2  0  0 -2 -1 -1 -1 -1 -1 -4
-4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4  1
"""


def blosum62() -> np.ndarray:
    """The 24x24 BLOSUM62 substitution matrix (int32, row-major, ALPHABET order).

    The paper scores with BLOSUM62 (Section 4.1, experimental design).
    """
    m = np.array(_BLOSUM62_ROWS.split(), dtype=np.int32).reshape(24, 24)
    return m


# Background amino-acid frequencies of Robinson & Robinson (1991), per mille,
# in ALPHABET order for the 20 standard residues (the set BLAST uses).
_ROBINSON_PER_MILLE = {
    "A": 78.05, "R": 51.29, "N": 44.87, "D": 53.64, "C": 19.25,
    "Q": 42.64, "E": 62.95, "G": 73.77, "H": 21.99, "I": 51.42,
    "L": 90.19, "K": 57.44, "M": 22.43, "F": 38.56, "P": 52.03,
    "S": 71.20, "T": 58.41, "W": 13.30, "Y": 32.16, "V": 64.41,
}


def background_freqs() -> np.ndarray:
    """Normalised background frequencies of the 20 standard residues."""
    f = np.array([_ROBINSON_PER_MILLE[a] for a in ALPHABET[:N_STANDARD]], dtype=np.float64)
    return f / f.sum()


def encode(seq: str) -> np.ndarray:
    """ASCII residues -> uint8 codes in ALPHABET order (unknown letters -> X)."""
    lut = np.full(256, ALPHABET.index("X"), dtype=np.uint8)
    for i, a in enumerate(ALPHABET):
        lut[ord(a)] = i
        lut[ord(a.lower())] = i
    return lut[np.frombuffer(seq.encode("ascii"), dtype=np.uint8)]


def decode(codes: np.ndarray) -> str:
    return "".join(ALPHABET[int(c)] for c in codes)


def _residue_lut() -> np.ndarray:
    """65,536-entry table mapping a uniform 16-bit integer to a residue code
    with the background frequencies (quantised to 1/65536)."""
    cdf = np.cumsum(background_freqs())
    cdf[-1] = 1.0
    u = (np.arange(65536, dtype=np.float64) + 0.5) / 65536.0
    return np.searchsorted(cdf, u, side="right").astype(np.uint8)


_LUT = None


def random_residues(rng: np.random.Generator, n: int, chunk: int = 1 << 26) -> np.ndarray:
    """n residues drawn i.i.d. from the background frequencies (uint8 codes 0..19),
    generated in chunks so that billions of residues need no float buffers."""
    global _LUT
    if n <= 0:
        return np.zeros(0, dtype=np.uint8)
    if _LUT is None:
        _LUT = _residue_lut()
    out = np.empty(n, dtype=np.uint8)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = _LUT[rng.integers(0, 65536, size=e - s, dtype=np.uint16)]
    return out


def lognormal_lengths(rng: np.random.Generator, count: int, mean: float,
                      lo: int, hi: int, sigma: float = 0.75) -> np.ndarray:
    """Lognormal lengths with the given arithmetic mean (before clipping).

    mu = ln(mean) - sigma^2/2 so that E[len] = mean for the unclipped law;
    the paper gives no spread, sigma = 0.75 is this build's reading.
    """
    mu = np.log(mean) - 0.5 * sigma * sigma
    x = rng.lognormal(mu, sigma, count)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def loguniform_lengths(rng: np.random.Generator, count: int, lo: float, hi: float) -> np.ndarray:
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), count))
    return np.clip(np.rint(x), int(np.ceil(lo)), int(hi)).astype(np.int64)


def geometric_grid(count: int, lo: int, hi: int) -> np.ndarray:
    """Deterministic log-uniform grid round(lo * (hi/lo)^(i/(count-1)))."""
    if count == 1:
        return np.array([lo], dtype=np.int64)
    i = np.arange(count, dtype=np.float64)
    return np.rint(lo * (hi / lo) ** (i / (count - 1))).astype(np.int64)


@dataclasses.dataclass
class SeqSet:
    """Sequences as one concatenated uint8 code array plus n+1 offsets."""
    residues: np.ndarray  # uint8
    offsets: np.ndarray   # int64, len n+1

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def seq(self, i: int) -> np.ndarray:
        return self.residues[self.offsets[i]:self.offsets[i + 1]]


def seqset_from_lengths(rng: np.random.Generator, lengths) -> SeqSet:
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    residues = random_residues(rng, int(offsets[-1]))
    return SeqSet(residues, offsets)


def seqset_from_list(seqs) -> SeqSet:
    seqs = [np.asarray(s, dtype=np.uint8) for s in seqs]
    lengths = np.array([len(s) for s in seqs], dtype=np.int64)
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    residues = np.concatenate(seqs) if seqs else np.zeros(0, dtype=np.uint8)
    return SeqSet(residues.astype(np.uint8), offsets)


@dataclasses.dataclass
class Workload:
    name: str
    queries: SeqSet
    db: SeqSet
    matrix: np.ndarray
    gap_open: int
    gap_extend: int
    top_k: int

    @property
    def cells(self) -> int:
        return int(self.queries.lengths.sum()) * int(self.db.lengths.sum())


SEED = 20220301

# Named workloads.  Sizes follow the paper's experiment (Section 4.1) and
# the larger cases the hot path is measured on.
# Serving: requests of lengths lognormal mean 400 (30..8000) against a large
# resident database (lognormal mean 360); the full size is 20M sequences, the
# benchmark runs a stated fraction of it.
SERVING_DB_SEQS = 20_000_000


def serving_database(seed: int = SEED, db_scale: float = 0.1) -> SeqSet:
    rng = np.random.default_rng(seed + 5)
    n = max(1, int(round(SERVING_DB_SEQS * db_scale)))
    return seqset_from_lengths(rng, lognormal_lengths(rng, n, 360.0, 2, 35_000))


def serving_requests(count: int, seed: int = SEED) -> SeqSet:
    rng = np.random.default_rng(seed + 6)
    return seqset_from_lengths(rng, lognormal_lengths(rng, count, 400.0, 30, 8000))


WORKLOADS = {
    "db2k_q100": "1 query of length 100 vs 2,000 sequences (lognormal mean 350, 20..1000)",
    "swissprot_like_20q": "20 queries 144..5478 (log grid) vs 565,000 sequences "
                          "(lognormal mean 360, 2..35,000, one of 35,000)",
    "long_4q_50k": "4 queries 5k/10k/20k/35k vs 50,000 sequences, 10% log-uniform in (3072, 35000]",
    "batched_512q": "512 queries uniform 50..5,000 vs the 565,000-sequence database",
}


def make_workload(name: str, seed: int = SEED, db_scale: float = 1.0, db: SeqSet | None = None) -> Workload:
    """Build a named workload.  db_scale < 1 shrinks the database count
    (used to make bounded samples of a workload; the full size is 1.0).
    For batched_512q, db may pass the already generated database of
    swissprot_like_20q (same seed and scale) instead of generating it again."""
    mat = blosum62()
    if name == "db2k_q100":
        rng = np.random.default_rng(seed + 1)
        n = max(1, int(round(2000 * db_scale)))
        db = seqset_from_lengths(rng, lognormal_lengths(rng, n, 350.0, 20, 1000))
        q = seqset_from_lengths(rng, [100])
        return Workload(name, q, db, mat, 10, 1, 10)
    if name == "swissprot_like_20q":
        rng = np.random.default_rng(seed + 2)
        n = max(1, int(round(565_000 * db_scale)))
        lens = lognormal_lengths(rng, n, 360.0, 2, 35_000)
        lens[rng.integers(0, n)] = 35_000  # the database's longest entry
        db = seqset_from_lengths(rng, lens)
        q = seqset_from_lengths(rng, geometric_grid(20, 144, 5478))
        return Workload(name, q, db, mat, 10, 1, 10)
    if name == "long_4q_50k":
        rng = np.random.default_rng(seed + 3)
        n = max(10, int(round(50_000 * db_scale)))
        n_long = n // 10
        short = lognormal_lengths(rng, n - n_long, 360.0, 2, 3072)
        long_ = loguniform_lengths(rng, n_long, 3073, 35_000)
        lens = np.concatenate([short, long_])
        rng.shuffle(lens)
        db = seqset_from_lengths(rng, lens)
        q = seqset_from_lengths(rng, [5000, 10000, 20000, 35000])
        return Workload(name, q, db, mat, 10, 1, 10)
    if name == "batched_512q":
        base_db = db if db is not None else make_workload("swissprot_like_20q", seed, db_scale).db
        rng = np.random.default_rng(seed + 4)
        q = seqset_from_lengths(rng, rng.integers(50, 5001, 512))
        return Workload(name, q, base_db, mat, 10, 1, 10)
    raise KeyError(name)


def random_matrix(rng: np.random.Generator, A: int, lo: int, hi: int,
                  symmetric: bool = False) -> np.ndarray:
    m = rng.integers(lo, hi + 1, size=(A, A)).astype(np.int32)
    if symmetric:
        m = np.triu(m) + np.triu(m, 1).T
    return m


def random_seqset(rng: np.random.Generator, count: int, lo: int, hi: int, A: int) -> SeqSet:
    lens = rng.integers(lo, hi + 1, count)
    offsets = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    res = rng.integers(0, A, int(offsets[-1])).astype(np.uint8)
    return SeqSet(res, offsets)
