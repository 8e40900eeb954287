"""Seeded synthetic profiles and protein databases.

This module is the one input generator that both the CUDA scan library and
the scalar oracle are fed from.  It produces bytes and holds none of the
scan arithmetic: the MSV/SSV recurrences live only in the CUDA kernels and,
independently, in the oracle.

What it generates (the paper's datasets -- env_nr, est_human and Pfam 27.0
models, Sec. 4 and Table 2 -- are not available, so these stand in for them
with the same shapes: mean sequence lengths near 197-511 residues and model
lengths 7-2405):

* Profiles.  Match emissions per node are Dirichlet with concentration 20
  times the background (mean = background), log-odds ``sc = ln(p / bg)``,
  quantised in the HMMER3 byte convention of the MSV filter (Eddy 2011,
  cited in Sec. 2.1): ``scale = 3 / ln 2`` units per nat, ``base = 190``,
  ``bias = round(scale * max sc)``, ``cost = min(255, bias - round(scale *
  sc))``, ``tbm = round(-scale ln(2 / (M (M + 1))))``, ``tec = round(-scale
  ln 1/2)`` and ``tjb(L) = round(-scale ln(3 / (L + 3)))`` as a per-length
  table.  ``round`` is half away from zero.
* Databases.  Residues are i.i.d. from the background (digital codes 0..19 in
  the order ``ACDEFGHIKLMNPQRSTVWY``); lengths are lognormal with the given
  arithmetic mean and sigma_log 0.6, clipped; an optional long tail draws a
  fraction of lengths log-uniformly; optional planted segments overwrite a
  window of a sequence with residues sampled from a profile's match
  emissions along a diagonal.

Background composition: the BLOSUM62 background frequencies as commonly
quoted (ARNDCQEGHILKMFPSTWYV: .074 .052 .045 .054 .025 .034 .054 .074 .026
.068 .099 .058 .025 .047 .039 .057 .051 .013 .032 .073), renormalised.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

ALPHABET = "ACDEFGHIKLMNPQRSTVWY"
_BG_ARND = dict(zip("ARNDCQEGHILKMFPSTWYV",
                    [.074, .052, .045, .054, .025, .034, .054, .074, .026, .068,
                     .099, .058, .025, .047, .039, .057, .051, .013, .032, .073]))
BACKGROUND = np.array([_BG_ARND[a] for a in ALPHABET], dtype=np.float64)
BACKGROUND /= BACKGROUND.sum()

SCALE = 3.0 / math.log(2.0)
BASE = 190
MAX_TJB_LEN = 35_000


def round_half_away(x):
    x = np.asarray(x, dtype=np.float64)
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


@dataclass
class Profile:
    """Byte-quantised MSV/SSV profile (the inputs of ``mpf_profile_create``)."""
    M: int
    K: int
    cost: np.ndarray            # K x M uint8, row-major [residue][node]
    bias: int
    tbm: int
    tec: int
    tjb_fixed: int
    tjb_by_len: Optional[np.ndarray]   # uint8 per length 0..n-1, or None
    scale: float
    base: int
    emit: Optional[np.ndarray] = None  # M x 20 match emission probabilities


@dataclass
class Database:
    residues: np.ndarray        # uint8 digital codes
    offsets: np.ndarray         # uint64 start of each sequence in residues
    lengths: np.ndarray         # uint32

    @property
    def n_seqs(self) -> int:
        return int(self.lengths.size)

    @property
    def n_residues(self) -> int:
        return int(self.lengths.sum(dtype=np.uint64))


def tjb_table(n: int = MAX_TJB_LEN + 1, scale: float = SCALE) -> np.ndarray:
    L = np.arange(n, dtype=np.float64)
    t = round_half_away(-scale * np.log(3.0 / (L + 3.0)))
    return np.clip(t, 0, 255).astype(np.uint8)


def quantise_profile(emit: np.ndarray, bg: np.ndarray = BACKGROUND, scale: float = SCALE,
                     base: int = BASE, tjb_len: int = MAX_TJB_LEN + 1) -> Profile:
    """Quantise match emissions (M x 20) into the biased byte costs."""
    M = emit.shape[0]
    with np.errstate(divide="ignore"):
        sc = np.log(emit / bg[None, :])          # -inf where p == 0
    smax = float(np.max(sc))
    bias = int(np.clip(round_half_away(scale * smax), 0, 255))
    q = round_half_away(np.where(np.isfinite(sc), scale * sc, -1e9))
    cost = np.clip(bias - q, 0, 255).astype(np.uint8).T.copy()   # K x M
    tbm = int(np.clip(round_half_away(-scale * math.log(2.0 / (M * (M + 1.0)))), 0, 255))
    tec = int(np.clip(round_half_away(-scale * math.log(0.5)), 0, 255))
    tjb = tjb_table(tjb_len, scale)
    return Profile(M=M, K=emit.shape[1], cost=cost, bias=bias, tbm=tbm, tec=tec,
                   tjb_fixed=int(tjb[min(350, tjb.size - 1)]), tjb_by_len=tjb,
                   scale=float(np.float32(scale)), base=base, emit=emit)


def make_profile(M: int, rng: np.random.Generator, concentration: float = 20.0) -> Profile:
    alpha = concentration * BACKGROUND
    emit = rng.dirichlet(alpha, size=M)
    return quantise_profile(emit)


def _residue_lut(bg: np.ndarray = BACKGROUND) -> np.ndarray:
    cdf = np.cumsum(bg)
    cdf[-1] = 1.0
    u = (np.arange(65536, dtype=np.float64) + 0.5) / 65536.0
    return np.searchsorted(cdf, u, side="right").astype(np.uint8)


def draw_residues(n: int, rng: np.random.Generator, chunk: int = 1 << 26) -> np.ndarray:
    """i.i.d. background residues through a 16-bit inverse-CDF table."""
    lut = _residue_lut()
    out = np.empty(n, dtype=np.uint8)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = lut[rng.integers(0, 65536, size=e - s, dtype=np.uint16)]
    return out


def draw_lengths(n: int, mean: float, lo: int, hi: int, rng: np.random.Generator,
                 sigma: float = 0.6, tail_frac: float = 0.0, tail=(5000, 35000)) -> np.ndarray:
    mu = math.log(mean) - 0.5 * sigma * sigma
    L = np.rint(rng.lognormal(mu, sigma, size=n))
    if tail_frac > 0:
        pick = rng.random(n) < tail_frac
        L[pick] = np.rint(np.exp(rng.uniform(math.log(tail[0]), math.log(tail[1]), pick.sum())))
    return np.clip(L, lo, hi).astype(np.uint32)


def make_database(n_seqs: int, mean: float, lo: int, hi: int, rng: np.random.Generator,
                  sigma: float = 0.6, tail_frac: float = 0.0, tail=(5000, 35000)) -> Database:
    lengths = draw_lengths(n_seqs, mean, lo, hi, rng, sigma, tail_frac, tail)
    offsets = np.zeros(n_seqs, dtype=np.uint64)
    if n_seqs > 1:
        np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
    residues = draw_residues(int(lengths.sum(dtype=np.uint64)), rng)
    return Database(residues=residues, offsets=offsets, lengths=lengths)


def plant_segments(db: Database, profiles: List[Profile], frac: float,
                   rng: np.random.Generator, seg=(30, 300)) -> np.ndarray:
    """Overwrite a window of ``frac`` of the sequences with a diagonal run of
    residues sampled from one profile's match emissions.  Returns the indices
    of the planted sequences."""
    n = db.n_seqs
    chosen = np.flatnonzero(rng.random(n) < frac)
    for s in chosen:
        L = int(db.lengths[s])
        if L == 0:
            continue
        p = profiles[int(rng.integers(len(profiles)))]
        k0 = int(rng.integers(p.M))
        ell = int(rng.integers(seg[0], seg[1] + 1))
        ell = min(ell, p.M - k0, L)
        w = int(rng.integers(0, L - ell + 1))
        cdf = np.cumsum(p.emit[k0:k0 + ell], axis=1)
        u = rng.random(ell)[:, None] * cdf[:, -1:]
        codes = np.minimum((u >= cdf).sum(axis=1), 19).astype(np.uint8)
        o = int(db.offsets[s]) + w
        db.residues[o:o + ell] = codes
    return chosen


# ----------------------------------------------------------------------------
# The five workloads.  Each is seeded with its own index.

@dataclass
class Workload:
    name: str
    profiles: List[Profile]
    db: Database
    planted: Optional[np.ndarray] = None
    arrivals: Optional[np.ndarray] = None     # serving: arrival times (s)
    meta: dict = field(default_factory=dict)


WORKLOADS = {
    0: dict(name="plain_M100_10k", Ms=[100], n_seqs=10_000, mean=350, clip=(20, 5000)),
    1: dict(name="msweep_500k", Ms=[48, 100, 200, 400, 800, 1600, 2405], n_seqs=500_000,
            mean=355, clip=(10, 35_000)),
    2: dict(name="overflow_batch_64q_2M", n_queries=64, M_uniform=(50, 2500), n_seqs=2_000_000,
            mean=270, clip=(10, 35_000), planted=0.05),
    3: dict(name="serving_5M", M_loguniform=(50, 2000), n_seqs=5_000_000, mean=355,
            clip=(10, 35_000), n_queries=256, rates=(10, 50, 100, 200, 500)),
    4: dict(name="throughput_1000q_10M", n_queries=1000, M_loguniform=(48, 2405),
            n_seqs=10_000_000, mean=350, clip=(10, 35_000), tail_frac=1e-4),
}


def make_workload(idx: int, n_seqs: Optional[int] = None, n_queries: Optional[int] = None) -> Workload:
    """Build workload ``idx`` (0..4).  ``n_seqs``/``n_queries`` shrink it for
    tests; the draws for the first sequences and queries do not depend on the
    totals (profiles, lengths and residues come from separate streams)."""
    spec = WORKLOADS[idx]
    ss = np.random.SeedSequence(idx)
    r_prof, r_len, r_res, r_extra = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(4)]
    if "Ms" in spec:
        Ms = list(spec["Ms"])
    elif "M_uniform" in spec:
        nq = spec["n_queries"]
        lo, hi = spec["M_uniform"]
        Ms = [int(m) for m in r_prof.integers(lo, hi + 1, size=nq)]
    else:
        nq = spec["n_queries"]
        lo, hi = spec["M_loguniform"]
        Ms = [int(round(math.exp(v))) for v in r_prof.uniform(math.log(lo), math.log(hi), size=nq)]
    if n_queries is not None:
        Ms = Ms[:n_queries]
    profiles = [make_profile(M, r_prof) for M in Ms]
    n = spec["n_seqs"] if n_seqs is None else int(n_seqs)
    lo, hi = spec["clip"]
    lengths = draw_lengths(n, spec["mean"], lo, hi, r_len, tail_frac=spec.get("tail_frac", 0.0))
    offsets = np.zeros(n, dtype=np.uint64)
    if n > 1:
        np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
    residues = draw_residues(int(lengths.sum(dtype=np.uint64)), r_res)
    db = Database(residues=residues, offsets=offsets, lengths=lengths)
    wl = Workload(name=spec["name"], profiles=profiles, db=db, meta=dict(spec))
    if spec.get("planted"):
        wl.planted = plant_segments(db, profiles, spec["planted"], r_extra)
    if "rates" in spec:
        wl.meta["poisson_seed"] = idx
    return wl


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of ``n`` requests from a Poisson process."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, int(rate * 1000)])))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def random_profile(M: int, K: int, rng: np.random.Generator, cost_hi: int = 255,
                   bias=None, tbm=None, tec=None, tjb=None, base: int = BASE,
                   with_lut: bool = False) -> Profile:
    """Adversarial profile: uniform random cost bytes and free special bytes
    (for edge-case tests; not shaped like a real model)."""
    cost = rng.integers(0, cost_hi + 1, size=(K, M), dtype=np.int64).astype(np.uint8)
    b = int(rng.integers(0, 64)) if bias is None else int(bias)
    lut = None
    if with_lut:
        lut = rng.integers(0, 40, size=int(rng.integers(1, 50)), dtype=np.int64).astype(np.uint8)
    return Profile(M=M, K=K, cost=cost, bias=b,
                   tbm=int(rng.integers(0, 60)) if tbm is None else int(tbm),
                   tec=int(rng.integers(0, 8)) if tec is None else int(tec),
                   tjb_fixed=int(rng.integers(0, 40)) if tjb is None else int(tjb),
                   tjb_by_len=lut, scale=float(np.float32(SCALE)), base=int(base))


def random_database(n: int, max_len: int, rng: np.random.Generator, alphabet: int = 32,
                    min_len: int = 0) -> Database:
    lengths = rng.integers(min_len, max_len + 1, size=n).astype(np.uint32)
    offsets = np.zeros(n, dtype=np.uint64)
    if n > 1:
        np.cumsum(lengths[:-1], dtype=np.uint64, out=offsets[1:])
    residues = rng.integers(0, alphabet, size=int(lengths.sum()), dtype=np.int64).astype(np.uint8)
    return Database(residues=residues, offsets=offsets, lengths=lengths)


# ----------------------------------------------------------------------------
# Viterbi filter profiles (Eq. 1): match emissions, the seven node transitions
# and the special states in the HMMER3 16-bit word convention
# (scale 500 / ln 2 words per nat, base 12000).

VIT_SCALE = 500.0 / math.log(2.0)
VIT_BASE = 12000
NEG16 = -32768


@dataclass
class VitProfile:
    M: int
    K: int
    msc: np.ndarray        # K x M int16 match scores
    trans: np.ndarray      # 8 x M int16: BM, MM, IM, DM, MI, II, MD, DD (node k at k-1)
    special: np.ndarray    # 8 int16: NN, NB, EC, CC, CT, EJ, JJ, JB
    base: int
    scale: float


def _words(p, scale=VIT_SCALE):
    with np.errstate(divide="ignore"):
        w = round_half_away(np.where(p > 0, scale * np.log(np.maximum(p, 1e-300)), -1e9))
    return np.clip(w, NEG16, 32767).astype(np.int16)


def make_vit_profile(M: int, rng: np.random.Generator, L: int = 350,
                     concentration: float = 20.0) -> VitProfile:
    """Match emissions as in make_profile; per-node transitions drawn from
    Dirichlets around a typical Plan-7 model (M->M 0.96, M->I 0.02, M->D 0.02,
    I->M/I->I and D->M/D->D 0.5/0.5); uniform local entry 2 / (M (M + 1)); the
    N, C and J loops and moves configured for sequence length L, multi-hit
    (E->C = E->J = 1/2)."""
    emit = rng.dirichlet(concentration * BACKGROUND, size=M)
    msc = _words(emit / BACKGROUND[None, :]).T.copy()
    tm = rng.dirichlet([96.0, 2.0, 2.0], size=M)     # from M_k: MM, MI, MD
    ti = rng.dirichlet([5.0, 5.0], size=M)            # from I_k: IM, II
    td = rng.dirichlet([5.0, 5.0], size=M)            # from D_k: DM, DD
    trans = np.full((8, M), NEG16, dtype=np.int16)
    trans[0] = _words(np.full(M, 2.0 / (M * (M + 1.0))))
    if M > 1:
        trans[1, 1:] = _words(tm[:-1, 0])    # M_{k-1} -> M_k
        trans[2, 1:] = _words(ti[:-1, 0])    # I_{k-1} -> M_k
        trans[3, 1:] = _words(td[:-1, 0])    # D_{k-1} -> M_k
        trans[4, :-1] = _words(tm[:-1, 1])   # M_k -> I_k
        trans[5, :-1] = _words(ti[:-1, 1])   # I_k -> I_k
        trans[6, 1:] = _words(tm[:-1, 2])    # M_{k-1} -> D_k
    if M > 2:
        trans[7, 2:] = _words(td[1:-1, 1])   # D_{k-1} -> D_k
    loop = L / (L + 3.0)
    move = 3.0 / (L + 3.0)
    special = _words(np.array([loop, move, 0.5, loop, move, 0.5, loop, move]))
    return VitProfile(M=M, K=20, msc=msc, trans=trans, special=special, base=VIT_BASE,
                      scale=float(np.float32(VIT_SCALE)))


def random_vit_profile(M: int, K: int, rng: np.random.Generator, lo: int = -32768,
                       hi: int = 32767, base=None, moves_hi=None) -> VitProfile:
    """Adversarial Viterbi profile: uniform int16 scores in [lo, hi]; with
    ``moves_hi`` the transition and special scores are drawn from
    [lo, moves_hi] instead (moves_hi=0: log-probability-like signs)."""
    def u(shape, top=hi):
        return rng.integers(lo, top + 1, size=shape, dtype=np.int64).astype(np.int16)
    mh = hi if moves_hi is None else min(hi, moves_hi)
    return VitProfile(M=M, K=K, msc=u((K, M)), trans=u((8, M), mh), special=u(8, mh),
                      base=int(rng.integers(-32768, 32768)) if base is None else int(base),
                      scale=float(np.float32(VIT_SCALE)))


def positive_chain_vit_profile(M: int, K: int, rng: np.random.Generator, kind: int) -> VitProfile:
    """Adversarial Viterbi profile with positive delete moves and a begin
    state near -32768: kind 0, large positive D->D and D->M (the delete chain
    climbs from -32768 across many nodes and reaches the upper bound);
    kind 1, small positive D->D, large positive D->M and nonnegative match
    scores (a row reads the previous row's delete scores through D->M)."""
    v = random_vit_profile(M, K, rng, lo=-3000, hi=3000)
    if kind == 0:
        v.trans[7] = rng.integers(1, 3000, M).astype(np.int16)
        v.trans[3] = rng.integers(0, 3000, M).astype(np.int16)
    else:
        v.trans[7] = rng.integers(1, 100, M).astype(np.int16)
        v.trans[3] = rng.integers(10000, 25000, M).astype(np.int16)
        v.msc[:] = rng.integers(0, 3000, v.msc.shape).astype(np.int16)
    v.base = -32000
    return v
