"""Seeded synthetic inputs for Aggregate Risk Analysis (ARA).

This module builds the three input tables of the paper's Section IV-A (the
Year Event Table of Eq. 1, the Event Loss Tables of Eq. 2 and the layers of
Eq. 3) with the shapes and distributions of the workloads described there:
trials of roughly 800-1500 time-ordered events drawn from a global event
catalogue, ELTs of 10,000-30,000 event losses, layers of 3-30 ELTs.

It holds none of the method's arithmetic (no financial terms, no sums over
trials, no risk metrics).  It is the only code shared by the CUDA path's
tests/benchmark and the CPU oracle: both receive the arrays built here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream k is mix64(key_k + (i + 1) * GAMMA).  Integer
draws are therefore identical on every platform; Poisson counts use NumPy's
Philox-based Generator.
"""
from __future__ import annotations

import json
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U64 = np.uint64


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (in place on a uint64 array, which is returned)."""
    with np.errstate(over="ignore"):
        z ^= z >> _U64(30)
        z *= _M1
        z ^= z >> _U64(27)
        z *= _M2
        z ^= z >> _U64(31)
    return z


def stream_key(seed: int, *tags: int) -> np.uint64:
    """Key of an independent stream: the seed and integer tags folded through mix64."""
    k = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    for t in tags:
        with np.errstate(over="ignore"):
            k = mix64(k + GAMMA * _U64(t & 0xFFFFFFFFFFFFFFFF) + _U64(0x632BE59BD9B4E019))
    return k[0]


def draws(key: np.uint64, start: int, count: int) -> np.ndarray:
    """Raw 64-bit draws start .. start+count-1 of the stream `key`."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        i *= GAMMA
        i += key
    return mix64(i)


def uniform01(key, start, count) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws(key, start, count) >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def below(key, start, count, n: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Uniform integers in [0, n) (n < 2**32) by the multiply-shift map of the top 32 bits."""
    assert 0 < n < (1 << 32)
    z = draws(key, start, count) >> _U64(32)
    with np.errstate(over="ignore"):
        z *= _U64(n)
    z >>= _U64(32)
    if out is None:
        return z.astype(np.int32)
    out[...] = z
    return out


def lognormal(key, start, count, mu: float, sigma: float) -> np.ndarray:
    """Lognormal(mu, sigma) by the Box-Muller transform of two uniform streams."""
    u1 = 1.0 - uniform01(key, start, count)              # (0, 1]
    u2 = uniform01(stream_key(int(key), 1), start, count)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return np.exp(mu + sigma * z)


def distinct(key, k: int, n: int) -> np.ndarray:
    """k distinct integers of [0, n), in first-draw order (sampling without replacement)."""
    assert k <= n
    got = np.empty(0, dtype=np.int64)
    pos, batch = 0, max(16, int(k * 1.25) + 16)
    while True:
        c = below(key, pos, batch, n).astype(np.int64)
        pos += batch
        allc = np.concatenate([got, c])
        _, first = np.unique(allc, return_index=True)
        first.sort()
        got = allc[first]
        if got.size >= k:
            return got[:k].astype(np.int32)


# --------------------------------------------------------------------------------------------
# Data model of Section IV-A
# --------------------------------------------------------------------------------------------

@dataclass
class Portfolio:
    """ELTs (Eq. 2) with per-ELT terms and layers (Eq. 3) with occurrence/aggregate terms."""
    catalogue: int
    elt_ids: List[np.ndarray]          # per ELT: int32 event IDs, unique, < catalogue
    elt_losses: List[np.ndarray]       # per ELT: float64 losses (float32-representable when f32)
    elt_ret: np.ndarray                # per ELT occurrence retention  (float64)
    elt_lim: np.ndarray                # per ELT occurrence limit      (float64, may be inf)
    layer_elts: List[List[int]]        # per layer: indices of its ELTs, in order
    occ_ret: np.ndarray                # per layer (float64)
    occ_lim: np.ndarray
    agg_ret: np.ndarray
    agg_lim: np.ndarray
    losses_f32: bool = False

    @property
    def n_elts(self) -> int:
        return len(self.elt_ids)

    @property
    def n_layers(self) -> int:
        return len(self.layer_elts)

    def layer_csr(self):
        off = np.zeros(self.n_layers + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(l) for l in self.layer_elts])
        ids = np.array([j for l in self.layer_elts for j in l], dtype=np.int32)
        return off, ids

    def terms_dict(self) -> dict:
        f = lambda a: [float(x) for x in np.asarray(a)]
        return {"elt_ret": f(self.elt_ret), "elt_lim": f(self.elt_lim), "occ_ret": f(self.occ_ret),
                "occ_lim": f(self.occ_lim), "agg_ret": f(self.agg_ret), "agg_lim": f(self.agg_lim)}

    def with_terms(self, t: dict) -> "Portfolio":
        g = lambda k: np.asarray(t[k], dtype=np.float64)
        return Portfolio(self.catalogue, self.elt_ids, self.elt_losses, g("elt_ret"), g("elt_lim"),
                         self.layer_elts, g("occ_ret"), g("occ_lim"), g("agg_ret"), g("agg_lim"),
                         self.losses_f32)


@dataclass
class YET:
    """Year Event Table (Eq. 1) as CSR: trial t owns events offsets[t] .. offsets[t+1]-1."""
    offsets: np.ndarray                # int64 [n_trials + 1]
    event_ids: np.ndarray              # int32 [n_events], time-ordered within each trial
    timestamps: Optional[np.ndarray] = None   # float32 [n_events] in [0, 365), ascending per trial

    @property
    def n_trials(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def n_events(self) -> int:
        return int(self.offsets[-1])


def make_elts(seed: int, n_elts: int, nnz: int, catalogue: int, mu: float, sigma: float,
              f32: bool):
    ids, losses = [], []
    for j in range(n_elts):
        ids.append(distinct(stream_key(seed, 1, j), nnz, catalogue))
        x = lognormal(stream_key(seed, 2, j), 0, nnz, mu, sigma)
        if f32:
            x = x.astype(np.float32).astype(np.float64)
        losses.append(x)
    return ids, losses


def percentile_terms(losses: List[np.ndarray], lo: float = 20.0, hi: float = 95.0):
    """Per-ELT retention R = P_lo and limit L = P_hi, the lo-th and hi-th percentiles of that
    ELT's losses (NumPy's default linear interpolation); L is the limit amount, so the cover
    pays min(max(x - P_lo, 0), P_hi)."""
    r = np.array([np.percentile(x, lo) if x.size else 0.0 for x in losses], dtype=np.float64)
    l = np.array([np.percentile(x, hi) if x.size else 0.0 for x in losses], dtype=np.float64)
    return r, l


def _fill_ids(out: np.ndarray, key, catalogue: int, nthreads: int):
    n = out.size
    chunk = 1 << 22
    starts = list(range(0, n, chunk))

    def work(s):
        e = min(n, s + chunk)
        below(key, s, e - s, catalogue, out=out[s:e])

    if nthreads <= 1 or len(starts) <= 1:
        for s in starts:
            work(s)
    else:
        with ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(work, starts))


def make_yet(seed: int, counts: np.ndarray, catalogue: int, with_timestamps: bool = True,
             ids_out: Optional[np.ndarray] = None, nthreads: Optional[int] = None) -> YET:
    """Trials with the given event counts; IDs uniform over the catalogue with replacement;
    timestamps uniform on [0, 365), sorted within each trial (ascending time order, Eq. 1)."""
    counts = np.asarray(counts, dtype=np.int64)
    offsets = np.zeros(counts.size + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    n = int(offsets[-1])
    ids = ids_out if ids_out is not None else np.empty(n, dtype=np.int32)
    assert ids.size == n and ids.dtype == np.int32
    _fill_ids(ids, stream_key(seed, 3), catalogue, nthreads or min(16, os.cpu_count() or 1))
    ts = None
    if with_timestamps:
        u = uniform01(stream_key(seed, 4), 0, n) * 365.0
        tr = np.repeat(np.arange(counts.size, dtype=np.int64), counts)
        order = np.lexsort((u, tr))
        ts = u[order].astype(np.float32)
    return YET(offsets, ids, ts)


def poisson_counts(seed: int, lam, n_trials: int) -> np.ndarray:
    g = np.random.Generator(np.random.Philox(key=seed & 0xFFFFFFFFFFFFFFFF))
    return g.poisson(lam, size=n_trials).astype(np.int64)


# --------------------------------------------------------------------------------------------
# Workload recipes (the five workload configurations: tiny, paper scale, batched, adjoint,
# serving).  Layer and aggregate terms that depend on the loss model beyond per-ELT
# percentiles are read from the terms manifests next to this file.
# --------------------------------------------------------------------------------------------

HERE = os.path.dirname(os.path.abspath(__file__))


def load_terms(name: str) -> dict:
    with open(os.path.join(HERE, f"terms_{name}.json")) as f:
        return json.load(f)


def tiny(seed: int = 0):
    """1 layer of 4 ELTs over a 10,000-event catalogue; 1,000 trials of Poisson(100) events."""
    C = 10_000
    ids, losses = make_elts(seed, 4, 1000, C, 10.0, 1.5, f32=False)
    r, l = percentile_terms(losses)
    pf = Portfolio(C, ids, losses, r, l, [[0, 1, 2, 3]], np.array([1e4]), np.array([1e6]),
                   np.array([5e4]), np.array([5e6]), losses_f32=False)
    yet = make_yet(seed, poisson_counts(seed, 100.0, 1000), C)
    return pf, yet


def paper_scale_portfolio(seed: int = 0, terms: Optional[dict] = None) -> Portfolio:
    """1 layer of 15 ELTs x 20,000 events over a 2,000,000-event catalogue, FP32 lognormal(11, 2)."""
    C = 2_000_000
    ids, losses = make_elts(seed, 15, 20_000, C, 11.0, 2.0, f32=True)
    r, l = percentile_terms(losses)
    nan = np.array([np.nan])
    pf = Portfolio(C, ids, losses, r, l, [list(range(15))], nan, nan, nan, nan, losses_f32=True)
    if terms is None:
        terms = load_terms("paper_scale")
    return pf.with_terms(terms)


def paper_scale_yet(seed: int = 0, n_trials: int = 1_000_000, events_per_trial: int = 1000,
                    ids_out: Optional[np.ndarray] = None) -> YET:
    """n_trials x exactly events_per_trial events (no timestamps: the YLT does not read them)."""
    counts = np.full(n_trials, events_per_trial, dtype=np.int64)
    return make_yet(seed, counts, 2_000_000, with_timestamps=False, ids_out=ids_out)


def _pool(seed: int, n_elts: int, nnz: int = 20_000, catalogue: int = 2_000_000):
    ids, losses = make_elts(seed, n_elts, nnz, catalogue, 11.0, 2.0, f32=True)
    r, l = percentile_terms(losses)
    return ids, losses, r, l


def adjoint_portfolio(seed: int = 0, terms: Optional[dict] = None) -> Portfolio:
    """16 layers x 15 ELTs (each layer its own 15 ELTs of 20,000 events, 2,000,000-event
    catalogue, FP32 lognormal(11, 2) losses); layer terms from terms_adjoint.json."""
    ids, losses, r, l = _pool(seed + 1000, 16 * 15)
    layers = [list(range(15 * k, 15 * k + 15)) for k in range(16)]
    nan = np.full(16, np.nan)
    pf = Portfolio(2_000_000, ids, losses, r, l, layers, nan, nan, nan, nan, losses_f32=True)
    return pf.with_terms(load_terms("adjoint") if terms is None else terms)


def adjoint_yet(seed: int = 0, n_trials: int = 200_000, ids_out: Optional[np.ndarray] = None) -> YET:
    counts = np.full(n_trials, 1000, dtype=np.int64)
    return make_yet(seed + 1000, counts, 2_000_000, with_timestamps=False, ids_out=ids_out)


def batched_portfolio(seed: int = 0, terms: Optional[dict] = None) -> Portfolio:
    """64 layers, each of U{3..30} distinct ELTs drawn from a pool of 200 ELTs (20,000 events,
    2,000,000-event catalogue, FP32 lognormal(11, 2)); layer terms from terms_batched.json."""
    ids, losses, r, l = _pool(seed + 2000, 200)
    key = stream_key(seed, 5)
    sizes = 3 + below(key, 0, 64, 28)                       # U{3..30}
    layers = []
    for k in range(64):
        pick = distinct(stream_key(seed, 6, k), int(sizes[k]), 200)
        layers.append(sorted(int(x) for x in pick))
    nan = np.full(64, np.nan)
    pf = Portfolio(2_000_000, ids, losses, r, l, layers, nan, nan, nan, nan, losses_f32=True)
    return pf.with_terms(load_terms("batched") if terms is None else terms)


def batched_term_factors(seed: int = 0) -> np.ndarray:
    """Per-layer multipliers U(0.5, 1.5) of (OccR, OccL, AggR, AggL) around the percentile rule."""
    return 0.5 + uniform01(stream_key(seed, 7), 0, 64 * 4).reshape(64, 4)


def batched_yet(seed: int = 0, n_trials: int = 200_000, ids_out: Optional[np.ndarray] = None) -> YET:
    """Trials with Poisson event counts whose per-trial mean is uniform on [200, 2000]."""
    mu = 200.0 + 1800.0 * uniform01(stream_key(seed, 8), 0, n_trials)
    counts = poisson_counts(seed + 2000, mu, n_trials)
    return make_yet(seed + 2000, counts, 2_000_000, with_timestamps=False, ids_out=ids_out)


def serving_pool(seed: int = 0) -> Portfolio:
    """Resident pool of 500 ELTs x 20,000 events (2,000,000-event catalogue, FP32 lognormal(11, 2)),
    per-ELT terms by the percentile rule, no layers (queries bring their own)."""
    ids, losses, r, l = _pool(seed + 3000, 500)
    z = np.zeros(0)
    return Portfolio(2_000_000, ids, losses, r, l, [], z, z, z, z, losses_f32=True)


def serving_yet(seed: int = 0, n_trials: int = 1_000_000, ids_out: Optional[np.ndarray] = None) -> YET:
    """Resident YET of n_trials x Poisson(1000) events."""
    counts = poisson_counts(seed + 3000, 1000.0, n_trials)
    return make_yet(seed + 3000, counts, 2_000_000, with_timestamps=False, ids_out=ids_out)


def serving_trace(pool: Portfolio, n_trials: int, n_requests: int = 200, rate: float = 200.0,
                  seed: int = 0, adjoint_share: float = 0.2):
    """Seeded request trace: Poisson arrivals at `rate` per second from 32 tenants; each query has
    U{1..32} layers of U{5..20} distinct pool ELTs over a contiguous slice of U[1e4, 1e6] trials
    (clipped to the YET), 20 % with the adjoint.  Layer terms are set from the raw loss quantiles
    of the layer's ELTs (no financial terms are evaluated here): OccR = max_j P50_j,
    OccL = sum_j P95_j, AggR = 10 sum_j P50_j, AggL = 200 sum_j P95_j."""
    g = np.random.Generator(np.random.Philox(key=seed + 4000))
    p50 = np.array([np.percentile(x, 50) for x in pool.elt_losses])
    p95 = np.array([np.percentile(x, 95) for x in pool.elt_losses])
    t = np.cumsum(g.exponential(1.0 / rate, n_requests))
    out = []
    for k in range(n_requests):
        nl = int(g.integers(1, 33))
        layers = [sorted(g.choice(pool.n_elts, size=int(g.integers(5, 21)), replace=False).tolist())
                  for _ in range(nl)]
        n = int(min(n_trials, g.integers(10_000, 1_000_001)))
        t0 = int(g.integers(0, n_trials - n + 1))
        out.append(dict(arrival=float(t[k]), tenant=int(g.integers(0, 32)), layer_elts=layers,
                        occ_ret=[float(p50[l].max()) for l in layers],
                        occ_lim=[float(p95[l].sum()) for l in layers],
                        agg_ret=[float(10 * p50[l].sum()) for l in layers],
                        agg_lim=[float(200 * p95[l].sum()) for l in layers],
                        trials=(t0, t0 + n), want_adjoint=bool(g.random() < adjoint_share)))
    return out
