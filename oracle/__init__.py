"""FP64 CPU oracle for Aggregate Risk Analysis.  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package.  It shares no code with the CUDA library (the product
path) and neither imports the other; both receive their inputs from ``synth``.

Contents
--------
ylt()            YLT by the plain loops of Algorithm 3 (Section IV-B), in C (ara_oracle.c).
brute_ylt()      The same quantity written differently (pure Python, event-major, dicts
                 instead of direct-access tables); pins ylt() on tiny inputs.
pml(), tvar()    Risk metrics named in Section IV-A ("PML", "TVaR"); the paper gives no
                 formula, so this package reads them as empirical order statistics of the
                 YLT: PML at return period RP is the ceil(N/RP)-th largest year loss, TVaR
                 at level p is the mean of the ceil(N(1-p)) largest year losses.  RP and p
                 are read as the decimal numbers they print as (exact rational arithmetic).
adjoint()        Gradient of a weighted sum of year losses (mean, or TVaR's top set)
                 w.r.t. every retention, limit and ELT loss, by the chain rule applied
                 occurrence by occurrence (ara_oracle.c).

Parity status: every function here is pinned by tests/test_oracle_pins.py (hand-worked
portfolio, closed forms, monotonicity, brute force, telescoping, permutation invariance,
sorted-order statistics, exact finite differences of a piecewise-linear objective).
"""
from __future__ import annotations

import ctypes
import math
import os
from fractions import Fraction
from typing import Dict, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

_lib = None


def build(verbose: bool = False) -> str:
    """Compile ara_oracle.c into liboracle.so (plain gcc, OpenMP when available, IEEE FP)."""
    import subprocess
    src = os.path.join(HERE, "ara_oracle.c")
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = LIB_PATH + ".tmp"
    for extra in (["-fopenmp"], []):
        cmd = base + extra + [src, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB_PATH)
            return LIB_PATH
        if verbose:
            print(r.stderr)
    raise RuntimeError("oracle build failed: " + r.stderr)


def lib():
    global _lib
    if _lib is None:
        src = os.path.join(HERE, "ara_oracle.c")
        if (not os.path.exists(LIB_PATH)) or os.path.getmtime(LIB_PATH) < os.path.getmtime(src):
            build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        L.orc_ylt.argtypes = [i64, i32, P, P, P, P, P, i32, P, P, P, P, P, P, i64, P, P, i64, P, P, P]
        L.orc_ylt.restype = ctypes.c_int
        L.orc_ylt_oep.argtypes = [i64, P, P, P, P, P, i32, P, P, P, P, i64, P, P, i64, P, P]
        L.orc_ylt_oep.restype = ctypes.c_int
        L.orc_adjoint.argtypes = [i64, P, P, P, P, P, i32, P, P, P, P, P, P, i64, P, P, P, P, P, P, P]
        L.orc_adjoint.restype = ctypes.c_int
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def threads() -> int:
    return int(lib().orc_max_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _records(pf):
    off = np.zeros(pf.n_elts + 1, dtype=np.int64)
    off[1:] = np.cumsum([x.size for x in pf.elt_ids])
    ids = np.ascontiguousarray(np.concatenate(pf.elt_ids) if pf.n_elts else np.zeros(0, np.int32),
                               dtype=np.int32)
    losses = np.ascontiguousarray(np.concatenate(pf.elt_losses) if pf.n_elts else np.zeros(0),
                                  dtype=np.float64)
    return off, ids, losses


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def ylt(pf, yet, trials: Optional[Sequence[int]] = None, return_agg: bool = False):
    """Year losses [n_layers, n_out] (n_out = len(trials) or all trials), FP64.
    With return_agg, also the aggregate losses before the aggregate terms."""
    L = lib()
    off, ids, losses = _records(pf)
    loff, lel = pf.layer_csr()
    toff = np.ascontiguousarray(yet.offsets, dtype=np.int64)
    ev = np.ascontiguousarray(yet.event_ids, dtype=np.int32)
    sel = None if trials is None else np.ascontiguousarray(np.asarray(trials, dtype=np.int64))
    n_out = yet.n_trials if sel is None else sel.size
    out = np.zeros((pf.n_layers, n_out), dtype=np.float64)
    agg = np.zeros((pf.n_layers, n_out), dtype=np.float64) if return_agg else None
    rc = L.orc_ylt(pf.catalogue, pf.n_elts, _p(off), _p(ids), _p(losses), _p(_f64(pf.elt_ret)),
                   _p(_f64(pf.elt_lim)), pf.n_layers, _p(loff), _p(lel), _p(_f64(pf.occ_ret)),
                   _p(_f64(pf.occ_lim)), _p(_f64(pf.agg_ret)), _p(_f64(pf.agg_lim)), yet.n_trials,
                   _p(toff), _p(ev), 0 if sel is None else sel.size,
                   None if sel is None else _p(sel), _p(out), None if agg is None else _p(agg))
    if rc != 0:
        raise ValueError("oracle: invalid input (event ID out of range, duplicate ELT record, "
                         "bad trial index) or out of memory")
    return (out, agg) if return_agg else out


def ylt_oep(pf, yet, trials: Optional[Sequence[int]] = None):
    """Occurrence year losses [n_layers, n_out]: the largest occurrence loss of each trial net of
    the ELT and occurrence terms (the loss basis of occurrence exceedance probabilities; the
    aggregate terms do not apply)."""
    L = lib()
    off, ids, losses = _records(pf)
    loff, lel = pf.layer_csr()
    sel = None if trials is None else np.ascontiguousarray(np.asarray(trials, dtype=np.int64))
    n_out = yet.n_trials if sel is None else sel.size
    out = np.zeros((pf.n_layers, n_out), dtype=np.float64)
    rc = L.orc_ylt_oep(pf.catalogue, _p(off), _p(ids), _p(losses), _p(_f64(pf.elt_ret)),
                       _p(_f64(pf.elt_lim)), pf.n_layers, _p(loff), _p(lel), _p(_f64(pf.occ_ret)),
                       _p(_f64(pf.occ_lim)), yet.n_trials,
                       _p(np.ascontiguousarray(yet.offsets, dtype=np.int64)),
                       _p(np.ascontiguousarray(yet.event_ids, dtype=np.int32)),
                       0 if sel is None else sel.size, None if sel is None else _p(sel), _p(out))
    if rc != 0:
        raise ValueError("oracle: invalid input")
    return out


# ------------------------------------------------------------------------------------------
# Second, independent formulation (pin P5): event-major, dictionaries, pure Python.
# ------------------------------------------------------------------------------------------

def brute_ylt(pf, yet):
    """Year losses by a different route: first the net loss of every distinct event under
    each layer (dict lookups per ELT record), then per trial a sum over its occurrences."""
    out = np.zeros((pf.n_layers, yet.n_trials))
    dicts = [dict(zip(i.tolist(), x.tolist())) for i, x in zip(pf.elt_ids, pf.elt_losses)]
    for l, elts in enumerate(pf.layer_elts):
        occ_net = {}
        for e in set(yet.event_ids.tolist()):
            tot = 0.0
            for j in elts:
                x = dicts[j].get(e, 0.0)
                tot += min(max(x - float(pf.elt_ret[j]), 0.0), float(pf.elt_lim[j]))
            occ_net[e] = min(max(tot - float(pf.occ_ret[l]), 0.0), float(pf.occ_lim[l]))
        for t in range(yet.n_trials):
            a = 0.0
            for e in yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]].tolist():
                a += occ_net[e]
            out[l, t] = min(max(a - float(pf.agg_ret[l]), 0.0), float(pf.agg_lim[l]))
    return out


# ------------------------------------------------------------------------------------------
# Risk metrics (Section IV-A names PML and TVaR; definitions are this package's reading)
# ------------------------------------------------------------------------------------------

def rank_for_return_period(n: int, rp: float) -> int:
    """k = ceil(N / RP) with RP read as the decimal it prints as."""
    k = math.ceil(Fraction(n) / Fraction(repr(float(rp))))
    if not (1 <= k <= n):
        raise ValueError("return period out of range")
    return int(k)


def tail_count(n: int, p: float) -> int:
    """m = ceil(N (1 - p)) with p read as the decimal it prints as."""
    m = math.ceil(Fraction(n) * (1 - Fraction(repr(float(p)))))
    if not (1 <= m <= n):
        raise ValueError("TVaR level out of range")
    return int(m)


def pml(y: np.ndarray, rp: float) -> float:
    ys = np.sort(np.asarray(y, dtype=np.float64))[::-1]
    return float(ys[rank_for_return_period(ys.size, rp) - 1])


def tvar(y: np.ndarray, p: float) -> float:
    ys = np.sort(np.asarray(y, dtype=np.float64))[::-1]
    m = tail_count(ys.size, p)
    return math.fsum(ys[:m].tolist()) / m


def risk_metrics(ylt_: np.ndarray, rps: Sequence[float], levels: Sequence[float]):
    ylt_ = np.atleast_2d(ylt_)
    P = np.array([[pml(r, rp) for rp in rps] for r in ylt_])
    T = np.array([[tvar(r, p) for p in levels] for r in ylt_])
    return P, T


# ------------------------------------------------------------------------------------------
# Adjoint
# ------------------------------------------------------------------------------------------

def objective_weights(ylt_: np.ndarray, objective: str, level: float = 0.99):
    """Per-trial weights w_t of J = sum_t w_t y_t: 1/N for the mean year loss; for TVaR_p, with
    m = ceil(N(1-p)) and v the m-th largest year loss, 1/m on every y_t > v and the remaining
    weight (m - #{y > v}) / m shared equally by the trials with y_t == v (the mean over every
    choice of the top-m set).  Returns (w, tie): tie reports that the top-m set is not unique
    (#{y >= v} > m), so TVaR is not differentiable in the usual sense there."""
    ylt_ = np.atleast_2d(ylt_)
    nl, n = ylt_.shape
    w = np.zeros((nl, n))
    ties = []
    for l in range(nl):
        if objective == "mean":
            w[l, :] = 1.0 / n
            ties.append(False)
        elif objective == "tvar":
            m = tail_count(n, level)
            v = np.sort(ylt_[l])[::-1][m - 1]
            gt = ylt_[l] > v
            eq = ylt_[l] == v
            c_gt, c_eq = int(gt.sum()), int(eq.sum())
            w[l, gt] = 1.0 / m
            w[l, eq] = (m - c_gt) / (c_eq * m)
            ties.append(c_gt + c_eq > m)
        else:
            raise ValueError(objective)
    return w, ties


def adjoint_weighted(pf, yet, w: np.ndarray) -> Dict[str, np.ndarray]:
    """Gradient of J_l = sum_t w[l, t] y_{l,t} for every layer l."""
    L = lib()
    off, ids, losses = _records(pf)
    loff, lel = pf.layer_csr()
    w = np.ascontiguousarray(np.broadcast_to(w, (pf.n_layers, yet.n_trials)), dtype=np.float64)
    nnz = np.array([pf.elt_ids[j].size for l in pf.layer_elts for j in l], dtype=np.int64)
    per_layer = np.array([sum(pf.elt_ids[j].size for j in l) for l in pf.layer_elts], dtype=np.int64)
    g_loss_off = np.zeros(pf.n_layers + 1, dtype=np.int64)
    g_loss_off[1:] = np.cumsum(per_layer)
    g_elt = np.zeros((int(loff[-1]), 2))
    g_layer = np.zeros((pf.n_layers, 4))
    g_loss = np.zeros(int(g_loss_off[-1]))
    rc = L.orc_adjoint(pf.catalogue, _p(off), _p(ids), _p(losses), _p(_f64(pf.elt_ret)),
                       _p(_f64(pf.elt_lim)), pf.n_layers, _p(loff), _p(lel),
                       _p(_f64(pf.occ_ret)), _p(_f64(pf.occ_lim)), _p(_f64(pf.agg_ret)),
                       _p(_f64(pf.agg_lim)), yet.n_trials,
                       _p(np.ascontiguousarray(yet.offsets, dtype=np.int64)),
                       _p(np.ascontiguousarray(yet.event_ids, dtype=np.int32)), _p(w), _p(g_elt),
                       _p(g_layer), _p(g_loss_off), _p(g_loss))
    if rc != 0:
        raise ValueError("oracle adjoint: invalid input or out of memory")
    return {"elt": g_elt, "layer": g_layer, "loss": g_loss, "loss_offsets": g_loss_off,
            "elt_offsets": loff, "record_counts": nnz}


def adjoint(pf, yet, objective: str = "mean", level: float = 0.99):
    y = ylt(pf, yet)
    w, ties = objective_weights(y, objective, level)
    g = adjoint_weighted(pf, yet, w)
    g["ties"] = ties
    return g
