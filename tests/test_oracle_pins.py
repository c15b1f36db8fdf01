"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics, not by the
oracle itself: a hand-worked portfolio (P1), closed forms (P2, P3), monotonicity (P4), an
independently written second oracle (P5), the telescoping reading of Algorithm 3 (P6),
permutation invariance and trial independence (P7), order statistics (P8) and exact finite
differences of the piecewise-linear objective (P9)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

INF = math.inf


def load_p1(golden_dir):
    with open(os.path.join(golden_dir, "p1_hand_worked.json")) as f:
        g = json.load(f)
    el = g["elts"]
    lay = g["layer"]
    pf = synth.Portfolio(
        g["catalogue"], [np.array(e["ids"], np.int32) for e in el],
        [np.array(e["losses"], np.float64) for e in el], np.array([e["ret"] for e in el]),
        np.array([e["lim"] for e in el]), [lay["elts"]], np.array([lay["occ_ret"]]),
        np.array([lay["occ_lim"]]), np.array([lay["agg_ret"]]), np.array([lay["agg_lim"]]))
    yet = trials_to_yet(g["trials"])
    return pf, yet, g["expected"]


def trials_to_yet(trials):
    counts = np.array([len(t) for t in trials], np.int64)
    off = np.zeros(len(trials) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    ids = np.array([e for t in trials for e in t], np.int32)
    return synth.YET(off, ids)


def random_case(seed, catalogue=300, n_elts=5, nnz=60, n_layers=3, n_trials=80, lam=25,
                inf_limits=False):
    rng = np.random.default_rng(seed)
    ids = [rng.choice(catalogue, size=nnz, replace=False).astype(np.int32) for _ in range(n_elts)]
    losses = [rng.lognormal(5, 1.2, nnz) for _ in range(n_elts)]
    r = np.array([np.percentile(x, 20) for x in losses])
    l = np.array([np.percentile(x, 95) for x in losses])
    if inf_limits:
        l[:] = INF
    layers = [sorted(rng.choice(n_elts, size=rng.integers(1, n_elts + 1), replace=False).tolist())
              for _ in range(n_layers)]
    occ_r = rng.uniform(0, 200, n_layers)
    occ_l = rng.uniform(200, 800, n_layers)
    agg_r = rng.uniform(0, 1500, n_layers)
    agg_l = rng.uniform(1000, 6000, n_layers)
    pf = synth.Portfolio(catalogue, ids, losses, r, l, layers, occ_r, occ_l, agg_r, agg_l)
    counts = rng.poisson(lam, n_trials)
    counts[0] = 0
    off = np.zeros(n_trials + 1, np.int64)
    off[1:] = np.cumsum(counts)
    yet = synth.YET(off, rng.integers(0, catalogue, int(off[-1])).astype(np.int32))
    return pf, yet


# ---------------------------------------------------------------------------------- P1
def test_p1_hand_worked_ylt(golden_dir):
    pf, yet, exp = load_p1(golden_dir)
    y, agg = oracle.ylt(pf, yet, return_agg=True)
    assert y[0].tolist() == exp["ylt"]
    assert agg[0].tolist() == exp["agg_loss"]


def test_p1_hand_worked_risk_metrics(golden_dir):
    pf, yet, exp = load_p1(golden_dir)
    y = oracle.ylt(pf, yet)[0]
    for rp, v in exp["pml"].items():
        assert oracle.pml(y, float(rp)) == v
    for p, v in exp["tvar"].items():
        assert oracle.tvar(y, float(p)) == v


@pytest.mark.parametrize("objective,key,level", [("mean", "adjoint_mean", 0.99),
                                                 ("tvar", "adjoint_tvar_0.6", 0.6)])
def test_p1_hand_worked_adjoint(golden_dir, objective, key, level):
    pf, yet, exp = load_p1(golden_dir)
    g = oracle.adjoint(pf, yet, objective, level)
    e = exp[key]
    np.testing.assert_allclose(g["elt"], e["elt_ret_lim"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(g["layer"][0], [e["occ_ret"], e["occ_lim"], e["agg_ret"],
                                               e["agg_lim"]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(g["loss"], e["loss"], rtol=0, atol=1e-15)
    assert g["ties"] == [False]


# ---------------------------------------------------------------------------------- P2, P3
def test_p2_single_elt_identity_terms_is_raw_loss_sum():
    pf, yet = random_case(1, n_elts=1, n_layers=1)
    pf.layer_elts = [[0]]
    pf.elt_ret[:] = 0.0
    pf.elt_lim[:] = INF
    pf.occ_ret, pf.occ_lim = np.array([0.0]), np.array([INF])
    pf.agg_ret, pf.agg_lim = np.array([0.0]), np.array([INF])
    dense = np.zeros(pf.catalogue)
    dense[pf.elt_ids[0]] = pf.elt_losses[0]
    per_event = dense[yet.event_ids]
    trial = np.repeat(np.arange(yet.n_trials), np.diff(yet.offsets))
    expect = np.bincount(trial, weights=per_event, minlength=yet.n_trials)
    y = oracle.ylt(pf, yet)[0]
    np.testing.assert_allclose(y, expect, rtol=1e-13, atol=0)
    assert y[0] == 0.0                                   # the empty trial


def test_p3_zero_retention_infinite_limits_make_terms_identity():
    pf, yet = random_case(2, n_layers=2, inf_limits=True)
    pf.elt_ret[:] = 0.0
    pf.occ_ret[:] = 0.0
    pf.occ_lim[:] = INF
    pf.agg_ret[:] = 0.0
    pf.agg_lim[:] = INF
    y = oracle.ylt(pf, yet)
    trial = np.repeat(np.arange(yet.n_trials), np.diff(yet.offsets))
    for l, elts in enumerate(pf.layer_elts):
        dense = np.zeros(pf.catalogue)
        for j in elts:
            np.add.at(dense, pf.elt_ids[j], pf.elt_losses[j])
        expect = np.bincount(trial, weights=dense[yet.event_ids], minlength=yet.n_trials)
        np.testing.assert_allclose(y[l], expect, rtol=1e-13, atol=0)


# ---------------------------------------------------------------------------------- P4
@pytest.mark.parametrize("seed", [3, 4, 5])
def test_p4_monotone_in_limits_antitone_in_retentions(seed):
    pf, yet = random_case(seed)
    base = oracle.ylt(pf, yet)
    rng = np.random.default_rng(seed)
    fields = ["elt_ret", "elt_lim", "occ_ret", "occ_lim", "agg_ret", "agg_lim"]
    moved_somewhere = 0
    for name in fields:
        for _ in range(3):
            arr = getattr(pf, name).copy()
            i = rng.integers(arr.size)
            bumped = pf.with_terms({**pf.terms_dict(), name: arr})
            getattr(bumped, name)[i] = arr[i] * rng.uniform(1.05, 1.6) + 1.0
            y = oracle.ylt(bumped, yet)
            if name.endswith("lim"):
                assert np.all(y >= base)
            else:
                assert np.all(y <= base)
            moved_somewhere += int(np.any(y != base))
    assert moved_somewhere > 0


# ---------------------------------------------------------------------------------- P5
@pytest.mark.parametrize("seed", [6, 7])
def test_p5_brute_force_second_oracle_agrees_bitwise(seed):
    pf, yet = random_case(seed, n_trials=40)
    assert np.array_equal(oracle.ylt(pf, yet), oracle.brute_ylt(pf, yet))


def test_p5_brute_force_on_tiny_workload_sample():
    pf, yet = synth.tiny(0)
    sub = synth.YET(yet.offsets[:41] - 0, yet.event_ids[:int(yet.offsets[40])])
    assert np.array_equal(oracle.ylt(pf, sub), oracle.brute_ylt(pf, sub))


# ---------------------------------------------------------------------------------- P6
def test_p6_cumulative_clamp_increments_telescope_to_year_loss():
    """Second reading of Algorithm 3: aggregate terms applied to the running total after each
    event, the year loss being the sum of the increments.  Same result (C is monotone, o >= 0)."""
    pf, yet = random_case(8)
    y = oracle.ylt(pf, yet)
    for l, elts in enumerate(pf.layer_elts):
        dense = np.zeros((len(elts), pf.catalogue))
        for q, j in enumerate(elts):
            dense[q, pf.elt_ids[j]] = pf.elt_losses[j]
        net = np.minimum(np.maximum(dense - pf.elt_ret[elts][:, None], 0), pf.elt_lim[elts][:, None])
        o = np.minimum(np.maximum(net.sum(0) - pf.occ_ret[l], 0), pf.occ_lim[l])
        C = lambda s: min(max(s - pf.agg_ret[l], 0.0), pf.agg_lim[l])
        for t in range(yet.n_trials):
            run, tot = 0.0, 0.0
            for e in yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]]:
                new = run + o[e]
                tot += C(new) - C(run)
                run = new
            assert abs(tot - y[l, t]) <= 1e-9 * max(1.0, abs(y[l, t]))


# ---------------------------------------------------------------------------------- P7
def test_p7_permutation_invariance_within_trials():
    pf, yet = random_case(9)
    rng = np.random.default_rng(9)
    ids = yet.event_ids.copy()
    for t in range(yet.n_trials):
        seg = ids[yet.offsets[t]:yet.offsets[t + 1]]
        rng.shuffle(seg)
    y1 = oracle.ylt(pf, yet)
    y2 = oracle.ylt(pf, synth.YET(yet.offsets, ids))
    np.testing.assert_allclose(y2, y1, rtol=1e-12, atol=1e-9)


def test_p7_trial_independence_subset_and_order():
    pf, yet = random_case(10)
    full = oracle.ylt(pf, yet)
    sel = np.array([5, 0, 17, 3, 3, 60])
    assert np.array_equal(oracle.ylt(pf, yet, trials=sel), full[:, sel])
    # Rebuilding a YET from a subset of trials gives the same year losses (no cross-trial state).
    trials = [yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]].tolist() for t in sel]
    assert np.array_equal(oracle.ylt(pf, trials_to_yet(trials)), full[:, sel])


# ---------------------------------------------------------------------------------- P8
def test_p8_hand_computed_order_statistics(golden_dir):
    with open(os.path.join(golden_dir, "p8_order_statistics.json")) as f:
        g = json.load(f)
    y = np.array(g["ylt"])
    for rp, v in g["pml"].items():
        assert oracle.pml(y, float(rp)) == v
    for p, v in g["tvar"].items():
        assert oracle.tvar(y, float(p)) == pytest.approx(v, rel=1e-15)


@pytest.mark.parametrize("n", [1, 7, 1000, 1001])
def test_p8_matches_sorted_definition(n):
    rng = np.random.default_rng(n)
    y = np.round(rng.lognormal(8, 2, n), 1)          # rounded: many ties
    y[: n // 3] = 0.0
    ys = sorted(y.tolist(), reverse=True)
    for rp in [1.0, 2.0, 10.0, 100.0, 250.0, 1000.0]:
        k = max(1, math.ceil(n / rp - 1e-12))
        if k > n:
            continue
        assert oracle.pml(y, rp) == ys[k - 1]
    for p in [0.0, 0.5, 0.9, 0.99, 0.996]:
        m = max(1, math.ceil(n * (1 - p) - 1e-9))
        assert oracle.tvar(y, p) == pytest.approx(sum(ys[:m]) / m, rel=1e-14)


def test_p8_decimal_reading_of_levels():
    # 1000 * (1 - 0.99) is 10.000000000000009 in binary floating point; the level is read as
    # the decimal 0.99, so the tail holds exactly 10 trials.
    assert oracle.tail_count(1000, 0.99) == 10
    assert oracle.tail_count(10 ** 6, 0.99) == 10_000
    assert oracle.rank_for_return_period(1000, 100.0) == 10
    assert oracle.rank_for_return_period(1000, 250.0) == 4
    assert oracle.rank_for_return_period(10 ** 6, 250.0) == 4000


# ---------------------------------------------------------------------------------- P9
def _regimes(pf, yet):
    """Regime signature of every clamp the objective passes through (used to certify that a
    finite-difference interval contains no kink)."""
    y, agg = oracle.ylt(pf, yet, return_agg=True)
    sig = [np.sign(agg - pf.agg_ret[:, None]), np.sign(agg - pf.agg_ret[:, None] - pf.agg_lim[:, None])]
    for l, elts in enumerate(pf.layer_elts):
        dense = np.zeros((len(elts), pf.catalogue))
        for q, j in enumerate(elts):
            dense[q, pf.elt_ids[j]] = pf.elt_losses[j]
        ex = dense - pf.elt_ret[elts][:, None]
        sig += [np.sign(ex), np.sign(ex - pf.elt_lim[elts][:, None])]
        net = np.minimum(np.maximum(ex, 0), pf.elt_lim[elts][:, None]).sum(0)
        sig += [np.sign(net - pf.occ_ret[l]), np.sign(net - pf.occ_ret[l] - pf.occ_lim[l])]
    return y, sig


@pytest.mark.parametrize("objective", ["mean", "tvar"])
def test_p9_adjoint_equals_exact_central_differences(objective):
    """The objective is piecewise linear in every term and loss, so where no clamp changes
    regime (and TVaR's top set is unchanged) inside [theta - h, theta + h] the central
    difference equals the derivative up to rounding."""
    pf, yet = random_case(11, n_trials=300, lam=30)
    level = 0.9
    g = oracle.adjoint(pf, yet, objective, level)
    y0 = oracle.ylt(pf, yet)
    w, _ = oracle.objective_weights(y0, objective, level)
    top0 = [set(np.nonzero(w[l])[0].tolist()) for l in range(pf.n_layers)]

    def J(p):
        y = oracle.ylt(p, yet)
        if objective == "mean":
            return y.mean(1)
        return np.array([oracle.tvar(y[l], level) for l in range(p.n_layers)])

    checked = 0
    params = [("elt_ret", i) for i in range(pf.n_elts)] + [("elt_lim", i) for i in range(pf.n_elts)]
    params += [(n, l) for n in ["occ_ret", "occ_lim", "agg_ret", "agg_lim"] for l in range(pf.n_layers)]
    for name, i in params:
        theta = getattr(pf, name)[i]
        h = 1e-4 * abs(theta)
        pp, pm = pf.with_terms(pf.terms_dict()), pf.with_terms(pf.terms_dict())
        getattr(pp, name)[i] = theta + h
        getattr(pm, name)[i] = theta - h
        yp, sp = _regimes(pp, yet)
        ym, sm = _regimes(pm, yet)
        if any(not np.array_equal(a, b) for a, b in zip(sp, sm)):
            continue
        if objective == "tvar":
            wp, _ = oracle.objective_weights(yp, objective, level)
            wm, _ = oracle.objective_weights(ym, objective, level)
            if any(set(np.nonzero(wp[l])[0].tolist()) != top0[l] or
                   set(np.nonzero(wm[l])[0].tolist()) != top0[l] for l in range(pf.n_layers)):
                continue
        fd = (J(pp) - J(pm)) / (2 * h)
        for l, elts in enumerate(pf.layer_elts):
            if name.startswith("elt"):
                if i not in elts:
                    assert fd[l] == pytest.approx(0.0, abs=1e-9)
                    continue
                row = int(pf.layer_csr()[0][l]) + elts.index(i)
                an = g["elt"][row, 0 if name == "elt_ret" else 1]
            else:
                if l != i:
                    continue
                an = g["layer"][l, ["occ_ret", "occ_lim", "agg_ret", "agg_lim"].index(name)]
            assert fd[l] == pytest.approx(an, rel=1e-6, abs=1e-9), (name, i, l)
            checked += 1
    assert checked >= 10
    # Losses: perturb a few records that sit inside every regime.
    rng = np.random.default_rng(12)
    for _ in range(12):
        j = int(rng.integers(pf.n_elts))
        r = int(rng.integers(pf.elt_ids[j].size))
        x = pf.elt_losses[j][r]
        h = 1e-4 * x
        lp = [a.copy() for a in pf.elt_losses]
        lm = [a.copy() for a in pf.elt_losses]
        lp[j][r] = x + h
        lm[j][r] = x - h
        pp = synth.Portfolio(pf.catalogue, pf.elt_ids, lp, pf.elt_ret, pf.elt_lim, pf.layer_elts,
                             pf.occ_ret, pf.occ_lim, pf.agg_ret, pf.agg_lim)
        pm = synth.Portfolio(pf.catalogue, pf.elt_ids, lm, pf.elt_ret, pf.elt_lim, pf.layer_elts,
                             pf.occ_ret, pf.occ_lim, pf.agg_ret, pf.agg_lim)
        yp, sp = _regimes(pp, yet)
        ym, sm = _regimes(pm, yet)
        if any(not np.array_equal(a, b) for a, b in zip(sp, sm)):
            continue
        fd = (J(pp) - J(pm)) / (2 * h)
        for l, elts in enumerate(pf.layer_elts):
            if j not in elts:
                continue
            pos = int(g["loss_offsets"][l]) + sum(pf.elt_ids[k].size for k in elts[:elts.index(j)]) + r
            assert fd[l] == pytest.approx(g["loss"][pos], rel=1e-6, abs=1e-9)
            checked += 1


# ---------------------------------------------------------------------------------- invariants
def test_invariants_range_and_absent_events():
    pf, yet = random_case(13)
    y = oracle.ylt(pf, yet)
    assert np.all(y >= 0) and np.all(y <= pf.agg_lim[:, None])
    # a trial made only of events that no ELT contains loses nothing
    covered = set(np.concatenate(pf.elt_ids).tolist())
    free = [e for e in range(pf.catalogue) if e not in covered][:5]
    y2 = oracle.ylt(pf, trials_to_yet([free, []]))
    assert np.all(y2 == 0.0)


def test_tiny_workload_regimes_are_not_degenerate():
    pf, yet = synth.tiny(0)
    y, agg = oracle.ylt(pf, yet, return_agg=True)
    below = np.mean(agg[0] <= pf.agg_ret[0])
    above = np.mean(agg[0] >= pf.agg_ret[0] + pf.agg_lim[0])
    assert 0.0 < 1 - below - above
    assert np.mean(y[0] > 0) > 0.5


def test_tvar_weights_share_the_boundary_among_ties():
    """Symmetric tie rule: y = 10, 5, 5, 5, 0 and p = 0.6 give m = 2 and v = 5; the trial above
    v gets 1/2 and the three tied trials share the remaining 1/2 (1/6 each); the weighted sum
    is TVaR = (10 + 5) / 2 = 7.5."""
    y = np.array([[10.0, 5.0, 5.0, 5.0, 0.0]])
    w, ties = oracle.objective_weights(y, "tvar", 0.6)
    assert w[0].tolist() == [0.5, 1 / 6, 1 / 6, 1 / 6, 0.0]
    assert ties == [True]
    assert float(w[0] @ y[0]) == pytest.approx(oracle.tvar(y[0], 0.6), rel=1e-15)
    w, ties = oracle.objective_weights(np.array([[10.0, 5.0, 4.0]]), "tvar", 0.5)
    assert w[0].tolist() == [0.5, 0.5, 0.0] and ties == [False]


# ---------------------------------------------------------------------------------- OEP basis
def test_oep_hand_worked(golden_dir):
    pf, yet, exp = load_p1(golden_dir)
    assert oracle.ylt_oep(pf, yet)[0].tolist() == exp["ylt_oep"]


def test_oep_properties():
    """max <= sum (with identity aggregate terms); one-event trials give o(e) itself; the same
    quantity written differently (numpy over dense tables) agrees exactly."""
    pf, yet = random_case(14)
    oep = oracle.ylt_oep(pf, yet)
    ident = pf.with_terms({**pf.terms_dict(), "agg_ret": [0.0] * pf.n_layers,
                           "agg_lim": [INF] * pf.n_layers})
    assert np.all(oep <= oracle.ylt(ident, yet) + 1e-9)
    for l, elts in enumerate(pf.layer_elts):
        dense = np.zeros((len(elts), pf.catalogue))
        for q, j in enumerate(elts):
            dense[q, pf.elt_ids[j]] = pf.elt_losses[j]
        net = np.minimum(np.maximum(dense - pf.elt_ret[elts][:, None], 0), pf.elt_lim[elts][:, None])
        s = np.zeros(pf.catalogue)
        for q in range(len(elts)):          # layer order, as the definition
            s = s + net[q]
        o = np.minimum(np.maximum(s - pf.occ_ret[l], 0), pf.occ_lim[l])
        want = np.array([o[yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]]].max(initial=0.0)
                         for t in range(yet.n_trials)])
        assert np.array_equal(oep[l], want)
    one = synth.YET(np.arange(51, dtype=np.int64), np.arange(50, dtype=np.int32) * 5)
    assert np.all(oracle.ylt_oep(pf, one) == oracle.ylt(ident.with_terms({**ident.terms_dict()}), one))
