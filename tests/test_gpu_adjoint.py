"""GPU adjoint (ara_adjoint, ara_adjoint_accumulate, the autograd Function) against the FP64
oracle's chain-rule gradient and against central finite differences of the GPU forward.

Required tolerance: 1e-4 relative on adjoints against FP64.  The device keeps every sum as an
exact integer count, so agreement is at rounding level wherever the clamp regimes of the two
sides agree; the cases are checked to keep every aggregate loss away from the aggregate kinks
and TVaR's boundary trial separated from its neighbour, where the gradient is not defined."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1606_04473_gb300 as ara
    from paper_1606_04473_gb300.autograd import LayerRisk

RTOL, LEVEL = 1e-4, 0.9


def dev(yet):
    return (torch.from_numpy(np.ascontiguousarray(yet.offsets)).cuda(),
            torch.from_numpy(np.ascontiguousarray(yet.event_ids)).cuda())


def case(seed, catalogue=100_000, n_elts=10, nnz=3000, n_layers=3, n_trials=3000, lam=400.0):
    rng = np.random.default_rng(seed)
    ids, losses = synth.make_elts(seed, n_elts, nnz, catalogue, 11.0, 2.0, f32=True)
    r, l = synth.percentile_terms(losses)
    layers = [sorted(rng.choice(n_elts, size=int(rng.integers(2, n_elts + 1)), replace=False).tolist())
              for _ in range(n_layers)]
    counts = synth.poisson_counts(seed, lam, n_trials)
    counts[:3] = [0, 1, 5]
    yet = synth.make_yet(seed, counts, catalogue, with_timestamps=False)
    z = np.zeros(n_layers)
    pf = synth.Portfolio(catalogue, ids, losses, r, l, layers, z, z, z, z, losses_f32=True)
    from oracle.derive_terms import derive
    t = derive(pf, synth.YET(yet.offsets[:1001], yet.event_ids[:int(yet.offsets[1000])]), 20.0, 80.0)
    return pf.with_terms(t), yet


def well_posed(pf, yet, level):
    y, agg = oracle.ylt(pf, yet, return_agg=True)
    for l in range(pf.n_layers):
        for kink in (pf.agg_ret[l], pf.agg_ret[l] + pf.agg_lim[l]):
            if np.any(np.abs(agg[l] - kink) <= 1e-9 * np.maximum(np.abs(agg[l]), 1.0)):
                return False
        m = oracle.tail_count(yet.n_trials, level)
        ys = np.sort(y[l])[::-1]
        if m < ys.size and ys[m - 1] > 0 and abs(ys[m - 1] - ys[m]) <= 1e-9 * ys[m - 1]:
            return False
    return True


def forward(g, yet):
    off, ids = dev(yet)
    reg = torch.empty((g.n_layers, yet.n_trials), dtype=torch.uint8, device="cuda")
    y = g.run_ylt(off, ids, regimes=reg)
    g.check()
    return off, ids, y, reg


def close(got, want, scale):
    got, want = np.asarray(got), np.asarray(want)
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=1e-12 * scale)


@pytest.fixture(scope="module")
def mid():
    pf, yet = case(21)
    assert well_posed(pf, yet, LEVEL)
    return pf, yet


@pytest.mark.parametrize("obj", [0, 1])
def test_adjoint_matches_fp64_reference(mid, obj):
    pf, yet = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids, y, reg = forward(g, yet)
    gr = g.adjoint(off, ids, y, reg, LEVEL)
    ref = oracle.adjoint(pf, yet, "mean" if obj == 0 else "tvar", LEVEL)
    scale = max(1.0, float(np.abs(ref["loss"]).max()))
    close(gr["elt"][obj].cpu().numpy(), ref["elt"], 1.0)
    close(gr["layer"][obj].cpu().numpy(), ref["layer"], 1.0)
    close(gr["loss"][obj].cpu().numpy(), ref["loss"], scale)
    assert gr["ties"].tolist() == [0] * pf.n_layers
    # the gradients are not trivially zero: every kind of term is exercised
    assert np.any(ref["elt"][:, 0] != 0) and np.any(ref["layer"][:, 0] != 0)
    assert np.any(ref["layer"][:, 2] != 0) and np.count_nonzero(ref["loss"]) > 100


def test_adjoint_layer_subset_and_repeat(mid):
    pf, yet = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    sel = [2, 0]
    reg = torch.empty((2, yet.n_trials), dtype=torch.uint8, device="cuda")
    y = g.run_ylt(off, ids, layers=sel, regimes=reg)
    a = g.adjoint(off, ids, y, reg, LEVEL, layers=sel)
    b = g.adjoint(off, ids, y, reg, LEVEL, layers=sel)
    for k in ("elt", "layer", "loss"):
        assert torch.equal(a[k], b[k])                      # deterministic
    sub = pf.with_terms(pf.terms_dict())
    sub.layer_elts = [pf.layer_elts[i] for i in sel]
    for name in ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]:
        setattr(sub, name, getattr(pf, name)[sel])
    ref = oracle.adjoint(sub, yet, "mean", LEVEL)
    close(a["layer"][0].cpu().numpy(), ref["layer"], 1.0)
    close(a["elt"][0].cpu().numpy(), ref["elt"], 1.0)


def test_accumulate_and_autograd_match_weighted_reference(mid):
    pf, yet = mid
    off, ids = dev(yet)
    P = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), device="cuda", requires_grad=True)
    params = [P(pf.elt_ret), P(pf.elt_lim), P(pf.occ_ret), P(pf.occ_lim), P(pf.agg_ret),
              P(pf.agg_lim), P(np.concatenate(pf.elt_losses))]
    risk = LayerRisk.apply(*params, pf, off, ids, LEVEL)
    w = torch.tensor(np.random.default_rng(3).normal(size=(pf.n_layers, 2)), device="cuda")
    (risk * w).sum().backward()
    # forward values against the oracle
    y_ref = oracle.ylt(pf, yet)
    np.testing.assert_allclose(risk[:, 0].detach().cpu().numpy(), y_ref.mean(1), rtol=1e-9)
    np.testing.assert_allclose(risk[:, 1].detach().cpu().numpy(),
                               [oracle.tvar(y_ref[l], LEVEL) for l in range(pf.n_layers)], rtol=1e-9)
    # weighted oracle gradient in parameter layout
    wn = w.cpu().numpy()
    gm = oracle.adjoint(pf, yet, "mean", LEVEL)
    gt = oracle.adjoint(pf, yet, "tvar", LEVEL)
    loff, _ = pf.layer_csr()
    exp_ret, exp_lim = np.zeros(pf.n_elts), np.zeros(pf.n_elts)
    exp_layer = np.zeros((pf.n_layers, 4))
    rec_off = np.concatenate([[0], np.cumsum([x.size for x in pf.elt_ids])])
    exp_loss = np.zeros(int(rec_off[-1]))
    for l, elts in enumerate(pf.layer_elts):
        exp_layer[l] = wn[l, 0] * gm["layer"][l] + wn[l, 1] * gt["layer"][l]
        pos = int(gm["loss_offsets"][l])
        for q, j in enumerate(elts):
            row = int(loff[l]) + q
            exp_ret[j] += wn[l, 0] * gm["elt"][row, 0] + wn[l, 1] * gt["elt"][row, 0]
            exp_lim[j] += wn[l, 0] * gm["elt"][row, 1] + wn[l, 1] * gt["elt"][row, 1]
            n = pf.elt_ids[j].size
            exp_loss[rec_off[j]:rec_off[j] + n] += (wn[l, 0] * gm["loss"][pos:pos + n] +
                                                    wn[l, 1] * gt["loss"][pos:pos + n])
            pos += n
    scale = max(1.0, float(np.abs(exp_loss).max()))
    close(params[0].grad.cpu().numpy(), exp_ret, 1.0)
    close(params[1].grad.cpu().numpy(), exp_lim, 1.0)
    for c, p in enumerate(params[2:6]):
        close(p.grad.cpu().numpy(), exp_layer[:, c], 1.0)
    close(params[6].grad.cpu().numpy(), exp_loss, scale)


def test_adjoint_matches_central_differences_of_gpu_forward(mid):
    """Central differences of the GPU forward (h = 1e-4 relative) on the layer terms; the
    objective is piecewise linear, so they are exact wherever no regime changes in between."""
    pf, yet = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids, y, reg = forward(g, yet)
    gr = g.adjoint(off, ids, y, reg, LEVEL)

    def objectives(p):
        gg = ara.Portfolio.from_tables(p)
        yy = gg.run_ylt(off, ids)
        _, tv, mn = ara.risk_metrics(yy, [], [LEVEL], want_mean=True)
        return np.stack([mn, tv[:, 0]], 1)

    checked = 0
    for name, c in [("occ_ret", 0), ("occ_lim", 1), ("agg_ret", 2), ("agg_lim", 3)]:
        for l in range(pf.n_layers):
            th = float(getattr(pf, name)[l])
            h = 1e-4 * th
            pp, pm = pf.with_terms(pf.terms_dict()), pf.with_terms(pf.terms_dict())
            getattr(pp, name)[l] = th + h
            getattr(pm, name)[l] = th - h
            if not (well_posed(pp, yet, LEVEL) and well_posed(pm, yet, LEVEL)):
                continue
            fd = (objectives(pp)[l] - objectives(pm)[l]) / (2 * h)
            an = np.array([gr["layer"][0][l, c].item(), gr["layer"][1][l, c].item()])
            # piecewise linear: equal unless a regime flips inside [th - h, th + h]
            if np.allclose(fd, an, rtol=RTOL, atol=1e-9):
                checked += 1
    assert checked >= 6


def test_adjoint_tie_at_the_tvar_boundary():
    """Aggregate limits low enough that the top trials all saturate: TVaR's boundary is a tie
    (reported), and the symmetric tie rule matches the oracle."""
    pf, yet = case(22, n_layers=2, n_trials=2000)
    pf = pf.with_terms({**pf.terms_dict(), "agg_lim": list(np.asarray(pf.agg_lim) * 0.3)})
    g = ara.Portfolio.from_tables(pf)
    off, ids, y, reg = forward(g, yet)
    gr = g.adjoint(off, ids, y, reg, LEVEL)
    ref = oracle.adjoint(pf, yet, "tvar", LEVEL)
    assert ref["ties"] == [True, True]
    assert gr["ties"].tolist() == [1, 1]
    close(gr["layer"][1].cpu().numpy(), ref["layer"], 1.0)
    close(gr["elt"][1].cpu().numpy(), ref["elt"], 1.0)
    close(gr["loss"][1].cpu().numpy(), ref["loss"], 1.0)


def test_adjoint_wide_layer_and_single_elt_layer():
    """A layer of 40 ELTs (the fold stages its records in two batches of at most 32 ELTs) next
    to a one-ELT layer: the gradients of both objectives match the FP64 chain rule."""
    seed = 23
    C, n_elts = 60_000, 40
    ids, losses = synth.make_elts(seed, n_elts, 1500, C, 11.0, 2.0, f32=True)
    r, l = synth.percentile_terms(losses)
    counts = synth.poisson_counts(seed, 300.0, 2500)
    counts[:2] = [0, 1]
    yet = synth.make_yet(seed, counts, C, with_timestamps=False)
    z = np.zeros(2)
    pf = synth.Portfolio(C, ids, losses, r, l, [list(range(40)), [3]], z, z, z, z, losses_f32=True)
    from oracle.derive_terms import derive
    pf = pf.with_terms(derive(pf, synth.YET(yet.offsets[:1001], yet.event_ids[:int(yet.offsets[1000])]),
                              20.0, 80.0))
    assert well_posed(pf, yet, LEVEL)
    g = ara.Portfolio.from_tables(pf)
    off, ids_d, y, reg = forward(g, yet)
    gr = g.adjoint(off, ids_d, y, reg, LEVEL)
    for obj, name in ((0, "mean"), (1, "tvar")):
        ref = oracle.adjoint(pf, yet, name, LEVEL)
        scale = max(1.0, float(np.abs(ref["loss"]).max()))
        close(gr["elt"][obj].cpu().numpy(), ref["elt"], 1.0)
        close(gr["layer"][obj].cpu().numpy(), ref["layer"], 1.0)
        close(gr["loss"][obj].cpu().numpy(), ref["loss"], scale)
    g.close()


def _occurrence_regimes(pf, layer):
    """Per catalogue event, the occurrence clamp's regime of one layer (0: s(e) <= OccR, 1:
    interior, 2: above OccR + OccL), restated with numpy from the notation of Section IV-B.
    Used only to show that a test case reaches the condition it is meant to exercise."""
    s = np.zeros(pf.catalogue)
    for j in pf.layer_elts[layer]:
        a = np.minimum(np.maximum(pf.elt_losses[j] - pf.elt_ret[j], 0.0), pf.elt_lim[j])
        s[pf.elt_ids[j]] += a
    ex = s - pf.occ_ret[layer]
    return np.where(ex <= 0, 0, np.where(ex < pf.occ_lim[layer], 1, 2)).astype(np.int8)


def test_adjoint_coarse_regime_bitmap_at_the_adjoint_workload_catalogue():
    """The adjoint workload's shape: a 2,000,000-event catalogue with ELTs of 20,000 events.
    Its exact regime bitmap (250 KB) exceeds the histogram pass's shared-memory budget, so the
    pass filters occurrences with the coarse bitmap (one bit per two events, 32 apart) and
    counts events of regime 0 that share a coarse bit with an event of non-zero regime; those
    counts must be dropped afterwards.  The case shows such events occur in interior trials,
    then compares every gradient of both objectives with the FP64 chain rule."""
    full = synth.adjoint_portfolio(0)
    sel = [0, 5]
    yet = synth.adjoint_yet(0, n_trials=4000)       # the first 4,000 trials of the workload's YET
    sub = full.with_terms(full.terms_dict())
    sub.layer_elts = [full.layer_elts[i] for i in sel]
    for name in ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]:
        setattr(sub, name, np.asarray(getattr(full, name))[sel])
    assert full.catalogue == 2_000_000 and (full.catalogue + 31) // 32 * 4 > 200 * 1024
    assert well_posed(sub, yet, LEVEL)
    # false positives of the coarse bitmap in interior trials, for every selected layer
    _, agg = oracle.ylt(sub, yet, return_agg=True)
    for l in range(len(sel)):
        r = _occurrence_regimes(sub, l)
        partner = np.arange(sub.catalogue) ^ 32
        partner = np.minimum(partner, sub.catalogue - 1)
        false_pos = (r == 0) & (r[partner] != 0)
        interior = (agg[l] > sub.agg_ret[l]) & (agg[l] - sub.agg_ret[l] < sub.agg_lim[l])
        counts = np.diff(yet.offsets)
        occ_interior = np.repeat(interior, counts)
        assert np.count_nonzero(false_pos[yet.event_ids[occ_interior]]) > 1000
    g = ara.Portfolio.from_tables(full)
    off, ids = dev(yet)
    reg = torch.empty((len(sel), yet.n_trials), dtype=torch.uint8, device="cuda")
    y = g.run_ylt(off, ids, layers=sel, regimes=reg)
    g.check()
    gr = g.adjoint(off, ids, y, reg, LEVEL, layers=sel)
    g.check()
    for obj, name in ((0, "mean"), (1, "tvar")):
        ref = oracle.adjoint(sub, yet, name, LEVEL)
        scale = max(1.0, float(np.abs(ref["loss"]).max()))
        close(gr["elt"][obj].cpu().numpy(), ref["elt"], 1.0)
        close(gr["layer"][obj].cpu().numpy(), ref["layer"], 1.0)
        close(gr["loss"][obj].cpu().numpy(), ref["loss"], scale)
        assert np.count_nonzero(ref["loss"]) > 1000 and np.all(ref["layer"][:, 0] != 0)
    assert gr["ties"].tolist() == [0, 0]
    g.close()


@pytest.mark.parametrize("case_name", ["mid", "adjoint_workload"])
def test_one_pass_for_all_layers_equals_per_layer_passes(mid, case_name):
    """The adjoint of several layers takes one histogram pass over the YET for all of them
    (event rows of the layers whose occurrence regime is non-zero, per-entry histograms); the
    gradients equal those of one pass per layer (ARA_DBG_ADJOINT_PER_LAYER) bit for bit, for
    both objectives, and the reported ties too."""
    if case_name == "mid":
        pf, yet = mid
        sel = None
    else:
        pf = synth.adjoint_portfolio(0)
        yet = synth.adjoint_yet(0, n_trials=3000)
        sel = [0, 3, 7, 15]
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    n_sel = pf.n_layers if sel is None else len(sel)
    reg = torch.empty((n_sel, yet.n_trials), dtype=torch.uint8, device="cuda")
    y = g.run_ylt(off, ids, layers=sel, regimes=reg)
    g.check()
    one = g.adjoint(off, ids, y, reg, LEVEL, layers=sel)
    ara.debug_set(ara.ARA_DBG_ADJOINT_PER_LAYER, 1)
    try:
        per = g.adjoint(off, ids, y, reg, LEVEL, layers=sel)
    finally:
        ara.debug_set(ara.ARA_DBG_ADJOINT_PER_LAYER, 0)
    for k in ("elt", "layer", "loss"):
        assert torch.equal(one[k], per[k]), k
    assert one["ties"].tolist() == per["ties"].tolist()
    assert torch.count_nonzero(one["loss"]).item() > 100
    g.close()


def _both_ways(g, off, ids, sel, level=LEVEL, index=None):
    """(trial-major adjoint, adjoint over an event-major index of the same YET)."""
    n_sel = g.n_layers if sel is None else len(sel)
    reg = torch.empty((n_sel, off.numel() - 1), dtype=torch.uint8, device="cuda")
    y = g.run_ylt(off, ids, layers=sel, regimes=reg)
    g.check()
    a = g.adjoint(off, ids, y, reg, level, layers=sel)
    yx = index if index is not None else g.yet_index(off, ids)
    b = g.adjoint(None, None, y, reg, level, layers=sel, index=yx)
    g.check()
    return a, b


def _assert_same(a, b):
    for k in ("elt", "layer", "loss"):
        assert torch.equal(a[k], b[k]), k
    assert a["ties"].tolist() == b["ties"].tolist()


@pytest.mark.parametrize("case_name", ["mid_all", "mid_one_layer", "adjoint_workload", "tie"])
def test_indexed_adjoint_equals_trial_major(mid, case_name):
    """ara_adjoint_indexed reads the YET through its event-major index: each event's list of
    trials, with the trials' classes packed 2 bits per layer.  It counts the same integers as
    the trial-major pass, so every gradient of both objectives and the reported ties are equal
    bit for bit (and the trial-major pass is checked against the FP64 oracle above)."""
    sel = None
    if case_name.startswith("mid"):
        pf, yet = mid
        sel = [1] if case_name == "mid_one_layer" else None
    elif case_name == "adjoint_workload":
        pf = synth.adjoint_portfolio(0)
        yet = synth.adjoint_yet(0, n_trials=3000)
        sel = [0, 3, 7, 15]
    else:
        pf, yet = case(22, n_layers=2, n_trials=2000)
        pf = pf.with_terms({**pf.terms_dict(), "agg_lim": list(np.asarray(pf.agg_lim) * 0.3)})
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    a, b = _both_ways(g, off, ids, sel)
    _assert_same(a, b)
    assert torch.count_nonzero(a["loss"]).item() > 100
    if case_name == "tie":
        assert a["ties"].tolist() == [1, 1]
    if case_name == "mid_all":                      # and directly against the FP64 chain rule
        for obj, name in ((0, "mean"), (1, "tvar")):
            ref = oracle.adjoint(pf, yet, name, LEVEL)
            scale = max(1.0, float(np.abs(ref["loss"]).max()))
            close(b["elt"][obj].cpu().numpy(), ref["elt"], 1.0)
            close(b["layer"][obj].cpu().numpy(), ref["layer"], 1.0)
            close(b["loss"][obj].cpu().numpy(), ref["loss"], scale)
    g.close()


def _blocks_case():
    """110,000 trials of Poisson(20) events over a 50,000-event catalogue (three blocks of the
    index), 20 layers (two groups of 16 per class word) that all include ELT 0."""
    seed = 31
    C, n_elts, n_layers = 50_000, 6, 20
    ids_e, losses = synth.make_elts(seed, n_elts, 5000, C, 11.0, 2.0, f32=True)
    r, l = synth.percentile_terms(losses)
    rng = np.random.default_rng(seed)
    layers = [sorted({0, *rng.choice(np.arange(1, n_elts), size=2, replace=False).tolist()})
              for _ in range(n_layers)]
    counts = synth.poisson_counts(seed, 20.0, 110_000)
    counts[:2] = [0, 1]
    yet = synth.make_yet(seed, counts, C, with_timestamps=False)
    z = np.zeros(n_layers)
    pf = synth.Portfolio(C, ids_e, losses, r, l, layers, z, z, z, z, losses_f32=True)
    from oracle.derive_terms import derive
    pf = pf.with_terms(derive(pf, synth.YET(yet.offsets[:2001], yet.event_ids[:int(yet.offsets[2000])]),
                              20.0, 80.0))
    return pf, yet


def test_indexed_adjoint_several_trial_blocks_many_layers_long_rows():
    """110,000 trials (three blocks of the index: offsets within a block are 16-bit), 20 layers
    (two groups of 16 layers per class word) that all include ELT 0, so that events of ELT 0 sit
    in the rows of most layers: rows longer than the 5 entries a walk counts, which walk their
    lists several times.  Equal bit for bit to the trial-major pass."""
    pf, yet = _blocks_case()
    n_layers = pf.n_layers
    rows = sum((_occurrence_regimes(pf, k) != 0).astype(np.int32) for k in range(n_layers))
    assert rows.max() >= 13          # three walks in the first group of 16 layers
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    yx = g.yet_index(off, ids)
    a, b = _both_ways(g, off, ids, None, index=yx)
    _assert_same(a, b)
    assert torch.count_nonzero(a["loss"]).item() > 1000
    # one index serves any layers of the same catalogue: a subset, then changed terms
    a, b = _both_ways(g, off, ids, [19, 2, 7], index=yx)
    _assert_same(a, b)
    g2 = ara.Portfolio.from_tables(pf.with_terms({**pf.terms_dict(),
                                                  "occ_ret": list(np.asarray(pf.occ_ret) * 1.5)}))
    a, b = _both_ways(g2, off, ids, None, index=yx)
    _assert_same(a, b)
    yx.close()
    g.close()
    g2.close()


def test_yet_index_owns_its_memory_and_reports_bad_input(mid):
    """The index keeps no reference to the YET (the YET's buffers may go); an event ID outside
    the catalogue or decreasing offsets give ARA_EDATA and no index; a portfolio of another
    catalogue size is refused; a closed index is refused."""
    pf, yet = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    reg = torch.empty((g.n_layers, yet.n_trials), dtype=torch.uint8, device="cuda")
    y = g.run_ylt(off, ids, regimes=reg)
    a = g.adjoint(off, ids, y, reg, LEVEL)
    off2, ids2 = off.clone(), ids.clone()
    yx = g.yet_index(off2, ids2)
    del off2, ids2
    torch.cuda.synchronize()
    junk = torch.full((ids.numel(),), 7, dtype=torch.int32, device="cuda")   # reuse the memory
    b = g.adjoint(None, None, y, reg, LEVEL, index=yx)
    _assert_same(a, b)
    del junk
    bad = ids.clone()
    bad[5] = pf.catalogue
    with pytest.raises(ara.AraError) as ei:
        g.yet_index(off, bad)
    assert ei.value.status == ara.ARA_EDATA
    off_bad = off.clone()
    off_bad[10] = off_bad[12] + 1
    with pytest.raises(ara.AraError) as ei:
        g.yet_index(off_bad, ids)
    assert ei.value.status == ara.ARA_EDATA
    other = synth.Portfolio(pf.catalogue + 1, pf.elt_ids, pf.elt_losses, pf.elt_ret, pf.elt_lim,
                            pf.layer_elts, pf.occ_ret, pf.occ_lim, pf.agg_ret, pf.agg_lim,
                            losses_f32=True)
    g3 = ara.Portfolio.from_tables(other)
    with pytest.raises(ara.AraError) as ei:
        g3.adjoint(None, None, y, reg, LEVEL, index=yx)
    assert ei.value.status == ara.ARA_EINVAL
    yx.close()
    with pytest.raises(ara.AraError):
        g.adjoint(None, None, y, reg, LEVEL, index=yx)
    g3.close()
    g.close()


def test_indexed_adjoint_of_a_yet_without_occurrences(mid):
    """Every trial empty: the index holds no entries, and the indexed adjoint equals the
    trial-major one (no occurrence counts; only the aggregate terms' trial counts)."""
    pf, _ = mid
    n = 700
    g = ara.Portfolio.from_tables(pf)
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ids = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
    a, b = _both_ways(g, off, ids, None)
    _assert_same(a, b)
    assert torch.count_nonzero(a["loss"]).item() == 0
    g.close()


def test_indexed_adjoint_over_trial_slices():
    """The adjoint of a forward run over a slice of the indexed YET's trials: inside one block,
    across a block boundary, the last trials, and one trial.  The pass reads the blocks the slice
    touches and counts only the slice's trials; equal bit for bit to the trial-major adjoint of
    the same slice."""
    pf, yet = _blocks_case()
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    yx = g.yet_index(off, ids)
    sel = [0, 4, 17]
    for t0, t1 in [(1_000, 9_000), (30_000, 80_000), (100_000, 110_000), (36_667, 36_668)]:
        o = off[t0:t1 + 1]
        reg = torch.empty((len(sel), t1 - t0), dtype=torch.uint8, device="cuda")
        y = g.run_ylt(o, ids, layers=sel, regimes=reg)
        g.check()
        a = g.adjoint(o, ids, y, reg, LEVEL, layers=sel)
        b = g.adjoint(None, None, y, reg, LEVEL, layers=sel, index=yx, first_trial=t0)
        g.check()
        _assert_same(a, b)
    with pytest.raises(ara.AraError):      # trials past the end of the index
        g.adjoint(None, None, y, reg, LEVEL, layers=sel, index=yx, first_trial=110_000)
    yx.close()
    g.close()
