"""GPU parity of the batched-portfolio plan (ara_plan_batched / ara_plan_launch): every selected
layer in one YET pass, replayed as a CUDA graph.  Its YLT must equal the single-layer path bit
for bit (same folds, same fixed point, exact integer sums) and the FP64 oracle within the YLT
tolerance."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1606_04473_gb300 as ara


def dev(yet):
    return (torch.from_numpy(np.ascontiguousarray(yet.offsets)).cuda(),
            torch.from_numpy(np.ascontiguousarray(yet.event_ids)).cuda())


def small_batched(seed=0, n_trials=3000):
    """The batched recipe at reduced size: 20 layers of U{3..30} ELTs from a pool of 40 ELTs
    over a 200,000-event catalogue, uneven trial lengths (Poisson, mean U[20, 400])."""
    rng = np.random.default_rng(seed)
    C, pool = 200_000, 40
    ids, losses = synth.make_elts(seed, pool, 2000, C, 11.0, 2.0, f32=True)
    r, l = synth.percentile_terms(losses)
    layers = [sorted(rng.choice(pool, size=int(rng.integers(3, 31)), replace=False).tolist())
              for _ in range(20)]
    lam = rng.uniform(20, 400, n_trials)
    counts = synth.poisson_counts(seed, lam, n_trials)
    counts[:4] = [0, 1, 0, 3]
    yet = synth.make_yet(seed, counts, C, with_timestamps=False)
    z = np.zeros(20)
    pf = synth.Portfolio(C, ids, losses, r, l, layers, z, z, z, z, losses_f32=True)
    from oracle.derive_terms import derive
    t = derive(pf, synth.YET(yet.offsets[:1001], yet.event_ids[:int(yet.offsets[1000])]), 20.0, 80.0)
    return pf.with_terms(t), yet


@pytest.fixture(scope="module")
def case():
    pf, yet = small_batched()
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    return pf, yet, ref, agg


@pytest.mark.parametrize("autotune", [False, True])
def test_plan_equals_single_layer_path_and_oracle(case, autotune):
    pf, yet, ref, agg = case
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    reg_a = torch.empty((pf.n_layers, yet.n_trials), dtype=torch.uint8, device="cuda")
    reg_b = torch.empty_like(reg_a)
    single = g.run_ylt(off, ids, regimes=reg_a).clone()
    plan = ara.BatchedPlan(g, off, ids, regimes=reg_b, autotune=autotune)
    for _ in range(2):                      # replays recompute everything
        plan.out.fill_(-1.0)
        y = plan.launch()
        g.check()
        assert torch.equal(y, single)
        assert torch.equal(reg_b, reg_a)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= 1e-6 * np.abs(ref) + 1e-12 * np.abs(agg))
    info = plan.info()
    assert info["warps"] in (8, 16, 32) and info["blocks_per_sm"] in (1, 2, 4)
    assert info["accumulator_copies"] in (1, 2, 4) and info["trials_per_grab"] in (1, 2, 4)
    if autotune:
        assert info["tuned_ms"] > 0
    plan.close()


def test_plan_layer_subset_and_rebound_inputs(case):
    pf, yet, ref, agg = case
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    plan = ara.BatchedPlan(g, off, ids, layers=[5, 0, 19], autotune=False)
    y = plan.launch().clone()
    np.testing.assert_allclose(y.cpu().numpy(), ref[[5, 0, 19]], rtol=1e-6,
                               atol=1e-12 * float(np.abs(agg).max()))
    ids.copy_(torch.flip(ids, [0]))          # new YET contents in the bound buffer
    y2 = plan.launch()
    single = g.run_ylt(off, ids, layers=[5, 0, 19])
    assert torch.equal(y2, single)
    plan.close()


def test_plan_with_many_layers_equals_single_layer_path():
    """130 layers of 1-4 ELTs (more than two groups of 64 layer slots in the table): the plan's
    YLT equals the single-layer path bit for bit, and the oracle's raw trial sums (zero
    retentions, infinite limits at the layer level) within the YLT tolerance."""
    rng = np.random.default_rng(5)
    C, pool, nl = 200_000, 40, 130
    ids, losses = synth.make_elts(5, pool, 2000, C, 11.0, 2.0, f32=True)
    r, l = synth.percentile_terms(losses)
    layers = [sorted(rng.choice(pool, size=int(rng.integers(1, 5)), replace=False).tolist())
              for _ in range(nl)]
    counts = synth.poisson_counts(5, 200.0, 1500)
    counts[:3] = [0, 1, 2]
    yet = synth.make_yet(5, counts, C, with_timestamps=False)
    z, inf = np.zeros(nl), np.full(nl, np.inf)
    pf = synth.Portfolio(C, ids, losses, r, l, layers, z, inf, z, inf, losses_f32=True)
    g = ara.Portfolio.from_tables(pf)
    off, ev = dev(yet)
    single = g.run_ylt(off, ev).clone()
    plan = ara.BatchedPlan(g, off, ev, autotune=False)
    y = plan.launch()
    g.check()
    assert torch.equal(y, single)
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= 1e-6 * np.abs(ref) + 1e-12 * np.abs(agg))
    plan.close()
    g.close()


def test_plan_skips_and_reports_out_of_range_ids(case):
    """Event IDs outside the catalogue (the catalogue size, -1, 2^31 - 1) at the first, the
    33rd and the 65th occurrence of a trial and at its last: the plan reports ARA_EDATA, and
    every other trial's YLT equals the single-layer path's bit for bit."""
    pf, yet, _, _ = case
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    counts = np.diff(yet.offsets)
    t = int(np.nonzero(counts >= 100)[0][0])
    b = int(yet.offsets[t])
    bad = ids.clone()
    for k, v in ((0, pf.catalogue), (32, -1), (64, 2**31 - 1), (int(counts[t]) - 1, pf.catalogue + 7)):
        bad[b + k] = v
    single = g.run_ylt(off, ids).clone()
    g.check()
    plan = ara.BatchedPlan(g, off, bad, autotune=False)
    y = plan.launch()
    with pytest.raises(ara.AraError) as e:
        g.check()
    assert e.value.status == ara.ARA_EDATA
    keep = torch.ones(yet.n_trials, dtype=torch.bool, device="cuda")
    keep[t] = False
    assert torch.equal(y[:, keep], single[:, keep])
    plan.close()
    g.close()


@pytest.mark.parametrize("requests", [
    # (layer_begin, layer_end, trial_begin, trial_end): trials [1500, 2400) are covered by the
    # first and the third request but not the middle one, whose entries those trials skip
    [(0, 7, 0, 2400), (7, 9, 1000, 1500), (9, 20, 1200, 3000)],
    # four requests: a middle pair uncovered together, single-request stretches, a one-trial
    # request and a request covering everything
    [(0, 3, 0, 900), (3, 5, 100, 101), (5, 12, 400, 700), (12, 20, 0, 3000)],
    # one request over every layer and trial: the plain batched pass
    [(0, 20, 0, 3000)],
])
def test_requests_in_one_pass_equal_each_request_alone(case, requests):
    """ara_run_ylt_requests: several requests' layers over different trial slices in one pass.
    Each request's YLT and regimes equal the single-layer path on its own layers and slice, bit
    for bit, and the oracle within the YLT tolerance."""
    pf, yet, ref, agg = case
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    ys, regs = g.run_ylt_requests(off, ids, requests, regimes=True)
    g.check()
    for (l0, l1, t0, t1), y, rg in zip(requests, ys, regs):
        sub_off = off[t0:t1 + 1]
        reg = torch.empty((l1 - l0, t1 - t0), dtype=torch.uint8, device="cuda")
        alone = g.run_ylt(sub_off, ids, layers=list(range(l0, l1)), regimes=reg)
        g.check()
        assert torch.equal(y, alone)
        assert torch.equal(rg, reg)
        err = np.abs(y.cpu().numpy() - ref[l0:l1, t0:t1])
        assert np.all(err <= 1e-6 * np.abs(ref[l0:l1, t0:t1]) + 1e-12 * np.abs(agg[l0:l1, t0:t1]))
    g.close()


def test_requests_in_one_pass_reject_bad_arguments(case):
    pf, yet, _, _ = case
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    bad = [[(0, 10, 0, 100)],                                   # layers not all covered
           [(0, 10, 0, 100), (10, 20, 50, 3001)],               # trials past the end
           [(0, 10, 5, 5), (10, 20, 0, 10)],                    # empty trial range
           [(0, 4, 0, 9), (4, 8, 0, 9), (8, 12, 0, 9), (12, 16, 0, 9), (16, 20, 0, 9)]]  # 5 requests
    for rq in bad:
        with pytest.raises(ara.AraError) as e:
            g.run_ylt_requests(off, ids, rq)
        assert e.value.status in (ara.ARA_EINVAL, ara.ARA_ERANGE)
    g.close()


def test_batched_workload_full_size_sampled():
    """The batched workload at its full size (64 layers of U{3..30} ELTs from a pool of 200,
    2,000,000-event catalogue, 2x10^5 trials of Poisson(U[200, 2000]) events) through the
    autotuned plan that bench.py times: 256 sampled trials of every layer against the oracle
    (which evaluates only those trials), and the selected layers' rows equal to single-layer
    runs bit for bit."""
    pf = synth.batched_portfolio(0)
    yet = synth.batched_yet(0, n_trials=200_000)
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    plan = ara.BatchedPlan(g, off, ids, autotune=True)
    y = plan.launch()
    g.check()
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(yet.n_trials, size=256, replace=False))
    ref, agg = oracle.ylt(pf, yet, trials=sample, return_agg=True)
    got = y[:, torch.from_numpy(sample).cuda()].cpu().numpy()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-6 * np.abs(ref) + 1e-12 * np.abs(agg))
    assert np.count_nonzero(ref) > 0.1 * ref.size
    for l in (0, 31, 63):
        single = g.run_ylt(off, ids, layers=[l])
        assert torch.equal(single[0], y[l])
    plan.close()
    g.close()


def test_merged_requests_on_the_serving_pool_sampled():
    """Four requests of the serving trace (their own layers of the 500-ELT pool, 2,000,000-event
    catalogue) merged in one pass over their slices (scaled from the trace's 10^6 trials to a
    2x10^5-trial Poisson(1000) YET): every request's YLT equals its run alone bit for bit, and
    128 sampled trials of each match the oracle."""
    pool_t = synth.serving_pool(0)
    n = 200_000
    yet = synth.serving_yet(0, n_trials=n)
    trace = synth.serving_trace(pool_t, 1_000_000, 8, 200.0, seed=0)[:4]
    for q in trace:   # the trace's slices of a 10^6-trial YET, scaled to this one
        q["trials"] = (q["trials"][0] * n // 1_000_000, max(q["trials"][1] * n // 1_000_000,
                                                             q["trials"][0] * n // 1_000_000 + 1))
    layers = [l for q in trace for l in q["layer_elts"]]
    terms = {k: np.asarray([x for q in trace for x in q[k]]) for k in ("occ_ret", "occ_lim", "agg_ret", "agg_lim")}
    tab = synth.Portfolio(pool_t.catalogue, pool_t.elt_ids, pool_t.elt_losses, pool_t.elt_ret,
                          pool_t.elt_lim, layers, terms["occ_ret"], terms["occ_lim"],
                          terms["agg_ret"], terms["agg_lim"], losses_f32=True)
    if sum(len(q["layer_elts"]) for q in trace) > 255:
        pytest.skip("more than 255 layers in the group")
    g = ara.Portfolio.from_tables(tab)
    off, ids = dev(yet)
    reqs, l0 = [], 0
    for q in trace:
        nl = len(q["layer_elts"])
        reqs.append((l0, l0 + nl, q["trials"][0], q["trials"][1]))
        l0 += nl
    ys = g.run_ylt_requests(off, ids, reqs)
    g.check()
    rng = np.random.default_rng(7)
    for (a, b, t0, t1), y in zip(reqs, ys):
        alone = g.run_ylt(off[t0:t1 + 1], ids, layers=list(range(a, b)))
        assert torch.equal(y, alone)
        sample = np.sort(rng.choice(np.arange(t0, t1), size=min(128, t1 - t0), replace=False))
        sub = tab.with_terms(tab.terms_dict())
        sub.layer_elts = tab.layer_elts[a:b]
        for name in ("occ_ret", "occ_lim", "agg_ret", "agg_lim"):
            setattr(sub, name, np.asarray(getattr(tab, name))[a:b])
        ref, agg = oracle.ylt(sub, yet, trials=sample, return_agg=True)
        got = y[:, torch.from_numpy(sample - t0).cuda()].cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref) + 1e-12 * np.abs(agg))
    g.close()
