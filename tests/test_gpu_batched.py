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
