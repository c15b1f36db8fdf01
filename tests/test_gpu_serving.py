"""GPU tests of serving: layer sets over a resident ELT pool and the native request server
(continuous admission by a device-memory budget, requests overlapping on separate streams).
Each request's results must be the same alone and in the mix (the per-request computation is
deterministic: exact integer trial sums and an exact selection), and agree with the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1606_04473_gb300 as ara

C, POOL = 200_000, 40


@pytest.fixture(scope="module")
def world():
    ids, losses = synth.make_elts(5, POOL, 3000, C, 11.0, 2.0, f32=True)
    r, l = synth.percentile_terms(losses)
    pool_tables = synth.Portfolio(C, ids, losses, r, l, [], np.zeros(0), np.zeros(0), np.zeros(0),
                                  np.zeros(0), losses_f32=True)
    counts = synth.poisson_counts(5, 300.0, 6000)
    yet = synth.make_yet(5, counts, C, with_timestamps=False)
    pool = ara.Portfolio.from_tables(pool_tables)
    off = torch.from_numpy(yet.offsets).cuda()
    ev = torch.from_numpy(yet.event_ids).cuda()
    return pool_tables, yet, pool, off, ev


def random_queries(n, seed, n_trials):
    rng = np.random.default_rng(seed)
    qs = []
    for k in range(n):
        nl = int(rng.integers(1, 7))
        layers = [sorted(rng.choice(POOL, size=int(rng.integers(3, 11)), replace=False).tolist())
                  for _ in range(nl)]
        t0 = int(rng.integers(0, n_trials - 500))
        t1 = int(rng.integers(t0 + 200, min(n_trials, t0 + 4000) + 1))
        scale = rng.uniform(0.5, 2.0, (4, nl))
        qs.append(dict(layer_elts=layers, occ_ret=2e4 * scale[0], occ_lim=2e6 * scale[1],
                       agg_ret=5e6 * scale[2], agg_lim=2e8 * scale[3], trials=(t0, t1),
                       return_periods=[10.0, 50.0], tvar_levels=[0.9], want_mean=True,
                       want_adjoint=bool(k % 3 == 0), adjoint_level=0.9,
                       flags=ara.ARA_RUN_BATCHED if k % 2 else 0, tenant=k % 5))
    return qs


def test_layer_set_equals_full_portfolio(world):
    pool_tables, yet, pool, off, ev = world
    layers = [[0, 3, 5, 7], [1, 2], [39, 10, 20]]
    terms = dict(occ_ret=[1e4, 2e4, 3e4], occ_lim=[1e6, 3e6, 5e6], agg_ret=[1e6, 2e6, 3e6],
                 agg_lim=[1e8, 1e8, 1e7])
    ls = pool.layer_set(layers, **terms)
    full_tables = synth.Portfolio(C, pool_tables.elt_ids, pool_tables.elt_losses, pool_tables.elt_ret,
                                  pool_tables.elt_lim, layers, *[np.array(terms[k]) for k in
                                  ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]], losses_f32=True)
    full = ara.Portfolio.from_tables(full_tables)
    a = ls.run_ylt(off, ev)
    b = full.run_ylt(off, ev)
    ls.check()
    assert torch.equal(a, b)
    ref, agg = oracle.ylt(full_tables, yet, return_agg=True)
    err = np.abs(a.cpu().numpy() - ref)
    assert np.all(err <= 1e-6 * np.abs(ref) + 1e-12 * np.abs(agg))
    ls.close()


def test_server_results_same_alone_and_in_the_mix(world):
    pool_tables, yet, pool, off, ev = world
    qs = random_queries(24, 7, yet.n_trials)
    srv = ara.Server(pool, off, ev, max_concurrent=4)
    tickets = [srv.submit(**q) for q in qs]          # all at once: they overlap on the device
    mixed = [srv.wait(t) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert stats["peak_running"] >= 2
    alone_srv = ara.Server(pool, off, ev, max_concurrent=1)
    for q, m in zip(qs, mixed):
        a = alone_srv.wait(alone_srv.submit(**q))
        for k in ("pml", "tvar", "mean", "grad_layer"):
            if a[k] is None:
                assert m[k] is None
            else:
                assert np.array_equal(a[k], m[k]), k
    alone_srv.close()
    # a few against the oracle
    for q, m in list(zip(qs, mixed))[:4]:
        t0, t1 = q["trials"]
        sub = synth.YET(yet.offsets[t0:t1 + 1] - yet.offsets[t0],
                        yet.event_ids[yet.offsets[t0]:yet.offsets[t1]])
        tab = synth.Portfolio(C, pool_tables.elt_ids, pool_tables.elt_losses, pool_tables.elt_ret,
                              pool_tables.elt_lim, q["layer_elts"], np.asarray(q["occ_ret"]),
                              np.asarray(q["occ_lim"]), np.asarray(q["agg_ret"]),
                              np.asarray(q["agg_lim"]))
        y = oracle.ylt(tab, sub)
        p, t = oracle.risk_metrics(y, q["return_periods"], q["tvar_levels"])
        np.testing.assert_allclose(m["pml"], p, rtol=1e-6)
        np.testing.assert_allclose(m["tvar"], t, rtol=1e-6)
        np.testing.assert_allclose(m["mean"], y.mean(1), rtol=1e-6)


def test_server_admission_by_memory_budget(world):
    pool_tables, yet, pool, off, ev = world
    qs = random_queries(8, 11, yet.n_trials)
    srv = ara.Server(pool, off, ev, max_concurrent=4, memory_budget=1)   # every request alone
    res = [srv.wait(t) for t in [srv.submit(**q) for q in qs]]
    assert srv.stats()["peak_running"] == 1
    srv.close()
    srv = ara.Server(pool, off, ev, max_concurrent=4, memory_budget=1 << 40)
    res2 = [srv.wait(t) for t in [srv.submit(**q) for q in qs]]
    srv.close()
    for a, b in zip(res, res2):
        assert np.array_equal(a["pml"], b["pml"]) and np.array_equal(a["tvar"], b["tvar"])


def test_server_rejects_invalid_queries(world):
    pool_tables, yet, pool, off, ev = world
    srv = ara.Server(pool, off, ev, max_concurrent=2)
    good = random_queries(1, 3, yet.n_trials)[0]
    bad = [dict(good, trials=(0, yet.n_trials + 1)), dict(good, layer_elts=[[POOL]]),
           dict(good, return_periods=[0.5]), dict(good, tvar_levels=[1.0])]
    for q in bad:
        with pytest.raises(ara.AraError) as e:
            srv.submit(**q)
        assert e.value.status == ara.ARA_EINVAL
    srv.wait(srv.submit(**good))
    srv.close()


def test_server_merges_overlapping_requests_with_identical_results(world):
    """Queued requests whose slices overlap run merged, several per pass over the union of their
    slices; every result (PML, TVaR, mean, layer-term gradients) equals the same request served
    with merging off, bit for bit, and the oracle within the YLT tolerance."""
    pool_tables, yet, pool, off, ev = world
    rng = np.random.default_rng(17)
    qs = random_queries(16, 13, yet.n_trials)
    for q in qs:                                      # heavily overlapping slices
        t0 = int(rng.integers(0, 1500))
        q["trials"] = (t0, int(rng.integers(4000, yet.n_trials + 1)))
    srv = ara.Server(pool, off, ev, max_concurrent=1, max_merge=4, min_overlap=0.1)
    merged = [srv.wait(t) for t in [srv.submit(**q) for q in qs]]
    cnt = srv.counters()
    srv.close()
    assert cnt["merged_requests"] >= 2 and cnt["passes"] < len(qs)
    alone_srv = ara.Server(pool, off, ev, max_concurrent=1, max_merge=1)
    for q, m in zip(qs, merged):
        a = alone_srv.wait(alone_srv.submit(**q))
        for k in ("pml", "tvar", "mean", "grad_layer"):
            if a[k] is None:
                assert m[k] is None
            else:
                assert np.array_equal(a[k], m[k]), k
    assert alone_srv.counters()["merged_requests"] == 0
    alone_srv.close()
    for q, m in list(zip(qs, merged))[:3]:
        t0, t1 = q["trials"]
        sub = synth.YET(yet.offsets[t0:t1 + 1] - yet.offsets[t0],
                        yet.event_ids[yet.offsets[t0]:yet.offsets[t1]])
        tab = synth.Portfolio(C, pool_tables.elt_ids, pool_tables.elt_losses, pool_tables.elt_ret,
                              pool_tables.elt_lim, q["layer_elts"], np.asarray(q["occ_ret"]),
                              np.asarray(q["occ_lim"]), np.asarray(q["agg_ret"]),
                              np.asarray(q["agg_lim"]))
        y = oracle.ylt(tab, sub)
        p, t = oracle.risk_metrics(y, q["return_periods"], q["tvar_levels"])
        np.testing.assert_allclose(m["pml"], p, rtol=1e-6)
        np.testing.assert_allclose(m["tvar"], t, rtol=1e-6)
        np.testing.assert_allclose(m["mean"], y.mean(1), rtol=1e-6)


def test_server_merging_arguments(world):
    pool_tables, yet, pool, off, ev = world
    srv = ara.Server(pool, off, ev, max_concurrent=1)
    for bad in [(0, 0.3), (5, 0.3), (2, 0.0), (2, 1.5)]:
        with pytest.raises(ara.AraError):
            srv.set_merging(*bad)
    srv.set_merging(1)
    srv.close()


def test_blocked_request_is_passed_by_smaller_ones_a_bounded_number_of_times(world):
    """Admission: while a long request runs, a queued request too large for the rest of the
    budget is passed by smaller queued requests that fit (at most 4 times), and still runs
    afterwards; every result equals the same request served alone."""
    pool_tables, yet, pool, off, ev = world
    rng = np.random.default_rng(29)
    big_layers = [sorted(rng.choice(POOL, size=10, replace=False).tolist()) for _ in range(24)]
    base = random_queries(1, 31, yet.n_trials)[0]
    long_q = dict(base, layer_elts=big_layers[:6], occ_ret=[2e4] * 6, occ_lim=[2e6] * 6,
                  agg_ret=[5e6] * 6, agg_lim=[2e8] * 6, trials=(0, yet.n_trials), want_adjoint=True)
    head_q = dict(base, layer_elts=big_layers, occ_ret=[2e4] * 24, occ_lim=[2e6] * 24,
                  agg_ret=[5e6] * 24, agg_lim=[2e8] * 24, trials=(0, yet.n_trials), want_adjoint=False)
    small = [dict(base, layer_elts=[big_layers[k][:3]], occ_ret=[2e4], occ_lim=[2e6], agg_ret=[5e6],
                  agg_lim=[2e8], trials=(100 * k, 100 * k + 300), want_adjoint=False)
             for k in range(6)]
    probe = ara.Server(pool, off, ev, max_concurrent=1)
    est = {name: probe.estimate_bytes(**q) for name, q in
           (("long", long_q), ("head", head_q), ("small", small[0]))}
    probe.close()
    assert est["head"] > 2 * est["small"]
    budget = est["long"] + est["small"] + 4096     # the head does not fit beside the long one
    srv = ara.Server(pool, off, ev, max_concurrent=2, memory_budget=budget, max_merge=1)
    tickets = [srv.submit(**long_q), srv.submit(**head_q)] + [srv.submit(**q) for q in small]
    res = [srv.wait(t) for t in tickets]
    cnt = srv.counters()
    srv.close()
    assert 1 <= cnt["head_passed"] <= 4
    alone = ara.Server(pool, off, ev, max_concurrent=1, max_merge=1)
    for q, m in zip([long_q, head_q] + small, res):
        a = alone.wait(alone.submit(**q))
        for k in ("pml", "tvar", "mean", "grad_layer"):
            assert (a[k] is None and m[k] is None) or np.array_equal(a[k], m[k]), k
    alone.close()


def test_server_adjoints_over_the_yet_index_are_identical(world):
    """With the server's index of its resident YET, adjoint requests whose slice covers at least
    half of the index blocks it touches read the index; every result equals the same request on
    a server without the index, bit for bit.  The index can change only while the server is
    idle."""
    pool_tables, yet, pool, off, ev = world
    rng = np.random.default_rng(23)
    qs = random_queries(12, 29, yet.n_trials)
    for k, q in enumerate(qs):
        q["want_adjoint"] = True
        if k % 3:                                     # long slices read the index
            t0 = int(rng.integers(0, 1000))
            q["trials"] = (t0, int(rng.integers(4000, yet.n_trials + 1)))
    plain = ara.Server(pool, off, ev, max_concurrent=1, max_merge=4)
    want = [plain.wait(t) for t in [plain.submit(**q) for q in qs]]
    assert plain.counters()["indexed_adjoints"] == 0
    plain.close()
    srv = ara.Server(pool, off, ev, max_concurrent=1, max_merge=4)
    srv.set_adjoint_index(True)
    got = [srv.wait(t) for t in [srv.submit(**q) for q in qs]]
    cnt = srv.counters()
    assert 0 < cnt["indexed_adjoints"] < len(qs)
    for a, b in zip(want, got):
        for k in ("pml", "tvar", "mean", "grad_layer"):
            assert np.array_equal(a[k], b[k]), k
    tickets = [srv.submit(**q) for q in qs]
    with pytest.raises(ara.AraError) as ei:          # requests queued: refused
        srv.set_adjoint_index(False)
    assert ei.value.status == ara.ARA_EBUSY
    for t in tickets:
        srv.wait(t)
    srv.close()
