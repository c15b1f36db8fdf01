"""GPU parity of the YLT path (C ABI through the binding) against the FP64 CPU oracle.

Tolerance (every YLT entry): |y_gpu - y_ref| <= 1e-6 |y_ref| + 1e-12 S_ref, where S_ref is
the oracle's aggregate loss before the aggregate terms.  The relative part is the required
1e-6; the absolute part covers the rounding of any reordered FP64 summation of a trial
(about n_t * 2^-53 * S_ref, below 1e-12 S_ref for the trial lengths used) and of the fixed
point the device sums in (a quantum of at most 2^-54 of the layer's bound on o(e)),
which dominate only where y_ref is tiny next to S_ref (the aggregate retention kink).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1606_04473_gb300 as ara

INF = float("inf")
FLAG_SETS = [0, 2, 4, 6, 8, 10, 12]  # bulk-staged folded; no filter; FP64 sums; both; LDG variants


def dev(yet):
    return (torch.from_numpy(np.ascontiguousarray(yet.offsets)).cuda(),
            torch.from_numpy(np.ascontiguousarray(yet.event_ids)).cuda())


def assert_ylt_close(got, ref, agg):
    got = np.asarray(got)
    err = np.abs(got - ref)
    tol = 1e-6 * np.abs(ref) + 1e-12 * np.abs(agg)
    bad = err > tol
    assert not bad.any(), (f"{bad.sum()} of {bad.size} entries out of tolerance; worst "
                           f"{np.max(err / np.maximum(tol, 1e-300)):.3g}x tol")


def mid_case(seed, catalogue=200_000, n_elts=12, nnz=4000, n_layers=4, n_trials=5003,
             lam=300.0, f32=True, max_le=None):
    """Mid-size portfolio spanning many tiles, ragged trial lengths (empty, 1..7 events,
    Poisson bulk), varied terms so that all clamp regimes occur."""
    rng = np.random.default_rng(seed)
    ids, losses = synth.make_elts(seed, n_elts, nnz, catalogue, 11.0, 2.0, f32=f32)
    r, l = synth.percentile_terms(losses)
    layers = []
    for k in range(n_layers):
        m = int(rng.integers(1, (max_le or n_elts) + 1))
        layers.append(sorted(rng.choice(n_elts, size=min(m, n_elts), replace=False).tolist()))
    counts = synth.poisson_counts(seed, lam, n_trials)
    counts[:8] = [0, 1, 2, 3, 4, 5, 6, 7]
    counts[-3:] = [0, 9, 1]
    yet = synth.make_yet(seed, counts, catalogue, with_timestamps=False)
    pf = synth.Portfolio(catalogue, ids, losses, r, l, layers, np.zeros(n_layers),
                         np.zeros(n_layers), np.zeros(n_layers), np.zeros(n_layers), losses_f32=f32)
    # layer terms from the oracle's own event/trial losses: retention at the 20th percentile,
    # limits low enough that a share of trials saturates
    from oracle.derive_terms import derive
    nh = min(1000, n_trials)
    head = synth.YET(yet.offsets[:nh + 1], yet.event_ids[:int(yet.offsets[nh])])
    t = derive(pf, head, 20.0, 70.0)
    return pf.with_terms(t), yet


@pytest.fixture(scope="module")
def tiny():
    pf, yet = synth.tiny(0)
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    return pf, yet, ref, agg


@pytest.fixture(scope="module")
def mid():
    pf, yet = mid_case(1)
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    return pf, yet, ref, agg


@pytest.mark.parametrize("flags", FLAG_SETS)
def test_tiny_workload_matches_oracle(tiny, flags):
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(*dev(yet), flags=flags)
    g.check()
    assert_ylt_close(y.cpu().numpy(), ref, agg)


@pytest.mark.parametrize("seed", range(5))
def test_tiny_workload_seeds_ylt_and_metrics(seed):
    """The tiny configuration (4 ELTs of 1,000 events over a 10,000-event catalogue, 1,000 trials
    of Poisson(100) events, the literal absolute layer terms) at seeds 0-4.  The YLT is within the
    stated tolerance of the oracle's; PML100, PML250 and TVaR99 are within 1e-6 of the oracle's
    metrics of its own YLT; the PML is the exact order statistic of the GPU's YLT, TVaR within
    1e-12 of the tail mean of that YLT, and the mean year loss within 1e-9 of the oracle's."""
    pf, yet = synth.tiny(seed)
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(*dev(yet))
    g.check()
    y_np = y.cpu().numpy()
    assert_ylt_close(y_np, ref, agg)
    p, t, mean = ara.risk_metrics(y, [100.0, 250.0], [0.99], want_mean=True)
    rp, rt = oracle.risk_metrics(ref, [100.0, 250.0], [0.99])
    np.testing.assert_allclose(p, rp, rtol=1e-6, atol=0)
    np.testing.assert_allclose(t, rt, rtol=1e-6, atol=0)
    gp, gt = oracle.risk_metrics(y_np, [100.0, 250.0], [0.99])
    assert np.array_equal(p, gp)
    np.testing.assert_allclose(t, gt, rtol=1e-12, atol=0)
    np.testing.assert_allclose(mean, ref.mean(axis=1), rtol=1e-9, atol=0)


def test_tiny_workload_per_elt_literal_path_equals_folded_bitwise(tiny):
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf, dense_tables=True)
    off, ids = dev(yet)
    a = g.run_ylt(off, ids, flags=ara.ARA_RUN_PER_ELT)
    b = g.run_ylt(off, ids)
    g.check()
    assert torch.equal(a, b)
    assert_ylt_close(a.cpu().numpy(), ref, agg)


@pytest.mark.parametrize("flags", FLAG_SETS)
def test_mid_size_multi_layer_ragged(mid, flags):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(*dev(yet), flags=flags)
    g.check()
    assert_ylt_close(y.cpu().numpy(), ref, agg)


def test_mid_size_regimes_all_present_and_recorded(mid):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    reg = torch.empty((pf.n_layers, yet.n_trials), dtype=torch.uint8, device="cuda")
    g.run_ylt(off, ids, regimes=reg)
    g.check()
    reg = reg.cpu().numpy()
    ex = agg - pf.agg_ret[:, None]
    want = np.where((ex > 0) & (ex < pf.agg_lim[:, None]), 1, np.where(ex > pf.agg_lim[:, None], 2, 0))
    near = np.abs(ex) <= 1e-9 * np.abs(agg) + 1e-6
    near |= np.abs(ex - pf.agg_lim[:, None]) <= 1e-9 * np.abs(agg) + 1e-6
    assert np.array_equal(reg[~near], want[~near])
    for r in (0, 1, 2):
        assert (want == r).any(), f"regime {r} absent from the test case"


def test_layer_subset_and_order(mid):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(*dev(yet), layers=[3, 0, 3])
    assert_ylt_close(y.cpu().numpy(), ref[[3, 0, 3]], agg[[3, 0, 3]])


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_unaligned_event_id_pointer(mid, shift):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    buf = torch.empty(ids.numel() + 4, dtype=torch.int32, device="cuda")
    view = buf[shift:shift + ids.numel()]
    view.copy_(ids)
    assert (view.data_ptr() // 4) % 4 == shift % 4
    y = g.run_ylt(off, view)
    g.check()
    assert_ylt_close(y.cpu().numpy(), ref, agg)


def test_large_catalogue_coarse_filter():
    """A 6M-event catalogue: the shared-memory hit bitmap must be coarsened (one bit per 2^k
    events); results stay exact."""
    pf, yet = mid_case(2, catalogue=6_000_000, n_elts=6, nnz=30_000, n_layers=2, n_trials=1500,
                       lam=500.0)
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    g = ara.Portfolio.from_tables(pf)
    for flags in (0, 2):
        y = g.run_ylt(*dev(yet), flags=flags)
        g.check()
        assert_ylt_close(y.cpu().numpy(), ref, agg)


def test_per_elt_path_many_elts_and_fp64_losses():
    """Layers wider than a warp (40 ELTs), a one-ELT layer and an empty layer; FP64 losses."""
    pf, yet = mid_case(3, catalogue=50_000, n_elts=40, nnz=800, n_layers=1, n_trials=700,
                       lam=200.0, f32=False)
    pf.layer_elts = [list(range(40)), [7], []]
    for name in ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]:
        setattr(pf, name, np.repeat(getattr(pf, name), 3))
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    g = ara.Portfolio.from_tables(pf, dense_tables=True)
    off, ids = dev(yet)
    a = g.run_ylt(off, ids, flags=ara.ARA_RUN_PER_ELT)
    b = g.run_ylt(off, ids)
    g.check()
    assert torch.equal(a, b)
    assert_ylt_close(a.cpu().numpy(), ref, agg)
    assert np.all(ref[2] == 0.0)


def test_fold_windows_dense_elts_and_empty_groups():
    """The fold stages a tile's records in windows of a few hundred: dense ELTs (70 % of a
    6,000-event catalogue, about 1,400 records per ELT and tile) straddle several windows each,
    and a second group of ELTs (a layer of 40 ELTs, searched 32 at a time) has records only in
    the first tile, so the other tiles meet groups without records.  The folded YLT equals the
    literal per-ELT path (Algorithm 3's lookups, the same ELT order) bit for bit, and the FP64
    oracle within tolerance; per-ELT, occurrence and aggregate retentions all bind."""
    catalogue = 6000
    dense_ids, dense_losses = synth.make_elts(21, 32, 4200, catalogue, 11.0, 2.0, f32=True)
    sparse_ids, sparse_losses = synth.make_elts(22, 8, 100, 500, 11.0, 2.0, f32=True)
    ids, losses = dense_ids + sparse_ids, dense_losses + sparse_losses
    r, l = synth.percentile_terms(losses)
    layers = [list(range(40)), [5], [33, 0, 39, 12], list(range(32, 40))]
    n = len(layers)
    counts = synth.poisson_counts(23, 200.0, 600)
    counts[:3] = [0, 1, 2]
    yet = synth.make_yet(23, counts, catalogue, with_timestamps=False)
    pf = synth.Portfolio(catalogue, ids, losses, r, l, layers, np.zeros(n), np.zeros(n),
                         np.zeros(n), np.zeros(n), losses_f32=True)
    from oracle.derive_terms import derive
    pf = pf.with_terms(derive(pf, yet, 20.0, 70.0))
    ref, agg = oracle.ylt(pf, yet, return_agg=True)
    g = ara.Portfolio.from_tables(pf, dense_tables=True)
    off, ev = dev(yet)
    a = g.run_ylt(off, ev, flags=ara.ARA_RUN_PER_ELT)
    b = g.run_ylt(off, ev)
    g.check()
    assert torch.equal(a, b)
    assert_ylt_close(b.cpu().numpy(), ref, agg)
    for k in range(n):   # the aggregate clamp is exercised in every layer
        assert np.any(ref[k] == 0.0) and np.any(ref[k] > 0.0)


def test_identity_terms_give_raw_loss_sums():
    pf, yet = mid_case(4, n_layers=2, n_trials=900)
    pf = pf.with_terms({**pf.terms_dict(), "elt_ret": [0.0] * pf.n_elts, "elt_lim": [INF] * pf.n_elts,
                        "occ_ret": [0.0, 0.0], "occ_lim": [INF, INF], "agg_ret": [0.0, 0.0],
                        "agg_lim": [INF, INF]})
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(*dev(yet)).cpu().numpy()
    trial = np.repeat(np.arange(yet.n_trials), np.diff(yet.offsets))
    for l, elts in enumerate(pf.layer_elts):
        dense = np.zeros(pf.catalogue)
        for j in elts:
            np.add.at(dense, pf.elt_ids[j], pf.elt_losses[j])
        expect = np.bincount(trial, weights=dense[yet.event_ids], minlength=yet.n_trials)
        np.testing.assert_allclose(y[l], expect, rtol=1e-12, atol=0)


def test_warp_reduction_of_large_partials_is_exact():
    """Table values near the fixed point's maximum (every lane partial has all three 27-bit
    limbs of the warp reduction in use) and trials of up to 3e5 events: the bulk stream's YLT
    equals, bit for bit, the register-staged kernel's, which adds every value with carries and
    reduces differently; both equal the correctly rounded sums of the losses."""
    import math
    catalogue = 4096
    ids = [np.arange(catalogue, dtype=np.int32)] * 2
    rng = np.random.default_rng(11)
    losses = [(1e6 * (0.9 + 0.1 * rng.random(catalogue))).astype(np.float32).astype(np.float64)
              for _ in range(2)]
    pf = synth.Portfolio(catalogue, ids, losses, np.zeros(2), np.full(2, INF), [[0, 1]],
                         np.zeros(1), np.full(1, INF), np.zeros(1), np.full(1, INF), losses_f32=True)
    counts = np.array([300_000, 0, 1, 250_000, 31, 32, 33, 4096, 123_457, 7], dtype=np.int64)
    yet = synth.make_yet(12, counts, catalogue, with_timestamps=False)
    g = ara.Portfolio.from_tables(pf)
    off, ev = dev(yet)
    y_bulk = g.run_ylt(off, ev)
    y_ldg = g.run_ylt(off, ev, flags=ara.ARA_RUN_LDG)
    g.check()
    assert torch.equal(y_bulk, y_ldg)
    dense = losses[0] + losses[1]
    expect = [math.fsum(dense[yet.event_ids[yet.offsets[t]:yet.offsets[t + 1]]].tolist())
              for t in range(yet.n_trials)]
    np.testing.assert_allclose(y_bulk.cpu().numpy()[0], expect, rtol=1e-14, atol=0)


def test_edge_cases_empty_inputs(tiny):
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf)
    off0 = torch.zeros(1, dtype=torch.int64, device="cuda")
    ids0 = torch.zeros(0, dtype=torch.int32, device="cuda")
    y = g.run_ylt(off0, ids0)
    assert y.shape == (1, 0)
    offz = torch.zeros(65, dtype=torch.int64, device="cuda")     # 64 empty trials
    y = g.run_ylt(offz, ids0)
    g.check()
    assert torch.all(y == 0)


def test_device_side_data_errors_are_reported_and_recoverable(tiny):
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    bad = ids.clone()
    bad[17] = pf.catalogue          # event ID outside the catalogue
    g.run_ylt(off, bad)
    with pytest.raises(ara.AraError) as e:
        g.check()
    assert e.value.status == ara.ARA_EDATA
    boff = off.clone()
    boff[5] = boff[6] + 1           # decreasing offsets
    g.run_ylt(boff, ids)
    with pytest.raises(ara.AraError):
        g.check()
    y = g.run_ylt(off, ids)          # a good run afterwards is unaffected
    g.check()
    assert_ylt_close(y.cpu().numpy(), ref, agg)


def test_warp_range_at_the_stream_limit_is_a_data_error(tiny):
    """One trial of 2^31 - 256 events: the default stream kernel gives each warp a contiguous
    trial range and accepts ranges below 2^31 - 512 events only.  Its range check runs before any
    event ID is read (the 8 GB ID buffer is left uninitialised), the run reports ARA_EDATA, and
    the next run is unaffected."""
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf)
    n = (1 << 31) - 256
    big = torch.empty(n, dtype=torch.int32, device="cuda")
    off1 = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    g.run_ylt(off1, big)
    with pytest.raises(ara.AraError) as e:
        g.check()
    assert e.value.status == ara.ARA_EDATA
    del big
    torch.cuda.empty_cache()
    off, ids = dev(yet)
    y = g.run_ylt(off, ids)
    g.check()
    assert_ylt_close(y.cpu().numpy(), ref, agg)


def test_repeatable_bitwise(mid):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    a = g.run_ylt(off, ids).clone()
    b = g.run_ylt(off, ids)
    assert torch.equal(a, b)


def test_host_pipeline_equals_device_path(mid):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    y_dev = g.run_ylt(*dev(yet))
    y_host = g.run_ylt_host(yet.offsets, yet.event_ids)
    assert np.array_equal(y_dev.cpu().numpy(), y_host)
    y2, p, t = g.run_ylt_host(yet.offsets, yet.event_ids, layers=[2, 1], return_periods=[100.0, 250.0],
                              tvar_levels=[0.99])
    assert np.array_equal(y2, y_host[[2, 1]])
    p_dev, t_dev = ara.risk_metrics(y_dev[[2, 1]].contiguous(), [100.0, 250.0], [0.99])
    assert np.array_equal(p, p_dev) and np.array_equal(t, t_dev)
    _, p3, t3 = g.run_ylt_host(yet.offsets, yet.event_ids, return_periods=[10.0], tvar_levels=[0.5],
                               want_ylt=False)
    rp, rt = oracle.risk_metrics(ref, [10.0], [0.5])
    np.testing.assert_allclose(p3, rp, rtol=1e-6)
    np.testing.assert_allclose(t3, rt, rtol=1e-6)


def test_host_pipeline_multi_chunk():
    """More than one 16M-event chunk through the host pipeline, pinned host memory."""
    pf = synth.paper_scale_portfolio(0)
    n = 40_000
    ids = torch.empty(n * 1000, dtype=torch.int32).pin_memory()
    yet = synth.paper_scale_yet(0, n_trials=n, ids_out=ids.numpy())
    g = ara.Portfolio.from_tables(pf)
    y_host = g.run_ylt_host(yet.offsets, ids.numpy())
    y_dev = g.run_ylt(torch.from_numpy(yet.offsets).cuda(), ids.cuda()).cpu().numpy()
    assert np.array_equal(y_host, y_dev)
    sample = np.arange(0, n, 97)
    ref, agg = oracle.ylt(pf, yet, trials=sample, return_agg=True)
    assert_ylt_close(y_host[:, sample], ref, agg)


def test_host_pipeline_rejects_decreasing_offsets(tiny):
    """Host offsets are validated before anything is queued: a decreasing pair anywhere (here
    the last) is ARA_EINVAL in both host modes, and the portfolio stays usable."""
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf)
    bad = np.array(yet.offsets, dtype=np.int64)
    bad[-2] = bad[-1] + 1
    for flags in (0, ara.ARA_RUN_HOST_DIRECT):
        with pytest.raises(ara.AraError) as e:
            g.run_ylt_host(bad, yet.event_ids, flags=flags)
        assert e.value.status == ara.ARA_EINVAL
    y = g.run_ylt_host(yet.offsets, yet.event_ids)
    assert_ylt_close(y, ref, agg)


def test_host_direct_reads_pinned_host_memory(mid):
    """ARA_RUN_HOST_DIRECT: the kernel reads the pinned host YET in place; same YLT as the
    device path.  Pageable memory is read in place too on platforms where the device can
    address it (coherent CPU-GPU systems); elsewhere it is refused with ARA_EINVAL."""
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    ids_p = torch.from_numpy(yet.event_ids).pin_memory()
    off_p = torch.from_numpy(yet.offsets).pin_memory()
    y_dev = g.run_ylt(off_p.cuda(), ids_p.cuda()).cpu().numpy()
    y_dir = g.run_ylt_host(off_p.numpy(), ids_p.numpy(), flags=ara.ARA_RUN_HOST_DIRECT)
    assert np.array_equal(y_dev, y_dir)
    try:
        y_pg = g.run_ylt_host(np.array(yet.offsets), np.array(yet.event_ids),
                              flags=ara.ARA_RUN_HOST_DIRECT)
        assert np.array_equal(y_pg, y_dev)
    except ara.AraError as e:
        assert e.status == ara.ARA_EINVAL


def test_paper_scale_full_size_sampled():
    """The paper-scale workload (1 layer of 15 ELTs, 2M-event catalogue, 10^6 trials x 1000
    events) in the benchmark's launch configuration; 4000 sampled trials against the oracle,
    range and determinism properties on all entries."""
    pf = synth.paper_scale_portfolio(0)
    n = 1_000_000
    ids_h = torch.empty(n * 1000, dtype=torch.int32).pin_memory()
    yet = synth.paper_scale_yet(0, n_trials=n, ids_out=ids_h.numpy())
    g = ara.Portfolio.from_tables(pf)
    off = torch.from_numpy(yet.offsets).cuda()
    ids = ids_h.cuda()
    y = g.run_ylt(off, ids)
    y2 = g.run_ylt(off, ids)
    g.check()
    assert torch.equal(y, y2)
    yc = y.cpu().numpy()
    assert np.all(yc >= 0) and np.all(yc <= pf.agg_lim[0])
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([rng.integers(0, n, 3990), [0, 1, n - 2, n - 1]]))
    ref, agg = oracle.ylt(pf, yet, trials=sample, return_agg=True)
    assert_ylt_close(yc[:, sample], ref, agg)
    del ids


def test_every_stream_shape_gives_identical_ylt(mid):
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    shapes = ara.stream_shapes()
    assert len(shapes) >= 2
    try:
        outs = []
        for i in range(len(shapes)):
            ara.set_stream_shape(i)
            outs.append(g.run_ylt(off, ids).clone())
            g.check()
    finally:
        ara.set_stream_shape(0)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    assert_ylt_close(outs[0].cpu().numpy(), ref, agg)


def test_bounded_copy_wait_times_out_and_reports(tiny):
    """Every wait for a bulk copy is bounded: with copies that announce more bytes than they
    deliver, each wait runs out after the (shortened) limit, the kernel returns, and the host
    reads ARA_ETIMEOUT; the context stays usable."""
    pf, yet, ref, agg = tiny
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    try:
        ara.debug_set(ara.ARA_DBG_WAIT_LIMIT_NS, 2_000_000)
        ara.debug_set(ara.ARA_DBG_STARVE_COPIES, 16)
        g.run_ylt(off, ids)
        with pytest.raises(ara.AraError) as e:
            g.check()
        assert e.value.status == ara.ARA_ETIMEOUT
    finally:
        ara.debug_set(ara.ARA_DBG_STARVE_COPIES, 0)
        ara.debug_set(ara.ARA_DBG_WAIT_LIMIT_NS, 1_000_000_000)
    y = g.run_ylt(off, ids)
    g.check()
    assert_ylt_close(y.cpu().numpy(), ref, agg)


def test_occurrence_basis_oep(mid):
    """ARA_RUN_OEP: the largest occurrence loss per trial, against the oracle's OEP basis."""
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(*dev(yet), flags=ara.ARA_RUN_OEP)
    g.check()
    want = oracle.ylt_oep(pf, yet)
    got = y.cpu().numpy()
    # one occurrence loss, rounded once to the layer's fixed point: q = rint(o 2^f) with
    # 2^(55-f) the first power of two above the layer's bound B on o(e), so |err| <= 2^-55 B
    # (the bound below restates B from the per-ELT maxima through the monotone clamps)
    clamp = lambda x, r, l: min(max(x - r, 0.0), l)
    for l, elts in enumerate(pf.layer_elts):
        s = sum(clamp(float(np.max(pf.elt_losses[j])), pf.elt_ret[j], pf.elt_lim[j]) for j in elts)
        bound = clamp(s, pf.occ_ret[l], pf.occ_lim[l]) * (1 + 1e-9)
        err = np.abs(got[l] - want[l])
        assert np.all(err <= 2.0 ** -55 * bound), (l, err.max(), bound)
        assert np.all(err <= 1e-6 * np.abs(want[l]))
    with pytest.raises(ara.AraError):
        g.run_ylt(*dev(yet), flags=ara.ARA_RUN_OEP | ara.ARA_RUN_LDG)


def test_fp32_storage_widens_exactly():
    """FP32 loss storage gives the same YLT, bit for bit, as FP64 storage of the same values:
    the fold widens binary32 losses to binary64 exactly, for zeros of both signs, subnormals
    with every leading-bit position, normals across the whole exponent range and the largest
    finite float.  Terms are open (zero retentions, infinite limits) so that every loss reaches
    the sums, and each layer's fixed point resolves its own smallest losses."""
    rng = np.random.default_rng(41)
    C = 4096
    sub = np.array([0x00000000, 0x80000000, 0x00000001, 0x00000003, 0x007fffff, 0x00400000,
                    0x00000400, 0x00800000, 0x00c00000], dtype=np.uint32)
    lead = rng.integers(0, 23, 400).astype(np.uint32)                       # subnormals
    frac = (np.uint32(1) << lead) | (rng.integers(0, 1 << 23, 400).astype(np.uint32) &
                                      ((np.uint32(1) << lead) - np.uint32(1)))
    small = (rng.integers(1, 11, 200).astype(np.uint32) << 23) | rng.integers(0, 1 << 23, 200).astype(np.uint32)
    sub = np.concatenate([sub, frac, small])
    wide = np.concatenate([np.array([0x7f7fffff, 0x3f800000, 0x00800000], dtype=np.uint32),
                           (rng.integers(1, 255, 700).astype(np.uint32) << 23) |
                           rng.integers(0, 1 << 23, 700).astype(np.uint32)])
    ordinary = rng.lognormal(11.0, 2.0, 500).astype(np.float32)
    tabs = [sub.view(np.float32), wide.view(np.float32), ordinary]
    ids = [np.sort(rng.choice(C, size=t.size, replace=False)).astype(np.int32) for t in tabs]
    losses = [t.astype(np.float64)[np.argsort(rng.random(t.size))] for t in tabs]
    layers = [[0], [1], [2, 0], [0, 1, 2]]
    z, inf = np.zeros(len(layers)), np.full(len(layers), INF)
    counts = synth.poisson_counts(41, 60.0, 3001)
    yet = synth.make_yet(41, counts, C, with_timestamps=False)
    off, ev = dev(yet)
    out = []
    for f32 in (True, False):
        pf = synth.Portfolio(C, ids, losses, np.zeros(3), np.full(3, INF), layers, z, inf, z, inf,
                             losses_f32=f32)
        g = ara.Portfolio.from_tables(pf)
        out.append(g.run_ylt(off, ev))
        torch.cuda.synchronize()
        g.check()
        g.close()
    assert torch.equal(out[0], out[1])
    assert (out[0][0] > 0).any() and (out[0][1] > 0).any()


@pytest.mark.parametrize("flags", [0, 2, 4, 8, 64])
def test_prepared_fold_slots_equal_unprepared_runs(mid, flags):
    """ara_prepare_ylt queues the fold (and coarse bitmap) into slot 0 or 1; runs with
    ARA_RUN_PREPARED (| ARA_RUN_SLOT1) stream against it and equal an ordinary run bit for bit,
    for both slots, a layer subset, and with the two slots holding different layer sets."""
    pf, yet, ref, agg = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    want = g.run_ylt(off, ids, flags=flags).clone()
    g.prepare_ylt(slot=0, flags=flags)
    a = g.run_ylt(off, ids, flags=flags | ara.ARA_RUN_PREPARED).clone()
    g.prepare_ylt(layers=[3, 1], slot=1, flags=flags)
    b = g.run_ylt(off, ids, layers=[3, 1], flags=flags | ara.ARA_RUN_PREPARED | ara.ARA_RUN_SLOT1)
    c = g.run_ylt(off, ids, flags=flags | ara.ARA_RUN_PREPARED)       # slot 0 still holds all
    g.check()
    assert torch.equal(a, want) and torch.equal(c, want)
    assert torch.equal(b[0], want[3]) and torch.equal(b[1], want[1])
    if flags != 64:
        assert_ylt_close(a.cpu().numpy(), ref, agg)
    g.close()


def test_prepared_fold_pipelined_over_two_streams_at_paper_scale_catalogue():
    """The paper-scale portfolio (2,000,000-event catalogue: the stream kernel reads the coarse
    bitmap, built by the prepare) on 3,000 trials x 1,000 events: folds queued on a second
    stream into alternating slots while the first stream runs the YET against the other slot,
    as bench.py schedules its steps; every run equals an ordinary run bit for bit."""
    pf = synth.paper_scale_portfolio(0)
    yet = synth.paper_scale_yet(0, n_trials=3000)
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    want = g.run_ylt(off, ids).clone()
    A = torch.cuda.current_stream()
    C = torch.cuda.Stream()
    outs = [torch.empty_like(want) for _ in range(6)]
    ev_fold = [torch.cuda.Event() for _ in range(6)]
    ev_run = [torch.cuda.Event() for _ in range(6)]
    for k in range(6):
        s = k % 2
        if k >= 2:
            C.wait_event(ev_run[k - 2])          # the run two steps back read this slot
        g.prepare_ylt(slot=s, stream=C)
        ev_fold[k].record(C)
        A.wait_event(ev_fold[k])
        g.run_ylt(off, ids, out=outs[k], flags=ara.ARA_RUN_PREPARED | (ara.ARA_RUN_SLOT1 if s else 0))
        ev_run[k].record(A)
    torch.cuda.synchronize()
    g.check()
    for o in outs:
        assert torch.equal(o, want)
    sample = np.arange(0, 3000, 97)
    ref, agg = oracle.ylt(pf, yet, trials=sample, return_agg=True)
    assert_ylt_close(want[:, torch.from_numpy(sample).cuda()].cpu().numpy(), ref, agg)
    g.close()


def test_prepared_fold_flag_rules(mid):
    pf, yet, _, _ = mid
    g = ara.Portfolio.from_tables(pf)
    off, ids = dev(yet)
    P, S1 = ara.ARA_RUN_PREPARED, ara.ARA_RUN_SLOT1
    for flags in (S1, P | ara.ARA_RUN_BATCHED):
        with pytest.raises(ara.AraError) as e:
            g.run_ylt(off, ids, flags=flags)
        assert e.value.status == ara.ARA_EINVAL
    with pytest.raises(ara.AraError):           # slot 1 never prepared on this portfolio
        g.run_ylt(off, ids, flags=P | S1)
    for bad in ((2, 0), (0, ara.ARA_RUN_BATCHED), (0, P)):
        with pytest.raises(ara.AraError):
            g.prepare_ylt(slot=bad[0], flags=bad[1])
    with pytest.raises(ara.AraError):
        g.run_ylt_host(yet.offsets, yet.event_ids, flags=P)
    g.close()
