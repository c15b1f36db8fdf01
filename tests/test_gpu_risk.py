"""GPU parity of PML / TVaR selection (ara_risk_metrics) against the oracle's order
statistics.  Inputs are YLTs from the generator or the oracle, never from the CUDA path,
except in the end-to-end test, which compares GPU(YLT_gpu) with oracle(YLT_oracle)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1606_04473_gb300 as ara

RPS = [1.0, 2.0, 10.0, 100.0, 250.0]
LEVELS = [0.0, 0.5, 0.9, 0.99]


def check(ylt, rps=RPS, levels=LEVELS):
    ylt = np.atleast_2d(ylt)
    n = ylt.shape[1]
    rps = [r for r in rps if np.ceil(n / r) >= 1]
    p, t = ara.risk_metrics(torch.from_numpy(ylt).cuda(), rps, levels)
    rp, rt = oracle.risk_metrics(ylt, rps, levels)
    assert np.array_equal(p, rp)                       # PML is a copy of a YLT entry
    np.testing.assert_allclose(t, rt, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [1, 2, 10, 1000, 4097, 100_003])
def test_lognormal_ylt(n):
    rng = np.random.default_rng(n)
    check(rng.lognormal(14, 2, n))


def test_many_ties_and_zeros():
    rng = np.random.default_rng(1)
    y = np.round(rng.lognormal(5, 1, 20_000), 0)
    y[:12_000] = 0.0
    y[12_000:12_500] = 5e6
    check(y)


def test_signed_and_special_values():
    rng = np.random.default_rng(2)
    y = rng.normal(0, 1e3, 5000)
    y[:10] = [0.0, -0.0, 1e-310, -1e-310, 1e300, -1e300, 5e-324, 3.0, 3.0, 3.0]
    check(y, levels=[0.5, 0.99, 0.999])   # tails contain +1e300 but not -1e300


def test_multiple_layers_independent():
    rng = np.random.default_rng(3)
    y = np.stack([rng.lognormal(10, s, 30_000) for s in (0.5, 1.0, 2.0, 3.0)])
    check(y)


def test_hand_computed_example(golden_dir):
    import json, os
    g = json.load(open(os.path.join(golden_dir, "p8_order_statistics.json")))
    y = np.array(g["ylt"])
    rps = [float(k) for k in g["pml"]]
    lv = [float(k) for k in g["tvar"]]
    p, t = ara.risk_metrics(torch.from_numpy(y).cuda(), rps, lv)
    assert p[0].tolist() == [g["pml"][k] for k in g["pml"]]
    np.testing.assert_allclose(t[0], [g["tvar"][k] for k in g["tvar"]], rtol=1e-15)


def test_end_to_end_tiny_workload():
    pf, yet = synth.tiny(0)
    g = ara.Portfolio.from_tables(pf)
    y = g.run_ylt(torch.from_numpy(yet.offsets).cuda(), torch.from_numpy(yet.event_ids).cuda())
    p, t = ara.risk_metrics(y, [100.0, 250.0], [0.99])
    ref = oracle.ylt(pf, yet)
    rp, rt = oracle.risk_metrics(ref, [100.0, 250.0], [0.99])
    np.testing.assert_allclose(p, rp, rtol=1e-6)
    np.testing.assert_allclose(t, rt, rtol=1e-6)


def test_many_layers_several_launches_and_slices_beyond_shared_memory():
    """200 layers: one block per layer, so the layers are split over more than one cooperative
    launch, and each block's slice (30k values) is larger than the shared-memory cache, so the
    passes read the row from global memory."""
    rng = np.random.default_rng(5)
    y = rng.lognormal(12, 1.5, (200, 30_000))
    y[:, :5_000] = 0.0
    y[7, 100:400] = 3e9                                  # ties at the top of one row
    check(y, rps=[10.0, 100.0, 250.0], levels=[0.99, 0.5])


def test_async_metrics_equal_synchronous_bitwise():
    rng = np.random.default_rng(6)
    y = torch.from_numpy(rng.lognormal(13, 2, (3, 50_001))).cuda()
    rps, lv = [100.0, 250.0], [0.99, 0.9]
    p, t, m = ara.risk_metrics(y, rps, lv, want_mean=True)
    pd = torch.full((3, 2), -1.0, dtype=torch.float64, device="cuda")
    td = torch.full((3, 2), -1.0, dtype=torch.float64, device="cuda")
    md = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    sd = torch.full((1,), 123, dtype=torch.int32, device="cuda")
    ara.risk_metrics_async(y, rps, lv, pd, td, sd, mean=md)
    torch.cuda.synchronize()
    assert int(sd.item()) == 0
    assert np.array_equal(pd.cpu().numpy(), p) and np.array_equal(td.cpu().numpy(), t)
    assert np.array_equal(md.cpu().numpy(), m)
    with pytest.raises(ValueError):
        ara.risk_metrics_async(y, rps, lv, pd[:2], td, sd)


def test_grid_barrier_timeout_is_reported():
    """The selection's blocks skip their barrier arrivals (test hook): every bounded wait runs
    out, the call reports ARA_ETIMEOUT (sync) or sets the device status (async), and the next
    call is correct again.  No fault, no hang: the waits end after 2 ms."""
    rng = np.random.default_rng(8)
    y = torch.from_numpy(rng.lognormal(13, 2, (1, 20_000))).cuda()
    try:
        ara.debug_set(ara.ARA_DBG_WAIT_LIMIT_NS, 2_000_000)
        ara.debug_set(ara.ARA_DBG_SKIP_BARRIER_ARRIVAL, 1)
        with pytest.raises(ara.AraError) as e:
            ara.risk_metrics(y, [100.0], [0.99])
        assert e.value.status == ara.ARA_ETIMEOUT
        pd = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
        td = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
        sd = torch.zeros((1,), dtype=torch.int32, device="cuda")
        ara.risk_metrics_async(y, [100.0], [0.99], pd, td, sd)
        torch.cuda.synchronize()
        assert int(sd.item()) & ara.ARA_DEVICE_TIMEOUT
    finally:
        ara.debug_set(ara.ARA_DBG_SKIP_BARRIER_ARRIVAL, 0)
        ara.debug_set(ara.ARA_DBG_WAIT_LIMIT_NS, 1_000_000_000)
    check(y.cpu().numpy(), rps=[100.0], levels=[0.99])


def test_large_tie_group_at_the_targets():
    """A tie group of 200k values (two thirds of the row) where the PML ranks and a TVaR
    boundary fall: the selected key is the tied value and the TVaR mean shares it."""
    rng = np.random.default_rng(9)
    y = rng.lognormal(12, 1, 300_000)
    y[:200_000] = 123456.0
    check(y, rps=[2.0, 3.0, 100.0], levels=[0.5, 0.99])


def test_layers_stopping_after_different_passes():
    """In one launch, layers whose targets fall on distinct values (the selection stops once
    each target's bin holds one key) next to layers with a tie group at the targets (all 8
    passes) and a layer of one repeated value: each layer's result is exact."""
    rng = np.random.default_rng(21)
    n = 50_000
    rows = [rng.lognormal(14, 2, n), rng.lognormal(14, 2, n), rng.lognormal(14, 2, n),
            np.full(n, 7.25)]
    rows[1][: n // 2] = 4.5e6                     # tie group holding every target
    rows[2][::2] = np.nextafter(rows[2][1::2], 0)  # near-equal pairs: unique only in the last bits
    check(np.stack(rows), rps=[1.0, 2.0, 100.0, 250.0, float(n)], levels=[0.0, 0.5, 0.99])


def test_results_unchanged_after_releasing_pooled_memory():
    """Scratch comes from the library's own memory pool, which keeps freed memory for the next
    call; ara_release_memory hands the idle part back.  Calls before and after (the pool then
    maps fresh memory) give the same, oracle-checked results."""
    rng = np.random.default_rng(44)
    y = rng.lognormal(14, 2, (3, 50_000))
    check(y)
    ara.release_memory()
    check(y)
    check(y)
    ara.release_memory()
