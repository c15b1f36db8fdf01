"""The allocation-free risk-metrics entry point (ara_risk_metrics_static).

It serves callers that cannot allocate device memory: a process whose GPU memory is already
reserved in full by another allocator, or a latency-critical loop that cannot pay for an
allocation or for cudaFree's implicit synchronisation.  Its scratch is a fixed array inside
libara.  This test calls it through the C ABI, twice in a row on different inputs (the array
keeps the previous call's contents, which must not leak into the next result), and compares
each result with the allocating entry point ara_risk_metrics, within the tolerances the other
risk-metric tests use: PML exactly (it is a copy of a YLT entry), TVaR and the mean to 1e-12
relative.  It also checks that a request too large for the array is refused with ARA_ERANGE.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_1606_04473_gb300 as ara
    from paper_1606_04473_gb300 import build as ara_build


def _lib():
    import os
    if not os.path.exists(ara.LIB_PATH):
        ara_build.build()
    return ara.lib()


def _call(fn, y_dev, rps, levels):
    """Call one of the two C entry points directly; returns (status, pml, tvar, mean)."""
    nl, n = y_dev.shape
    rp = np.ascontiguousarray(rps, dtype=np.float64)
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    pml = np.full((nl, rp.size), np.nan)
    tvar = np.full((nl, lv.size), np.nan)
    mean = np.full(nl, np.nan)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(ctypes.c_void_p(y_dev.data_ptr()), n, nl, rp.size, p(rp), lv.size, p(lv), p(pml),
            p(tvar), p(mean), stream)
    return st, pml, tvar, mean


def _ylt(seed, n_layers, n):
    rng = np.random.default_rng(seed)
    y = rng.lognormal(14.0, 2.0, (n_layers, n))
    y[:, : n // 5] = 0.0                              # a block of zero years, as under a retention
    y[:, n // 5: n // 5 + 50] = 7.5e6                 # ties
    return torch.from_numpy(y).cuda()


def test_no_alloc_matches_allocating_entry_point_on_two_calls():
    L = _lib()
    cases = [(_ylt(1, 3, 100_003), [100.0, 250.0, 10.0], [0.99, 0.5]),
             (_ylt(2, 5, 4_097), [2.0], [0.9, 0.99, 0.0])]
    for y, rps, levels in cases:          # first call sets the device address up, second reuses
        st_s, p_s, t_s, m_s = _call(L.ara_risk_metrics_static, y, rps, levels)
        st_a, p_a, t_a, m_a = _call(L.ara_risk_metrics, y, rps, levels)
        assert st_s == ara.ARA_OK and st_a == ara.ARA_OK
        assert np.array_equal(p_s, p_a)
        np.testing.assert_allclose(t_s, t_a, rtol=1e-12, atol=0)
        np.testing.assert_allclose(m_s, m_a, rtol=1e-12, atol=0)


def test_no_alloc_refuses_requests_beyond_its_capacity():
    L = _lib()
    y = _ylt(3, 200, 64)                  # 200 layers x 16 levels needs ~26 MB of scratch
    st, *_ = _call(L.ara_risk_metrics_static, y, [1.0] * 8, [0.5] * 8)
    assert st == ara.ARA_ERANGE
    st, *_ = _call(L.ara_risk_metrics, y, [1.0] * 8, [0.5] * 8)   # the allocating one copes
    assert st == ara.ARA_OK
