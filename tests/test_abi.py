"""CPU checks of the C ABI: the library loads, exports every function include/ara.h declares,
and rejects invalid arguments on the host before touching a device."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_1606_04473_gb300 as ara
from paper_1606_04473_gb300 import build as ara_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(ara.LIB_PATH):
        ara_build.build()
    return ara.lib()


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"ARA_API\s+[\w\s\*]*?\b(ara_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_function_is_exported(L):
    names = header_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    for s in [0, -1, -2, -3, -4, -5, -6, -7]:
        assert ara.status_string(s) not in ("", "unknown status")


def _create(L, C=10, rec_off=(0, 2), ids=(1, 3), loss=(5.0, 7.0), ret=(1.0,), lim=(math.inf,),
            layer_off=(0, 1), layer_elts=(0,), occ=(0.0, math.inf), agg=(0.0, math.inf), flags=0):
    a = lambda v, t: np.ascontiguousarray(np.array(v, dtype=t))
    ro, ii, ll = a(rec_off, np.int64), a(ids, np.int32), a(loss, np.float64)
    er, el = a(ret, np.float64), a(lim, np.float64)
    lo, le = a(layer_off, np.int32), a(layer_elts, np.int32)
    n_layers = len(layer_off) - 1
    orr, ol = a([occ[0]] * n_layers, np.float64), a([occ[1]] * n_layers, np.float64)
    ar, al = a([agg[0]] * n_layers, np.float64), a([agg[1]] * n_layers, np.float64)
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    h = ctypes.c_void_p()
    st = L.ara_create_portfolio(C, len(rec_off) - 1, p(ro), p(ii), p(ll), p(er), p(el), n_layers,
                                p(lo), p(le), p(orr), p(ol), p(ar), p(al), flags, ctypes.byref(h))
    if st == 0:
        L.ara_destroy_portfolio(h)
    return st


@pytest.mark.parametrize("kw", [
    dict(C=0),                                   # empty catalogue
    dict(ids=(1, 10)),                           # event ID == catalogue size
    dict(ids=(-1, 3)),                           # negative event ID
    dict(ids=(3, 3)),                            # duplicate record within an ELT
    dict(loss=(5.0, -1.0)),                      # negative loss
    dict(loss=(5.0, float("nan"))),              # NaN loss
    dict(loss=(5.0, float("inf"))),              # infinite loss
    dict(ret=(-1.0,)),                           # negative retention
    dict(ret=(math.inf,)),                       # infinite retention
    dict(lim=(float("nan"),)),                   # NaN limit
    dict(rec_off=(1, 2)),                        # offsets must start at 0
    dict(rec_off=(0, 2, 1), ret=(1.0, 1.0), lim=(1.0, 1.0)),  # decreasing offsets
    dict(layer_elts=(1,)),                       # layer refers to a missing ELT
    dict(layer_off=(0, 2), layer_elts=(0, -1)),  # negative ELT index
    dict(occ=(-1.0, 1.0)),                       # negative occurrence retention
    dict(agg=(0.0, -2.0)),                       # negative aggregate limit
    dict(flags=1, loss=(5.0, 0.1)),              # FP32 storage of a non-FP32 loss
    dict(flags=64),                              # unknown flag
])
def test_create_rejects_invalid_tables_on_host(L, kw):
    assert _create(L, **kw) == ara.ARA_EINVAL


def test_create_without_device_reports_cuda_error(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    assert _create(L) == ara.ARA_ECUDA


def test_risk_metrics_rejects_invalid_levels(L):
    p = ctypes.c_void_p(256)          # never dereferenced: arguments fail first
    out = np.zeros(4)
    po = out.ctypes.data_as(ctypes.c_void_p)

    def call(n, rps, lv):
        r = np.ascontiguousarray(rps, dtype=np.float64)
        v = np.ascontiguousarray(lv, dtype=np.float64)
        return L.ara_risk_metrics(p, n, 1, r.size, r.ctypes.data_as(ctypes.c_void_p), v.size,
                                  v.ctypes.data_as(ctypes.c_void_p), po, po, None, None)
    assert call(0, [10.0], []) == ara.ARA_EINVAL          # no trials
    assert call(100, [0.5], []) == ara.ARA_EINVAL         # return period < 1
    assert call(100, [], [1.0]) == ara.ARA_EINVAL         # level 1 -> empty tail
    assert call(100, [], [-0.1]) == ara.ARA_EINVAL
    assert call(100, [], []) == ara.ARA_EINVAL            # nothing requested
    assert call(100, [2.0] * 17, []) == ara.ARA_EINVAL    # more than 16 targets


def test_run_rejects_null_portfolio(L):
    assert L.ara_run_ylt(None, 1, None, 0, None, None, 0, None, None, None, 0, None) == ara.ARA_EINVAL
    assert L.ara_check(None, None) == ara.ARA_EINVAL
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert L.ara_timing_read(99, ctypes.byref(ms), ctypes.byref(n)) == ara.ARA_EINVAL


def test_new_entry_points_reject_null_handles_on_host(L):
    """The multi-request pass, the server's merging and estimate calls, and the plan table reject
    missing handles and arguments before touching a device; releasing pooled memory with no pool
    created is a no-op."""
    p = ctypes.c_void_p(256)          # never dereferenced: the handle check fails first
    first = np.array([0, 1], dtype=np.int32)
    tb, te = np.array([0], dtype=np.int64), np.array([1], dtype=np.int64)
    ptrs = (ctypes.c_void_p * 1)(256)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert L.ara_run_ylt_requests(None, 1, p, 0, p, 1, P(first), P(tb), P(te),
                                  ctypes.cast(ptrs, ctypes.c_void_p), None, None) == ara.ARA_EINVAL
    assert L.ara_server_set_merging(None, 2, 0.3) == ara.ARA_EINVAL
    b = ctypes.c_int64()
    assert L.ara_server_estimate_bytes(None, None, ctypes.byref(b)) == ara.ARA_EINVAL
    n = ctypes.c_int64()
    assert L.ara_server_counters(None, ctypes.byref(n), ctypes.byref(n), ctypes.byref(n),
                                 ctypes.byref(n)) == ara.ARA_EINVAL
    assert L.ara_server_set_adjoint_index(None, 1) == ara.ARA_EINVAL
    assert L.ara_plan_table(None, None, ctypes.byref(n)) == ara.ARA_EINVAL
    assert L.ara_plan_info(None, None, None, None, None, None) == ara.ARA_EINVAL
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        assert L.ara_release_memory() == ara.ARA_OK


def test_timing_classes_of_the_host_pipeline_are_readable(L):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    for k in (ara.ARA_K_TRANSFER, ara.ARA_K_HOST_CHECK):
        assert L.ara_timing_read(k, ctypes.byref(ms), ctypes.byref(n)) == ara.ARA_OK
    assert L.ara_timing_read(7, ctypes.byref(ms), ctypes.byref(n)) == ara.ARA_EINVAL


def test_yet_index_entry_points_reject_bad_arguments_on_host(L):
    """The event-major YET index and the adjoint over it refuse missing handles and outputs
    before touching a device, leave the output handle null, and accept destroying null."""
    p = ctypes.c_void_p(256)          # never dereferenced: the argument checks fail first
    out = ctypes.c_void_p(1234)
    assert L.ara_yet_index_create(None, 10, p, 100, p, None, ctypes.byref(out)) == ara.ARA_EINVAL
    assert out.value is None
    assert L.ara_yet_index_create(p, 10, p, 100, p, None, None) == ara.ARA_EINVAL
    L.ara_yet_index_destroy(None)
    assert L.ara_adjoint_indexed(None, p, 0, 0, 0, None, p, p, 0.99, p, p, p, None, None) == ara.ARA_EINVAL
    assert L.ara_adjoint_indexed(p, None, 0, 0, 0, None, p, p, 0.99, p, p, p, None, None) == ara.ARA_EINVAL
