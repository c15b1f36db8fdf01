"""Aggregate Risk Analysis on GB300 (sm_103a): Python binding of libara.so.

This module only marshals arguments to the C ABI declared in include/ara.h; every step of
the computation runs in the library's CUDA kernels.  PyTorch provides device memory and
streams.  There is no CPU fallback: if libara.so is missing or cannot be loaded, every
call raises.

Paper mapping (arXiv 1606.04473, Section IV):
  Portfolio          ELTs (Eq. 2) with terms I, layers (Eq. 3) with terms T
  Portfolio.run_ylt  Algorithm 1 around Algorithm 3 for a YET already on the device
  Portfolio.run_ylt_host  the same with the transfer of Algorithm 2 overlapped
  risk_metrics       PML and TVaR of the YLT (named in Section IV-A)
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libara.so")

ARA_OK, ARA_EINVAL, ARA_ENOMEM, ARA_ECUDA, ARA_ETIMEOUT, ARA_EBUSY, ARA_EDATA = 0, -1, -2, -3, -4, -5, -6
ARA_ERANGE = -7
ARA_STATIC_SELECT_BYTES = 4 << 20
ARA_LOSSES_F32, ARA_DENSE_TABLES = 1, 2
ARA_RUN_FOLDED, ARA_RUN_PER_ELT, ARA_RUN_NO_FILTER, ARA_RUN_F64_SUM, ARA_RUN_LDG = 0, 1, 2, 4, 8
ARA_RUN_HOST_DIRECT = 16
ARA_RUN_BATCHED = 32
ARA_RUN_OEP = 64


class Query(ctypes.Structure):
    """ara_query (include/ara.h)."""
    _fields_ = [("n_layers", ctypes.c_int32), ("layer_elt_offsets", ctypes.c_void_p),
                ("layer_elt_ids", ctypes.c_void_p), ("occ_ret", ctypes.c_void_p),
                ("occ_lim", ctypes.c_void_p), ("agg_ret", ctypes.c_void_p),
                ("agg_lim", ctypes.c_void_p), ("trial_begin", ctypes.c_int64),
                ("trial_end", ctypes.c_int64), ("n_rp", ctypes.c_int32),
                ("return_periods", ctypes.c_void_p), ("n_tvar", ctypes.c_int32),
                ("tvar_levels", ctypes.c_void_p), ("want_mean", ctypes.c_int32),
                ("want_adjoint", ctypes.c_int32), ("adjoint_level", ctypes.c_double),
                ("flags", ctypes.c_int32), ("tenant", ctypes.c_int32)]
ARA_K_FOLD, ARA_K_YLT, ARA_K_SELECT, ARA_K_ADJOINT, ARA_K_BATCHED = 0, 1, 2, 3, 4
ARA_K_TRANSFER, ARA_K_HOST_CHECK = 5, 6
ARA_RUN_PREPARED, ARA_RUN_SLOT1 = 256, 512
ARA_PLAN_AUTOTUNE = 1

_lib = None


class AraError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def lib() -> ctypes.CDLL:
    """Load libara.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libara.so not found at {LIB_PATH}; build it with "
                           "paper_1606_04473_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.ara_create_portfolio.argtypes = [i64, i32, P, P, P, P, P, i32, P, P, P, P, P, P, i32,
                                       ctypes.POINTER(P)]
    L.ara_destroy_portfolio.argtypes = [P]
    L.ara_destroy_portfolio.restype = None
    L.ara_run_ylt.argtypes = [P, i64, P, i64, P, P, i32, P, P, P, i32, P]
    L.ara_run_ylt_host.argtypes = [P, i64, P, P, i32, P, P, i32, P, i32, P, P, P, P, i32, P]
    L.ara_check.argtypes = [P, P]
    L.ara_risk_metrics.argtypes = [P, i64, i32, i32, P, i32, P, P, P, P, P]
    L.ara_risk_metrics_static.argtypes = [P, i64, i32, i32, P, i32, P, P, P, P, P]
    L.ara_risk_metrics_async.argtypes = [P, i64, i32, i32, P, i32, P, P, P, P, P, P]
    L.ara_launch_count.restype = i64
    L.ara_stream_shapes.argtypes = [P, P, i32]
    L.ara_stream_shapes.restype = i32
    L.ara_set_stream_shape.argtypes = [i32]
    L.ara_set_stream_shape.restype = i32
    L.ara_debug_set.argtypes = [i32, i64]
    L.ara_debug_set.restype = i32
    L.ara_plan_batched.argtypes = [P, i64, P, i64, P, i32, P, P, P, i32, P, ctypes.POINTER(P)]
    L.ara_plan_batched.restype = i32
    L.ara_plan_launch.argtypes = [P, P]
    L.ara_plan_launch.restype = i32
    L.ara_plan_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                ctypes.POINTER(d), ctypes.POINTER(i32)]
    L.ara_plan_info.restype = i32
    L.ara_plan_table.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(i64)]
    L.ara_plan_table.restype = i32
    L.ara_plan_destroy.argtypes = [P]
    L.ara_plan_destroy.restype = None
    L.ara_create_layer_set.argtypes = [P, i32, P, P, P, P, P, P, P, ctypes.POINTER(P)]
    L.ara_create_layer_set.restype = i32
    L.ara_server_create.argtypes = [P, i64, P, i64, P, i32, i64, ctypes.POINTER(P)]
    L.ara_server_create.restype = i32
    L.ara_server_submit.argtypes = [P, ctypes.POINTER(Query), ctypes.POINTER(i64)]
    L.ara_server_submit.restype = i32
    L.ara_server_wait.argtypes = [P, i64, P, P, P, P, P]
    L.ara_server_wait.restype = i32
    L.ara_server_stats.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64)]
    L.ara_server_stats.restype = i32
    L.ara_prepare_ylt.argtypes = [P, i32, P, i32, i32, P]
    L.ara_prepare_ylt.restype = i32
    L.ara_run_ylt_requests.argtypes = [P, i64, P, i64, P, i32, P, P, P, P, P, P]
    L.ara_run_ylt_requests.restype = i32
    L.ara_release_memory.argtypes = []
    L.ara_release_memory.restype = i32
    L.ara_server_estimate_bytes.argtypes = [P, ctypes.POINTER(Query), ctypes.POINTER(i64)]
    L.ara_server_estimate_bytes.restype = i32
    L.ara_server_set_merging.argtypes = [P, i32, d]
    L.ara_server_set_merging.restype = i32
    L.ara_server_counters.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64)]
    L.ara_server_set_adjoint_index.argtypes = [P, i32]
    L.ara_server_set_adjoint_index.restype = i32
    L.ara_server_counters.restype = i32
    L.ara_server_destroy.argtypes = [P]
    L.ara_server_destroy.restype = None
    L.ara_adjoint.argtypes = [P, i64, P, i64, P, i32, P, P, P, d, P, P, P, P, P]
    L.ara_adjoint.restype = i32
    L.ara_adjoint_accumulate.argtypes = [P, i64, P, i64, P, i32, P, P, P, d, P, P, P, P, P, P]
    L.ara_adjoint_accumulate.restype = i32
    L.ara_yet_index_create.argtypes = [P, i64, P, i64, P, P, ctypes.POINTER(P)]
    L.ara_yet_index_create.restype = i32
    L.ara_yet_index_destroy.argtypes = [P]
    L.ara_yet_index_destroy.restype = None
    L.ara_adjoint_indexed.argtypes = [P, P, i64, i64, i32, P, P, P, d, P, P, P, P, P]
    L.ara_adjoint_indexed.restype = i32
    L.ara_timing_enable.argtypes = [i32]
    L.ara_timing_enable.restype = None
    L.ara_timing_reset.restype = None
    L.ara_timing_read.argtypes = [i32, ctypes.POINTER(d), ctypes.POINTER(i64)]
    L.ara_status_string.argtypes = [i32]
    L.ara_status_string.restype = ctypes.c_char_p
    for fn in ["ara_create_portfolio", "ara_run_ylt", "ara_run_ylt_host", "ara_check",
               "ara_risk_metrics", "ara_risk_metrics_static", "ara_timing_read"]:
        getattr(L, fn).restype = i32
    _lib = L
    return L


def status_string(s: int) -> str:
    try:
        return lib().ara_status_string(int(s)).decode()
    except Exception:
        return "unknown"


def _check(st: int, what: str):
    if st != ARA_OK:
        raise AraError(st, what)


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream (or the current stream when None)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Portfolio:
    """A portfolio resident on the current CUDA device (ara_create_portfolio)."""

    def __init__(self, catalogue: int, elt_ids: Sequence[np.ndarray], elt_losses: Sequence[np.ndarray],
                 elt_ret, elt_lim, layer_elts: Sequence[Sequence[int]], occ_ret, occ_lim,
                 agg_ret, agg_lim, losses_f32: bool = False, dense_tables: bool = False):
        L = lib()
        n_elts = len(elt_ids)
        off = np.zeros(n_elts + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(x) for x in elt_ids])
        ids = np.ascontiguousarray(np.concatenate(elt_ids) if n_elts else np.zeros(0), dtype=np.int32)
        loss = np.ascontiguousarray(np.concatenate(elt_losses) if n_elts else np.zeros(0), dtype=np.float64)
        loff = np.zeros(len(layer_elts) + 1, dtype=np.int32)
        loff[1:] = np.cumsum([len(l) for l in layer_elts])
        lel = np.ascontiguousarray([j for l in layer_elts for j in l], dtype=np.int32)
        f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        self._keep = [off, ids, loss, loff, lel]
        er, el, orr, ol, ar, al = (f(elt_ret), f(elt_lim), f(occ_ret), f(occ_lim), f(agg_ret), f(agg_lim))
        flags = (ARA_LOSSES_F32 if losses_f32 else 0) | (ARA_DENSE_TABLES if dense_tables else 0)
        h = ctypes.c_void_p()
        st = L.ara_create_portfolio(int(catalogue), n_elts, _np_ptr(off), _np_ptr(ids), _np_ptr(loss),
                                    _np_ptr(er), _np_ptr(el), len(layer_elts), _np_ptr(loff),
                                    _np_ptr(lel), _np_ptr(orr), _np_ptr(ol), _np_ptr(ar), _np_ptr(al),
                                    flags, ctypes.byref(h))
        _check(st, "ara_create_portfolio")
        self._h = h
        self.catalogue = int(catalogue)
        self.n_layers = len(layer_elts)
        self.n_elts = n_elts
        self.layer_elts = [list(map(int, l)) for l in layer_elts]
        self.elt_nnz = [int(len(x)) for x in elt_ids]
        self.n_records = int(off[-1])

    @classmethod
    def from_tables(cls, pf, dense_tables: bool = False) -> "Portfolio":
        """From an object with the fields of the paper's tables (catalogue, elt_ids, elt_losses,
        elt_ret, elt_lim, layer_elts, occ_ret, occ_lim, agg_ret, agg_lim, losses_f32)."""
        return cls(pf.catalogue, pf.elt_ids, pf.elt_losses, pf.elt_ret, pf.elt_lim, pf.layer_elts,
                   pf.occ_ret, pf.occ_lim, pf.agg_ret, pf.agg_lim,
                   losses_f32=bool(getattr(pf, "losses_f32", False)), dense_tables=dense_tables)

    def close(self):
        if getattr(self, "_h", None):
            lib().ara_destroy_portfolio(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sel(self, layers):
        if layers is None:
            return 0, None, self.n_layers, None
        sel = np.ascontiguousarray(np.asarray(layers, dtype=np.int32).reshape(-1))
        return sel.size, _np_ptr(sel), sel.size, sel

    def run_ylt(self, offsets, event_ids, layers=None, out=None, regimes=None, flags: int = 0,
                stream=None, timestamps=None):
        """YLT [n_layers_selected, n_trials] (float64, on the device) of a device-resident YET.
        Asynchronous on `stream`; call check() to surface device-side data errors."""
        import torch
        n_trials = offsets.numel() - 1
        n_sel, sel_p, n_out, _sel = self._sel(layers)
        if out is None:
            out = torch.empty((n_out, n_trials), dtype=torch.float64, device=offsets.device)
        st = lib().ara_run_ylt(self._h, n_trials, _dev_ptr(offsets, torch.int64, "offsets"),
                               event_ids.numel(), _dev_ptr(event_ids, torch.int32, "event_ids"),
                               None if timestamps is None else _dev_ptr(timestamps, torch.float32, "timestamps"),
                               n_sel, sel_p, _dev_ptr(out, torch.float64, "out"),
                               None if regimes is None else _dev_ptr(regimes, torch.uint8, "regimes"),
                               int(flags), _stream_handle(stream))
        _check(st, "ara_run_ylt")
        return out

    def prepare_ylt(self, layers=None, slot: int = 0, flags: int = 0, stream=None):
        """Queue the fold of the selected layers into fold slot 0 or 1 (ara_prepare_ylt); a later
        run_ylt with flags ARA_RUN_PREPARED (| ARA_RUN_SLOT1 for slot 1) streams against it."""
        n_sel, sel_p, _n_out, _sel = self._sel(layers)
        _check(lib().ara_prepare_ylt(self._h, n_sel, sel_p, int(slot), int(flags),
                                     _stream_handle(stream)), "ara_prepare_ylt")

    def run_ylt_requests(self, offsets, event_ids, requests, regimes: bool = False, stream=None):
        """Several requests in one pass (ara_run_ylt_requests): requests is a list of
        (layer_begin, layer_end, trial_begin, trial_end) covering the portfolio's layers in
        order.  Returns one YLT tensor [its layers, its trials] per request (and the regime
        tensors when regimes=True)."""
        import torch
        n_trials = offsets.numel() - 1
        n = len(requests)
        first = np.ascontiguousarray([r[0] for r in requests] + [requests[-1][1]], dtype=np.int32)
        tb = np.ascontiguousarray([r[2] for r in requests], dtype=np.int64)
        te = np.ascontiguousarray([r[3] for r in requests], dtype=np.int64)
        ys = [torch.empty((r[1] - r[0], r[3] - r[2]), dtype=torch.float64, device=offsets.device)
              for r in requests]
        rs = [torch.empty((r[1] - r[0], r[3] - r[2]), dtype=torch.uint8, device=offsets.device)
              for r in requests] if regimes else None
        yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        rp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in rs]) if regimes else None
        st = lib().ara_run_ylt_requests(self._h, n_trials, _dev_ptr(offsets, torch.int64, "offsets"),
                                        event_ids.numel(), _dev_ptr(event_ids, torch.int32, "event_ids"),
                                        n, _np_ptr(first), _np_ptr(tb), _np_ptr(te),
                                        ctypes.cast(yp, ctypes.c_void_p),
                                        ctypes.cast(rp, ctypes.c_void_p) if regimes else None,
                                        _stream_handle(stream))
        _check(st, "ara_run_ylt_requests")
        return (ys, rs) if regimes else ys

    def run_ylt_host(self, offsets: np.ndarray, event_ids: np.ndarray, layers=None, out=None,
                     return_periods: Sequence[float] = (), tvar_levels: Sequence[float] = (),
                     want_ylt: bool = True, want_mean: bool = False, flags: int = 0, stream=None):
        """The whole analysis from host memory (synchronous): YLT [n_layers_selected, n_trials]
        on the host, plus (PML, TVaR) when return periods / levels are given.  Pinned host
        arrays (e.g. from torch pin_memory) transfer at full link bandwidth."""
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        event_ids = np.ascontiguousarray(event_ids, dtype=np.int32)
        n_trials = offsets.size - 1
        n_sel, sel_p, n_out, _sel = self._sel(layers)
        if want_ylt and out is None:
            out = np.empty((n_out, n_trials), dtype=np.float64)
        if out is not None:
            assert out.dtype == np.float64 and out.flags.c_contiguous and out.shape == (n_out, n_trials)
        rp = np.ascontiguousarray(return_periods, dtype=np.float64)
        lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
        pml = np.zeros((n_out, rp.size))
        tvar = np.zeros((n_out, lv.size))
        mean = np.zeros(n_out) if want_mean else None
        st = lib().ara_run_ylt_host(self._h, n_trials, _np_ptr(offsets), _np_ptr(event_ids), n_sel,
                                    sel_p, _np_ptr(out), rp.size, _np_ptr(rp), lv.size, _np_ptr(lv),
                                    _np_ptr(pml), _np_ptr(tvar), _np_ptr(mean), int(flags),
                                    _stream_handle(stream))
        _check(st, "ara_run_ylt_host")
        if want_mean:
            return out, pml, tvar, mean
        if rp.size or lv.size:
            return out, pml, tvar
        return out

    def adjoint(self, offsets, event_ids, ylt, regimes, tvar_level: float = 0.99, layers=None,
                stream=None, index: "YetIndex" = None, first_trial: int = 0):
        """Gradients of each selected layer's mean year loss (objective 0) and TVaR (objective 1)
        from a forward run's YLT and regimes (ara_adjoint; with `index`, a YetIndex of a YET whose
        trials [first_trial, first_trial + ylt columns) the forward ran over,
        ara_adjoint_indexed, and offsets / event_ids may be None).  Returns a dict of device
        tensors: 'elt' [2, K, 2] (d/dR, d/dL per ELT slot), 'layer' [2, n_sel, 4] (OccR, OccL,
        AggR, AggL), 'loss' [2, M] (per record of each slot, creation order), and 'ties' (numpy
        int32)."""
        import torch
        n_sel, sel_p, n_out, sel = self._sel(layers)
        lay = list(range(self.n_layers)) if sel is None else [int(x) for x in sel]
        K = sum(len(self.layer_elts[l]) for l in lay)
        M = sum(self.elt_nnz[j] for l in lay for j in self.layer_elts[l])
        dev = ylt.device
        ge = torch.zeros((2, max(K, 1), 2), dtype=torch.float64, device=dev)
        gl = torch.zeros((2, n_out, 4), dtype=torch.float64, device=dev)
        gx = torch.zeros((2, max(M, 1)), dtype=torch.float64, device=dev)
        ties = np.zeros(n_out, dtype=np.int32)
        if index is not None:
            st = lib().ara_adjoint_indexed(self._h, index._handle(), int(first_trial),
                                           int(ylt.shape[-1]), n_sel, sel_p,
                                           _dev_ptr(ylt, torch.float64, "ylt"),
                                           _dev_ptr(regimes, torch.uint8, "regimes"), float(tvar_level),
                                           _dev_ptr(ge, torch.float64, "g"), _dev_ptr(gl, torch.float64, "g"),
                                           _dev_ptr(gx, torch.float64, "g"), _np_ptr(ties),
                                           _stream_handle(stream))
            _check(st, "ara_adjoint_indexed")
        else:
            n_trials = offsets.numel() - 1
            st = lib().ara_adjoint(self._h, n_trials, _dev_ptr(offsets, torch.int64, "offsets"),
                                   event_ids.numel(), _dev_ptr(event_ids, torch.int32, "event_ids"),
                                   n_sel, sel_p, _dev_ptr(ylt, torch.float64, "ylt"),
                                   _dev_ptr(regimes, torch.uint8, "regimes"), float(tvar_level),
                                   _dev_ptr(ge, torch.float64, "g"), _dev_ptr(gl, torch.float64, "g"),
                                   _dev_ptr(gx, torch.float64, "g"), _np_ptr(ties), _stream_handle(stream))
            _check(st, "ara_adjoint")
        return {"elt": ge[:, :K], "layer": gl, "loss": gx[:, :M], "ties": ties}

    def yet_index(self, offsets, event_ids, stream=None) -> "YetIndex":
        """Event-major index of a device YET for this portfolio's catalogue
        (ara_yet_index_create), for adjoint(..., index=...) calls over the same YET."""
        return YetIndex(self, offsets, event_ids, stream)

    def adjoint_accumulate(self, offsets, event_ids, ylt, regimes, weights, tvar_level: float = 0.99,
                           layers=None, out=None, stream=None):
        """Upstream-weighted gradients in parameter layout (ara_adjoint_accumulate): weights
        [n_sel, 2] for (mean, TVaR) of each selected layer; returns (or adds into `out`) the dict
        'elt_ret' [n_elts], 'elt_lim' [n_elts], 'layer' [n_layers, 4], 'loss' [n_records]."""
        import torch
        n_trials = offsets.numel() - 1
        n_sel, sel_p, n_out, _s = self._sel(layers)
        dev = offsets.device
        if out is None:
            out = {"elt_ret": torch.zeros(max(self.n_elts, 1), dtype=torch.float64, device=dev),
                   "elt_lim": torch.zeros(max(self.n_elts, 1), dtype=torch.float64, device=dev),
                   "layer": torch.zeros((max(self.n_layers, 1), 4), dtype=torch.float64, device=dev),
                   "loss": torch.zeros(max(self.n_records, 1), dtype=torch.float64, device=dev)}
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(n_out, 2))
        st = lib().ara_adjoint_accumulate(
            self._h, n_trials, _dev_ptr(offsets, torch.int64, "offsets"), event_ids.numel(),
            _dev_ptr(event_ids, torch.int32, "event_ids"), n_sel, sel_p,
            _dev_ptr(ylt, torch.float64, "ylt"), _dev_ptr(regimes, torch.uint8, "regimes"),
            float(tvar_level), _np_ptr(w), _dev_ptr(out["elt_ret"], torch.float64, "g"),
            _dev_ptr(out["elt_lim"], torch.float64, "g"), _dev_ptr(out["layer"], torch.float64, "g"),
            _dev_ptr(out["loss"], torch.float64, "g"), _stream_handle(stream))
        _check(st, "ara_adjoint_accumulate")
        return out

    def layer_set(self, layer_elts, occ_ret, occ_lim, agg_ret, agg_lim, stream=None) -> "Portfolio":
        """New layers over this portfolio's resident ELTs (ara_create_layer_set)."""
        loff = np.zeros(len(layer_elts) + 1, dtype=np.int32)
        loff[1:] = np.cumsum([len(l) for l in layer_elts])
        lel = np.ascontiguousarray([j for l in layer_elts for j in l], dtype=np.int32)
        f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        orr, ol, ar, al = f(occ_ret), f(occ_lim), f(agg_ret), f(agg_lim)
        h = ctypes.c_void_p()
        st = lib().ara_create_layer_set(self._h, len(layer_elts), _np_ptr(loff), _np_ptr(lel), _np_ptr(orr),
                                        _np_ptr(ol), _np_ptr(ar), _np_ptr(al), _stream_handle(stream),
                                        ctypes.byref(h))
        _check(st, "ara_create_layer_set")
        ls = Portfolio.__new__(Portfolio)
        ls._h, ls._keep, ls._pool = h, [loff, lel], self
        ls.catalogue, ls.n_layers, ls.n_elts = self.catalogue, len(layer_elts), self.n_elts
        ls.layer_elts = [list(map(int, l)) for l in layer_elts]
        ls.elt_nnz, ls.n_records = self.elt_nnz, self.n_records
        return ls

    def check(self, stream=None):
        _check(lib().ara_check(self._h, _stream_handle(stream)), "ara_check")


class YetIndex:
    """An event-major index of a device YET (ara_yet_index_create).  It owns its device memory;
    the YET may change or go afterwards."""

    def __init__(self, portfolio: Portfolio, offsets, event_ids, stream=None):
        import torch
        self.n_trials = offsets.numel() - 1
        h = ctypes.c_void_p()
        st = lib().ara_yet_index_create(portfolio._h, self.n_trials,
                                        _dev_ptr(offsets, torch.int64, "offsets"), event_ids.numel(),
                                        _dev_ptr(event_ids, torch.int32, "event_ids"),
                                        _stream_handle(stream), ctypes.byref(h))
        _check(st, "ara_yet_index_create")
        self._h = h

    def _handle(self):
        if not getattr(self, "_h", None):
            raise AraError(ARA_EINVAL, "YetIndex is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().ara_yet_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchedPlan:
    """Every selected layer in one pass over a device YET, as one CUDA graph (ara_plan_batched).
    The YET and output buffers are bound at construction; launch() recomputes the YLT."""

    def __init__(self, portfolio: Portfolio, offsets, event_ids, layers=None, out=None, regimes=None,
                 autotune: bool = True, stream=None):
        import torch
        n_trials = offsets.numel() - 1
        n_sel, sel_p, n_out, _sel = portfolio._sel(layers)
        if out is None:
            out = torch.empty((n_out, n_trials), dtype=torch.float64, device=offsets.device)
        self.out, self.regimes = out, regimes
        self._keep = (portfolio, offsets, event_ids, _sel)
        h = ctypes.c_void_p()
        st = lib().ara_plan_batched(portfolio._h, n_trials, _dev_ptr(offsets, torch.int64, "offsets"),
                                    event_ids.numel(), _dev_ptr(event_ids, torch.int32, "event_ids"),
                                    n_sel, sel_p, _dev_ptr(out, torch.float64, "out"),
                                    None if regimes is None else _dev_ptr(regimes, torch.uint8, "regimes"),
                                    ARA_PLAN_AUTOTUNE if autotune else 0, _stream_handle(stream),
                                    ctypes.byref(h))
        _check(st, "ara_plan_batched")
        self._h = h

    def launch(self, stream=None):
        _check(lib().ara_plan_launch(self._h, _stream_handle(stream)), "ara_plan_launch")
        return self.out

    def info(self):
        w, c, t, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        k = ctypes.c_int32()
        _check(lib().ara_plan_info(self._h, ctypes.byref(w), ctypes.byref(c), ctypes.byref(t),
                                   ctypes.byref(ms), ctypes.byref(k)), "ara_plan_info")
        return {"warps": w.value, "blocks_per_sm": c.value, "trials_per_grab": t.value,
                "accumulator_copies": k.value, "tuned_ms": ms.value}

    def table(self):
        """(row descriptors, entries): the plan's event-major table for measurement
        (ara_plan_table) as an int64 device tensor [catalogue] viewing the plan's own array (valid
        while the plan lives; bits 32..39 of a descriptor: the event's number of entries), and
        the table's entry count."""
        import torch
        p, n = ctypes.c_void_p(), ctypes.c_int64()
        _check(lib().ara_plan_table(self._h, ctypes.byref(p), ctypes.byref(n)), "ara_plan_table")

        class _View:
            pass
        v = _View()
        v.__cuda_array_interface__ = {"shape": (self._keep[0].catalogue,), "typestr": "<i8",
                                      "data": (p.value, False), "version": 3}
        return torch.as_tensor(v, device=self._keep[1].device), n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().ara_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Native request server over this pool's resident ELTs and a resident device YET
    (ara_server_*).  submit() queues a query and returns a ticket; wait() returns its results."""

    def __init__(self, pool: Portfolio, offsets, event_ids, max_concurrent: int = 4,
                 memory_budget: int = 0, max_merge: int = 4, min_overlap: float = 0.6):
        import torch
        self._keep = (pool, offsets, event_ids)
        self.n_trials = offsets.numel() - 1
        h = ctypes.c_void_p()
        st = lib().ara_server_create(pool._h, self.n_trials, _dev_ptr(offsets, torch.int64, "offsets"),
                                     event_ids.numel(), _dev_ptr(event_ids, torch.int32, "event_ids"),
                                     int(max_concurrent), int(memory_budget), ctypes.byref(h))
        _check(st, "ara_server_create")
        self._h = h
        self._shapes = {}
        self.set_merging(max_merge, min_overlap)

    def set_merging(self, max_merge: int, min_overlap: float = 0.6):
        """Merge up to max_merge queued requests with overlapping slices into one pass
        (ara_server_set_merging; 1 = no merging)."""
        _check(lib().ara_server_set_merging(self._h, int(max_merge), float(min_overlap)),
               "ara_server_set_merging")

    def counters(self):
        a, b, c, x = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ara_server_counters(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                         ctypes.byref(x)), "ara_server_counters")
        return {"passes": a.value, "merged_requests": b.value, "head_passed": c.value,
                "indexed_adjoints": x.value}

    def set_adjoint_index(self, on: bool = True):
        """Build (or release) an event-major index of the resident YET for adjoint requests
        (ara_server_set_adjoint_index; only while the server is idle)."""
        _check(lib().ara_server_set_adjoint_index(self._h, 1 if on else 0), "ara_server_set_adjoint_index")

    @staticmethod
    def _query(layer_elts, occ_ret, occ_lim, agg_ret, agg_lim, trials, return_periods=(),
               tvar_levels=(), want_mean=False, want_adjoint=False, adjoint_level=0.99, flags=0,
               tenant=0):
        """(ara_query, the arrays it points into: keep them alive while it is used)."""
        loff = np.zeros(len(layer_elts) + 1, dtype=np.int32)
        loff[1:] = np.cumsum([len(l) for l in layer_elts])
        lel = np.ascontiguousarray([j for l in layer_elts for j in l] or [0], dtype=np.int32)
        f = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
        arrs = [loff, lel, f(occ_ret), f(occ_lim), f(agg_ret), f(agg_lim), f(return_periods or [0.0]),
                f(tvar_levels or [0.0])]
        q = Query(len(layer_elts), *[a.ctypes.data for a in arrs[:6]], int(trials[0]), int(trials[1]),
                  len(return_periods), arrs[6].ctypes.data, len(tvar_levels), arrs[7].ctypes.data,
                  int(want_mean), int(want_adjoint), float(adjoint_level), int(flags), int(tenant))
        return q, arrs

    def estimate_bytes(self, **query) -> int:
        """The device memory the server's admission assumes for this query
        (ara_server_estimate_bytes)."""
        q, _arrs = self._query(**query)
        b = ctypes.c_int64()
        _check(lib().ara_server_estimate_bytes(self._h, ctypes.byref(q), ctypes.byref(b)),
               "ara_server_estimate_bytes")
        return b.value

    def submit(self, layer_elts, occ_ret, occ_lim, agg_ret, agg_lim, trials, return_periods=(),
               tvar_levels=(), want_mean=False, want_adjoint=False, adjoint_level=0.99, flags=0,
               tenant=0) -> int:
        q, arrs = self._query(layer_elts, occ_ret, occ_lim, agg_ret, agg_lim, trials, return_periods,
                              tvar_levels, want_mean, want_adjoint, adjoint_level, flags, tenant)
        t = ctypes.c_int64()
        _check(lib().ara_server_submit(self._h, ctypes.byref(q), ctypes.byref(t)), "ara_server_submit")
        self._shapes[t.value] = (len(layer_elts), len(return_periods), len(tvar_levels), want_mean,
                                 want_adjoint)
        return t.value

    def wait(self, ticket: int):
        nl, nr, nt, wm, wa = self._shapes.pop(ticket)
        pml, tvar = np.zeros((nl, nr)), np.zeros((nl, nt))
        mean = np.zeros(nl) if wm else None
        grad = np.zeros((2, nl, 4)) if wa else None
        times = np.zeros(3)
        st = lib().ara_server_wait(self._h, ticket, _np_ptr(pml), _np_ptr(tvar), _np_ptr(mean),
                                   _np_ptr(grad), _np_ptr(times))
        _check(st, "request")
        return {"pml": pml, "tvar": tvar, "mean": mean, "grad_layer": grad,
                "queued_s": times[0], "run_s": times[1], "latency_s": times[2]}

    def stats(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        c, d = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ara_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                      ctypes.byref(d)), "ara_server_stats")
        return {"in_flight": a.value, "peak_running": b.value, "peak_bytes": c.value, "budget": d.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().ara_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def risk_metrics(ylt, return_periods: Sequence[float] = (), tvar_levels: Sequence[float] = (),
                 stream=None, want_mean: bool = False):
    """(PML [n_layers, n_rp], TVaR [n_layers, n_tvar][, mean [n_layers]]) of a device YLT
    [n_layers, n_trials]."""
    import torch
    ylt2 = ylt if ylt.dim() == 2 else ylt.reshape(1, -1)
    nl, n = ylt2.shape
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    pml = np.zeros((nl, rp.size))
    tvar = np.zeros((nl, lv.size))
    mean = np.zeros(nl) if want_mean else None
    st = lib().ara_risk_metrics(_dev_ptr(ylt2, torch.float64, "ylt"), n, nl, rp.size, _np_ptr(rp),
                                lv.size, _np_ptr(lv), _np_ptr(pml), _np_ptr(tvar), _np_ptr(mean),
                                _stream_handle(stream))
    _check(st, "ara_risk_metrics")
    return (pml, tvar, mean) if want_mean else (pml, tvar)


ARA_DEVICE_TIMEOUT = 4


def risk_metrics_async(ylt, return_periods: Sequence[float], tvar_levels: Sequence[float],
                       pml, tvar, status, mean=None, stream=None):
    """Stream-ordered risk metrics (ara_risk_metrics_async): queues the selection on `stream`
    and returns at once.  pml [n_layers, n_rp], tvar [n_layers, n_tvar], mean [n_layers] (or
    None) are float64 CUDA tensors and status a 1-element int32 CUDA tensor, all written when
    the queued work completes (status & ARA_DEVICE_TIMEOUT: a device-side wait ran out)."""
    import torch
    ylt2 = ylt if ylt.dim() == 2 else ylt.reshape(1, -1)
    nl, n = ylt2.shape
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    if tuple(pml.shape) != (nl, rp.size) or tuple(tvar.shape) != (nl, lv.size):
        raise ValueError("pml / tvar must be [n_layers, n_rp] / [n_layers, n_tvar]")
    if mean is not None and tuple(mean.shape) != (nl,):
        raise ValueError("mean must be [n_layers]")
    if status.numel() != 1 or status.dtype != torch.int32 or not status.is_cuda:
        raise ValueError("status must be a 1-element int32 CUDA tensor")
    st = lib().ara_risk_metrics_async(
        _dev_ptr(ylt2, torch.float64, "ylt"), n, nl, rp.size, _np_ptr(rp), lv.size, _np_ptr(lv),
        _dev_ptr(pml, torch.float64, "pml") if rp.size else None,
        _dev_ptr(tvar, torch.float64, "tvar") if lv.size else None,
        _dev_ptr(mean, torch.float64, "mean") if mean is not None else None,
        ctypes.c_void_p(status.data_ptr()), _stream_handle(stream))
    _check(st, "ara_risk_metrics_async")


def risk_metrics_static(ylt, return_periods: Sequence[float] = (), tvar_levels: Sequence[float] = (),
                        stream=None, want_mean: bool = False):
    """risk_metrics() without any device allocation (ara_risk_metrics_static), for callers whose
    device memory is owned by another allocator or who cannot pay for an allocation: scratch
    comes from a fixed array inside libara.  Raises AraError(ARA_ERANGE) when the request does
    not fit that array; concurrent calls on one device must be serialised by the caller."""
    import torch
    ylt2 = ylt if ylt.dim() == 2 else ylt.reshape(1, -1)
    nl, n = ylt2.shape
    rp = np.ascontiguousarray(return_periods, dtype=np.float64)
    lv = np.ascontiguousarray(tvar_levels, dtype=np.float64)
    pml = np.zeros((nl, rp.size))
    tvar = np.zeros((nl, lv.size))
    mean = np.zeros(nl) if want_mean else None
    st = lib().ara_risk_metrics_static(_dev_ptr(ylt2, torch.float64, "ylt"), n, nl, rp.size,
                                       _np_ptr(rp), lv.size, _np_ptr(lv), _np_ptr(pml),
                                       _np_ptr(tvar), _np_ptr(mean), _stream_handle(stream))
    _check(st, "ara_risk_metrics_static")
    return (pml, tvar, mean) if want_mean else (pml, tvar)


def release_memory():
    """Return the idle memory of the library's pools to the system (ara_release_memory)."""
    _check(lib().ara_release_memory(), "ara_release_memory")


def launch_count() -> int:
    return int(lib().ara_launch_count())


def stream_shapes():
    """Compiled (warps per block, ring stages) shapes of the YET-stream kernel."""
    w = np.zeros(64, dtype=np.int32)
    st = np.zeros(64, dtype=np.int32)
    n = lib().ara_stream_shapes(_np_ptr(w), _np_ptr(st), 64)
    return [(int(w[i]), int(st[i])) for i in range(n)]


def set_stream_shape(index: int):
    _check(lib().ara_set_stream_shape(int(index)), "ara_set_stream_shape")


ARA_DBG_WAIT_LIMIT_NS, ARA_DBG_STARVE_COPIES, ARA_DBG_SKIP_BARRIER_ARRIVAL = 1, 2, 3
ARA_DBG_ADJOINT_PER_LAYER = 4


def debug_set(key: int, value: int):
    """Failure-detection hooks for tests (see ara_debug_set in include/ara.h)."""
    _check(lib().ara_debug_set(int(key), int(value)), "ara_debug_set")


def timing_enable(on: bool = True):
    lib().ara_timing_enable(1 if on else 0)


def timing_reset():
    lib().ara_timing_reset()


def timing_read(kernel_class: int):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().ara_timing_read(int(kernel_class), ctypes.byref(ms), ctypes.byref(n)), "ara_timing_read")
    return ms.value, n.value
