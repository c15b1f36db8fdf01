"""torch.autograd.Function around the library's forward (YLT, mean year loss, TVaR) and its
hand-written adjoint kernels: gradients of each layer's mean year loss and TVaR w.r.t. every
retention and limit (per-ELT terms and layer terms of Section IV-B) and every ELT loss.

    risk = LayerRisk.apply(elt_ret, elt_lim, occ_ret, occ_lim, agg_ret, agg_lim, losses,
                           tables, offsets, event_ids, tvar_level)
    # risk: [n_layers, 2] = (mean year loss, TVaR) per layer; risk.backward(...) fills .grad

`tables` carries the fixed structure (catalogue, per-ELT event IDs, layer composition, FP32
storage flag); `losses` is the flat vector of every ELT's losses in ELT order.  The forward
builds a device portfolio from the current parameter values, runs ara_run_ylt (recording the
aggregate regimes) and ara_risk_metrics; backward calls ara_adjoint_accumulate with the
upstream gradient as weights.  All arithmetic runs in libara's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Portfolio, risk_metrics


class LayerRisk(torch.autograd.Function):
    @staticmethod
    def forward(ctx, elt_ret, elt_lim, occ_ret, occ_lim, agg_ret, agg_lim, losses, tables,
                offsets, event_ids, tvar_level):
        h = lambda t: t.detach().cpu().numpy().astype(np.float64)
        flat = h(losses)
        split = np.cumsum([len(x) for x in tables.elt_ids])[:-1]
        pf = Portfolio(tables.catalogue, tables.elt_ids, np.split(flat, split), h(elt_ret), h(elt_lim),
                       tables.layer_elts, h(occ_ret), h(occ_lim), h(agg_ret), h(agg_lim),
                       losses_f32=bool(getattr(tables, "losses_f32", False)))
        n_trials = offsets.numel() - 1
        reg = torch.empty((pf.n_layers, n_trials), dtype=torch.uint8, device=offsets.device)
        ylt = pf.run_ylt(offsets, event_ids, regimes=reg)
        pf.check()
        _, tvar, mean = risk_metrics(ylt, [], [tvar_level], want_mean=True)
        ctx.pf, ctx.level = pf, float(tvar_level)
        ctx.save_for_backward(offsets, event_ids, ylt, reg)
        ctx.shapes = (elt_ret.shape, elt_lim.shape, occ_ret.shape, losses.shape)
        out = np.stack([mean, tvar[:, 0]], axis=1)
        return torch.from_numpy(out).to(device=elt_ret.device)

    @staticmethod
    def backward(ctx, grad_out):
        offsets, event_ids, ylt, reg = ctx.saved_tensors
        pf = ctx.pf
        w = grad_out.detach().double().cpu().numpy()
        g = pf.adjoint_accumulate(offsets, event_ids, ylt, reg, w, ctx.level)
        dev = grad_out.device
        n_e, n_l = pf.n_elts, pf.n_layers
        lay = g["layer"][:n_l]
        grads = (g["elt_ret"][:n_e], g["elt_lim"][:n_e], lay[:, 0], lay[:, 1], lay[:, 2], lay[:, 3],
                 g["loss"][:pf.n_records])
        grads = tuple(x.to(dev) for x in grads)
        return grads + (None, None, None, None)
