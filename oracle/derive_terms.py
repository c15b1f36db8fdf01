"""Write the terms manifests of the synthetic workloads whose layer terms depend on the loss
model (run:  python -m oracle.derive_terms).  TEST INFRASTRUCTURE: it calls only this oracle
package and the input generator, and its output is an input file (terms), never an expected
value.

Rule (the tiny workload's percentile rule carried to paper scale, where the tiny workload's
absolute layer terms would saturate every trial):
every cover has retention R = P20 and limit amount L = P95, the 20th and 95th percentiles of
the losses it applies to:
  * per-ELT terms: percentiles of that ELT's losses (as in the tiny case);
  * layer occurrence terms: percentiles of the non-zero combined event loss s(e) (per-ELT
    terms applied, summed across the layer's ELTs) over the catalogue;
  * aggregate terms: percentiles of the trial aggregate loss (occurrence terms applied,
    summed over the trial) over the first 10,000 trials of the YET.
"""
from __future__ import annotations

import json
import os

import numpy as np

import oracle
import synth

INF = float("inf")


def layer_event_losses(pf, layer):
    """s(e) for every catalogue event under one layer: the oracle run on one-event trials with
    identity occurrence and aggregate terms."""
    one = synth.YET(np.arange(pf.catalogue + 1, dtype=np.int64),
                    np.arange(pf.catalogue, dtype=np.int32))
    p = pf.with_terms({**pf.terms_dict(), "occ_ret": [0.0] * pf.n_layers, "occ_lim": [INF] * pf.n_layers,
                       "agg_ret": [0.0] * pf.n_layers, "agg_lim": [INF] * pf.n_layers})
    return oracle.ylt(p, one)[layer]


def derive(pf, yet_head, lo=20.0, hi=95.0):
    t = pf.terms_dict()
    for l in range(pf.n_layers):
        s = layer_event_losses(pf, l)
        nz = s[s > 0]
        t["occ_ret"][l] = float(np.percentile(nz, lo))
        t["occ_lim"][l] = float(np.percentile(nz, hi))
    p = pf.with_terms({**t, "agg_ret": [0.0] * pf.n_layers, "agg_lim": [INF] * pf.n_layers})
    agg = oracle.ylt(p, yet_head)
    for l in range(pf.n_layers):
        t["agg_ret"][l] = float(np.percentile(agg[l], lo))
        t["agg_lim"][l] = float(np.percentile(agg[l], hi))
    return t


def blank(n):
    return {"occ_ret": [0.0] * n, "occ_lim": [0.0] * n, "agg_ret": [0.0] * n, "agg_lim": [0.0] * n}


def write(name, t):
    t["_rule"] = __doc__.split("Rule")[1].strip()
    out = os.path.join(synth.HERE, f"terms_{name}.json")
    with open(out, "w") as f:
        json.dump(t, f, indent=1)
    print("wrote", out)


def main_adjoint(seed=0):
    base = synth.adjoint_portfolio(seed, terms={"elt_ret": [0.0] * 240, "elt_lim": [0.0] * 240, **blank(16)})
    r, l = synth.percentile_terms(base.elt_losses)
    pf = base.with_terms({**base.terms_dict(), "elt_ret": r.tolist(), "elt_lim": l.tolist()})
    t = derive(pf, synth.adjoint_yet(seed, n_trials=5000))
    t["_seed"] = seed
    write("adjoint", t)


def main_batched(seed=0):
    base = synth.batched_portfolio(seed, terms={"elt_ret": [0.0] * 200, "elt_lim": [0.0] * 200, **blank(64)})
    r, l = synth.percentile_terms(base.elt_losses)
    pf = base.with_terms({**base.terms_dict(), "elt_ret": r.tolist(), "elt_lim": l.tolist()})
    t = derive(pf, synth.batched_yet(seed, n_trials=2000))
    f = synth.batched_term_factors(seed)
    for c, k in enumerate(["occ_ret", "occ_lim", "agg_ret", "agg_lim"]):
        t[k] = [float(v * f[i, c]) for i, v in enumerate(t[k])]
    t["_seed"] = seed
    t["_randomised"] = "each layer term multiplied by U(0.5, 1.5) (synth.batched_term_factors)"
    write("batched", t)


def main():
    seed = 0
    pf = synth.paper_scale_portfolio(seed, terms={"elt_ret": [0.0] * 15, "elt_lim": [0.0] * 15,
                                                  "occ_ret": [0.0], "occ_lim": [0.0],
                                                  "agg_ret": [0.0], "agg_lim": [0.0]})
    r, l = synth.percentile_terms(pf.elt_losses)
    pf = pf.with_terms({**pf.terms_dict(), "elt_ret": r.tolist(), "elt_lim": l.tolist()})
    head = synth.paper_scale_yet(seed, n_trials=10_000)
    t = derive(pf, head)
    t["_rule"] = __doc__.split("Rule")[1].strip()
    t["_seed"] = seed
    out = os.path.join(synth.HERE, "terms_paper_scale.json")
    with open(out, "w") as f:
        json.dump(t, f, indent=1)
    print("wrote", out, {k: t[k] for k in ["occ_ret", "occ_lim", "agg_ret", "agg_lim"]})


if __name__ == "__main__":
    import sys
    which = sys.argv[1:] or ["paper_scale", "adjoint", "batched"]
    if "paper_scale" in which:
        main()
    if "adjoint" in which:
        main_adjoint()
    if "batched" in which:
        main_batched()
