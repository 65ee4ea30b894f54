"""Residual balancing of the consensus penalty r between ADMM iterations.

The paper runs OD2P with fixed (eta, r) and names their automatic choice
future work (section 4.3).  This module supplies the standard residual-balancing
rule for an ADMM penalty (He, Yang and Wang 2000; Boyd, Parikh, Chu, Peleato,
Eckstein 2011, section 3.4.1) for the consensus penalty r: every `every`
iterations it compares the primal residual of the consensus constraint -- the
relative disagreement of the subdomain copies on their overlaps,
od2p_consensus_residual -- with a dual residual, r times the relative change of
the iterate (the RE of section 4, from od2p_metrics).  If the primal residual
is more than `ratio` times the dual one, r is multiplied by `factor`; if the
dual one is more than `ratio` times the primal one, r is divided by it; the
change goes through od2p_set_penalties, which keeps the unscaled multipliers.

All arithmetic of the iteration runs in the library; this is a host control
loop over its entry points.
"""
from __future__ import annotations

from . import api


def decide(r: float, primal: float, dual: float, ratio: float = 10.0, factor: float = 2.0,
           r_min: float = 1e-4, r_max: float = 1e4) -> float:
    """The new consensus penalty for residuals (primal, dual) at penalty r."""
    if primal > ratio * dual:
        return min(r * factor, r_max)
    if dual > ratio * primal:
        return max(r / factor, r_min)
    return r


def iterate_balanced(plan: api.Plan, n_iter: int, every: int = 10, ratio: float = 10.0, factor: float = 2.0,
                     r_min: float = 1e-4, r_max: float = 1e4) -> list[dict]:
    """Run n_iter iterations of plan, rebalancing r every `every` iterations.

    Returns one record per check: iterations done, RF, RE, consensus residual
    and the penalty r in force for the next block of iterations.
    """
    if every < 1:
        raise ValueError("every must be >= 1")
    eta, r = float(plan.geom.eta), float(plan.geom.r)
    history, done = [], 0
    while done < n_iter:
        k = min(every, n_iter - done)
        api.od2p_iterate(plan, k)
        done += k
        rf, re = api.od2p_metrics(plan)
        rc = api.od2p_consensus_residual(plan)
        r_new = decide(r, rc, r * re, ratio, factor, r_min, r_max) if plan.n_pairs else r
        if r_new != r and done < n_iter:
            api.od2p_set_penalties(plan, eta, r_new)
            r = r_new
        history.append({"iterations": done, "rf": rf, "re": re, "consensus": rc, "r": r})
    return history
