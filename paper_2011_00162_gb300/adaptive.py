"""Residual balancing of the consensus penalty r between ADMM iterations.

The paper runs OD2P with fixed (eta, r) and names their automatic choice
future work (section 4.3).  This module supplies the standard residual-balancing
rule for an ADMM penalty (He, Yang and Wang 2000; Boyd, Parikh, Chu, Peleato,
Eckstein 2011, section 3.4.1) for the consensus penalty r, and optionally for
the frame penalty eta (iterate_balanced(..., balance_eta=True)): every `every`
iterations it compares the primal residual of the consensus constraint -- the
relative disagreement of the subdomain copies on their overlaps,
od2p_consensus_residual -- with a dual residual, r times the relative change of
the iterate (the RE of section 4, from od2p_metrics).  If the primal residual
is more than `ratio` times the dual one, r is multiplied by `factor`; if the
dual one is more than `ratio` times the primal one, r is divided by it; the
change goes through od2p_set_penalties, which keeps the unscaled multipliers.

The module also gives the paper's own sufficient choice of (r, eta) inside the
parameter set K of Lemma 2.4 (eq. paramsSet, stated for two subdomains and
taken here over all subdomains and ordered overlap pairs), for which the
augmented Lagrangian does not increase: select_in_K reads the operator norms of
a nonblind plan from the library and params_in_K applies the lemma's bounds.

All arithmetic of the iteration runs in the library; this is a host control
loop over its entry points.
"""
from __future__ import annotations

from . import api


def params_in_K(norms: tuple[float, float], eps: float, margin: float = 1.01) -> tuple[float, float]:
    """(r, eta) inside K for operator norms (max ||A_d^* A_d||, max ||pi_{d,e} A_d^*||^2)
    and ST-AGM truncation eps, by the sufficient choice that follows eq. (paramsSet):
    eta > max(6L + 2L^2 + 2 (c1 / c0^2) (L + 1)^2, 1) and r > c0 eta, with
    L = 2/eps - 1 (Lemma 2.1), c0 = max(2 ||A^*A||, ||pi A^*||), c1 = 2 ||pi A^*||^2;
    each bound exceeded by the factor `margin` (> 1)."""
    if not margin > 1.0:
        raise ValueError("margin must exceed 1 (the bounds are strict)")
    if not 0.0 < eps < 1.0:
        raise ValueError("eps must lie in (0, 1)")
    a, b = float(norms[0]), float(norms[1])
    if not a > 0.0:
        raise ValueError("the illumination is zero")
    L = 2.0 / eps - 1.0
    c0 = max(2.0 * a, b ** 0.5)
    c1 = 2.0 * b
    eta = margin * max(6.0 * L + 2.0 * L * L + 2.0 * (c1 / c0 ** 2) * (L + 1.0) ** 2, 1.0)
    return margin * c0 * eta, eta


def in_K(r: float, eta: float, norms: tuple[float, float], eps: float) -> bool:
    """The three inequalities of eq. (paramsSet) for these operator norms."""
    a, b = float(norms[0]), float(norms[1])
    L = 2.0 / eps - 1.0
    c0 = max(2.0 * a, b ** 0.5)
    return (eta - 1.0 >= 0.0 and r - eta * c0 > 0.0
            and (eta - 3.0 * L) / 2.0 - L * L / eta - 2.0 * (L + eta) ** 2 / r ** 2 * b > 0.0)


def select_in_K(plan: api.Plan, margin: float = 1.01) -> tuple[float, float]:
    """params_in_K for a nonblind plan, its operator norms measured by the library."""
    return params_in_K(api.od2p_operator_norms(plan), float(plan.geom.eps), margin)


def decide(r: float, primal: float, dual: float, ratio: float = 10.0, factor: float = 2.0,
           r_min: float = 1e-4, r_max: float = 1e4) -> float:
    """The new consensus penalty for residuals (primal, dual) at penalty r."""
    if primal > ratio * dual:
        return min(r * factor, r_max)
    if dual > ratio * primal:
        return max(r / factor, r_min)
    return r


def iterate_balanced(plan: api.Plan, n_iter: int, every: int = 10, ratio: float = 10.0, factor: float = 2.0,
                     r_min: float = 1e-4, r_max: float = 1e4, balance_eta: bool = False,
                     eta_min: float | None = None, eta_max: float = 1e4) -> list[dict]:
    """Run n_iter iterations of plan, rebalancing r (and, with balance_eta, eta)
    every `every` iterations.

    r: primal = the consensus residual, dual = r * RE.  eta (balance_eta): primal
    = the frame constraint's relative residual ||Gamma^{n+1} - Gamma^n|| / ||sqrt f||
    of the block's last iteration (od2p_frame_residual), dual = eta * RE -- the
    same rule with the relative change of u standing in for the dual residual of
    either constraint.  eta stays above eta_min, by default 1.01 (1 - eps) / eps:
    at or below (1 - eps) / eps the ST-AGM prox of eq. (Prox_sol) jumps at y = 0
    (only its AGM branch is reachable), which makes runs sensitive to rounding.
    Returns one record per check: iterations done, RF, RE, the residuals and the
    penalties in force for the next block.
    """
    if every < 1:
        raise ValueError("every must be >= 1")
    eta, r = float(plan.geom.eta), float(plan.geom.r)
    if eta_min is None:
        eps = float(plan.geom.eps)
        eta_min = 1.01 * (1.0 - eps) / eps
    history, done = [], 0
    while done < n_iter:
        k = min(every, n_iter - done)
        if balance_eta:
            if k > 1:
                api.od2p_iterate(plan, k - 1)
            api.od2p_gamma_snapshot(plan)
            api.od2p_iterate(plan, 1)
        else:
            api.od2p_iterate(plan, k)
        done += k
        rf, re = api.od2p_metrics(plan)
        rc = api.od2p_consensus_residual(plan)
        rec = {"iterations": done, "rf": rf, "re": re, "consensus": rc}
        r_new = decide(r, rc, r * re, ratio, factor, r_min, r_max) if plan.n_pairs else r
        eta_new = eta
        if balance_eta:
            fr = api.od2p_frame_residual(plan)
            rec["frame_residual"] = fr
            eta_new = decide(eta, fr, eta * re, ratio, factor, eta_min, eta_max)
        if (r_new != r or eta_new != eta) and done < n_iter:
            api.od2p_set_penalties(plan, eta_new, r_new)
            eta, r = eta_new, r_new
        rec["r"], rec["eta"] = r, eta
        history.append(rec)
    return history
