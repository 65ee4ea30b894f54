"""Host logic of the consensus-penalty balancing rule (no GPU needed)."""
from paper_2011_00162_gb300 import adaptive


def test_decide_balances_and_clamps():
    assert adaptive.decide(1.0, 1.0, 1.0) == 1.0          # balanced: unchanged
    assert adaptive.decide(1.0, 11.0, 1.0) == 2.0         # primal lags: raise r
    assert adaptive.decide(1.0, 1.0, 11.0) == 0.5         # dual lags: lower r
    assert adaptive.decide(1.0, 10.0, 1.0) == 1.0         # the ratio is strict
    assert adaptive.decide(3e3, 1e3, 1.0, r_max=4e3) == 4e3
    assert adaptive.decide(2e-4, 1.0, 1e3, r_min=1.5e-4) == 1.5e-4
    assert adaptive.decide(1.0, 5.0, 1.0, ratio=4.0, factor=3.0) == 3.0


class _FakePlan:
    """A stand-in for api.Plan that records the driver's calls."""

    def __init__(self, eta, r, eps=0.5, n_pairs=2):
        import types
        self.geom = types.SimpleNamespace(eta=eta, r=r, eps=eps)
        self.n_pairs = n_pairs
        self.calls = []


def _fake_api(monkeypatch, residuals):
    """Route adaptive's api calls to a script: residuals[i] = (rf, re, consensus, frame)."""
    from paper_2011_00162_gb300 import adaptive as ad
    state = {"check": 0}

    def iterate(plan, n):
        plan.calls.append(("iterate", n))

    def snapshot(plan):
        plan.calls.append(("snapshot",))

    def metrics(plan):
        return residuals[state["check"]][:2]

    def consensus(plan):
        return residuals[state["check"]][2]

    def frame(plan):
        v = residuals[state["check"]][3]
        state["check"] += 1
        return v

    def set_penalties(plan, eta, r):
        plan.calls.append(("set", eta, r))
        plan.geom.eta, plan.geom.r = eta, r

    monkeypatch.setattr(ad.api, "od2p_iterate", iterate)
    monkeypatch.setattr(ad.api, "od2p_gamma_snapshot", snapshot)
    monkeypatch.setattr(ad.api, "od2p_metrics", metrics)
    monkeypatch.setattr(ad.api, "od2p_consensus_residual", consensus)
    monkeypatch.setattr(ad.api, "od2p_frame_residual", frame)
    monkeypatch.setattr(ad.api, "od2p_set_penalties", set_penalties)


def test_balanced_eta_schedule(monkeypatch):
    """balance_eta: Gamma is kept right before each block's last iteration; eta
    rises when the frame residual dominates, falls when the dual one does, never
    to the prox continuity bound (1 - eps)/eps or below; the last block changes
    nothing."""
    _fake_api(monkeypatch, [
        (0.5, 0.01, 1e-3, 1.0),    # frame residual >> eta*RE: eta 2 -> 4; consensus balanced vs r*RE
        (0.4, 0.5, 1e-3, 1e-3),    # eta*RE >> frame residual: eta 4 -> 2; r*RE >> consensus: r 0.1 -> 0.05
        (0.3, 0.5, 1e-3, 1e-3),    # eta 2 -> 1.01 (the floor), r 0.05 -> 0.025
        (0.2, 0.5, 1e-3, 1e-3),    # last block: no change
    ])
    plan = _FakePlan(eta=2.0, r=0.1)
    hist = adaptive.iterate_balanced(plan, 40, every=10, balance_eta=True)
    assert [c for c in plan.calls if c[0] != "set"][:3] == [("iterate", 9), ("snapshot",), ("iterate", 1)]
    sets = [c for c in plan.calls if c[0] == "set"]
    assert sets == [("set", 4.0, 0.1), ("set", 2.0, 0.05), ("set", 1.01, 0.025)]
    assert [h["eta"] for h in hist] == [4.0, 2.0, 1.01, 1.01]
    assert hist[-1]["frame_residual"] == 1e-3


def test_balanced_r_only_takes_no_snapshot(monkeypatch):
    _fake_api(monkeypatch, [(0.5, 1.0, 1e-3, 0.0), (0.5, 1.0, 1e-3, 0.0)])
    plan = _FakePlan(eta=2.0, r=1.0)
    hist = adaptive.iterate_balanced(plan, 7, every=5)
    assert ("snapshot",) not in plan.calls
    assert [c for c in plan.calls if c[0] == "iterate"] == [("iterate", 5), ("iterate", 2)]
    assert hist[0]["r"] == 0.5 and hist[-1]["iterations"] == 7
