"""Host logic of the learned closure (no GPU).

closure.failed_checks decides when a corrected coarse run is handed to the fine solver: a healthy
state passes; each limit (non-finite nodes, phi range, max |u|, sum phi drift) fails on its own,
with a reason that names it; limits can be overridden one at a time.  closure.equal_accuracy prices
the plain grid of the corrected run's accuracy from two plain grids."""
from paper_2501_00846_b300 import closure


def _obs(**kw):
    o = {"n_nonfinite": 0.0, "phi_min": 0.0, "phi_max": 1.0, "umax": 0.03, "sum_phi": 1000.0}
    o.update(kw)
    return o


def test_healthy_state_passes():
    assert closure.failed_checks(_obs(), _obs()) == []
    # just inside every default limit
    lim = closure.DEFAULT_LIMITS
    inside = _obs(phi_min=lim["phi_min"], phi_max=lim["phi_max"], umax=lim["umax"],
                  sum_phi=1000.0 * (1 + 0.999 * lim["sum_phi_drift"]))
    assert closure.failed_checks(inside, _obs()) == []


def test_each_limit_fails_on_its_own():
    cases = {
        "non-finite": _obs(n_nonfinite=3.0),
        "phi in": _obs(phi_min=-0.2),
        "max |u|": _obs(umax=0.5),
        "sum phi drifted": _obs(sum_phi=1002.0),
    }
    for word, o in cases.items():
        bad = closure.failed_checks(o, _obs())
        assert len(bad) == 1 and word in bad[0], (word, bad)
    assert "phi in" in closure.failed_checks(_obs(phi_max=1.3), _obs())[0]
    # a non-finite state is reported as such, whatever the other fields hold
    assert len(closure.failed_checks(_obs(n_nonfinite=1.0, umax=float("nan")), _obs())) == 1


def test_limits_can_be_overridden():
    o = _obs(umax=0.25)
    assert closure.failed_checks(o, _obs())
    assert closure.failed_checks(o, _obs(), {"umax": 0.3}) == []
    assert closure.failed_checks(_obs(sum_phi=1002.0), _obs(), {"sum_phi_drift": 1e-2}) == []


def test_equal_accuracy_fit_recovers_power_laws():
    """closure.equal_accuracy on a ladder made from exact power laws: e(L) = 3 L^-2 and
    t(L) = 1e-6 L^4 (cost per unit physical time under acoustic scaling) recover p = 2 and q = 4, and
    a corrected run with the error of the plain 128^3 grid is priced at t(128)."""
    def plain(L):
        return {"phi_rms_mean": 3.0 * L ** -2.0, "ms_per_coarse_step": 1e-6 * L ** 4.0}
    ladder = {"runs": {"plain_64": plain(64), "plain_96": plain(96),
                       "closure_64": {"phi_rms_mean": 3.0 * 128 ** -2.0, "ms_per_coarse_step": 0.5}}}
    r = closure.equal_accuracy(ladder, coarse=64, finer=96)
    assert abs(r["error_exponent"] - 2.0) < 1e-12 and abs(r["cost_exponent"] - 4.0) < 1e-12
    assert abs(r["equal_accuracy_grid"] - 128.0) < 1e-9
    assert abs(r["plain_ms_at_equal_accuracy"] - 1e-6 * 128 ** 4) < 1e-9
    assert abs(r["speedup"] - 1e-6 * 128 ** 4 / 0.5) < 1e-9
