"""CPU checks of the warm-up tuner's host logic (paper_2204_14241_gb300/tuning.py) with a stand-in
for the library's trajectory: acceptance from dH, the Eq. (acc_ineq) step-size walk, the back-off
to a stable production-length trajectory, and the Eq. (ESJD) choice of n_max."""

import math

import pytest

from paper_2204_14241_gb300.tuning import Tuner


class FakeCtx:
    """trajectory() with dH, status and the proposal's jump from closed forms of (eps, n_leap)."""

    def __init__(self, dH, status=lambda eps, n: 0, jump2=lambda eps, n: 1.0):
        self.dH, self.status, self.jump2 = dH, status, jump2
        self.calls = []

    def trajectory(self, phis, sigmas, eps, n_leap, **kw):
        self.calls.append((eps, n_leap, kw.get("counter")))
        st = self.status(eps, n_leap)
        dH = self.dH(eps, n_leap) if st == 0 else float("nan")
        return {"dH": [dH], "status": st, "accepted": [st == 0 and dH <= 0.0], "jump2": [self.jump2(eps, n_leap)]}


def tuner(ctx):
    return Tuner(ctx, phi=None, sigma=None)


def test_acceptance_from_dH_and_failures():
    ctx = FakeCtx(dH=lambda eps, n: {1: -0.3, 2: 0.7}[n], status=lambda eps, n: 2 if n == 3 else 0)
    t = tuner(ctx)
    assert t.propose(0.1, 1)[0] == 1.0                          # dH <= 0
    assert t.propose(0.1, 2)[0] == pytest.approx(math.exp(-0.7))
    a, _, dH, acc = t.propose(0.1, 3)                           # a failed update counts as alpha = 0
    assert a == 0.0 and math.isnan(dH) and not acc
    assert [c[2] for c in ctx.calls] == [0, 1, 2]               # Philox counter = proposal index
    assert len(t.log) == 3


@pytest.mark.parametrize("eps0", [0.01, 2.0])
def test_step_size_walk_settles_at_the_inequality_boundary(eps0):
    # single-step acceptance alpha(eps) = exp(-k eps^2): alpha(eps/2)^2 <= 2 alpha(eps) holds
    # exactly for eps^2 <= 2 ln 2 / k, so the walk settles within one factor `grow` of that step
    k, grow = 4.0, 1.2
    ctx = FakeCtx(dH=lambda eps, n: k * eps * eps)
    eps, hist = tuner(ctx).tune_eps(eps0, rounds=60, window=1, grow=grow, stop_after_turns=3)
    star = math.sqrt(2 * math.log(2) / k)
    assert star / grow <= eps <= star * grow
    # the walk moved towards the boundary from either side
    first = hist[0][0]
    assert (hist[1][0] > first) == (first < star)


def test_step_size_shrinks_when_every_proposal_fails():
    ctx = FakeCtx(dH=lambda eps, n: 0.0, status=lambda eps, n: 2)
    eps, hist = tuner(ctx).tune_eps(1.0, rounds=5, window=2, grow=2.0)
    assert eps == pytest.approx(1.0 / 2 ** 5)
    assert all(a1 == 0.0 and a2 == 0.0 for _, a1, a2 in hist)


def test_back_off_to_a_stable_trajectory():
    # a 40-step trajectory is unstable above eps = 0.1 (solver failure) and has |dH| > 1 up to 0.06
    def status(eps, n):
        return 2 if eps > 0.1 else 0

    def dH(eps, n):
        return -5.0 if eps > 0.06 else 0.3

    eps, tries = tuner(FakeCtx(dH, status)).stabilize_eps(0.384, 40, max_tries=8, shrink=1.5)
    assert eps <= 0.06 and eps * 1.5 > 0.06
    assert [ok for _, _, ok in tries] == [False] * (len(tries) - 1) + [True]
    assert tries[0][0] == pytest.approx(0.384)


def test_back_off_gives_up_after_max_tries():
    eps, tries = tuner(FakeCtx(lambda eps, n: 0.0, lambda eps, n: 2)).stabilize_eps(1.0, 40, max_tries=3,
                                                                                   shrink=2.0)
    assert len(tries) == 3 and not any(ok for _, _, ok in tries)
    assert eps == pytest.approx(1.0 / 8)


def test_n_max_maximises_the_expected_squared_jump():
    # harmonic mode of frequency w: jump^2 = 2 (1 - cos(n eps w)), all proposals accepted
    eps, w = 0.1, 2.0
    ctx = FakeCtx(dH=lambda e, n: 0.0, jump2=lambda e, n: 2.0 * (1.0 - math.cos(n * e * w)))
    n_max, esjd = tuner(ctx).tune_nmax(eps, candidates=list(range(1, 31)), per_candidate=2)
    assert n_max == round(math.pi / (eps * w))
    assert esjd[n_max] == pytest.approx(4.0, rel=1e-3)
