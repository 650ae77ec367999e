"""Host logic of the transition searches, with the PIC runs replaced by a
known backflow curve per setting (no GPU)."""
import numpy as np
import pytest

from paper_2605_07083_gb300 import surrogate as S


def _fake(crossing, width=0.08e19):
    """backflow(setting i, flux g) = logistic((g - crossing_i) / width)."""
    def ev(settings, gammas, cost, **kw):
        cost["runs"] += len(gammas)
        cost["rounds"] += 1
        cost["gpu_ms"] += 1.0
        cost["particle_steps"] += len(gammas)
        return np.array([1.0 / (1.0 + np.exp(-(g - crossing[s["i"]]) / width))
                         for s, g in zip(settings, gammas)])
    return ev


@pytest.fixture
def world(monkeypatch):
    rng = np.random.default_rng(3)
    n = 40
    crossing = rng.uniform(4.0e19, 10.0e19, n)          # some outside [5, 9]e19
    settings = [{"i": i} for i in range(n)]
    monkeypatch.setattr(S, "_eval", _fake(crossing))
    return settings, crossing


def _inside(crossing):
    return (crossing > S.LO + S.TOL) & (crossing < S.HI - S.TOL)


def test_bisection_and_ksection_find_the_crossing(world):
    settings, crossing = world
    n = len(settings)
    for fn, max_rounds in ((S._bisect, 6), (S._ksect, 3)):
        a, b = np.full(n, S.LO), np.full(n, S.HI)
        est = np.full(n, np.nan)
        open_ = _inside(crossing).copy()
        cost = {"gpu_ms": 0.0, "particle_steps": 0, "runs": 0, "rounds": 0}
        fn(settings, a, b, open_, est, cost)
        ok = _inside(crossing)
        assert np.all(np.abs(est[ok] - crossing[ok]) <= 2 * S.TOL)
        assert not open_.any()
        assert cost["rounds"] <= max_rounds     # 4e19 / 2^6 and 4e19 / 4^3 < 2 x 0.05e19


def test_plain_search_classifies_every_setting(world):
    settings, crossing = world
    est, _ = S.plain_search(settings)
    ok = _inside(crossing)
    assert np.all(np.abs(est[ok] - crossing[ok]) <= 2 * S.TOL)
    out = ~ok
    assert np.all(np.isnan(est[out]) | (np.abs(est[out] - crossing[out]) <= 2 * S.TOL))


@pytest.mark.parametrize("bias", [0.0, 0.6e19])
def test_guided_search_agrees_with_plain_whether_or_not_the_surrogate_is_right(world, monkeypatch,
                                                                                bias):
    settings, crossing = world
    grid = np.linspace(S.LO, S.HI, 161)

    def fake_crossing(model, sets, n_grid=161):
        bf = np.array([1.0 / (1.0 + np.exp(-(grid - crossing[s["i"]] - bias) / 0.08e19))
                       for s in sets])
        est = np.full(len(sets), np.nan)
        for i in range(len(sets)):
            up = np.nonzero((bf[i, :-1] < 0.5) & (bf[i, 1:] >= 0.5))[0]
            if up.size:
                k = up[0]
                f = (0.5 - bf[i, k]) / (bf[i, k + 1] - bf[i, k])
                est[i] = grid[k] + f * (grid[k + 1] - grid[k])
        return est, bf, grid

    monkeypatch.setattr(S, "surrogate_crossing", fake_crossing)
    est_p, cost_p = S.plain_search(settings)
    est_g, cost_g = S.guided_search(None, settings, max_err=0.02)
    same = np.isnan(est_p) == np.isnan(est_g)
    assert same.mean() >= 0.9
    both = ~np.isnan(est_p) & ~np.isnan(est_g)
    assert np.all(np.abs(est_p[both] - est_g[both]) <= 4 * S.TOL)
    if bias == 0.0:
        # a right surrogate settles nearly everything in its first round
        assert cost_g["runs"] < cost_p["runs"] and cost_g["rounds"] < cost_p["rounds"]
