"""Host-side checks of the seeded workload recipes (no GPU)."""
import math

import numpy as np

from paper_2605_07083_gb300 import workloads as W


def test_flux_scan_is_the_paper_diode_at_table2_fluxes():
    ps = W.paper_flux_scan(ppc=1000, n_steps=4_500_000)
    assert [round(p["gamma_emit"] / 1e19, 2) for p in ps] == list(W.TABLE2_FLUXES)
    for p in ps:
        # Sec. 2.1: dt = 0.2 dz / v_te = 6.722e-12 s, w0 = n0 dz / 1000 = 1.2207e7 m^-2
        assert math.isclose(p["dt"], 6.722e-12, rel_tol=2e-4)
        assert math.isclose(p["weight"], 1.2207e7, rel_tol=1e-4)
        assert p["window_start"] == 3_000_000 and p["replenish"] == 1
        assert p["V"] == 40.0 and p["Nz"] == 4096 and p["L"] == 0.10
        assert p["sigma_exc0"] == 0.0 and p["lotz_a"] == 0.0          # elastic + CX only
        assert p["T_gas_e_K"] == 300.0 and p["T_gas_i_K"] == 1740.0
    assert len({p["seed"] for p in ps}) == len(ps)
    # fewer particles per cell -> proportionally heavier macro-particles
    q = W.paper_flux_scan(ppc=250)[0]
    assert math.isclose(q["weight"], 4 * ps[0]["weight"], rel_tol=1e-12)


def test_table3_cases_switch_one_thing_each():
    base = W.paper_flux_scan((1.0,), ppc=250)[0]
    cs = {c["label"]: c for c in W.paper_table3_cases(ppc=250)}
    assert len(cs) == 8
    for k in ("1 exc", "2 exc", "3 exc", "4 exc", "5 exc"):
        assert cs[k]["sigma_exc0"] > 0 and cs[k]["sigma_cx_i"] == base["sigma_cx_i"]
    assert cs["6 Tne=1740K"]["T_gas_e_K"] == 1740.0 and cs["6 Tne=1740K"]["sigma_exc0"] == 0
    assert cs["7 CX off"]["sigma_cx_i"] == 0.0
    assert cs["8 2x ppc"]["ppc"] == 500 and math.isclose(cs["8 2x ppc"]["weight"],
                                                         base["weight"] / 2, rel_tol=1e-12)
    assert [c["gamma_emit"] / 1e19 for c in cs.values()] == [1.5, 4.5, 5.0, 8.0, 10.0, 7.0,
                                                            10.0, 10.0]


def test_initial_plasma_is_uniform_and_maxwellian():
    p = W.paper_flux_scan(ppc=8)[0]
    st = W.paper_initial_plasma(p, seed=3)
    n = 8 * p["Nz"]
    assert st[0][0].size == 0 and st[1][0].size == n and st[2][0].size == n
    for sp, T, m in ((1, p["T_e0_eV"], W.M_E), (2, p["T_i0_eV"], p["m_ion"])):
        z, vx, vy, vz = st[sp]
        assert z.dtype == np.float32 and z.min() >= 0 and z.max() < np.float32(p["L"])
        assert abs(z.mean() / p["L"] - 0.5) < 0.01
        s = math.sqrt(W.E_CHARGE * T / m)
        for v in (vx, vy, vz):
            assert abs(v.std() / s - 1) < 0.02 and abs(v.mean()) < 0.02 * s


def test_window_stationarity_check():
    """Block means that scatter around one value are stationary; a drift of
    many standard errors between the halves is not; too few blocks give no
    verdict."""
    from paper_2605_07083_gb300.flux_scan import stationarity
    rng = np.random.default_rng(5)
    flat = 0.47 + 0.005 * rng.standard_normal(12)
    assert stationarity(flat)["stationary"] is True
    drift = 0.40 + 0.01 * np.arange(12) + 0.002 * rng.standard_normal(12)
    r = stationarity(drift)
    assert r["stationary"] is False and r["difference"] > r["two_sigma"]
    assert stationarity([0.5, 0.5, 0.5])["stationary"] is None
    assert stationarity([0.4, float("nan"), 0.41, 0.4, 0.42])["blocks"] == 4


def test_setting_diode_step_count_rules():
    """A surrogate setting runs five vacuum transits, at least min_steps, or
    exactly n_steps; the window is the last 40 % of the run."""
    s = {"gamma_emit": 7e19, "T_wall_K": 2500.0, "log10_n_gas": 21.5, "gap_m": 3e-3,
         "bias_V": 10.0}
    base = W.setting_diode(s, cell_m=2.5e-6)
    assert base["n_steps"] == math.ceil(5.0 * W.vacuum_transit_time(3e-3, 10.0) / base["dt"])
    assert W.setting_diode(s, cell_m=2.5e-6, min_steps=10 * base["n_steps"])["n_steps"] == \
        10 * base["n_steps"]
    fixed = W.setting_diode(s, cell_m=2.5e-6, n_steps=20000, min_steps=10 ** 9)
    assert fixed["n_steps"] == 20000 and fixed["window_start"] == 12000
    # children's capacity grows with the electrons in flight
    big = W.setting_diode(s, n_flight=4e6)
    assert big["capacity"][1] >= 8e6 and big["capacity"][2] >= 8e6


def test_flight_counts_are_log_uniform_in_range():
    n = W.flight_counts(20000, 3)
    assert n.min() >= 5e4 and n.max() <= 4e6
    u = (np.log10(n) - np.log10(5e4)) / (np.log10(4e6) - np.log10(5e4))
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.003
    assert np.array_equal(n, W.flight_counts(20000, 3))
