"""Pins of the oracle's late-time profiles (Sec. 3 averaged potential and
species densities) and of its Eq. 9-10 post-processing.  CPU only."""
import math

import numpy as np

from conftest import load_golden
from paper_2605_07083_gb300 import workloads as W
from parity_util import mixed_state

QE, EPS0, KB = 1.602176634e-19, 8.8541878128e-12, 1.380649e-23


def _golden():
    return {r[0]: tuple(float(x) for x in r[1:]) for r in load_golden("eq9_10_virtual_cathode.txt")}


def test_eq10_and_eq9_reproduce_the_printed_example(oracle_mod):
    g = _golden()
    T = g["T_emit_eV"][0]
    ratio, phi_printed, tol = g["phi_vc_eff"]
    phi_min, eta_printed, tol9 = g["eta_vc"]
    # a profile whose near-cathode minimum is the printed -2.2e-3 V
    Nz, L = 400, 0.1
    z = np.arange(Nz + 1) * (L / Nz)
    phi = 40.0 * (z / L) ** 3
    phi[3] = phi_min
    vc = oracle_mod.virtual_cathode(phi, L, T, ratio, near_fraction=0.05)
    assert abs(vc["phi_vc_eff"] - phi_printed) <= tol
    assert abs(vc["eta_vc"] - eta_printed) <= tol9
    assert vc["phi_min"] == phi_min and math.isclose(vc["z_min"], 3 * L / Nz, rel_tol=1e-15)
    # Eq. 9 inverts Eq. 10: the barrier of the mapped efficiency transmits it
    assert math.isclose(math.exp(vc["phi_vc_eff"] / T), ratio, rel_tol=1e-14)
    # a potential that never dips has its minimum at the wall, phi_w = 0
    vc0 = oracle_mod.virtual_cathode(40.0 * z / L, L, T, 1.0)
    assert vc0["phi_min"] == 0.0 and vc0["z_min"] == 0.0 and vc0["eta_vc"] == 1.0
    assert vc0["phi_vc_eff"] == 0.0
    assert math.isnan(oracle_mod.virtual_cathode(phi, L, T, 0.0)["phi_vc_eff"])
    # the region bound: a deeper dip beyond near_fraction*L is not the near-cathode minimum
    phi2 = phi.copy()
    phi2[200] = -1.0
    assert oracle_mod.virtual_cathode(phi2, L, T, ratio, near_fraction=0.05)["phi_min"] == phi_min
    assert oracle_mod.virtual_cathode(phi2, L, T, ratio, near_fraction=0.5)["phi_min"] == -1.0


def _quiet(**kw):
    p = W.single_diode_small(seed=5)
    p.update(n_gas=0.0, gamma_emit=0.0, replenish=0, window_start=0)
    p.update(kw)
    return p


def test_vacuum_profile_is_the_linear_potential(oracle_mod):
    p = _quiet(V=7.0, window_start=2)
    o = oracle_mod.Oracle(p)
    o.set_profile_period(3)
    o.step(12)                      # samples after steps 2, 5, 8, 11
    phi_sum, counts, k = o.profiles()
    assert k == 4
    z = np.arange(p["Nz"] + 1) * (p["L"] / p["Nz"])
    phi, dens = oracle_mod.profile_averages(phi_sum, counts, k, p["weight"], p["L"], p["Nz"])
    np.testing.assert_allclose(phi, p["V"] * z / p["L"], rtol=0, atol=1e-12 * p["V"])
    assert not counts.any() and not dens.any()


def test_frozen_lattice_density_is_the_closed_form(oracle_mod):
    """m electrons and m ions at rest on every cell centre: the net charge is
    zero, so with V = 0 nothing moves; each interior node then holds m
    particles' worth from its two half cells (2^24 m units), each electrode
    node half that, and the density is m w / dz everywhere."""
    p = _quiet(V=0.0, window_start=1)
    Nz, L, m = p["Nz"], p["L"], 3
    zc = ((np.arange(Nz) + 0.5) * (L / Nz)).astype(np.float32)
    z = np.repeat(zc, m)
    zero = np.zeros_like(z)
    o = oracle_mod.Oracle(p)
    o.inject(1, z, zero, zero, zero)
    o.inject(2, z, zero, zero, zero)
    o.set_profile_period(2)
    o.step(6)                       # samples after steps 1, 3, 5
    phi_sum, counts, k = o.profiles()
    assert k == 3
    np.testing.assert_array_equal(o.state(1)["z"], z.astype(np.float64))
    # the cell centres are exact in FP32 only up to rounding of z*Nz/L: use
    # the rule's own Q = trunc(f 2^24) total, which must still sum to 2^24 m
    # per cell -- and with f = 1/2 exactly where z*Nz/L is a half-integer
    interior = counts[1, 1:-1]
    assert counts[1].sum() == k * m * Nz * (1 << 24)
    assert np.array_equal(counts[1], counts[2]) and not counts[0].any()
    s = (zc * np.float32(Nz / L)).astype(np.float32)
    exact = s == np.floor(s) + np.float32(0.5)
    assert exact.mean() > 0.5
    half = (1 << 23) * m * k
    for j in np.nonzero(exact[1:] & exact[:-1])[0] + 1:
        assert interior[j - 1] == 2 * half
    phi, dens = oracle_mod.profile_averages(phi_sum, counts, k, p["weight"], L, Nz)
    ok = np.zeros(Nz + 1, bool)
    ok[1:-1] = exact[1:] & exact[:-1]
    ok[0], ok[-1] = exact[0], exact[-1]
    np.testing.assert_allclose(dens[1][ok], m * p["weight"] / (L / Nz), rtol=1e-14)
    assert not phi.any()


def test_live_run_profiles_are_consistent_samples(oracle_mod):
    """A collisional run with emission: the sums are samples of the states
    after the sampled steps (charge totals match the live counts at those
    steps), and the averaged potential is the Poisson solution of the averaged
    charge (Poisson is linear), which ties the two accumulators to the same
    states."""
    p = W.single_diode_small(seed=3)
    p.update(window_start=4, n_gas=3e22)
    st = mixed_state(p, 8, 600, 300)
    o = oracle_mod.Oracle(p)
    for sp in (0, 1, 2):
        o.inject(sp, *st[sp])
    period, n_steps = 3, 17
    o.set_profile_period(period)
    live = np.zeros(3, np.int64)
    for n in range(n_steps):
        o.step(1)
        if n >= p["window_start"] and (n - p["window_start"]) % period == 0:
            live += [o.count(s) for s in range(3)]
    phi_sum, counts, k = o.profiles()
    assert k == len(range(p["window_start"], n_steps, period)) == 5
    np.testing.assert_array_equal(counts.sum(axis=1), live * (1 << 24))
    Nz, L = p["Nz"], p["L"]
    dz = L / Nz
    rho_fix = (counts[2] - counts[0] - counts[1]).astype(np.float64) / k
    rhs = dz * dz * rho_fix * QE * p["weight"] / (16777216.0 * dz) / EPS0
    rhs[0] = rhs[-1] = 0.0
    phi_of_mean = oracle_mod.thomas(Nz, p["V"], rhs)
    np.testing.assert_allclose(phi_sum / k, phi_of_mean, rtol=0, atol=1e-11 * p["V"])
    # densities integrate to the mean live count times the weight
    _, dens = oracle_mod.profile_averages(phi_sum, counts, k, p["weight"], L, Nz)
    vol = np.full(Nz + 1, dz)
    vol[0] = vol[-1] = dz / 2
    np.testing.assert_allclose((dens * vol).sum(axis=1), live / k * p["weight"], rtol=1e-12)
    # re-arming clears the sums
    o.set_profile_period(period)
    assert o.profiles()[2] == 0 and not o.profiles()[1].any()
