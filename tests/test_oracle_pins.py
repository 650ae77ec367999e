"""Pins of the CPU oracle against facts fixed outside it (closed forms, the
paper's printed tables, invariants, textbook limits).  CPU only."""
import math

import numpy as np
import pytest
from scipy import stats

from conftest import load_golden
from paper_2605_07083_gb300 import workloads as W

QE, ME, EPS0, KB = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12, 1.380649e-23


def quiet(p, **kw):
    """Collisionless, emission-free, space-charge-free variant of a diode."""
    q = dict(p)
    q.update(n_gas=0.0, gamma_emit=0.0, weight=1e-12, replenish=0)
    q.update(kw)
    return q


# ---------------------------------------------------------------- Philox
def test_philox_uniform_and_bijective(oracle_mod):
    O = oracle_mod
    key = np.array([0x12345678, 0x9ABCDEF0], np.uint32)
    words = np.array([O.philox4x32_10([i, 7, 0, 1], key) for i in range(1 << 13)])
    # distinct counters -> distinct 128-bit outputs (a keyed bijection)
    assert len({tuple(r) for r in words}) == words.shape[0]
    for w in range(4):
        hist = np.bincount(words[:, w] >> 24, minlength=256)
        assert stats.chisquare(hist).pvalue > 1e-4
    # one-bit counter change flips about half of the 128 output bits
    base = O.philox4x32_10([5, 7, 0, 1], key)
    flips = []
    for bit in range(32):
        o = O.philox4x32_10([5 ^ (1 << bit), 7, 0, 1], key)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, o)))
    assert 56 <= np.mean(flips) <= 72
    # key changes the stream
    assert not np.array_equal(base, O.philox4x32_10([5, 7, 0, 1], key ^ np.uint32(1)))


def test_philox2x32_uniform_and_bijective(oracle_mod):
    O = oracle_mod
    key = 0x2468ACE1
    # for a fixed key the 10-round map of the 64-bit counter is a bijection:
    # distinct counters never collide on the full output, and word 0 alone
    # spreads uniformly
    w = np.array([O.philox2x32_10_w0(i, 7, key) for i in range(1 << 14)], np.uint64)
    assert np.unique(w).size > (1 << 14) - 4           # 32-bit birthday collisions only
    hist = np.bincount((w >> np.uint64(24)).astype(np.int64), minlength=256)
    assert stats.chisquare(hist).pvalue > 1e-4
    # the fraction below a threshold is the threshold (the candidate test)
    t = 1 << 30
    frac = (w < t).mean()
    assert abs(frac - 0.25) < 4 * math.sqrt(0.25 * 0.75 / w.size)
    flips = [bin(O.philox2x32_10_w0(5, 7, key) ^ O.philox2x32_10_w0(5 ^ (1 << b), 7, key)).count("1")
             for b in range(32)]
    assert 12 <= np.mean(flips) <= 20
    assert O.philox2x32_10_w0(5, 7, key) != O.philox2x32_10_w0(5, 8, key)


# ---------------------------------------------------------------- Poisson
def test_thomas_uniform_charge_is_exact_quadratic(oracle_mod):
    """-phi'' = rho/eps0 with constant rho: the 3-point Laplacian is exact for
    the quadratic V z/L + rho z (L - z) / (2 eps0)."""
    Nz, L, V, rho = 200, 2e-3, 7.5, 3.0e-4
    dz = L / Nz
    rhs = np.full(Nz + 1, dz * dz * rho / EPS0)
    phi = oracle_mod.thomas(Nz, V, rhs)
    z = np.arange(Nz + 1) * dz
    exact = V * z / L + rho * z * (L - z) / (2 * EPS0)
    np.testing.assert_allclose(phi, exact, rtol=1e-11, atol=1e-12 * abs(exact).max())


def test_thomas_residual_random(oracle_mod):
    rng = np.random.default_rng(0)
    Nz, V = 513, -3.0
    rhs = rng.standard_normal(Nz + 1)
    phi = oracle_mod.thomas(Nz, V, rhs)
    assert phi[0] == 0.0 and phi[Nz] == V
    res = -phi[:-2] + 2 * phi[1:-1] - phi[2:] - rhs[1:-1]
    assert np.abs(res).max() < 1e-9 * np.abs(phi).max()


def test_field_of_uniform_fixed_point_charge(oracle_mod):
    """Ions exactly on every interior node (power-of-two grid, f = 0) give a
    uniform rho; phi must be the exact quadratic and E its derivative."""
    Nz, L, V, k = 64, 2.0 ** -10, 4.0, 3
    dz = L / Nz
    p = quiet(W.single_diode_small(), L=L, Nz=Nz, V=V, weight=2.0e9)
    o = oracle_mod.Oracle(p)
    z = np.repeat(np.arange(1, Nz) * dz, k).astype(np.float32)
    zero = np.zeros_like(z)
    o.inject(2, z, zero, zero, zero)
    rho_fix = o.rho_fixed()
    assert np.all(rho_fix[1:-1] == k * (1 << 24)) and rho_fix[0] == 0 and rho_fix[-1] == 0
    rho_si = k * QE * p["weight"] / dz
    phi, E = o.field()
    zz = np.arange(Nz + 1) * dz
    exact = V * zz / L + rho_si * zz * (L - zz) / (2 * EPS0)
    np.testing.assert_allclose(phi, exact, rtol=1e-11, atol=1e-11 * abs(exact).max())
    dphi = V / L + rho_si * (L - 2 * zz) / (2 * EPS0)
    # central differences are exact for a quadratic inside
    np.testing.assert_allclose(E[1:-1], -dphi[1:-1], rtol=1e-9, atol=1e-9 * abs(dphi).max())


def test_vacuum_field_is_uniform(oracle_mod):
    p = quiet(W.single_diode_small())
    phi, E = oracle_mod.Oracle(p).field()
    np.testing.assert_allclose(E, -p["V"] / p["L"], rtol=1e-12)
    np.testing.assert_allclose(phi, p["V"] * np.arange(p["Nz"] + 1) / p["Nz"], rtol=1e-12,
                               atol=1e-14)


# ---------------------------------------------------------------- deposit
def test_deposit_charge_sum_and_centroid(oracle_mod):
    p = W.single_diode_small()
    rng = np.random.default_rng(1)
    o = oracle_mod.Oracle(p)
    ne, ni = 3001, 1777
    ze = W.clamp_inside(rng.random(ne) * p["L"], p["L"])
    zi = W.clamp_inside(rng.random(ni) * p["L"], p["L"])
    o.inject(1, ze, *(np.zeros(ne, np.float32),) * 3)
    o.inject(2, zi, *(np.zeros(ni, np.float32),) * 3)
    rho = o.rho_fixed()
    assert rho.sum() == (ni - ne) * (1 << 24)
    # single particles: the linear weights put the charge centroid at z
    dz = p["L"] / p["Nz"]
    for zval in rng.random(50) * p["L"]:
        o1 = oracle_mod.Oracle(p)
        zf = np.float32(zval)
        o1.inject(2, [zf], [0.0], [0.0], [0.0])
        r = o1.rho_fixed()
        assert r.sum() == 1 << 24 and (r >= 0).all() and np.count_nonzero(r) <= 2
        centroid = (r * np.arange(p["Nz"] + 1)).sum() / float(1 << 24) * dz
        assert abs(centroid - float(zf)) <= dz * 2.0 ** -23 + 4e-7 * float(zf)


# ---------------------------------------------------------------- push
@pytest.mark.parametrize("species", [0, 2])
def test_leapfrog_uniform_field_closed_form(oracle_mod, species):
    """Constant acceleration a = qE/m, E = -V/L: v_n = v0 + n a dt and
    z_n = z0 + n v0 dt + a dt^2 n (n+1) / 2 (leapfrog is exact here)."""
    p = quiet(W.single_diode_small(), L=1e-2)
    o = oracle_mod.Oracle(p)
    n = 200
    z0 = np.array([2e-3, 5e-3, 7e-3], np.float32)
    v0 = np.array([1e3, -2e3, 0.0], np.float32)
    zero = np.zeros(3, np.float32)
    o.inject(species, z0, zero, zero, v0)
    o.step(n)
    st = o.state(species)
    q = -QE if species < 2 else QE
    m = ME if species < 2 else p["m_ion"]
    a = q * (-p["V"] / p["L"]) / m
    dt = p["dt"]
    order = np.argsort(st["id"])
    z_exact = z0.astype(np.float64) + n * v0 * dt + a * dt * dt * n * (n + 1) / 2
    v_exact = v0.astype(np.float64) + n * a * dt
    alive = (z_exact >= 0) & (z_exact < p["L"])
    assert st["z"].size == alive.sum()
    np.testing.assert_allclose(st["z"][order], z_exact[alive], rtol=1e-10)
    np.testing.assert_allclose(st["vz"][order], v_exact[alive], rtol=1e-10, atol=1e-9)


def test_free_streaming(oracle_mod):
    p = quiet(W.single_diode_small(), V=0.0)
    o = oracle_mod.Oracle(p)
    z0 = np.array([1e-4, 5e-4, 9e-4], np.float32)
    v0 = np.array([3e3, -1e3, 0.0], np.float32)
    zero = np.zeros(3, np.float32)
    o.inject(1, z0, zero, zero, v0)
    o.step(20)
    st = o.state(1)
    np.testing.assert_allclose(st["z"], z0 + 20 * v0.astype(np.float64) * p["dt"], rtol=1e-12)
    # the residual field of three 1e-12 m^-2 macro-particles is ~1e-17 V/m
    np.testing.assert_allclose(st["vz"], v0, rtol=1e-15, atol=1e-12)


def test_absorption_counts_and_energy_closed_form(oracle_mod):
    """Test-particle limit: every electron started at rest is absorbed at the
    anode at the first n with z_n >= L; the tallied KE is 1/2 m v_n^2 w."""
    p = quiet(W.single_diode_small(), window_start=0)
    o = oracle_mod.Oracle(p)
    rng = np.random.default_rng(2)
    N = 64
    z0 = (rng.random(N) * 0.5 * p["L"]).astype(np.float32)
    vx = (rng.standard_normal(N) * 1e4).astype(np.float32)
    zero = np.zeros(N, np.float32)
    o.inject(0, z0, vx, zero, zero)
    a = QE * p["V"] / p["L"] / ME
    dt = p["dt"]
    nmax = 4000
    o.step(nmax)
    assert o.count(0) == 0
    t = o.tallies()
    assert t["count"][0, 1] == N and t["count"][0, 0] == 0
    ke = 0.0
    for zi, vxi in zip(z0.astype(np.float64), vx.astype(np.float64)):
        n = 1
        while zi + a * dt * dt * n * (n + 1) / 2 < p["L"]:
            n += 1
        ke += 0.5 * ME * (vxi * vxi + (n * a * dt) ** 2) * p["weight"]
    assert t["ke"][0, 1] == pytest.approx(ke, rel=1e-9)


@pytest.mark.slow
def test_child_langmuir_limit(oracle_mod):
    """Cold emission at twice the vacuum Child-Langmuir flux, no collisions:
    the anode-collected flux settles at J_CL/e = (4 eps0/9) sqrt(2e/m)
    V^1.5 / d^2 / e (4.607e20 m^-2 s^-1 at 10 V, 1 mm)."""
    d, V = 1e-3, 10.0
    j_cl = 4 * EPS0 / 9 * math.sqrt(2 * QE / ME) * V ** 1.5 / d ** 2
    g_cl = j_cl / QE
    assert g_cl == pytest.approx(4.607e20, rel=1e-3)
    p = W.single_diode_small()
    p.update(n_gas=0.0, T_wall_K=10.0, gamma_emit=2 * g_cl, window_start=3000)
    p["weight"] = W.weight_for_in_flight(g_cl, d, V, 1.5e4)
    o = oracle_mod.Oracle(p)
    o.step(5000)
    dg = o.diag()
    assert dg["gamma_anode"] == pytest.approx(g_cl, rel=0.05)
    # the excess is returned to the cathode by the space-charge barrier
    assert dg["gamma_ref"] == pytest.approx(2 * g_cl - dg["gamma_anode"], rel=0.1)


# ---------------------------------------------------------------- MCC
def _beam(p, n, E_eV, species=0):
    m = ME if species < 2 else p["m_ion"]
    v = math.sqrt(2 * E_eV * QE / m)
    rng = np.random.default_rng(3)
    z = (0.25 + 0.5 * rng.random(n)) * p["L"]
    zero = np.zeros(n, np.float32)
    return z.astype(np.float32), zero, zero, np.full(n, v, np.float32), v


def test_null_collision_bound_covers_all_energies(oracle_mod):
    p = W.single_diode_small()
    o = oracle_mod.Oracle(p)
    nu_max = o.derived()["nu_max"]
    mu = ME * p["m_gas"] / (ME + p["m_gas"])
    E = np.linspace(1e-3, p["E_cap_e_eV"], 20001)
    sig = np.array([p["sigma_el_e"] + oracle_mod.sigma_exc(p, e) + oracle_mod.sigma_iz(p, e)
                    for e in E])
    nu = p["n_gas"] * sig * np.sqrt(2 * E * QE / mu)
    assert nu.max() <= nu_max[0] * (1 + 1e-12)
    assert nu.max() >= 0.95 * nu_max[0]
    # the Lotz curve peaks at P*e with value a q / (e P^2)
    P, a, q = p["E_iz_eV"], p["lotz_a"], p["lotz_q"]
    grid = np.linspace(P, 10 * P, 200001)
    lz = np.array([oracle_mod.sigma_iz(p, e) for e in grid[::100]])
    assert lz.max() == pytest.approx(a * q / (math.e * P * P), rel=1e-4)
    assert oracle_mod.sigma_iz(p, P) == 0.0 and oracle_mod.sigma_exc(p, p["E_exc_eV"]) == 0.0


def test_elastic_collision_rate_matches_constant_sigma(oracle_mod):
    """Cold gas (T_n = 0), monoenergetic 10 eV beam, constant sigma: elastic
    events in one step ~ Binomial(N, P_cand * nu / nu_max), nu = n sigma v."""
    p = quiet(W.single_diode_small(), n_gas=2e23, sigma_exc0=0.0, lotz_a=0.0,
              T_gas_e_K=0.0, window_start=0, V=0.0)
    o = oracle_mod.Oracle(p)
    N = 200_000
    z, zx, zy, vz, v = _beam(p, N, 10.0)
    o.inject(0, z, zx, zy, vz)
    d = o.derived()
    o.step(1)
    t = o.tallies()
    mu = ME * p["m_gas"] / (ME + p["m_gas"])
    g_max = math.sqrt(2 * p["E_cap_e_eV"] * QE / mu)
    p_cand = d["t_cand"][0] / 2.0 ** 32
    assert p_cand == pytest.approx(-math.expm1(-p["n_gas"] * p["sigma_el_e"] * g_max * p["dt"]),
                                   rel=1e-6)
    prob = p_cand * v / g_max
    mean, sd = N * prob, math.sqrt(N * prob * (1 - prob))
    assert abs(t["coll"][1] - mean) < 4 * sd
    assert abs(t["candidates"][0] - N * p_cand) < 4 * math.sqrt(N * p_cand)
    # scattered directions are isotropic (cos theta mean 0, second moment 1/3)
    ev = o.events()
    ids = set(ev["id"][ev["process"] == 1].tolist())
    st = o.state(0)
    sel = np.array([i in ids for i in st["id"]])
    sp = np.sqrt(st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2)[sel]
    cos = st["vz"][sel] / sp
    n = cos.size
    assert abs(cos.mean()) < 4 / math.sqrt(3 * n)
    assert abs((cos ** 2).mean() - 1 / 3) < 4 * math.sqrt(4 / 45 / n)
    # and lose at most 4 m/M of their energy (cold target)
    ke_ratio = sp ** 2 / (v * v)
    assert ke_ratio.max() <= 1 + 1e-9 and ke_ratio.min() >= 1 - 4 * ME / p["m_gas"] - 1e-9


def test_two_body_conserves_momentum_and_energy(oracle_mod):
    rng = np.random.default_rng(4)
    for _ in range(200):
        m, M = ME, W.M_HE
        v = rng.standard_normal(3) * 1e6
        vn = rng.standard_normal(3) * 1e3
        g = np.linalg.norm(v - vn)
        r1, r2 = (int(x) for x in rng.integers(0, 2 ** 32, 2))
        vo, vno = oracle_mod.two_body(m, M, v, vn, g, r1, r2)
        p0, p1 = m * v + M * vn, m * vo + M * vno
        np.testing.assert_allclose(p1, p0, rtol=1e-12, atol=1e-12 * np.abs(p0).max())
        e0 = m * v @ v + M * vn @ vn
        e1 = m * vo @ vo + M * vno @ vno
        assert e1 == pytest.approx(e0, rel=1e-12)
        assert np.linalg.norm(vo - vno) == pytest.approx(g, rel=1e-12)


def test_charge_exchange_gives_neutral_maxwellian(oracle_mod):
    """Fast ions (|v| >> v_n): CX hands the ion the neutral's velocity, so
    the collided ions are Maxwellian at T_n,i (collision weight ~ flat)."""
    p = quiet(W.single_diode_small(), n_gas=5e23, sigma_el_i=0.0, T_gas_i_K=1740.0,
              E_cap_i_eV=20000.0, window_start=0, V=0.0)
    o = oracle_mod.Oracle(p)
    N = 100_000
    z, zx, zy, vz, v = _beam(p, N, 10000.0, species=2)
    o.inject(2, z, zx, zy, vz)
    o.step(1)
    ev = o.events()
    cx = set(ev["id"][ev["process"] == 4].tolist())
    st = o.state(2)
    sel = np.array([i in cx for i in st["id"]])
    assert sel.sum() > 2000
    s_n = math.sqrt(KB * p["T_gas_i_K"] / p["m_gas"])
    for comp in ("vx", "vy"):
        assert stats.kstest(st[comp][sel] / s_n, "norm").pvalue > 1e-3
    # the axial component is shifted by O(v_n^2 / v) only
    assert stats.kstest(st["vz"][sel] / s_n, "norm").pvalue > 1e-4


def test_ionisation_children_energy_and_ids(oracle_mod):
    """Ionisation only, cold gas: the two electrons share E_rel - P exactly,
    the ion child is at rest, children are ordered by parent id."""
    p = quiet(W.single_diode_small(), n_gas=1e24, sigma_el_e=0.0, sigma_exc0=0.0,
              T_gas_e_K=0.0, window_start=0, V=0.0)
    o = oracle_mod.Oracle(p)
    N = 50_000
    E0 = 50.0
    z, zx, zy, vz, v = _beam(p, N, E0)
    o.inject(0, z, zx, zy, vz)
    o.step(1)
    t = o.tallies()
    n_iz = t["coll"][3]
    assert n_iz > 100
    assert o.count(1) == n_iz and o.count(2) == n_iz
    e_child = o.state(1)
    ions = o.state(2)
    assert np.all(ions["vx"] == 0) and np.all(ions["vz"] == 0)
    # ids: e child then ion for each event, in parent-id order
    np.testing.assert_array_equal(e_child["id"], N + 2 * np.arange(n_iz))
    np.testing.assert_array_equal(ions["id"], N + 2 * np.arange(n_iz) + 1)
    ev = o.events()
    parents = np.sort(ev["id"][ev["process"] == 3])
    prim = o.state(0)
    pos = {int(i): k for k, i in enumerate(prim["id"])}
    mu = ME * p["m_gas"] / (ME + p["m_gas"])
    E_rel = 0.5 * mu * v * v / QE - p["E_iz_eV"]
    for j, par in enumerate(parents):
        k = pos[int(par)]
        e1 = 0.5 * ME * (prim["vx"][k] ** 2 + prim["vy"][k] ** 2 + prim["vz"][k] ** 2) / QE
        e2 = 0.5 * ME * (e_child["vx"][j] ** 2 + e_child["vy"][j] ** 2
                         + e_child["vz"][j] ** 2) / QE
        assert e1 + e2 == pytest.approx(E_rel, rel=1e-6)
        assert e_child["z"][j] == prim["z"][k] and ions["z"][j] == prim["z"][k]


def test_excitation_removes_threshold_energy(oracle_mod):
    p = quiet(W.single_diode_small(), n_gas=1e24, sigma_el_e=0.0, lotz_a=0.0,
              sigma_exc0=5e-21, T_gas_e_K=0.0, window_start=0, V=0.0)
    o = oracle_mod.Oracle(p)
    N = 50_000
    z, zx, zy, vz, v = _beam(p, N, 30.0)
    o.inject(0, z, zx, zy, vz)
    o.step(1)
    ev = o.events()
    exc = set(ev["id"][ev["process"] == 2].tolist())
    assert len(exc) > 100
    st = o.state(0)
    sel = np.array([i in exc for i in st["id"]])
    ke = 0.5 * ME * (st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2) / QE
    mu = ME * p["m_gas"] / (ME + p["m_gas"])
    # cold heavy target: lab energy after = (E_rel - E_th) * (m/mu) up to O(m/M)
    target = (0.5 * mu * v * v / QE - p["E_exc_eV"])
    assert np.all(np.abs(ke[sel] - target) < 4 * ME / p["m_gas"] * 30.0 + 1e-9)
    assert np.all(ke[~sel] == pytest.approx(30.0, rel=1e-6))


# ---------------------------------------------------------------- injection
def test_thermionic_emission_count_and_distribution(oracle_mod):
    """N_emit = Gamma dt / w with a stochastic fraction (Sec. 2.2); flux-
    weighted half-Maxwellian: v_z Rayleigh, v_x, v_y normal, <KE> = 2 k T_w,
    z = v_z dt."""
    p = quiet(W.single_diode_small(), window_start=0)
    x = 40000.37
    p["gamma_emit"] = 7.25e19
    p["weight"] = p["gamma_emit"] * p["dt"] / x
    o = oracle_mod.Oracle(p)
    d = o.derived()
    assert d["emit_x"] == pytest.approx(x, rel=1e-12)
    o.step(1)
    st = o.state(0)
    assert st["z"].size in (40000, 40001)
    s = math.sqrt(KB * p["T_wall_K"] / ME)
    assert stats.kstest(st["vz"] / s, "rayleigh").pvalue > 1e-3
    assert stats.kstest(st["vx"] / s, "norm").pvalue > 1e-3
    assert stats.kstest(st["vy"] / s, "norm").pvalue > 1e-3
    ke = 0.5 * ME * (st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2)
    # Var(KE) for this law is 4 (kT)^2 -> sd of the mean = 2 kT / sqrt(N)
    assert abs(ke.mean() - 2 * KB * p["T_wall_K"]) < 4 * 2 * KB * p["T_wall_K"] / math.sqrt(ke.size)
    np.testing.assert_allclose(st["z"], st["vz"] * p["dt"], rtol=1e-15)
    assert np.all(st["vz"] > 0)


def test_emission_fraction_is_stochastic_with_right_mean(oracle_mod):
    p = quiet(W.single_diode_small(), window_start=0, gamma_emit=7.25e19)
    p["weight"] = p["gamma_emit"] * p["dt"] / 0.3      # x = 0.3 per step
    p["V"] = 0.0
    o = oracle_mod.Oracle(p)
    n = 20000
    o.step(n)
    t = o.tallies()
    assert abs(t["emitted"] - 0.3 * n) < 4 * math.sqrt(n * 0.3 * 0.7)


def test_replenishment_pairs(oracle_mod):
    """Sec. 2.1: ions lost to the walls are replaced by the same number of
    e-ion pairs at one uniform position, Maxwellian at Te0 / Ti0."""
    p = quiet(W.single_diode_small(), replenish=1, window_start=0, V=0.0)
    o = oracle_mod.Oracle(p)
    N = 20000
    z = np.full(N, np.float32(p["L"]) - np.float32(1e-9), np.float32)
    zero = np.zeros(N, np.float32)
    o.inject(2, z, zero, zero, np.full(N, 1e5, np.float32))
    o.step(1)
    t = o.tallies()
    assert t["count"][2, 1] == N and t["replenished"] == N
    e, i = o.state(1), o.state(2)
    assert e["z"].size == N and i["z"].size == N
    np.testing.assert_array_equal(e["z"], i["z"])
    assert stats.kstest(e["z"] / p["L"], "uniform").pvalue > 1e-3
    se = math.sqrt(p["T_e0_eV"] * QE / ME)
    si = math.sqrt(p["T_i0_eV"] * QE / p["m_ion"])
    for c in ("vx", "vy", "vz"):
        assert stats.kstest(e[c] / se, "norm").pvalue > 1e-3
        assert stats.kstest(i[c] / si, "norm").pvalue > 1e-3


def test_runs_are_deterministic(oracle_mod):
    p = W.single_diode_small()
    a, b = oracle_mod.Oracle(p), oracle_mod.Oracle(p)
    a.step(300)
    b.step(300)
    np.testing.assert_array_equal(a.rho_fixed(), b.rho_fixed())
    sa, sb = a.state(0), b.state(0)
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k])


# ---------------------------------------------------------------- diagnostics
def test_eq1_eq2_reproduce_table4_emission_power(oracle_mod):
    for row in load_golden("table4_energy_budget.txt"):
        g = float(row[0]) * 1e19
        d = oracle_mod.postprocess(g, 0.2, 1.0, 1.0, np.zeros((3, 2)), np.zeros((3, 2)), 0)
        assert d["q_emit_theory"] == pytest.approx(float(row[1]), abs=0.006), row


def test_eq4_to_eq5_reproduce_table4_cooling(oracle_mod):
    """Feed the table's reheating terms as tallies; Eq. 4-5 must give the
    printed cooling metrics (all columns rounded to 0.01)."""
    T, w = 1e-6, 1e7
    for row in load_golden("table4_energy_budget.txt"):
        vals = [float(x) for x in row]
        g = vals[0] * 1e19
        ke = np.zeros((3, 2))
        ke[0, 0], ke[1, 0], ke[2, 0] = vals[2] * T, vals[3] * T, vals[4] * T
        cnt = np.zeros((3, 2))
        cnt[2, 0] = vals[5] / (QE * 24.59) * T / w
        d = oracle_mod.postprocess(g, 0.2, w, T, cnt, ke, 0)
        assert d["q_ion_cath_recomb"] == pytest.approx(vals[5], rel=1e-12)
        assert d["q_cooling_1"] == pytest.approx(vals[6], abs=0.025), row
        assert d["q_cooling_2"] == pytest.approx(vals[7], abs=0.035), row


def test_flux_identities_reproduce_table2(oracle_mod):
    T, w = 1e-6, 1e7
    for row in load_golden("table2_flux_scan.txt"):
        g, gref, gnet, gan, pct = (float(x) for x in row)
        cnt = np.zeros((3, 2))
        cnt[0, 0] = gref * 1e19 * T / w
        cnt[0, 1] = gan * 1e19 * T / w
        d = oracle_mod.postprocess(g * 1e19, 0.2, w, T, cnt, np.zeros((3, 2)), 0)
        assert d["gamma_net"] / 1e19 == pytest.approx(gnet, abs=0.011), row
        # ratio from the rounded fluxes agrees with the printed ratio to the
        # rounding of Gamma_ref (0.005e19), except the two rows the table
        # itself prints inconsistently (see the fixture header)
        if g not in (4.50, 12.00):
            assert 100 * d["backflow_ratio"] == pytest.approx(pct, abs=100 * 0.0051 / g + 0.01), row
        assert d["net_efficiency"] + d["backflow_ratio"] == pytest.approx(1.0, rel=1e-12)
        assert d["collection_efficiency"] == pytest.approx(gan / g, rel=1e-12)


def test_paper_diode_derived_constants():
    """The paper-diode parameter set reproduces the constants printed in
    Sec. 2.1-2.2 (catches unit slips in the workload recipe)."""
    p = W.paper_diode()
    n0, Te0, Ti0, Tc = 5e14, 3.0, 0.15, 0.2
    mi = 6.64e-27
    dz = p["L"] / p["Nz"]
    vals = {
        "lambda_D_m": math.sqrt(EPS0 * Te0 / (n0 * QE)),
        "v_te_m_s": math.sqrt(QE * Te0 / ME),
        "v_ti_m_s": math.sqrt(QE * Ti0 / mi),
        "v_emit_m_s": math.sqrt(QE * Tc / ME),
        "c_s_m_s": math.sqrt(QE * Te0 / mi),
        "dz_m": dz,
        "omega_pe_rad_s": math.sqrt(n0 * QE * QE / (ME * EPS0)),
        "omega_pe_dt": math.sqrt(n0 * QE * QE / (ME * EPS0)) * p["dt"],
        "w0_m2": p["weight"],
        "lambda_e_m": 1 / (p["n_gas"] * p["sigma_el_e"]),
        "lambda_i_m": 1 / (p["n_gas"] * p["sigma_cx_i"]),
    }
    for name, val, tol in load_golden("derived_constants.txt"):
        assert vals[name] == pytest.approx(float(val), rel=float(tol)), name
    assert KB * p["T_wall_K"] / QE == pytest.approx(Tc, rel=1e-12)


@pytest.mark.parametrize("species", [0, 2])
def test_process_selection_splits_by_cross_section(oracle_mod, species):
    """Two channels at once: each is chosen with probability
    P_cand * n sigma_k(E) g / nu_max (cumulative selection, null otherwise)."""
    p = quiet(W.single_diode_small(), n_gas=3e23, T_gas_e_K=0.0, T_gas_i_K=0.0,
              window_start=0, V=0.0, lotz_a=0.0, sigma_exc0=8e-20, sigma_el_i=1e-19,
              E_cap_i_eV=200.0)
    o = oracle_mod.Oracle(p)
    N = 300_000
    E0 = 40.0
    z, zx, zy, vz, v = _beam(p, N, E0, species=species)
    o.inject(species, z, zx, zy, vz)
    d = o.derived()
    o.step(1)
    t = o.tallies()
    m = ME if species < 2 else p["m_ion"]
    mu = m * p["m_gas"] / (m + p["m_gas"])
    E_rel = 0.5 * mu * v * v / QE
    p_cand = d["t_cand"][species] / 2.0 ** 32
    nu_max = d["nu_max"][species]
    if species == 0:
        sig = {1: p["sigma_el_e"], 2: p["sigma_exc0"] * (1 - p["E_exc_eV"] / E_rel)}
    else:
        sig = {4: p["sigma_cx_i"], 5: p["sigma_el_i"]}
    for code, s in sig.items():
        prob = p_cand * p["n_gas"] * s * v / nu_max
        mean, sd = N * prob, math.sqrt(N * prob * (1 - prob))
        assert mean > 300
        assert abs(t["coll"][code] - mean) < 4 * sd, (code, t["coll"][code], mean)
