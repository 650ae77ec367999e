"""GPU (C-ABI) vs CPU oracle parity of the rarer parts of one step.

* the excitation channel of the electrons and the elastic channel of the
  ions (Sec. 2.2 null-collision MCC; Table 3 switches excitation on),
* ion-loss replenishment of electron-ion pairs (Sec. 2.1),
* the Eq. 1-8 post-processing of the window tallies (Sec. 2.3-2.4), exact,
  on a run whose ions reach both electrodes,
* a non-zero instance of a batched handle of uneven diodes.

Needs a GPU.
"""
import math

import numpy as np
import pytest

from parity_util import by_id, compare_species, mixed_state
from paper_2605_07083_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIAG_FIELDS = [
    "window_time", "gamma_emit", "gamma_emit_realized", "gamma_ref", "gamma_net",
    "gamma_anode", "backflow_ratio", "net_efficiency", "collection_efficiency", "T_c_eV",
    "W_F_eff", "q_emit_theory", "q_back_em_cath", "q_back_p_cath", "q_ion_cath",
    "gamma_ion_cath", "q_ion_cath_recomb", "q_cooling_1", "q_cooling_2", "q_out_em_anode",
    "q_out_p_anode", "q_ion_anode", "gamma_ion_anode", "q_ion_anode_recomb",
    "q_anode_total_1", "q_anode_total_2",
]


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import oracle as O
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import pic
    pic.load()
    return pic, O


def _iso(rng, n, speed):
    mu = 1.0 - 2.0 * rng.random(n)
    ph = 2.0 * math.pi * rng.random(n)
    s = np.sqrt(1.0 - mu * mu)
    return ((speed * s * np.cos(ph)).astype(np.float32), (speed * s * np.sin(ph)).astype(np.float32),
            (speed * mu).astype(np.float32))


def _beam(rng, n, L, E_lo, E_hi, mass):
    """n particles in the middle of the gap, energies uniform on [E_lo, E_hi]
    eV, isotropic directions."""
    z = ((0.2 + 0.6 * rng.random(n)) * L).astype(np.float32)
    E = E_lo + (E_hi - E_lo) * rng.random(n)
    return (z,) + _iso(rng, n, np.sqrt(2.0 * E * W.E_CHARGE / mass))


def _step_both(env, p, state, step0=23, instance=0, gpu=None):
    pic, O = env
    if gpu is None:
        gpu = pic.Diode(p)
        for sp in range(3):
            gpu.inject(sp, *state[sp])
    ora = O.Oracle(p)
    for sp in range(3):
        ora.inject(sp, *state[sp])
    gpu.set_step(step0)
    ora.set_step(step0)
    gpu.step(1)
    ora.step(1)
    ev = ora.events()
    flips = set(ev["id"][ev["margin"] < 1e-5].tolist())
    return gpu, ora, ev, flips


def _compare_all(gpu, ora, flips, instance=0):
    for sp in range(3):
        g, o = gpu.state(sp, instance=instance), ora.state(sp)
        bad, n, bad_ids = compare_species(g, o, sp, flips)
        if o["id"].size:
            assert n > 0
        assert bad == 0, (sp, bad, n, bad_ids[:10])
        assert abs(g["id"].size - o["id"].size) <= 1, (sp, g["id"].size, o["id"].size)


def test_excitation_and_ion_elastic_channels_match_the_oracle(env):
    """Electrons of 20-50 eV (above the 19.8 eV excitation threshold) in both
    electron species and 5-40 eV He+ with a non-zero He+-He elastic cross
    section, in a dense gas: every channel of the MCC fires (elastic,
    excitation, ionisation; CX, ion elastic) and the collided particles
    match the oracle per id."""
    p = W.single_diode_small()
    p.update(V=0.0, n_gas=1e24, sigma_exc0=5e-20, sigma_el_i=2e-19, window_start=0,
             gamma_emit=0.0)
    rng = np.random.default_rng(41)
    e0 = _beam(rng, 12000, p["L"], 20.0, 50.0, W.M_E)
    e1 = _beam(rng, 12001, p["L"], 20.0, 50.0, W.M_E)
    ions = _beam(rng, 60003, p["L"], 5.0, 40.0, p["m_ion"])
    state = {0: e0, 1: e1, 2: ions}
    gpu, ora, ev, flips = _step_both(env, p, state)
    _compare_all(gpu, ora, flips)
    dg, to = gpu.diagnostics(), ora.tallies()
    assert len(flips) <= max(2, ev.size // 1000)
    np.testing.assert_array_equal(dg["candidates"], to["candidates"])
    assert np.abs(dg["collisions"] - to["coll"]).sum() <= 2 * len(flips)
    # every channel really ran, on both sides
    for code in (1, 2, 3, 4, 5):
        assert to["coll"][code] > 100, (code, to["coll"])
        assert dg["collisions"][code] > 100, (code, dg["collisions"])
    assert dg["energy_cap_exceeded"] == 0 and to["cap_exceeded"] == 0
    # the per-id comparison above covered these excited electrons
    exc = set(ev["id"][(ev["process"] == 2) & (ev["margin"] >= 1e-5)].tolist())
    assert len(exc) > 100
    gpu.close()


def _wall_state(rng, p, n_wall=4000):
    """Particles of every species just inside both electrodes moving out
    (absorbed in the first step), plus a mixed bulk."""
    L = p["L"]
    st = mixed_state(p, 42, 20000, 6000, edge=False)
    out = {}
    for sp, mass in ((0, W.M_E), (1, W.M_E), (2, p["m_ion"])):
        v = math.sqrt(2 * 5.0 * W.E_CHARGE / mass)        # 5 eV outward
        step_len = v * p["dt"]
        zc = (rng.random(n_wall) * 0.5 * step_len).astype(np.float32)
        za = (L - rng.random(n_wall) * 0.5 * step_len).astype(np.float32)
        za = np.minimum(za, np.nextafter(np.float32(L), np.float32(0)))
        z = np.concatenate([st[sp][0], zc, za])
        vx = np.concatenate([st[sp][1], rng.standard_normal(2 * n_wall).astype(np.float32) * v * 0.1])
        vy = np.concatenate([st[sp][2], rng.standard_normal(2 * n_wall).astype(np.float32) * v * 0.1])
        vz = np.concatenate([st[sp][3], np.full(n_wall, -v, np.float32),
                             np.full(n_wall, v, np.float32)])
        out[sp] = (z, vx, vy, vz)
    return out


def test_replenishment_reinjects_pairs_like_the_oracle(env):
    """Ions leaving through both electrodes in one step: as many e-He+ pairs
    are re-injected as ions were lost (Sec. 2.1), with the oracle's ids,
    positions and velocities."""
    p = W.single_diode_small()
    p.update(replenish=1, window_start=0)
    rng = np.random.default_rng(43)
    state = _wall_state(rng, p)
    gpu, ora, ev, flips = _step_both(env, p, state)
    _compare_all(gpu, ora, flips)
    dg, to = gpu.diagnostics(), ora.tallies()
    assert to["replenished"] == to["count"][2].sum()
    assert to["replenished"] >= 7000
    assert dg["replenished"] == to["replenished"]
    np.testing.assert_array_equal(dg["count"], to["count"])
    # the new pairs: same ids on both sides, each electron beside its ion
    ge, gi = by_id(gpu.state(1)), by_id(gpu.state(2))
    n_new = int(dg["replenished"])
    new_e, new_i = ge["id"][-n_new:], gi["id"][-n_new:]
    np.testing.assert_array_equal(new_e + 1, new_i)
    np.testing.assert_array_equal(ge["z"][-n_new:], gi["z"][-n_new:])
    gpu.close()


def test_eq1_to_8_postprocessing_matches_the_oracle_exactly(env):
    """pic_diagnostics' Eq. 1-8 fields equal the oracle's post-processing of
    the same window tallies (the GPU's own counts and energies) to 1e-12, on
    a run where every species reaches both electrodes, so the
    recombination terms of Eq. 3, 5, 7 and 8 are non-zero."""
    pic, O = env
    p = W.single_diode_small()
    p.update(replenish=1, window_start=0, n_gas=2e22)
    rng = np.random.default_rng(44)
    state = _wall_state(rng, p)
    gpu = pic.Diode(p)
    for sp in range(3):
        gpu.inject(sp, *state[sp])
    gpu.step(40)
    dg = gpu.diagnostics()
    gpu.close()
    assert (dg["count"] > 0).all(), dg["count"]
    T_c = W.K_B * p["T_wall_K"] / W.E_CHARGE
    want = O.postprocess(p["gamma_emit"], T_c, p["weight"], dg["window_time"], dg["count"],
                         dg["ke"], dg["emitted"])
    assert dg["window_time"] == pytest.approx(40 * p["dt"], rel=1e-15)
    for k in DIAG_FIELDS:
        assert want[k] != 0.0, k
        assert dg[k] == pytest.approx(want[k], rel=1e-12, abs=0.0), (k, dg[k], want[k])
    assert dg["q_ion_cath_recomb"] > 0 and dg["q_ion_anode_recomb"] > 0
    assert dg["q_cooling_2"] < dg["q_cooling_1"]
    assert dg["q_anode_total_2"] > dg["q_anode_total_1"]


def test_one_step_on_instance_2_of_an_uneven_batch_matches_the_oracle(env):
    """Three diodes of different gaps, cell counts, gas densities and
    particle counts in one handle: instance 2 (uneven segment and node
    offsets before it) matches the oracle's step of that diode alone."""
    pic, O = env
    ps = W.batched_sweep(n_instances=3, seed=700, n_steps=100)
    for p in ps:
        p.update(window_start=0, replenish=1)
        p["n_gas"] *= 30.0                     # collisional in one step
    sizes = [(30011, 9001), (5003, 1999), (70001, 20011)]
    states = [mixed_state(p, 50 + i, a, b) for i, (p, (a, b)) in enumerate(zip(ps, sizes))]
    gpu = pic.Diode(ps)
    for i, st in enumerate(states):
        for sp in range(3):
            gpu.inject(sp, *st[sp], instance=i)
    assert len({p["Nz"] for p in ps}) == 3
    gpu, ora, ev, flips = _step_both(env, ps[2], states[2], gpu=gpu)
    _compare_all(gpu, ora, flips, instance=2)
    dg, to = gpu.diagnostics(2), ora.tallies()
    np.testing.assert_array_equal(dg["candidates"], to["candidates"])
    assert np.abs(dg["collisions"] - to["coll"]).sum() <= 2 * len(flips)
    assert dg["collisions"][1:].sum() > 100
    assert np.abs(dg["count"] - to["count"]).sum() <= 2
    assert dg["emitted"] == to["emitted"] and dg["replenished"] == to["replenished"]
    # charge of the new state: exact up to FP32/FP64 positions that straddle
    # a 2^-24 cell fraction
    rg, ro = gpu.rho_fixed(2), ora.rho_fixed()
    assert rg.sum() == ro.sum()
    assert np.abs(rg - ro).sum() <= 1e-5 * np.abs(ro).sum()
    gpu.close()
