"""GPU (C-ABI) vs CPU oracle parity.  Needs a GPU."""
import math

import numpy as np
import pytest

from parity_util import REL, by_id, compare_species, load_both, mixed_state
from paper_2605_07083_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _pair(env, p, state):
    pic, O = env
    gpu = pic.Diode(p)
    ora = O.Oracle(p)
    load_both(gpu, ora, state)
    return gpu, ora


# ------------------------------------------------------------ deposit / field
@pytest.mark.parametrize("which,n_emit,n_pairs", [
    ("small", 7, 3),                 # fewer particles than one quad per species
    ("small", 20001, 9999),          # ragged, several blocks
    ("production", 100003, 50001),   # 2048 cells, ragged tail
])
def test_fixed_point_charge_is_bit_exact(env, which, n_emit, n_pairs):
    p = W.single_diode_small() if which == "small" else W.single_diode_production()
    gpu, ora = _pair(env, p, mixed_state(p, 11, n_emit, n_pairs))
    rg, ro = gpu.rho_fixed(), ora.rho_fixed()
    assert rg.dtype == np.int64 and np.array_equal(rg, ro)
    n_e = 2 * 5 + n_emit + n_pairs
    n_i = 5 + n_pairs
    assert rg.sum() == (n_i - n_e) * (1 << 24)


def test_empty_diode_field_is_vacuum(env):
    p = W.single_diode_small()
    gpu, ora = _pair(env, p, {0: [np.zeros(0, np.float32)] * 4, 1: [np.zeros(0, np.float32)] * 4,
                              2: [np.zeros(0, np.float32)] * 4})
    assert not gpu.rho_fixed().any()
    phi, E = gpu.field()
    np.testing.assert_allclose(E, -p["V"] / p["L"], rtol=1e-6)
    np.testing.assert_allclose(phi, p["V"] * np.arange(p["Nz"] + 1) / p["Nz"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("which", ["small", "production"])
def test_field_matches_oracle(env, which):
    p = W.single_diode_small() if which == "small" else W.single_diode_production()
    p["weight"] *= 50.0                      # strong space charge
    gpu, ora = _pair(env, p, mixed_state(p, 12, 30011, 7001))
    phi_g, E_g = gpu.field()
    phi_o, E_o = ora.field()
    np.testing.assert_allclose(phi_g, phi_o, rtol=0, atol=1e-9 * np.abs(phi_o).max())
    np.testing.assert_allclose(E_g, E_o, rtol=0, atol=2e-6 * np.abs(E_o).max())


# ------------------------------------------------------------ one time step
def _one_step_case(env, p, state, step0=17):
    gpu, ora = _pair(env, p, state)
    gpu.set_step(step0)
    ora.set_step(step0)
    gpu.step(1)
    ora.step(1)
    ev = ora.events()
    # MCC decisions within a relative margin of 1e-5 of a channel boundary may
    # flip between FP32 (GPU) and FP64 (oracle)
    flips = set(ev["id"][ev["margin"] < 1e-5].tolist())
    return gpu, ora, ev, flips


def _wall_flip_ids(ora_state_before, p):
    return set()


@pytest.mark.parametrize("n_gas", [2e21, 3e23])
def test_one_step_matches_oracle(env, n_gas):
    p = W.single_diode_small()
    p.update(n_gas=n_gas, replenish=1, window_start=0)
    state = mixed_state(p, 13, 40000, 20000)
    _check_one_step(env, p, state, n_gas > 1e22)


def test_one_step_matches_oracle_on_the_paper_diode(env):
    """The paper's 10 cm, 4096-cell, 40 V diode of the Table 2 scan (elastic +
    CX, T_n,i = 1740 K, replenishment) at 7.25e19, from a mixed state."""
    p = W.paper_flux_scan((7.25,), ppc=250)[0]
    p["window_start"] = 0
    p["n_gas"] = 3e23                      # many collisions in one step
    state = mixed_state(p, 16, 100000, 200000)
    _check_one_step(env, p, state, True)


def _check_one_step(env, p, state, many_collisions):
    gpu, ora, ev, flips = _one_step_case(env, p, state)
    for sp in range(3):
        g, o = gpu.state(sp), ora.state(sp)
        bad, n, bad_ids = compare_species(g, o, sp, flips)
        assert n > 0
        assert bad == 0, (sp, bad, n, bad_ids[:10])
        # live populations agree exactly unless a wall decision flipped
        assert abs(g["id"].size - o["id"].size) <= 1, (sp, g["id"].size, o["id"].size)
    dg = gpu.diagnostics()
    to = ora.tallies()
    assert len(flips) <= max(2, ev.size // 1000)
    np.testing.assert_array_equal(dg["candidates"], to["candidates"])
    assert np.abs(dg["collisions"] - to["coll"]).sum() <= 2 * len(flips)
    assert np.abs(dg["count"] - to["count"]).sum() <= 2
    np.testing.assert_allclose(dg["ke"], to["ke"], rtol=1e-5, atol=1e-30)
    assert dg["emitted"] == to["emitted"] and dg["replenished"] == to["replenished"]
    if many_collisions:
        assert dg["collisions"][1:].sum() > 100     # the case really exercises the MCC


def test_one_step_rho_after_step_matches(env):
    """Charge after one step (push + appends) agrees with the oracle's deposit of
    its own post-step state except where FP32/FP64 positions straddle a 2^-24
    cell fraction."""
    p = W.single_diode_small()
    state = mixed_state(p, 14, 30000, 10000)
    gpu, ora, ev, flips = _one_step_case(env, p, state)
    rg, ro = gpu.rho_fixed(), ora.rho_fixed()
    assert rg.sum() == ro.sum()
    tot = np.abs(ro).sum()
    assert np.abs(rg - ro).sum() <= 1e-5 * tot


def test_ionisation_children_match(env):
    p = W.single_diode_small()
    p.update(V=0.0, n_gas=1e24, sigma_el_e=0.0, sigma_exc0=0.0, T_gas_e_K=300.0,
             window_start=0, gamma_emit=0.0)
    n = 20000
    v = math.sqrt(2 * 50.0 * W.E_CHARGE / W.M_E)
    rng = np.random.default_rng(15)
    z = ((0.2 + 0.6 * rng.random(n)) * p["L"]).astype(np.float32)
    zero = np.zeros(n, np.float32)
    st = {0: (z, zero, zero, np.full(n, v, np.float32)),
          1: (np.zeros(0, np.float32),) * 4, 2: (np.zeros(0, np.float32),) * 4}
    gpu, ora, ev, flips = _one_step_case(env, p, st)
    n_iz = int((ev["process"] == 3).sum())
    assert n_iz > 50
    for sp in range(3):
        g, o = by_id(gpu.state(sp)), by_id(ora.state(sp))
        if not flips:
            np.testing.assert_array_equal(g["id"], o["id"])
        bad, cnt, _ = compare_species(gpu.state(sp), ora.state(sp), sp, flips)
        assert bad == 0, (sp, bad, cnt)
    assert gpu.diagnostics()["collisions"][3] == n_iz


# ------------------------------------------------------------ determinism
def test_run_to_run_determinism(env):
    pic, O = env
    p = W.single_diode_small()
    p["n_gas"] = 2e22
    outs = []
    for _ in range(2):
        d = pic.Diode(p)
        d.step(300)
        st = [by_id(d.state(sp)) for sp in range(3)]
        outs.append((d.rho_fixed(), st, d.diagnostics()))
        d.close()
    (r1, s1, d1), (r2, s2, d2) = outs
    assert np.array_equal(r1, r2)
    for a, b in zip(s1, s2):
        for k in a:
            assert np.array_equal(a[k], b[k])
    assert np.array_equal(d1["count"], d2["count"]) and np.array_equal(d1["ke"], d2["ke"])


# ------------------------------------------------------------ errors
def test_capacity_errors_are_reported(env):
    pic, O = env
    p = W.single_diode_small()
    p["capacity"] = (64, 64, 64)
    d = pic.Diode(p)
    z = np.full(100, 1e-4, np.float32)
    with pytest.raises(pic.PicError) as e:
        d.inject(1, z, z * 0, z * 0, z * 0)
    assert e.value.code == pic.PIC_ECAPACITY
    # emission outgrows the 64-slot emitted species on the device: sticky error
    d.step(20)
    diag = d.diagnostics(check=False)
    assert diag["rc"] == pic.PIC_ECAPACITY and diag["n_live"][0] <= 64
    with pytest.raises(pic.PicError):
        d.step(1)
    d.close()


def test_positions_outside_the_gap_are_rejected(env):
    """A z outside [0, L) anywhere in a call (host or device arrays, NaN
    included) rejects the whole call and leaves the instance as it was: the
    next valid call appends from the same slot and id."""
    pic, O = env
    import torch
    p = W.single_diode_small()
    d = pic.Diode(p)
    bad = np.array([p["L"] * 1.5], np.float32)
    with pytest.raises(pic.PicError) as e:
        d.inject(0, bad, bad * 0, bad * 0, bad * 0)
    assert e.value.code == pic.PIC_EINVAL
    z = np.linspace(0.0, p["L"] * 0.99, 1000).astype(np.float32)
    for k, v in ((0, np.nan), (999, -1e-9), (500, p["L"])):
        zz = z.copy()
        zz[k] = v
        for dev in (False, True):
            arr = torch.from_numpy(zz).cuda() if dev else zz
            with pytest.raises(pic.PicError) as e:
                d.inject(0, arr, arr * 0, arr * 0, arr * 0)
            assert e.value.code == pic.PIC_EINVAL
    assert d.state(0)["z"].size == 0
    d.inject(0, z, z * 0, z * 0, z * 0)
    st = d.state(0)
    assert np.array_equal(st["z"], z) and np.array_equal(st["id"], np.arange(1000, dtype=np.uint32))
    d.close()


# ------------------------------------------------------------ batching
def test_batched_instances_equal_separate_runs(env):
    pic, O = env
    ps = W.batched_sweep(n_instances=3, seed=500, n_steps=100)
    for p in ps:
        p["weight"] *= 20.0            # keep the test small
    both = pic.Diode(ps)
    sep = [pic.Diode(p) for p in ps]
    both.step(60)
    for i, d in enumerate(sep):
        d.step(60)
        assert np.array_equal(both.rho_fixed(i), d.rho_fixed())
        for sp in range(3):
            a, b = by_id(both.state(sp, instance=i)), by_id(d.state(sp))
            for k in a:
                assert np.array_equal(a[k], b[k]), (i, sp, k)
        da, db = both.diagnostics(i), d.diagnostics()
        assert np.array_equal(da["count"], db["count"])


def test_many_instances_equal_separate_runs(env):
    """13 diodes in one handle split k_mid's work over fewer blocks per diode
    (its field and absorbed lists) than a handle of one: states, charge and
    wall counts still match bit for bit, the FP64 energy tallies to
    rounding (their sums are grouped by those blocks)."""
    pic, O = env
    ps = W.batched_sweep(n_instances=13, seed=900, n_steps=100)
    for p in ps:
        p["weight"] *= 40.0            # keep the test small
        p["window_start"] = 0
    both = pic.Diode(ps)
    both.step(40)
    for i, p in enumerate(ps):
        d = pic.Diode(p)
        d.step(40)
        assert np.array_equal(both.rho_fixed(i), d.rho_fixed())
        for sp in range(3):
            a, b = by_id(both.state(sp, instance=i)), by_id(d.state(sp))
            for k in a:
                assert np.array_equal(a[k], b[k]), (i, sp, k)
        da, db = both.diagnostics(i), d.diagnostics()
        assert np.array_equal(da["count"], db["count"])
        np.testing.assert_allclose(da["ke"], db["ke"], rtol=1e-12)
        d.close()
    both.close()


# ------------------------------------------------------------ sort
def test_sort_is_a_stable_permutation_by_cell(env):
    pic, O = env
    p = W.single_diode_production()
    state = mixed_state(p, 16, 50000, 20000)
    d = pic.Diode(p)
    for sp in range(3):
        d.inject(sp, *state[sp])
    r0 = d.rho_fixed()
    before = [d.state(sp) for sp in range(3)]
    d.sort()
    assert np.array_equal(d.rho_fixed(), r0)
    inv = np.float32(p["Nz"] / p["L"])
    for sp in range(3):
        a, b = before[sp], d.state(sp)
        cell_a = np.clip(np.floor(a["z"] * inv), 0, p["Nz"] - 1).astype(np.int64)
        order = np.argsort(cell_a, kind="stable")
        for k in ("z", "vx", "vy", "vz", "id"):
            assert np.array_equal(b[k], a[k][order]), (sp, k)


def test_periodic_sort_leaves_the_physics_bit_identical(env):
    """Sorting only reorders the arrays: with Philox streams keyed by particle
    id and integer charge, the id-ordered state, the charge and the counts
    after 120 steps are identical with and without a sort every 10 steps
    (graphs on, sort-aligned)."""
    pic, O = env
    p = W.single_diode_small()
    p["n_gas"] = 2e22
    state = mixed_state(p, 17, 20000, 8000)
    runs = []
    for period in (0, 10):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *state[sp])
        if period:
            d.tune(sort_period=period, graph_steps=20)
        d.step(120)
        runs.append((d.rho_fixed(), [by_id(d.state(sp)) for sp in range(3)], d.diagnostics()))
        d.close()
    (r0, s0, d0), (r1, s1, d1) = runs
    assert np.array_equal(r0, r1)
    for a, b in zip(s0, s1):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(d0["count"], d1["count"])
    np.testing.assert_allclose(d0["ke"], d1["ke"], rtol=1e-12)


def test_sort_steps_are_the_same_with_and_without_graphs(env):
    """A sort period that does not divide graph_steps (7 and 16: the graphs
    become 21 and 7 steps long) and step counts that start off the sort
    phase: the raw array order, which shows where every sort fell, and the
    charge match a run of single launches with the same period."""
    pic, O = env
    p = W.single_diode_small()
    p["n_gas"] = 2e22
    state = mixed_state(p, 23, 20000, 8000)
    runs = []
    for graphs in (-1, 16):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *state[sp])
        d.tune(sort_period=7, graph_steps=graphs)
        rhos = []
        for n in (3, 50, 1, 66, 29):
            d.step(n)
            rhos.append(d.rho_fixed())
        runs.append((rhos, [d.state(sp) for sp in range(3)], d.diagnostics()))
        d.close()
    (ra, sa, da), (rb, sb, db) = runs
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    for a, b in zip(sa, sb):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert da["step"] == db["step"] == 149
    assert np.array_equal(da["count"], db["count"])


def test_prepared_graphs_run_the_same_steps(env):
    """pic_prepare_steps only captures: a handle that prepared 37 steps (and,
    with a sort period of 5, 12 more from an unaligned step) ends in the same
    state as one that did not."""
    pic, O = env
    p = W.single_diode_small()
    p["n_gas"] = 2e22
    state = mixed_state(p, 29, 20000, 8000)
    runs = []
    for prep in (False, True):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *state[sp])
        if prep:
            d.prepare(37)
        d.step(37)
        d.tune(sort_period=5, graph_steps=16)
        d.step(3)
        if prep:
            d.prepare(12)
        d.step(12)
        runs.append(([d.state(sp) for sp in range(3)], d.rho_fixed(), d.diagnostics()))
        d.close()
    (sa, ra, da), (sb, rb, db) = runs
    assert np.array_equal(ra, rb)
    for a, b in zip(sa, sb):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert da["step"] == db["step"] == 52


def test_autotuner_times_its_grid_and_keeps_the_fastest(env):
    """The autotuner on a reduced grid: one trial per distinct graph length,
    each timed over whole sort periods, and the handle left on the fastest
    shape, which still steps."""
    pic, O = env
    from paper_2605_07083_gb300 import autotune as A
    p = W.single_diode_small()
    d = pic.Diode(p)
    d.inject(0, *mixed_state(p, 5, 20000, 10)[0])
    res = A.autotune(d, steps=50, settle=10, threads=(128, 384), sort_periods=(0, 25),
                     graph_steps=(16, 20, 64))
    # sort period 25 rounds 16 and 20 up to 25 and 64 up to 75
    assert len(res["trials"]) == 2 * (3 + 2)
    assert res["ms_per_step"] == min(t["ms_per_step"] for t in res["trials"])
    assert all(t["ms_per_step"] > 0 for t in res["trials"])
    s0 = d.diagnostics()["step"]
    d.step(30)
    assert d.diagnostics()["step"] == s0 + 30
    d.close()


def test_production_determinism_over_many_steps(env):
    """The 2048-cell production diode (a 2.6M-particle preload of the same
    recipe): two runs give identical fixed-point charge at steps 1, 100 and
    2000 and identical states and tallies."""
    pic, O = env
    p = W.single_diode_production(seed=9)
    # ~750 electrons are emitted per step and few leave within 2000 steps
    p["capacity"] = (4_000_000, 1_000_000, 1_000_000)
    st = W.scaled_preload(p, seed=31, n_emit=2_000_000, n_pairs=300_000)
    runs = []
    for _ in range(2):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *st[sp])
        rhos = []
        for n in (1, 99, 1900):
            d.step(n)
            rhos.append(d.rho_fixed())
        runs.append((rhos, [by_id(d.state(sp)) for sp in range(3)], d.diagnostics()))
        d.close()
    (ra, sa, da), (rb, sb, db) = runs
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y)
    for x, y in zip(sa, sb):
        for k in x:
            assert np.array_equal(x[k], y[k])
    assert np.array_equal(da["count"], db["count"]) and np.array_equal(da["ke"], db["ke"])
    assert da["step"] == 2000 and da["emitted"] == db["emitted"]


def test_forced_wait_timeout_is_reported_and_the_context_stays_usable(env):
    """A push kernel told to give up its bulk-copy waits at once reports
    PIC_ETIMEOUT (after letting its copies in flight land); the device stays
    usable and a fresh handle steps normally."""
    pic, O = env
    p = W.single_diode_small()
    st = mixed_state(p, 17, 20001, 5001)
    d = pic.Diode(p)
    for sp in range(3):
        d.inject(sp, *st[sp])
    d.tune(wait_polls=-1)
    d.step(3)
    assert d.synchronize() == pic.PIC_ETIMEOUT
    assert d.diagnostics(check=False)["error_flags"] & (1 << 4)
    with pytest.raises(pic.PicError):
        d.step(1)                          # the error is sticky
    d.close()
    fresh = pic.Diode(p)
    for sp in range(3):
        fresh.inject(sp, *st[sp])
    fresh.step(5)
    assert fresh.synchronize() == 0
    assert fresh.diagnostics()["step"] == 5


def test_energy_above_the_null_collision_bound_is_reported(env):
    """Electrons far above E_cap make candidates whose collision rate exceeds
    nu_max: the step flags PIC_EENERGYCAP and counts them (the null-collision
    method of Sec. 2.2 needs nu <= nu_max)."""
    pic, O = env
    p = W.single_diode_small()
    p.update(V=0.0, n_gas=1e24, E_cap_e_eV=1.0, gamma_emit=0.0, window_start=0)
    n = 20000
    rng = np.random.default_rng(18)
    v = math.sqrt(2 * 50.0 * W.E_CHARGE / W.M_E)
    z = ((0.2 + 0.6 * rng.random(n)) * p["L"]).astype(np.float32)
    zero = np.zeros(n, np.float32)
    d = pic.Diode(p)
    d.inject(0, z, zero, zero, np.full(n, v, np.float32))
    d.step(1)
    assert d.synchronize() == pic.PIC_EENERGYCAP
    dg = d.diagnostics(check=False)
    assert dg["rc"] == pic.PIC_EENERGYCAP and dg["energy_cap_exceeded"] > 100


def test_results_do_not_depend_on_the_push_chunk(env):
    """Streaming 32- or 64-quad warp chunks changes nothing: 20 collisional
    steps give bit-identical states, charge and tallies."""
    pic, O = env
    p = W.single_diode_small()
    p.update(n_gas=3e22, replenish=1, window_start=0)
    st = mixed_state(p, 21, 30001, 10001)
    out = []
    for chunk in (64, 32):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *st[sp])
        d.tune(push_chunk=chunk)
        d.step(20)
        out.append(([d.state(sp) for sp in range(3)], d.rho_fixed(), d.diagnostics()))
        d.close()
    (sa, ra, da), (sb, rb, db) = out
    assert np.array_equal(ra, rb)
    for x, y in zip(sa, sb):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    for k in ("count", "ke", "collisions", "candidates"):
        assert np.array_equal(da[k], db[k]), k
    d = pic.Diode(p)
    with pytest.raises(pic.PicError) as e:
        d.tune(push_chunk=48)
    assert e.value.code == pic.PIC_EINVAL
    d.close()


@pytest.mark.parametrize("threads", [160, 320, 384])
def test_results_do_not_depend_on_the_push_block_size(env, threads):
    """The partition of the particles over push blocks changes nothing: the
    charge is exact, absorbed lists are merged in slot order and every draw
    is keyed by particle id, so 20 collisional steps give bit-identical
    states, charge and tallies with 256 and with other block sizes."""
    pic, O = env
    p = W.single_diode_small()
    p.update(n_gas=3e22, replenish=1, window_start=0)
    st = mixed_state(p, 19, 30001, 10001)
    out = []
    for t in (256, threads):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *st[sp])
        d.tune(push_threads=t)
        d.step(20)
        out.append(([d.state(sp) for sp in range(3)], d.rho_fixed(), d.diagnostics()))
        d.close()
    (sa, ra, da), (sb, rb, db) = out
    assert np.array_equal(ra, rb)
    for x, y in zip(sa, sb):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    for k in ("count", "ke", "collisions", "candidates"):
        assert np.array_equal(da[k], db[k]), k
