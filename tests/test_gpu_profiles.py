"""Late-time profiles (Sec. 3 averaged potential, species densities) and the
Eq. 9-10 virtual-cathode estimate through the C ABI, against the oracle.
Needs a GPU."""
import numpy as np
import pytest

from parity_util import load_both, mixed_state
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


def _params(window_start=4):
    p = W.single_diode_small(seed=3)
    p.update(window_start=window_start, n_gas=3e22)
    return p


def _oracle_of_gpu_state(O, p, gpu):
    """An oracle holding exactly the GPU's current particles (FP32 values)."""
    o = O.Oracle(p)
    for sp in range(3):
        s = gpu.state(sp)
        o.inject(sp, s["z"], s["vx"], s["vy"], s["vz"])
    return o


def test_sums_are_samples_of_the_stepped_states(env):
    """Step one step at a time; at each sampled step the oracle bins the GPU's
    own state: the species sums must agree bit for bit and the potential sum
    to FP64 round-off (prefix-sum solve vs Thomas)."""
    pic, O = env
    p = _params()
    st = mixed_state(p, 8, 20001, 9999)
    gpu = pic.Diode(p)
    for sp in range(3):
        gpu.inject(sp, *st[sp])
    period, n_steps = 3, 17
    gpu.set_profile_period(period)
    nn = p["Nz"] + 1
    want_cnt = np.zeros((3, nn), np.int64)
    want_phi = np.zeros(nn)
    k = 0
    for n in range(n_steps):
        gpu.step(1)
        if n >= p["window_start"] and (n - p["window_start"]) % period == 0:
            o = _oracle_of_gpu_state(O, p, gpu)
            for sp in range(3):
                want_cnt[sp] += o.species_fixed(sp)
            want_phi += o.field()[0]
            k += 1
            o.close()
    got = gpu.profiles()
    assert got["samples"] == k == 5
    assert np.array_equal(got["counts"], want_cnt)
    np.testing.assert_allclose(got["phi"] * k, want_phi, rtol=0, atol=1e-9 * k * p["V"])
    # the host post-processing is the oracle's formula
    phi, dens = O.profile_averages(want_phi, want_cnt, k, p["weight"], p["L"], p["Nz"])
    np.testing.assert_allclose(got["density"], dens, rtol=1e-14, atol=0)
    np.testing.assert_allclose(got["phi"], phi, rtol=0, atol=1e-9 * p["V"])


def test_graph_launches_sample_the_same_steps(env):
    """pic_step over CUDA graphs (the sampling rule is tested on the device)
    gives the same sums as single-step launches."""
    pic, O = env
    p = _params(window_start=10)
    st = mixed_state(p, 9, 5003, 2001)
    runs = []
    for mode in ("single", "graph"):
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *st[sp])
        d.set_profile_period(7)
        if mode == "single":
            for _ in range(117):
                d.step(1)
        else:
            d.step(117)
        runs.append(d.profiles())
        d.close()
    a, b = runs
    assert a["samples"] == b["samples"] == len(range(10, 117, 7))
    assert np.array_equal(a["counts"], b["counts"])
    assert np.array_equal(a["phi"], b["phi"])


def test_run_profiles_agree_with_the_oracle_run(env):
    """GPU and oracle advanced side by side from one state: the averaged
    potential and densities agree to the FP32-vs-FP64 drift of a few steps."""
    pic, O = env
    p = _params()
    st = mixed_state(p, 10, 20001, 9999)
    gpu, ora = pic.Diode(p), O.Oracle(p)
    load_both(gpu, ora, st)
    gpu.set_profile_period(2)
    ora.set_profile_period(2)
    gpu.step(12)
    ora.step(12)
    g = gpu.profiles()
    phi_o, cnt_o, k = ora.profiles()
    assert g["samples"] == k == 4
    np.testing.assert_allclose(g["phi"], phi_o / k, rtol=0, atol=1e-6 * p["V"])
    for sp in range(3):
        tot = max(cnt_o[sp].sum(), 1)
        assert np.abs(g["counts"][sp] - cnt_o[sp]).sum() <= 1e-3 * tot


def test_virtual_cathode_is_the_oracle_post_processing(env):
    pic, O = env
    p = W.single_diode_small(seed=4)
    p.update(window_start=100, weight=p["weight"] * 3.0)   # stronger space charge
    gpu = pic.Diode(p)
    gpu.set_profile_period(10)
    gpu.step(400)
    prof = gpu.profiles()
    d = gpu.diagnostics()
    for frac in (0.05, 0.25, 1.0):
        vc = gpu.virtual_cathode(near_fraction=frac)
        ref = O.virtual_cathode(prof["phi"], p["L"], d["T_c_eV"], d["net_efficiency"], frac)
        assert vc["samples"] == prof["samples"] == 30
        for key in ("phi_vc_eff", "phi_min", "z_min", "eta_vc", "T_emit_eV", "net_efficiency"):
            assert vc[key] == pytest.approx(ref[key], rel=1e-12, abs=1e-15), key
        assert vc["phi_min"] <= 0.0 and 0.0 < vc["eta_vc"] <= 1.0


def test_profiles_need_sampling_and_samples(env):
    pic, O = env
    p = _params()
    d = pic.Diode(p)
    with pytest.raises(pic.PicError):
        d.profiles()
    d.set_profile_period(5)
    d.step(2)                          # before the window: no samples
    got = d.profiles()
    assert got["samples"] == 0 and np.isnan(got["phi"]).all()
    with pytest.raises(pic.PicError):
        d.virtual_cathode()
    with pytest.raises(pic.PicError):
        d.set_profile_period(-1)
    # turning sampling off stops the sums; turning it on again clears them
    d.step(10)
    k = d.profiles()["samples"]
    assert k > 0
    d.set_profile_period(0)
    d.step(10)
    assert d.profiles()["samples"] == 0
