"""Statistical and full-size parity of the GPU path against the oracle.  GPU."""
import math

import numpy as np
import pytest

from parity_util import compare_species, load_both
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


KEYS = ("backflow_ratio", "collection_efficiency", "q_cooling_1", "q_anode_total_1")


def test_steady_state_diagnostics_within_3_sigma(env):
    """The 1 mm, 128-cell diode (2000 steps, empty start) with 8 seeds on each
    side: GPU and oracle means of the late-time diagnostics agree within 3
    sigma of the ensemble scatter."""
    pic, O = env
    seeds = range(1, 9)
    g_rows, o_rows = [], []
    for s in seeds:
        p = W.single_diode_small(seed=s)
        p["n_gas"] = 2e22            # collisional enough that backflow is not rare
        d = pic.Diode(p)
        d.step(p["n_steps"])
        dg = d.diagnostics()
        d.close()
        o = O.Oracle(p)
        o.step(p["n_steps"])
        do = o.diag()
        g_rows.append([dg[k] for k in KEYS])
        o_rows.append([do[k] for k in KEYS])
    g, o = np.array(g_rows), np.array(o_rows)
    n = len(seeds)
    for j, k in enumerate(KEYS):
        se = math.sqrt(g[:, j].var(ddof=1) / n + o[:, j].var(ddof=1) / n)
        assert se > 0, k
        assert abs(g[:, j].mean() - o[:, j].mean()) <= 3 * se, (k, g[:, j].mean(), o[:, j].mean(), se)


def test_full_production_state_one_step(env):
    """The bench workload (5 mm, 2048 cells, ~10M particles, same launch
    shape): bit-exact charge of the loaded state and one step of every
    particle against the oracle."""
    pic, O = env
    p = W.single_diode_production()
    p["capacity"] = (8_000_000, 3_000_000, 3_000_000)
    state = W.production_preload(p, seed=20)
    gpu = pic.Diode(p)
    ora = O.Oracle(p)
    load_both(gpu, ora, state)
    rg, ro = gpu.rho_fixed(), ora.rho_fixed()
    assert np.array_equal(rg, ro)
    assert rg.sum() == (2_000_000 - 8_000_000) * (1 << 24)
    gpu.set_step(1000)
    ora.set_step(1000)
    gpu.step(1)
    ora.step(1)
    ev = ora.events()
    flips = set(ev["id"][ev["margin"] < 1e-5].tolist())
    assert len(flips) <= 20
    for sp in range(3):
        g, o = gpu.state(sp), ora.state(sp)
        bad, n, ids = compare_species(g, o, sp, flips)
        assert n > 1_000_000
        assert bad == 0, (sp, bad, ids[:10])
        assert abs(g["id"].size - o["id"].size) <= 2
    dg, to = gpu.diagnostics(), ora.tallies()
    np.testing.assert_array_equal(dg["candidates"], to["candidates"])
    assert np.abs(dg["count"] - to["count"]).sum() <= 2
    assert dg["emitted"] == to["emitted"]
    gpu.close()
