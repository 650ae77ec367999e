"""Checkpoint / resume through the C ABI: a run cut in two by save and load
continues bit for bit as the uninterrupted run.  Needs a GPU."""
import numpy as np
import pytest

from parity_util import mixed_state
from paper_2605_07083_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import pic as P
    P.load()
    return P


def _snapshot(d, n_inst=1):
    out = []
    for i in range(n_inst):
        st = [d.state(sp, instance=i) for sp in range(3)]      # array order, not by id
        diag = d.diagnostics(i)
        phi, E = d.field(i)
        out.append((st, d.rho_fixed(i), phi, E, diag))
    return out


def _same(a, b):
    for (sa, ra, pa, Ea, da), (sb, rb, pb, Eb, db) in zip(a, b):
        for x, y in zip(sa, sb):
            for k in x:
                assert np.array_equal(x[k], y[k]), k
        assert np.array_equal(ra, rb)
        assert np.array_equal(pa, pb) and np.array_equal(Ea, Eb)
        for k, v in da.items():
            if isinstance(v, np.ndarray):
                assert np.array_equal(v, db[k]), k
            else:
                assert v == db[k] or (v != v and db[k] != db[k]), k


def _diode(pic, p, st):
    d = pic.Diode(p)
    for sp in range(3):
        d.inject(sp, *st[sp])
    return d


@pytest.mark.parametrize("cut", [1, 130])
def test_resume_is_bit_identical(pic, cut):
    p = W.single_diode_small(seed=6)
    p.update(n_gas=2e22, window_start=50, replenish=1)
    st = mixed_state(p, 21, 9001, 3001)
    total = 300
    a = _diode(pic, p, st)
    a.set_profile_period(5)
    a.step(total)
    b = _diode(pic, p, st)
    b.set_profile_period(5)
    b.step(cut)
    blob = b.save()
    b.close()
    c = pic.Diode(p)                    # empty handle, same configuration
    c.load(blob)
    c.step(total - cut)
    _same(_snapshot(a), _snapshot(c))
    pa, pc = a.profiles(), c.profiles()
    assert pa["samples"] == pc["samples"] > 0
    assert np.array_equal(pa["counts"], pc["counts"]) and np.array_equal(pa["phi"], pc["phi"])
    assert a.diagnostics()["step"] == c.diagnostics()["step"] == total


def test_batched_resume_is_bit_identical(pic):
    ps = W.batched_sweep(n_instances=3, seed=700, n_steps=100)
    for q in ps:
        q["weight"] *= 20.0
    a = pic.Diode(ps)
    a.step(90)
    b = pic.Diode(ps)
    b.step(40)
    blob = b.save()
    c = pic.Diode(ps)
    c.load(blob)
    c.step(50)
    _same(_snapshot(a, 3), _snapshot(c, 3))


def test_load_rejects_other_runs_and_damaged_buffers(pic):
    p = W.single_diode_small(seed=6)
    st = mixed_state(p, 22, 1001, 301)
    b = _diode(pic, p, st)
    b.step(7)
    blob = b.save()
    other = dict(p, seed=p["seed"] + 1)
    c = pic.Diode(other)
    with pytest.raises(pic.PicError):
        c.load(blob)
    assert c.diagnostics()["step"] == 0 and c.diagnostics()["n_live"] == [0, 0, 0]
    d = pic.Diode(p)
    with pytest.raises(pic.PicError):
        d.load(blob[:-4])
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(pic.PicError):
        d.load(bytes(bad))
    assert d.diagnostics()["step"] == 0
    d.load(blob)                        # the intact buffer still loads
    assert d.diagnostics()["step"] == 7
    assert d.diagnostics()["n_live"] == b.diagnostics()["n_live"]


def test_running_out_of_particle_ids_is_reported(pic):
    """A diode whose id counter is about to pass 2^32 reports PIC_ECAPACITY
    instead of reusing ids (they key the random streams).  The counter is set
    by editing a checkpoint: 56-byte header, the configs, capacities and live
    counts (4 bytes per segment each), then the per-diode records, whose
    next-id field follows the 8-byte step."""
    import struct
    p = W.single_diode_small(seed=6)          # ~19 electrons emitted per step
    d = pic.Diode(p)
    d.step(2)
    blob = bytearray(d.save())
    cfg_bytes = pic.load().pic_sizeof(0)
    at = 56 + cfg_bytes + 2 * 3 * 4 + 8
    # nothing has left the gap yet: every id handed out is a live particle
    assert struct.unpack_from("<I", blob, at)[0] == sum(d.diagnostics()["n_live"])
    struct.pack_into("<I", blob, at, 0xFFFFFFFF - 30)
    c = pic.Diode(p)
    c.load(bytes(blob))
    c.step(1)
    assert c.synchronize() == 0                # 30 ids left, ~19 used
    c.step(3)
    assert c.synchronize() == pic.PIC_ECAPACITY
