"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/pic.h; the ctypes mirrors match the C struct sizes."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import pic
    return pic.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pic_create", "pic_inject", "pic_step", "pic_diagnostics", "pic_get_state",
                 "pic_get_rho_fixed", "pic_set_step", "pic_destroy", "pic_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2605_07083_gb300 import pic
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in pic.ENTRY_POINTS, "binding lacks " + name


def test_struct_sizes_match(lib):
    from paper_2605_07083_gb300 import pic
    for i, st in enumerate((pic.PicConfig, pic.PicTuning, pic.PicDiag, pic.PicProfile)):
        assert lib.pic_sizeof(i) == C.sizeof(st)
    assert lib.pic_sizeof(99) == 0
    assert lib.pic_abi_version() == 1


def test_error_strings_and_argument_checks(lib):
    from paper_2605_07083_gb300 import pic
    assert lib.pic_strerror(0) == b"ok"
    assert b"capacity" in lib.pic_strerror(-4)
    # argument validation happens before any CUDA call
    h = C.c_void_p()
    assert lib.pic_create(None, 1, None, None, C.byref(h)) == pic.PIC_EINVAL
    cfg = pic.PicConfig()
    cfg.size = 7                                   # wrong ABI size
    assert lib.pic_create(C.byref(cfg), 1, None, None, C.byref(h)) == pic.PIC_EINVAL
    assert lib.pic_step(None, 1) == pic.PIC_EINVAL
    assert lib.pic_prepare_steps(None, 1) == pic.PIC_EINVAL
    lib.pic_destroy(None)


def test_config_marshalling_roundtrip():
    from paper_2605_07083_gb300 import pic, workloads as W
    p = W.single_diode_production()
    c = pic.make_config(p)
    assert c.size == C.sizeof(pic.PicConfig)
    assert c.n_cells == 2048 and c.gap_m == p["L"] and c.dt_s == p["dt"]
    assert c.weight == p["weight"] and c.seed == 2
