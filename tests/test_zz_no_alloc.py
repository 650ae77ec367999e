"""The allocation-free sort entry point (pic_sort_by_cell_static).

Some callers cannot allocate device memory once they run -- a real-time loop
or a host application that reserved its memory up front, where a cudaMalloc
could fail, block or synchronise the device.  This entry point takes its
scratch from a fixed array inside the library.  It is checked through the C
ABI against the handle's own sort (pic_sort) on two calls in a row, the
second reusing the scratch the first left behind.  GPU.
"""
import ctypes as C

import numpy as np
import pytest

from parity_util import mixed_state
from paper_2605_07083_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_sort_matches_the_handle_sort_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import pic
    lib = pic.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(W.single_diode_production(), 31, 60000, 25000),
             (W.single_diode_small(), 32, 20001, 7003)]
    for p, seed, n_emit, n_pairs in cases:
        state = mixed_state(p, seed, n_emit, n_pairs)
        d = pic.Diode(p)
        for sp in range(3):
            d.inject(sp, *state[sp])
        before = [d.state(sp, device=True) for sp in range(3)]
        d.sort()
        after = [d.state(sp) for sp in range(3)]
        for sp in range(3):
            src = before[sp]
            n = src["z"].numel()
            out = {k: torch.empty_like(src[k]) for k in ("z", "vx", "vy", "vz", "id")}
            args = [C.c_void_p(src[k].data_ptr()) for k in ("z", "vx", "vy", "vz", "id")]
            outs = [C.c_void_p(out[k].data_ptr()) for k in ("z", "vx", "vy", "vz", "id")]
            rc = lib.pic_sort_by_cell_static(*args, n, p["Nz"], p["L"], *outs, C.c_void_p(stream))
            assert rc == pic.PIC_OK
            torch.cuda.synchronize()
            for k in ("z", "vx", "vy", "vz"):
                assert np.array_equal(out[k].cpu().numpy(), after[sp][k]), (sp, k)
            assert np.array_equal(out["id"].cpu().numpy().view(np.uint32), after[sp]["id"])
        d.close()


def test_static_sort_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07083_gb300 import pic
    lib = pic.load()
    t = torch.zeros(16, dtype=torch.float32, device="cuda")
    ptr = C.c_void_p(t.data_ptr())
    # 4096 cells x ceil(3M / 8192) columns > 2^20 entries: refused before any launch
    rc = lib.pic_sort_by_cell_static(ptr, ptr, ptr, ptr, ptr, 3_000_000, 4096, 1e-3,
                                     ptr, ptr, ptr, ptr, ptr, None)
    assert rc == pic.PIC_ECAPACITY
    # one cell keeps the histogram small, but 2^31 particles would overflow
    # the 32-bit output positions: refused before any launch
    rc = lib.pic_sort_by_cell_static(ptr, ptr, ptr, ptr, ptr, 1 << 31, 1, 1e-3,
                                     ptr, ptr, ptr, ptr, ptr, None)
    assert rc == pic.PIC_ECAPACITY
    assert lib.pic_sort_by_cell_static(ptr, ptr, ptr, ptr, ptr, 10, 0, 1e-3,
                                       ptr, ptr, ptr, ptr, ptr, None) == pic.PIC_EINVAL
