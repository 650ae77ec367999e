"""Thin ctypes binding of the C ABI in include/pic.h.

Only argument marshalling lives here: every step of the method runs in the
CUDA library (``_build/libpic.so``).  Importing this module loads that
library and fails loudly if it is missing or was built without a GPU target;
there is no CPU fallback.  PyTorch supplies device memory (the caching
allocator is handed to the library as its allocator) and the CUDA stream.

Module-level functions carry the C names (``pic_create``, ``pic_inject``,
``pic_step``, ``pic_diagnostics``, ...); :class:`Diode` wraps one handle.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA = 0, -1, -2, -3
PIC_ECAPACITY, PIC_ETIMEOUT, PIC_EENERGYCAP = -4, -5, -6
SPECIES = ("emitted", "plasma_e", "ion")


class PicError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, strerror(code), code))


class PicConfig(C.Structure):
    _fields_ = [
        ("size", C.c_uint32), ("n_cells", C.c_int32),
        ("gap_m", C.c_double), ("bias_V", C.c_double), ("dt_s", C.c_double),
        ("gamma_emit", C.c_double), ("T_wall_K", C.c_double), ("n_gas", C.c_double),
        ("T_gas_e_K", C.c_double), ("T_gas_i_K", C.c_double), ("T_e0_eV", C.c_double),
        ("T_i0_eV", C.c_double), ("weight", C.c_double), ("m_ion", C.c_double),
        ("m_gas", C.c_double), ("sigma_el_e", C.c_double), ("sigma_cx_i", C.c_double),
        ("sigma_el_i", C.c_double), ("E_exc_eV", C.c_double), ("sigma_exc0", C.c_double),
        ("E_iz_eV", C.c_double), ("lotz_a", C.c_double), ("lotz_q", C.c_double),
        ("E_cap_e_eV", C.c_double), ("E_cap_i_eV", C.c_double),
        ("replenish", C.c_int32), ("reserved0", C.c_int32),
        ("window_start", C.c_int64), ("seed", C.c_uint64), ("capacity", C.c_int64 * 3),
    ]


class PicAllocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("ctx", C.c_void_p)]


class PicTuning(C.Structure):
    _fields_ = [("size", C.c_uint32), ("push_threads", C.c_int32),
                ("push_blocks_per_sm", C.c_int32), ("sort_period", C.c_int32),
                ("graph_steps", C.c_int32), ("wait_polls", C.c_int32),
                ("push_chunk", C.c_int32), ("reserved", C.c_int32 * 1)]


_DIAG_DOUBLES = [
    "gamma_emit", "gamma_emit_realized", "gamma_ref", "gamma_net", "gamma_anode",
    "backflow_ratio", "net_efficiency", "collection_efficiency", "T_c_eV", "W_F_eff",
    "q_emit_theory", "q_back_em_cath", "q_back_p_cath", "q_ion_cath", "gamma_ion_cath",
    "q_ion_cath_recomb", "q_cooling_1", "q_cooling_2", "q_out_em_anode", "q_out_p_anode",
    "q_ion_anode", "gamma_ion_anode", "q_anode_total_1", "q_ion_anode_recomb",
    "q_anode_total_2",
]


class PicDiag(C.Structure):
    _fields_ = ([("step", C.c_int64), ("window_steps", C.c_int64), ("window_time", C.c_double),
                 ("n_live", C.c_int64 * 3), ("count", (C.c_int64 * 2) * 3),
                 ("ke", (C.c_double * 2) * 3), ("emitted", C.c_int64),
                 ("replenished", C.c_int64), ("collisions", C.c_int64 * 6),
                 ("candidates", C.c_int64 * 3), ("energy_cap_exceeded", C.c_int64),
                 ("particles_pushed", C.c_int64)]
                + [(n, C.c_double) for n in _DIAG_DOUBLES]
                + [("error_flags", C.c_int32), ("reserved", C.c_int32)])


class PicProfile(C.Structure):
    _fields_ = [("steps", C.c_int64), ("ms_push", C.c_double), ("ms_mcc", C.c_double),
                ("ms_post", C.c_double), ("ms_sort", C.c_double), ("ms_total", C.c_double),
                ("particle_steps", C.c_int64), ("launches", C.c_int64),
                ("push_launches", C.c_int64)]


class PicVC(C.Structure):
    _fields_ = [("samples", C.c_int64), ("T_emit_eV", C.c_double),
                ("net_efficiency", C.c_double), ("phi_vc_eff", C.c_double),
                ("phi_min", C.c_double), ("z_min", C.c_double), ("eta_vc", C.c_double)]


# every entry point declared in include/pic.h: name -> (restype, argtypes)
_P = C.c_void_p
ENTRY_POINTS = {
    "pic_create": (C.c_int, [C.POINTER(PicConfig), C.c_int, _P, C.POINTER(PicAllocator),
                             C.POINTER(_P)]),
    "pic_inject": (C.c_int, [_P, C.c_int, C.c_int, C.c_int64, _P, _P, _P, _P, C.c_int]),
    "pic_step": (C.c_int, [_P, C.c_int64]),
    "pic_prepare_steps": (C.c_int, [_P, C.c_int64]),
    "pic_profile_steps": (C.c_int, [_P, C.c_int64, C.POINTER(PicProfile)]),
    "pic_diagnostics": (C.c_int, [_P, C.c_int, C.POINTER(PicDiag)]),
    "pic_get_state": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, _P, _P, C.c_int64,
                                C.POINTER(C.c_int64), C.c_int]),
    "pic_get_rho_fixed": (C.c_int, [_P, C.c_int, _P, C.c_int64]),
    "pic_get_field": (C.c_int, [_P, C.c_int, _P, _P, C.c_int64]),
    "pic_set_step": (C.c_int, [_P, C.c_int64]),
    "pic_set_profile_period": (C.c_int, [_P, C.c_int64]),
    "pic_get_profiles": (C.c_int, [_P, C.c_int, C.c_int64, _P, _P, _P, C.POINTER(C.c_int64)]),
    "pic_virtual_cathode": (C.c_int, [_P, C.c_int, C.c_double, C.POINTER(PicVC)]),
    "pic_checkpoint_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "pic_save": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "pic_load": (C.c_int, [_P, _P, C.c_size_t]),
    "pic_tune": (C.c_int, [_P, C.POINTER(PicTuning)]),
    "pic_sort": (C.c_int, [_P]),
    "pic_synchronize": (C.c_int, [_P]),
    "pic_last_error": (C.c_char_p, [_P]),
    "pic_destroy": (None, [_P]),
    "pic_strerror": (C.c_char_p, [C.c_int]),
    "pic_abi_version": (C.c_int, []),
    "pic_sizeof": (C.c_size_t, [C.c_int]),
    "pic_sort_by_cell_static": (C.c_int, [_P, _P, _P, _P, _P, C.c_int64, C.c_int32, C.c_double,
                                          _P, _P, _P, _P, _P, _P]),
    "pic_mlp_scratch_bytes": (C.c_size_t, [C.c_int64]),
    "pic_mlp_cast_bf16": (C.c_int, [_P, _P, _P]),
    "pic_mlp_forward": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P]),
    "pic_mlp_grad": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P, _P, C.c_size_t, _P]),
    "pic_mlp_train_step": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_float, C.c_float, C.c_float,
                                     C.c_float, _P, _P, C.c_int64, _P, _P, C.c_size_t, _P]),
}
MLP_PARAMS = 34308

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libpic.so (build it first with build.build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError("CUDA library %s is missing: run build() first" % path)
            try:
                import torch  # noqa: F401  (loads the CUDA runtime the library links)
            except ImportError:
                pass
            lib = C.CDLL(path)
            for name, (res, args) in ENTRY_POINTS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            for i, st in enumerate((PicConfig, PicTuning, PicDiag, PicProfile, PicVC)):
                if lib.pic_sizeof(i) != C.sizeof(st):
                    raise ImportError("struct %s: C size %d != ctypes size %d"
                                      % (st.__name__, lib.pic_sizeof(i), C.sizeof(st)))
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    try:
        return load().pic_strerror(code).decode()
    except ImportError:
        return "error %d" % code


def _check(rc: int, what: str, h=None):
    if rc != PIC_OK:
        err = PicError(rc, what)
        if h is not None and rc == PIC_ECUDA:
            msg = load().pic_last_error(h)
            if msg:
                err.args = (err.args[0] + " [" + msg.decode() + "]",)
        raise err


def make_config(p: dict) -> PicConfig:
    """Marshal a workload parameter dict into the C config struct."""
    c = PicConfig()
    c.size = C.sizeof(PicConfig)
    c.n_cells = int(p["Nz"])
    c.gap_m = p["L"]
    c.bias_V = p["V"]
    c.dt_s = p["dt"]
    for name in ("gamma_emit", "T_wall_K", "n_gas", "T_gas_e_K", "T_gas_i_K", "T_e0_eV",
                 "T_i0_eV", "weight", "m_ion", "m_gas", "sigma_el_e", "sigma_cx_i",
                 "sigma_el_i", "E_exc_eV", "sigma_exc0", "E_iz_eV", "lotz_a", "lotz_q",
                 "E_cap_e_eV", "E_cap_i_eV"):
        setattr(c, name, float(p.get(name, 0.0)))
    c.replenish = int(p.get("replenish", 0))
    c.window_start = int(p.get("window_start", 0))
    c.seed = int(p.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    cap = p.get("capacity", (0, 0, 0))
    for s in range(3):
        c.capacity[s] = int(cap[s])
    return c


def _torch_allocator():
    import torch

    @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    @C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a = PicAllocator()
    a.alloc = _alloc
    a.free = _free
    a.ctx = None
    return a, (_alloc, _free)


# ---------------------------------------------------------------- C names
def pic_create(configs, stream=None, allocator=None):
    lib = load()
    arr = (PicConfig * len(configs))(*configs)
    h = C.c_void_p()
    _check(lib.pic_create(arr, len(configs), stream, allocator, C.byref(h)), "pic_create")
    return h


def pic_inject(h, instance, species, z, vx, vy, vz):
    """z, vx, vy, vz: numpy float32 arrays (host) or CUDA float32 tensors."""
    on_dev = hasattr(z, "is_cuda") and z.is_cuda
    if on_dev:
        keep = [t.float().contiguous() for t in (z, vx, vy, vz)]   # alive across the call
        ptrs = [t.data_ptr() for t in keep]
        n = keep[0].numel()
    else:
        keep = [np.ascontiguousarray(a, dtype=np.float32) for a in (z, vx, vy, vz)]
        ptrs = [a.ctypes.data for a in keep]
        n = keep[0].size
    rc = load().pic_inject(h, instance, species, n, *[C.c_void_p(p) for p in ptrs], int(on_dev))
    _check(rc, "pic_inject", h)


def pic_step(h, n_steps):
    _check(load().pic_step(h, int(n_steps)), "pic_step", h)


def pic_prepare_steps(h, n_steps):
    _check(load().pic_prepare_steps(h, int(n_steps)), "pic_prepare_steps", h)


def pic_profile_steps(h, n_steps) -> dict:
    prof = PicProfile()
    _check(load().pic_profile_steps(h, int(n_steps), C.byref(prof)), "pic_profile_steps")
    return {n: getattr(prof, n) for n, _ in PicProfile._fields_}


def pic_diagnostics(h, instance=0, check=True) -> dict:
    d = PicDiag()
    rc = load().pic_diagnostics(h, instance, C.byref(d))
    if check:
        _check(rc, "pic_diagnostics")
    out = {"step": d.step, "window_steps": d.window_steps, "window_time": d.window_time,
           "n_live": list(d.n_live), "error_flags": d.error_flags, "rc": rc,
           "count": np.array([[d.count[s][w] for w in range(2)] for s in range(3)], np.int64),
           "ke": np.array([[d.ke[s][w] for w in range(2)] for s in range(3)], np.float64),
           "emitted": d.emitted, "replenished": d.replenished,
           "collisions": np.array(list(d.collisions), np.int64),
           "candidates": np.array(list(d.candidates), np.int64),
           "energy_cap_exceeded": d.energy_cap_exceeded,
           "particles_pushed": d.particles_pushed}
    for n in _DIAG_DOUBLES:
        out[n] = getattr(d, n)
    return out


def pic_get_state(h, instance, species, device=False):
    lib = load()
    n = C.c_int64()
    rc = lib.pic_get_state(h, instance, species, None, None, None, None, None, 0, C.byref(n), 0)
    if rc not in (PIC_OK, PIC_ECAPACITY):
        _check(rc, "pic_get_state")
    cnt = n.value
    if device:
        import torch
        bufs = [torch.empty(cnt, dtype=torch.float32, device="cuda") for _ in range(4)]
        ids = torch.empty(cnt, dtype=torch.int32, device="cuda")
        ptrs = [b.data_ptr() for b in bufs] + [ids.data_ptr()]
    else:
        bufs = [np.empty(cnt, np.float32) for _ in range(4)]
        ids = np.empty(cnt, np.uint32)
        ptrs = [b.ctypes.data for b in bufs] + [ids.ctypes.data]
    rc = lib.pic_get_state(h, instance, species, *[C.c_void_p(p) for p in ptrs], cnt,
                           C.byref(n), int(device))
    _check(rc, "pic_get_state")
    if device:
        ids = ids.view(torch.int32)
    return {"z": bufs[0], "vx": bufs[1], "vy": bufs[2], "vz": bufs[3], "id": ids}


def pic_get_rho_fixed(h, instance, n_nodes):
    out = np.empty(n_nodes, np.int64)
    _check(load().pic_get_rho_fixed(h, instance, out.ctypes.data_as(C.c_void_p), n_nodes),
           "pic_get_rho_fixed")
    return out


def pic_get_field(h, instance, n_nodes):
    phi = np.empty(n_nodes, np.float64)
    E = np.empty(n_nodes, np.float32)
    _check(load().pic_get_field(h, instance, phi.ctypes.data_as(C.c_void_p),
                                E.ctypes.data_as(C.c_void_p), n_nodes), "pic_get_field")
    return phi, E


def pic_set_step(h, step):
    _check(load().pic_set_step(h, int(step)), "pic_set_step")


def pic_set_profile_period(h, period):
    _check(load().pic_set_profile_period(h, int(period)), "pic_set_profile_period")


def pic_get_profiles(h, instance, n_nodes) -> dict:
    phi = np.empty(n_nodes, np.float64)
    dens = np.empty((3, n_nodes), np.float64)
    cnt = np.empty((3, n_nodes), np.int64)
    k = C.c_int64()
    _check(load().pic_get_profiles(h, instance, n_nodes, phi.ctypes.data_as(C.c_void_p),
                                   dens.ctypes.data_as(C.c_void_p),
                                   cnt.ctypes.data_as(C.c_void_p), C.byref(k)),
           "pic_get_profiles")
    return {"phi": phi, "density": dens, "counts": cnt, "samples": k.value}


def pic_virtual_cathode(h, instance=0, near_fraction=0.1) -> dict:
    v = PicVC()
    _check(load().pic_virtual_cathode(h, instance, float(near_fraction), C.byref(v)),
           "pic_virtual_cathode")
    return {n: getattr(v, n) for n, _ in PicVC._fields_}


def pic_save(h) -> bytes:
    lib = load()
    n = C.c_size_t()
    _check(lib.pic_checkpoint_bytes(h, C.byref(n)), "pic_checkpoint_bytes")
    buf = C.create_string_buffer(n.value)
    w = C.c_size_t()
    _check(lib.pic_save(h, buf, n.value, C.byref(w)), "pic_save")
    return buf.raw[:w.value]


def pic_load(h, data: bytes):
    buf = C.create_string_buffer(bytes(data), len(data))
    _check(load().pic_load(h, buf, len(data)), "pic_load")


def pic_tune(h, push_threads=0, push_blocks_per_sm=0, sort_period=0, graph_steps=0,
             wait_polls=0, push_chunk=0):
    t = PicTuning()
    t.size = C.sizeof(PicTuning)
    t.push_threads = push_threads
    t.push_chunk = push_chunk
    t.push_blocks_per_sm = push_blocks_per_sm
    t.sort_period = sort_period
    t.graph_steps = graph_steps
    t.wait_polls = wait_polls
    _check(load().pic_tune(h, C.byref(t)), "pic_tune")


def pic_sort(h):
    _check(load().pic_sort(h), "pic_sort")


def pic_synchronize(h):
    return load().pic_synchronize(h)


def pic_destroy(h):
    load().pic_destroy(h)


# ---------------------------------------------------------------- wrapper
class Diode:
    """One handle holding one or more independent diodes (instances)."""

    def __init__(self, params, stream=None, torch_memory=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the PIC-MCC library needs a CUDA device")
        plist = params if isinstance(params, (list, tuple)) else [params]
        self.params = [dict(p) for p in plist]
        self.n_instances = len(self.params)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._alloc_keep = None
        alloc = None
        if torch_memory:
            a, keep = _torch_allocator()
            self._alloc_keep = (a, keep)
            alloc = C.byref(a)
        self._h = pic_create([make_config(p) for p in self.params],
                             C.c_void_p(self.stream.cuda_stream), alloc)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nodes(self, instance=0):
        return int(self.params[instance]["Nz"]) + 1

    def inject(self, species, z, vx, vy, vz, instance=0):
        pic_inject(self._h, instance, species, z, vx, vy, vz)

    def step(self, n=1):
        pic_step(self._h, n)

    def prepare(self, n):
        """Capture now the step graphs that step(n) will launch."""
        pic_prepare_steps(self._h, n)

    def profile(self, n):
        return pic_profile_steps(self._h, n)

    def diagnostics(self, instance=0, check=True):
        return pic_diagnostics(self._h, instance, check)

    def state(self, species, instance=0, device=False):
        return pic_get_state(self._h, instance, species, device)

    def rho_fixed(self, instance=0):
        return pic_get_rho_fixed(self._h, instance, self.nodes(instance))

    def field(self, instance=0):
        return pic_get_field(self._h, instance, self.nodes(instance))

    def set_step(self, step):
        pic_set_step(self._h, step)

    def tune(self, **kw):
        pic_tune(self._h, **kw)

    def set_profile_period(self, period):
        pic_set_profile_period(self._h, period)

    def profiles(self, instance=0):
        return pic_get_profiles(self._h, instance, self.nodes(instance))

    def virtual_cathode(self, instance=0, near_fraction=0.1):
        return pic_virtual_cathode(self._h, instance, near_fraction)

    def save(self) -> bytes:
        return pic_save(self._h)

    def load(self, data: bytes):
        pic_load(self._h, data)

    def sort(self):
        pic_sort(self._h)

    def synchronize(self):
        return pic_synchronize(self._h)
