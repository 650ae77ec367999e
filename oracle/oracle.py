"""ctypes front end of the CPU oracle (arXiv 2605.07083, Sec. 2.1-2.4).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and
bench.py's cpu_baseline / reference leg may import this module.  It builds
``pic_oracle.cpp`` with g++ (FP contraction off) into ``oracle/_build/`` and
wraps it with numpy.  It imports nothing from the CUDA library package.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "pic_oracle.cpp")]
_HDR = os.path.join(_HERE, "pic_oracle.h")
_lock = threading.Lock()
_lib = None

E_CHARGE = 1.602176634e-19
K_BOLTZMANN = 1.380649e-23


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + ".tmp%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp] + _SRC
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


class OCfg(C.Structure):
    _fields_ = [
        ("L", C.c_double), ("V", C.c_double), ("Nz", C.c_int32), ("replenish", C.c_int32),
        ("dt", C.c_double), ("gamma_emit", C.c_double), ("T_wall_K", C.c_double),
        ("n_gas", C.c_double), ("T_gas_e_K", C.c_double), ("T_gas_i_K", C.c_double),
        ("T_e0_eV", C.c_double), ("T_i0_eV", C.c_double), ("weight", C.c_double),
        ("m_ion", C.c_double), ("m_gas", C.c_double), ("sigma_el_e", C.c_double),
        ("sigma_cx_i", C.c_double), ("sigma_el_i", C.c_double), ("E_exc_eV", C.c_double),
        ("sigma_exc0", C.c_double), ("E_iz_eV", C.c_double), ("lotz_a", C.c_double),
        ("lotz_q", C.c_double), ("E_cap_e_eV", C.c_double), ("E_cap_i_eV", C.c_double),
        ("window_start", C.c_int64), ("seed", C.c_uint64),
    ]


class OTally(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("count", (C.c_int64 * 2) * 3), ("ke", (C.c_double * 2) * 3),
        ("emitted", C.c_int64), ("replenished", C.c_int64), ("coll", C.c_int64 * 6),
        ("candidates", C.c_int64 * 3), ("cap_exceeded", C.c_int64),
    ]


_DIAG_FIELDS = [
    "window_time", "gamma_emit", "gamma_emit_realized", "gamma_ref", "gamma_net",
    "gamma_anode", "backflow_ratio", "net_efficiency", "collection_efficiency", "T_c_eV",
    "W_F_eff", "q_emit_theory", "q_back_em_cath", "q_back_p_cath", "q_ion_cath",
    "gamma_ion_cath", "q_ion_cath_recomb", "q_cooling_1", "q_cooling_2", "q_out_em_anode",
    "q_out_p_anode", "q_ion_anode", "gamma_ion_anode", "q_ion_anode_recomb",
    "q_anode_total_1", "q_anode_total_2",
]


class ODiag(C.Structure):
    _fields_ = [(n, C.c_double) for n in _DIAG_FIELDS]


class OEvent(C.Structure):
    _fields_ = [("species", C.c_int32), ("id", C.c_uint32), ("process", C.c_int32),
                ("margin", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.oracle_create.restype = P
            L.oracle_create.argtypes = [C.POINTER(OCfg)]
            L.oracle_destroy.argtypes = [P]
            L.oracle_inject.argtypes = [P, C.c_int, C.c_int64, P, P, P, P]
            L.oracle_set_step.argtypes = [P, C.c_int64]
            L.oracle_get_step.restype = C.c_int64
            L.oracle_get_step.argtypes = [P]
            L.oracle_next_id.restype = C.c_uint32
            L.oracle_next_id.argtypes = [P]
            L.oracle_step.argtypes = [P, C.c_int64]
            L.oracle_count.restype = C.c_int64
            L.oracle_count.argtypes = [P, C.c_int]
            L.oracle_get_state.argtypes = [P, C.c_int, P, P, P, P, P]
            L.oracle_rho_fixed.argtypes = [P, P]
            L.oracle_field.argtypes = [P, P, P]
            L.oracle_tallies.argtypes = [P, C.POINTER(OTally)]
            L.oracle_diag.argtypes = [P, C.POINTER(ODiag)]
            L.oracle_events.restype = C.c_int64
            L.oracle_events.argtypes = [P, P, C.c_int64]
            L.oracle_derived.argtypes = [P, P, P, P, P]
            L.oracle_philox4x32_10.argtypes = [P, P, P]
            L.oracle_philox2x32_10_w0.restype = C.c_uint32
            L.oracle_philox2x32_10_w0.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
            L.oracle_thomas.argtypes = [C.c_int32, C.c_double, P, P]
            L.oracle_two_body.argtypes = [C.c_double, C.c_double, P, P, C.c_double,
                                          C.c_uint32, C.c_uint32, P, P]
            L.oracle_postprocess.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                                             P, P, C.c_double, C.POINTER(ODiag)]
            L.oracle_species_fixed.argtypes = [P, C.c_int, P]
            L.oracle_set_profile_period.argtypes = [P, C.c_int64]
            L.oracle_profiles.restype = C.c_int64
            L.oracle_profiles.argtypes = [P, P, P]
            L.oracle_sigma_exc.restype = C.c_double
            L.oracle_sigma_exc.argtypes = [C.POINTER(OCfg), C.c_double]
            L.oracle_sigma_iz.restype = C.c_double
            L.oracle_sigma_iz.argtypes = [C.POINTER(OCfg), C.c_double]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def make_cfg(p: dict) -> OCfg:
    """Fill the oracle's own config struct from a plain parameter dict."""
    c = OCfg()
    for name, _ in OCfg._fields_:
        if name in p:
            setattr(c, name, p[name])
    return c


def _diag_dict(d: ODiag) -> dict:
    return {n: getattr(d, n) for n in _DIAG_FIELDS}


class Oracle:
    """One oracle diode.  ``params`` is a plain dict (see the workload module)."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._cfg = make_cfg(self.params)
        self._L = lib()
        self._h = self._L.oracle_create(C.byref(self._cfg))
        if not self._h:
            raise ValueError("oracle_create rejected the configuration")

    def close(self):
        if self._h:
            self._L.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def inject(self, species, z, vx, vy, vz):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (z, vx, vy, vz)]
        n = arrs[0].size
        if self._L.oracle_inject(self._h, species, n, *[_ptr(a) for a in arrs]) != 0:
            raise ValueError("oracle_inject failed")

    def set_step(self, step):
        self._L.oracle_set_step(self._h, step)

    @property
    def step_index(self):
        return self._L.oracle_get_step(self._h)

    @property
    def next_id(self):
        return self._L.oracle_next_id(self._h)

    def step(self, n=1):
        self._L.oracle_step(self._h, n)

    def count(self, species):
        return self._L.oracle_count(self._h, species)

    def state(self, species):
        n = self.count(species)
        z, vx, vy, vz = (np.empty(n, np.float64) for _ in range(4))
        ids = np.empty(n, np.uint32)
        self._L.oracle_get_state(self._h, species, _ptr(z), _ptr(vx), _ptr(vy), _ptr(vz),
                                 _ptr(ids))
        return {"z": z, "vx": vx, "vy": vy, "vz": vz, "id": ids}

    def rho_fixed(self):
        out = np.empty(self.params["Nz"] + 1, np.int64)
        self._L.oracle_rho_fixed(self._h, _ptr(out))
        return out

    def field(self):
        n = self.params["Nz"] + 1
        phi = np.empty(n, np.float64)
        E = np.empty(n, np.float64)
        self._L.oracle_field(self._h, _ptr(phi), _ptr(E))
        return phi, E

    def species_fixed(self, species):
        out = np.empty(self.params["Nz"] + 1, np.int64)
        self._L.oracle_species_fixed(self._h, species, _ptr(out))
        return out

    def set_profile_period(self, period):
        """Sample profiles every `period` steps inside the window (0 = off);
        clears the sums."""
        self._L.oracle_set_profile_period(self._h, int(period))

    def profiles(self):
        """(phi_sum [Nz+1], counts [3, Nz+1] int64, samples)."""
        n = self.params["Nz"] + 1
        phi = np.zeros(n, np.float64)
        cnt = np.zeros((3, n), np.int64)
        k = self._L.oracle_profiles(self._h, _ptr(phi), _ptr(cnt))
        return phi, cnt, int(k)

    def tallies(self) -> dict:
        t = OTally()
        self._L.oracle_tallies(self._h, C.byref(t))
        return {
            "steps": t.steps,
            "count": np.array([[t.count[k][w] for w in range(2)] for k in range(3)], np.int64),
            "ke": np.array([[t.ke[k][w] for w in range(2)] for k in range(3)], np.float64),
            "emitted": t.emitted, "replenished": t.replenished,
            "coll": np.array(list(t.coll), np.int64),
            "candidates": np.array(list(t.candidates), np.int64),
            "cap_exceeded": t.cap_exceeded,
        }

    def diag(self) -> dict:
        d = ODiag()
        self._L.oracle_diag(self._h, C.byref(d))
        return _diag_dict(d)

    def events(self) -> np.ndarray:
        n = self._L.oracle_events(self._h, None, 0)
        buf = (OEvent * max(n, 1))()
        self._L.oracle_events(self._h, C.cast(buf, C.c_void_p), n)
        out = np.zeros(n, dtype=[("species", np.int32), ("id", np.uint32),
                                 ("process", np.int32), ("margin", np.float64)])
        for i in range(n):
            out[i] = (buf[i].species, buf[i].id, buf[i].process, buf[i].margin)
        return out

    def derived(self) -> dict:
        nu = np.empty(3, np.float64)
        tc = np.empty(3, np.uint32)
        x = C.c_double()
        tf = C.c_uint32()
        self._L.oracle_derived(self._h, _ptr(nu), _ptr(tc), C.byref(x), C.byref(tf))
        return {"nu_max": nu, "t_cand": tc, "emit_x": x.value, "t_frac": tf.value}


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.empty(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox2x32_10_w0(c0: int, c1: int, key: int) -> int:
    return int(lib().oracle_philox2x32_10_w0(c0, c1, key))


def thomas(Nz: int, V: float, rhs: np.ndarray) -> np.ndarray:
    r = np.ascontiguousarray(rhs, np.float64)
    phi = np.empty(Nz + 1, np.float64)
    lib().oracle_thomas(Nz, V, _ptr(r), _ptr(phi))
    return phi


def two_body(m, M, v, vn, gnew, r_cos, r_phi):
    v = np.ascontiguousarray(v, np.float64)
    vn = np.ascontiguousarray(vn, np.float64)
    vo = np.empty(3, np.float64)
    vno = np.empty(3, np.float64)
    lib().oracle_two_body(m, M, _ptr(v), _ptr(vn), gnew, r_cos, r_phi, _ptr(vo), _ptr(vno))
    return vo, vno


def postprocess(gamma_emit, T_c_eV, weight, window_time, count, ke, emitted) -> dict:
    cnt = np.ascontiguousarray(count, np.float64).reshape(3, 2)
    k = np.ascontiguousarray(ke, np.float64).reshape(3, 2)
    d = ODiag()
    lib().oracle_postprocess(gamma_emit, T_c_eV, weight, window_time, _ptr(cnt), _ptr(k),
                             float(emitted), C.byref(d))
    return _diag_dict(d)


def sigma_exc(params: dict, E_eV: float) -> float:
    c = make_cfg(params)
    return lib().oracle_sigma_exc(C.byref(c), E_eV)


def sigma_iz(params: dict, E_eV: float) -> float:
    c = make_cfg(params)
    return lib().oracle_sigma_iz(C.byref(c), E_eV)


def profile_averages(phi_sum, counts, samples, weight, L, Nz):
    """Late-time averages (Sec. 3) from sampled sums.

    phi_avg = phi_sum / K in V.  Number density of species s at node j:
    counts[s, j] / 2^24 particles times the weight w, divided by K and by the
    node's length, dz inside and dz / 2 at the two electrodes (the boundary
    node collects charge from half a cell only)."""
    if samples <= 0:
        raise ValueError("no samples")
    dz = L / Nz
    vol = np.full(Nz + 1, dz)
    vol[0] = vol[-1] = 0.5 * dz
    phi = np.asarray(phi_sum, np.float64) / samples
    dens = np.asarray(counts, np.float64) / 16777216.0 * weight / (samples * vol)
    return phi, dens


def virtual_cathode(phi_avg, L, T_emit_eV, net_efficiency, near_fraction=0.1) -> dict:
    """Eq. 9-10 of Sec. 3.

    Eq. 10 maps the window's net transport efficiency to an effective
    barrier, phi_vc_eff = T_emit ln(Gamma_net / Gamma_emit) (NaN when the
    efficiency is not positive).  The near-cathode minimum phi_min of the
    averaged potential is taken over the nodes j <= floor(near_fraction Nz)
    (at least node 1); Eq. 9 gives its transmission eta_VC = exp((phi_min -
    phi_w) / T_emit) with the wall at phi_w = 0."""
    phi = np.asarray(phi_avg, np.float64)
    Nz = phi.size - 1
    jmax = min(Nz, max(1, int(math.floor(near_fraction * Nz))))
    seg = phi[:jmax + 1]
    j = int(np.argmin(seg))
    phi_min = float(seg[j])
    eff = float(net_efficiency)
    return {
        "T_emit_eV": float(T_emit_eV),
        "net_efficiency": eff,
        "phi_vc_eff": T_emit_eV * math.log(eff) if eff > 0 else float("nan"),
        "phi_min": phi_min,
        "z_min": j * (L / Nz),
        "eta_vc": math.exp(phi_min / T_emit_eV),
    }
