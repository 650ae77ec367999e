"""Shared helpers of the GPU-vs-oracle parity tests."""
import numpy as np

from paper_2605_07083_gb300 import workloads as W

# one push/MCC step: |gpu - oracle| <= REL * (|oracle| + floor)
REL = 1e-5
V_FLOOR = {0: 1e5, 1: 1e5, 2: 1e2}       # m/s: FP32 Box-Muller/direction error scale
Z_FLOOR = 1e-9                           # m


def mixed_state(p, seed, n_emit, n_pairs, edge=True):
    """Seeded state of all three species; adds edge positions (z = 0, the
    last float below L, exact node positions) when edge is set."""
    rng = np.random.default_rng(seed)
    em = list(W.emitted_fill(rng, n_emit, p["L"], p["T_wall_K"]))
    pe, pi = W.uniform_plasma(rng, n_pairs, p["L"], p.get("T_e0_eV", 3.0), p.get("T_i0_eV", 0.15))
    pe, pi = list(pe), list(pi)
    if edge:
        Lf = np.float32(p["L"])
        extra = np.array([0.0, np.nextafter(Lf, np.float32(0)), p["L"] / p["Nz"],
                          p["L"] / 2, 3 * p["L"] / p["Nz"]], np.float32)
        for arrs in (em, pe, pi):
            arrs[0] = np.concatenate([arrs[0], extra])
            for k in (1, 2, 3):
                arrs[k] = np.concatenate([arrs[k], np.zeros(extra.size, np.float32)])
    return {0: tuple(em), 1: tuple(pe), 2: tuple(pi)}


def load_both(gpu, ora, state, instance=0):
    for sp in (0, 1, 2):
        gpu.inject(sp, *state[sp], instance=instance)
        ora.inject(sp, *state[sp])


def by_id(st):
    o = np.argsort(st["id"], kind="stable")
    return {k: np.asarray(v)[o] for k, v in st.items()}


def compare_species(g, o, sp, flip_ids=(), rel=REL):
    """Match by id; return (n_bad, n) over ids present on both sides."""
    g, o = by_id(g), by_id(o)
    common, gi, oi = np.intersect1d(g["id"], o["id"], return_indices=True)
    keep = ~np.isin(common, np.asarray(list(flip_ids), np.uint32))
    bad = np.zeros(common.size, bool)
    for k in ("z", "vx", "vy", "vz"):
        a = g[k][gi].astype(np.float64)
        b = o[k][oi]
        floor = Z_FLOOR if k == "z" else V_FLOOR[sp]
        bad |= np.abs(a - b) > rel * (np.abs(b) + floor)
    bad &= keep
    return int(bad.sum()), int(common.size), common[bad]
