"""Emission-flux scan of the paper's benchmark diode (Sec. 2.1-2.2, Sec. 3.1
Table 2, Sec. 3 potential profiles and Eq. 9-10) as one batched job.

Every flux of the scan is one instance of a single library handle, so the
whole scan advances in one launch sequence per step.  The run reports, per
flux, the window diagnostics (fluxes, backflow ratio, Eq. 1-8 energy terms),
the late-time averaged potential profile and the Eq. 9-10 virtual-cathode
estimate, plus the particle-steps per second of the whole job.

    python -m paper_2605_07083_gb300.flux_scan --ppc 250 --steps 4500000 --out scan.json
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import pic
from . import workloads as W

_DIAG_KEYS = ("gamma_emit", "gamma_emit_realized", "gamma_ref", "gamma_net", "gamma_anode",
              "backflow_ratio", "net_efficiency", "collection_efficiency", "T_c_eV", "W_F_eff",
              "q_emit_theory", "q_back_em_cath", "q_back_p_cath", "q_ion_cath",
              "q_ion_cath_recomb", "q_cooling_1", "q_cooling_2", "q_anode_total_1",
              "q_anode_total_2", "window_time", "window_steps", "energy_cap_exceeded")


def stationarity(blocks) -> dict:
    """Reading of Sec. 3's "late-time window" check: split the window's block
    means (equal-length blocks of steps) into halves and call the window
    stationary when the two half means differ by no more than twice the
    standard error of their difference, sqrt(s1^2/n1 + s2^2/n2) from the
    block scatter.  Needs at least two blocks per half."""
    b = np.asarray([x for x in blocks if np.isfinite(x)], np.float64)
    if b.size < 4:
        return {"blocks": b.size, "stationary": None}
    h = b.size // 2
    a, c = b[:h], b[b.size - h:]
    se = math.sqrt(a.var(ddof=1) / a.size + c.var(ddof=1) / c.size)
    diff = float(c.mean() - a.mean())
    return {"blocks": int(b.size), "first_half": float(a.mean()), "second_half": float(c.mean()),
            "difference": diff, "two_sigma": 2.0 * se, "stationary": bool(abs(diff) <= 2.0 * se)}


def run(fluxes=W.TABLE2_FLUXES, ppc=1000, n_steps=4_500_000, window_start=None,
        profile_period=1000, chunk=50_000, max_seconds=None, seed=3, log=sys.stderr,
        profile_points=512, table3=False, kernel_times=0) -> dict:
    """Run the scan (or, with table3, the Table 3 sensitivity cases) as one
    batched job; stop early (and say so) if max_seconds would be passed."""
    import torch
    if table3:
        ps = W.paper_table3_cases(ppc=ppc, n_steps=n_steps, window_start=window_start)
        fluxes = tuple(p["gamma_emit"] / 1e19 for p in ps)
    else:
        ps = W.paper_flux_scan(fluxes, ppc=ppc, n_steps=n_steps, window_start=window_start,
                               seed=seed)
    d = pic.Diode(ps)
    for i, p in enumerate(ps):
        st = W.paper_initial_plasma(p, seed=1000 + i)
        for sp in (1, 2):
            d.inject(sp, *st[sp], instance=i)
    d.set_profile_period(profile_period)
    t0 = time.time()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pushed0 = sum(d.diagnostics(i)["particles_pushed"] for i in range(len(ps)))
    ev0.record(d.stream)
    done, complete = 0, True
    # block means of the backflow ratio inside the window, one per chunk
    prev = [None] * len(ps)
    blocks = [[] for _ in ps]
    while done < n_steps:
        n = min(chunk, n_steps - done)
        d.step(n)
        d.synchronize()
        done += n
        for i, p in enumerate(ps):
            dg = d.diagnostics(i, check=False)
            cur = (dg["window_steps"], int(dg["count"][0][0]))
            if prev[i] is not None and cur[0] - prev[i][0] == n:
                dt = n * p["dt"]
                blocks[i].append((cur[1] - prev[i][1]) * p["weight"] / dt / p["gamma_emit"])
            prev[i] = cur
        el = time.time() - t0
        live = [sum(d.diagnostics(i)["n_live"]) for i in range(len(ps))]
        print("step %d/%d  %.0f s  live %.3g" % (done, n_steps, el, float(sum(live))), file=log,
              flush=True)
        if max_seconds is not None and done < n_steps and el * (done + n) / done > max_seconds:
            complete = False
            break
    ev1.record(d.stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    pushed = sum(d.diagnostics(i)["particles_pushed"] for i in range(len(ps))) - pushed0
    rows = []
    for i, p in enumerate(ps):
        dg = d.diagnostics(i, check=False)
        row = {"gamma_emit_1e19": p["gamma_emit"] / 1e19, "seed": p["seed"],
               "label": p.get("label", ""), "ppc": p["ppc"], "n_live": dg["n_live"],
               "rc": dg["rc"], "collisions": dg["collisions"].tolist()}
        row.update({k: dg[k] for k in _DIAG_KEYS})
        row["backflow_blocks"] = blocks[i]
        row["stationarity"] = stationarity(blocks[i])
        prof = d.profiles(i)
        if prof["samples"] > 0:
            vc = d.virtual_cathode(i, near_fraction=0.05)
            row["virtual_cathode"] = vc
            stride = max(1, (p["Nz"] + 1) // profile_points)
            row["phi_profile"] = {"z_m": (np.arange(0, p["Nz"] + 1, stride) * p["L"] / p["Nz"]).tolist(),
                                  "phi_V": prof["phi"][::stride].tolist()}
            row["profile_samples"] = prof["samples"]
        rows.append(row)
    kt = None
    if kernel_times > 0:
        # after the rows: per-kernel device time (one launch at a time) and the
        # CUDA-graph step, on the final state
        prof = d.profile(kernel_times)
        n = max(prof["steps"], 1)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d.prepare(1000)                       # graphs captured outside the timing
        d.synchronize()
        g0.record(d.stream)
        d.step(1000)
        g1.record(d.stream)
        g1.synchronize()
        kt = {"steps": n, "push_us": 1e3 * prof["ms_push"] / n, "mcc_us": 1e3 * prof["ms_mcc"] / n,
              "post_us": 1e3 * prof["ms_post"] / n, "graph_step_us": g0.elapsed_time(g1),
              "live": int(sum(sum(d.diagnostics(i, check=False)["n_live"]) for i in range(len(ps))))}
    d.close()
    return {"config": {"fluxes_1e19": list(fluxes), "ppc": ppc, "n_steps": n_steps,
                       "steps_done": done, "complete": complete,
                       "window_start": ps[0]["window_start"], "profile_period": profile_period,
                       "dt_s": ps[0]["dt"], "weight_m2": ps[0]["weight"], "L_m": ps[0]["L"],
                       "Nz": ps[0]["Nz"], "V": ps[0]["V"], "E_cap_eV": ps[0]["E_cap_e_eV"]},
            "rows": rows,
            "kernel_times": kt,
            "gpu_ms": ms, "particle_steps": int(pushed),
            "particle_steps_per_s": pushed / (ms * 1e-3) if ms > 0 else math.nan,
            "wall_s": time.time() - t0}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--ppc", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=4_500_000)
    ap.add_argument("--window-start", type=int, default=None)
    ap.add_argument("--profile-period", type=int, default=1000)
    ap.add_argument("--chunk", type=int, default=50_000)
    ap.add_argument("--max-seconds", type=float, default=None)
    ap.add_argument("--fluxes", type=str, default=None,
                    help="comma-separated fluxes in 1e19 m^-2 s^-1 (default: Table 2)")
    ap.add_argument("--table3", action="store_true",
                    help="run the Table 3 sensitivity cases instead of the flux scan")
    ap.add_argument("--kernel-times", type=int, default=0,
                    help="after the run, time this many steps kernel by kernel and 1000 as graphs")
    ap.add_argument("--out", type=str, default=None)
    a = ap.parse_args(argv)
    fl = tuple(float(x) for x in a.fluxes.split(",")) if a.fluxes else W.TABLE2_FLUXES
    res = run(fl, ppc=a.ppc, n_steps=a.steps, window_start=a.window_start,
              profile_period=a.profile_period, chunk=a.chunk, max_seconds=a.max_seconds,
              table3=a.table3, kernel_times=a.kernel_times)
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    print(json.dumps({k: v for k, v in res.items() if k != "rows"}))
    for r in res["rows"]:
        print("%-12s %6.2f  backflow %.4f  net %.4f  anode %.4f  q_cool1 %.2f  phi_eff %s  "
              "stationary %s" % (
                  r["label"], r["gamma_emit_1e19"], r["backflow_ratio"], r["net_efficiency"],
                  r["collection_efficiency"], r["q_cooling_1"],
                  "%.4f" % r["virtual_cathode"]["phi_vc_eff"] if "virtual_cathode" in r else "-",
                  r["stationarity"]["stationary"]))


if __name__ == "__main__":
    main()
