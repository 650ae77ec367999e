"""Throughput of the PIC-MCC diode step on GB300.

Workload: the production-size single He diode (5 mm gap, 2048 cells, dt 5e-13
s, 10 V; elastic + excitation + Lotz ionisation for e-He, CX for He+-He),
preloaded with a synthetic state of 6M emitted-type electrons and 2M plasma
e-He+ pairs (~10M macro-particles, 200 MB of streamed state: larger than L2).
One bench step = one PIC time step of the whole hot path: deposit/field,
gather+push+absorb, MCC, compaction, emission, replenishment.

Metric: particle-steps/s (sum over steps of live particles pushed / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank advances its own independent replica
diode (different seed), no data-path collective; value is the sum over ranks.
The reference arm times the CPU oracle on a bounded sample of the same state.
Rank 0 also reports, in the same JSON line, the 64-diode batched sweep
(10,000 steps in one autotuned handle against the same diodes one by one;
--no-batched skips it) and the small 128-cell diode.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_07083_gb300 import workloads as W  # noqa: E402

ALG_BYTES_PER_PARTICLE = 20      # read z, v_z, id + write z, v_z (FP32/u32)
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def measured_traffic():
    """DRAM bytes per k_push launch from the committed ncu summary, if the
    kernel source it was taken on is the one built now (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_kernels_production_diode.md")
    csrc = os.path.join(ROOT, "paper_2605_07083_gb300", "csrc")
    try:
        h = hashlib.sha1()
        for f in ("pic_kernels.cu", "pic_internal.cuh"):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
        want = h.hexdigest()[:16]
        traffic, sha = None, None
        with open(path) as fh:
            for line in fh:
                if line.startswith("traffic_bytes_per_launch(k_push):"):
                    traffic = float(line.split(":")[1])
                if line.startswith("kernel_source_sha1_16:"):
                    sha = line.split(":")[1].strip()
        return traffic if sha == want else None
    except OSError:
        return None


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload(seed_offset=0):
    p = W.single_diode_production(seed=2 + seed_offset)
    p["capacity"] = (8_000_000, 3_000_000, 3_000_000)
    return p


def describe(p, n0):
    return {"workload": "single He diode 5 mm, 2048 cells, dt 5e-13 s, 10 V, preloaded "
                        "6M emitted e + 2M plasma e-He+ pairs",
            "cells": p["Nz"], "particles_initial": int(n0), "dt_s": p["dt"],
            "weight_m2": p["weight"], "l2": "inputs larger than L2 (~200 MB streamed per step)",
            "pic_steps_per_bench_step": 1}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for n, v in zip(names, r[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def reduce_over_ranks(ms, pushed, e2e_s, e2e_ps, device="cpu"):
    """Whole-job numbers of independent replicas: the slowest rank's times and
    the sum of the particle-steps of all ranks (no collective in the data path;
    this is the only exchange, after the timed region)."""
    import torch
    vals = torch.tensor([ms, float(pushed), e2e_s, float(e2e_ps)], dtype=torch.float64,
                        device=device)
    try:
        import torch.distributed as td
        dist = td.is_available() and td.is_initialized() and td.get_world_size() > 1
    except Exception:
        dist = False
    if not dist:
        return ms, float(pushed), e2e_s, float(e2e_ps)
    mx = vals.clone()
    td.all_reduce(mx, op=td.ReduceOp.MAX)
    sm = vals.clone()
    td.all_reduce(sm, op=td.ReduceOp.SUM)
    return mx[0].item(), sm[1].item(), mx[2].item(), sm[3].item()


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import torch
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import pic

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    p = workload(seed_offset=rank)
    state = W.production_preload(p, seed=20 + rank)
    n0 = sum(state[s][0].size for s in range(3))
    dist = world > 1
    if dist:
        import torch.distributed as td

    def barrier():
        if dist:
            td.barrier()
        torch.cuda.synchronize()

    d = pic.Diode(p)
    for sp in range(3):
        d.inject(sp, *state[sp])
    d.step(args.warmup)
    d.prepare(args.steps)                 # the timed steps' graphs, captured untimed
    d.synchronize()
    stream = d.stream
    # --- timed region 1: graph-launched steps (value)
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    pushed0 = d.diagnostics()["particles_pushed"]
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    pushed = d.diagnostics()["particles_pushed"] - pushed0
    # --- timed region 2: same steps with CUDA events around every kernel
    pushed1 = d.diagnostics()["particles_pushed"]
    prof = d.profile(args.steps)
    pushed_prof = d.diagnostics()["particles_pushed"] - pushed1
    ck = clocks.stop()
    diag = d.diagnostics()
    d.close()
    del d
    torch.cuda.synchronize()

    # --- end to end through the C ABI: host (pinned) state in, K steps, diag out
    pinned = {}
    h2d = 0
    for sp in range(3):
        pinned[sp] = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in state[sp]]
        h2d += sum(t.numel() * 4 for t in pinned[sp])
    lib = pic.load()
    import ctypes as C
    h = pic.pic_create([pic.make_config(p)], C.c_void_p(stream.cuda_stream),
                       None)
    barrier()
    t0 = time.perf_counter()
    for sp in range(3):
        n = pinned[sp][0].numel()
        rc = lib.pic_inject(h, 0, sp, n, *[C.c_void_p(t.data_ptr()) for t in pinned[sp]], 0)
        assert rc == 0, rc
    lib.pic_step(h, args.warmup + args.steps)
    dg = pic.PicDiag()
    rc = lib.pic_diagnostics(h, 0, C.byref(dg))
    t1 = time.perf_counter()
    barrier()
    e2e_ps = dg.particles_pushed
    lib.pic_destroy(h)
    e2e_s = t1 - t0
    n_e2e_steps = args.warmup + args.steps

    # --- reduce over ranks
    ms_max, pushed_tot, e2e_max, e2e_tot = reduce_over_ranks(ms, pushed, e2e_s, e2e_ps,
                                                             device="cuda")
    if rank != 0:
        return None
    value = pushed_tot / (ms_max * 1e-3)
    peak, peak_kind = hbm_peak()
    push_ms = prof["ms_push"] / max(prof["push_launches"], 1)
    n_per_launch = pushed_prof / max(prof["push_launches"], 1)
    achieved = ALG_BYTES_PER_PARTICLE * n_per_launch / (push_ms * 1e-3) / 1e9
    # the same algorithmic bytes over push + MCC: k_push (which also draws
    # every particle's null-collision candidate word) and k_mid (which
    # applies the candidates' collisions, in blocks that run beside the
    # field solve and the absorbed lists, so its whole time is counted)
    mcc_ms = prof["ms_mcc"] / max(prof["push_launches"], 1)
    achieved_pm = ALG_BYTES_PER_PARTICLE * n_per_launch / ((push_ms + mcc_ms) * 1e-3) / 1e9
    # and over the whole graph-launched step (push, k_mid, compaction and
    # injection), from the timed region of ``value``
    step_ms = ms_max / max(args.steps, 1)
    achieved_step = ALG_BYTES_PER_PARTICLE * (pushed_tot / max(args.steps, 1)) / (step_ms * 1e-3) / 1e9
    cpu = cpu_baseline(p, state) if not args.no_cpu else None
    batched = run_batched() if not args.no_batched else None
    if batched is not None and not args.no_cpu:
        batched["cpu_baseline"] = cpu_baseline_batched()
    small = run_small() if not args.no_batched else None
    launches = 3 * args.steps
    out = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": describe(p, n0),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(),
                     "kernel": "k_push", "peak_kind": peak_kind + " (hbm_gbs)",
                     "alg_bytes_per_particle": ALG_BYTES_PER_PARTICLE,
                     "particles_per_launch": n_per_launch, "avg_launch_ms": push_ms,
                     "push_mcc": {"achieved": achieved_pm, "frac": achieved_pm / peak,
                                  "ms": push_ms + mcc_ms, "target_frac": 0.60,
                                  "kernels": "k_push + k_mid, each launched alone"},
                     "step": {"achieved": achieved_step, "frac": achieved_step / peak,
                              "ms": step_ms, "kernels": "k_push + k_mid + k_post in CUDA graphs"},
                     "ms_mcc_per_step": prof["ms_mcc"] / max(args.steps, 1),
                     "ms_post_per_step": prof["ms_post"] / max(args.steps, 1),
                     "ms_step_profiled": prof["ms_total"] / max(args.steps, 1)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_tot / e2e_max, "unit": "particle-steps/s",
                "h2d_bytes_per_step": h2d / n_e2e_steps,
                "d2h_bytes_per_step": C.sizeof(pic.PicDiag) / n_e2e_steps,
                "steps": n_e2e_steps, "includes": "pic_inject from pinned host + pic_step + "
                                                   "pic_diagnostics"},
        "gpu_launches": launches,
        "batched_sweep": batched,
        "small_diode": small,
        "clocks": ck,
        "diag": {"n_live": diag["n_live"], "backflow_ratio": diag["backflow_ratio"],
                 "candidates": diag["candidates"].tolist()},
    }
    return out


def batched_instance(p, i, seed=1000, steps=100):
    """Diode i of the sweep preloaded with its target in-flight emitted
    population (uniform positions, T_w velocities); sets its capacities."""
    n = int(p["target_in_flight"])
    rng = np.random.default_rng(seed + 7919 * (i + 1))
    em = W.emitted_fill(rng, n, p["L"], p["T_wall_K"])
    em = (W.clamp_inside(em[0], p["L"]),) + tuple(em[1:])
    x = p["gamma_emit"] * p["dt"] / p["weight"]
    p["capacity"] = (int(n + 1.3 * x * (3 * steps + 400)) + 4096, 65536, 65536)
    return em


def batched_workload(n_instances=64, seed=1000, steps=100):
    """The uneven 64-diode sweep, each diode preloaded (batched_instance)."""
    ps = W.batched_sweep(n_instances=n_instances, seed=seed, n_steps=steps)
    states = [batched_instance(p, i, seed, steps) for i, p in enumerate(ps)]
    return ps, states


def _oracle_instance(args):
    """One sweep diode on the oracle (a worker process): (particle-steps, s)."""
    i, n_steps = args
    from oracle import oracle as O
    p = W.batched_sweep(n_instances=64, seed=1000, n_steps=100)[i]
    em = batched_instance(p, i)
    o = O.Oracle(p)
    o.inject(0, *em)
    ps = 0
    t0 = time.perf_counter()
    for _ in range(n_steps):
        n = o.count(0) + o.count(1) + o.count(2)
        o.step(1)
        ps += n
    el = time.perf_counter() - t0
    o.close()
    return ps, el


def cpu_baseline_batched(n_steps=16):
    """The 64 sweep diodes as independent oracle processes over all host
    cores (a bounded number of steps each, from the same preload)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(cores, 64)) as pool:
        res = pool.map(_oracle_instance, [(i, n_steps) for i in range(64)], chunksize=1)
    wall = time.perf_counter() - t0
    ps = sum(r[0] for r in res)
    busy = sum(r[1] for r in res)
    return {"value": ps / busy * min(cores, 64), "unit": "particle-steps/s", "cores": min(cores, 64),
            "kind": "oracle",
            "sample": "64 sweep diodes, %d steps each from the preload, one process per core; "
                      "value = particle-steps / summed step time x cores (%.1f s wall incl. "
                      "start-up)" % (n_steps, wall)}


def run_batched(steps=10_000, warmup=200, tune_steps=400):
    """The 64-diode sweep for 10,000 steps: one batched handle (tuned by the
    autotuner on a copy of the job first) against the same diodes run one
    after another on their own handles with the default shape.  Results do
    not depend on the launch shape, so every diode's wall tallies must come
    out identical both ways."""
    import torch
    from paper_2605_07083_gb300 import pic
    from paper_2605_07083_gb300 import autotune as A
    ps, states = batched_workload(steps=steps)
    n_tot = sum(s[0].size for s in states)

    def make():
        h = pic.Diode(ps)
        for i, st in enumerate(states):
            h.inject(0, *st, instance=i)
        return h

    t0 = time.perf_counter()
    d = make()
    tuning = A.autotune(d, steps=tune_steps)
    d.close()
    del d
    tune_s = time.perf_counter() - t0
    d = make()
    A.apply(d, tuning)
    d.step(warmup)
    d.prepare(steps)
    d.synchronize()
    p0 = sum(d.diagnostics(i)["particles_pushed"] for i in range(len(ps)))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(d.stream)
    d.step(steps)
    e1.record(d.stream)
    e1.synchronize()
    ms_b = e0.elapsed_time(e1)
    diag_b = [d.diagnostics(i) for i in range(len(ps))]
    pushed_b = sum(x["particles_pushed"] for x in diag_b) - p0
    d.close()
    del d
    ms_seq, pushed_s, same = 0.0, 0, 0
    for i, (p, st) in enumerate(zip(ps, states)):
        s1 = pic.Diode(p)
        s1.inject(0, *st)
        s1.step(warmup)
        s1.prepare(steps)
        s1.synchronize()
        q0 = s1.diagnostics()["particles_pushed"]
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s1.stream)
        s1.step(steps)
        b.record(s1.stream)
        b.synchronize()
        ms_seq += a.elapsed_time(b)
        dg = s1.diagnostics()
        pushed_s += dg["particles_pushed"] - q0
        same += int(np.array_equal(dg["count"], diag_b[i]["count"])
                    and dg["emitted"] == diag_b[i]["emitted"]
                    and np.array_equal(dg["n_live"], diag_b[i]["n_live"]))
        s1.close()
    bf = np.array([x["backflow_ratio"] for x in diag_b], np.float64)
    gam = np.array([p["gamma_emit"] for p in ps], np.float64)
    ok = np.isfinite(bf)
    return {"instances": len(ps), "particles_initial": int(n_tot),
            "particles_final": int(sum(int(np.sum(x["n_live"])) for x in diag_b)),
            "steps": steps, "warmup": warmup,
            "ms_per_step_batched": ms_b / steps, "ms_per_step_sequential": ms_seq / steps,
            "speedup": ms_seq / ms_b,
            "value_batched": pushed_b / (ms_b * 1e-3), "value_sequential": pushed_s / (ms_seq * 1e-3),
            "unit": "particle-steps/s",
            "instances_with_identical_tallies": same,
            "launch": "one CUDA graph per %d steps, 3 kernels per step (push, mid, post) "
                      "over all 64 diodes" % A.graph_length(tuning["graph_steps"],
                                                            tuning["sort_period"]),
            "tuning": {k: tuning[k] for k in ("push_threads", "push_chunk", "sort_period",
                                              "graph_steps", "ms_per_step")},
            "autotune": {"trials": len(tuning["trials"]), "timed_steps_per_trial": tune_steps,
                         "seconds": tune_s,
                         "grid": "threads 128..384 step 32 x sort period {0,25,50,100,200} "
                                 "x graph steps {16,64,256} (rounded to whole sort periods)"},
            "backflow_ratio_window": {"min": float(bf[ok].min()) if ok.any() else None,
                                      "max": float(bf[ok].max()) if ok.any() else None,
                                      "corr_with_gamma": float(np.corrcoef(gam[ok], bf[ok])[0, 1])
                                      if ok.sum() > 2 else None},
            "workload": "64 He diodes: Gamma U[5,9]e19, gap U[1,5] mm (cells = gap/2.5 um), "
                        "n_He logU[1e21,1e22], 5e4-4e6 emitted e preloaded (log-uniform), 10 V"}


def run_small(steps=2000):
    """The 1 mm, 128-cell diode from an empty start (~2e4 emitted electrons
    in flight once filled): launch-latency-bound and L2-resident, so it
    carries no roofline claim."""
    import torch
    from paper_2605_07083_gb300 import pic
    p = W.single_diode_small(seed=1)
    d = pic.Diode(p)
    d.step(50)
    d.prepare(steps)
    d.synchronize()
    p0 = d.diagnostics()["particles_pushed"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(d.stream)
    d.step(steps)
    e1.record(d.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    dg = d.diagnostics()
    d.close()
    pushed = dg["particles_pushed"] - p0
    return {"workload": "He diode 1 mm, 128 cells, dt 1e-12 s, 10 V, empty start, steps 50-2050",
            "steps": steps, "ms_per_step": ms / steps, "value": pushed / (ms * 1e-3),
            "unit": "particle-steps/s", "particles_final": int(sum(dg["n_live"])),
            "note": "launch-latency-bound, L2-resident: no roofline claim"}


def cpu_baseline(p, state, budget_s=12.0):
    """The oracle as it stands, on the host, single thread: a bounded number of
    steps of the same preloaded production state."""
    from oracle import oracle as O
    o = O.Oracle(p)
    for sp in range(3):
        o.inject(sp, *state[sp])
    n = sum(o.count(s) for s in range(3))
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 > budget_s or steps >= 50:
            break
    el = time.perf_counter() - t0
    return {"value": n * steps / el, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": "full %d-particle production state, %d steps, single-threaded FP64 C++"
                      % (n, steps)}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import oracle as O
    O.build()
    p = workload()
    full = W.production_preload(p, seed=20)
    n_full = sum(full[s][0].size for s in range(3))
    # each step: the oracle advances a fixed random subsample of the state
    total_budget = 90.0
    per_step_particles = 2.0e7 * total_budget / max(args.steps + args.warmup, 1)
    frac = min(1.0, per_step_particles / n_full)
    rng = np.random.default_rng(5)
    sample = {}
    for sp in range(3):
        n = full[sp][0].size
        idx = np.sort(rng.choice(n, max(1, int(n * frac)), replace=False))
        sample[sp] = tuple(a[idx] for a in full[sp])
    o = O.Oracle(p)
    for sp in range(3):
        o.inject(sp, *sample[sp])
    for _ in range(args.warmup):
        o.step(1)
    done = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        done += sum(o.count(s) for s in range(3))
        o.step(1)
    el = time.perf_counter() - t0
    v = done / el
    return {"impl": "reference", "metric": "particle-steps/s", "value": v,
            "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": describe(p, n_full),
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "%.4f of the production state per step (%d particles)"
                                       % (frac, sum(sample[s][0].size for s in range(3)))},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-diode sweep and the small-diode line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
    out = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if out is not None:
        print(json.dumps(out))
    if world > 1 and args.impl == "ours":
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
