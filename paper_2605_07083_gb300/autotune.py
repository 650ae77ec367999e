"""Launch-shape autotuner for a PIC handle.

Runs real simulation steps through pic_step -- the CUDA-graph path a caller
uses -- for every candidate shape on a grid of

  * threads per block of the particle kernels (128 ... 384 in steps of 32),
  * optionally the push's warp chunk (64 or 32 quads),
  * the period of the counting sort by cell (0 = never),
  * the number of steps captured in one CUDA graph,

times each with CUDA events on the handle's stream and leaves the handle on
the fastest.  A trial first settles (the push kernel's per-block shares adapt
to a new shape within a few steps, and the graphs of the shape are built
then), starts on a sort-aligned step, and times a whole number of sort
periods, so every trial pays for its sorts.  The steps it runs are ordinary
simulation steps: tune a copy of the job, or accept that the tuned handle has
advanced.
"""
from __future__ import annotations

THREADS = tuple(range(128, 385, 32))
SORT_PERIODS = (0, 25, 50, 100, 200)
GRAPH_STEPS = (16, 64, 256)
CHUNKS = (64,)


def graph_length(graph_steps: int, sort_period: int) -> int:
    """Steps in the longest graph the library captures for this pair: with a
    sort, graph_steps rounded up to a whole number of sort periods."""
    if sort_period <= 0:
        return graph_steps
    return -(-graph_steps // sort_period) * sort_period


def apply(diode, tuning: dict):
    """Set a tuning returned by autotune on a (fresh) handle."""
    diode.tune(push_threads=tuning["push_threads"],
               sort_period=tuning["sort_period"] if tuning["sort_period"] else -1,
               graph_steps=tuning["graph_steps"], push_chunk=tuning.get("push_chunk", 0))


def autotune(diode, steps: int = 400, settle: int = 50, threads=THREADS,
             sort_periods=SORT_PERIODS, graph_steps=GRAPH_STEPS, chunks=CHUNKS) -> dict:
    """Return {"push_threads", "push_chunk", "sort_period", "graph_steps",
    "ms_per_step", "trials"} for the fastest shape and apply it to
    ``diode``.

    ``steps`` must be a multiple of every sort period tried.  Graph lengths
    that a sort period rounds to the same length are tried once."""
    import torch
    for s in sort_periods:
        if s > 0 and steps % s:
            raise ValueError("steps=%d is not a multiple of sort period %d" % (steps, s))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    trials = []
    for t, cq in ((t, cq) for cq in chunks for t in threads):
        for s in sort_periods:
            seen = set()
            for g in graph_steps:
                glen = graph_length(g, s)
                if glen in seen:
                    continue
                seen.add(glen)
                tuning = {"push_threads": t, "push_chunk": cq, "sort_period": s,
                          "graph_steps": g}
                apply(diode, tuning)
                diode.step(settle)
                if s > 0:                      # start the timed steps on a sort
                    step = diode.diagnostics(0)["step"]
                    diode.step((s - step % s) % s)
                diode.prepare(steps)           # graphs captured outside the timing
                diode.synchronize()
                e0.record(diode.stream)
                diode.step(steps)
                e1.record(diode.stream)
                e1.synchronize()
                tuning["graph_length"] = glen
                tuning["ms_per_step"] = e0.elapsed_time(e1) / steps
                trials.append(tuning)
    best = min(trials, key=lambda r: r["ms_per_step"])
    apply(diode, best)
    out = dict(best)
    out["trials"] = trials
    out["timed_steps_per_trial"] = steps
    return out
