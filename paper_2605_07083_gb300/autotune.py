"""Launch-shape autotuner for a PIC handle.

Times a few real steps (CUDA events around every kernel, pic_profile_steps)
for each candidate shape -- threads per block of the particle kernels, a cap
on resident blocks per SM, and the period of the counting sort -- and leaves
the handle on the fastest.  The steps it runs are ordinary simulation steps.
"""
from __future__ import annotations


def autotune(diode, steps: int = 20, threads=(128, 256), blocks_per_sm=(0,),
             sort_periods=(0, 50)) -> dict:
    """Return {"push_threads", "push_blocks_per_sm", "sort_period", "ms_per_step",
    "trials"} for the best shape and apply it to ``diode``."""
    trials = []
    for t in threads:
        for b in blocks_per_sm:
            for s in sort_periods:
                diode.tune(push_threads=t, push_blocks_per_sm=b, sort_period=s if s else -1)
                diode.profile(max(2, steps // 4))              # settle
                prof = diode.profile(steps)
                ms = prof["ms_total"] / max(prof["steps"], 1)
                trials.append({"push_threads": t, "push_blocks_per_sm": b, "sort_period": s,
                               "ms_per_step": ms})
    best = min(trials, key=lambda r: r["ms_per_step"])
    diode.tune(push_threads=best["push_threads"], push_blocks_per_sm=best["push_blocks_per_sm"],
               sort_period=best["sort_period"] if best["sort_period"] else -1)
    out = dict(best)
    out["trials"] = trials
    return out
