"""Autotuner of the FFT plans: per grid size, the radix order and tile width of
the y/z passes and of the x passes, picked by timing the transform on the GPU
and cached as JSON.

Candidates are the ordered factorisations of the pass length into one to
three supported radices, with 2, 4, 8 or 16 sequences per tile; the library
refuses the plans its kernels cannot run (cwthf_set_fft_plan).  The y/z plan
is tuned first with the built-in x plan, then the x plan with the chosen y/z
plan; each candidate is timed as a whole cwthf_transform (best of `reps`
after one warm-up), and the built-in rule is kept unless a candidate beats it
by more than `margin`.
"""
from __future__ import annotations

import itertools
import json
import os
from pathlib import Path

RADICES = (2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 30, 32)
TILES = (2, 4, 8, 16)


def factorisations(n: int, max_stages: int = 3, radices=RADICES) -> list[tuple[int, ...]]:
    """Ordered factorisations of n into 1..max_stages factors from `radices`."""
    out = []
    for k in range(1, max_stages + 1):
        for combo in itertools.product(radices, repeat=k):
            prod = 1
            for r in combo:
                prod *= r
            if prod == n:
                out.append(combo)
    return out


def candidates(n: int, limit: int = 48) -> list[tuple[int, tuple[int, ...]]]:
    """(tile width, radices) candidates for a pass of length n: the
    factorisations with the largest smallest radix first (fewer stages and
    threads), at most `limit` of them, each with every tile width."""
    fs = sorted(factorisations(n), key=lambda f: (-min(f), len(f), f))[:limit]
    return [(c, f) for f in fs for c in TILES]


def default_cache() -> Path:
    return Path(os.environ.get("CWTHF_FFT_PLANS", Path.home() / ".cache" / "cwthf" / "fft_plans.json"))


def load(path=None) -> dict:
    p = Path(path) if path else default_cache()
    if not p.exists():
        return {}
    return {int(k): v for k, v in json.loads(p.read_text()).items()}


def save(plans: dict, path=None) -> Path:
    p = Path(path) if path else default_cache()
    p.parent.mkdir(parents=True, exist_ok=True)
    p.write_text(json.dumps({str(k): v for k, v in sorted(plans.items())}, indent=1) + "\n")
    return p


def apply(ctx, plans: dict):
    """Set the cached plans of every grid size on a context."""
    for ng, entry in plans.items():
        for which, key in ((0, "yz"), (1, "x")):
            if entry.get(key):
                c, rad = entry[key]
                ctx.set_fft_plan(int(ng), which, c, rad)


def tune_size(ctx, ng: int, reps: int = 5, margin: float = 0.02, box: float | None = None) -> dict:
    """Best (tile width, radices) for the y/z and x passes of grid size ng on
    this context (whose max_ng must be >= ng), by timing cwthf_transform."""
    import torch
    L = box or ng * 0.78125
    g = torch.randint(0, 1 << 34, (ng, ng, ng), dtype=torch.int64, device=ctx.device)
    out = torch.empty((ng, ng, ng), dtype=torch.float32, device=ctx.device)
    s = torch.cuda.current_stream(ctx.device)

    def timed():
        ctx.transform(g, L, 2.0, cwt=out, stream=s)
        ctx.check(what=f"autotune {ng}")
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ctx.transform(g, L, 2.0, cwt=out, stream=s)
            e1.record(s)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    result = {"ng": ng}
    for which, key, n in ((0, "yz", ng), (1, "x", ng // 2)):
        ctx.set_fft_plan(ng, which)  # built-in rule
        t0 = timed()
        best_t, best = t0, None
        tried = 0
        for c, rad in candidates(n):
            if not ctx.set_fft_plan(ng, which, c, rad):
                continue
            tried += 1
            t = timed()
            if t < best_t:
                best_t, best = t, [c, list(rad)]
        if best is not None and best_t < t0 * (1.0 - margin):
            ctx.set_fft_plan(ng, which, best[0], best[1])
            result[key] = best
        else:
            ctx.set_fft_plan(ng, which)
            result[key] = None  # the built-in rule stays
        result[f"{key}_ms"] = [t0, min(best_t, t0)]
        result[f"{key}_tried"] = tried
    del g, out
    return result


def tune(device, sizes, reps: int = 5, path=None) -> dict:
    """Tune every grid size in `sizes`, save and return {ng: entry}."""
    from . import _lib
    ctx = _lib.Context(device, max_ng=max(sizes), max_np=1, max_scales=1)
    try:
        plans = {ng: tune_size(ctx, ng, reps) for ng in sorted(set(sizes))}
    finally:
        ctx.close()
    save(plans, path)
    return plans
