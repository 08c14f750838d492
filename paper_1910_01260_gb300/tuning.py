"""Cache of tuned launch plans for the batched reduced solve.

st_rom_solve_tune times every candidate plan (panel width, CTAs per SM, queue
order) on a batch and installs the fastest.  The result depends on the GPU,
the basis sizes, the precision and the batch's size mix, so it is cached in a
JSON file under a key built from those; load_or_tune installs the cached plan
when the key is present and tunes (and stores) otherwise.

File layout: {key: {"plan": {"panel", "ctas_per_sm", "order"},
                    "precision": int, "best_ms": float, "default_ms": float,
                    "n_candidates": int}}
"""
from __future__ import annotations

import json
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "solve_plans.json")


def plan_key(device: str, ns: int, nt: int, precision: int, refine: int, n_mu: int, sizes=None) -> str:
    """Cache key: device name, basis sizes, precision and refinement steps,
    batch size and the sorted set of (ns_p, nt_p) classes of the batch."""
    mix = "full" if sizes is None else ",".join(f"{a}x{b}" for a, b in sorted({tuple(map(int, x)) for x in sizes}))
    return f"{device}|ns={ns}|nt={nt}|precision={precision}|refine={refine}|n_mu={n_mu}|sizes={mix}"


def load(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(entries: dict, path: str = DEFAULT_CACHE) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)


def load_or_tune(model, key: str, precision: int, n_mu: int, theta, ns_nt, uhat, path: str = DEFAULT_CACHE,
                 reps: int = 2, write: bool = True) -> dict:
    """Install the cached plan for `key`, or tune on this batch and cache it.
    Returns the cache entry with "source" = "cache" or "tuned"."""
    entries = load(path)
    if key in entries:
        e = dict(entries[key])
        model.st_rom_solve_set_plan(precision, e["plan"])
        e["source"] = "cache"
        return e
    r = model.st_rom_solve_tune(n_mu, theta, ns_nt, uhat, reps=reps)
    e = {"plan": r["best"], "precision": int(precision), "best_ms": r["best_ms"], "default_ms": r["default_ms"],
         "n_candidates": r["n_candidates"]}
    if write:
        entries[key] = e
        try:
            store(entries, path)
        except OSError:
            pass
    out = dict(e)
    out["source"] = "tuned"
    out["candidates"] = r["candidates"]
    return out
