"""Launch-option autotuner for qsg_sweep.

Every option of ``qsg_set_option`` that shapes the sweep launch (tau chunk per
work unit, kernel form, persistent multi-group launch, CUDA-graph batch, work
units per block of the generic kernel, slots swept in shorter chunks at the
end of a launch) leaves the sampled bits unchanged, so the choice is purely
one of speed.  The tuner times each valid combination of the first four on the
caller's own context with CUDA events on the context's stream, then (when a
group runs the generic kernel) the units per block, then the tail lengths with
the best launch of each of the four fastest chunk lengths, keeps the fastest,
and caches the choice in a JSON file keyed by the group shapes, the device
name and the library build.

Tuning runs real sweeps, so the spins and counters of every group are saved
to the host first and put back afterwards: a tuned run samples exactly what an
untuned one does.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os
from dataclasses import asdict

from . import qsg as Q

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")

# option id -> name used in the cache and in reports
_NAMES = {Q.OPT_CHUNK: "chunk", Q.OPT_WAVEFRONT_VARIANT: "variant", Q.OPT_PERSISTENT: "persistent",
          Q.OPT_GRAPH: "graph", Q.OPT_TAIL: "tail", Q.OPT_UNITS_PER_BLOCK: "upb"}
DEFAULTS = {"chunk": 0, "variant": 0, "persistent": 0, "graph": 0, "tail": 0, "upb": 0}
UPB = [1, 2, 4, 8, 16]  # units per block of the generic kernel, tried after the first stage
COMPILED_L = (8, 12, 16, 20, 24)  # lattice sizes with a compiled one-unit-per-block kernel
TAILS = [0, 16, 24, 28, 32, 40, 48, 64]  # slots swept in quarter-length chunks, tried after the rest
VARIANTS = [0, 1, 2, 3]  # forms of the wavefront kernel (QSG_OPT_WAVEFRONT_VARIANT)


def _library_id() -> str:
    h = hashlib.sha256()
    with open(Q._LIB_PATH, "rb") as f:
        for block in iter(lambda: f.read(1 << 20), b""):
            h.update(block)
    return h.hexdigest()[:16]


def cache_key(shapes, device_name: str) -> str:
    desc = json.dumps([asdict(s) for s in shapes], sort_keys=True)
    return hashlib.sha256(f"{desc}|{device_name}|{_library_id()}".encode()).hexdigest()[:24]


def candidate_chunks(shapes, largest=512):
    """Tau planes per work unit that every group accepts: multiples of 16
    dividing every L_tau, plus 0 (the library's own choice)."""
    out = [0]
    c = 16
    while c <= min(largest, min(s.Ltau for s in shapes)):
        if all(s.Ltau % c == 0 for s in shapes):
            out.append(c)
        c += 16
    return out


def candidates(shapes, sweeps_per_call, space=None):
    """Launch options of the first stage; `space` may restrict any of
    "chunk", "variant", "persistent", "graph" (and "upb", the later stage's
    units per block) to a list of values."""
    space = space or {}
    chunks = [c for c in candidate_chunks(shapes) if c in space.get("chunk", [c])]
    persistent = [1, 2, 3] if len(shapes) > 1 else [1]
    persistent = [p for p in persistent if p in space.get("persistent", [p])]
    graph = [0, sweeps_per_call] if sweeps_per_call > 1 else [0]
    graph = [g for g in graph if g in space.get("graph", [g])]
    variants = [v for v in VARIANTS if v in space.get("variant", [v])]
    for chunk, variant, pers, gr in itertools.product(chunks, variants, persistent, graph):
        yield {"chunk": chunk, "variant": variant, "persistent": pers, "graph": gr, "tail": 0, "upb": 0}


def uses_generic_kernel(shapes, variant):
    """True if some group is swept by the generic wavefront kernel (a lattice
    size without a compiled kernel, or the generic form asked for)."""
    return variant == 2 or any(s.L not in COMPILED_L for s in shapes)


def apply(ctx, choice: dict) -> None:
    """Set every tuned option on ctx (raises QSGError if one is invalid)."""
    ctx.qsg_set_option(Q.OPT_GRAPH, 0)  # the chunk check depends on it; set last
    ctx.qsg_set_option(Q.OPT_CHUNK, int(choice["chunk"]))
    ctx.qsg_set_option(Q.OPT_WAVEFRONT_VARIANT, int(choice["variant"]))
    ctx.qsg_set_option(Q.OPT_PERSISTENT, int(choice["persistent"]))
    ctx.qsg_set_option(Q.OPT_TAIL, int(choice.get("tail", 0)))
    ctx.qsg_set_option(Q.OPT_UNITS_PER_BLOCK, int(choice.get("upb", 0)))
    ctx.qsg_set_option(Q.OPT_GRAPH, int(choice["graph"]))


def _time_call(ctx, n_sweeps, reps):
    import torch
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(ctx.stream):
        ctx.qsg_sweep(n_sweeps)  # warm-up: graph capture, first-use attribute setup
        torch.cuda.synchronize(ctx.device)
        best = float("inf")
        for _ in range(reps):
            start.record(ctx.stream)
            ctx.qsg_sweep(n_sweeps)
            stop.record(ctx.stream)
            stop.synchronize()
            best = min(best, start.elapsed_time(stop) / n_sweeps)
    return best


def tune(ctx, sweeps_per_call=10, reps=3, cache_path=DEFAULT_CACHE, use_cache=True, verbose=False, space=None):
    """Choose the fastest sweep launch options for ctx, apply them, and return
    ``{"options": {...}, "ms_per_sweep": t, "cached": bool, "table": [...]}``.

    ``sweeps_per_call`` is the number of sweeps the caller passes to one
    qsg_sweep call (the sweeps between tempering steps); it is also the graph
    batch tried.  Spins and counters are restored before returning.
    """
    import torch
    dev_name = torch.cuda.get_device_name(ctx.device)
    key = cache_key(ctx.shapes, dev_name) + f"|{sweeps_per_call}" + (
        "|" + json.dumps(space, sort_keys=True) if space else "")
    cache = {}
    if use_cache and cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        entry = cache[key]
        apply(ctx, entry["options"])
        return {"options": entry["options"], "ms_per_sweep": entry["ms_per_sweep"], "cached": True, "table": []}

    spins = [ctx.qsg_get_spins(g) for g in range(len(ctx.shapes))]
    counters = ctx.qsg_get_counters()
    table = []
    try:
        for cand in candidates(ctx.shapes, sweeps_per_call, space):
            try:
                apply(ctx, cand)
            except Q.QSGError:
                continue
            t = _time_call(ctx, sweeps_per_call, reps)
            table.append((t, cand))
            if verbose:
                print(f"  {cand} {t:.4f} ms/sweep", flush=True)
        # units per block of the generic kernel, with the best launch so far
        if table:
            t0, first = min(table, key=lambda tc: tc[0])
            if uses_generic_kernel(ctx.shapes, first["variant"]):
                for upb in [u for u in UPB if u in (space or {}).get("upb", UPB)]:
                    cand = dict(first, upb=upb)
                    try:
                        apply(ctx, cand)
                    except Q.QSGError:
                        continue
                    t = _time_call(ctx, sweeps_per_call, reps)
                    table.append((t, cand))
                    if verbose:
                        print(f"  {cand} {t:.4f} ms/sweep", flush=True)
        # the tail lengths with the best launch of each chunk length (a longer
        # chunk that fills the last wave badly without a tail can win with one)
        best_per_chunk = {}
        for t, cand in table:
            c = cand["chunk"]
            if c not in best_per_chunk or t < best_per_chunk[c][0]:
                best_per_chunk[c] = (t, cand)
        for _, first in sorted(best_per_chunk.values(), key=lambda tc: tc[0])[:4]:
            for tail in TAILS[1:]:
                cand = dict(first, tail=tail)
                try:
                    apply(ctx, cand)
                except Q.QSGError:
                    continue
                t = _time_call(ctx, sweeps_per_call, reps)
                table.append((t, cand))
                if verbose:
                    print(f"  {cand} {t:.4f} ms/sweep", flush=True)
    finally:
        for g, s in enumerate(spins):
            ctx.qsg_set_spins(g, s)
        ctx.qsg_set_counters(counters[0], counters[1], counters[2])
    if not table:
        apply(ctx, DEFAULTS)
        return {"options": dict(DEFAULTS), "ms_per_sweep": None, "cached": False, "table": []}
    t_best, best = min(table, key=lambda tc: tc[0])
    apply(ctx, best)
    if cache_path:
        cache[key] = {"options": best, "ms_per_sweep": t_best, "device": dev_name,
                      "shapes": [asdict(s) for s in ctx.shapes]}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return {"options": best, "ms_per_sweep": t_best, "cached": False, "table": table}
