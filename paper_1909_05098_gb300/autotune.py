"""Autotuner for the time-loop launch knobs.

Every kernel family, tile size and element order gives bit-identical
temperatures (the per-node summation order is fixed by the input mesh), so
the choice is purely one of speed.  ``tune`` times each candidate on the live context with CUDA
events, restores the context's state afterwards (checkpoint API), applies the
fastest candidate and caches it under a signature of the mesh, precision and
device.
"""
from __future__ import annotations

import json
import os
import time

from . import fedfem as ff

CACHE = os.environ.get("FEDFEM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "fedfem_tune.json"))


def candidates(elem_type: int, precision: int):
    """(kernel, block, tile_nodes, blocks_per_sm); 0 = the library's default."""
    out = [(ff.KERNEL_PERSISTENT, 0, 0, 0)]
    sizes = (0, 128, 256, 384) if elem_type == ff.HEX8 else (0, 64, 96, 128, 192)
    staged = (0, 384, 512, 576, 640) if elem_type == ff.HEX8 else (0, 128, 192, 224, 256)
    staged1024 = (1024, 1280) if elem_type == ff.HEX8 else (512,)   # one block of 1024 threads per SM
    if precision == ff.FP64:
        sizes = tuple(s // 2 for s in sizes if s)[:2] + (0,)
        staged, staged1024 = (0,), ()
    out += [(ff.KERNEL_TILED, 0, b, 0) for b in sizes]
    out += [(ff.KERNEL_TILED_STAGED, 0, b, 0) for b in staged]
    out += [(ff.KERNEL_TILED_STAGED, 1024, b, 0) for b in staged1024]
    # replicated rows: at most one owned node per thread (512 or 256 threads)
    if elem_type == ff.HEX8:
        rep = [(0, b) for b in ((0, 448, 480, 512) if precision != ff.FP64 else (0, 256))]
        rep += [(256, b) for b in ((224, 256) if precision != ff.FP64 else (128,))]
    else:
        rep = [(256, b) for b in (0, 96, 128, 192)]
    out += [(ff.KERNEL_TILED_REP, blk, b, 0) for blk, b in rep]
    return out


def variant(solver) -> str:
    """The options of a solver's problem that change which kernel builds run
    (and so which configuration is fastest, or allowed at all)."""
    p = getattr(solver, "problem", None)
    parts = []
    if p is not None:
        if getattr(getattr(p, "material", None), "table", None) is not None:
            parts.append("table")
        if getattr(p, "regions", None) is not None:
            parts.append(f"regions{len(p.region_materials)}")
        if getattr(p, "hex_rule", "one-point") != "one-point":
            parts.append("hex" + getattr(p, "hex_rule"))
        if getattr(p, "lumping", "element") != "element":
            parts.append("uniform")
        if len(getattr(p, "schedule_factor", ())):
            parts.append("schedule")
    if getattr(solver, "dose_model", False):
        parts.append("dose")
    if getattr(solver, "matrix_free", False):
        parts.append("mf")
    return "+".join(parts)


def signature(info: dict, device_name: str, variant_tag: str = "") -> str:
    return (f"{device_name}|nv{info['elem_type']}|p{info['precision']}|N{info['n_nodes']}|E{info['n_elems']}|"
            f"F{info['n_free']}|C{info['n_convective']}|o{info['order']}|b{info['algorithmic_bytes_per_step']}|"
            f"v{variant_tag}")


def _load_cache():
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _save_cache(d):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        json.dump(d, open(CACHE, "w"), indent=1)
    except Exception:
        pass


def tune(solver, dt: float, steps: int = 30, use_cache: bool = True, stream=None, verbose: bool = False) -> dict:
    """Pick the fastest launch configuration for ``solver`` (a fedfem.Solver)
    and apply it.  Returns {"kernel", "block", "tile_nodes", "blocks_per_sm", "us_per_step", "trials"}."""
    import torch
    ctx = solver.ctx
    info = ff.fedfem_get_info(ctx)
    sig = signature(info, torch.cuda.get_device_name(), variant(solver))
    cache = _load_cache() if use_cache else {}
    if sig in cache:
        best = cache[sig]
        ff.fedfem_set_tile(ctx, best["kernel"], best.get("block", 0), best["tile_nodes"], best["blocks_per_sm"])
        best = dict(best, cached=True)
        return best
    saved = ff.fedfem_get_state(ctx)
    s = stream if stream is not None else torch.cuda.current_stream()
    trials = []
    for kern, blk, B, bps in candidates(info["elem_type"], info["precision"]):
        try:
            t0 = time.perf_counter()
            ff.fedfem_set_tile(ctx, kern, blk, B, bps)
            ff.fedfem_step(ctx, dt, 3)            # builds tiles on first use, warms up
            ff.fedfem_sync(ctx)
            setup = time.perf_counter() - t0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ff.fedfem_step(ctx, dt, steps)
            e1.record(s)
            ff.fedfem_sync(ctx)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / steps
            trials.append({"kernel": kern, "block": blk, "tile_nodes": B, "blocks_per_sm": bps, "us_per_step": us,
                           "setup_s": setup})
            if verbose:
                print(f"tune: kernel {kern} block {blk} tile {B} bps {bps}: {us:.1f} us/step (setup {setup:.2f} s)")
        except ff.FedfemError as ex:
            trials.append({"kernel": kern, "block": blk, "tile_nodes": B, "blocks_per_sm": bps, "error": str(ex)})
        finally:
            ff.fedfem_set_state(ctx, saved)
    ok = [t for t in trials if "us_per_step" in t]
    best = min(ok, key=lambda t: t["us_per_step"])
    ff.fedfem_set_tile(ctx, best["kernel"], best["block"], best["tile_nodes"], best["blocks_per_sm"])
    result = {k: best[k] for k in ("kernel", "block", "tile_nodes", "blocks_per_sm", "us_per_step")}
    if use_cache:
        cache[sig] = result
        _save_cache(cache)
    return dict(result, trials=trials, cached=False)


def tune_order(make_solver, dt_of, orders=None, **kw):
    """The element (and node) order is fixed when a context is built, so it is
    tuned by building one solver per order: ``make_solver(order)`` returns a
    fedfem.Solver, ``dt_of(solver)`` the step to time with.  Each is tuned with
    ``tune(**kw)``; the fastest solver is kept (the others are closed) and
    returned with its result, which gains an "order" key and the trials of
    every order.  Results do not depend on the order (each node sums its
    loads in input element order), so the choice is one of speed."""
    if orders is None:
        orders = (ff.ORDER_MORTON, ff.ORDER_RCM)
    best, best_r, trials = None, None, []
    for order in orders:
        s = make_solver(order)
        try:
            r = tune(s, dt_of(s), **kw)
        except Exception:
            s.close()
            raise
        trials += [dict(t, order=order) for t in r.get("trials", [])]
        r = dict(r, order=order)
        if best is None or r["us_per_step"] < best_r["us_per_step"]:
            if best is not None:
                best.close()
            best, best_r = s, r
        else:
            s.close()
    best_r["trials"] = trials
    return best, best_r
