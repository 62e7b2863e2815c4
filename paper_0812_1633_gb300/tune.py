"""Choice of the neighbour-list skin by measurement.

The skin trades list length (every step scans rc + skin) against rebuild
frequency (a rebuild once some atom has moved more than half the skin,
Example section); the trajectories do not depend on it beyond summation order,
so a workload that does not fix it can take the fastest.  A context's list
capacity and layout follow from its skin, so each candidate gets a context of
its own: `make(skin)` builds it, its launch shape is autotuned, and the same
advance + exchange cycles are timed on each; the fastest context is kept,
restored to its state before the timed cycles, and the others are closed.
"""
from __future__ import annotations

import time

DEFAULT_SKINS = (0.2, 0.3, 0.4, 0.5, 0.6)


def _cycles(ctx, budgets, n):
    for c in range(n):
        ctx.advance(None if budgets is None else budgets[c % len(budgets)])
        ctx.exchange()


def choose_skin(make, candidates=DEFAULT_SKINS, cycles=20, budgets=None, warm=5, tune_steps=40,
                agree=None):
    """Returns (skin, context, {skin: ms per cycle}) for the fastest candidate.

    make(skin) -> a new Context; budgets: per-cycle step budgets (cycles x
    n_rep, reused cyclically) or None for the context's N_x.  Each candidate:
    autotune of the launch shape, a checkpoint of the fresh state (the
    autotuner restores the state it tuned on), `warm` untimed cycles, then
    `cycles` timed cycles (host clock around synchronised work).  agree(ms) ->
    ms, when given, turns a local time into one every process agrees on (the
    maximum over ranks), so that all ranks keep the same skin.  The kept
    context is restored from its checkpoint: its step and rebuild counters,
    trajectory and launch shape are those it had before the timed cycles, so
    a tuned workload starts where a fixed-skin one does."""
    best = None
    timings = {}
    for skin in candidates:
        ctx = make(float(skin))
        ctx.autotune(steps=tune_steps)
        ckpt = ctx.checkpoint()
        _cycles(ctx, budgets, warm)
        ctx.sync()
        t0 = time.perf_counter()
        _cycles(ctx, budgets, cycles)
        ctx.sync()
        ms = (time.perf_counter() - t0) / cycles * 1e3
        if agree is not None:
            ms = agree(ms)
        timings[float(skin)] = ms
        if best is None or ms < best[0]:
            if best is not None:
                best[2].close()
            best = (ms, float(skin), ctx, ckpt)
        else:
            ctx.close()
    _, skin, ctx, ckpt = best
    ctx.restore(ckpt)
    return skin, ctx, timings
