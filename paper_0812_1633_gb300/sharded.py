"""One replica ladder sharded over processes, one GPU each.

Every rank holds a contiguous block of the ladder's members in its own
context, created with ``id_offset`` = the global id of its first member so
that every replica keeps its own random streams.  One exchange attempt is the
paper's synchronous variant (Implementation section): each rank contributes
(attempt, global id, T, lam, U) of its members to one all-gather; every rank
computes the same decisions from the gathered ladder with the library's
stateless exchange kernel (identical inputs give identical outputs on every
GPU) and applies those of its own members with ``Context.apply_exchange``.

Failures are detected on the host between steps and change no state: a rank
whose message never comes makes the collective fail on the others after the
process group's timeout; a message that belongs to another attempt (a rank
that dropped one) or an incomplete ladder is rejected on every rank.
"""
from __future__ import annotations

import numpy as np


class ExchangeFailed(RuntimeError):
    """An exchange attempt could not be completed; no replica was changed."""


class ContextShard:
    """The local block of a ladder held by one context."""

    def __init__(self, ctx):
        self.ctx = ctx

    def advance(self, steps):
        self.ctx.advance(steps)

    def params(self):
        return self.ctx.temps(), self.ctx.lambdas(), self.ctx.energies()[0]

    def apply(self, T, lam, vscale, uscale):
        self.ctx.apply_exchange(T, vscale, lam, uscale)


def device_decide(T, lam, U, seed, attempt, parity_mode, distance):
    """The decisions of one attempt over the whole ladder, computed by the
    library's exchange kernel on this rank's GPU."""
    import torch
    from . import exchange_device_h
    cu = lambda a: torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")
    out = exchange_device_h(cu(T), cu(lam), cu(U), seed, attempt, parity_mode, distance)
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def torch_gather(group=None):
    """All-gather of every rank's message through torch.distributed (any
    backend; the process group's timeout bounds the wait)."""
    import torch.distributed as dist

    def gather(msg):
        out = [None] * dist.get_world_size(group)
        dist.all_gather_object(out, msg, group=group)
        return out
    return gather


class ShardedLadder:
    """Exchange attempts over a ladder of `n_total` members whose members
    [offset, offset + n_local) are held by `local` (a ContextShard or any object
    with advance/params/apply).  `decide` computes the decisions of a whole
    ladder (default: the library's device kernel); `gather` all-gathers the
    per-rank messages (default: torch.distributed)."""

    def __init__(self, local, offset, n_total, seed, parity_mode=0, distance=1, decide=None,
                 gather=None):
        self.local = local
        self.offset = int(offset)
        self.n_total = int(n_total)
        self.seed = int(seed)
        self.parity_mode = int(parity_mode)
        self.distance = int(distance)
        self.decide = decide or device_decide
        self.gather = gather or torch_gather()
        self.attempt = 0
        # attempts / acceptances per lower ladder position (as re_accept_stats)
        self.pair_att = np.zeros(max(self.n_total - 1, 1), np.int64)
        self.pair_acc = np.zeros(max(self.n_total - 1, 1), np.int64)

    def message(self):
        T, lam, U = self.local.params()
        n = len(T)
        m = np.empty((n, 5))
        m[:, 0] = self.attempt
        m[:, 1] = self.offset + np.arange(n)
        m[:, 2], m[:, 3], m[:, 4] = T, lam, U
        return m

    def exchange(self):
        """One attempt; returns (partner, accepted) over the whole ladder."""
        msg = self.message()
        try:
            parts = self.gather(msg)
        except Exception as e:  # a missing rank: the collective timed out or broke
            raise ExchangeFailed(f"attempt {self.attempt}: a rank's message did not arrive "
                                 f"({type(e).__name__}: {e})") from e
        m = np.concatenate(parts)
        ids = m[:, 1].astype(np.int64)
        if (len(m) != self.n_total or np.any(m[:, 0] != self.attempt)
                or not np.array_equal(np.sort(ids), np.arange(self.n_total))):
            got = sorted(set(m[:, 0].astype(np.int64).tolist()))
            raise ExchangeFailed(f"attempt {self.attempt}: messages of attempts {got} for "
                                 f"{len(m)} of {self.n_total} members")
        m = m[np.argsort(ids)]
        T, lam, U = m[:, 2], m[:, 3], m[:, 4]
        Tn, ln, partner, acc, vs, us = self.decide(T, lam, U, self.seed, self.attempt,
                                                   self.parity_mode, self.distance)
        mine = slice(self.offset, self.offset + len(msg))
        self.local.apply(Tn[mine], ln[mine], vs[mine], us[mine])
        # ladder statistics, the same on every rank
        key = T / lam
        rank = np.empty(self.n_total, np.int64)
        rank[np.lexsort((np.arange(self.n_total), key))] = np.arange(self.n_total)
        for a in range(self.n_total):
            b = int(partner[a])
            if b > a:
                q = min(rank[a], rank[b])
                self.pair_att[q] += 1
                self.pair_acc[q] += int(acc[a])
        self.attempt += 1
        return partner, acc
