"""A ladder sharded over two processes (gloo on CPU, 127.0.0.1).  Each rank
holds half of an 8-member ladder; the local replicas are oracle replicas (test
stand-ins for a GPU context) and the decisions come from the oracle's exchange
(the same definition as the library's kernel).  Checked: the sharded run equals
one unsharded ensemble bit for bit; a late message changes nothing; a dropped
message and a missing rank are detected on the host and change no state."""
import ctypes as C
import os
import socket
import sys
import time
from datetime import timedelta

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, R, SEED, NX, CYCLES, D = 32, 8, 2024, 15, 5, 2
TEMPS = list(0.8 * 1.06 ** np.arange(R))
LAMS = list(1.0 - 0.03 * np.arange(R))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def box():
    return (N / 0.8442) ** (1.0 / 3.0) * 1.3


class OracleShard:
    """Members [offset, offset + n) of the ladder as oracle replicas."""

    def __init__(self, offset, n):
        import oracle as O
        self.O = O
        self.reps = [O.Replica(N, box(), TEMPS[g], SEED, g, lam=LAMS[g])
                     for g in range(offset, offset + n)]
        self.arr = (C.POINTER(O.Rep) * n)(*[C.pointer(r.rep) for r in self.reps])

    def advance(self, steps):
        for r in self.reps:
            r.steps(steps)

    def params(self):
        return (np.array([r.T for r in self.reps]), np.array([r.lam for r in self.reps]),
                np.array([r.U for r in self.reps]))

    def apply(self, T, lam, vs, us):
        dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(
            C.POINTER(C.c_double))
        self.O.lib().orc_apply_exchange_h(self.arr, len(self.reps), dp(T), dp(lam), dp(vs), dp(us))


def oracle_decide(T, lam, U, seed, attempt, mode, distance):
    import oracle as O
    Tn, ln, p, a, vs, us, _ = O.exchange_h(T, lam, U, seed, attempt, mode, distance)
    return Tn, ln, p, a, vs, us


def _worker(rank, ws, port, scenario, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_0812_1633_gb300.sharded import ExchangeFailed, ShardedLadder, torch_gather
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=timedelta(seconds=3))
    n = R // ws
    shard = OracleShard(rank * n, n)
    lad = ShardedLadder(shard, rank * n, R, SEED, 0, D, decide=oracle_decide,
                        gather=torch_gather())
    res = {"pairs": [], "error": None, "failed_at": None}
    for c in range(CYCLES):
        shard.advance(NX)
        if scenario == "late" and rank == 1 and c == 2:
            time.sleep(1.0)
        if scenario == "dropped" and rank == 1 and c == 2:
            lad.attempt += 1          # this rank's message for attempt 2 is lost
            continue
        if scenario == "missing" and rank == 1 and c == 2:
            time.sleep(6.0)           # never joins the collective within the timeout
            break
        before = shard.params()
        try:
            p, a = lad.exchange()
        except ExchangeFailed as e:
            after = shard.params()
            res["error"] = str(e)
            res["failed_at"] = c
            res["unchanged"] = all(np.array_equal(x, y) for x, y in zip(before, after))
            break
        res["pairs"].append((p.tolist(), a.tolist()))
    T, lam, U = shard.params()
    res["T"], res["lam"], res["U"] = T.tolist(), lam.tolist(), U.tolist()
    res["x"] = [r.x.copy() for r in shard.reps]
    out[rank] = res
    if scenario in ("normal", "late"):
        dist.barrier()
        dist.destroy_process_group()


def run(scenario):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, port, scenario, out), nprocs=ws, join=True)
        return dict(out)


def reference():
    import oracle as O
    ens = O.Ensemble(N, box(), TEMPS, SEED, lams=LAMS, distance=D)
    pairs = []
    for c in range(CYCLES):
        ens.advance([NX] * R)
        p, a = ens.exchange()
        pairs.append((p.tolist(), a.tolist()))
    return ens, pairs


@pytest.mark.parametrize("scenario", ["normal", "late"])
def test_sharded_ladder_equals_one_ensemble(scenario):
    res = run(scenario)
    ens, pairs = reference()
    for rank in (0, 1):
        assert res[rank]["error"] is None
        assert res[rank]["pairs"] == pairs         # every rank sees the whole ladder's decisions
        for k, x in enumerate(res[rank]["x"]):
            r = ens.reps[rank * (R // 2) + k]
            assert np.array_equal(x, r.x)
        assert res[rank]["T"] == ens.temps()[rank * 4:(rank + 1) * 4].tolist()
        assert res[rank]["lam"] == ens.lams()[rank * 4:(rank + 1) * 4].tolist()
    assert sum(1 for p, a in pairs for v in a if v) > 0   # some swaps happened


def test_dropped_message_is_detected_on_every_rank():
    res = run("dropped")
    # rank 0 sends attempt 2, rank 1 attempt 3: both reject the gathered ladder
    assert res[0]["failed_at"] == 2 and "attempts [2, 3]" in res[0]["error"]
    assert res[1]["failed_at"] == 3 and "attempts [2, 3]" in res[1]["error"]
    assert res[0]["unchanged"] and res[1]["unchanged"]
    assert len(res[0]["pairs"]) == 2


def test_missing_rank_times_out_without_changing_state():
    t0 = time.time()
    res = run("missing")
    assert res[0]["failed_at"] == 2 and "did not arrive" in res[0]["error"]
    assert res[0]["unchanged"]
    assert time.time() - t0 < 60
