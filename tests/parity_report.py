"""Measured error of every GPU result against the FP64 oracle, as one JSON
report (run on a machine with the GPU; test infrastructure, not a test):

    python tests/parity_report.py > parity.json

Each entry states the quantity compared, the workload and the largest error
seen; the tolerances the tests enforce are in the test files."""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle as O  # noqa: E402
from paper_0812_1633_gb300 import inputs  # noqa: E402


def rms(f):
    return math.sqrt((f ** 2).sum(1).mean())


def state_err(ctx, ens, N, L):
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    dx = dv = du = dk = dh = 0.0
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        dx = max(dx, float(np.abs(d).max()))
        dv = max(dv, float(np.abs(v[k * N:(k + 1) * N] - r.v).max()))
        du = max(du, abs(U[k] - r.U) / abs(r.U))
        dk = max(dk, abs(K[k] - r.K) / abs(r.K))
        dh = max(dh, abs(H[k] - r.H) / abs(r.H))
    return {"max_abs_dx": dx, "max_abs_dv": dv, "max_rel_dU": du, "max_rel_dK": dk,
            "max_rel_dH": dh}


def main():
    import torch
    import paper_0812_1633_gb300 as re
    from paper_0812_1633_gb300 import build
    build.build()
    out = {}

    # forces and potential energy at one configuration (after 50 steps from the
    # lattice); the mixed path at the skins the tuner chooses from, whose longer
    # lists give longer FP32 sums per sub-list, in its default launch shape
    rows = []
    # (and with one thread per atom: one FP32 sum over the whole list, the
    # shape the tuner picks for the 256 x 4000 and 1024 x 2048 workloads)
    cases = ([("fp64", 0.5, 0)] + [("mixed", sk, 0) for sk in (0.2, 0.3, 0.5, 0.6)] +
             [("mixed", sk, 1) for sk in (0.3, 0.6)])
    for prec, skin, at in cases:
        for N in (256, 864, 2048, 4000):
            L = inputs.box_length(N)
            kw = dict(atom_threads=1, cluster=4 if N > 1024 else 1) if at else {}
            ctx = re.Context(N, L, 2.5, [0.8, 1.2], 7, precision=prec, skin=skin, **kw)
            ctx.advance(50)
            x, _ = ctx.get_state()
            f = ctx.forces()
            U, _, _ = ctx.energies()
            ef = eu = eun = 0.0
            for k in range(2):
                fo, Uo = O.forces_brute(x[k * N:(k + 1) * N], L)
                ef = max(ef, float(np.sqrt(((f[k * N:(k + 1) * N] - fo) ** 2).sum(1)).max()) / rms(fo))
                eu = max(eu, abs(U[k] - Uo) / abs(Uo))
                eun = max(eun, abs(U[k] - Uo) / N)
            cfg = ctx.config()
            rows.append({"precision": prec, "skin": skin, "N": N,
                         "threads_per_atom": cfg["atom_threads"],
                         "list_entries_per_atom": 0.8442 * 4 / 3 * math.pi * (2.5 + skin) ** 3,
                         "max_force_err_over_rms": ef, "rel_U_err": eu, "U_err_per_atom": eun})
            ctx.close()
    out["forces_and_U"] = rows

    # FP64 MD steps, both paths
    N = 500
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, 3)
    md = {}
    for path in ("batched", "plain"):
        ctx = re.Context(N, L, 2.5, temps, 11, precision="fp64", path=path)
        ens = O.Ensemble(N, L, temps, 11)
        ctx.advance([7, 30, 0])
        ens.advance([7, 30, 0])
        md[path] = state_err(ctx, ens, N, L)
    out["fp64_md_3x500_budgets_7_30_0"] = md
    # mixed MD steps
    N = 864
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, [0.7, 2.0], 4, skin=0.3)
    ens = O.Ensemble(N, L, [0.7, 2.0], 4, skin=0.3)
    ctx.advance([10, 10])
    ens.advance([10, 10])
    e = state_err(ctx, ens, N, L)
    U, K, _ = ctx.energies()
    e["max_dU_per_atom"] = max(abs(U[k] - r.U) / N for k, r in enumerate(ens.reps))
    e["max_dK_per_atom"] = max(abs(K[k] - r.K) / N for k, r in enumerate(ens.reps))
    out["mixed_md_2x864_10_steps"] = e

    # exchange decisions
    mism = 0
    cases = 0
    vmax = 0.0
    for R in (2, 7, 64, 1024, 4096):
        for mode in (0, 1):
            for d in (1, 2, 3):
                for seed in range(3):
                    T, U = inputs.random_temps_energies(R, seed + 100 * R, u_sd=5.0)
                    lam = np.random.default_rng(seed).uniform(0.7, 1.3, R) if d > 1 else None
                    for att in (0, 1, 17):
                        To, lo, po, ao, vo, uo, _ = O.exchange_h(T, lam, U, 1234 + seed, att, mode, d)
                        cu = lambda a: torch.tensor(a, device="cuda")
                        Tg, lg, pg, ag, vg, ug = re.exchange_device_h(
                            cu(T), None if lam is None else cu(lam), cu(U), 1234 + seed, att, mode, d)
                        cases += 1
                        ok = (np.array_equal(pg.cpu().numpy(), po) and np.array_equal(ag.cpu().numpy(), ao)
                              and np.array_equal(Tg.cpu().numpy(), To))
                        mism += 0 if ok else 1
                        vmax = max(vmax, float(np.abs(vg.cpu().numpy() / vo - 1).max()))
    out["exchange_decisions"] = {"attempts": cases, "mismatched": mism, "max_rel_vscale_err": vmax,
                                 "replicas": [2, 7, 64, 1024, 4096], "distances": [1, 2, 3]}

    # a replica-exchange run and the free-running scheme, FP64
    N, R = 256, 8
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, 12345, precision="fp64")
    ens = O.Ensemble(N, L, temps, 12345)
    dec = 0
    for c in range(4):
        ctx.advance(100)
        ens.advance([100] * R)
        pg, ag = ctx.exchange(outputs=True)
        po, ao = ens.exchange()
        dec += int(not (np.array_equal(pg, po) and np.array_equal(ag, ao)))
    out["re_run_8x256_fp64_4_cycles"] = dict(state_err(ctx, ens, N, L), mismatched_attempts=dec)
    ctx = re.Context(N, L, 2.5, temps, 41, precision="fp64")
    ens = O.Ensemble(N, L, temps, 41)
    steps, T, partner, acc = ctx.run_free(12, 10, log=True)
    prev = np.zeros(R, np.int64)
    dec = 0
    for k in range(12):
        ens.advance([int(s) for s in steps[k] - prev])
        po, ao = ens.exchange()
        dec += int(not (np.array_equal(partner[k], po) and np.array_equal(acc[k].astype(bool), ao.astype(bool))))
        prev = steps[k].copy()
    out["free_running_8x256_fp64_12_attempts"] = dict(state_err(ctx, ens, N, L), mismatched_attempts=dec)

    # the oracle's energy drift on the drift study's systems (common window)
    N, R, steps, chunk, dt = 4000, 8, 4000, 100, 0.005
    L = inputs.box_length(N)
    ens = O.Ensemble(N, L, inputs.geometric_ladder(0.75, 1.8, R), 12345)
    t, H = [], []
    t0 = time.perf_counter()
    for c in range(steps // chunk):
        ens.advance([chunk] * R)
        H.append([r.H for r in ens.reps])
        t.append((c + 1) * chunk * dt)
    tt = np.asarray(t)
    Hn = np.asarray(H) / N
    tc = tt - tt.mean()
    sl = (tc[:, None] * (Hn - Hn.mean(0))).sum(0) / (tc * tc).sum()
    out["oracle_drift_8x4000_4000_steps"] = {"mean": float(sl.mean()), "max_abs": float(np.abs(sl).max()),
                                             "wall_s": time.perf_counter() - t0}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
