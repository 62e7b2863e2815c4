"""The FP64 oracle's legs of bench.py's precision study (host only; the
oracle is test infrastructure, so its legs live here):

    python tests/precision_oracle.py [steps] > precision_oracle.json

The same 16 replicas (the coldest of the 256-replica ladder T 0.75-1.8,
N = 4000, FCC start, seed 12345): the energy drift of H~ per atom per tau
for the two ends of the ladder without exchanges, and the exchange
acceptance per ladder pair with an attempt every 10 steps."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle as O  # noqa: E402
from paper_0812_1633_gb300 import inputs  # noqa: E402


def main():
    S = int(sys.argv[1]) if len(sys.argv) > 1 else 100000
    N, R, seed = bench.PREC_N, bench.PREC_R, bench.PREC_SEED
    L = inputs.box_length(N)
    temps = bench.precision_temps()
    out = {"workload": "as bench.py --study precision", "steps": S,
           "threads": os.cpu_count()}
    # drift: the two ends of the ladder, no exchanges
    ens = O.Ensemble(N, L, temps, seed)
    ends = np.zeros(R, np.int32)
    ends[[0, R - 1]] = 1
    t, H = [], []
    t0 = time.perf_counter()
    for c in range(S // 100):
        ens.advance(ends * 100)
        H.append([r.H for r in ens.reps])
        t.append((c + 1) * 100 * 0.005)
    sl = bench.drift_slopes(t, H, N)[[0, R - 1]]
    out["drift"] = {"replicas": [0, R - 1], "slopes": sl.tolist(),
                    "wall_s": time.perf_counter() - t0}
    print(json.dumps(out["drift"]), file=sys.stderr, flush=True)
    # exchanges every 10 steps, all 16 replicas
    ens = O.Ensemble(N, L, temps, seed)
    att = np.zeros(R - 1)
    acc = np.zeros(R - 1)
    t0 = time.perf_counter()
    for c in range(S // 10):
        ens.advance([10] * R)
        T = ens.temps()
        partner, ok = ens.exchange()
        order = np.argsort(T)
        for k in range(R - 1):
            a, b = order[k], order[k + 1]
            if partner[a] == b:
                att[k] += 1
                acc[k] += ok[a]
    out["exchange"] = {"acceptance_per_pair": (acc / np.maximum(att, 1)).tolist(),
                       "attempts_per_pair": att.tolist(), "wall_s": time.perf_counter() - t0}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
