"""Parity at the full workload sizes, in the launch shapes the benchmark
times.  Every replica of the ladder runs on the GPU; a sample of them is rerun
one by one by the FP64 oracle from the same lattice, seed and random streams
and compared (positions, potential and kinetic energy, within the mixed
path's tolerances); the exchange decisions over the whole ladder are compared
bit for bit with the oracle's exchange rule (Implementation section) applied
to the GPU's energies; the sampled replicas then take their exchange result
and run a second stretch, compared again (the velocity rescaling at full size).
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_0812_1633_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def re():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0812_1633_gb300 import build
    build.build()
    import paper_0812_1633_gb300 as m
    m.lib()
    return m


# name: (N, R, T_min, T_max, skin, steps per stretch, launch shape, sampled replicas)
WORKLOADS = {
    # the benchmark: 2-CTA clusters of 864 threads, 2 lanes per atom, lists in global memory
    "64x864": (864, 64, 0.7, 2.0, 0.3, 10,
               dict(cluster=2, atom_threads=2, cell_div=2, lists_smem=0), [0, 21, 42, 63]),
    "256x4000": (4000, 256, 0.75, 1.8, 0.5, 10, dict(cluster=4, atom_threads=1), [0, 128, 255]),
    "1024x2048": (2048, 1024, 0.7, 3.0, 0.5, 1, dict(cluster=2, atom_threads=1),
                  [0, 511, 1023]),
}


def compare(x, U, K, reps, sample, N, L):
    for k in sample:
        r = reps[k]
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < 1e-6, (k, np.abs(d).max())
        assert abs(U[k] - r.U) / N < 1e-5, (k, U[k], r.U)
        assert abs(K[k] - r.K) / N < 1e-5, (k, K[k], r.K)


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_full_size_sampled_replicas_match_oracle(re, name):
    N, R, t0, t1, skin, nsteps, launch, sample = WORKLOADS[name]
    seed = 2024
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(t0, t1, R)
    ctx = re.Context(N, L, 2.5, temps, seed, skin=skin, precision="mixed", **launch)
    cfg = ctx.config()
    assert cfg["cluster"] == launch["cluster"] and cfg["atom_threads"] == launch["atom_threads"]
    reps = {k: O.Replica(N, L, float(temps[k]), seed, k, skin=skin) for k in sample}

    ctx.advance(nsteps)
    for r in reps.values():
        r.steps(nsteps)
    x, _ = ctx.get_state()
    U, K, _ = ctx.energies()
    compare(x, U, K, reps, sample, N, L)
    steps, _ = ctx.counters()
    assert np.all(steps == nsteps)

    # the whole ladder's decisions from the GPU's energies, bit for bit
    T = ctx.temps()
    To, po, ao, vo, n = O.exchange(T, U, seed, 0, 0)
    pg, ag = ctx.exchange(outputs=True)
    assert np.array_equal(pg, po) and np.array_equal(ag, ao)
    assert np.array_equal(ctx.temps(), To)
    assert n == int(ao.sum()) // 2

    # the sampled replicas take their result (new T, velocities scaled) and run on
    for k in sample:
        arr = (C.POINTER(O.Rep) * 1)(C.pointer(reps[k].rep))
        one = lambda a: np.ascontiguousarray([a], dtype=np.float64)
        Tk, lk, vk, uk = one(To[k]), one(1.0), one(vo[k]), one(1.0)
        O.lib().orc_apply_exchange_h(arr, 1, O._dp(Tk), O._dp(lk), O._dp(vk), O._dp(uk))
        assert reps[k].T == To[k]
    ctx.advance(nsteps)
    for r in reps.values():
        r.steps(nsteps)
    x, _ = ctx.get_state()
    U, K, _ = ctx.energies()
    compare(x, U, K, reps, sample, N, L)
    ctx.close()
