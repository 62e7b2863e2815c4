"""The temperature-diffusion analysis (Diffusion in temperature space, the
Fig. 1(a) analogue) end to end on the GPU against the FP64 oracle: the same
trajectory helpers bench.py's study uses record the temperature of every
replica after each attempt, in the synchronous scheme and in the free-running
asynchronous one; on the FP64 path the exchange decisions replay bit for bit,
so the temperature trajectories, the step counts and the diffusion
coefficient of ln T must equal the oracle's exactly."""
import numpy as np
import pytest

import bench
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


N, R, SEED, NX, A = 256, 8, 71, 5, 60


def setup(re):
    L = inputs.box_length(N)
    temps = inputs.paper_ladder(R, ratio=1.06)
    ctx = re.Context(N, L, 2.5, temps, SEED, precision="fp64", skin=0.3)
    ens = O.Ensemble(N, L, temps, SEED, skin=0.3)
    return ctx, ens


def test_diffusion_sync_matches_oracle(re):
    ctx, ens = setup(re)
    Tg, sg = bench.diffusion_sync_trajectory(ctx, NX, A)
    To, so = [], []
    for k in range(A):
        ens.advance([NX] * R)
        ens.exchange()
        To.append(ens.temps())
        so.append([r.step for r in ens.reps])
    To, so = np.array(To), np.array(so, dtype=np.float64)
    assert np.array_equal(Tg, To)
    assert np.array_equal(sg, so)
    # the ladder is explored: some replica's temperature changed
    assert (Tg != Tg[0]).any()
    assert bench.msd_diffusion(Tg, sg) == bench.msd_diffusion(To, so) > 0


def test_diffusion_async_matches_oracle(re):
    ctx, ens = setup(re)
    Tg, sg = bench.diffusion_async_trajectory(ctx, NX, A)
    To, so = [], []
    prev = np.zeros(R, np.int64)
    for k in range(A):
        made = sg[k].astype(np.int64) - prev
        assert made[k % R] == NX                    # the rotating master's own stride
        ens.advance([int(x) for x in made])
        ens.exchange()
        To.append(ens.temps())
        so.append([r.step for r in ens.reps])
        prev = sg[k].astype(np.int64)
    To, so = np.array(To), np.array(so, dtype=np.float64)
    assert np.array_equal(Tg, To)
    assert np.array_equal(sg, so)
    assert (Tg != Tg[0]).any()
    assert bench.msd_diffusion(Tg, sg) == bench.msd_diffusion(To, so) > 0
