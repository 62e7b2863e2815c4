"""Every launch shape the autotuner can pick, against the FP64 oracle.

The tuner chooses, per workload, CTAs per replica (cluster 1, 2, 3, 4 or 8),
threads per atom (1, 2, 4 or 8 sub-lists), list cells per list radius (or
none: all pairs) and where the lists live (global or shared memory); the
results must
not depend on that choice beyond rounding.  One ensemble of three replicas of
864 atoms at T 0.7-2.0, skin 0.3 (several list rebuilds), uneven budgets
13 / 7 / 10: positions, velocities and energies after the budgets against the
oracle (FP64: the tolerances of the FP64 parity tests, and the rebuild
counts equal; mixed: the tolerances of the mixed MD test)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_0812_1633_gb300 import inputs

pytestmark = pytest.mark.gpu

N, SEED, SKIN = 864, 21, 0.3
TEMPS = inputs.geometric_ladder(0.7, 2.0, 3)
BUDGETS = [13, 7, 10]
SHAPES = list(itertools.product([1, 2, 3, 4, 8], [1, 2, 4, 8], [1, 2, 3], [-1, 1]))


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


@pytest.fixture(scope="module")
def reference():
    L = inputs.box_length(N)
    ens = O.Ensemble(N, L, TEMPS, SEED, skin=SKIN)
    ens.advance(BUDGETS)
    return ens


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_every_tunable_shape_matches_the_oracle(re, reference, prec):
    L = inputs.box_length(N)
    ran, refused = [], []
    for cl, at, cd, ls in SHAPES:
        want = dict(cluster=cl, atom_threads=at, cell_div=cd, lists_smem=ls)
        try:
            ctx = re.Context(N, L, 2.5, TEMPS, SEED, precision=prec, skin=SKIN, **want)
        except re.REError as e:
            assert e.code == re.RE_EINVAL, (want, str(e))
            refused.append(want)
            continue
        cfg = ctx.config()
        assert (cfg["cluster"], cfg["atom_threads"]) == (cl, at), (want, cfg)
        # a cell division whose cells cost more to visit than all pairs (here
        # 1: three cells a side; 3: 343 cells visited per atom) falls back to
        # all pairs, the tuner's cell_div 0
        assert cfg["cell_div"] in (cd, 0), (want, cfg)
        # lists asked for in shared memory stay in global memory when they do
        # not fit there
        assert cfg["lists_smem"] in ((0, 1) if ls > 0 else (0,)), (want, cfg)
        try:
            ctx.advance(BUDGETS)
        except re.REError as e:
            # a shape whose lists do not fit is refused at its first launch
            assert e.code == re.RE_EINVAL, (want, str(e))
            refused.append(want)
            ctx.close()
            continue
        x, v = ctx.get_state()
        U, K, H = ctx.energies()
        steps, rebuilds = ctx.counters()
        for k, r in enumerate(reference.reps):
            d = x[k * N:(k + 1) * N] - r.x
            d -= L * np.rint(d / L)
            if prec == "fp64":
                assert np.abs(d).max() < 1e-10, want
                assert np.abs(v[k * N:(k + 1) * N] - r.v).max() < 1e-10, want
                assert U[k] == pytest.approx(r.U, rel=1e-11), want
                assert H[k] == pytest.approx(r.H, rel=1e-11), want
            else:
                assert np.abs(d).max() < 1e-6, want
                assert abs(U[k] - r.U) / N < 1e-5, want
                assert abs(K[k] - r.K) / N < 1e-5, want
            assert steps[k] == BUDGETS[k]
            if prec == "fp64":
                assert rebuilds[k] == r.nrebuild, want
        ran.append(want)
        ctx.close()
    # the shapes the tuner considers for this workload all run
    assert len(ran) >= 60, (len(ran), refused)
