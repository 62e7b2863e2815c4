"""Degenerate and boundary cases of the method through the context path,
against the oracle: a ladder of one replica (no pair to exchange), an odd
ladder (one member sits out every attempt), zero step budgets, a skin so small
that the lists are rebuilt almost every step, and a replica too large for the
batched kernel's thread-block clusters (refused before any launch)."""
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


def same_state(ctx, ens, N, L, xtol=1e-10, etol=1e-11):
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < xtol
        assert np.abs(v[k * N:(k + 1) * N] - r.v).max() < xtol
        assert U[k] == pytest.approx(r.U, rel=etol)
        assert K[k] == pytest.approx(r.K, rel=etol)
        assert H[k] == pytest.approx(r.H, rel=etol)


def test_single_replica_ladder(re):
    N, seed = 256, 5
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, [1.3], seed, precision="fp64")
    ens = O.Ensemble(N, L, [1.3], seed)
    for _ in range(3):
        ctx.advance([25])
        ens.advance([25])
        partner, acc = ctx.exchange(outputs=True)
        assert partner.tolist() == [-1] and acc.tolist() == [0]
        assert ctx.temps().tolist() == [1.3]
    same_state(ctx, ens, N, L)
    att, acc = ctx.accept_stats()
    assert att.size == 0 or att.sum() == 0
    ctx.close()


def test_odd_ladder_matches_oracle(re):
    N, R, seed = 256, 5, 21
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64")
    ens = O.Ensemble(N, L, temps, seed)
    for cyc in range(6):
        ctx.advance([20] * R)
        ens.advance([20] * R)
        pg, ag = ctx.exchange(outputs=True)
        po, ao = ens.exchange()
        assert np.array_equal(pg, po) and np.array_equal(ag, ao)
        assert (pg == -1).sum() == 1  # one member of an odd ladder sits out
        assert np.array_equal(ctx.temps(), ens.temps())
    same_state(ctx, ens, N, L, xtol=1e-9, etol=1e-9)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_zero_budgets_change_nothing(re, prec):
    N, R = 500, 3
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, inputs.geometric_ladder(0.7, 1.4, R), 9, precision=prec)
    ctx.advance([12, 3, 7])
    x0, v0 = ctx.get_state()
    e0 = ctx.energies()
    c0 = ctx.counters()
    for _ in range(3):
        ctx.advance([0, 0, 0])
    x1, v1 = ctx.get_state()
    e1 = ctx.energies()
    c1 = ctx.counters()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)
    for a, b in zip(e0 + c0, e1 + c1):
        assert np.array_equal(a, b)
    ctx.close()


@pytest.mark.parametrize("path", ["batched", "plain"])
def test_tiny_skin_rebuilds_match_oracle(re, path):
    """Skin 0.01: lists rebuilt every few steps; the rebuild decisions (counts)
    and the trajectory follow the oracle."""
    N, R, seed, skin = 256, 2, 13, 0.01
    L = inputs.box_length(N)
    temps = [0.9, 1.8]
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", path=path, skin=skin)
    ens = O.Ensemble(N, L, temps, seed, skin=skin)
    ctx.advance([40, 40])
    ens.advance([40, 40])
    same_state(ctx, ens, N, L, xtol=1e-10, etol=1e-10)
    steps, rebuilds = ctx.counters()
    assert [int(r.nrebuild) for r in ens.reps] == rebuilds.tolist()
    assert rebuilds.min() >= 8  # a rebuild at least every five steps
    ctx.close()


@pytest.mark.parametrize("N,prec,why", [(4 * 20 ** 3, "mixed", "1024 threads"),
                                         (4 * 12 ** 3, "fp64", "shared memory")])
def test_replica_too_large_for_one_cluster_is_refused(re, N, prec, why):
    """32,000 atoms need more than 8 CTAs of 1024 threads; 6,912 FP64 atoms fit
    the threads but not a CTA's shared memory.  Both are refused at creation,
    before any launch."""
    L = inputs.box_length(N)
    with pytest.raises(re.REError) as e:
        re.Context(N, L, 2.5, [1.0, 1.1], 1, precision=prec)
    assert e.value.code == re.RE_EINVAL
    assert why in str(e.value)
