"""The split launch (re_opts.wide_launch): the hottest replicas run in a second,
concurrent launch with clusters of twice the CTAs.  Which replicas are hot is decided
on the device from the current temperatures, so after exchanges the classes
change members.  With equal threads per atom the trajectories must not change:
bit for bit on the mixed path (exact integer sums), and within the FP64
tolerances against the oracle on the FP64 path."""
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


def test_split_launch_is_bit_identical_on_the_mixed_path(re):
    """The benchmark's shape: 64 x 864, 2-CTA clusters, 2 threads per atom;
    split, the 12 hottest replicas take 4-CTA clusters (the 24 SMs the uniform
    launch leaves idle)."""
    N, R = 864, 64
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    kw = dict(skin=0.3, cluster=2, atom_threads=2, cell_div=2)
    a = re.Context(N, L, 2.5, temps, 31, wide_launch=1, **kw)
    b = re.Context(N, L, 2.5, temps, 31, wide_launch=-1, **kw)
    ca, cb = a.config(), b.config()
    assert ca["wide_n"] == 12 and ca["wide_cluster"] == 4 and cb["wide_n"] == 0, (ca, cb)
    assert ca["wide_atom_threads"] == 2
    bud = inputs.random_budgets(R, 6, 5, 20, 4)
    for c in range(6):
        for ctx in (a, b):
            ctx.advance(bud[c])
            ctx.exchange()
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.temps(), b.temps())
    assert np.array_equal(a.energies()[2], b.energies()[2])
    assert np.array_equal(a.counters()[1], b.counters()[1])
    # the hot class did change members: the ladder moved
    assert not np.array_equal(a.temps(), temps)


def test_split_launch_fp64_matches_oracle(re):
    N, R, seed = 500, 6, 19
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", cluster=2, atom_threads=2,
                     wide_launch=1)
    cfg = ctx.config()
    assert cfg["wide_n"] == R - 1 and cfg["wide_cluster"] == 4, cfg
    ens = O.Ensemble(N, L, temps, seed)
    bud = inputs.random_budgets(R, 3, 5, 30, 6)
    for c in range(3):
        ctx.advance(bud[c])
        ens.advance(bud[c])
        pg, ag = ctx.exchange(outputs=True)
        po, ao = ens.exchange()
        assert np.array_equal(pg, po) and np.array_equal(ag, ao)
        assert np.array_equal(ctx.temps(), ens.temps())
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    steps, rebuilds = ctx.counters()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < 1e-10
        assert np.abs(v[k * N:(k + 1) * N] - r.v).max() < 1e-10
        assert U[k] == pytest.approx(r.U, rel=1e-11)
        assert H[k] == pytest.approx(r.H, rel=1e-11)
        assert steps[k] == r.step and rebuilds[k] == r.nrebuild


def test_split_launch_in_a_graph_equals_eager(re):
    N, R = 864, 32
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    kw = dict(skin=0.3, cluster=2, atom_threads=2, wide_launch=1)
    a = re.Context(N, L, 2.5, temps, 8, **kw)
    b = re.Context(N, L, 2.5, temps, 8, **kw)
    assert a.config()["wide_n"] > 0
    bud = inputs.random_budgets(R, 4, 5, 30, 3)
    a.run(4, bud, graph=True)
    for c in range(4):
        b.advance(bud[c])
        b.exchange()
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.temps(), b.temps())
