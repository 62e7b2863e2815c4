"""The sharded-ladder pieces on the GPU, in one process: two contexts hold
the halves of an 8-member (T, lam) ladder (id_offset 0 and 4), the decisions
come from the library's exchange kernel over the gathered ladder and are
applied with apply_exchange.  The result must equal one context holding the
whole ladder (FP64, same launch shape)."""
import numpy as np
import pytest

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


def test_two_shards_equal_one_context(re):
    from paper_0812_1633_gb300.sharded import ContextShard, ShardedLadder
    N, R, seed, nx, cycles = 256, 8, 99, 25, 6
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.3, R)
    lam = np.linspace(1.0, 0.85, R)
    shape = dict(precision="fp64", cluster=1, atom_threads=2, cell_div=2, exch_distance=2)
    whole = re.Context(N, L, 2.5, temps, seed, lam=lam, **shape)
    halves = [re.Context(N, L, 2.5, temps[4 * k:4 * k + 4], seed, lam=lam[4 * k:4 * k + 4],
                         id_offset=4 * k, **shape) for k in range(2)]
    hub = {}

    def gather_for(rank):
        def g(msg):
            hub[rank] = msg
            return [hub[0], hub[1]]
        return g
    lads = [ShardedLadder(ContextShard(h), 4 * k, R, seed, 0, 2, gather=gather_for(k))
            for k, h in enumerate(halves)]
    for c in range(cycles):
        whole.advance(nx)
        for h in halves:
            h.advance(nx)
        pw, aw = whole.exchange(outputs=True)
        hub[1] = lads[1].message()
        p0, a0 = lads[0].exchange()
        p1, a1 = lads[1].exchange()
        assert np.array_equal(p0, pw) and np.array_equal(p1, pw)
        assert np.array_equal(a0.astype(bool), aw.astype(bool))
    Tw = whole.temps()
    assert np.array_equal(np.concatenate([h.temps() for h in halves]), Tw)
    assert np.array_equal(np.concatenate([h.lambdas() for h in halves]), whole.lambdas())
    xw, vw = whole.get_state()
    Uw, Kw, Hw = whole.energies()
    for k, h in enumerate(halves):
        x, v = h.get_state()
        U, K, H = h.energies()
        sl = slice(4 * k * N, (4 * k + 4) * N)
        assert np.allclose(x, xw[sl], rtol=0, atol=1e-12)
        assert np.allclose(v, vw[sl], rtol=0, atol=1e-12)
        assert np.allclose(U, Uw[4 * k:4 * k + 4], rtol=1e-12, atol=0)
        assert np.allclose(H, Hw[4 * k:4 * k + 4], rtol=1e-12, atol=0)
    att, acc = whole.accept_stats()
    assert np.array_equal(lads[0].pair_att, att) and np.array_equal(lads[0].pair_acc, acc)
