"""Host-side bookkeeping of the C ABI on the GPU: the device copy of the step
budgets that re_advance keeps (a call with the budgets of the last upload
copies nothing; every other writer of that buffer drops it), and the
free-running call's narrower resident shape on the mixed path."""
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


def _twins(re, **kw):
    N, R = 500, 6
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    return [re.Context(N, L, 2.5, temps, 17, **kw) for _ in range(2)]


def test_repeated_budgets_equal_explicit_runs(re):
    """advance(b1), advance(b1) (kept copy), advance(b2), advance(b1), each
    followed by an exchange, against re_run with the same budgets passed
    explicitly (its own device buffer): bit-identical states and counters."""
    a, b = _twins(re)
    R = a.n_rep
    b1 = inputs.random_budgets(R, 1, 5, 15, 1)[0]
    b2 = inputs.random_budgets(R, 1, 5, 15, 2)[0]
    seq = [b1, b1, b2, b1]
    for s in seq:
        a.advance(s)
        a.exchange()
    b.run(len(seq), np.stack(seq), graph=False)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.counters()[0], b.counters()[0])
    assert np.array_equal(a.counters()[0], np.sum(seq, axis=0))
    a.close()
    b.close()


def test_kept_budgets_dropped_by_other_writers(re):
    """set_state rebuilds the lists with a zero-budget launch through the same
    device buffer, and autotune writes its trial budgets there: the next
    advance with the earlier budgets must upload them again."""
    a, _ = _twins(re)
    R = a.n_rep
    b1 = inputs.random_budgets(R, 1, 5, 15, 3)[0]
    a.advance(b1)
    s0 = a.counters()[0].copy()
    x, v = a.get_state()
    a.set_state(x, v)
    a.advance(b1)
    assert np.array_equal(a.counters()[0] - s0, b1)
    a.autotune(steps=4)
    s1 = a.counters()[0].copy()
    a.advance(b1)
    assert np.array_equal(a.counters()[0] - s1, b1)
    a.close()


def test_free_running_mixed_in_a_narrower_shape(re):
    """96 replicas of 864 atoms: the tuned budget shape (2-CTA clusters) cannot
    have them all resident; the free-running call runs anyway, in a narrower
    shape, and leaves a valid state: T a permutation of the ladder, pairs
    mutual, finite energies, and budget cycles run afterwards."""
    N, R, nx, A = 864, 96, 5, 10
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    ctx = re.Context(N, L, 2.5, temps, 9, skin=0.3, cluster=2, atom_threads=2)
    steps, T, partner, acc = ctx.run_free(A, nx, log=True)
    assert (steps[-1] >= 0).all()
    for k in range(A):
        p = partner[k]
        paired = p >= 0
        assert np.array_equal(p[p[paired]], np.arange(R)[paired])
    assert np.array_equal(np.sort(ctx.temps()), np.sort(temps))
    U, K, H = ctx.energies()
    assert np.isfinite(U).all() and np.isfinite(H).all()
    assert ctx.config()["cluster"] == 2 and ctx.config()["atom_threads"] == 2
    s0 = ctx.counters()[0].copy()
    ctx.advance(10)
    ctx.exchange()
    assert np.array_equal(ctx.counters()[0] - s0, np.full(R, 10))
    assert np.isfinite(ctx.energies()[2]).all()
    ctx.close()
