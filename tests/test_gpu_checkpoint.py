"""Checkpoint and resume: a context restored from a checkpoint continues bit
for bit as the original would have (positions, velocities, temperatures,
energies, step and rebuild counters, exchange decisions and statistics),
across list rebuilds, spatial re-sorts and exchanges, whatever launch shape
the restoring context was created with; checkpoints of another shape or seed,
and truncated ones, are refused and leave the context as it was."""
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


N, R, SEED = 500, 6, 31
CYCLES = 8
BUDGETS = inputs.random_budgets(R, CYCLES, 5, 15, 4)


def make(re, prec, path, **kw):
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    return re.Context(N, L, 2.5, temps, SEED, precision=prec, path=path, skin=0.3,
                      sort_interval=20, **kw)


def finish(ctx):
    """Cycles 3..7 (advance by the budgets, exchange), then everything observable."""
    dec = []
    for c in range(3, CYCLES):
        ctx.advance(BUDGETS[c])
        dec.append(ctx.exchange(outputs=True))
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    steps, reb = ctx.counters()
    att, acc = ctx.accept_stats()
    return dict(x=x, v=v, T=ctx.temps(), U=U, K=K, H=H, steps=steps, reb=reb, att=att, acc=acc,
                partners=np.array([d[0] for d in dec]), accepted=np.array([d[1] for d in dec]))


def assert_same(a, b):
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec,path", [("mixed", "batched"), ("fp64", "batched"),
                                       ("fp64", "plain")])
def test_resume_is_bit_exact(re, prec, path):
    a = make(re, prec, path)
    for c in range(3):
        a.advance(BUDGETS[c])
        a.exchange()
    ck = a.checkpoint()
    ra = finish(a)
    assert ra["reb"].sum() > R  # the run crossed list rebuilds
    # a fresh context created with another launch shape takes the saved one
    other = dict(cluster=4, atom_threads=1) if path == "batched" else {}
    b = make(re, prec, path, **other)
    b.restore(ck)
    if path == "batched":
        assert b.config()["cluster"] == a.config()["cluster"]
    assert_same(ra, finish(b))
    # and the original, rewound to its own checkpoint, repeats itself
    a.restore(ck)
    assert_same(ra, finish(a))
    a.close()
    b.close()


def test_foreign_checkpoints_are_refused(re):
    a = make(re, "mixed", "batched")
    a.advance(BUDGETS[0])
    ck = a.checkpoint()
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    twin = make(re, "mixed", "batched")
    victims = [re.Context(N, L, 2.5, temps[:R - 1], SEED, skin=0.3, sort_interval=20),  # shape
               re.Context(N, L, 2.5, temps, SEED + 1, skin=0.3, sort_interval=20),     # seed
               make(re, "mixed", "batched")]                                            # truncated
    for k, ctx in enumerate(victims):
        with pytest.raises(re.REError) as e:
            ctx.restore(ck[:-8] if k == 2 else ck)
        assert e.value.code == re.RE_EINVAL
    with pytest.raises(re.REError):
        victims[2].restore(np.zeros(64, np.uint8))  # not a checkpoint at all
    # a refused restore changed nothing
    victims[2].advance(BUDGETS[1])
    twin.advance(BUDGETS[1])
    xa, va = victims[2].get_state()
    xb, vb = twin.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    for ctx in victims + [a, twin]:
        ctx.close()


def test_group_resume_is_bit_exact(re):
    """A group of uneven ensembles (one launch) resumes bit for bit too."""
    specs = [(256, 3, 0.7, 1.6), (500, 2, 0.8, 1.4)]

    def group():
        members = [re.Context(n, inputs.box_length(n), 2.5, inputs.geometric_ladder(t0, t1, r),
                              50 + k, skin=0.3, sort_interval=20)
                   for k, (n, r, t0, t1) in enumerate(specs)]
        g = re.Context.group(members)
        for m in members:
            m.close()
        return g

    bud = inputs.random_budgets(5, 6, 5, 15, 9)
    a = group()
    for c in range(2):
        a.advance(bud[c])
        a.exchange()
    ck = a.checkpoint()

    def rest(ctx):
        dec = []
        for c in range(2, 6):
            ctx.advance(bud[c])
            dec.append(ctx.exchange(outputs=True))
        x, v = ctx.get_state()
        return dict(x=x, v=v, T=ctx.temps(), U=ctx.energies()[0], steps=ctx.counters()[0],
                    att=ctx.accept_stats()[0], partners=np.array([d[0] for d in dec]),
                    accepted=np.array([d[1] for d in dec]))

    ra = rest(a)
    b = group()
    b.restore(ck)
    assert_same(ra, rest(b))
    a.close()
    b.close()
