"""The exchange step of a context (ladders of up to 256 replicas: one CTA per
ensemble ordering them by counting ranks; longer ones: a cluster of CTAs per
ensemble, each ranking a slice of the ladder) against
the oracle's exchange on the same temperatures, potential scales and
energies (Implementation section: sort, pair neighbours, Metropolis with the
lower replica id's uniform, rescale velocities by sqrt(T_new/T_old)):
partners, decisions, new temperatures and scales bit-exact, kinetic energies
to rounding.  And re_run_record: the per-cycle record it copies back equals
what the per-call API reports, and an FP64 run of it follows the oracle."""
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


@pytest.mark.parametrize("R", [2, 3, 64, 256, 257, 600])
@pytest.mark.parametrize("variant", ["neighbours", "random_parity", "hamiltonian_d2"])
def test_context_exchange_matches_oracle(re, R, variant):
    N = 256
    L = inputs.box_length(N)
    parity = 1 if variant == "random_parity" else 0
    dist = 2 if variant == "hamiltonian_d2" else 1
    temps = inputs.geometric_ladder(0.7, 2.5, R)
    # T rises and lam falls along the ladder: the keys T/lam stay distinct
    lams = inputs.geometric_ladder(1.0, 0.8, R) if variant == "hamiltonian_d2" else None
    seed = 1000 + R
    ctx = re.Context(N, L, 2.5, temps, seed, pair_parity=parity, exch_distance=dist, lam=lams)
    ctx.advance(3)
    n_acc = 0
    for attempt in range(3):
        T, lam = ctx.temps(), ctx.lambdas()
        U, K, _ = ctx.energies()
        Tn, ln, po, ao, vs, us, n = O.exchange_h(T, lam, U, seed, attempt, parity, dist)
        pg, ag = ctx.exchange(outputs=True)
        assert np.array_equal(pg, po)
        assert np.array_equal(ag, ao)
        assert np.array_equal(ctx.temps(), Tn)
        assert np.array_equal(ctx.lambdas(), ln)
        U2, K2, _ = ctx.energies()
        assert np.allclose(K2, K * vs ** 2, rtol=1e-14, atol=0)
        assert np.allclose(U2, U * us, rtol=1e-14, atol=0)
        n_acc += n
        ctx.advance(2)
    att, acc = ctx.accept_stats()
    assert acc.sum() == n_acc
    ctx.close()


def _twins(re, **kw):
    N, R = 500, 12
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    return [re.Context(N, L, 2.5, temps, 31, **kw) for _ in range(2)]


@pytest.mark.parametrize("kw", [dict(), dict(precision="fp64"), dict(path="plain")],
                         ids=["mixed", "fp64", "plain"])
def test_run_record_equals_the_per_call_api(re, kw):
    a, b = _twins(re, **kw)
    cycles = 6
    bud = inputs.random_budgets(a.n_rep, cycles, 5, 20, 9)
    rec = a.run_record(cycles, bud)
    for k in range(cycles):
        b.advance(bud[k])
        pg, ag = b.exchange(outputs=True)
        U, K, H = b.energies()
        assert np.array_equal(rec["partner"][k], pg)
        assert np.array_equal(rec["accepted"][k], ag)
        assert np.array_equal(rec["T"][k], b.temps())
        assert np.array_equal(rec["U"][k], U)
        assert np.array_equal(rec["K"][k], K)
        assert np.array_equal(rec["H"][k], H)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.counters()[0], b.counters()[0])
    # a second call reuses the record areas; without budgets every replica
    # makes nx steps
    rec2 = a.run_record(2)
    for k in range(2):
        b.advance()
        pg, _ = b.exchange(outputs=True)
        assert np.array_equal(rec2["partner"][k], pg)
        assert np.array_equal(rec2["H"][k], b.energies()[2])
    a.close()
    b.close()


@pytest.mark.parametrize("kw", [dict(), dict(precision="fp64")], ids=["mixed", "fp64"])
def test_run_record_graph_equals_eager(re, kw):
    """The graph form of re_run_record: the same records and states as the
    eager form, also on the next call, which replays the kept graph with new
    budgets."""
    a, b = _twins(re, **kw)
    cycles = 5
    for call in range(2):
        bud = inputs.random_budgets(a.n_rep, cycles, 5, 20, 20 + call)
        ra = a.run_record(cycles, bud, graph=True)
        rb = b.run_record(cycles, bud)
        for key in ("partner", "accepted", "T", "U", "K", "H"):
            assert np.array_equal(ra[key], rb[key]), (call, key)
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_run_record_fp64_follows_the_oracle(re):
    """8 x 256 replicas, FP64, uneven budgets: the record of every cycle
    against the oracle ensemble run with the same budgets."""
    N, R, seed = 256, 8, 777
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64")
    ens = O.Ensemble(N, L, temps, seed)
    cycles = 4
    bud = inputs.random_budgets(R, cycles, 5, 30, 4)
    rec = ctx.run_record(cycles, bud)
    for k in range(cycles):
        ens.advance([int(s) for s in bud[k]])
        po, ao = ens.exchange()
        assert np.array_equal(rec["partner"][k], po)
        assert np.array_equal(rec["accepted"][k], ao)
        assert np.array_equal(rec["T"][k], ens.temps())
        assert np.allclose(rec["U"][k], ens.energies(), rtol=1e-9, atol=0)
        assert np.allclose(rec["H"][k], [r.H for r in ens.reps], rtol=1e-9, atol=0)
    ctx.close()


def test_run_record_of_a_group(re):
    """Two ensembles in one context: each cycle's record against the members
    run alone in the same launch shape (replica ids concatenated)."""
    kw = dict(cluster=2, atom_threads=2, cell_div=2)
    specs = [(256, 4, 0.7, 1.6), (500, 6, 0.8, 2.0)]
    mk = lambda: [re.Context(N, inputs.box_length(N), 2.5, inputs.geometric_ladder(t0, t1, R),
                             50 + i, **kw) for i, (N, R, t0, t1) in enumerate(specs)]
    g = re.Context.group(mk())
    alone = mk()
    cycles = 3
    bud = inputs.random_budgets(g.n_rep, cycles, 5, 15, 2)
    rec = g.run_record(cycles, bud)
    for k in range(cycles):
        off = 0
        for m in alone:
            m.advance(bud[k][off:off + m.n_rep])
            pg, ag = m.exchange(outputs=True)
            sl = slice(off, off + m.n_rep)
            assert np.array_equal(rec["partner"][k][sl], pg)
            assert np.array_equal(rec["accepted"][k][sl], ag)
            assert np.array_equal(rec["T"][k][sl], m.temps())
            assert np.array_equal(rec["H"][k][sl], m.energies()[2])
            off += m.n_rep
    for m in alone:
        m.close()
    g.close()


def test_run_record_rejects_negative_budgets(re):
    a, b = _twins(re)
    bud = np.full((2, a.n_rep), 5, np.int32)
    bud[1, 3] = -1
    with pytest.raises(re.REError):
        a.run_record(2, bud)
    a.close()
    b.close()


def test_group_exchange_with_a_long_ladder_matches_oracle(re):
    """A group whose longest ladder (300 replicas) takes the cluster form of the
    exchange, beside a 5-replica ensemble run by the same launch: every
    ensemble's partners, decisions and temperatures against the oracle's
    exchange on its own ladder."""
    specs = [(256, 300, 0.7, 2.5, 71), (256, 5, 0.8, 1.4, 72)]
    members = [re.Context(N, inputs.box_length(N), 2.5, inputs.geometric_ladder(t0, t1, R), sd)
               for (N, R, t0, t1, sd) in specs]
    g = re.Context.group(members)
    for m in members:
        m.close()
    g.advance(4)
    for attempt in range(3):
        T, lam = g.temps(), g.lambdas()
        U = g.energies()[0]
        pg, ag = g.exchange(outputs=True)
        Tg = g.temps()
        off = 0
        for (N, R, _, _, sd) in specs:
            sl = slice(off, off + R)
            Tn, _, po, ao, _, _, _ = O.exchange_h(T[sl], lam[sl], U[sl], sd, attempt, 0, 1)
            assert np.array_equal(pg[sl], po)
            assert np.array_equal(ag[sl], ao)
            assert np.array_equal(Tg[sl], Tn)
            off += R
        g.advance(2)
    g.close()


def test_run_record_graph_of_a_group(re):
    """A group with per-ensemble launches (forked onto their own streams inside
    the capture): the graph form of re_run_record equals the eager one, on the
    capturing call and on a replay with new budgets."""
    specs = [(256, 4, 0.7, 1.6), (500, 6, 0.8, 2.0)]
    mk = lambda: re.Context.group([
        re.Context(N, inputs.box_length(N), 2.5, inputs.geometric_ladder(t0, t1, R), 60 + i)
        for i, (N, R, t0, t1) in enumerate(specs)])
    a, b = mk(), mk()
    assert len(a.config()["classes"]) == 2
    for call in range(2):
        bud = inputs.random_budgets(a.n_rep, 3, 5, 15, 30 + call)
        ra = a.run_record(3, bud, graph=True)
        rb = b.run_record(3, bud)
        for key in ("partner", "accepted", "T", "H"):
            assert np.array_equal(ra[key], rb[key]), (call, key)
    xa, _ = a.get_state()
    xb, _ = b.get_state()
    assert np.array_equal(xa, xb)
    a.close()
    b.close()
