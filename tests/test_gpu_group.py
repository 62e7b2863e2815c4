"""Uneven ensembles advanced by one launch (re_group) against the FP64 oracle,
through the C ABI.

Each ensemble of a group is an independent ladder (Implementation section:
exchanges never mix ensembles); replicas advance by per-replica budgets drawn
uniformly in 5..50 between attempts, the asynchronous stride of the Example
section.  The oracle runs every ensemble on its own (its own seed and random
streams) with the same budgets.

FP64: x, v within 1e-10, U, K, H~ within 1e-11 relative; partners, decisions
and temperatures bit-exact.  Mixed, at the full uneven workload: a sample of
replicas per ensemble within the mixed tolerances, the whole ladders'
decisions bit-exact on the GPU's energies.
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


def make_group(re, specs, seed0, **kw):
    members = []
    for i, (N, R, t0, t1) in enumerate(specs):
        L = inputs.box_length(N)
        members.append(re.Context(N, L, 2.5, inputs.geometric_ladder(t0, t1, R), seed0 + i, **kw))
    g = re.Context.group(members)
    for m in members:
        m.close()
    return g


@pytest.mark.parametrize("launch", [{}, dict(cluster=4, atom_threads=1),
                                    dict(cluster=2, atom_threads=2, cell_div=2)],
                         ids=["default", "c4p1", "c2p2m2"])
def test_uneven_group_fp64_matches_oracle(re, launch):
    specs = [(256, 3, 0.7, 2.5), (500, 4, 0.7, 2.5), (864, 2, 0.7, 2.5)]
    seed0 = 60
    g = make_group(re, specs, seed0, precision="fp64", **launch)
    ens = [O.Ensemble(N, inputs.box_length(N), inputs.geometric_ladder(t0, t1, R), seed0 + i)
           for i, (N, R, t0, t1) in enumerate(specs)]
    Rtot = sum(s[1] for s in specs)
    bud = inputs.random_budgets(Rtot, 4, 5, 50, 21)
    for c in range(4):
        g.advance(bud[c])
        off = 0
        for e, (N, R, _, _) in zip(ens, specs):
            e.advance(bud[c][off:off + R])
            off += R
        U, K, H = g.energies()
        pg, ag = g.exchange(outputs=True)
        Tg = g.temps()
        off = 0
        for e, (N, R, _, _) in zip(ens, specs):
            assert np.allclose(U[off:off + R], e.energies(), rtol=1e-11, atol=0)
            po, ao = e.exchange()
            assert np.array_equal(pg[off:off + R], po), (c, N)
            assert np.array_equal(ag[off:off + R], ao), (c, N)
            assert np.array_equal(Tg[off:off + R], e.temps()), (c, N)
            off += R
    x, v = g.get_state()
    U, K, H = g.energies()
    steps, rebuilds = g.counters()
    a0 = r0 = 0
    for e, (N, R, _, _) in zip(ens, specs):
        L = inputs.box_length(N)
        for k, r in enumerate(e.reps):
            d = x[a0:a0 + N] - r.x
            d -= L * np.rint(d / L)
            assert np.abs(d).max() < 1e-10, (N, k)
            assert np.abs(v[a0:a0 + N] - r.v).max() < 1e-10, (N, k)
            assert U[r0 + k] == pytest.approx(r.U, rel=1e-11)
            assert K[r0 + k] == pytest.approx(r.K, rel=1e-11)
            assert H[r0 + k] == pytest.approx(r.H, rel=1e-11)
            assert steps[r0 + k] == r.step and rebuilds[r0 + k] == r.nrebuild
            a0 += N
        r0 += R


def test_uneven_group_full_size_sampled_match_oracle(re):
    """The uneven workload at full size (16x256, 32x500, 48x864, 64x2048,
    96x4000 in one launch, T 0.7-2.5, mixed, skin 0.4, the launch shape the
    benchmark's autotuner picks): first, middle and last replica of every
    ensemble rerun by the oracle; two stretches with the exchange between
    (the second from the GPU's state, see below).  Budgets are drawn in 5..15
    here (the FP64 test above takes the workload's 5..50): over longer
    stretches the mixed and FP64 trajectories part far enough that pairs near
    the cutoff, where the truncated force jumps, end up on different sides of
    it in the two runs."""
    specs = [(256, 16, 0.7, 2.5), (500, 32, 0.7, 2.5), (864, 48, 0.7, 2.5),
             (2048, 64, 0.7, 2.5), (4000, 96, 0.7, 2.5)]
    seed0, skin = 3030, 0.4
    g = make_group(re, specs, seed0, precision="mixed", skin=skin, cluster=4, atom_threads=1)
    Rtot = sum(s[1] for s in specs)
    bud = inputs.random_budgets(Rtot, 2, 5, 15, 77)
    sample = {}
    off = 0
    for i, (N, R, t0, t1) in enumerate(specs):
        L = inputs.box_length(N)
        temps = inputs.geometric_ladder(t0, t1, R)
        for k in (0, R // 2, R - 1):
            sample[off + k] = (O.Replica(N, L, float(temps[k]), seed0 + i, k, skin=skin), N, L)
        off += R
    starts = np.cumsum([0] + [N * R for (N, R, _, _) in specs])
    rstarts = np.cumsum([0] + [R for (_, R, _, _) in specs])

    def check(nsteps):
        # Position tolerance of the full-size tests (1e-6 after 10 steps),
        # scaled by (n / 10)^2 for a stretch of n steps: a force error held for
        # n steps moves an atom by (error) dt^2 n^2 / 2.  Energies per atom
        # keep the mixed tolerance 1e-5.
        x, _ = g.get_state()
        U, K, _ = g.energies()
        for gr, (rep, N, L) in sample.items():
            e = int(np.searchsorted(rstarts, gr, side="right")) - 1
            a = int(starts[e] + (gr - rstarts[e]) * N)
            d = x[a:a + N] - rep.x
            d -= L * np.rint(d / L)
            tol = 1e-6 * max(1.0, (nsteps[gr] / 10.0) ** 2)
            assert np.abs(d).max() < tol, (gr, nsteps[gr], np.abs(d).max())
            assert abs(U[gr] - rep.U) / N < 1e-5, gr
            assert abs(K[gr] - rep.K) / N < 1e-5, gr
        return U

    g.advance(bud[0])
    for gr, (rep, _, _) in sample.items():
        rep.steps(int(bud[0][gr]))
    U = check(bud[0])
    # The second stretch starts the sampled oracle replicas again from the
    # GPU's state (mixed and FP64 trajectories part exponentially, so each
    # stretch is compared from a common start); they then take the exchange
    # result and both sides run the second stretch.
    x0, v0 = g.get_state()
    for gr in list(sample):
        rep, N, L = sample[gr]
        e = int(np.searchsorted(rstarts, gr, side="right")) - 1
        a = int(starts[e] + (gr - rstarts[e]) * N)
        sample[gr] = (O.Replica(N, L, rep.T, seed0 + e, int(gr - rstarts[e]), skin=skin,
                                x=x0[a:a + N], v=v0[a:a + N], step=rep.step), N, L)
    T = g.temps()
    pg, ag = g.exchange(outputs=True)
    Tg = g.temps()
    for e, (N, R, _, _) in enumerate(specs):
        lo, hi = rstarts[e], rstarts[e + 1]
        To, po, ao, vo, _ = O.exchange(T[lo:hi], U[lo:hi], seed0 + e, 0, 0)
        assert np.array_equal(pg[lo:hi], po) and np.array_equal(ag[lo:hi], ao), N
        assert np.array_equal(Tg[lo:hi], To), N
        for gr in range(lo, hi):
            if gr in sample:
                rep = sample[gr][0]
                arr = (C.POINTER(O.Rep) * 1)(C.pointer(rep.rep))
                one = lambda a: np.ascontiguousarray([a], dtype=np.float64)
                Tk, lk, vk, uk = one(To[gr - lo]), one(1.0), one(vo[gr - lo]), one(1.0)
                O.lib().orc_apply_exchange_h(arr, 1, O._dp(Tk), O._dp(lk), O._dp(vk), O._dp(uk))
    g.advance(bud[1])
    for gr, (rep, _, _) in sample.items():
        rep.steps(int(bud[1][gr]))
    check(bud[1])
    steps, _ = g.counters()
    assert np.array_equal(steps, bud.sum(0))
    g.close()


def test_per_ensemble_launches_equal_one_launch(re):
    """Budget mode of a group: one launch per ensemble (each in its own shape,
    here the same explicit shape) gives bit for bit what one launch of all
    replicas gives (mixed path)."""
    specs = [(256, 4, 0.7, 2.5), (500, 3, 0.7, 2.5), (864, 3, 0.7, 2.5)]
    kw = dict(precision="mixed", skin=0.4, cluster=2, atom_threads=2, cell_div=2)
    a = make_group(re, specs, 90, group_launch=0, **kw)
    b = make_group(re, specs, 90, group_launch=-1, **kw)
    assert len(a.config()["classes"]) == 3 and "classes" not in b.config()
    Rtot = sum(s[1] for s in specs)
    bud = inputs.random_budgets(Rtot, 4, 5, 50, 5)
    for c in range(4):
        for g in (a, b):
            g.advance(bud[c])
            g.exchange()
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.energies()[2], b.energies()[2])
    assert np.array_equal(a.temps(), b.temps())


def test_group_switches_between_launch_layouts(re):
    """A group with per-ensemble launches in their default shapes (threads per
    atom differ between the ensembles and from the uniform launch) runs budget
    cycles, then the free-running exchange (one uniform launch), then budget
    cycles again.  The lists are rebuilt in the other layout at each switch
    (not counted as list-rule rebuilds); trajectories, decisions and energies
    replay on the FP64 oracle.  Rebuild counts equal the oracle's up to the
    first switch; after it the fresh lists' reference positions set when the
    list rule fires next, so the counts may part."""
    specs = [(256, 4, 0.8, 1.6), (500, 4, 0.8, 1.6)]
    seed0, nx, A = 120, 5, 4
    g = make_group(re, specs, seed0, precision="fp64")
    cls = g.config()["classes"]
    assert len(cls) == 2
    ens = [O.Ensemble(N, inputs.box_length(N), inputs.geometric_ladder(t0, t1, R), seed0 + i)
           for i, (N, R, t0, t1) in enumerate(specs)]
    Rtot = sum(s[1] for s in specs)
    r0s = np.cumsum([0] + [R for (_, R, _, _) in specs])

    def budget_cycle(b):
        g.advance(b)
        for i, e in enumerate(ens):
            e.advance(b[r0s[i]:r0s[i + 1]])

    bud = inputs.random_budgets(Rtot, 2, 5, 30, 8)
    budget_cycle(bud[0])
    base, reb = g.counters()
    assert np.array_equal(reb, np.concatenate([[r.nrebuild for r in e.reps] for e in ens]))
    steps, T, partner, acc = g.run_free(A, nx, log=True)
    for i, e in enumerate(ens):
        R = specs[i][1]
        prev = base[r0s[i]:r0s[i + 1]].copy()
        for k in range(A):
            st = steps[k, r0s[i]:r0s[i + 1]]
            e.advance([int(x) for x in st - prev])
            po, ao = e.exchange()
            assert np.array_equal(partner[k, r0s[i]:r0s[i + 1]], po), (i, k)
            assert np.array_equal(acc[k, r0s[i]:r0s[i + 1]].astype(bool), ao.astype(bool))
            assert np.array_equal(T[k, r0s[i]:r0s[i + 1]], e.temps())
            prev = st.copy()
        # the replicas' steps after their last attempt, up to where they stopped
        e.advance([int(x) for x in g.counters()[0][r0s[i]:r0s[i + 1]] - prev])
    budget_cycle(bud[1])
    x, v = g.get_state()
    U, K, H = g.energies()
    steps_now, rebuilds = g.counters()
    a0 = 0
    for i, e in enumerate(ens):
        N, R = specs[i][0], specs[i][1]
        L = inputs.box_length(N)
        for k, r in enumerate(e.reps):
            d = x[a0:a0 + N] - r.x
            d -= L * np.rint(d / L)
            assert np.abs(d).max() < 1e-9, (i, k)
            assert np.abs(v[a0:a0 + N] - r.v).max() < 1e-9, (i, k)
            assert U[r0s[i] + k] == pytest.approx(r.U, rel=1e-10)
            assert steps_now[r0s[i] + k] == r.step
            a0 += N


def test_group_graph_replay_after_a_free_running_call(re):
    """A group with per-ensemble launches captures its budget cycles in a CUDA
    graph, runs the free-running exchange (which lays the lists out for the
    uniform launch), then replays the cached graph: the lists must be laid out
    for the per-ensemble launches again before the replay.  FP64: the whole
    sequence -- graph cycles, the free-running attempts replayed from their
    log, graph cycles again -- follows the oracle."""
    specs = [(256, 4, 0.8, 1.6), (500, 4, 0.8, 1.6)]
    seed0, nx, A, cyc = 150, 5, 3, 3
    g = make_group(re, specs, seed0, precision="fp64", nx=nx)
    assert len(g.config()["classes"]) == 2
    ens = [O.Ensemble(N, inputs.box_length(N), inputs.geometric_ladder(t0, t1, R), seed0 + i)
           for i, (N, R, t0, t1) in enumerate(specs)]
    r0s = np.cumsum([0] + [R for (_, R, _, _) in specs])

    def oracle_cycles(n):
        for _ in range(n):
            for e in ens:
                e.advance([nx] * len(e.reps))
                e.exchange()

    g.run(cyc, graph=True)
    oracle_cycles(cyc)
    base = g.counters()[0]
    steps, T, partner, acc = g.run_free(A, nx, log=True)
    for i, e in enumerate(ens):
        prev = base[r0s[i]:r0s[i + 1]].copy()
        for k in range(A):
            st = steps[k, r0s[i]:r0s[i + 1]]
            e.advance([int(x) for x in st - prev])
            po, ao = e.exchange()
            assert np.array_equal(partner[k, r0s[i]:r0s[i + 1]], po), (i, k)
            prev = st.copy()
        e.advance([int(x) for x in g.counters()[0][r0s[i]:r0s[i + 1]] - prev])
    g.run(cyc, graph=True)
    oracle_cycles(cyc)
    x, v = g.get_state()
    U, _, _ = g.energies()
    assert np.array_equal(g.temps(), np.concatenate([e.temps() for e in ens]))
    a0 = 0
    for i, e in enumerate(ens):
        N = specs[i][0]
        L = inputs.box_length(N)
        for k, r in enumerate(e.reps):
            d = x[a0:a0 + N] - r.x
            d -= L * np.rint(d / L)
            assert np.abs(d).max() < 1e-9, (i, k)
            assert np.abs(v[a0:a0 + N] - r.v).max() < 1e-9, (i, k)
            assert U[r0s[i] + k] == pytest.approx(r.U, rel=1e-10)
            a0 += N
