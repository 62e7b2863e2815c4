"""Free-running (asynchronous) mode of the batched kernel (Implementation section).

The master replica of each ensemble (replica attempt mod R) performs exactly
N_x steps; every other replica stops at the first step boundary after the
master has finished.  The number of steps a replica makes is thus decided by
timing, but its trajectory is not: given the step counts the GPU reports, the
FP64 oracle run for those counts must land on the same states (the stop rule
only chooses where the velocity-Verlet / thermostat sequence ends).
"""
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


def compare(ctx, ens, N, L, tol=1e-10):
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < tol, k
        assert np.abs(v[k * N:(k + 1) * N] - r.v).max() < tol, k
        assert U[k] == pytest.approx(r.U, rel=1e-11)
        assert K[k] == pytest.approx(r.K, rel=1e-11)
        assert H[k] == pytest.approx(r.H, rel=1e-11)


def test_async_fp64_matches_oracle_at_reported_step_counts(re):
    N, R, seed, nx = 500, 4, 31, 20
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64")
    ens = O.Ensemble(N, L, temps, seed)
    prev = np.zeros(R, np.int64)
    for cyc in range(3):
        ctx.advance_async(nx)
        steps, _ = ctx.counters()
        made = steps - prev
        prev = steps.copy()
        master = cyc % R            # the attempt counter rotates the master
        assert made[master] == nx
        assert (made >= 1).all() and (made <= 16 * nx + 16).all(), made
        ens.advance([int(s) for s in made])
        compare(ctx, ens, N, L)
        pg, ag = ctx.exchange(outputs=True)
        po, ao = ens.exchange()
        assert np.array_equal(pg, po) and np.array_equal(ag, ao)
        assert np.array_equal(ctx.temps(), ens.temps())


def test_async_graph_run_counts(re):
    N, R, nx, cycles = 256, 8, 10, 6
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, 5)
    ctx.run_async(cycles, nx, graph=True)
    steps, _ = ctx.counters()
    # every replica steps at least once per cycle; masters exactly nx
    assert (steps >= cycles).all()
    for k in range(R):
        n_master = sum(1 for c in range(cycles) if c % R == k)
        assert steps[k] >= n_master * nx + (cycles - n_master)
    U, K, H = ctx.energies()
    assert np.isfinite(U).all() and np.isfinite(K).all() and np.isfinite(H).all()
    att, _ = ctx.accept_stats()
    assert att.sum() == sum(1 for c in range(cycles) for k in range(c & 1, R - 1, 2))


def test_async_replicas_run_alongside_the_master(re):
    """All replicas resident at once (64 x 864, mixed): the others make about as
    many steps as the master, hot replicas (more list rebuilds) somewhat fewer."""
    N, R, nx = 864, 64, 100
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    ctx = re.Context(N, L, 2.5, temps, 3, skin=0.3)
    ctx.advance(50)
    s0, _ = ctx.counters()
    ctx.advance_async(nx)
    made = ctx.counters()[0] - s0
    assert made[0] == nx
    assert 0.5 * nx <= made.mean() <= 1.5 * nx, made


def test_async_needs_batched_path(re):
    N = 256
    ctx = re.Context(N, inputs.box_length(N), 2.5, [1.0, 1.2], 1, path="plain")
    with pytest.raises(re.REError):
        ctx.advance_async(5)


# ---------------------------------------------------------------------------
# exchanges inside one persistent launch (re_run_free)

def test_free_running_fp64_replays_on_the_oracle(re):
    """The log gives, per attempt, the step at which each replica took part;
    the oracle advanced to those steps and exchanging there must take the same
    decisions and land on the same states."""
    N, R, seed, nx, A = 256, 8, 41, 10, 12
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64")
    ens = O.Ensemble(N, L, temps, seed)
    steps, T, partner, acc = ctx.run_free(A, nx, log=True)
    prev = np.zeros(R, np.int64)
    for k in range(A):
        m = k % R
        # the master issues attempt k nx of its own steps after its attempt k - 1
        assert steps[k, m] - prev[m] == nx, (k, steps[k], prev)
        made = steps[k] - prev
        assert (made >= 1).all(), made
        ens.advance([int(x) for x in made])
        po, ao = ens.exchange()
        assert np.array_equal(partner[k], po), (k, partner[k], po)
        assert np.array_equal(acc[k].astype(bool), ao.astype(bool)), k
        assert np.array_equal(T[k], ens.temps()), k
        prev = steps[k].copy()
    assert np.array_equal(ctx.counters()[0], prev)
    compare(ctx, ens, N, L, tol=1e-9)
    att, _ = ctx.accept_stats()
    assert att.sum() == sum(1 for k in range(A) for q in range(k & 1, R - 1, 2))


def test_free_running_mixed_many_replicas(re):
    N, R, nx, A = 864, 64, 10, 40
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, R)
    ctx = re.Context(N, L, 2.5, temps, 3, skin=0.3)
    ctx.advance(20)
    s0, _ = ctx.counters()
    steps, T, partner, acc = ctx.run_free(A, nx, log=True)
    for k in range(A):
        assert np.array_equal(np.sort(T[k]), np.sort(temps))      # still a permutation
        p = partner[k]
        for r in range(R):                                          # pairs are mutual
            if p[r] >= 0:
                assert p[p[r]] == r and acc[k, r] == acc[k, p[r]]
    per_attempt = (steps[-1] - s0) / A                              # <N_x> per replica
    assert 0.5 * nx <= per_attempt.mean() <= 2.0 * nx, per_attempt
    U, K, H = ctx.energies()
    assert np.isfinite(U).all() and np.isfinite(K).all()
    assert np.array_equal(ctx.temps(), T[-1])
    # the context goes on with ordinary cycles afterwards
    ctx.advance(10)
    ctx.exchange()
    ctx.run_free(5, nx)
    assert np.isfinite(ctx.energies()[0]).all()


def test_free_running_falls_back_to_a_resident_shape(re):
    """160 replicas in 8-CTA clusters with 8 threads per atom (1280 CTAs) cannot
    all be resident; the free-running call runs in a narrower shape that can
    (fewer CTAs and threads per replica, lists rebuilt in its layout) and
    replays on the oracle; budget cycles afterwards, back in the tuned shape,
    follow the oracle too."""
    N, R, seed, nx, A = 256, 160, 43, 10, 6
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", cluster=8, atom_threads=8)
    ens = O.Ensemble(N, L, temps, seed)
    steps, T, partner, acc = ctx.run_free(A, nx, log=True)
    prev = np.zeros(R, np.int64)
    for k in range(A):
        made = steps[k] - prev
        assert (made >= 1).all(), made
        ens.advance([int(x) for x in made])
        po, ao = ens.exchange()
        assert np.array_equal(partner[k], po), k
        assert np.array_equal(acc[k].astype(bool), ao.astype(bool)), k
        assert np.array_equal(T[k], ens.temps()), k
        prev = steps[k].copy()
    compare(ctx, ens, N, L, tol=1e-9)
    assert ctx.config()["cluster"] == 8 and ctx.config()["atom_threads"] == 8
    ctx.advance(7)
    ens.advance([7] * R)
    compare(ctx, ens, N, L, tol=1e-9)


def test_free_running_refuses_non_resident_launch(re):
    N, R = 256, 1000
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, inputs.geometric_ladder(0.7, 2.0, R), 1)
    with pytest.raises(re.REError):
        ctx.run_free(2, 5)


def test_free_running_timeout_leaves_a_consistent_state(re):
    """Failure detection of the free-running exchange (Implementation section:
    the blocking pair receive becomes a bounded device wait).  Replica w stops
    answering in attempt 3 of the launch (host-side fault injection: it sends
    no pair message and leaves at that step boundary); its partner's wait runs
    out after 5 ms, the call returns RE_ETIMEOUT, and every replica stops at
    a step boundary.  Replayed on the FP64 oracle from the log: the earlier
    attempts and the pairs of attempt 3 that completed take the oracle's
    decisions, the pair of w swaps nothing, and the final x, v, T of every
    replica equal the oracle's at the reported step counts.  The context then
    goes on with ordinary calls.  (The replicas that are not waiting keep
    stepping until the abort reaches them, a wait limit's worth of steps: the
    limit is kept short so that the FP64 trajectories still agree to 1e-9.)"""
    N, R, seed, nx, A, w, ks = 256, 8, 43, 10, 6, 3, 3
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64")
    ens = O.Ensemble(N, L, temps, seed)
    ctx.set_wait_limit(0.005)
    ctx.inject_stall(w, ks)
    with pytest.raises(re.REError) as e:
        ctx.run_free(A, nx, log=True)
    assert e.value.code == re.RE_ETIMEOUT
    steps, T, partner, acc = e.value.log
    final, _ = ctx.counters()
    prev = np.zeros(R, np.int64)
    for k in range(ks):                       # complete attempts: as the replay test
        assert (steps[k] >= 0).all()
        ens.advance([int(x) for x in steps[k] - prev])
        po, ao = ens.exchange()
        assert np.array_equal(partner[k], po) and np.array_equal(acc[k].astype(bool), ao.astype(bool))
        assert np.array_equal(T[k], ens.temps())
        prev = steps[k].copy()
    took = steps[ks] >= 0
    assert not took[w] and final[w] >= prev[w]
    # every other replica had seen the pattern before the abort
    assert took.sum() == R - 1, steps[ks]
    # to the step of its part in attempt ks (w: to where it stopped)
    at = np.where(took, steps[ks], final)
    ens.advance([int(x) for x in at - prev])
    To, lo, po, ao, vs, us, _ = O.exchange_h(ens.temps(), ens.lams(), ens.energies(), seed, ks,
                                             0, 1)
    p = po[w]
    assert p >= 0 and partner[ks, p] == w and acc[ks, p] == 0   # the stalled pair: no swap
    for r in range(R):
        if r in (w, p):
            To[r], vs[r] = ens.reps[r].T, 1.0
        else:
            assert partner[ks, r] == po[r] and bool(acc[ks, r]) == bool(ao[r]), r
    assert np.array_equal(np.sort(To), np.sort(temps))       # still a permutation
    O.lib().orc_apply_exchange_h(ens._arr, R, O._dp(To), O._dp(lo), O._dp(vs), O._dp(us))
    ens.advance([int(x) for x in final - at])
    assert np.array_equal(ctx.temps(), ens.temps())
    compare(ctx, ens, N, L, tol=1e-9)
    # the context goes on: ordinary cycles, then a free-running launch
    ctx.advance(10)
    ctx.exchange()
    ctx.run_free(2, nx)
    assert np.isfinite(ctx.energies()[0]).all()
    assert np.array_equal(np.sort(ctx.temps()), np.sort(temps))
