"""GPU path against the FP64 CPU oracle, through the C ABI.

Tolerances (fixed by the method's target):
  FP64 forces: max |F_gpu - F_oracle| <= 1e-12 * rms|F|; FP64 energies 1e-12 relative.
  mixed forces: max |F_gpu - F_oracle| <= 1e-5 * rms|F|; energies 1e-6 relative per atom.
  exchange patterns and decisions: bit-exact given identical T, U, seed, attempt.
"""
import math

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


def force_err(f, fo):
    rms = math.sqrt((fo ** 2).sum(1).mean())
    return np.sqrt(((f - fo) ** 2).sum(1)).max() / rms


def melted_state(N, R, seed, temps):
    """Per replica: oracle run from the lattice for 200 steps (a liquid-like state)."""
    L = inputs.box_length(N)
    reps = [O.Replica(N, L, float(t), seed, k) for k, t in enumerate(temps)]
    for r in reps:
        r.steps(200)
    return L, reps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [256, 500, 864, 2048])
def test_initial_state_matches_oracle(re, prec, N):
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 2.0, 3)
    ctx = re.Context(N, L, 2.5, temps, 99, precision=prec)
    x, v = ctx.get_state()
    for k, t in enumerate(temps):
        xo = O.fcc_lattice(N, L)
        vo = O.init_velocities(N, t, 99, k)
        assert np.abs(x[k * N:(k + 1) * N] - xo).max() < 1e-12 * L
        assert np.abs(v[k * N:(k + 1) * N] - vo).max() < 1e-12
    U, K, H = ctx.energies()
    for k, t in enumerate(temps):
        _, Uo = O.forces_brute(O.fcc_lattice(N, L), L)
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert abs(U[k] - Uo) <= tol * abs(Uo)
        # mixed path: kinetic energy summed from FP32 squares (exact integer sum)
        assert K[k] == pytest.approx(0.5 * (3 * N - 3) * t, rel=tol)


@pytest.mark.parametrize("prec,ftol,utol", [("fp64", 1e-12, 1e-12), ("mixed", 1e-5, 1e-6)])
@pytest.mark.parametrize("N", [256, 500, 864, 2048, 4000])
def test_forces_match_brute_force(re, prec, ftol, utol, N):
    temps = [0.8, 1.9]
    L, reps = melted_state(N, 2, 5, temps)
    x = np.concatenate([r.x for r in reps])
    v = np.concatenate([r.v for r in reps])
    ctx = re.Context(N, L, 2.5, temps, 5, precision=prec)
    ctx.set_state(x, v)
    f = ctx.forces()
    U, K, H = ctx.energies()
    for k, r in enumerate(reps):
        fo, Uo = O.forces_brute(r.x, L)
        assert force_err(f[k * N:(k + 1) * N], fo) <= ftol
        assert abs(U[k] - Uo) / N <= utol * abs(Uo / N)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lj_forces_device_entry(re, prec):
    import torch
    N = 864
    L, reps = melted_state(N, 1, 3, [1.2])
    fo, Uo = O.forces_brute(reps[0].x, L)
    x = torch.tensor(reps[0].x, device="cuda", dtype=torch.float64)
    f, U = re.lj_forces_device(x, L, precision=prec)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert force_err(f.cpu().numpy(), fo) <= tol
    assert abs(U.item() - Uo) <= (1e-12 if prec == "fp64" else 1e-6) * abs(Uo)


@pytest.mark.parametrize("path", ["batched", "plain"])
def test_fp64_md_steps_match_oracle(re, path):
    N, seed = 500, 11
    temps = inputs.geometric_ladder(0.8, 1.6, 3)
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", path=path)
    ens = O.Ensemble(N, L, temps, seed)
    budgets = [7, 30, 0]
    ctx.advance(budgets)
    ens.advance(budgets)
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    steps, rebuilds = ctx.counters()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < 1e-10
        assert np.abs(v[k * N:(k + 1) * N] - r.v).max() < 1e-10
        assert U[k] == pytest.approx(r.U, rel=1e-11)
        assert K[k] == pytest.approx(r.K, rel=1e-11)
        assert H[k] == pytest.approx(r.H, rel=1e-11)
        assert steps[k] == budgets[k] == r.step
        assert rebuilds[k] == r.nrebuild


def test_mixed_md_steps_track_oracle(re):
    N, seed = 864, 4
    temps = inputs.geometric_ladder(0.7, 2.0, 2)
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="mixed", skin=0.3)
    ens = O.Ensemble(N, L, temps, seed, skin=0.3)
    ctx.advance([10, 10])
    ens.advance([10, 10])
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < 1e-6
        assert abs(U[k] - r.U) / N < 1e-5
        assert abs(K[k] - r.K) / N < 1e-5


@pytest.mark.parametrize("R", [2, 3, 7, 64, 1024, 4096])
@pytest.mark.parametrize("mode", [0, 1])
def test_exchange_device_bit_exact(re, R, mode):
    import torch
    for seed in range(3):
        T, U = inputs.random_temps_energies(R, seed + 100 * R, u_sd=5.0)
        for attempt in (0, 1, 17):
            To, po, ao, vo, n = O.exchange(T, U, 1234 + seed, attempt, mode)
            Tg, pg, ag, vg = re.exchange_device(torch.tensor(T, device="cuda"),
                                                torch.tensor(U, device="cuda"), 1234 + seed,
                                                attempt, mode)
            assert np.array_equal(pg.cpu().numpy(), po)
            assert np.array_equal(ag.cpu().numpy(), ao)
            assert np.array_equal(Tg.cpu().numpy(), To)
            assert np.allclose(vg.cpu().numpy(), vo, rtol=1e-15, atol=0)


def test_replica_exchange_run_matches_oracle(re):
    """8 x 256 replicas, T 0.8-1.6, stride 100, FP64: 4 cycles of advance + exchange."""
    N, R, seed = 256, 8, 12345
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64")
    ens = O.Ensemble(N, L, temps, seed)
    for cyc in range(4):
        ctx.advance(100)
        ens.advance([100] * R)
        U, _, _ = ctx.energies()
        assert np.allclose(U, ens.energies(), rtol=1e-9, atol=0)
        pg, ag = ctx.exchange(outputs=True)
        po, ao = ens.exchange()
        assert np.array_equal(pg, po) and np.array_equal(ag, ao)
        assert np.array_equal(ctx.temps(), ens.temps())
    att, acc = ctx.accept_stats()
    assert att.sum() == sum(1 for c in range(4) for k in range(c & 1, R - 1, 2))


def test_graph_run_equals_eager(re):
    N, R = 500, 6
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.7, 1.5, R)
    bud = inputs.random_budgets(R, 5, 5, 50, 3)
    a = re.Context(N, L, 2.5, temps, 8)
    b = re.Context(N, L, 2.5, temps, 8)
    a.run(5, bud, graph=True)
    for c in range(5):
        b.advance(bud[c])
        b.exchange()
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.temps(), b.temps())
    assert np.array_equal(a.counters()[0], bud.sum(0))


def test_uneven_group_matches_members(re):
    """Ensembles of 256, 500 and 864 atoms in one launch give the results each
    gives alone (same launch shape)."""
    kw = dict(cluster=2, atom_threads=2, cell_div=2)
    specs = [(256, 3, 0.7, 2.5), (500, 4, 0.7, 2.5), (864, 2, 0.7, 2.5)]
    alone, members = [], []
    for i, (N, R, t0, t1) in enumerate(specs):
        L = inputs.box_length(N)
        temps = inputs.geometric_ladder(t0, t1, R)
        alone.append(re.Context(N, L, 2.5, temps, 40 + i, **kw))
        members.append(re.Context(N, L, 2.5, temps, 40 + i, **kw))
    g = re.Context.group(members)
    Rtot = sum(s[1] for s in specs)
    bud = inputs.random_budgets(Rtot, 3, 5, 50, 9)
    for c in range(3):
        g.advance(bud[c])
        g.exchange()
        off = 0
        for ctx, (N, R, _, _) in zip(alone, specs):
            ctx.advance(bud[c][off:off + R])
            ctx.exchange()
            off += R
    xg, vg = g.get_state()
    Ug = g.energies()[0]
    a0 = r0 = 0
    for ctx, (N, R, _, _) in zip(alone, specs):
        x, v = ctx.get_state()
        assert np.array_equal(xg[a0:a0 + N * R], x)
        assert np.array_equal(vg[a0:a0 + N * R], v)
        assert np.array_equal(Ug[r0:r0 + R], ctx.energies()[0])
        a0 += N * R
        r0 += R


def test_neighbour_overflow_is_reported(re):
    N = 864
    L = inputs.box_length(N)
    ctx = None
    with pytest.raises(re.REError) as e:
        ctx = re.Context(N, L, 2.5, [1.0, 1.1], 1, nbr_capacity=8)
    assert e.value.code == re.RE_EOVERFLOW
    del ctx


def test_non_finite_energy_is_reported(re):
    N = 256
    L = inputs.box_length(N)
    ctx = re.Context(N, L, 2.5, [1.0], 1)
    x, v = ctx.get_state()
    x[1] = x[0]  # two atoms on top of each other: infinite pair energy
    with pytest.raises(re.REError) as e:
        ctx.set_state(x, v)
    assert e.value.code == re.RE_ENUMERIC


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_small_blocks_match_oracle(re, prec):
    """32 atoms and 32 threads per CTA (clusters of 8): fewer threads than
    thermostat records per chunk; every CTA of a replica must still hold the
    same records (budgets run past record 32 of the first chunk)."""
    N, seed = 256, 3
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.4, 3)
    ctx = re.Context(N, L, 2.5, temps, seed, precision=prec, cluster=8, atom_threads=1)
    assert ctx.config()["threads"] == 32
    ens = O.Ensemble(N, L, temps, seed)
    budgets = [70, 40, 65]
    ctx.advance(budgets)
    ens.advance(budgets)
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    steps, _ = ctx.counters()
    tol = 1e-10 if prec == "fp64" else 1e-5
    for k, r in enumerate(ens.reps):
        assert steps[k] == budgets[k]
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < (tol if prec == "fp64" else 1e-4)
        assert abs(U[k] - r.U) / N < (1e-12 if prec == "fp64" else 1e-5)
        assert abs(K[k] - r.K) / N < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lists_in_shared_memory_equal_global(re, prec):
    """Where the neighbour lists live (global memory, or copied into shared
    memory at every launch) must not change a single bit."""
    N = 500
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.6, 4)
    a = re.Context(N, L, 2.5, temps, 17, precision=prec, lists_smem=0)
    b = re.Context(N, L, 2.5, temps, 17, precision=prec, lists_smem=1)
    assert a.config()["lists_smem"] == 0 and b.config()["lists_smem"] == 1
    for c in range(6):
        for ctx in (a, b):
            ctx.advance(15)
            ctx.exchange()
    xa, va = a.get_state()
    xb, vb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert np.array_equal(a.energies()[2], b.energies()[2])
