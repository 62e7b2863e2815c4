"""Generalised exchanges on the GPU against the FP64 oracle: potential-scale
(Hamiltonian) ladders, parameter sets (T, lam), and pairs at ladder distance d
(the extensions the Implementation section mentions)."""
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


def random_ladder(R, rng):
    """Distinct keys T/lam: a temperature ladder and potential scales."""
    T = rng.permutation(0.7 * 1.03 ** np.arange(R))
    lam = rng.uniform(0.6, 1.4, R)
    return T, lam


@pytest.mark.parametrize("R", [2, 5, 64, 1000])
@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("mode", [0, 1])
def test_exchange_device_h_bit_exact(re, R, d, mode):
    import torch
    rng = np.random.default_rng(R * 10 + d)
    for trial in range(3):
        T, lam = random_ladder(R, rng)
        U = rng.normal(-4.0 * 864, 6.0, R) * lam
        for attempt in (0, 1, 7):
            To, lo, po, ao, vo, uo, _ = O.exchange_h(T, lam, U, 99 + trial, attempt, mode, d)
            cu = lambda a: torch.tensor(a, device="cuda")
            Tg, lg, pg, ag, vg, ug = re.exchange_device_h(cu(T), cu(lam), cu(U), 99 + trial,
                                                          attempt, mode, d)
            assert np.array_equal(pg.cpu().numpy(), po)
            assert np.array_equal(ag.cpu().numpy(), ao)
            assert np.array_equal(Tg.cpu().numpy(), To)
            assert np.array_equal(lg.cpu().numpy(), lo)
            assert np.allclose(vg.cpu().numpy(), vo, rtol=1e-15, atol=0)
            assert np.allclose(ug.cpu().numpy(), uo, rtol=1e-15, atol=0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_scaled_forces_and_energy(re, prec, tol):
    N = 864
    L = inputs.box_length(N)
    temps = [0.8, 1.0, 1.2]
    lam = [1.0, 0.6, 1.3]
    ctx = re.Context(N, L, 2.5, temps, 5, precision=prec, lam=lam)
    ctx.advance(30)
    x, _ = ctx.get_state()
    f = ctx.forces()
    U, _, _ = ctx.energies()
    assert np.array_equal(ctx.lambdas(), lam)
    for k in range(3):
        fo, Uo = O.forces_brute(x[k * N:(k + 1) * N], L)
        fo = lam[k] * fo
        rms = np.sqrt((fo ** 2).sum(1).mean())
        assert np.sqrt(((f[k * N:(k + 1) * N] - fo) ** 2).sum(1)).max() <= tol * rms
        assert abs(U[k] - lam[k] * Uo) <= (tol if prec == "fp64" else 1e-6) * abs(lam[k] * Uo)


@pytest.mark.parametrize("path", ["batched", "plain"])
def test_scaled_md_steps_match_oracle(re, path):
    N, seed = 500, 21
    L = inputs.box_length(N)
    temps = [0.9, 0.9, 1.1]
    lam = [1.0, 0.8, 1.25]
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", path=path, lam=lam)
    ens = O.Ensemble(N, L, temps, seed, lams=lam)
    budgets = [12, 40, 5]
    ctx.advance(budgets)
    ens.advance(budgets)
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < 1e-10
        assert np.abs(v[k * N:(k + 1) * N] - r.v).max() < 1e-10
        assert U[k] == pytest.approx(r.U, rel=1e-11)
        assert H[k] == pytest.approx(r.H, rel=1e-11)


def test_hamiltonian_exchange_run_matches_oracle(re):
    """8 x 256, FP64, temperatures and potential scales both varying, pairs at
    ladder distance 2; decisions bit-exact over 6 cycles, states after."""
    N, R, seed = 256, 8, 314
    L = inputs.box_length(N)
    temps = inputs.geometric_ladder(0.8, 1.2, R)
    lam = np.linspace(1.0, 0.8, R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", lam=lam, exch_distance=2)
    ens = O.Ensemble(N, L, temps, seed, lams=list(lam), distance=2)
    for cyc in range(6):
        ctx.advance(40)
        ens.advance([40] * R)
        U, _, _ = ctx.energies()
        assert np.allclose(U, ens.energies(), rtol=1e-9, atol=0)
        pg, ag = ctx.exchange(outputs=True)
        po, ao = ens.exchange()
        assert np.array_equal(pg, po) and np.array_equal(ag, ao)
        assert np.array_equal(ctx.temps(), ens.temps())
        assert np.array_equal(ctx.lambdas(), ens.lams())
    ctx.advance(20)
    ens.advance([20] * R)
    x, v = ctx.get_state()
    U, K, H = ctx.energies()
    for k, r in enumerate(ens.reps):
        d = x[k * N:(k + 1) * N] - r.x
        d -= L * np.rint(d / L)
        assert np.abs(d).max() < 1e-8
        assert U[k] == pytest.approx(r.U, rel=1e-9)
        assert H[k] == pytest.approx(r.H, rel=1e-9)


def test_free_running_hamiltonian_replays_on_the_oracle(re):
    N, R, seed, nx, A = 256, 8, 17, 10, 10
    L = inputs.box_length(N)
    temps = [1.0] * R            # a pure potential-scale ladder at one temperature
    lam = 1.0 - 0.05 * np.arange(R)
    ctx = re.Context(N, L, 2.5, temps, seed, precision="fp64", lam=lam, exch_distance=2)
    ens = O.Ensemble(N, L, temps, seed, lams=list(lam), distance=2)
    steps, T, partner, acc = ctx.run_free(A, nx, log=True)
    prev = np.zeros(R, np.int64)
    for k in range(A):
        ens.advance([int(s) for s in steps[k] - prev])
        po, ao = ens.exchange()
        assert np.array_equal(partner[k], po), k
        assert np.array_equal(acc[k].astype(bool), ao.astype(bool)), k
        prev = steps[k].copy()
    assert np.array_equal(ctx.lambdas(), ens.lams())
    U, _, H = ctx.energies()
    for k, r in enumerate(ens.reps):
        assert U[k] == pytest.approx(r.U, rel=1e-9)
        assert H[k] == pytest.approx(r.H, rel=1e-9)
