"""Pins of the FP64 CPU oracle against things other than itself.

Each test fixes a fact that the paper, a library routine or the mathematics
determines: numpy's Philox4x64-10, scipy's Gamma/normal distributions, closed
forms of the LJ pair, finite differences, an independent FCC lattice sum,
brute-force pair enumeration, conservation laws and hand-worked Metropolis
decisions.  A dropped term, wrong sign or wrong index in the oracle fails one.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O

RHO = 0.8442


def box(N):
    return (N / RHO) ** (1.0 / 3.0)


# ------------------------------------------------------------------ Philox
@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((5, 6, 7, 8), (11, 12)),
    ((2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1), (2**64 - 1, 2**64 - 1)),
    ((123456789, 4, 3, 0), (12345, 977)),
    ((0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0, 0x082EFA98EC4E6C89),
     (0x452821E638D01377, 0xBE5466CF34E90C6C)),
])
def test_philox_matches_numpy(ctr, key):
    # numpy's Philox (4x64, 10 rounds) increments its counter before each block.
    prev = list(ctr)
    i = 0
    while True:
        if prev[i] == 0:
            prev[i] = 2**64 - 1
            i += 1
            continue
        prev[i] -= 1
        break
    bg = np.random.Philox(counter=np.array(prev, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(4)]
    assert O.philox4x64(ctr, key) == ref


def test_uniform_is_top_53_bits():
    bg = np.random.Philox(counter=[6, 4, 2, 0], key=[99, 3])
    raw = bg.random_raw(4)
    u = O.uniform4(99, 3, 7, 4, 2)
    assert np.array_equal(u, (raw >> np.uint64(11)).astype(np.float64) * 2.0**-53)
    assert np.all((u >= 0) & (u < 1))


def test_box_muller_closed_form():
    for u0, u1 in [(0.3, 0.1), (0.999, 0.77), (0.0, 0.5), (0.5, 0.0)]:
        g0, g1 = O.box_muller(u0, u1)
        assert math.isclose(g0 * g0 + g1 * g1, -2 * math.log(1 - u0), rel_tol=1e-14, abs_tol=1e-300)
        if u0 > 0:
            ang = math.atan2(g1, g0) % (2 * math.pi)
            assert math.isclose(ang, (2 * math.pi * u1) % (2 * math.pi), abs_tol=1e-12)


def test_gaussian_stream_is_standard_normal():
    g = []
    for i in range(4000):
        u = O.uniform4(5, 1, i, O.TAG_VEL)
        g.extend(O.box_muller(u[0], u[1]))
    assert stats.kstest(g, "norm").pvalue > 1e-3


@pytest.mark.parametrize("a", [1.0, 2.5, 64.5, 1294.5])
def test_gamma_marsaglia_tsang_distribution(a):
    draws = np.array([O.gamma_mt(a, 2024, 3, i)[0] for i in range(3000)])
    assert stats.kstest(draws, "gamma", args=(a,)).pvalue > 1e-3
    se = math.sqrt(a / len(draws))
    assert abs(draws.mean() - a) < 5 * se


# ------------------------------------------------------------------ SVR
def test_svr_c1_is_identity():
    a, Kn = O.svr_alpha(123.0, 100.0, 300, 1.0, 0.7, 290.0)
    assert Kn == pytest.approx(123.0, rel=1e-15) and a == pytest.approx(1.0, rel=1e-15)


def test_svr_alpha_squared_is_kinetic_ratio():
    K, Kbar, Nf, c = 80.0, 100.0, 200, math.exp(-0.01)
    for R1, S in [(0.3, 190.0), (-1.2, 210.0), (2.0, 150.0)]:
        a, Kn = O.svr_alpha(K, Kbar, Nf, c, R1, S)
        assert a > 0 and a * a == pytest.approx(Kn / K, rel=1e-14)
        expect = c * K + (1 - c) * Kbar * (R1 * R1 + S) / Nf + 2 * R1 * math.sqrt(c * (1 - c) * Kbar * K / Nf)
        assert Kn == pytest.approx(expect, rel=1e-14)


def test_svr_alpha_sign_rule():
    # alpha < 0 exactly when R1 + sqrt(c Nf K / ((1-c) Kbar)) < 0.
    K, Kbar, Nf, c = 1.0, 1.0, 3, 0.01
    thr = -math.sqrt(c * Nf * K / ((1 - c) * Kbar))
    a_neg, _ = O.svr_alpha(K, Kbar, Nf, c, thr - 0.05, 2.0)
    a_pos, _ = O.svr_alpha(K, Kbar, Nf, c, thr + 0.05, 2.0)
    assert a_neg < 0 < a_pos


def test_svr_c0_gives_canonical_kinetic_energy():
    # c = 0: K' = Kbar (R1^2 + S)/Nf with R1^2 + S ~ chi^2_Nf, i.e. K' ~ Gamma(Nf/2, scale T).
    N, T = 32, 1.3
    Nf = 3 * N - 3
    Kbar = 0.5 * Nf * T
    out = []
    for n in range(3000):
        u = O.uniform4(7, 0, n, O.TAG_SVR_R1)
        R1, _ = O.box_muller(u[0], u[1])
        S = 2.0 * O.gamma_mt(0.5 * (Nf - 1), 7, 0, n)[0]
        out.append(O.svr_alpha(40.0, Kbar, Nf, 0.0, R1, S)[1])
    assert stats.kstest(out, "gamma", args=(Nf / 2, 0, T)).pvalue > 1e-3


def test_svr_mean_relaxation():
    # E[K'] = c K + (1 - c) Kbar for any c.
    K, Kbar, Nf, c = 50.0, 100.0, 189, 0.9
    out = []
    for n in range(4000):
        u = O.uniform4(11, 0, n, O.TAG_SVR_R1)
        R1, _ = O.box_muller(u[0], u[1])
        S = 2.0 * O.gamma_mt(0.5 * (Nf - 1), 11, 0, n)[0]
        out.append(O.svr_alpha(K, Kbar, Nf, c, R1, S)[1])
    out = np.array(out)
    assert abs(out.mean() - (c * K + (1 - c) * Kbar)) < 5 * out.std() / math.sqrt(len(out))


# ------------------------------------------------------------------ LJ pair
def test_lj_shift_value():
    assert O.lj_shift(2.5, 1) == pytest.approx(-0.016316891136, rel=1e-9)
    assert O.lj_shift(2.5, 0) == 0.0


def test_lj_pair_closed_forms():
    Uc = O.lj_shift(2.5)
    u, fs = O.lj_pair(1.0, Uc)
    assert u == pytest.approx(-Uc, abs=1e-15) and fs == pytest.approx(24.0, rel=1e-15)
    rmin2 = 2.0 ** (1.0 / 3.0)
    u, fs = O.lj_pair(rmin2, 0.0)
    assert u == pytest.approx(-1.0, rel=1e-14) and abs(fs) < 1e-13


@pytest.mark.parametrize("r", [0.9, 1.0, 1.3, 2.0, 2.45])
def test_lj_force_is_minus_gradient(r):
    h = 1e-5
    up, _ = O.lj_pair((r + h) ** 2)
    um, _ = O.lj_pair((r - h) ** 2)
    _, fs = O.lj_pair(r * r)
    # fs = -(1/r) du/dr
    assert fs == pytest.approx(-(up - um) / (2 * h) / r, rel=1e-8)


# ------------------------------------------------------------------ forces
def melted(N, seed=0, amp=0.12):
    L = box(N)
    rng = np.random.default_rng(seed)
    x = O.fcc_lattice(N, L) + rng.uniform(-amp, amp, size=(N, 3))
    return x % L, L


def test_two_atoms_across_boundary():
    L = 8.0
    x = np.array([[0.2, 4.0, 4.0], [L - 0.9, 4.0, 4.0]])  # minimum-image distance 1.1
    f, U = O.forces_brute(x, L)
    u, fs = O.lj_pair(1.1 ** 2, O.lj_shift(2.5))
    assert U == pytest.approx(u, rel=1e-14)
    # force on atom 0 points away from atom 1, i.e. along +x (atom 1 sits at -1.1)
    assert f[0, 0] == pytest.approx(fs * 1.1, rel=1e-14) and f[0, 0] > 0
    assert np.allclose(f[0], -f[1], rtol=0, atol=1e-14)


def test_forces_are_minus_gradient_of_energy():
    x, L = melted(32, seed=3, amp=0.2)
    f, _ = O.forces_brute(x, L)
    h = 1e-6
    for i, k in [(0, 0), (5, 1), (17, 2), (31, 0)]:
        xp = x.copy(); xp[i, k] += h
        xm = x.copy(); xm[i, k] -= h
        g = (O.forces_brute(xp, L)[1] - O.forces_brute(xm, L)[1]) / (2 * h)
        assert f[i, k] == pytest.approx(-g, rel=1e-6, abs=1e-6)


@pytest.mark.parametrize("N", [32, 108, 256])
def test_newton_third_law_and_translation(N):
    x, L = melted(N, seed=N)
    f, U = O.forces_brute(x, L)
    rms = math.sqrt((f * f).sum(1).mean())
    assert np.abs(f.sum(0)).max() < 1e-12 * rms * math.sqrt(N)
    shift = np.array([0.37, -1.91, 2.2])
    f2, U2 = O.forces_brute((x + shift) % L, L)
    assert U2 == pytest.approx(U, rel=1e-12)
    assert np.abs(f2 - f).max() < 1e-11 * rms


def fcc_lattice_sum(a, rc=2.5):
    """U per atom of an infinite FCC lattice (cube side a), shifted LJ, r < rc.

    Enumerates lattice vectors (a/2)(n1, n2, n3) with n1 + n2 + n3 even; no
    periodic box and no minimum image are involved."""
    Uc = 4 * (rc ** -12 - rc ** -6)
    m = int(math.ceil(2 * rc / a)) + 1
    tot = 0.0
    for n1 in range(-m, m + 1):
        for n2 in range(-m, m + 1):
            for n3 in range(-m, m + 1):
                if (n1 + n2 + n3) % 2 or (n1 == n2 == n3 == 0):
                    continue
                r = 0.5 * a * math.sqrt(n1 * n1 + n2 * n2 + n3 * n3)
                if r < rc:
                    tot += 4 * (r ** -12 - r ** -6) - Uc
    return 0.5 * tot


@pytest.mark.parametrize("N", [256, 500, 864])
def test_perfect_fcc(N):
    L = box(N)
    x = O.fcc_lattice(N, L)
    k = round((N / 4) ** (1 / 3))
    assert 4 * k ** 3 == N
    f, U = O.forces_brute(x, L)
    assert np.abs(f).max() < 1e-12
    assert U / N == pytest.approx(fcc_lattice_sum(L / k), rel=1e-12)
    # every site is distinct and inside the box
    assert len({tuple(np.round(p, 9)) for p in x}) == N
    assert x.min() >= 0 and x.max() < L


@pytest.mark.parametrize("N,rlist", [(32, 3.0), (108, 3.0), (256, 3.0), (864, 2.8), (2048, 3.0)])
def test_verlet_list_matches_brute_force(N, rlist):
    x, L = melted(N, seed=N + 1)
    pi, pj = O.build_list(x, L, rlist)
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.rint(d / L)
    r2 = (d * d).sum(-1)
    iu = np.triu_indices(N, 1)
    want = {(int(i), int(j)) for i, j in zip(*iu) if r2[i, j] < rlist * rlist}
    got = set(zip(pi.tolist(), pj.tolist()))
    assert got == want and len(got) == len(pi)
    fb, Ub = O.forces_brute(x, L)
    fl, Ul = O.forces_list(x, L, pi, pj)
    rms = math.sqrt((fb * fb).sum(1).mean())
    assert np.abs(fl - fb).max() < 1e-13 * rms
    assert Ul == pytest.approx(Ub, rel=1e-13)


# ------------------------------------------------------------------ set-up
@pytest.mark.parametrize("N,T", [(256, 0.8), (864, 2.0)])
def test_initial_velocities(N, T):
    v = O.init_velocities(N, T, 12345, 3)
    assert np.abs(v.sum(0)).max() < 1e-11
    Nf = 3 * N - 3
    assert (v * v).sum() / Nf == pytest.approx(T, rel=1e-13)
    z = (v / math.sqrt(T)).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_init_replica_is_lattice_plus_velocities():
    N, L = 256, box(256)
    r = O.Replica(N, L, 0.9, 77, 2, tau=0.5)
    assert np.array_equal(r.x, O.fcc_lattice(N, L))
    assert np.array_equal(r.v, O.init_velocities(N, 0.9, 77, 2))
    assert r.K == pytest.approx(0.5 * (r.v ** 2).sum(), rel=1e-15)
    assert r.step == 0 and r.nrebuild == 1


# ------------------------------------------------------------------ MD
def test_nve_time_reversibility():
    x, L = melted(108, seed=9, amp=0.15)
    v = O.init_velocities(108, 1.0, 1, 0)
    r = O.Replica(108, L, 1.0, 1, 0, tau=0.0, x=x, v=v)
    x0, v0 = r.x.copy(), r.v.copy()
    r.steps(100)
    r.v *= -1.0
    r.refresh()
    r.steps(100)
    d = r.x - x0
    d -= L * np.rint(d / L)
    assert np.abs(d).max() < 1e-9
    assert np.abs(r.v + v0).max() < 1e-9


def nve_fluct(dt, nsteps, x, v, L):
    r = O.Replica(len(x), L, 1.0, 1, 0, tau=0.0, dt=dt, x=x, v=v)
    H = []
    for _ in range(nsteps // 10):
        r.steps(10)
        H.append(r.U + r.K)
    return np.std(H), r


def test_nve_energy_error_scales_as_dt_squared():
    N = 108
    x, L = melted(N, seed=4, amp=0.1)
    v = O.init_velocities(N, 1.0, 2, 0)
    s1, r1 = nve_fluct(0.004, 400, x, v, L)
    s2, r2 = nve_fluct(0.002, 800, x, v, L)
    ratio = s1 / s2
    assert 3.0 < ratio < 5.3
    # momentum stays zero
    assert np.abs(r1.v.sum(0)).max() < 1e-10


def test_thermostat_keeps_temperature_and_effective_energy():
    N, T = 108, 1.2
    L = box(N)
    r = O.Replica(N, L, T, 5, 0, tau=0.1)
    r.steps(400)
    Ts, H = [], []
    for _ in range(300):
        r.steps(5)
        Ts.append(2 * r.K / (3 * N - 3))
        H.append(r.H)
    Ts = np.array(Ts)
    # block standard error (blocks of 20 samples = 100 steps >> tau/dt)
    blocks = Ts.reshape(-1, 20).mean(1)
    se = blocks.std(ddof=1) / math.sqrt(len(blocks))
    assert abs(Ts.mean() - T) < 3.5 * se + 1e-3
    # effective energy H~ = U + K + econs is conserved up to the integrator error
    assert (max(H) - min(H)) / N < 5e-3
    assert np.abs(r.v.sum(0)).max() < 1e-10


def test_rebuild_criterion_half_skin():
    # no pair within rc may be missed: list forces equal brute force after many steps
    N = 256
    L = box(N)
    r = O.Replica(N, L, 2.0, 3, 1, skin=0.3, tau=0.5)
    r.steps(300)
    assert r.nrebuild > 2
    fb, Ub = O.forces_brute(r.x, L)
    rms = math.sqrt((fb * fb).sum(1).mean())
    assert np.abs(r.f - fb).max() < 1e-12 * rms
    assert r.U == pytest.approx(Ub, rel=1e-12)


# ------------------------------------------------------------------ exchange
def test_exchange_hand_cases():
    seed, att = 42, 0
    r0 = O.uniform4(seed, 0, att, O.TAG_EXCH)[0]
    # D >= 0 always accepted: cold replica 0 has the higher energy
    Tn, partner, acc, vs, n = O.exchange([1.0, 2.0], [-10.0, -20.0], seed, att)
    assert n == 1 and list(partner) == [1, 0] and list(acc) == [1, 1]
    assert list(Tn) == [2.0, 1.0]
    assert vs[0] == pytest.approx(math.sqrt(2.0)) and vs[1] == pytest.approx(math.sqrt(0.5))
    # D < 0: accept iff r < exp(D); D = (1/1 - 1/2)(U0 - U1) = 0.5 (U0 - U1)
    D_below = math.log(r0) + 1e-9   # exp(D) slightly above r -> accept
    D_above = math.log(r0) - 1e-9   # exp(D) slightly below r -> reject
    for D, want in [(D_below, 1), (D_above, 0)]:
        U = [-20.0 + 2 * D, -20.0]
        Tn, partner, acc, vs, n = O.exchange([1.0, 2.0], U, seed, att)
        assert n == want and list(partner) == [1, 0]
        assert list(Tn) == ([2.0, 1.0] if want else [1.0, 2.0])


def test_exchange_uses_lower_id_random_number():
    # replica 1 is colder than replica 0; the uniform must be replica 0's.
    seed, att = 9, 4   # even attempt: offset 0, so the two replicas form a pair
    r0 = O.uniform4(seed, 0, att, O.TAG_EXCH)[0]
    r1 = O.uniform4(seed, 1, att, O.TAG_EXCH)[0]
    assert abs(r0 - r1) > 0.05
    lo, hi = sorted([r0, r1])
    D = math.log(0.5 * (lo + hi))  # accept with r_lo, reject with r_hi
    want = 1 if r0 < math.exp(D) else 0
    T = [2.0, 1.0]
    U = [-20.0, -20.0 + 2 * D]   # D = (1/T_cold - 1/T_hot)(U_cold - U_hot) = 0.5 * (U1 - U0)
    Tn, partner, acc, vs, n = O.exchange(T, U, seed, att)
    assert n == want


def test_exchange_pattern_parity_and_permutation():
    rng = np.random.default_rng(0)
    R = 9
    ladder = 0.7 * 1.0275 ** np.arange(R)
    T = rng.permutation(ladder)
    for att in range(40):
        U = rng.normal(-5000, 30, R)
        order = np.argsort(T)
        Tn, partner, acc, vs, n = O.exchange(T, U, 1, att)
        p = att & 1
        # pairs are sorted-temperature neighbours starting at position p
        pairs = [(order[k], order[k + 1]) for k in range(p, R - 1, 2)]
        assert int((partner >= 0).sum()) == 2 * len(pairs)
        for a, b in pairs:
            assert partner[a] == b and partner[b] == a
            assert acc[a] == acc[b]
        assert sorted(Tn) == sorted(ladder)
        assert n == sum(acc) // 2
        T = Tn


@pytest.mark.parametrize("D", [-0.2, -1.0, -2.5])
def test_acceptance_frequency_is_metropolis(D):
    n = 20000
    U = [-10.0 + 2 * D, -10.0]
    acc = sum(O.exchange([1.0, 2.0], U, 31, a)[4] for a in range(0, 2 * n, 2))
    p = math.exp(D)
    se = math.sqrt(p * (1 - p) / n)
    assert abs(acc / n - p) < 3 * se


def test_random_parity_mode_draws_both_offsets():
    ps = set()
    for att in range(20):
        _, partner, _, _, _ = O.exchange([1.0, 1.1, 1.2], [0.0, 0.0, 0.0], 5, att, parity_mode=1)
        ps.add(int(partner[0] >= 0))
    assert ps == {0, 1}


def test_exchange_rescales_and_keeps_effective_energy():
    N = 32
    L = box(N) * 1.3
    ens = O.Ensemble(N, L, [0.7, 0.9], seed=3, tau=0.5)
    ens.advance([20, 20])
    v0 = [r.v.copy() for r in ens.reps]
    KE0 = [r.K + r.econs for r in ens.reps]
    ens.reps[0].rep.U, ens.reps[1].rep.U = 0.0, -100.0   # force acceptance (D > 0)
    partner, acc = ens.exchange()
    assert list(acc) == [1, 1] and list(partner) == [1, 0]
    assert ens.temps().tolist() == [0.9, 0.7]
    assert np.allclose(ens.reps[0].v, v0[0] * math.sqrt(0.9 / 0.7), rtol=1e-15, atol=0)
    assert np.allclose(ens.reps[1].v, v0[1] * math.sqrt(0.7 / 0.9), rtol=1e-15, atol=0)
    for r, ke in zip(ens.reps, KE0):
        assert r.K == pytest.approx(0.5 * (r.v ** 2).sum(), rel=1e-12)
        # econs absorbs the kinetic change, so H~ = U + K + econs stays continuous
        assert r.K + r.econs == pytest.approx(ke, rel=1e-12)


def test_budgets_are_per_replica_and_thread_independent():
    N = 32
    L = box(N) * 1.2
    a = O.Ensemble(N, L, [0.8, 1.0, 1.2], seed=8)
    b = O.Ensemble(N, L, [0.8, 1.0, 1.2], seed=8)
    a.advance([5, 17, 0], nthreads=3)
    for r, s in zip(b.reps, [5, 17, 0]):
        r.steps(s)
    for ra, rb, s in zip(a.reps, b.reps, [5, 17, 0]):
        assert ra.step == s
        assert np.array_equal(ra.x, rb.x) and np.array_equal(ra.v, rb.v)


# ------------------------------------------- generalised (Hamiltonian) exchange
def test_generalised_exchange_reduces_to_temperature_exchange():
    rng = np.random.default_rng(3)
    for R in (2, 5, 9):
        for att in range(12):
            T = rng.permutation(0.7 * 1.03 ** np.arange(R))
            U = rng.normal(-4000, 40, R)
            a = O.exchange(T, U, 77, att, att % 2)
            b = O.exchange_h(T, None, U, 77, att, att % 2, 1)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[2])
            assert np.array_equal(a[2], b[3]) and np.array_equal(a[3], b[4])
            assert np.array_equal(b[1], np.ones(R)) and np.array_equal(b[5], np.ones(R))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_distance_d_pattern(d):
    rng = np.random.default_rng(d)
    R = 11
    ladder = 0.7 * 1.0275 ** np.arange(R)
    T = rng.permutation(ladder)
    for att in range(8):
        U = rng.normal(-5000, 30, R)
        rank = np.argsort(np.argsort(T))   # ladder position of every replica
        order = np.argsort(T)
        Tn, _, partner, acc, _, _, n = O.exchange_h(T, None, U, 1, att, 0, d)
        o = (att & 1) * d
        # expected pairs written out: blocks of 2d from offset o, (q, q + d)
        want = [(order[q], order[q + d]) for q in range(o, R - d) if (q - o) % (2 * d) < d]
        assert int((partner >= 0).sum()) == 2 * len(want)
        for a, b in want:
            assert partner[a] == b and partner[b] == a
            assert abs(int(rank[a]) - int(rank[b])) == d
        assert sorted(Tn) == sorted(ladder)
        T = Tn


def test_lambda_exchange_hand_cases():
    """Equal temperatures, potential scales 1 and 0.5: D = (1 - 0.5)/T (u_a - u_b),
    u = U/lam; the lower id's uniform decides."""
    seed, att, T = 13, 0, 1.5
    r0 = O.uniform4(seed, 0, att, O.TAG_EXCH)[0]
    lam = [1.0, 0.5]
    # ladder order by T/lam: replica 0 (1.5) before replica 1 (3.0)
    for D, want in [(math.log(r0) + 1e-9, 1), (math.log(r0) - 1e-9, 0), (0.3, 1)]:
        ub = -100.0
        ua = ub + D * T / 0.5         # (1/T - 0.5/T) (ua - ub) = D
        U = [1.0 * ua, 0.5 * ub]       # stored energies are lam * u
        Tn, ln, partner, acc, vs, us, n = O.exchange_h([T, T], lam, U, seed, att)
        assert list(partner) == [1, 0] and n == want
        if want:
            assert list(ln) == [0.5, 1.0] and list(us) == [0.5, 2.0]
            assert list(vs) == [1.0, 1.0] and list(Tn) == [T, T]
        else:
            assert list(ln) == lam and list(us) == [1.0, 1.0]


@pytest.mark.parametrize("D", [-0.3, -1.5])
def test_lambda_acceptance_frequency_is_metropolis(D):
    n, T = 20000, 1.0
    lam = [1.0, 0.6]
    ub = -50.0
    ua = ub + D * T / (1.0 - 0.6)
    U = [ua, 0.6 * ub]
    acc = sum(O.exchange_h([T, T], lam, U, 31, a)[6] for a in range(0, 2 * n, 2))
    p = math.exp(D)
    assert abs(acc / n - p) < 3 * math.sqrt(p * (1 - p) / n)


def test_lambda_scales_forces_and_energy():
    # two atoms: closed-form pair force and energy, scaled by lam
    L, r = 10.0, 1.3
    x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    v = np.zeros((2, 3))
    a = O.Replica(2, L, 1.0, 1, 0, x=x, v=v)
    b = O.Replica(2, L, 1.0, 1, 0, x=x, v=v, lam=0.37)
    uc = 4.0 * (2.5 ** -12 - 2.5 ** -6)
    u = 4.0 * (r ** -12 - r ** -6) - uc
    fx = 24.0 * (2.0 * r ** -13 - r ** -7)
    assert a.U == pytest.approx(u, rel=1e-14) and b.U == pytest.approx(0.37 * u, rel=1e-14)
    assert b.f[1, 0] == pytest.approx(0.37 * fx, rel=1e-13) and b.f[0, 0] == -b.f[1, 0]
    # a liquid: every force component scales
    xs, Lb = melted(108, seed=2, amp=0.12)
    vs = O.init_velocities(108, 1.0, 1, 0)
    p = O.Replica(108, Lb, 1.0, 1, 0, x=xs, v=vs)
    q = O.Replica(108, Lb, 1.0, 1, 0, x=xs, v=vs, lam=0.8)
    assert np.allclose(q.f, 0.8 * p.f, rtol=1e-14, atol=0) and q.U == pytest.approx(0.8 * p.U)


def test_lambda_nve_conserves_scaled_hamiltonian():
    N = 108
    x, L = melted(N, seed=4, amp=0.1)
    v = O.init_velocities(N, 1.0, 2, 0)
    r = O.Replica(N, L, 1.0, 1, 0, tau=0.0, dt=0.002, x=x, v=v, lam=0.7)
    H0 = r.U + r.K
    for _ in range(20):
        r.steps(10)
        assert abs(r.U + r.K - H0) / N < 2e-4


def test_lambda_swap_keeps_effective_energy():
    N = 32
    L = box(N) * 1.3
    ens = O.Ensemble(N, L, [1.0, 1.0], seed=3, tau=0.5, lams=[1.0, 0.5])
    ens.advance([20, 20])
    f0 = [r.f.copy() for r in ens.reps]
    H0 = [r.H for r in ens.reps]
    # force acceptance: u0 well above u1 makes D = (1 - 0.5)(u0 - u1) > 0
    ens.reps[0].rep.U, ens.reps[1].rep.U = 0.0, 0.5 * -100.0
    H0 = [0.0 + ens.reps[0].K + ens.reps[0].econs, -50.0 + ens.reps[1].K + ens.reps[1].econs]
    partner, acc = ens.exchange()
    assert list(acc) == [1, 1]
    assert ens.lams().tolist() == [0.5, 1.0] and ens.temps().tolist() == [1.0, 1.0]
    assert np.allclose(ens.reps[0].f, 0.5 * f0[0], rtol=1e-15, atol=0)
    assert np.allclose(ens.reps[1].f, 2.0 * f0[1], rtol=1e-15, atol=0)
    assert ens.reps[1].U == pytest.approx(-100.0)
    for r, h in zip(ens.reps, H0):
        assert r.H == pytest.approx(h, rel=1e-12)   # econs absorbs the change of U
