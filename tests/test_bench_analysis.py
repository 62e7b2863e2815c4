"""The analysis code behind the reported numbers, pinned to closed forms (CPU):
the unique in-cutoff pair count that the roofline's algorithmic flops use, and
the diffusion-coefficient estimator of ln T (Diffusion in temperature space)."""
import itertools

import numpy as np

import bench
from paper_0812_1633_gb300 import inputs


def fcc(N, L):
    """Perfect FCC lattice of N = 4 k^3 atoms in a cube of side L (built here,
    independently of the oracle and of the library)."""
    k = round((N / 4) ** (1 / 3))
    a = L / k
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.array(list(itertools.product(range(k), repeat=3)), dtype=float)
    return ((cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) + 0.25) * a


def test_in_cutoff_pairs_on_the_fcc_lattice():
    # FCC shells at a * sqrt(n / 2): n = 1..4 (12, 6, 24, 12 neighbours) lie
    # inside rc = 2.5 at rho = 0.8442 (a = 1.6796; shell 5 at 2.656 is outside),
    # so every atom has 54 neighbours: 27 unique pairs per atom
    for N in (256, 500, 864):
        L = inputs.box_length(N)
        cfg = ("", [(N, 1, 1.0, 1.0)])
        assert bench.in_cutoff_pairs_per_atom(fcc(N, L), cfg) == 27.0


def test_in_cutoff_pairs_uniform_gas():
    # an ideal gas: rho * 4/3 pi rc^3 / 2 unique pairs per atom on average
    N = 2048
    L = inputs.box_length(N)
    rng = np.random.default_rng(3)
    cfg = ("", [(N, 4, 1.0, 1.0)])
    x = rng.random((4 * N, 3)) * L
    want = N / L ** 3 * 4.0 / 3.0 * np.pi * 2.5 ** 3 / 2
    got = bench.in_cutoff_pairs_per_atom(x, cfg)
    assert abs(got - want) < 0.02 * want


def test_diffusion_estimator_recovers_a_known_coefficient():
    # ln T performs a random walk with variance 2 D (steps between attempts)
    rng = np.random.default_rng(7)
    D, A, R = 3e-5, 20000, 16
    ds = rng.integers(5, 16, size=(A, R))             # uneven strides, as in the async scheme
    steps = np.cumsum(ds, axis=0)
    y = np.cumsum(rng.normal(0.0, np.sqrt(2 * D * ds)), axis=0)
    got = bench.msd_diffusion(np.exp(y), steps)
    assert abs(got - D) < 0.05 * D


def test_drift_slope_estimator_recovers_known_slopes():
    # H~/N rising linearly in time at a known rate per replica, plus noise
    rng = np.random.default_rng(11)
    N, R = 4000, 5
    t = np.arange(0.0, 100.0, 0.5)
    rates = np.array([1e-6, -2e-6, 0.0, 5e-7, 3e-6])
    H = N * (rates[None, :] * t[:, None] + rng.normal(0.0, 1e-7, (t.size, R))) - 5.0 * N
    got = bench.drift_slopes(t, H, N)
    assert np.allclose(got, rates, atol=5e-9)
