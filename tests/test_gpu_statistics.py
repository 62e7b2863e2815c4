"""Long-run statistics of the GPU mixed path against the FP64 oracle.

Trajectories diverge (molecular dynamics is chaotic), so long runs are compared
statistically: exchange acceptance per sorted-temperature pair within 3
standard errors (batch means), and the paper's own figure of about 30 %
acceptance for the ladder T_k = 0.7 * 1.0275^k at N = 4000 (Example section).
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


def batch_rates(acc, n_batches=10):
    """acc: (attempts, pairs) 0/1 for attempted pairs, nan where not attempted.
    Returns per-pair rate and batch-means standard error."""
    B = len(acc) // n_batches
    means = np.array([np.nanmean(acc[b * B:(b + 1) * B], axis=0) for b in range(n_batches)])
    return np.nanmean(acc[:B * n_batches], axis=0), means.std(axis=0, ddof=1) / math.sqrt(n_batches)


def run_gpu(re, N, temps, seed, cycles, nx, burn):
    ctx = re.Context(N, inputs.box_length(N), 2.5, temps, seed, precision="mixed")
    R = len(temps)
    rows = []
    for c in range(burn + cycles):
        ctx.advance(nx)
        T_before = ctx.temps()
        partner, acc = ctx.exchange(outputs=True)
        if c >= burn:
            rows.append(pair_row(T_before, partner, acc, R))
    return np.array(rows)


def pair_row(T, partner, acc, R):
    """Acceptance (1/0) of each sorted-temperature pair position, nan if not attempted."""
    order = np.argsort(T)
    row = np.full(R - 1, np.nan)
    for k in range(R - 1):
        a, b = order[k], order[k + 1]
        if partner[a] == b:
            row[k] = float(acc[a])
    return row


def run_oracle(N, temps, seed, cycles, nx, burn):
    ens = O.Ensemble(N, inputs.box_length(N), temps, seed)
    R = len(temps)
    rows = []
    for c in range(burn + cycles):
        ens.advance([nx] * R)
        T_before = ens.temps()
        partner, acc = ens.exchange()
        if c >= burn:
            rows.append(pair_row(T_before, partner, acc, R))
    return np.array(rows)


def test_acceptance_per_pair_matches_oracle(re):
    N, R, seed = 256, 8, 2024
    temps = inputs.geometric_ladder(0.8, 1.6, R)
    cycles, nx, burn = 2000, 10, 100
    g = run_gpu(re, N, temps, seed, cycles, nx, burn)
    o = run_oracle(N, temps, seed + 1, cycles, nx, burn)
    pg, sg = batch_rates(g)
    po, so = batch_rates(o)
    for k in range(R - 1):
        se = math.sqrt(sg[k] ** 2 + so[k] ** 2)
        assert abs(pg[k] - po[k]) <= 3 * se + 1e-9, (k, pg[k], po[k], se)
    # the acceptance decreases with temperature only mildly on a geometric ladder
    assert 0.05 < pg.mean() < 0.95


def test_paper_acceptance_about_30_percent(re):
    """N = 4000 at reduced density 0.844-ish, T_k = 0.7 * 1.0275^k: about 30 %
    acceptance (Example section).  The liquid is prepared by melting at high
    temperature, then equilibrated on the ladder."""
    N, R, seed = 4000, 8, 77
    L = inputs.box_length(N)
    hot = inputs.geometric_ladder(1.6, 1.9, R)
    melt = re.Context(N, L, 2.5, hot, seed)
    melt.advance(3000)
    x, v = melt.get_state()
    temps = inputs.paper_ladder(R)
    ctx = re.Context(N, L, 2.5, temps, seed + 1)
    scale = np.repeat(np.sqrt(temps / hot), N)[:, None]
    ctx.set_state(x, v * scale)
    ctx.advance(2000)
    att0, acc0 = ctx.accept_stats()
    for _ in range(1000):
        ctx.advance(10)
        ctx.exchange()
    att, acc = ctx.accept_stats()
    rate = (acc - acc0).sum() / (att - att0).sum()
    assert 0.2 < rate < 0.4, rate
