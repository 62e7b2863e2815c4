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


def paper_workload_rows(advance, exchange, temps, cycles, nx):
    rows = []
    for _ in range(cycles):
        advance(nx)
        T_before = temps()
        partner, acc = exchange()
        rows.append(pair_row(T_before, partner, acc, len(T_before)))
    return np.array(rows)


def test_paper_workload_acceptance_matches_oracle(re):
    """The Example section's workload: N = 4000 at density 0.8442, cutoff 2.5,
    list radius 3.0, T_k = 0.7 * 1.0275^k (8 replicas), the liquid melted at
    high temperature first.  The GPU's acceptance must match the FP64 oracle's
    on the same recipe (independent trajectories, batch-mean errors).  The
    paper quotes "approximately 30 %" for this ladder with no error bar; both
    implementations give about 20 % here (recorded as a reading of the paper),
    so the band below is loose and the oracle comparison is the pin."""
    N, R, cycles, nx = 4000, 8, 1200, 10
    L = inputs.box_length(N)
    hot = inputs.geometric_ladder(1.6, 1.9, R)
    temps = inputs.paper_ladder(R)
    scale = np.sqrt(temps / hot)
    # GPU
    melt = re.Context(N, L, 2.5, hot, 77)
    melt.advance(1500)
    x, v = melt.get_state()
    ctx = re.Context(N, L, 2.5, temps, 78)
    ctx.set_state(x, v * np.repeat(scale, N)[:, None])
    ctx.advance(1000)
    g = paper_workload_rows(lambda n: ctx.advance(n), lambda: ctx.exchange(outputs=True),
                            ctx.temps, cycles, nx)
    # oracle, its own melt
    om = O.Ensemble(N, L, hot, 177)
    om.advance([1500] * R)
    xs = np.array([r.x for r in om.reps])
    vs = np.array([r.v * scale[k] for k, r in enumerate(om.reps)])
    ens = O.Ensemble.from_state(N, L, temps, 178, xs, vs)
    ens.advance([1000] * R)
    o = paper_workload_rows(lambda n: ens.advance([n] * R), ens.exchange, ens.temps, cycles, nx)
    ag = np.nanmean(g)
    ao = np.nanmean(o)
    # batch means of the all-pair acceptance: 20 batches of 60 attempts (the
    # error estimate of 10 batches was itself uncertain by about a quarter)
    nb = 20
    bg = np.array([np.nanmean(b) for b in np.array_split(g, nb)])
    bo = np.array([np.nanmean(b) for b in np.array_split(o, nb)])
    se = math.sqrt(bg.var(ddof=1) / nb + bo.var(ddof=1) / nb)
    assert abs(ag - ao) <= 3 * se + 1e-9, (ag, ao, se)
    assert 0.12 < ag < 0.45, ag
