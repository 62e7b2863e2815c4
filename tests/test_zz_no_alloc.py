"""The allocation-free force entry point (for callers that cannot call
cudaMalloc) against the allocating one and against the FP64 oracle, through the
C ABI, on calls in a row (each call finds the previous call's data in the
shared scratch array).  Collected last on purpose."""
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


def rel_force_err(f, fo):
    rms = math.sqrt((fo ** 2).sum(1).mean())
    return np.sqrt(((f - fo) ** 2).sum(1)).max() / rms


def check_call(re, x, L, with_alloc=True):
    """One no-allocation call: equal to the allocating FP64 entry point (where
    that one accepts the shape) and to the oracle's brute-force sum within the
    FP64 force tolerance (1e-12 of the rms force, energies 1e-12 relative)."""
    import torch
    xt = torch.tensor(x, device="cuda", dtype=torch.float64)
    f, U = re.lj_forces_device_noalloc(xt, L)
    torch.cuda.synchronize()
    f = f.cpu().numpy()
    if with_alloc:
        f_ref, U_ref = re.lj_forces_device(xt, L, precision="fp64")
        torch.cuda.synchronize()
        assert rel_force_err(f, f_ref.cpu().numpy()) <= 1e-12
        assert abs(U.item() - U_ref.item()) <= 1e-12 * abs(U_ref.item())
    fo, Uo = O.forces_brute(x, L)
    assert rel_force_err(f, fo) <= 1e-12
    assert abs(U.item() - Uo) <= 1e-12 * abs(Uo)


def liquid_like(N, seed, amp=0.1):
    L = inputs.box_length(N)
    return inputs.jittered_lattice(N, L, amp, seed, O.fcc_lattice(N, L)), L


def test_no_alloc_matches_allocating_entry_point_and_oracle(re):
    # larger, then smaller: the second call must not see the first call's atoms
    for N, seed in [(864, 11), (500, 12)]:
        x, L = liquid_like(N, seed)
        check_call(re, x, L)


def test_no_alloc_smaller_then_largest(re):
    # smaller, then the largest size the fixed array holds (4096 atoms)
    for N, seed in [(256, 13), (4000, 14)]:
        x, L = liquid_like(N, seed)
        check_call(re, x, L)
    N = 4096
    L = inputs.box_length(N)
    rng = np.random.default_rng(15)
    # 4096 atoms on a jittered 16^3 simple-cubic grid at the liquid density
    g = (np.stack(np.meshgrid(*[np.arange(16)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5)
    x = (g * (L / 16) + rng.uniform(-0.05, 0.05, g.shape)) % L
    check_call(re, x, L)


def test_no_alloc_all_pairs_fallback(re):
    """4096 atoms in a dilute box of side 80: the cell table would not fit the
    list build's shared memory, so the call takes the all-pairs list path.
    (The allocating entry point refuses this shape: its batched kernel would
    need the same table in shared memory.)"""
    N, L = 4096, 80.0
    rng = np.random.default_rng(16)
    g = (np.stack(np.meshgrid(*[np.arange(16)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5)
    x = (g * (L / 16) + rng.uniform(-1.5, 1.5, g.shape)) % L
    check_call(re, x, L, with_alloc=False)


def test_no_alloc_limits_and_errors(re):
    import torch
    # one atom beyond the fixed array's limit: refused before any device work
    N = 4097
    x = torch.zeros((N, 3), device="cuda", dtype=torch.float64)
    with pytest.raises(re.REError) as e:
        re.lj_forces_device_noalloc(x, 30.0)
    assert e.value.code == re.RE_EINVAL
    # 500 atoms squeezed into a 4.5-sigma cube of a 16-sigma box: far more
    # neighbours per atom than the capacity taken from the mean density
    rng = np.random.default_rng(17)
    g = (np.stack(np.meshgrid(*[np.arange(8)] * 3, indexing="ij"), -1).reshape(-1, 3)[:500] + 0.5)
    xc = g * 0.56 + rng.uniform(-0.02, 0.02, g.shape) + 5.0
    with pytest.raises(re.REError) as e:
        re.lj_forces_device_noalloc(torch.tensor(xc, device="cuda", dtype=torch.float64), 16.0)
    assert e.value.code == re.RE_EOVERFLOW
    # the shared array is usable again after a refused call
    x, L = liquid_like(864, 18)
    check_call(re, x, L)
