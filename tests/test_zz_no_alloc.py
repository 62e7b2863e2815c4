"""The allocation-free force entry point (for callers that cannot call
cudaMalloc) against the allocating one, through the C ABI, on two calls in a
row (the second call finds the first call's data in the shared scratch).
Collected last on purpose."""
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


def test_no_alloc_matches_allocating_entry_point(re):
    import torch
    for call, (N, seed) in enumerate([(864, 11), (500, 12)]):
        L = inputs.box_length(N)
        x = inputs.jittered_lattice(N, L, 0.1, seed, O.fcc_lattice(N, L))
        xt = torch.tensor(x, device="cuda", dtype=torch.float64)
        f_ref, U_ref = re.lj_forces_device(xt, L, precision="fp64")
        f, U = re.lj_forces_device_noalloc(xt, L)
        torch.cuda.synchronize()
        f_ref, f = f_ref.cpu().numpy(), f.cpu().numpy()
        rms = math.sqrt((f_ref ** 2).sum(1).mean())
        # FP64 tolerance of the force tests: 1e-12 of the rms force, 1e-12 relative energy
        assert np.sqrt(((f - f_ref) ** 2).sum(1)).max() <= 1e-12 * rms, call
        assert abs(U.item() - U_ref.item()) <= 1e-12 * abs(U_ref.item()), call
