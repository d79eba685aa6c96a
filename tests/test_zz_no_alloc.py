"""The pressure apply that allocates no device memory, checked against vd_apply_op.

Callers that cannot allocate (a host framework's memory pool owns the device, plugins with
a fixed device footprint, loops that must not synchronise through an allocation) use
vd_apply_pressure_noalloc, which keeps every intermediate in one fixed device array.  Its
output must equal the workspace-based vd_apply_op's within the apply tolerance of the other
parity tests (1e-12 relative, max norm), on two calls in a row (the array keeps the last
call's contents), and grids too large for the array must be refused with a clear error.
This file is collected last so that a run stopping at the first failure has run the rest.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    ((256,), (2 * math.pi,)),
    ((48, 30), (2 * math.pi, 1.5)),
    ((20, 12, 30), (2 * math.pi, 1.0, 3.0)),
    ((64, 64, 64), (2 * math.pi,) * 3),
    ((512, 1024), (1.0, 2.0)),
]


def relmax(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("n,L", CASES)
def test_noalloc_matches_apply_op_twice(n, L):
    shape = tuple(reversed(n))
    f = inputs.smooth_random_field(n, L, 3, kmax=4)
    f = (f - f.min()) / (f.max() - f.min())
    rho = torch.from_numpy(1.0 + 3.0 * f).cuda()
    G = vd.Grid(n, L)
    G.set_density(rho)
    for seed in (11, 12):
        x = torch.from_numpy(inputs.random_field(shape, seed)).cuda()
        ref = G.apply("pressure", x)
        out = torch.full_like(x, float("nan"))
        vd.vd_apply_pressure_noalloc(n, L, rho, x, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert relmax(out, ref) < 1e-12


def test_noalloc_refuses_grids_beyond_the_array():
    n, L = (128, 128, 128), (2 * math.pi,) * 3
    rho = torch.ones(tuple(reversed(n)), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(rho)
    out = torch.zeros_like(rho)
    with pytest.raises(vd.VDError) as e:
        vd.vd_apply_pressure_noalloc(n, L, rho, x, out)
    assert e.value.status == vd.VD_ERR_INVALID_ARG and "too large" in str(e.value)


def test_noalloc_rejects_bad_density():
    n, L = (16, 12), (1.0, 1.0)
    rho = torch.full((12, 16), -1.0, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(rho)
    out = torch.zeros_like(rho)
    with pytest.raises(vd.VDError) as e:
        vd.vd_apply_pressure_noalloc(n, L, rho, x, out)
    assert e.value.status == vd.VD_ERR_INVALID_ARG
