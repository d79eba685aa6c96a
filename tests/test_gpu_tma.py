"""The TMA-staged y and z passes against the register four-step passes they replace.

Both kernels run the same arithmetic on every line (only the way the input reaches the
registers differs: a tensor-memory-accelerator box in shared memory instead of per-thread
loads), so every result must be bit-for-bit the same: plain float transforms (forward and
inverse z passes), and whole mixed-precision solves whose inner operator chains use the y and
z passes with derivative, symbol and accumulating transforms.  Grids cover lengths 128 and 256,
planes whose column count is not a multiple of the 16-column tile (box fill at the end), odd
and even h0 (the odd-row box of a y tile starts one column early when h0 is odd), 2D and 3D,
and the transforms are also checked against the oracle's DFT.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import spectral as sp

pytestmark = pytest.mark.gpu

STAGED = 128   # launch-table choice of the TMA-staged kernel
GRIDS = [((32, 24, 256), (2 * math.pi, 1.0, 2 * math.pi)), ((64, 16, 128), (2 * math.pi,) * 3),
         ((48, 40, 256), (1.0, 2.0, 3.0))]


def _force(n, choice, axes=(2,)):
    for axis in axes:
        for d in (-1, 1):
            vd.vd_autotune_set(0, 1, n, axis, d, choice)


@pytest.fixture(autouse=True)
def _restore_table():
    yield
    for n in (128, 256):
        _force(n, -1, (1, 2))


@pytest.mark.parametrize("n,L", GRIDS)
def test_staged_transforms_bitwise_equal_register_kernel(n, L):
    g = sp.Grid(n, L)
    f = inputs.random_field(g.shape, 5)
    G = vd.Grid(n, L)
    x = torch.from_numpy(f).float().cuda()
    out = {}
    for choice in (0, STAGED):
        _force(n[2], choice)
        xh = G.fft_r2c(x, "mixed")
        back = G.fft_c2r(xh, "mixed")
        torch.cuda.synchronize()
        out[choice] = (xh.clone(), back.clone())
    assert torch.equal(out[0][0], out[STAGED][0])
    assert torch.equal(out[0][1], out[STAGED][1])
    ref = sp.fwd(f)[..., : n[0] // 2 + 1]
    got = out[STAGED][0].cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-5


# y tiles are two pair-row boxes, one column early for the odd rows when h0 is odd: both
# parities of h0 (n0 = 30, 90: h0 = 16, 46; n0 = 32, 64: h0 = 17, 33), y lengths 128 and 256
SOLVE_GRIDS = [((32, 24, 256), (2 * math.pi, 1.0, 2 * math.pi)), ((30, 128, 128), (2 * math.pi,) * 3),
               ((32, 128, 128), (2 * math.pi, 1.0, 2.0)), ((90, 256, 16), (2 * math.pi, 2.0, 1.0)),
               ((30, 256), (2 * math.pi, 3.0)), ((64, 256), (1.0, 3.0))]


@pytest.mark.parametrize("precision", ["mixed", "mixed_dd"])
@pytest.mark.parametrize("solver", ["cg", "gmres"])
@pytest.mark.parametrize("n,L", SOLVE_GRIDS)
def test_staged_solves_bitwise_equal_register_kernel(precision, solver, n, L):
    g = sp.Grid(n, L)
    ax = len(n) - 1
    rho = inputs.slab_density(g.n, g.L, 12.0, ax, 0.4 * L[ax], 0.5 * L[ax], 3 * L[ax] / n[ax])
    f = inputs.smooth_random_field(g.n, g.L, 9, kmax=5)
    G = vd.Grid(n, L)
    G.set_density(torch.from_numpy(rho).cuda())
    b = torch.from_numpy(f).cuda()
    res = {}
    for choice in (0, STAGED):
        for m in (128, 256):
            _force(m, choice, (1, 2))
        x, info = G.solve("pressure", solver, b, tol=1e-10, max_it=500, precision=precision)
        assert info["status"] == "converged", info
        res[choice] = (x.clone(), info["iters"])
    assert res[0][1] == res[STAGED][1]
    assert torch.equal(res[0][0], res[STAGED][0])
    # and the solution is the FP64 one within the parity bound
    x64, i64 = G.solve("pressure", solver, b, tol=1e-12, max_it=500, precision="fp64")
    assert float(torch.linalg.vector_norm(res[0][0] - x64) / torch.linalg.vector_norm(x64)) < 12 * 1e-10
