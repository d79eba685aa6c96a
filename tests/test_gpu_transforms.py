"""Plain transforms through the C ABI (vd_fft_r2c / vd_fft_c2r) against the oracle's DFT.

The half spectrum of the library is the first n0/2 + 1 x-columns of the oracle's full
unnormalised DFT (oracle.spectral.fwd); the inverse divides by N.  Double transforms are
compared element by element at 1e-12 of the largest coefficient, float-pair ones at 1e-12
(their rounding is ~2^-48 per operation), float ones at 1e-5.  Sizes span radix 2, 3 and 5,
the register four-step kernels (lengths 128/256, x half-length 64/128/256) and ragged tiles.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import spectral as sp

pytestmark = pytest.mark.gpu

GRIDS = [((240,), (2 * math.pi,)), ((48, 30), (2 * math.pi, 1.5)), ((256, 256), (1.0, 1.0)),
         ((20, 12, 30), (2 * math.pi, 1.0, 3.0)), ((128, 128, 16), (2 * math.pi,) * 3),
         ((512, 40, 10), (2 * math.pi,) * 3)]
TOL = {"fp64": 1e-12, "mixed_dd": 1e-12, "mixed": 1e-5}


@pytest.mark.parametrize("n,L", GRIDS)
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_dd"])
def test_r2c_c2r_match_oracle(n, L, precision):
    g = sp.Grid(n, L)
    f = inputs.random_field(g.shape, 7)
    ref = sp.fwd(f)[..., : n[0] // 2 + 1]
    G = vd.Grid(n, L)
    dt = torch.float32 if precision == "mixed" else torch.float64
    x = torch.from_numpy(f).to(dt).cuda()
    xh = G.fft_r2c(x, precision)
    got = xh.cpu().numpy().astype(np.complex128)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < TOL[precision], err
    # inverse of the oracle's half spectrum
    refh = torch.from_numpy(np.ascontiguousarray(ref)).to(torch.complex64 if precision == "mixed" else torch.complex128)
    back = G.fft_c2r(refh.cuda(), precision).cpu().numpy().astype(np.float64)
    err2 = np.max(np.abs(back - f)) / np.max(np.abs(f))
    assert err2 < TOL[precision], err2
