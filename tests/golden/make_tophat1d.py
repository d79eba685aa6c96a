"""Write tophat1d.json: oracle figures of the 1D top-hat workload (N = 256 on [0, 2 pi),
rho = 1 + (r-1)/2 (tanh((x-pi/2)/d) - tanh((x-3pi/2)/d)), r = 3, d = 0.05; the 16-mode rhs of
seed 1), the case of the paper's Sec. 3.2 pressure study with its density ratio and interface.

Values, all from the oracle (oracle/ only):
* condition numbers from dense assembly, as the paper measures them (SVD, Sec. 3.1/3.2), on
  the range of the operator: kappa of L~, of the left- and right-preconditioned M+ L~ and
  L~ M+, and the eigenvalue ratio of M+ L~ (bounded by rho_max / rho_min = 3);
* the oracle's CG, GMRES(30) and RMR iteration counts to a 1e-12 relative residual from
  x0 = 0, with the true residual of each result.

Run: python tests/golden/make_tophat1d.py   (rewrites tests/golden/tophat1d.json)
"""

import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import dense, operators as op, solvers as sv, spectral as sp  # noqa: E402
from paper_2403_06654_gb300 import inputs  # noqa: E402


def compute():
    n = 256
    g = sp.Grid((n,), (2 * math.pi,))
    rho = inputs.tophat_1d(n=n)
    f = sp.project_range(inputs.modes_rhs_1d(n=n), g)
    A = dense.assemble(lambda v: op.apply_pressure(rho, v, g), g.shape)
    M = dense.assemble(lambda v: sp.precond_pressure(v, g), g.shape)
    w = dense.eig_range(M @ A)
    out = {"workload": "1D periodic N=256 top-hat r=3 d=0.05, 16-mode rhs (seed 1)",
           "kappa_L": dense.cond_on_range(A), "kappa_left_MA": dense.cond_on_range(M @ A),
           "kappa_right_AM": dense.cond_on_range(A @ M),
           "eig_ratio_MA": float(np.max(w.real) / np.min(w.real)),
           "eig_bound_rho_ratio": float(rho.max() / rho.min()), "solvers": {}}
    Af, Mf = op.pressure_system(rho, g)
    for name in ("cg", "gmres", "rmr"):
        r = sv.solve(name, Af, Mf, f, tol=1e-12, maxit=400, restart=30)
        out["solvers"][name] = {"iters": r.iters, "status": r.status, "relres_true": r.relres_true}
    return out


if __name__ == "__main__":
    data = compute()
    with open(os.path.join(HERE, "tophat1d.json"), "w") as fh:
        json.dump(data, fh, indent=1)
    print(json.dumps(data, indent=1))
