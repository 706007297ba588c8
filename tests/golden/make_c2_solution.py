"""Write the CPU oracle's solution of the 3D diffusion workload (40000 fibres,
H = 1/16, replicate 0) to c2_oracle_solution.npz.

The GPU parity test at the full workload size compares the library's solutions
with this file.  Only the oracle and the input generator run here: assembly,
the Schwarz preconditioner with dense Cholesky factors of every star and of
A_0, and textbook PCG (Section 4.2) to a relative residual of 1e-12, so that
the stored solution is far more accurate than the 1e-6 the test asks for.

Run from the repository root:  python tests/golden/make_c2_solution.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.solve import OracleSolver  # noqa: E402
from paper_2207_07488_gb300 import networks as nw  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_oracle_solution.npz")


def main():
    t0 = time.time()
    p = nw.config2(0)
    S = OracleSolver(p)
    res = S.solve(rtol=1e-12, maxit=2000)
    assert res.converged, res.true_relres
    np.savez_compressed(OUT, u=res.u, iters=res.iters, relres=res.true_relres,
                        n_nodes=p.net.n_nodes, n_free=S.A.shape[0])
    print(f"wrote {OUT}: {p.net.n_nodes} nodes, {res.iters} steps, relres {res.true_relres:.2e}, "
          f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
