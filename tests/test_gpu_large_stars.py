"""Stars of several thousand dofs (coarse elements holding many nodes).

The serving stream chooses H so that about 300 nodes fall in each coarse
element, which gives stars of 1-3 thousand dofs whose elimination ends in a
dense block larger than the set-up's first scratch size; set-up then repeats
with a larger block.  Here a 2D network of 3000 fibres at H = 1/6 (stars of up
to about 4300 dofs) is compared with the oracle: B r (Sections 4.1-4.2) at the
tolerance of the parity tests, and whole solves (Section 4.2) to a recomputed
residual of 1e-8 and a relative error of at most 1e-6, one right-hand side and
several stepped together.
"""
import functools

import numpy as np
import pytest

from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402

PREC = {"fp64": spnet.PREC_FP64, "mixed": spnet.PREC_MIXED}
TOL = {"fp64": 1e-10, "mixed": 2e-4}


@functools.lru_cache(maxsize=None)
def problem():
    net = nw.fiber_network_2d(3000, 0.1, 77)
    return nw.scalar_band_problem(net, 1.0 / 6, name="2d-3000fib-H6")


@functools.lru_cache(maxsize=None)
def oracle():
    return OracleSolver(problem(), local="dense")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_stars_against_the_oracle(prec):
    p = problem()
    o = oracle()
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=PREC[prec], batch_rhs=3)
    assert pc.info.max_star == max(o.B.star_sizes) and pc.info.max_star > 4000
    r = np.random.default_rng(8).standard_normal(o.A.shape[0])
    assert rel(pc.apply(r), o.B.apply(r)) <= TOL[prec]
    u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-8)
    ref = o.solve(rtol=1e-8, flexible=(prec == "mixed"))
    assert st[0].converged and st[0].relres <= 1e-8
    assert rel(u, ref.u) <= 1e-6
    # three right-hand sides stepped together
    rng = np.random.default_rng(9)
    F = rng.uniform(0.0, 1.0, size=(3, p.n_dof))
    G = np.tile(p.dirichlet_vals, (3, 1))
    U, st3 = spnet.pcg_solve(op, pc, F, G, rtol=1e-8)
    for j in range(3):
        assert st3[j].converged and st3[j].relres <= 1e-8, j
        b = o.rhs(F[j], G[j])
        assert np.linalg.norm(b - o.A @ U[j][o.free]) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6), j
