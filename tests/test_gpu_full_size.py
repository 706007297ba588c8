"""Parity at the full size of the measured workload (3D diffusion, 40000 fibres,
H = 1/16: 168,801 free dofs, 3375 stars, 595 coarse tiles), on the paths the
benchmark times.

- The star term and B r of the one-vector path, element-wise against the
  oracle: in FP64 every entry within 1e-9 of the size of the stars that hold
  it (so one wrong star among 3375 fails), in mixed precision every star's
  dofs within 1e-2 and all dofs within 2e-4 (FP32 factors of stars whose
  condition numbers reach ~5e5).
- Whole solves, one request at a time and through the server (the served
  mixed path of the benchmark, with its star-mapping tuner and the coarse
  product over all tiles), against the oracle's solution stored in
  tests/golden/c2_oracle_solution.npz (written by make_c2_solution.py, which
  calls only the oracle): recomputed residual <= 1e-8, relative error <= 1e-6.
"""
import functools
import os

import numpy as np
import pytest

from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw
from parity_checks import check_entries, check_star_term, rel, star_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_oracle_solution.npz")
PREC = {"fp64": spnet.PREC_FP64, "mixed": spnet.PREC_MIXED}


@functools.lru_cache(maxsize=None)
def problem():
    return nw.config2(0)


@functools.lru_cache(maxsize=None)
def oracle():
    return OracleSolver(problem(), local="dense")


@functools.lru_cache(maxsize=None)
def lib(prec):
    p = problem()
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=PREC[prec])
    return op, pc


@functools.lru_cache(maxsize=None)
def residual():
    return np.random.default_rng(41).standard_normal(oracle().A.shape[0])


@functools.lru_cache(maxsize=None)
def scale():
    return star_scale(oracle(), residual())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_star_term_and_B_elementwise(prec):
    o = oracle()
    _, pc = lib(prec)
    assert pc.info.n_stars == o.B.n_stars == 3375
    r = residual()
    sref = check_star_term(o, r, pc.stars(r), prec, sc=scale() if prec == "fp64" else None)
    cref = o.B.coarse_term(r)
    got = pc.apply(r)
    if prec == "fp64":
        check_entries(got, cref + sref, 1e-9 * (scale() + np.abs(cref).max()), "B")
    else:
        assert rel(got, cref + sref) <= 2e-4


def _golden():
    d = np.load(GOLDEN)
    u = d["u"]
    assert u.size == problem().net.n_nodes and float(d["relres"]) <= 1e-12
    return u


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_solution_against_oracle(prec):
    p = problem()
    o = oracle()
    op, pc = lib(prec)
    u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-8)
    assert st[0].converged == 1 and st[0].relres <= 1e-8
    b = o.rhs()
    assert np.linalg.norm(b - o.A @ u[o.free]) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert rel(u, _golden()) <= 1e-6


def test_full_size_served_solution_against_oracle():
    # the benchmark's request: host arrays through the server, mixed precision, the
    # star mapping tuned per size class, four requests in flight
    p = problem()
    sv = spnet.Server(max_inflight=4)
    try:
        tickets = [sv.submit(p, precision=spnet.PREC_MIXED, rtol=1e-8) for _ in range(4)]
        outs = [sv.wait(t) for t in tickets]
    finally:
        sv.close()
    ref = _golden()
    for x, res in outs:
        assert res["status"] == 0 and res["relres"] <= 1e-8
        assert rel(x, ref) <= 1e-6
    for x, _ in outs[1:]:
        np.testing.assert_array_equal(x, outs[0][0])
