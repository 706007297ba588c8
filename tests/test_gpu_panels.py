"""Dense blocks of large stars solved by panels on tensor cores (k right-hand sides, FP32).

On a 2D network whose stars hold 1500-2000 dofs, the elimination of every star
ends in a dense block of well over 32 nodes; with batch_rhs >= 2 the library
solves those blocks by 16-row panels with tensor-core products instead of level
by level.  Checked against the oracle (Section 4.1, eq. defPj: the exact local
solves): the star term per column, per star within 1e-2 and over all dofs within
2e-4 (the mixed-precision bounds of the other parity tests), whole batched
solves to relative error 1e-6, agreement with the level-by-level solve of the
same blocks, and a column's result independent of the other columns.
"""
import functools

import numpy as np
import pytest

from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw
from parity_checks import check_star_term, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402


@functools.lru_cache(maxsize=None)
def problem():
    net = nw.fiber_network_2d(2500, 0.1, seed=77)
    return nw.scalar_band_problem(net, 1.0 / 8, name="2d-2500fib-H8")


@functools.lru_cache(maxsize=None)
def oracle():
    return OracleSolver(problem(), local="dense")


@functools.lru_cache(maxsize=None)
def lib(panels, batch=32):
    p = problem()
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED, batch_rhs=batch,
                              panels=panels)
    return op, pc


def test_dense_blocks_are_solved_by_panels():
    _, pc = lib(True)
    core = pc.export(spnet.EXPORT_STAR_CORE)
    assert pc.info.panel_stars == int((core >= 32).sum()) > 0
    assert np.median(core) >= 64
    _, pc0 = lib(False)
    assert pc0.info.panel_stars == 0


@pytest.mark.parametrize("k", [3, 8, 32])
def test_star_term_against_the_oracle(k):
    o = oracle()
    _, pc = lib(True)
    _, pc0 = lib(False)
    R = np.random.default_rng(50 + k).standard_normal((k, o.A.shape[0]))
    Zs = pc.apply_batch(R, which=2)
    Z0 = pc0.apply_batch(R, which=2)
    for j in sorted({0, k // 2, k - 1}):
        check_star_term(o, R[j], Zs[j], "mixed")
        # the same blocks solved level by level: the same star term up to FP32 rounding
        assert rel(Zs[j], Z0[j]) <= 1e-4, j
    Z = pc.apply_batch(R)
    assert rel(Z[0], o.B.apply(R[0])) <= 2e-4


def test_batched_solve_against_the_oracle():
    p = problem()
    o = oracle()
    op, pc = lib(True)
    rng = np.random.default_rng(61)
    F = rng.uniform(0.0, 1.0, size=(32, p.n_dof))
    G = np.tile(p.dirichlet_vals, (32, 1))
    U, st = spnet.pcg_solve(op, pc, F, G, rtol=1e-8)
    assert all(s.converged and s.relres <= 1e-8 for s in st)
    op0, pc0 = lib(False)
    U0, st0 = spnet.pcg_solve(op0, pc0, F, G, rtol=1e-8)
    for j in (0, 31):
        ref = o.solve(f=F[j], g=G[j], rtol=1e-8, flexible=True)
        assert rel(U[j], ref.u) <= 1e-6, j
        assert abs(st[j].iterations - st0[j].iterations) <= 3, (st[j].iterations, st0[j].iterations)


def test_a_column_does_not_depend_on_its_neighbours():
    o = oracle()
    _, pc = lib(True)
    R = np.random.default_rng(70).standard_normal((9, o.A.shape[0]))
    Za = pc.apply_batch(R[[0, 1, 2, 3]], which=2)
    Zb = pc.apply_batch(R[[4, 0, 5, 6]], which=2)
    Zc = pc.apply_batch(R[[7, 8, 0]], which=2)  # 3 columns: the same padded width 4
    np.testing.assert_array_equal(Za[0], Zb[1])
    np.testing.assert_array_equal(Za[0], Zc[2])


@functools.lru_cache(maxsize=None)
def downscaled_large():
    # the 400000-fibre workload's geometry scaled by 4 into the unit cube (fibres of length
    # 0.4, contacts below 0.016, 400000 / 4^3 = 6250 fibres, H = 4/32): a quarter-size cube of
    # that network, 139k nodes, 343 stars of ~2400 dofs whose eliminations end in dense blocks
    net = nw.fiber_network_3d(6250, 0.4, 0.016, nw.config_seed(5, 1))
    p = nw.scalar_band_problem(net, 1.0 / 8, name="3d-6250fib-L0.4-H8")
    return p, OracleSolver(p, local="sparse")


def test_downscaled_large_network_32_rhs():
    p, o = downscaled_large()
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED, batch_rhs=32)
    assert pc.info.panel_stars > 0
    R = np.random.default_rng(80).standard_normal((32, o.A.shape[0]))
    Zs = pc.apply_batch(R, which=2)
    Z = pc.apply_batch(R)
    for j in (0, 31):
        check_star_term(o, R[j], Zs[j], "mixed")
        assert rel(Z[j], o.B.apply(R[j])) <= 2e-4
    rng = np.random.default_rng(81)
    F = rng.uniform(0.0, 1.0, size=(32, p.n_dof))
    G = np.tile(p.dirichlet_vals, (32, 1))
    U, st = spnet.pcg_solve(op, pc, F, G, rtol=1e-8)
    assert all(s.converged and s.relres <= 1e-8 for s in st)
    ref = o.solve(f=F[5], g=G[5], rtol=1e-8, flexible=True)
    assert rel(U[5], ref.u) <= 1e-6
