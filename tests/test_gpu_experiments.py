"""The convergence-rate experiment of Section 6.2 (Table lap_conv) through the library,
against the oracle on networks small enough for it: the K-norm errors of PCG after
every step and the rates tau_l must agree (the same FP64 textbook iteration on both
sides, so the rates agree to rounding), on the uniform fibre network of Section 6.1
with gamma = 1 and gamma ~ U[0.1, 1], and on the grid network."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.pcg import convergence_rates
from oracle.solve import OracleSolver
from paper_2207_07488_gb300 import networks as nw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300.experiments import pcg_rates  # noqa: E402


def _oracle_rates(p, reduction=1e-8):
    S = OracleSolver(p, local="dense")
    b = S.rhs()
    u = spla.spsolve(S.A.tocsc(), b)
    its = []
    S.solve(rtol=1e-13, callback=lambda x, i: its.append(x.copy()))
    taus, errs = convergence_rates(S.A, u, its)
    last = int(np.nonzero(errs <= reduction * errs[0])[0][0])
    return errs[: last + 1], taus[: last - 1]


def _cases():
    net = nw.fiber_heat_network(11, total_length=80.0)
    yield "fibre-H4", nw.fiber_heat_problem(net, 0.25)
    yield "fibre-H8", nw.fiber_heat_problem(net, 0.125)
    yield "fibre-weighted-H4", nw.fiber_heat_problem(net, 0.25, gamma=nw.heat_weights(net, 12))
    yield "grid5-H4", nw.grid_heat_problem(5, 0.25)


@pytest.mark.parametrize("name,p", list(_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_rates_match_the_oracle(name, p):
    errs_o, taus_o = _oracle_rates(p)
    got = pcg_rates(p)
    assert got["steps"] == errs_o.size - 1, (got["steps"], errs_o.size - 1)
    np.testing.assert_allclose(got["errors"] / got["errors"][0], errs_o / errs_o[0], rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(got["taus"], taus_o, atol=1e-6)
    assert got["max"] < 1.0


def test_recorded_iterates_are_the_iterates():
    """spnet_pc_record_iterates: row l of the record is the result of the same solve
    stopped after l steps (a deterministic textbook iteration), bit for bit."""
    import torch
    from paper_2207_07488_gb300 import spnet
    net = nw.fiber_heat_network(11, total_length=80.0)
    p = nw.fiber_heat_problem(net, 0.25)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_FP64, star_set=spnet.STARS_ALL,
                              patch=p.patch, flexible=0, max_restarts=0)
    free = np.setdiff1d(np.arange(p.n_dof), p.dirichlet_dofs)
    hist = torch.full((6, int(op.info.n_free)), float("nan"), dtype=torch.float64, device="cuda")
    pc.record_iterates(hist)
    u, st = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-12, maxit=500, raise_on_noconv=False)
    pc.record_iterates(None)
    H = hist.cpu().numpy()
    assert np.all(H[0] == 0.0)
    for l in (1, 2, 5):
        x, _ = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-300, maxit=l, raise_on_noconv=False)
        assert np.array_equal(H[l], x[free]), l
    assert st[0].iterations > 5
    # recording stopped: a later solve leaves the buffer alone
    hist.fill_(-1.0)
    spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-12, maxit=500, raise_on_noconv=False)
    assert bool((hist == -1.0).all())
    pc.close()
    op.close()


def test_record_iterates_rejects_bad_buffers():
    import ctypes as C
    import torch
    from paper_2207_07488_gb300 import spnet
    p = nw.grid_heat_problem(5, 0.25)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_FP64, star_set=spnet.STARS_ALL,
                              patch=p.patch)
    lib = spnet.load()
    host = np.zeros((4, int(op.info.n_free)))
    assert lib.spnet_pc_record_iterates(pc.handle, C.c_void_p(host.ctypes.data), 4) == spnet.ERR_BAD_INPUT
    dev = torch.zeros((4, int(op.info.n_free)), dtype=torch.float64, device="cuda")
    assert lib.spnet_pc_record_iterates(pc.handle, None, 4) == spnet.ERR_BAD_INPUT
    assert lib.spnet_pc_record_iterates(pc.handle, C.c_void_p(dev.data_ptr()), 0) == spnet.ERR_BAD_INPUT
    assert lib.spnet_pc_record_iterates(pc.handle, C.c_void_p(dev.data_ptr()), -1) == spnet.ERR_BAD_INPUT
    assert lib.spnet_pc_record_iterates(pc.handle, C.c_void_p(dev.data_ptr() + 4), 1) == spnet.ERR_BAD_INPUT
    with pytest.raises(ValueError):
        pc.record_iterates(dev[:, :-1])
    pc.close()
    op.close()
