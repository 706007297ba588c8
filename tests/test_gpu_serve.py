"""Serving (spnet_server_*): requests against the direct calls, alone and in the mix.

A request runs the same kernels as the direct calls (assembly, operator,
preconditioner, PCG), and every kernel reduces in a fixed order, so a
request's solution must be bitwise the same whether it runs alone or among
other requests of different sizes and models, and the same as the direct
calls on the same problem.
"""
import numpy as np
import pytest

from paper_2207_07488_gb300 import networks as nw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402


def _small3d(seed=31, n=1500):
    # (seed, n) pairs whose coarse matrix is SPD at H = 1/4; sparser draws can
    # leave coarse functions linearly dependent on the free nodes
    net = nw.fiber_network_3d(n, 0.2, 0.01, seed=seed)
    return nw.scalar_band_problem(net, 0.25, name=f"small3d-{seed}")


def _truss():
    net = nw.fiber_network_3d(1200, 0.25, 0.02, seed=41, keep="clamped_x")
    return nw.truss_band_problem(net, 0.25, name="truss")


def _direct(p, precision):
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=precision,
                              star_set=spnet.STARS_ALL if p.star_set == "all" else spnet.STARS_INTERIOR)
    u, _ = spnet.pcg_solve(op, pc, p.f, p.dirichlet_vals, rtol=1e-8)
    return u


@pytest.mark.parametrize("precision", [spnet.PREC_FP64, spnet.PREC_MIXED])
def test_request_matches_direct_calls(precision):
    p = nw.config1()
    ref = _direct(p, precision)
    sv = spnet.Server(max_inflight=2)
    x, res = sv.wait(sv.submit(p, precision=precision))
    sv.close()
    assert res["status"] == 0, res["message"]
    assert res["relres"] <= 1e-8
    assert np.array_equal(x[0], ref)
    assert 0.0 <= res["queue_ms"] <= res["latency_ms"]
    assert res["device_end_ms"] > res["device_start_ms"] >= 0.0


def test_result_is_the_same_alone_and_in_the_mix():
    a = _small3d()
    sv = spnet.Server(max_inflight=1)
    xa, ra = sv.wait(sv.submit(a))
    sv.close()
    assert ra["status"] == 0, ra["message"]
    mix = [nw.config1(), _small3d(seed=7, n=2500), a, _truss(), _small3d(seed=5, n=2000), a]
    sv = spnet.Server(max_inflight=4)
    tickets = [sv.submit(p) for p in mix]
    out = [sv.wait(t) for t in tickets]
    sv.close()
    for (x, res), p in zip(out, mix):
        assert res["status"] == 0, (p.name, res["message"])
        assert res["relres"] <= 1e-8, p.name
    assert np.array_equal(out[2][0], xa)
    assert np.array_equal(out[5][0], xa)
    # the work overlapped: some request started on the device before another ended
    spans = sorted((r["device_start_ms"], r["device_end_ms"]) for _, r in out)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_several_right_hand_sides_in_one_request():
    p = _small3d()
    rng = np.random.default_rng(5)
    F = rng.uniform(0.0, 1.0, size=(3, p.n_dof))
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED)
    ref, _ = spnet.pcg_solve(op, pc, F, np.broadcast_to(p.dirichlet_vals, (3, len(p.dirichlet_vals))), rtol=1e-8)
    sv = spnet.Server(max_inflight=2)
    x, res = sv.wait(sv.submit(p, f=F))
    sv.close()
    assert res["status"] == 0, res["message"]
    assert np.array_equal(x, ref)


def test_batched_right_hand_sides_alone_and_in_the_mix():
    # a request whose right-hand sides are stepped together (batch_rhs) runs the
    # batched kernels; its result is that of the direct calls, alone and in the mix
    p = _small3d()
    rng = np.random.default_rng(6)
    F = rng.uniform(0.0, 1.0, size=(6, p.n_dof))
    G = np.broadcast_to(p.dirichlet_vals, (6, len(p.dirichlet_vals)))
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED, batch_rhs=6)
    ref, st = spnet.pcg_solve(op, pc, F, G, rtol=1e-8)
    assert all(s.converged for s in st)
    sv = spnet.Server(max_inflight=3)
    tickets = [sv.submit(_small3d(seed=7, n=2500)), sv.submit(p, f=F, batch_rhs=6), sv.submit(_truss()),
               sv.submit(p, f=F, batch_rhs=6)]
    out = [sv.wait(t) for t in tickets]
    sv.close()
    for x, res in out:
        assert res["status"] == 0, res["message"]
    np.testing.assert_array_equal(out[1][0], ref)
    np.testing.assert_array_equal(out[3][0], ref)


def test_a_failing_request_does_not_disturb_the_others():
    good = _small3d()
    bad = _small3d(seed=3)
    bad.H = 0.3  # does not divide the unit cube
    sv = spnet.Server(max_inflight=2)
    t1, t2, t3 = sv.submit(good), sv.submit(bad), sv.submit(good)
    (x1, r1), (_, r2), (x3, r3) = sv.wait(t1), sv.wait(t2), sv.wait(t3)
    sv.close()
    assert r1["status"] == 0 and r3["status"] == 0
    assert r2["status"] == spnet.ERR_BAD_H
    assert np.array_equal(x1, x3)
