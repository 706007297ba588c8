"""Serving (spnet_server_*): requests against the direct calls, alone and in the mix.

A request runs the same kernels as the direct calls (assembly, operator,
preconditioner, PCG), and every kernel reduces in a fixed order, so a
request's solution must be bitwise the same whether it runs alone or among
other requests of different sizes and models, and the same as the direct
calls on the same problem.  Admission: a budget that holds one request makes
the others queue; a request beyond the budget is refused; non-finite data is
bad input; a queued request can be cancelled and a finished one polled.
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
    net = nw.fiber_network_3d(n, 0.2, 0.01, seed=seed)
    return nw.scalar_band_problem(net, 0.25, name=f"small3d-{seed}")


def _truss():
    net = nw.fiber_network_3d(1200, 0.25, 0.02, seed=41, keep="clamped_x")
    return nw.truss_band_problem(net, 0.25, name="truss")


def _direct(p, precision):
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=precision,
                              star_set=spnet.STARS_ALL if p.star_set == "all" else spnet.STARS_INTERIOR,
                              patch=p.patch)
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
    # seed 3 draws linearly dependent coarse functions (a singular A_0 handled by dropping them)
    mix = [nw.config1(), _small3d(seed=7, n=2500), a, _truss(), _small3d(seed=3), _small3d(seed=5, n=2000), a]
    sv = spnet.Server(max_inflight=4)
    tickets = [sv.submit(p) for p in mix]
    out = [sv.wait(t) for t in tickets]
    sv.close()
    for (x, res), p in zip(out, mix):
        assert res["status"] == 0, (p.name, res["message"])
        assert res["relres"] <= 1e-8, p.name
    assert np.array_equal(out[2][0], xa)
    assert np.array_equal(out[6][0], xa)
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


def _server_with_budget(multiple, p):
    """A server whose budget is about `multiple` times the estimate of request p."""
    est = spnet.request_estimate(p)
    free, _ = torch.cuda.mem_get_info()
    reserve = int(free - multiple * est)
    sv = spnet.Server(max_inflight=3, reserve_bytes=reserve)
    return sv, est


def test_a_small_budget_makes_requests_queue():
    # a budget of 1.5 estimates holds one request at a time: three requests submitted
    # together run one after the other, and the later ones wait in the queue
    p = _small3d()
    sv, est = _server_with_budget(1.5, p)
    try:
        b = sv.budget()
        assert est <= b < 2 * est, (est, b)
        tickets = [sv.submit(p) for _ in range(3)]
        out = [sv.wait(t) for t in tickets]
    finally:
        sv.close()
    for x, res in out:
        assert res["status"] == 0, res["message"]
        np.testing.assert_array_equal(x, out[0][0])
    spans = sorted((r["device_start_ms"], r["device_end_ms"]) for _, r in out)
    assert all(spans[i + 1][0] >= spans[i][1] for i in range(2)), spans
    assert max(r["queue_ms"] for _, r in out) > 0.0


def test_a_request_beyond_the_budget_is_refused():
    p = _small3d()
    sv, est = _server_with_budget(0.5, p)
    try:
        assert sv.budget() < est
        with pytest.raises(spnet.SpnetError) as ei:
            sv.submit(p)
        assert ei.value.code == spnet.ERR_NO_MEMORY
    finally:
        sv.close()


def test_non_finite_input_is_bad_input():
    p = nw.config1()
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED)
    free = np.setdiff1d(np.arange(p.n_dof), p.dirichlet_dofs)
    f = p.f.copy()
    f[free[17]] = np.nan
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.pcg_solve(op, pc, f, p.dirichlet_vals)
    assert ei.value.code == spnet.ERR_BAD_INPUT and "non-finite" in str(ei.value)
    g = p.dirichlet_vals.copy()
    g[3] = np.inf
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.pcg_solve(op, pc, p.f, g)
    assert ei.value.code == spnet.ERR_BAD_INPUT
    # a NaN at a Dirichlet dof of f is ignored, as documented
    f2 = p.f.copy()
    f2[p.dirichlet_dofs[0]] = np.nan
    u, st = spnet.pcg_solve(op, pc, f2, p.dirichlet_vals)
    assert st[0].converged
    # the batched path checks every column
    pcb = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED, batch_rhs=4)
    F = np.tile(p.f, (4, 1))
    F[2, free[5]] = np.nan
    with pytest.raises(spnet.SpnetError) as ei:
        spnet.pcg_solve(op, pcb, F, np.tile(p.dirichlet_vals, (4, 1)))
    assert ei.value.code == spnet.ERR_BAD_INPUT
    # through the server: the request fails with BAD_INPUT, the next one runs
    sv = spnet.Server(max_inflight=1)
    try:
        t1, t2 = sv.submit(p, f=f), sv.submit(p)
        (_, r1), (_, r2) = sv.wait(t1), sv.wait(t2)
    finally:
        sv.close()
    assert r1["status"] == spnet.ERR_BAD_INPUT and "non-finite" in r1["message"]
    assert r2["status"] == 0


def test_poll_and_cancel():
    big = _small3d(seed=7, n=2500)
    small = _small3d()
    sv = spnet.Server(max_inflight=1)
    try:
        t1 = sv.submit(big)
        t2 = sv.submit(small)
        t3 = sv.submit(small)
        assert sv.cancel(t3)              # still queued behind t1 and t2
        import time
        deadline = time.time() + 120
        got = None
        while got is None and time.time() < deadline:
            got = sv.poll(t1)
            if got is None:
                time.sleep(0.002)
        assert got is not None and got[1]["status"] == 0
        x2, r2 = sv.wait(t2)
        assert r2["status"] == 0
        _, r3 = sv.wait(t3)
        assert r3["status"] == spnet.ERR_CANCELLED
        with pytest.raises(spnet.SpnetError):
            sv.cancel(t3)                 # retired tickets are unknown
        t4 = sv.submit(small)
        x4, r4 = sv.wait(t4)
    finally:
        sv.close()
    np.testing.assert_array_equal(x2, x4)
