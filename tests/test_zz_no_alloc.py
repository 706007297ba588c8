"""The allocation-free restriction entry point against the ordinary one.

spnet_pc_restrict_static serves callers that cannot allocate device memory
during the call: hosts whose device memory is all reserved up front by
another allocator, and loops that must not enter cudaMalloc.  It must give
the same r_c = R_0 r as spnet_pc_restrict and as the oracle's R_0 r, on two
calls in a row (the shared static scratch keeps the previous call's
contents, which must not leak into the next result), for 2D and 3D meshes
and for 1 and 3 dofs per node.  Collected last so that a failure here leaves
every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import operator as oop  # noqa: E402
from oracle.coarse import CoarseSpace  # noqa: E402
from paper_2207_07488_gb300 import networks as nw  # noqa: E402
from paper_2207_07488_gb300 import spnet  # noqa: E402


def _problem(case):
    if case == "2d":
        return nw.config1()
    if case == "3d":
        net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=31)
        return nw.scalar_band_problem(net, 0.25)
    net = nw.fiber_network_3d(1200, 0.25, 0.02, seed=41, keep="clamped_x")
    return nw.truss_band_problem(net, 0.25)


@pytest.mark.parametrize("case", ["2d", "3d", "3d_3dof"])
def test_static_restrict_matches_restrict_twice(case):
    p = _problem(case)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED)
    free, A, _ = oop.split(p)
    R0 = CoarseSpace(p, free, A.tocsr()).R0
    rng = np.random.default_rng(11 + len(case))
    n, m0 = op.info.n_free, pc.info.m0
    assert n == free.size and m0 == R0.shape[0]
    rc_out = torch.full((m0,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        r = rng.standard_normal(n) * (1 + call)
        ref = pc.restrict(r)
        got = pc.restrict_static(torch.from_numpy(r).cuda(), rc_out).cpu().numpy()
        # every entry within 1e-13 of the sum of magnitudes it adds up: against the
        # ordinary entry point and against the oracle's R_0 r
        bound = 1e-13 * (abs(R0) @ np.abs(r)) + 1e-300
        assert np.all(np.abs(got - ref) <= bound)
        assert np.all(np.abs(got - R0 @ r) <= bound)


def _grid_patch(k=300, h_div=10, lo=0.45):
    """A square grid patch inside the unit square, on a mesh of k x k elements."""
    n = k // 10 * h_div          # nodes per side: the patch spans k/10 elements
    h = 1.0 / (k * h_div)
    ids = np.arange(n * n)
    ix, iy = ids % n, ids // n
    X = np.stack([lo + ix * h, lo + iy * h], axis=1)
    right = ids[ix < n - 1]
    up = ids[iy < n - 1]
    E = np.concatenate([np.stack([right, right + 1], 1), np.stack([up, up + n], 1)]).astype(np.int64)
    m = E.shape[0]
    net = nw.Network(2, X, E, np.zeros(m, np.int8), np.full(m, 1.0 / h), np.full(m, 1.0 / h),
                     np.zeros((m, 2)), (1.0, 1.0))
    dd = ids[ix == 0].astype(np.int64)
    return nw.Problem(net, 1, "scalar", dd, np.zeros(dd.size), np.ones(n * n), 1.0 / k, (0,))


def test_static_restrict_rejects_oversized_mesh():
    p = _grid_patch()   # 300 x 300 elements x 4 corners = 360000 corner sums > 2^18
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED)
    assert pc.info.n_elem * 4 > 2 ** 18
    r = torch.zeros(op.info.n_free, dtype=torch.float64, device="cuda")
    rc = torch.zeros(max(pc.info.m0, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(spnet.SpnetError) as ei:
        pc.restrict_static(r, rc)
    assert ei.value.code == -7 and "static scratch" in str(ei.value)
    # the ordinary entry point still serves this mesh
    rr = np.random.default_rng(5).standard_normal(op.info.n_free)
    assert np.all(np.isfinite(pc.restrict(rr)))


def test_static_restrict_rejects_bad_tensors():
    # checked in the binding before the library is called (no launch)
    p = _problem("2d")
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED)
    n, m0 = op.info.n_free, pc.info.m0
    r = torch.zeros(n, dtype=torch.float64, device="cuda")
    rc = torch.zeros(m0, dtype=torch.float64, device="cuda")
    bad = [(r.float(), rc), (r, rc.float()), (r[:-1], rc), (r, rc[:-1]), (r.cpu(), rc),
           (torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2], rc)]
    for a, b in bad:
        with pytest.raises(ValueError):
            pc.restrict_static(a, b)
