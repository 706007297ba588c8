"""The allocation-free restriction entry point against the ordinary one.

spnet_pc_restrict_static serves callers that cannot allocate device memory
during the call (for example code inside CUDA stream capture).  It must give
the same r_c = R_0 r as spnet_pc_restrict, on two calls in a row (the shared
static scratch keeps the previous call's contents, which must not leak into
the next result).  Collected last so that a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import networks as nw  # noqa: E402
from paper_2207_07488_gb300 import spnet  # noqa: E402


def _case(dim):
    if dim == 2:
        p = nw.config1()
    else:
        net = nw.fiber_network_3d(1500, 0.2, 0.01, seed=31)
        p = nw.scalar_band_problem(net, 0.25)
    op = spnet.Operator.from_problem(p)
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED)
    return op, pc


@pytest.mark.parametrize("dim", [2, 3])
def test_static_restrict_matches_restrict_twice(dim):
    op, pc = _case(dim)
    rng = np.random.default_rng(11 + dim)
    n, m0 = op.info.n_free, pc.info.m0
    rc_out = torch.full((m0,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        r = rng.standard_normal(n) * (1 + call)
        ref = pc.restrict(r)
        got = pc.restrict_static(torch.from_numpy(r).cuda(), rc_out).cpu().numpy()
        # the same arithmetic in the same order: equal to the ordinary entry point
        # within the tolerance of the restriction parity test
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


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
