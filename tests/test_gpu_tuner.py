"""The tuner on the 40000-fibre workload: the three choices (star-solve mapping, SpMV lanes
per row, right-hand sides per warp of the batched star solve) are measured once per size
class, reused by the next set-up of the class, saved to a file and taken from it by a
cleared cache without measuring; solutions are bitwise the same with the reused choices."""
import numpy as np
import pytest

from paper_2207_07488_gb300 import networks as nw

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2207_07488_gb300 import spnet  # noqa: E402


def _setup(p, op):
    pc = spnet.Preconditioner(op, p.H, p.gamma_faces, precision=spnet.PREC_MIXED, batch_rhs=32)
    return pc, (pc.info.star_warps_per_block, pc.info.tuned)


def test_choices_are_measured_once_reused_and_persisted(tmp_path):
    p = nw.config2()
    op = spnet.Operator.from_problem(p)
    spnet.tune_cache_clear()
    pc1, c1 = _setup(p, op)
    measured, reused = spnet.tune_counts()
    assert measured == 3 and reused == 0
    lanes, jw = c1[1] % 256, c1[1] // 256
    assert 1 <= lanes <= 32 and jw in (2, 4) and 1 <= c1[0] <= 8
    u1, _ = spnet.pcg_solve(op, pc1, p.f, p.dirichlet_vals)
    pc1.close()
    pc2, c2 = _setup(p, op)
    assert c2 == c1 and spnet.tune_counts() == (3, 3)
    u2, _ = spnet.pcg_solve(op, pc2, p.f, p.dirichlet_vals)
    np.testing.assert_array_equal(u1, u2)
    pc2.close()
    path = str(tmp_path / "tune.tsv")
    spnet.tune_cache_save(path)
    spnet.tune_cache_clear()
    spnet.tune_cache_load(path)
    pc3, c3 = _setup(p, op)
    assert c3 == c1 and spnet.tune_counts() == (0, 3)
    u3, _ = spnet.pcg_solve(op, pc3, p.f, p.dirichlet_vals)
    np.testing.assert_array_equal(u1, u3)
