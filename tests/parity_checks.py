"""Element-wise comparisons of the library's preconditioner steps with the oracle's
(shared by the GPU parity tests)."""
import numpy as np


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def star_scale(o, r):
    """Per free dof, the largest |A_j^{-1} r_j|_inf over the stars j that hold it
    (the oracle's own local solves): the size of what each star adds there."""
    sc = np.zeros(o.A.shape[0])
    for j, S in enumerate(o.B.stars):
        w = o.B.local_solve(j, r[S])
        np.maximum.at(sc, S, np.abs(w).max(initial=0.0))
    return sc


def check_star_term(o, r, got, prec, sc=None):
    """Element-wise comparison of a star term with the oracle's.

    FP64 (the same window kernels as FP32, on FP64 coefficients): every entry within
    1e-9 of the scale of the stars that hold it, so one wrong star anywhere fails by
    orders of magnitude.  Mixed (FP32 factors, condition numbers of the stars up to
    ~5e5): the relative error over every star's dofs within 1e-2, and over all
    dofs within 2e-4."""
    ref = o.B.star_term(r)
    d = np.abs(got - ref)
    if prec == "fp64":
        sc = star_scale(o, r) if sc is None else sc
        bad = np.nonzero(d > 1e-9 * sc)[0]
        assert bad.size == 0, (bad[:10], d[bad[:10]], sc[bad[:10]])
    else:
        worst = max(np.linalg.norm(d[S]) / np.linalg.norm(ref[S]) for S in o.B.stars)
        assert worst <= 1e-2, worst
        assert rel(got, ref) <= 2e-4
    return ref


def check_entries(got, ref, bound, what):
    d = np.abs(np.asarray(got) - np.asarray(ref))
    bad = np.nonzero(d > bound)[0]
    assert bad.size == 0, (what, bad[:10], d[bad[:10]], np.asarray(bound)[bad[:10]])
