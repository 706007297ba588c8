"""End-to-end oracle solve of a problem (test infrastructure)."""
from __future__ import annotations

import numpy as np

from . import operator as op
from .pcg import pcg
from .schwarz import SchwarzPreconditioner


class OracleSolver:
    """Assembly, splitting, preconditioner set-up and PCG for one problem."""

    def __init__(self, problem, local="dense", star_set=None):
        self.problem = problem
        self.K = op.assemble(problem)
        self.free, self.A, self.KID = op.split(problem, self.K)
        self.B = SchwarzPreconditioner(problem, self.free, self.A, local=local, star_set=star_set)

    def rhs(self, f=None, g=None):
        p = self.problem
        f = p.f if f is None else f
        g = p.dirichlet_vals if g is None else g
        return op.lifted_rhs(p, f, g, self.free, self.KID)

    def solve(self, f=None, g=None, rtol=1e-8, maxit=1000, flexible=False, callback=None):
        p = self.problem
        g = p.dirichlet_vals if g is None else g
        b = self.rhs(f, g)
        res = pcg(self.A, b, self.B.apply, rtol=rtol, maxit=maxit, flexible=flexible,
                  callback=callback)
        res.u = op.expand(p, self.free, res.x, g)
        res.b = b
        return res


def solve(problem, rtol=1e-8, **kw):
    return OracleSolver(problem).solve(rtol=rtol, **kw)
