"""The convergence-rate experiments of Section 6.2, run through the library.

PCG's error in the K-norm after each step, |u - u^(l)|_K, and the rates
tau_l = |u - u^(l)|_K / |u - u^(l-1)|_K for l >= 2 (eq. conv_rate, read with the
ratio the right way up: the tables report values below one), averaged until the
error has fallen by a given factor (Table lap_conv reports the mean and the
largest rate).

One solve gives both: FP64 factors and coarse inverse, textbook (non-flexible)
PCG without restarts, run to a relative residual of 1e-13, is the reference
solution u, and the library records every iterate u^(l) of that same run
(spnet_pc_record_iterates) on the device.  The K-norms use the library's product
with A = K_II.
"""
from __future__ import annotations

import numpy as np

from . import spnet


def pcg_rates(problem, reduction: float = 1e-8, max_steps: int = 300):
    """K-norm errors and rates of PCG on `problem` (a networks.Problem).

    Returns a dict: errors |e_l|_K for l = 0..L (L the first step at which the
    error is at most `reduction` times the initial one), rates tau_l for
    l = 2..L, their mean and maximum, L, and the sizes of the problem.
    """
    op = spnet.Operator.from_problem(problem)
    pc = spnet.Preconditioner(op, problem.H, problem.gamma_faces, precision=spnet.PREC_FP64,
                              star_set=spnet.STARS_ALL if problem.star_set == "all" else spnet.STARS_INTERIOR,
                              patch=problem.patch, flexible=0, max_restarts=0,
                              coarse=getattr(problem, "coarse", "q1"))
    import torch
    free = np.setdiff1d(np.arange(problem.n_dof), problem.dirichlet_dofs)
    hist = torch.empty((max_steps + 1, int(op.info.n_free)), dtype=torch.float64,
                       device=torch.device("cuda", torch.cuda.current_device()))
    pc.record_iterates(hist)
    u, st = spnet.pcg_solve(op, pc, problem.f, problem.dirichlet_vals, rtol=1e-13, maxit=20 * max_steps,
                            raise_on_noconv=False)
    pc.record_iterates(None)
    torch.cuda.synchronize()
    kept = min(max_steps, int(st[0].iterations)) + 1
    uf = u[free]

    def knorm(xf):
        e = uf - xf
        return float(np.sqrt(max(float(e @ op.spmv(e)), 0.0)))

    errs = [knorm(hist[0].cpu().numpy())]
    steps = 0
    for l in range(1, kept):
        errs.append(knorm(hist[l].cpu().numpy()))
        steps = l
        if errs[-1] <= reduction * errs[0]:
            break
    del hist
    errs = np.array(errs)
    taus = errs[2:] / errs[1:-1]
    info = pc.info
    out = {"errors": errs, "taus": taus, "mean": float(taus.mean()) if taus.size else float("nan"),
           "max": float(taus.max()) if taus.size else float("nan"), "steps": steps,
           "n_free": int(op.info.n_free), "stars": int(info.n_stars), "m0": int(info.m0),
           "exact_relres": float(st[0].relres), "max_star": int(info.max_star),
           "max_dense_block": int(pc.export(spnet.EXPORT_STAR_CORE).max()) if info.n_stars else 0,
           "solve_ms": float(st[0].solve_ms), "reference_steps": int(st[0].iterations),
           "setup_ms": float(info.setup_ms)}
    pc.close()
    op.close()
    return out
