"""Preconditioned conjugate gradients (oracle; test infrastructure).

Section 4.2 applies the conjugate gradient method to (B K u, v) = (B f, v)
with P = B K symmetric in the K inner product (eq. TTsym); the paper does not
print the iteration, so this is the textbook Hestenes-Stiefel PCG:

    r = b - A x,  z = B r,  p = z,  rho = (r, z)
    repeat:  q = A p,  alpha = rho / (p, q),  x += alpha p,  r -= alpha q
             stop if |r|_2 <= rtol |b|_2
             z = B r,  beta = (r, z) / rho   [flexible: (r, z - z_old) / rho]
             rho = (r, z),  p = z + beta p

After the recursive residual meets the tolerance the true residual b - A x is
recomputed; if it does not, the iteration restarts from it (at most twice).
The flexible (Polak-Ribiere) beta is the standard choice when B is applied
inexactly and is no longer exactly symmetric.

Convergence rates (Section 6.2, eq. conv_rate): with e_l = u - u^(l),
tau_l = |e_l|_K / |e_{l-1}|_K for l >= 2 (the printed ratio is the reciprocal
of this; the tables report values below one).
"""
from __future__ import annotations

import numpy as np


class PCGResult:
    def __init__(self, x, iters, relres_hist, true_relres, converged, restarts, alphas=(),
                 betas=()):
        self.alphas = list(alphas)
        self.betas = list(betas)
        self.x = x
        self.iters = iters
        self.relres_hist = relres_hist
        self.true_relres = true_relres
        self.converged = converged
        self.restarts = restarts


def pcg(A, b, apply_B, rtol=1e-8, maxit=1000, x0=None, flexible=False, max_restarts=2,
        callback=None):
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return PCGResult(np.zeros(n), 0, [0.0], 0.0, True, 0)
    tol = rtol * bnorm
    r = b - A @ x
    hist = [float(np.linalg.norm(r)) / bnorm]
    it = 0
    restarts = 0
    alphas, betas = [], []
    if callback is not None:
        callback(x, it)
    while True:
        if np.linalg.norm(r) > tol and it < maxit:
            z = apply_B(r)
            rho = float(r @ z)
            p = z.copy()
            while it < maxit:
                q = A @ p
                alpha = rho / float(p @ q)
                alphas.append(alpha)
                x = x + alpha * p
                r = r - alpha * q
                it += 1
                rn = float(np.linalg.norm(r))
                hist.append(rn / bnorm)
                if callback is not None:
                    callback(x, it)
                if rn <= tol:
                    break
                z_old = z
                z = apply_B(r)
                rz = float(r @ z)
                if flexible:
                    beta = (rz - float(r @ z_old)) / rho
                else:
                    beta = rz / rho
                betas.append(beta)
                rho = rz
                p = z + beta * p
        rtrue = b - A @ x
        true_rel = float(np.linalg.norm(rtrue)) / bnorm
        if true_rel <= rtol or restarts >= max_restarts or it >= maxit:
            return PCGResult(x, it, hist, true_rel, true_rel <= rtol, restarts, alphas, betas)
        r = rtrue
        restarts += 1


def k_norm(A, e):
    return float(np.sqrt(max(e @ (A @ e), 0.0)))


def convergence_rates(A, u_exact, iterates):
    """tau_l = |u - u^(l)|_K / |u - u^(l-1)|_K for l >= 2; returns (taus, errors)."""
    errs = np.array([k_norm(A, u_exact - x) for x in iterates])
    taus = errs[2:] / errs[1:-1]
    return taus, errs


def lanczos_extremes(alphas, betas):
    """Extreme Ritz values of the PCG-generated Lanczos tridiagonal matrix.

    From the CG coefficients alpha_l (step lengths) and beta_l the Lanczos
    matrix T has diagonal 1/alpha_l + beta_{l-1}/alpha_{l-1} and off-diagonal
    sqrt(beta_l)/alpha_l; its eigenvalues approximate the spectrum of B A.
    """
    m = len(alphas)
    T = np.zeros((m, m))
    for l in range(m):
        T[l, l] = 1.0 / alphas[l] + (betas[l - 1] / alphas[l - 1] if l > 0 else 0.0)
        if l + 1 < m:
            T[l, l + 1] = T[l + 1, l] = np.sqrt(betas[l]) / alphas[l]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])
