"""Right-preconditioned flexible GMRES with CGS2 (Sec. 4).

The paper solves every Jacobian system with right-preconditioned full GMRES
(no restart), zero initial guess, stopped when the residual norm has dropped
by the factor tol.  With a fixed linear preconditioner the flexible form (the
preconditioned directions z_j are stored and x = Z y) produces the same
iterates as right-preconditioned GMRES.

Per iteration j (0-based):
    z_j = M^-1 v_j;  w = J z_j;  w0 = ||w||
    classical Gram-Schmidt twice: h = V^T w; w -= V h; h' = V^T w; w -= V h';
    h += h';  h_{j+1,j} = ||w||
    previous Givens rotations applied to column j, a new rotation zeroes
    h_{j+1,j}; g_{j+1} = -s_j g_j, g_j = c_j g_j
    stop when |g_{j+1}| / beta <= tol, or when h_{j+1,j} <= 1e-14 w0
    (breakdown: the Krylov space is invariant)
Then y solves the triangular system R y = g and x = Z y.  The true residual
||b - J x|| / ||b|| is returned.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class Result:
    x: np.ndarray
    iters: int
    relres: float
    est: float
    history: list = field(default_factory=list)
    converged: bool = False


def fgmres(Jmv, M, b: np.ndarray, tol: float = 1e-8, maxit: int = 500) -> Result:
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return Result(np.zeros(n), 0, 0.0, 0.0, [], True)
    V = np.zeros((maxit + 1, n))
    Z = np.zeros((maxit, n))
    Hh = np.zeros((maxit + 1, maxit))
    cs = np.zeros(maxit)
    sn = np.zeros(maxit)
    g = np.zeros(maxit + 1)
    g[0] = beta
    V[0] = b / beta
    hist = [1.0]
    k = 0
    est = 1.0
    for j in range(maxit):
        Z[j] = M(V[j])
        w = Jmv(Z[j])
        w0 = float(np.linalg.norm(w))
        Vj = V[:j + 1]
        h = Vj @ w
        w = w - Vj.T @ h
        h2 = Vj @ w
        w = w - Vj.T @ h2
        h = h + h2
        hn = float(np.linalg.norm(w))
        col = np.zeros(j + 2)
        col[:j + 1] = h
        col[j + 1] = hn
        for i in range(j):
            t = cs[i] * col[i] + sn[i] * col[i + 1]
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
            col[i] = t
        r = float(np.hypot(col[j], col[j + 1]))
        cs[j] = col[j] / r
        sn[j] = col[j + 1] / r
        col[j] = r
        col[j + 1] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        Hh[:j + 2, j] = col
        k = j + 1
        est = abs(g[j + 1]) / beta
        hist.append(est)
        breakdown = hn <= 1e-14 * w0
        if not breakdown:
            V[j + 1] = w / hn
        if est <= tol or breakdown:
            break
    y = sla.solve_triangular(Hh[:k, :k], g[:k], lower=False)
    x = Z[:k].T @ y
    relres = float(np.linalg.norm(b - Jmv(x)) / beta)
    return Result(x, k, relres, est, hist, relres <= tol or est <= tol)
