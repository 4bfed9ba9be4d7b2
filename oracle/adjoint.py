"""Adjoint solve: J^T lambda = g with the transposed preconditioners.

The preconditioners are the inexact block factorisations of Eq. P1 / Eq. P2,
M^-1 = U^-1 D^-1 L^-1 (in the permuted orders of Eq. Q1 / Eq. Q2); their
transposes M^-T = L^-T D^-T U^-T applied to w read, written out:

app_tpu^T (from Eq. P1):
  t_p = T^-T w_p
  t_u = w_u + C2^T (H~^-T w_t) - Q2^T t_p
  v_u = AMG^T(S~, t_u)
  v_p = t_p - T^-T (Q1^T v_u)
  v_t = H~^-T (C1^T v_u - w_t)

app_tup^T (from Eq. P2):
  t_u = w_u + C2^T (H~^-T w_t)
  s_u = AMG^T(S1, t_u)
  t_p = w_p - Q1^T s_u
  v_p = S~2^-T t_p
  v_u = s_u - AMG^T(S1, Q2^T v_p)
  v_t = H~^-T (C1^T v_u - w_t)

app_tup_star^T = (D2^-1 L2^-1)^T = L2^-T D2^-T (from Eq. LDU2):
  z_t = -H~^-T w_t,  z_u = AMG^T(S1, w_u),  z_p = S~2^-T w_p
  v_p = z_p
  v_u = z_u - AMG^T(S1, Q2^T z_p)
  v_t = z_t + H~^-T (C1^T v_u)

AMG^T is the transposed V-cycle (oracle.amg.AMG.vcycle_t); T and S~2 are
symmetric and their scalar V-cycles are symmetric operators.  The solve is
the same flexible GMRES on J^T.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import sparse as osp
from .fgmres import fgmres
from .precond import BlockPreconditioner


def _inv_t(solver):
    """Transpose of an inner solver: the transposed V-cycle for AMG, the
    transposed sparse LU solve for the exact inner solver."""
    if hasattr(solver, "vcycle_t"):
        return solver.vcycle_t
    lu = solver.lu
    return (lambda f: lu.solve(f, trans="T")) if lu is not None else (lambda f: np.zeros_like(f))


class AdjointPreconditioner:
    def __init__(self, M: BlockPreconditioner):
        self.M = M
        b = M.b
        self.C1T = b["C1"].T.tocsr()
        self.C2T = b["C2"].T.tocsr()
        self.Q1T = b["Q1"].T.tocsr()
        self.Q2T = b["Q2"].T.tocsr()
        self.HinvT = M.Hinv.T.tocsr()
        self.u_t = _inv_t(M.u_inv)
        self.p_t = _inv_t(M.p_inv)

    def __call__(self, w):
        M = self.M
        w = np.asarray(w, dtype=np.float64)
        w_u, w_t, w_p = M.split(w)
        if M.variant == "tpu":
            t_p = self.p_t(w_p)
            t_u = w_u + self.C2T @ (self.HinvT @ w_t) - self.Q2T @ t_p
            v_u = self.u_t(t_u)
            v_p = t_p - self.p_t(self.Q1T @ v_u)
            v_t = self.HinvT @ (self.C1T @ v_u - w_t)
        elif M.variant == "tup_star":
            z_t = -(self.HinvT @ w_t)
            z_u = self.u_t(w_u)
            z_p = self.p_t(w_p)
            v_p = z_p
            v_u = z_u - self.u_t(self.Q2T @ z_p)
            v_t = z_t + self.HinvT @ (self.C1T @ v_u)
        else:
            t_u = w_u + self.C2T @ (self.HinvT @ w_t)
            s_u = self.u_t(t_u)
            t_p = w_p - self.Q1T @ s_u
            v_p = self.p_t(t_p)
            v_u = s_u - self.u_t(self.Q2T @ v_p)
            v_t = self.HinvT @ (self.C1T @ v_u - w_t)
        return np.concatenate([v_u, v_t, v_p])


def solve_adjoint(P, M: BlockPreconditioner, g, tol=1e-8, maxit=500):
    JT = osp.jacobian(P).T.tocsr()
    return fgmres(lambda v: JT @ v, AdjointPreconditioner(M), g, tol, maxit)


def dense_adjoint(P, g):
    J = osp.jacobian(P).toarray()
    return np.linalg.solve(J.T, g)


def operator_matrix(apply, n):
    """Dense matrix of a linear operator, column by column (tiny cases)."""
    cols = [apply(e) for e in np.eye(n)]
    return np.array(cols).T


def aperture_gradient(P, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dL/da_f = -lambda^T (dJ/da_f) x from the derivative entries of the
    transmissibility T and the coupling Q2 (rows are pressure equations)."""
    d = P.dk
    nu, nt = 3 * P.n_node, 3 * P.n_face
    lam_p = lam[nu + nt:]
    x_u, x_p = x[:nu], x[nu + nt:]
    t = d["block"] == 0
    xv = np.empty(len(d["val"]))
    xv[t] = x_p[d["col"][t]]
    xv[~t] = x_u[3 * d["col"][~t] + d["comp"][~t]]
    contrib = lam_p[d["row"]] * d["val"] * xv
    return -np.bincount(d["face"], weights=contrib, minlength=P.n_face)
