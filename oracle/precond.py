"""The two block preconditioners, applied exactly as Alg. 2 and Alg. 4, and
the incomplete t-u-p form M2* = D2^-1 L2^-1 (Sec. 3.2, the remark after
Prop. 3.2: the factor U2^-1 of Eq. P2 is dropped).

Inner solves are pluggable:
* ``u_solver``: "amg" (one AMG V-cycle on S~ or S1, the paper's AMG(K, y)) or
  "exact" (sparse LU of S~ or S1, the paper's nested direct solver,
  Sec. 4.1).
* ``p_solver``: "amg" (one scalar AMG V-cycle on T or S~2) or "exact"
  (sparse LU of T or S~2; the paper applies these inverses exactly).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import schur
from . import sparse as osp
from .amg import AMG, AmgOptions


class _Exact:
    def __init__(self, M: sp.csr_matrix):
        self.lu = spla.splu(M.tocsc()) if M.shape[0] else None

    def __call__(self, f):
        return self.lu.solve(f) if self.lu is not None else np.zeros_like(f)


def _solver(M, B, kind, opt, aggregates=None, near_null=None):
    if kind == "amg":
        return AMG(M, B, opt, aggregates=aggregates, near_null=near_null)
    if kind == "exact":
        return _Exact(M)
    raise ValueError(kind)


class BlockPreconditioner:
    """M1^-1 (variant "tpu", Alg. 1-2), M2^-1 (variant "tup", Alg. 3-4) or
    the incomplete M2*^-1 = D2^-1 L2^-1 (variant "tup_star", built by Alg. 3
    like M2)."""

    def __init__(self, P, variant: str, u_solver: str = "amg", p_solver: str = "amg",
                 opt: AmgOptions | None = None, blk: dict | None = None,
                 opt_p: AmgOptions | None = None, u_matrix=None, p_matrix=None,
                 u_aggregates=None, p_aggregates=None, u_near_null=None):
        """``u_matrix`` / ``p_matrix`` replace the matrix the inner u / p
        solver is built on (S~ or S1, T or S~2); used to form the exact block
        factorisation of Eq. P1 / Eq. P2 on tiny cases.  ``u_aggregates`` /
        ``p_aggregates`` rebuild the AMG hierarchies on the aggregates of an
        earlier setup (``AMG.aggregates()``): the numeric refresh for new
        values of the same patterns.  ``u_near_null``: candidate vectors for
        the elasticity AMG (e.g. the six rigid modes of ``amg.rigid_modes``)
        instead of the three translations."""
        self.P = P
        self.variant = variant
        b = blk or osp.blocks(P)
        self.b = b
        self.nu, self.nt, self.np_ = 3 * P.n_node, 3 * P.n_face, P.n_face
        self.Hinv = schur.htilde_inv(P, b["H"])                      # H~^-1 (Alg. 1, Alg. 3)
        opt = opt or AmgOptions()
        opt_p = opt_p or opt
        if variant == "tpu":
            self.S1 = schur.s1(P, b)
            self.Su = schur.s_tilde(P, b, self.S1)                    # S~ (Alg. 1)
            self.u_inv = _solver(self.Su if u_matrix is None else u_matrix, 3, u_solver, opt, u_aggregates,
                                 u_near_null)
            self.p_inv = _solver(b["T"] if p_matrix is None else p_matrix, 1, p_solver, opt_p, p_aggregates)
        elif variant in ("tup", "tup_star"):
            self.S1 = schur.s1(P, b)                                  # S1 (Alg. 3)
            self.Su = self.S1
            self.S2 = schur.s2_tilde(P, self.S1, b)                   # S~2 = T - FS (Alg. 3)
            self.u_inv = _solver(self.S1 if u_matrix is None else u_matrix, 3, u_solver, opt, u_aggregates,
                                 u_near_null)
            self.p_inv = _solver(self.S2 if p_matrix is None else p_matrix, 1, p_solver, opt_p, p_aggregates)
        else:
            raise ValueError(variant)

    def split(self, w):
        return w[:self.nu], w[self.nu:self.nu + self.nt], w[self.nu + self.nt:]

    # The applications are written factor by factor from the block LDU forms
    # (Eq. P1 in the order (t, p, u), Eq. P2 in the order (t, u, p)); Alg. 2
    # and Alg. 4 are the same products with every inner inverse applied once.

    def apply_tpu(self, w):
        """M1^-1 w = U1^-1 D1^-1 L1^-1 w (Eq. P1), the operator of Alg. 2."""
        b = self.b
        w_u, w_t, w_p = self.split(w)
        hw = self.Hinv @ w_t                                  # H~^-1 w_t
        tw = self.p_inv(w_p)                                  # T^-1 w_p
        # L1^-1 then D1^-1: t -> -H~^-1 w_t, p -> T^-1 w_p,
        # u -> S~^-1 (w_u + C1 H~^-1 w_t - Q1 T^-1 w_p)
        z_u = self.u_inv(w_u + b["C1"] @ hw - b["Q1"] @ tw)
        # U1^-1: p -= T^-1 Q2 u, t += H~^-1 C2 u
        v_p = tw - self.p_inv(b["Q2"] @ z_u)
        v_t = -hw + self.Hinv @ (b["C2"] @ z_u)
        return np.concatenate([z_u, v_t, v_p])

    def _tup_lower_diag(self, w):
        """D2^-1 L2^-1 w (Eq. LDU2): t -> -H~^-1 w_t, u -> S~1^-1 y_u with
        y_u = w_u + C1 H~^-1 w_t, p -> S~2^-1 (w_p - Q2 S~1^-1 y_u); the
        S~1^-1 y_u of both factors is one AMG application."""
        b = self.b
        w_u, w_t, w_p = self.split(w)
        hw = self.Hinv @ w_t
        z_u = self.u_inv(w_u + b["C1"] @ hw)
        z_p = self.p_inv(w_p - b["Q2"] @ z_u)
        return z_u, -hw, z_p

    def apply_tup(self, w):
        """M2^-1 w = U2^-1 (D2^-1 L2^-1 w) (Eq. P2), the operator of Alg. 4:
        U2^-1 takes u -= S~1^-1 Q1 p, then t += H~^-1 C2 u."""
        b = self.b
        z_u, z_t, z_p = self._tup_lower_diag(w)
        v_u = z_u - self.u_inv(b["Q1"] @ z_p)
        v_t = z_t + self.Hinv @ (b["C2"] @ v_u)
        return np.concatenate([v_u, v_t, z_p])

    def apply_tup_star(self, w):
        """M2*^-1 w = D2^-1 L2^-1 w: Eq. P2 without its first factor (the
        incomplete form of the remark after Prop. 3.2)."""
        z_u, z_t, z_p = self._tup_lower_diag(w)
        return np.concatenate([z_u, z_t, z_p])

    def __call__(self, w):
        w = np.asarray(w, dtype=np.float64)
        if self.variant == "tpu":
            return self.apply_tpu(w)
        if self.variant == "tup":
            return self.apply_tup(w)
        return self.apply_tup_star(w)
