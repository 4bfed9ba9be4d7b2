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


def _solver(M, B, kind, opt, aggregates=None):
    if kind == "amg":
        return AMG(M, B, opt, aggregates=aggregates)
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
                 u_aggregates=None, p_aggregates=None):
        """``u_matrix`` / ``p_matrix`` replace the matrix the inner u / p
        solver is built on (S~ or S1, T or S~2); used to form the exact block
        factorisation of Eq. P1 / Eq. P2 on tiny cases.  ``u_aggregates`` /
        ``p_aggregates`` rebuild the AMG hierarchies on the aggregates of an
        earlier setup (``AMG.aggregates()``): the numeric refresh for new
        values of the same patterns."""
        self.P = P
        self.variant = variant
        b = blk or osp.blocks(P)
        self.b = b
        self.nu, self.nt, self.np_ = 3 * P.n_node, 3 * P.n_face, P.n_face
        self.Hinv = schur.htilde_inv(P, b["H"])                      # Alg. 1/3 line 1
        opt = opt or AmgOptions()
        opt_p = opt_p or opt
        if variant == "tpu":
            self.S1 = schur.s1(P, b)
            self.Su = schur.s_tilde(P, b, self.S1)                    # Alg. 1 line 3
            self.u_inv = _solver(self.Su if u_matrix is None else u_matrix, 3, u_solver, opt, u_aggregates)
            self.p_inv = _solver(b["T"] if p_matrix is None else p_matrix, 1, p_solver, opt_p, p_aggregates)
        elif variant in ("tup", "tup_star"):
            self.S1 = schur.s1(P, b)                                  # Alg. 3 line 2
            self.Su = self.S1
            self.S2 = schur.s2_tilde(P, self.S1, b)                   # Alg. 3 line 3
            self.u_inv = _solver(self.S1 if u_matrix is None else u_matrix, 3, u_solver, opt, u_aggregates)
            self.p_inv = _solver(self.S2 if p_matrix is None else p_matrix, 1, p_solver, opt_p, p_aggregates)
        else:
            raise ValueError(variant)

    def split(self, w):
        return w[:self.nu], w[self.nu:self.nu + self.nt], w[self.nu + self.nt:]

    def apply_tpu(self, w):
        """Alg. 2, app_tpu."""
        b = self.b
        w_u, w_t, w_p = self.split(w)
        t_p = self.p_inv(w_p)                          # 1: t_p = T^-1 w_p
        t_t = self.Hinv @ w_t                          # 2: t_t = H~^-1 w_t
        t_u = w_u + b["C1"] @ t_t - b["Q1"] @ t_p      # 3
        v_u = self.u_inv(t_u)                          # 4: AMG(S~, t_u)
        s_p = b["Q2"] @ v_u                            # 5
        s_t = b["C2"] @ v_u                            # 6
        v_p = t_p - self.p_inv(s_p)                    # 7
        v_t = -t_t + self.Hinv @ s_t                   # 8
        return np.concatenate([v_u, v_t, v_p])

    def apply_tup(self, w):
        """Alg. 4, app_tup."""
        b = self.b
        w_u, w_t, w_p = self.split(w)
        t_t = self.Hinv @ w_t                          # 1
        t_u = w_u + b["C1"] @ t_t                      # 2
        s_u = self.u_inv(t_u)                          # 3: AMG(S1, t_u)
        t_p = w_p - b["Q2"] @ s_u                      # 4
        v_p = self.p_inv(t_p)                          # 5: S~2^-1 t_p
        t_u = b["Q1"] @ v_p                            # 6
        v_u = self.u_inv(t_u)                          # 7: AMG(S1, t_u)
        v_u = s_u - v_u                                # 8
        s_t = b["C2"] @ v_u                            # 9
        v_t = -t_t + self.Hinv @ s_t                   # 10
        return np.concatenate([v_u, v_t, v_p])

    def apply_tup_star(self, w):
        """M2*^-1 w = D2^-1 (L2^-1 w) with the factors of Eq. LDU2, in the
        (t, u, p) order of Eq. Q2:
          L2^-1: y_t = w_t, y_u = w_u + C1 H~^-1 w_t, y_p = w_p - Q2 S~1^-1 y_u
          D2^-1: v_t = -H~^-1 y_t, v_u = S~1^-1 y_u, v_p = S~2^-1 y_p
        S~1^-1 y_u appears in both factors; it is one AMG call."""
        b = self.b
        w_u, w_t, w_p = self.split(w)
        t_t = self.Hinv @ w_t                          # H~^-1 w_t
        y_u = w_u + b["C1"] @ t_t                      # L2^-1, u block
        s_u = self.u_inv(y_u)                          # S~1^-1 y_u = AMG(S1, y_u)
        y_p = w_p - b["Q2"] @ s_u                      # L2^-1, p block
        v_p = self.p_inv(y_p)                          # D2^-1, p block
        v_u = s_u                                      # D2^-1, u block
        v_t = -t_t                                     # D2^-1, t block
        return np.concatenate([v_u, v_t, v_p])

    def __call__(self, w):
        w = np.asarray(w, dtype=np.float64)
        if self.variant == "tpu":
            return self.apply_tpu(w)
        if self.variant == "tup":
            return self.apply_tup(w)
        return self.apply_tup_star(w)
