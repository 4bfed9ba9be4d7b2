"""Smoothed-aggregation AMG and its V-cycle (plain FP64 reference).

The paper applies S~^-1 and S1^-1 by an aggregation-based AMG (Sec. 3.1:
GAMG, smoothed aggregation in the family of Vanek, Mandel and Brezina) and
gives no settings.  This is the explicit algorithm both implementations
follow; every step is written out in its plain order:

Setup, on level l with block size B (3 for S1/S~, 1 for T/S~2):
 1. strength: a stored off-diagonal block S_ij is strong when
        ||S_ij||_F^2 > theta_l^2 * ||S_ii||_F * ||S_jj||_F,
    theta_l = theta0 * decay^l; ||.||_F^2 summed entry by entry in row-major
    order.  Weight w_ij = ||S_ij||_F^2 / (||S_ii||_F ||S_jj||_F).  The
    undirected strength graph has edge {i,j} when i->j or j->i is strong, with
    weight max of the strong directions.  Nodes without edges are left out
    (no coarse unknown).
 2. roots: greedy distance-2 maximal independent set on that graph, nodes
    visited by descending 64-bit key (SplitMix64 draw, stream 10, with its
    low 26 bits replaced by the node index).
 3. aggregates: round 1 puts each neighbour of a root into its strongest
    root (ties: lower index); round 2 puts each still-unassigned node into
    the aggregate of its strongest round-1-assigned neighbour; remaining
    nodes seed singletons.  Aggregates are numbered by their seed's index.
 4. P_tent(i, agg(i)) = I_B / sqrt(|agg(i)|).
 5. lambda^ = ||D^-1 S v|| / ||v|| after 15 normalised power steps from
    v0 = U(-1,1) (stream 11); D = B x B block diagonal of S.
 6. P = (I - omega D^-1 S) P_tent, omega = (4/3) / lambda^.
 7. S_c = P^T S P.  Stop when n <= coarse_max, at max_levels, or when
    n_c > max_ratio * n.  Coarsest level: dense LU, partial pivoting.

Apply: V(1,1) cycle, zero initial guess on every level, Chebyshev smoother of
degree 2 for D^-1 S on [lo * 1.1 lambda^, 1.1 lambda^] (Saad, Iterative
Methods for Sparse Linear Systems, Alg. 12.1), the same smoother before and
after the coarse correction.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import rng


@dataclass
class AmgOptions:
    theta0: float = 0.08
    theta_decay: float = 0.5
    coarse_max: int = 200         # block rows
    max_levels: int = 12
    max_ratio: float = 0.8
    power_steps: int = 15
    omega_num: float = 4.0 / 3.0
    cheb_degree: int = 2
    cheb_hi: float = 1.1
    cheb_lo: float = 0.1
    seed: int = 0
    dense_limit: int = 20000      # scalar rows allowed on the coarsest level


@dataclass
class Level:
    S: sp.csr_matrix
    B: int
    n: int
    Dinv: np.ndarray | None = None
    lam: float = 0.0
    P: sp.csr_matrix | None = None
    R: sp.csr_matrix | None = None
    agg: np.ndarray | None = None
    nc: int = 0
    info: dict = field(default_factory=dict)


def block_norms2(Sb: sp.bsr_matrix) -> np.ndarray:
    """||block||_F^2 per stored block, summed entry by entry in row-major order."""
    B2 = Sb.data.shape[1] * Sb.data.shape[2]
    flat = Sb.data.reshape(-1, B2)
    s = np.zeros(flat.shape[0])
    for k in range(B2):
        s = s + flat[:, k] * flat[:, k]
    return s


def to_bsr(S: sp.csr_matrix, B: int) -> sp.bsr_matrix:
    Sb = sp.bsr_matrix(S, blocksize=(B, B))
    Sb.sort_indices()
    return Sb


def diag_blocks(Sb: sp.bsr_matrix, B: int) -> np.ndarray:
    n = Sb.shape[0] // B
    D = np.zeros((n, B, B))
    rows = np.repeat(np.arange(n), np.diff(Sb.indptr))
    on = rows == Sb.indices
    D[rows[on]] = Sb.data[on]
    return D


def strength_graph(S: sp.csr_matrix, B: int, level: int, opt: AmgOptions):
    """Undirected strength graph (CSR, sorted, no self loops) with weights."""
    Sb = to_bsr(S, B)
    n = Sb.shape[0] // B
    s = block_norms2(Sb)
    rows = np.repeat(np.arange(n), np.diff(Sb.indptr))
    cols = Sb.indices
    dsq = np.zeros(n)
    on = rows == cols
    dsq[rows[on]] = s[on]
    d = np.sqrt(dsq)
    theta = opt.theta0 * opt.theta_decay ** level
    thr = (theta * theta) * (d[rows] * d[cols])
    strong = (rows != cols) & (s > thr)
    w = s[strong] / (d[rows[strong]] * d[cols[strong]])
    Wd = sp.csr_matrix((w, (rows[strong], cols[strong])), shape=(n, n))
    W = Wd.maximum(Wd.T).tocsr()
    W.sort_indices()
    return W


def priority_keys(n: int, level: int, seed: int) -> np.ndarray:
    r = rng.rand_u64(seed, rng.STREAM_PRIORITY, rng.level_index(level, np.arange(n)))
    mask = np.uint64((1 << 26) - 1)
    return (r & ~mask) | np.arange(n, dtype=np.uint64)


def mis2_greedy(W: sp.csr_matrix, keys: np.ndarray) -> np.ndarray:
    """Greedy distance-2 maximal independent set, by descending key."""
    n = W.shape[0]
    deg = np.diff(W.indptr)
    cand = np.nonzero(deg > 0)[0]
    order = cand[np.argsort(keys[cand])[::-1]]
    blocked = np.zeros(n, dtype=bool)
    is_root = np.zeros(n, dtype=bool)
    ip, ix = W.indptr, W.indices
    for v in order:
        if blocked[v]:
            continue
        is_root[v] = True
        n1 = ix[ip[v]:ip[v + 1]]
        blocked[v] = True
        blocked[n1] = True
        for u in n1:
            blocked[ix[ip[u]:ip[u + 1]]] = True
    return is_root


def aggregate(W: sp.csr_matrix, is_root: np.ndarray):
    """Two assignment rounds; returns (agg index per node or -1, n_coarse)."""
    n = W.shape[0]
    deg = np.diff(W.indptr)
    rows = np.repeat(np.arange(n), deg)
    cols = W.indices
    w = W.data
    owner = np.full(n, -1, dtype=np.int64)      # node index of the seed
    owner[is_root] = np.nonzero(is_root)[0]
    # round 1: neighbours of roots join the strongest root (ties: lower index)
    m = (~is_root[rows]) & is_root[cols]
    r1, c1, w1 = rows[m], cols[m], w[m]
    o = np.lexsort((c1, -w1, r1))
    r1, c1 = r1[o], c1[o]
    first = np.ones(len(r1), dtype=bool)
    first[1:] = r1[1:] != r1[:-1]
    owner[r1[first]] = c1[first]
    assigned1 = owner >= 0
    # round 2: remaining nodes join the aggregate of their strongest
    # round-1-assigned neighbour
    m = (~assigned1[rows]) & assigned1[cols]
    r2, c2, w2 = rows[m], cols[m], w[m]
    o = np.lexsort((c2, -w2, r2))
    r2, c2 = r2[o], c2[o]
    first = np.ones(len(r2), dtype=bool)
    first[1:] = r2[1:] != r2[:-1]
    new_owner = owner.copy()
    new_owner[r2[first]] = owner[c2[first]]
    owner = new_owner
    # leftovers with edges seed their own aggregate
    left = (owner < 0) & (deg > 0)
    owner[left] = np.nonzero(left)[0]
    seeds = np.zeros(n, dtype=bool)
    seeds[is_root] = True
    seeds[left] = True
    seed_idx = np.full(n, -1, dtype=np.int64)
    seed_idx[seeds] = np.arange(int(seeds.sum()))
    agg = np.where(owner >= 0, seed_idx[np.maximum(owner, 0)], -1)
    return agg, int(seeds.sum())


def tentative(agg: np.ndarray, nc: int, B: int) -> sp.csr_matrix:
    n = len(agg)
    has = agg >= 0
    size = np.bincount(agg[has], minlength=nc).astype(np.float64)
    rows, cols, vals = [], [], []
    nodes = np.nonzero(has)[0]
    for c in range(B):
        rows.append(B * nodes + c)
        cols.append(B * agg[nodes] + c)
        vals.append(1.0 / np.sqrt(size[agg[nodes]]))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n * B, nc * B))


def rigid_modes(coords: np.ndarray) -> np.ndarray:
    """The six rigid-body motions of nodes at `coords` (n x 3): three
    translations and three rotations (x, y, z interleaved per node)."""
    n = coords.shape[0]
    Z = np.zeros((3 * n, 6))
    for d in range(3):
        Z[d::3, d] = 1.0
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    Z[0::3, 3], Z[1::3, 3] = -y, x
    Z[1::3, 4], Z[2::3, 4] = -z, y
    Z[0::3, 5], Z[2::3, 5] = z, -x
    return Z


def tentative_nullspace(agg: np.ndarray, nc: int, B: int, Z: np.ndarray, tol: float = 1e-10):
    """Tentative prolongator that reproduces the candidate vectors Z (B n x k)
    on every aggregate (smoothed aggregation with a general near-null space,
    Vanek, Mandel and Brezina): per aggregate, the thin QR of Z restricted to
    the aggregate's rows gives the block of P_tent (Q) and the coarse
    candidates (R), so that P_tent Z_c = Z there.  A column of R whose
    diagonal falls below tol times the largest (an aggregate too small or too
    flat to carry all k modes) is a dead coarse dof: its column of P_tent is
    zero.  Returns (P_tent, Z_c (k nc x k), dead mask over the k nc coarse
    dofs)."""
    k = Z.shape[1]
    rows_p, cols_p, vals_p = [], [], []
    Zc = np.zeros((k * nc, k))
    dead = np.zeros(k * nc, dtype=bool)
    nodes_of = [[] for _ in range(nc)]
    for i in np.nonzero(agg >= 0)[0]:
        nodes_of[agg[i]].append(i)
    for a in range(nc):
        nodes = np.array(nodes_of[a], dtype=np.int64)
        r = (B * nodes[:, None] + np.arange(B)).ravel()
        Q, R = np.linalg.qr(Z[r], mode="complete" if len(r) < k else "reduced")
        Q, R = Q[:, :k], R[:k]
        if Q.shape[1] < k:                      # fewer rows than candidates
            Q = np.hstack([Q, np.zeros((len(r), k - Q.shape[1]))])
            R = np.vstack([R, np.zeros((k - R.shape[0], k))])
        diag = np.abs(np.diag(R))
        off = diag <= tol * max(diag.max(), 1e-300)
        Q[:, off] = 0.0
        R[off] = 0.0
        dead[k * a + np.nonzero(off)[0]] = True
        Zc[k * a:k * a + k] = R
        rr, cc = np.nonzero(Q)
        rows_p.append(r[rr])
        cols_p.append(k * a + cc)
        vals_p.append(Q[rr, cc])
    Pt = sp.csr_matrix((np.concatenate(vals_p), (np.concatenate(rows_p), np.concatenate(cols_p))),
                       shape=(len(agg) * B, nc * k))
    return Pt, Zc, dead


def apply_blockdiag(Dinv: np.ndarray, r: np.ndarray) -> np.ndarray:
    B = Dinv.shape[1]
    return np.einsum("nij,nj->ni", Dinv, r.reshape(-1, B)).reshape(-1)


def power_lambda(S, Dinv, B, level, opt: AmgOptions) -> float:
    """lambda^ of D^-1 S: 15 normalised power steps from a U(-1,1) start."""
    nb = S.shape[0]
    v = 2.0 * rng.uniform(opt.seed, rng.STREAM_POWER, rng.level_index(level, np.arange(nb))) - 1.0
    lam = 0.0
    for _ in range(opt.power_steps):
        w = apply_blockdiag(Dinv, S @ v)
        nw = np.linalg.norm(w)
        lam = nw / np.linalg.norm(v)
        v = w / nw
    return float(lam)


class AMG:
    """Hierarchy and V-cycle for one operator (block size B)."""

    def __init__(self, S: sp.csr_matrix, B: int, opt: AmgOptions | None = None,
                 aggregates: list | None = None, near_null: np.ndarray | None = None):
        """``aggregates``: the (agg, n_coarse) pair of every coarsening step of
        an earlier hierarchy.  Given, the hierarchy is rebuilt on new values
        of S with those aggregates (no strength graph, no MIS-2): the same
        levels, with D^-1, lambda, P, R and the Galerkin products recomputed.
        ``near_null``: candidate vectors (rows of S x k), e.g. the six rigid
        modes of ``rigid_modes``; P_tent then reproduces them aggregate by
        aggregate (``tentative_nullspace``), every coarse level has k x k
        blocks, and dead coarse dofs get a unit diagonal in S_c.  None: the
        translations I_B / sqrt|agg| of step 4."""
        self.opt = opt or AmgOptions()
        self.B = B
        Z = near_null
        self.levels: list[Level] = []
        S = S.tocsr()
        S.sort_indices()
        lvl = 0
        while True:
            n = S.shape[0] // B
            L = Level(S=S, B=B, n=n)
            self.levels.append(L)
            if aggregates is not None:
                if lvl >= len(aggregates):
                    break
                agg, nc = aggregates[lvl]
                is_root = np.zeros(n, dtype=bool)
            else:
                if n <= self.opt.coarse_max or lvl + 1 >= self.opt.max_levels:
                    break
                W = strength_graph(S, B, lvl, self.opt)
                is_root = mis2_greedy(W, priority_keys(n, lvl, self.opt.seed))
                agg, nc = aggregate(W, is_root)
                if nc == 0 or nc > self.opt.max_ratio * n:
                    break
            Sb = to_bsr(S, B)
            D = diag_blocks(Sb, B)
            Dinv = np.linalg.inv(D)
            lam = power_lambda(S, Dinv, B, lvl, self.opt)
            if Z is None:
                Pt, Bc, dead = tentative(agg, nc, B), B, None
            else:
                Pt, Z, dead = tentative_nullspace(agg, nc, B, Z)
                Bc = Z.shape[1]
            omega = self.opt.omega_num / lam
            Dinv_sp = sp.block_diag(list(Dinv), format="csr")
            P = (Pt - omega * (Dinv_sp @ (S @ Pt))).tocsr()
            R = P.T.tocsr()
            Sc = (R @ S @ P).tocsr()
            if dead is not None and dead.any():
                Sc = (Sc + sp.diags(dead.astype(float))).tocsr()
            Sc.sort_indices()
            L.Dinv, L.lam, L.P, L.R, L.agg = Dinv, lam, P, R, agg
            L.info = dict(n_coarse=nc, n_roots=int(is_root.sum()), dead=int(dead.sum()) if dead is not None else 0)
            L.nc = nc
            S = Sc
            B = Bc
            lvl += 1
        last = self.levels[-1]
        if last.S.shape[0] > self.opt.dense_limit:
            raise RuntimeError(f"coarsest level too large for a dense solve: {last.S.shape[0]}")
        self.lu = sla.lu_factor(last.S.toarray()) if last.S.shape[0] else None

    def aggregates(self) -> list:
        """(agg, n_coarse) of every coarsening step, for a numeric rebuild."""
        return [(L.agg, L.nc) for L in self.levels[:-1]]

    # -------------------------------------------------------------- apply
    def _cheb(self, L: Level, f: np.ndarray, x0: np.ndarray | None) -> np.ndarray:
        hi = self.opt.cheb_hi * L.lam
        lo = self.opt.cheb_lo * hi
        theta = 0.5 * (hi + lo)
        delta = 0.5 * (hi - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        if x0 is None:
            r = f
            x = np.zeros_like(f)
        else:
            r = f - L.S @ x0
            x = x0
        d = apply_blockdiag(L.Dinv, r) / theta
        x = x + d
        for _ in range(1, self.opt.cheb_degree):
            rho_new = 1.0 / (2.0 * sigma - rho)
            r = f - L.S @ x
            d = (rho_new * rho) * d + (2.0 * rho_new / delta) * apply_blockdiag(L.Dinv, r)
            x = x + d
            rho = rho_new
        return x

    def vcycle(self, f: np.ndarray, lvl: int = 0) -> np.ndarray:
        L = self.levels[lvl]
        if lvl == len(self.levels) - 1:
            if L.S.shape[0] == 0:
                return np.zeros_like(f)
            return sla.lu_solve(self.lu, f)
        x = self._cheb(L, f, None)
        r = f - L.S @ x
        ec = self.vcycle(L.R @ r, lvl + 1)
        x = x + L.P @ ec
        return self._cheb(L, f, x)

    def __call__(self, f: np.ndarray) -> np.ndarray:
        return self.vcycle(np.asarray(f, dtype=np.float64))

    # -------------------------------------------------------------- transpose
    # The V-cycle is a linear operator B(S).  With the same polynomial
    # smoother before and after the correction and R = P^T, its transpose is
    # the same cycle run on the transposed level operators S_l^T (the
    # Galerkin coarse operators transpose accordingly: R S^T P = (R S P)^T),
    # with the transposed diagonal blocks and the transposed coarsest solve.
    def _cheb_t(self, L: Level, f: np.ndarray, x0):
        St = L.S.T.tocsr()
        DinvT = np.transpose(L.Dinv, (0, 2, 1))
        hi = self.opt.cheb_hi * L.lam
        lo = self.opt.cheb_lo * hi
        theta = 0.5 * (hi + lo)
        delta = 0.5 * (hi - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        if x0 is None:
            r = f
            x = np.zeros_like(f)
        else:
            r = f - St @ x0
            x = x0
        d = apply_blockdiag(DinvT, r) / theta
        x = x + d
        for _ in range(1, self.opt.cheb_degree):
            rho_new = 1.0 / (2.0 * sigma - rho)
            r = f - St @ x
            d = (rho_new * rho) * d + (2.0 * rho_new / delta) * apply_blockdiag(DinvT, r)
            x = x + d
            rho = rho_new
        return x

    def vcycle_t(self, f: np.ndarray, lvl: int = 0) -> np.ndarray:
        """Apply B^T, the transpose of the V-cycle operator."""
        f = np.asarray(f, dtype=np.float64)
        L = self.levels[lvl]
        if lvl == len(self.levels) - 1:
            if L.S.shape[0] == 0:
                return np.zeros_like(f)
            return sla.lu_solve(self.lu, f, trans=1)
        x = self._cheb_t(L, f, None)
        r = f - L.S.T @ x
        ec = self.vcycle_t(L.R @ r, lvl + 1)
        x = x + L.P @ ec
        return self._cheb_t(L, f, x)

    def describe(self) -> list[tuple[int, int]]:
        return [(L.n, L.S.nnz) for L in self.levels]
