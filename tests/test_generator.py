"""Pins of the synthetic input generator against facts the paper and the
mathematics fix (Sec. 2.2 item list, Eq. block_def, Eq. Q2vsQ1)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import fracgen
from oracle import sparse as osp

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_u64(name):
    vals = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            vals.append(int(line, 16))
    return vals


def test_splitmix64_reference_outputs():
    # seed 0, stream 0 gives key mix64(0) = 0, i.e. the raw sequence from state 0
    ref = _golden_u64("splitmix64_seed0.txt")
    assert [fracgen.rand_u64(0, 0, i) for i in range(4)] == ref


def _rigid_modes(X):
    n = X.shape[0]
    Z = np.zeros((3 * n, 6))
    for d in range(3):
        Z[d::3, d] = 1.0
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    Z[0::3, 3], Z[1::3, 3] = -y, x
    Z[1::3, 4], Z[2::3, 4] = -z, y
    Z[0::3, 5], Z[2::3, 5] = z, -x
    return Z


def test_hex8_symmetric_rigid_nullspace_and_rank():
    K = fracgen.hex8_stiffness(0.25)
    assert np.allclose(K, K.T, atol=1e-15)
    X = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    Z = _rigid_modes(X)
    assert np.abs(K @ Z).max() < 1e-14
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-12) == 6 and ev.min() > -1e-14
    # uniaxial strain e_xx = 1 on the unit cube: strain energy = (lambda+2G)/2
    nu = 0.25
    lam, G = nu / ((1 + nu) * (1 - 2 * nu)), 1 / (2 * (1 + nu))
    u = np.zeros(24)
    u[0::3] = X[:, 0]
    assert np.isclose(0.5 * u @ K @ u, 0.5 * (lam + 2 * G), rtol=1e-13)
    # pure shear gamma_xy = 1: energy = G/2
    u = np.zeros(24)
    u[0::3] = X[:, 1]
    assert np.isclose(0.5 * u @ K @ u, 0.5 * G, rtol=1e-13)


def _coords(P):
    N1 = P.N + 1
    g = P.node_grid
    return np.stack([g % N1, (g // N1) % N1, g // (N1 * N1)], 1) / P.N


@pytest.mark.parametrize("name,kw", [("tiny8", {}), ("planes64", dict(N=8)),
                                     ("rects128", dict(N=12)), ("network96", dict(N=16, spacing=4))])
def test_A_symmetric_and_rigid_modes_of_each_piece(name, kw):
    P = fracgen.generate(name, **kw)
    A = osp.csr(P.A)
    assert abs(A - A.T).max() <= 1e-12 * abs(A).max()
    X = _coords(P)
    Z = _rigid_modes(X)
    # rows not coupled to a constrained dof see zero force from rigid motions;
    # rigid motions of the whole body are rigid on every split piece
    # the block pattern keeps every pair of copies sharing a cell, so a block
    # row touches a constrained dof iff one of its column copies carries one
    node_dir = P.dirichlet.reshape(-1, 3).any(axis=1)
    rp, ci = P.A.row_ptr, P.A.col_idx
    touched = np.array([node_dir[ci[rp[i]:rp[i + 1]]].any() for i in range(P.n_node)])
    free = np.repeat(~touched, 3)
    R = A @ Z
    assert np.abs(R[free]).max() <= 1e-11 * abs(A).max()

def test_A_blind_to_a_rigid_motion_of_one_side_of_a_full_plane():
    """The node split of S3: one fracture plane through the whole cube cuts
    it in two pieces that share no cell, so a translation of the + piece
    alone (every copy of a cell beyond the plane, the + copies on it) is a
    rigid motion of each piece and A sees no force in any row that no
    roller touches.  A copy shared across the plane (a wrong split) would
    couple the pieces and fail this."""
    P = fracgen.generate("tiny8")
    A = osp.csr(P.A)
    N1 = P.N + 1
    ix = P.node_grid % N1
    m = P.N // 2
    assert np.all(P.face_geom[:, 0] == 0) and np.all(P.face_geom[:, 1] == m)
    plus = (ix > m) | np.isin(np.arange(P.n_node), P.face_copies[:, 1, :])
    assert not np.any(np.isin(P.face_copies[:, 0, :], np.nonzero(plus)[0]))
    node_dir = P.dirichlet.reshape(-1, 3).any(axis=1)
    rp, ci = P.A.row_ptr, P.A.col_idx
    touched = np.array([node_dir[ci[rp[i]:rp[i + 1]]].any() for i in range(P.n_node)])
    free = np.repeat(~touched, 3)
    assert free.sum() > 0
    for d in range(3):
        v = np.zeros(A.shape[0])
        v[3 * np.nonzero(plus)[0] + d] = 1.0
        r = A @ v
        assert np.abs(r[free]).max() <= 1e-12 * abs(A).max()
        # and it is not blind to the same motion of a piece that crosses
        # the plane (the pin has teeth)
        w = np.zeros(A.shape[0])
        w[3 * np.nonzero(ix >= m - 1)[0] + d] = 1.0
        assert np.abs((A @ w)[free]).max() > 1e-3 * abs(A).max()


def test_A_patch_test_linear_field():
    # homogeneous material: a linear displacement field is an exact solution
    P = fracgen.generate("planes64", N=8, p_stick=1.0, p_slip=0.0, sigma_E=0.0)
    A = osp.csr(P.A)
    X = _coords(P)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((3, 3))
    u = (X @ G.T).reshape(-1)
    r = A @ u
    # nodes of a single copy with 8 cells, no constrained neighbours and away
    # from the fractures: the assembled force of a linear field vanishes
    N1 = P.N + 1
    g = P.node_grid
    I, J, K = g % N1, (g // N1) % N1, g // (N1 * N1)
    interior = (I >= 2) & (I <= P.N - 2) & (J >= 2) & (J <= P.N - 2) & (K >= 2) & (K <= P.N - 2)
    far = (np.abs(I - P.N // 2) >= 2) & (np.abs(J - P.N // 2) >= 2) & (np.abs(K - P.N // 2) >= 2)
    sel = np.repeat(interior & far, 3)
    assert sel.sum() > 0
    assert np.abs(r[sel]).max() <= 1e-11 * abs(A).max()


def test_stick_invariants(tiny):
    """All stick: C2 = C1^T and Q2 = 0, so J is reducible (Sec. 2.2 items 2, 4)."""
    P = tiny
    assert np.all(P.state == 0)
    b = osp.blocks(P)
    assert (b["C2"] - b["C1"].T).count_nonzero() == 0
    assert b["Q2"].count_nonzero() == 0


def test_Q1_is_minus_normal_column_of_C1():
    """Q1 = -([[eta_N]], chi) is minus the normal-traction column of C1 (Eq. block_def)."""
    P = fracgen.generate("rects128", N=12)
    b = osp.blocks(P)
    C1n = b["C1"][:, 0::3]
    assert abs(b["Q1"] + C1n).max() == 0.0


def test_C1_partition_of_unity():
    """Per face and side the C1 blocks add up to +-h^2 R_f^T (integral of the
    nodal basis over the face) where no boundary row is eliminated."""
    P = fracgen.generate("planes64", N=8)
    C1 = osp.csr(P.C1).toarray()
    h2 = P.h ** 2
    for f in range(P.n_face):
        a, m, p, q = P.face_geom[f]
        cps = P.face_copies[f]
        rows_dir = P.dirichlet.reshape(-1, 3)[cps.ravel()].any()
        if rows_dir or np.any(cps[0] == cps[1]):
            continue
        R = np.zeros((3, 3))
        R[0, a] = R[1, (a + 1) % 3] = R[2, (a + 2) % 3] = 1.0
        for side, sg in ((0, -1.0), (1, 1.0)):
            tot = sum(C1[3 * c:3 * c + 3, 3 * f:3 * f + 3] for c in cps[side])
            assert np.allclose(tot, sg * h2 * R.T, rtol=1e-14, atol=1e-18)


def test_T_symmetric_spd_rowsums():
    """T: SPD 2-D TPFA Laplacian plus stabilisation; its rows sum to the
    Dirichlet corner terms only (Sec. 2.2 item 5, Eq. FV_inner_product)."""
    P = fracgen.generate("rects128", N=12)
    T = osp.csr(P.T)
    assert abs(T - T.T).max() <= 1e-14 * abs(T).max()
    ev = np.linalg.eigvalsh(T.toarray())
    assert ev.min() > 0
    rs = np.asarray(T.sum(axis=1)).ravel()
    nonzero = np.abs(rs) > 1e-12 * abs(T).max()
    # only corner faces of fractures carry Dirichlet edges
    corners = set()
    for a, m, p0, q0, p1, q1 in P.rects:
        for p, q in ((p0, q0), (p1, q0), (p0, q1), (p1, q1)):
            hit = np.nonzero((P.face_geom[:, 0] == a) & (P.face_geom[:, 1] == m) &
                             (P.face_geom[:, 2] == p) & (P.face_geom[:, 3] == q))[0]
            corners.update(hit.tolist())
    assert set(np.nonzero(nonzero)[0].tolist()) <= corners
    # each Dirichlet edge adds the one-sided transmissibility of its face
    k = np.nonzero(nonzero)[0]
    ratio = rs[k] / P.ups_face[k]
    assert np.allclose(ratio, np.round(ratio), rtol=1e-12) and np.all(np.round(ratio) >= 1)


def test_H_singular_in_stick_and_Htilde_regular():
    """H is singular (Sec. 2.2 item 3); its 3x3 diagonal blocks are not."""
    P = fracgen.generate("tiny8")
    H = osp.csr(P.H).toarray()
    # constant traction field over a stick-only plane is in the kernel of j_t
    c = np.tile([1.0, 0.0, 0.0], P.n_face)
    assert np.abs(H @ c).max() <= 1e-14 * np.abs(H).max()
    P2 = fracgen.generate("planes64", N=8)
    Hb = osp.csr(P2.H).toarray()
    for f in range(P2.n_face):
        blk = Hb[3 * f:3 * f + 3, 3 * f:3 * f + 3]
        assert abs(np.linalg.det(blk)) > 0


def _flux_residual_rows(P, g_open):
    """[chi_K, p^l]_F as a function of the apertures of open faces:
    TPFA with one-sided transmissibility 2 C_f / mu, series average over each
    pair of faces sharing an edge, Dirichlet corner edges (Eq. FV_inner_product)."""
    nf = P.n_face
    C_f = P.C_f0 + g_open ** 3 / 12.0
    ups = 2.0 * C_f / P.mu
    N1 = P.N + 1
    edges = {}
    for f in range(nf):
        a, m, p, q = P.face_geom[f]
        t1, t2 = (a + 1) % 3, (a + 2) % 3
        for e in range(4):
            g = [0, 0, 0]
            g[a] = m
            if e < 2:
                g[t1], g[t2], d = p, q + e, t1
            else:
                g[t1], g[t2], d = p + e - 2, q, t2
            key = (g[0] + N1 * (g[1] + N1 * g[2])) * 3 + d
            edges.setdefault(key, []).append((f, e))
    out = np.zeros(nf, dtype=ups.dtype)
    pl = P.pl
    for key, lst in edges.items():
        fs = [f for f, _ in lst]
        for i in range(len(fs)):
            for j in range(i + 1, len(fs)):
                K, L = fs[i], fs[j]
                u = ups[K] * ups[L] / (ups[K] + ups[L])
                out[K] += u * (pl[K] - pl[L])
                out[L] += u * (pl[L] - pl[K])
    for a, m, p0, q0, p1, q1 in P.rects:
        seen = set()
        for (p, q) in ((p0, q0), (p1, q0), (p0, q1), (p1, q1)):
            hit = np.nonzero((P.face_geom[:, 0] == a) & (P.face_geom[:, 1] == m) &
                             (P.face_geom[:, 2] == p) & (P.face_geom[:, 3] == q))[0]
            if len(hit) == 0 or hit[0] in seen:
                continue
            K = hit[0]
            seen.add(K)
            t1, t2 = (a + 1) % 3, (a + 2) % 3
            for e in range(4):
                g = [0, 0, 0]
                g[a] = m
                if e < 2:
                    g[t1], g[t2], d = p, q + e, t1
                    outer = (e == 0 and q == q0) or (e == 1 and q == q1)
                else:
                    g[t1], g[t2], d = p + e - 2, q, t2
                    outer = (e == 2 and p == p0) or (e == 3 and p == p1)
                key = (g[0] + N1 * (g[1] + N1 * g[2])) * 3 + d
                if outer and len(edges[key]) == 1:
                    out[K] += ups[K] * pl[K]
    return out


def test_Q2_equals_storage_term_plus_complex_step_flux_derivative():
    """Q2 = -Psi(Q1^T)/dt + F_u (Eq. Q2vsQ1), F_u by complex-step
    differentiation of the TPFA flux w.r.t. u through the open apertures
    g_K = a_K + mean normal jump."""
    P = fracgen.generate("planes64", N=6, p_stick=0.4, p_slip=0.2)
    b = osp.blocks(P)
    Q1, Q2 = b["Q1"], b["Q2"]
    open_ = P.state == 2
    Psi = sp.diags(open_.astype(float)) @ Q1.T
    Fu = (Q2 + Psi / P.dt).toarray()
    nu = 3 * P.n_node
    rng = np.random.default_rng(3)
    for _ in range(4):
        du = rng.standard_normal(nu)
        du[P.dirichlet] = 0.0
        hstep = 1e-30
        U = (hstep * 1j) * du
        jump = np.zeros(P.n_face, dtype=complex)
        for f in range(P.n_face):
            a = P.face_geom[f, 0]
            cm, cp = P.face_copies[f]
            jump[f] = 0.25 * (U[3 * cp + a].sum() - U[3 * cm + a].sum())
        g = P.aperture.astype(complex) + np.where(open_, jump, 0.0)
        d = _flux_residual_rows(P, g).imag / hstep
        assert np.allclose(Fu @ du, d, rtol=1e-10, atol=1e-12 * np.abs(d).max())


# ---------------------------------------------------------------- slip and open faces
def _normal(seed: int, stream: int, i: int) -> float:
    """Standard normal by Box-Muller from the counter draws 2i and 2i+1."""
    u1 = 1.0 - fracgen.uniform(seed, stream, 2 * i)
    u2 = fracgen.uniform(seed, stream, 2 * i + 1)
    return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2))


def _slip_data(P, f):
    """Seeded slip data of face f: t_N = -(5 + 10 U) MPa (stream 3), slip
    direction at angle 2 pi U (stream 4), |Delta g_T| = 1e-4 exp(0.5 Z) m
    (stream 5)."""
    s = P.cfg.seed
    tN = -(5.0 + 10.0 * fracgen.uniform(s, 3, f))
    phi = 2.0 * np.pi * fracgen.uniform(s, 4, f)
    dg = 1e-4 * np.exp(0.5 * _normal(s, 5, f))
    return tN, np.array([np.cos(phi), np.sin(phi)]), dg


TAN_THETA = np.tan(np.deg2rad(30.0))   # friction angle 30 degrees, cohesion 0


def _friction_law(dgT, tN):
    """t_T* = tau_max(t_N) Delta g_T / ||Delta g_T|| with the static Coulomb
    limit tau_max = c - t_N tan(theta) (Sec. 2.1); written with sqrt(x.x)
    so that a complex step differentiates it."""
    tau = 0.0 - tN * TAN_THETA
    return tau * dgT / np.sqrt(dgT[0] * dgT[0] + dgT[1] * dgT[1])


def _frame(a):
    R = np.zeros((3, 3))
    R[0, a] = R[1, (a + 1) % 3] = R[2, (a + 2) % 3] = 1.0
    return R


def _k(P, f):
    # k = Ebar_f / (8 h): the generator's reading of the paper's k
    return P.Ebar_face[f] / (8.0 * P.h)


def test_C2_slip_rows_are_the_friction_law_derivative():
    """Eq. C2def on a slip face: the normal row is (mu_N, [[eta_N]]) as for
    stick; the tangential rows are -(1/k)(mu_T, dt_T*/dDelta g_T .
    [[eta_T]]).  The derivative is taken here by complex step of the
    friction law itself at the seeded slip data, and the face integral of
    the jump of a nodal basis function is +-h^2/4 (+ copy, - copy), so C2's
    (face, copy) block is fixed entry by entry.  A flipped sign of the
    derivative, a missing tangential projection (I - g g^T), k for 1/k or
    swapped sides all fail it."""
    P = fracgen.generate("planes64", N=6, p_stick=0.2, p_slip=0.7, seed=5)
    C2 = osp.csr(P.C2).toarray()
    dirichlet = P.dirichlet.reshape(-1, 3)
    w = P.h ** 2 / 4.0
    slip = np.nonzero(P.state == 1)[0]
    assert slip.size > 10
    checked = 0
    for f in slip:
        tN, ghat, dg = _slip_data(P, f)
        D = np.zeros((2, 2))
        for j in range(2):
            e = np.zeros(2, dtype=complex)
            e[j] = 1e-30j
            D[:, j] = _friction_law(dg * ghat + e, tN).imag / 1e-30
        R = _frame(P.face_geom[f, 0])
        cm, cp = P.face_copies[f]
        for side, sg in ((0, -1.0), (1, 1.0)):
            for k in range(4):
                c = (cm, cp)[side][k]
                got = C2[3 * f:3 * f + 3, 3 * c:3 * c + 3]
                if cm[k] == cp[k]:
                    # a fracture tip: one copy, zero jump
                    assert np.all(got == 0.0)
                    continue
                jump = sg * w * R                 # d/du_c of the face integral of [[u]] in (n, t1, t2)
                exp = np.vstack([jump[0], -(1.0 / _k(P, f)) * D @ jump[1:]])
                exp[:, dirichlet[c]] = 0.0
                assert np.allclose(got, exp, rtol=1e-12, atol=1e-14 * np.abs(exp).max())
                checked += 1
    assert checked > 40


def test_H_slip_and_open_blocks_follow_the_linearisation():
    """Eq. Hdef.  An open face's row and column of H hold only its diagonal
    block -(1/k)(mu, mu) = -(h^2/k) I (no j_t on open faces, Sec. 2.2 item
    3).  A slip face's diagonal block is its stick block (the j_t part, set
    by geometry and material alone) plus -(h^2/k) on the tangential diagonal
    and (h^2/k) dt_T*/dt_N in the tangential rows of the normal column, the
    derivative by complex step of t_T* in t_N.  Compared with the same
    instance in all-stick state.  A flipped friction term, h^2 k for h^2/k
    or j_t kept on open faces fail it."""
    over = dict(N=6, seed=5)
    P = fracgen.generate("planes64", p_stick=0.2, p_slip=0.5, **over)
    P0 = fracgen.generate("planes64", p_stick=1.0, p_slip=0.0, **over)
    assert np.array_equal(P.face_geom, P0.face_geom) and np.array_equal(P.E_cell, P0.E_cell)
    H = osp.csr(P.H).toarray()
    H0 = osp.csr(P0.H).toarray()
    kinds = {0: 0, 1: 0, 2: 0}
    for f in range(P.n_face):
        blk = H[3 * f:3 * f + 3, 3 * f:3 * f + 3]
        hk = P.h ** 2 / _k(P, f)
        st = int(P.state[f])
        kinds[st] += 1
        if st == 0:
            assert np.array_equal(blk, H0[3 * f:3 * f + 3, 3 * f:3 * f + 3])
        elif st == 2:
            assert np.allclose(blk, -hk * np.eye(3), rtol=1e-14, atol=0)
            row = H[3 * f:3 * f + 3].copy()
            row[:, 3 * f:3 * f + 3] = 0.0
            col = H[:, 3 * f:3 * f + 3].copy()
            col[3 * f:3 * f + 3] = 0.0
            assert not row.any() and not col.any()
        else:
            tN, ghat, dg = _slip_data(P, f)
            dtdn = _friction_law(dg * ghat + 0j, tN + 1e-30j).imag / 1e-30
            exp = np.zeros((3, 3))
            exp[1, 1] = exp[2, 2] = -hk
            exp[1:, 0] = hk * dtdn
            diff = blk - H0[3 * f:3 * f + 3, 3 * f:3 * f + 3]
            assert np.allclose(diff, exp, rtol=1e-12, atol=1e-14 * hk)
    assert min(kinds.values()) > 5


def _edge_pairs(P):
    """Pairs of faces sharing a grid edge (the TPFA connections of every
    fracture, intersections included), with a coplanarity flag."""
    N1 = P.N + 1
    edges = {}
    for f in range(P.n_face):
        a, m, p, q = P.face_geom[f]
        t1, t2 = (a + 1) % 3, (a + 2) % 3
        for e in range(4):
            g = [0, 0, 0]
            g[a] = m
            if e < 2:
                g[t1], g[t2], d = p, q + e, t1
            else:
                g[t1], g[t2], d = p + e - 2, q, t2
            edges.setdefault((g[0] + N1 * (g[1] + N1 * g[2])) * 3 + d, []).append(f)
    out = {}
    for fs in edges.values():
        for i in range(len(fs)):
            for j in range(i + 1, len(fs)):
                K, L = fs[i], fs[j]
                cop = (P.face_geom[K, 0] == P.face_geom[L, 0]) and (P.face_geom[K, 1] == P.face_geom[L, 1])
                out[(min(K, L), max(K, L))] = bool(cop)
    return out


def test_T_is_tpfa_plus_normal_projection_of_jt_over_dt():
    """Eq. Tdef: T = d[chi, p]_F/dp + (1/dt) j_p with j_p the normal
    projection of j_t on every pair of coplanar faces, in every state
    (Sec. 2.2).  Off the diagonal: T_KL = -Ups_K Ups_L / (Ups_K + Ups_L)
    for every pair of faces sharing an edge (series TPFA, one-sided
    2 C_f / mu, C_f = C_f0 + a^3 / 12, Eq. cond_def), plus H0_KL[N, N] / dt
    for coplanar pairs, H0 the stabilisation of the same instance in
    all-stick state (j_t then spans every coplanar edge); zero elsewhere.
    Dropping the 1/dt, projecting on a tangential component, a harmonic
    mean (twice the series value) or no flow across intersections fail it."""
    over = dict(N=6, seed=2)
    P = fracgen.generate("planes64", **over)
    P0 = fracgen.generate("planes64", p_stick=1.0, p_slip=0.0, **over)
    assert np.array_equal(P.aperture, P0.aperture)
    T = osp.csr(P.T).toarray()
    H0 = osp.csr(P0.H).toarray()
    ups = 2.0 * (P.C_f0 + P.aperture ** 3 / 12.0) / P.mu
    exp = np.zeros_like(T)
    pairs = _edge_pairs(P)
    assert any(pairs.values()) and not all(pairs.values())
    for (K, L), cop in pairs.items():
        v = -ups[K] * ups[L] / (ups[K] + ups[L])
        if cop:
            v += H0[3 * K, 3 * L] / P.dt
            assert H0[3 * K, 3 * L] < 0
        exp[K, L] = exp[L, K] = v
    off = ~np.eye(P.n_face, dtype=bool)
    assert np.allclose(T[off], exp[off], rtol=1e-13, atol=1e-15 * np.abs(T).max())
