"""GPU parity of the adjoint path (transposed products, transposed V-cycles,
M^-T, FGMRES on J^T) against the oracle, the dense adjoint on the 8^3 case,
and the gradient of 0.5 ||p - p_obs||^2 w.r.t. b through
torch.autograd (central differences)."""
import numpy as np
import pytest

import fracgen
from oracle import adjoint, schur
from oracle import sparse as osp
from oracle.amg import AMG, AmgOptions
from oracle.precond import BlockPreconditioner

from fields import assert_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "tiny8": ("tiny8", {}, 64, 16),
    "planes8": ("planes64", dict(N=8), 32, 16),
    "rects16": ("rects128", dict(N=16), 50, 30),
}


@pytest.fixture(scope="module")
def fs():
    import paper_2112_12397_gb300 as m
    m.load(build_if_missing=True)
    return m


_cache = {}


def case(name, fs):
    if name not in _cache:
        preset, over, cm, cmp = CASES[name]
        P = fracgen.generate(preset, **over)
        ctx = fs.context_for(P, fs.default_options(coarse_max=cm, coarse_max_p=cmp))
        _cache[name] = (P, ctx, AmgOptions(coarse_max=cm), AmgOptions(coarse_max=cmp))
    return _cache[name]


def cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name", sorted(CASES))
def test_transposed_products(fs, name):
    P, ctx, opt, optp = case(name, fs)
    JT = osp.jacobian(P).T.tocsr()
    x = np.random.default_rng(0).standard_normal(P.n)
    y = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    ctx.spmv_adjoint(cuda(x), y)
    assert np.all(np.abs(y.cpu().numpy() - JT @ x) <= 2e-14 * (abs(JT) @ np.abs(x)))
    S1 = schur.s1(P)
    for hier, M in ((fs.FC_H_TUP_U, S1), (fs.FC_H_TPU_U, schur.s_tilde(P, S1=S1))):
        ref = AMG(M, 3, opt)
        f = np.random.default_rng(hier).standard_normal(M.shape[0])
        xo = torch.zeros(M.shape[0], dtype=torch.float64, device="cuda")
        ctx.vcycle_adjoint(hier, cuda(f), xo)
        assert rel(xo.cpu().numpy(), ref.vcycle_t(f)) <= 1e-10


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("variant", ["tpu", "tup", "tup_star"])
def test_adjoint_preconditioner_and_solve(fs, name, variant):
    P, ctx, opt, optp = case(name, fs)
    M = BlockPreconditioner(P, variant, opt=opt, opt_p=optp)
    Mt = adjoint.AdjointPreconditioner(M)
    w = np.random.default_rng(9).standard_normal(P.n)
    v = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    ctx.apply_prec_adjoint(variant, cuda(w), v)
    assert_fields(P, v.cpu().numpy(), Mt(w), 1e-10, f"{name} {variant} M^-T w")
    g = np.zeros(P.n)
    g[-P.n_face:] = np.random.default_rng(4).standard_normal(P.n_face)
    lam = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    # M2*^-T leaves the same attainable-accuracy floor near 1e-8 (its p/u
    # blocks are uncorrected); the other two forms must reach tol
    star = variant == "tup_star"
    rc, it, rr = ctx.solve_adjoint(variant, cuda(g), lam, 1e-8, 400, allow_fail=star)
    ref = adjoint.solve_adjoint(P, M, g, 1e-8, 400)
    assert abs(it - ref.iters) <= 1
    assert_fields(P, lam.cpu().numpy(), ref.x, 1e-8, f"{name} {variant} lambda")
    JT = osp.jacobian(P).T.tocsr()
    assert np.linalg.norm(g - JT @ lam.cpu().numpy()) / np.linalg.norm(g) <= (3e-8 if star else 1e-8)


def test_adjoint_matches_dense_on_8cubed(fs):
    P, ctx, _, _ = case("tiny8", fs)
    g = np.zeros(P.n)
    g[-P.n_face:] = np.random.default_rng(1).standard_normal(P.n_face)
    lam_d = adjoint.dense_adjoint(P, g)
    for variant in ("tpu", "tup"):
        lam = torch.zeros(P.n, dtype=torch.float64, device="cuda")
        ctx.solve_adjoint(variant, cuda(g), lam, 1e-12, 400, allow_fail=True)
        assert_fields(P, lam.cpu().numpy(), lam_d, 1e-8, f"tiny8 {variant} lambda vs dense")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autograd_gradient_wrt_rhs(fs, precision):
    from paper_2112_12397_gb300.autograd import frac_solve
    P = fracgen.generate("planes64", N=8, seed=3)
    ctx = fs.context_for(P, fs.default_options(precision=precision, coarse_max=32, coarse_max_p=16))
    b = cuda(P.b).requires_grad_(True)
    p_obs = cuda(np.random.default_rng(5).standard_normal(P.n_face))

    def loss_of(bb, grad=False):
        x = frac_solve(bb, ctx, "tup", 1e-8, 600)
        return 0.5 * ((x[-P.n_face:] - p_obs) ** 2).sum()

    L = loss_of(b)
    L.backward()
    grad = b.grad.detach().cpu().numpy()
    rs = np.random.default_rng(6)
    with torch.no_grad():
        for _ in range(5):
            d = rs.standard_normal(P.n)
            d[:3 * P.n_node][P.dirichlet] = 0.0
            # the loss is quadratic in b, so central differences carry no
            # truncation error; a unit step keeps the solves' 1e-8 residual
            # error far below the 1e-5 tolerance
            h = 1.0
            lp = float(loss_of(b + h * cuda(d)))
            lm = float(loss_of(b - h * cuda(d)))
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grad @ d) <= 1e-5 * abs(grad @ d)
    ctx.close()


# ------------------------------------------------------------------ apertures
def test_aperture_gradient_kernel(fs):
    P = fracgen.generate("planes64", N=8, p_stick=0.4, p_slip=0.3, seed=5)
    ctx = fs.context_for(P, fs.default_options(coarse_max=32, coarse_max_p=16))
    rs = np.random.default_rng(1)
    x, lam = rs.standard_normal(P.n), rs.standard_normal(P.n)
    grad = torch.zeros(P.n_face, dtype=torch.float64, device="cuda")
    ctx.aperture_gradient(fs.device_dk(P), cuda(x), cuda(lam), grad)
    ref = adjoint.aperture_gradient(P, x, lam)
    assert rel(grad.cpu().numpy(), ref) <= 1e-13
    ctx.close()


def test_aperture_gradient_rejects_malformed_entries(fs):
    """Out-of-range rows, columns or components and a decreasing face_ptr
    are reported as FC_BAD_ARG instead of being read."""
    P = fracgen.generate("planes64", N=8, p_stick=0.4, p_slip=0.3, seed=5)
    ctx = fs.context_for(P, fs.default_options(coarse_max=32, coarse_max_p=16))
    rs = np.random.default_rng(1)
    x, lam = cuda(rs.standard_normal(P.n)), cuda(rs.standard_normal(P.n))
    grad = torch.zeros(P.n_face, dtype=torch.float64, device="cuda")
    good = fs.device_dk(P)
    q2 = int(torch.nonzero(good["block"] == 1)[0])
    t = int(torch.nonzero(good["block"] == 0)[0])
    cases = []
    for key, e, v in (("row", t, P.n_face), ("col", t, -1), ("col", q2, P.n_node), ("comp", q2, 3)):
        d = {k: a.clone() for k, a in good.items()}
        d[key][e] = v
        cases.append(d)
    d = {k: a.clone() for k, a in good.items()}
    d["face_ptr"][2], d["face_ptr"][3] = good["face_ptr"][3], good["face_ptr"][2] - 1
    cases.append(d)
    for d in cases:
        with pytest.raises(fs.FcError):
            ctx.aperture_gradient(d, x, lam, grad)
    ctx.aperture_gradient(good, x, lam, grad)
    ref = adjoint.aperture_gradient(P, x.cpu().numpy(), lam.cpu().numpy())
    assert rel(grad.cpu().numpy(), ref) <= 1e-13
    ctx.close()


def test_aperture_gradient_matches_dense_adjoint_8cubed(fs):
    """8^3 case: forward and adjoint solved on the GPU, gradient against the
    oracle's dense adjoint gradient."""
    P = fracgen.generate("tiny8")
    ctx = fs.context_for(P, fs.default_options(coarse_max=64, coarse_max_p=16))
    J = osp.jacobian(P).toarray()
    xs = np.linalg.solve(J, P.b)
    p_obs = xs[-P.n_face:] * 1.1
    g = np.zeros(P.n)
    g[-P.n_face:] = xs[-P.n_face:] - p_obs
    lam_d = np.linalg.solve(J.T, g)
    ref = adjoint.aperture_gradient(P, xs, lam_d)
    x = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    ctx.solve("tup", cuda(P.b), x, 1e-12, 400, allow_fail=True)
    gg = np.zeros(P.n)
    gg[-P.n_face:] = x[-P.n_face:].cpu().numpy() - p_obs
    lam = torch.zeros_like(x)
    ctx.solve_adjoint("tup", cuda(gg), lam, 1e-12, 400, allow_fail=True)
    grad = torch.zeros(P.n_face, dtype=torch.float64, device="cuda")
    ctx.aperture_gradient(fs.device_dk(P), x, lam, grad)
    assert rel(grad.cpu().numpy(), ref) <= 1e-8
    ctx.close()


def test_autograd_aperture_gradient_by_central_differences(fs):
    """Gradient of 0.5 ||p - p_obs||^2 w.r.t. the apertures through
    FracSolveAperture (GPU forward + adjoint + aperture kernel) against
    central differences of dense solves, step 1e-6 relative, 20 directions."""
    from paper_2112_12397_gb300.autograd import ApertureSystem, frac_solve_aperture
    cfg = fracgen.preset("planes64", N=6, p_stick=0.4, p_slip=0.3, seed=11)
    P = fracgen.generate(cfg)
    system = ApertureSystem(cfg, fs.default_options(coarse_max=32, coarse_max_p=16))
    a = cuda(P.aperture).requires_grad_(True)
    b = cuda(P.b).requires_grad_(True)
    p_obs = np.random.default_rng(4).standard_normal(P.n_face) * 10
    x = frac_solve_aperture(a, b, system, "tup", 1e-8, 600)
    L = 0.5 * ((x[-P.n_face:] - cuda(p_obs)) ** 2).sum()
    L.backward()
    grad = a.grad.cpu().numpy()

    def loss(av):
        Pa = fracgen.generate(cfg, aperture=av)
        xx = np.linalg.solve(osp.jacobian(Pa).toarray(), Pa.b)
        return 0.5 * np.sum((xx[-P.n_face:] - p_obs) ** 2)

    rs = np.random.default_rng(7)
    errs = []
    for _ in range(20):
        d = rs.standard_normal(P.n_face) * P.aperture
        h = 1e-6
        fd = (loss(P.aperture + h * d) - loss(P.aperture - h * d)) / (2 * h)
        errs.append(abs(fd - grad @ d) / abs(fd))
    assert max(errs) <= 1e-5, max(errs)
    system.ctx.close()
