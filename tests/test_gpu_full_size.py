"""Full-size parity: the CUDA path at the sizes of the measured workloads
against the CPU oracle, field by field.

* Three central planes at 64^3 (911,640 unknowns), FP64, both variants:
  iterations within +-1 of the oracle's FGMRES and every field of x within
  1e-8 of the oracle's solution.
* The adjoint workload on the same instance: forward solve, p_obs from a
  forward solve with the apertures a exp(0.1 Z), adjoint of
  0.5 ||p - p_obs||^2 by FGMRES on J^T; each side runs the whole chain on
  its own, and lambda is compared field by field (1e-8), iterations +-1.
* The fracture network (planes every 8 cells on all axes, 23% face
  unknowns) at 48^3 (610,632 unknowns), the largest size the oracle solves
  in about a minute: FP64 both variants against the oracle as above; the
  mixed form to FP64 true residual 1e-8 with at most 15% more iterations,
  its per-field error against the oracle's FP64 solution stated and bounded.

The oracle solves run in a spawn process pool while the GPU works.
"""
import multiprocessing as mp
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

import fracgen
from oracle import sparse as osp

import oracle_jobs
from fields import assert_fields, field_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, MAXIT = 1e-8, 600
NET = ("network96", dict(N=48))


@pytest.fixture(scope="module")
def fs():
    import paper_2112_12397_gb300 as m
    m.load(build_if_missing=True)
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def oracle():
    """Every oracle job of this module, submitted at once."""
    ex = ProcessPoolExecutor(max_workers=5, mp_context=mp.get_context("spawn"))
    jobs = {
        ("planes64", "tpu"): ex.submit(oracle_jobs.forward, "planes64", {}, "tpu", TOL, MAXIT),
        ("planes64", "adjoint"): ex.submit(oracle_jobs.forward_and_adjoint, "planes64", {}, "tup", TOL, MAXIT),
        ("network48", "tpu"): ex.submit(oracle_jobs.forward, NET[0], NET[1], "tpu", TOL, MAXIT),
        ("network48", "tup"): ex.submit(oracle_jobs.forward, NET[0], NET[1], "tup", TOL, MAXIT),
    }
    yield lambda key: jobs[key].result(timeout=1800)
    ex.shutdown(wait=True, cancel_futures=True)


def cuda(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def solve(ctx, variant, P, b=None):
    b = cuda(P.b if b is None else b)
    x = torch.zeros_like(b)
    rc, it, rr = ctx.solve(variant, b, x, TOL, MAXIT)
    return it, rr, x.cpu().numpy()


def true_relres(J, b, x):
    return float(np.linalg.norm(b - J @ x) / np.linalg.norm(b))


@pytest.mark.parametrize("variant", ["tpu", "tup"])
def test_planes64_fp64_against_oracle(fs, oracle, variant):
    P = fracgen.generate("planes64")
    ctx = fs.context_for(P, fs.default_options(variants=fs.variant_bit(variant)))
    it, rr, x = solve(ctx, variant, P)
    ctx.close()
    ref = oracle(("planes64", "tpu")) if variant == "tpu" else oracle(("planes64", "adjoint"))
    J = osp.jacobian(P)
    assert true_relres(J, P.b, x) <= TOL
    assert abs(it - ref["iters"]) <= 1, (it, ref["iters"])
    e = assert_fields(P, x, ref["x"], 1e-8, f"planes64 {variant} x")
    print(f"planes64 fp64 {variant}: iters {it} (oracle {ref['iters']}) " +
          " ".join(f"{f} {v[0]:.1e}/{v[1]:.1e}" for f, v in e.items()))


def test_planes64_adjoint_against_oracle(fs, oracle):
    """The adjoint workload run through the C-ABI on the GPU and by the
    oracle, each chain on its own inputs from the generator."""
    P = fracgen.generate("planes64")
    ctx = fs.context_for(P, fs.default_options(variants=2))
    it, rr, x = solve(ctx, "tup", P)
    Q = fracgen.generate("planes64", aperture=oracle_jobs.perturbed_apertures(P))
    cq = fs.context_for(Q, fs.default_options(variants=2))
    _, _, xq = solve(cq, "tup", Q)
    cq.close()
    g = np.zeros(P.n)
    g[-P.n_face:] = x[-P.n_face:] - xq[-P.n_face:]
    lam = torch.zeros(P.n, dtype=torch.float64, device="cuda")
    rc, ita, rra = ctx.solve_adjoint("tup", cuda(g), lam, TOL, MAXIT)
    lam = lam.cpu().numpy()
    ctx.close()
    ref = oracle(("planes64", "adjoint"))
    JT = osp.jacobian(P).T.tocsr()
    assert true_relres(JT, g, lam) <= TOL
    assert abs(ita - ref["adj_iters"]) <= 1, (ita, ref["adj_iters"])
    # the two chains' right-hand sides agree to the forward solves' accuracy
    ge = field_errors(P, g, ref["g"])["p"]
    assert ge[0] <= 1e-9, ge
    e = assert_fields(P, lam, ref["lam"], 1e-8, "planes64 adjoint lambda")
    print(f"planes64 adjoint: iters {ita} (oracle {ref['adj_iters']}) g diff {ge[0]:.1e} " +
          " ".join(f"{f} {v[0]:.1e}/{v[1]:.1e}" for f, v in e.items()))


# per-field bound of the mixed form's solution against the FP64 oracle
# solution on the network (measured 1e-13 .. 5e-13): the FP32 preconditioner
# changes the Krylov directions at ~1e-7 relative, which moves the
# minimum-residual solution only to second order (times its ~1e-10 distance
# from the exact solution)
MIXED_FIELD_BOUND = 1e-9


@pytest.mark.parametrize("variant", ["tpu", "tup"])
def test_network48_fp64_and_mixed(fs, oracle, variant):
    P = fracgen.generate(NET[0], **NET[1])
    assert 4 * P.n_face / P.n > 0.2
    J = osp.jacobian(P)
    res = {}
    for prec in ("fp64", "mixed"):
        ctx = fs.context_for(P, fs.default_options(precision=prec, variants=fs.variant_bit(variant)))
        res[prec] = solve(ctx, variant, P)
        ctx.close()
    ref = oracle(("network48", variant))
    it64, _, x64 = res["fp64"]
    itm, _, xm = res["mixed"]
    assert true_relres(J, P.b, x64) <= TOL and true_relres(J, P.b, xm) <= TOL
    assert abs(it64 - ref["iters"]) <= 1, (it64, ref["iters"])
    assert_fields(P, x64, ref["x"], 1e-8, f"network48 fp64 {variant} x")
    assert itm <= 1.15 * it64, (itm, it64)
    e = assert_fields(P, xm, ref["x"], MIXED_FIELD_BOUND, f"network48 mixed {variant} x vs FP64 oracle")
    print(f"network48 {variant}: fp64 iters {it64} (oracle {ref['iters']}), mixed {itm}; mixed vs oracle " +
          " ".join(f"{f} {v[0]:.1e}/{v[1]:.1e}" for f, v in e.items()))
