"""Oracle solves of the full-size parity tests, run in worker processes.

The CPU oracle needs one to a few minutes per solve at 64^3; the full-size
GPU tests submit these jobs to a process pool (spawn start method, so no
worker inherits a CUDA context) when the module starts, do their GPU work,
and collect the results.  Nothing here touches the CUDA path: every input is
made by the seeded generator from the arguments given.
"""
from __future__ import annotations

import os

# one BLAS thread per worker: several workers run side by side
for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_k, "1")

import time  # noqa: E402

import numpy as np  # noqa: E402


def perturbed_apertures(P, scale: float = 0.1, stream: int = 12) -> np.ndarray:
    """a_f exp(scale Z_f), Z_f standard normal by Box-Muller from the
    generator's counter draws (u1, u2) = U(seed, stream, 2f), U(.., 2f + 1)."""
    import fracgen
    seed = P.cfg.seed
    u1 = np.array([fracgen.uniform(seed, stream, 2 * f) for f in range(P.n_face)])
    u2 = np.array([fracgen.uniform(seed, stream, 2 * f + 1) for f in range(P.n_face)])
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return P.aperture * np.exp(scale * z)


def forward(preset: str, over: dict, variant: str, tol: float, maxit: int, amg: dict | None = None,
            aperture: np.ndarray | None = None) -> dict:
    """FP64 oracle: setup of Alg. 1 / Alg. 3 and right-preconditioned FGMRES
    (Sec. 4) on one seeded instance."""
    import fracgen
    from oracle import sparse as osp
    from oracle.amg import AmgOptions
    from oracle.fgmres import fgmres
    from oracle.precond import BlockPreconditioner
    P = fracgen.generate(preset, aperture=aperture, **over)
    J = osp.jacobian(P)
    amg = amg or {}
    t0 = time.perf_counter()
    M = BlockPreconditioner(P, variant, opt=AmgOptions(**amg.get("u", {})), opt_p=AmgOptions(**amg.get("p", {})))
    t1 = time.perf_counter()
    r = fgmres(lambda v: J @ v, M, P.b, tol, maxit)
    t2 = time.perf_counter()
    return {"iters": r.iters, "x": r.x, "relres": r.relres, "setup_s": t1 - t0, "solve_s": t2 - t1}


def forward_and_adjoint(preset: str, over: dict, variant: str, tol: float, maxit: int) -> dict:
    """The adjoint workload: forward solve, a second forward solve with the
    apertures a exp(0.1 Z) (stream 12) whose pressures are p_obs, then
    J^T lambda = g with g = p - p_obs on the pressure rows (the gradient of
    0.5 ||p - p_obs||^2), by FGMRES with the transposed preconditioner."""
    import fracgen
    from oracle import adjoint
    from oracle import sparse as osp
    from oracle.fgmres import fgmres
    from oracle.precond import BlockPreconditioner
    P = fracgen.generate(preset, **over)
    J = osp.jacobian(P)
    M = BlockPreconditioner(P, variant)
    fw = fgmres(lambda v: J @ v, M, P.b, tol, maxit)
    Q = fracgen.generate(preset, aperture=perturbed_apertures(P), **over)
    JQ = osp.jacobian(Q)
    ob = fgmres(lambda v: JQ @ v, BlockPreconditioner(Q, variant), Q.b, tol, maxit)
    g = np.zeros(P.n)
    g[-P.n_face:] = fw.x[-P.n_face:] - ob.x[-P.n_face:]
    ad = adjoint.solve_adjoint(P, M, g, tol, maxit)
    return {"iters": fw.iters, "x": fw.x, "obs_iters": ob.iters, "p_obs": ob.x[-P.n_face:],
            "adj_iters": ad.iters, "lam": ad.x, "g": g}
