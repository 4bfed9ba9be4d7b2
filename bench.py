#!/usr/bin/env python3
"""Benchmark: time to solve the block-preconditioned contact/flow Jacobian to
relative residual 1e-8 on one GB300, FP32-preconditioner (mixed) form against
the all-FP64 form, plus the finest-level smoother's HBM bandwidth.

One step = one system solution as the paper counts it (Sec. 4: "CPU time for
a single system solution"): fc_setup (H~^-1, S1 / S~, fixed-stress S~2, AMG
hierarchies; Alg. 1 / Alg. 3) followed by fc_solve (right-preconditioned
FGMRES-CGS2 with Alg. 2 / Alg. 4 to relative residual 1e-8), on a Jacobian
already resident in HBM.  The e2e figure repeats the step through the public
C-ABI with host buffers: the Jacobian blocks and b are copied from pinned host
memory, the solution is copied back.

Workload (default): 128^3 unit-cube grid, ten seeded fracture rectangles,
60/30/10 stick/slip/open, ~6.7M unknowns; synthetic seeded data standing in
for the paper's private meshes.  Matrices are several GB, far above the
129 MB L2, so no flush is needed between steps.

The bench line's cpu_baseline times the CPU oracle (the tests' reference
implementation) once on a bounded sample, the same workload family at
--cpu-sample-n cells per side (40 by default, about 9 s on one Grace core); --impl
reference times it once per warm-up and timed step at --ref-sample-n cells
per side (32 by default, about 4 s per solve), so that the whole reference
run ends within minutes.  Both are reported as measured, with the sample's
own size.  --cpu-full runs the oracle at the workload's full size instead
(minutes per solve at 128^3; not part of the default run).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve s to rel-res 1e-8 (FP32-AMG vs FP64) at 1 GB300; V-cycle HBM GB/s % peak"
WORKLOADS = {
    "rects128": "unit cube, 10 seeded fracture rectangles (extents 0.2-0.8), 60/30/10 stick/slip/open",
    "planes64": "unit cube, three central fracture planes, 60/30/10 stick/slip/open",
    "network96": "unit cube, fracture planes every 8 cells, 50/40/10 stick/slip/open",
    "tiny8": "unit cube, one fracture plane, all stick",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rects128", choices=sorted(WORKLOADS))
    ap.add_argument("--N", type=int, default=0,
                    help="override the workload's grid size (cells per side; 0: the workload's own)")
    ap.add_argument("--variant", default="tup", choices=["tup", "tpu", "tup_star"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=600)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--variant-steps", type=int, default=1,
                    help="timed solves per preconditioner variant on one shared setup (0: skip)")
    ap.add_argument("--update-steps", type=int, default=1,
                    help="timed fc_update calls per update case (0: skip)")
    ap.add_argument("--other-workloads", type=int, default=1,
                    help="1: after the timed region, measure the other workloads (three planes 64^3 FP64, "
                         "fracture network 96^3 mixed and FP64, the 64^3 adjoint, seeds 0-2 of the bench "
                         "workload) on instances from fc_generate; 0: skip")
    ap.add_argument("--adjoint-steps", type=int, default=1,
                    help="timed adjoint solves + aperture gradients after the timed region (0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-sample-n", type=int, default=40,
                    help="grid size of the cpu_baseline's bounded oracle sample (cells per side)")
    ap.add_argument("--ref-sample-n", type=int, default=32,
                    help="grid size of the reference arm's oracle sample per step (cells per side)")
    ap.add_argument("--cpu-full", action="store_true",
                    help="time the oracle at the workload's full size (long: minutes per solve)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--verbose", type=int, default=0, help="library diagnostics (setup phase times) to stderr")
    ap.add_argument("--mode", default="bench", choices=["bench", "vcycle", "generate"],
                    help="vcycle: fc_setup then two V-cycles of the elasticity hierarchy (profiling case); "
                         "generate: fc_generate of the workload, --steps times (profiling case)")
    return ap.parse_args()


# nominal dense FP64 rate of a GB300 (the FMA pipes, not the tensor cores)
FP64_NOMINAL_TFLOPS = 1.25

# DRAM traffic of the fused Chebyshev step from one ncu capture of the same
# kernel (finest S1 level of the 64^3 three-plane workload, a launch that
# reads the previous direction): dram__bytes_read.sum + dram__bytes_write.sum
# against that launch's algorithmic bytes.  The 128^3 launch is too large to
# capture with the full metric set; its traffic is scaled by the algorithmic
# bytes (blocks and rows grow together).
SMOOTHER_CAPTURE = {"dram_bytes": 329515776 + 3683584, "alg_bytes": 329392804}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import fracgen
from oracle import sparse as osp
from oracle.precond import BlockPreconditioner
from oracle.fgmres import fgmres
P = fracgen.generate({workload!r}, N={n})
J = osp.jacobian(P)
t0 = time.perf_counter()
M = BlockPreconditioner(P, {variant!r})
t1 = time.perf_counter()
r = fgmres(lambda v: J @ v, M, P.b, {tol!r}, {maxit})
t2 = time.perf_counter()
print(json.dumps(dict(n=P.n, setup=t1 - t0, solve=t2 - t1, iters=r.iters, relres=r.relres)))
"""


def run_oracle_sample(workload, n_cells, variant, tol, maxit, timeout=900):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ORACLE_SNIPPET.format(root=ROOT, workload=workload, n=n_cells, variant=variant, tol=tol, maxit=maxit)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=timeout)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


FULL_N = {"rects128": 128, "planes64": 64, "network96": 96, "tiny8": 8}


def oracle_cells(args, sample_n: int) -> int:
    """Cells per side of the oracle's run: the bounded sample, or the full
    workload with --cpu-full (or when the sample is not smaller)."""
    full = args.N or FULL_N[args.workload]
    return full if args.cpu_full else min(sample_n, full)


def cpu_baseline(args):
    n = oracle_cells(args, args.cpu_sample_n)
    s = run_oracle_sample(args.workload, n, args.variant, args.tol, args.maxit,
                          timeout=7200 if args.cpu_full else 900)
    t = s["setup"] + s["solve"]
    full = n == (args.N or FULL_N[args.workload])
    return {"value": t, "unit": "s", "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
            "setup_s": s["setup"], "solve_s": s["solve"], "iters": s["iters"], "relres": s["relres"],
            "unknowns": s["n"], "grid": n,
            "sample": (f"oracle (FP64, one thread) {args.variant} setup+solve measured at {n}^3 "
                       f"({s['n']} unknowns, {s['iters']} iterations)"
                       + ("" if full else ", the bounded sample of the same workload family; not scaled"))}


# ------------------------------------------------------------------ reference arm
def reference(args, rank):
    if rank != 0:
        return
    import fracgen
    fracgen.build()
    n = oracle_cells(args, args.ref_sample_n)
    times, setups, solves = [], [], []
    last = None
    for k in range(args.warmup + args.steps):
        s = run_oracle_sample(args.workload, n, args.variant, args.tol, args.maxit,
                              timeout=7200 if args.cpu_full else 900)
        last = s
        if k >= args.warmup:
            times.append(s["setup"] + s["solve"])
            setups.append(s["setup"])
            solves.append(s["solve"])
    v = statistics.mean(times)
    sample = (f"oracle (FP64, one thread) {args.variant} setup+solve measured at {n}^3 "
              f"({last['n']} unknowns, {last['iters']} iterations) per step; not scaled")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} family at {n}^3", "description": WORKLOADS[args.workload],
                   "grid": n, "unknowns": last["n"], "variant": args.variant, "tol": args.tol},
        "breakdown": {"setup_s": statistics.mean(setups), "solve_s": statistics.mean(solves),
                      "iters": last["iters"], "relres": last["relres"]},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ per-field differences
def field_diffs(a, ref, n_node: int, n_face: int) -> dict:
    """Relative difference of two solutions per field of [u; t; p]
    (||a_f - r_f|| / ||r_f|| and max |a_f - r_f| / max |r_f|): the tractions
    are orders of magnitude larger than the displacements, so one norm of
    the whole vector would describe t alone."""
    import numpy as np
    nu, nt = 3 * n_node, 3 * n_face
    out = {}
    for f, sl in (("u", slice(0, nu)), ("t", slice(nu, nu + nt)), ("p", slice(nu + nt, nu + nt + n_face))):
        d, r = a[sl] - ref[sl], ref[sl]
        if r.size == 0:
            continue
        out[f] = {"rel2": float(np.linalg.norm(d) / max(np.linalg.norm(r), 1e-300)),
                  "relmax": float(np.abs(d).max() / max(np.abs(r).max(), 1e-300)),
                  "norm": float(np.linalg.norm(r))}
    return out


# ------------------------------------------------------------------ other workloads
def perturbed_apertures(aperture, seed: int, n_face: int, scale: float = 0.1, stream: int = 12):
    """a exp(scale Z), Z standard normal by Box-Muller from the generator's
    counter draws 2f, 2f + 1 of `stream` (the adjoint workload's p_obs run)."""
    import numpy as np

    import fracgen
    u1 = np.array([fracgen.uniform(seed, stream, 2 * f) for f in range(n_face)])
    u2 = np.array([fracgen.uniform(seed, stream, 2 * f + 1) for f in range(n_face)])
    return aperture * np.exp(scale * np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2))


def other_workloads(fs, args, stream):
    """The workloads besides the bench's own, each assembled on the device by
    fc_generate (seed 0 unless stated), timed with CUDA events on `stream`
    outside the bench's timed region: setup and solve times, iterations, FP64
    true residuals, and per-field differences of the mixed solution from the
    FP64 one."""
    import torch

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def run(inst, precision, variant, repeat=2):
        ctx = fs.Context(fs.default_options(precision=precision, variants=fs.variant_bit(variant)))
        out = None
        for _ in range(repeat):
            x = torch.zeros_like(inst.b)
            e0, e1, e2 = ev(), ev(), ev()
            e0.record(stream)
            ctx.setup(inst.blocks(), inst.n_node, inst.n_face)
            e1.record(stream)
            rc, it, rr = ctx.solve(variant, inst.b, x, args.tol, args.maxit, allow_fail=True)
            e2.record(stream)
            torch.cuda.synchronize()
            out = {"setup_s": e0.elapsed_time(e1) / 1e3, "solve_s": e1.elapsed_time(e2) / 1e3, "iters": it,
                   "relres": rr}
        return ctx, out, x

    res = {}
    # three central planes, 64^3, FP64, both variants
    inst = fs.generate("planes64")
    res["planes64_fp64"] = {"unknowns": int(inst.n)}
    for v in ("tpu", "tup"):
        ctx, o, _ = run(inst, "fp64", v)
        res["planes64_fp64"][v] = o
        ctx.close()
    # the adjoint workload on the same instance: p_obs from a forward solve
    # with perturbed apertures, then J^T lambda = g, g = p - p_obs
    ctx, o, x = run(inst, "fp64", "tup", repeat=1)
    a = inst.field("aperture").cpu().numpy()
    ia = fs.generate("planes64", aperture=torch.from_numpy(perturbed_apertures(a, 0, inst.n_face)))
    cq, oq, xq = run(ia, "fp64", "tup", repeat=1)
    nf = inst.n_face
    g = torch.zeros_like(inst.b)
    g[-nf:] = x[-nf:] - xq[-nf:]
    lam = torch.zeros_like(inst.b)
    ctx.solve_adjoint("tup", g, lam, args.tol, args.maxit, allow_fail=True)   # builds the J^T data
    e0, e1 = ev(), ev()
    e0.record(stream)
    rc, ita, rra = ctx.solve_adjoint("tup", g, lam, args.tol, args.maxit, allow_fail=True)
    e1.record(stream)
    torch.cuda.synchronize()
    res["adjoint64_fp64"] = {"forward": o, "p_obs_forward_iters": oq["iters"],
                             "adjoint_solve_s": e0.elapsed_time(e1) / 1e3, "adjoint_iters": ita,
                             "adjoint_relres": rra}
    for c in (ctx, cq):
        c.close()
    ia.close()
    inst.close()
    # the fracture network, 96^3, mixed against FP64, both variants
    inst = fs.generate("network96")
    res["network96"] = {"unknowns": int(inst.n), "face_share": 4.0 * inst.n_face / inst.n}
    for v in ("tpu", "tup"):
        r = {}
        xs = {}
        for prec in ("mixed", "fp64"):
            ctx, r[prec], xs[prec] = run(inst, prec, v)
            ctx.close()
        r["mixed_vs_fp64_per_field"] = field_diffs(xs["mixed"].cpu().numpy(), xs["fp64"].cpu().numpy(),
                                                   inst.n_node, inst.n_face)
        res["network96"][v] = r
    inst.close()
    # seeds 0, 1, 2 of the bench workload (mixed, the bench's variant)
    steps = []
    for seed in (0, 1, 2):
        inst = fs.generate(args.workload, seed=seed)
        ctx, o, _ = run(inst, "mixed", args.variant)
        o["seed"], o["unknowns"] = seed, int(inst.n)
        o["step_s"] = o["setup_s"] + o["solve_s"]
        steps.append(o)
        ctx.close()
        inst.close()
    res[f"{args.workload}_seeds"] = {"runs": steps,
                                     "median_step_s": statistics.median([o["step_s"] for o in steps]),
                                     "median_iters": statistics.median([o["iters"] for o in steps])}
    return res


# ------------------------------------------------------------------ ranks
def max_over_ranks(value: float, dist, device: str = "cuda") -> float:
    """The largest value over the ranks (the slowest replica's step time);
    the value itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_env() -> tuple[int, int, int]:
    """RANK, WORLD_SIZE, LOCAL_RANK of a torchrun launch (0, 1, 0 without)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ our arm
def ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import fracgen
    import paper_2112_12397_gb300 as fs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fracgen.build()
    P = fracgen.generate(args.workload, seed=rank, **({"N": args.N} if args.N else {}))
    blocks = fs.device_blocks(P)
    b = torch.from_numpy(P.b).cuda()
    x = torch.zeros_like(b)
    variant_bit = fs.variant_bit(args.variant)

    def make_ctx(prec):
        ctx = fs.Context(fs.default_options(precision=prec, variants=variant_bit, verbose=args.verbose))
        return ctx

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()

    def run_steps(ctx, nsteps, record):
        setup_ms, solve_ms, its, rrs = [], [], [], []
        for _ in range(nsteps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            ctx.setup(blocks, P.n_node, P.n_face)
            e1.record(stream)
            rc, it, rr = ctx.solve(args.variant, b, x, args.tol, args.maxit, allow_fail=True)
            e2.record(stream)
            torch.cuda.synchronize()
            if record:
                setup_ms.append(e0.elapsed_time(e1))
                solve_ms.append(e1.elapsed_time(e2))
                its.append(it)
                rrs.append(rr)
        return setup_ms, solve_ms, its, rrs

    ctx = make_ctx(args.precision)
    run_steps(ctx, args.warmup, False)
    peak, peak_kind = measured_peaks()
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True)
    l0 = fs.launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    setup_ms, solve_ms, its, rrs = run_steps(ctx, args.steps, True)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = fs.launch_count() - l0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    sm_launch, sm_ms, sm_bytes = ctx.kernel_stats(fs.FC_K_SMOOTH0)
    jac = ctx.kernel_stats(fs.FC_K_JAC)
    cgs = ctx.kernel_stats(fs.FC_K_CGS)
    prec = ctx.kernel_stats(fs.FC_K_PREC)
    detail = {}
    for name, k in (("vcycle_u", fs.FC_K_VCYCLE), ("vcycle_p", fs.FC_K_VCYCLE_P), ("resid0", fs.FC_K_RESID0),
                    ("restrict0", fs.FC_K_RESTRICT0), ("prolong0", fs.FC_K_PROLONG0), ("coarse0", fs.FC_K_COARSE0),
                    ("smooth0", fs.FC_K_SMOOTH0), ("jac", fs.FC_K_JAC), ("cgs", fs.FC_K_CGS)):
        n_, ms_, b_ = ctx.kernel_stats(k)
        if n_:
            detail[name] = {"ms_per_launch": ms_ / n_, "launches_per_step": n_ / args.steps,
                            "GBps_alg": (b_ / (ms_ * 1e-3) / 1e9) if (b_ and ms_) else None}
    ctx.profile(False)
    # the FP64-ALU-bound kernels: J z does one FMA per stored scalar of J;
    # a Gram-Schmidt pass against j basis vectors does about (2 j + 1) n,
    # n (k + 2) per pass on average over k iterations
    fp64_peak = FP64_NOMINAL_TFLOPS * 1e3 / 2.0   # GFMA/s
    if "jac" in detail:
        gf = sum(int(t[2].numel()) for t in blocks.values()) / (detail["jac"]["ms_per_launch"] * 1e-3) / 1e9
        detail["jac"].update({"bound": "alu", "GFMA_per_s": gf, "fp64_peak_GFMA_per_s": fp64_peak,
                              "frac_fp64": gf / fp64_peak})
    if "cgs" in detail:
        gf = P.n * (its[-1] + 2) / (detail["cgs"]["ms_per_launch"] * 1e-3) / 1e9
        detail["cgs"].update({"bound": "alu", "GFMA_per_s": gf, "fp64_peak_GFMA_per_s": fp64_peak,
                              "frac_fp64": gf / fp64_peak})
    x_mixed = x.cpu().numpy().copy()

    # max over ranks
    step_ms = max_over_ranks(total_ms / args.steps, dist)

    # end to end through the C-ABI with host buffers: fc_setup_host copies
    # the seven blocks from pinned host memory, fc_solve_host copies b in and
    # x out.  Measured right after the headline steps, with the one context a
    # user's process holds; pinned_h2d_GBps records the host-to-device rate of
    # this run (it varies between runs on these machines).
    e2e = None
    if args.e2e_steps > 0:
        host = {}
        h2d = 0
        for name, t in blocks.items():
            rp, ci, val = (a.cpu().pin_memory() for a in t[:3])
            host[name] = (rp, ci, val) + tuple(t[3:])
            h2d += sum(a.numel() * a.element_size() for a in (rp, ci, val))
        hb = torch.from_numpy(P.b).pin_memory()
        hx = torch.zeros_like(hb).pin_memory()
        h2d += hb.numel() * 8
        d2h = hx.numel() * 8
        times, t_setup = [], []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.setup_host(host, P.n_node, P.n_face)
            t1 = time.perf_counter()
            rc, it, rr = ctx.solve_host(args.variant, hb, hx, args.tol, args.maxit, allow_fail=True)
            torch.cuda.synchronize()
            if k > 0:
                times.append(time.perf_counter() - t0)
                t_setup.append(t1 - t0)
        # the host-to-device bandwidth alone: one pinned copy of A's values
        a_h, a_d = host["A"][2], blocks["A"][2]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a_d.copy_(a_h, non_blocking=True)
        torch.cuda.synchronize()
        h2d_gbs = a_h.numel() * 8 / (time.perf_counter() - t0) / 1e9
        e2e = {"value": statistics.mean(times), "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "api": "fc_setup_host + fc_solve_host",
               "setup_host_s": statistics.mean(t_setup), "pinned_h2d_GBps": h2d_gbs}
        del host

    # FP64 form on the same workload for the FP32-vs-FP64 comparison
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        del ctx
        torch.cuda.empty_cache()
        c64 = make_ctx("fp64")
        run_steps(c64, 1, False)
        s64, v64, i64, r64 = run_steps(c64, args.fp64_steps, True)
        x64 = x.cpu().numpy()
        fp64 = {"setup_s": statistics.mean(s64) / 1e3, "solve_s": statistics.mean(v64) / 1e3,
                "step_s": (statistics.mean(s64) + statistics.mean(v64)) / 1e3, "iters": i64[-1],
                "relres": r64[-1],
                "mixed_vs_fp64_per_field": field_diffs(x_mixed, x64, P.n_node, P.n_face)}
        del c64
        ctx = make_ctx(args.precision)

    # the three preconditioners on one setup (outside the timed region):
    # iterations against time per iteration
    variants = None
    if args.variant_steps > 0:
        del ctx
        torch.cuda.empty_cache()
        cv = fs.Context(fs.default_options(precision=args.precision, variants=3, verbose=args.verbose))
        cv.setup(blocks, P.n_node, P.n_face)
        variants = {}
        for name in ("tpu", "tup", "tup_star"):
            cv.solve(name, b, x, args.tol, args.maxit, allow_fail=True)
            cv.profile(True)
            ts = []
            for _ in range(args.variant_steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rc, it_v, rr_v = cv.solve(name, b, x, args.tol, args.maxit, allow_fail=True)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            pr = cv.kernel_stats(fs.FC_K_PREC)
            cv.profile(False)
            variants[name] = {"solve_s": statistics.mean(ts) / 1e3, "iters": it_v, "relres": rr_v,
                              "prec_apply_ms": pr[1] / max(pr[0], 1)}
        # t-u-p with the geometric fixed stress (Eq. FS) instead of the
        # algebraic one: cell volume 2 h^3 and mean bulk modulus per face
        omega = torch.full((P.n_face,), 2.0 * P.h ** 3, dtype=torch.float64, device="cuda")
        kbar = torch.from_numpy(P.Ebar_face / (3.0 * (1.0 - 2.0 * P.nu))).cuda()
        cv.set_geometric_fs(omega, kbar, P.dt)
        cv.update(blocks, P.n_node, P.n_face)
        cv.solve("tup", b, x, args.tol, args.maxit, allow_fail=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, it_v, rr_v = cv.solve("tup", b, x, args.tol, args.maxit, allow_fail=True)
        e1.record(stream)
        torch.cuda.synchronize()
        variants["tup_geometric_fs"] = {"solve_s": e0.elapsed_time(e1) / 1e3, "iters": it_v, "relres": rr_v}
        del cv
        ctx = make_ctx(args.precision)

    # numeric refresh (fc_update) against a full setup, same patterns: a
    # hydraulic update (T and Q2 change, S1 and its hierarchy do not) and an
    # update of every block (A scaled too, so every hierarchy is rebuilt)
    update = None
    if args.update_steps > 0:
        def scaled(src, factors):
            out = dict(src)
            for name, f in factors.items():
                rp, ci, val = src[name][:3]
                out[name] = (rp, ci, val * f) + tuple(src[name][3:])
            return out
        cases = {"hydraulic_T_Q2": scaled(blocks, {"T": 1.3, "Q2": 0.7}),
                 "all_blocks": scaled(blocks, {"A": 1.1, "T": 1.3, "Q2": 0.7})}
        update = {}
        for name, blk in cases.items():
            ts, its_u = [], None
            for _ in range(args.update_steps):
                ctx.setup(blocks, P.n_node, P.n_face)
                torch.cuda.synchronize()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                ctx.update(blk, P.n_node, P.n_face)
                e1.record(stream)
                rc, its_u, rr_u = ctx.solve(args.variant, b, x, args.tol, args.maxit, allow_fail=True)
                e2.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            update[name] = {"update_s": statistics.mean(ts) / 1e3, "solve_iters_after": its_u,
                            "relres_after": rr_u}
        update["full_setup_s"] = statistics.mean(setup_ms) / 1e3

    # adjoint (the gradient of 0.5 ||p - p_obs||^2 through J^T lambda = g):
    # the transposed solve with the transposed preconditioner, and dJ/da by
    # the aperture-derivative contraction, after one forward solve
    adjoint = None
    if args.adjoint_steps > 0:
        ctx.setup(blocks, P.n_node, P.n_face)
        ctx.solve(args.variant, b, x, args.tol, args.maxit, allow_fail=True)
        g = torch.zeros_like(b)
        pn = P.n_face
        p_obs = torch.from_numpy(np.random.default_rng(12).standard_normal(pn)).cuda()
        g[-pn:] = x[-pn:] - p_obs
        lam = torch.zeros_like(b)
        ctx.solve_adjoint(args.variant, g, lam, args.tol, args.maxit, allow_fail=True)   # builds J^T data
        dk = fs.device_dk(P)
        grad = torch.zeros(pn, dtype=torch.float64, device="cuda")
        ts, tg = [], []
        for _ in range(args.adjoint_steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            rc, it_a, rr_a = ctx.solve_adjoint(args.variant, g, lam, args.tol, args.maxit, allow_fail=True)
            e1.record(stream)
            ctx.aperture_gradient(dk, x, lam, grad)
            e2.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            tg.append(e1.elapsed_time(e2))
        adjoint = {"solve_s": statistics.mean(ts) / 1e3, "iters": it_a, "relres": rr_a,
                   "aperture_gradient_ms": statistics.mean(tg), "dk_entries": int(dk["val"].numel())}


    # the instance assembled on the device by fc_generate (same seed and
    # workload), and a step that starts from the seed: generate + setup +
    # solve with x copied to the host
    generator = None
    if args.e2e_steps > 0 and not args.N:
        gcfg = dict(seed=rank)
        inst = fs.generate(args.workload, **gcfg)
        inst.close()
        gen_ms, seed_s = [], []
        for k in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            inst = fs.generate(args.workload, **gcfg)
            t1 = time.perf_counter()
            ctx.setup(inst.blocks(), inst.n_node, inst.n_face)
            xs = torch.zeros_like(inst.b)
            rc, it_g, rr_g = ctx.solve(args.variant, inst.b, xs, args.tol, args.maxit, allow_fail=True)
            hx.copy_(xs)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if k > 0:
                gen_ms.append((t1 - t0) * 1e3)
                seed_s.append(t2 - t0)
            bytes_out = sum(a.numel() * a.element_size() for v in inst.blocks().values() for a in v[:3])
            same = all(torch.equal(a, b) for v, w in zip(inst.blocks().values(), blocks.values())
                       for a, b in zip(v[:2], w[:2]))
            inst.close()
        generator = {"fc_generate_ms": statistics.mean(gen_ms), "bytes_of_blocks": int(bytes_out),
                     "GBps_written": bytes_out / (statistics.mean(gen_ms) * 1e-3) / 1e9,
                     "patterns_equal_host_generator": bool(same),
                     "e2e_from_seed_s": statistics.mean(seed_s), "iters": it_g, "relres": rr_g}

    others = None
    if args.other_workloads and not args.N:
        del ctx
        torch.cuda.empty_cache()
        others = other_workloads(fs, args, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args)
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": "s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    if rank != 0:
        return
    achieved = sm_bytes / (sm_ms * 1e-3) / 1e9 if sm_ms > 0 else None
    alg_launch = sm_bytes / max(sm_launch, 1)
    traffic = (alg_launch * SMOOTHER_CAPTURE["dram_bytes"] / SMOOTHER_CAPTURE["alg_bytes"]
               if args.precision == "mixed" and sm_launch else None)
    roofline = {"bound": "hbm", "kernel": "fused Chebyshev step, finest level of the S1 hierarchy",
                "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "traffic_source": "ncu capture on the 64^3 three-plane workload, scaled by algorithmic bytes",
                "launches": sm_launch, "avg_launch_ms": sm_ms / max(sm_launch, 1),
                "alg_bytes_per_launch": sm_bytes / max(sm_launch, 1)}
    mean_setup = statistics.mean(setup_ms) / 1e3
    mean_solve = statistics.mean(solve_ms) / 1e3
    out = {
        "metric": METRIC, "value": step_ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "unknowns": P.n,
                   "grid": P.N,
                   "variant": args.variant, "precision": args.precision, "tol": args.tol,
                   "l2": "matrices of several GB, larger than L2; no flush"},
        "breakdown": {"setup_s": mean_setup, "solve_s": mean_solve, "iters": its[-1], "relres": rrs[-1],
                      "prec_apply_ms": prec[1] / max(prec[0], 1), "jac_ms": jac[1] / max(jac[0], 1),
                      "cgs_pass_ms": cgs[1] / max(cgs[0], 1),
                      "smoother_share_of_solve": (sm_ms / (sum(solve_ms))) if solve_ms else None,
                      "kernels": detail},
        "fp64": fp64,
        "variants": variants,
        "update": update,
        "adjoint": adjoint,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "generator": generator,
        "other_workloads": others,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(out))


def vcycle_case(args):
    """Small profiling case: setup, then two V-cycles on the S1 (t-u-p) or
    S~ (t-p-u) hierarchy; the finest level's operator is several hundred MB."""
    import torch

    import fracgen
    import paper_2112_12397_gb300 as fs
    fracgen.build()
    P = fracgen.generate(args.workload)
    ctx = fs.context_for(P, fs.default_options(precision=args.precision, variants=fs.variant_bit(args.variant)))
    hier = fs.FC_H_TPU_U if args.variant == "tpu" else fs.FC_H_TUP_U
    f = torch.randn(3 * P.n_node, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(f)
    for _ in range(2):
        ctx.vcycle(hier, f, x)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "vcycle", "workload": args.workload, "norm": float(x.norm())}))


def generate_case(args):
    """fc_generate of the workload, timed with CUDA events (the instance is
    freed between calls)."""
    import torch

    import paper_2112_12397_gb300 as fs
    fs.load()
    ms = []
    for k in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        inst = fs.generate(args.workload, **({"N": args.N} if args.N else {}))
        e1.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ms.append(e0.elapsed_time(e1))
        n = inst.n
        inst.close()
    print(json.dumps({"mode": "generate", "workload": args.workload, "unknowns": int(n),
                      "ms": statistics.mean(ms) if ms else None}))


def main():
    args = parse()
    if args.mode == "vcycle":
        vcycle_case(args)
        return
    if args.mode == "generate":
        generate_case(args)
        return
    rank, world, local_rank = rank_env()
    if args.impl == "reference":
        reference(args, rank)
    else:
        ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
