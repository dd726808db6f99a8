"""Benchmark of the AMG-PCG solve phase (time to FP64 relative residual 1e-8).

One step = one complete PCG solve, preconditioned by one V-cycle, of the
seeded synthetic 3D P1 elasticity system on 64^3 vertices (774,144 dofs,
3x3 blocks) from a zero initial guess to ||r|| <= 1e-8 ||f||: every row of
the solve phase (BSR SpMV, block-l1 smoother, restriction, prolongation,
coarsest solve, V-cycle, PCG) runs inside the timed region; the hierarchy
(setup + device Galerkin products) is built before it.  Inputs live in HBM
when the timed region starts; A_0 alone (280 MB) is larger than L2.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
Multi-GPU (torchrun): independent replicas, one per GPU (the solve phase of
one system does not shard without a halo exchange, which is not built).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

# No thread-count variables are set here: with some OpenBLAS builds (e.g. on
# aarch64) OPENBLAS_NUM_THREADS=1 also pins the process-wide OpenMP thread
# count, which the library's host setup uses.  The CPU oracle's solve phase is
# single-threaded anyway (scipy.sparse products, numpy element-wise ops).

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
WORKLOADS = {
    "cube64": ("3D P1 elasticity, unit cube, 64^3 vertices (Kuhn tetrahedra, +-20% h "
               "perturbation, seed 2), E=1, nu=0.3, clamped x=0, body force (0,0,-1); "
               "774,144 dofs, 3x3 BSR"),
    "square32": ("2D P1 elasticity, unit square, 33x33 vertices (seed 1), E=1, nu=0.3, "
                 "clamped x=0, body force (0,-1); 2,112 dofs, 2x2 BSR"),
    "cube128jump": ("3D P1 elasticity, 128^3 vertices, 200 inclusion boxes E=10^U(-3,3), "
                    "nu U[0.25,0.45] (seed 3); 6.24M dofs"),
    "cube96nu": ("3D P1 elasticity, unit cube, 96^3 vertices (seed 5), E=1, nu per element "
                 "U[0.3,0.45], clamped x=0, body force (0,0,-1); 2.65M dofs; level-0 smoother: the "
                 "learned MLP trained on ten 32^3 meshes (seeds 100-109)"),
    "beam": ("the paper's vector model problem (Sec. 7): 3D P1 elasticity on the beam "
             "[0,10]x[0,1]^2, h=1/32 (321x33x33 vertices, seed 6), mu=1, lambda=0, clamped x=0, "
             "body force (0,0,-1); 1.05M dofs"),
    "jump11": ("the paper's difficult vector problem (Sec. 7): unit cube, 67^3 vertices (seed 7), "
               "mu=lambda=1e4 in the eleven diagonal boxes [(i-1)/11,i/11]^3, 1 elsewhere, clamped "
               "x=0, body force (0,0,-1); 888,822 dofs; 4 matching passes first, 3 later"),
    "poisson": ("the paper's scalar model problem (Sec. 7): -Laplace u = 1 on the unit cube, "
                "128^3 vertices (seed 8), u = 0 on the boundary; 2,000,376 unknowns, 1x1 blocks; "
                "mu_s alone, 4 / 3 matching passes, row caps 4, coarse size min(1600, n/1250)"),
    "batch64": ("64 independent 3D P1 elasticity boxes, vertices per axis U{16..48}, h=1/32, "
                "E U[0.1,10], nu U[0.2,0.4] per system (seed 4), clamped x=0, 6 load cases "
                "(unit body forces +-x, +-y, +-z) each"),
}
PREC_NAMES = {0: "fp64", 1: "fp32_vcycle", 2: "bf16_storage", 3: "bf16_coarse"}


def make_workload(name):
    from workloads import configs
    if name == "cube64":
        return configs.cube64()
    if name == "square32":
        return configs.square32()
    if name == "cube128jump":
        return configs.cube128jump()
    if name == "cube96nu":
        return configs.cube96nu()
    if name == "beam":
        return configs.beam()
    if name == "jump11":
        return configs.jump11()
    if name == "poisson":
        return configs.poisson()
    raise SystemExit(f"unknown workload {name}")


def setup_params(name, problem=None):
    """amg_setup parameters the paper gives for this workload (Sec. 7)."""
    from workloads import configs
    prm = dict(configs.SETUP.get(name, {}))
    if problem is not None and configs.coarse_size(name, problem.n_free):
        prm["coarse_max"] = configs.coarse_size(name, problem.n_free)
    return prm


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes_per_iteration(levels, prec, nr=1, gs=False):
    """Bytes one PCG iteration must move at least once (matrices, smoother
    blocks, vectors), from the actual level sizes; with nr load cases solved
    together the operators are read once and the vectors nr times.  gs: the
    hybrid Gauss-Seidel V-cycle, whose pre-smoothing is a full sweep (A_l read
    three times per level instead of twice)."""
    # matrix value bytes per level (BF16 coarse: FP32 on level 0, BF16 below)
    wl = lambda l: {0: 8, 1: 4, 2: 2, 3: 4 if l == 0 else 2}[prec]
    wv = 8 if prec == 0 else 4            # V-cycle vector / smoother bytes
    n0, k0 = levels[0]["n_rows"], levels[0]["block"]
    N0 = n0 * k0
    A0 = levels[0]["nnzb"] * (k0 * k0 * 8 + 4) + 4 * (n0 + 1)
    mat = A0
    vec = N0 * 8 * 2                                   # q = A p (p read, q written)
    vec += N0 * 8 * 2 + N0 * 8 * 3 + N0 * 8 * 6        # dots and updates
    for l, L in enumerate(levels):
        n, k = L["n_rows"], L["block"]
        N = n * k
        if l == len(levels) - 1:
            mat += (N * N) * 8
            vec += 2 * N * wv
            continue
        w = wl(l)
        Ab = L["nnzb"] * (k * k * w + 4) + 4 * (n + 1)
        kc = levels[l + 1]["block"]
        Pb = L["nnzb_P"] * (k * kc * w + 4) + 4 * (n + 1)
        Rb = L["nnzb_P"] * (k * kc * w + 4) + 4 * (levels[l + 1]["n_rows"] + 1)
        Mb = n * k * k * wv
        Nc = levels[l + 1]["n_rows"] * kc
        mat += 2 * Mb + (3 if gs else 2) * Ab + Rb + Pb
        vec += (3 if gs else 2) * N * wv + 3 * N * wv   # pre-smoothing ; t = b - A x
        vec += N * wv + Nc * wv + Nc * wv + 2 * N * wv   # restriction, prolongation
        vec += 3 * N * wv                           # y = x + M(b - A x)
    if prec:
        vec += N0 * (8 + 4) * 2
    return mat + nr * vec


def spmv_bytes(L):
    n, k = L["n_rows"], L["block"]
    return L["nnzb"] * (k * k * 8 + 4) + 4 * (n + 1) + 2 * n * k * 8


def traffic_record(kernel):
    """dram bytes per launch of `kernel` from the committed ncu summary
    (profiles/ncu_traffic.json, one record per kernel), if the kernel's
    source has not changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        recs = json.load(f)
    if isinstance(recs, dict):
        recs = [recs]
    for rec in recs:
        if rec.get("kernel_name") != kernel:
            continue
        src = os.path.join(ROOT, rec["source"])
        if os.path.exists(src) and rec.get("kernel_source_sha1") == kernel_source_sha1(
                src, kernel.split("<")[0]):
            return rec
    return None


def scaled_traffic(rec, algorithmic_bytes):
    """DRAM bytes per launch of the dominant kernel on this workload.  The
    record holds one capture; on another workload the launch reads each
    block and block row once as well, so its traffic grows with the
    algorithmic bytes: the captured traffic is scaled by their ratio.
    Returns (bytes, how it was obtained), or (None, None) without a record."""
    if not rec:
        return None, None
    ref = rec["algorithmic_bytes_per_launch"]
    if int(algorithmic_bytes) == int(ref):
        return int(rec["bytes_per_launch"]), f"ncu capture ({rec.get('workload', 'same workload')})"
    t = int(round(rec["bytes_per_launch"] * algorithmic_bytes / ref))
    return t, (f"scaled from the {rec.get('workload', 'recorded')} ncu capture by algorithmic "
               f"bytes ({int(algorithmic_bytes)} / {ref})")


def kernel_source_sha1(path, name):
    """SHA-1 of the source text of the __global__ function `name` (from the
    template line before its definition to its closing brace): the traffic
    record stays valid while that kernel is unchanged."""
    import hashlib
    import re
    text = open(path).read()
    m = re.search(r"__global__[^;{]*?\b" + re.escape(name) + r"\(", text)
    if m is None:
        raise ValueError(f"no __global__ {name} in {path}")
    i = m.end()
    start = text.rindex("template <", 0, i)
    end = text.index("\n}\n", i) + 3
    return hashlib.sha1(text[start:end].encode()).hexdigest()


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------


def max_over_ranks(value, ws, device):
    """The largest of every rank's value (the timing of a multi-replica run is
    that of its slowest replica); the value itself for one rank."""
    if ws <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cube128jump", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2, 3],
                    help="V-cycle precision of the timed path: 0 fp64, 1 fp32 (default), 2 bf16 "
                         "storage, 3 bf16 storage on the levels below 0; the CG is FP64 in all")
    ap.add_argument("--cg-operator", default="auto", choices=["auto", "double_float", "fp64"],
                    help="arithmetic of the CG operator q = A_0 p: auto (default: double-float "
                         "pairs on the FP32 pipe with the FP32 / BF16 V-cycles, FP64 with the "
                         "FP64 V-cycle), double_float, fp64")
    ap.add_argument("--variants", default="auto",
                    help="comma list of other precisions timed for comparison ('auto': the two "
                         "others, '': none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the oracle's tight solve (energy-norm errors); for profiling")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--pcg-mode", default="graph", choices=["graph", "host"],
                    help="graph: whole PCG in one CUDA graph (default); host: the same kernels "
                         "launched one by one (per-kernel view for profilers)")
    ap.add_argument("--smoother", default="auto", choices=["auto", "l1", "gs", "learned"],
                    help="smoother of the timed solve: l1 block-l1 Jacobi, gs block-l1 hybrid "
                         "Gauss-Seidel (colour classes), learned (level 0; cube96nu); auto: "
                         "learned for cube96nu, block-l1 Jacobi otherwise")
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--systems", type=int, default=64,
                    help="batch64: number of systems (the workload has 64)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.smoother == "auto":
        args.smoother = "learned" if args.workload == "cube96nu" else "l1"
    if args.workload == "batch64":
        # the 64 meshes are generated in a spawn pool before any CUDA call
        problems = batch_problems(args.systems)
    train_problems = None
    if args.smoother == "learned" and args.impl != "reference":
        train_problems = training_problems()

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.impl == "reference":
        if args.workload == "batch64":
            return run_reference_batch(args, ws, rank, local, problems)
        return run_reference(args, ws, rank, local)
    if args.workload == "batch64":
        return run_batch(args, ws, rank, local, problems)
    return run_single(args, ws, rank, local, train_problems)


def operator_complexity(levels):
    """Sec. 7's operator complexity: nonzero entries of the matrices of all
    levels over those of the finest (blocks hold k^2 entries), and the same
    ratio counted in blocks."""
    ent = [L["nnzb"] * L["block"] ** 2 for L in levels]
    blk = [L["nnzb"] for L in levels]
    return {"entries": round(sum(ent) / ent[0], 3), "blocks": round(sum(blk) / blk[0], 3),
            "vertex": round(sum(L["n_rows"] for L in levels) / levels[0]["n_rows"], 3)}


def run_single(args, ws, rank, local, train_problems):
    import torch
    from paper_2011_13325_gb300 import amg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # one non-default stream for the library and for torch's own ops (graph
    # capture is not allowed on the legacy default stream)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    cg_mode = {"auto": amg.AMG_CG_AUTO, "double_float": amg.AMG_CG_DOUBLE_FLOAT,
               "fp64": amg.AMG_CG_FP64}[args.cg_operator]

    t0 = time.perf_counter()
    problem = make_workload(args.workload)
    gen_s = time.perf_counter() - t0

    ctx = amg.Context(local, stream.cuda_stream)
    ctx.set_pcg_graph(args.pcg_mode == "graph")
    ctx.set_cg_operator(cg_mode)
    t0 = time.perf_counter()
    main_sm = amg.AMG_SMOOTHER_HYBRID_GS if args.smoother == "gs" else amg.AMG_SMOOTHER_L1_JACOBI
    ctx.setup(problem, args.precision, main_sm, **setup_params(args.workload, problem))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    setup_parts = {k: round(v, 2) for k, v in ctx.setup_times().items()}
    levels = [ctx.level_info(l) for l in range(ctx.n_levels)]
    learned_info = None
    if args.smoother == "learned":
        net, learned_info = train_learned(amg, train_problems, local, epochs=args.train_epochs)
        t0 = time.perf_counter()
        lam, w = ctx.set_learned_smoother(net, problem.coords[problem.free])
        learned_info.update(lambda_lanczos=lam, omega=w,
                            install_s=round(time.perf_counter() - t0, 3))
    f = torch.from_numpy(np.ascontiguousarray(problem.b[0])).to(dev)
    u = torch.zeros_like(f)

    def run_steps(c, k, record):
        times, its = [], []
        for _ in range(k):
            u.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, it, rr = c.pcg_solve(f, u, rtol=args.rtol, maxit=1000)
            e1.record(stream)
            if record:
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                its.append(it[0])
        return times, its

    run_steps(ctx, args.warmup, False)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.15)
    t_wall = time.perf_counter()
    times, its = run_steps(ctx, args.steps, True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    if ws > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(float(np.mean(times)), ws, dev)
    u_main = u.cpu().numpy()

    # final FP64 true residual (computed on the device by the library)
    res = torch.zeros_like(f)
    ctx.residual(0, f, u, res)
    true_rel = float(torch.linalg.norm(res) / torch.linalg.norm(f))
    P_list = [ctx.download_prolongation(l) for l in range(ctx.n_levels - 1)]

    def upload(prec, cg, smoother=None):
        smoother = main_sm if smoother is None else smoother
        c2 = amg.Context(local, stream.cuda_stream)
        c2.set_pcg_graph(args.pcg_mode == "graph")
        c2.set_cg_operator(cg)
        Ps = [type("P", (), dict(n_rows=n, n_cols=m, rowptr=rp, colidx=ci, vals=v))
              for (n, m, rp, ci, v) in P_list]
        c2.upload_hierarchy(problem.A, Ps, prec, smoother)
        return c2

    solutions = {}

    def variant(c2, name, base=None):
        # a variant that does not reach rtol in 1000 iterations is reported
        # as such (the BF16-storage V-cycle can lose definiteness on A_0)
        try:
            run_steps(c2, args.warmup, False)
            tv, iv = run_steps(c2, args.steps, True)
        except amg.AmgError as e:
            return {"converged": False, "error": str(e)[:120]}
        c2.residual(0, f, u, res)
        solutions[name] = u.cpu().numpy()
        out = {"ms": round(float(np.mean(tv)), 3), "iters": float(np.mean(iv)),
               "true_relres": float(torch.linalg.norm(res) / torch.linalg.norm(f)),
               "ms_ratio_to_main": round(float(np.mean(tv)) / ms, 3)}
        if base is not None:
            out["solve_gbs"] = round(algorithmic_bytes_per_iteration(levels, base, gs=(name == "hybrid_gs" or (name != "l1_jacobi" and args.smoother == "gs"))) * float(np.mean(iv)) /
                                     (float(np.mean(tv)) * 1e-3) / 1e9, 1)
        return out

    # the plain FP64 method: FP64 V-cycle and FP64 CG operator (the comparator
    # of the mixed-precision, batched and learned forms)
    variants = {}
    c2 = upload(amg.AMG_PREC_FP64, amg.AMG_CG_FP64)
    plain = variant(c2, "plain_fp64", 0)
    c2.close()
    if args.variants == "auto":
        vlist = [] if args.smoother == "learned" else [p for p in (1, 2, 3) if p != args.precision]
    else:
        vlist = [int(v) for v in args.variants.split(",") if v.strip()]
    for prec in vlist:
        c2 = upload(prec, cg_mode)
        variants[PREC_NAMES[prec]] = variant(c2, PREC_NAMES[prec], prec)
        c2.close()
    # the other smoother of Sec. 7's block-l1 family (hybrid Gauss-Seidel with
    # colour classes, or block-l1 Jacobi), same hierarchy, precision and CG
    # operator
    if args.smoother in ("l1", "gs") and args.variants == "auto":
        other_sm = amg.AMG_SMOOTHER_L1_JACOBI if args.smoother == "gs" else amg.AMG_SMOOTHER_HYBRID_GS
        name = "l1_jacobi" if args.smoother == "gs" else "hybrid_gs"
        c2 = upload(args.precision, cg_mode, other_sm)
        variants[name] = variant(c2, name, args.precision)
        c2.close()
    # the timed configuration with the other CG operator arithmetic
    main_df = "pcg_spmv_dot_sell_df_kernel" in ctx.describe()
    other = amg.AMG_CG_FP64 if main_df else amg.AMG_CG_DOUBLE_FLOAT
    ctx.set_cg_operator(other)
    variants["cg_operator_" + ("fp64" if other == amg.AMG_CG_FP64 else "double_float")] = \
        variant(ctx, "other_cg_operator")
    ctx.set_cg_operator(cg_mode)
    # the same solve with plain launches (no programmatic dependent launch)
    ctx.set_launch_overlap(False)
    run_steps(ctx, args.warmup, False)
    tv, iv = run_steps(ctx, args.steps, True)
    ctx.set_launch_overlap(True)
    variants["no_launch_overlap"] = {"ms": round(float(np.mean(tv)), 3), "iters": float(np.mean(iv)),
                                     "ms_ratio_to_main": round(float(np.mean(tv)) / ms, 3)}

    # end-to-end through the host entry point (H2D f, u0; D2H u inside)
    fh = torch.from_numpy(np.ascontiguousarray(problem.b[0])).pin_memory()
    uh = torch.zeros_like(fh).pin_memory()
    for _ in range(2):
        uh.zero_()
        ctx.pcg_solve_host(fh, uh, rtol=args.rtol, maxit=1000)
    et = []
    for _ in range(args.steps):
        uh.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.pcg_solve_host(fh, uh, rtol=args.rtol, maxit=1000)
        e1.record(stream)
        e1.synchronize()
        et.append(e0.elapsed_time(e1))
    n_dof = int(f.numel())

    fine_smoother = ctx.download_smoother(0) if args.smoother == "learned" else None
    if args.smoother == "learned":
        # the method's own block-l1 Jacobi on the same hierarchy and precision
        ctx.reset_smoother()
        variants["l1_jacobi"] = variant(ctx, "l1_jacobi")

    # dominant kernel of the solve: the CG operator q = A_0 p (per-launch
    # time by CUDA events on the library's stream), and every CG step
    pk, pk_kind = peaks()
    pcg_prof = ctx.profile_pcg(reps=20)
    pcg_kernels = []
    for step, us_k, by in pcg_prof:
        gbs_k = by / (us_k * 1e-6) / 1e9
        pcg_kernels.append({"step": step, "us": round(us_k, 2), "mbytes": round(by / 1e6, 2),
                            "gbs": round(gbs_k, 1), "frac_hbm": round(gbs_k / pk["hbm_gbs"], 3)})
    _, op_us, op_bytes = pcg_prof[2]
    achieved = op_bytes / (op_us * 1e-6) / 1e9
    df_used = "pcg_spmv_dot_sell_df_kernel" in ctx.describe()
    kb = levels[0]["block"]
    kname = (f"pcg_spmv_dot_sell_df_kernel<{kb}>" if df_used else f"pcg_spmv_dot_sell_kernel<{kb}>")
    traffic, traffic_kind = scaled_traffic(traffic_record(kname), op_bytes)
    fp64_gflops, fp32_gflops = ctx.probe_fma_rate()
    k_flops = 2.0 * levels[0]["nnzb"] * levels[0]["block"] ** 2
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / pk["hbm_gbs"], 3), "traffic": traffic,
                "traffic_kind": traffic_kind,
                "kernel": f"{kname} q = A_0 p with p.q partials (CG operator, "
                          f"{'double-float' if df_used else 'FP64'} arithmetic)",
                "bytes_per_launch": int(op_bytes), "us_per_launch": round(op_us, 2),
                "peak_kind": f"{pk_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "flops_per_launch": int(k_flops),
                "tflops": round(k_flops / (op_us * 1e-6) / 1e12, 3),
                "fp64_fma_peak_tflops": round(fp64_gflops / 1e3, 3),
                "fp32_fma_peak_tflops": round(fp32_gflops / 1e3, 1)}

    it_mean = float(np.mean(its))
    per_it_bytes = algorithmic_bytes_per_iteration(levels, args.precision, gs=args.smoother == "gs")
    solve_gbs = per_it_bytes * it_mean / (ms * 1e-3) / 1e9
    per_it, fixed = ctx.pcg_launches()
    launches = fixed + int(round(it_mean)) * per_it

    # the CPU oracle: its own solve phase on the same prolongations (C, all
    # host cores), its own iteration count to rtol, the energy-norm errors of
    # every GPU solution against its tight solve, and its timing
    cpu, accuracy = None, None
    if rank == 0 and ws == 1 and not (args.no_cpu_baseline and args.no_accuracy):
        cpu, accuracy = oracle_leg(problem, P_list, fine_smoother, args, u_main, solutions,
                                   int(round(it_mean)), skip_timing=args.no_cpu_baseline,
                                   skip_accuracy=args.no_accuracy)

    line = {
        "metric": "AMG-PCG time-to-1e-8 (FP64 residual), " + ("3D Poisson" if problem.k == 1 else
                                                                "3D elasticity"),
        "value": round(ms, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f64", 1: "f64 CG + f32 V-cycle", 2: "f64 CG + f32 V-cycle (bf16 storage)",
                  3: "f64 CG + f32 V-cycle (bf16 storage below level 0)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                   "precision": PREC_NAMES[args.precision] + " V-cycle, fp64 CG (FP64 residual 1e-8)",
                   "cg_operator": args.cg_operator,
                   "rtol": args.rtol,
                   "pcg_mode": args.pcg_mode,
                   "levels": [L["n_rows"] for L in levels],
                   "nnzb": [L["nnzb"] for L in levels],
                   "l2": f"inputs larger than L2 (A_0 values {levels[0]['nnzb'] * levels[0]['block'] ** 2 * 8 / 1e6:.0f} MB)",
                   "parallelism": f"replicas x{ws}"},
        "plain_fp64": None if plain is None else dict(plain, speedup_of_main=round(plain["ms"] / ms, 3),
                                                      what="FP64 V-cycle and FP64 CG operator"),
        "iters": it_mean, "true_relres": true_rel, "accuracy": accuracy,
        "operator_complexity": operator_complexity(levels),
        "setup_s": round(setup_s, 2), "setup_parts": setup_parts,
        "generate_s": round(gen_s, 2), "solve_gbs": round(solve_gbs, 1),
        "bytes_per_iteration": int(per_it_bytes), "solves_per_s": round(ws * 1e3 / ms, 2),
        "wall_s_timed": round(wall, 3),
        "roofline": roofline, "clocks": clocks, "variants": variants,
        "e2e": {"value": round(float(np.mean(et)), 3), "unit": "ms",
                "h2d_bytes_per_step": 2 * n_dof * 8, "d2h_bytes_per_step": n_dof * 8},
        "gpu_launches": launches * args.steps, "gpu_launches_per_step": launches,
        "cpu_baseline": cpu,
    }
    line["pcg_kernels"] = pcg_kernels
    line["kernels"] = [ln for ln in ctx.describe().splitlines()]
    # every V-cycle kernel: live time per launch vs its algorithmic bytes
    kr = []
    for lev, step, us_k, by in ctx.profile_vcycle(reps=20):
        gbs_k = by / (us_k * 1e-6) / 1e9 if us_k > 0 else 0.0
        kr.append({"level": lev, "step": step, "us": round(us_k, 2), "mbytes": round(by / 1e6, 2),
                   "gbs": round(gbs_k, 1), "frac_hbm": round(gbs_k / pk["hbm_gbs"], 3)})
    line["vcycle_kernels"] = kr
    line["config"]["smoother"] = {"l1": "block-l1 Jacobi",
                                  "gs": "block-l1 hybrid Gauss-Seidel (colour classes)"}.get(args.smoother)
    if learned_info is not None:
        line["config"]["smoother"] = "learned MLP (level 0), block-l1 Jacobi below"
        line["learned"] = learned_info
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def oracle_leg(problem, P_list, fine_smoother, args, u_main, solutions, gpu_iters,
               skip_timing=False, skip_accuracy=False, single_budget_s=20.0):
    """The CPU oracle on this machine's host cores, on the same prolongations
    and with the timed solve's smoother (block-l1 Jacobi, hybrid Gauss-Seidel,
    or the learned level-0 blocks over block-l1 Jacobi): its C solve phase
    (oracle/csolve.c) builds its own coarse matrices and solves to rtol with
    all cores (timed, its own iteration count); one core runs a bounded
    sample of iterations (scaled to that count); the energy-norm error
    ||u - u_o||_A / ||u_o||_A of every GPU solution is taken against the
    oracle's continuation of its solve to 1e-12."""
    from oracle import csolve, solve
    t0 = time.perf_counter()
    A0 = solve.mat_from(problem.A)
    Ps = [solve.Mat(n, m, rp.astype(np.int64), ci.astype(np.int64), v) for (n, m, rp, ci, v) in P_list]
    smoother = oracle_smoother(args)
    try:
        H = csolve.Hierarchy(A0, Ps, smoother=smoother)
    except np.linalg.LinAlgError as e:
        why = f"oracle coarsest Cholesky failed on this hierarchy: {e}"
        return ({"value": None, "unit": "ms", "cores": 0, "kind": "oracle", "unavailable": why},
                {"unavailable": why})
    if fine_smoother is not None:
        H.Minv[0] = np.ascontiguousarray(fine_smoother)
        H._pack()
    prep_s = time.perf_counter() - t0
    f = problem.b[0]
    cores = csolve.max_threads()
    t0 = time.perf_counter()
    u_o, it_o, hist = H.pcg(f, rtol=args.rtol, maxit=1000)
    all_ms = (time.perf_counter() - t0) * 1e3
    cpu = None
    if not skip_timing:
        csolve.set_threads(1)
        try:
            t0 = time.perf_counter()
            H.pcg(f, rtol=0.0, maxit=1)
            t1 = time.perf_counter() - t0
            m = int(max(1, min(it_o, single_budget_s / max(t1, 1e-6))))
            t0 = time.perf_counter()
            H.pcg(f, rtol=0.0, maxit=m)
            dt = time.perf_counter() - t0
        finally:
            csolve.set_threads(cores)
        cpu = {"value": round(all_ms, 1), "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": (f"the oracle's FP64 PCG (C solve phase, oracle/csolve.c, {smoother} "
                          f"smoother) on the same "
                          f"prolongations, run to its own rtol {args.rtol:g} ({it_o} iterations, "
                          f"GPU {gpu_iters}) on {cores} host threads, timed whole; coarse matrices, "
                          f"smoother blocks and factor built beforehand in {prep_s:.1f} s"),
               "iters": it_o,
               "single_thread": {"value": round(dt / m * it_o * 1e3, 1), "unit": "ms", "cores": 1,
                                 "sample": f"{m} iterations ({dt:.1f} s) on 1 thread, scaled to "
                                           f"{it_o} iterations"}}
    accuracy = None
    if not skip_accuracy:
        ue, it_e, hist_e = H.pcg(f, rtol=1e-12, maxit=2000, x0=u_o)
        Aue = csolve.spmv(A0, ue)
        unorm = float(np.sqrt(ue @ Aue))

        def energy(u):
            e = u - ue
            return float(np.sqrt(max(e @ csolve.spmv(A0, e), 0.0)) / unorm)
        accuracy = {"energy_error": energy(u_main),
                    "variants": {k: energy(v) for k, v in solutions.items()},
                    "oracle_1e8": energy(u_o),
                    "reference": (f"the oracle's own solve (C solve phase, same prolongations) "
                                  f"continued to rtol 1e-12 ({it_o} + {it_e} iterations, relres "
                                  f"{hist_e[-1]:.1e})")}
    return cpu, accuracy


def oracle_smoother(args):
    """The oracle's smoother for the timed solve's --smoother (the learned
    smoother's blocks replace level 0's block-l1 Jacobi blocks)."""
    return "hybrid_gs" if getattr(args, "smoother", "l1") == "gs" else "l1_jacobi"


def run_reference(args, ws, rank, local):
    """The CPU oracle on this machine's host cores, on the same workload:
    the prolongations come from the library's setup (Algorithm 1 and the
    smoothed prolongation on the host; the oracle's own Python setup would
    take hours on 2M vertices), everything after them is the oracle's (C
    solve phase): coarse matrices, smoothers, coarsest factor, PCG with its
    own iteration count; each step a bounded sample of its iterations."""
    import torch
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    from oracle import csolve, solve
    from paper_2011_13325_gb300 import amg
    problem = make_workload(args.workload)
    ctx = amg.Context(local)
    ctx.setup(problem, amg.AMG_PREC_FP64, **setup_params(args.workload, problem))
    P_list = [ctx.download_prolongation(l) for l in range(ctx.n_levels - 1)]
    ctx.close()
    A0 = solve.mat_from(problem.A)
    Ps = [solve.Mat(n, m, rp.astype(np.int64), ci.astype(np.int64), v) for (n, m, rp, ci, v) in P_list]
    smoother = oracle_smoother(args)
    H = csolve.Hierarchy(A0, Ps, smoother=smoother)
    f = problem.b[0]
    cores = csolve.max_threads()
    t0 = time.perf_counter()
    _, it_o, _ = H.pcg(f, rtol=args.rtol, maxit=1000)
    full_s = time.perf_counter() - t0
    budget = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    m = int(max(1, min(it_o, budget / max(full_s / max(it_o, 1), 1e-6))))
    per_step = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        H.pcg(f, rtol=0.0, maxit=m)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            per_step.append(dt / m * it_o * 1e3)
    v = float(np.mean(per_step))
    line = {"impl": "reference", "metric": "AMG-PCG time-to-1e-8 (FP64 residual), 3D elasticity",
            "value": round(v, 1), "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                       "smoother": {"hybrid_gs": "block-l1 hybrid Gauss-Seidel (colour classes)",
                                    "l1_jacobi": "block-l1 Jacobi"}[smoother]},
            "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": (f"each step: {m} iterations of the oracle's FP64 PCG (C solve "
                                        f"phase, {smoother} smoother, on {cores} threads) scaled to "
                                        f"its own {it_o} iterations "
                                        f"to rtol {args.rtol:g} (one full solve: {full_s:.1f} s)")},
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# learned smoother: training on the library's own patch-inverse targets
# ---------------------------------------------------------------------------

def _train_problem(seed):
    from workloads import configs
    return configs.training_meshes(seeds=[seed])[0]


def training_problems():
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(10) as pool:
        return pool.map(_train_problem, list(range(100, 110)), chunksize=1)


def train_learned(amg, problems, local, epochs=40, batch=1024, lr=2e-3):
    """Features and FP64 patch-inverse targets of the training meshes (their
    own hierarchies), then Adam on the device."""
    import torch
    t0 = time.perf_counter()
    ctxs, _ = batch_setup(amg, problems, amg.AMG_PREC_FP64, local)
    setup_s = time.perf_counter() - t0
    sizes = [c.level_info(0)["n_rows"] for c in ctxs]
    total = sum(sizes)
    X = torch.zeros((total, 13), dtype=torch.float32, device=f"cuda:{local}")
    T = torch.zeros((total, 9), dtype=torch.float32, device=f"cuda:{local}")
    t0 = time.perf_counter()
    off = 0
    for c, p, n in zip(ctxs, problems, sizes):
        c.learned_features(p.coords[p.free], X[off:off + n])
        c.learned_targets(T32=T[off:off + n])
        off += n
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    net = amg.Mlp(local, seed=1)
    l0, _ = net.loss_grad(X, T)
    t0 = time.perf_counter()
    hist = net.train(X, T, epochs=epochs, batch=batch, lr=lr, seed=2)
    train_s = time.perf_counter() - t0
    return net, {"meshes": len(problems), "samples": int(total), "epochs": epochs, "batch": batch,
                 "lr": lr, "loss_initial": l0, "loss_final": float(hist[-1]),
                 "setup_s": round(setup_s, 2), "features_targets_s": round(data_s, 3),
                 "train_s": round(train_s, 3)}


# ---------------------------------------------------------------------------
# batched workload: 64 systems x 6 load cases, one graph launch per step
# ---------------------------------------------------------------------------

def _batch_problem(spec):
    from workloads import configs
    return configs.batch_problem(spec)


def batch_problems(n_systems):
    import multiprocessing as mp
    from workloads import configs
    specs = configs.batch_specs(64)[:n_systems]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_batch_problem, specs, chunksize=1)


def batch_setup(amg, problems, prec, local):
    """Library setup of every system, side by side on the host cores (one
    OpenMP thread per setup); returns the contexts and their prolongations."""
    from concurrent.futures import ThreadPoolExecutor
    ctxs = [amg.Context(local) for _ in problems]

    def one(i):
        ctxs[i].setup(problems[i], prec, host_threads=1)
        return [ctxs[i].download_prolongation(l) for l in range(ctxs[i].n_levels - 1)]

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        P_lists = list(ex.map(one, range(len(problems))))
    return ctxs, P_lists


def batch_upload(amg, problems, P_lists, prec, local):
    ctxs = []
    for p, P_list in zip(problems, P_lists):
        c = amg.Context(local)
        Ps = [type("P", (), dict(n_rows=n, n_cols=m, rowptr=rp, colidx=ci, vals=v))
              for (n, m, rp, ci, v) in P_list]
        c.upload_hierarchy(p.A, Ps, prec)
        ctxs.append(c)
    return ctxs


def stacked(B, problems):
    total = B.layout(0)[2]
    f = np.zeros(total)
    for s, p in enumerate(problems):
        off, n, _ = B.layout(s)
        f[off:off + 6 * n] = p.b.reshape(-1)
    return f


def batch_stage_roofline(levels_per_system, tuned, prec, hbm_gbs, nr=6):
    """Per grouped product stage of the batch: its tuned time per launch (from
    the tuner's CUDA events) against its algorithmic bytes over all systems
    (values + indices + row pointers once, vectors of the nr load cases
    once, updated outputs twice, smoother blocks for the smoothing)."""
    import re
    w = {0: 8, 1: 4, 2: 2}[prec]
    wv = 8 if prec == 0 else 4
    out = []
    for ln in tuned:
        m = re.search(r"(init|iteration): (.*?) (\d+)x(\d+): .* ([0-9.]+) us$", ln)
        if not m:
            continue
        name, br, bc, us = m.group(2), int(m.group(3)), int(m.group(4)), float(m.group(5))
        lv = re.search(r"level (\d+)", name)
        total = 0.0
        for levels in levels_per_system:
            if "A_0" in name:            # FP64 CG operator (init residual, q = A p)
                L = levels[0]
                n, k = L["n_rows"], L["block"]
                total += L["nnzb"] * (k * k * 8 + 4) + 4 * (n + 1) + (3 if "f -" in name else 2) * n * k * nr * 8
                continue
            l = int(lv.group(1))
            if l >= len(levels) - 1:
                continue
            L, C = levels[l], levels[l + 1]
            n, k, nc, kc = L["n_rows"], L["block"], C["n_rows"], C["block"]
            if L["block"] != br and "A x" in name:
                continue
            if "t = b - A x" in name:
                total += L["nnzb"] * (k * k * w + 4) + 4 * (n + 1) + 3 * n * k * nr * wv
            elif "M^+(b - A x)" in name:
                total += L["nnzb"] * (k * k * w + 4) + 4 * (n + 1) + 3 * n * k * nr * wv + n * k * k * wv
            elif "b_c = R t" in name:
                total += L["nnzb_P"] * (k * kc * w + 4) + 4 * (nc + 1) + (n * k + nc * kc) * nr * wv
            elif "x += P y_c" in name:
                total += L["nnzb_P"] * (k * kc * w + 4) + 4 * (n + 1) + (nc * kc + 2 * n * k) * nr * wv
        if total and us > 0:
            gbs = total / (us * 1e-6) / 1e9
            out.append({"stage": name, "block": f"{br}x{bc}", "us": us, "mbytes": round(total / 1e6, 1),
                        "gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm_gbs, 3)})
    return out


def run_batch(args, ws, rank, local, problems):
    import torch
    from paper_2011_13325_gb300 import amg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = args.precision
    t0 = time.perf_counter()
    ctx_main, P_lists = batch_setup(amg, problems, prec, local)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    levels_per_system = [[c.level_info(l) for l in range(c.n_levels)] for c in ctx_main]
    B = amg.Batch(ctx_main, 6)
    fh = stacked(B, problems)
    f = torch.from_numpy(fh).to(dev)
    u = torch.zeros_like(f)
    total = f.numel()

    def run(Bx, k, record):
        times, its = [], None
        for _ in range(k):
            u.zero_()
            torch.cuda.synchronize()
            _, it, rr, ms = Bx.pcg_solve(f, u, rtol=args.rtol, maxit=1000)
            if record:
                times.append(ms)
                its = it
        return times, its

    run(B, args.warmup, False)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.15)
    t_wall = time.perf_counter()
    times, its = run(B, args.steps, True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    if ws > 1:
        torch.distributed.barrier()
    ms = max_over_ranks(float(np.mean(times)), ws, dev)
    uh = u.cpu().numpy()

    # FP64 true residual of every load case (library residual kernel)
    worst = 0.0
    for s, c in enumerate(ctx_main):
        off, n, _ = B.layout(s)
        for j in range(6):
            fj = f[off + j * n:off + (j + 1) * n]
            uj = u[off + j * n:off + (j + 1) * n]
            r = torch.empty_like(fj)
            c.residual(0, fj, uj, r)
            worst = max(worst, float(torch.linalg.norm(r) / torch.linalg.norm(fj)))

    # the same batch with the FP64 V-cycle (one graph launch)
    variants = {}
    ctx64 = batch_upload(amg, problems, P_lists, 0, local) if prec != 0 else ctx_main
    if prec != 0:
        B64 = amg.Batch(ctx64, 6)
        run(B64, 3, False)
        t64, it64 = run(B64, args.steps, True)
        variants["batch_fp64"] = {"ms": round(float(np.mean(t64)), 3), "iters_max": max(it64),
                                  "iters_mean": round(float(np.mean(it64)), 2)}
        B64.close()
    # the same batch with the other arithmetic of the CG product
    main_df = "(double-float)" in B.describe()
    ctx_op = batch_upload(amg, problems, P_lists, prec, local)
    for c in ctx_op:
        c.set_cg_operator(amg.AMG_CG_FP64 if main_df else amg.AMG_CG_DOUBLE_FLOAT)
    Bop = amg.Batch(ctx_op, 6)
    run(Bop, 3, False)
    top, itop = run(Bop, args.steps, True)
    variants["cg_product_" + ("fp64" if main_df else "double_float")] = {
        "ms": round(float(np.mean(top)), 3), "iters_max": max(itop),
        "iters_mean": round(float(np.mean(itop)), 2)}
    Bop.close()
    for c in ctx_op:
        c.close()
    # plain FP64 GPU PCG, one system and one load case at a time (384 graph
    # launches per step), device time summed
    seq_steps = 2
    seq = []
    seq_its = []
    for step in range(1 + seq_steps):
        tot = 0.0
        for s, c in enumerate(ctx64):
            off, n, _ = B.layout(s)
            for j in range(6):
                fj = f[off + j * n:off + (j + 1) * n]
                uj = torch.zeros_like(fj)
                _, it, _ = c.pcg_solve(fj, uj, rtol=args.rtol, maxit=1000)
                tot += c.last_solve_ms()
                if step == 1:
                    seq_its.append(it[0])
        if step >= 1:
            seq.append(tot)
    variants["sequential_fp64"] = {"ms": round(float(np.mean(seq)), 3),
                                   "solves_per_step": 6 * len(ctx64),
                                   "iters_mean": round(float(np.mean(seq_its)), 2),
                                   "ms_ratio_to_main": round(float(np.mean(seq)) / ms, 2)}

    # end to end: host buffers, copies inside the call and its timing
    fpin = torch.from_numpy(fh).pin_memory()
    upin = torch.zeros_like(fpin).pin_memory()
    et = []
    for k in range(2 + args.steps):
        upin.zero_()
        _, _, _, e_ms = B.pcg_solve_host(fpin, upin, rtol=args.rtol, maxit=1000)
        if k >= 2:
            et.append(e_ms)

    per_step_bytes = 0
    for s, levels in enumerate(levels_per_system):
        it = its[s * 6:(s + 1) * 6]
        per_step_bytes += algorithmic_bytes_per_iteration(levels, prec, nr=6) * max(it)
    pk, pk_kind = peaks()
    gbs = per_step_bytes / (ms * 1e-3) / 1e9
    per_it, fixed = B.launches()
    launches = fixed + max(its) * per_it
    tuned = [ln for ln in B.describe().splitlines() if "lanes/row" in ln or "SELL-32" in ln]
    # dominant kernel: the grouped CG product q = A_0 p (6 load cases); in
    # FP64 bound by the FP64 pipe, in double-float arithmetic by HBM; its
    # per-launch time from the tuner's CUDA events
    import re
    cg_us = [float(re.search(r"([0-9.]+) us$", ln).group(1)) for ln in tuned if "q = A_0 p" in ln]
    nnzb0 = sum(levels[0]["nnzb"] * levels[0]["block"] ** 2 for levels in levels_per_system)
    cg_flops = 2.0 * 6 * nnzb0
    fp64_gflops, _ = ctx_main[0].probe_fma_rate()
    roof = None
    if cg_us and main_df:
        # values as pairs (8 bytes each) and column indices once, p pairs
        # read and q written for the 6 load cases of every dof
        cg_bytes = sum(L[0]["nnzb"] * (L[0]["block"] ** 2 * 8 + 4) + 4 * (L[0]["n_rows"] + 1) +
                       2 * 8 * 6 * L[0]["n_rows"] * L[0]["block"] for L in levels_per_system)
        ach = cg_bytes / (cg_us[0] * 1e-6) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / pk["hbm_gbs"], 3), "traffic": None,
                "kernel": "grouped CG product q = A_0 p in double-float arithmetic (gsell_df_kernel), "
                          "all systems, 6 load cases",
                "bytes_per_launch": int(cg_bytes), "us_per_launch": cg_us[0],
                "flops_per_launch": int(cg_flops), "tflops": round(cg_flops / (cg_us[0] * 1e-6) / 1e12, 3),
                "peak_kind": pk_kind}
    elif cg_us:
        ach = cg_flops / (cg_us[0] * 1e-6) / 1e12
        roof = {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp64_gflops / 1e3, 3),
                "unit": "TFLOP/s", "frac": round(ach / (fp64_gflops / 1e3), 3), "traffic": None,
                "kernel": "grouped FP64 CG product q = A_0 p, all systems, 6 load cases",
                "flops_per_launch": int(cg_flops), "us_per_launch": cg_us[0],
                "peak_kind": "FP64 FMA rate measured live (amg_probe_fma_rate)"}
    n_dofs = [levels[0]["n_rows"] * levels[0]["block"] for levels in levels_per_system]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import csolve
        ob = OracleBatch(problems, P_lists, args.rtol)
        all_ms, its_o = ob.solve_all()
        cores = csolve.max_threads()
        csolve.set_threads(1)
        try:
            v1, sample = ob.sample(budget_s=20.0)
        finally:
            csolve.set_threads(cores)
        cpu = {"value": round(all_ms, 1), "unit": "ms", "cores": cores, "kind": "oracle",
               "sample": (f"the oracle's FP64 PCG (C solve phase, oracle/csolve.c) on the same "
                          f"prolongations, every load case of every system to its own rtol "
                          f"{args.rtol:g} on {cores} host threads, timed whole (iterations: max "
                          f"{max(its_o)}, mean {np.mean(its_o):.1f}; GPU: max {max(its)}, mean "
                          f"{np.mean(its):.1f})"),
               "iters_max": max(its_o), "iters_mean": round(float(np.mean(its_o)), 2),
               "single_thread": {"value": round(v1, 1), "unit": "ms", "cores": 1, "sample": sample}}

    line = {
        "metric": "batched AMG-PCG time-to-1e-8 (FP64 residual), 64 systems x 6 load cases",
        "value": round(ms, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f64", 1: "f64 CG + f32 V-cycle", 2: "f64 CG + f32 V-cycle (bf16 storage)",
                  3: "f64 CG + f32 V-cycle (bf16 storage below level 0)"}[prec],
        "data": "synthetic",
        "config": {"workload": "batch64", "description": WORKLOADS["batch64"],
                   "systems": len(problems), "load_cases": 6, "dofs_total": int(sum(n_dofs)),
                   "dofs_min_max": [int(min(n_dofs)), int(max(n_dofs))],
                   "precision": PREC_NAMES[prec] + " V-cycle, fp64 CG (FP64 residual 1e-8)",
                   "rtol": args.rtol,
                   "l2": "inputs larger than L2 (operators of all systems > 1 GB)",
                   "parallelism": f"replicas x{ws}"},
        "iters_max": max(its), "iters_mean": round(float(np.mean(its)), 2),
        "true_relres_max": worst, "setup_s": round(setup_s, 2),
        "solve_gbs": round(gbs, 1), "bytes_per_step": int(per_step_bytes),
        "roofline": roof,
        "whole_solve_hbm": {"achieved": round(gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": round(gbs / pk["hbm_gbs"], 3),
                            "what": "algorithmic bytes of every V-cycle and CG kernel / graph time"},
        "wall_s_timed": round(wall, 3), "clocks": clocks, "variants": variants,
        "e2e": {"value": round(float(np.mean(et)), 3), "unit": "ms",
                "h2d_bytes_per_step": 2 * total * 8, "d2h_bytes_per_step": total * 8},
        "gpu_launches": launches * args.steps, "gpu_launches_per_step": launches,
        "autotuned_products": tuned,
        "stage_kernels": batch_stage_roofline(levels_per_system, tuned, prec, pk["hbm_gbs"]),
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


class OracleBatch:
    """The CPU oracle on the batched workload: per system the C solve phase
    (oracle/csolve.c: its own coarse matrices, block-l1 Jacobi blocks and
    coarsest factor) on the library's downloaded prolongations.
    solve_all() solves every load case of every system to rtol on all host
    threads (the oracle's own iteration counts, timed whole); sample() times
    load case 0 of the first systems, `maxit` = that case's own count, until
    about budget_s of CPU time, and scales the cost per dof-iteration to
    every load case at its own count.  Hierarchies are built once, outside
    the timed regions."""

    def __init__(self, problems, P_lists, rtol):
        self.problems, self.P_lists, self.rtol = problems, P_lists, rtol
        self._H = {}
        self.its = None

    def hierarchy(self, s):
        from oracle import csolve, solve
        if s not in self._H:
            A0 = solve.mat_from(self.problems[s].A)
            Ps = [solve.Mat(n, m, rp.astype(np.int64), ci.astype(np.int64), v)
                  for (n, m, rp, ci, v) in self.P_lists[s]]
            self._H[s] = csolve.Hierarchy(A0, Ps)
        return self._H[s]

    def solve_all(self):
        """(ms of all solves on all threads, iteration counts: 6 per system)"""
        its, spent = [], 0.0
        for s, p in enumerate(self.problems):
            H = self.hierarchy(s)
            for j in range(p.b.shape[0]):
                t0 = time.perf_counter()
                _, it, _ = H.pcg(p.b[j], rtol=self.rtol, maxit=1000)
                spent += time.perf_counter() - t0
                its.append(int(it))
            if s >= 1:     # keep the hierarchies of the first systems only
                self._H.pop(s, None)
        self.its = its
        return spent * 1e3, its

    def sample(self, budget_s):
        """(ms for the whole batch scaled from the sample, its description)"""
        spent, dof_its, used = 0.0, 0.0, 0
        for s, p in enumerate(self.problems):
            H = self.hierarchy(s)
            m = max(1, self.its[s * p.b.shape[0]])
            t0 = time.perf_counter()
            H.pcg(p.b[0], rtol=0.0, maxit=m)
            spent += time.perf_counter() - t0
            dof_its += m * p.b.shape[1]
            used += 1
            if spent >= budget_s:
                break
        per = spent / dof_its
        k = 0
        want = 0.0
        for p in self.problems:
            for _ in range(p.b.shape[0]):
                want += self.its[k] * p.b.shape[1]
                k += 1
        return per * want * 1e3, (f"oracle PCG (C solve phase) of load case 0 on the first {used} "
                                  f"systems ({spent:.1f} s), scaled per dof-iteration to all {k} "
                                  f"load cases at the oracle's own iteration counts")


def run_reference_batch(args, ws, rank, local, problems):
    """The CPU oracle on the batched workload (OracleBatch): the library's
    setup supplies the prolongations, the oracle's C solve phase solves every
    load case to rtol once (its own iteration counts), and every step times a
    bounded sample of it on all host threads."""
    import torch
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    from oracle import csolve
    from paper_2011_13325_gb300 import amg
    ctxs, P_lists = batch_setup(amg, problems, amg.AMG_PREC_FP64, local)
    for c in ctxs:
        c.close()
    ob = OracleBatch(problems, P_lists, args.rtol)
    all_ms, its_o = ob.solve_all()
    cores = csolve.max_threads()
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    per_step, sample = [], ""
    for s in range(args.warmup + args.steps):
        v, sample = ob.sample(budget)
        if s >= args.warmup:
            per_step.append(v)
    v = float(np.mean(per_step))
    line = {"impl": "reference",
            "metric": "batched AMG-PCG time-to-1e-8 (FP64 residual), 64 systems x 6 load cases",
            "value": round(v, 1), "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batch64", "description": WORKLOADS["batch64"],
                       "smoother": "block-l1 Jacobi"},
            "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": (f"each step: {sample}, on {cores} threads; one full pass "
                                        f"over all load cases: {all_ms / 1e3:.1f} s, iterations "
                                        f"max {max(its_o)}, mean {np.mean(its_o):.1f}")},
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
