"""Benchmark: matrix-free neo-Hookean tangent matvecs inside Newton + Jacobi-PCG
implicit Newmark steps on the 64x8x8-hex, P = 8 cantilever (6.50 M DOFs).

One step = one implicit Newmark step of the load ramp (Newton iterations with
a float64 residual, each solved by Jacobi-PCG whose iterations run the
tangent matvec), i.e. one pass of the whole hot path.  Inputs are synthetic
(seeded workload ``beam_p8``: E = 1000, nu = 0.45, dead tip shear traction
calibrated by the oracle), resident in HBM; every working vector and the
per-Gauss-point state exceed the 129 MB L2, so no flush is needed.

    python bench.py [--steps K] [--warmup W] [--precision mixed|fp64] [--basis sdme_h]
    python bench.py --impl reference      # the FP64 CPU oracle on host cores

Prints one JSON line (rank 0).  Multi-GPU: independent replicas (the single
mesh is not sharded), launched one rank per GPU by torchrun.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import load_magnitude, workload  # noqa: E402

METRIC = ("tangent-matvec DOF/s and Newton-PCG time per implicit step, SDME vs nodal, FP64 vs mixed at 1e-8")
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
FP64_PEAK_TFLOPS = 1.25                               # GB300 FP64 rate (profiling recipe table)


def lame(E, nu):
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def tangent_flops_per_element(P, nodal=False):
    """Float ops of one element's tangent action as the kernel computes it,
    with the even-odd (mirror) split of every 1D contraction.  Per line:
    interpolation between n modes and Q points 2 (QH n + [Q odd] NE) + 2 QH + 2,
    collocated derivative 2 (2 QH^2 + [Q odd] 2 QH) + 4 QH, the same for the
    transposed forms; a nodal basis adds n - 2 pairing adds per mode-side
    line.  Lines per component and direction: n^2 + nQ + Q^2 interpolations
    and 3 Q^2 derivatives; 207 flops of pointwise linearised stress per Gauss
    point.  (The plain contraction count, 4 x 3 (n^3 Q + n^2 Q^2 + n Q^3 +
    3 Q^4) + 207 Q^3, is 1.46x this at P = 8.)"""
    n, Q = P + 1, P + 2
    QH, NE, odd = Q // 2, 1 + P // 2, Q % 2
    interp = 2 * (QH * n + odd * NE) + 2 * QH + 2 + (n - 2 if nodal else 0)
    deriv = 2 * (2 * QH * QH + odd * 2 * QH) + 4 * QH
    per_dir = (n * n + n * Q + Q * Q) * interp + 3 * Q * Q * deriv
    return 3 * 2 * per_dir + 207 * Q ** 3


def algorithmic_flops_per_element(P):
    """Algorithmic float ops of one element's tangent action, the unit the
    roofline is quoted in: plain sum factorisation (no even-odd split),
    f1 = n Q (n^2 + n Q + Q^2) + 3 Q^4 multiply-adds per component and
    direction of application, forward and transposed for 3 components
    (12 f1 flops), plus 207 flops of pointwise linearised stress per Gauss
    point.  859,680 per element at P = 8."""
    n, Q = P + 1, P + 2
    f1 = n * Q * (n * n + n * Q + Q * Q) + 3 * Q ** 4
    return 12 * f1 + 207 * Q ** 3


def tangent_bytes(P, nelem, ndof, word_state, word_vec):
    """Algorithmic DRAM bytes of one tangent launch: the per-Gauss-point
    state (10 words), x read once, y read and written once."""
    Q = P + 2
    return 10 * Q ** 3 * nelem * word_state + 3 * ndof * word_vec


KERNEL_SOURCES = ("elem_kernels.cuh", "common.cuh", "elem_launch.cuh")


def profiled_traffic(precision):
    """DRAM bytes per tangent launch from the committed ncu summary, or None
    when the kernel sources changed since that capture (hash mismatch)."""
    import hashlib
    name = "tangent_kernel_f32_beam_p8.md" if precision == "mixed" else "tangent_kernel_f64_beam_p8.md"
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2104_13466_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    vals = {}
    for line in open(path):
        line = line.strip()
        for key in ("traffic_bytes_per_launch:", "kernel_source_sha256:"):
            if line.startswith(key):
                vals[key] = line.split(":", 1)[1].strip()
    if vals.get("kernel_source_sha256:") != h.hexdigest():
        return None
    try:
        return float(vals["traffic_bytes_per_launch:"])
    except (KeyError, ValueError):
        return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, device):
    """The slowest rank's time (replicas: the job ends when the last one does);
    the local time when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws, ndof, matvecs, ms):
    """Whole-job DOF/s of ws identical replicas timed to the slowest one."""
    return ws * ndof * matvecs / (ms * 1e-3)


def cpu_oracle_matvec(w, basis, nsample, seed=0):
    """The FP64 oracle's tangent action on a bounded sample of elements of
    the same mesh; returns (DOF/s scaled to the whole mesh, seconds, cores)."""
    from oracle.assembly import Discretization
    from oracle.basis1d import Basis1D
    from oracle.hexmesh import BoxMesh
    from oracle.material import lame as olame
    from synthetic import random_vector
    mu, lam = olame(w["E"], w["nu"])
    mesh = BoxMesh(*w["elems"], w["P"], w["lengths"])
    for f, comps in w["clamp"].items():
        mesh.clamp(f, comps)
    d = Discretization(mesh, Basis1D(w["P"], basis), mu, lam, w["rho"])
    u = random_vector(mesh.ndof, seed + 1, 1e-4)
    x = random_vector(mesh.ndof, seed + 2)
    els = np.arange(min(nsample, mesh.nelem))
    t0 = time.perf_counter()
    for s in range(0, len(els), 64):
        e = els[s:s + 64]
        Ue, Xe = d.gather(u, e), d.gather(x, e)
        Ye = d.ref.tangent_action(Ue, Xe, mu, lam) + 4.0 * d.ref.mass_action(Xe, w["rho"])
        d.scatter(Ye, e)
    dt = time.perf_counter() - t0
    dofs_per_s = mesh.ndof * (len(els) / mesh.nelem) / dt
    return dofs_per_s, dt, os.cpu_count()


def cpu_oracle_extras(w, basis, nsample):
    """The other timings the CPU-baseline plan names, on the oracle as it
    stands: config 1 (the 4^3-hex unit cube at P = 4) in full, 10 implicit
    Newmark steps with Jacobi-PCG (rtol 1e-10, Newton 1e-8) in SDME-H; and
    one internal-force evaluation on the cantilever's sample of elements,
    scaled to the mesh (a Newton step of the 6.5 M-DOF cantilever would take
    the oracle hours)."""
    from oracle import solvers
    from oracle.assembly import Discretization
    from oracle.basis1d import Basis1D
    from oracle.hexmesh import BoxMesh
    from oracle.material import lame as olame
    from synthetic import random_vector
    out = {}
    wc = workload("cube_p4")
    mu, lam = olame(wc["E"], wc["nu"])
    mesh = BoxMesh(*wc["elems"], wc["P"], wc["lengths"])
    for f, comps in wc["clamp"].items():
        mesh.clamp(f, comps)
    d = Discretization(mesh, Basis1D(wc["P"], "sdme_h"), mu, lam, wc["rho"])
    unit = d.traction_load(wc["traction_face"], lambda X, t: np.broadcast_to(wc["traction_dir"], X.shape))
    smag = load_magnitude(wc["load_key"])
    u = np.zeros(mesh.ndof)
    v, a = u.copy(), u.copy()
    t0 = time.perf_counter()
    newton = 0
    for k in range(1, wc["steps"] + 1):
        u, v, a, st = solvers.newmark_step(d, u, v, a, unit * smag * k / wc["steps"], wc["dt"],
                                           tol=wc["newton_tol"], pcg_rtol=wc["pcg_rtol"])
        newton += len(st["pcg_iters"])
    dt = time.perf_counter() - t0
    out["cube_p4_newmark"] = {"ms_per_step": dt * 1e3 / wc["steps"], "steps": wc["steps"],
                              "newton_iters_per_step": newton / wc["steps"], "basis": "sdme_h"}
    mu, lam = olame(w["E"], w["nu"])
    mesh = BoxMesh(*w["elems"], w["P"], w["lengths"])
    for f, comps in w["clamp"].items():
        mesh.clamp(f, comps)
    d = Discretization(mesh, Basis1D(w["P"], basis), mu, lam, w["rho"])
    uu = random_vector(mesh.ndof, 11, 1e-4)
    els = np.arange(min(nsample, mesh.nelem))
    t0 = time.perf_counter()
    for s0 in range(0, len(els), 64):
        e = els[s0:s0 + 64]
        d.scatter(d.ref.internal_force(d.gather(uu, e), mu, lam), e)
    dt = time.perf_counter() - t0
    out["beam_internal_force"] = {"dofs_per_s": mesh.ndof * (len(els) / mesh.nelem) / dt,
                                  "sample": "%d of %d elements, scaled to the mesh" % (len(els), mesh.nelem)}
    return out


def workload_config(args, w, ws):
    """The `config` object of the default line, identical for both arms."""
    ne, P = w["elems"], w["P"]
    nelem = int(np.prod(ne))
    n = 3 * int(np.prod([e * P + 1 for e in ne]))
    wstate = 4 if args.precision == "mixed" else 8
    return {"workload": "beam_p8: [0,8]x[0,1]^2 cantilever, 64x8x8 hexes, P=8, %d DOFs, basis %s, "
                        "%s, Newton tol %g, dt %g" % (n, args.basis, args.precision, w["newton_tol"], w["dt"]),
            "global_batch": 1, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "inputs larger than L2 (vectors 52 MB each, Gauss-point state %d MB)"
                  % (10 * (P + 2) ** 3 * nelem * wstate // 2 ** 20)}


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    per_step = []
    sample = args.ref_sample
    for i in range(args.warmup + args.steps):
        v, dt, cores = cpu_oracle_matvec(w, args.basis, sample, seed=i)
        if i >= args.warmup:
            per_step.append((v, dt))
    value = float(np.mean([v for v, _ in per_step]))
    ms = float(np.mean([dt for _, dt in per_step]) * 1e3)
    desc = "FP64 numpy oracle tangent action on %d of %d elements per step, scaled to the mesh" % (
        sample, int(np.prod(w["elems"])))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w, ws),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_context(sd, w, basis, prec, lam_h=None):
    mu, lam = lame(w["E"], w["nu"])
    return sd.Context(w["elems"], w["lengths"], w["clamp"], mu, lam, w["rho"], w["P"], basis, precision=prec,
                      k=w["k"], lam_h=w["lam"] if lam_h is None else lam_h)


class Ramp:
    """Implicit Newmark steps of a workload's load ramp on one context, from
    rest: step k applies the traction at level min(k, steps) / steps.  Each
    step is timed with CUDA events on the current stream (the context runs on
    the legacy default stream, which orders with it)."""

    def __init__(self, sd, torch, ctx, w, opts):
        self.sd, self.torch, self.ctx, self.w, self.opts = sd, torch, ctx, w, opts
        n = ctx.ndof
        self.unit = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.traction_load(w["traction_face"], np.array(w["traction_dir"], dtype=float), self.unit)
        self.smag = load_magnitude(w["load_key"])
        self.u, self.v, self.a, self.Pn = (torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(4))
        self.k = 0

    def state(self):
        return self.k, self.u.clone(), self.v.clone(), self.a.clone()

    def set_state(self, st):
        self.k = st[0]
        for dst, src in zip((self.u, self.v, self.a), st[1:]):
            dst.copy_(src)

    def step(self):
        torch = self.torch
        self.k += 1
        level = min(self.k, self.w["steps"])
        torch.mul(self.unit, self.smag * level / self.w["steps"], out=self.Pn)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = self.ctx.implicit_newmark_step(self.u, self.v, self.a, self.w["dt"], self.Pn,
                                            allow=(self.sd.NEWTON_DIVERGED,), **self.opts)
        e1.record(stream)
        e1.synchronize()
        st["ms"] = e0.elapsed_time(e1)
        st["level"] = level
        return st


def step_summary(st):
    return {"level": st["level"], "ms": round(st["ms"], 3), "converged": st["converged"],
            "newton_iters": st["newton_iters"], "pcg_iters_total": st["pcg_iters_total"],
            "residual_rel": st["residual_rel"], "lin_rel_max": st["lin_rel_max"],
            "refine_sweeps": st["refine_sweeps"]}


def arm_summary(n, steps):
    ms = sum(s["ms"] for s in steps)
    mv = sum(s["matvecs"] for s in steps)
    return {"steps": len(steps), "levels": [s["level"] for s in steps],
            "converged_steps": sum(1 for s in steps if s["converged"]),
            "ms_per_step": ms / max(1, len(steps)), "matvec_dofs_per_s": n * mv / (ms * 1e-3) if ms > 0 else None,
            "newton_iters_per_step": sum(s["newton_iters"] for s in steps) / max(1, len(steps)),
            "pcg_iters_per_newton": mv / max(1, sum(s["newton_iters"] for s in steps)),
            "ms": [round(s["ms"], 2) for s in steps]}


def newton_opts(args, w):
    return dict(newton_tol=w["newton_tol"], pcg_rtol=w["pcg_rtol"], mixed_rtol=args.mixed_rtol,
                pcg_maxit=args.pcg_maxit, max_newton=args.max_newton, forcing=args.forcing)


def compare_block(args, w, n_main, main_steps, saved, prec_main):
    """The metric's comparisons beside the timed line (rank 0):
    * fp64 vs mixed on the cantilever: one float64 step from the main arm's
      own input state at each saved level, against the main arm's step there;
    * bases on the cantilever: each other basis from rest over the first
      levels of the ramp, against the main arm's steps at the same levels;
    * the unit cube of 4^3 hexes at P = 4 (14,739 DOFs, bottom clamped, top
      traction ramped over 10 steps of dt = 0.01): every basis in both
      precisions over the whole ramp."""
    import torch
    import paper_2104_13466_gb300 as sd
    out = {}
    opts = newton_opts(args, w)
    other = sd.FP64 if prec_main == sd.MIXED_FP32 else sd.MIXED_FP32
    ctx = make_context(sd, w, args.basis, other)
    ramp = Ramp(sd, torch, ctx, w, opts)
    rows = []
    for lvl_state in saved:
        ramp.set_state(lvl_state)
        st = ramp.step()
        mine = main_steps[lvl_state[0]]
        rows.append({"level": st["level"], "mixed_ms" if prec_main == sd.MIXED_FP32 else "fp64_ms": mine["ms"],
                     "fp64_ms" if prec_main == sd.MIXED_FP32 else "mixed_ms": st["ms"],
                     "mixed_converged": mine["converged"] if prec_main == sd.MIXED_FP32 else st["converged"],
                     "fp64_converged": st["converged"] if prec_main == sd.MIXED_FP32 else mine["converged"],
                     "fp64_newton_iters": (st if prec_main == sd.MIXED_FP32 else mine)["newton_iters"],
                     "mixed_newton_iters": (mine if prec_main == sd.MIXED_FP32 else st)["newton_iters"]})
    ctx.close()
    for r in rows:
        r["mixed_speedup"] = r["fp64_ms"] / r["mixed_ms"]
    out["beam_fp64_vs_mixed"] = rows
    m = min(args.compare_levels, len(main_steps))
    bases = {args.basis: arm_summary(n_main, main_steps[:m])}
    for basis in [b for b in args.compare_bases.split(",") if b and b != args.basis]:
        ctx = make_context(sd, w, basis, prec_main)
        n = ctx.ndof
        ramp = Ramp(sd, torch, ctx, w, opts)
        bases[basis] = arm_summary(n, [ramp.step() for _ in range(m)])
        ctx.close()
    out["beam_bases"] = {"precision": "mixed" if prec_main == sd.MIXED_FP32 else "fp64", "arms": bases}
    wc = workload("cube_p4")
    cube = {}
    for pname, pr in (("mixed", sd.MIXED_FP32), ("fp64", sd.FP64)):
        for basis in ("nodal", "modal", "sdme_m", "sdme_h"):
            ctx = make_context(sd, wc, basis, pr)
            o = newton_opts(args, wc)
            warm = Ramp(sd, torch, ctx, wc, o)
            warm.step()
            ramp = Ramp(sd, torch, ctx, wc, o)
            cube["%s/%s" % (basis, pname)] = arm_summary(ctx.ndof, [ramp.step() for _ in range(wc["steps"])])
            ctx.close()
    out["cube_p4"] = cube
    if args.compare_batch_steps > 0:
        r = run_batch(args, workload("batch_cubes"), steps=args.compare_batch_steps, quiet=True, basis="sdme_h")
        out["batch_cubes"] = {k: r[k] for k in ("problems", "total_dofs", "elements", "steps", "ms_per_step",
                                                "matvec_dofs_per_s", "all_converged", "newton_iters_mean",
                                                "pcg_iters_per_newton_mean", "pcg_iters_per_newton_max",
                                                "persistent", "tuning")}
    return out


def run_gpu(args, w):
    import torch
    import paper_2104_13466_gb300 as sd

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = sd.MIXED_FP32 if args.precision == "mixed" else sd.FP64
    ctx = make_context(sd, w, args.basis, prec)
    tangent_grid = ctx.set_tangent_grid(args.tangent_grid)
    n = ctx.ndof
    dev = torch.device("cuda", local)
    opts = newton_opts(args, w)
    ramp = Ramp(sd, torch, ctx, w, opts)
    # input states of the fp64-vs-mixed comparison: the first timed step and
    # the last ramp level reached
    total = args.warmup + args.steps
    cmp_levels = sorted({args.warmup + 1, min(total, w["steps"])})
    saved = []
    all_steps = []

    def one_step():
        if ramp.k + 1 in cmp_levels and rank == 0 and not args.no_compare:
            saved.append(ramp.state())
        st = ramp.step()
        all_steps.append(st)
        return st

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ctx.set_timing(True)
    t0 = ctx.timing()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(one_step())
        e1.record(stream)
        torch.cuda.synchronize()
    ctx.set_timing(False)
    t1 = ctx.timing()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    matvecs = sum(s["matvecs"] for s in stats)
    unconverged = sum(1 for s in all_steps if not s["converged"])
    value = replica_throughput(ws, n, matvecs, ms) if unconverged == 0 else None
    tan_ms = (t1["tangent_ms"] - t0["tangent_ms"])
    tan_launches = t1["tangent_launches"] - t0["tangent_launches"]
    avg_tan = tan_ms / max(1, tan_launches)
    wstate = 4 if prec == sd.MIXED_FP32 else 8
    flops = algorithmic_flops_per_element(w["P"]) * ctx.nelem
    flops_impl = tangent_flops_per_element(w["P"], args.basis == "nodal") * ctx.nelem
    nbytes = tangent_bytes(w["P"], ctx.nelem, n, wstate, wstate)
    achieved_tf = flops / (avg_tan * 1e-3) / 1e12
    alu_peak = FP32_PEAK_TFLOPS if prec == sd.MIXED_FP32 else FP64_PEAK_TFLOPS
    hbm_peak, hbm_src = _peaks()
    achieved_gbs = nbytes / (avg_tan * 1e-3) / 1e9

    # end to end through the public API: host state and load in, host state
    # out, for the step after the timed ones (same load level as the last)
    pin = [torch.zeros(n, dtype=torch.float64).pin_memory() for _ in range(4)]
    for p_, d_ in zip(pin, (ramp.u, ramp.v, ramp.a, ramp.unit)):
        p_.copy_(d_)
    out = [torch.zeros(n, dtype=torch.float64).pin_memory() for _ in range(3)]
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_mv, e2e_conv = 0, True
    e2.record(stream)
    for _ in range(args.e2e_steps):
        for p_, d_ in zip(pin, (ramp.u, ramp.v, ramp.a, ramp.unit)):
            d_.copy_(p_, non_blocking=True)
        ramp.k -= 1  # the same load level as the last timed step
        st = ramp.step()
        e2e_mv += st["matvecs"]
        e2e_conv = e2e_conv and st["converged"]
        for o_, d_ in zip(out, (ramp.u, ramp.v, ramp.a)):
            o_.copy_(d_, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2.elapsed_time(e3)
    e2e_value = ws * n * e2e_mv / (e2e_ms * 1e-3) if args.e2e_steps > 0 and e2e_ms > 0 and e2e_conv else None
    ctx.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cv, cdt, cores = cpu_oracle_matvec(w, args.basis, args.ref_sample)
        cpu = {"value": cv, "unit": "DOF/s", "cores": cores, "kind": "oracle",
               "sample": "FP64 numpy oracle tangent action on %d of %d elements (%.1f s), scaled to the mesh"
                         % (args.ref_sample, int(np.prod(w["elems"])), cdt)}
        if args.cpu_extras:
            cpu["extra"] = cpu_oracle_extras(w, args.basis, args.ref_sample)
    clocks = clk.summary()
    compare = None
    if rank == 0 and not args.no_compare:
        compare = compare_block(args, w, n, all_steps, saved, prec)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-matvec/f64-residual" if prec == sd.MIXED_FP32 else "f64",
            "data": "synthetic",
            "config": workload_config(args, w, ws),
            "newton_pcg_ms_per_step": ms / args.steps,
            "unconverged_steps": unconverged,
            "steps_detail": [step_summary(s) for s in all_steps[args.warmup:]],
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved_tf / alu_peak,
                         "traffic": profiled_traffic(args.precision) if w["P"] == 8 and args.workload == "beam_p8"
                         else None,
                         "kernel": "tangent_kernel<8,%s>" % ("float,float" if prec == sd.MIXED_FP32 else "double,double"),
                         "avg_launch_ms": avg_tan, "launches": tan_launches, "tangent_grid": tangent_grid,
                         "flops_per_launch": flops, "flops_unit": "plain sum factorisation, 859,680 per P=8 element",
                         "flops_per_launch_even_odd": flops_impl,
                         "peak_src": "derived from recipe unit counts and max clock",
                         "hbm_view": {"bytes_per_launch": nbytes, "achieved_gbs": achieved_gbs, "peak_gbs": hbm_peak,
                                      "frac": achieved_gbs / hbm_peak, "peak_src": hbm_src}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "DOF/s", "steps": args.e2e_steps,
                    "h2d_bytes_per_step": 4 * n * 8, "d2h_bytes_per_step": 3 * n * 8},
            "gpu_launches": int(t1["kernel_launches"] - t0["kernel_launches"]),
            "clocks": clocks,
        }
        if compare is not None:
            line["compare"] = compare
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if unconverged:
        sys.exit(1)


def run_kernel_only(args, w):
    """A few PCG iterations at the full bench size: linearise at a seeded
    displacement, then run ``--kernel-iters`` iterations (rtol 0), timing
    every tangent launch with CUDA events.  Used for kernel profiles."""
    import torch
    import paper_2104_13466_gb300 as sd
    from synthetic import random_vector
    prec = sd.MIXED_FP32 if args.precision == "mixed" else sd.FP64
    mu, lam = lame(w["E"], w["nu"])
    ctx = sd.Context(w["elems"], w["lengths"], w["clamp"], mu, lam, w["rho"], w["P"], args.basis, precision=prec)
    n = ctx.ndof
    u = torch.from_numpy(random_vector(n, 1, 1e-4)).cuda()
    b = torch.from_numpy(random_vector(n, 2)).cuda()
    x = torch.zeros_like(u)
    grid = ctx.set_tangent_grid(args.tangent_grid)
    ctx.set_timing(True)
    its, rel = ctx.pcg_solve(u, 4.0, b, x, rtol=0.0, maxit=args.kernel_iters, allow_maxit=True)
    t = ctx.timing()
    avg = t["tangent_ms"] / max(1, t["tangent_launches"])
    flops = algorithmic_flops_per_element(w["P"]) * ctx.nelem
    flops_eo = tangent_flops_per_element(w["P"], args.basis == "nodal") * ctx.nelem
    print(json.dumps({"mode": "kernel-only", "precision": args.precision, "basis": args.basis, "iters": its,
                      "tangent_grid": grid,
                      "tangent_avg_ms": avg, "tflops": flops / (avg * 1e-3) / 1e12,
                      "tflops_even_odd_count": flops_eo / (avg * 1e-3) / 1e12, "launches": t["tangent_launches"]}),
          flush=True)
    ctx.close()


def run_compare(args, w):
    """The metric's comparison: Newton-PCG time per implicit step for each
    basis and precision on identical inputs (same mesh, load ramp, steps).
    One JSON line per (basis, precision), rank 0 only."""
    import torch
    import paper_2104_13466_gb300 as sd
    mu, lam = lame(w["E"], w["nu"])
    for prec_name in args.precisions.split(","):
        prec = sd.MIXED_FP32 if prec_name == "mixed" else sd.FP64
        for basis in args.bases.split(","):
            ctx = sd.Context(w["elems"], w["lengths"], w["clamp"], mu, lam, w["rho"], w["P"], basis,
                             precision=prec)
            n = ctx.ndof
            unit = torch.zeros(n, dtype=torch.float64, device="cuda")
            ctx.traction_load(w["traction_face"], np.array(w["traction_dir"], dtype=float), unit)
            smag = load_magnitude(w["load_key"])
            u, v, a, Pn = (torch.zeros_like(unit) for _ in range(4))
            opts = dict(newton_tol=w["newton_tol"], pcg_rtol=w["pcg_rtol"], mixed_rtol=args.mixed_rtol,
                        pcg_maxit=args.pcg_maxit, max_newton=args.max_newton, forcing=args.forcing)
            res = []
            for k in range(1, args.warmup + args.steps + 1):
                torch.mul(unit, smag * min(k, w["steps"]) / w["steps"], out=Pn)
                ctx.set_timing(k > args.warmup)
                t0 = ctx.timing()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = ctx.implicit_newmark_step(u, v, a, w["dt"], Pn, allow=(sd.NEWTON_DIVERGED, sd.PCG_MAXIT),
                                               **opts)
                e1.record()
                torch.cuda.synchronize()
                if k > args.warmup:
                    t1 = ctx.timing()
                    res.append({"step": k, "ms": e0.elapsed_time(e1), "newton_iters": st["newton_iters"],
                                "pcg_iters": st["pcg_iters"], "converged": st["converged"],
                                "residual_rel": st["residual_final"] / max(st["residual0"], 1e-300),
                                "tangent_avg_ms": (t1["tangent_ms"] - t0["tangent_ms"]) /
                                max(1, t1["tangent_launches"] - t0["tangent_launches"])})
            tot_ms = sum(r["ms"] for r in res)
            mv = sum(sum(r["pcg_iters"]) for r in res)
            print(json.dumps({"mode": "compare", "workload": args.workload, "basis": basis, "precision": prec_name,
                              "ms_per_step": tot_ms / len(res), "matvec_dofs_per_s": n * mv / (tot_ms * 1e-3),
                              "pcg_iters_per_newton": mv / max(1, sum(r["newton_iters"] for r in res)),
                              "steps": res}), flush=True)
            ctx.close()


def run_explicit(args, w):
    """Explicit central-difference run (config 2 shape): v0 projected from the
    seeded sinusoidal field, dt = 0.5 dt_crit from a power iteration, N steps
    without load in float64 and in mixed precision on identical inputs;
    reports time per step, energy drift and the mixed-vs-float64 difference.
    The configuration is the unit cube (nx = ny = nz) with all faces clamped."""
    import torch
    import paper_2104_13466_gb300 as sd
    from synthetic import random_uniform
    mu, lam = lame(w["E"], w["nu"])
    amp = w["v_amp"] * (1.0 + 0.01 * float(random_uniform(1, w["seed"])[0]))
    out = {"mode": "explicit", "workload": args.workload, "basis": args.basis, "amplitude": amp}
    v0 = None
    results = {}
    for prec_name in ("fp64", "mixed"):
        prec = sd.MIXED_FP32 if prec_name == "mixed" else sd.FP64
        ctx = sd.Context(w["elems"], w["lengths"], w["clamp"], mu, lam, w["rho"], w["P"], args.basis,
                         precision=prec)
        n = ctx.ndof
        if v0 is None:
            # L2 projection of v0 = A sin(pi x) sin(pi y) sin(pi z) e_z (float64 context)
            X = ctx.gauss_point_coords()
            fq = torch.zeros(X.shape[0], 3, X.shape[1], dtype=torch.float64, device="cuda")
            fq[:, 2, :] = amp * torch.sin(np.pi * X[..., 0]) * torch.sin(np.pi * X[..., 1]) * \
                torch.sin(np.pi * X[..., 2])
            b = torch.zeros(n, dtype=torch.float64, device="cuda")
            ctx.body_load(fq.contiguous(), b)
            v0 = torch.zeros_like(b)
            ctx.mass_solve(b, v0, rtol=1e-13)
            dt_crit, lam_max = ctx.estimate_dt_crit(torch.zeros_like(b), iters=args.dt_iters)
            dt = w["cfl"] * dt_crit
            out.update({"dt_crit": dt_crit, "dt": dt, "ndof": n})
        zero = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = ctx.explicit_state(torch.zeros_like(zero), torch.zeros_like(zero), torch.zeros_like(zero))
        rtol = w["mass_rtol"] if prec == sd.FP64 else w["mass_rtol_mixed"]
        ctx.explicit_start(st, dt, zero, v0, rtol=rtol)
        E0, _ = ctx.energy(v=v0)
        energies, its_total = [], 0
        torch.cuda.synchronize()
        t_ms = 0.0
        prev = st.u_prev.clone()
        for k in range(1, args.explicit_steps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            its_total += ctx.explicit_step(st, dt, zero, rtol=rtol)
            e1.record()
            torch.cuda.synchronize()
            t_ms += e0.elapsed_time(e1)
            if k % args.energy_every == 0:
                v = ((st.u - prev) / (2 * dt)).contiguous()
                ke, se = ctx.energy(st.u_prev, v)
                energies.append((k, (ke + se) / E0 - 1.0))
            prev.copy_(st.u_prev)
        results[prec_name] = {"u": st.u.clone(), "ms_per_step": t_ms / args.explicit_steps,
                              "mass_pcg_iters_per_step": its_total / args.explicit_steps,
                              "energy_rel_dev_max": max(abs(e) for _, e in energies),
                              "energy_rel_dev_last": energies[-1][1], "energy_trace": energies[::5]}
        ctx.close()
    u64, u32 = results["fp64"].pop("u"), results["mixed"].pop("u")
    out["mixed_vs_fp64_u_rel"] = float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64))
    out["fp64"], out["mixed"] = results["fp64"], results["mixed"]
    print(json.dumps(out), flush=True)


def run_adjoint(args, w):
    """Differentiated explicit run (config 5 shape): u_N of a checkpointed
    central-difference trajectory under a constant dead tip traction, the
    objective J = |u_N - target|^2 over the tip face, and dJ/d(mu, lambda) by
    the hand-written discrete adjoint; compared with central finite
    differences (h = fd_rel_h relative) of the same GPU forward run."""
    import torch
    import paper_2104_13466_gb300 as sd
    from synthetic import random_uniform
    mu, lam = lame(w["E"], w["nu"])
    ctx = sd.Context(w["elems"], w["lengths"], w["clamp"], mu, lam, w["rho"], w["P"], args.basis)
    n = ctx.ndof
    Nx, Ny, Nz = ctx.N
    zero = torch.zeros(n, dtype=torch.float64, device="cuda")
    f = torch.zeros_like(zero)
    ctx.traction_load(w["traction_face"], w["traction"], f)
    dt_crit, _ = ctx.estimate_dt_crit(zero, iters=args.dt_iters)
    dt = w["cfl"] * dt_crit
    # tip-face DOF indices (x = Nx - 1) and the seeded target
    j, k = np.meshgrid(np.arange(Ny), np.arange(Nz), indexing="xy")
    node = ((k * Ny + j) * Nx + (Nx - 1)).ravel()
    idx = np.concatenate([c * Nx * Ny * Nz + node for c in range(3)])
    xi = random_uniform(node.size, w["seed"])
    target = np.zeros(idx.size)
    target[2 * node.size:] = -w["tip_delta"] * (1.0 + 0.1 * xi)
    idx_t = torch.from_numpy(idx).cuda()
    tgt = torch.from_numpy(target).cuda()
    steps, every, rtol = w["steps"], w["every"], w["mass_rtol"]
    tape = sd.Tape(ctx, steps, every)
    uN = torch.zeros_like(zero)

    def objective(mu_, lam_):
        ctx.set_material(mu_, lam_)
        tape.forward(dt, zero, zero, uN, f=f, rtol=rtol)
        return float(((uN[idx_t] - tgt) ** 2).sum())

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    objective(mu, lam)  # warm-up (kernel attributes, graph capture)
    launches0 = ctx.timing()["kernel_launches"]
    J, t_fwd = timed(lambda: objective(mu, lam))
    gN = torch.zeros_like(zero)
    gN[idx_t] = 2.0 * (uN[idx_t] - tgt)
    (gmu, glam), t_adj = timed(lambda: tape.adjoint(gN))
    launches = ctx.timing()["kernel_launches"] - launches0
    h_mu, h_lam = w["fd_rel_h"] * mu, w["fd_rel_h"] * lam
    fd_mu = (objective(mu + h_mu, lam) - objective(mu - h_mu, lam)) / (2 * h_mu)
    fd_lam = (objective(mu, lam + h_lam) - objective(mu, lam - h_lam)) / (2 * h_lam)
    out = {"mode": "adjoint", "workload": args.workload, "basis": args.basis, "ndof": n, "steps": steps,
           "checkpoint_every": every, "dt": dt, "dt_crit": dt_crit, "J": J,
           "forward_ms": t_fwd, "adjoint_ms": t_adj, "adjoint_over_forward": t_adj / t_fwd,
           "dJ_dmu": gmu, "dJ_dlambda": glam, "fd_dmu": fd_mu, "fd_dlambda": fd_lam,
           "rel_err_mu": abs(gmu - fd_mu) / abs(fd_mu), "rel_err_lambda": abs(glam - fd_lam) / abs(fd_lam),
           "gpu_launches_fwd_plus_adj": launches, "fd_rel_h": w["fd_rel_h"], "mass_rtol": rtol}
    tape.close()
    ctx.close()
    print(json.dumps(out), flush=True)


def compare_sequential(args, w, probs, b_full, f_full, dt, steps):
    """The first K problems of the batch solved (a) as one batch and (b) one
    context at a time, `steps` Newmark steps each on identical inputs;
    prints both wall times (the batching gain) and the largest difference
    between the two solutions."""
    import torch
    import paper_2104_13466_gb300 as sd
    K = args.batch_vs_sequential
    sub = probs[:K]
    prec = sd.MIXED_FP32 if args.precision == "mixed" else sd.FP64
    fh = [b_full.segment(f_full, i).clone() for i in range(K)]
    opts = dict(newton_tol=w["newton_tol"], mixed_rtol=args.mixed_rtol, pcg_maxit=args.pcg_maxit)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    b = sd.Batch(sub, args.basis, precision=prec, k=w["k"], lam_h=w["lam"])
    if not args.no_tune:
        b.tune(reps=3)
    fb = b.zeros()
    for i in range(K):
        b.segment(fb, i).copy_(fh[i])

    def run_batch():
        u, v, a = b.zeros(), b.zeros(), b.zeros()
        for n in range(1, steps + 1):
            b.newmark_step(u, v, a, dt, fb * (n / w["steps"]), **opts)
        return u

    ctxs = [sd.Context(pr["elems"], pr["lengths"], pr["clamp"], pr["mu"], pr["lam"], pr["rho"], pr["P"], args.basis,
                       precision=prec, k=w["k"], lam_h=w["lam"]) for pr in sub]

    def run_seq():
        us = []
        for i, c in enumerate(ctxs):
            u, v, a = (torch.zeros(c.ndof, dtype=torch.float64, device="cuda") for _ in range(3))
            for n in range(1, steps + 1):
                c.implicit_newmark_step(u, v, a, dt, fh[i] * (n / w["steps"]), **opts)
            us.append(u)
        return us

    run_batch()  # warm-up
    run_seq()
    ub, t_batch = timed(run_batch)
    us, t_seq = timed(run_seq)
    diff = max(float((b.segment(ub, i) - us[i]).abs().max() / us[i].abs().max()) for i in range(K))
    print(json.dumps({"mode": "batch-vs-sequential", "problems": K, "steps": steps, "dofs": int(sum(b.ndofs)),
                      "batch_ms": t_batch, "sequential_ms": t_seq, "speedup": t_seq / t_batch,
                      "max_rel_diff": diff}), flush=True)


def run_batch(args, w, steps=None, persist=None, quiet=False, basis=None):
    """Batched independent solves (config 4 shape): 256 seeded cubes of uneven
    size, order and material, each taking `steps` implicit Newmark steps of a
    ramped top traction, all problems advanced together (one set of launches
    per step, PCG chunks replayed as one CUDA graph for the whole batch), in
    mixed precision (float32 tangent and PCG inside the float64 Newton
    residual).  Reports the aggregate tangent-matvec DOF/s over the timed
    steps, the wall time, the tuner's launch configuration per order and the
    persistent cross-order operator's tiles and timing (persist: 1 / 0 / -1
    forces it on, off, or lets the tuner decide)."""
    import torch
    import paper_2104_13466_gb300 as sd
    from synthetic import batch_draws, load_magnitude
    side, orders, E, nu = batch_draws(w)
    probs = []
    for i in range(w["count"]):
        mu, lam = lame(E[i], nu[i])
        probs.append(dict(elems=(side[i],) * 3, lengths=(1.0, 1.0, 1.0), clamp=w["clamp"], mu=mu, lam=lam,
                          rho=w["rho"], P=orders[i]))
    prec = sd.MIXED_FP32 if args.precision == "mixed" else sd.FP64
    basis = basis or args.basis
    t0 = time.time()
    b = sd.Batch(probs, basis, precision=prec, k=w["k"], lam_h=w["lam"])
    t_create = time.time() - t0
    persist = args.batch_persist if persist is None else persist
    b.set_persistent(persist)
    smag = load_magnitude(w["load_key"])
    f = b.zeros()
    scale = (w["load_scale"] if args.batch_load_scale is None else args.batch_load_scale) * smag / 1.0e3
    b.traction_load(w["traction_face"], [(0.0, 0.0, -scale * E[i]) for i in range(w["count"])], f)
    tuning = b.tune(reps=3) if not args.no_tune else []
    if persist != -1:
        b.set_persistent(persist)   # keep the forced form (the tuner's tiles stay)
    steps = steps or args.batch_steps or w["steps"]
    dt = w["dt"]

    def run(nsteps, time_it):
        u, v, a = b.zeros(), b.zeros(), b.zeros()
        stats, ms = [], 0.0
        for n in range(1, nsteps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            st = b.newmark_step(u, v, a, dt, f * (n / w["steps"]), newton_tol=w["newton_tol"],
                                mixed_rtol=args.mixed_rtol, pcg_maxit=args.pcg_maxit,
                                allow=(sd.NONPOSITIVE_J, sd.NEWTON_DIVERGED, sd.NAN))
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            stats.append(st)
        return stats, ms

    if args.batch_vs_sequential:
        compare_sequential(args, w, probs, b, f, dt, steps=2)
        b.close()
        return
    run(1, False)  # warm-up: kernel attributes, graph capture
    l0 = b.launches()
    stats, ms = run(steps, True)
    launches = b.launches() - l0
    dof_matvecs = sum(b.ndofs[i] * st[i]["matvecs"] for st in stats for i in range(b.nprob))
    conv = all(st[i]["converged"] for st in stats for i in range(b.nprob))
    failed = sorted({i for st in stats for i in range(b.nprob) if not st[i]["converged"]})
    newton = [st[i]["newton_iters"] for st in stats for i in range(b.nprob)]
    pcg = [st[i]["pcg_iters_total"] / max(1, st[i]["newton_iters"]) for st in stats for i in range(b.nprob)]
    out = {"mode": "batch", "workload": "batch_cubes", "basis": basis, "precision": args.precision,
           "problems": b.nprob, "total_dofs": int(sum(b.ndofs)), "elements": int(sum(s_ ** 3 for s_ in side)),
           "steps": steps, "dt": dt, "wall_ms": ms, "ms_per_step": ms / steps,
           "matvec_dofs_per_s": dof_matvecs / (ms * 1e-3), "all_converged": conv,
           "failed": [{"i": i, "side": side[i], "P": orders[i], "E": E[i], "nu": nu[i]} for i in failed][:20],
           "newton_iters_mean": float(np.mean(newton)), "newton_iters_max": int(np.max(newton)),
           "pcg_iters_per_newton_mean": float(np.mean(pcg)), "pcg_iters_per_newton_max": float(np.max(pcg)),
           "gpu_launches": launches, "create_s": t_create,
           "tuning": [{"P": p_, "grid": g_, "tangent_ms": m_} for p_, g_, m_ in tuning],
           "persistent": b.persistent_info()}
    b.close()
    if not quiet:
        print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--basis", default=None,
                    choices=["nodal", "modal", "sdme_m", "sdme_k", "sdme_h", "nodal_lumped"],
                    help="default: the workload's basis (sdme_k for the quasi-static cantilever, else sdme_h)")
    ap.add_argument("--workload", default="beam_p8")
    ap.add_argument("--mixed-rtol", type=float, default=1e-4)
    ap.add_argument("--pcg-maxit", type=int, default=20000)
    ap.add_argument("--max-newton", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--ref-sample", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-extras", action="store_true",
                    help="also time the oracle on config 1 in full and a sampled internal force (minutes of CPU)")
    ap.add_argument("--kernel-only", action="store_true")
    ap.add_argument("--compare", action="store_true")
    ap.add_argument("--explicit", action="store_true")
    ap.add_argument("--explicit-steps", type=int, default=2000)
    ap.add_argument("--energy-every", type=int, default=50)
    ap.add_argument("--dt-iters", type=int, default=100)
    ap.add_argument("--bases", default="nodal,modal,sdme_m,sdme_h")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the basis / precision / unit-cube comparisons printed beside the default line")
    ap.add_argument("--compare-bases", default="nodal,modal,sdme_m,sdme_k,sdme_h")
    ap.add_argument("--compare-levels", type=int, default=5)
    ap.add_argument("--precisions", default="mixed,fp64")
    ap.add_argument("--kernel-iters", type=int, default=20)
    ap.add_argument("--tangent-grid", type=int, default=0,
                    help="CTAs of the PCG tangent launch: 0 one per element, -1 the resident CTAs, > 0 that many")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--forcing", type=int, default=1, choices=[0, 1],
                    help="1: Eisenstat-Walker forcing terms for the inner PCG tolerance (0: fixed tolerance)")
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--batch-load-scale", type=float, default=None)
    ap.add_argument("--batch-vs-sequential", type=int, default=0)
    ap.add_argument("--batch-persist", type=int, default=-1, choices=[-1, 0, 1],
                    help="batched PCG operator: 1 one persistent launch across orders, 0 one launch per order, "
                         "-1 as the tuner decides")
    ap.add_argument("--compare-batch-steps", type=int, default=3,
                    help="steps of the 256-cube batch in the comparison block (0: skip)")
    args = ap.parse_args()
    if args.batch and args.workload == "beam_p8":
        args.workload = "batch_cubes"
    if args.adjoint and args.workload == "beam_p8":
        args.workload = "beam_p6_adjoint"
    if args.explicit and args.workload == "beam_p8":
        args.workload = "cube_p6_explicit"
    w = workload(args.workload)
    if args.basis is None:
        args.basis = w.get("basis", "sdme_h")
    if args.batch:
        run_batch(args, w)
    elif args.adjoint:
        run_adjoint(args, w)
    elif args.kernel_only:
        run_kernel_only(args, w)
    elif args.compare:
        run_compare(args, w)
    elif args.explicit:
        run_explicit(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
