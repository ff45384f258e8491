"""Benchmark: time-to-1e-8 per system of a GMRES-SDR sequence on one GB300.

Workload: 3D convection-diffusion 128^3 (N = 2,097,152, 7-point upwind,
convection (20, 10, 5)); 20 systems A^(i) = A0 + i 1e-3 D with D = diag(U[0,1]),
b^(i) ~ N(0,1); m = 100, k = 20, t = 2, s = 480, zeta = 8, rel_tol 1e-8,
exact recycling (SAU recomputed for each new matrix).  One step = one system:
sdr_recycle(exact) + sdr_solve to ||b - A x|| < 1e-8 ||b||.

Output: one JSON line.  value = wall time per system on the device (CUDA
events, inputs resident in HBM); e2e = the same through the C ABI with the
system's inputs copied from pinned host memory and x copied back inside the
timed region.  roofline = the dominant kernel class, algorithmic bytes / CUDA
event time of its launches in the timed region.  cpu_baseline = the FP64 CPU
oracle on a bounded sample of the same workload (single thread).

--impl reference runs the oracle instead (host cores only).

--workload vcdiff_512_adjoint measures the adjoint form: ten gradient-descent
steps on L = ||x(theta) - x_t||^2 for the 512 x 512 variable-coefficient
operator, each a forward and an adjoint solve, with recycled spaces and from
cold starts.

--workload cd2d_batch64 measures the batched form: 64 independent 2D systems
(sides U{32..512}) x 5-system sequences, solved in lockstep and one at a time.

--workload cd3d_256_seq20_fp32ir measures the refined form instead: 3D
convection-diffusion 256^3 (N = 16,777,216), the same perturbed sequence,
m = 80, k = 20, s = 400, true relative residual 1e-10, solved by the float64
GPU path and by the float32 solver inside float64 refinement on the same
systems; value = the refined form's ms per system, with the float64 path's
time and the relative difference of the two solutions beside it.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="cd3d_128_seq20", n=128, conv=(20.0, 10.0, 5.0), systems=20, eps=1e-3,
                m=100, k=20, t=2, s=480, zeta=8, rel_tol=1e-8, seed=231114206)
METRIC = "time-to-1e-8 residual per system in sequence; cycle HBM GB/s vs ~8 TB/s peak"
UNIT = "ms/system"
# Arnoldi-step equivalents per system of this workload (Arnoldi steps + true-residual
# checks + k SpMVs of the exact recycling) used to scale the oracle's per-step time to
# a per-system time.  Measured on the GPU arm (the oracle's cycle counts agree within
# one cycle per system in the parity tests); overwritten by the GPU arm's own count
# whenever it runs in the same process.
STEP_EQUIV_PER_SYSTEM = 400
# DRAM bytes (read + write) per row of one k_spmv_dots launch, from an ncu capture of that
# kernel at 96^3 (dram__bytes_read.sum + dram__bytes_write.sum over three launches: 106.55 MB
# read and 0.78 to 4.23 MB written per launch, mean 108.6 MB, at 884,736 rows; the write
# share depends on when L2 writes w back); set to None when the kernel changes until it is
# captured again.
SPMV_DRAM_BYTES_PER_ROW = (106.552e6 + 2.058e6) / 884736


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", os.environ.get("LOCAL_RANK", "0")],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- inputs
def make_inputs(cfg):
    import numpy as np
    import workloads as W
    A0 = W.make_cd3d(cfg["n"], cfg["conv"])
    dvec = W.diag_perturbation(A0.n)
    rows = np.repeat(np.arange(A0.n), np.diff(A0.rowptr.astype(np.int64)))
    diag_pos = np.nonzero(A0.col.astype(np.int64) == rows)[0]
    return A0, dvec, diag_pos


def system_values(A0, dvec, diag_pos, i, eps):
    """Values of A^(i) = A0 + i eps D (same sparsity pattern as A0)."""
    v = A0.val.copy()
    v[diag_pos] += i * eps * dvec
    return v


# --------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world):
    import numpy as np
    import torch
    import workloads as W
    import paper_2311_14206_gb300 as P

    cfg = dict(WORKLOAD)
    if args.n:  # a smaller grid of the same workload (profiler captures)
        cfg["n"] = args.n
        cfg["workload"] = f"cd3d_{args.n}_seq{cfg['systems']}"
    if args.systems:
        cfg["systems"] = args.systems
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda")
    A0, dvec, diag_pos = make_inputs(cfg)
    N, nnz = A0.n, A0.nnz
    nsys = cfg["systems"]
    rowptr = torch.as_tensor(A0.rowptr, device=dev)
    col = torch.as_tensor(A0.col, device=dev)
    vals = [torch.as_tensor(system_values(A0, dvec, diag_pos, i + 1, cfg["eps"]), device=dev) for i in range(nsys)]
    # each replica solves its own right-hand sides (weak scaling)
    bs = [torch.as_tensor(W.rhs(N, replica_rhs_seed(rank, i)), device=dev) for i in range(nsys)]
    mats = [P.CSRDevice(N, rowptr, col, v) for v in vals]
    solver = P.Solver(N, cfg["m"], cfg["k"], cfg["t"], cfg["s"], cfg["zeta"], cfg["seed"], cfg["rel_tol"])
    xs = torch.zeros(N, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    seq = {"i": 0}

    def step(stats_out=None):
        i = seq["i"] % nsys
        A = mats[i]
        if seq["i"] > 0:
            solver.recycle(A, 0)
        xs.zero_()
        st, stats = P.sdr_solve(solver.h, A, bs[i], xs)
        if st != 0:
            raise RuntimeError(f"system {i}: status {st} {stats}")
        seq["i"] += 1
        if stats_out is not None:
            stats_out.append(stats)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    # ---- timed region: inputs resident in HBM, cycles replayed from CUDA graphs ----
    clocks = ClockSampler()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t_wall = time.perf_counter()
    stats_list = []
    launches = 0
    for _ in range(args.steps):
        step(stats_list)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    # kernels of this library in the timed region: the solves' own count plus four
    # kernels per recycled column of the exact SAU recomputation (the recycle
    # space a solve leaves is what the next system's recycle recomputes)
    launches = sum(s_["kernel_launches"] for s_ in stats_list) + 4 * sum(
        s_["recycle_dim"] for s_ in stats_list[:-1]) + 4 * stats_list[0]["recycle_dim"]
    # ---- per-kernel-class times: a separate pass with CUDA events around every launch ----
    P.sdr_profile(solver.h, True)
    if args.trace:
        P.sdr_trace(solver.h, 1 << 20)
    prof_stats = []
    for _ in range(min(args.steps, 3)):
        step(prof_stats)
    torch.cuda.synchronize()
    prof = P.sdr_profile_get(solver.h)
    if args.trace:
        with open(args.trace, "w") as f:
            f.write("class,stream,start_us,end_us\n")
            for c_, s_, t0_, t1_ in P.sdr_trace_get(solver.h):
                f.write(f"{c_},{s_},{t0_:.2f},{t1_:.2f}\n")
        P.sdr_trace(solver.h, 0)
    P.sdr_profile(solver.h, False)
    # ---- e2e: the same steps through the C ABI from pinned host buffers ----
    host_vals = [v.cpu().pin_memory() for v in vals]
    host_bs = [b.cpu().pin_memory() for b in bs]
    host_x = torch.empty(N, dtype=torch.float64).pin_memory()
    dval = torch.empty_like(vals[0])
    db = torch.empty_like(bs[0])
    dA = P.CSRDevice(N, rowptr, col, dval)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        i = seq["i"] % nsys
        dval.copy_(host_vals[i], non_blocking=True)
        db.copy_(host_bs[i], non_blocking=True)
        solver.recycle(dA, 0)
        xs.zero_()
        st, _ = P.sdr_solve(solver.h, dA, db, xs)
        host_x.copy_(xs, non_blocking=True)
        seq["i"] += 1
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = f0.elapsed_time(f1) / e2e_steps
    h2d = (vals[0].numel() + bs[0].numel()) * 8
    d2h = N * 8
    solver.close()

    # ---- roofline of the dominant kernel class ----
    agg = {k: 0 for k in ("steps", "checks", "cycles", "sau", "svd")}
    for s_ in prof_stats:
        agg["svd"] += s_["full_svd_cycles"]
        agg["steps"] += s_["arnoldi_steps"]
        agg["checks"] += s_["true_res_evals"]
        agg["cycles"] += s_["cycles"]
    m, t = cfg["m"], cfg["t"]
    mat_bytes = 12 * nnz + 4 * (N + 1)
    vec = 8 * N
    # spmv_dots: matrix + x gather + w write + (t-1) window reads (none at j = 0)
    steps_j0 = agg["cycles"]
    bytes_spmv = agg["steps"] * (mat_bytes + 2 * vec) + (agg["steps"] - steps_j0) * (t - 1) * vec
    # update_sketch: w and window reads + v_{j+1} write
    bytes_upd = agg["steps"] * (2 * vec) + (agg["steps"] - steps_j0) * (t - 1) * vec + steps_j0 * 0
    kprime = cfg["k"] + 1
    avg_d = (agg["steps"] / max(agg["cycles"], 1)) + kprime
    bytes_gemm = agg["cycles"] * vec * (avg_d + kprime)
    hbm, peak_kind = peaks()
    classes = {
        "spmv_dots": (bytes_spmv, "hbm"),
        "update_sketch": (bytes_upd, "hbm"),
        "recycle_gemm": (bytes_gemm, "hbm"),
    }
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    rf_name = dom if dom in classes else max(classes, key=lambda c: prof[c][1])
    rb, bound = classes[rf_name]
    rl, rms = prof[rf_name]
    achieved = rb / (rms * 1e-3) / 1e9 if rms > 0 else 0.0
    systems = args.steps
    agg_timed = {k: 0 for k in ("steps", "checks", "cycles", "svd")}
    for s_ in stats_list:
        agg_timed["svd"] += s_["full_svd_cycles"]
        agg_timed["steps"] += s_["arnoldi_steps"]
        agg_timed["checks"] += s_["true_res_evals"]
        agg_timed["cycles"] += s_["cycles"]
    # Whole-job algorithmic HBM bytes of the timed region: per Arnoldi step the SpMV
    # (matrix, x, window, w) and the update (w, window, v_hat); per check the tall
    # GEMV over [U V] and the residual (matrix, b, x_trial, r); per cycle the recycle
    # product ([U V] read, U_new written); per system the exact SAU (k SpMVs).
    d_avg = agg_timed["steps"] / max(agg_timed["cycles"], 1) + cfg["k"]
    job_bytes = (agg_timed["steps"] * (mat_bytes + vec * (t + 1) + vec * (t + 2))
                 + agg_timed["checks"] * (vec * (d_avg + 2) + mat_bytes + 3 * vec)
                 + agg_timed["cycles"] * vec * (d_avg + cfg["k"] + 1)
                 + systems * cfg["k"] * (mat_bytes + 2 * vec))
    cycle_gbs = job_bytes / (ms * 1e-3) / 1e9
    result = dict(ms=ms, wall=wall, clocks=ck, prof=prof, e2e_ms=e2e_ms, h2d=h2d, d2h=d2h, launches=launches,
                  roofline=dict(kernel=rf_name, bound=bound, achieved=achieved, peak=hbm,
                                peak_kind=peak_kind, unit="GB/s", frac=achieved / hbm,
                                bytes_per_launch=rb / max(rl, 1), launches=rl, ms_per_launch=rms / max(rl, 1),
                                traffic=(SPMV_DRAM_BYTES_PER_ROW * N if rf_name == "spmv_dots" else None)),
                  systems=systems, agg=agg_timed, N=N, nnz=nnz, workload=cfg["workload"],
                  cycle_hbm=dict(achieved=cycle_gbs, unit="GB/s", frac_of_measured=cycle_gbs / hbm,
                                 frac_of_8tbs=cycle_gbs / 8000.0, bytes_per_system=job_bytes / systems))
    return result


# --------------------------------------------------------------------------- refined form
F32IR = dict(workload="cd3d_256_seq20_fp32ir", n=256, conv=(20.0, 10.0, 5.0), systems=20, eps=1e-3,
             m=80, k=20, t=2, s=400, zeta=8, rel_tol=1e-10, inner_rel_tol=1e-4, seed=231114206)


def run_form_f32ir(args):
    """Time-to-1e-10 per system: float64 GPU path vs float32 + float64 refinement."""
    import torch
    import workloads as W
    import paper_2311_14206_gb300 as P

    cfg = F32IR
    dev = torch.device("cuda")
    A0, dvec, diag_pos = make_inputs(cfg)
    N, nnz = A0.n, A0.nnz
    rowptr = torch.as_tensor(A0.rowptr, device=dev)
    col = torch.as_tensor(A0.col, device=dev)
    nsys = args.warmup + args.steps
    vals = [torch.as_tensor(system_values(A0, dvec, diag_pos, i + 1, cfg["eps"]), device=dev) for i in range(nsys)]
    mats = [P.CSRDevice(N, rowptr, col, v, v.to(torch.float32)) for v in vals]
    bs = [torch.as_tensor(W.rhs(N, i), device=dev) for i in range(nsys)]
    stream = torch.cuda.current_stream()
    out = {}
    xs = {}
    for name, prec in (("fp64", P.SDR_PREC_F64), ("f32_refined", P.SDR_PREC_F32_REFINED)):
        solver = P.Solver(N, cfg["m"], cfg["k"], cfg["t"], cfg["s"], cfg["zeta"], cfg["seed"], cfg["rel_tol"],
                          precision=prec, inner_rel_tol=cfg["inner_rel_tol"])
        x = torch.zeros(N, dtype=torch.float64, device=dev)
        stats_list = []
        clocks = ClockSampler()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        xs[name] = []
        for i in range(nsys):
            if i == args.warmup:
                torch.cuda.synchronize()
                clocks.start()
                e0.record(stream)
            if i > 0:
                solver.recycle(mats[i], 0)
            x.zero_()
            st, stats = P.sdr_solve(solver.h, mats[i], bs[i], x)
            if st != 0:
                raise RuntimeError(f"{name} system {i}: status {st} {stats}")
            if i >= args.warmup:
                stats_list.append(stats)
                e1.record(stream)
                torch.cuda.synchronize()
                xs[name].append(x.clone())
                e0b = torch.cuda.Event(enable_timing=True)
                e0b.record(stream)
                out.setdefault(name + "_ms", []).append(e0.elapsed_time(e1))
                e0 = e0b
        ck = clocks.stop()
        if args.breakdown:
            # one more system with CUDA events around every launch (not part of the timing)
            P.sdr_profile(solver.h, True)
            solver.recycle(mats[0], 0)
            x.zero_()
            P.sdr_solve(solver.h, mats[0], bs[0], x)
            torch.cuda.synchronize()
            prof = P.sdr_profile_get(solver.h)
            P.sdr_profile(solver.h, False)
            tot = sum(v[1] for v in prof.values())
            print(f"{name}:", file=sys.stderr)
            for k_, (n_, t_) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:12]:
                print(f"  {k_:16s} launches {n_:7d}  {t_:10.2f} ms  {100 * t_ / max(tot, 1e-9):5.1f}%  "
                      f"{1e3 * t_ / max(n_, 1):9.2f} us/launch", file=sys.stderr)
        out[name] = dict(ms_per_system=sum(out[name + "_ms"]) / len(out[name + "_ms"]), clocks=ck,
                         cycles=sum(s_["cycles"] for s_ in stats_list) / len(stats_list),
                         refinements=sum(s_["refinements"] for s_ in stats_list) / len(stats_list),
                         arnoldi_steps=sum(s_["arnoldi_steps"] for s_ in stats_list) / len(stats_list),
                         final_rel_res=max(s_["final_rel_res"] for s_ in stats_list))
        solver.close()
    errs = [float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(xs["f32_refined"], xs["fp64"])]
    f32, f64 = out["f32_refined"], out["fp64"]
    return dict(
        metric="time-to-1e-10 true relative residual per system, float32 solver in float64 refinement",
        value=f32["ms_per_system"], unit="ms/system", n_gpus=1, steps=args.steps, warmup=args.warmup,
        ms_per_step=f32["ms_per_system"], higher_is_better=False, scaling="weak", vs_baseline=None,
        dtype="f32 (inner) / f64 (refinement, sketched QR, eigenproblem)", data="synthetic",
        config=dict(workload=cfg["workload"], N=N, nnz=nnz, m=cfg["m"], k=cfg["k"], t=cfg["t"], s=cfg["s"],
                    zeta=cfg["zeta"], rel_tol=cfg["rel_tol"], inner_rel_tol=cfg["inner_rel_tol"],
                    recycling="exact", l2="inputs larger than L2"),
        fp64_gpu=dict(ms_per_system=f64["ms_per_system"], cycles=f64["cycles"], arnoldi_steps=f64["arnoldi_steps"],
                      final_rel_res=f64["final_rel_res"]),
        refined=dict(refinements=f32["refinements"], inner_cycles=f32["cycles"], final_rel_res=f32["final_rel_res"]),
        speedup_vs_fp64=f64["ms_per_system"] / f32["ms_per_system"],
        x_rel_diff_vs_fp64=dict(max=max(errs), mean=sum(errs) / len(errs)),
        clocks=f32["clocks"])


# --------------------------------------------------------------------------- adjoint form
ADJ = dict(workload="vcdiff_512_adjoint", n=512, conv=(10.0, 10.0), theta_sd=0.5, opt_steps=10,
           m=60, k=15, t=2, s=300, zeta=8, rel_tol=1e-8, seed=231114206, lr=0.05)


def run_form_adjoint(args):
    """Ten gradient-descent steps on L = ||x(theta) - x_t||^2 at 512 x 512: each
    step a forward and an adjoint GMRES-SDR solve (autograd through SDRSolve),
    with the recycle spaces carried from step to step, and the same steps with
    every solve started from an empty recycle space."""
    import torch
    import workloads as W
    import paper_2311_14206_gb300 as P
    from paper_2311_14206_gb300.adjoint import solve
    from workloads.vcdiff_torch import vcdiff_pattern, vcdiff_values

    cfg = ADJ
    n = cfg["n"]
    N = n * n
    rp, cl = vcdiff_pattern(n)
    rp = torch.as_tensor(rp, device="cuda")
    cl = torch.as_tensor(cl, device="cuda")
    theta0 = torch.as_tensor(W.theta_field(n, cfg["theta_sd"]), device="cuda")
    b = torch.as_tensor(W.rhs(N, 0), device="cuda")
    x_t = torch.as_tensor(W.target_field(N) / (n + 1) ** 2, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    for mode in ("recycled", "cold"):
        pair = P.AdjointPair(N, rp, cl, cfg["m"], cfg["k"], cfg["t"], cfg["s"], cfg["zeta"], cfg["seed"],
                             cfg["rel_tol"])
        theta = theta0.clone()
        step_ms, losses, cyc = [], [], []
        scale = None
        for it in range(args.warmup + cfg["opt_steps"]):
            if mode == "cold":
                pair.fwd.recycle(None, 2)
                pair.adj.recycle(None, 2)
            th = theta.clone().requires_grad_(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            x = solve(vcdiff_values(n, th), b, pair)
            L = torch.sum((x - x_t) ** 2)
            L.backward()
            e1.record(stream)
            torch.cuda.synchronize()
            g = th.grad
            if scale is None:
                scale = float(g.abs().max())
            with torch.no_grad():
                theta -= cfg["lr"] * g / scale
            if it >= args.warmup:
                step_ms.append(e0.elapsed_time(e1))
                losses.append(float(L.detach()))
                cyc.append(pair.last_stats["forward"]["cycles"] + pair.last_stats["adjoint"]["cycles"])
        if args.breakdown and mode == "recycled":
            # one more step with CUDA events around every launch (not part of the timing)
            P.sdr_profile(pair.fwd.h, True)
            P.sdr_profile(pair.adj.h, True)
            th = theta.clone().requires_grad_(True)
            x = solve(vcdiff_values(n, th), b, pair)
            torch.sum((x - x_t) ** 2).backward()
            torch.cuda.synchronize()
            for name, hh in (("forward", pair.fwd.h), ("adjoint", pair.adj.h)):
                prof = P.sdr_profile_get(hh)
                tot = sum(v[1] for v in prof.values())
                _, logs = P.sdr_get_history(hh)
                sw = [g_["svd_sweeps"] for g_ in logs if g_["flags"] & 1]
                ndep = sum(1 for g_ in logs if g_["flags"] & 8)
                print(f"{name} solve: {pair.last_stats[name]['cycles']} cycles, "
                      f"{pair.last_stats[name]['arnoldi_steps']} steps, truncated-SVD cycles {len(sw)}, "
                      f"Jacobi sweeps {sum(sw) / max(len(sw), 1):.1f} mean / {max(sw) if sw else 0} max, "
                      f"ell {[g_['ell'] for g_ in logs][:6]}, cycles with a dependent eigenvector {ndep}",
                      file=sys.stderr)
                for k_, (n_, t_) in sorted(prof.items(), key=lambda kv: -kv[1][1])[:10]:
                    print(f"  {k_:16s} launches {n_:7d}  {t_:10.2f} ms  {100 * t_ / max(tot, 1e-9):5.1f}%  "
                          f"{1e3 * t_ / max(n_, 1):9.2f} us/launch", file=sys.stderr)
            P.sdr_profile(pair.fwd.h, False)
            P.sdr_profile(pair.adj.h, False)
        pair.close()
        out[mode] = dict(ms_per_opt_step=sum(step_ms) / len(step_ms), loss_first=losses[0], loss_last=losses[-1],
                         cycles_per_opt_step=sum(cyc) / len(cyc))
    r, c = out["recycled"], out["cold"]
    return dict(
        metric="time per optimisation step (forward + adjoint solve to 1e-8) with recycled spaces",
        value=r["ms_per_opt_step"], unit="ms/step", n_gpus=1, steps=cfg["opt_steps"], warmup=args.warmup,
        ms_per_step=r["ms_per_opt_step"], higher_is_better=False, scaling="weak", vs_baseline=None,
        dtype="f64", data="synthetic",
        config=dict(workload=cfg["workload"], N=N, m=cfg["m"], k=cfg["k"], t=cfg["t"], s=cfg["s"], zeta=cfg["zeta"],
                    rel_tol=cfg["rel_tol"], optimiser=f"gradient descent, step {cfg['lr']} / max|g_0|"),
        recycled=r, cold_start=c, speedup_vs_cold=c["ms_per_opt_step"] / r["ms_per_opt_step"])


# --------------------------------------------------------------------------- batched form
BATCH = dict(workload="cd2d_batch64", count=64, nmin=32, nmax=512, seq=5, eps=1e-3,
             m=40, k=10, t=2, s=100, zeta=8, rel_tol=1e-8, seed=231114206)


def run_form_batch(args):
    """64 independent 2D systems (sides U{32..512}, convection U[1,50]^2), each a
    5-system perturbed sequence with its own recycle space: all systems solved
    in lockstep by sdr_solve_batch (one stream pair per handle, cycles replayed
    from CUDA graphs), against the same solves issued one system at a time."""
    import numpy as np
    import torch
    import workloads as W
    import paper_2311_14206_gb300 as P

    cfg = BATCH
    specs = W.batch_systems(cfg["count"], cfg["nmin"], cfg["nmax"])
    mats, rhs, sizes = [], [], []
    for i, (n, conv) in enumerate(specs):
        A0 = W.make_cd2d(n, conv)
        dvec = W.diag_perturbation(A0.n, tag=i)
        rows = np.repeat(np.arange(A0.n), np.diff(A0.rowptr.astype(np.int64)))
        dpos = np.nonzero(A0.col.astype(np.int64) == rows)[0]
        rp = torch.as_tensor(A0.rowptr, device="cuda")
        cl = torch.as_tensor(A0.col, device="cuda")
        seq = []
        for j in range(cfg["seq"]):
            v = A0.val.copy()
            v[dpos] += (j + 1) * cfg["eps"] * dvec
            seq.append(P.CSRDevice(A0.n, rp, cl, torch.as_tensor(v, device="cuda")))
        mats.append(seq)
        rhs.append([torch.as_tensor(W.rhs(A0.n, 1000 * i + j), device="cuda") for j in range(cfg["seq"])])
        sizes.append(A0.n)
    out = {}
    for mode in ("batched", "one_at_a_time"):
        hs = [P.Solver(N, cfg["m"], cfg["k"], cfg["t"], cfg["s"], cfg["zeta"], cfg["seed"], cfg["rel_tol"],
                       stream=torch.cuda.Stream()) for N in sizes]
        xs = [torch.zeros(N, dtype=torch.float64, device="cuda") for N in sizes]
        handles = [h.h for h in hs]

        def run_seq(record):
            cyc, worst, conv = 0, 0.0, 0
            for j in range(cfg["seq"]):
                A_j = [m_[j] for m_ in mats]
                b_j = [r_[j] for r_ in rhs]
                for x in xs:
                    x.zero_()
                if mode == "batched":
                    if j > 0:
                        P.sdr_recycle_batch(handles, A_j, 0)
                    st, stats = P.sdr_solve_batch(handles, A_j, b_j, xs)
                else:
                    stats = []
                    for i, h in enumerate(hs):
                        if j > 0:
                            h.recycle(A_j[i], 0)
                        _, st1 = P.sdr_solve(h.h, A_j[i], b_j[i], xs[i])
                        stats.append(st1)
                if record:
                    cyc += sum(s_["cycles"] for s_ in stats)
                    worst = max(worst, max(s_["final_rel_res"] for s_ in stats))
                    conv += sum(s_["converged"] for s_ in stats)
            return cyc, worst, conv

        # warm-up: capture every handle's cycle graphs on the first system, then drop the recycle spaces
        run_seq(False)
        P.sdr_recycle_batch(handles, None, 2)
        torch.cuda.synchronize()
        clocks = ClockSampler()
        clocks.start()
        t0 = time.perf_counter()
        cyc, worst, conv = run_seq(True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[mode] = dict(total_s=wall, ms_per_solve=1e3 * wall / (cfg["count"] * cfg["seq"]), cycles=cyc,
                         converged_solves=conv, solves=cfg["count"] * cfg["seq"], max_final_rel_res=worst,
                         clocks=clocks.stop())
        for h in hs:
            h.close()
    b_, s_ = out["batched"], out["one_at_a_time"]
    return dict(
        metric="time per system solve to 1e-8, 64 independent systems x 5-system sequences",
        value=b_["ms_per_solve"], unit="ms/solve", n_gpus=1, steps=1, warmup=1, ms_per_step=1e3 * b_["total_s"],
        higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=cfg["workload"], systems=cfg["count"], sequence=cfg["seq"],
                    N_total=int(sum(sizes)), N_min=int(min(sizes)), N_max=int(max(sizes)), m=cfg["m"], k=cfg["k"],
                    t=cfg["t"], s=cfg["s"], zeta=cfg["zeta"], rel_tol=cfg["rel_tol"],
                    timing="host wall clock around the whole sequence (the solves synchronise every cycle)"),
        batched=b_, one_at_a_time=s_, speedup_vs_one_at_a_time=s_["total_s"] / b_["total_s"],
        clocks=b_["clocks"])


# --------------------------------------------------------------------------- the paper's Section 6.3 experiment
PAPER_CD = dict(workload="cd_paper_section_6_3", n=500, alpha=(0.0, 5.0, 20.0), m=80, k=20, t=2, s=480, zeta=8,
                rel_tol=1e-2, max_cycles=10, seed=231114206)
# the counts of the paper's table for this experiment (MATLAB, DCT sketch with s = 640), context only
PAPER_CD_TABLE = dict(gmres_sdr_exact=1971, gmres_sdr_inexact=1886)


def run_form_paper_cd(args):
    """The paper's Section 6.3 sequence (three 2D convection-diffusion problems,
    n = 500, alpha = 0, 5, 20, b = ones, 80 Arnoldi steps + 20 recycled, at most
    10 restarts, target 1e-2 relative) through the C ABI: exact recycling, the
    inexact variant and the inexact variant with the stale-SAU rule, with the
    sparse sign and with the paper's subsampled DCT (s = 480), and the paper's
    own configuration (the DCT at s = 640).  Reports products
    with A (Arnoldi steps + true-residual checks + the k products of each exact
    recycle, counted as the paper counts matrix-vector products) and the time
    per problem, beside the oracle's counts for the same runs."""
    import numpy as np
    import torch
    import workloads as W
    import paper_2311_14206_gb300 as P

    cfg = PAPER_CD
    As = [W.make_cd_paper(cfg["n"], a) for a in cfg["alpha"]]
    N = As[0].n
    mats = [P.CSRDevice.from_numpy(A) for A in As]
    b = torch.ones(N, dtype=torch.float64, device="cuda")
    gold = {}
    sketches = (("sparse_sign", 0, 480, "paper_cd_sparse_sign_s480.json"), ("dct", 1, 480, "paper_cd_dct_s480.json"),
                ("dct_s640", 1, 640, "paper_cd_dct_s640.json"))
    for sk, _, _, fname in sketches:
        path = os.path.join(ROOT, "tests", "golden", fname)
        if os.path.exists(path):
            with open(path) as f:
                gold[sk] = json.load(f)["variants"]
    runs = {}
    for sk, kind, s_, _ in sketches:
        for variant in ("exact", "inexact", "inexact_stale_check"):
            if kind == 1 and variant == "inexact_stale_check":
                continue
            solver = P.Solver(N, cfg["m"], cfg["k"], cfg["t"], s_, cfg["zeta"], cfg["seed"], cfg["rel_tol"],
                              max_cycles=cfg["max_cycles"], stale_check=variant == "inexact_stale_check",
                              sketch_kind=kind)
            if kind == 1:
                solver.set_sketch_draws(*W.dct_draws(cfg["seed"], N, s_))
            probs, total_mv, total_ms = [], 0, 0.0
            for rep in range(2):  # the first pass captures the cycle graphs
                probs, total_mv, total_ms = [], 0, 0.0
                solver.recycle(None, 2)
                for i, Ad in enumerate(mats):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    extra = 0
                    if i > 0:
                        kd = P.sdr_recycle_dim(solver.h)
                        solver.recycle(Ad, 0 if variant == "exact" else 1)
                        extra = kd if variant == "exact" else 0
                    x, st, stats = solver.solve(Ad, b)
                    torch.cuda.synchronize()
                    ms = 1e3 * (time.perf_counter() - t0)
                    mv = stats["arnoldi_steps"] + stats["true_res_evals"] + extra + stats["refresh_matvecs"]
                    probs.append(dict(converged=bool(stats["converged"]), cycles=stats["cycles"], matvecs=mv,
                                      rel_res=stats["final_rel_res"], ms=ms, sau_refreshes=stats["sau_refreshes"]))
                    total_mv += mv
                    total_ms += ms
            solver.close()
            ref = gold.get(sk, {}).get(variant)
            runs[f"{sk}/{variant}"] = dict(
                problems=probs, total_matvecs=total_mv, total_ms=total_ms,
                oracle_total_matvecs=ref["total_matvecs"] if ref else None,
                oracle_converged=[r_["converged"] for r_ in ref["problems"]] if ref else None)
    ex = runs["sparse_sign/exact"]
    return dict(
        metric="Section 6.3 sequence: time per problem and products with A", value=ex["total_ms"] / 3.0,
        unit="ms/system", n_gpus=1, steps=1, warmup=1, ms_per_step=ex["total_ms"], higher_is_better=False,
        scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=cfg["workload"], N=N, m=cfg["m"], k=cfg["k"], t=cfg["t"], s=cfg["s"],
                    zeta=cfg["zeta"], rel_tol=cfg["rel_tol"], max_cycles=cfg["max_cycles"],
                    timing="host wall clock per problem (each solve synchronises every cycle), second pass"),
        runs=runs, paper_table_matvecs=PAPER_CD_TABLE,
        note="the paper's counts were taken in MATLAB with a DCT sketch of s = 640 (its own draws); the "
             "dct_s640 runs use the same sketch family and size with this repository's draws; context, not a target")


# --------------------------------------------------------------------------- oracle arm
# Arnoldi steps of the bounded oracle sample: about 10-15 s of one host core on the GPU machine.
# The oracle's cost per step grows with the steps of its cycle (its basis is an N x (m+1)
# row-major array, so every column access strides over more memory), so a longer sample is
# also closer to the workload's m = 100 than a short one.
ORACLE_SAMPLE_STEPS = 32


def oracle_sample(steps=ORACLE_SAMPLE_STEPS, system=1):
    """Time the oracle on the first `steps` Arnoldi steps of one system of the
    workload (single thread) and return seconds per Arnoldi-step equivalent."""
    import numpy as np
    import workloads as W
    from oracle import sdr as osdr
    from oracle.sketch import SparseSign
    cfg = WORKLOAD
    A0, dvec, diag_pos = make_inputs(cfg)
    A = W.CSR(A0.n, A0.rowptr, A0.col, system_values(A0, dvec, diag_pos, system, cfg["eps"]))
    b = W.rhs(A.n, system)
    S = SparseSign(cfg["seed"], A.n, cfg["s"], cfg["zeta"])
    t0 = time.perf_counter()
    # a bounded cycle: `steps` Arnoldi steps with the true-residual check at the end
    c = osdr.cycle(A, b, None, None, None, S, cfg["rel_tol"] * np.linalg.norm(b), steps, cfg["t"], cfg["k"])
    dt = time.perf_counter() - t0
    return dt / (steps + 1), dict(steps=steps, seconds=dt)


def run_oracle_subprocess(steps=ORACLE_SAMPLE_STEPS):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; r = bench.oracle_sample(%d); "
            "print(json.dumps({'per_step': r[0], 'info': r[1]}))" % (ROOT, steps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(step_equiv):
    r = run_oracle_subprocess()
    per_system_ms = r["per_step"] * step_equiv * 1e3
    return dict(value=per_system_ms, unit=UNIT, cores=1, kind="oracle", extrapolated=True,
                sampled_step_equivalents=r["info"]["steps"] + 1, step_equivalents_per_system=step_equiv,
                sample=(f"FP64 numpy oracle, 1 thread: first {r['info']['steps']} Arnoldi steps of system 1 "
                        f"(N=2,097,152) plus one true-residual check took {r['info']['seconds']:.1f} s; "
                        f"scaled by {step_equiv:.0f} step-equivalents per system"))


def replica_rhs_seed(rank, i):
    """Seed of the right-hand side of system i on replica `rank`: every replica solves
    its own right-hand sides (weak scaling), distinct for i < 1000."""
    return 1000 * rank + i


def reduce_over_ranks(ms, e2e_ms, systems, world, device):
    """Whole-job times over `world` replicas.  ms: one replica's timed region (the
    `systems` solves); e2e_ms: its end-to-end time per system.  Both are maxed over the
    ranks (the slowest replica ends the job); every rank returns the same pair: ms per
    system of the whole job (all ranks' systems / the slowest region) and the
    end-to-end figure on the same footing."""
    if world == 1:
        return ms / systems, e2e_ms
    import torch
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t[0]) / (systems * world), float(t[1]) / world


def run_reference(args, rank, world):
    if rank != 0:
        return None
    per = []
    for _ in range(args.warmup):
        run_oracle_subprocess(4)  # warm-up: imports and caches only
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = run_oracle_subprocess(ORACLE_SAMPLE_STEPS)
        per.append(r["per_step"])
    wall = time.perf_counter() - t0
    value = statistics.mean(per) * STEP_EQUIV_PER_SYSTEM * 1e3
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=value, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD["workload"], N=2097152, m=100, k=20, t=2, s=480, zeta=8,
                            systems=20, rel_tol=1e-8),
                cpu_baseline=dict(kind="oracle", cores=1, value=value, unit=UNIT, extrapolated=True,
                                  sampled_step_equivalents=ORACLE_SAMPLE_STEPS + 1,
                                  step_equivalents_per_system=STEP_EQUIV_PER_SYSTEM,
                                  sample=(f"each step: FP64 numpy oracle (1 thread) on {ORACLE_SAMPLE_STEPS} Arnoldi "
                                          f"steps + one check of system 1, scaled by {STEP_EQUIV_PER_SYSTEM} "
                                          f"step-equivalents per system; {wall:.0f} s for the timed steps")),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--breakdown", action="store_true", help="print the per-kernel-class times to stderr")
    ap.add_argument("--trace", default="", help="write every launch of the per-kernel pass (class, stream, "
                    "start and end in us) to this CSV file")
    ap.add_argument("--n", type=int, default=0, help="grid side of a smaller case of the default workload "
                    "(for profiler captures; the bench line names it)")
    ap.add_argument("--systems", type=int, default=0, help="systems of the sequence kept on the device")
    ap.add_argument("--workload", default=WORKLOAD["workload"],
                    choices=[WORKLOAD["workload"], F32IR["workload"], ADJ["workload"], BATCH["workload"],
                             PAPER_CD["workload"]])
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    import torch
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        torch.distributed.init_process_group("nccl")
    import __graft_entry__ as g
    g.build()
    if args.workload in (F32IR["workload"], ADJ["workload"], BATCH["workload"], PAPER_CD["workload"]):
        if rank == 0:
            fn = {F32IR["workload"]: run_form_f32ir, ADJ["workload"]: run_form_adjoint,
                  BATCH["workload"]: run_form_batch, PAPER_CD["workload"]: run_form_paper_cd}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return
    res = run_gpu(args, rank, world)
    ms_per_system, e2e_per_system = reduce_over_ranks(res["ms"], res["e2e_ms"], res["systems"], world, "cuda")
    if rank == 0:
        agg = res["agg"]
        step_equiv = (agg["steps"] + agg["checks"] + WORKLOAD["k"] * res["systems"]) / max(res["systems"], 1)
        cpu = None if args.no_cpu_baseline else cpu_baseline(step_equiv)
        rf = res["roofline"]
        line = dict(
            metric=METRIC, value=ms_per_system, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=res["ms"] / res["systems"], higher_is_better=False, scaling="weak", vs_baseline=None,
            dtype="f64", data="synthetic",
            config=dict(workload=res["workload"], N=res["N"], nnz=res["nnz"], m=100, k=20, t=2, s=480,
                        zeta=8, systems=20, rel_tol=1e-8, recycling="exact", l2="inputs larger than L2",
                        parallelism=f"replicas{world}"),
            roofline=dict(bound=rf["bound"], achieved=rf["achieved"], peak=rf["peak"], unit=rf["unit"],
                          frac=rf["frac"], traffic=rf["traffic"], kernel=rf["kernel"],
                          peak_source=f"{rf['peak_kind']} HBM copy (MEASURED_PEAKS.json hbm_gbs)",
                          bytes_per_launch=rf["bytes_per_launch"], ms_per_launch=rf["ms_per_launch"]),
            clocks=res["clocks"],
            e2e=dict(value=e2e_per_system, unit=UNIT, h2d_bytes_per_step=res["h2d"], d2h_bytes_per_step=res["d2h"]),
            gpu_launches=res["launches"],
            cycle_hbm=res["cycle_hbm"],
            cpu_baseline=cpu,
            per_system=dict(arnoldi_steps=agg["steps"] / res["systems"], checks=agg["checks"] / res["systems"],
                            cycles=agg["cycles"] / res["systems"], svd_path_cycles=agg["svd"]),
        )
        if args.breakdown:
            tot = sum(v[1] for v in res["prof"].values())
            for k, (n, t) in sorted(res["prof"].items(), key=lambda kv: -kv[1][1]):
                print(f"  {k:16s} launches {n:7d}  {t:10.2f} ms  {100 * t / max(tot, 1e-9):5.1f}%  "
                      f"{1e3 * t / max(n, 1):9.2f} us/launch", file=sys.stderr)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
