"""Benchmark of the implicit-stage hot path on one GB300 per rank.

Workload (per rank): the 256 x 256 jittered periodic mesh of the synthetic
family (131,072 triangles, 196,608 edges), p = 3, dt = 1e-3, nu = 1e-3.  One
step is one implicit stage of the paper's pressure projection:
  b_S = G^T vhat                      (divergence of the dual velocity, eq. ins.1)
  b_c = sum_j U_ij^T vhat_c,j         (eq. d2m right-hand side, both components)
  S p = b_S                           (pressure Schur solve, eq. pressure_final)
  H vbar_c = b_c                      (viscous solves, eq. ad5 with lambda = nu)
all to relative residual 1e-10, FP32 inner CG under FP64 refinement.  vhat
is the Taylor-Green velocity sampled at the dual nodes plus seeded N(0, 1e-2)
noise.  Metric: CG DOF*iterations per second (all solves of the step).

Legs: the device-resident GPU leg (value), an end-to-end leg through the
C-ABI from pinned host buffers (e2e), one FP64-CG step (the one-solve-at-a-
time FP64 baseline), and the oracle timed on the host cores (cpu_baseline).
`--impl reference` times the oracle alone on the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(N=256, p=3, dt=1e-3, nu=1e-3, seed=0, noise=1e-2, tol=1e-10)
METRIC = "Schur-CG DOF*iters/s"
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes (read + write) per matrix row per CG iteration of the persistent
# CG kernel, from one ncu capture each (dram__bytes_read.sum +
# dram__bytes_write.sum over a 200-iteration launch at 256x256, p = 3, and
# 50-iteration launches at 1024x1024, p = 2 and p = 4; FP32 couplings).  Keyed
# by (p, precision); a kernel change invalidates it.
NCU_DRAM_BYTES_PER_ROW_ITER = {(3, "f32"): 171.1, (2, "f32"): 169.0, (4, "f32"): 290.9}


def workload_name(args):
    return (f"pressure Schur solve + velocity update + 2 viscous Helmholtz solves to 1e-10, {args.N}x{args.N} jittered "
            f"periodic mesh, p={args.p}")


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f32", "bf16", "f64"], default="f32")
    ap.add_argument("--N", type=int, default=WORKLOAD["N"])
    ap.add_argument("--p", type=int, default=WORKLOAD["p"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-precond", action="store_true",
                    help="skip the block-Jacobi preconditioned run of the same stage")
    ap.add_argument("--no-mg", action="store_true",
                    help="skip the multigrid preconditioned run of the same stage")
    ap.add_argument("--no-sl", action="store_true",
                    help="skip the semi-Lagrangian transport of the stage's velocity")
    ap.add_argument("--sl-dt", type=float, default=0.01)
    ap.add_argument("--sl-reps", type=int, default=100,
                    help="sl workload: transport calls per timed step")
    ap.add_argument("--c3-degrees", type=str, default="2,4")
    ap.add_argument("--workload", choices=["stage", "batch", "serve", "cg", "sl", "ns", "advdiff", "c3", "mg"],
                    default="stage",
                    help="stage: implicit stage (default line); batch: many solves in one launch; "
                         "serve: Poisson request sweep through the server; cg: one FP32 inner CG "
                         "launch capped at --cg-iters iterations (the case the profiles capture)")
    ap.add_argument("--cg-iters", type=int, default=200)
    ap.add_argument("--precond", action="store_true",
                    help="cg, batch and serve workloads: block-Jacobi preconditioned CG")
    ap.add_argument("--batch-solves", type=int, default=512)
    ap.add_argument("--batch-nmax", type=int, default=256)
    ap.add_argument("--batch-paths", type=str, default="multigrid",
                    help="comma list of engine, engine-bj, multigrid (each path's systems stay on the "
                         "operators: at the full 512-solve size run one path per process)")
    ap.add_argument("--batch-engine-iters", type=int, default=0,
                    help="batch workload: cap the engine paths at this many CG passes per refinement step and "
                         "one refinement (a throughput probe of the engine at full size: its solves stop unconverged)")
    ap.add_argument("--batch-split", action="store_true",
                    help="batch workload: also time the right-hand sides as one request each")
    ap.add_argument("--rhs", type=int, default=8)
    ap.add_argument("--serve-nmax", type=int, default=1024)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="serve workload: arrivals per rate at most (the window is shortened to about this "
                         "many requests at high rates; above the server's capacity they queue)")
    ap.add_argument("--serve-rates", type=str, default="10,30,100,300,1000,2000")
    ap.add_argument("--serve-precond", choices=["none", "block-jacobi", "multigrid"], default="multigrid")
    ap.add_argument("--serve-budget", type=float, default=150e9)
    ap.add_argument("--serve-sample-rate", type=float, default=10.0)
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving sample of the default line")
    ap.add_argument("--cpu-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-iters", type=int, default=10, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        under = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(under), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    """(rank, world, local_rank); NCCL only for the timing barrier / max."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return rank, world, local


def dual_velocity(op, seed):
    """Taylor-Green velocity at the dual nodes plus N(0, 1e-2) noise,
    [2][n_edge][n_psi] in the library's internal edge order."""
    import numpy as np
    from paper_2401_17806_gb300 import synth
    xy = op.node_coords(1)
    u, v = synth.taylor_green_velocity(xy[:, 0], xy[:, 1])
    noise = synth.standard_normal((2, op.n_dual), seed + 1, WORKLOAD["noise"])
    return np.stack([u, v]) + noise


def bytes_per_row_iter(nphi, coupling_bytes, vec_bytes, precond=False):
    """Algorithmic bytes per matrix row per CG iteration of the persistent
    kernel: the row's 4*N_phi coupling coefficients, its share of the column
    indices (4 int32 per triangle), and its vector accesses: 10 for plain CG
    (read p, x, r, w, s; write them), 12 with the block-Jacobi preconditioner
    (read p, x, u, r, w, s; write them) plus the row of P (N_phi values in the
    vector precision); the couplings are then those of A P, of the same size."""
    if precond:
        return 4 * nphi * coupling_bytes + nphi * vec_bytes + 16.0 / nphi + 12 * vec_bytes
    return 4 * nphi * coupling_bytes + 16.0 / nphi + 10 * vec_bytes


class Stage:
    """Device buffers and the calls of one implicit stage: divergence of the dual
    velocity, the two d2m right-hand sides, the pressure Schur solve, the velocity
    update of the projection and the two viscous Helmholtz solves."""

    def __init__(self, op, vhat_np, precision):
        import torch
        from paper_2401_17806_gb300 import dgsl
        self.op = op
        self.dgsl = dgsl
        n = op.n_dof
        self.vhat = torch.tensor(vhat_np.ravel(), dtype=torch.float64, device="cuda")
        self.bS = torch.empty(n, dtype=torch.float64, device="cuda")
        self.bH = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        self.p = torch.empty(n, dtype=torch.float64, device="cuda")
        self.vbar = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        self.vnew = torch.empty_like(self.vhat)
        prec = {"f32": dgsl.PREC_F32_IR, "bf16": dgsl.PREC_BF16_IR, "f64": dgsl.PREC_F64}[precision]
        self.opts = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=prec)

    def run(self, stream, opts=None):
        op, d = self.op, self.dgsl
        o = opts or self.opts
        op.dgsl_apply_div(self.vhat, self.bS, stream=stream)
        op.dgsl_project_d2m_rhs(self.vhat, self.bH, n_rhs=2, stream=stream)
        infos = op.dgsl_cg_solve(d.SCHUR, WORKLOAD["dt"], self.bS, self.p, opts=o, stream=stream)
        # velocity update of the projection (eq. nc.2): vnew = vhat - dt^2 Mhat^-1 G p
        op.dgsl_velocity_update(WORKLOAD["dt"] ** 2, self.vhat, self.p, self.vnew, stream=stream)
        infos += op.dgsl_cg_solve(d.HELMHOLTZ, WORKLOAD["nu"] * WORKLOAD["dt"], self.bH, self.vbar,
                                  n_rhs=2, opts=o, stream=stream)
        for i in infos:
            if i.status != d.OK:
                raise RuntimeError(f"solve failed: status {i.status}, relres {i.relres:.3e}")
        return infos


def gpu_leg(args, rank, world, local):
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(local)
    N, p = args.N, args.p
    seed = WORKLOAD["seed"] + rank
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    t0 = time.time()
    store = dgsl.STORE_F64 | dgsl.STORE_F32 | (dgsl.STORE_BF16 if args.precision == "bf16" else 0)
    op = dgsl.Operator(xy, tri, per, p, device=local, store=store, factored=True)
    build_s = time.time() - t0
    vhat = dual_velocity(op, seed)
    st = Stage(op, vhat, args.precision)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            st.run(stream)
    stream.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    l0 = dgsl.dgsl_launch_count()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            infos += st.run(stream)
        ev1.record(stream)
    stream.synchronize()
    barrier()
    clk = clocks.stop()
    launches = dgsl.dgsl_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    dof_iters = sum(op.n_dof * i.iters for i in infos)
    schur_iters = sum(i.iters for k, i in enumerate(infos) if k % 3 == 0)
    kern_ms = sum(i.cg_kernel_ms for i in infos)
    res = dict(ms=ms, dof_iters=dof_iters, schur_iters_per_step=schur_iters / args.steps,
               helm_iters_per_step=(sum(i.iters for i in infos) - schur_iters) / args.steps,
               refinements=sum(i.refinements for i in infos) / args.steps,
               relres_max=max(i.relres for i in infos), kern_ms=kern_ms, launches=launches,
               cg_launches=sum(i.cg_launches for i in infos), grid=infos[0].grid,
               clocks=clk, build_s=build_s, op=op, stage=st, stream=stream,
               iters_total=sum(i.iters for i in infos), device_bytes=op.device_bytes)
    # divergence of the projected velocity relative to that of the input (eq. nc.1)
    with torch.cuda.stream(stream):
        ydiv = torch.empty_like(st.bS)
        op.dgsl_apply_div(st.vnew, ydiv, stream=stream)
    stream.synchronize()
    res["div_rel"] = float(torch.linalg.norm(ydiv) / torch.linalg.norm(st.bS))
    # ---- end to end: pinned host input -> device, stage, device -> pinned host
    vh_host = torch.from_numpy(vhat.ravel().copy()).pin_memory()
    p_host = torch.empty(op.n_dof, dtype=torch.float64).pin_memory()
    v_host = torch.empty(2 * op.n_dof, dtype=torch.float64).pin_memory()
    vn_host = torch.empty(st.vnew.numel(), dtype=torch.float64).pin_memory()
    barrier()
    e_infos = []
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            st.vhat.copy_(vh_host, non_blocking=True)
            e_infos += st.run(stream)
            p_host.copy_(st.p, non_blocking=True)
            v_host.copy_(st.vbar, non_blocking=True)
            vn_host.copy_(st.vnew, non_blocking=True)
        ev1.record(stream)
    stream.synchronize()
    barrier()
    res["e2e_ms"] = ev0.elapsed_time(ev1)
    res["e2e_dof_iters"] = sum(op.n_dof * i.iters for i in e_infos)
    res["h2d"] = vh_host.numel() * 8
    res["d2h"] = (p_host.numel() + v_host.numel() + vn_host.numel()) * 8
    # ---- one-solve-at-a-time FP64 CG on the same stage
    if not args.no_fp64_baseline and args.precision != "f64":
        o64 = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F64)
        barrier()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            f_infos = st.run(stream, o64)
            ev1.record(stream)
        stream.synchronize()
        res["fp64"] = dict(ms=ev0.elapsed_time(ev1), iters=sum(i.iters for i in f_infos),
                           dof_iters=sum(op.n_dof * i.iters for i in f_infos),
                           kern_ms=sum(i.cg_kernel_ms for i in f_infos))
    # ---- the same stage with block-Jacobi preconditioned CG (an extension);
    # the first run builds and keeps the blocks of both systems
    if not args.no_precond:
        ob = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=st.opts.precision,
                             precond=dgsl.PRECOND_BLOCK_JACOBI)
        with torch.cuda.stream(stream):
            st.run(stream, ob)
        stream.synchronize()
        barrier()
        b_infos = []
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                b_infos += st.run(stream, ob)
            ev1.record(stream)
        stream.synchronize()
        bs = sum(i.iters for k, i in enumerate(b_infos) if k % 3 == 0)
        res["bj"] = dict(ms=ev0.elapsed_time(ev1), schur_iters=bs / args.steps,
                         helm_iters=(sum(i.iters for i in b_infos) - bs) / args.steps,
                         iters_total=sum(i.iters for i in b_infos),
                         kern_ms=sum(i.cg_kernel_ms for i in b_infos),
                         relres_max=max(i.relres for i in b_infos))
    # ---- the same stage with the two-level multigrid preconditioned CG (an
    # extension); the first run builds and keeps the hierarchies of both systems
    if not args.no_mg:
        om = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=st.opts.precision, precond=dgsl.PRECOND_MULTIGRID)
        t0 = time.time()
        with torch.cuda.stream(stream):
            st.run(stream, om)
        stream.synchronize()
        setup_s = time.time() - t0
        barrier()
        l1 = dgsl.dgsl_launch_count()
        m_infos = []
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                m_infos += st.run(stream, om)
            ev1.record(stream)
        stream.synchronize()
        ms_ = sum(i.iters for k, i in enumerate(m_infos) if k % 3 == 0)
        res["mg"] = dict(ms=ev0.elapsed_time(ev1), schur_iters=ms_ / args.steps,
                         helm_iters=(sum(i.iters for i in m_infos) - ms_) / args.steps,
                         refinements=sum(i.refinements for i in m_infos) / args.steps,
                         relres_max=max(i.relres for i in m_infos), first_run_s=setup_s,
                         launches_per_step=(dgsl.dgsl_launch_count() - l1) / args.steps)
        # the same multigrid stage in FP64 throughout (one untimed run builds
        # the FP64 hierarchies): the iterations the FP32 inner solves cost extra
        if args.precision != "f64":
            om64 = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F64, precond=dgsl.PRECOND_MULTIGRID)
            with torch.cuda.stream(stream):
                st.run(stream, om64)
                ev0.record(stream)
                f_infos = st.run(stream, om64)
                ev1.record(stream)
            stream.synchronize()
            res["mg"]["fp64"] = dict(ms=ev0.elapsed_time(ev1), schur_iters=f_infos[0].iters,
                                     helm_iters=sum(i.iters for i in f_infos[1:]),
                                     relres_max=max(i.relres for i in f_infos))
    # ---- semi-Lagrangian transport of the stage's main-grid velocity (two
    # components) by itself over dt, on the same mesh (Sec. 2.5, eq. intstage)
    if not args.no_sl:
        vb = st.vbar.clone()  # [2][n_dof]: the viscous solve's velocity
        cs = torch.empty_like(vb)
        ng = dgsl.sl_quadrature(op.p)[1].size
        stp = torch.zeros(op.n_tri * ng, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream):
            op.dgsl_sl_transport(WORKLOAD["dt"], vb, vb, cs, 2, steps=stp, stream=stream)
        stream.synchronize()
        reps = 20
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(reps):
                op.dgsl_sl_transport(WORKLOAD["dt"], vb, vb, cs, 2, stream=stream)
            ev1.record(stream)
        stream.synchronize()
        res["sl"] = dict(ms=ev0.elapsed_time(ev1) / reps, trajectories=op.n_tri * ng,
                         crossed=float(stp.sum().item()) / (op.n_tri * ng))
    return res


# ---------------------------------------------------------------- batch and serving legs

def fourier_rhs(op, seed, dt):
    """b = dt^2 Mbar f at the main nodes, f a 32-mode Fourier field (|k| <= 16,
    amplitude ~ |k|^-2); Mbar applied by the library (Helmholtz with nu_dt = 0)."""
    import torch
    from paper_2401_17806_gb300 import synth
    xy = torch.tensor(op.node_coords(0), device="cuda")
    k, amp, phase = synth.fourier_modes(seed)
    # the field sum evaluated on the device (synth.fourier_field's formula; the
    # host loop over 32 modes took minutes on the 10M-node pool meshes)
    fd = torch.zeros(xy.shape[0], dtype=torch.float64, device="cuda")
    tp = 2.0 * math.pi
    for (kx, ky), a, ph in zip(k, amp, phase):
        fd += float(a) * torch.cos(tp * (float(kx) * xy[:, 0] + float(ky) * xy[:, 1]) + float(ph))
    fd *= dt * dt
    b = torch.empty_like(fd)
    op.dgsl_apply_helmholtz(0.0, fd, b)
    return b


def cg_leg(args):
    """One persistent FP32 CG launch (Schur operator, dt = 1e-3, random right-hand
    side) capped at --cg-iters iterations on the N x N mesh, block-Jacobi
    preconditioned with --precond: the case the ncu summaries under profiles/
    capture.  Runs it twice (the first launch also builds the preconditioned
    operator) and prints the event-timed cost per iteration of the second."""
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    xy, tri, per = synth.jittered_periodic_mesh(args.N, WORKLOAD["seed"])
    op = dgsl.Operator(xy, tri, per, args.p, store=dgsl.STORE_F64 | dgsl.STORE_F32)
    b = torch.tensor(synth.standard_normal(op.n_dof, 1), device="cuda")
    x = torch.zeros_like(b)
    o = dgsl.solve_opts(tol=1e-30, max_iters=args.cg_iters, max_refine=1, precision=dgsl.PREC_F32_IR,
                        precond=dgsl.PRECOND_BLOCK_JACOBI if args.precond else dgsl.PRECOND_NONE)
    for _ in range(2):  # the first launch warms up (module load, attributes); the second is reported
        info = op.dgsl_cg_solve(dgsl.SCHUR, WORKLOAD["dt"], b, x, opts=o, check=False)[0]
    kind = "block-Jacobi preconditioned " if args.precond else ""
    print(json.dumps({"workload": f"one {kind}FP32 CG launch, {args.N}x{args.N}, p={args.p}", "iters": info.iters,
                      "grid": info.grid, "us_per_iter": 1e3 * info.cg_kernel_ms / max(1, info.iters)}))


def mg_leg(args):
    """One multigrid-preconditioned Schur solve (FP32 inner PCG under FP64
    refinement to 1e-10, Fourier right-hand side) on the N x N mesh, run
    twice (the first builds the hierarchy); prints the second's event-timed
    cost: the case the multigrid profiles capture."""
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    xy, tri, per = synth.jittered_periodic_mesh(args.N, WORKLOAD["seed"])
    op = dgsl.Operator(xy, tri, per, args.p)
    b = fourier_rhs(op, 11, WORKLOAD["dt"])
    x = torch.zeros_like(b)
    om = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F32_IR, precond=dgsl.PRECOND_MULTIGRID)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        x.zero_()
        torch.cuda.synchronize()
        l0 = dgsl.dgsl_launch_count()
        ev0.record()
        info = op.dgsl_cg_solve(dgsl.SCHUR, WORKLOAD["dt"], b, x, opts=om, check=False)[0]
        ev1.record()
        torch.cuda.synchronize()
    print(json.dumps({"workload": f"one multigrid PCG Schur solve, {args.N}x{args.N}, p={args.p}",
                      "status": info.status, "iters": info.iters, "refinements": info.refinements,
                      "relres": info.relres, "ms": ev0.elapsed_time(ev1),
                      "us_per_iter": 1e3 * ev0.elapsed_time(ev1) / max(1, info.iters),
                      "launches": dgsl.dgsl_launch_count() - l0}))


def c3_leg(args):
    """The precision configuration: 1024 x 1024 mesh, p = 2 and p = 4, Fourier
    right-hand side (32 modes, |k| <= 16, amplitude ~ |k|^-2, dt = 1e-3), the
    Schur system solved to relative residual 1e-10 under FP64 refinement with
    FP32 and with BF16 couplings (multigrid preconditioned PCG), and the
    persistent CG kernel's cost per iteration with each coupling type (one
    launch capped at --cg-iters iterations)."""
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    peak, peak_src = measured_hbm_peak()
    N = args.N if args.N != WORKLOAD["N"] else 1024
    out = []
    for p in [int(v) for v in args.c3_degrees.split(",")]:
        xy, tri, per = synth.jittered_periodic_mesh(N, WORKLOAD["seed"])
        t0 = time.time()
        op = dgsl.Operator(xy, tri, per, p, store=dgsl.STORE_F64 | dgsl.STORE_F32 | dgsl.STORE_BF16)
        build_s = time.time() - t0
        b = fourier_rhs(op, 11, WORKLOAD["dt"])
        for prec, name, cb in ((dgsl.PREC_F32_IR, "f32", 4), (dgsl.PREC_BF16_IR, "bf16", 2)):
            entry = {"p": p, "couplings": name, "n_dof": op.n_dof, "operator_build_s": build_s}
            # persistent CG kernel alone (plain, capped): the HBM roofline
            r = torch.tensor(synth.standard_normal(op.n_dof, 1), device="cuda")
            x = torch.zeros_like(r)
            oc = dgsl.solve_opts(tol=1e-30, max_iters=args.cg_iters, max_refine=1, precision=prec)
            for _ in range(2):
                ic = op.dgsl_cg_solve(dgsl.SCHUR, WORKLOAD["dt"], r, x, opts=oc, check=False)[0]
            per_row = bytes_per_row_iter(op.n_phi, cb, 4)
            us = 1e3 * ic.cg_kernel_ms / max(1, ic.iters)
            gbs = op.n_dof * per_row / (us * 1e-6) / 1e9
            entry["k_cg"] = {"us_per_iter": us, "bytes_per_row_iter": per_row, "achieved_gbs": gbs,
                             "frac": gbs / peak, "peak": peak, "peak_source": peak_src, "grid": ic.grid}
            tr = NCU_DRAM_BYTES_PER_ROW_ITER.get((p, name))
            if tr is not None:  # the DRAM traffic ncu measured for this kernel and size
                dram_gbs = op.n_dof * tr / (us * 1e-6) / 1e9
                entry["k_cg"].update({"ncu_dram_bytes_per_row_iter": tr, "dram_gbs": dram_gbs,
                                      "dram_frac": dram_gbs / peak})
            # the full solve with the multigrid preconditioner
            om = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=prec, precond=dgsl.PRECOND_MULTIGRID)
            x.zero_()
            t0 = time.time()
            op.dgsl_cg_solve(dgsl.SCHUR, WORKLOAD["dt"], b, x, opts=om, check=False)   # builds the hierarchy
            torch.cuda.synchronize()
            first_s = time.time() - t0
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.zero_()
            torch.cuda.synchronize()
            ev0.record()
            im = op.dgsl_cg_solve(dgsl.SCHUR, WORKLOAD["dt"], b, x, opts=om, check=False)[0]
            ev1.record()
            torch.cuda.synchronize()
            entry["multigrid_solve"] = {"status": "converged" if im.status == dgsl.OK else f"status {im.status}",
                                        "iters": im.iters, "refinements": im.refinements, "relres": im.relres,
                                        "ms": ev0.elapsed_time(ev1), "first_solve_s": first_s,
                                        "dof_iters_per_s": op.n_dof * im.iters / (ev0.elapsed_time(ev1) * 1e-3)}
            out.append(entry)
            print(json.dumps(entry), file=sys.stderr, flush=True)
        del op
        torch.cuda.empty_cache()
    print(json.dumps({"workload": f"precision: {N}x{N} mesh, Schur solve to 1e-10 under FP64 refinement",
                      "data": "synthetic", "results": out}))


def sl_flops(p, nf):
    """Algorithmic FP64 operations of the semi-Lagrangian walk (FMA = 2), with
    a polynomial of degree p evaluated by nested Horner (h = p(p+1)/2 + p
    FMAs): per cell visited, the reference coordinates (8), the two velocity
    components (4 h), the barycentric rates (6 + 3), the exit tests (9) and the
    move (8); per trajectory, the start point (8), the final reference
    coordinates (8), the fields at the foot (2 h nf) and its share of the
    projection (2 N_phi nf)."""
    nphi = (p + 1) * (p + 2) // 2
    h = p * (p + 1) // 2 + p
    per_visit = 8 + 4 * h + 9 + 9 + 8
    per_traj = 8 + 8 + 2 * h * nf + 2 * nphi * nf
    return per_visit, per_traj


def sl_leg(args):
    """Semi-Lagrangian transport (Sec. 2.5, eq. intstage) on the N x N mesh:
    the backward characteristic of every Gauss point over dt through the
    Taylor-Green velocity (nodal interpolation on the main grid), both
    velocity components transported.  Gauss-point trajectories per second,
    device-timed, inputs resident; the walk's FP64 operation rate against the
    GB300 FP64 peak."""
    import numpy as np
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    N, p, dt = args.N, args.p, args.sl_dt
    xy, tri, per = synth.jittered_periodic_mesh(N, WORKLOAD["seed"])
    op = dgsl.Operator(xy, tri, per, p, store=dgsl.STORE_F64)
    X = op.node_coords(0)
    tp = 2.0 * np.pi
    u = np.sin(tp * X[:, 0]) * np.cos(tp * X[:, 1])
    v = -np.cos(tp * X[:, 0]) * np.sin(tp * X[:, 1])
    vbar = torch.tensor(np.concatenate([u, v]), device="cuda")
    cstar = torch.empty_like(vbar)
    ng = dgsl.sl_quadrature(p)[1].size
    nt = op.n_tri * ng
    steps = torch.zeros(nt, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            op.dgsl_sl_transport(dt, vbar, vbar, cstar, 2, steps=steps, stream=stream)
    stream.synchronize()
    visits = float(steps.sum().item()) + nt  # cells visited: crossings + the first
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = dgsl.dgsl_launch_count()
    calls = args.steps * args.sl_reps
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(calls):
            op.dgsl_sl_transport(dt, vbar, vbar, cstar, 2, stream=stream)
        ev1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    launches = dgsl.dgsl_launch_count() - l0
    ms = ev0.elapsed_time(ev1) / calls
    pv, pt = sl_flops(p, 2)
    flops = pv * visits + pt * nt
    # the FP64 FMA rate measured on this device by the library's probe (the
    # walk is FP64-pipe bound); the nominal 1.25 TFLOP/s only if it fails
    try:
        peak = dgsl.dgsl_measure_fma_rate(fp64=True) / 1e9
        peak_src = "measured: dgsl_measure_fma_rate (event-timed FP64 FMA chains, 2 flop per FMA)"
    except dgsl.DgslError:
        peak, peak_src = 1250.0, "nominal GB300 FP64 rate (the probe failed)"
    line = {
        "metric": "semi-Lagrangian Gauss-point trajectories/s", "workload": "sl", "data": "synthetic",
        "value": nt / (ms * 1e-3), "unit": "trajectories/s", "ms_per_call": ms, "steps": args.steps,
        "calls_per_step": args.sl_reps,
        "warmup": args.warmup, "gpu_launches": launches, "dtype": "f64",
        "cells_crossed_per_trajectory": visits / nt - 1.0, "cell_visits_per_s": visits / (ms * 1e-3),
        "config": {"N": N, "p": p, "n_tri": op.n_tri, "gauss_points": ng, "trajectories": nt, "dt": dt,
                   "velocity": "Taylor-Green, nodal interpolation", "fields": 2,
                   "l2": "mesh records and fields (~%d MB) L2-resident; no flush (the walk re-reads them)"
                         % int((op.n_tri * (144 + 2 * 8 * op.n_phi * 3)) / 1e6)},
        "roofline": {"kernel": "k_sl_walk", "bound": "alu", "achieved": flops / (ms * 1e-3) / 1e9,
                     "peak": peak, "unit": "GFLOP/s (FP64)", "frac": flops / (ms * 1e-3) / 1e9 / peak,
                     "peak_source": peak_src,
                     "flops_per_cell_visit": pv, "flops_per_trajectory": pt},
        "clocks": clk,
        "stages": sl_stage_timings(op, vbar, cstar, dt, calls, stream, nt),
    }
    print(json.dumps(line))


def _tg_exact_feet(x0, dt, sub=400):
    """Backward characteristics of the Taylor-Green velocity over dt from the
    points x0 [m, 2], by classical RK4 with `sub` substeps (error ~1e-16)."""
    import numpy as np
    tp = 2.0 * np.pi

    def f(z):
        return -np.stack([np.sin(tp * z[:, 0]) * np.cos(tp * z[:, 1]),
                          -np.cos(tp * z[:, 0]) * np.sin(tp * z[:, 1])], axis=1)

    z, h = np.array(x0, dtype=np.float64), dt / sub
    for _ in range(sub):
        k1 = f(z)
        k2 = f(z + 0.5 * h * k1)
        k3 = f(z + 0.5 * h * k2)
        k4 = f(z + h * k3)
        z = z + h / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return z


def sl_stage_timings(op, vbar, cstar, dt, calls, stream, nt):
    """The stage-trajectory transport (dgsl_sl_transport_imex, R = 0, 1, 2) on
    the same mesh and fields: time per call at dt, and the feet's one-step
    error against the exact characteristics on 256 sampled Gauss points at
    dt = 0.16, 0.08, 0.04 (observed order = log2 of the ratios)."""
    import numpy as np
    import torch
    out = {}
    foot = torch.zeros(2 * nt, dtype=torch.float64, device="cuda")
    steps = torch.zeros(nt, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        op.dgsl_sl_transport_imex(0, 0.0, vbar, foot=foot, stream=stream)  # dt = 0: the Gauss points
    stream.synchronize()
    rng = np.random.default_rng(11)
    idx = rng.choice(nt, 256, replace=False)
    x0 = foot.view(nt, 2).cpu().numpy()[idx]
    for R in (0, 1, 2):
        with torch.cuda.stream(stream):
            op.dgsl_sl_transport_imex(R, dt, vbar, vbar, cstar, 2, steps=steps, stream=stream)
        stream.synchronize()
        crossed = float(steps.sum().item()) / nt
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(calls):
                op.dgsl_sl_transport_imex(R, dt, vbar, vbar, cstar, 2, stream=stream)
            ev1.record(stream)
        stream.synchronize()
        ms = ev0.elapsed_time(ev1) / calls
        errs = []
        for h in (0.16, 0.08, 0.04):
            with torch.cuda.stream(stream):
                op.dgsl_sl_transport_imex(R, h, vbar, foot=foot, stream=stream)
            stream.synchronize()
            d = foot.view(nt, 2).cpu().numpy()[idx] - _tg_exact_feet(x0, h)
            errs.append(float(np.abs(d - np.round(d)).max()))
        out["R%d" % R] = {"ms_per_call": ms, "trajectories_per_s": nt / (ms * 1e-3),
                          "cells_crossed_per_trajectory": crossed,
                          "one_step_foot_error": {"dt": [0.16, 0.08, 0.04], "max_abs": errs,
                                                  "observed_order": [float(np.log2(errs[0] / errs[1])),
                                                                     float(np.log2(errs[1] / errs[2]))]}}
    return out


def ns_leg(args):
    """First-order semi-Lagrangian Navier-Stokes steps (dgsl_ns_step) of the
    Taylor-Green vortex on the N x N mesh (dt = 1e-3, nu = 1e-3, FP32 inner CG
    under FP64 refinement to 1e-10, block-Jacobi preconditioned, the pressure
    solve started from the extrapolation of the last two steps' pressures):
    steps per second, device-timed.  Then the temporal order on a 64 x 64, p = 2 mesh:
    the error against the exact decay exp(-8 pi^2 nu t) at t = 0.1 for dt =
    0.05, 0.025, 0.0125 (nu = 0.01).  Key "imex": the SL-IMEX stages
    (dgsl_ns_imex_step) for R = 1, 2 timed the same way, and their temporal
    order (R = 0, 1, 2) on 32 x 32, p = 3 with 2, 4, 8 and 16 steps."""
    import numpy as np
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    tp = 2.0 * np.pi

    def tg_dual(op):
        X = op.node_coords(1)
        return torch.tensor(np.concatenate([np.sin(tp * X[:, 0]) * np.cos(tp * X[:, 1]),
                                            -np.cos(tp * X[:, 0]) * np.sin(tp * X[:, 1])]), device="cuda")

    N, p = args.N, args.p
    op = dgsl.Operator(*synth.jittered_periodic_mesh(N, WORKLOAD["seed"]), p, factored=True)
    # the pressure solve starts from the extrapolation 2 p^n - p^{n-1} of the last two steps' pressures
    opts = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F32_IR, precond=dgsl.PRECOND_BLOCK_JACOBI,
                           use_x0=2)
    v = tg_dual(op)
    pr = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        op.dgsl_ns_step(WORKLOAD["dt"], WORKLOAD["nu"], v, v, pr, opts=opts)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    clocks.start()
    l0 = dgsl.dgsl_launch_count()
    infos = []
    ev0.record()
    for _ in range(args.steps):
        infos += op.dgsl_ns_step(WORKLOAD["dt"], WORKLOAD["nu"], v, v, pr, opts=opts)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = dgsl.dgsl_launch_count() - l0
    # temporal order (the exact Taylor-Green decay)
    opo = dgsl.Operator(*synth.jittered_periodic_mesh(64, 3), 2, factored=True)
    o2 = dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F32_IR, precond=dgsl.PRECOND_BLOCK_JACOBI)
    v0 = tg_dual(opo)
    nu, T = 0.01, 0.1
    ref = v0 * np.exp(-8.0 * np.pi ** 2 * nu * T)
    errs = []
    for n in (2, 4, 8):
        w = v0.clone()
        for _ in range(n):
            opo.dgsl_ns_step(T / n, nu, w, w, opts=o2)
        errs.append(float(torch.linalg.norm(w - ref) / torch.linalg.norm(ref)))
    # the SL-IMEX stages (dgsl_ns_imex_step): time per step on the same mesh, order on 32 x 32, p = 3
    imex = {}
    for R in (1, 2):
        v = tg_dual(op)
        pr = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            op.dgsl_ns_imex_step(R, WORKLOAD["dt"], WORKLOAD["nu"], v, v, pr, opts=opts)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        its = 0
        for _ in range(args.steps):
            its += sum(i.iters for i in op.dgsl_ns_imex_step(R, WORKLOAD["dt"], WORKLOAD["nu"], v, v, pr, opts=opts))
        e1.record()
        torch.cuda.synchronize()
        imex["R%d" % R] = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "cg_iters_per_step": its / args.steps}
    op3 = dgsl.Operator(*synth.jittered_periodic_mesh(32, 3), 3, factored=True)
    o3 = dgsl.solve_opts(tol=1e-11, precision=dgsl.PREC_F64, precond=dgsl.PRECOND_BLOCK_JACOBI)
    w0 = tg_dual(op3)
    ref3 = w0 * np.exp(-8.0 * np.pi ** 2 * nu * T)
    for R in (0, 1, 2):
        ierrs = []
        for n in (2, 4, 8, 16):
            w = w0.clone()
            for _ in range(n):
                op3.dgsl_ns_imex_step(R, T / n, nu, w, w, opts=o3)
            ierrs.append(float(torch.linalg.norm(w - ref3) / torch.linalg.norm(ref3)))
        imex.setdefault("temporal_order", {"mesh": "32x32, p=3", "nu": nu, "t": T,
                                           "dt": [T / 2, T / 4, T / 8, T / 16]})["R%d" % R] = {
            "rel_error": ierrs, "observed_order": [float(np.log2(ierrs[k] / ierrs[k + 1])) for k in range(3)]}
    print(json.dumps({
        "metric": "first-order semi-Lagrangian Navier-Stokes steps/s", "workload": "ns", "data": "synthetic",
        "value": 1e3 / ms, "unit": "steps/s", "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
        "gpu_launches": launches, "dtype": "f32+f64",
        "schur_iters_per_step": sum(i.iters for k, i in enumerate(infos) if k % 3 == 2) / args.steps,
        "helmholtz_iters_per_step": sum(i.iters for k, i in enumerate(infos) if k % 3 != 2) / args.steps,
        "config": {"N": N, "p": p, "n_dof": op.n_dof, "dt": WORKLOAD["dt"], "nu": WORKLOAD["nu"],
                   "tol": WORKLOAD["tol"], "initial": "Taylor-Green vortex (nodal on the dual grid)",
                   "solves": "FP32 inner CG, FP64 refinement, block-Jacobi; pressure started from 2 p^n - p^(n-1)"},
        "temporal_order": {"mesh": "64x64, p=2", "nu": nu, "t": T, "dt": [T / 2, T / 4, T / 8], "rel_error": errs,
                           "observed_order": [float(np.log2(errs[0] / errs[1])), float(np.log2(errs[1] / errs[2]))]},
        "clocks": clk,
        "imex": imex,
    }))


def advdiff_leg(args):
    """SL-IMEX steps of the advection-diffusion model (dgsl_advdiff_step) on the
    N x N mesh: a scalar carried by the steady Taylor-Green velocity and
    diffused (alpha = 1e-3, dt = 0.01, block-Jacobi FP32 inner CG under FP64
    refinement to 1e-10), steps per second for R = 0, 1, 2, device-timed.  Then the global
    order in time on 48 x 48, p = 4: the exact solution exp(-alpha |k|^2 t)
    sin(k.(x - V t)) for a constant V (alpha = 0.2, k = (2 pi, 0)) at t = 0.2
    with dt = 0.05, 0.025, 0.0125."""
    import numpy as np
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    N, p = args.N, args.p
    op = dgsl.Operator(*synth.jittered_periodic_mesh(N, WORKLOAD["seed"]), p)
    X = op.node_coords(0)
    tp = 2.0 * np.pi
    vb = torch.tensor(np.concatenate([np.sin(tp * X[:, 0]) * np.cos(tp * X[:, 1]),
                                      -np.cos(tp * X[:, 0]) * np.sin(tp * X[:, 1])]), device="cuda")
    c0 = torch.tensor(np.exp(-20.0 * ((X[:, 0] - 0.5) ** 2 + (X[:, 1] - 0.5) ** 2)), device="cuda")
    opts = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F32_IR, precond=dgsl.PRECOND_BLOCK_JACOBI)
    dt, alpha = 0.01, 1e-3
    clocks = ClockSampler(0)
    clocks.start()
    legs = {}
    for R in (0, 1, 2):
        c = c0.clone()
        for _ in range(args.warmup):
            op.dgsl_advdiff_step(R, dt, alpha, vb, c, c, opts=opts)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = dgsl.dgsl_launch_count()
        iters = 0
        ev0.record()
        for _ in range(args.steps):
            iters += sum(i.iters for i in op.dgsl_advdiff_step(R, dt, alpha, vb, c, c, opts=opts))
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        legs["R%d" % R] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "cg_iters_per_step": iters / args.steps,
                           "gpu_launches_per_step": (dgsl.dgsl_launch_count() - l0) / args.steps}
    clk = clocks.stop()
    # global order in time
    opo = dgsl.Operator(*synth.jittered_periodic_mesh(48, 3), 4)
    Xo = opo.node_coords(0)
    V = np.array([0.8, 0.5])
    k = np.array([tp, 0.0])
    a2 = 0.2
    lam = a2 * (k @ k)
    vo = torch.tensor(np.concatenate([np.full(opo.n_dof, V[0]), np.full(opo.n_dof, V[1])]), device="cuda")
    # (FP64 bottoms out near 1e-12 on these Helmholtz systems; 1e-11 is far below the errors measured)
    o2 = dgsl.solve_opts(tol=1e-11, precision=dgsl.PREC_F64, precond=dgsl.PRECOND_BLOCK_JACOBI)
    T = 0.2
    order = {}
    for R in (0, 1, 2):
        errs = []
        for nstep in (4, 8, 16):
            c = torch.tensor(np.sin(Xo @ k), device="cuda")
            for _ in range(nstep):
                opo.dgsl_advdiff_step(R, T / nstep, a2, vo, c, c, opts=o2)
            ex = np.exp(-lam * T) * np.sin(Xo @ k - (k @ V) * T)
            errs.append(float(np.abs(c.cpu().numpy() - ex).max()))
        order["R%d" % R] = {"max_abs_error": errs,
                            "observed_order": [float(np.log2(errs[0] / errs[1])), float(np.log2(errs[1] / errs[2]))]}
    r2 = legs["R2"]
    print(json.dumps({
        "metric": "SL-IMEX advection-diffusion steps/s (R = 2)", "workload": "advdiff", "data": "synthetic",
        "value": r2["steps_per_s"], "unit": "steps/s", "ms_per_step": r2["ms_per_step"], "steps": args.steps,
        "warmup": args.warmup, "dtype": "f32+f64", "by_R": legs,
        "config": {"N": N, "p": p, "n_dof": op.n_dof, "dt": dt, "alpha": alpha, "tol": WORKLOAD["tol"],
                   "velocity": "Taylor-Green, steady", "initial": "Gaussian bump",
                   "solves": "Helmholtz per stage: FP32 inner CG, FP64 refinement, block-Jacobi, started from the stage value"},
        "temporal_order": {"mesh": "48x48, p=4", "alpha": a2, "V": V.tolist(), "k": k.tolist(), "t": T,
                           "dt": [T / 4, T / 8, T / 16], **order},
        "clocks": clk,
    }))


def engine_bytes_per_row_pass(nphi, cb, R):
    """Algorithmic bytes per matrix row per CG pass of the batched engine for a
    request with R right-hand sides: the row's 4 N_phi couplings and its share
    of the column indices (both shared by the R right-hand sides) and 10 FP32
    vector accesses per right-hand side."""
    return 4 * nphi * cb + 16.0 / nphi + 10 * 4 * R


def batch_leg(args):
    """The batching configuration: independent Schur solves of random meshes
    (N uniform in 8..nmax, p uniform in 1..4, per-solve seeds), each with R
    Fourier right-hand sides, all in ONE call: the persistent engine (one
    cooperative launch; plain or block-Jacobi CG) and the multigrid path
    (concurrent solves on worker streams); versus one-solve-at-a-time FP64 CG
    on a sample of the right-hand sides."""
    import numpy as np
    import torch
    from paper_2401_17806_gb300 import build, dgsl, synth
    build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(1234)
    nsol, R, dt = args.batch_solves, args.rhs, WORKLOAD["dt"]
    Ns = rng.integers(8, args.batch_nmax + 1, nsol)
    ps = rng.integers(1, 5, nsol)
    store = dgsl.STORE_F64 | dgsl.STORE_F32 | (dgsl.STORE_BF16 if args.precision == "bf16" else 0)
    t0 = time.time()
    ops = build_operators([(N, p, 1000 + i) for i, (N, p) in enumerate(zip(Ns, ps))], store)
    build_s = time.time() - t0
    reqs, split, bufs = [], [], []
    for i, op in enumerate(ops):
        b = torch.cat([fourier_rhs(op, 5000 + i * R + j, dt) for j in range(R)])
        x = torch.zeros_like(b)
        xs = torch.zeros_like(b) if args.batch_split else None
        bufs.append((op, b, x, xs))  # requests hold raw pointers: keep every tensor alive
        reqs.append(dgsl.request(op, dgsl.SCHUR, dt, b, x, n_rhs=R))
        n = op.n_dof
        if args.batch_split:
            split += [dgsl.request(op, dgsl.SCHUR, dt, b[j * n:(j + 1) * n], xs[j * n:(j + 1) * n])
                      for j in range(R)]
    prec = dgsl.PREC_BF16_IR if args.precision == "bf16" else dgsl.PREC_F32_IR
    cb = 2 if args.precision == "bf16" else 4
    peak, peak_src = measured_hbm_peak()

    def timed(rs, opts):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = dgsl.dgsl_launch_count()
        ev0.record()
        out = dgsl.dgsl_cg_solve_batch(rs, opts)
        ev1.record()
        torch.cuda.synchronize()
        return out, ev0.elapsed_time(ev1), dgsl.dgsl_launch_count() - l0

    result = {}
    for name in args.batch_paths.split(","):
        pc = {"engine": dgsl.PRECOND_NONE, "engine-bj": dgsl.PRECOND_BLOCK_JACOBI,
              "multigrid": dgsl.PRECOND_MULTIGRID}[name]
        capped = args.batch_engine_iters > 0 and pc != dgsl.PRECOND_MULTIGRID
        opts = (dgsl.engine_opts(precision=prec, precond=pc, max_iters=args.batch_engine_iters, max_refine=1)
                if capped else dgsl.engine_opts(precision=prec, precond=pc))
        t = time.perf_counter()
        if pc != dgsl.PRECOND_NONE:  # build every system's preconditioner once, outside the timing
            dgsl.dgsl_cg_solve_batch(reqs, dgsl.engine_opts(precision=prec, precond=pc, max_iters=1, max_refine=1))
        else:
            dgsl.dgsl_cg_solve_batch(reqs[:2], opts)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t
        infos, ms, launches = timed(reqs, opts)
        iters = sorted(i.iters for i in infos)
        entry = {"solves_per_s": nsol / (ms * 1e-3), "rhs_solves_per_s": nsol * R / (ms * 1e-3), "ms_total": ms,
                 "converged": int(sum(i.status == dgsl.OK for i in infos)), "requests": nsol,
                 "iters_p50": iters[len(iters) // 2], "iters_max": iters[-1],
                 "max_relres": max(i.relres for i in infos), "gpu_launches": launches,
                 "preconditioner_setup_s": setup_s}
        if capped:
            entry["capped_passes"] = args.batch_engine_iters
            entry["note"] = "throughput probe: every solve stops after the capped passes (not converged)"
        if name == "engine":
            # the engine's algorithmic bytes: every request's passes over its couplings
            alg = sum(i.iters * op.n_dof * engine_bytes_per_row_pass(op.n_phi, cb, R) for i, op in zip(infos, ops))
            entry["engine_achieved_gbs"] = alg / (ms * 1e-3) / 1e9
            entry["engine_frac"] = entry["engine_achieved_gbs"] / peak
            entry["bytes_per_row_pass_per_rhs"] = float(np.mean([engine_bytes_per_row_pass(op.n_phi, cb, R) / R
                                                                 for op in ops]))
            entry["peak_source"] = peak_src
            if args.batch_split:
                sinfos, ms_split, _ = timed(split, opts)
                entry["split_rhs_solves_per_s"] = nsol * R / (ms_split * 1e-3)
                entry["multi_rhs_speedup"] = ms_split / ms
        result[name] = entry
        print(json.dumps({name: entry}), file=sys.stderr, flush=True)
    # one-solve-at-a-time FP64 CG on a sample of the same right-hand sides
    sample = rng.choice(nsol * R, size=min(16, nsol * R), replace=False)
    o64 = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F64)
    t64 = 0.0
    for k in sample:
        op, b, _, _ = bufs[k // R]
        n = op.n_dof
        bk = b[(k % R) * n:(k % R + 1) * n].clone()
        x = torch.zeros_like(bk)
        torch.cuda.synchronize()
        t = time.perf_counter()
        op.dgsl_cg_solve(dgsl.SCHUR, dt, bk, x, opts=o64, check=False)
        torch.cuda.synchronize()
        t64 += time.perf_counter() - t
    base_rate = len(sample) / t64
    for e in result.values():
        e["speedup_vs_fp64_one_at_a_time"] = e["rhs_solves_per_s"] / base_rate
    print(json.dumps({
        "metric": "batched Schur solves/s", "workload": "batch", "data": "synthetic",
        "dtype": {"bf16": "bf16+f32+f64"}.get(args.precision, "f32+f64"),
        "config": {"solves": nsol, "rhs_per_solve": R, "N_range": [8, args.batch_nmax], "p_range": [1, 4],
                   "tol": WORKLOAD["tol"], "dt": dt, "operator_build_s": build_s,
                   "total_dof": int(sum(op.n_dof for op in ops))},
        "paths": result,
        "fp64_one_at_a_time": {"rhs_solves_per_s": base_rate, "sample_rhs": len(sample)}}))


SERVE_SIZES = (16, 32, 64, 128, 256, 512, 1024)


def build_operators(specs, store=None):
    """dgsl.Operator for every (N, p, seed) of specs, built by host threads
    (the C-ABI build releases the interpreter lock); returns them in order."""
    import concurrent.futures as cf
    from paper_2401_17806_gb300 import dgsl, synth
    st = store if store is not None else 0

    def one(spec):
        N, p, seed = spec
        return dgsl.Operator(*synth.jittered_periodic_mesh(int(N), int(seed)), int(p), store=st)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, specs))


def serve_pool(sizes, dt):
    """One operator per (N, p) of the pool (p = 1..4) and 8 Fourier right-hand
    sides each."""
    import torch
    keys = [(N, p) for N in sizes for p in range(1, 5)]
    ops = build_operators([(N, p, 300 + N + p) for N, p in keys])
    pool = {}
    for (N, p), op in zip(keys, ops):
        rhs = torch.cat([fourier_rhs(op, 9000 + 10 * N + 8 * p + j, dt) for j in range(8)])
        pool[(N, p)] = (op, rhs)
    return pool


def fp64_service_times(pool, dt, full_nmax=256, cap=200):
    """Service time of one Schur solve to 1e-10 by one-at-a-time FP64 CG
    (unpreconditioned, the paper's solver) for every pool operator: measured
    in full for N <= full_nmax; above it, the measured cost of one iteration
    (a capped solve) times the iteration count of the same degree at
    full_nmax scaled by N / full_nmax (CG iterations grow like 1/h)."""
    import torch
    from paper_2401_17806_gb300 import dgsl
    o64 = dgsl.solve_opts(tol=WORKLOAD["tol"], precision=dgsl.PREC_F64)
    svc, how, iters = {}, {}, {}
    for (N, p), (op, rhs) in sorted(pool.items()):
        b0 = rhs[:op.n_dof].clone()
        x = torch.zeros_like(b0)
        if N <= full_nmax:
            torch.cuda.synchronize()
            t = time.perf_counter()
            info = op.dgsl_cg_solve(dgsl.SCHUR, dt, b0, x, opts=o64, check=False)[0]
            torch.cuda.synchronize()
            svc[(N, p)] = time.perf_counter() - t
            iters[(N, p)] = info.iters
            how[(N, p)] = "measured"
        else:
            oc = dgsl.solve_opts(tol=1e-30, precision=dgsl.PREC_F64, max_iters=cap, max_refine=1)
            op.dgsl_cg_solve(dgsl.SCHUR, dt, b0, x, opts=oc, check=False)
            torch.cuda.synchronize()
            t = time.perf_counter()
            info = op.dgsl_cg_solve(dgsl.SCHUR, dt, b0, x, opts=oc, check=False)[0]
            torch.cuda.synchronize()
            per_iter = (time.perf_counter() - t) / max(1, info.iters)
            ref = max(n for n in pool if n[1] == p and n[0] <= full_nmax)
            est = iters[ref] * N / ref[0]
            svc[(N, p)] = per_iter * est
            iters[(N, p)] = est
            how[(N, p)] = f"extrapolated: {per_iter * 1e3:.3f} ms/iteration x {est:.0f} iterations"
    return svc, how, iters


def serve_trace(pool, svc, rate, seconds, seed, precond, budget, nmax, max_rhs=8):
    """One open-loop Poisson trace through the server (multi-RHS requests:
    N log-uniform in 16..nmax rounded to the pool, p uniform in 1..4, 1..max_rhs
    right-hand sides), with its FIFO one-at-a-time FP64 CG counterpart on the
    same arrivals (service times svc)."""
    import numpy as np
    import torch
    from paper_2401_17806_gb300 import dgsl
    dt = WORKLOAD["dt"]
    sizes = sorted({n for n, _ in pool})
    rng = np.random.default_rng(seed)
    arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.5) + 8))
    arr = arr[arr < seconds]
    lnN = rng.uniform(np.log(16), np.log(nmax), len(arr))
    Nr = [min(sizes, key=lambda s: abs(np.log(s) - v)) for v in lnN]
    pr = rng.integers(1, 5, len(arr))
    kr = rng.integers(1, max_rhs + 1, len(arr))
    xs = [torch.zeros(int(k) * pool[(int(N), int(p))][0].n_dof, dtype=torch.float64, device="cuda")
          for N, p, k in zip(Nr, pr, kr)]
    torch.cuda.synchronize()
    srv = dgsl.Server(dgsl.engine_opts(hbm_budget_bytes=int(budget), idle_us=2000, precond=precond))
    owner, outstanding = {}, []
    done_t = np.full(len(arr), np.nan)
    status = np.zeros(len(arr), dtype=np.int64)
    relres = np.full(len(arr), np.nan)
    floor = np.zeros(len(arr))
    start = time.perf_counter()
    i = 0
    while True:
        now = time.perf_counter() - start
        while i < len(arr) and arr[i] <= now:
            op, rhs = pool[(int(Nr[i]), int(pr[i]))]
            k = int(kr[i])
            t = srv.dgsl_submit(dgsl.request(op, dgsl.SCHUR, dt, rhs[:k * op.n_dof], xs[i], n_rhs=k))
            owner[t] = i
            outstanding.append(t)
            i += 1
        if outstanding:
            flags, infos = srv.dgsl_poll_many(np.array(outstanding, dtype=np.uint64))
            tnow = time.perf_counter() - start
            keep = []
            for t, f, inf in zip(outstanding, flags, infos):
                if f == 1:
                    done_t[owner[t]] = tnow
                    status[owner[t]] = inf.status
                    relres[owner[t]] = inf.relres
                    floor[owner[t]] = inf.relres_floor
                else:
                    keep.append(t)
            outstanding = keep
        if i >= len(arr) and not outstanding:
            break
        if time.perf_counter() - start > seconds + 300:
            break
        time.sleep(0.0002)
    stats = srv.stats()
    srv.close()
    lat = done_t - arr
    fin = np.isfinite(lat)
    end = np.nanmax(done_t) if fin.any() else seconds
    free_at, blat = 0.0, []
    for a, N, p, k in zip(arr, Nr, pr, kr):
        begin = max(a, free_at)
        free_at = begin + int(k) * svc[(int(N), int(p))]
        blat.append(free_at - a)
    blat = np.array(blat)
    nsolves = int(sum(int(k) for k, f in zip(kr, fin) if f))
    failed = [{"N": int(Nr[j]), "p": int(pr[j]), "rhs": int(kr[j]), "status": int(status[j]),
               "relres": float(relres[j]), "fp64_floor": float(floor[j])}
              for j in range(len(arr)) if fin[j] and status[j] != 0][:10]
    return {
        "rate": rate, "requests": int(len(arr)), "completed": int(fin.sum()),
        "right_hand_sides": int(kr.sum()), "all_converged": bool(np.all(status[fin] == 0)),
        # a request short of the tolerance whose residual is at FP64's own floor
        # (the residual of its exact solution rounded to FP64, reported by the
        # library) is at the accuracy FP64 allows, not a failed solve
        "all_converged_or_at_fp64_floor": bool(np.all((status[fin] == 0) | (relres[fin] <= floor[fin]))),
        "not_converged": failed,
        "max_relres": float(np.nanmax(relres)) if fin.any() else None,
        "requests_per_s": float(fin.sum() / end), "solves_per_s": float(nsolves / end),
        "p50_ms": float(np.nanpercentile(lat, 50) * 1e3), "p99_ms": float(np.nanpercentile(lat, 99) * 1e3),
        "engine_launches": stats["engine_launches"], "admitted_while_running": stats["admitted_running"],
        "fp64_one_at_a_time": {"requests_per_s": float(len(arr) / free_at),
                               "solves_per_s": float(kr.sum() / free_at),
                               "p50_ms": float(np.percentile(blat, 50) * 1e3),
                               "p99_ms": float(np.percentile(blat, 99) * 1e3)}}


def serve_leg(args):
    """Open-loop Poisson arrivals through the server: mesh N log-uniform in
    16..nmax (rounded to the pool of powers of two), p uniform in 1..4, 1..8
    RHS per request (one multi-RHS request each), FP32 inner CG + FP64
    refinement to 1e-10, every right-hand side's relative residual reported.
    Latency = request done - arrival.  Baseline: the same trace served FIFO by
    one-at-a-time FP64 CG (service times measured on this GPU, extrapolated
    above N = 256)."""
    import torch
    from paper_2401_17806_gb300 import build, dgsl
    build.build()
    torch.cuda.set_device(0)
    dt = WORKLOAD["dt"]
    sizes = [n for n in SERVE_SIZES if n <= args.serve_nmax]
    t0 = time.time()
    pool = serve_pool(sizes, dt)
    build_s = time.time() - t0
    svc, how, _ = fp64_service_times(pool, dt)
    pc = {"none": dgsl.PRECOND_NONE, "block-jacobi": dgsl.PRECOND_BLOCK_JACOBI,
          "multigrid": dgsl.PRECOND_MULTIGRID}[args.serve_precond]
    warm_requests(pool, pc, dt)
    results = []
    for k, rate in enumerate(float(v) for v in args.serve_rates.split(",")):
        window = min(args.serve_seconds, args.serve_requests / rate)
        results.append(serve_trace(pool, svc, rate, window, 77 + k, pc, args.serve_budget,
                                   args.serve_nmax))
        results[-1]["arrival_window_s"] = window
        print(json.dumps(results[-1]), file=sys.stderr, flush=True)
    print(json.dumps({
        "metric": "served Schur solves/s and p50/p99 latency", "workload": "serve", "data": "synthetic",
        "config": {"N_pool": sizes, "p_range": [1, 4], "rhs_per_request": [1, 8], "tol": WORKLOAD["tol"],
                   "precond": args.serve_precond, "hbm_budget_bytes": args.serve_budget,
                   "seconds_per_rate": args.serve_seconds, "max_requests_per_rate": args.serve_requests,
                   "operator_pool_build_s": build_s,
                   "fp64_service_times": {f"{n}x{n} p={p}": h for (n, p), h in sorted(how.items())},
                   "sample": f"N log-uniform in 16..{args.serve_nmax}"},
        "sweep": results}))


def serve_sample(args):
    """The serving half of the metric in the default line: one fixed seeded
    trace of the serving configuration (N log-uniform in 16..1024, p in 1..4,
    1..8 right-hand sides per request, FP32 couplings with FP64 refinement to
    1e-10, 150 GB budget) at --serve-sample-rate requests/s for 10 s through the multigrid
    server, against the same arrivals served one at a time by FP64 CG."""
    import torch
    from paper_2401_17806_gb300 import dgsl
    dt = WORKLOAD["dt"]
    t0 = time.time()
    pool = serve_pool(SERVE_SIZES, dt)
    build_s = time.time() - t0
    svc, how, _ = fp64_service_times(pool, dt)
    warm_requests(pool, dgsl.PRECOND_MULTIGRID, dt)
    r = serve_trace(pool, svc, args.serve_sample_rate, 10.0, 1234, dgsl.PRECOND_MULTIGRID, 150e9, 1024)
    fp = r["fp64_one_at_a_time"]
    r.update({
        "metric": "served Schur solves/s and p50/p99 latency at 1e-10",
        "sample": f"one seeded Poisson trace, {args.serve_sample_rate:g} requests/s for 10 s; N log-uniform 16..1024 (pool of powers of "
                  "two), p uniform 1..4, 1..8 right-hand sides; multigrid-preconditioned FP32 CG under FP64 "
                  "refinement, 8 concurrent solves, 150 GB budget",
        "baseline": "the same arrivals served FIFO by one-at-a-time unpreconditioned FP64 CG on this GPU: service "
                    "times measured for N <= 256, extrapolated above (per-iteration cost x iterations scaled by N)",
        "solves_per_s_vs_fp64": r["solves_per_s"] / fp["solves_per_s"] if fp["solves_per_s"] else None,
        "p99_vs_fp64": fp["p99_ms"] / r["p99_ms"] if r["p99_ms"] else None,
        "operator_pool_build_s": build_s,
        "fp64_service_s": {f"{n}x{n} p={p}": round(v, 4) for (n, p), v in sorted(svc.items())},
    })
    del pool
    torch.cuda.empty_cache()
    return r


def warm_requests(pool, pc, dt):
    """One request per pool operator before a trace, so that every operator's
    preconditioner (block-Jacobi blocks or multigrid hierarchy) is built."""
    import torch
    from paper_2401_17806_gb300 import dgsl
    if pc == dgsl.PRECOND_NONE:
        return
    wx = [torch.zeros(op.n_dof, dtype=torch.float64, device="cuda") for op, _ in pool.values()]
    warm = [dgsl.request(op, dgsl.SCHUR, dt, rhs[:op.n_dof], x) for (op, rhs), x in zip(pool.values(), wx)]
    dgsl.dgsl_cg_solve_batch(warm, dgsl.engine_opts(precond=pc, max_iters=1, max_refine=1))
    torch.cuda.synchronize()


# ---------------------------------------------------------------- oracle legs

def oracle_setup(N, p):
    """The oracle's Schur operator and right-hand side for the workload (host
    only; used by the CPU baseline and by --impl reference)."""
    import numpy as np
    from oracle import assemble as OA
    from oracle import fields as OF
    from oracle import operators as OP
    from paper_2401_17806_gb300 import synth
    xy, tri, per = synth.jittered_periodic_mesh(N, WORKLOAD["seed"])
    orc = OP.Operators(OA.assemble(xy, tri, per, p))
    Y = OF.dual_nodes(orc.bl.conn, p).reshape(-1, 2)
    u, v = synth.taylor_green_velocity(Y[:, 0], Y[:, 1])
    vhat = np.stack([u, v]) + synth.standard_normal((2, Y.shape[0]), WORKLOAD["seed"] + 1,
                                                    WORKLOAD["noise"])
    b = orc.G.T @ vhat.ravel()
    return orc, b


def oracle_cg_rate(orc, b, iters):
    """DOF*iterations/s of the oracle's plain FP64 CG (fixed iteration count)."""
    from oracle import operators as OP
    dt = WORKLOAD["dt"]
    t = time.perf_counter()
    _, it, _ = OP.cg(lambda v: orc.apply_schur(v, dt), b, tol=0.0, maxit=iters, mean_zero=True)
    el = time.perf_counter() - t
    return orc.n * it / el, it, el


def host_cpu_info():
    """Cores this process may run on (os.sched_getaffinity) and the CPU model
    (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return cores, model or platform.processor() or platform.machine()


def _oracle_worker(iters):
    """One forked worker: the oracle's CG for a fixed number of iterations on
    the operator built by the parent (shared copy-on-write)."""
    rate, it, el = oracle_cg_rate(_ORACLE[0], _ORACLE[1], iters)
    return _ORACLE[0].n * it, el


_ORACLE = []


def oracle_all_cores(orc, b, iters, cores):
    """DOF*iterations/s of `cores` single-threaded copies of the oracle's CG
    running at once (forked after the operator is built; this process never
    touches the GPU): the host's whole throughput on independent solves."""
    import multiprocessing as mp
    _ORACLE[:] = [orc, b]
    ctx = mp.get_context("fork")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [1] * cores)          # warm every worker
        t = time.perf_counter()
        res = pool.map(_oracle_worker, [iters] * cores)
        el = time.perf_counter() - t
    return sum(w for w, _ in res) / el


def cpu_leg_main(args):
    """Host-only subprocess: the oracle on one thread and on every core."""
    orc, b = oracle_setup(args.N, args.p)
    rate1, it, el = oracle_cg_rate(orc, b, args.cpu_iters)
    cores, model = host_cpu_info()
    rate_all = oracle_all_cores(orc, b, args.cpu_iters, cores) if cores > 1 else rate1
    print(json.dumps({"value": rate1, "iters": it, "seconds": el, "n_dof": int(orc.n), "cores": cores,
                      "cpu_model": model, "value_all_cores": rate_all}))


def run_cpu_baseline(args):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--N", str(args.N), "--p", str(args.p),
           "--cpu-iters", str(args.cpu_iters)]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
        out = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, never fatal to the GPU number
        return {"value": None, "unit": "DOF*iters/s", "cores": 1, "kind": "oracle",
                "sample": f"failed: {type(e).__name__}"}
    return {"value": out["value_all_cores"], "unit": "DOF*iters/s", "cores": out["cores"], "kind": "oracle",
            "cpu_model": out["cpu_model"],
            "single_thread": {"value": out["value"], "cores": 1},
            "sample": (f"{out['iters']} FP64 CG iterations of the Schur solve on the same "
                       f"{args.N}x{args.N}, p={args.p} mesh ({out['n_dof']} DOF) per worker, the oracle's "
                       f"scipy/numpy code single-threaded in each of {out['cores']} forked workers at once "
                       f"(all cores of os.sched_getaffinity) and alone on one thread; operator build excluded")}


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    orc, b = oracle_setup(args.N, args.p)
    cores, model = host_cpu_info()
    import multiprocessing as mp
    _ORACLE[:] = [orc, b]
    ctx = mp.get_context("fork")            # this process never touches the GPU
    with ctx.Pool(cores) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_worker, [2] * cores)
        t = time.perf_counter()
        dof_iters = 0
        for _ in range(args.steps):
            dof_iters += sum(w for w, _ in pool.map(_oracle_worker, [args.cpu_iters] * cores))
        el = time.perf_counter() - t
    value = dof_iters / el
    sample = (f"each step: {args.cpu_iters} FP64 CG iterations of the Schur solve on the "
              f"{args.N}x{args.N}, p={args.p} mesh in each of {cores} single-threaded forked workers at once")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF*iters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "N": args.N, "p": args.p, "n_dof": int(orc.n)},
        "cpu_baseline": {"value": value, "unit": "DOF*iters/s", "cores": cores, "kind": "oracle",
                         "cpu_model": model, "sample": sample},
        "e2e": {"value": value, "unit": "DOF*iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------- main

def aggregate_ranks(ms, e2e_ms, dof_iters, e2e_dof_iters, device=None):
    """Whole-job numbers across ranks (replicas, no data exchange): the slowest
    rank's times (MAX) and the total work (SUM).  Single process: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, e2e_ms, dof_iters, e2e_dof_iters
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([dof_iters, e2e_dof_iters], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return t[0].item(), t[1].item(), w[0].item(), w[1].item()


def main():
    args = parse_args()
    if args.cpu_leg:
        cpu_leg_main(args)
        return
    if args.impl == "reference":
        reference_main(args)
        return
    if args.workload == "batch":
        batch_leg(args)
        return
    if args.workload == "serve":
        serve_leg(args)
        return
    if args.workload == "cg":
        cg_leg(args)
        return
    if args.workload == "c3":
        c3_leg(args)
        return
    if args.workload == "mg":
        mg_leg(args)
        return
    if args.workload == "sl":
        sl_leg(args)
        return
    if args.workload == "ns":
        ns_leg(args)
        return
    if args.workload == "advdiff":
        advdiff_leg(args)
        return
    rank, world, local = dist_setup(args)
    import torch
    res = gpu_leg(args, rank, world, local)
    ms, e2e_ms = res["ms"], res["e2e_ms"]
    dof_iters, e2e_dof_iters = float(res["dof_iters"]), float(res["e2e_dof_iters"])
    ms, e2e_ms, dof_iters, e2e_dof_iters = aggregate_ranks(ms, e2e_ms, dof_iters, e2e_dof_iters,
                                                           device="cuda")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(args)
    serve = None
    if rank == 0 and not args.no_serve:
        serve = serve_sample(args)
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    op = res["op"]
    cb, vb = {"f32": (4, 4), "bf16": (2, 4), "f64": (8, 8)}[args.precision]
    per_row = bytes_per_row_iter(op.n_phi, cb, vb)
    alg_bytes = res["iters_total"] * op.n_dof * per_row
    achieved = alg_bytes / (res["kern_ms"] * 1e-3) / 1e9 if res["kern_ms"] > 0 else None
    peak, peak_src = measured_hbm_peak()
    line = {
        "metric": METRIC,
        "value": dof_iters / (ms * 1e-3),
        "unit": "DOF*iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32+f64", "bf16": "bf16+f32+f64", "f64": "f64"}[args.precision],
        "data": "synthetic",
        "config": {
            "workload": workload_name(args), "N": args.N, "p": args.p, "n_dof": op.n_dof,
            "n_tri": op.n_tri, "n_edge": op.n_edge, "dt": WORKLOAD["dt"], "nu": WORKLOAD["nu"],
            "tol": WORKLOAD["tol"],
            "precision": {"f32": "FP32 couplings + FP32 inner CG, FP64 refinement",
                          "bf16": "BF16 couplings, FP32 inner CG, FP64 refinement",
                          "f64": "FP64 CG"}[args.precision],
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2: FP32 + FP64 couplings "
                  f"{(op.device_bytes / 1e6):.0f} MB resident, couplings streamed every iteration",
            "schur_iters_per_step": res["schur_iters_per_step"],
            "helmholtz_iters_per_step": res["helm_iters_per_step"],
            "refinements_per_step": res["refinements"],
            "max_relres": res["relres_max"],
            "projected_velocity_div_rel": res["div_rel"],
            "operator_build_s": res["build_s"],
            "cg_grid_ctas": res["grid"],
        },
        "roofline": {
            "kernel": "k_cg (persistent CG, FP32 couplings)" if args.precision == "f32" else "k_cg",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": (NCU_DRAM_BYTES_PER_ROW_ITER[(args.p, args.precision)] * op.n_dof
                        * res["iters_total"] / max(1, res["cg_launches"])
                        if (args.p, args.precision) in NCU_DRAM_BYTES_PER_ROW_ITER else None),
            "traffic_unit": "bytes per launch (ncu DRAM bytes per row-iteration x rows x mean iterations per launch)",
            "alg_bytes_per_launch": alg_bytes / max(1, res["cg_launches"]),
            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
            "bytes_per_row_iter": per_row,
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_dof_iters / (e2e_ms * 1e-3), "unit": "DOF*iters/s",
                "h2d_bytes_per_step": res["h2d"], "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
    }
    if "fp64" in res:
        f = res["fp64"]
        line["fp64_cg_baseline"] = {"value": f["dof_iters"] / (f["ms"] * 1e-3), "unit": "DOF*iters/s",
                                    "ms_per_step": f["ms"], "iters_per_step": f["iters"],
                                    "speedup_of_value": (dof_iters / ms) / (f["dof_iters"] / f["ms"]),
                                    "stage_time_ratio": f["ms"] / (ms / args.steps)}
    if "bj" in res:
        bj = res["bj"]
        per_row_bj = bytes_per_row_iter(op.n_phi, cb, vb, precond=True)
        ach = bj["iters_total"] * op.n_dof * per_row_bj / (bj["kern_ms"] * 1e-3) / 1e9
        line["block_jacobi"] = {
            "what": "same stage, CG preconditioned by the inverse diagonal blocks (extension)",
            "ms_per_step": bj["ms"] / args.steps,
            "stage_speedup": (ms / args.steps) / (bj["ms"] / args.steps),
            "schur_iters_per_step": bj["schur_iters"],
            "helmholtz_iters_per_step": bj["helm_iters"],
            "max_relres": bj["relres_max"],
            "kernel_achieved_gbs": ach, "kernel_frac": ach / peak if peak else None,
            "bytes_per_row_iter": per_row_bj,
        }
    if "mg" in res:
        mg = res["mg"]
        line["multigrid"] = {
            "what": "same stage, PCG with the two-level multigrid preconditioner (block-Jacobi smoother, "
                    "P1 vertex coarse space, smoothed-aggregation V-cycle; extension)",
            "ms_per_step": mg["ms"] / args.steps,
            "stage_speedup": (ms / args.steps) / (mg["ms"] / args.steps),
            "speedup_vs_fp64_cg_stage": (res["fp64"]["ms"] / (mg["ms"] / args.steps)) if "fp64" in res else None,
            "schur_iters_per_step": mg["schur_iters"], "helmholtz_iters_per_step": mg["helm_iters"],
            "refinements_per_step": mg["refinements"], "max_relres": mg["relres_max"],
            "hierarchy_build_and_first_stage_s": mg["first_run_s"],
            "kernel_launches_per_step": mg["launches_per_step"],
        }
        if "fp64" in mg:
            f = mg["fp64"]
            line["multigrid"]["fp64_multigrid"] = {
                "what": "the same stage with the multigrid PCG in FP64 throughout (one step)",
                "ms_per_step": f["ms"], "schur_iters_per_step": f["schur_iters"],
                "helmholtz_iters_per_step": f["helm_iters"], "max_relres": f["relres_max"],
                "fp32_ir_iteration_overhead": (mg["schur_iters"] + mg["helm_iters"])
                / max(1, f["schur_iters"] + f["helm_iters"]) - 1.0,
                "fp32_ir_stage_speedup": f["ms"] / (mg["ms"] / args.steps)}
    if serve is not None:
        line["serving"] = serve
    if "sl" in res:
        sl = res["sl"]
        line["sl_transport"] = {
            "what": "semi-Lagrangian transport of the stage's main-grid velocity by itself over dt (Sec. 2.5)",
            "ms_per_call": sl["ms"], "trajectories_per_s": sl["trajectories"] / (sl["ms"] * 1e-3),
            "gauss_point_trajectories": sl["trajectories"], "cells_crossed_per_trajectory": sl["crossed"],
        }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
