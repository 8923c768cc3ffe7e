"""Benchmark: cell-collision evaluations per second of the spectral Boltzmann
collision operator on one GB300 (or N, one process per GPU, weak scaling).

Workload (default): 65536 independent cells, 2-D velocity grid 32x32 on
[-10,10]^2, hard-sphere (VHS) kernel, each cell two shifted Maxwellians with
Mach 0-3 drift.  One step = one collide_batch over all cells (forward DFT,
mode sum, inverse DFT).  Inputs (268 MB) and outputs exceed the 129 MB L2, so
no L2 flush is needed between steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead, on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_V, L_BOX, GAMMA = 32, 10.0, 1.0
CELLS = 65536
SEED = 1003
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
# DRAM bytes (read + write) of the mode-sum launch of one step on the
# 65536-cell workload (the autotuned FP32x2 kernel on 16-cell tiles, three CTAs
# per SM), from one ncu capture of dram__bytes_read.sum and
# dram__bytes_write.sum of that kernel; reported only for that workload.
MODESUM_TRAFFIC_65536 = 261291008 + 207005184
METRIC = "cell-collision evals/s at N_v=32^2: mixed-precision vs FP64 GPU, rel-L2 err stated"
WORKLOAD = "65536 cells, 2-D 32x32 velocity grid on [-10,10]^2, VHS kernel, shifted Maxwellians Mach 0-3"
FAST_WORKLOAD = ("65536 cells, 2-D 32x32 velocity grid on [-10,10]^2, Maxwell molecules, fast spectral "
                 "(Carleman) form with %d directions, shifted Maxwellians Mach 0-3")


def fast_flops_per_cell(N, ndirs):
    """Algorithmic FP32 work of one fast-form evaluation (mode-sum phase):
    nominal 5 n log2 n flops per complex length-n FFT; per direction (and once
    more for the loss term) one complex multiply per retained mode, 2h+1 row
    and P column transforms of length P, and one multiply-add per padded
    point; then P/2-length real transforms of the P columns (plus the 10-flop
    untangling of each kept row) and h+1 row transforms.  For an even number
    of directions, direction p + A/2 gives direction p's product, so A/2
    products are formed."""
    h = N // 2 - 1
    M = 2 * h + 1
    P = next(L for L in (2, 3, 4, 6, 8, 12, 16, 24, 32, 48) if L >= 3 * h + 1)
    fft = lambda n: 5.0 * n * math.log2(n)
    per_dir = 6.0 * M * M + (M + P) * fft(P) + 2.0 * P * P
    final = P * (fft(P // 2) + 10.0 * (h + 1)) + (h + 1) * fft(P)
    nconv = ndirs // 2 if ndirs % 2 == 0 else ndirs     # paired directions share one product
    return (nconv + 1) * per_dir + final


def _env_rank():
    from paper_2103_14890_gb300.dist import rank_env
    return rank_env()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(f_host, budget_s=15.0, check_idx=(), ndirs=0):
    """The cpu_baseline leg: time the FP64 oracle on the host cores on a bounded
    sample of cells (the cells in check_idx plus the first cells of the batch,
    sized to about budget_s of work).  Returns the baseline entry, the sampled
    cell indices and the oracle's Q on them (used to state the GPU error).
    ndirs > 0: the oracle's fast (Carleman) modes, Maxwell molecules."""
    import numpy as np
    import oracle
    k = oracle.FastKernel(N_V, L_BOX, ndirs) if ndirs else oracle.Kernel(2, N_V, L_BOX, GAMMA)
    probe = f_host[:8].astype(np.float64)
    t0 = time.perf_counter()
    k.collide(probe)
    per_cell = (time.perf_counter() - t0) / len(probe)
    n = int(max(8, min(len(f_host), budget_s / max(per_cell, 1e-6))))
    idx = np.unique(np.concatenate([np.asarray(check_idx, dtype=np.int64),
                                    np.arange(max(0, n - len(check_idx)), dtype=np.int64)]))
    sample = f_host[idx].astype(np.float64)
    t0 = time.perf_counter()
    Qr = k.collide(sample)
    dt = time.perf_counter() - t0
    entry = {"value": len(idx) / dt, "unit": "cell-collision evals/s", "cores": oracle.num_threads(),
             "kind": "oracle",
             "sample": "%d of the %d cells (FP64 %s, OpenMP over cells)" % (
                 len(idx), len(f_host), "fast-form pair sum" if ndirs else "direct sum")}
    return entry, idx, Qr, k


def reference_arm(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import numpy as np
    from paper_2103_14890_gb300 import workloads
    f = workloads.shifted_maxwellians(4096, 2, N_V, L_BOX, seed=SEED)
    base, _, _, k = cpu_baseline(f, budget_s=4.0)
    per_step = max(8, int(base["value"] * 4.0))
    per_step = min(per_step, len(f))
    sample = f[:per_step]
    for _ in range(args.warmup):
        k.collide(sample[:8])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        k.collide(sample)
    el = time.perf_counter() - t0
    value = per_step * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cell-collision evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded sample per step: %d cells)" % per_step},
            "cpu_baseline": {"value": value, "unit": "cell-collision evals/s", "cores": base["cores"],
                             "kind": "oracle", "sample": "%d cells per step" % per_step},
            "e2e": {"value": value, "unit": "cell-collision evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=CELLS, help="cells per GPU (small cases for ncu captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the IMEX-step and grouped-batch measurements")
    ap.add_argument("--method", default="direct", choices=["direct", "fast"],
                    help="fast: time the fast spectral form (Maxwell molecules) as the main line instead")
    ap.add_argument("--ndirs", type=int, default=8, help="collision directions of the fast form")
    ap.add_argument("--form", default="fp32", choices=["fp32", "fp32x2"],
                    help="precision form of the timed line (fp32x2: the double-float mode sum)")
    ap.add_argument("--sections", default="forms,transport,imex,grouped,fast",
                    help="comma list of the extra measurements to run (forms, transport, imex, grouped, fast)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    rank, world, local = _env_rank()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2103_14890_gb300 import binding as bz, build as bzbuild, workloads
    bzbuild.build()
    bz.load()

    grid = bz.Grid(2, N_V, L_BOX)
    fast = args.method == "fast"
    modes = bz.FastModes(grid, args.ndirs) if fast else bz.Modes(grid, GAMMA)
    cells = args.cells
    f_host = workloads.shifted_maxwellians(cells, 2, N_V, L_BOX, seed=SEED + rank).astype(np.float32)
    f = torch.from_numpy(f_host).cuda()
    Q = torch.empty_like(f)

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    form = args.form

    def step():
        bz.collide_batch(modes, f, Q, precision=form)

    for _ in range(max(3, args.warmup)):
        step()
    bz.check()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    bz.profile(True)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    prof = bz.profile_read()
    bz.profile(False)
    clk = clocks.stop()
    bz.check()
    from paper_2103_14890_gb300.dist import max_over_ranks
    ms = max_over_ranks(ms, device="cuda")          # the slowest rank sets the job's time
    value = cells * world / (ms / 1e3)

    # dominant kernel: the mode sum (or the fast form's convolutions)
    ms_name = "fast_f32" if fast else "modesum_x2" if form == "fp32x2" else \
        "modesum_f32" if "modesum_f32" in prof else "modesum_f32_generic"
    launches, ktot = prof.get(ms_name, (0, float("nan")))
    k_ms = ktot / max(1, launches)
    if "modesum_f32_tail" in prof:          # the last partial wave runs as a second launch
        tl, tt = prof["modesum_f32_tail"]
        k_ms += tt / max(1, tl)
    # the X2 form's unit of work is the same pair count (its extra instructions
    # are the precision, not more pairs)
    flops_launch = (fast_flops_per_cell(N_V, args.ndirs) if fast else 10.0 * modes.pairs_sym) * cells
    achieved = flops_launch / (k_ms / 1e3) / 1e12
    gpu_launches = sum(c for c, _ in prof.values())

    # FP64 plain form on the same workload
    Q64 = None
    value64 = ms64 = float("nan")
    if args.fp64_steps > 0:
        Q64 = torch.empty((cells, N_V * N_V), dtype=torch.float64, device="cuda")
        f64 = f.double()
        bz.collide_batch(modes, f64, Q64, precision="fp64")
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.fp64_steps):
            bz.collide_batch(modes, f64, Q64, precision="fp64")
        e1.record(st)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        value64 = cells * world / (ms64 / 1e3)

    extra = {}
    sections = set(args.sections.split(",")) if not args.no_extra and not fast else set()
    if "transport" in sections:
        extra["transport"] = _transport_measure(bz, workloads, st, check=not args.no_cpu_baseline)
    if "forms" in sections:
        extra["precision_forms"] = _forms_measure(bz, workloads, st, f, f_host, check=not args.no_cpu_baseline)
    if "imex" in sections:
        extra["imex_step"] = _imex_measure(bz, workloads, barrier, check=not args.no_cpu_baseline)
    if "grouped" in sections:
        extra["grouped"] = _group_measure(bz, workloads, barrier, check=not args.no_cpu_baseline)
    if "fast" in sections:
        extra["fast_spectral"] = _fast_measure(bz, f, f_host, st, args.ndirs, check=not args.no_cpu_baseline)

    # end to end: pinned host f -> device, collide, device -> pinned host Q
    e2e_val = None
    if not args.no_e2e:
        e2e_val = _e2e(args, bz, modes, f_host, f, barrier, st, e0, e1, cells, world)

    line = None
    if rank == 0:
        _report(args, bz, modes, f_host, Q, Q64, cells, world, ms, value, ms64, value64, prof, ms_name, k_ms,
                flops_launch, achieved, gpu_launches, e2e_val, clk, extra)
    if dist:
        tdist.barrier()
        tdist.destroy_process_group()
    return 0


def _e2e(args, bz, modes, f_host, f, barrier, st, e0, e1, cells, world):
    """End to end through the host-buffer entry point: pinned host f in, the
    library pipelines the copies to the device, the collisions and the copies
    of Q back; the timed region ends when Q is on the host."""
    import torch
    fh = torch.from_numpy(f_host).pin_memory()
    qh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        bz.collide_batch_host(modes, fh, qh, precision=args.form, stream=st)
    barrier()
    e0.record(st)
    for _ in range(args.steps):
        bz.collide_batch_host(modes, fh, qh, precision=args.form, stream=st)
    e1.record(st)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    return cells * world / (e2e_ms / 1e3)


def workloads_mod():
    from paper_2103_14890_gb300 import workloads
    return workloads


def torch_index(idx):
    import torch
    return torch.from_numpy(idx).to("cuda")


def _timed(fn, steps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _transport_measure(bz, workloads, st, check=True):
    """Transport step of the finite-volume scheme on the 19802-triangle mesh
    with the 32^2 velocity grid (the explosion-problem states): the residual
    <L(f^w)>_x (CWENO degree 1 + Rusanov) in FP32 and FP64, its HBM roofline
    (algorithmic bytes: f read once, L written once), the ARS(2,2,2) step
    coupled to it (VHS direct sum; Maxwell fast form), and the oracle's rate
    on a 50x50-lattice mesh."""
    import numpy as np
    import torch
    pts, tri = workloads.sod_triangulation()
    mesh = bz.Mesh(pts, tri, order=2)
    P = pts[tri]
    bary = P.mean(axis=1)
    g = bz.Grid(2, N_V, L_BOX)
    fh = workloads.mesh_states(bary, N_V, L_BOX, jump=True)
    out = {"cells": int(mesh.n_cells), "velocities": N_V * N_V, "order": 2,
           "mesh": "jittered 100x100 lattice, Delaunay, 19802 triangles",
           "l2": "a 256 MB buffer is written before every timed call (f alone, 81 MB in FP32, would fit L2)"}
    hbm = _measured_hbm()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")     # 256 MB > L2, written between calls
    for prec, dt_, steps in (("fp32", torch.float32, 20), ("fp64", torch.float64, 5)):
        f = torch.from_numpy(fh).to("cuda", dt_)
        Lr = torch.empty_like(f)
        for _ in range(3):
            bz.transport_residual(mesh, g, f, Lr, precision=prec)
        bz.check()
        bz.profile(True)
        ms = 0.0
        for _ in range(steps):
            flush.fill_(1)
            ms += _timed(lambda: bz.transport_residual(mesh, g, f, Lr, precision=prec), 1, st)
        ms /= steps
        prof = bz.profile_read()
        bz.profile(False)
        es = 4 if prec == "fp32" else 8
        alg = 2.0 * f.numel() * es
        kern = {k: v[1] / max(1, v[0]) for k, v in prof.items()}
        ent = {"ms_per_call": ms, "cell_velocity_updates_per_s": f.numel() / (ms / 1e3), "kernel_ms": kern,
               "algorithmic_bytes": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9}
        if prec == "fp32":
            ent["roofline"] = {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                               "frac": alg / (ms / 1e3) / 1e9 / hbm,
                               "note": "two passes: the reconstruction writes the values at the 3 face midpoints per "
                                       "(cell, velocity), which the flux pass reads back (0.65 GB of DRAM traffic "
                                       "per call at the least)"}
        out[prec] = ent
    # the same residual in a closed box: every boundary edge a wall at rest
    # with full accommodation (the wall flux pass: one CTA per cell holds all
    # 1024 velocities for the wall's mass balance)
    bedges = _boundary_edges(tri)
    mesh_w = bz.Mesh(pts, tri, order=2)
    mesh_w.set_walls(bedges, np.tile([[1.0, 0.0, 0.0]], (len(bedges), 1)))
    f = torch.from_numpy(fh).to("cuda", torch.float32)
    Lr = torch.empty_like(f)
    for _ in range(3):
        bz.transport_residual(mesh_w, g, f, Lr, precision="fp32")
    bz.check()
    bz.profile(True)
    msw = 0.0
    for _ in range(10):
        flush.fill_(1)
        msw += _timed(lambda: bz.transport_residual(mesh_w, g, f, Lr, precision="fp32"), 1, st)
    msw /= 10
    profw = bz.profile_read()
    bz.profile(False)
    out["fp32_walls"] = {"ms_per_call": msw, "wall_edges": int(len(bedges)),
                         "kernel_ms": {k: v[1] / max(1, v[0]) for k, v in profw.items()}}

    def timed_residual(m, f, Lr, reps):
        for _ in range(3):
            bz.transport_residual(m, g, f, Lr, precision="fp32")
        bz.check()
        bz.profile(True)
        ms = 0.0
        for _ in range(reps):
            flush.fill_(1)
            ms += _timed(lambda: bz.transport_residual(m, g, f, Lr, precision="fp32"), 1, st)
        prof = bz.profile_read()
        bz.profile(False)
        return ms / reps, {k: v[1] / max(1, v[0]) for k, v in prof.items()}

    # the third-order residual (CWENO of degree 2, two Gauss points per face)
    f = torch.from_numpy(fh).to("cuda", torch.float32)
    Lr = torch.empty_like(f)
    ms3, k3 = timed_residual(bz.Mesh(pts, tri, order=3), f, Lr, 10)
    out["fp32_order3"] = {"ms_per_call": ms3, "kernel_ms": k3,
                          "cell_velocity_updates_per_s": f.numel() / (ms3 / 1e3),
                          "note": "5 coefficients per (cell, velocity) written and read back; 4 velocities per thread "
                                  "(FP32x2 on triangle meshes)"}
    # a periodic Voronoi mesh (the polygonal cells of the vortex study), orders 2 and 3
    vp, vc = workloads.periodic_voronoi(2603)
    vbary = np.array([np.asarray(vp)[c].mean(axis=0) for c in vc])
    fv_ = torch.from_numpy(workloads.mesh_states(vbary / 10.0, N_V, L_BOX, jump=True)).to("cuda", torch.float32)
    Lv = torch.empty_like(fv_)
    for order in (2, 3):
        msv, kv = timed_residual(bz.Mesh(vp, vc, order=order, periodic=(10.0, 10.0)), fv_, Lv, 10)
        out["fp32_voronoi_order%d" % order] = {"ms_per_call": msv, "kernel_ms": kv, "cells": len(vc),
                                              "cell_velocity_updates_per_s": fv_.numel() / (msv / 1e3)}
    # the coupled step
    hmesh = float(np.sqrt(np.abs(0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                                        (P[:, 2, 0] - P[:, 0, 0]) * (P[:, 1, 1] - P[:, 0, 1]))).mean()))
    dtt = 0.5 * hmesh / (math.sqrt(2.0) * L_BOX)
    f = torch.from_numpy(fh).to("cuda", torch.float32)
    y = torch.empty_like(f)
    for name, m, model in (("vhs_direct", bz.Modes(g, GAMMA), "boltzmann"),
                           ("maxwell_fast_A8", bz.FastModes(g, 8), "boltzmann"),
                           ("bgk", bz.Modes(g, GAMMA), "bgk")):
        bz.imex_step_fv(m, mesh, f, dtt, 5e-3, f_out=y, precision="fp32", model=model)
        bz.check()
        msi = _timed(lambda: bz.imex_step_fv(m, mesh, f, dtt, 5e-3, f_out=y, precision="fp32", model=model), 5, st)
        out["imex_step_fv_fp32_" + name] = {"ms_per_step": msi, "dt": dtt, "eps": 5e-3,
                                            "cell_steps_per_s": f.shape[0] / (msi / 1e3)}
    # the paper's Table comp_time measure: the collision operator's share over the BGK run,
    # tau_coll = (T_Boltzmann - T_BGK) / T_BGK in percent
    tb = out["imex_step_fv_fp32_bgk"]["ms_per_step"]
    for name in ("vhs_direct", "maxwell_fast_A8"):
        out["imex_step_fv_fp32_" + name]["tau_coll_pct"] = 100.0 * (
            out["imex_step_fv_fp32_" + name]["ms_per_step"] - tb) / tb
    if check:
        from oracle import fv
        p2, t2 = workloads.sod_triangulation(n_side=50)
        om = fv.Mesh(p2, t2)
        f2 = workloads.mesh_states(om.bary, N_V, L_BOX, jump=True)
        t0 = time.perf_counter()
        fv.transport_residual(om, f2, N_V, L_BOX, order=2)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"kind": "oracle", "value": f2.size / el, "unit": "cell-velocity updates/s",
                               "sample": "%d-triangle mesh, 32^2 velocities (numpy, one process)" % len(t2)}
    return out


def _boundary_edges(cells):
    """Vertex pairs of the edges that belong to one cell only."""
    count = {}
    for c in cells:
        c = [int(v) for v in c]
        for q in range(len(c)):
            e = frozenset((c[q], c[(q + 1) % len(c)]))
            count[e] = count.get(e, 0) + 1
    import numpy as np
    return np.array([sorted(e) for e, n in count.items() if n == 1], dtype=np.int64)


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fp:
            return float(json.load(fp)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def _imex_measure(bz, workloads, barrier, check=True):
    """One ARS(2,2,2) step on the ~19.6k-cell triangulated Sod-like mesh
    (32x32 grid on [-10,10]^2, VHS, eps = 5e-3, dt = h / (2 max|v|)), FP32,
    FP32X2 and FP64, the step captured as a CUDA graph (non-default stream);
    f^{n+1} against the oracle's step on 256 cells spread over the mesh."""
    import math
    import torch
    f, hmesh = workloads.sod_cells(32, 10.0)
    dt = 0.5 * hmesh / (math.sqrt(2.0) * 10.0)
    m = bz.Modes(bz.Grid(2, 32, 10.0), 1.0)
    s = torch.cuda.Stream()
    out = {}
    import numpy as np
    fin = f.astype(np.float32).astype(np.float64)
    idx = np.unique(np.linspace(0, f.shape[0] - 1, 256).astype(np.int64))
    want = None
    if check:
        import oracle
        want = oracle.Kernel(2, 32, 10.0, 1.0).imex_step(fin[idx], dt, 5e-3)
    with torch.cuda.stream(s):
        for prec, steps in (("fp32", 10), ("fp32x2", 3), ("fp64", 1)):
            x = torch.from_numpy(fin).to("cuda", torch.float64 if prec == "fp64" else torch.float32)
            y = torch.empty_like(x)
            for _ in range(2):
                bz.imex_step(m, x, dt, 5e-3, f_out=y, precision=prec, stream=s)
            bz.check(s)
            ms = _timed(lambda: bz.imex_step(m, x, dt, 5e-3, f_out=y, precision=prec, stream=s), steps, s)
            out[prec] = {"ms_per_step": ms, "cell_collision_evals_per_s": 2 * x.shape[0] / (ms / 1e3)}
            if want is not None:
                got = y[torch_index(idx)].double().cpu().numpy()
                out[prec]["rel_l2_fnp1_vs_oracle"] = float(np.linalg.norm(got - want) / np.linalg.norm(want))
    out["oracle_cells"] = int(len(idx))
    out["cells"] = int(f.shape[0])
    out["workload"] = "ARS(2,2,2) step, %d-cell Delaunay mesh, 32x32 grid, VHS, eps=5e-3, dt=%.3g, CUDA graph" % (
        f.shape[0], dt)
    return out


def _oracle_err(k, f_in, got, idx=None):
    """rel-L2 of got against the FP64 oracle on the rows idx (all rows if None)."""
    import numpy as np
    if idx is None:
        idx = np.arange(f_in.shape[0])
    Qr = k.collide(f_in[idx])
    return float(np.linalg.norm(got[idx] - Qr) / np.linalg.norm(Qr)), len(idx)


def _forms_measure(bz, workloads, st, f3, f3_host, check=True):
    """The three precision forms on the small and noisy configurations and the
    FP32X2 form on the benchmark workload: throughput and rel-L2 against the
    FP64 oracle (FP32-rounded inputs, the same values the device sees).
      config 1: 64 cells, 16^2 on [-8,8]^2, Maxwell molecules, bi-Maxwellians
      config 2: 4096 cells, 32^2 on [-10,10]^2, VHS, bi-Maxwellians x (1 + 5 % noise)
      config 3: the benchmark workload (65536 cells), FP32X2 only; its FP32 and
                FP64 numbers are the main line and fp64_form"""
    import numpy as np
    import oracle
    import torch
    out = {}
    cfgs = (("config1", 2, 16, 8.0, 0.0, workloads.bi_maxwellian(64, 2, 16, 8.0, seed=1001), 50),
            ("config2", 2, 32, 10.0, 1.0, workloads.bi_maxwellian(4096, 2, 32, 10.0, seed=1002, noise=0.05), 5))
    for name, d, N, L, gam, f, reps in cfgs:
        m = bz.Modes(bz.Grid(d, N, L), gam)
        fin = f.astype(np.float32).astype(np.float64)
        k = oracle.Kernel(d, N, L, gam) if check else None
        res = {"cells": f.shape[0], "grid": "%d^%d on [-%g,%g]^%d" % (N, d, L, L, d), "gamma": gam}
        for prec in ("fp32", "fp32x2", "fp64"):
            x = torch.from_numpy(fin).to("cuda", torch.float64 if prec == "fp64" else torch.float32)
            Q = torch.empty_like(x)
            bz.collide_batch(m, x, Q, precision=prec, stream=st)
            bz.check(st)
            ms = _timed(lambda: bz.collide_batch(m, x, Q, precision=prec, stream=st), reps, st)
            r = {"ms": ms, "cell_collision_evals_per_s": f.shape[0] / (ms / 1e3)}
            if check:
                r["rel_l2_vs_oracle"], r["oracle_cells"] = _oracle_err(k, fin, Q.double().cpu().numpy())
            res[prec] = r
        out[name] = res
    m = bz.Modes(bz.Grid(2, N_V, L_BOX), GAMMA)
    Q = torch.empty_like(f3)
    bz.collide_batch(m, f3, Q, precision="fp32x2", stream=st)
    bz.check(st)
    ms = _timed(lambda: bz.collide_batch(m, f3, Q, precision="fp32x2", stream=st), 3, st)
    r = {"ms": ms, "cell_collision_evals_per_s": f3.shape[0] / (ms / 1e3)}
    if check:
        idx = np.unique(np.linspace(0, f3.shape[0] - 1, 2048).astype(np.int64))
        k = oracle.Kernel(2, N_V, L_BOX, GAMMA)
        r["rel_l2_vs_oracle"], r["oracle_cells"] = _oracle_err(k, f3_host.astype(np.float64), Q.double().cpu().numpy(),
                                                               idx)
    out["config3_fp32x2"] = r
    out["note"] = ("fp32x2: FP64 forward DFT, double-float (compensated) mode sum on the FP32 pipe, FP32 inverse "
                   "DFT; FP32 arrays in and out")
    return out


def _group_measure(bz, workloads, barrier, check=True):
    """Heterogeneous batch in one group_collide call: 8 instances with cell
    counts log-uniform in [1e3, 5e4] and N in {16, 24, 32, 48}, plus two 3-D
    16^3 instances of 1000 cells; the FP32, FP32X2 and FP64 forms on the same
    FP32-rounded inputs, each against the FP64 oracle on 32 cells of every
    instance (and FP32 against FP64 over all cells)."""
    import numpy as np
    import torch
    items = workloads.grouped_instances()
    grids = {}
    hosts = []
    total = 0
    for it in items:
        key = (it["dim"], it["N"])
        if key not in grids:
            grids[key] = bz.Modes(bz.Grid(it["dim"], it["N"], it["L"]), 1.0)
        hosts.append(workloads.bi_maxwellian(it["n_cells"], it["dim"], it["N"], it["L"], seed=it["seed"]))
        total += it["n_cells"]
    s = torch.cuda.current_stream()
    out = {"cells": total, "instances": [(it["dim"], it["N"], it["n_cells"]) for it in items],
           "variants": {"%dd N=%d" % k: m.modesum_variant for k, m in grids.items()}}
    results = {}
    for prec in ("fp32", "fp32x2", "fp64"):
        dt = torch.float64 if prec == "fp64" else torch.float32
        entries = []
        for it, f in zip(items, hosts):
            x = torch.from_numpy(f.astype(np.float32)).to("cuda", dt)
            entries.append((grids[(it["dim"], it["N"])], x, torch.empty_like(x)))
        bz.group_collide(entries, precision=prec)
        bz.check()
        ms = _timed(lambda: bz.group_collide(entries, precision=prec), 1, s)
        out[prec] = {"ms_per_call": ms, "cell_collision_evals_per_s": total / (ms / 1e3)}
        results[prec] = [Q for (_, _, Q) in entries]
        del entries
    if check:
        # every instance against the FP64 oracle on 32 cells spread over it
        import oracle
        per = []
        for prec in ("fp32", "fp32x2", "fp64"):
            num = den = 0.0
            worst = 0.0
            for i, (it, f) in enumerate(zip(items, hosts)):
                k = oracle.Kernel(it["dim"], it["N"], it["L"], 1.0)
                idx = np.unique(np.linspace(0, it["n_cells"] - 1, 32).astype(np.int64))
                fin = f[idx].astype(np.float32).astype(np.float64)
                Qr = k.collide(fin)
                got = results[prec][i][torch_index(idx)].double().cpu().numpy()
                e2, q2 = float(((got - Qr) ** 2).sum()), float((Qr ** 2).sum())
                num += e2
                den += q2
                worst = max(worst, (e2 / q2) ** 0.5)
                if prec == "fp32x2":
                    per.append({"dim": it["dim"], "N": it["N"], "rel_l2_fp32x2": (e2 / q2) ** 0.5})
            out[prec]["rel_l2_vs_oracle"] = (num / den) ** 0.5
            out[prec]["worst_instance_rel_l2_vs_oracle"] = worst
        out["oracle_cells_per_instance"] = 32
        out["fp32x2_per_instance"] = per
        out["speedup_fp32x2_over_fp64"] = out["fp64"]["ms_per_call"] / out["fp32x2"]["ms_per_call"]
    # FP32 form against the FP64 GPU form on every cell of every instance
    num = den = 0.0
    for a, b in zip(results["fp32"], results["fp64"]):
        num += ((a.double() - b) ** 2).sum().item()
        den += (b ** 2).sum().item()
    out["rel_l2_fp32_vs_fp64_gpu"] = (num / den) ** 0.5
    out["speedup_fp32_over_fp64"] = out["fp64"]["ms_per_call"] / out["fp32"]["ms_per_call"]
    return out


def _fast_measure(bz, f, f_host, st, ndirs, check=True):
    """The fast spectral (Carleman) form on the same 65536 cells, Maxwell
    molecules: FP32 and FP64 throughput, the FP32 direct sum with the same
    kernel for comparison, the fast kernel's roofline on the FP32 peak, and
    the FP32 error against the oracle's fast modes on sampled cells."""
    import numpy as np
    import torch
    cells = f.shape[0]
    grid = bz.Grid(2, N_V, L_BOX)
    out = {"workload": FAST_WORKLOAD % ndirs, "ndirs": ndirs}
    mf = bz.FastModes(grid, ndirs)
    out["pad"] = mf.pad
    Q = torch.empty_like(f)
    for _ in range(3):
        bz.collide_batch(mf, f, Q, precision="fp32")
    bz.check()
    bz.profile(True)
    ms = _timed(lambda: bz.collide_batch(mf, f, Q, precision="fp32"), 10, st)
    prof = bz.profile_read()
    bz.profile(False)
    kl, kt = prof.get("fast_f32", (1, float("nan")))
    k_ms = kt / max(1, kl)
    fl = fast_flops_per_cell(N_V, ndirs) * cells
    out["fp32"] = {"ms_per_step": ms, "cell_collision_evals_per_s": cells / (ms / 1e3),
                   "kernel_ms": {k: v[1] / max(1, v[0]) for k, v in prof.items()}}
    out["roofline"] = {"bound": "alu", "kernel": "fast_f32", "kernel_ms": k_ms, "flops_per_launch": fl,
                       "achieved": fl / (k_ms / 1e3) / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": fl / (k_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                       "flop_count": "nominal 5 n log2 n per complex length-n FFT (bench.fast_flops_per_cell)"}
    f64 = f.double()
    Q64 = torch.empty_like(f64)
    bz.collide_batch(mf, f64, Q64, precision="fp64")
    ms64 = _timed(lambda: bz.collide_batch(mf, f64, Q64, precision="fp64"), 1, st)
    out["fp64"] = {"ms_per_step": ms64, "cell_collision_evals_per_s": cells / (ms64 / 1e3)}
    md = bz.Modes(grid, 0.0)
    Qd = torch.empty_like(f)
    bz.collide_batch(md, f, Qd, precision="fp32")
    msd = _timed(lambda: bz.collide_batch(md, f, Qd, precision="fp32"), 10, st)
    out["direct_fp32_same_kernel"] = {"ms_per_step": msd, "cell_collision_evals_per_s": cells / (msd / 1e3)}
    out["speedup_fast_over_direct_fp32"] = msd / ms
    # 48^2 grid (zero-padded to 72^2), 16384 cells: fast form against the direct sum
    g48 = bz.Grid(2, 48, L_BOX)
    f48 = torch.from_numpy(workloads_mod().shifted_maxwellians(16384, 2, 48, L_BOX, seed=SEED + 48)).to(
        "cuda", torch.float32)
    q48 = torch.empty_like(f48)
    res48 = {}
    for name, m48 in (("fast", bz.FastModes(g48, ndirs)), ("direct", bz.Modes(g48, 0.0))):
        bz.collide_batch(m48, f48, q48, precision="fp32")
        t48 = _timed(lambda: bz.collide_batch(m48, f48, q48, precision="fp32"), 5, st)
        res48[name] = {"ms_per_step": t48, "cell_collision_evals_per_s": f48.shape[0] / (t48 / 1e3)}
    res48["speedup_fast_over_direct"] = res48["direct"]["ms_per_step"] / res48["fast"]["ms_per_step"]
    out["grid_48x48_16384_cells_fp32"] = res48
    # the paper's production configuration: ARS(2,2,2) steps with the fast
    # operator (Maxwell molecules) on the 19802-cell mesh, CUDA graph
    fs, hmesh = workloads_mod().sod_cells(N_V, L_BOX)
    dt = 0.5 * hmesh / (math.sqrt(2.0) * L_BOX)
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        x = torch.from_numpy(fs).to("cuda", torch.float32)
        y = torch.empty_like(x)
        for _ in range(2):
            bz.imex_step(mf, x, dt, 5e-3, f_out=y, precision="fp32", stream=s2)
        bz.check(s2)
        msi = _timed(lambda: bz.imex_step(mf, x, dt, 5e-3, f_out=y, precision="fp32", stream=s2), 10, s2)
    out["imex_step_fp32"] = {"ms_per_step": msi, "cell_collision_evals_per_s": 2 * x.shape[0] / (msi / 1e3),
                             "workload": "ARS(2,2,2) step, %d-cell Delaunay mesh, eps=5e-3, CUDA graph" % x.shape[0]}
    bz.check()
    out["rel_l2_fp32_vs_fp64_gpu_all_cells"] = ((Q.double() - Q64).norm() / Q64.norm()).item()
    if check:
        import oracle
        k = oracle.FastKernel(N_V, L_BOX, ndirs)
        idx = np.linspace(0, cells - 1, 12).astype(np.int64)
        fs = f_host[idx].astype(np.float64)
        Qr = k.collide(fs)
        q32 = Q[torch_index(idx)].double().cpu().numpy()
        rho = fs.sum(1, keepdims=True) * k.dv ** 2
        out["fp32_vs_oracle"] = {"rel_l2": float(np.linalg.norm(q32 - Qr) / np.linalg.norm(Qr)),
                                 "loss_scaled": float(np.linalg.norm(q32 - Qr) / np.linalg.norm(rho * fs)),
                                 "cells": len(idx)}
    return out


def _report(args, bz, modes, f_host, Q, Q64, cells, world, ms, value, ms64, value64, prof, ms_name, k_ms,
            flops_launch, achieved, gpu_launches, e2e_val, clk, extra):
    import numpy as np
    # errors: against the FP64 oracle on the cells its timed run covers (same
    # FP32-rounded inputs), else the FP32 form against the FP64 GPU form
    cpu = None
    err32 = err64 = loss32 = None
    err32_vs64 = None
    if Q64 is not None:
        d = (Q.double() - Q64).norm().item()
        err32_vs64 = d / Q64.norm().item()
    if not args.no_cpu_baseline:
        spread = np.linspace(0, cells - 1, 24).astype(np.int64)
        cpu, idx, Qr, k = cpu_baseline(f_host, budget_s=15.0, check_idx=spread,
                                       ndirs=args.ndirs if args.method == "fast" else 0)
        ti = torch_index(idx)
        q32 = Q[ti].double().cpu().numpy()
        err32 = float(np.linalg.norm(q32 - Qr) / np.linalg.norm(Qr))
        if Q64 is not None:
            err64 = float(np.linalg.norm(Q64[ti].cpu().numpy() - Qr) / np.linalg.norm(Qr))
        fs = f_host[idx].astype(np.float64)
        rho = fs.sum(1, keepdims=True) * k.dv ** 2
        loss32 = float(np.linalg.norm(q32 - Qr) / np.linalg.norm(rho * fs))   # error / |loss rate ~ rho f|
        nchk = len(idx)
    else:
        nchk = 0
    line = {
        "metric": METRIC, "value": value, "unit": "cell-collision evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (FAST_WORKLOAD % args.ndirs if args.method == "fast" else WORKLOAD).replace(
                       str(CELLS), str(cells)),
                   "cells_per_gpu": cells, "N_v": N_V * N_V, "L": L_BOX,
                   "kernel": ("Maxwell molecules (gamma=0, b0=1/(2pi)), fast form, %d directions" % args.ndirs
                              if args.method == "fast" else "VHS hard spheres (gamma=1, b0=1/(2pi))"),
                   "precision_form": args.form,
                   "l2": "inputs and outputs (268 MB each) exceed L2: no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "rel_l2_err": {"form": args.form, "fp32_vs_oracle": err32, "fp64_vs_oracle": err64, "fp32_loss_scaled": loss32,
                       "oracle_cells": nchk, "fp32_vs_fp64_gpu_all_cells": err32_vs64},
        "fp64_form": {"value": value64, "unit": "cell-collision evals/s", "ms_per_step": ms64,
                      "speedup_fp32_over_fp64": value / value64} if Q64 is not None else None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": MODESUM_TRAFFIC_65536 if cells == CELLS and args.method == "direct" else None,
                     "kernel": ms_name,
                     "kernel_ms": k_ms, "flops_per_launch": flops_launch,
                     "peak_note": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz" + (
                         "; fp32x2 counts the same 10 flops per pair, its double-float arithmetic executes ~54 FP32 "
                         "instructions per pair" if args.form == "fp32x2" else "")},
        "kernel_times_ms": {k2: v[1] / max(1, v[0]) for k2, v in prof.items()},
        "gpu_launches": gpu_launches,
        "imex_step": extra.get("imex_step"),
        "grouped": extra.get("grouped"),
        "precision_forms": extra.get("precision_forms"),
        "fast_spectral": extra.get("fast_spectral"),
        "transport": extra.get("transport"),
        "e2e": {"value": e2e_val, "unit": "cell-collision evals/s",
                "h2d_bytes_per_step": int(Q.numel() * 4), "d2h_bytes_per_step": int(Q.numel() * 4)},
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    sys.exit(main())
