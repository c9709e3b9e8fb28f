"""Benchmark of the batched SF-AWRI gradient (one JSON line on rank 0).

Workload (per GPU): the frequency-dependent batch of 128 surface sources x 3 frequencies
(3 Hz on 64^3, 5 Hz on 96^3, 8 Hz on 128^3 physical nodes, each plus a 10-cell absorbing
layer: 84^3, 116^3, 148^3 computational nodes), 96 borehole receivers, seeded layered +
anomaly model, source-free mode, complex64 stencils with FP64 reductions.  One step = one
gradient evaluation of all 384 systems: right-hand sides, ``--iters`` CGLS iterations per
system (the fused, batched, graph-captured phases), the source-weight estimates and the
gradient/objective accumulation.

value = systems (source x frequency gradients) per second over all ranks.  With N ranks
every rank evaluates its own shot record of 384 systems (weak scaling) and the gradients
and objectives are summed over ranks (the method's one exchange step).  The working set
(~40 GB per GPU) is far larger than L2, so no flush is needed between steps.

``--impl reference`` times the CPU oracle (the repository has no other reference
implementation: the C++/OpenMP complex128 CGLS of ``oracle/cpu_cgls.cpp`` on every host core) on a
bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WRI gradient src·freq/s at 128³ (GPt·iter/s, % HBM roofline) vs plain path"
UNIT = "src·freq/s"
BYTES_PER_NODE_SYS = 80.0  # one CGLS iteration, per node and system: phase 1 48 B + phase 2 32 B (c64)
# grouped-update configurations: x read and written every m-th iteration, with m - 1 extra p reads
# then: phase 1 (m 32 + 16 + 8 (m - 1)) / m = 44 B (m = 2) or 42 B (m = 4)
XSTEPS = {22: 2, 23: 2, 24: 4}
MODEL_BYTES = 8.0          # m (float32) read by both phases, per node of a group, shared by its systems
K_POLL = 2                 # CG iterations per body of the iteration graph's device-side loop
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "cg_iteration_traffic.json")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--iters", type=int, default=300, help="CGLS iterations per system per step")
    p.add_argument("--nsrc", type=int, default=128)
    p.add_argument("--small", action="store_true", help="tiny workload (debugging only)")
    p.add_argument("--only-group", type=int, default=-1,
                   help="keep only one frequency group (0: 3 Hz, 1: 5 Hz, 2: 8 Hz); profiling cases")
    p.add_argument("--no-extras", action="store_true", help="skip plain-path, e2e and CPU legs")
    p.add_argument("--kernel", type=int, default=0, help="0 auto, 1 z-march only, 2+c TMA configuration c")
    p.add_argument("--order", type=int, default=0, help="TMA work order (0 = library default)")
    p.add_argument("--zsplit", type=int, default=0, help="z-chunks per tile column (0 = library choice)")
    p.add_argument("--promo", type=int, default=0, help="TMA L2 promotion: 0 auto, 1 none, 2 64B, 3 128B, 4 256B")
    p.add_argument("--cpu-seconds", type=float, default=4.0,
                   help="seconds of oracle CGLS per CPU sample (one per step in the reference arm; the GPU "
                        "arm's cpu_baseline takes one sample of 5x this)")
    p.add_argument("--group-sweep", default="",
                   help="comma-separated systems per call (e.g. 1,2,4,8,16,32): instead of the bench line, time "
                        "one CGLS iteration of that many systems of the 148^3 group in one batched call and "
                        "print one JSON line for each (the grouping sweep of Eq. Mmatrix2)")
    p.add_argument("--camembert-shape", action="store_true",
                   help="instead of the bench line, time one misfit + gradient evaluation on the shape of the "
                        "paper's timing case (61^3 nodes, 9 sources, 2025 receivers, 5 Hz, residual 1e-6) with "
                        "n_b = 9, 4 and 1 systems per call, and print one JSON line")
    return p.parse_args()


def workload(args, shard=0):
    import synth
    if args.small:
        groups = synth.workload_c4(nsrc=min(args.nsrc, 8), freqs=((3.0, 24), (5.0, 32), (8.0, 40)), nrec=24,
                                   shard=shard)
    else:
        groups = synth.workload_c4(nsrc=args.nsrc, shard=shard)
    if args.only_group >= 0:
        groups = [groups[args.only_group]]
    return groups


def workload_name(args):
    if args.small:
        return "c4-batch-small"
    base = "c4-batch: {} src x {{3 Hz 84^3, 5 Hz 116^3, 8 Hz 148^3}}".format(args.nsrc)
    return base if args.only_group < 0 else base + f" (group {args.only_group} only)"


def bytes_per_node_sys(opts):
    """Algorithmic bytes of one CGLS iteration per node and system for the configuration of opts."""
    k = int(opts.kernel)
    m = XSTEPS.get(k - 2, 1) if k >= 2 else 1
    return BYTES_PER_NODE_SYS - 16.0 + (16.0 + 8.0 * (m - 1)) / m


def phase_kernel_name(opts):
    """Name of the CGLS phase kernel a configuration launches (see wri_solve_opts.kernel)."""
    k = int(opts.kernel)
    if k == 1:
        return "k_march"
    cfg = k - 2 if k >= 2 else 8
    return "k_phase_tma" if cfg <= 3 else "k_phase_tma2" if cfg <= 8 else "k_phase_ws"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.path = f"/tmp/wri_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.out = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.dev), "-lms", "200"], stdout=self.out,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle legs
def _cpu_system(groups):
    """Arguments of the C++ oracle CGLS for the first system of the largest grid."""
    big = max(groups, key=lambda g: g.spec.n)
    rec = big.rec_idx[big.rec_off[0]:big.rec_off[1]]
    d = big.d[big.rec_off[0]:big.rec_off[1]]
    return big, (big.spec.shape, big.spec.h, big.omega, big.m, big.spec.npml, big.v_max, big.src[0], rec, d, big.lam)


def cpu_sample(sysargs, iters, threads):
    """Seconds of one oracle CGLS solve of ``iters`` iterations (set-up included)."""
    from oracle import cpu_cgls
    t0 = time.perf_counter()
    cpu_cgls.cgls(*sysargs, tol=0.0, max_iter=iters, nthreads=threads)
    return time.perf_counter() - t0


def cpu_calibrate(sysargs, threads, seconds):
    """(set-up seconds, iterations that take about ``seconds``) of the oracle CGLS on this system.
    One untimed solve first (thread start-up, first touch of the pages); the per-iteration time is
    the difference of a 1- and a 5-iteration solve, or, if timing noise makes that implausibly
    small, the 5-iteration solve's time per iteration (an upper bound, so the sample stays short)."""
    cpu_sample(sysargs, 2, threads)
    ta = cpu_sample(sysargs, 1, threads)
    tb = cpu_sample(sysargs, 5, threads)
    per_iter = (tb - ta) / 4.0
    if not per_iter > 0.05 * tb / 5.0:
        per_iter = tb / 5.0
    return max(ta - per_iter, 0.0), max(2, int(round(seconds / per_iter)))


def cpu_rate(groups, step_iters, seconds, threads):
    """Throughput of the C++/OpenMP oracle CGLS (complex128, every host core), extrapolated to the
    bench step from one bounded sample on the largest grid: the per-node-iteration rate of a solve of
    k iterations (k sized to take about ``seconds``; its set-up, timed separately, removed).

    Returns (src·freq/s, node-iterations/s, seconds sampled, iterations sampled)."""
    big, sysargs = _cpu_system(groups)
    setup, k = cpu_calibrate(sysargs, threads, seconds)
    secs = cpu_sample(sysargs, k, threads) - setup
    node_iter_rate = big.spec.n * k / secs
    node_iters = sum(g.nsys * g.spec.n for g in groups) * step_iters
    nsys = sum(g.nsys for g in groups)
    return nsys * node_iter_rate / node_iters, node_iter_rate, secs, k


def cpu_sample_text(groups, k):
    big = max(groups, key=lambda g: g.spec.n)
    return (f"C++/OpenMP oracle CGLS (complex128, matrix-free) on one system of the {big.spec.nx}^3 group: "
            f"{k} iterations, set-up removed; the per-node-iteration rate is scaled to the step "
            f"({sum(g.nsys for g in groups)} systems x the step's iterations on their own grids)")


def host_threads():
    return len(os.sched_getaffinity(0))


def run_reference(args, ws, rank):
    """The reference arm: the oracle as it stands, on the host cores, one bounded sample of the
    workload per step (rank 0 only)."""
    if rank != 0:
        return
    from oracle import cpu_cgls
    groups = workload(args)
    nsys = sum(g.nsys for g in groups)
    thr = host_threads()
    big, sysargs = _cpu_system(groups)
    setup, k = cpu_calibrate(sysargs, thr, args.cpu_seconds)
    for _ in range(args.warmup):
        cpu_sample(sysargs, k, thr)
    secs = sum(cpu_sample(sysargs, k, thr) - setup for _ in range(args.steps))
    rate = big.spec.n * k * args.steps / secs
    node_iters = sum(g.nsys * g.spec.n for g in groups) * args.iters
    value = nsys * rate / node_iters
    cb = {"value": value, "unit": UNIT, "cores": cpu_cgls.threads() if thr <= 0 else thr, "kind": "oracle",
          "sample": cpu_sample_text(groups, k) + f"; one sample per step, {args.steps} steps",
          "gpt_iter_s": rate / 1e9, "seconds_sampled": secs, "host_threads": thr}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic", "ms_per_step": 1e3 * nsys / value,
            "config": {"workload": workload_name(args), "systems": nsys, "iters_per_system": args.iters,
                       "l2": "working set >> L2 (no flush needed)"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- grouping sweep
def run_group_sweep(args):
    """Grouping (Eq. Mmatrix2): one CGLS iteration of n_b systems of the largest grid advanced by
    one batched call, for every n_b of ``--group-sweep`` (the default TMA configuration and
    order unless ``--kernel`` / ``--order`` say otherwise; no autotuning, so every n_b runs the
    same kernel).  The per-iteration time is the difference of two solves of 20 and 80
    iterations (tol = 0, CUDA events on the launching stream, best of two each), which removes
    the set-up; algorithmic bytes are those of the bench line."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2410_18429_gb300 import wri
    from paper_2410_18429_gb300.problem import to_device

    sizes = [int(x) for x in args.group_sweep.split(",") if x.strip()]
    groups = workload(args)
    g0 = max(groups, key=lambda g: g.spec.n)
    if not sizes or min(sizes) < 1 or max(sizes) > g0.nsys:
        raise SystemExit(f"--group-sweep sizes must lie in 1..{g0.nsys}")
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        peak = 6800.0
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    n = g0.spec.n
    for nb in sizes:
        sub = synth.Group(g0.spec, g0.freq, g0.v, g0.src[:nb], g0.rec_off[:nb + 1] - g0.rec_off[0],
                          g0.rec_idx[g0.rec_off[0]:g0.rec_off[nb]], g0.lam, g0.v_max, g0.pml_R, g0.alpha[:nb],
                          g0.d[g0.rec_off[0]:g0.rec_off[nb]])
        spec = to_device(sub, wri.C64, dev)
        base = wri.make_opts(tol=0.0, max_iter=1, dtype=wri.C64, poll_every=K_POLL, kernel=args.kernel,
                             order=args.order, zsplit=args.zsplit, l2_promotion=args.promo)
        work = torch.empty(wri.workspace_size([spec], base), dtype=torch.uint8, device=dev)

        def timed(iters):
            o = wri.WriSolveOpts.from_buffer_copy(base)
            o.max_iter = iters
            ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev[0].record(stream)
            wri.solve([spec], o, workspace=work)
            ev[1].record(stream)
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) * 1e-3

        timed(20)
        ta = min(timed(20) for _ in range(2))
        tb = min(timed(80) for _ in range(2))
        t_iter = (tb - ta) / 60.0
        alg = n * (bytes_per_node_sys(base) * nb + MODEL_BYTES)
        print(json.dumps({"group_sweep": nb, "grid": f"{g0.spec.nx}x{g0.spec.ny}x{g0.spec.nz}",
                          "ms_per_iter": t_iter * 1e3, "us_per_system_iter": t_iter / nb * 1e6,
                          "gpt_iter_s": nb * n / t_iter / 1e9, "hbm_gbs": alg / t_iter / 1e9,
                          "frac_of_measured_hbm": alg / t_iter / 1e9 / peak,
                          "cg_vector_mb": 6 * nb * n * 8 / 1e6, "kernel": int(base.kernel), "order": int(base.order),
                          "device": torch.cuda.get_device_name(dev)}), flush=True)
        del spec, work
        torch.cuda.empty_cache()


# ---------------------------------------------------------------- GPU arm
def run_camembert_shape(args):
    """One misfit + gradient evaluation on the shape of the paper's timing case (Sec. "Evaluation of
    GPU Acceleration Efficiency", Table CMPTime: a 3 km cube at h = 50 m, 61^3 nodes, 9 sources,
    2025 receivers, 5 Hz, relative residual 1e-6), with synthetic model and data on a 10-cell
    absorbing layer (81^3 computational nodes), and on the nearest cube whose x extent the TMA phases
    take (60^3 + layer, 80^3).  Certified precision configuration, refined to an
    FP64 normal-equation residual of 1e-6 (every system must end with status OK).  The 9 systems
    are evaluated in batched calls of n_b systems (9, 4 and 1, so 1, 3 and 9 calls), each call a
    solve, a source estimate and a gradient, after one untimed evaluation; CUDA events on the
    launching stream, SM clocks sampled.  Prints one JSON line per grid."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    for nphys in (61, 60):
        camembert_case(args, synth.workload_camembert_shape(nphys), dev, stream)


def camembert_case(args, G, dev, stream):
    """The evaluations of run_camembert_shape on one grid (61^3 physical: x extent 81, z-march
    kernels; 60^3: x extent 80, TMA phases)."""
    import torch

    import synth
    from paper_2410_18429_gb300 import wri
    from paper_2410_18429_gb300.problem import to_device

    def part(a, b):
        return synth.Group(G.spec, G.freq, G.v, G.src[a:b], G.rec_off[a:b + 1] - G.rec_off[a],
                           G.rec_idx[G.rec_off[a]:G.rec_off[b]], G.lam, G.v_max, G.pml_R, G.alpha[a:b],
                           G.d[G.rec_off[a]:G.rec_off[b]])

    opts = solve_opts(wri, args, iters=400000, max_refine=8, refine_tol=1e-6, inner_tol=1e-3)
    full = with_u64([to_device(G, wri.C64, dev)], dev)
    work = torch.empty(wri.workspace_size(full, opts), dtype=torch.uint8, device=dev)
    if int(opts.kernel) == 0:
        opts = wri.autotune(full, opts, trial_iters=8, workspace=work)
    grad = torch.zeros(G.spec.nz, G.spec.ny, G.spec.nx, dtype=torch.float64, device=dev)
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    runs = []
    for nb in (9, 4, 1):
        calls = []
        for a in range(0, G.nsys, nb):
            sp = with_u64([to_device(part(a, min(a + nb, G.nsys)), wri.C64, dev)], dev)
            calls.append((sp, torch.empty(wri.workspace_size(sp, opts), dtype=torch.uint8, device=dev)))

        def evaluate():
            out = []
            grad.zero_()
            f.zero_()
            for sp, w in calls:
                for s_ in sp:
                    s_.u.zero_()
                    s_.u64.zero_()
                it, rr, st = wri.solve(sp, opts, workspace=w)
                wri.source_estimate(sp, wri.C64, workspace=w)
                wri.gradient_refined(sp, opts, w, grads=[grad], f=f)
                out.append((it, rr, st))
            return out

        evaluate()
        torch.cuda.synchronize()
        clk = Clocks(0)
        clk.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = evaluate()
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        its = torch.cat([r[0] for r in res]).cpu().tolist()
        rrs = torch.cat([r[1] for r in res]).cpu().tolist()
        sts = torch.cat([r[2] for r in res]).cpu().tolist()
        runs.append({"n_b": nb, "calls": len(calls), "seconds": e0.elapsed_time(e1) / 1e3, "iters": its,
                     "fp64_relres_max": max(rrs), "status_all_ok": all(v == wri.SYS_OK for v in sts),
                     "f": float(f.item()), "clocks": clocks})
    g = G.spec
    print(json.dumps({"camembert_shape": {
        "grid": f"{g.nx}x{g.ny}x{g.nz} computational nodes ({g.nx - 2 * g.npml}^3 physical + {g.npml}-cell layer), "
                f"h = {g.h} m",
        "phase_kernels": "TMA" if g.nx % 4 == 0 else "z-march (x extent not a multiple of 4)",
        "freq_hz": G.freq, "systems": int(G.nsys), "receivers_per_system": int(G.rec_off[1] - G.rec_off[0]),
        "precision": "complex64 CGLS inside FP64 iterative refinement to an FP64 normal-equation residual of 1e-6; "
                     "FP64 source estimate and gradient from the refinement's residual",
        "kernel": {"config": int(opts.kernel) - 2 if int(opts.kernel) >= 2 else None, "order": int(opts.order)},
        "data": "synthetic (Gaussian anomaly in 2500 m/s; homogeneous Green's-function traces)",
        "runs": runs, "library": wri.version()}}))


def solve_opts(wri, args, certified=True, iters=None, **kw):
    """Options of the bench step.  certified: the precision configuration whose converged results
    meet the stated accuracy (complex64 CGLS with FP32 stencils and FP64 reductions inside FP64
    iterative refinement; the FP64 residual decides and is reported; the FP64 wavefield feeds an
    FP64 source estimate and gradient).  With refine_tol = 0 and an unreachable inner tolerance the
    one refinement step runs exactly ``iters`` CGLS iterations, then its FP64 residual check."""
    base = dict(tol=0.0, max_iter=args.iters if iters is None else iters, dtype=wri.C64, poll_every=K_POLL,
                kernel=args.kernel, order=args.order, zsplit=args.zsplit, l2_promotion=args.promo)
    if certified:
        base.update(max_refine=1, refine_tol=0.0, inner_tol=1e-300)
    base.update(kw)
    return wri.make_opts(**base)


def step_launches(iters, k, certified, ngroups):
    """Kernels of libwri in one step (the claim of the bench line).  Both configurations: the
    receiver bitmaps, the z tables, the right-hand sides, the initial S^H b, the loop of phase 1 +
    phase 2 in bodies of K iterations with one control kernel each (the P1 after the last iteration
    is the x-only pass), the export and the source estimate.  Certified: the refinement's receiver
    map, init and cold start (r2), its update, one FP64 residual step of 3 kernels (residual,
    forcing, S^H), the final rounding, and the gradient from that residual (one kernel per group).
    Unrefined: the gradient's z tables, gradient kernel and data term."""
    bodies = -(-(iters + 1) // k)
    loop = bodies * (2 * k + 1)
    fixed = 1 + 1 + 1 + 1 + 1 + 1
    fixed += (1 + 1 + 1 + 1 + 3 + 1 + ngroups) if certified else 3
    return loop + fixed


def subset(groups, per_group):
    """The first ``per_group`` systems of every group (same grids, model and geometry)."""
    import synth
    out = []
    for g in groups:
        k = min(per_group, g.nsys)
        out.append(synth.Group(g.spec, g.freq, g.v, g.src[:k], g.rec_off[:k + 1] - g.rec_off[0],
                               g.rec_idx[g.rec_off[0]:g.rec_off[k]], g.lam, g.v_max, g.pml_R, g.alpha[:k],
                               g.d[g.rec_off[0]:g.rec_off[k]]))
    return out


def true_relres(wri, grp, u64, dev):
    """||S^H (b - S u)|| / ||S^H b|| of every system of a group in FP64, for FP64 wavefields u64
    [nsys, n], with the complex128 operator of libwri on the float32 model and complex64 data the
    complex64 solves saw (a measurement of the bench: the vector arithmetic around the two operator
    applications is torch's).  Source-free mode."""
    import numpy as np
    import torch
    from paper_2410_18429_gb300.problem import to_device
    m32 = grp.m.astype(np.float32).astype(np.float64)
    d32 = grp.d.astype(np.complex64).astype(np.complex128)
    sp = to_device(grp, wri.C128, dev, m=m32, d=d32)
    out = []
    for s in range(grp.nsys):
        us = u64[s:s + 1]
        Au = wri.apply_A(sp, us)[0]
        Au[int(grp.src[s])] = 0
        rec = torch.as_tensor(grp.rec_idx[grp.rec_off[s]:grp.rec_off[s + 1]].astype(np.int64), device=dev)
        d = torch.as_tensor(d32[grp.rec_off[s]:grp.rec_off[s + 1]], device=dev)
        r2 = grp.lam * (d - us[0, rec])
        sv = wri.apply_A(sp, (-Au)[None], adjoint=True)[0]
        sv[rec] += grp.lam * r2
        sb = torch.zeros_like(sv)
        sb[rec] = grp.lam ** 2 * d
        out.append(float(sv.norm() / sb.norm()))
    return out


def with_u64(specs, dev):
    import torch
    for s_ in specs:
        s_.u64 = torch.zeros(s_.nsys, s_.n, dtype=torch.complex128, device=dev)
    return specs


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.group_sweep:
        run_group_sweep(args)
        return
    if args.camembert_shape:
        run_camembert_shape(args)
        return
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import wri
    from paper_2410_18429_gb300.parallel_sum import allreduce_gradient
    from paper_2410_18429_gb300.problem import to_device

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    groups = workload(args, shard=rank)
    specs = with_u64([to_device(g, wri.C64, dev) for g in groups], dev)
    nsys = sum(g.nsys for g in groups)
    node_sys = sum(g.nsys * g.spec.n for g in groups)
    opts = solve_opts(wri, args)
    work = torch.empty(wri.workspace_size(specs, opts), dtype=torch.uint8, device=dev)
    if args.kernel == 0 and args.order == 0:
        opts = wri.autotune(specs, opts, trial_iters=8, workspace=work)  # before the warm-up, not timed
    grads = [torch.zeros(g.spec.nz, g.spec.ny, g.spec.nx, dtype=torch.float64, device=dev) for g in groups]
    f = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def gradient_of_solve(sp, o, a, g_out, f_out, w):
        """g and f of the wavefields the last solve left: from the refined solve's FP64 residual (no
        stencil pass) in the certified configuration, else the gradient kernel on the wavefields."""
        if int(o.max_refine) > 0 and all(s_.u64 is not None for s_ in sp):
            wri.gradient_refined(sp, o, w, grads=g_out, f=f_out)
        else:
            wri.gradient(sp, wri.C64, a, grads=g_out, f=f_out, workspace=w)

    def step(sp, o, solve_events=None):
        if solve_events is not None:
            solve_events[0].record(stream)
        it, rr, st = wri.solve(sp, o, workspace=work)
        if solve_events is not None:
            solve_events[1].record(stream)
        a = wri.source_estimate(sp, wri.C64, workspace=work)
        for g in grads:
            g.zero_()
        f.zero_()
        gradient_of_solve(sp, o, a, grads, f, work)
        if ws > 1:
            allreduce_gradient(grads, f)
        return it, rr, st

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(t):
        if ws > 1:
            import torch.distributed as dist
            tt = torch.tensor([t], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t

    for _ in range(args.warmup):
        step(specs, opts)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    solve_ev = [(ev(), ev()) for _ in range(args.steps)]
    e0, e1 = ev(), ev()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(args.steps):
        it, rr, st = step(specs, opts, solve_ev[k])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    iters_done = int(it.min().item())
    relres_fp64 = [float(rr.min().item()), float(rr.max().item())]
    value = ws * nsys * args.steps / t
    gpt = ws * node_sys * iters_done * args.steps / t / 1e9
    t_solve = statistics.mean(a.elapsed_time(b) for a, b in solve_ev) / 1e3

    # ---- roofline of one fused CG iteration (phase 1 + phase 2 over every system).  The solve of a
    # step is its fixed part (set-up, the FP64 residual steps of the refinement) plus iters_done
    # iterations; the per-iteration time is the difference of two solves of the step's configuration
    # with iters_done and iters_done / 3 iterations (CUDA events on the stream the iteration graph is
    # launched on, best of two each), which removes the fixed part.
    def timed_solve(iters):
        o = wri.WriSolveOpts.from_buffer_copy(opts)
        o.max_iter = iters
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        wri.solve(specs, o, workspace=work)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    lo_iters = max(2, iters_done // 3)
    t_hi = min(timed_solve(iters_done) for _ in range(2))
    t_lo = min(timed_solve(lo_iters) for _ in range(2))
    t_iter = (t_hi - t_lo) / (iters_done - lo_iters)
    alg_bytes = node_sys * bytes_per_node_sys(opts) + sum(g.spec.n for g in groups) * MODEL_BYTES
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / t_iter / 1e9
    # DRAM traffic per iteration from the ncu record of this build and kernel configuration
    traffic = None
    cfg = int(opts.kernel) - 2 if int(opts.kernel) >= 2 else None
    try:
        prof = json.load(open(TRAFFIC_FILE))
        rec = prof.get("configs", {}).get(str(cfg))
        if prof.get("kernel_version") == wri.version() and rec:
            traffic = rec["bytes_per_node_system"] * node_sys
    except (OSError, KeyError, ValueError):
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "algorithmic_bytes": alg_bytes,
                "kernel": f"{phase_kernel_name(opts)} phase 1 + phase 2 (one fused CGLS iteration over all systems)",
                "t_iter_ms": t_iter * 1e3, "solve_fixed_ms": (t_solve - iters_done * t_iter) * 1e3,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback"}

    extras = {}
    if not args.no_extras and rank == 0:
        # ---- the same step without refinement and with FP32 stencils on the complex64 wavefield in
        # the estimate and gradient (faster, but its gradient misses the 1e-4 target: labelled variant)
        fast = solve_opts(wri, args, certified=False, kernel=int(opts.kernel), order=int(opts.order))
        plain_specs = [to_device(g, wri.C64, dev) for g in groups]
        step(plain_specs, fast)
        torch.cuda.synchronize()
        nv = 3
        v0, v1 = ev(), ev()
        v0.record(stream)
        for _ in range(nv):
            step(plain_specs, fast)
        v1.record(stream)
        torch.cuda.synchronize()
        tv = v0.elapsed_time(v1) / 1e3 / nv
        extras["variant_fp32_gradient"] = {
            "value": nsys / tv, "unit": UNIT, "ms_per_step": tv * 1e3,
            "precision": "complex64 CGLS (FP32 stencils, FP64 reductions), no refinement; FP32 stencils on the "
                         "complex64 wavefield in the source estimate and gradient (gradient error ~1e-3: misses "
                         "the 1e-4 target)"}
        del plain_specs
        torch.cuda.empty_cache()

        # ---- plain (unbatched, unfused, host-read scalars) path, per iteration on one system of the
        # largest grid
        import synth
        big_i = max(range(len(groups)), key=lambda i: groups[i].spec.n)
        g0 = groups[big_i]
        sp1 = to_device(subset([g0], 1)[0], wri.C64, dev)

        def timed_plain(iters):
            o = wri.make_opts(tol=0.0, max_iter=iters, dtype=wri.C64, plain=True)
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            wri.solve([sp1], o)
            torch.cuda.synchronize()
            return time.perf_counter() - h0

        timed_plain(5)
        pa, pb = timed_plain(10), timed_plain(60)
        plain_per_sys_iter = (pb - pa) / 50.0
        fused_per_sys_iter_big = t_iter * (g0.spec.n / node_sys)
        extras["plain"] = {"per_system_iter_ms_148": plain_per_sys_iter * 1e3,
                           "fused_per_system_iter_ms_148": fused_per_sys_iter_big * 1e3,
                           "speedup_per_iteration": plain_per_sys_iter / fused_per_sys_iter_big}
        del sp1

        # ---- measured at the adaptive schedule's loosest tolerance (1e-2): a whole gradient (solve to
        # tolerance, source estimate, gradient) of the first 8 sources of every group in one batched
        # call, certified configuration (the FP64 residual decides), CUDA events and clocks; and the
        # same gradient of the first source of every group on the plain path (same tolerance)
        ntol = 8
        tol_groups = subset(groups, ntol)
        tsp = with_u64([to_device(g, wri.C64, dev) for g in tol_groups], dev)
        tol_opts = solve_opts(wri, args, iters=200000, max_refine=4, refine_tol=1e-2, inner_tol=1e-3,
                              kernel=int(opts.kernel), order=int(opts.order))
        twork = torch.empty(wri.workspace_size(tsp, tol_opts), dtype=torch.uint8, device=dev)
        tgr = [torch.zeros(g.spec.nz, g.spec.ny, g.spec.nx, dtype=torch.float64, device=dev) for g in tol_groups]
        tf = torch.zeros(1, dtype=torch.float64, device=dev)

        def grad_at_tol(sp, o, w):
            if w is None:
                w = torch.empty(wri.workspace_size(sp, o), dtype=torch.uint8, device=dev)
            it_, rr_, st_ = wri.solve(sp, o, workspace=w)
            a_ = wri.source_estimate(sp, wri.C64, workspace=w)
            for g in tgr[:len(sp)]:
                g.zero_()
            tf.zero_()
            gradient_of_solve(sp, o, a_, tgr[:len(sp)], tf, w)
            return it_, rr_, st_

        tclk = Clocks(local)
        tclk.start()
        a0, a1 = ev(), ev()
        torch.cuda.synchronize()
        a0.record(stream)
        it_t, rr_t, st_t = grad_at_tol(tsp, tol_opts, twork)
        a1.record(stream)
        torch.cuda.synchronize()
        t_tol = a0.elapsed_time(a1) / 1e3
        clk_tol = tclk.stop()
        its = it_t.cpu().numpy()
        offs = np.cumsum([0] + [g.nsys for g in tol_groups])
        nt = int(offs[-1])
        del twork
        # the first source of every group, one call: the fused path (certified configuration) and the
        # plain path (one system at a time, scalars read by the host), same systems and tolerance
        one_groups = subset(groups, 1)

        def timed_grad(sp, o):
            b0, b1 = ev(), ev()
            torch.cuda.synchronize()
            b0.record(stream)
            res = grad_at_tol(sp, o, None)
            b1.record(stream)
            torch.cuda.synchronize()
            return res, b0.elapsed_time(b1) / 1e3

        fsp = with_u64([to_device(g, wri.C64, dev) for g in one_groups], dev)
        (fit, _, fst), t_fused3 = timed_grad(fsp, tol_opts)
        f_true = [true_relres(wri, g, sp_.u64, dev)[0] for g, sp_ in zip(one_groups, fsp)]
        # the same stopping rule as the plain path: unrefined, the FP32 recurrence's residual decides
        usp = with_u64([to_device(g, wri.C64, dev) for g in one_groups], dev)
        u_opts = solve_opts(wri, args, certified=False, tol=1e-2, max_iter=200000, kernel=int(opts.kernel),
                            order=int(opts.order))
        (uit, _, ust), t_unref3 = timed_grad(usp, u_opts)
        u_true = [true_relres(wri, g, sp_.u64, dev)[0] for g, sp_ in zip(one_groups, usp)]
        psp = with_u64([to_device(g, wri.C64, dev) for g in one_groups], dev)
        p_opts = wri.make_opts(tol=1e-2, max_iter=200000, dtype=wri.C64, plain=True)
        (pit, prr, pst), t_plain = timed_grad(psp, p_opts)
        p_true = [true_relres(wri, g, sp_.u64, dev)[0] for g, sp_ in zip(one_groups, psp)]
        extras["at_tolerance"] = {
            "tol": 1e-2, "systems": nt, "sources_per_group": ntol, "measured": True,
            "ms_per_step": t_tol * 1e3, "value": nt / t_tol, "unit": UNIT,
            "iters_per_group": [float(its[offs[i]:offs[i + 1]].mean()) for i in range(len(tol_groups))],
            "fp64_relres_max": float(rr_t.max().item()),
            "status_all_ok": bool(int(st_t.max().item()) == wri.SYS_OK),
            "clocks": clk_tol,
            "same_systems": {
                "systems": "the first source of every group (3 systems), one call per path, tol 1e-2; "
                           "true_relres = ||S^H (b - S u)|| / ||S^H b|| of the returned wavefield in FP64",
                "fused_unrefined": {"ms": t_unref3 * 1e3, "iters_per_group": [int(x) for x in uit.cpu().tolist()],
                                    "status_all_ok": bool(int(ust.max().item()) == wri.SYS_OK),
                                    "true_relres": u_true},
                "plain": {"ms": t_plain * 1e3, "iters_per_group": [int(x) for x in pit.cpu().tolist()],
                          "status_all_ok": bool(int(pst.max().item()) == wri.SYS_OK), "true_relres": p_true},
                "fused_certified": {"ms": t_fused3 * 1e3, "iters_per_group": [int(x) for x in fit.cpu().tolist()],
                                    "status_all_ok": bool(int(fst.max().item()) == wri.SYS_OK),
                                    "true_relres": f_true},
                "speedup_vs_plain_same_rule": t_plain / t_unref3,
                "speedup_vs_plain_certified": t_plain / t_fused3},
            "speedup_vs_plain_per_system": (t_plain / len(psp)) / (t_tol / nt)}
        del tsp, psp, fsp, usp
        torch.cuda.empty_cache()

        if ws == 1:
            thr = host_threads()
            val, rate, secs, k = cpu_rate(groups, iters_done, 5 * args.cpu_seconds, thr)
            extras["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                                      "sample": cpu_sample_text(groups, k), "gpt_iter_s": rate / 1e9,
                                      "seconds_sampled": secs, "host_threads": thr}

    # ---- end to end through the public API with host buffers, on every rank (the gradient sum
    # over ranks included), timed like the device-resident steps (barrier, max over ranks)
    if not args.no_extras:
        m_host = [torch.from_numpy(np.ascontiguousarray(g.m, dtype=np.float32).reshape(g.spec.shape)).pin_memory()
                  for g in groups]
        d_host = [torch.from_numpy(np.ascontiguousarray(g.d, dtype=np.complex64)).pin_memory() for g in groups]
        g_host = [torch.empty(g.spec.shape, dtype=torch.float64).pin_memory() for g in groups]
        f_host = torch.empty(1, dtype=torch.float64).pin_memory()
        a_host = torch.empty(nsys, dtype=torch.complex128).pin_memory()
        h2d = sum(x.numel() * x.element_size() for x in m_host + d_host)
        d2h = sum(x.numel() * x.element_size() for x in g_host) + 8 + a_host.numel() * 16

        def e2e_step():
            for s_, mh, dh in zip(specs, m_host, d_host):
                s_.m.copy_(mh, non_blocking=True)
                s_.d.copy_(dh, non_blocking=True)
            wri.solve(specs, opts, workspace=work)
            a = wri.source_estimate(specs, wri.C64, workspace=work)
            for g in grads:
                g.zero_()
            f.zero_()
            gradient_of_solve(specs, opts, a, grads, f, work)
            if ws > 1:
                allreduce_gradient(grads, f)
            for gh, g in zip(g_host, grads):
                gh.copy_(g, non_blocking=True)
            f_host.copy_(f, non_blocking=True)
            a_host.copy_(a, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        c0, c1 = ev(), ev()
        ne = max(2, args.steps // 2)
        c0.record(stream)
        for _ in range(ne):
            e2e_step()
        c1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(c0.elapsed_time(c1) / 1e3)
        extras["e2e"] = {"value": ws * nsys * ne / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h}

    launches = step_launches(iters_done, int(opts.poll_every) or K_POLL, True, len(groups))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
                "config": {"workload": workload_name(args), "systems_per_gpu": nsys,
                           "iters_per_system": iters_done, "tol": 0.0,
                           "value_is": f"gradients per second at a fixed budget of {iters_done} CGLS iterations "
                                       "per system (every step the same work); at_tolerance holds the measured "
                                       "rate of gradients solved to tol 1e-2",
                           "nodes": [g.spec.n for g in groups],
                           "parallelism": f"data parallel x{ws}: one shot record per GPU, gradient all-reduce",
                           "precision": "certified: complex64 CGLS (FP32 stencils and vector updates, FP64 "
                                        "reductions and scalars) inside one FP64 iterative-refinement step (FP64 "
                                        "wavefield and normal-equation residual); FP64 source estimate on the FP64 "
                                        "wavefield and FP64 gradient from the refinement's FP64 residual",
                           "kernel": {"config": int(opts.kernel) - 2 if opts.kernel >= 2 else int(opts.kernel),
                                      "order": int(opts.order),
                                      "chosen_by": "wri_autotune" if args.kernel == 0 and args.order == 0
                                      else "command line"},
                           "l2": "working set >> L2 (no flush needed)"},
                "gpt_iter_s": gpt, "t_cg_iter_ms": t_iter * 1e3, "fp64_relres": relres_fp64,
                "roofline": roofline, "clocks": clk, "gpu_launches": launches * args.steps,
                "library": wri.version()}
        line.update(extras)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
