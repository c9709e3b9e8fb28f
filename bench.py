"""Benchmark of the batched SF-AWRI gradient (one JSON line on rank 0).

Workload (N = 1): the frequency-dependent batch of 128 surface sources x 3
frequencies (3 Hz on 64^3, 5 Hz on 96^3, 8 Hz on 128^3 physical nodes, each plus
a 10-cell absorbing layer: 84^3, 116^3, 148^3 computational nodes), 96 borehole
receivers, seeded layered + anomaly model, source-free mode, complex64 stencils with
FP64 reductions.  One step = one gradient evaluation of all 384 systems: right-hand
sides, ``--iters`` CGLS iterations per system (the fused, batched, graph-captured
phases), the source-weight estimates and the gradient/objective accumulation.

value = systems (source x frequency gradients) per second over all ranks.  The
working set (~40 GB) is far larger than L2, so no flush is needed between steps.
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
BYTES_PER_NODE_ITER = 80.0   # algorithmic bytes of one fused CGLS iteration per node and system (c64)
MODEL_BYTES = 8.0            # m read by both phases (float32), shared by the systems of a group


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
    p.add_argument("--order", type=int, default=0,
                   help="TMA work order: 0 auto, 1 system-major, 2 tile-major, 3 z-chunk-major")
    p.add_argument("--zsplit", type=int, default=0, help="z-chunks per tile column (0 = library choice)")
    p.add_argument("--promo", type=int, default=0, help="TMA L2 promotion: 0 auto, 1 none, 2 64B, 3 128B, 4 256B")
    return p.parse_args()


def workload(nsrc, small):
    import synth
    if small:
        return synth.workload_c4(nsrc=min(nsrc, 8), freqs=((3.0, 24), (5.0, 32), (8.0, 40)), nrec=24)
    return synth.workload_c4(nsrc=nsrc)


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
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull if False else "/tmp/wri_clocks.csv", "w")
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
        for line in open("/tmp/wri_clocks.csv"):
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(grp, iters=25):
    """Oracle CGLS (scipy.sparse, complex128) on one system: seconds per iteration."""
    import numpy as np

    import oracle as O
    n = grp.spec.n
    A = O.helmholtz_matrix(grp.spec.shape, grp.spec.h, grp.omega, grp.m, grp.spec.npml, grp.v_max, grp.pml_R)
    rec = grp.rec_idx[grp.rec_off[0]:grp.rec_off[1]]
    S = O.augmented_operator(A, O.restriction(n, rec), grp.src[0], grp.lam, True)
    b = O.rhs(n, grp.src[0], grp.d[grp.rec_off[0]:grp.rec_off[1]], grp.lam)
    t0 = time.perf_counter()
    O.cgls(S, b, tol=0.0, max_iter=2)
    t1 = time.perf_counter()
    O.cgls(S, b, tol=0.0, max_iter=2 + iters)
    t2 = time.perf_counter()
    return ((t2 - t1) - (t1 - t0)) / iters, (t2 - t0) + (t1 - t0)


def cpu_equivalent(groups, iters):
    """CPU-oracle throughput for the bench step, from a bounded sample on the largest grid."""
    big = max(groups, key=lambda g: g.spec.n)
    per_it, secs = cpu_oracle_rate(big)
    rate = big.spec.n / per_it                       # node-iterations per second (one system)
    node_iters = sum(g.nsys * g.spec.n for g in groups) * iters
    step_s = node_iters / rate
    nsys = sum(g.nsys for g in groups)
    return {"value": nsys / step_s, "gpt_iter_s": rate / 1e9, "cores": 1, "kind": "oracle",
            "sample": f"oracle CGLS (scipy.sparse complex128, serial) on 1 system of the "
                      f"{big.spec.nx}^3 group, 25 iterations ({secs:.1f} s incl. warm-up); per-node rate "
                      f"scaled to {nsys} systems x {iters} iterations", "unit": "src·freq/s"}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    groups = workload(args.nsrc, args.small)
    cb = cpu_equivalent(groups, args.iters)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "src·freq/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "ms_per_step": 1e3 * sum(g.nsys for g in groups) / cb["value"],
            "config": {"workload": "c4-batch", "iters_per_system": args.iters},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "src·freq/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2410_18429_gb300 import wri
    from paper_2410_18429_gb300.problem import to_device
    from paper_2410_18429_gb300.parallel_sum import allreduce_gradient

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    groups = workload(args.nsrc, args.small)
    if args.only_group >= 0:
        groups = [groups[args.only_group]]
    specs = [to_device(g, wri.C64, dev) for g in groups]
    nsys = sum(g.nsys for g in groups)
    n_nodes = [g.spec.n for g in groups]
    K = 2
    opts = wri.make_opts(tol=0.0, max_iter=args.iters, dtype=wri.C64, poll_every=K, kernel=args.kernel, order=args.order,
                         zsplit=args.zsplit, l2_promotion=args.promo)
    wsz = wri.workspace_size(specs, opts)
    work = torch.empty(wsz, dtype=torch.uint8, device=dev)
    grads = [torch.zeros(g.spec.nz, g.spec.ny, g.spec.nx, dtype=torch.float64, device=dev) for g in groups]
    f = torch.zeros(1, dtype=torch.float64, device=dev)

    def step():
        it, rr, st = wri.solve(specs, opts, workspace=work)
        a = wri.source_estimate(specs, wri.C64, workspace=work)
        for g in grads:
            g.zero_()
        f.zero_()
        wri.gradient(specs, wri.C64, a, grads=grads, f=f, workspace=work)
        if ws > 1:
            allreduce_gradient(grads, f)
        return it

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        it = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    iters_done = int(it.min().item())
    value = ws * nsys * args.steps / t
    node_iters = sum(g.nsys * g.spec.n for g in groups) * iters_done
    gpt = ws * node_iters * args.steps / t / 1e9

    # ---- roofline of the fused CG iteration (phase 1 + phase 2 kernels), live with CUDA events
    def timed_solve(iters):
        o = wri.make_opts(tol=0.0, max_iter=iters, dtype=wri.C64, poll_every=K, kernel=args.kernel, order=args.order,
                         zsplit=args.zsplit, l2_promotion=args.promo)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        wri.solve(specs, o, workspace=work)
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / 1e3

    timed_solve(10)
    ta, tb = timed_solve(10), timed_solve(70)
    t_iter = (tb - ta) / 60.0
    alg_bytes = sum(g.nsys * g.spec.n * BYTES_PER_NODE_ITER + g.spec.n * MODEL_BYTES for g in groups)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = alg_bytes / t_iter / 1e9
    traffic = None
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "cg_iteration_traffic.json")))
        if prof.get("kernel_version") == wri.version():
            traffic = prof.get("bytes_per_iteration")
    except OSError:
        pass
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_march phase1+phase2 (one fused CGLS iteration, all systems)",
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    extras = {}
    if not args.no_extras and rank == 0:
        # ---- plain (unbatched, unfused, host-read scalars) path on one system of the largest grid
        import synth
        big_i = max(range(len(groups)), key=lambda i: groups[i].spec.n)
        g0 = groups[big_i]
        one = synth.Group(g0.spec, g0.freq, g0.v, g0.src[:1], g0.rec_off[:2] - g0.rec_off[0],
                          g0.rec_idx[g0.rec_off[0]:g0.rec_off[1]], g0.lam, g0.v_max, g0.pml_R, g0.alpha[:1],
                          g0.d[g0.rec_off[0]:g0.rec_off[1]])
        sp1 = to_device(one, wri.C64, dev)

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
        fused_per_sys_iter_big = t_iter * (g0.spec.n / sum(g.nsys * g.spec.n for g in groups))
        plain_step = sum(g.nsys * g.spec.n for g in groups) * iters_done * plain_per_sys_iter / g0.spec.n
        extras["plain"] = {"per_system_iter_ms_148": plain_per_sys_iter * 1e3,
                           "fused_per_system_iter_ms_148": fused_per_sys_iter_big * 1e3,
                           "speedup_per_iteration": plain_per_sys_iter / fused_per_sys_iter_big,
                           "value_equivalent": nsys / plain_step}
        del sp1

        # ---- end to end through the public API with host buffers
        m_host = [torch.from_numpy(np.ascontiguousarray(g.m, dtype=np.float32).reshape(g.spec.shape)).pin_memory()
                  for g in groups]
        d_host = [torch.from_numpy(np.ascontiguousarray(g.d, dtype=np.complex64)).pin_memory() for g in groups]
        g_host = [torch.empty(g.spec.shape, dtype=torch.float64).pin_memory() for g in groups]
        f_host = torch.empty(1, dtype=torch.float64).pin_memory()
        a_host = torch.empty(nsys, dtype=torch.complex128).pin_memory()
        h2d = sum(x.numel() * x.element_size() for x in m_host + d_host)
        d2h = sum(x.numel() * x.element_size() for x in g_host) + 8 + a_host.numel() * 16

        def e2e_step():
            for s, mh, dh in zip(specs, m_host, d_host):
                s.m.copy_(mh, non_blocking=True)
                s.d.copy_(dh, non_blocking=True)
            wri.solve(specs, opts, workspace=work)
            a = wri.source_estimate(specs, wri.C64, workspace=work)
            for g in grads:
                g.zero_()
            f.zero_()
            wri.gradient(specs, wri.C64, a, grads=grads, f=f, workspace=work)
            for gh, g in zip(g_host, grads):
                gh.copy_(g, non_blocking=True)
            f_host.copy_(f, non_blocking=True)
            a_host.copy_(a, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ne = max(2, args.steps // 2)
        c0.record(stream)
        for _ in range(ne):
            e2e_step()
        c1.record(stream)
        torch.cuda.synchronize()
        te = c0.elapsed_time(c1) / 1e3
        extras["e2e"] = {"value": nsys * ne / te, "unit": "src·freq/s", "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h}
        if ws == 1:
            extras["cpu_baseline"] = cpu_equivalent(groups, iters_done)

    # kernel launches per step: setup + init + export, 2 per CG iteration (graph batches of K), estimate,
    # gradient + data term
    graph_launches = -(-(iters_done + 1) // K)
    launches = 3 + 2 * K * graph_launches + 1 + 2
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "src·freq/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp64 reductions)", "data": "synthetic",
                "config": {"workload": "c4-batch: 128 src x {3 Hz 84^3, 5 Hz 116^3, 8 Hz 148^3}"
                                       if not args.small else "c4-batch-small",
                           "systems": nsys, "iters_per_system": iters_done, "tol": 0.0,
                           "nodes": n_nodes, "parallelism": f"replicas x{ws} (sources sharded, gradient all-reduce)",
                           "l2": "working set >> L2 (no flush needed)"},
                "gpt_iter_s": gpt, "t_cg_iter_ms": t_iter * 1e3, "roofline": roofline, "clocks": clk,
                "gpu_launches": launches * args.steps}
        line.update(extras)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
