#!/usr/bin/env python3
"""Benchmark of the GB300 LASTO interstitial Poisson step.

Metric: converged Poisson solves per second (relative residual <= 1e-10), one
step = one whole solve (density, pseudo-density deposit, boundary multipoles,
faces, multigrid-preconditioned CG, sphere projection) of the Pd55 Mackay
icosahedron on the graded 129^3 mesh (0.12 -> 0.6 bohr, 10 bohr vacuum) with a
seeded synthetic Slater-model density.  `value` is the mixed-precision form
(FP32 multigrid preconditioner inside FP64 CG); the plain FP64 form is reported
beside it.  The 17-70 MB working set of this workload fits the 129 MB L2, so L2
is flushed (a 512 MiB write) before every timed step and each step is timed alone
with CUDA events on the launch stream.

`--impl reference` times the FP64 CPU oracle on the same workload and metric (the
reference arm; the paper publishes no implementation or timing).

Multi-GPU: the step does not shard; N ranks run N independent replicas (weak
scaling), value = solves of all ranks / max over ranks of the timed span.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged Poisson solves/sec (resid <=1e-10)"
UNIT = "solves/s"
WORKLOAD = "Pd55 Mackay icosahedron, graded 129^3 (0.12->0.6 bohr, 10 bohr vacuum), synthetic Slater density seed 1"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--quiet", action="store_true")
    p.add_argument("--no-batch64", action="store_true")
    p.add_argument("--profile", choices=["smoother", "solve"], default=None,
                   help="run one kernel family for a profiler and exit: 'smoother' = one FP32 red-black sweep "
                        "on an n^3 graded mesh, 'solve' = one mixed solve of the workload with direct launches")
    p.add_argument("--n", type=int, default=257, help="grid size of --profile smoother")
    p.add_argument("--direct", action="store_true",
                   help="launch the kernels directly instead of one CUDA graph per solve (for ncu)")
    return p.parse_args()


# ------------------------------------------------------------------ distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Largest value over the ranks (identity for one rank)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, ws: int, device=None) -> float:
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0, period_ms=100):
        self.idx, self.period, self.rows, self.proc = gpu_index, period_ms, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", f"-lms={self.period}"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ CPU oracle timing
def oracle_solves(cl, n_solves, tol=1e-10):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    out = None
    for _ in range(n_solves):
        out = oracle.poisson_solve(cl, tol=tol, max_cycles=200)
    dt = time.perf_counter() - t0
    return dt, out


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, one whole solve per step, on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    cl = synth.pd55_graded129()
    for _ in range(args.warmup):
        oracle_solves(cl, 1)
    times = []
    out = None
    for _ in range(args.steps):
        dt, out = oracle_solves(cl, 1)
        times.append(dt)
    total = sum(times)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": "129^3 graded", "precision": "f64 (CPU oracle, stationary V(2,2))",
                   "l2": "n/a (CPU)", "cycles": out["cycles"], "rel_resid": out["rel_resid"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": f"{args.steps} whole solves of the workload (after {args.warmup} warm-up)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import synth
    from paper_0806_1723_gb300 import binding as B

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    if args.profile:
        return run_profile(args, B)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    B.load()

    cl = synth.pd55_graded129()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(precision):
        return B.Poisson(n_max=cl.n, max_atoms=cl.n_atoms, precision=precision, launch=1 if args.direct else 0)

    dc = B.DeviceCluster(cl)
    vlm = torch.empty((cl.n_atoms, 25), dtype=torch.float64, device=dev)

    def timed_solves(solver, steps, warmup):
        st = None
        for _ in range(warmup):
            st = solver.solve(dc, vlm)
        torch.cuda.synchronize()
        assert st[0].status == 0 and st[0].rel_resid <= 1e-10, (st[0].status, st[0].rel_resid)
        fixed, per_it, per_out = solver.kernel_counts() if not args.direct else (0, 0, 0)
        ms, launches, cycles = [], 0, []
        for _ in range(steps):
            flush.fill_(1.0)                       # evict the working set from L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solver.solve(dc, vlm)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            cycles.append((st[0].cycles, st[0].outer))
            launches += fixed + st[0].cycles * per_it + st[0].outer * per_out
            assert st[0].status == 0 and st[0].rel_resid <= 1e-10
        return ms, launches, cycles, st[0]

    mixed, plain = make(B.LASTO_PREC_MIXED), make(B.LASTO_PREC_FP64)
    # warm both, then time the plain form and the chosen form with clock sampling
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms_plain, _, cyc_plain, st_plain = timed_solves(plain, args.steps, args.warmup)
        barrier(ws)
        torch.cuda.synchronize()
        ms_mixed, launches, cyc_mixed, st_mixed = timed_solves(mixed, args.steps, args.warmup)
        torch.cuda.synchronize()
        barrier(ws)
    span_ms = sum(ms_mixed)
    span_max = max_over_ranks(span_ms, ws, dev)
    value = (args.steps * ws) / (span_max / 1e3)
    plain_value = (args.steps * ws) / (max_over_ranks(sum(ms_plain), ws, dev) / 1e3)

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: torch.as_tensor(np.ascontiguousarray(getattr(cl, k), dtype=np.float64)).pin_memory()
                for k in ("pos", "Z", "R", "slater_w", "slater_zeta", "c_lm")}
        devbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
        vlm_host = torch.empty((cl.n_atoms, 25), dtype=torch.float64).pin_memory()
        dce = B.DeviceCluster(cl)
        dce.pos, dce.Z, dce.R = devbuf["pos"], devbuf["Z"], devbuf["R"]
        dce.w, dce.zeta, dce.clm = devbuf["slater_w"], devbuf["slater_zeta"], devbuf["c_lm"]
        axes = [torch.empty(cl.n, dtype=torch.float64, device=dev) for _ in range(3)]
        dce.x, dce.y, dce.z = axes
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = vlm_host.numel() * vlm_host.element_size()
        lib = B.load()

        def e2e_step():
            for k in host:
                devbuf[k].copy_(host[k], non_blocking=True)
            for a in range(3):
                lib.lasto_mesh_axis(cl.n, float(cl.centre[a]), cl.half_width, cl.h_min, cl.h_max, cl.p_max,
                                    B._ptr(axes[a]), None, B._stream(None))
            st = mixed.solve(dce, vlm)
            vlm_host.copy_(vlm, non_blocking=True)
            return st

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        ms_e2e = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = e2e_step()
            e1.record(stream)
            e1.synchronize()
            ms_e2e.append(e0.elapsed_time(e1))
            assert st[0].status == 0
        e2e_val = (args.steps * ws) / (max_over_ranks(sum(ms_e2e), ws, dev) / 1e3)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---------------- batched forms (one graph launch per batch, clusters as concurrent branches)
    batch8 = batch_throughput(B, [synth.pd55_graded129(seed=1 + k) for k in range(8)], B.LASTO_PREC_MIXED,
                              max(2, args.steps // 4), flush, stream, dev)
    b64 = None
    if not args.no_batch64:
        b64 = batch_throughput(B, synth.batch64(), B.LASTO_PREC_MIXED, 2, flush, stream, dev, warmup=1)

    # ---------------- roofline of the dominant kernel (FP32 red-black half sweep)
    roof = smoother_roofline(B, stream, flush, dev)
    dep = kernel_roofline(B, cl, dc, stream, flush, dev, 1)
    roof["deposit_fp32pair_ms"] = dep["ms"]
    roof["deposit_fp64_ms"] = kernel_roofline(B, cl, dc, stream, flush, dev, 0)["ms"]

    # ---------------- CPU baseline: the oracle as it stands, one whole solve
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, out = oracle_solves(cl, 1)
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": f"1 whole solve of the workload to 1e-10 ({out['cycles']} V(2,2) cycles), {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": span_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "FP64 defect correction around FP32 multigrid-preconditioned CG; FP32-pair density",
                       "l2": "flushed before every timed step (512 MiB write)", "cycles": cyc_mixed[-1][0], "defect_correction_steps": cyc_mixed[-1][1],
                       "rel_resid": st_mixed.rel_resid, "parallelism": f"replicas x{ws}"},
            "plain_fp64": {"value": plain_value, "unit": UNIT, "ms_per_step": sum(ms_plain) / args.steps,
                           "cycles": cyc_plain[-1][0], "rel_resid": st_plain.rel_resid},
            "batched_pd55x8": batch8,
            "batch64_uneven": b64,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_profile(args, B):
    """One kernel family for ncu (no timing of its own)."""
    import torch

    import synth
    if args.profile == "smoother":
        n = args.n
        axes = [B.lasto_mesh_axis(n, 0.0, 30.0, 0.12, 0.6, 6.0) for _ in range(3)]
        u = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
        b = torch.rand(n ** 3, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        B.lasto_op_smooth(*axes, u, b, sweeps=1)
    else:
        cl = synth.pd55_graded129()
        solver = B.Poisson(n_max=cl.n, max_atoms=cl.n_atoms, precision=B.LASTO_PREC_MIXED, launch=1)
        dc = B.DeviceCluster(cl)
        v = torch.empty((cl.n_atoms, 25), dtype=torch.float64, device="cuda")
        st = solver.solve(dc, v)
        torch.cuda.synchronize()
        assert st[0].status == 0
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "ok": True}))
    return 0


def batch_throughput(B, clusters, precision, steps, flush, stream, dev, warmup=2):
    """Solves/s of a batch of clusters solved in one call (one graph launch)."""
    import torch
    n_max = max(c.n for c in clusters)
    solver = B.Poisson(n_max=n_max, max_atoms=max(c.n_atoms for c in clusters), max_batch=len(clusters),
                       precision=precision)
    dcs = [B.DeviceCluster(c) for c in clusters]
    vlm = torch.empty((sum(c.n_atoms for c in clusters), 25), dtype=torch.float64, device=dev)
    for _ in range(warmup):
        st = solver.solve(dcs, vlm)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = solver.solve(dcs, vlm)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ok = all(s.status == 0 and s.rel_resid <= 1e-10 for s in st)
    solver.close()
    del dcs, vlm
    torch.cuda.empty_cache()
    return {"value": len(clusters) * steps / (sum(ms) / 1e3), "unit": UNIT, "clusters": len(clusters),
            "ms_per_batch": sum(ms) / steps, "all_converged": ok,
            "max_cycles": max(s.cycles for s in st), "nodes": sum(c.n ** 3 for c in clusters)}


def smoother_roofline(B, stream, flush, dev):
    """FP32 red-black half sweep on the 385^3 graded Pd561 mesh (456 MB of u and b, far beyond
    L2).  Algorithmic bytes per half sweep: every node's u read once (4 B), the colour's b read
    and u written (8 B per updated node) = 8 B per node.  Time per launch from a 1-sweep and a
    3-sweep call (the difference is 4 launches), L2 flushed before each call."""
    import json as _json
    import torch

    import synth
    cl = synth.pd561_graded385(n_densities=1)[0]
    n = cl.n
    axes = [B.lasto_mesh_axis(n, 0.0, cl.half_width, cl.h_min, cl.h_max, cl.p_max) for _ in range(3)]
    u = torch.zeros(n ** 3, dtype=torch.float32, device=dev)
    b = torch.rand(n ** 3, dtype=torch.float32, device=dev)

    def timed(sweeps):
        ts = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.lasto_op_smooth(*axes, u, b, sweeps=sweeps)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    timed(1)
    t_launch = (timed(3) - timed(1)) / 4 / 1e3
    bytes_per_launch = 8.0 * n ** 3
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = bytes_per_launch / t_launch / 1e9
    del u, b
    torch.cuda.empty_cache()
    return {"kernel": "k_rbgs<float> (red-black half sweep, 385^3 graded)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
            "bytes_per_launch": bytes_per_launch, "us_per_launch": t_launch * 1e6,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}


def kernel_roofline(B, cl, dc, stream, flush, dev, precision=1):
    """The deposit kernel family timed alone with CUDA events (median of 5, L2 flushed)."""
    import torch
    B.lasto_op_deposit(dc, precision=precision)   # warm
    torch.cuda.synchronize()
    ms = []
    for _ in range(5):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.lasto_op_deposit(dc, precision=precision)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) / 1e3
    pairs = cl.n ** 3 * cl.n_atoms
    return {"kernel": f"lasto_op_deposit precision={precision}", "bound": "alu", "unit": "Gpair/s",
            "achieved": pairs / t / 1e9, "peak": None, "frac": None, "traffic": None, "ms": t * 1e3}


if __name__ == "__main__":
    sys.exit(main())
