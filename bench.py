#!/usr/bin/env python3
"""Benchmark of the GB300 LASTO interstitial Poisson step.

Metric: converged Poisson solves per second (relative residual <= 1e-10).  One solve =
density, pseudo-density deposit, boundary multipoles, faces, iteration to 1e-10, sphere
projection, for a Pd55 Mackay icosahedron on the graded 129^3 mesh (0.12 -> 0.6 bohr,
10 bohr vacuum) with a seeded synthetic Slater-model density.

`value` is the chosen form: 8 such clusters (density seeds 1..8) per call, solved as
independent branches of one CUDA graph, each started from the learned guess (the U-Net
runs inside the graph, once for the batch), with FP64 defect correction around FP32
multigrid-preconditioned CG and the FP32-pair density deposit.  A step is one batch of 8
solves.  The plain form (one cluster per call, zero start, FP64 throughout) is timed in the
same clock-sampled region and reported beside it, as are the forms between the two.  The
working set fits the 129 MB L2, so L2 is flushed (a 512 MiB write) before every timed step
and each step is timed alone with CUDA events on the launch stream.

`--impl reference` times the FP64 CPU oracle on the same workload and metric (the
reference arm; the paper publishes no implementation or timing).

Multi-GPU: the step does not shard; N ranks run N independent replicas (weak scaling),
value = solves of all ranks / max over ranks of the timed span.
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
WORKLOAD = ("Pd55 Mackay icosahedron, graded 129^3 (0.12->0.6 bohr, 10 bohr vacuum), synthetic Slater densities; "
            "8 clusters (density seeds 1-8) per step")
FORM = ("learned initial guess (U-Net in the graph) + FP64 defect correction around FP32 multigrid-preconditioned CG "
        "+ FP32-pair density; 8 clusters per graph launch")
BATCH = 8


# ncu dram__bytes_read.sum + dram__bytes_write.sum per half sweep at 257^3, one block per row, in
# steady state (launches 5-8 of 4 sweeps, caches not flushed between launches, so each launch also
# writes back what the one before left dirty in L2): mean of the four launches, by launch shape
# (0 = one block per row, else threads per block).  FP32 rows: 130.3 MB read + 67.6 MB written,
# flat 128: 129.3 + 66.3, flat 256: 129.5 + 66.3; FP64 rows: 403.3 + 134.5 MB.  A launch shape
# without a capture reports null.
DRAM_BYTES_257 = {0: 197.9e6, 128: 195.6e6, 256: 195.8e6}
DRAM_BYTES_257_F64 = 537.7e6

# FP64 FMA throughput of one GB300 (a DFMA chain over every SM, CUDA events: 1.19 TFLOP/s at
# 1995 MHz); the copy and BF16 peaks come from the measured-peaks file
FP64_TFLOPS = 1.19


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
    p.add_argument("--no-pd561", action="store_true")
    p.add_argument("--no-hs", action="store_true")
    p.add_argument("--profile", choices=["smoother", "solve", "guess", "pd561", "hs", "batch"], default=None,
                   help="run one kernel family for a profiler and exit: 'smoother' = one FP32 red-black sweep "
                        "on an n^3 graded mesh, 'solve' = one mixed solve of the workload with direct launches, "
                        "'guess' = the same with the learned initial guess, 'pd561' = one chosen-form solve "
                        "of the Pd561 graded 385^3 workload with direct launches, 'hs' = one interstitial H and S "
                        "call (tensor cores) for Pd55 on the graded 129^3 mesh, 'batch' = one graph launch of the "
                        "chosen form over the 8 Pd55 clusters of the workload (for ncu --graph-profiling graph)")
    p.add_argument("--n", type=int, default=257, help="grid size of --profile smoother")
    p.add_argument("--threads", type=int, default=256,
                   help="launch shape of --profile smoother: threads per block, 0 = one block per row")
    p.add_argument("--sweeps", type=int, default=1, help="red-black sweeps of --profile smoother")
    p.add_argument("--fp64", action="store_true", help="--profile smoother in FP64 (the plain form's smoother)")
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

    cls8 = [synth.pd55_graded129(seed=1 + k) for k in range(BATCH)]
    cl = cls8[0]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    launch = 1 if args.direct else 0

    def make(precision, batch=1, guess=False):
        s_ = B.Poisson(n_max=cl.n, max_atoms=cl.n_atoms, max_batch=batch, precision=precision, launch=launch)
        if guess:
            s_.set_guess()
        return s_

    dcs8 = [B.DeviceCluster(c) for c in cls8]
    vlm8 = torch.empty((BATCH * cl.n_atoms, 25), dtype=torch.float64, device=dev)
    dc = dcs8[0]
    vlm = vlm8[:cl.n_atoms]

    def timed(solver, dcs, out, steps, warmup):
        """steps timed calls (L2 flushed before each); kernel launches counted from the graph."""
        st = None
        for _ in range(warmup):
            st = solver.solve(dcs, out)
        torch.cuda.synchronize()
        assert all(x.status == 0 and x.rel_resid <= 1e-10 for x in st), [(x.status, x.rel_resid) for x in st]
        fixed, per_it, per_out = solver.kernel_counts() if not args.direct else (0, 0, 0)
        ms, launches = [], 0
        for _ in range(steps):
            flush.fill_(1.0)                       # evict the working set from L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solver.solve(dcs, out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            launches += fixed + sum(x.cycles * per_it + x.outer * per_out for x in st)
            assert all(x.status == 0 and x.rel_resid <= 1e-10 for x in st)
        return {"ms": ms, "launches": launches, "stats": list(st)}

    def summary(r, nclusters):
        st = r["stats"]
        return {"value": nclusters * len(r["ms"]) / (sum(r["ms"]) / 1e3), "unit": UNIT,
                "ms_per_call": sum(r["ms"]) / len(r["ms"]), "clusters_per_call": nclusters,
                "cycles": [x.cycles for x in st], "outer": [x.outer for x in st],
                "max_rel_resid": max(x.rel_resid for x in st), "learned_guess": [x.guess for x in st]}

    plain = make(B.LASTO_PREC_FP64)
    chosen = make(B.LASTO_PREC_MIXED, BATCH, guess=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        r_plain = timed(plain, dc, vlm, args.steps, args.warmup)
        barrier(ws)
        torch.cuda.synchronize()
        r_chosen = timed(chosen, dcs8, vlm8, args.steps, args.warmup)
        torch.cuda.synchronize()
        barrier(ws)
    tuned = [line.split() for line in chosen.tune_table().strip().splitlines()]
    smoother_choice = {f"{r[0]}x{r[1]}x{r[2]}/{'f32' if r[3] == '4' else 'f64'}":
                       ((f"in-place half sweeps, {r[5]} threads" if r[5] != "0" else "in-place half sweeps, one block per row")
                        if r[4] == "0" else
                        f"fused {r[9]}-sweep passes, tile {r[6]}x{r[7]}x{r[8]}") + f" ({float(r[10]):.1f} us)"
                       for r in tuned}
    span_max = max_over_ranks(sum(r_chosen["ms"]), ws, dev)
    value = (BATCH * args.steps * ws) / (span_max / 1e3)
    plain_value = (args.steps * ws) / (max_over_ranks(sum(r_plain["ms"]), ws, dev) / 1e3)

    # ---------------- the forms between plain and chosen (one factor at a time)
    steps_b = max(3, args.steps // 4)
    mixed1 = make(B.LASTO_PREC_MIXED)
    forms = {"mixed_single": summary(timed(mixed1, dc, vlm, steps_b, 2), 1)}
    mixed1.set_guess()
    forms["mixed_learned_single"] = summary(timed(mixed1, dc, vlm, steps_b, 2), 1)
    mixed1.close()
    mixed8 = make(B.LASTO_PREC_MIXED, BATCH)
    forms["mixed_batched"] = summary(timed(mixed8, dcs8, vlm8, steps_b, 2), BATCH)
    mixed8.close()

    # ---------------- end to end through the C ABI with host buffers (the chosen form)
    e2e = None
    if not args.no_e2e:
        fields = ("pos", "Z", "R", "slater_w", "slater_zeta", "c_lm")
        host = [{k: torch.as_tensor(np.ascontiguousarray(getattr(c, k), dtype=np.float64)).pin_memory()
                 for k in fields} for c in cls8]
        devbuf = [{k: torch.empty_like(v, device=dev) for k, v in hb.items()} for hb in host]
        vlm_host = torch.empty((BATCH * cl.n_atoms, 25), dtype=torch.float64).pin_memory()
        dces = []
        for c, dbuf in zip(cls8, devbuf):
            d = B.DeviceCluster(c)
            d.pos, d.Z, d.R = dbuf["pos"], dbuf["Z"], dbuf["R"]
            d.w, d.zeta, d.clm = dbuf["slater_w"], dbuf["slater_zeta"], dbuf["c_lm"]
            d.x, d.y, d.z = (torch.empty(c.n, dtype=torch.float64, device=dev) for _ in range(3))
            dces.append(d)
        h2d = sum(v.numel() * v.element_size() for hb in host for v in hb.values())
        d2h = vlm_host.numel() * vlm_host.element_size()
        lib = B.load()

        def e2e_step():
            for hb, dbuf in zip(host, devbuf):
                for k in fields:
                    dbuf[k].copy_(hb[k], non_blocking=True)
            for c, d in zip(cls8, dces):
                for a, ax in enumerate((d.x, d.y, d.z)):
                    lib.lasto_mesh_axis(c.n, float(c.centre[a]), c.half_width, c.h_min, c.h_max, c.p_max,
                                        B._ptr(ax), None, B._stream(None))
            st = chosen.solve(dces, vlm8)
            vlm_host.copy_(vlm8, non_blocking=True)
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
            assert all(x.status == 0 for x in st)
        e2e_val = (BATCH * args.steps * ws) / (max_over_ranks(sum(ms_e2e), ws, dev) / 1e3)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---------------- the uneven batch of 64 (Pd13/55/147 on 65^3 .. 193^3), chosen form
    b64 = None
    if not args.no_batch64:
        b64 = batch_throughput(B, synth.batch64(), B.LASTO_PREC_MIXED, 2, flush, stream, dev, warmup=1, guess=True)

    # ---------------- Pd561 on the graded 385^3 mesh: 8 SCF-like densities back to back
    pd561 = None
    if not args.no_pd561:
        pd561 = pd561_sequence(B, synth, flush, stream, dev)

    # ---------------- the interstitial H and S contraction (Eq. 3.11-3.14)
    hs = None
    if not args.no_hs:
        hs = interstitial_hs(B, synth, flush, stream, dev)

    # ---------------- the inner Dirichlet problem, exact faces and raw-density deposit
    rows = None
    if not args.no_hs:
        rows = next_rows(B, synth, flush, stream, dev)

    # ---------------- roofline of the dominant kernel (FP32 red-black half sweep)
    roof = smoother_roofline(B, stream, flush, dev)
    roof["deposit_fp32pair_ms"] = kernel_roofline(B, cl, dc, stream, flush, dev, 1)["ms"]
    roof["deposit_fp64_ms"] = kernel_roofline(B, cl, dc, stream, flush, dev, 0)["ms"]

    # ---------------- CPU baseline: the oracle as it stands, one whole solve
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, out = oracle_solves(cl, 1)
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": f"1 whole solve of one cluster of the workload to 1e-10 ({out['cycles']} V(2,2) cycles), "
                         f"{dt:.1f} s"}

    if rank == 0:
        ch = summary(r_chosen, BATCH)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": span_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32+bf16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": FORM, "l2": "flushed before every timed step (512 MiB write)",
                       "cycles": ch["cycles"], "defect_correction_steps": ch["outer"],
                       "max_rel_resid": ch["max_rel_resid"], "parallelism": f"replicas x{ws}",
                       "smoother_tuned": smoother_choice},
            "plain_fp64": {"value": plain_value, "unit": UNIT, "ms_per_step": sum(r_plain["ms"]) / args.steps,
                           "cycles": r_plain["stats"][0].cycles, "rel_resid": r_plain["stats"][0].rel_resid,
                           "form": "one cluster per call, zero start, FP64 deposit and FP64 multigrid-preconditioned CG"},
            "chosen_over_plain": value / plain_value,
            "forms": forms,
            "batch64_uneven": b64,
            "pd561_graded385": pd561,
            "interstitial_hs": hs,
            "inner_faces_raw": rows,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": r_chosen["launches"],
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
    if args.profile == "hs":
        cl = synth.pd55_graded129()
        dc = B.DeviceCluster(cl)
        x, y, z = (t.cpu().numpy() for t in (dc.x, dc.y, dc.z))
        V = torch.as_tensor(synth.potential_energy(cl.pos, x, y, z, seed=5)).cuda()
        B.lasto_op_interstitial_hs(dc.x, dc.y, dc.z, dc.pos, dc.R, V)   # untimed first call
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        B.lasto_op_interstitial_hs(dc.x, dc.y, dc.z, dc.pos, dc.R, V)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif args.profile == "batch":
        cls = [synth.pd55_graded129(seed=1 + k) for k in range(BATCH)]
        solver = B.Poisson(n_max=cls[0].n, max_atoms=cls[0].n_atoms, max_batch=BATCH, precision=B.LASTO_PREC_MIXED)
        solver.set_guess()
        dcs = [B.DeviceCluster(c) for c in cls]
        v = torch.empty((BATCH * cls[0].n_atoms, 25), dtype=torch.float64, device="cuda")
        st = solver.solve(dcs, v)     # first solve: smoother tuning, graph capture
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        st = solver.solve(dcs, v)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        assert all(x.status == 0 for x in st)
    elif args.profile == "smoother":
        n = args.n
        axes = [B.lasto_mesh_axis(n, 0.0, 30.0, 0.12, 0.6, 6.0) for _ in range(3)]
        dt = torch.float64 if args.fp64 else torch.float32
        u = torch.zeros(n ** 3, dtype=dt, device="cuda")
        b = torch.rand(n ** 3, dtype=dt, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        B.lasto_op_smooth(*axes, u, b, sweeps=args.sweeps, threads=args.threads)
    else:
        cl = synth.pd561_graded385(n_densities=1)[0] if args.profile == "pd561" else synth.pd55_graded129()
        solver = B.Poisson(n_max=cl.n, max_atoms=cl.n_atoms, precision=B.LASTO_PREC_MIXED, launch=1)
        if args.profile in ("guess", "pd561"):
            solver.set_guess()
        # under a profiler the tuner's timings mean nothing; take the choice it makes without one
        # on these levels (in-place half sweeps, 256 threads)
        sizes, m = [], cl.n
        while m > 9:
            sizes.append(m)
            m = (m + 1) // 2
        solver.set_tune_table("".join(f"{m} {m} {m} 4 0 256 0 0 0 0 0\n" for m in sizes))
        dc = B.DeviceCluster(cl)
        v = torch.empty((cl.n_atoms, 25), dtype=torch.float64, device="cuda")
        st = solver.solve(dc, v)      # first solve: smoother tuning, network upload
        torch.cuda.synchronize()
        torch.cuda.profiler.start()   # ncu --profile-from-start off captures this solve only
        st = solver.solve(dc, v)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        assert st[0].status == 0
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "ok": True}))
    return 0


def batch_throughput(B, clusters, precision, steps, flush, stream, dev, warmup=2, guess=False):
    """Solves/s of a batch of clusters solved in one call (one graph launch)."""
    import torch
    n_max = max(c.n for c in clusters)
    solver = B.Poisson(n_max=n_max, max_atoms=max(c.n_atoms for c in clusters), max_batch=len(clusters),
                       precision=precision)
    if guess:
        solver.set_guess()
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
            "ms_per_batch": sum(ms) / steps, "all_converged": ok, "mean_cycles": sum(s.cycles for s in st) / len(st),
            "max_cycles": max(s.cycles for s in st), "learned_guess": sum(s.guess for s in st),
            "nodes": sum(c.n ** 3 for c in clusters)}


def pd561_sequence(B, synth, flush, stream, dev):
    """Chosen form (learned guess, FP64 defect correction around FP32 multigrid-preconditioned
    CG) on 8 successive Pd561 densities (graded 385^3, 57 M nodes), one solve per call, after
    one untimed solve; the plain FP64 form on the first density for comparison."""
    import torch
    cls = synth.pd561_graded385()
    c0 = cls[0]
    mk = lambda prec: B.Poisson(n_max=c0.n, max_atoms=c0.n_atoms, precision=prec)
    out = {}
    for name, prec, seq in (("chosen", B.LASTO_PREC_MIXED, cls), ("plain_fp64", B.LASTO_PREC_FP64, cls[:1])):
        solver = mk(prec)
        if name == "chosen":
            solver.set_guess()
        v = torch.empty((c0.n_atoms, 25), dtype=torch.float64, device=dev)
        dc = B.DeviceCluster(c0)
        st = solver.solve(dc, v)   # capture, tuning
        torch.cuda.synchronize()
        ms, cyc, res = [], [], []
        for c in seq:
            dc = B.DeviceCluster(c)
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solver.solve(dc, v)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            cyc.append(st[0].cycles)
            res.append(st[0].rel_resid)
            assert st[0].status == 0 and st[0].rel_resid <= 1e-10
        out[name] = {"value": len(seq) / (sum(ms) / 1e3), "unit": UNIT, "ms_per_solve": sum(ms) / len(seq),
                     "cycles": cyc, "max_rel_resid": max(res), "learned_guess": st[0].guess}
        if name == "chosen":
            out["smoother_tuned"] = solver.tune_table().strip().splitlines()
        solver.close()
        del v, dc
        torch.cuda.empty_cache()
    out["nodes"] = c0.n ** 3
    out["chosen_over_plain"] = out["chosen"]["value"] / out["plain_fp64"]["value"]
    return out


def interstitial_hs(B, synth, flush, stream, dev):
    """The interstitial H and S contributions (Eq. 3.11-3.14) of Table 1's basis (25 functions
    per Pd atom) for Pd55 on the graded 129^3 mesh, V a seeded potential-energy field: the
    whole call and its stages (CUDA events inside the call), tensor-core and SIMT contractions.
    Tensor-pipe work per interstitial node: 9 MMAs of 128 x 128 x 16 per 16 nodes per
    upper-triangle tile pair (3 for S, 6 for 2H, hi*hi + hi*lo + lo*hi each); algorithmic work:
    6 flops per node per (a <= b) entry (S: 1 product, 2H: 2)."""
    import json as _json
    import torch
    cl = synth.pd55_graded129()
    dc = B.DeviceCluster(cl)
    x, y, z = (t.cpu().numpy() for t in (dc.x, dc.y, dc.z))
    V = torch.as_tensor(synth.potential_energy(cl.pos, x, y, z, seed=5)).to(dev)
    out = {"workload": f"{cl.name}, Table 1 basis (25 functions per atom)"}
    for name, mode in (("tensor", B.LASTO_HS_TENSOR), ("simt", B.LASTO_HS_SIMT)):
        st = B.lasto_hs_stats()
        B.lasto_op_interstitial_hs(dc.x, dc.y, dc.z, dc.pos, dc.R, V, mode=mode)   # warm-up
        ms = []
        for _ in range(3 if name == "tensor" else 1):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S, H = B.lasto_op_interstitial_hs(dc.x, dc.y, dc.z, dc.pos, dc.R, V, mode=mode, stats=st)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[name] = {"ms": min(ms), "ms_contract": st.ms_contract, "ms_tables": st.ms_tables, "ms_list": st.ms_list,
                     "ms_mirror": st.ms_mirror, "chunks": st.chunks, "tile": st.tile}
        M = S.shape[0]
        nodes = st.interstitial_nodes
        out["M"], out["interstitial_nodes"] = M, nodes
        del S, H
    nT = (out["M"] + 127) // 128
    pairs = nT * (nT + 1) // 2
    tensor_flops = 9 * 2 * 128 * 128 * pairs * out["interstitial_nodes"]
    alg_flops = 6 * (out["M"] * (out["M"] + 1) // 2) * out["interstitial_nodes"]
    peaks = {}
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    # the MMAs are kind::f16 on FP16 operands: the dense FP16 rate equals the BF16 one
    f16_peak = peaks.get("bf16_tflops", 1900.0)
    t = out["tensor"]["ms_contract"] / 1e3
    out["roofline"] = {"kernel": "k_hs_gemm_tc", "bound": "tensor", "achieved": tensor_flops / t / 1e12,
                       "peak": f16_peak, "unit": "TFLOP/s", "frac": tensor_flops / t / 1e12 / f16_peak,
                       "traffic": None,
                       "peak_source": ("measured bf16 burst (FP16 dense rate = BF16)" if "bf16_tflops" in peaks
                                       else "fallback bf16 burst")}
    out["algorithmic_tflops"] = {"tensor": alg_flops / t / 1e12,
                                 "simt": alg_flops / (out["simt"]["ms_contract"] / 1e3) / 1e12}
    out["tensor_over_simt"] = out["simt"]["ms"] / out["tensor"]["ms"]
    return out


def next_rows(B, synth, flush, stream, dev):
    """The rows built beyond the Poisson step, each timed alone with CUDA events (median of 5,
    L2 flushed) on the Pd55 graded 129^3 workload: the inner Dirichlet problem (Eq. 3.4-3.7:
    rho_LM on the 429-point logarithmic mesh of every sphere, then the radial solve), the
    exact-superposition faces (f2) and the raw-density deposit (Eq. 3.1, f4; its inputs are the
    model's deposit and the GPU's rho_00 tables, which only set the values, not the cost)."""
    import torch
    cl = synth.pd55_graded129()
    dc = B.DeviceCluster(cl)
    na, n_rad, nq = cl.n_atoms, 429, 16 * 32

    def median_ms(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(5):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    rho, _ = B.lasto_op_sphere_density(dc, n_rad=n_rad)
    vR = torch.zeros((na, 25), dtype=torch.float64, device=dev)
    t_sd = median_ms(lambda: B.lasto_op_sphere_density(dc, n_rad=n_rad))
    t_in = median_ms(lambda: B.lasto_op_inner_solve(dc.R, dc.Z, rho, vR))
    u = torch.zeros((cl.n,) * 3, dtype=torch.float64, device=dev)
    t_bx = median_ms(lambda: B.lasto_op_boundary_exact(dc, u))
    b, _, _ = B.lasto_op_deposit(dc, precision=B.LASTO_PREC_MIXED)
    rc = B.RawCluster(cl.pos, cl.Z, cl.R, dc.x, dc.y, dc.z, cl.centre, (b / (4 * 3.141592653589793)).reshape(-1),
                      rho[:, 0, :].contiguous())
    t_raw = median_ms(lambda: B.lasto_op_raw_deposit(rc))
    t_dep = median_ms(lambda: B.lasto_op_deposit(dc, precision=B.LASTO_PREC_MIXED))
    faces = 6 * cl.n * cl.n
    return {
        "workload": cl.name,
        "inner_sphere_density": {"ms": t_sd, "unit": "Gpair/s",
                                 "achieved": na * n_rad * nq * na / (t_sd / 1e3) / 1e9,
                                 "work": f"{na} spheres x {n_rad} radii x {nq} quadrature points x {na} atoms"},
        "inner_solve": {"ms": t_in, "points": na * 25 * n_rad},
        "boundary_exact": {"ms": t_bx, "unit": "Gpair/s", "achieved": faces * na / (t_bx / 1e3) / 1e9,
                           "work": f"{faces} face nodes x {na} atoms"},
        "raw_deposit": {"ms": t_raw, "model_deposit_ms": t_dep},
    }


def smoother_roofline(B, stream, flush, dev):
    """FP32 red-black half sweep on the 385^3 graded Pd561 mesh (456 MB of u and b, far beyond
    L2).  Algorithmic bytes per half sweep: every node's u read once (4 B), the colour's b read
    and u written (8 B per updated node) = 8 B per node.  Time per launch from a 1-sweep and a
    3-sweep call (the difference is 4 launches), L2 flushed before each call, for each launch
    shape the solver's tuner chooses among; the fastest is reported."""
    import json as _json
    import torch

    import synth
    cl = synth.pd561_graded385(n_densities=1)[0]
    n = cl.n
    axes = [B.lasto_mesh_axis(n, 0.0, cl.half_width, cl.h_min, cl.h_max, cl.p_max) for _ in range(3)]
    u = torch.zeros(n ** 3, dtype=torch.float32, device=dev)
    b = torch.rand(n ** 3, dtype=torch.float32, device=dev)

    def timed(sweeps, threads):
        ts = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.lasto_op_smooth(*axes, u, b, sweeps=sweeps, threads=threads)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    # the launch shapes the solver's tuner chooses among (flat 128/256/512, one block per row)
    per = {}
    for threads in (0, 128, 256, 512):
        timed(1, threads)
        per[threads] = (timed(3, threads) - timed(1, threads)) / 4 / 1e3
    best = min(per, key=per.get)
    t_launch = per[best]
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
    # DRAM bytes per launch: ncu dram__bytes_read.sum + dram__bytes_write.sum of the chosen
    # launch shape at 257^3 (steady state), scaled by the node count
    traffic_257 = DRAM_BYTES_257.get(best)
    traffic = traffic_257 * (n / 257.0) ** 3 if traffic_257 else None
    name = "k_rbgs_row<float>, one block per row" if best == 0 else f"k_rbgs<float>, {best} threads per block"
    return {"kernel": f"{name} (red-black half sweep, 385^3 graded)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "bytes_per_launch": bytes_per_launch, "us_per_launch": t_launch * 1e6,
            "us_per_launch_by_shape": {("rows" if k == 0 else str(k)): v * 1e6 for k, v in per.items()},
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "plain_fp64": fp64_half_sweep(B, cl, axes, timed_fn=lambda uu, bb, sw, th: _timed_smooth(
                B, axes, uu, bb, sw, th, flush, stream), peak=peak)}


def _timed_smooth(B, axes, u, b, sweeps, threads, flush, stream):
    import torch
    ts = []
    for _ in range(3):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.lasto_op_smooth(*axes, u, b, sweeps=sweeps, threads=threads)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def fp64_half_sweep(B, cl, axes, timed_fn, peak):
    """The plain form's FP64 red-black half sweep at the same 385^3 mesh, one block per row.
    Algorithmic bytes per launch: u read once (8 B per node), the colour's b and 1/diagonal read
    and u written (24 B per updated node) = 20 B per node.  FP64 work per updated node: one
    multiply, five FMAs, a subtraction and the multiply by 1/diagonal = 13 FLOP in 8 FP64
    instructions; GB300's FP64 pipe (1.19 TFLOP/s of DFMA measured = 0.595 T instructions/s)
    therefore caps this sweep near 0.45 of the HBM copy peak in algorithmic bytes."""
    import torch
    n = cl.n
    u = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    b = torch.rand(n ** 3, dtype=torch.float64, device="cuda")
    timed_fn(u, b, 1, 0)
    t = (timed_fn(u, b, 3, 0) - timed_fn(u, b, 1, 0)) / 4 / 1e3
    upd = (n - 2) ** 3 / 2
    del u, b
    torch.cuda.empty_cache()
    bytes_per_launch = 20.0 * n ** 3
    return {"kernel": "k_rbgs_row<double> (FP64 red-black half sweep, 385^3 graded)", "us_per_launch": t * 1e6,
            "achieved_gbs": bytes_per_launch / t / 1e9, "hbm_frac": bytes_per_launch / t / 1e9 / peak,
            "fp64_tflops": 13 * upd / t / 1e12, "fp64_peak_tflops": FP64_TFLOPS,
            "fp64_issue_frac": 8 * upd / t / (FP64_TFLOPS / 2 * 1e12), "bytes_per_launch": bytes_per_launch,
            "traffic": DRAM_BYTES_257_F64 * (n / 257.0) ** 3}


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
