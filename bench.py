#!/usr/bin/env python3
"""Benchmark of the GB300 LASTO interstitial Poisson step.

Metric: converged Poisson solves per second (relative residual <= 1e-10).  One solve =
density, pseudo-density deposit, boundary multipoles, faces, iteration to 1e-10, sphere
projection (V_LM, Eq. 3.6).

`value` is the largest single-GPU workload: the Pd561 five-shell icosahedron on the graded
385^3 mesh (57 M nodes, 0.12 -> 0.6 bohr, 10 bohr vacuum) with 8 SCF-like densities (seeded
1 % perturbations of the Slater weights and nonspherical coefficients) solved back to back.
A step is the sequence of 8 solves, in the chosen form: FP64 defect correction around FP32
multigrid-preconditioned CG, FP32-pair density; the first density starts from the learned
guess (the U-Net inside the solve's graph), each later one from the previous density's
potential (an SCF loop has it).  The plain form (FP64 throughout, zero start) is timed beside
it, and so are the other starts (zero, learned guess for every density).  Every result
carries its error against the FP64 oracle: max |dV_LM| / max |V_LM| over the spheres, from
the oracle's answers stored by tests/golden/make_oracle_vlm.py (null when that file is
absent).  The working set (~6 GB) is far beyond L2; L2 is flushed anyway before each step.

Extra keys: the former headline (8 Pd55 clusters on graded 129^3 in one graph launch), the
uneven batch of 64 Pd13/Pd55/Pd147 clusters, the interstitial H and S contraction and the
other rows beyond the Poisson step, the roofline of the dominant kernel (the FP32 smoother
at 385^3), the arithmetic ceilings measured by the library's FMA probe, and the FP64 CPU
oracle timed on a bounded sample of the same workload.

`--impl reference` times the FP64 CPU oracle on the same workload and metric (the
reference arm; the paper publishes no implementation or timing), one bounded sample per
step: the deposit on 4 planes of the 385^3 grid and one and two stationary V(2,2) cycles on
the whole grid, extrapolated to a whole solve with the oracle's own cycle count to 1e-10.

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
sys.path.insert(0, os.path.join(ROOT, "tests"))

METRIC = "converged Poisson solves/sec (resid <=1e-10)"
UNIT = "solves/s"
SEQ = 8            # densities per step
WORKLOAD = ("Pd561 5-shell icosahedron, graded 385^3 (57 M nodes; 0.12->0.6 bohr, 10 bohr vacuum), synthetic Slater "
            "densities; 8 SCF-like densities (seed 4, 1% perturbations) solved back to back per step")
FORM = ("FP64 defect correction around FP32 multigrid-preconditioned CG + FP32-pair density; first density from the "
        "learned guess (U-Net in the graph), each later density warm-started from the previous potential")
PD55_WORKLOAD = ("Pd55 Mackay icosahedron, graded 129^3 (0.12->0.6 bohr, 10 bohr vacuum); 8 clusters (density seeds "
                 "1-8) per graph launch")
BATCH = 8


# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch at 257^3 (steady state: launches 5-8
# of a 4-sweep call, caches not flushed between launches), by launch shape: in-place half sweep
# with one block per row (0) or 128 / 256 threads per block; the FP32 wavefront sweep ("wave").
# Scaled to 385^3 by the node count (the traffic is proportional to the nodes beyond L2).
DRAM_BYTES_257 = {0: 197.9e6, 128: 195.6e6, 256: 195.8e6}
DRAM_BYTES_257_F64 = 537.7e6
# the half sweep over colour-split storage, one warp per row (k_rbgs_split_rows<6>), captured at
# 385^3 itself (third launch of `bench.py --profile smoother --n 385 --split --threads 0
# --sweeps 2`, ncu --set full: caches flushed before the launch): 230.9 MB read + 87.2 MB written
DRAM_BYTES_385_SPLIT_ROWS = 318.1e6
# the plane-staged half sweep over colour-split storage (k_rbgs_split_stage<6, 0>), captured the
# same way (`--threads 1`): 237.2 MB read + 76.6 MB written
DRAM_BYTES_385_SPLIT_STAGE = 313.8e6


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--quiet", action="store_true")
    p.add_argument("--no-batch64", action="store_true")
    p.add_argument("--no-pd561", action="store_true")
    p.add_argument("--no-hs", action="store_true")
    p.add_argument("--profile", choices=["smoother", "solve", "guess", "pd561", "pd561warm", "deposit", "hs", "batch",
                                          "train"],
                   default=None,
                   help="run one kernel family for a profiler and exit: 'smoother' = one FP32 red-black sweep "
                        "on an n^3 graded mesh, 'solve' = one mixed solve of the workload with direct launches, "
                        "'guess' = the same with the learned initial guess, 'pd561' = one chosen-form solve "
                        "of the Pd561 graded 385^3 workload with direct launches, 'pd561warm' = the second density "
                        "of that sequence warm-started from the first one's potential (the headline's steady "
                        "state), 'deposit' = two FP32-pair density deposits of the Pd561 graded 385^3 density, 'train' = one training step of the learned guess's U-Net on 8 grids of 33^3 (tcgen05 kernels; --wmma for the warp-level MMA ones), 'hs' = one interstitial H and S "
                        "call (tensor cores) for Pd55 on the graded 129^3 mesh, 'batch' = one graph launch of the "
                        "chosen form over the 8 Pd55 clusters of the workload (for ncu --graph-profiling graph)")
    p.add_argument("--n", type=int, default=257, help="grid size of --profile smoother")
    p.add_argument("--threads", type=int, default=256,
                   help="launch shape of --profile smoother: threads per block, 0 = one block per row")
    p.add_argument("--sweeps", type=int, default=1, help="red-black sweeps of --profile smoother")
    p.add_argument("--fp64", action="store_true", help="--profile smoother in FP64 (the plain form's smoother)")
    p.add_argument("--wmma", action="store_true", help="--profile train on the warp-level MMA kernels")
    p.add_argument("--split", action="store_true",
                   help="--profile smoother over colour-split storage (the finest FP32 level's layout)")
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


# ------------------------------------------------------------------ oracle: stored answers and CPU timing
def oracle_errors(group, clusters, vlm, first=0):
    """max |dV_LM| / max |V_LM| of each cluster of a concatenated GPU V_LM against the oracle's
    stored answer (clusters at positions first, first + 1, ... of the group); None when the
    stored answers are absent."""
    try:
        from golden.make_oracle_vlm import stored_vlm
    except ImportError:
        return None
    out, off = [], 0
    try:
        for q, cl in enumerate(clusters):
            ref = stored_vlm(group, cl, first + q)
            out.append(float(abs(vlm[off:off + cl.n_atoms] - ref).max() / abs(ref).max()))
            off += cl.n_atoms
    except (FileNotFoundError, IndexError, KeyError):
        return None
    return out


def oracle_cycles_to(tol, group="pd561", index=0, fallback=85):
    """Stationary V(2,2) cycles the oracle needs to reach `tol` on a stored cluster (its residual
    history), else `fallback`."""
    try:
        from golden.make_oracle_vlm import history
        h = history(group, index)
        return int(next(i for i, r in enumerate(h) if r <= tol)), "oracle residual history (stored)"
    except (ImportError, FileNotFoundError, KeyError, StopIteration):
        return fallback, "assumed"


def oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


class OracleSample:
    """A bounded sample of the oracle on the Pd561 workload: the deposit on `planes` planes at
    the middle of the 385^3 grid, and one and two stationary V(2,2) cycles on the whole grid.
    Extrapolated solve time = deposit per plane x 385 planes + cycles to 1e-10 x (t2 - t1) +
    (2 t1 - t2) (the cycle's fixed part: norms, hierarchy set-up)."""

    def __init__(self, planes=4):
        import numpy as np

        import oracle
        import synth
        oracle.build()
        self.oracle, self.planes = oracle, planes
        self.cl = synth.pd561_graded385(n_densities=1)[0]
        self.x, self.y, self.z = oracle.mesh(self.cl)
        n = self.cl.n
        self.b = np.random.default_rng(0).normal(size=(n, n, n))
        self.u = np.zeros((n, n, n))
        self.cycles, self.cycles_source = oracle_cycles_to(1e-10)

    def step(self):
        n, k0 = self.cl.n, self.cl.n // 2 - self.planes // 2
        t0 = time.perf_counter()
        self.oracle.deposit(self.cl, self.x, self.y, self.z[k0:k0 + self.planes])
        t1 = time.perf_counter()
        self.u[...] = 0.0
        self.oracle.mg_solve(self.x, self.y, self.z, self.b, self.u, max_cycles=1, tol=1e-30)
        t2 = time.perf_counter()
        self.u[...] = 0.0
        self.oracle.mg_solve(self.x, self.y, self.z, self.b, self.u, max_cycles=2, tol=1e-30)
        t3 = time.perf_counter()
        dep = (t1 - t0) / self.planes * n
        c1, c2 = t2 - t1, t3 - t2
        cyc = max(c2 - c1, 1e-9)
        solve = dep + self.cycles * cyc + max(2 * c1 - c2, 0.0)
        return {"sample_s": t3 - t0, "solve_s": solve, "deposit_s": dep, "cycle_s": cyc}

    def describe(self, steps):
        return (f"{steps} samples of the Pd561 385^3 workload: deposit on {self.planes} planes (x385/{self.planes}) and "
                f"1 and 2 stationary V(2,2) cycles on the whole grid; solve = deposit + {self.cycles} cycles to 1e-10 "
                f"({self.cycles_source}) + the cycle's fixed part")


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on the host cores, a bounded sample per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    smp = OracleSample()
    for _ in range(args.warmup):
        smp.step()
    res = [smp.step() for _ in range(args.steps)]
    solve_s = statistics.median(r["solve_s"] for r in res)
    value = 1.0 / solve_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * solve_s * SEQ,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "f64 (CPU oracle, stationary V(2,2) to 1e-10)",
                   "l2": "n/a (CPU)", "deposit_s": statistics.median(r["deposit_s"] for r in res),
                   "cycle_s": statistics.median(r["cycle_s"] for r in res), "cycles": smp.cycles,
                   "sample_s": statistics.median(r["sample_s"] for r in res)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                         "sample": smp.describe(args.steps)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def pd561_run(B, solvers, dcs, v, pot, start, stream, flush):
    """One pass over the density sequence.  start 'warm': the first density from the learned
    guess (solvers['learned']), each later one from the previous potential (solvers['warm']);
    'learned': every density from the learned guess; 'zero': every density from zero
    (solvers['zero']).  As in an SCF loop, each handle solves in one set of device arrays (its
    slot, solvers[name + '_slot']) into which the next density's Slater weights and
    nonspherical coefficients are copied on the device, so its captured graph is replayed.
    Returns (ms of the pass, stats per density, V_LM per density)."""
    import torch
    flush.fill_(1.0)
    e0, e1 = _events(torch, stream)
    e0.record(stream)
    stats, vl = [], []
    for s, dc in enumerate(dcs):
        name = "warm" if (start == "warm" and s > 0) else ("learned" if start in ("warm", "learned") else "zero")
        slot = solvers[name + "_slot"]
        slot.w.copy_(dc.w, non_blocking=True)
        slot.clm.copy_(dc.clm, non_blocking=True)
        if name == "warm":
            st = solvers[name].solve(slot, v, potential=pot, guess=pot)
        else:
            st = solvers[name].solve(slot, v, potential=pot)
        stats.append(st[0])
        vl.append(v.clone())
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), [(x.cycles, x.outer, x.rel_resid, x.status, x.guess) for x in stats], vl


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
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    launch = 1 if args.direct else 0

    # ---------------- the headline: Pd561 / graded 385^3, 8 SCF-like densities per step
    seq = synth.pd561_graded385()
    na, n = seq[0].n_atoms, seq[0].n
    dcs = [B.DeviceCluster(c) for c in seq]
    v = torch.empty((na, 25), dtype=torch.float64, device=dev)
    pot = torch.empty(n ** 3, dtype=torch.float64, device=dev)
    mk = lambda prec: B.Poisson(n_max=n, max_atoms=na, precision=prec, launch=launch)
    solvers = {"learned": mk(B.LASTO_PREC_MIXED), "warm": mk(B.LASTO_PREC_MIXED),
               "learned_slot": B.DeviceCluster(seq[0]), "warm_slot": B.DeviceCluster(seq[0])}
    solvers["learned"].set_guess()
    for _ in range(args.warmup):
        pd561_run(B, solvers, dcs, v, pot, "warm", stream, flush)
    torch.cuda.synchronize()
    counts = {k: (solvers[k].kernel_counts() if not args.direct else (0, 0, 0)) for k in ("learned", "warm")}
    barrier(ws)
    torch.cuda.synchronize()
    ms, launches, stats, vlms = [], 0, None, None
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            t, stats, vlms = pd561_run(B, solvers, dcs, v, pot, "warm", stream, flush)
            ms.append(t)
            for s, (c, o, _, _, _) in enumerate(stats):
                f_, i_, o_ = counts["warm" if s else "learned"]
                launches += f_ + c * i_ + o * o_
            assert all(st == 0 and r <= 1e-10 for _, _, r, st, _ in stats), stats
        torch.cuda.synchronize()
        barrier(ws)
    span_max = max_over_ranks(sum(ms), ws, dev)
    value = SEQ * args.steps * ws / (span_max / 1e3)
    err = oracle_errors("pd561", seq, torch.cat(vlms).cpu().numpy())
    tuned = solvers["warm"].tune_table().strip().splitlines()

    # ---------------- the other starts at 385^3 (one pass each) and the plain FP64 form
    starts = {"warm": {"ms_per_solve": sum(ms) / len(ms) / SEQ, "cycles": [c for c, *_ in stats],
                       "defect_correction_steps": [o for _, o, *_ in stats],
                       "oracle_error_max": max(err) if err else None}}
    solvers["zero"], solvers["zero_slot"] = mk(B.LASTO_PREC_MIXED), B.DeviceCluster(seq[0])
    for name in ("learned", "zero"):
        pd561_run(B, solvers, dcs[:1], v, pot, name, stream, flush)          # capture, tuning
        t, st_, vl = pd561_run(B, solvers, dcs, v, pot, name, stream, flush)
        e_ = oracle_errors("pd561", seq, torch.cat(vl).cpu().numpy())
        starts[name] = {"ms_per_solve": t / SEQ, "cycles": [c for c, *_ in st_],
                        "defect_correction_steps": [o for _, o, *_ in st_],
                        "oracle_error_max": max(e_) if e_ else None}
    solvers["zero"].close()
    plain = {"zero": mk(B.LASTO_PREC_FP64), "zero_slot": solvers["zero_slot"]}
    pd561_run(B, plain, dcs[:1], v, pot, "zero", stream, flush)
    pms, pst = [], None
    for _ in range(2):
        t, pst, pvl = pd561_run(B, plain, dcs[:1], v, pot, "zero", stream, flush)
        pms.append(t)
    plain_value = ws * len(pms) / (max_over_ranks(sum(pms), ws, dev) / 1e3)
    perr = oracle_errors("pd561", seq[:1], pvl[0].cpu().numpy())
    plain["zero"].close()

    # ---------------- end to end through the C ABI with host buffers (the chosen form)
    e2e = None
    if not args.no_e2e:
        fields = ("pos", "Z", "R", "slater_w", "slater_zeta", "c_lm")
        host = [{k: torch.as_tensor(np.ascontiguousarray(getattr(c, k), dtype=np.float64)).pin_memory()
                 for k in fields} for c in seq]
        # one set of device arrays per handle (as an SCF code keeps), filled from the host each solve
        slots = {}
        for name in ("learned", "warm"):
            d = B.DeviceCluster(seq[0])
            d.x, d.y, d.z = (torch.empty(n, dtype=torch.float64, device=dev) for _ in range(3))
            slots[name] = (d, {"pos": d.pos, "Z": d.Z, "R": d.R, "slater_w": d.w, "slater_zeta": d.zeta,
                               "c_lm": d.clm})
        vlm_host = torch.empty((SEQ, na, 25), dtype=torch.float64).pin_memory()
        h2d = sum(t_.numel() * t_.element_size() for hb in host for t_ in hb.values())
        d2h = vlm_host.numel() * vlm_host.element_size()
        lib = B.load()

        def e2e_step():
            sts = []
            for s, (c, hb) in enumerate(zip(seq, host)):
                name = "warm" if s else "learned"
                d, dbuf = slots[name]
                for k in fields:
                    dbuf[k].copy_(hb[k], non_blocking=True)
                for a, ax in enumerate((d.x, d.y, d.z)):
                    lib.lasto_mesh_axis(c.n, float(c.centre[a]), c.half_width, c.h_min, c.h_max, c.p_max,
                                        B._ptr(ax), None, B._stream(None))
                sv = solvers[name]
                sts.append((sv.solve(d, v, potential=pot, guess=pot) if s else sv.solve(d, v, potential=pot))[0])
                vlm_host[s].copy_(v, non_blocking=True)
            return sts

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        ms_e2e = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            sts = e2e_step()
            e1.record(stream)
            e1.synchronize()
            ms_e2e.append(e0.elapsed_time(e1))
            assert all(x.status == 0 and x.rel_resid <= 1e-10 for x in sts)
        e2e_err = oracle_errors("pd561", seq, vlm_host.reshape(SEQ * na, 25).numpy())
        e2e_val = SEQ * args.steps * ws / (max_over_ranks(sum(ms_e2e), ws, dev) / 1e3)
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "oracle_error_max": max(e2e_err) if e2e_err else None}
        del slots
    for k in ("learned", "warm"):
        solvers[k].close()
    del dcs, v, pot, solvers
    torch.cuda.empty_cache()

    # ---------------- the former headline: 8 Pd55 clusters per graph launch, and its forms
    pd55 = pd55_forms(B, synth, flush, stream, dev, args, launch)

    # ---------------- the uneven batch of 64 (Pd13/55/147 on 65^3 .. 193^3), chosen form
    b64 = None
    if not args.no_batch64:
        b64 = batch_throughput(B, synth.batch64(), B.LASTO_PREC_MIXED, 2, flush, stream, dev, warmup=1, guess=True,
                               group="batch64")

    # ---------------- the interstitial H and S contraction (Eq. 3.11-3.14) and the other rows
    hs = rows = None
    if not args.no_hs:
        hs = interstitial_hs(B, synth, flush, stream, dev)
        rows = next_rows(B, synth, flush, stream, dev)

    # ---------------- arithmetic ceilings (the library's FMA probe) and the roofline
    probes = fma_ceilings(B, stream, dev)
    training = training_rate(B, stream, dev)
    roof = smoother_roofline(B, stream, flush, dev, tuned, probes)
    dep = deposit_rate(B, synth, stream, flush, dev, probes)

    # ---------------- CPU baseline: the oracle as it stands, a bounded sample of the workload
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        smp = OracleSample()
        r = smp.step()
        cpu = {"value": 1.0 / r["solve_s"], "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
               "sample": smp.describe(1) + f"; {r['sample_s']:.1f} s of CPU work"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": span_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32+bf16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": FORM, "solves_per_step": SEQ,
                       "l2": "inputs far larger than L2 (~6 GB working set); flushed before every step anyway",
                       "cycles": [c for c, *_ in stats], "defect_correction_steps": [o for _, o, *_ in stats],
                       "learned_guess": [g for *_, g in stats],
                       "max_rel_resid": max(r for _, _, r, _, _ in stats), "parallelism": f"replicas x{ws}",
                       "oracle_error": {"max": max(err) if err else None, "per_density": err,
                                        "definition": "max|dV_LM|/max|V_LM| against the FP64 oracle solved to 1e-13"},
                       "smoother_tuned": tuned},
            "plain_fp64": {"value": plain_value, "unit": UNIT, "ms_per_solve": sum(pms) / len(pms),
                           "cycles": pst[0][0], "rel_resid": pst[0][2], "oracle_error": perr[0] if perr else None,
                           "form": "FP64 deposit and FP64 multigrid-preconditioned CG, zero start, first density"},
            "chosen_over_plain": value / plain_value,
            "starts_385": starts,
            "pd55_batch8": pd55,
            "batch64_uneven": b64,
            "interstitial_hs": hs,
            "inner_faces_raw": rows,
            "probes": probes,
            "guess_training": training,
            "deposit": dep,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": launches,
            # the dominant kernel of the Pd561 solve is the deposit (about 39 % of a warm solve,
            # ahead of the finest level's smoother at about 20 %): instruction-issue bound
            "roofline": {"kernel": dep["kernel"], "bound": "alu", "achieved": dep.get("issue_ginst_s"),
                         "peak": dep.get("issue_peak_ginst_s"), "unit": "Ginst/s", "frac": dep.get("frac"),
                         "traffic": DEPOSIT_DRAM_BYTES, "ms_per_launch": dep["ms"],
                         "achieved_rule": "warp instructions issued per launch (ncu smsp__inst_executed.sum) / "
                                          "CUDA-event launch time",
                         "peak_rule": "4 schedulers x 152 SMs x 1 warp instruction per cycle x 2070 MHz",
                         "fp32_tflops": dep.get("fp32_tflops"), "fp32_frac_of_measured_fma": dep.get("fp32_frac")},
            "roofline_smoother": roof,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def pd55_forms(B, synth, flush, stream, dev, args, launch):
    """The 8-cluster Pd55 / graded 129^3 batch (one graph launch, learned guess, mixed), the
    plain FP64 form (one cluster per call) and the forms between, each with its oracle error."""
    import torch
    cls8 = [synth.pd55_graded129(seed=1 + k) for k in range(BATCH)]
    cl = cls8[0]
    dcs8 = [B.DeviceCluster(c) for c in cls8]
    vlm8 = torch.empty((BATCH * cl.n_atoms, 25), dtype=torch.float64, device=dev)
    dc, vlm = dcs8[0], vlm8[:cl.n_atoms]

    def make(precision, batch=1, guess=False):
        s_ = B.Poisson(n_max=cl.n, max_atoms=cl.n_atoms, max_batch=batch, precision=precision, launch=launch)
        if guess:
            s_.set_guess()
        return s_

    def timed(solver, dcs, out, clusters, steps, warmup):
        st = None
        for _ in range(warmup):
            st = solver.solve(dcs, out)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            st = solver.solve(dcs, out)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            assert all(x.status == 0 and x.rel_resid <= 1e-10 for x in st)
        err = oracle_errors("pd55x8", clusters, out.cpu().numpy())
        nc = len(clusters)
        return {"value": nc * len(ms) / (sum(ms) / 1e3), "unit": UNIT, "ms_per_call": sum(ms) / len(ms),
                "clusters_per_call": nc, "cycles": [x.cycles for x in st], "outer": [x.outer for x in st],
                "max_rel_resid": max(x.rel_resid for x in st), "learned_guess": [x.guess for x in st],
                "oracle_error_max": max(err) if err else None}

    steps = max(3, args.steps)
    out = {"workload": PD55_WORKLOAD}
    s_ = make(B.LASTO_PREC_MIXED, BATCH, guess=True)
    out["chosen"] = timed(s_, dcs8, vlm8, cls8, steps, 2)
    s_.close()
    s_ = make(B.LASTO_PREC_FP64)
    out["plain_fp64"] = timed(s_, dc, vlm, cls8[:1], steps, 2)
    s_.close()
    s_ = make(B.LASTO_PREC_MIXED)
    out["mixed_single"] = timed(s_, dc, vlm, cls8[:1], steps, 2)
    s_.set_guess()
    out["mixed_learned_single"] = timed(s_, dc, vlm, cls8[:1], steps, 2)
    s_.close()
    s_ = make(B.LASTO_PREC_MIXED, BATCH)
    out["mixed_batched"] = timed(s_, dcs8, vlm8, cls8, steps, 2)
    s_.close()
    out["chosen_over_plain"] = out["chosen"]["value"] / out["plain_fp64"]["value"]
    del dcs8, vlm8
    torch.cuda.empty_cache()
    return out


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
        if args.split and not args.fp64:
            B.lasto_op_smooth_split(*axes, u, b, sweeps=args.sweeps, threads=args.threads)
        else:
            B.lasto_op_smooth(*axes, u, b, sweeps=args.sweeps, threads=args.threads)
    elif args.profile == "train":
        from paper_0806_1723_gb300 import unet
        net = unet.UNet(n=33, nb=8, seed=1, tc=not args.wmma)
        N = 8 * 33 ** 3
        g = torch.Generator(device="cuda").manual_seed(2)
        x = torch.randn(N, 16, generator=g, device="cuda") * 0.5
        x[:, 3:] = 0
        tgt = torch.randn(N, generator=g, device="cuda")
        mask = torch.ones(N, device="cuda")
        net._mask_count = float(N)

        def step():
            net.forward(x)
            net.loss_and_grad(tgt, mask)
            net.backward(net.dpred)
            net.adam(1e-4)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()   # ncu --profile-from-start off captures this step only
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif args.profile == "deposit":
        dc = B.DeviceCluster(synth.pd561_graded385(n_densities=1)[0])
        for _ in range(2):
            B.lasto_op_deposit(dc, precision=B.LASTO_PREC_MIXED)
    elif args.profile == "pd561warm":
        seq = synth.pd561_graded385(n_densities=2)
        solver = B.Poisson(n_max=385, max_atoms=561, precision=B.LASTO_PREC_MIXED, launch=1)
        # under a profiler the tuner's timings mean nothing; take the choices it makes without one
        # (the finest level in colour-split storage, plane-staged; in-place half sweeps below)
        solver.set_tune_table("385 385 385 4 3 1 0 0 0 0 0\n" +
                              "".join(f"{m} {m} {m} 4 0 128 0 0 0 0 0\n" for m in (193, 97, 49, 25)))
        v = torch.empty((561, 25), dtype=torch.float64, device="cuda")
        pot = torch.empty(385 ** 3, dtype=torch.float64, device="cuda")
        st = solver.solve(B.DeviceCluster(seq[0]), v, potential=pot)   # the previous density
        dc = B.DeviceCluster(seq[1])
        st = solver.solve(dc, v, potential=pot, guess=pot)              # tables, first launch of each kernel
        torch.cuda.synchronize()
        st = solver.solve(B.DeviceCluster(seq[0]), v, potential=pot)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()   # ncu --profile-from-start off captures this solve only
        st = solver.solve(dc, v, potential=pot, guess=pot)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        assert st[0].status == 0
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


def batch_throughput(B, clusters, precision, steps, flush, stream, dev, warmup=2, guess=False, group=None):
    """Solves/s of a batch of clusters solved in one call (one graph launch), with the oracle
    error of every cluster (max over the batch)."""
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
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        st = solver.solve(dcs, vlm)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ok = all(s.status == 0 and s.rel_resid <= 1e-10 for s in st)
    err = oracle_errors(group, clusters, vlm.cpu().numpy()) if group else None
    solver.close()
    del dcs, vlm
    torch.cuda.empty_cache()
    return {"value": len(clusters) * steps / (sum(ms) / 1e3), "unit": UNIT, "clusters": len(clusters),
            "ms_per_batch": sum(ms) / steps, "all_converged": ok, "mean_cycles": sum(s.cycles for s in st) / len(st),
            "max_cycles": max(s.cycles for s in st), "learned_guess": sum(s.guess for s in st),
            "nodes": sum(c.n ** 3 for c in clusters), "oracle_error_max": max(err) if err else None}


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
    # the fraction counts the method's own products (S_ab and 2H_ab over a <= b), not the three
    # hi/lo MMAs per product nor the padding of the 128 x 128 tiles
    out["roofline"] = {"kernel": "k_hs_gemm_tc", "bound": "tensor", "achieved": alg_flops / t / 1e12,
                       "peak": f16_peak, "unit": "TFLOP/s", "frac": alg_flops / t / 1e12 / f16_peak,
                       "traffic": None, "flops": "algorithmic: 6 per interstitial node per (a <= b) entry",
                       "peak_source": ("measured bf16 burst (FP16 dense rate = BF16)" if "bf16_tflops" in peaks
                                       else "fallback bf16 burst")}
    out["tensor_pipe_tflops"] = tensor_flops / t / 1e12   # all issued MMAs (3 per product, padded tiles)
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


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def training_rate(B, stream, dev, steps=10, warmup=3):
    """Training throughput of the learned guess's U-Net (batches of 8 grids of 33^3, one step =
    forward, masked MSE, backward, Adam), on the tcgen05 kernels and on the warp-level MMA
    kernels, with random inputs and targets (the rate does not depend on the values)."""
    import torch

    from paper_0806_1723_gb300 import unet
    out = {"batch": 8, "grid": "33^3", "steps": steps}
    for name, tc in (("tcgen05", True), ("wmma", False)):
        net = unet.UNet(n=33, nb=8, seed=1, tc=tc)
        g = torch.Generator(device=dev).manual_seed(2)
        N = 8 * 33 ** 3
        x = torch.randn(N, 16, generator=g, device=dev) * 0.5
        x[:, 3:] = 0
        tgt = torch.randn(N, generator=g, device=dev)
        mask = torch.ones(N, device=dev)
        net._mask_count = float(N)

        def step():
            net.forward(x)
            net.loss_and_grad(tgt, mask)
            net.backward(net.dpred)
            net.adam(1e-4)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "samples_per_s": 8 / (ms / 1e3)}
        if tc:
            out[name]["timeouts"] = int(net.tc_err.item())
        del net
        torch.cuda.empty_cache()
    return out


def fma_ceilings(B, stream, dev):
    """FP64 and FP32 fused multiply-add throughput of this GPU (the library's FMA-chain probe on
    every SM, CUDA events, best of 3): the ceilings of the ALU-bound kernels."""
    import torch
    out = {}
    for name, prec, dt, iters in (("fp64", 0, torch.float64, 200), ("fp32", 1, torch.float32, 4000)):
        blocks = 152 * 16
        buf = torch.empty(blocks * 256, dtype=dt, device=dev)
        B.lasto_probe_fma(prec, blocks, iters, buf)
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(3):
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            B.lasto_probe_fma(prec, blocks, iters, buf)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        flops = B.PROBE_FLOP_PER_THREAD_ITER * iters * blocks * 256
        out[f"{name}_tflops"] = flops / best / 1e12
        out[f"{name}_ms"] = best * 1e3
    out["how"] = "lasto_probe_fma: 8 independent FMA chains per thread, 2432 blocks x 256 threads, best of 3"
    return out


def smoother_roofline(B, stream, flush, dev, tuned, probes):
    """The second kernel of the headline: the FP32 smoother at 385^3, in the launch shape the
    tuner chose for that level.  Algorithmic bytes (the smoother's compulsory traffic, 12 B per
    node per FP32 sweep: u read, b read, u written): 6 B per node for one half-sweep launch (one
    colour; natural or colour-split storage), 12 B per node for one fused wavefront sweep.  Each
    shape is timed alone with CUDA events (L2 flushed before each call; the difference of a 9-
    and a 1-sweep call for the half sweeps, 16 launches back to back as in a cycle's smoothing,
    so table set-up and the first, cold launch cancel), and the line reports the tuner's choice; `traffic` is ncu's DRAM bytes per launch
    (dram__bytes_read.sum + dram__bytes_write.sum at 257^3 in steady state, scaled by nodes)."""
    import torch

    import synth
    cl = synth.pd561_graded385(n_densities=1)[0]
    n = cl.n
    axes = [B.lasto_mesh_axis(n, 0.0, cl.half_width, cl.h_min, cl.h_max, cl.p_max) for _ in range(3)]
    u = torch.zeros(n ** 3, dtype=torch.float32, device=dev)
    b = torch.rand(n ** 3, dtype=torch.float32, device=dev)
    o = torch.empty_like(u)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts) / 1e3

    shapes = {}
    names = {0: "rows", B.SPLIT_STAGED: "staged"}
    for th in (B.SPLIT_STAGED, 0, 128):   # half sweeps over colour-split storage (its data is irrelevant here)
        t = (timed(lambda: B.lasto_op_smooth_split(*axes, u, b, sweeps=9, threads=th)) -
             timed(lambda: B.lasto_op_smooth_split(*axes, u, b, sweeps=1, threads=th))) / 16
        shapes[f"split_{names.get(th, th)}"] = {"us_per_launch": t * 1e6, "bytes_per_launch": 6.0 * n ** 3,
                                                "launches_per_sweep": 2, "nt": th}
    for th in (0, 128, 256):   # in-place half sweeps: per launch (2 launches per sweep)
        t = (timed(lambda: B.lasto_op_smooth(*axes, u, b, sweeps=9, threads=th)) -
             timed(lambda: B.lasto_op_smooth(*axes, u, b, sweeps=1, threads=th))) / 16
        shapes[f"inplace_{th if th else 'rows'}"] = {"us_per_launch": t * 1e6, "bytes_per_launch": 6.0 * n ** 3,
                                                     "launches_per_sweep": 2, "nt": th}
    for tile in ((60, 16), (60, 12), (60, 8)):   # wavefront sweeps: per launch (1 per sweep)
        t = (timed(lambda: B.lasto_op_smooth_wave(*axes, u, o, b, sweeps=4, tile=tile)) -
             timed(lambda: B.lasto_op_smooth_wave(*axes, u, o, b, sweeps=2, tile=tile))) / 2
        shapes[f"wave_{tile[0]}x{tile[1]}"] = {"us_per_launch": t * 1e6, "bytes_per_launch": 12.0 * n ** 3,
                                               "launches_per_sweep": 1, "tile": list(tile)}
    del u, b, o
    torch.cuda.empty_cache()
    peaks = _peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    for v_ in shapes.values():
        v_["achieved_gbs"] = v_["bytes_per_launch"] / (v_["us_per_launch"] / 1e6) / 1e9
        v_["frac"] = v_["achieved_gbs"] / peak
        v_["us_per_sweep"] = v_["us_per_launch"] * v_["launches_per_sweep"]
    # the tuner's choice for the 385^3 FP32 level (table line: nx ny nz elem fused nt tx ty kz ns us)
    pick = None
    for line in tuned:
        f = line.split()
        if f[:4] == [str(n), str(n), str(n), "4"]:
            fused, nt, tx, ty = int(f[4]), int(f[5]), int(f[6]), int(f[7])
            pick = (f"wave_{tx}x{ty}" if fused == 2 else f"inplace_{nt if nt else 'rows'}" if fused == 0
                    else f"split_{names.get(nt, nt)}" if fused == 3 else None)
    if pick not in shapes:
        pick = min(shapes, key=lambda k: shapes[k]["us_per_sweep"])
    c = shapes[pick]
    traffic = None
    if pick.startswith("split"):
        traffic = (DRAM_BYTES_385_SPLIT_ROWS if c["nt"] == 0 else
                   DRAM_BYTES_385_SPLIT_STAGE if c["nt"] == B.SPLIT_STAGED else None) if n == 385 else None
        kernel = ("k_rbgs_split_rows<6> (red-black half sweep over colour-split storage, one warp per row, "
                  "385^3 graded)" if c["nt"] == 0 else
                  "k_rbgs_split_stage<6> (red-black half sweep over colour-split storage, tiles of 8 rows marching "
                  "through plane chunks, the other colour's planes bulk-copied into shared memory one plane ahead, "
                  "385^3 graded)" if c["nt"] == B.SPLIT_STAGED else
                  f"k_rbgs<float,split> (red-black half sweep over colour-split storage, {c['nt']} threads per "
                  "block, 385^3 graded)")
    elif pick.startswith("inplace"):
        t257 = DRAM_BYTES_257.get(c["nt"])
        kernel = ("k_rbgs_row<float> (in-place red-black half sweep, one block per row, 385^3 graded)" if c["nt"] == 0
                  else f"k_rbgs<float> (in-place red-black half sweep, {c['nt']} threads per block, 385^3 graded)")
    else:
        t257 = DRAM_BYTES_257.get("wave")
        kernel = f"k_rb_wave<float> (fused red-black wavefront sweep, tile {c['tile']}, 385^3 graded)"
    if not pick.startswith("split"):
        traffic = t257 * (n / 257.0) ** 3 if t257 else None
    return {"kernel": kernel, "bound": "hbm", "achieved": c["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": c["frac"], "traffic": traffic,
            "traffic_over_algorithmic": traffic / c["bytes_per_launch"] if traffic else None,
            "bytes_per_launch": c["bytes_per_launch"], "us_per_launch": c["us_per_launch"],
            "bytes_rule": "12 B per node per FP32 sweep (u read, b read, u written): 6 per half-sweep launch",
            "peak_source": "measured (hbm_gbs)" if "hbm_gbs" in peaks else "fallback",
            "shapes": shapes, "tuner_choice": pick,
            "plain_fp64": fp64_half_sweep(B, cl, axes, flush, stream, dev, peak, probes)}


def fp64_half_sweep(B, cl, axes, flush, stream, dev, peak, probes):
    """The plain form's FP64 red-black half sweep at 385^3, one block per row.  Algorithmic bytes
    per launch: 12 B per node (u read, the colour's b read and u written: 24 B per node per FP64
    sweep).  FP64 work per updated node: one multiply, five FMAs, a subtraction and the multiply by
    the stored 1/diagonal = 8 FP64 instructions (13 FLOP), against the FP64 FMA rate the probe
    measured (2 FLOP per FMA instruction)."""
    import torch
    n = cl.n
    u = torch.zeros(n ** 3, dtype=torch.float64, device=dev)
    b = torch.rand(n ** 3, dtype=torch.float64, device=dev)

    def timed(sweeps):
        B.lasto_op_smooth(*axes, u, b, sweeps=sweeps, threads=0)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            B.lasto_op_smooth(*axes, u, b, sweeps=sweeps, threads=0)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts) / 1e3

    t = (timed(3) - timed(1)) / 4
    upd = (n - 2) ** 3 / 2
    del u, b
    torch.cuda.empty_cache()
    bytes_per_launch = 12.0 * n ** 3
    fp64_peak = probes["fp64_tflops"]
    return {"kernel": "k_rbgs_row<double> (FP64 red-black half sweep, 385^3 graded)", "us_per_launch": t * 1e6,
            "achieved_gbs": bytes_per_launch / t / 1e9, "hbm_frac": bytes_per_launch / t / 1e9 / peak,
            "fp64_tflops": 13 * upd / t / 1e12, "fp64_fma_tflops_measured": fp64_peak,
            "fp64_issue_frac": 8 * upd / t / (fp64_peak / 2 * 1e12), "bytes_per_launch": bytes_per_launch,
            "traffic": DRAM_BYTES_257_F64 * (n / 257.0) ** 3}


def deposit_rate(B, synth, stream, flush, dev, probes):
    """The FP32-pair density deposit (the second kernel of the Pd561 solve) timed alone: (node,
    atom) pairs per second, and FP32 work per second against the FP32 FMA rate the probe
    measured, with the FP32 work per launch from ncu (DEPOSIT_FP32_FLOP)."""
    import torch
    cl = synth.pd561_graded385(n_densities=1)[0]
    dc = B.DeviceCluster(cl)
    B.lasto_op_deposit(dc, precision=B.LASTO_PREC_MIXED)
    torch.cuda.synchronize()
    ms = []
    for _ in range(3):
        flush.fill_(1.0)
        e0, e1 = _events(torch, stream)
        e0.record(stream)
        B.lasto_op_deposit(dc, precision=B.LASTO_PREC_MIXED)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) / 1e3
    pairs = cl.n ** 3 * cl.n_atoms
    out = {"kernel": "k_deposit_df (FP32-pair Slater sums, Pd561 graded 385^3)", "ms": t * 1e3,
           "gpair_s": pairs / t / 1e9, "pairs": pairs, "bound": "alu",
           "fp32_fma_tflops_measured": probes["fp32_tflops"]}
    if DEPOSIT_FP32_FLOP is not None:
        out["fp32_tflops"] = DEPOSIT_FP32_FLOP / t / 1e12
        out["fp32_frac"] = out["fp32_tflops"] / probes["fp32_tflops"]
    # the bound it meets: instruction issue (one warp instruction per cycle per scheduler, four
    # schedulers per SM, 152 SMs, at the sampled SM clock)
    if DEPOSIT_WARP_INST is not None:
        peak = 4 * 152 * MAX_SM_MHZ * 1e6 / 1e9
        out["issue_ginst_s"] = DEPOSIT_WARP_INST / t / 1e9
        out["issue_peak_ginst_s"] = peak
        out["frac"] = out["issue_ginst_s"] / peak
    del dc
    torch.cuda.empty_cache()
    return out


# One Pd561 385^3 deposit launch (k_deposit_df) under ncu (`bench.py --profile deposit`, second
# launch): FP32 FLOP from the sass thread-instruction counts (2 per FFMA: 132.4 G, 1 per FADD:
# 329.4 G and per FMUL: 89.9 G), the warp instructions issued (smsp__inst_executed.sum) and the
# DRAM bytes (read 14.6 MB + written 850.7 MB); the launch issued 0.87 instructions per cycle per
# scheduler.
DEPOSIT_FP32_FLOP = 684.0e9
DEPOSIT_WARP_INST = 32.623e9
DEPOSIT_DRAM_BYTES = 865.3e6
MAX_SM_MHZ = 2070.0   # the GB300's maximum SM clock (the clock the timed runs hold)


if __name__ == "__main__":
    sys.exit(main())
