#!/usr/bin/env python
"""Benchmark of the GB300 ORAS-GMRES closest point method solver.

One step = the whole hot path on one synthetic problem, the shifted surface
Poisson problem (c - Delta_S) u = f (arXiv 2110.06322, eq. shiftPoisson) on a
torus R = 1, r = 0.4 at h = 0.004 (about 5.7M band points, tricubic
interpolation), c = 10, f = 20 random Fourier modes in the torus angles:

  band build (Sigma_A, Sigma_G, E rows)  ->  Schwarz set-up (512 parts,
  overlap 2, ILU(0))  ->  mixed-precision solve M u = f  ->  mixed-precision
  adjoint solve M^T lambda = g, both to relative residual 1e-8.

Reported value: band-point iterations per second of the whole step, N_A times
the GMRES iterations of both solves (inner iterations of the refinement
included) divided by the step time.  Also reported: solves/s, and one plain
FP64 solve of the same system for comparison.

--impl reference times the FP64 CPU oracle (oracle/) on the host cores, each
step a bounded sample of the same workload (the same torus at h = 0.025 with
16 parts, so that each subdomain has about as many rows as in the GPU
workload), in the same unit.

Multi-GPU: the problems are independent, so N ranks run N replicas with no
collective on the data path ("scaling": "weak"); value = all ranks' band-point
iterations / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_06322_gb300 import inputs  # noqa: E402

WORKLOAD = "torus_h0.004"
SAMPLE = dict(h=0.025, nparts=16)  # oracle sample: same torus, same subdomain size
# DRAM bytes per stored factor entry of one FP32 Schwarz apply (dram__bytes_read.sum + dram__bytes_write.sum
# of one ncu capture on the torus h = 0.0125 / 64-part case, 564.35 MB over 88,019,898 entries; summary in
# profiles/k_schwarz_pk_fp32_torus_h0.0125.md).  Traffic grows with the stored entries, so a full launch moves
# this times Sigma nnz(A_j).  Re-measure when k_schwarz_pk changes.
SCHWARZ_TRAFFIC_PER_ENTRY = 564.354048e6 / 88019898
METRIC = "ORAS-GMRES band-pt*iters/s (full pipeline: band, set-up, mixed forward + adjoint solve at 1e-8)"
UNIT = "band-pt*iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(name):
    w = dict(inputs.WORKLOADS[name])
    return w


def rhs_pair(cp, w):
    f = inputs.torus_rhs(cp, inputs.torus_modes(w["seed"]))
    g = inputs.torus_rhs(cp, inputs.torus_modes(w["seed"] + 100))
    return f, g


# ---------------------------------------------------------------- clocks
class Clocks:
    """Samples nvidia-smi during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = sorted(float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------- ranks
def reduce_over_ranks(ms, iters, device="cpu"):
    """Whole-job numbers of a replicated run: the slowest rank's time and the
    band-point iterations summed over all ranks (no data-path collective:
    this is the only exchange)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(iters)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(it)
    return t.item(), it.item()


# ---------------------------------------------------------------- oracle sample (CPU)
def oracle_step(w, h, nparts):
    """One full pipeline of the FP64 oracle on the sample; returns (seconds,
    band-point iterations, solves)."""
    import oracle
    t0 = time.perf_counter()
    B = oracle.Band(w["kind"], w["params"], h, w["p"])
    M = B.M(w["c"])
    cp = B.export()[3][: B.n_active]
    f, g = rhs_pair(cp, w)
    P = oracle.ORAS(B, M, nparts, w["overlap"], robin=w["robin"], alpha=w.get("alpha", 4.0),
                    alpha_cross=w.get("alpha_cross", 20.0))
    u, i1 = oracle.gmres(M, f, P, restart=w["restart"], rtol=w["rtol"], maxit=20000)
    lam, i2 = oracle.gmres(M.transpose(), g, P, transpose=True, restart=w["restart"], rtol=w["rtol"], maxit=20000)
    dt = time.perf_counter() - t0
    return dt, B.n_active * (i1["iters"] + i2["iters"]), 2, B.n_active


def cpu_baseline(w):
    dt, bpi, solves, n = oracle_step(w, SAMPLE["h"], SAMPLE["nparts"])
    return {"value": bpi / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle (FP64, single thread) full pipeline on the same torus at h={SAMPLE['h']} "
                      f"({n} band points, {SAMPLE['nparts']} parts, overlap {w['overlap']}): band, M, "
                      f"ILU(0) set-up, forward + adjoint GMRES to {w['rtol']:g}; {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload)
    for _ in range(args.warmup):
        oracle_step(w, SAMPLE["h"], SAMPLE["nparts"])
    tot_t, tot_bpi, tot_solves = 0.0, 0, 0
    for _ in range(args.steps):
        dt, bpi, solves, n = oracle_step(w, SAMPLE["h"], SAMPLE["nparts"])
        tot_t += dt
        tot_bpi += bpi
        tot_solves += solves
    value = tot_bpi / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} (oracle sample h={SAMPLE['h']}, {SAMPLE['nparts']} parts)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: oracle full pipeline on the torus at h={SAMPLE['h']} "
                                       f"({n} band points)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2110_06322_gb300 import cpm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.workload)
    kind, prm, h, c = w["kind"], w["params"], w["h"], w["c"]
    robin = w["robin"]
    alpha, alpha_x = w.get("alpha", 4.0), w.get("alpha_cross", 20.0)
    stream = torch.cuda.current_stream()

    # inputs: the right-hand sides at the closest points (host, once), resident in HBM
    B0 = cpm.Band(kind, prm, h, w["p"])
    n = B0.n_active
    cp = B0.export()[3][:n].cpu().numpy()
    f_h, g_h = rhs_pair(cp, w)
    del B0
    f = torch.from_numpy(f_h).cuda()
    g = torch.from_numpy(g_h).cuda()
    fh_pin = torch.from_numpy(f_h).pin_memory()
    gh_pin = torch.from_numpy(g_h).pin_memory()
    uh_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    lh_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    kw = dict(restart=w["restart"], rtol=w["rtol"], maxit=50000, mixed=True, inner_rtol=1e-4, reorth=0)

    def step(fd, gd, timing=False):
        B = cpm.Band(kind, prm, h, w["p"])
        P = cpm.Schwarz(B, c, w["nparts"], w["overlap"], robin=robin, alpha=alpha, alpha_cross=alpha_x,
                        store=cpm.CPM_F32)
        u, i1 = cpm.solve(B, fd, P, timing=timing, **kw)
        lam, i2 = cpm.solve(B, gd, P, adjoint=True, timing=timing, **kw)
        if i1["status"] != 0 or i2["status"] != 0:
            raise RuntimeError(f"solve did not converge: {i1} {i2}")
        info = (i1, i2, P.total_nnz, P.total_rows)
        del P, B
        return u, lam, info

    for _ in range(args.warmup):
        step(f, g)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM
    L0 = cpm.cpm_kernel_launches()
    iters = 0
    prec_ms, prec_n, nnz, nloc = 0.0, 0, 0, 0
    with Clocks(local) as clk:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            u, lam, (i1, i2, nnz, nloc) = step(f, g, timing=True)
            iters += i1["iters"] + i2["iters"]
            prec_ms += i1["ms_precond"]  # forward solve: FP32 Schwarz applies
            prec_n += i1["n_precond"]
        e1.record(stream)
        barrier()
    launches = cpm.cpm_kernel_launches() - L0
    ms, all_iters = reduce_over_ranks(e0.elapsed_time(e1), iters, device="cuda")
    value = n * all_iters / (ms / 1000.0)
    solves_per_s = 2 * args.steps * world / (ms / 1000.0)

    # ---- end to end: host buffers in, host buffers out, copies timed
    barrier()
    t0 = time.perf_counter()
    e_iters = 0
    for _ in range(args.steps):
        fd = fh_pin.to("cuda", non_blocking=True)
        gd = gh_pin.to("cuda", non_blocking=True)
        u, lam, (i1, i2, _, _) = step(fd, gd)
        uh_pin.copy_(u, non_blocking=True)
        lh_pin.copy_(lam, non_blocking=True)
        e_iters += i1["iters"] + i2["iters"]
    torch.cuda.synchronize()
    e2e_s, e_all = reduce_over_ranks(time.perf_counter() - t0, e_iters, device="cuda")
    e2e_value = n * e_all / e2e_s

    # ---- plain FP64 solve of the same system (context: mixed vs FP64)
    B = cpm.Band(kind, prm, h, w["p"])
    P = cpm.Schwarz(B, c, w["nparts"], w["overlap"], robin=robin, alpha=alpha, alpha_cross=alpha_x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u64, i64 = cpm.solve(B, f, P, restart=w["restart"], rtol=w["rtol"], maxit=50000, mixed=False, reorth=0)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    u32, i32 = cpm.solve(B, f, P, **kw)
    torch.cuda.synchronize()
    mixed_s = time.perf_counter() - t0
    diff = ((u32 - u64).norm() / u64.norm()).item()
    del P, B

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    import json as _j
    peaks = {}
    try:
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    alg_bytes = 8.0 * nnz + 4.0 * nloc + 4.0 * n  # FP32 value + int32 column per entry; gather; scatter
    avg_ms = prec_ms / max(prec_n, 1)
    achieved = alg_bytes / (avg_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: torus R=1 r=0.4 h={h} p=3 c={c}, {n} band points, "
                               f"{w['nparts']} parts overlap {w['overlap']} "
                               f"{'P-ORAS' if robin else 'RAS'} ILU(0), GMRES({w['restart']}) rtol {w['rtol']:g}, "
                               "classical Gram-Schmidt (one pass), mixed FP32/FP64",
                   "parallelism": f"replicas x{world}", "l2": "working set (ORAS factors) far above L2"},
        "solves_per_s": solves_per_s,
        "iters_per_step": iters / args.steps,
        "fp64_solve_s": fp64_s, "fp64_iters": i64["iters"], "mixed_solve_s": mixed_s, "mixed_iters": i32["iters"],
        "mixed_vs_fp64_speedup": fp64_s / mixed_s, "mixed_vs_fp64_rel_diff": diff,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * n, "d2h_bytes_per_step": 2 * 8 * n},
        "gpu_launches": launches,
        "roofline": {"kernel": "k_schwarz<float,float> (FP32 Schwarz apply)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": SCHWARZ_TRAFFIC_PER_ENTRY * nnz, "alg_bytes_per_launch": alg_bytes,
                     "avg_ms": avg_ms},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
