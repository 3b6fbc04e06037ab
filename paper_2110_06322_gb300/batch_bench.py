"""Batched solves on the GPU: many independent problems of uneven size in one
cpm_solve_batch call, against the same systems solved one by one.

Problems (seeded): spheres of radius U[0.5, 1.5] and tori with R ~ U[0.8, 1.2],
r ~ U[0.2, 0.5] in equal numbers, grid spacing drawn from --hs, shift c
log-uniform in [0.1, 1000], 1-8 Gaussian right-hand sides each; a draw whose
band radius would exceed 0.9 of the surface's reach moves to the next finer
spacing.  Each problem gets a Schwarz preconditioner with about --rows
overlapping rows per subdomain.  Prints one JSON line.

    python -m paper_2110_06322_gb300.batch_bench --problems 96 --hs 0.05,0.025,0.0125
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from paper_2110_06322_gb300 import cpm, inputs


def draw_problems(nprob, hs, seed):
    u = inputs.uniform(seed, 8 * nprob).reshape(nprob, 8)
    hs = sorted(hs, reverse=True)
    out = []
    for q in range(nprob):
        sphere = q % 2 == 0
        if sphere:
            rho = 0.5 + u[q, 0]
            params = inputs.surface_params(inputs.SPHERE, a=rho)
            reach = rho
        else:
            R = 0.8 + 0.4 * u[q, 0]
            r = 0.2 + 0.3 * u[q, 1]
            params = inputs.surface_params(inputs.TORUS, a=R, b=r)
            reach = min(r, R - r)
        k = min(int(u[q, 2] * len(hs)), len(hs) - 1)
        while k < len(hs) - 1 and math.sqrt(17.0) * hs[k] >= 0.9 * reach:
            k += 1
        h = hs[k]
        if math.sqrt(17.0) * h >= 0.9 * reach:
            h = reach * 0.9 / math.sqrt(17.0) / 1.01
        c = 10.0 ** (-1.0 + 4.0 * u[q, 3])
        nrhs = 1 + min(int(u[q, 4] * 8), 7)
        out.append(dict(kind=inputs.SPHERE if sphere else inputs.TORUS, params=params, h=h, c=c, nrhs=nrhs,
                        seed=seed * 1000 + q))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=96)
    ap.add_argument("--hs", default="0.05,0.025,0.0125")
    ap.add_argument("--rows", type=int, default=13000)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--fp64", action="store_true", help="plain FP64 instead of FP32 applies in FP64 refinement")
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--skip-single", action="store_true")
    a = ap.parse_args()
    torch.cuda.set_device(0)
    hs = [float(x) for x in a.hs.split(",")]
    specs = draw_problems(a.problems, hs, a.seed)
    t0 = time.perf_counter()
    probs, rhs = [], []
    for sp in specs:
        B = cpm.Band(sp["kind"], sp["params"], sp["h"], 3)
        parts = max(1, int(round(B.n_active * 1.15 / a.rows)))
        P = cpm.Schwarz(B, sp["c"], parts, 2)
        F = np.stack([inputs.gaussian_vector(sp["seed"] + r, B.n_active) for r in range(sp["nrhs"])])
        probs.append((B, P, sp["c"]))
        rhs.append(torch.from_numpy(F).cuda())
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    opts = dict(rtol=a.rtol, maxit=100000, mixed=not a.fp64)
    # warm-up (builds nothing new; first-use costs of the kernels)
    cpm.solve_batch(probs[:2], rhs[:2], **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    U, infos = cpm.solve_batch(probs, rhs, **opts)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    n_sys = len(infos)
    pts = sum(int(b.n_active) * f.shape[0] for (b, _, _), f in zip(probs, rhs))
    pt_iters = 0
    q = 0
    for (b, _, _), f in zip(probs, rhs):
        for _ in range(f.shape[0]):
            pt_iters += int(b.n_active) * infos[q]["iters"]
            q += 1
    worst = max(i["rel_residual"] for i in infos)
    out = {
        "problems": len(probs), "systems": n_sys, "band_points_total": pts,
        "band_points_min": min(int(b.n_active) for b, _, _ in probs),
        "band_points_max": max(int(b.n_active) for b, _, _ in probs),
        "hs": hs, "mixed": not a.fp64, "rtol": a.rtol, "setup_s": t_setup, "batch_s": t_batch,
        "iters_total": sum(i["iters"] for i in infos), "iters_max": max(i["iters"] for i in infos),
        "converged": sum(1 for i in infos if i["status"] == 0), "worst_rel_residual": worst,
        "batch_solves_per_s": n_sys / t_batch, "batch_band_pt_iters_per_s": pt_iters / t_batch,
    }
    if not a.skip_single:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (B, P, c), f in zip(probs, rhs):
            for r in range(f.shape[0]):
                cpm.solve(B, f[r].contiguous(), P, c=c, **opts)
        torch.cuda.synchronize()
        t_single = time.perf_counter() - t0
        out.update(single_s=t_single, single_solves_per_s=n_sys / t_single, batch_speedup=t_single / t_batch)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
