"""One large torus solved twice on the GPU: mixed precision (FP32 operator and
preconditioner inside FP64 refinement) and plain FP64, to the same relative
residual; prints one JSON line with sizes, set-up and solve times, iteration
counts, the FP64 true residual of both solutions and their relative
difference.

    python -m paper_2110_06322_gb300.scale_case --workload torus_h0.002
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from paper_2110_06322_gb300 import cpm, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="torus_h0.002")
    ap.add_argument("--store", choices=["f32", "bf16"], default="f32")
    a = ap.parse_args()
    w = inputs.WORKLOADS[a.workload]
    torch.cuda.set_device(0)

    def tick():
        torch.cuda.synchronize()
        return time.perf_counter()
    t0 = tick()
    B = cpm.Band(w["kind"], w["params"], w["h"], w["p"])
    t1 = tick()
    n = B.n_active
    cp = B.export()[3][:n].cpu().numpy()
    f = torch.from_numpy(inputs.torus_rhs(cp, inputs.torus_modes(w["seed"]))).cuda()
    store = cpm.CPM_F32 if a.store == "f32" else cpm.CPM_BF16
    t2 = tick()
    P = cpm.Schwarz(B, w["c"], w["nparts"], w["overlap"], robin=w["robin"], store=store)
    t3 = tick()
    kw = dict(restart=w["restart"], rtol=w["rtol"], maxit=50000)
    um, im = cpm.solve(B, f, P, mixed=True, **kw)
    t4 = tick()
    ud, idd = cpm.solve(B, f, P, mixed=False, **kw)
    t5 = tick()

    def true_rel(u):
        r = torch.empty_like(u)
        B.apply(w["c"], u, out=r)
        return float(((f - r).norm() / f.norm()).item())
    out = {
        "workload": a.workload, "n_active": n, "n_ghost": B.n_ghost, "nparts": w["nparts"],
        "stored_entries": P.total_nnz, "max_levels": P.max_levels, "store": a.store,
        "band_s": t1 - t0, "schwarz_setup_s": t3 - t2,
        "mixed_s": t4 - t3, "mixed_iters": im["iters"], "mixed_ir_steps": im["ir_steps"],
        "fp64_s": t5 - t4, "fp64_iters": idd["iters"],
        "mixed_true_rel_residual": true_rel(um), "fp64_true_rel_residual": true_rel(ud),
        "mixed_vs_fp64_rel_diff": float(((um - ud).norm() / ud.norm()).item()),
        "mixed_speedup": (t5 - t4) / (t4 - t3),
        "mixed_band_pt_iters_per_s": n * im["iters"] / (t4 - t3),
        "fp64_band_pt_iters_per_s": n * idd["iters"] / (t5 - t4),
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
