"""Runs the pipeline step of bench.py (band build, Schwarz set-up, mixed
forward and adjoint solves) on a named workload, for profiling with ncu:
no clock sampler, no host oracle, nothing else on the GPU.

    python -m paper_2110_06322_gb300.profile_step --workload torus_h0.025 --warmup 3 --steps 1
"""
from __future__ import annotations

import argparse

import torch

from paper_2110_06322_gb300 import cpm, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="torus_h0.025")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--steps", type=int, default=1)
    a = ap.parse_args()
    w = inputs.WORKLOADS[a.workload]
    L0 = cpm.cpm_kernel_launches()
    B0 = cpm.Band(w["kind"], w["params"], w["h"], w["p"])
    cp = B0.export()[3][: B0.n_active].cpu().numpy()
    f = torch.from_numpy(inputs.torus_rhs(cp, inputs.torus_modes(w["seed"]))).cuda()
    g = torch.from_numpy(inputs.torus_rhs(cp, inputs.torus_modes(w["seed"] + 100))).cuda()
    del B0
    torch.cuda.synchronize()
    print(f"setup launches={cpm.cpm_kernel_launches() - L0}", flush=True)
    kw = dict(restart=w["restart"], rtol=w["rtol"], maxit=50000, mixed=True, inner_rtol=1e-4)
    for q in range(a.warmup + a.steps):
        L0 = cpm.cpm_kernel_launches()
        B = cpm.Band(w["kind"], w["params"], w["h"], w["p"])
        P = cpm.Schwarz(B, w["c"], w["nparts"], w["overlap"], robin=w["robin"], store=cpm.CPM_F32)
        u, i1 = cpm.solve(B, f, P, **kw)
        lam, i2 = cpm.solve(B, g, P, adjoint=True, **kw)
        torch.cuda.synchronize()
        print(f"step {q}: N_A={B.n_active} iters={i1['iters']}+{i2['iters']} "
              f"launches={cpm.cpm_kernel_launches() - L0}", flush=True)
        del P, B


if __name__ == "__main__":
    main()
