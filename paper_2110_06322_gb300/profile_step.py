"""Runs the pipeline step of bench.py (band build, Schwarz set-up, mixed
forward and adjoint solves) on a named workload, for profiling with ncu:
no clock sampler, no host oracle, nothing else on the GPU.

    python -m paper_2110_06322_gb300.profile_step --workload torus_h0.025 --warmup 3 --steps 1

With --setup-only a step is the set-up alone: band build, Schwarz set-up, and
one transposed operator and preconditioner apply (which build the transpose
map and the transposed factors on first use), each phase timed with CUDA
events.  With --apply-only KIND the band (and for KIND pc the Schwarz
preconditioner) is built once and a step is one FP32 apply of that kind: op
(the operator M), opT (its transpose) or pc (the Schwarz preconditioner), for
captures of those kernels alone.
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
    ap.add_argument("--setup-only", action="store_true")
    ap.add_argument("--apply-only", choices=["op", "opT", "pc"], default=None)
    ap.add_argument("--maxit", type=int, default=50000,
                    help="iteration cap of each solve (a short capture of the Krylov loop)")
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
    kw = dict(restart=w["restart"], rtol=w["rtol"], maxit=a.maxit, mixed=True, inner_rtol=1e-4, reorth=0)
    if a.apply_only:
        B = cpm.Band(w["kind"], w["params"], w["h"], w["p"])
        x = f.float()
        y = torch.empty_like(x)
        if a.apply_only == "pc":
            P = cpm.Schwarz(B, w["c"], w["nparts"], w["overlap"], robin=w["robin"], store=cpm.CPM_F32)
            run = lambda: P.apply(x, out=y)  # noqa: E731
        else:
            tr = a.apply_only == "opT"
            run = lambda: B.apply(w["c"], x, transpose=tr, out=y)  # noqa: E731
        run()  # first use builds the transpose map
        torch.cuda.synchronize()
        print(f"setup launches={cpm.cpm_kernel_launches() - L0}", flush=True)
        for q in range(a.warmup + a.steps):
            L1 = cpm.cpm_kernel_launches()
            run()
            torch.cuda.synchronize()
            print(f"apply step {q}: launches={cpm.cpm_kernel_launches() - L1}", flush=True)
        return
    if a.setup_only:
        for q in range(a.warmup + a.steps):
            L0 = cpm.cpm_kernel_launches()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record()
            B = cpm.Band(w["kind"], w["params"], w["h"], w["p"])
            ev[1].record()
            P = cpm.Schwarz(B, w["c"], w["nparts"], w["overlap"], robin=w["robin"], store=cpm.CPM_F32)
            ev[2].record()
            B.apply(w["c"], f.float(), transpose=True)
            ev[3].record()
            P.apply(f.float(), transpose=True)
            ev[4].record()
            torch.cuda.synchronize()
            ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
            print(f"setup step {q}: band {ms[0]:.1f} ms, schwarz {ms[1]:.1f} ms, first M^T apply {ms[2]:.1f} ms, "
                  f"first P^T apply {ms[3]:.1f} ms, launches={cpm.cpm_kernel_launches() - L0}", flush=True)
            del P, B
        return
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
