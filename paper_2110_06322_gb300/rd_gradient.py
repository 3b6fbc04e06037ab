"""Differentiable Schnakenberg run on the GPU (eq. schnack, Section 4.1.6): the
forward integration of `steps` semi-implicit Euler steps and the gradient of
L = 1/2 sum (u - u*)^2 + 1/2 sum (v - v*)^2 at the final step with respect to
D_u, D_v and the initial state, through the checkpointed adjoint.  Prints one
JSON line with the phase times, solve counts and gradient values.

    python -m paper_2110_06322_gb300.rd_gradient --workload schnakenberg_torus_h0.005 --steps 500

--fd-steps K additionally checks dL/dD_u and dL/dD_v of a K-step run against
central differences (relative step 1e-4; use --rtol 1e-13 so that the solves'
own error stays far below the differences).
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from paper_2110_06322_gb300 import autograd, cpm, inputs


def initial_state(w, n, device):
    us = 0.003 + 0.7
    vs = 0.7 / (us * us + 0.06)
    a = inputs.uniform(w["seed"], n)
    b = inputs.uniform(w["seed"] + 1, n)
    u0 = torch.from_numpy(us * (1.0 + 0.01 * (2.0 * a - 1.0))).to(device)
    v0 = torch.from_numpy(vs * (1.0 + 0.01 * (2.0 * b - 1.0))).to(device)
    return u0, v0, us, vs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="schnakenberg_torus_h0.005")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--checkpoint", type=int, default=None)
    ap.add_argument("--mixed", action="store_true", help="FP32 applies inside FP64 refinement for every solve")
    ap.add_argument("--fd-steps", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=None)
    a = ap.parse_args()
    w = inputs.WORKLOADS[a.workload]
    steps = a.steps if a.steps is not None else w["steps"]
    every = a.checkpoint if a.checkpoint is not None else w["checkpoint"]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    B = cpm.Band(w["kind"], w["params"], w["h"], w["p"])
    opts = dict(rtol=a.rtol if a.rtol is not None else w["rtol"], restart=w["restart"], maxit=50000)
    if a.mixed:
        opts.update(mixed=True)
    sim = autograd.Schnakenberg(B, dt=w["dt"], nparts=w["nparts"], overlap=w["overlap"], robin=w["robin"], **opts)
    n = B.n_active
    u0, v0, us, vs = initial_state(w, n, dev)
    cu, cv = sim.shifts(w["Du"], w["Dv"])
    sim._pc(cu)
    sim._pc(cv)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0

    ut = u0.clone().requires_grad_(True)
    vt = v0.clone().requires_grad_(True)
    Du = torch.tensor(w["Du"], dtype=torch.float64, device=dev, requires_grad=True)
    Dv = torch.tensor(w["Dv"], dtype=torch.float64, device=dev, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s0, i0 = sim.solves, len(sim.iters)
    uN, vN = sim.run(ut, vt, Du, Dv, steps=steps, checkpoint=every)
    loss = 0.5 * (((uN - us) ** 2).sum() + ((vN - vs) ** 2).sum())
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    s1, i1 = sim.solves, len(sim.iters)
    t0 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    s2 = sim.solves
    fit, bit = sim.iters[i0:i1], sim.iters[i1:]
    out = {
        "workload": a.workload, "n_active": n, "steps": steps, "checkpoint": every, "mixed": a.mixed,
        "c_u": cu, "c_v": cv, "setup_s": t_setup, "forward_s": t_fwd, "backward_s": t_bwd,
        "forward_solves": s1 - s0, "backward_solves": s2 - s1, "rtol": opts["rtol"],
        "forward_iters_u": sum(fit[0::2]), "forward_iters_v": sum(fit[1::2]), "backward_iters": sum(bit),
        "loss": loss.item(),
        "dL_dDu": Du.grad.item(), "dL_dDv": Dv.grad.item(), "grad_u0_norm": ut.grad.norm().item(),
        "grad_v0_norm": vt.grad.norm().item(),
    }
    if a.fd_steps > 0:
        k = a.fd_steps
        ut2 = u0.clone().requires_grad_(True)
        vt2 = v0.clone().requires_grad_(True)
        Du2 = torch.tensor(w["Du"], dtype=torch.float64, device=dev, requires_grad=True)
        Dv2 = torch.tensor(w["Dv"], dtype=torch.float64, device=dev, requires_grad=True)
        uK, vK = sim.run(ut2, vt2, Du2, Dv2, steps=k, checkpoint=every)
        (0.5 * (((uK - us) ** 2).sum() + ((vK - vs) ** 2).sum())).backward()

        def L(du, dv):
            with torch.no_grad():
                uu, vv = sim.run(u0, v0, du, dv, steps=k)
            return 0.5 * float(((uu - us) ** 2).sum() + ((vv - vs) ** 2).sum())
        fd = {}
        for name, g, d in (("Du", Du2.grad.item(), w["Du"]), ("Dv", Dv2.grad.item(), w["Dv"])):
            eps = 1e-4 * d
            p = {"Du": w["Du"], "Dv": w["Dv"]}
            m = dict(p)
            p[name] += eps
            m[name] -= eps
            f = (L(p["Du"], p["Dv"]) - L(m["Du"], m["Dv"])) / (2 * eps)
            fd[name] = {"adjoint": g, "central_difference": f, "rel_diff": abs(g - f) / abs(f)}
        out["fd_check"] = {"steps": k, **fd}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
