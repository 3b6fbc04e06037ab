"""Differentiable solves and semi-implicit reaction-diffusion steps on the band.

``solve(band, f, c, pc)``: u = M(c)^{-1} f with M(c) = c I - Delta_S^h, the
shifted Poisson problem (Section 1, eq. shiftPoisson).  Its backward pass is
one adjoint solve and one dot product (both in libcpm):

    dL/df = lambda = M(c)^{-T} dL/du,      dL/dc = -<lambda, u>

(d u / d c = -M^{-1} u because d M / d c = I).

``Schnakenberg``: semi-implicit Euler steps of eq. schnack (Section 4.1.6),
diffusion implicit and reaction explicit, one shifted Poisson solve per
species and step (c_u = 1 / (D_u dt), c_v = 1 / (D_v dt)).  ``run`` is
differentiable with respect to the initial state (u0, v0) and the diffusion
coefficients (D_u, D_v): the backward pass walks the steps in reverse, one
adjoint solve per species and step, with the reaction's transposed Jacobian
and the dL/dc sums formed by ``cpm_imex_rhs_adjoint``.  Only every
``checkpoint``-th state is kept from the forward pass; the states inside a
segment are recomputed from its checkpoint when the reverse sweep reaches it.

Argument marshalling and the loop over steps live here; every vector
operation of a step runs in libcpm's kernels.
"""
from __future__ import annotations

import torch

from . import cpm


def _fwd_solve(band, pc, c, f, opts, tally=None):
    u, info = cpm.solve(band, f.contiguous(), pc, c=float(c), **opts)
    if info["status"] != cpm.CPM_OK:
        raise cpm.CpmError(info["status"], f"solve did not reach rtol: {info}")
    if tally is not None:
        tally.append(info["iters"])
    return u


def _adj_solve(band, pc, c, g, opts, tally=None):
    lam, info = cpm.solve(band, g.contiguous(), pc, c=float(c), adjoint=True, **opts)
    if info["status"] != cpm.CPM_OK:
        raise cpm.CpmError(info["status"], f"adjoint solve did not reach rtol: {info}")
    if tally is not None:
        tally.append(info["iters"])
    return lam


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, c, band, pc, opts):
        cval = float(c)
        u = _fwd_solve(band, pc, cval, f, opts)
        ctx.save_for_backward(u)
        ctx.band, ctx.pc, ctx.c, ctx.opts = band, pc, cval, opts
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        lam = _adj_solve(ctx.band, ctx.pc, ctx.c, gu, ctx.opts)
        gc = None
        if ctx.needs_input_grad[1]:
            out = torch.empty(1, dtype=torch.float64, device=u.device)
            cpm.cpm_dot(ctx.band.handle, lam, u, out)
            gc = -out.reshape(())
        return lam, gc, None, None, None


def solve(band, f, c, pc=None, **opts):
    """u = M(c)^{-1} f, differentiable in f (FP64 CUDA vector of N_A) and c
    (a float or a 0-dim FP64 tensor).  opts go to cpm.solve (rtol, restart,
    maxit, mixed, ...)."""
    if not torch.is_tensor(c):
        c = torch.tensor(float(c), dtype=torch.float64, device=f.device)
    return _SolveFn.apply(f, c, band, pc, opts)


class Schnakenberg:
    """Semi-implicit Euler integrator of eq. schnack on a Band.

    delta1, delta2, lam: reaction parameters (defaults of Section 4.1.6);
    dt: time step; nparts, overlap, robin: the Schwarz preconditioner of each
    species' solve (one per distinct c); solve_opts: rtol, restart, maxit, ...
    """

    ARS_GAMMA = 1.0 - 0.5 ** 0.5  # implicit diagonal of ARS(2,2,2)

    def __init__(self, band, delta1=0.003, delta2=0.7, lam=0.06, dt=0.01, nparts=8, overlap=2, robin=False,
                 model=0, **solve_opts):
        self.band = band
        self.model = int(model)  # 0 Schnakenberg reaction, 1 none (heat equation per species)
        self.delta1, self.delta2, self.lam, self.dt = float(delta1), float(delta2), float(lam), float(dt)
        self.nparts, self.overlap, self.robin = int(nparts), int(overlap), bool(robin)
        self.opts = dict(rtol=1e-10, maxit=20000)
        self.opts.update(solve_opts)
        self._pcs = {}
        self.solves = 0
        self.iters = []  # GMRES iterations of every solve, in order

    def steady_state(self):
        u = self.delta1 + self.delta2
        return u, self.delta2 / (u * u + self.lam)

    def params(self, Du, Dv):
        return {"delta1": self.delta1, "delta2": self.delta2, "lambda": self.lam, "Du": float(Du), "Dv": float(Dv),
                "dt": self.dt, "model": self.model}

    def shifts(self, Du, Dv):
        return 1.0 / (float(Du) * self.dt), 1.0 / (float(Dv) * self.dt)

    def _pc(self, c):
        key = float(c)
        if key not in self._pcs:
            self._pcs[key] = cpm.Schwarz(self.band, key, self.nparts, self.overlap, robin=self.robin)
        return self._pcs[key]

    def step(self, u, v, Du, Dv):
        """One step: (u, v) -> (u', v')."""
        prm = self.params(Du, Dv)
        cu, cv = self.shifts(Du, Dv)
        bu, bv = torch.empty_like(u), torch.empty_like(v)
        cpm.cpm_imex_rhs(self.band.handle, prm, u, v, bu, bv)
        u1 = _fwd_solve(self.band, self._pc(cu), cu, bu, self.opts, self.iters)
        v1 = _fwd_solve(self.band, self._pc(cv), cv, bv, self.opts, self.iters)
        self.solves += 2
        return u1, v1

    def step_ars222(self, u, v, Du, Dv):
        """One second-order IMEX Runge-Kutta step, ARS(2,2,2): two stages, each
        one solve per species with c = 1 / (gamma D dt) (stage right-hand sides
        by cpm_imex2_rhs).  Not differentiable (forward integration only)."""
        prm = self.params(Du, Dv)
        g = self.ARS_GAMMA
        cu, cv = 1.0 / (g * float(Du) * self.dt), 1.0 / (g * float(Dv) * self.dt)
        bu, bv = torch.empty_like(u), torch.empty_like(v)
        cpm.cpm_imex2_rhs(self.band.handle, prm, 2, u, v, None, None, bu, bv)
        u2 = _fwd_solve(self.band, self._pc(cu), cu, bu, self.opts, self.iters)
        v2 = _fwd_solve(self.band, self._pc(cv), cv, bv, self.opts, self.iters)
        cpm.cpm_imex2_rhs(self.band.handle, prm, 3, u, v, u2, v2, bu, bv)
        u3 = _fwd_solve(self.band, self._pc(cu), cu, bu, self.opts, self.iters)
        v3 = _fwd_solve(self.band, self._pc(cv), cv, bv, self.opts, self.iters)
        self.solves += 4
        return u3, v3

    def integrate(self, u0, v0, Du, Dv, steps, scheme="ars222"):
        """Forward integration without gradients: `scheme` is "euler"
        (semi-implicit Euler) or "ars222" (second order)."""
        u, v = u0.contiguous(), v0.contiguous()
        for _ in range(int(steps)):
            u, v = (self.step_ars222 if scheme == "ars222" else self.step)(u, v, float(Du), float(Dv))
        return u, v

    def run(self, u0, v0, Du, Dv, steps, checkpoint=25):
        """(u_steps, v_steps) after `steps` steps from (u0, v0); differentiable
        in u0, v0, Du, Dv (0-dim FP64 tensors or floats)."""
        dev = u0.device
        if not torch.is_tensor(Du):
            Du = torch.tensor(float(Du), dtype=torch.float64, device=dev)
        if not torch.is_tensor(Dv):
            Dv = torch.tensor(float(Dv), dtype=torch.float64, device=dev)
        return _ImexRun.apply(u0, v0, Du, Dv, self, int(steps), max(1, int(checkpoint)))


class _ImexRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, v0, Du, Dv, sim, steps, every):
        du, dv = float(Du), float(Dv)
        u, v = u0.contiguous(), v0.contiguous()
        ckpt = {0: (u, v)}
        for n in range(steps):
            u, v = sim.step(u, v, du, dv)
            if (n + 1) % every == 0 and n + 1 < steps:
                ckpt[n + 1] = (u, v)
        ctx.sim, ctx.steps, ctx.every, ctx.D, ctx.ckpt = sim, steps, every, (du, dv), ckpt
        return u, v

    @staticmethod
    def backward(ctx, gu, gv):
        sim, steps, every, (du, dv) = ctx.sim, ctx.steps, ctx.every, ctx.D
        band = sim.band
        prm = sim.params(du, dv)
        cu, cv = sim.shifts(du, dv)
        pu, pv = sim._pc(cu), sim._pc(cv)
        u0 = ctx.ckpt[0][0]
        ub = gu.contiguous() if gu is not None else torch.zeros_like(u0)
        vb = gv.contiguous() if gv is not None else torch.zeros_like(u0)
        dcs = torch.zeros(2, dtype=torch.float64, device=u0.device)  # dL/dc_u, dL/dc_v (accumulated by the library)
        for start in range(((steps - 1) // every) * every, -1, -every):
            end = min(start + every, steps)
            states = [ctx.ckpt[start]]
            for _ in range(start, end):
                states.append(sim.step(*states[-1], du, dv))
            for n in range(end - 1, start - 1, -1):
                (u, v), (u1, v1) = states[n - start], states[n - start + 1]
                lu = _adj_solve(band, pu, cu, ub, sim.opts, sim.iters)
                lv = _adj_solve(band, pv, cv, vb, sim.opts, sim.iters)
                sim.solves += 2
                ub, vb = torch.empty_like(u), torch.empty_like(v)
                cpm.cpm_imex_rhs_adjoint(band.handle, prm, u, v, u1, v1, lu, lv, ub, vb, dcs)
        gDu = (dcs[0] * (-cu / du)).reshape(())
        gDv = (dcs[1] * (-cv / dv)).reshape(())
        return ub, vb, gDu, gDv, None, None, None
