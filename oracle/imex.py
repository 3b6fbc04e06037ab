"""Oracle of the semi-implicit Schnakenberg steps and of their discrete adjoint
(TEST INFRASTRUCTURE: only the tests may import it).

Model (Section 4.1.6, eq. schnack) on the band, with the CPM operator
M(c) = c I - Delta_S^h assembled by the oracle (``Band.M``):

    u_t = D_u Delta_S u + f(u, v),   f = delta1 - u + u^2 v + lambda v
    v_t = D_v Delta_S v + g(u, v),   g = delta2 - u^2 v - lambda v

One semi-implicit Euler step (diffusion implicit, reaction explicit):

    (u' - u) / dt = D_u Delta_S u' + f(u, v)
    <=>  M(c_u) u' = c_u (u + dt f(u, v)),   c_u = 1 / (D_u dt)

and the same for v with c_v = 1 / (D_v dt).  The solves are sparse direct
(scipy's SuperLU of the oracle's FP64 matrix).

The adjoint of a loss L(u_N, v_N) is the chain rule written out step by
step, last step first:

    lambda_u = M(c_u)^{-T} dL/du'      (and lambda_v likewise)
    dL/du   = c_u (1 + dt f_u) lambda_u + c_v dt g_u lambda_v
    dL/dv   = c_u dt f_v lambda_u + c_v (1 + dt g_v) lambda_v
    dL/dc_u = <lambda_u, u + dt f - u'>        (b = c_u (u + dt f), u' = M^{-1} b,
                                               d u'/d c_u = M^{-1} (b / c_u - u'))
    dL/dD_u = -(c_u / D_u) * sum over steps of dL/dc_u

with f_u = -1 + 2uv, f_v = u^2 + lambda, g_u = -2uv, g_v = -u^2 - lambda.
Pinned in the tests by central finite differences of the forward run and by
the invariance of the homogeneous steady state u* = delta1 + delta2,
v* = delta2 / (u*^2 + lambda).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla


def reaction(u, v, prm):
    """f(u, v), g(u, v) of eq. schnack; zero for model 1 (no reaction: the
    heat equation u_t = D Delta_S u of Section 4.1.3 for each species)."""
    if prm.get("model", 0) == 1:
        return np.zeros_like(u), np.zeros_like(v)
    d1, d2, lam = prm["delta1"], prm["delta2"], prm["lambda"]
    f = d1 - u + u * u * v + lam * v
    g = d2 - u * u * v - lam * v
    return f, g


def steady_state(prm):
    u = prm["delta1"] + prm["delta2"]
    return u, prm["delta2"] / (u * u + prm["lambda"])


class Imex:
    """Semi-implicit Euler steps of the Schnakenberg system on an oracle Band."""

    def __init__(self, band, prm):
        self.prm = dict(prm)
        dt = prm["dt"]
        self.cu = 1.0 / (prm["Du"] * dt)
        self.cv = 1.0 / (prm["Dv"] * dt)
        Mu = band.M(self.cu).to_scipy().tocsc()
        Mv = band.M(self.cv).to_scipy().tocsc()
        self.lu_u = sla.splu(Mu)
        self.lu_v = sla.splu(Mv)

    def step(self, u, v):
        dt = self.prm["dt"]
        f, g = reaction(u, v, self.prm)
        u1 = self.lu_u.solve(self.cu * (u + dt * f))
        v1 = self.lu_v.solve(self.cv * (v + dt * g))
        return u1, v1

    def run(self, u0, v0, steps):
        """All states s_0 .. s_steps."""
        states = [(np.asarray(u0, dtype=np.float64).copy(), np.asarray(v0, dtype=np.float64).copy())]
        for _ in range(steps):
            states.append(self.step(*states[-1]))
        return states

    def grad(self, u0, v0, steps, ubar, vbar):
        """Gradients of a loss whose derivative with respect to the final
        state is (ubar, vbar): returns dL/du0, dL/dv0, dL/dDu, dL/dDv."""
        dt, lam = self.prm["dt"], self.prm["lambda"]
        states = self.run(u0, v0, steps)
        gu, gv = np.asarray(ubar, dtype=np.float64), np.asarray(vbar, dtype=np.float64)
        dcu = dcv = 0.0
        for n in range(steps - 1, -1, -1):
            u, v = states[n]
            u1, v1 = states[n + 1]
            lu = self.lu_u.solve(gu, trans="T")
            lv = self.lu_v.solve(gv, trans="T")
            f, g = reaction(u, v, self.prm)
            dcu += float(np.dot(lu, u + dt * f - u1))
            dcv += float(np.dot(lv, v + dt * g - v1))
            fu, fv = -1.0 + 2.0 * u * v, u * u + lam
            gu_, gv_ = -2.0 * u * v, -u * u - lam
            gu = self.cu * (1.0 + dt * fu) * lu + self.cv * dt * gu_ * lv
            gv = self.cu * dt * fv * lu + self.cv * (1.0 + dt * gv_) * lv
        gDu = -(self.cu / self.prm["Du"]) * dcu
        gDv = -(self.cv / self.prm["Dv"]) * dcv
        return gu, gv, gDu, gDv


def steady_loss(states, prm):
    """L = 1/2 sum (u - u*)^2 + 1/2 sum (v - v*)^2 at the last state, and its
    derivative with respect to that state."""
    us, vs = steady_state(prm)
    u, v = states[-1]
    return 0.5 * float(np.sum((u - us) ** 2) + np.sum((v - vs) ** 2)), u - us, v - vs


# ---------------------------------------------------------------------------
# Second-order IMEX Runge-Kutta step, ARS(2,2,2) of Ascher, Ruuth & Spiteri
# (1997): the paper integrates its reaction-diffusion and heat examples with
# PETSc's IMEX Runge-Kutta schemes (Section 4.1.3, Section 4.1.5); this is a
# second-order, L-stable member of that family.  With gamma = 1 - 1/sqrt(2),
# delta = 1 - 1/(2 gamma), F the reaction (explicit) and G = D Delta_S the
# diffusion (implicit):
#
#   U1 = u
#   U2 = u + dt gamma F(U1) + dt gamma G(U2)
#   U3 = u + dt (delta F(U1) + (1 - delta) F(U2)) + dt ((1 - gamma) G(U2) + gamma G(U3))
#   u' = U3
#
# so each stage is one shifted Poisson solve with c = 1 / (gamma D dt):
#   M(c) U2 = c (u + gamma dt F(U1))
#   M(c) U3 = c (u + dt (delta F(U1) + (1 - delta) F(U2)) + (1 - gamma) dt G(U2)),
# where dt G(U2) = (U2 - u - gamma dt F(U1)) / gamma follows from the first
# equation (no operator apply needed).
# ---------------------------------------------------------------------------
ARS_GAMMA = 1.0 - 1.0 / np.sqrt(2.0)
ARS_DELTA = 1.0 - 1.0 / (2.0 * ARS_GAMMA)


class ImexArs2:
    """ARS(2,2,2) steps of the two-species system on an oracle Band."""

    def __init__(self, band, prm):
        self.prm = dict(prm)
        dt, g = prm["dt"], ARS_GAMMA
        self.cu = 1.0 / (g * prm["Du"] * dt)
        self.cv = 1.0 / (g * prm["Dv"] * dt)
        self.lu_u = sla.splu(band.M(self.cu).to_scipy().tocsc())
        self.lu_v = sla.splu(band.M(self.cv).to_scipy().tocsc())

    def step(self, u, v):
        dt, g, d = self.prm["dt"], ARS_GAMMA, ARS_DELTA
        f1, g1 = reaction(u, v, self.prm)
        u2 = self.lu_u.solve(self.cu * (u + g * dt * f1))
        v2 = self.lu_v.solve(self.cv * (v + g * dt * g1))
        f2, g2 = reaction(u2, v2, self.prm)
        gu2 = (u2 - u - g * dt * f1) / g   # dt D_u Delta u2
        gv2 = (v2 - v - g * dt * g1) / g
        u3 = self.lu_u.solve(self.cu * (u + dt * (d * f1 + (1.0 - d) * f2) + (1.0 - g) * gu2))
        v3 = self.lu_v.solve(self.cv * (v + dt * (d * g1 + (1.0 - d) * g2) + (1.0 - g) * gv2))
        return u3, v3

    def run(self, u0, v0, steps):
        u, v = np.asarray(u0, dtype=np.float64).copy(), np.asarray(v0, dtype=np.float64).copy()
        for _ in range(steps):
            u, v = self.step(u, v)
        return u, v
