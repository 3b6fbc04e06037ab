"""Pins of the oracle's semi-implicit Schnakenberg steps and their adjoint
(Section 4.1.6, eq. schnack), checked against facts the oracle does not
compute itself: the homogeneous steady state is a fixed point of every step,
and the adjoint gradients equal central finite differences of the forward
run (a wrong sign or a dropped term of the reaction Jacobian, of the shift
derivative or of the transposed solve fails them)."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import imex as oimex
from paper_2110_06322_gb300 import inputs

SPH = (0.0, 0.0, 0.0, 1.0)
PRM = {"delta1": 0.003, "delta2": 0.7, "lambda": 0.06, "Du": 0.05, "Dv": 0.5, "dt": 0.01}


@pytest.fixture(scope="module")
def band(oracle_mod):
    return oracle_mod.Band(0, SPH, 0.2, 3)


def _ic(n, seed, amp):
    us, vs = oimex.steady_state(PRM)
    a = inputs.gaussian_vector(seed, n)
    b = inputs.gaussian_vector(seed + 1, n)
    return us * (1.0 + amp * np.tanh(a)), vs * (1.0 + amp * np.tanh(b))


def test_steady_state_values():
    us, vs = oimex.steady_state(PRM)
    assert us == pytest.approx(0.703, abs=1e-15)
    assert vs == pytest.approx(0.7 / (0.703 ** 2 + 0.06), rel=1e-15)
    f, g = oimex.reaction(np.array([us]), np.array([vs]), PRM)
    assert abs(f[0]) < 1e-15 and abs(g[0]) < 1e-15


def test_steady_state_is_a_fixed_point(band):
    n = band.n_active
    us, vs = oimex.steady_state(PRM)
    sim = oimex.Imex(band, PRM)
    states = sim.run(np.full(n, us), np.full(n, vs), 5)
    u, v = states[-1]
    assert np.abs(u - us).max() < 1e-12 and np.abs(v - vs).max() < 1e-12


def test_adjoint_gradients_match_central_differences(band):
    n = band.n_active
    u0, v0 = _ic(n, 5, 0.2)
    steps = 4

    def loss(u0_, v0_, Du, Dv):
        p = dict(PRM, Du=Du, Dv=Dv)
        return oimex.steady_loss(oimex.Imex(band, p).run(u0_, v0_, steps), p)[0]

    sim = oimex.Imex(band, PRM)
    L, ub, vb = oimex.steady_loss(sim.run(u0, v0, steps), PRM)
    gu, gv, gDu, gDv = sim.grad(u0, v0, steps, ub, vb)
    for name, g, d in (("Du", gDu, PRM["Du"]), ("Dv", gDv, PRM["Dv"])):
        eps = 1e-5 * d
        kw = {"Du": PRM["Du"], "Dv": PRM["Dv"]}
        kp, km = dict(kw), dict(kw)
        kp[name] += eps
        km[name] -= eps
        fd = (loss(u0, v0, **kp) - loss(u0, v0, **km)) / (2 * eps)
        assert abs(g - fd) <= 1e-6 * abs(fd), (name, g, fd)
    for wseed in (11, 12):
        wu = inputs.gaussian_vector(wseed, n)
        wv = inputs.gaussian_vector(wseed + 50, n)
        eps = 1e-6
        fd = (loss(u0 + eps * wu, v0 + eps * wv, PRM["Du"], PRM["Dv"]) -
              loss(u0 - eps * wu, v0 - eps * wv, PRM["Du"], PRM["Dv"])) / (2 * eps)
        g = float(np.dot(gu, wu) + np.dot(gv, wv))
        assert abs(g - fd) <= 1e-6 * abs(fd), (g, fd)


# ------------------------------------------------------------------ second-order IMEX (ARS(2,2,2))
def test_ars_steady_state_is_a_fixed_point(band):
    n = band.n_active
    us, vs = oimex.steady_state(PRM)
    u, v = oimex.ImexArs2(band, PRM).run(np.full(n, us), np.full(n, vs), 3)
    assert np.abs(u - us).max() < 1e-12 and np.abs(v - vs).max() < 1e-12


def test_ars_heat_step_is_its_stability_function(band):
    """Without reaction (the heat equation, Section 4.1.3) one step is
    R(dt D Delta_h) u with R(z) = (1 + (1 - 2 gamma) z) / (1 - gamma z)^2, the
    stability function of the implicit tableau; evaluated here with sparse
    solves of I - gamma dt D Delta_h (Delta_h = -M(0))."""
    import scipy.sparse as sp
    prm = dict(PRM, model=1)
    n = band.n_active
    u0 = inputs.gaussian_vector(21, n)
    v0 = inputs.gaussian_vector(22, n)
    u1, v1 = oimex.ImexArs2(band, prm).run(u0, v0, 1)
    lap = -band.M(0.0).to_scipy().tocsc()
    g = oimex.ARS_GAMMA
    for x0, x1, D in ((u0, u1, prm["Du"]), (v0, v1, prm["Dv"])):
        z = prm["dt"] * D * lap
        A = (sp.identity(n, format="csc") - g * z).tocsc()
        want = sla.spsolve(A, sla.spsolve(A, x0 + (1.0 - 2.0 * g) * (z @ x0)))
        assert np.abs(x1 - want).max() <= 1e-11 * np.abs(want).max()


def test_ars_reaction_part_is_second_order_on_constants(band):
    """On spatially constant states the diffusion vanishes (Delta_h 1 = 0) and
    the step is the explicit tableau on the reaction ODE: errors against
    scipy's solve_ivp at tight tolerance fall by ~4 per halving of dt
    (semi-implicit Euler: ~2)."""
    from scipy.integrate import solve_ivp
    n = band.n_active
    u0, v0 = 1.2, 0.8
    T = 0.4

    def rhs(t, y):
        f, g = oimex.reaction(np.array([y[0]]), np.array([y[1]]), PRM)
        return [f[0], g[0]]
    ref = solve_ivp(rhs, (0.0, T), [u0, v0], method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = {"ars": [], "euler": []}
    for dt in (0.04, 0.02, 0.01):
        p = dict(PRM, dt=dt)
        steps = int(round(T / dt))
        u, v = oimex.ImexArs2(band, p).run(np.full(n, u0), np.full(n, v0), steps)
        errs["ars"].append(abs(u[0] - ref[0]) + abs(v[0] - ref[1]))
        u, v = oimex.Imex(band, p).run(np.full(n, u0), np.full(n, v0), steps)[-1]
        errs["euler"].append(abs(u[0] - ref[0]) + abs(v[0] - ref[1]))
    for k in range(2):
        assert 3.3 < errs["ars"][k] / errs["ars"][k + 1] < 4.7, errs
        assert 1.6 < errs["euler"][k] / errs["euler"][k + 1] < 2.4, errs


def test_ars_is_second_order_in_time_on_the_band(band):
    """Schnakenberg on the band: against a run with dt / 8, the ARS(2,2,2)
    error falls by ~4 per halving of dt."""
    n = band.n_active
    u0, v0 = _ic(n, 9, 0.3)
    T = 0.08
    p = dict(PRM, dt=T / 64)
    ref = oimex.ImexArs2(band, p).run(u0, v0, 64)
    errs = []
    for steps in (4, 8, 16):
        p = dict(PRM, dt=T / steps)
        u, v = oimex.ImexArs2(band, p).run(u0, v0, steps)
        errs.append(np.abs(u - ref[0]).max() + np.abs(v - ref[1]).max())
    for k in range(2):
        assert 3.2 < errs[k] / errs[k + 1] < 4.8, errs
