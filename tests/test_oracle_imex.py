"""Pins of the oracle's semi-implicit Schnakenberg steps and their adjoint
(Section 4.1.6, eq. schnack), checked against facts the oracle does not
compute itself: the homogeneous steady state is a fixed point of every step,
and the adjoint gradients equal central finite differences of the forward
run (a wrong sign or a dropped term of the reaction Jacobian, of the shift
derivative or of the transposed solve fails them)."""
import numpy as np
import pytest

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
