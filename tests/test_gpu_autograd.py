"""GPU parity of the differentiable solve and of the semi-implicit Schnakenberg
steps (Section 4.1.6, eq. schnack) against the oracle and against central
finite differences of the GPU forward pass.

Tolerances: FP64 solves at rtol 1e-13.  States agree with the oracle's direct
solves to 1e-10 relative; adjoint gradients agree with the oracle's discrete
adjoint to 1e-8 relative and with central differences (relative step 1e-5 for
the coefficients, 1e-6 along random directions for the initial state) to
1e-6 relative.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla
import torch

from oracle import imex as oimex
from paper_2110_06322_gb300 import inputs

pytestmark = pytest.mark.gpu

SPH = (0.0, 0.0, 0.0, 1.0)
TOR = (0.0, 0.0, 0.0, 1.0, 0.4)
PRM = {"delta1": 0.003, "delta2": 0.7, "lambda": 0.06, "Du": 0.05, "Dv": 0.5, "dt": 0.01}
TIGHT = dict(rtol=1e-13, maxit=20000)


@pytest.fixture(scope="module")
def cpm():
    from paper_2110_06322_gb300 import cpm as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def ag(cpm):
    from paper_2110_06322_gb300 import autograd as a
    return a


@pytest.fixture(scope="module")
def sphere(cpm, oracle_mod):
    return cpm.Band(0, SPH, 0.1, 3), oracle_mod.Band(0, SPH, 0.1, 3)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _ic(n, seed, amp):
    us, vs = oimex.steady_state(PRM)
    a = inputs.gaussian_vector(seed, n)
    b = inputs.gaussian_vector(seed + 1, n)
    return us * (1.0 + amp * np.tanh(a)), vs * (1.0 + amp * np.tanh(b))


def test_solve_gradients(cpm, ag, oracle_mod):
    """L = 1/2 |u|^2 with u = M(c)^{-1} f: dL/df = M^{-T} u and dL/dc = -<M^{-T} u, u>
    against the oracle's sparse direct solves, and dL/dc against a central
    difference of the GPU solve."""
    B = cpm.Band(1, TOR, 0.05, 3)
    O = oracle_mod.Band(1, TOR, 0.05, 3)
    c = 10.0
    P = cpm.Schwarz(B, c, 16, 2)
    f = inputs.gaussian_vector(21, B.n_active)
    ft = _cuda(f).requires_grad_(True)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda", requires_grad=True)
    u = ag.solve(B, ft, ct, P, **TIGHT)
    (0.5 * (u * u).sum()).backward()
    M = O.M(c).to_scipy().tocsc()
    lu = sla.splu(M)
    ud = lu.solve(f)
    lam = lu.solve(ud, trans="T")
    gf = ft.grad.cpu().numpy()
    assert np.linalg.norm(gf - lam) <= 1e-9 * np.linalg.norm(lam)
    gc_o = -float(np.dot(lam, ud))
    assert abs(ct.grad.item() - gc_o) <= 1e-9 * abs(gc_o)

    def L(cc):
        uu, info = cpm.solve(B, _cuda(f), P, c=cc, **TIGHT)
        return 0.5 * float((uu * uu).sum())
    eps = 1e-5 * c
    fd = (L(c + eps) - L(c - eps)) / (2 * eps)
    assert abs(ct.grad.item() - fd) <= 1e-6 * abs(fd)


def test_imex_forward_matches_oracle(cpm, ag, sphere):
    B, O = sphere
    n = B.n_active
    u0, v0 = _ic(n, 31, 0.2)
    sim = ag.Schnakenberg(B, dt=PRM["dt"], nparts=8, overlap=2, **TIGHT)
    uN, vN = sim.run(_cuda(u0), _cuda(v0), PRM["Du"], PRM["Dv"], steps=6)
    states = oimex.Imex(O, PRM).run(u0, v0, 6)
    uo, vo = states[-1]
    assert np.linalg.norm(uN.cpu().numpy() - uo) <= 1e-10 * np.linalg.norm(uo)
    assert np.linalg.norm(vN.cpu().numpy() - vo) <= 1e-10 * np.linalg.norm(vo)
    # the homogeneous steady state stays put
    us, vs = sim.steady_state()
    u1, v1 = sim.run(torch.full((n,), us, dtype=torch.float64, device="cuda"),
                     torch.full((n,), vs, dtype=torch.float64, device="cuda"), PRM["Du"], PRM["Dv"], steps=3)
    assert (u1 - us).abs().max().item() < 1e-11 and (v1 - vs).abs().max().item() < 1e-11


@pytest.mark.parametrize("checkpoint", [1, 4, 100])
def test_imex_gradients_match_oracle_adjoint(cpm, ag, sphere, checkpoint):
    B, O = sphere
    n = B.n_active
    steps = 6
    u0, v0 = _ic(n, 41, 0.2)
    sim = ag.Schnakenberg(B, dt=PRM["dt"], nparts=8, overlap=2, **TIGHT)
    ut = _cuda(u0).requires_grad_(True)
    vt = _cuda(v0).requires_grad_(True)
    Du = torch.tensor(PRM["Du"], dtype=torch.float64, device="cuda", requires_grad=True)
    Dv = torch.tensor(PRM["Dv"], dtype=torch.float64, device="cuda", requires_grad=True)
    uN, vN = sim.run(ut, vt, Du, Dv, steps=steps, checkpoint=checkpoint)
    us, vs = sim.steady_state()
    loss = 0.5 * (((uN - us) ** 2).sum() + ((vN - vs) ** 2).sum())
    loss.backward()
    osim = oimex.Imex(O, PRM)
    Lo, ub, vb = oimex.steady_loss(osim.run(u0, v0, steps), PRM)
    gu, gv, gDu, gDv = osim.grad(u0, v0, steps, ub, vb)
    assert abs(loss.item() - Lo) <= 1e-10 * Lo
    assert np.linalg.norm(ut.grad.cpu().numpy() - gu) <= 1e-8 * np.linalg.norm(gu)
    assert np.linalg.norm(vt.grad.cpu().numpy() - gv) <= 1e-8 * np.linalg.norm(gv)
    assert abs(Du.grad.item() - gDu) <= 1e-8 * abs(gDu)
    assert abs(Dv.grad.item() - gDv) <= 1e-8 * abs(gDv)


def test_imex_gradients_match_finite_differences(cpm, ag):
    """Torus h = 0.05: dL/dD_u, dL/dD_v and a directional derivative in the
    initial state against central differences of the GPU forward run."""
    B = cpm.Band(1, TOR, 0.05, 3)
    n = B.n_active
    steps = 5
    u0, v0 = _ic(n, 51, 0.2)
    sim = ag.Schnakenberg(B, dt=PRM["dt"], nparts=16, overlap=2, **TIGHT)
    us, vs = sim.steady_state()

    def L(uu0, vv0, Du, Dv):
        with torch.no_grad():
            uN, vN = sim.run(uu0, vv0, Du, Dv, steps=steps)
        return 0.5 * float(((uN - us) ** 2).sum() + ((vN - vs) ** 2).sum())

    ut = _cuda(u0).requires_grad_(True)
    vt = _cuda(v0).requires_grad_(True)
    Du = torch.tensor(PRM["Du"], dtype=torch.float64, device="cuda", requires_grad=True)
    Dv = torch.tensor(PRM["Dv"], dtype=torch.float64, device="cuda", requires_grad=True)
    uN, vN = sim.run(ut, vt, Du, Dv, steps=steps, checkpoint=2)
    (0.5 * (((uN - us) ** 2).sum() + ((vN - vs) ** 2).sum())).backward()
    for name, g, d in (("Du", Du.grad.item(), PRM["Du"]), ("Dv", Dv.grad.item(), PRM["Dv"])):
        eps = 1e-5 * d
        a = {"Du": PRM["Du"], "Dv": PRM["Dv"]}
        b = dict(a)
        a[name] += eps
        b[name] -= eps
        fd = (L(_cuda(u0), _cuda(v0), **a) - L(_cuda(u0), _cuda(v0), **b)) / (2 * eps)
        assert abs(g - fd) <= 1e-6 * abs(fd), (name, g, fd)
    wu = inputs.gaussian_vector(61, n)
    wv = inputs.gaussian_vector(62, n)
    eps = 1e-6
    fd = (L(_cuda(u0 + eps * wu), _cuda(v0 + eps * wv), PRM["Du"], PRM["Dv"]) -
          L(_cuda(u0 - eps * wu), _cuda(v0 - eps * wv), PRM["Du"], PRM["Dv"])) / (2 * eps)
    g = float(np.dot(ut.grad.cpu().numpy(), wu) + np.dot(vt.grad.cpu().numpy(), wv))
    assert abs(g - fd) <= 1e-6 * abs(fd), (g, fd)


def test_imex_rhs_adjoint_accumulates(cpm, sphere):
    """The dL/dc output of cpm_imex_rhs_adjoint accumulates; ubar and vbar
    are overwritten."""
    B, O = sphere
    n = B.n_active
    x = [_cuda(inputs.gaussian_vector(70 + k, n)) for k in range(6)]
    ub, vb = torch.empty_like(x[0]), torch.empty_like(x[0])
    dc = torch.zeros(2, dtype=torch.float64, device="cuda")
    cpm.cpm_imex_rhs_adjoint(B.handle, PRM, *x, ub, vb, dc)
    first = dc.clone()
    cpm.cpm_imex_rhs_adjoint(B.handle, PRM, *x, ub, vb, dc)
    assert torch.allclose(dc, 2 * first, rtol=1e-15, atol=0)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    cpm.cpm_dot(B.handle, x[0], x[1], out)
    ref = float(np.dot(x[0].cpu().numpy(), x[1].cpu().numpy()))
    assert abs(out.item() - ref) <= 1e-12 * np.linalg.norm(x[0].cpu().numpy()) * np.linalg.norm(x[1].cpu().numpy())


@pytest.mark.parametrize("model", [0, 1])
def test_ars222_steps_match_oracle(cpm, ag, oracle_mod, sphere, model):
    """Second-order IMEX steps (ARS(2,2,2)) on the GPU against the oracle's
    steps with sparse direct solves: Schnakenberg (model 0) and the heat
    equation per species (model 1), four steps, states to 1e-10 relative."""
    B, O = sphere
    prm = dict(PRM, model=model)
    n = B.n_active
    u0, v0 = _ic(n, 41, 0.2)
    sim = ag.Schnakenberg(B, dt=prm["dt"], nparts=8, overlap=2, model=model, **TIGHT)
    u, v = sim.integrate(_cuda(u0), _cuda(v0), prm["Du"], prm["Dv"], 4, scheme="ars222")
    wu, wv = oimex.ImexArs2(O, prm).run(u0, v0, 4)
    assert np.abs(u.cpu().numpy() - wu).max() <= 1e-10 * np.abs(wu).max()
    assert np.abs(v.cpu().numpy() - wv).max() <= 1e-10 * np.abs(wv).max()
    assert sim.solves == 16


def test_euler_heat_model_matches_oracle(cpm, ag, oracle_mod, sphere):
    """The first-order step with no reaction (heat equation) against the oracle."""
    B, O = sphere
    prm = dict(PRM, model=1)
    u0, v0 = _ic(B.n_active, 43, 0.2)
    sim = ag.Schnakenberg(B, dt=prm["dt"], nparts=8, overlap=2, model=1, **TIGHT)
    u, v = sim.integrate(_cuda(u0), _cuda(v0), prm["Du"], prm["Dv"], 3, scheme="euler")
    wu, wv = oimex.Imex(O, prm).run(u0, v0, 3)[-1]
    assert np.abs(u.cpu().numpy() - wu).max() <= 1e-10 * np.abs(wu).max()
    assert np.abs(v.cpu().numpy() - wv).max() <= 1e-10 * np.abs(wv).max()
