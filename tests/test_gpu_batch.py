"""GPU parity of the lockstep batched solver (cpm_solve_batch): problems with
different bands, shifts and numbers of right-hand sides in one call, checked
system by system against the oracle's sparse direct solves (FP64: 1e-10
relative at rtol 1e-12; mixed precision: 1e-8 at rtol 1e-10) and against the
single-system solver."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla
import torch

from paper_2110_06322_gb300 import inputs

pytestmark = pytest.mark.gpu

SPH = (0.0, 0.0, 0.0, 1.0)
SPH2 = (0.1, -0.2, 0.05, 0.7)
TOR = (0.0, 0.0, 0.0, 1.0, 0.4)


@pytest.fixture(scope="module")
def cpm():
    from paper_2110_06322_gb300 import cpm as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def batch(cpm, oracle_mod):
    """Three problems of uneven size: unit sphere h = 0.1 (c = 1, 2 RHS),
    torus h = 0.05 (c = 10, 3 RHS), small sphere h = 0.1 (c = 300, 1 RHS)."""
    specs = [(0, SPH, 0.1, 1.0, 2, 8), (1, TOR, 0.05, 10.0, 3, 16), (0, SPH2, 0.1, 300.0, 1, 4)]
    out = []
    for q, (kind, prm, h, c, k, parts) in enumerate(specs):
        B = cpm.Band(kind, prm, h, 3)
        O = oracle_mod.Band(kind, prm, h, 3)
        P = cpm.Schwarz(B, c, parts, 2)
        F = np.stack([inputs.gaussian_vector(100 + 10 * q + r, B.n_active) for r in range(k)])
        lu = sla.splu(O.M(c).to_scipy().tocsc())
        out.append(dict(B=B, P=P, c=c, F=F, lu=lu))
    return out


def _rhs(batch):
    return [torch.from_numpy(b["F"]).cuda() for b in batch]


def test_batch_fp64_matches_direct_solves(cpm, batch):
    U, infos = cpm.solve_batch([(b["B"], b["P"], b["c"]) for b in batch], _rhs(batch), rtol=1e-12, maxit=5000)
    q = 0
    for b, u in zip(batch, U):
        for r in range(b["F"].shape[0]):
            xd = b["lu"].solve(b["F"][r])
            got = u[r].cpu().numpy()
            assert infos[q]["status"] == 0 and infos[q]["rel_residual"] <= 1e-12, infos[q]
            assert np.linalg.norm(got - xd) <= 1e-10 * np.linalg.norm(xd)
            q += 1
    # the systems stop on their own: the easy one (c = 300) needs fewer iterations
    assert infos[-1]["iters"] < infos[0]["iters"]


def test_batch_matches_single_solves(cpm, batch):
    U, infos = cpm.solve_batch([(b["B"], b["P"], b["c"]) for b in batch], _rhs(batch), rtol=1e-11, maxit=5000)
    q = 0
    for b, u in zip(batch, U):
        for r in range(b["F"].shape[0]):
            us, info = cpm.solve(b["B"], torch.from_numpy(b["F"][r]).cuda(), b["P"], c=b["c"], rtol=1e-11,
                                 maxit=5000)
            assert abs(infos[q]["iters"] - info["iters"]) <= 1
            assert torch.linalg.norm(u[r] - us) <= 1e-9 * torch.linalg.norm(us)
            q += 1


def test_batch_mixed_precision(cpm, batch):
    U, infos = cpm.solve_batch([(b["B"], b["P"], b["c"]) for b in batch], _rhs(batch), rtol=1e-10, maxit=5000,
                               mixed=True)
    for b, u in zip(batch, U):
        for r in range(b["F"].shape[0]):
            xd = b["lu"].solve(b["F"][r])
            assert np.linalg.norm(u[r].cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    assert all(i["status"] == 0 and i["ir_steps"] >= 1 for i in infos)


def test_batch_adjoint(cpm, batch):
    U, infos = cpm.solve_batch([(b["B"], b["P"], b["c"]) for b in batch], _rhs(batch), rtol=1e-12, maxit=5000,
                               adjoint=True)
    for b, u in zip(batch, U):
        for r in range(b["F"].shape[0]):
            xd = b["lu"].solve(b["F"][r], trans="T")
            assert np.linalg.norm(u[r].cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)


def test_batch_edge_cases(cpm, batch):
    b0, b1 = batch[0], batch[1]
    F0 = b0["F"].copy()
    F0[1] = 0.0  # a zero right-hand side stays zero and takes no iteration
    rhs = [torch.from_numpy(F0).cuda(), torch.from_numpy(b1["F"][0]).cuda()]
    # problem 1 without a preconditioner
    U, infos = cpm.solve_batch([(b0["B"], b0["P"], b0["c"]), (b1["B"], None, b1["c"])], rhs, rtol=1e-10,
                               maxit=20000)
    assert infos[1]["iters"] == 0 and U[0][1].abs().max().item() == 0.0
    xd = b1["lu"].solve(b1["F"][0])
    assert np.linalg.norm(U[1].cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    # iteration limit: reported per system
    st, inf = cpm.cpm_solve_batch([b0["B"].handle], [b0["P"].handle], [b0["c"]], [2],
                                  torch.from_numpy(b0["F"].reshape(-1)).cuda(),
                                  torch.zeros(b0["F"].size, dtype=torch.float64, device="cuda"), rtol=1e-12, maxit=3)
    assert st == cpm.CPM_ERR_NOT_CONVERGED
    assert all(i["status"] == cpm.CPM_ERR_NOT_CONVERGED and i["iters"] == 3 for i in inf)
