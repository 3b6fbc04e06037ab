"""GPU parity: band construction and the matrix-free operator vs the FP64 oracle.

Band lists, cube bases, closest points and interpolation weights must be
bit-identical (Section 2.1).  The FP64 apply must agree with the oracle's
assembled M within 1e-14 relative (only the summation order differs); the
FP32 apply within 2e-6 relative, a bound from FP32 rounding (about 1e-7 per
weight and per multiply-add over the 84 contractions of a row, times the
cancellation-free 6/h^2 scale of the stencil).
"""
import numpy as np
import pytest
import torch

from paper_2110_06322_gb300 import inputs

pytestmark = pytest.mark.gpu

SPH = (0.0, 0.0, 0.0, 1.0)
TOR = (0.0, 0.0, 0.0, 1.0, 0.4)
CASES = [(0, SPH, 0.1, 3), (0, SPH, 0.2, 3), (1, TOR, 0.05, 3), (0, (0.013, 0.1, -0.07, 0.7), 0.03, 3),
         (1, (0.1, 0.0, -0.05, 1.1, 0.35), 0.04, 2)]


@pytest.fixture(scope="module")
def cpm():
    from paper_2110_06322_gb300 import cpm as m
    m.lib()
    return m


def _tensor_weights(w1d):
    """(w_x[u] w_y[v]) w_z[w] in cube order, evaluated in float64 with the same order."""
    P1 = w1d.shape[2]
    W = (w1d[:, 0, :, None] * w1d[:, 1, None, :])[:, :, :, None] * w1d[:, 2, None, None, :]
    return W.reshape(len(w1d), P1 ** 3)


@pytest.mark.parametrize("kind,prm,h,p", CASES)
def test_band_is_bit_identical(cpm, oracle_mod, kind, prm, h, p):
    B = cpm.Band(kind, prm, h, p)
    O = oracle_mod.Band(kind, prm, h, p)
    assert (B.n_active, B.n_ghost, B.n_tube) == (O.n_active, O.n_ghost, O.n_tube)
    ijkA, ijkG, base, cp, perm = [t.cpu().numpy() for t in B.export()]
    oA, oG, obase, ocp = O.export()
    assert np.array_equal(ijkA, oA)
    assert np.array_equal(ijkG, oG)
    assert np.array_equal(base, obase)
    assert np.array_equal(cp.view(np.uint64), ocp.view(np.uint64))
    assert np.array_equal(perm, np.arange(B.n_active))
    W = _tensor_weights(B.weights().cpu().numpy())
    rows = np.unique(np.concatenate([np.arange(0, B.n_rows, max(1, B.n_rows // 500)), [B.n_rows - 1]]))
    for r in rows:
        assert np.array_equal(W[r].view(np.uint64), O.erow_weights(int(r)).view(np.uint64))


@pytest.mark.parametrize("kind,prm,h,p", CASES)
def test_apply_matches_oracle(cpm, oracle_mod, kind, prm, h, p):
    c = 1.0 if kind == 0 else 10.0
    B = cpm.Band(kind, prm, h, p)
    O = oracle_mod.Band(kind, prm, h, p)
    M = O.M(c)
    x = inputs.gaussian_vector(31, B.n_active)
    want = M.matvec(x)
    got = B.apply(c, torch.from_numpy(x).cuda()).cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-14 * scale
    got32 = B.apply(c, torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    assert np.abs(got32 - want).max() <= 2e-6 * scale
    # transposed operator
    wantT = M.transpose().matvec(x)
    gotT = B.apply(c, torch.from_numpy(x).cuda(), transpose=True).cpu().numpy()
    assert np.abs(gotT - wantT).max() <= 1e-14 * np.abs(wantT).max()
    gotT32 = B.apply(c, torch.from_numpy(x).float().cuda(), transpose=True).double().cpu().numpy()
    assert np.abs(gotT32 - wantT).max() <= 2e-6 * np.abs(wantT).max()


def test_apply_several_rhs_with_their_own_shift(cpm, oracle_mod):
    B = cpm.Band(1, TOR, 0.05, 3)
    O = oracle_mod.Band(1, TOR, 0.05, 3)
    cs = [0.5, 10.0, 1000.0]
    X = np.stack([inputs.gaussian_vector(40 + q, B.n_active) for q in range(3)])
    Y = B.apply(cs, torch.from_numpy(X).cuda().reshape(-1)).cpu().numpy().reshape(3, -1)
    for q, c in enumerate(cs):
        want = O.M(c).matvec(X[q])
        assert np.abs(Y[q] - want).max() <= 1e-14 * np.abs(want).max()


def test_fp32_apply_of_18_rhs_with_their_own_shift(cpm, oracle_mod):
    """The FP32 forward apply (staged by bricks) over more right-hand sides
    than one launch takes (16), each with its own shift."""
    B = cpm.Band(0, (0.013, 0.1, -0.07, 0.7), 0.03, 3)
    O = oracle_mod.Band(0, (0.013, 0.1, -0.07, 0.7), 0.03, 3)
    cs = [0.1 * 2.0 ** q for q in range(18)]
    X = np.stack([inputs.gaussian_vector(60 + q, B.n_active) for q in range(18)])
    Y = B.apply(cs, torch.from_numpy(X).float().cuda().reshape(-1)).double().cpu().numpy().reshape(18, -1)
    for q, c in enumerate(cs):
        want = O.M(c).matvec(X[q])
        assert np.abs(Y[q] - want).max() <= 2e-6 * np.abs(want).max()


def test_constant_is_mapped_to_c(cpm):
    B = cpm.Band(1, TOR, 0.01, 3)
    y = B.apply(7.0, torch.ones(B.n_active, dtype=torch.float64, device="cuda"))
    assert (y - 7.0).abs().max().item() < 1e-12 * 6 / 0.01 ** 2


def test_band_errors(cpm):
    with pytest.raises(cpm.CpmError) as e:
        cpm.Band(1, (0, 0, 0, 1.0, 0.2), 0.05, 3)  # band radius 0.206 beyond the reach 0.2
    assert e.value.status == cpm.CPM_ERR_BAND
    with pytest.raises(cpm.CpmError) as e:
        cpm.Band(0, SPH, 0.1, 1)
    assert e.value.status == cpm.CPM_ERR_ARG
    with pytest.raises(cpm.CpmError) as e:
        cpm.Band(2, SPH, 0.1, 3)
    assert e.value.status == cpm.CPM_ERR_ARG
    B = cpm.Band(0, SPH, 0.2, 3)
    x = torch.zeros(B.n_active, dtype=torch.float64, device="cuda")
    with pytest.raises(cpm.CpmError):
        B.apply(float("nan"), x)


def test_full_size_torus_band_and_sampled_rows(cpm, oracle_mod):
    """Torus R = 1, r = 0.4 at h = 0.004 (the FP64 ORAS-GMRES workload): the
    whole band bit-identical, operator rows sampled against the oracle."""
    h = 0.004
    B = cpm.Band(1, TOR, h, 3)
    O = oracle_mod.Band(1, TOR, h, 3)
    assert (B.n_active, B.n_ghost, B.n_tube) == (O.n_active, O.n_ghost, O.n_tube)
    ijkA, ijkG, base, cp, _ = [t.cpu().numpy() for t in B.export()]
    oA, oG, obase, ocp = O.export()
    assert np.array_equal(ijkA, oA) and np.array_equal(ijkG, oG) and np.array_equal(base, obase)
    assert np.array_equal(cp.view(np.uint64), ocp.view(np.uint64))
    x = inputs.gaussian_vector(77, B.n_active)
    rows = np.unique(np.concatenate([np.random.default_rng(0).integers(0, B.n_active, 3000), [0, B.n_active - 1]]))
    y = B.apply(10.0, torch.from_numpy(x).cuda()).cpu().numpy()
    want = O.apply_rows(10.0, x, rows)
    assert np.abs(y[rows] - want).max() <= 1e-14 * np.abs(want).max()
    y32 = B.apply(10.0, torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    assert np.abs(y32[rows] - want).max() <= 2e-6 * np.abs(want).max()
    cols = rows[::10]
    yT = B.apply(10.0, torch.from_numpy(x).cuda(), transpose=True).cpu().numpy()
    wantT = O.apply_T_cols(10.0, x, cols)
    assert np.abs(yT[cols] - wantT).max() <= 1e-14 * np.abs(wantT).max()
