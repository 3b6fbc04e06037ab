"""Pins of the oracle's geometry: closest points, interpolation weights, band.

Each test checks the oracle against something other than its own formula:
closed forms, the defining minimisation, brute force, or invariants.
Paper: Section 2.1 (eq. cpFunc, the extension operator E, Sigma_A / Sigma_G).
"""
import math
import os

import numpy as np
import pytest

from paper_2110_06322_gb300 import inputs

SPH = (0.0, 0.0, 0.0, 1.0)
TOR = (0.0, 0.0, 0.0, 1.0, 0.4)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ closest points
def test_sphere_cp_is_the_minimiser(oracle_mod):
    rng = np.random.default_rng(0)
    # random points in a shell around an off-centre sphere
    prm = (0.3, -0.2, 0.1, 0.8)
    ys = rng.normal(size=(4000, 3))
    ys = prm[3] * ys / np.linalg.norm(ys, axis=1)[:, None] + np.array(prm[:3])
    for _ in range(200):
        d = rng.normal(size=3)
        x = np.array(prm[:3]) + (0.5 + rng.random()) * prm[3] * d / np.linalg.norm(d)
        st, cp, dist = oracle_mod.cp_dist(0, prm, x)
        assert st == 0
        assert abs(np.linalg.norm(cp - prm[:3]) - prm[3]) < 1e-14
        assert abs(np.linalg.norm(x - cp) - dist) < 1e-14
        # no point of the sphere is closer than cp
        assert np.linalg.norm(ys - x, axis=1).min() >= dist - 1e-12


def test_torus_cp_matches_brute_force_minimisation(oracle_mod):
    from scipy.optimize import minimize
    R, r = 1.0, 0.4
    rng = np.random.default_rng(1)

    def surf(t):
        th, ph = t
        return np.array([(R + r * math.cos(th)) * math.cos(ph), (R + r * math.cos(th)) * math.sin(ph),
                         r * math.sin(th)])

    th, ph = np.meshgrid(np.linspace(0, 2 * math.pi, 181), np.linspace(0, 2 * math.pi, 361), indexing="ij")
    grid = np.stack([(R + r * np.cos(th)) * np.cos(ph), (R + r * np.cos(th)) * np.sin(ph), r * np.sin(th)], -1)
    grid = grid.reshape(-1, 3)
    tgrid = np.stack([th.ravel(), ph.ravel()], -1)
    for _ in range(40):
        t0 = rng.random(2) * 2 * math.pi
        n = surf(t0) - np.array([R * math.cos(t0[1]), R * math.sin(t0[1]), 0.0])
        x = surf(t0) + (rng.random() - 0.5) * 0.5 * n  # within 0.1 of the surface
        st, cp, dist = oracle_mod.cp_dist(1, TOR, x)
        assert st == 0
        q = int(np.argmin(np.linalg.norm(grid - x, axis=1)))
        res = minimize(lambda t: float(np.sum((surf(t) - x) ** 2)), tgrid[q], method="Nelder-Mead",
                       options={"xatol": 1e-12, "fatol": 1e-20, "maxiter": 4000})
        y = surf(res.x)
        assert np.linalg.norm(y - cp) < 1e-6
        assert abs(np.linalg.norm(x - y) - dist) < 1e-9
        # cp lies on the torus
        assert abs((math.hypot(cp[0], cp[1]) - R) ** 2 + cp[2] ** 2 - r * r) < 1e-14


def test_reach(oracle_mod):
    L = oracle_mod.lib()
    assert L.orc_reach(0, np.array([0, 0, 0, 0.7, 0, 0, 0, 0.0])) == 0.7
    assert L.orc_reach(1, np.array([0, 0, 0, 1.0, 0.4, 0, 0, 0.0])) == 0.4
    assert L.orc_reach(1, np.array([0, 0, 0, 1.0, 0.7, 0, 0, 0.0])) == pytest.approx(0.3)


# ------------------------------------------------------------------ 1-D weights
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_weights_partition_of_unity_and_reproduction(oracle_mod, p):
    rng = np.random.default_rng(p)
    for s in np.concatenate([rng.random(300) * p, [0.5, 1.0 + 1e-15, 2.0 - 1e-13]]):
        w = oracle_mod.weights1d(p, s)
        assert abs(w.sum() - 1.0) <= 8 * np.finfo(float).eps
        for q in range(p + 1):  # reproduces every polynomial of degree <= p
            assert abs(np.dot(w, np.arange(p + 1.0) ** q) - s ** q) <= 1e-13 * max(1.0, s ** q) * p ** q
    # but not degree p + 1
    s = 0.37
    w = oracle_mod.weights1d(p, s)
    assert abs(np.dot(w, np.arange(p + 1.0) ** (p + 1)) - s ** (p + 1)) > 1e-6


@pytest.mark.parametrize("p", [2, 3])
def test_weights_equal_lagrange_product_form(oracle_mod, p):
    rng = np.random.default_rng(7)
    for s in rng.random(500) * p:
        w = oracle_mod.weights1d(p, s)
        lag = [np.prod([(s - k) / (j - k) for k in range(p + 1) if k != j]) for j in range(p + 1)]
        assert np.allclose(w, lag, rtol=0, atol=1e-14)
    for j in range(p + 1):  # nodes: unit vectors exactly
        e = np.zeros(p + 1)
        e[j] = 1.0
        assert np.array_equal(oracle_mod.weights1d(p, float(j)), e)


def test_band_lambda_is_sqrt17_h_for_cubic(oracle_mod):
    # (d-1)((p+1)/2)^2 + (1+(p+1)/2)^2 = 2*4 + 9 = 17 for d=3, p=3
    assert oracle_mod.band_lambda(0.1, 3) == 0.1 * math.sqrt(17.0)
    assert oracle_mod.band_lambda(1.0, 2) == math.sqrt(10.75)


# ------------------------------------------------------------------ band
def _tube_volume(kind, prm, lam):
    if kind == 0:
        rho = prm[3]
        return 4.0 / 3.0 * math.pi * ((rho + lam) ** 3 - (rho - lam) ** 3)
    R, r = prm[3], prm[4]
    return 2.0 * math.pi ** 2 * R * ((r + lam) ** 2 - (r - lam) ** 2)  # Pappus


@pytest.mark.parametrize("kind,prm,h,tol", [(0, SPH, 0.05, 0.01), (1, TOR, 0.025, 0.01), (0, (0.013, 0.1, -0.07, 0.7), 0.04, 0.015)])
def test_tube_count_matches_closed_form_volume(oracle_mod, kind, prm, h, tol):
    B = oracle_mod.Band(kind, prm, h, 3)
    lam = oracle_mod.band_lambda(h, 3)
    assert abs(B.n_tube * h ** 3 / _tube_volume(kind, prm, lam) - 1.0) < tol


@pytest.mark.parametrize("kind,prm,h", [(0, SPH, 0.2), (1, TOR, 0.08), (0, (0.013, 0.1, -0.07, 0.7), 0.09)])
def test_band_structure_and_closure(oracle_mod, kind, prm, h):
    B = oracle_mod.Band(kind, prm, h, 3)
    A, G, base, cp = B.export()
    # canonical order: strictly increasing lexicographic keys
    for X in (A, G):
        key = (X[:, 0].astype(np.int64) << 42) + (X[:, 1].astype(np.int64) << 21) + X[:, 2]
        assert np.all(np.diff(key) > 0)
    setA = set(map(tuple, A.tolist()))
    setG = set(map(tuple, G.tolist()))
    assert not (setA & setG)
    nb = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    # every 6-neighbour of an active node is active or ghost; every ghost touches an active node
    setR = setA | setG
    for (i, j, k) in A.tolist():
        for d in nb:
            assert (i + d[0], j + d[1], k + d[2]) in setR
    for (i, j, k) in G.tolist():
        assert any((i + d[0], j + d[1], k + d[2]) in setA for d in nb)
    # closure: every E-row cube lies in Sigma_A; cp is the closest point of its row node
    rows = np.concatenate([A, G])

    def key(X):
        X = X.astype(np.int64) + (1 << 20)
        return (X[..., 0] << 42) + (X[..., 1] << 21) + X[..., 2]

    keysA = np.sort(key(A))
    off = np.stack(np.meshgrid(range(4), range(4), range(4), indexing="ij"), -1).reshape(-1, 3)
    cube = key(base[:, None, :] + off[None, :, :]).ravel()
    pos = np.clip(np.searchsorted(keysA, cube), 0, len(keysA) - 1)
    assert np.all(keysA[pos] == cube)
    x = rows * h
    lam = oracle_mod.band_lambda(h, 3)
    d = np.linalg.norm(x - cp, axis=1)
    assert d.max() <= lam * (1 + 1e-12)
    # base = floor(cp / h - 1) and s in [1, 2)
    s = cp / h - base
    assert np.all(s >= 1.0 - 1e-12) and np.all(s < 2.0 + 1e-12)


def test_active_set_is_exactly_the_union_of_cubes(oracle_mod):
    """Brute force on a tiny band: Sigma_A = union over lattice x with
    dist(x) <= lambda of the cube at cp(x)."""
    h, prm = 0.2, (0.05, -0.02, 0.01, 1.0)
    B = oracle_mod.Band(0, prm, h, 3)
    A = set(map(tuple, B.export()[0].tolist()))
    lam = oracle_mod.band_lambda(h, 3)
    union = set()
    rng = range(-12, 13)
    for i in rng:
        for j in rng:
            for k in rng:
                x = np.array([i * h, j * h, k * h])
                st, cp, dist = oracle_mod.cp_dist(0, prm, x)
                if dist <= lam:
                    b = np.floor(cp / h - 1.0).astype(int)
                    for u in range(4):
                        for v in range(4):
                            for w in range(4):
                                union.add((b[0] + u, b[1] + v, b[2] + w))
    assert union == A


def test_sphere_band_is_symmetric_under_axis_swap(oracle_mod):
    B = oracle_mod.Band(0, SPH, 0.1, 3)
    A = B.export()[0]
    s1 = set(map(tuple, A.tolist()))
    s2 = set(map(tuple, A[:, [1, 0, 2]].tolist()))
    assert s1 == s2


def test_band_count_scales_like_the_papers_counts(oracle_mod):
    """The paper's torus unknown counts at h = 1/300, 1/420, 1/595, 1/600 keep
    N h^2 constant to 0.6 %; our band obeys the same law (N_A h^2 converges)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_unknown_counts.txt")) if ln.strip() and not ln.startswith("#")]
    nh2 = [int(n) / float(res) ** 2 for res, n in rows]
    assert max(nh2) / min(nh2) - 1.0 < 0.006
    vals = []
    for h in (0.05, 0.025, 0.0125):
        vals.append(oracle_mod.Band(1, TOR, h, 3).n_active * h * h)
    assert abs(vals[2] / vals[1] - 1) < abs(vals[1] / vals[0] - 1)
    assert abs(vals[2] / vals[1] - 1) < 0.01


@pytest.mark.parametrize("kind,prm,h,p", [(0, (0.0, 0.0, 0.0, 1.0), 0.1, 3), (1, (0.0, 0.0, 0.0, 1.0, 0.4), 0.05, 3),
                                           (0, (0.013, 0.1, -0.07, 0.7), 0.03, 2)])
def test_erow_cubes_lie_near_their_rows(oracle_mod, kind, prm, h, p):
    """Every E row's interpolation cube lies within 6 cells of the row per
    axis: active nodes are cube nodes, within 2 cells of a closest point per
    axis (so within 2 sqrt(3) h of S), ghosts one cell further (4.46 h), and a
    row's cube spans its closest point +-2 cells.  The FP32 apply that stages x
    by 16^3 bricks relies on this: a brick's box (its nodes and the cubes of
    the rows they need) spans at most 16 + 2 + 12 = 30 cells per axis."""
    B = oracle_mod.Band(kind, prm, h, p)
    A, G, base, cp = B.export()
    rows = np.concatenate([A, G])
    assert (base - rows).min() >= -6
    assert (base + p - rows).max() <= 6
    # the rows lie within 2 sqrt(3) h + h of the surface
    d = np.linalg.norm(cp / h - rows, axis=1)
    assert d.max() <= 2.0 * math.sqrt(3.0) + 1.0 + 1e-9


def test_reach_violation_is_rejected(oracle_mod):
    with pytest.raises(oracle_mod.BandError) as e:
        oracle_mod.Band(1, (0, 0, 0, 1.0, 0.2), 0.05, 3)  # lambda = 0.206 > r
    assert e.value.status == 4


def test_extension_reproduces_tricubic_polynomials(oracle_mod):
    B = oracle_mod.Band(1, TOR, 0.08, 3)
    A, G, base, cp = B.export()
    E = B.E().to_scipy()
    x = A * B.h
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b, c = rng.integers(0, 4, size=3)
        f = x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
        want = cp[:, 0] ** a * cp[:, 1] ** b * cp[:, 2] ** c
        assert np.abs(E @ f - want).max() < 1e-12
    assert np.abs(E @ np.ones(B.n_active) - 1.0).max() < 1e-14
