"""Pins of the oracle's operator, Schwarz preconditioners, ILU(0) and GMRES.

Paper: Section 2.1 eq. lapBel (stabilised Delta_S^h), Section 2.2 (RAS/ORAS),
Section 4.1.1 (GMRES, ILU(0) local solves, alpha = 4, alpha_cross = 20).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla
from scipy.sparse.csgraph import shortest_path

from paper_2110_06322_gb300 import inputs

SPH = (0.0, 0.0, 0.0, 1.0)
TOR = (0.0, 0.0, 0.0, 1.0, 0.4)
NB = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]


@pytest.fixture(scope="module")
def sphere02(oracle_mod):
    B = oracle_mod.Band(0, SPH, 0.2, 3)
    return B, B.M(1.0)


@pytest.fixture(scope="module")
def torus008(oracle_mod):
    B = oracle_mod.Band(1, TOR, 0.08, 3)
    return B, B.M(10.0)


def _key(X):
    X = np.asarray(X, dtype=np.int64) + (1 << 20)
    return (X[..., 0] << 42) + (X[..., 1] << 21) + X[..., 2]


def _lookup(sorted_keys, X):
    k = _key(X)
    pos = np.clip(np.searchsorted(sorted_keys, k), 0, len(sorted_keys) - 1)
    return np.where(sorted_keys[pos] == k, pos, -1)


# ------------------------------------------------------------------ operator
def test_operator_annihilates_constants(oracle_mod, torus008):
    B, M = torus008
    y = M.matvec(np.ones(B.n_active))
    assert np.abs(y - 10.0).max() < 1e-12 * 6.0 / B.h ** 2


def test_M_equals_library_product_of_definition(oracle_mod, torus008):
    """M = (c + 6/h^2) I - L_off E with L_off built from the 6-neighbour
    structure and the product taken by scipy (eq. lapBel)."""
    B, M = torus008
    A, G, _, _ = B.export()
    rows = np.concatenate([A, G])
    order = np.argsort(_key(rows))
    skeys = _key(rows)[order]
    nbr = np.stack([order[_lookup(skeys, A + np.array(d))] for d in NB], 1)
    coef = 1.0 / (B.h * B.h)
    Loff = sp.csr_matrix((np.full(nbr.size, coef), nbr.ravel(), np.arange(0, nbr.size + 1, 6)),
                         shape=(B.n_active, B.n_rows))
    want = (10.0 + 6.0 * coef) * sp.eye(B.n_active) - Loff @ B.E().to_scipy()
    got = M.to_scipy()
    diff = abs(got - want).max()
    assert diff < 1e-12 * 6.0 * coef


def test_sphere_harmonic_consistency_is_second_order(oracle_mod):
    """On the unit sphere u = Y(cp(x)) with Y = (x^2-y^2)z (Delta_S Y = -12 Y)
    has Delta(u o cp)(x) = -12 u / |x|^2, so (M u)_i -> c u_i + 12 u_i / r_i^2."""
    errs = []
    for h in (0.1, 0.05):
        B = oracle_mod.Band(0, SPH, h, 3)
        A, _, _, cp = B.export()
        u = inputs.y32(cp[: B.n_active])
        r = np.linalg.norm(A * h, axis=1)
        errs.append(np.abs(B.M(1.0).matvec(u) - (u + 12.0 * u / r ** 2)).max())
    assert errs[0] / errs[1] > 3.5


def test_sphere_solution_converges_at_second_order(oracle_mod):
    errs = []
    for h in (0.2, 0.1, 0.05):
        B = oracle_mod.Band(0, SPH, h, 3)
        cp = B.export()[3][: B.n_active]
        u = inputs.y32(cp)
        M = B.M(1.0)
        P = oracle_mod.ORAS(B, M, 8, 2)
        x, info = oracle_mod.gmres(M, 13.0 * u, P, rtol=1e-12)
        assert info["status"] == 0
        errs.append(np.abs(x - u).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() >= 1.8


def test_sampled_rows_and_transpose(oracle_mod, torus008):
    B, M = torus008
    x = inputs.gaussian_vector(11, B.n_active)
    y = inputs.gaussian_vector(12, B.n_active)
    rows = np.arange(0, B.n_active, 97)
    assert np.abs(B.apply_rows(10.0, x, rows) - M.matvec(x)[rows]).max() < 1e-9
    MT = M.transpose()
    assert abs(np.dot(M.matvec(x), y) - np.dot(x, MT.matvec(y))) < 1e-12 * np.abs(M.matvec(x)).sum()
    assert abs(MT.to_scipy() - M.to_scipy().T).max() == 0.0
    cols = np.arange(3, B.n_active, 311)
    assert np.abs(B.apply_T_cols(10.0, y, cols) - MT.matvec(y)[cols]).max() < 1e-9


# ------------------------------------------------------------------ partition / overlap
@pytest.mark.parametrize("nparts", [8, 13])
def test_partition_is_boxes_and_balanced(oracle_mod, torus008, nparts):
    B, M = torus008
    P = oracle_mod.ORAS(B, M, nparts, 0)
    part = P.partition()
    A = B.export()[0]
    assert part.min() == 0 and part.max() == nparts - 1
    counts = np.bincount(part, minlength=nparts)
    assert counts.max() <= 1.5 * B.n_active / nparts
    lo = np.array([A[part == j].min(0) for j in range(nparts)])
    hi = np.array([A[part == j].max(0) for j in range(nparts)])
    for j in range(nparts):
        inside = np.all((A >= lo[j]) & (A <= hi[j]), axis=1)
        assert np.all(part[inside] == j)  # each part is the band cut by its bounding box


def test_overlap_is_graph_ball(oracle_mod, sphere02):
    B, M = sphere02
    A = B.export()[0]
    skeys = np.sort(_key(A))
    ii, jj = [], []
    for d in NB:
        nb = _lookup(skeys, A + np.array(d))
        ok = nb >= 0
        ii.append(np.nonzero(ok)[0])
        jj.append(nb[ok])
    Gph = sp.csr_matrix((np.ones(sum(len(x) for x in ii)), (np.concatenate(ii), np.concatenate(jj))),
                        shape=(B.n_active, B.n_active))
    for NO in (1, 2):
        P = oracle_mod.ORAS(B, M, 6, NO)
        part = P.partition()
        for j in range(6):
            dist = shortest_path(Gph, unweighted=True, indices=np.nonzero(part == j)[0], directed=False).min(0)
            want = np.nonzero(dist <= NO)[0]
            assert np.array_equal(np.sort(P.sub_nodes(j)), want)


# ------------------------------------------------------------------ local solvers
@pytest.mark.parametrize("order", [0, 1, 2])
def test_ilu0_reproduces_A_on_its_pattern(oracle_mod, sphere02, order):
    B, M = sphere02
    P = oracle_mod.ORAS(B, M, 1, 0, order=order)
    A = P.sub_matrix(0).to_scipy()
    F = P.sub_factors(0).to_scipy()
    L = sp.tril(F, -1) + sp.eye(F.shape[0])
    U = sp.triu(F)
    LU = (L @ U).tocsr()
    pat = A.copy()
    pat.data[:] = 1.0
    diff = (LU - A).multiply(pat)
    assert abs(diff).max() < 1e-10 * abs(A).max()
    # ILU(0) of the whole operator is not its LU: fill-in was dropped
    assert abs(LU - A).max() > 1e-6


def test_single_subdomain_exact_solve_is_the_inverse(oracle_mod, sphere02):
    B, M = sphere02
    P = oracle_mod.ORAS(B, M, 1, 0, exact=True)
    f = inputs.gaussian_vector(3, B.n_active)
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    assert np.abs(P.apply(f) - xd).max() < 1e-12 * np.abs(xd).max()
    x, info = oracle_mod.gmres(M, f, P, rtol=1e-10)
    assert info["iters"] == 1


@pytest.mark.parametrize("robin", [False, True])
def test_stationary_schwarz_converges_to_direct_solve(oracle_mod, sphere02, robin):
    B, M = sphere02
    f = inputs.gaussian_vector(5, B.n_active)
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    P = oracle_mod.ORAS(B, M, 4, 2, robin=robin, exact=True)
    x = np.zeros(B.n_active)
    for _ in range(300):
        x = x + P.apply(f - M.matvec(x))
    assert np.abs(x - xd).max() < 1e-12 * np.abs(xd).max()


def test_robin_with_infinite_alpha_is_ras_bitwise(oracle_mod, torus008):
    B, M = torus008
    r = inputs.gaussian_vector(9, B.n_active)
    z0 = oracle_mod.ORAS(B, M, 8, 2).apply(r)
    z1 = oracle_mod.ORAS(B, M, 8, 2, robin=True, alpha=np.inf, alpha_cross=np.inf).apply(r)
    assert np.array_equal(z0, z1)
    z2 = oracle_mod.ORAS(B, M, 8, 2, robin=True).apply(r)
    assert not np.array_equal(z0, z2)


def test_transposed_preconditioner_is_the_adjoint(oracle_mod, torus008):
    B, M = torus008
    r = inputs.gaussian_vector(21, B.n_active)
    s = inputs.gaussian_vector(22, B.n_active)
    for robin in (False, True):
        P = oracle_mod.ORAS(B, M, 8, 2, robin=robin)
        a, b = np.dot(P.apply(r), s), np.dot(r, P.apply(s, transpose=True))
        assert abs(a - b) < 1e-12 * abs(a)


def test_canonical_local_order_breaks_ilu0(oracle_mod):
    """Reading taken for the local ILU(0) order: in canonical lexicographic
    order the factorisation meets negative pivots on the sphere at h = 0.05;
    in descending-distance order it does not."""
    B = oracle_mod.Band(0, SPH, 0.05, 3)
    M = B.M(1.0)
    neg = {}
    for order in (0, 1):
        P = oracle_mod.ORAS(B, M, 8, 2, order=order)
        neg[order] = sum(int((P.sub_factors(j).to_scipy().diagonal() < 0).sum()) for j in range(8))
    assert neg[0] > 0 and neg[1] == 0


def test_shell_order_is_shallower_and_faster(oracle_mod):
    """The distance-shell / lattice-colour local order (order 2) against the
    descending-distance order (order 1) on the torus at h = 0.025, 16 parts:
    the same nodes in each subdomain, no negative pivot, fewer dependency
    levels in both triangular sweeps and fewer GMRES iterations to 1e-8."""
    B = oracle_mod.Band(1, TOR, 0.025, 3)
    M = B.M(10.0)
    cp = B.export()[3][: B.n_active]
    f = inputs.torus_rhs(cp, inputs.torus_modes(2))
    res = {}
    for order in (1, 2):
        P = oracle_mod.ORAS(B, M, 16, 2, order=order)
        depth = max(max(P.depth(j, True), P.depth(j, False)) for j in range(16))
        neg = sum(int((P.sub_factors(j).to_scipy().diagonal() < 0).sum()) for j in range(16))
        x, info = oracle_mod.gmres(M, f, P, rtol=1e-8, maxit=2000)
        res[order] = (P, depth, neg, info)
    for j in range(16):
        assert np.array_equal(np.sort(res[1][0].sub_nodes(j)), np.sort(res[2][0].sub_nodes(j)))
    assert res[2][2] == 0 and res[1][2] == 0
    assert res[2][1] < 0.95 * res[1][1]
    assert res[2][3]["status"] == 0 and res[2][3]["iters"] < res[1][3]["iters"]


# ------------------------------------------------------------------ GMRES
@pytest.mark.parametrize("robin,exact", [(False, False), (True, False), (False, True), (True, True)])
def test_gmres_reaches_the_direct_solution(oracle_mod, torus008, sphere02, robin, exact):
    B, M = sphere02 if exact else torus008
    f = inputs.gaussian_vector(4, B.n_active)
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    P = oracle_mod.ORAS(B, M, 8, 2, robin=robin, exact=exact)
    x, info = oracle_mod.gmres(M, f, P, rtol=1e-13)
    assert info["status"] == 0
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_gmres_dense_agreement_and_restart(oracle_mod, sphere02):
    B, M = sphere02
    f = inputs.gaussian_vector(6, B.n_active)
    D = M.to_scipy().toarray()
    xd = oracle_mod.dense_solve(D, f)
    for restart in (5, 30):
        x, info = oracle_mod.gmres(M, f, None, restart=restart, rtol=1e-12)
        assert info["status"] == 0
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    x, info = oracle_mod.gmres(M, np.zeros(B.n_active))
    assert info["iters"] == 0 and not x.any()


def test_adjoint_solve(oracle_mod, sphere02):
    B, M = sphere02
    g = inputs.gaussian_vector(8, B.n_active)
    D = M.to_scipy().toarray()
    lam_d = oracle_mod.dense_solve(D, g, transpose=True)
    assert np.abs(D.T @ lam_d - g).max() < 1e-9
    P = oracle_mod.ORAS(B, M, 4, 2, robin=True)
    lam, info = oracle_mod.gmres(M.transpose(), g, P, transpose=True, rtol=1e-13)
    assert info["status"] == 0
    assert np.linalg.norm(lam - lam_d) <= 1e-10 * np.linalg.norm(lam_d)


# ------------------------------------------------------------------ two-level (coarse correction)
# The paper leaves a coarse grid correction to future releases (Section 4.1.1);
# the reading built here: coarse space Z with one constant per disjoint part,
# E0 = Z^T M Z, applied multiplicatively before the one-level apply,
# P2 = Q + P_RAS (I - M Q), Q = Z E0^{-1} Z^T.

def test_coarse_matrix_row_sums_and_entries(oracle_mod, torus008):
    """E0 = Z^T M Z: its row sums are c |part a| (M 1 = c 1), and every entry
    equals a scipy product of the indicator matrix with M."""
    B, M = torus008
    P = oracle_mod.ORAS(B, M, 13, 2, coarse=True)
    E = P.coarse_matrix()
    part = P.partition()
    sizes = np.bincount(part, minlength=13)
    assert np.allclose(E.sum(axis=1), 10.0 * sizes, rtol=1e-12, atol=1e-9)
    Z = sp.csr_matrix((np.ones(B.n_active), (np.arange(B.n_active), part)), shape=(B.n_active, 13))
    want = (Z.T @ (M.to_scipy() @ Z)).toarray()
    assert np.abs(E - want).max() <= 1e-12 * np.abs(want).max()


def test_two_level_reproduces_the_coarse_space(oracle_mod, torus008):
    """For v = Z c the coarse correction is exact and the one-level part sees
    a zero residual: P2 (M Z c) = Z c (a wrong, transposed or incomplete E0
    breaks it)."""
    B, M = torus008
    P = oracle_mod.ORAS(B, M, 13, 2, coarse=True)
    part = P.partition()
    c = inputs.gaussian_vector(71, 13)
    v = c[part]
    got = P.apply(M.matvec(v))
    assert np.abs(got - v).max() <= 1e-10 * np.abs(v).max()


def test_two_level_single_exact_subdomain_is_the_inverse(oracle_mod, sphere02):
    """N_S = 1 with an exact local solve: P_RAS = M^{-1}, so
    P2 = Q + M^{-1} (I - M Q) = M^{-1}."""
    B, M = sphere02
    P = oracle_mod.ORAS(B, M, 1, 0, exact=True, coarse=True)
    r = inputs.gaussian_vector(72, B.n_active)
    want = oracle_mod.dense_solve(M.to_scipy().toarray(), r)
    assert np.abs(P.apply(r) - want).max() <= 1e-10 * np.abs(want).max()


def test_two_level_transpose_is_the_adjoint(oracle_mod, torus008):
    B, M = torus008
    P = oracle_mod.ORAS(B, M, 13, 2, coarse=True)
    x = inputs.gaussian_vector(73, B.n_active)
    y = inputs.gaussian_vector(74, B.n_active)
    lhs, rhs = np.dot(P.apply(x), y), np.dot(x, P.apply(y, transpose=True))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.fixture(scope="module")
def torus008_direct(oracle_mod, torus008):
    B, M = torus008
    f = inputs.gaussian_vector(75, B.n_active)
    lu = sla.splu(M.to_scipy().tocsc())
    return B, M, f, lu.solve(f), lu.solve(f, trans="T")


@pytest.mark.parametrize("robin", [False, True])
def test_two_level_gmres_reaches_direct_solution_in_fewer_iterations(oracle_mod, torus008_direct, robin):
    B, M, f, xd, ld = torus008_direct
    MT = M.transpose()
    its = {}
    for coarse in (False, True):
        P = oracle_mod.ORAS(B, M, 24, 2, robin=robin, order=oracle_mod.ORAS.LOCAL_SHELLS, coarse=coarse)
        x, info = oracle_mod.gmres(M, f, P, rtol=1e-12)
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
        its[coarse] = info["iters"]
        lam, info = oracle_mod.gmres(MT, f, P, transpose=True, rtol=1e-12)
        assert np.linalg.norm(lam - ld) <= 1e-9 * np.linalg.norm(ld)
    assert its[True] < its[False], its
