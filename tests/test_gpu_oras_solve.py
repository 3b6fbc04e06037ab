"""GPU parity: Schwarz preconditioner and GMRES solver vs the FP64 oracle.

Partition and subdomain lists (in their local order) are integer data and
must be identical.  The preconditioner apply uses the same ILU(0) factors in
the same local order; only the summation order inside each row differs, so
FP64 agreement is required to 1e-12 relative (the triangular solves amplify
rounding by their growth, which stays below 1e3 on these bands).  Solutions:
FP64 solves agree with the oracle's direct solve to 1e-10 relative (both
sides at rtol 1e-13, Section 4.1.1 GMRES); the mixed-precision solve must
reach 1e-8 relative error.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla
import torch

from paper_2110_06322_gb300 import inputs

pytestmark = pytest.mark.gpu

SPH = (0.0, 0.0, 0.0, 1.0)
TOR = (0.0, 0.0, 0.0, 1.0, 0.4)


@pytest.fixture(scope="module")
def cpm():
    from paper_2110_06322_gb300 import cpm as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def torus005(cpm, oracle_mod):
    B = cpm.Band(1, TOR, 0.05, 3)
    O = oracle_mod.Band(1, TOR, 0.05, 3)
    return B, O, O.M(10.0)


@pytest.fixture(scope="module")
def torus005_lu(torus005):
    """Sparse LU of the oracle's M (library factorisation), shared by the tests."""
    return sla.splu(torus005[2].to_scipy().tocsc())


@pytest.fixture(scope="module")
def sphere01(cpm, oracle_mod):
    B = cpm.Band(0, SPH, 0.1, 3)
    O = oracle_mod.Band(0, SPH, 0.1, 3)
    return B, O, O.M(1.0)


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("nparts,overlap", [(1, 0), (8, 2), (13, 1), (64, 2), (64, 3)])
def test_partition_and_local_order_identical(cpm, oracle_mod, torus005, nparts, overlap, order):
    B, O, M = torus005
    P = cpm.Schwarz(B, 10.0, nparts, overlap, order=order)
    OP = oracle_mod.ORAS(O, M, nparts, overlap, order=order)
    part, sptr, nodes = [t.cpu().numpy() for t in P.export()]
    assert np.array_equal(part, OP.partition())
    for j in range(nparts):
        assert np.array_equal(nodes[sptr[j]:sptr[j + 1]], OP.sub_nodes(j))


@pytest.mark.parametrize("robin", [False, True])
def test_schwarz_apply_matches_oracle(cpm, oracle_mod, torus005, robin):
    B, O, M = torus005
    P = cpm.Schwarz(B, 10.0, 16, 2, robin=robin)  # default local order: shells and colours for p = 3
    OP = oracle_mod.ORAS(O, M, 16, 2, robin=robin, order=oracle_mod.ORAS.LOCAL_SHELLS)
    r = inputs.gaussian_vector(5, B.n_active)
    want = OP.apply(r)
    got = P.apply(_cuda(r)).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    got32 = P.apply(_cuda(r).float()).double().cpu().numpy()
    assert np.abs(got32 - want).max() <= 1e-4 * np.abs(want).max()
    wantT = OP.apply(r, transpose=True)
    gotT = P.apply(_cuda(r), transpose=True).cpu().numpy()
    assert np.abs(gotT - wantT).max() <= 1e-12 * np.abs(wantT).max()


def test_schwarz_several_rhs(cpm, oracle_mod, sphere01):
    B, O, M = sphere01
    P = cpm.Schwarz(B, 1.0, 8, 2, robin=True)
    OP = oracle_mod.ORAS(O, M, 8, 2, robin=True, order=oracle_mod.ORAS.LOCAL_SHELLS)
    R = np.stack([inputs.gaussian_vector(60 + q, B.n_active) for q in range(3)])
    Z = P.apply(_cuda(R).reshape(-1)).cpu().numpy().reshape(3, -1)
    for q in range(3):
        want = OP.apply(R[q])
        assert np.abs(Z[q] - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("robin", [False, True])
def test_fp64_solve_matches_direct_solve(cpm, oracle_mod, torus005, torus005_lu, robin):
    B, O, M = torus005
    f = inputs.gaussian_vector(4, B.n_active)
    xd = torus005_lu.solve(f)
    P = cpm.Schwarz(B, 10.0, 16, 2, robin=robin)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-13, maxit=5000)
    assert info["status"] == 0, info
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)
    # the oracle's own GMRES with the same preconditioner reaches the same u
    xo, oinfo = oracle_mod.gmres(M, f, oracle_mod.ORAS(O, M, 16, 2, robin=robin), rtol=1e-13)
    assert np.linalg.norm(u.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)


@pytest.mark.parametrize("reorth", [0, 1, 2])
def test_gram_schmidt_variants_reach_same_solution(cpm, oracle_mod, torus005, torus005_lu, reorth):
    """One classical pass, a conditional second pass and two passes: the same
    solution to 1e-10 (FP64, rtol 1e-12) and to 1e-8 in mixed precision."""
    B, O, M = torus005
    f = inputs.gaussian_vector(11, B.n_active)
    xd = torus005_lu.solve(f)
    P = cpm.Schwarz(B, 10.0, 16, 2, store=cpm.CPM_F32)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-12, maxit=5000, reorth=reorth)
    assert info["status"] == 0, info
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-10, maxit=5000, reorth=reorth, mixed=True)
    assert info["status"] == 0, info
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


def test_wide_basis_chunked_gram_schmidt(cpm, oracle_mod, sphere01):
    """Restart 40 without a preconditioner (full cycles of 40 iterations, a
    basis wider than one Gram-Schmidt kernel's 32 vectors): the chunked passes
    reach the direct solution."""
    B, O, M = sphere01
    f = inputs.gaussian_vector(12, B.n_active)
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    for reorth in (0, 2):
        u, info = cpm.solve(B, _cuda(f), None, c=1.0, rtol=1e-12, restart=40, maxit=20000, reorth=reorth)
        assert info["status"] == 0 and info["iters"] > 40, info
        assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)


def test_mixed_precision_solve_reaches_1e8(cpm, oracle_mod, torus005, torus005_lu):
    B, O, M = torus005
    f = inputs.gaussian_vector(7, B.n_active)
    xd = torus005_lu.solve(f)
    for store in (cpm.CPM_F32, cpm.CPM_BF16):
        P = cpm.Schwarz(B, 10.0, 16, 2, robin=True, store=store)
        u, info = cpm.solve(B, _cuda(f), P, rtol=1e-10, mixed=True, maxit=5000)
        assert info["status"] == 0 and info["ir_steps"] >= 1, info
        assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)


def test_sphere_harmonic_solution(cpm, oracle_mod, sphere01):
    B, O, M = sphere01
    cp = B.export()[3][: B.n_active].cpu().numpy()
    f = 13.0 * inputs.y32(cp)
    P = cpm.Schwarz(B, 1.0, 8, 2)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-13)
    assert info["status"] == 0
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)


def test_adjoint_solve(cpm, oracle_mod, torus005, torus005_lu):
    B, O, M = torus005
    g = inputs.gaussian_vector(8, B.n_active)
    lam_d = torus005_lu.solve(g, trans="T")
    for robin in (False, True):
        P = cpm.Schwarz(B, 10.0, 16, 2, robin=robin)
        lam, info = cpm.solve(B, _cuda(g), P, rtol=1e-13, adjoint=True, maxit=5000)
        assert info["status"] == 0, info
        assert np.linalg.norm(lam.cpu().numpy() - lam_d) <= 1e-10 * np.linalg.norm(lam_d)


def test_unpreconditioned_and_edge_cases(cpm, oracle_mod, sphere01):
    B, O, M = sphere01
    f = inputs.gaussian_vector(9, B.n_active)
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    u, info = cpm.solve(B, _cuda(f), None, c=1.0, rtol=1e-12, maxit=20000)
    assert info["status"] == 0
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    # zero right-hand side
    u, info = cpm.solve(B, torch.zeros(B.n_active, dtype=torch.float64, device="cuda"), None, c=1.0)
    assert info["status"] == 0 and info["iters"] == 0 and u.abs().max().item() == 0.0
    # iteration limit
    P = cpm.Schwarz(B, 1.0, 8, 2)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-12, maxit=3)
    assert info["status"] == cpm.CPM_ERR_NOT_CONVERGED and info["iters"] == 3
    # NaN in the right-hand side is reported, not propagated silently
    fn = f.copy()
    fn[17] = np.nan
    with pytest.raises(cpm.CpmError) as e:
        cpm.solve(B, _cuda(fn), P, rtol=1e-8)
    assert e.value.status == cpm.CPM_ERR_NAN
    # more parts than some boxes can fill: empty subdomains are harmless
    P2 = cpm.Schwarz(B, 1.0, 1000, 1)
    u, info = cpm.solve(B, _cuda(f), P2, rtol=1e-12, maxit=5000)
    assert info["status"] == 0


def test_full_size_torus_solve(cpm, oracle_mod):
    """Torus h = 0.004 (5.7M band points), 512 parts, overlap 2, RAS with
    ILU(0), GMRES(30): the FP64 solve at rtol 1e-8 and the mixed-precision
    solve at rtol 1e-10.  The true residual of the mixed solution is checked on
    sampled rows assembled by the oracle (|r_i| <= |r|_2 <= 1e-10 |f|_2), and
    the two solutions against each other."""
    h, c = 0.004, 10.0
    B = cpm.Band(1, TOR, h, 3)
    cp = B.export()[3][: B.n_active].cpu().numpy()
    f = inputs.torus_rhs(cp, inputs.torus_modes(2))
    P = cpm.Schwarz(B, c, 512, 2)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-8, maxit=20000)
    assert info["status"] == 0, info
    u32, info32 = cpm.solve(B, _cuda(f), P, rtol=1e-10, mixed=True, maxit=20000)
    assert info32["status"] == 0, info32
    un, u32n = u.cpu().numpy(), u32.cpu().numpy()
    O = oracle_mod.Band(1, TOR, h, 3)
    rows = np.random.default_rng(1).integers(0, B.n_active, 2000)
    res = O.apply_rows(c, u32n, rows) - f[rows]
    assert np.abs(res).max() <= 2e-10 * np.linalg.norm(f)
    assert np.linalg.norm(un - u32n) <= 1e-6 * np.linalg.norm(u32n)


@pytest.fixture(scope="module")
def torus0025(cpm, oracle_mod):
    """Torus h = 0.025 in 4 parts: subdomains of ~38k rows whose local vectors
    do not fit in shared memory (FP64 or FP32), about 175 rows per
    dependency level, so every level spans several factor chunks."""
    B = cpm.Band(1, TOR, 0.025, 3)
    O = oracle_mod.Band(1, TOR, 0.025, 3)
    M = O.M(10.0)
    return B, O, M, oracle_mod.ORAS(O, M, 4, 2, order=oracle_mod.ORAS.LOCAL_SHELLS)


def _rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


# BF16 factor storage rounds every stored factor entry to 8 significant bits
# (relative error <= 2^-9); through the two triangular sweeps of ~60-entry rows
# this bounds the apply's error at a few 1e-3 of max|z| on these bands; 2e-2
# leaves a margin while still failing any wrong entry, level or row.
BF16_TOL = 2e-2


@pytest.mark.parametrize("robin", [False, True])
def test_schwarz_global_slice_branch_matches_oracle(cpm, oracle_mod, torus005, robin):
    """The apply with every local vector in a global-memory slice (the branch
    large subdomains take), forced on the small torus: FP64, FP32 and BF16
    factors, forward and transposed, RAS and the Robin reading."""
    B, O, M = torus005
    OP = oracle_mod.ORAS(O, M, 16, 2, robin=robin, order=oracle_mod.ORAS.LOCAL_SHELLS)
    r = inputs.gaussian_vector(15, B.n_active)
    want, wantT = OP.apply(r), OP.apply(r, transpose=True)
    for store in (cpm.CPM_F32, cpm.CPM_BF16):
        P = cpm.Schwarz(B, 10.0, 16, 2, robin=robin, store=store)
        P.set_tuning(xplace=1)
        assert _rel(P.apply(_cuda(r)).cpu().numpy(), want) <= 1e-12
        assert _rel(P.apply(_cuda(r), transpose=True).cpu().numpy(), wantT) <= 1e-12
        got32 = P.apply(_cuda(r).float()).double().cpu().numpy()
        assert _rel(got32, want) <= (1e-4 if store == cpm.CPM_F32 else BF16_TOL)
        gotT32 = P.apply(_cuda(r).float(), transpose=True).double().cpu().numpy()
        assert _rel(gotT32, wantT) <= 1e-4
        # the same preconditioner with the shared-memory branch gives the same values
        P.set_tuning(xplace=0)
        assert _rel(P.apply(_cuda(r)).cpu().numpy(), want) <= 1e-12


@pytest.mark.parametrize("lanes", [4, 8, 16])
@pytest.mark.parametrize("xplace", [0, 1])
def test_schwarz_kernel_variants_match_oracle(cpm, oracle_mod, torus005, lanes, xplace):
    """Every lanes-per-row variant, in both local-vector placements and both
    subdomain schedules, against the oracle (FP64 1e-12, FP32 1e-4, forward
    and transposed)."""
    B, O, M = torus005
    OP = oracle_mod.ORAS(O, M, 16, 2, order=oracle_mod.ORAS.LOCAL_SHELLS)
    r = inputs.gaussian_vector(18, B.n_active)
    want, wantT = OP.apply(r), OP.apply(r, transpose=True)
    P = cpm.Schwarz(B, 10.0, 16, 2, store=cpm.CPM_F32)
    for schedule, ctas in ((0, 2), (1, 1), (0, 4)):
        P.set_tuning(xplace=xplace, lanes=lanes, schedule=schedule, ctas=ctas)
        assert P.tuning()["lanes"] == lanes
        assert _rel(P.apply(_cuda(r)).cpu().numpy(), want) <= 1e-12
        assert _rel(P.apply(_cuda(r), transpose=True).cpu().numpy(), wantT) <= 1e-12
        assert _rel(P.apply(_cuda(r).float()).double().cpu().numpy(), want) <= 1e-4


def test_schwarz_autotune_keeps_a_valid_setting(cpm, oracle_mod, torus005):
    B, O, M = torus005
    P = cpm.Schwarz(B, 10.0, 16, 2, store=cpm.CPM_F32)
    best, ms = P.autotune(cpm.CPM_F32, reps=2)
    assert ms > 0 and best["lanes"] in (4, 8, 16) and best["schedule"] in (0, 1) and best["probe_timeout"] == 0
    assert P.tuning() == best
    OP = oracle_mod.ORAS(O, M, 16, 2, order=oracle_mod.ORAS.LOCAL_SHELLS)
    r = inputs.gaussian_vector(19, B.n_active)
    assert _rel(P.apply(_cuda(r).float()).double().cpu().numpy(), OP.apply(r)) <= 1e-4


def test_schwarz_large_subdomains_multichunk_levels(cpm, oracle_mod, torus0025):
    """~38k-row subdomains (global-slice branch chosen by size, levels of
    several chunks): element-wise against the oracle in FP64 and FP32,
    forward and transposed, with two right-hand sides."""
    B, O, M, OP = torus0025
    P = cpm.Schwarz(B, 10.0, 4, 2, store=cpm.CPM_F32)
    part, sptr, nodes = [t.cpu().numpy() for t in P.export()]
    assert np.array_equal(part, OP.partition())
    for j in range(4):
        assert np.array_equal(nodes[sptr[j]:sptr[j + 1]], OP.sub_nodes(j))
    R = np.stack([inputs.gaussian_vector(20 + q, B.n_active) for q in range(2)])
    Z = P.apply(_cuda(R).reshape(-1)).cpu().numpy().reshape(2, -1)
    ZT = P.apply(_cuda(R).reshape(-1), transpose=True).cpu().numpy().reshape(2, -1)
    Z32 = P.apply(_cuda(R).reshape(-1).float()).double().cpu().numpy().reshape(2, -1)
    for q in range(2):
        want = OP.apply(R[q])
        assert _rel(Z[q], want) <= 1e-12
        assert _rel(Z32[q], want) <= 1e-4
        assert _rel(ZT[q], OP.apply(R[q], transpose=True)) <= 1e-12


# FP16 local vector (xplace 2 and 3): every stored sweep value is rounded to 11
# significant bits (relative error <= 2^-11) after a power-of-two scaling that
# keeps it in FP16's normal range; the sweeps' growth (below 3 on these bands)
# and ~60-entry rows bound the apply's error at a few 1e-3 of max|z|.  1e-2
# fails any wrong entry, level, scale or row (those give errors of order 1).
HALF_TOL = 1e-2


@pytest.mark.parametrize("xplace", [2, 3])
def test_schwarz_half_local_vector_matches_oracle(cpm, oracle_mod, torus0025, xplace):
    """~38k-row subdomains with an FP16 local vector in shared memory (FP32 and
    BF16 factors, forward and transposed, two right-hand sides) against the
    oracle; FP64 applies ignore the setting."""
    B, O, M, OP = torus0025
    R = np.stack([inputs.gaussian_vector(40 + q, B.n_active) for q in range(2)])
    # one right-hand side scaled far down: the per-subdomain power-of-two scale
    # must bring it back into FP16's range
    R[1] *= 1e-9
    want = [OP.apply(R[q]) for q in range(2)]
    wantT = [OP.apply(R[q], transpose=True) for q in range(2)]
    for store, tol in ((cpm.CPM_F32, HALF_TOL), (cpm.CPM_BF16, BF16_TOL + HALF_TOL)):
        P = cpm.Schwarz(B, 10.0, 4, 2, store=store)
        P.set_tuning(xplace=xplace)
        Z = P.apply(_cuda(R).reshape(-1).float()).double().cpu().numpy().reshape(2, -1)
        ZT = P.apply(_cuda(R).reshape(-1).float(), transpose=True).double().cpu().numpy().reshape(2, -1)
        for q in range(2):
            assert np.all(np.isfinite(Z[q])) and np.all(np.isfinite(ZT[q]))
            assert _rel(Z[q], want[q]) <= tol
            assert _rel(ZT[q], wantT[q]) <= tol
        Z64 = P.apply(_cuda(R[0])).cpu().numpy()
        assert _rel(Z64, want[0]) <= 1e-12


def test_mixed_solve_with_half_local_vector(cpm, oracle_mod, torus0025):
    """The flexible mixed-precision solve with the FP16 local vector reaches
    the same tolerance as with the FP32 one, in at most a few more
    iterations, and its solution satisfies sampled rows of the oracle's M."""
    B, O, M, OP = torus0025
    f = inputs.gaussian_vector(44, B.n_active)
    P = cpm.Schwarz(B, 10.0, 4, 2, store=cpm.CPM_F32)
    u32, i32 = cpm.solve(B, _cuda(f), P, rtol=1e-9, mixed=True, maxit=5000)
    P.set_tuning(xplace=2)
    u16, i16 = cpm.solve(B, _cuda(f), P, rtol=1e-9, mixed=True, maxit=5000)
    assert i32["status"] == 0 and i16["status"] == 0
    assert i16["rel_residual"] <= 1e-9
    assert i16["iters"] <= 1.1 * i32["iters"] + 3
    un = u16.cpu().numpy()
    rows = np.arange(0, B.n_active, 97)
    res = O.apply_rows(10.0, un, rows) - f[rows]
    assert np.abs(res).max() <= 1e-8 * np.linalg.norm(f)
    assert np.linalg.norm(un - u32.cpu().numpy()) <= 1e-6 * np.linalg.norm(un)


def test_schwarz_timeout_is_reported_and_recovers(cpm, oracle_mod, torus005, torus005_lu):
    """Failure path of the bounded waits, without a GPU fault: with the probe
    on, the first chunk wait of every subdomain waits on a barrier nothing
    completes and runs out after 1,000 polls; each CTA drains the copies it
    issued and returns, and the solve reports CPM_ERR_TIMEOUT.  With the
    probe off the same handles solve to the direct solution."""
    B, O, M = torus005
    f = inputs.gaussian_vector(16, B.n_active)
    P = cpm.Schwarz(B, 10.0, 16, 2, store=cpm.CPM_F32)
    for mixed in (False, True):
        P.set_tuning(probe_timeout=1, wait_polls=1000)
        with pytest.raises(cpm.CpmError) as e:
            cpm.solve(B, _cuda(f), P, rtol=1e-10, maxit=200, mixed=mixed)
        assert e.value.status == cpm.CPM_ERR_TIMEOUT
        P.set_tuning()
        u, info = cpm.solve(B, _cuda(f), P, rtol=1e-12, maxit=5000, mixed=mixed)
        assert info["status"] == 0, info
        xd = torus005_lu.solve(f)
        assert np.linalg.norm(u.cpu().numpy() - xd) <= (1e-10 if not mixed else 1e-8) * np.linalg.norm(xd)


@pytest.mark.parametrize("nparts,overlap", [(16, 2), (64, 2)])
def test_shell_colour_order_matches_oracle(cpm, oracle_mod, torus005, nparts, overlap):
    """The second local order (distance shells of width h, then lattice-parity
    colours): subdomain lists identical to the oracle's order 2, and the
    Schwarz apply with its factors element-wise equal (FP64 1e-12, FP32 1e-4),
    forward and transposed."""
    B, O, M = torus005
    P = cpm.Schwarz(B, 10.0, nparts, overlap, order=2)
    OP = oracle_mod.ORAS(O, M, nparts, overlap, order=oracle_mod.ORAS.LOCAL_SHELLS)
    part, sptr, nodes = [t.cpu().numpy() for t in P.export()]
    assert np.array_equal(part, OP.partition())
    for j in range(nparts):
        assert np.array_equal(nodes[sptr[j]:sptr[j + 1]], OP.sub_nodes(j))
    assert P.max_levels == max(max(OP.depth(j, True), OP.depth(j, False)) for j in range(nparts))
    r = inputs.gaussian_vector(17, B.n_active)
    want = OP.apply(r)
    assert _rel(P.apply(_cuda(r)).cpu().numpy(), want) <= 1e-12
    assert _rel(P.apply(_cuda(r).float()).double().cpu().numpy(), want) <= 1e-4
    assert _rel(P.apply(_cuda(r), transpose=True).cpu().numpy(), OP.apply(r, transpose=True)) <= 1e-12


@pytest.fixture(scope="module")
def torus005_p2(cpm, oracle_mod):
    """Tri-quadratic interpolation (p = 2, 27-point cubes), the degree of the
    paper's scaling runs (Section 5)."""
    B = cpm.Band(1, TOR, 0.05, 2)
    O = oracle_mod.Band(1, TOR, 0.05, 2)
    M = O.M(10.0)
    return B, O, M, sla.splu(M.to_scipy().tocsc())


@pytest.mark.parametrize("robin", [False, True])
def test_p2_schwarz_apply_matches_oracle(cpm, oracle_mod, torus005_p2, robin):
    B, O, M, _ = torus005_p2
    P = cpm.Schwarz(B, 10.0, 16, 2, robin=robin)
    OP = oracle_mod.ORAS(O, M, 16, 2, robin=robin)
    part, sptr, nodes = [t.cpu().numpy() for t in P.export()]
    assert np.array_equal(part, OP.partition())
    for j in range(16):
        assert np.array_equal(nodes[sptr[j]:sptr[j + 1]], OP.sub_nodes(j))
    r = inputs.gaussian_vector(31, B.n_active)
    want = OP.apply(r)
    assert _rel(P.apply(_cuda(r)).cpu().numpy(), want) <= 1e-12
    assert _rel(P.apply(_cuda(r).float()).double().cpu().numpy(), want) <= 1e-4
    assert _rel(P.apply(_cuda(r), transpose=True).cpu().numpy(), OP.apply(r, transpose=True)) <= 1e-12


def test_p2_solves_match_direct_solve(cpm, oracle_mod, torus005_p2):
    """p = 2: FP64 and mixed-precision forward solves and the FP64 adjoint
    solve against the sparse LU of the oracle's M."""
    B, O, M, lu = torus005_p2
    f = inputs.gaussian_vector(32, B.n_active)
    xd = lu.solve(f)
    P = cpm.Schwarz(B, 10.0, 16, 2, store=cpm.CPM_F32)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-13, maxit=5000)
    assert info["status"] == 0, info
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-10, maxit=5000, mixed=True)
    assert info["status"] == 0, info
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
    lam, info = cpm.solve(B, _cuda(f), P, rtol=1e-13, maxit=5000, adjoint=True)
    assert info["status"] == 0, info
    ld = lu.solve(f, trans="T")
    assert np.linalg.norm(lam.cpu().numpy() - ld) <= 1e-10 * np.linalg.norm(ld)


# ------------------------------------------------------------------ two-level (coarse correction)
@pytest.mark.parametrize("robin", [False, True])
def test_two_level_apply_matches_oracle(cpm, oracle_mod, torus005, robin):
    """Coarse correction on one constant per disjoint part, then the
    one-level apply (the oracle's two-level variant): FP64 forward and
    transposed to 1e-12, FP32 forward to 1e-4, two right-hand sides."""
    B, O, M = torus005
    P = cpm.Schwarz(B, 10.0, 16, 2, robin=robin, coarse=True)
    OP = oracle_mod.ORAS(O, M, 16, 2, robin=robin, order=oracle_mod.ORAS.LOCAL_SHELLS, coarse=True)
    R = np.stack([inputs.gaussian_vector(80 + q, B.n_active) for q in range(2)])
    Z = P.apply(_cuda(R).reshape(-1)).cpu().numpy().reshape(2, -1)
    ZT = P.apply(_cuda(R).reshape(-1), transpose=True).cpu().numpy().reshape(2, -1)
    Z32 = P.apply(_cuda(R).reshape(-1).float()).double().cpu().numpy().reshape(2, -1)
    for q in range(2):
        want = OP.apply(R[q])
        assert _rel(Z[q], want) <= 1e-12
        assert _rel(Z32[q], want) <= 1e-4
        assert _rel(ZT[q], OP.apply(R[q], transpose=True)) <= 1e-12


def test_two_level_solves_match_direct_solve_in_fewer_iterations(cpm, oracle_mod, torus005, torus005_lu):
    B, O, M = torus005
    f = inputs.gaussian_vector(85, B.n_active)
    xd = torus005_lu.solve(f)
    iters = {}
    for coarse in (False, True):
        P = cpm.Schwarz(B, 10.0, 32, 2, coarse=coarse)
        u, info = cpm.solve(B, _cuda(f), P, rtol=1e-13, maxit=5000)
        assert info["status"] == 0, info
        assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)
        iters[coarse] = info["iters"]
        u, info = cpm.solve(B, _cuda(f), P, rtol=1e-10, maxit=5000, mixed=True)
        assert info["status"] == 0, info
        assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-8 * np.linalg.norm(xd)
        lam, info = cpm.solve(B, _cuda(f), P, rtol=1e-13, maxit=5000, adjoint=True)
        assert info["status"] == 0, info
        ld = torus005_lu.solve(f, trans="T")
        assert np.linalg.norm(lam.cpu().numpy() - ld) <= 1e-10 * np.linalg.norm(ld)
    assert iters[True] < iters[False], iters


def test_two_level_small_shift_matches_oracle(cpm, oracle_mod):
    """A small shift (c = 0.337) on a thinner torus in 12 parts.  The coarse
    step solves for q of size |r| / c on the coarse space and forms r - M q,
    which cancels to ~c / |M| of its terms, so the apply's rounding grows with
    |M|_inf / c: the 1e-12 (FP64) and 1e-4 (FP32) bounds of the c = 10 tests,
    where |M|_inf / c ~ 600, are scaled by (|M|_inf / c) / 600 (~120 here).
    The GPU solves converge in about the oracle's iteration count (FP64) or a
    few times it at most (the flexible mixed solve)."""
    tor = (0.0, 0.0, 0.0, 1.1327777047085716, 0.3907496930152238)
    c = 0.33743553695361456
    B = cpm.Band(1, tor, 0.025, 3)
    O = oracle_mod.Band(1, tor, 0.025, 3)
    M = O.M(c)
    amp = max(1.0, float(np.abs(M.to_scipy()).sum(axis=1).max()) / c / 600.0)
    P = cpm.Schwarz(B, c, 12, 2, coarse=True)
    OP = oracle_mod.ORAS(O, M, 12, 2, order=oracle_mod.ORAS.LOCAL_SHELLS, coarse=True)
    r = inputs.gaussian_vector(88, B.n_active)
    want = OP.apply(r)
    assert _rel(P.apply(_cuda(r)).cpu().numpy(), want) <= 1e-12 * amp
    assert _rel(P.apply(_cuda(r).float()).double().cpu().numpy(), want) <= 1e-4 * amp
    f = inputs.gaussian_vector(4015, B.n_active)
    _, oinfo = oracle_mod.gmres(M, f, OP, restart=30, maxit=3000, rtol=1e-8)
    assert oinfo["status"] == 0, oinfo
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-8, maxit=3000, mixed=False)
    assert info["status"] == 0 and info["iters"] <= 1.2 * oinfo["iters"] + 5, (info, oinfo)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-8, maxit=3000, mixed=True)
    assert info["status"] == 0 and info["iters"] <= 3 * oinfo["iters"] + 10, (info, oinfo)


def test_two_level_with_empty_parts(cpm, oracle_mod, sphere01):
    """More parts than the band can fill: empty parts get a decoupled unit
    row in Z^T M Z and the solve is unaffected."""
    B, O, M = sphere01
    f = inputs.gaussian_vector(86, B.n_active)
    xd = sla.spsolve(M.to_scipy().tocsc(), f)
    P = cpm.Schwarz(B, 1.0, 1000, 1, coarse=True)
    u, info = cpm.solve(B, _cuda(f), P, rtol=1e-12, maxit=5000)
    assert info["status"] == 0, info
    assert np.linalg.norm(u.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)
