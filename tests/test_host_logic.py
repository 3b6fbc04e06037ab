"""Host-side logic that needs no GPU: argument validation of the C ABI (the
calls below return before any CUDA call), the batched workload's problem
draws and the differentiable workload's initial state."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from paper_2110_06322_gb300 import inputs


@pytest.fixture(scope="module")
def lib():
    from paper_2110_06322_gb300 import build, cpm
    build.build()
    return cpm.lib()


def _msg(lib):
    return lib.cpm_last_error().decode()


def test_null_arguments_are_rejected(lib):
    from paper_2110_06322_gb300 import cpm
    c = (C.c_double * 1)(1.0)
    assert lib.cpm_apply(None, c, None, None, cpm.CPM_F64, 1, 0, None) == cpm.CPM_ERR_ARG
    assert "null" in _msg(lib)
    out = C.c_void_p()
    assert lib.oras_setup(None, None, 1.0, None, C.byref(out)) == cpm.CPM_ERR_ARG
    assert lib.cpm_dot(None, None, None, None, None) == cpm.CPM_ERR_ARG
    assert lib.cpm_imex_rhs(None, None, None, None, None, None, None) == cpm.CPM_ERR_ARG
    assert lib.cpm_imex_rhs_adjoint(None, None, None, None, None, None, None, None, None, None, None,
                                    None) == cpm.CPM_ERR_ARG


def test_batch_arguments_are_rejected(lib):
    from paper_2110_06322_gb300 import cpm
    prm = cpm.cpm_solve_params(30, 100, 1e-8, 0, 0, 1e-4, 0)
    info = (cpm.cpm_solve_info * 4)()
    bands = (C.c_void_p * 2)(None, None)
    cs = (C.c_double * 2)(1.0, 2.0)
    nr = (C.c_int32 * 2)(1, 1)
    f = C.c_void_p(16)
    u = C.c_void_p(32)
    assert lib.cpm_solve_batch(0, bands, None, cs, nr, f, u, C.byref(prm), info, 0, None) == cpm.CPM_ERR_ARG
    assert lib.cpm_solve_batch(2, bands, None, cs, nr, f, u, C.byref(prm), info, 0, None) == cpm.CPM_ERR_ARG
    assert "null band for problem 0" in _msg(lib)
    bad = cpm.cpm_solve_params(0, 100, 1e-8, 0, 0, 1e-4, 0)
    assert lib.cpm_solve_batch(2, bands, None, cs, nr, f, u, C.byref(bad), info, 0, None) == cpm.CPM_ERR_ARG
    assert "restart" in _msg(lib)


def test_batch_problem_draws():
    import bench
    hs = [0.05, 0.025, 0.0125, 0.00625]
    a = bench.draw_problems(96, hs, 4)
    b = bench.draw_problems(96, hs, 4)
    assert a == b  # seeded
    assert [p["kind"] for p in a[:4]] == [inputs.SPHERE, inputs.TORUS, inputs.SPHERE, inputs.TORUS]
    for p in a:
        prm = p["params"]
        reach = prm[3] if p["kind"] == inputs.SPHERE else min(prm[4], prm[3] - prm[4])
        assert math.sqrt(17.0) * p["h"] < 0.9 * reach  # the band stays well inside the reach
        assert 0.1 <= p["c"] <= 1000.0 and 1 <= p["nrhs"] <= 8
        if p["kind"] == inputs.SPHERE:
            assert 0.5 <= prm[3] <= 1.5
        else:
            assert 0.8 <= prm[3] <= 1.2 and 0.2 <= prm[4] <= 0.5
    assert len({round(p["h"], 6) for p in a}) >= 4


def test_bench_local_vector_placement_override():
    """The headline workload holds its Schwarz local vectors in FP16 in shared
    memory (oras_tuning.xplace 3); --xplace replaces that for any workload."""
    import bench
    try:
        assert bench.workload("torus_h0.002")["xplace"] == 3
        assert "xplace" not in bench.workload("torus_h0.004")
        args = bench.parse(["--xplace", "0"])
        bench._XPLACE = args.xplace
        assert bench.workload("torus_h0.002")["xplace"] == 0
        assert bench.workload("torus_h0.004")["xplace"] == 0
        assert bench.parse([]).xplace is None
    finally:
        bench._XPLACE = None


def test_schnakenberg_initial_state():
    import bench
    w = inputs.WORKLOADS["schnakenberg_torus_h0.005"]
    u0, v0, us, vs = bench.schnakenberg_initial_state(w, 1000)
    assert us == pytest.approx(0.703) and vs == pytest.approx(0.7 / (0.703 ** 2 + 0.06))
    du = u0 / us - 1.0
    dv = v0 / vs - 1.0
    assert np.abs(du).max() <= 0.01 and np.abs(dv).max() <= 0.01
    assert abs(du.mean()) < 2e-3 and du.std() > 4e-3  # uniform on [-1 %, 1 %]
    assert 1.0 / (w["Du"] * w["dt"]) == pytest.approx(1e5) and 1.0 / (w["Dv"] * w["dt"]) == pytest.approx(1e3)


def test_apply_wrappers_check_their_vectors(lib):
    """The binding's operator wrappers reject vectors that are not whole
    right-hand sides, a mismatched output and a shift list of the wrong
    length before anything reaches the library (checked with a fake band
    size on CPU tensors)."""
    from paper_2110_06322_gb300 import cpm
    h = C.c_void_p(0x1000)
    cpm.Band._sizes[h.value] = 10
    try:
        x = torch.zeros(20, dtype=torch.float64)
        assert cpm._apply_args(h, [1.0, 2.0], x, torch.zeros(20, dtype=torch.float64))[0] == 2
        with pytest.raises(ValueError):
            cpm._apply_args(h, 1.0, torch.zeros(15, dtype=torch.float64), torch.zeros(15, dtype=torch.float64))
        with pytest.raises(ValueError):
            cpm._apply_args(h, [1.0], x, torch.zeros(20, dtype=torch.float64))
        with pytest.raises(ValueError):
            cpm._apply_args(h, 1.0, x, torch.zeros(20, dtype=torch.float32))
        with pytest.raises(ValueError):
            cpm._apply_args(h, 1.0, x, torch.zeros(10, dtype=torch.float64))
    finally:
        cpm.Band._sizes.pop(h.value)


def test_tuning_arguments_are_rejected(lib):
    from paper_2110_06322_gb300 import cpm
    t = cpm.oras_tuning(0, 0, 0, 0, 0, 0)
    assert lib.oras_set_tuning(None, C.byref(t)) == cpm.CPM_ERR_ARG
    assert lib.oras_get_tuning(None, C.byref(t)) == cpm.CPM_ERR_ARG
    assert lib.oras_autotune(None, cpm.CPM_F32, 3, None, None, None) == cpm.CPM_ERR_ARG
    assert lib.cpm_device_allocations() >= 0
