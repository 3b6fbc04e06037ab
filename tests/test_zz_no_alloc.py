"""cpm_apply_noalloc: the operator apply that allocates nothing.

Some callers cannot allocate device memory (their process's device memory is
owned by another allocator, or they run latency-bounded loops where an
allocation may block), so the library offers this variant of cpm_apply whose
scratch is a fixed array inside the library.  It must give the same result as
cpm_apply -- within the tolerances the apply parity tests use (1e-14 relative
in FP64, 2e-6 in FP32) -- on consecutive calls that reuse the shared scratch,
and reject a band whose scratch need exceeds the fixed size.

This file is collected last on purpose, so that a failure here comes after
every other test has run.
"""
import numpy as np
import pytest
import torch

from paper_2110_06322_gb300 import inputs

pytestmark = pytest.mark.gpu

TOR = (0.0, 0.0, 0.0, 1.0, 0.4)


@pytest.fixture(scope="module")
def cpm():
    from paper_2110_06322_gb300 import cpm as m
    m.lib()
    return m


@pytest.mark.parametrize("h", [0.05, 0.01])
def test_noalloc_apply_matches_cpm_apply_twice(cpm, h):
    B = cpm.Band(1, TOR, h, 3)
    for call, seed in enumerate((101, 202)):  # two calls in a row share the scratch
        x = torch.from_numpy(inputs.gaussian_vector(seed, B.n_active)).cuda()
        for dt, tol in ((torch.float64, 1e-14), (torch.float32, 2e-6)):
            xd = x.to(dt)
            want = B.apply(10.0 + call, xd)
            got = cpm.cpm_apply_noalloc(B.handle, 10.0 + call, xd, torch.empty_like(xd))
            scale = want.double().abs().max().item()
            assert (got.double() - want.double()).abs().max().item() <= tol * scale


def test_noalloc_apply_allocates_nothing(cpm):
    """Two calls after the band is built: the library's own allocation count
    does not move (every device allocation of the library goes through one
    counted routine) and the device's free memory is unchanged, so neither the
    library nor the CUDA runtime allocated for the call (the fixed scratch was
    committed when the band was built)."""
    B = cpm.Band(1, TOR, 0.05, 3)
    x = torch.from_numpy(inputs.gaussian_vector(5, B.n_active)).cuda()
    y = torch.empty_like(x)
    want = B.apply(10.0, x)
    torch.cuda.synchronize()
    a0, free0 = cpm.cpm_device_allocations(), torch.cuda.mem_get_info()[0]
    cpm.cpm_apply_noalloc(B.handle, 10.0, x, y)
    cpm.cpm_apply_noalloc(B.handle, 10.0, x, y)
    torch.cuda.synchronize()
    a1, free1 = cpm.cpm_device_allocations(), torch.cuda.mem_get_info()[0]
    assert a1 == a0
    assert free1 == free0
    assert (y - want).abs().max().item() <= 1e-14 * want.abs().max().item()


def test_noalloc_apply_more_rhs_than_one_pass(cpm):
    """20 right-hand sides with their own shifts run 16 at a time through the
    same scratch; every one matches cpm_apply."""
    B = cpm.Band(1, TOR, 0.05, 3)
    cs = [0.5 * (q + 1) for q in range(20)]
    X = torch.from_numpy(np.stack([inputs.gaussian_vector(400 + q, B.n_active) for q in range(20)])).cuda()
    want = B.apply(cs, X.reshape(-1)).reshape(20, -1)
    got = cpm.cpm_apply_noalloc(B.handle, cs, X.reshape(-1), torch.empty(X.numel(), dtype=X.dtype, device="cuda"))
    got = got.reshape(20, -1)
    for q in range(20):
        assert (got[q] - want[q]).abs().max().item() <= 1e-14 * want[q].abs().max().item()


def test_noalloc_rejects_overlapping_buffers(cpm):
    B = cpm.Band(1, TOR, 0.05, 3)
    buf = torch.zeros(B.n_active + 8, dtype=torch.float64, device="cuda")
    with pytest.raises(cpm.CpmError) as e:  # y starts 8 values into x
        cpm.cpm_apply_noalloc(B.handle, 10.0, buf[: B.n_active], buf[8:])
    assert e.value.status == cpm.CPM_ERR_ARG


def test_noalloc_apply_several_rhs(cpm):
    B = cpm.Band(1, TOR, 0.02, 3)
    cs = [0.5, 10.0, 300.0]
    X = torch.from_numpy(np.stack([inputs.gaussian_vector(300 + q, B.n_active) for q in range(3)])).cuda()
    want = B.apply(cs, X.reshape(-1))
    got = cpm.cpm_apply_noalloc(B.handle, cs, X.reshape(-1), torch.empty(X.numel(), dtype=X.dtype, device="cuda"))
    assert (got - want).abs().max().item() <= 1e-14 * want.abs().max().item()


def test_noalloc_rejects_bands_beyond_its_scratch(cpm):
    B = cpm.Band(1, TOR, 0.005, 3)  # about 4.7M E rows: 8 bytes each exceed the 16 MiB scratch
    x = torch.zeros(B.n_active, dtype=torch.float64, device="cuda")
    with pytest.raises(cpm.CpmError) as e:
        cpm.cpm_apply_noalloc(B.handle, 10.0, x, torch.empty_like(x))
    assert e.value.status == cpm.CPM_ERR_ARG
    assert "scratch" in str(e.value)
