"""The allocation-free residual check (hz_residual_noalloc) against hz_residual.

Callers that cannot allocate device memory when they check a solution
(allocation-free serving or real-time loops, frameworks that own all device memory)
use hz_residual_noalloc, whose scratch is a fixed array inside the library.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1909_01299_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01299_gb300 import build
    build.build()
    from paper_1909_01299_gb300 import hz
    return torch, hz


def test_noalloc_residual_matches_residual_on_two_calls(env):
    torch, hz = env
    w = W.tiny_pml(40, 36, 24, 2, 2, rim=5, pml=2, nrhs=3)
    plan = hz.Plan.from_workload(w)
    f = torch.from_numpy(w.f).cuda()
    u_exact = plan.solve(f)
    rng = np.random.default_rng(9)
    # two different (f, u) pairs in a row: the second call must not see the first's scratch
    u_pert = u_exact + torch.from_numpy(1e-6 * rng.standard_normal(w.f.shape) + 0j).cuda()
    f2 = torch.from_numpy(np.ascontiguousarray(w.f[:2] * 3.0)).cuda()
    u2 = plan.solve(f2) + torch.from_numpy(1e-3 * rng.standard_normal(w.f[:2].shape) + 0j).cuda()
    for ff, uu in ((f, u_pert), (f2, u2)):
        ref = plan.residual(ff, uu)
        got = hz.residual_noalloc(plan, ff, uu)
        assert got.shape == ref.shape
        assert np.allclose(got, ref, rtol=1e-10, atol=0.0), (got, ref)


def test_noalloc_residual_allocates_nothing_and_rejects_oversize(env):
    torch, hz = env
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=2)
    plan = hz.Plan.from_workload(w)
    f = torch.from_numpy(w.f).cuda()
    u = plan.solve(f)
    hz.residual_noalloc(plan, f, u)                 # first call on this device: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    r1 = hz.residual_noalloc(plan, f, u)
    r2 = hz.residual_noalloc(plan, f, u)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(r1, r2)
    big = torch.zeros((65, w.nz, w.ny, w.nx), dtype=torch.complex128, device="cuda")
    with pytest.raises(hz.HzError) as e:
        hz.residual_noalloc(plan, big, big)
    assert e.value.code == 1
