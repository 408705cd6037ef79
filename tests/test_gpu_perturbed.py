"""Locally perturbed layered medium: GMRES around the layered solve against the oracle's
sparse LU of the perturbed operator (needs a GB300)."""
import numpy as np
import pytest

from oracle import hz_oracle as O
from paper_1909_01299_gb300 import workloads as W
from tests.parity import rel
from tests import oracle_pins as pins

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


@pytest.mark.parametrize("precision,rtol,tol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8)])
def test_perturbed_medium_matches_lu(env, precision, rtol, tol):
    torch, hz = env
    w = W.tiny_pml(30, 26, 16, 2, 2, rim=4, pml=2, nrhs=2)
    P = O.Problem.from_workload(w)
    dk2 = pins.perturbation(P, amp=0.3)
    ref = O.solve_perturbed(P, w.f, dk2)
    plan = hz.Plan.from_workload(w, precision=precision)
    u, iters, relres = plan.solve_perturbed(torch.from_numpy(dk2).cuda(), torch.from_numpy(w.f).cuda(),
                                            rtol=rtol, max_iter=300, restart=25)
    u = u.cpu().numpy()
    assert 0 < iters < 300
    assert rel(u, ref) < tol
    assert np.all(relres < tol)
    assert np.allclose(relres, O.residual_perturbed(P, u, w.f, dk2), rtol=1e-2, atol=1e-14)


def test_zero_perturbation_is_the_layered_solve(env):
    torch, hz = env
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=3)
    plan = hz.Plan.from_workload(w, precision="fp64")
    f = torch.from_numpy(w.f).cuda()
    zero = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.complex128, device="cuda")
    u, iters, relres = plan.solve_perturbed(zero, f, rtol=1e-12)
    assert iters == 0
    assert rel(u.cpu().numpy(), plan.solve(f).cpu().numpy()) < 1e-14
    assert np.all(relres < 1e-10)


def test_perturbed_not_converged_is_reported(env):
    torch, hz = env
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=1)
    P = O.Problem.from_workload(w)
    dk2 = pins.perturbation(P, amp=0.3)
    plan = hz.Plan.from_workload(w, precision="fp64")
    with pytest.raises(hz.HzError) as e:
        plan.solve_perturbed(torch.from_numpy(dk2).cuda(), torch.from_numpy(w.f).cuda(), rtol=1e-14, max_iter=2)
    assert e.value.code == 5
