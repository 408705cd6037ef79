"""The named full-size workloads on the GPU against the CPU oracle (needs a GB300).

At full size the oracle is used where it finishes in seconds: its sparse operator
gives every RHS's residual ||M f - A u|| / ||M f||, and its block solver gives
sampled right-hand sides element by element.
"""
import numpy as np
import pytest

from oracle import hz_oracle as O
from paper_1909_01299_gb300 import workloads as W
from tests.parity import rel

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


def test_uniform_320_mixed_4x4_blocks(env):
    torch, hz = env
    w = W.uniform_320x320x200(nrhs=8)
    plan = hz.Plan.from_workload(w, precision="mixed", rtol=1e-8)
    f = torch.from_numpy(w.f).cuda()
    u = plan.solve(f)
    info = plan.info()
    assert info["rel_residual"] <= 1e-8
    u_h = u.cpu().numpy()
    del u, f
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    assert np.all(O.residual(P, u_h, w.f, A) <= 1e-8)
    # two of the eight RHS element by element (first and last source)
    for r in (0, 7):
        ref = O.block_solve(P, w.f[r:r + 1], A)
        assert rel(u_h[r:r + 1], ref) < 1e-8, r


def test_uniform_320_fp64_sampled(env):
    torch, hz = env
    w = W.uniform_320x320x200(nrhs=2)
    plan = hz.Plan.from_workload(w, precision="fp64")
    u_h = plan.solve(torch.from_numpy(w.f).cuda()).cpu().numpy()
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    assert np.all(O.residual(P, u_h, w.f, A) <= 1e-10)
    ref = O.block_solve(P, w.f[1:2], A)
    assert rel(u_h[1:2], ref) < 1e-10


@pytest.fixture(scope="module")
def adj192(env):
    w = W.adjoint_192x192x128(nsrc=16)
    rec = w.extra["rec_flat"]
    # observed data from the true model, computed by the oracle's block solver
    P_true = O.Problem.from_workload(w, k2=w.extra["k2_true"])
    A_true, _ = O.assemble(P_true)
    d_obs = O.block_solve(P_true, w.f, A_true).reshape(w.nrhs, -1)[:, rec]
    return w, rec, d_obs


def test_adjoint_gradient_192_against_oracle(env, adj192):
    torch, hz = env
    w, rec, d_obs = adj192
    nsub = 4                                   # oracle gradient over 4 of the 16 sources
    P = O.Problem.from_workload(w)
    J_o, G_o, _, lam_o = O.misfit_gradient(P, w.f[:nsub], rec, d_obs[:nsub])
    plan = hz.Plan.from_workload(w, precision="fp64")
    u = plan.solve(torch.from_numpy(np.ascontiguousarray(w.f[:nsub])).cuda())
    J, g = O.misfit(u.cpu().numpy(), rec, d_obs[:nsub])
    assert abs(J - J_o) <= 1e-10 * abs(J_o)
    lam = plan.solve_adjoint(torch.from_numpy(g).cuda())
    assert rel(lam.cpu().numpy(), lam_o) < 1e-9
    G = plan.grad_layers(u, lam)
    assert rel(G, G_o) < 1e-6


def test_adjoint_gradient_192_central_differences(env, adj192):
    torch, hz = env
    w, rec, d_obs = adj192
    plan = hz.Plan.from_workload(w, precision="fp64")
    f = torch.from_numpy(w.f).cuda()
    rec_t = torch.from_numpy(rec).cuda()
    d_t = torch.from_numpy(d_obs).cuda()

    def J_of(k2):
        plan.set_k2(k2)
        u = plan.solve(f).reshape(w.nrhs, -1)
        return 0.5 * float((u[:, rec_t] - d_t).abs().pow(2).sum())

    J_of(w.k2)
    u = plan.solve(f)
    flat = u.reshape(w.nrhs, -1)
    g = torch.zeros_like(flat)
    g[:, rec_t] = flat[:, rec_t] - d_t
    lam = plan.solve_adjoint(g.reshape(u.shape).contiguous())
    G = plan.grad_layers(u, lam)
    eps = 1e-6
    layers = [0, 7, 15, 31]                    # a sample of the 32 layers, top to bottom
    fd_re, fd_im = [], []
    for L in layers:
        e = np.zeros(len(w.k2), complex)
        e[L] = eps
        fd_re.append((J_of(w.k2 + e) - J_of(w.k2 - e)) / (2 * eps))
        fd_im.append((J_of(w.k2 + 1j * e) - J_of(w.k2 - 1j * e)) / (2 * eps))
    fd_re, fd_im = np.array(fd_re), np.array(fd_im)
    assert np.linalg.norm(G[layers].real - fd_re) <= 1e-6 * np.linalg.norm(fd_re)
    assert np.linalg.norm(-G[layers].imag - fd_im) <= 1e-6 * np.linalg.norm(fd_im)
