"""The CPU oracle against closed forms, brute force and invariants (no GPU)."""
import numpy as np
import pytest

from oracle import hz_oracle as O
from paper_1909_01299_gb300 import workloads as W
from tests import oracle_pins as pins


def test_sine_eigenpairs_closed_form():
    assert pins.sine_eigenpair_error(9, 0.7) < 1e-13
    assert pins.sine_eigenpair_error(32, 1.0) < 1e-13


@pytest.mark.parametrize("axis", ["pml160_global", "pml160_block0", "pml160_block1", "ramp_z"])
def test_eigen_identity_nonuniform(axis):
    hx = W.rim_axis(128)
    if axis == "pml160_global":
        err = pins.eigen_identity_error(hx)
    elif axis == "pml160_block0":
        err = pins.eigen_identity_error(hx, 0, 79)
    elif axis == "pml160_block1":
        err = pins.eigen_identity_error(hx, 80, 80)
    else:
        err = pins.eigen_identity_error(W.ramp_z(64))
    assert err < 1e-12


@pytest.mark.parametrize("sigma", [False, True])
def test_kronecker_form_matches_stencil(sigma):
    w = W.tiny_pml(5, 4, 6, 2, 2, sigma=sigma, rim=1, pml=1)
    assert pins.stencil_error(w) < 1e-14


@pytest.mark.parametrize("method", ["lu", "blk"])
@pytest.mark.parametrize("blocks", [(1, 1), (2, 2), (3, 2)])
def test_quadratic_exact_solution(method, blocks):
    w = W.tiny_pml(13, 11, 9, blocks[0], blocks[1])
    assert pins.quadratic_error(w, method) < 1e-12


def test_quadratic_exact_on_pml160_rim_axis():
    # the full 160-node PML axis of the two-block workload, with a short z axis
    hx = W.rim_axis(128)
    w = W.Workload("q", hx, hx[:41].copy(), W.ramp_z(6), np.array([0, 3, 6], np.int32),
                   np.array([0.2 + 0.01j, 0.4 + 0.01j]), W.default_ifaces(160, 2),
                   W.default_ifaces(40, 2), np.zeros((1, 6, 40, 160), complex))
    assert pins.quadratic_error(w, "blk") < 1e-11


@pytest.mark.parametrize("blocks", [(1, 1), (2, 2), (3, 2)])
def test_single_mode_closed_form(blocks):
    assert pins.single_mode_error(blocks=blocks) < 1e-12


def test_poisson_special_case():
    # k^2 = 0 reduces to the discrete Poisson problem; its quadratic solution is exact
    w = W.tiny_pml(9, 8, 7, 2, 2)
    w.k2[:] = 0
    assert pins.quadratic_error(w, "blk") < 1e-12


@pytest.mark.parametrize("kw", [dict(), dict(bx=3, by=2), dict(bx=1, by=1), dict(sigma=True),
                                dict(nx=16, ny=16, nz=16, bx=4, by=4, rim=4, pml=2)])
def test_block_solver_matches_lu(kw):
    w = W.tiny_pml(**kw)
    assert pins.blk_vs_lu_error(w) < 1e-12


def test_partition_invariance():
    base = W.tiny_pml(16, 14, 8, 1, 1, rim=4, pml=2)
    P = O.Problem.from_workload(base)
    A, _ = O.assemble(P)
    ref = O.block_solve(P, base.f, A)
    for bx, by in [(2, 2), (4, 4), (3, 1)]:
        P2 = O.Problem(base.hx, base.hy, base.hz, base.z_begin, base.k2, None,
                       W.default_ifaces(16, bx), W.default_ifaces(14, by))
        u = O.block_solve(P2, base.f, A)
        assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-12


def test_residual_support_after_block_solves():
    assert pins.residual_support_error(W.tiny_pml()) < 1e-12


def test_residual_against_node_by_node_stencil():
    # per-RHS ||M f - A u|| / ||M f|| from the loop-assembled stencil, u = exact + perturbation
    assert pins.residual_error(W.tiny_pml(6, 5, 4, 2, 2, rim=1, pml=1)) < 1e-12


def test_residual_perturbed_against_node_by_node_stencil():
    # nonzero dk2: the perturbed residual from the loop-assembled perturbed stencil
    assert pins.residual_perturbed_error(W.tiny_pml(6, 5, 4, 2, 2, rim=1, pml=1, nrhs=2)) < 1e-11


def test_residual_of_block_solution():
    w = W.tiny_pml(16, 16, 16, 4, 4, rim=4, pml=2)
    P = O.Problem.from_workload(w)
    u = O.block_solve(P, w.f)
    assert np.all(O.residual(P, u, w.f) < 1e-12)


def test_operator_symmetric_and_reciprocity():
    w = W.tiny_pml(7, 6, 5, 2, 2, rim=2, pml=1)
    P = O.Problem.from_workload(w)
    A, mdiag = O.assemble(P)
    assert abs(A - A.T).max() == 0
    # point sources at s and r: u_s[r] / m_s = u_r[s] / m_r with m the weights of M
    nz, ny, nx = P.shape
    s, r = (1, 2, 3), (3, 4, 1)
    fs = np.zeros((1, nz, ny, nx), complex)
    fr = np.zeros_like(fs)
    fs[0][s] = 1.0
    fr[0][r] = 1.0
    us, ur = O.block_solve(P, fs, A), O.block_solve(P, fr, A)
    ms = O.weighted_rhs(P, fs)[0][s]
    mr = O.weighted_rhs(P, fr)[0][r]
    assert abs(us[0][r] / ms - ur[0][s] / mr) < 1e-12 * abs(us[0][r] / ms)


def test_adjoint_conjugation_identity():
    assert pins.adjoint_error(W.tiny_pml()) < 1e-12


def test_adjoint_dot_product():
    w = W.tiny_pml()
    P = O.Problem.from_workload(w)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(w.f.shape) + 1j * rng.standard_normal(w.f.shape)
    lam = O.adjoint_solve(P, g)
    x = O.block_solve_weighted(P, w.f)
    # <A^{-H} g, h> = <g, A^{-1} h>
    lhs = np.vdot(lam, w.f)
    rhs = np.vdot(g, x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_layer_gradient_central_differences():
    w = W.tiny_pml(9, 8, 9, 2, 2, nrhs=2)
    nz, ny, nx = w.nz, w.ny, w.nx
    rng = np.random.default_rng(11)
    rec = rng.choice(nx * ny * nz, 6, replace=False)
    P_true = O.Problem.from_workload(w, k2=w.k2 * 1.1)
    d_obs = O.solve(P_true, w.f).reshape(w.nrhs, -1)[:, rec]
    P = O.Problem.from_workload(w)
    J, G, _, _ = O.misfit_gradient(P, w.f, rec, d_obs)

    def J_at(k2):
        Pk = O.Problem.from_workload(w, k2=k2)
        u = O.solve(Pk, w.f)
        return O.misfit(u, rec, d_obs)[0]

    eps = 1e-6
    g_re, g_im = [], []
    for L in range(len(w.k2)):
        e = np.zeros(len(w.k2), complex)
        e[L] = eps
        g_re.append((J_at(w.k2 + e) - J_at(w.k2 - e)) / (2 * eps))
        g_im.append((J_at(w.k2 + 1j * e) - J_at(w.k2 - 1j * e)) / (2 * eps))
    g_re, g_im = np.array(g_re), np.array(g_im)
    assert np.linalg.norm(G.real - g_re) / np.linalg.norm(g_re) < 1e-6
    assert np.linalg.norm(-G.imag - g_im) / np.linalg.norm(g_im) < 1e-6


def test_workload_shapes():
    w = W.pml_160x160x128(nrhs=1)
    assert (w.nx, w.ny, w.nz) == (160, 160, 128)
    assert len(w.hx) == 161 and list(w.x_iface) == [79]
    assert np.sum(w.hx.imag != 0) == 18           # 9 complex steps per side
    assert abs(w.hz[0] - 0.5) < 1e-15 and abs(w.hz[-1] - 2.0) < 1e-15
    w3 = W.uniform_320x320x200(nrhs=1)
    assert list(w3.x_iface) == [79, 159, 239]
    w5 = W.adjoint_192x192x128(nsrc=2)
    assert len(w5.hx) == 193 and list(w5.x_iface) == [95]


def test_perturbed_solve_bruteforce():
    # dense node-by-node assembly with the perturbed k^2 (tiny grid, 2x2 blocks irrelevant here)
    w = W.tiny_pml(9, 8, 6, 2, 2, rim=2, pml=1, nrhs=2)
    assert pins.perturbed_bruteforce_error(w) < 1e-12


def test_perturbed_solve_born_series():
    w = W.tiny_pml(16, 14, 10, 2, 2, rim=3, pml=2, nrhs=2)
    assert pins.perturbed_born_series_error(w) < 1e-11


def test_perturbed_solve_zero_perturbation():
    w = W.tiny_pml(13, 11, 9, 2, 2, nrhs=1)
    P = O.Problem.from_workload(w)
    u0 = O.solve(P, w.f)
    u1 = O.solve_perturbed(P, w.f, np.zeros(P.shape, dtype=np.complex128))
    assert np.linalg.norm(u1 - u0) <= 1e-14 * np.linalg.norm(u0)
    assert np.all(O.residual_perturbed(P, u1, w.f, np.zeros(P.shape)) < 1e-12)


def test_rhs_gradient_against_central_differences():
    # complex (PML) steps make M complex, so a missing conjugate or a missing M is visible
    assert pins.rhs_gradient_fd_error(W.tiny_pml(9, 8, 6, 2, 2, rim=3, pml=2, nrhs=2)) < 1e-6
