"""CUDA path against the CPU oracle on the same seeded inputs (needs a GB300).

Tolerances: relative L2 error <= 1e-10 for the FP64 path and <= 1e-8 for the
mixed path after refinement, as the target states; residual checks use the
oracle's sparse operator.  Every call goes through the C ABI (hz.Plan).
"""
import numpy as np
import pytest

from oracle import hz_oracle as O
from paper_1909_01299_gb300 import workloads as W
from tests.parity import rel

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-8


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01299_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def hz(torch_cuda):
    from paper_1909_01299_gb300 import hz as mod
    return mod


def gpu_solve(hz, torch, w, precision="fp64", f=None, **kw):
    plan = hz.Plan.from_workload(w, precision=precision, **kw)
    fd = torch.from_numpy(w.f if f is None else f).cuda()
    u = plan.solve(fd).cpu().numpy()
    return plan, u


@pytest.mark.parametrize("kw", [
    dict(nx=13, ny=11, nz=9, bx=2, by=2),
    dict(nx=13, ny=11, nz=9, bx=3, by=2),
    dict(nx=13, ny=11, nz=9, bx=1, by=1),
    dict(nx=13, ny=11, nz=9, bx=2, by=1),
    dict(nx=13, ny=11, nz=9, bx=1, by=3),
    dict(nx=13, ny=11, nz=9, bx=2, by=2, sigma=True),
    dict(nx=16, ny=16, nz=16, bx=4, by=4, rim=4, pml=2),
    dict(nx=70, ny=45, nz=33, bx=3, by=2, rim=6, pml=3, nrhs=3),      # several tiles + ragged tails
])
def test_fp64_matches_lu(hz, torch_cuda, kw):
    w = W.tiny_pml(**kw)
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    _, u = gpu_solve(hz, torch_cuda, w)
    assert rel(u, ref) < TOL64


def test_fp64_quadratic_exact_solution(hz, torch_cuda):
    from tests.oracle_pins import quadratic_solution
    w = W.tiny_pml(40, 37, 21, 3, 2, rim=5, pml=2)
    u_ex, f = quadratic_solution(w)
    _, u = gpu_solve(hz, torch_cuda, w, f=f[None].copy())
    assert rel(u[0], u_ex) < TOL64


def test_single_block_32_matches_oracle(hz, torch_cuda):
    w = W.single_block_32()
    P = O.Problem.from_workload(w)
    ref = O.block_solve(P, w.f)
    plan, u = gpu_solve(hz, torch_cuda, w)
    assert rel(u, ref) < TOL64
    assert np.all(O.residual(P, u, w.f) < 1e-12)


@pytest.fixture(scope="module")
def pml160(hz, torch_cuda):
    w = W.pml_160x160x128()
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    ref = O.block_solve(P, w.f, A)
    return w, P, A, ref


def test_two_block_pml_full_size_fp64(hz, torch_cuda, pml160):
    w, P, A, ref = pml160
    plan, u = gpu_solve(hz, torch_cuda, w)
    for r in range(w.nrhs):
        assert rel(u[r], ref[r]) < TOL64
    assert np.all(O.residual(P, u, w.f, A) < 1e-10)
    # the library's own FP64 residual agrees with the oracle's
    fd = torch_cuda.from_numpy(w.f).cuda()
    res = plan.residual(fd, torch_cuda.from_numpy(u).cuda())
    assert np.allclose(res, O.residual(P, u, w.f, A), rtol=1e-3, atol=1e-15)


def test_two_block_pml_full_size_mixed(hz, torch_cuda, pml160):
    w, P, A, ref = pml160
    plan, u = gpu_solve(hz, torch_cuda, w, precision="mixed", rtol=1e-10, max_refine=12)
    info = plan.info()
    assert info["rel_residual"] <= 1e-10
    for r in range(w.nrhs):
        assert rel(u[r], ref[r]) < TOLMIX
    assert np.all(O.residual(P, u, w.f, A) < 1e-8)


@pytest.mark.parametrize("kw", [dict(nx=13, ny=11, nz=9, bx=2, by=2),
                                dict(nx=70, ny=45, nz=33, bx=3, by=2, rim=6, pml=3, nrhs=2)])
def test_mixed_matches_lu(hz, torch_cuda, kw):
    w = W.tiny_pml(**kw)
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    plan, u = gpu_solve(hz, torch_cuda, w, precision="mixed")
    assert rel(u, ref) < TOLMIX
    assert plan.info()["rel_residual"] <= 1e-8


def test_partition_invariance_gpu(hz, torch_cuda):
    base = W.tiny_pml(48, 40, 20, 1, 1, rim=6, pml=3)
    _, u1 = gpu_solve(hz, torch_cuda, base)
    for bx, by in [(2, 2), (4, 3), (3, 1)]:
        w = W.tiny_pml(48, 40, 20, bx, by, rim=6, pml=3)
        _, u = gpu_solve(hz, torch_cuda, w)
        assert rel(u, u1) < TOL64


def test_in_place_and_host_entry_points(hz, torch_cuda):
    torch = torch_cuda
    w = W.tiny_pml(30, 28, 17, 2, 2, rim=4, pml=2, nrhs=2)
    plan = hz.Plan.from_workload(w)
    fd = torch.from_numpy(w.f).cuda()
    u = plan.solve(fd).cpu().numpy()
    fd2 = torch.from_numpy(w.f).cuda()
    plan.solve(fd2, out=fd2)                                   # f == u
    assert rel(fd2.cpu().numpy(), u) < 1e-14
    uh = plan.solve_host(w.f)                                  # host buffers
    assert rel(uh, u) < 1e-14
    plan.set_options(precision="mixed")
    fd3 = torch.from_numpy(w.f).cuda()
    plan.solve(fd3, out=fd3)                                   # in place with refinement
    assert rel(fd3.cpu().numpy(), u) < TOLMIX


@pytest.mark.parametrize("nrhs", [1, 3, 5, 9])
def test_host_entry_point_chunks(hz, torch_cuda, nrhs):
    # host buffers: 1 RHS in one piece; 3, 5 and 9 RHS in up to eight uneven chunks whose
    # uploads, solves and downloads overlap; every RHS against the device-buffer solve
    torch = torch_cuda
    w = W.tiny_pml(30, 28, 17, 2, 2, rim=4, pml=2, nrhs=nrhs)
    plan = hz.Plan.from_workload(w, precision="fp64")
    u = plan.solve(torch.from_numpy(w.f).cuda()).cpu().numpy()
    for precision, tol in (("fp64", 1e-14), ("mixed", TOLMIX)):
        plan.set_options(precision=precision)
        uh = plan.solve_host(w.f)
        for r in range(nrhs):
            assert rel(uh[r], u[r]) < tol, (precision, r)
        if precision == "mixed":
            assert plan.info()["rel_residual"] <= 1e-8


def test_ragged_rhs_counts(hz, torch_cuda):
    torch = torch_cuda
    w = W.tiny_pml(33, 29, 19, 2, 3, rim=4, pml=2, nrhs=5)
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    plan = hz.Plan.from_workload(w)
    for R in (1, 5, 3):
        u = plan.solve(torch.from_numpy(w.f[:R].copy()).cuda()).cpu().numpy()
        assert rel(u, ref[:R]) < TOL64


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 5, 3), (6, 1, 4), (7, 6, 1), (5, 4, 2)])
def test_degenerate_sizes(hz, torch_cuda, shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(5)
    w = W.Workload("deg", W.uniform_steps(nx, 0.9), W.uniform_steps(ny, 1.1), W.ramp_z(nz),
                   np.array([0, nz], np.int32), np.array([0.3 + 0.02j]), np.zeros(0, np.int32),
                   np.zeros(0, np.int32), rng.standard_normal((2, nz, ny, nx)) + 0j)
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    _, u = gpu_solve(hz, torch_cuda, w)
    assert rel(u, ref) < TOL64


def test_single_node_blocks(hz, torch_cuda):
    # interfaces two nodes apart leave blocks of one node
    w = W.tiny_pml(9, 8, 6, 1, 1, rim=2, pml=1)
    w.x_iface = np.array([1, 3, 5, 7], np.int32)
    w.y_iface = np.array([2, 4], np.int32)
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    _, u = gpu_solve(hz, torch_cuda, w)
    assert rel(u, ref) < TOL64


def test_frequency_rescaling(hz, torch_cuda):
    torch = torch_cuda
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2)
    plan = hz.Plan.from_workload(w)
    fd = torch.from_numpy(w.f).cuda()
    for om in (0.5, 1.5):
        plan.set_frequency(om)
        u = plan.solve(fd).cpu().numpy()
        P = O.Problem.from_workload(w, k2=w.k2 * om * om)
        assert rel(u, O.solve(P, w.f)) < TOL64


def test_adjoint_and_layer_gradient(hz, torch_cuda):
    torch = torch_cuda
    w = W.tiny_pml(24, 22, 16, 2, 2, rim=3, pml=2, nrhs=2)
    rng = np.random.default_rng(2)
    rec = rng.choice(w.nx * w.ny * w.nz, 10, replace=False)
    d_obs = O.solve(O.Problem.from_workload(w, k2=w.k2 * 1.05), w.f).reshape(2, -1)[:, rec]
    P = O.Problem.from_workload(w)
    J_o, G_o, u_o, lam_o = O.misfit_gradient(P, w.f, rec, d_obs, method="lu")
    plan = hz.Plan.from_workload(w)
    u = plan.solve(torch.from_numpy(w.f).cuda())
    _, g = O.misfit(u.cpu().numpy(), rec, d_obs)
    lam = plan.solve_adjoint(torch.from_numpy(g).cuda())
    assert rel(lam.cpu().numpy(), lam_o) < TOL64
    G = plan.grad_layers(u, lam)
    assert rel(G, G_o) < 1e-9


def test_autograd_wrapper_against_finite_differences(hz, torch_cuda):
    torch = torch_cuda
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=1)
    plan = hz.Plan.from_workload(w)
    rng = np.random.default_rng(4)
    rec = torch.from_numpy(rng.choice(w.nx * w.ny * w.nz, 8, replace=False)).cuda()
    d = torch.from_numpy(rng.standard_normal(8) * 1e-2 + 0j).cuda()
    f = torch.from_numpy(w.f).cuda()

    def loss(k2):
        u = hz.HzSolve.apply(k2, f, plan)
        return 0.5 * (u.reshape(-1)[rec] - d).abs().pow(2).sum()

    k2 = torch.tensor(w.k2, dtype=torch.complex128, requires_grad=True)
    L = loss(k2)
    L.backward()
    eps = 1e-6
    for Lyr in range(len(w.k2)):
        e = torch.zeros_like(k2.detach())
        e[Lyr] = eps
        fd_re = (loss(k2.detach() + e) - loss(k2.detach() - e)).item() / (2 * eps)
        fd_im = (loss(k2.detach() + 1j * e) - loss(k2.detach() - 1j * e)).item() / (2 * eps)
        g = k2.grad[Lyr].item()
        assert abs(g.real - fd_re) <= 1e-6 * max(abs(fd_re), 1e-12) + 1e-12
        assert abs(g.imag - fd_im) <= 1e-6 * max(abs(fd_im), 1e-12) + 1e-12


def test_autograd_rhs_gradient(hz, torch_cuda):
    # f.grad = M^H lam from hz_grad_rhs: against the oracle's right-hand-side gradient of its
    # adjoint state and against central differences in Re f and Im f (PML grid: complex M)
    torch = torch_cuda
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=2)
    plan = hz.Plan.from_workload(w)
    rng = np.random.default_rng(5)
    rec_np = rng.choice(w.nx * w.ny * w.nz, 8, replace=False)
    d_np = rng.standard_normal((2, 8)) * 1e-2 + 0j
    rec = torch.from_numpy(rec_np).cuda()
    d = torch.from_numpy(d_np).cuda()
    k2 = torch.tensor(w.k2, dtype=torch.complex128)

    def loss(f):
        u = hz.HzSolve.apply(k2, f, plan)
        return 0.5 * (u.reshape(2, -1)[:, rec] - d).abs().pow(2).sum()

    f = torch.from_numpy(w.f).cuda().requires_grad_()
    loss(f).backward()
    gf = f.grad.cpu().numpy()
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    _, g = O.misfit(O.solve(P, w.f, A), rec_np, d_np)
    ref = O.rhs_gradient(P, O.adjoint_solve(P, g, A, method="lu"))
    assert rel(gf, ref) < TOL64
    eps = 1e-6
    f0 = torch.from_numpy(w.f).cuda()
    for (r, k, j, i) in ((0, 3, 4, 5), (1, 6, 9, 10), (0, 11, 17, 19)):
        e = torch.zeros_like(f0)
        e[r, k, j, i] = eps
        with torch.no_grad():
            fd_re = (loss(f0 + e) - loss(f0 - e)).item() / (2 * eps)
            fd_im = (loss(f0 + 1j * e) - loss(f0 - 1j * e)).item() / (2 * eps)
        scale = abs(fd_re) + abs(fd_im)
        assert abs(gf[r, k, j, i].real - fd_re) <= 1e-6 * scale
        assert abs(gf[r, k, j, i].imag - fd_im) <= 1e-6 * scale


def test_singular_mode_is_reported(hz, torch_cuda):
    # one x and one y node (lambda = mu = 2) and k^2 = 6 make the z matrix of the only mode
    # tridiag(-1, 0, -1): its first pivot is exactly zero
    with pytest.raises(hz.HzError) as e:
        hz.Plan(W.uniform_steps(1), W.uniform_steps(1), W.uniform_steps(3), [0, 3], [6.0 + 0j])
    assert e.value.code == 3


def _complex_z(w):
    """Give the z axis an absorbing (complex) end: the last 3 steps times (1 + 0.5i)."""
    hz = w.hz.copy()
    hz[-3:] *= (1 + 0.5j)
    w.hz = hz
    return w


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_complex_z_steps(hz, torch_cuda, precision):
    # complex z steps make the z off-diagonals complex (the general sweep and stencil paths)
    w = _complex_z(W.tiny_pml(26, 22, 15, 2, 2, rim=3, pml=2, nrhs=2))
    ref = O.solve(O.Problem.from_workload(w), w.f)
    plan, u = gpu_solve(hz, torch_cuda, w, precision=precision)
    assert rel(u, ref) < (TOL64 if precision == "fp64" else TOLMIX)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_layers(hz, torch_cuda, precision):
    w = W.tiny_pml(30, 26, 17, 3, 2, rim=4, pml=2, nrhs=2, sigma=True)
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    plan, u = gpu_solve(hz, torch_cuda, w, precision=precision)
    assert rel(u, ref) < (TOL64 if precision == "fp64" else TOLMIX)
    res = plan.residual(torch_cuda.from_numpy(w.f).cuda(), torch_cuda.from_numpy(u).cuda())
    assert np.allclose(res, O.residual(P, u, w.f), rtol=1e-3, atol=1e-15)


def test_mixed_adjoint_and_host_entry(hz, torch_cuda):
    torch = torch_cuda
    w = W.tiny_pml(28, 24, 16, 2, 2, rim=3, pml=2, nrhs=2)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(w.f.shape) + 1j * rng.standard_normal(w.f.shape)
    lam_o = O.adjoint_solve(O.Problem.from_workload(w), g, method="lu")
    plan = hz.Plan.from_workload(w, precision="mixed")
    lam = plan.solve_adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    assert rel(lam, lam_o) < TOLMIX
    uh = plan.solve_host(w.f)
    assert rel(uh, O.solve(O.Problem.from_workload(w), w.f)) < TOLMIX


def test_refinement_not_converged_is_reported(hz, torch_cuda):
    # zero corrections allowed and an unreachable tolerance: the mixed path must say so
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=1)
    plan = hz.Plan.from_workload(w, precision="mixed", rtol=1e-15, max_refine=0)
    with pytest.raises(hz.HzError) as e:
        plan.solve(torch_cuda.from_numpy(w.f).cuda())
    assert e.value.code == 5


def test_nonfinite_input_is_reported(hz, torch_cuda):
    w = W.tiny_pml(20, 18, 12, 2, 2, rim=3, pml=2, nrhs=1)
    f = w.f.copy()
    f[0, 3, 4, 5] = np.nan
    plan = hz.Plan.from_workload(w)
    fd = torch_cuda.from_numpy(f).cuda()
    u = plan.solve(fd)
    with pytest.raises(hz.HzError) as e:
        plan.residual(fd, u)
    assert e.value.code == 4


def _uniform_mix_workload(nrhs=2):
    # x uniform in three blocks of 17, 18, 17 nodes (all take the closed-form sine pairs and
    # the folded transforms, odd and even widths); y = 4 rim nodes | 35 uniform core nodes |
    # 4 rim nodes, so one transform set mixes folded and dense complex blocks
    rng = np.random.default_rng(11)
    nx, ny, nz = 54, 45, 9
    hx = W.uniform_steps(nx, 1.0)
    hy = W.rim_axis(ny - 8, rim_nodes=4, ratio=1.3, pml_nodes=2)
    k2 = np.array([0.2 + 0.01j, 0.35 + 0.02j])
    return W.Workload("uniform-mix", hx, hy, W.ramp_z(nz), np.array([0, 4, nz], np.int32), k2,
                      np.array([17, 36], np.int32), np.array([4, 40], np.int32),
                      rng.standard_normal((nrhs, nz, ny, nx)) + 1j * rng.standard_normal((nrhs, nz, ny, nx)))


@pytest.mark.parametrize("precision,fast", [("fp64", 1), ("fp64", 0), ("mixed", 2), ("mixed", 1)])
def test_uniform_blocks_sine_path(hz, torch_cuda, precision, fast):
    # x blocks 17 (n + 1 = 18 = 2 x 3 x 3: fast sine transform), 18 (19 is prime: folded dense),
    # 17; y core block of 35 (36 = 4 x 3 x 3) between dense complex rim blocks
    w = _uniform_mix_workload()
    P = O.Problem.from_workload(w)
    ref = O.solve(P, w.f)
    plan = hz.Plan.from_workload(w, precision=precision)
    plan.set_fast_sine(fast)
    u = plan.solve(torch_cuda.from_numpy(w.f).cuda()).cpu().numpy()
    assert rel(u, ref) < (TOL64 if precision == "fp64" else TOLMIX)
    assert plan.info()["eig_max_residual"] < 1e-12
    assert plan.info()["fast_sine"] == fast


def test_fast_sine_many_tiles_against_lu_and_dense(hz, torch_cuda):
    # uniform 160 x 99 x 7 grid: x blocks of 79 and 80 nodes (n + 1 = 80 = 16 x 5, split by
    # the prime-factor map, and 81 = 3^4, as in the 320-node benchmark grid), y one block of 99
    # (100 = 4 x 5 x 5, mixed radix with twiddles);
    # 3 RHS give 2079 and 3339 rows per transform launch (ragged last row tile)
    torch = torch_cuda
    rng = np.random.default_rng(17)
    nx, ny, nz = 160, 99, 7
    f = rng.standard_normal((3, nz, ny, nx)) + 1j * rng.standard_normal((3, nz, ny, nx))
    w = W.Workload("uniform-fast-sine", W.uniform_steps(nx, 0.8), W.uniform_steps(ny, 1.2), W.ramp_z(nz),
                   np.array([0, 3, nz], np.int32), np.array([0.3 + 0.02j, 0.15 + 0.01j]),
                   np.array([79], np.int32), np.zeros(0, np.int32), f)
    ref = O.solve(O.Problem.from_workload(w), w.f)
    plan = hz.Plan.from_workload(w, precision="fp64")
    fd = torch.from_numpy(w.f).cuda()
    u_fast = plan.solve(fd).cpu().numpy()
    assert plan.info()["fast_sine"] == 1
    plan.set_fast_sine(0)
    u_dense = plan.solve(fd).cpu().numpy()
    assert rel(u_fast, ref) < TOL64
    assert rel(u_fast, u_dense) < 1e-12
    # the mixed path: bulk transforms of these all-uniform blocks by the FP32 fast sine kernel
    plan.set_options(precision="mixed", rtol=1e-10, max_refine=12)
    plan.set_fast_sine(2)
    u_mix = plan.solve(fd).cpu().numpy()
    assert plan.info()["rel_residual"] <= 1e-10
    assert rel(u_mix, ref) < TOLMIX


def test_fast_sine_adjoint(hz, torch_cuda):
    # the conjugating inverse transform of the FP64 adjoint through the fast sine kernel
    torch = torch_cuda
    w = _uniform_mix_workload()
    rng = np.random.default_rng(13)
    g = rng.standard_normal(w.f.shape) + 1j * rng.standard_normal(w.f.shape)
    lam_o = O.adjoint_solve(O.Problem.from_workload(w), g, method="lu")
    plan = hz.Plan.from_workload(w, precision="fp64")
    lam = plan.solve_adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    assert plan.info()["fast_sine"] == 1
    assert rel(lam, lam_o) < TOL64


def test_uniform_blocks_mixed_adjoint(hz, torch_cuda):
    # the conjugating transforms run on CUDA cores in FP32: the folded path with conj_out
    torch = torch_cuda
    w = _uniform_mix_workload()
    rng = np.random.default_rng(12)
    g = rng.standard_normal(w.f.shape) + 1j * rng.standard_normal(w.f.shape)
    lam_o = O.adjoint_solve(O.Problem.from_workload(w), g, method="lu")
    plan = hz.Plan.from_workload(w, precision="mixed")
    lam = plan.solve_adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    assert rel(lam, lam_o) < TOLMIX


def test_auto_partition_matches_lu(hz, torch_cuda):
    # HZ_BLOCKS_AUTO: the FP64 plan picks round(sqrt(3 N / 7)) blocks of >= 16 nodes per axis,
    # the mixed plan blocks about 80 nodes wide
    torch = torch_cuda
    w = W.tiny_pml(96, 66, 8, 1, 1, rim=8, pml=3, nrhs=1)
    ref = O.solve(O.Problem.from_workload(w), w.f)
    for precision, tol, counts in (("fp64", TOL64, (6, 4)), ("mixed", TOLMIX, (1, 1))):
        plan = hz.Plan(w.hx, w.hy, w.hz, w.z_begin, w.k2, w.sigma, nbx=0, nby=0, precision=precision)
        u = plan.solve(torch.from_numpy(w.f).cuda()).cpu().numpy()
        info = plan.info()
        assert (info["nbx"], info["nby"]) == counts
        assert rel(u, ref) < tol


_REFS = {}


def _oracle_ref(key, make):
    """The oracle's sparse-LU solution of a seeded workload, computed once per module."""
    if key not in _REFS:
        w = make()
        _REFS[key] = (w, O.solve(O.Problem.from_workload(w), w.f))
    return _REFS[key]


@pytest.mark.parametrize("z_sweep", [0, 1, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_long_z_few_modes(hz, torch_cuda, precision, z_sweep):
    # few modes, long z: 13 x 11 nodes in 2 x 2 blocks, 1536 ramped z steps, 2 RHS (the
    # automatic choice takes the chunked sweep here)
    w, ref = _oracle_ref("long_z", lambda: W.long_z(nx=13, ny=11, nz=1536, nrhs=2))
    plan = hz.Plan.from_workload(w, precision=precision)
    plan.set_z_sweep(z_sweep)
    u = plan.solve(torch_cuda.from_numpy(w.f).cuda()).cpu().numpy()
    assert plan.info()["z_sweep"] == z_sweep
    assert rel(u, ref) < (TOL64 if precision == "fp64" else TOLMIX)


@pytest.mark.parametrize("z_sweep", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kw", [dict(nx=70, ny=45, nz=33, bx=3, by=2, rim=6, pml=3, nrhs=3),   # ragged z chunk
                                dict(nx=23, ny=19, nz=1, bx=2, by=3, rim=4, pml=2, nrhs=2),
                                dict(nx=23, ny=19, nz=17, bx=2, by=3, rim=4, pml=2, nrhs=1, sigma=True)])
def test_z_sweep_variants(hz, torch_cuda, kw, precision, z_sweep):
    # every z sweep variant on the same input: one or two RHS per thread, z in register
    # chunks of 16 (33 and 17 planes leave a short last chunk, 1 plane no back substitution)
    w, ref = _oracle_ref(repr(sorted(kw.items())), lambda: W.tiny_pml(**kw))
    plan = hz.Plan.from_workload(w, precision=precision)
    plan.set_z_sweep(z_sweep)
    u = plan.solve(torch_cuda.from_numpy(w.f).cuda()).cpu().numpy()
    assert rel(u, ref) < (TOL64 if precision == "fp64" else TOLMIX)
