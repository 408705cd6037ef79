"""Mixed path at the edges of its tiling and storage (needs a GB300).

Blocks wider than one tensor-core column tile (the table rows of the later tiles start at a
non-zero row of the block's tensor map), one and two z planes (the complex64 z sweep with
no back-substitution step), odd block starts and odd right-hand-side counts; every result
is compared with the oracle's sparse LU on the same seeded input.
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


def solve_and_check(hz, torch, w, precision):
    ref = O.solve(O.Problem.from_workload(w), w.f)
    plan = hz.Plan.from_workload(w, precision=precision)
    u = plan.solve(torch.from_numpy(w.f).cuda()).cpu().numpy()
    info = plan.info()
    if precision == "mixed":
        assert info["tensor_cores"] == 1
        assert info["rel_residual"] <= 1e-8
    assert rel(u, ref) < (TOL64 if precision == "fp64" else TOLMIX)


# x block of 150 nodes: two column tiles of 144 and 160 real columns; y block of 170
# nodes: three tiles of 112, 112 and 128
@pytest.mark.parametrize("kw", [dict(nx=150, ny=20, nz=6, bx=1, by=2, rim=6, pml=3, nrhs=1),
                                dict(nx=30, ny=170, nz=5, bx=2, by=1, rim=6, pml=3, nrhs=3)])
def test_mixed_blocks_wider_than_one_tile(hz, torch_cuda, kw):
    solve_and_check(hz, torch_cuda, W.tiny_pml(**kw), "mixed")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nz", [1, 2])
def test_one_and_two_z_planes(hz, torch_cuda, nz, precision):
    solve_and_check(hz, torch_cuda, W.tiny_pml(nx=23, ny=19, nz=nz, bx=2, by=3, rim=4, pml=2, nrhs=3),
                    precision)


def test_single_product_tf32_mixed_precision(hz, torch_cuda):
    # HZ_MIXED_TF32: one TF32 product per bulk transform (about 1e-3 per transform) reaches the
    # same tolerance through more corrections than the 3xTF32 form
    torch = torch_cuda
    w = W.tiny_pml(70, 45, 33, 3, 2, rim=6, pml=3, nrhs=2)
    ref = O.solve(O.Problem.from_workload(w), w.f)
    f = torch.from_numpy(w.f).cuda()
    refinements = {}
    for precision in ("mixed_tf32", "mixed"):
        plan = hz.Plan.from_workload(w, precision=precision, rtol=1e-10, max_refine=20)
        u = plan.solve(f).cpu().numpy()
        info = plan.info()
        assert info["tensor_cores"] == 1
        assert info["rel_residual"] <= 1e-10
        assert rel(u, ref) < TOLMIX
        refinements[precision] = info["refinements"]
    assert refinements["mixed_tf32"] > refinements["mixed"]


@pytest.mark.parametrize("real_tables", [True, False])
def test_real_table_kernel(hz, torch_cuda, real_tables):
    # real steps everywhere (real block tables): x one block of 130 (two real-table tiles of
    # 64 and 80 columns), y blocks of 40 and 79; 3 RHS x 5 planes give ragged row tiles
    torch = torch_cuda
    rng = np.random.default_rng(23)
    nx, ny, nz = 130, 120, 5
    rim = 1.2 ** np.arange(1, 6)                                        # real geometric rim
    hy = np.concatenate([rim[::-1], np.ones(ny - 9), rim]).astype(np.complex128)
    f = rng.standard_normal((3, nz, ny, nx)) + 1j * rng.standard_normal((3, nz, ny, nx))
    w = W.Workload("real-tables", W.uniform_steps(nx, 0.9), hy, W.ramp_z(nz), np.array([0, 2, nz], np.int32),
                   np.array([0.3 + 0.02j, 0.2 + 0.01j]), np.zeros(0, np.int32), np.array([40], np.int32), f)
    ref = O.solve(O.Problem.from_workload(w), w.f)
    plan = hz.Plan.from_workload(w, precision="mixed", rtol=1e-10, max_refine=12)
    plan.set_real_tables(real_tables)
    u = plan.solve(torch.from_numpy(w.f).cuda()).cpu().numpy()
    info = plan.info()
    assert info["tensor_cores"] == 1 and info["real_tables"] == int(real_tables)
    assert info["rel_residual"] <= 1e-10
    assert rel(u, ref) < TOLMIX
