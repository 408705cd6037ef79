"""Seeded synthetic inputs for the layered-medium Helmholtz solver.

This module builds grids, layer tables, block partitions and right-hand sides
only.  It holds none of the solver's arithmetic (no operator, no transform, no
elimination), so both the CPU oracle and the CUDA path may use it.

Grids follow the paper's setting (Sec. 1, Sec. 2): a tensor-product grid
S_x x S_y x S_z whose x/y axes have a fine uniform survey core, a rim
coarsened geometrically outwards and complex ("PML") steps on the outer part
of the rim; z is layered.  Every axis with N interior (unknown) nodes carries
N+1 steps h_0..h_N; step h_n joins node n-1 to node n, and nodes -1 and N are
homogeneous Dirichlet nodes.

Random draws use numpy's PCG64 generator seeded with 190901299 + the
1-based workload number, in the order: layer k^2, layer boundaries, source
locations, noise.  Complex noise is re + i*im with both parts N(0, 1).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 190901299


@dataclasses.dataclass
class Workload:
    """One synthetic layered-medium problem (all arrays are host numpy)."""
    name: str
    hx: np.ndarray            # (Nx+1,) complex128 steps
    hy: np.ndarray            # (Ny+1,) complex128 steps
    hz: np.ndarray            # (Nz+1,) complex128 steps
    z_begin: np.ndarray       # (nlayers+1,) int32 node index where each layer starts
    k2: np.ndarray            # (nlayers,) complex128 per-layer k^2
    x_iface: np.ndarray       # (nbx-1,) int32 interface node indices in x
    y_iface: np.ndarray       # (nby-1,) int32 interface node indices in y
    f: np.ndarray             # (nrhs, Nz, Ny, Nx) complex128 right-hand sides
    sigma: Optional[np.ndarray] = None   # (nlayers,) float64 per-layer sigma, None = 1
    precision: str = "fp64"   # "fp64" or "mixed"
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def nx(self) -> int:
        return len(self.hx) - 1

    @property
    def ny(self) -> int:
        return len(self.hy) - 1

    @property
    def nz(self) -> int:
        return len(self.hz) - 1

    @property
    def nrhs(self) -> int:
        return self.f.shape[0]

    @property
    def unknowns(self) -> int:
        return self.nx * self.ny * self.nz

    def k2_nodes(self) -> np.ndarray:
        """Per-node k^2 expanded from the layer table (layer L = nodes [z_begin[L], z_begin[L+1]))."""
        out = np.empty(self.nz, dtype=np.complex128)
        for L in range(len(self.k2)):
            out[self.z_begin[L]:self.z_begin[L + 1]] = self.k2[L]
        return out


def default_ifaces(n: int, nblocks: int) -> np.ndarray:
    """Interface node positions p_b = floor(b (N+1) / B) - 1, b = 1..B-1."""
    return np.array([(b * (n + 1)) // nblocks - 1 for b in range(1, nblocks)], dtype=np.int32)


def uniform_steps(n: int, h: float = 1.0) -> np.ndarray:
    """N+1 equal real steps for N interior nodes."""
    return np.full(n + 1, h, dtype=np.complex128)


def rim_axis(core_nodes: int, rim_nodes: int = 16, ratio: float = 1.3, pml_nodes: int = 8,
             h_core: float = 1.0) -> np.ndarray:
    """Steps of a survey axis: uniform core, geometric rim, complex-stepped outer rim.

    The core has `core_nodes` nodes spaced h_core.  Going outwards from each core
    edge the n-th step (n = 1..rim_nodes+1) is h_core * ratio**n; step
    rim_nodes+1 reaches the Dirichlet node.  Steps n > rim_nodes - pml_nodes are
    multiplied by (1 + 1i), which puts the last `pml_nodes` rim nodes (and the
    step to the boundary) in the complex-stepped absorbing layer.
    """
    n = np.arange(1, rim_nodes + 2)
    rim = h_core * ratio ** n.astype(np.float64)
    rim = rim.astype(np.complex128)
    rim[n > rim_nodes - pml_nodes] *= (1.0 + 1.0j)
    core = np.full(core_nodes - 1, h_core, dtype=np.complex128)
    return np.concatenate([rim[::-1], core, rim])


def ramp_z(nz: int, h0: float = 0.5, h1: float = 2.0) -> np.ndarray:
    """Deterministic geometric ramp of N+1 steps from h0 to h1: h_n = h0 (h1/h0)^(n/N)."""
    n = np.arange(nz + 1, dtype=np.float64)
    return (h0 * (h1 / h0) ** (n / nz)).astype(np.complex128)


def _cnoise(rng: np.random.Generator, shape) -> np.ndarray:
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def point_source_plane(nz, ny, nx, k, j, i) -> np.ndarray:
    f = np.zeros((nz, ny, nx), dtype=np.complex128)
    f[k, j, i] = 1.0
    return f


def gaussian_source(nz, ny, nx, center, sigma=2.0) -> np.ndarray:
    """exp(-rho^2 / (2 sigma^2)) in node units, truncated at rho > 4 sigma, peak 1."""
    kc, jc, ic = center
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho2 = (kk - kc) ** 2 + (jj - jc) ** 2 + (ii - ic) ** 2
    g = np.exp(-rho2 / (2.0 * sigma * sigma))
    g[rho2 > (4.0 * sigma) ** 2] = 0.0
    return g.astype(np.complex128)


# ---------------------------------------------------------------------------
# The five named workloads
# ---------------------------------------------------------------------------

def single_block_32(nrhs: int = 1) -> Workload:
    """Uniform 32^3 grid, h = 1, one block, 4 layers of 8 planes; point source + 1e-3 noise."""
    rng = np.random.default_rng(SEED_BASE + 1)
    n = 32
    k2 = np.array([0.10, 0.25, 0.15, 0.40]) * (1 + 0.05j)
    z_begin = np.array([0, 8, 16, 24, 32], dtype=np.int32)
    f = np.empty((nrhs, n, n, n), dtype=np.complex128)
    for r in range(nrhs):
        f[r] = point_source_plane(n, n, n, 16, 16, 16) + 1e-3 * _cnoise(rng, (n, n, n))
    return Workload("uniform-32x32x32-1x1blocks-fp64", uniform_steps(n), uniform_steps(n),
                    uniform_steps(n), z_begin, k2.astype(np.complex128),
                    np.zeros(0, np.int32), np.zeros(0, np.int32), f)


def pml_160x160x128(nrhs: int = 4) -> Workload:
    """160x160x128, PML rim in x/y, ramped z, 12 layers, 2x2 blocks, 4 point sources."""
    rng = np.random.default_rng(SEED_BASE + 2)
    nx = ny = 160
    nz = 128
    nlayers = 12
    k2 = rng.uniform(0.05, 0.5, nlayers) * (1 + 0.02j)
    z_begin = np.array([(nz * L) // nlayers for L in range(nlayers + 1)], dtype=np.int32)
    src = np.stack([rng.integers(16, 144, nrhs), rng.integers(16, 144, nrhs),
                    rng.integers(8, 120, nrhs)], axis=1)       # (x, y, z)
    f = np.empty((nrhs, nz, ny, nx), dtype=np.complex128)
    for r in range(nrhs):
        f[r] = point_source_plane(nz, ny, nx, src[r, 2], src[r, 1], src[r, 0])
    hx = rim_axis(128)
    return Workload("pml-160x160x128-2x2blocks-4rhs-fp64", hx, hx.copy(), ramp_z(nz), z_begin,
                    k2.astype(np.complex128), default_ifaces(nx, 2), default_ifaces(ny, 2), f,
                    extra={"sources_xyz": src})


def uniform_320x320x200(nrhs: int = 8) -> Workload:
    """320x320x200, h = 1, 4 layers of 50 planes, 4x4 blocks, 8 Gaussian sources; mixed path."""
    rng = np.random.default_rng(SEED_BASE + 3)
    nx = ny = 320
    nz = 200
    k2 = (np.array([0.10, 0.25, 0.15, 0.40]) * (1 + 0.05j)).astype(np.complex128)
    z_begin = np.array([0, 50, 100, 150, 200], dtype=np.int32)
    cen = np.stack([rng.integers(8, nz - 8, nrhs), rng.integers(8, ny - 8, nrhs),
                    rng.integers(8, nx - 8, nrhs)], axis=1)     # (z, y, x)
    f = np.empty((nrhs, nz, ny, nx), dtype=np.complex128)
    for r in range(nrhs):
        f[r] = gaussian_source(nz, ny, nx, cen[r])
    return Workload("uniform-320x320x200-4x4blocks-8rhs", uniform_steps(nx), uniform_steps(ny),
                    uniform_steps(nz), z_begin, k2, default_ifaces(nx, 4), default_ifaces(ny, 4), f,
                    precision="mixed", extra={"centres_zyx": cen})


def uniform_320x320x40(nrhs: int = 2) -> Workload:
    """The 320 x 320 grid of the benchmark workload with 40 planes and 2 RHS (same blocks of
    79 and 80 nodes, inputs of 131 MB, above the L2 size): a small case for kernel captures."""
    rng = np.random.default_rng(SEED_BASE + 103)
    nx = ny = 320
    nz = 40
    k2 = (np.array([0.10, 0.25, 0.15, 0.40]) * (1 + 0.05j)).astype(np.complex128)
    cen = np.stack([rng.integers(8, nz - 8, nrhs), rng.integers(8, ny - 8, nrhs),
                    rng.integers(8, nx - 8, nrhs)], axis=1)     # (z, y, x)
    f = np.empty((nrhs, nz, ny, nx), dtype=np.complex128)
    for r in range(nrhs):
        f[r] = gaussian_source(nz, ny, nx, cen[r])
    return Workload("uniform-320x320x40-4x4blocks-2rhs", uniform_steps(nx), uniform_steps(ny),
                    uniform_steps(nz), np.array([0, 10, 20, 30, 40], dtype=np.int32), k2,
                    default_ifaces(nx, 4), default_ifaces(ny, 4), f, precision="mixed")


def long_z(nx: int = 32, ny: int = 32, nz: int = 4096, nrhs: int = 4, bx: int = 2, by: int = 2) -> Workload:
    """Few modes, long z: a narrow column (nx x ny nodes, h = 1, bx x by blocks) of nz ramped
    z steps with 64 layers, seeded complex noise.  The regime where one z sweep per mode leaves
    most of the GPU idle (nx ny nrhs sweeps of length nz)."""
    rng = np.random.default_rng(SEED_BASE + 6)
    nl = 64
    k2 = (rng.uniform(0.05, 0.5, nl) * (1 + 0.02j)).astype(np.complex128)
    z_begin = np.array([(nz * L) // nl for L in range(nl + 1)], dtype=np.int32)
    f = _cnoise(rng, (nrhs, nz, ny, nx))
    return Workload(f"longz-{nx}x{ny}x{nz}-{bx}x{by}blocks-{nrhs}rhs", uniform_steps(nx), uniform_steps(ny),
                    ramp_z(nz, 0.5, 1.0), z_begin, k2, default_ifaces(nx, bx), default_ifaces(ny, by), f)


def adjoint_192x192x128(nsrc: int = 16) -> Workload:
    """192x192x128, PML rim in x/y, uniform z, 32 layers of 4 planes, 2x2 blocks.

    Sources and receivers sit at distinct seeded core (x, y) positions on z-plane 4.
    `extra` holds the receiver indices and the "true" layer k^2 (drawn with seed + 1000)
    from which observed data are synthesised.
    """
    rng = np.random.default_rng(SEED_BASE + 5)
    nx = ny = 192
    nz = 128
    nlayers = 32
    k2 = (rng.uniform(0.05, 0.5, nlayers) * (1 + 0.02j)).astype(np.complex128)
    z_begin = np.arange(0, nz + 1, 4, dtype=np.int32)
    core = np.arange(16, 176)
    cells = rng.choice(len(core) * len(core), size=2 * nsrc, replace=False)
    xs, ys = core[cells % len(core)], core[cells // len(core)]
    src_xy = np.stack([xs[:nsrc], ys[:nsrc]], axis=1)
    rec_xy = np.stack([xs[nsrc:], ys[nsrc:]], axis=1)
    f = np.empty((nsrc, nz, ny, nx), dtype=np.complex128)
    for r in range(nsrc):
        f[r] = point_source_plane(nz, ny, nx, 4, src_xy[r, 1], src_xy[r, 0])
    rng_true = np.random.default_rng(SEED_BASE + 5 + 1000)
    k2_true = (rng_true.uniform(0.05, 0.5, nlayers) * (1 + 0.02j)).astype(np.complex128)
    hx = rim_axis(160)
    rec_flat = 4 * ny * nx + rec_xy[:, 1] * nx + rec_xy[:, 0]
    return Workload("pml-192x192x128-2x2blocks-adjoint-grad", hx, hx.copy(), uniform_steps(nz),
                    z_begin, k2, default_ifaces(nx, 2), default_ifaces(ny, 2), f,
                    extra={"src_xy": src_xy, "rec_xy": rec_xy, "rec_flat": rec_flat.astype(np.int64),
                           "k2_true": k2_true})


def batched_models(n_models: int = 48):
    """Uneven batch: cubic grids from {64,96,128,160}^3, 8..24 layers, 4 frequencies, 2..16 RHS.

    Returns a list of (Workload, omegas).  Each model's k^2 is the base table; the
    frequency scales it by omega^2.
    """
    rng = np.random.default_rng(SEED_BASE + 4)
    sizes = np.array([64, 96, 128, 160])
    omegas = np.array([0.5, 1.0, 1.5, 2.0])
    out = []
    for mi in range(n_models):
        n = int(sizes[rng.integers(0, 4)])
        nl = int(rng.integers(8, 25))
        k2 = (rng.uniform(0.05, 0.5, nl) * (1 + 0.02j)).astype(np.complex128)
        inner = np.sort(rng.choice(np.arange(1, n), size=nl - 1, replace=False))
        z_begin = np.concatenate([[0], inner, [n]]).astype(np.int32)
        nrhs = int(rng.integers(2, 17))
        src = np.stack([rng.integers(4, n - 4, nrhs) for _ in range(3)], axis=1)
        f = np.empty((nrhs, n, n, n), dtype=np.complex128)
        for r in range(nrhs):
            f[r] = point_source_plane(n, n, n, src[r, 2], src[r, 1], src[r, 0])
        w = Workload(f"batch-model{mi}-{n}^3", uniform_steps(n), uniform_steps(n), uniform_steps(n),
                     z_begin, k2, default_ifaces(n, 2), default_ifaces(n, 2), f, precision="mixed")
        out.append((w, omegas.copy()))
    return out


def tiny_pml(nx=13, ny=11, nz=9, bx=2, by=2, nrhs=2, seed=7, sigma=False, rim=3, pml=2) -> Workload:
    """Small non-uniform problem with every feature of the big ones (for brute-force checks).

    x/y: a uniform core plus a `rim`-node geometric rim per side whose outer `pml`
    nodes have complex steps; z: ramped steps; layered complex k^2; optional sigma.
    """
    rng = np.random.default_rng(seed)
    hx = rim_axis(nx - 2 * rim, rim_nodes=rim, ratio=1.3, pml_nodes=pml)
    hy = rim_axis(ny - 2 * rim, rim_nodes=rim, ratio=1.3, pml_nodes=pml)
    hz = ramp_z(nz)
    nl = min(3, nz)
    k2 = (rng.uniform(0.05, 0.5, nl) * (1 + 0.05j)).astype(np.complex128)
    z_begin = np.array([(nz * L) // nl for L in range(nl + 1)], dtype=np.int32)
    f = _cnoise(rng, (nrhs, nz, ny, nx))
    sig = rng.uniform(0.5, 2.0, nl) if sigma else None
    return Workload(f"tiny-{nx}x{ny}x{nz}-{bx}x{by}", hx, hy, hz, z_begin, k2,
                    default_ifaces(nx, bx), default_ifaces(ny, by), f, sigma=sig)


NAMED = {
    "uniform32": single_block_32,
    "pml160": pml_160x160x128,
    "uniform320": uniform_320x320x200,
    "uniform320x40": uniform_320x320x40,
    "longz": long_z,
    "adjoint192": adjoint_192x192x128,
}
