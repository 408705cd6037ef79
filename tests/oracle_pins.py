"""Checks that pin the CPU oracle to facts outside itself.

Each function returns a scalar error (0 = exact).  The pins come from closed
forms, brute-force assembly from the stencil Eq. (fd), exact polynomial
solutions and invariants of the method of Sec. 2; none of them re-types an
oracle formula.  `test_oracle_pins.py` asserts the bounds and
`test_oracle_mutations.py` plants mistakes in the oracle and checks that some
pin catches each one.
"""
from __future__ import annotations

import numpy as np

from oracle import hz_oracle as O
from paper_1909_01299_gb300 import workloads as W


def sine_eigenpair_error(n=9, h=0.7):
    """Uniform real block: lambda_m = (4/h^2) sin^2(m pi / (2(N+1))),
    W_im = sqrt(2/((N+1)h)) sin(i m pi/(N+1)) (1-based i, m), up to sign per column."""
    steps = np.full(n + 1, h, dtype=np.complex128)
    lam, Wm = O.block_eig(steps, 0, n)
    m = np.arange(1, n + 1)
    lam_ref = 4.0 / h ** 2 * np.sin(m * np.pi / (2 * (n + 1))) ** 2
    i = np.arange(1, n + 1)
    W_ref = np.sqrt(2.0 / ((n + 1) * h)) * np.sin(np.outer(i, m) * np.pi / (n + 1))
    sign = np.sign((Wm * W_ref).sum(axis=0).real)
    e_lam = np.max(np.abs(lam - lam_ref)) / np.max(lam_ref)
    e_w = np.max(np.abs(Wm * sign[None, :] - W_ref))
    return max(e_lam, e_w)


def eigen_identity_error(h, start=0, size=None):
    """Relative ||K W - M W Lambda|| and ||W^T M W - I|| / cond(W) on a (block of an) axis."""
    n = len(h) - 1
    size = n - start if size is None else size
    lam, Wm = O.block_eig(h, start, size)
    kd, ko = O.stiffness(h)
    m = O.dual_lengths(h)
    sl = slice(start, start + size)
    K = O.tridiag_dense(kd[sl], ko[start:start + size - 1])
    M = np.diag(m[sl])
    e1 = np.linalg.norm(K @ Wm - M @ Wm @ np.diag(lam)) / (np.linalg.norm(K) * np.linalg.norm(Wm))
    e2 = np.linalg.norm(Wm.T @ M @ Wm - np.eye(size)) / np.linalg.cond(Wm)
    return max(e1, e2)


def stencil_matrix_loops(P: O.Problem):
    """Dense A assembled node by node from the 7-point finite-volume stencil Eq. (fd).

    Sign convention -div(sigma grad u) - k^2 u.  Steps: h[n] joins node n-1 and n.
    sigma: node value for the x/y fluxes, half-node value for the z flux.
    """
    nz, ny, nx = P.shape
    hx, hy, hz = P.hx, P.hy, P.hz
    hhx = [(hx[i] + hx[i + 1]) / 2 for i in range(nx)]
    hhy = [(hy[j] + hy[j + 1]) / 2 for j in range(ny)]
    hhz = [(hz[k] + hz[k + 1]) / 2 for k in range(nz)]
    layer_of = [max(L for L in range(len(P.z_begin) - 1) if P.z_begin[L] <= k) for k in range(nz)]
    k2 = [P.k2[layer_of[k]] for k in range(nz)]
    sig = [1.0 if P.sigma is None else P.sigma[layer_of[k]] for k in range(nz)]

    def sig_step(n):          # sigma on the step between node n-1 and node n
        if n == 0:
            return sig[0]
        if n == nz:
            return sig[nz - 1]
        a, b = sig[n - 1], sig[n]
        return 2 * a * b / (a + b)

    N = nx * ny * nz
    A = np.zeros((N, N), dtype=np.complex128)
    idx = lambda i, j, k: (k * ny + j) * nx + i
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = idx(i, j, k)
                # x fluxes: sigma_k * hhat_y * hhat_z * [(u_i - u_{i-1})/h_i - (u_{i+1} - u_i)/h_{i+1}]
                cx = sig[k] * hhy[j] * hhz[k]
                A[row, row] += cx * (1 / hx[i] + 1 / hx[i + 1])
                if i > 0:
                    A[row, idx(i - 1, j, k)] -= cx / hx[i]
                if i < nx - 1:
                    A[row, idx(i + 1, j, k)] -= cx / hx[i + 1]
                cy = sig[k] * hhx[i] * hhz[k]
                A[row, row] += cy * (1 / hy[j] + 1 / hy[j + 1])
                if j > 0:
                    A[row, idx(i, j - 1, k)] -= cy / hy[j]
                if j < ny - 1:
                    A[row, idx(i, j + 1, k)] -= cy / hy[j + 1]
                cz = hhx[i] * hhy[j]
                A[row, row] += cz * (sig_step(k) / hz[k] + sig_step(k + 1) / hz[k + 1])
                if k > 0:
                    A[row, idx(i, j, k - 1)] -= cz * sig_step(k) / hz[k]
                if k < nz - 1:
                    A[row, idx(i, j, k + 1)] -= cz * sig_step(k + 1) / hz[k + 1]
                A[row, row] -= k2[k] * hhx[i] * hhy[j] * hhz[k]
    return A


def stencil_error(w):
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    Ad = stencil_matrix_loops(P)
    return np.max(np.abs(A.toarray() - Ad)) / np.max(np.abs(Ad))


def quadratic_solution(w):
    """Exact discrete solution for sigma = 1 on any (complex) tensor grid.

    With node coordinates x_i = sum_{n<=i} h_n (Dirichlet nodes at 0 and L) and
    q(x) = x (L - x), the three-point finite-volume difference of a quadratic is
    exact: -(K q)_i / hhat_i = q'' = -2.  Hence u = qx qy qz solves A u = M f for
    f = 2 (qy qz + qx qz + qx qy) - k^2(z) qx qy qz, node by node.
    """
    def q(h):
        x = np.cumsum(h)[:-1]
        L = np.sum(h)
        return x * (L - x)
    qx, qy, qz = q(w.hx), q(w.hy), q(w.hz)
    k2n = w.k2_nodes()
    Qx = qx[None, None, :]
    Qy = qy[None, :, None]
    Qz = qz[:, None, None]
    u = Qx * Qy * Qz
    f = 2 * (Qy * Qz + Qx * Qz + Qx * Qy) - k2n[:, None, None] * u
    return u, f


def quadratic_error(w, method="blk"):
    assert w.sigma is None
    u_ex, f = quadratic_solution(w)
    P = O.Problem.from_workload(w)
    solver = O.block_solve if method == "blk" else O.solve
    u = solver(P, f[None])
    return np.linalg.norm(u[0] - u_ex) / np.linalg.norm(u_ex)


def single_mode_error(n=(10, 9, 8), h=(1.0, 0.8, 1.3), k2=0.3 + 0.02j, modes=(3, 2, 5), blocks=(1, 1)):
    """Uniform grid, constant k^2: f = sin(l pi x) sin(m pi y) sin(n pi z) gives
    u = f / (lambda_l + mu_m + nu_n - k^2) with the sine eigenvalues of each axis."""
    nx, ny, nz = n
    hx, hy, hz = h
    l, m, nn = modes
    sx = np.sin(l * np.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(m * np.pi * np.arange(1, ny + 1) / (ny + 1))
    sz = np.sin(nn * np.pi * np.arange(1, nz + 1) / (nz + 1))
    lam = lambda mm, N, hh: 4.0 / hh ** 2 * np.sin(mm * np.pi / (2 * (N + 1))) ** 2
    f = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    u_ex = f / (lam(l, nx, hx) + lam(m, ny, hy) + lam(nn, nz, hz) - k2)
    P = O.Problem(np.full(nx + 1, hx, complex), np.full(ny + 1, hy, complex),
                  np.full(nz + 1, hz, complex), [0, nz], [k2], None,
                  W.default_ifaces(nx, blocks[0]), W.default_ifaces(ny, blocks[1]))
    u = O.block_solve(P, f[None].astype(complex))[0]
    return np.linalg.norm(u - u_ex) / np.linalg.norm(u_ex)


def blk_vs_lu_error(w):
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    u1 = O.solve(P, w.f, A)
    u2 = O.block_solve(P, w.f, A)
    return np.linalg.norm(u1 - u2) / np.linalg.norm(u1)


def residual_support_error(w):
    """After steps 1-3, r = b - A v vanishes off the interfaces (Sec. 2, residual support)."""
    P = O.Problem.from_workload(w)
    st = {}
    O.block_solve(P, w.f, stages=st)
    mask = O.iface_mask(P)
    off = np.where(mask[None, None], 0.0, st["r_full"])
    on = np.where(mask[None, None], st["r_full"], 0.0)
    return np.max(np.abs(off)) / np.max(np.abs(on))


def adjoint_error(w):
    """A^{-H} g from the conjugation identity against a direct solve with conj(A)^T."""
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    g = w.f
    lam = O.adjoint_solve(P, g, A, method="blk")
    AH = A.conj().T.tocsc()
    import scipy.sparse.linalg as spla
    R = g.shape[0]
    ref = spla.spsolve(AH, g.reshape(R, -1).T).T.reshape(g.shape)
    return np.linalg.norm(lam - ref) / np.linalg.norm(ref)


def perturbation(P: O.Problem, amp=0.15, seed=3):
    """A local complex perturbation of k^2 on a box in the middle of the grid (zero elsewhere)."""
    nz, ny, nx = P.shape
    rng = np.random.default_rng(seed)
    d = np.zeros((nz, ny, nx), dtype=np.complex128)
    kz, jy, ix = slice(nz // 4, 3 * nz // 4 + 1), slice(ny // 4, 3 * ny // 4 + 1), slice(nx // 4, 3 * nx // 4 + 1)
    shape = d[kz, jy, ix].shape
    d[kz, jy, ix] = amp * (rng.uniform(0.5, 1.0, shape) + 0.1j * rng.uniform(0.0, 1.0, shape))
    return d


def perturbed_bruteforce_error(w, amp=0.15):
    """Perturbed operator assembled node by node from the stencil (Eq. (fd) with k^2 -> k^2 + dk2
    at each node) and solved densely, against the oracle's perturbed solve."""
    P = O.Problem.from_workload(w)
    dk2 = perturbation(P, amp)
    Ad = stencil_matrix_loops(P)
    nz, ny, nx = P.shape
    hhx = [(P.hx[i] + P.hx[i + 1]) / 2 for i in range(nx)]
    hhy = [(P.hy[j] + P.hy[j + 1]) / 2 for j in range(ny)]
    hhz = [(P.hz[k] + P.hz[k + 1]) / 2 for k in range(nz)]
    b = np.zeros((w.f.shape[0], nz * ny * nx), dtype=np.complex128)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = (k * ny + j) * nx + i
                vol = hhx[i] * hhy[j] * hhz[k]
                Ad[row, row] -= dk2[k, j, i] * vol
                b[:, row] = w.f[:, k, j, i] * vol
    ref = np.linalg.solve(Ad, b.T).T.reshape(w.f.shape)
    u = O.solve_perturbed(P, w.f, dk2)
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def perturbed_born_series_error(w, amp=0.02, terms=40):
    """For a weak perturbation the solution is the Born (Neumann) series
    u = sum_n (S dk2)^n S f with S the layered solve; only layered solves are used."""
    P = O.Problem.from_workload(w)
    dk2 = perturbation(P, amp)
    A, _ = O.assemble(P)
    term = O.solve(P, w.f, A)
    u = term.copy()
    for _ in range(terms):
        term = O.solve(P, dk2[None] * term, A)
        u += term
    ref = O.solve_perturbed(P, w.f, dk2, A)
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def _loop_weights(P: O.Problem):
    """Control-volume weight hhat^x_i hhat^y_j hhat^z_k of every node, written out node by node."""
    nz, ny, nx = P.shape
    vol = np.empty((nz, ny, nx), dtype=np.complex128)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                vol[k, j, i] = ((P.hx[i] + P.hx[i + 1]) / 2) * ((P.hy[j] + P.hy[j + 1]) / 2) \
                    * ((P.hz[k] + P.hz[k + 1]) / 2)
    return vol


def _loop_relres(Ad, vol, u, f):
    """Per-RHS ||b - Ad u|| / ||b|| with b = vol * f, from the node-by-node matrix Ad."""
    R = u.shape[0]
    out = np.empty(R)
    for r in range(R):
        b = (vol * f[r]).ravel()
        out[r] = np.linalg.norm(b - Ad @ u[r].ravel()) / np.linalg.norm(b)
    return out


def residual_error(w, scales=(1e-1, 1e-4)):
    """The oracle's relative residual ||M f - A u|| / ||M f|| (per RHS) against the same quantity
    formed from the node-by-node stencil matrix and control-volume weights, on
    u = exact quadratic solution + a seeded perturbation of a different size per RHS (so that a
    residual pooled over RHS, taken without M, or divided by ||f|| instead of ||M f||, differs).
    Also u = 0 must give exactly 1 and the exact solution a residual at the rounding level."""
    P = O.Problem.from_workload(w)
    u_ex, f1 = quadratic_solution(w)
    rng = np.random.default_rng(21)
    R = len(scales)
    f = np.stack([f1 * (1.0 + 0.5 * r) for r in range(R)])
    u = np.stack([u_ex * (1.0 + 0.5 * r) for r in range(R)])
    for r, s in enumerate(scales):
        u[r] = u[r] + s * np.max(np.abs(u_ex)) * (rng.standard_normal(u_ex.shape)
                                                  + 1j * rng.standard_normal(u_ex.shape))
    Ad = stencil_matrix_loops(P)
    vol = _loop_weights(P)
    ref = _loop_relres(Ad, vol, u, f)
    got = O.residual(P, u, f)
    e = np.max(np.abs(got - ref) / ref)
    zero = O.residual(P, np.zeros_like(u), f)
    e = max(e, np.max(np.abs(zero - 1.0)))
    exact = O.residual(P, u_ex[None], f1[None])
    return max(e, float(exact[0]) * 1e-2)        # exact solution: residual <= 1e-10 passes


def residual_perturbed_error(w, amp=0.15):
    """The oracle's perturbed residual ||M f - (A - diag(M dk2)) u|| / ||M f|| against the same
    quantity from the node-by-node perturbed matrix (stencil with k^2 -> k^2 + dk2 per node),
    for a seeded u that solves nothing (so every term of the residual counts)."""
    P = O.Problem.from_workload(w)
    dk2 = perturbation(P, amp)
    Ad = stencil_matrix_loops(P)
    vol = _loop_weights(P)
    nz, ny, nx = P.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = (k * ny + j) * nx + i
                Ad[row, row] -= dk2[k, j, i] * vol[k, j, i]
    rng = np.random.default_rng(22)
    u = rng.standard_normal(w.f.shape) + 1j * rng.standard_normal(w.f.shape)
    # a u close to the solution too: the residual is then dominated by the dk2 term's balance
    u[0] = O.solve_perturbed(P, w.f[:1], dk2)[0] * (1 + 1e-3)
    ref = _loop_relres(Ad, vol, u, w.f)
    got = O.residual_perturbed(P, u, w.f, dk2)
    return np.max(np.abs(got - ref) / ref)


def rhs_gradient_fd_error(w, entries=((0, 1, 2, 3), (0, 3, 1, 2), (1, 2, 4, 1)), eps=1e-6):
    """Central differences of J(f) = 1/2 sum |P u(f) - d|^2 (u by sparse LU) in Re f and Im f
    at a few entries against the oracle's right-hand-side gradient of the adjoint state."""
    P = O.Problem.from_workload(w)
    A, _ = O.assemble(P)
    rng = np.random.default_rng(31)
    rec = rng.choice(w.nx * w.ny * w.nz, 6, replace=False)
    R = w.f.shape[0]
    d = rng.standard_normal((R, 6)) * 1e-2 + 0j

    def J(f):
        return O.misfit(O.solve(P, f, A), rec, d)[0]

    _, g = O.misfit(O.solve(P, w.f, A), rec, d)
    gr = O.rhs_gradient(P, O.adjoint_solve(P, g, A, method="lu"))
    err = 0.0
    for (r, k, j, i) in entries:
        e = np.zeros_like(w.f)
        e[r, k, j, i] = eps
        fd_re = (J(w.f + e) - J(w.f - e)) / (2 * eps)
        fd_im = (J(w.f + 1j * e) - J(w.f - 1j * e)) / (2 * eps)
        scale = abs(fd_re) + abs(fd_im)
        err = max(err, abs(gr[r, k, j, i].real - fd_re) / scale, abs(gr[r, k, j, i].imag - fd_im) / scale)
    return err
