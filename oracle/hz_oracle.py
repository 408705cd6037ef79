"""CPU FP64 oracle for the layered-medium Helmholtz solve (Druskin & Zaslavsky, Sec. 2).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
CPU-baseline leg of the benchmark may import this module; the product path
never does, and this module imports nothing from the product.

It is deliberately plain: numpy/scipy complex128 throughout, no blocking,
fusion or reordering beyond what the paper's definitions and algorithm state.

Problem (Eq. (wave2) with the readings below)
---------------------------------------------
    -sigma(z) (u_xx + u_yy) - (sigma(z) u_z)_z - k^2(z) u = f

on a tensor grid S_x x S_y x S_z with homogeneous Dirichlet conditions.  Each
axis has N interior nodes and N+1 (possibly complex, "PML") steps h_0..h_N;
step h_n joins node n-1 to node n.  The finite-volume scheme Eq. (fd) in
Kronecker form Eq. (fdmtr) reads (vector index k-major, then j, then i)

    A = (S_z (x) My (x) Kx) + (S_z (x) Ky (x) Mx) + (Tz (x) My (x) Mx),
    A u = (Mz (x) My (x) Mx) f,

with M_d = diag(hhat), hhat_i = (h_i + h_{i+1}) / 2 the control-volume edge
lengths, K_d the 3-point stiffness of -d^2/dd^2 (diagonal 1/h_i + 1/h_{i+1},
off-diagonal -1/h_{i+1}), S_z = diag(sigma_k hhat^z_k), and
Tz = K_z^sigma - diag(k^2_k hhat^z_k) with sigma at half nodes in K_z^sigma.

Readings of the paper taken here (each is listed in the design notes):
  * Eq. (wave2) has lambda u with real constant lambda; here lambda -> k^2(z),
    node-based and complex, and the equation's overall sign is flipped so that
    A = -(paper's A) with lambda = k^2.  Separability is unchanged because k^2
    varies only with z.
  * The paper's transformed quantities (W)^* (x) (W)^* (x) I use the
    transpose, not the conjugate transpose: the pencils (K_d, M_d) are complex
    symmetric.  With the normalisation W^T M W = I the forward transform of a
    weighted vector b = M f is W^T b and the inverse transform is W.
  * sigma at the half node of a step inside a layer is that layer's sigma; on
    a step joining two layers it is the harmonic mean of the two nodes'
    sigma; the two boundary steps take the adjacent node's sigma.
  * Steps 5 and 6 of the algorithm carry the typos "v" for "w" and
    "u~" for "v~"; they are read as w~ and v~.
  * Step 6 moves the known interface values to the right-hand side:
    A_{int,int} w = -A_{int,iface} w_iface in each block.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------

class Problem:
    """Grid, layered coefficients and block partition, as plain arrays.

    hx, hy, hz : complex steps, lengths Nx+1, Ny+1, Nz+1.
    z_begin    : nlayers+1 node indices; layer L holds z nodes [z_begin[L], z_begin[L+1]).
    k2         : per-layer complex k^2.
    sigma      : per-layer positive sigma, or None for sigma = 1.
    x_iface, y_iface : interface node indices (sorted, strictly inside the axis).
    """

    def __init__(self, hx, hy, hz, z_begin, k2, sigma=None, x_iface=(), y_iface=()):
        self.hx = np.asarray(hx, dtype=np.complex128)
        self.hy = np.asarray(hy, dtype=np.complex128)
        self.hz = np.asarray(hz, dtype=np.complex128)
        self.z_begin = np.asarray(z_begin, dtype=np.int64)
        self.k2 = np.asarray(k2, dtype=np.complex128)
        self.sigma = None if sigma is None else np.asarray(sigma, dtype=np.float64)
        self.x_iface = np.asarray(x_iface, dtype=np.int64)
        self.y_iface = np.asarray(y_iface, dtype=np.int64)

    @classmethod
    def from_workload(cls, w, k2=None):
        return cls(w.hx, w.hy, w.hz, w.z_begin, w.k2 if k2 is None else k2, w.sigma,
                   w.x_iface, w.y_iface)

    @property
    def shape(self):
        return (len(self.hz) - 1, len(self.hy) - 1, len(self.hx) - 1)

    def node_values(self, per_layer):
        """Expand a per-layer table to the Nz z nodes."""
        nz = len(self.hz) - 1
        out = np.empty(nz, dtype=np.asarray(per_layer).dtype)
        for L in range(len(self.z_begin) - 1):
            out[self.z_begin[L]:self.z_begin[L + 1]] = per_layer[L]
        return out


# ---------------------------------------------------------------------------
# 1D operators: Eq. (fd), Eq. (fdmtr)
# ---------------------------------------------------------------------------

def dual_lengths(h):
    """hhat_i = (h_i + h_{i+1}) / 2: lengths of the control-volume edges (Eq. (fd))."""
    h = np.asarray(h)
    return 0.5 * (h[:-1] + h[1:])


def stiffness(h, s_half=None):
    """3-point stiffness of -d/dx(s du/dx) on N nodes from N+1 steps (Eq. (fd)).

    Returns (diag, off): diag_i = s_i/h_i + s_{i+1}/h_{i+1}, off_i = K[i, i+1] = -s_{i+1}/h_{i+1}.
    """
    h = np.asarray(h, dtype=np.complex128)
    s = np.ones(len(h)) if s_half is None else np.asarray(s_half)
    flux = s / h
    return flux[:-1] + flux[1:], -flux[1:-1]


def tridiag_dense(diag, off):
    return np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)


def sigma_half(sig_nodes):
    """sigma on the Nz+1 z steps from node values (harmonic mean across a layer change)."""
    s = np.asarray(sig_nodes, dtype=np.float64)
    out = np.empty(len(s) + 1)
    out[0], out[-1] = s[0], s[-1]
    out[1:-1] = 2.0 * s[:-1] * s[1:] / (s[:-1] + s[1:])
    return out


def z_coefficients(P: Problem):
    """z-direction pieces: Tz (diag, off), Mz = hhat^z and S_z = sigma hhat^z (Eq. (fdmtr))."""
    nz = len(P.hz) - 1
    sig = np.ones(nz) if P.sigma is None else P.node_values(P.sigma)
    mz = dual_lengths(P.hz)
    kd, ko = stiffness(P.hz, sigma_half(sig))
    k2n = P.node_values(P.k2)
    return kd - k2n * mz, ko, mz, sig * mz


def assemble(P: Problem):
    """Sparse A of Eq. (fdmtr) (vector index (k, j, i), i fastest) and the diagonal of M."""
    kxd, kxo = stiffness(P.hx)
    kyd, kyo = stiffness(P.hy)
    tzd, tzo, mz, sz = z_coefficients(P)
    mx, my = dual_lengths(P.hx), dual_lengths(P.hy)
    Kx = sp.diags([kxo, kxd, kxo], [-1, 0, 1], format="csr")
    Ky = sp.diags([kyo, kyd, kyo], [-1, 0, 1], format="csr")
    Tz = sp.diags([tzo, tzd, tzo], [-1, 0, 1], format="csr")
    Mx, My = sp.diags(mx), sp.diags(my)
    Sz = sp.diags(sz)
    A = (sp.kron(Sz, sp.kron(My, Kx)) + sp.kron(Sz, sp.kron(Ky, Mx))
         + sp.kron(Tz, sp.kron(My, Mx)))
    mdiag = np.kron(mz, np.kron(my, mx))
    return A.tocsr(), mdiag


def weighted_rhs(P: Problem, f):
    """b = (Mz (x) My (x) Mx) f for f of shape (nrhs, Nz, Ny, Nx)."""
    mx, my, mz = dual_lengths(P.hx), dual_lengths(P.hy), dual_lengths(P.hz)
    return f * mz[None, :, None, None] * my[None, None, :, None] * mx[None, None, None, :]


def apply_A(P: Problem, u, A=None):
    """A u for u of shape (nrhs, Nz, Ny, Nx)."""
    if A is None:
        A, _ = assemble(P)
    R = u.shape[0]
    return (A @ u.reshape(R, -1).T).T.reshape(u.shape)


def residual(P: Problem, u, f, A=None):
    """Per-RHS relative residual ||M f - A u||_2 / ||M f||_2 (weighted form)."""
    b = weighted_rhs(P, f)
    r = b - apply_A(P, u, A)
    R = u.shape[0]
    return (np.linalg.norm(r.reshape(R, -1), axis=1) / np.linalg.norm(b.reshape(R, -1), axis=1))


def solve_direct(P: Problem, b, A=None):
    """O-LU: x = A^{-1} b by sparse LU (b already weighted), shape (nrhs, Nz, Ny, Nx)."""
    if A is None:
        A, _ = assemble(P)
    lu = spla.splu(A.tocsc())
    R = b.shape[0]
    x = lu.solve(np.ascontiguousarray(b.reshape(R, -1).T))
    return x.T.reshape(b.shape)


def solve(P: Problem, f, A=None):
    """u = A^{-1} (M f) by sparse LU: the plain definition of the solution."""
    return solve_direct(P, weighted_rhs(P, f), A)


# ---------------------------------------------------------------------------
# Generalised eigenpairs (the display after Eq. (fdmtrprj); global ones before Eq. (fdmtrprjfrerr))
# ---------------------------------------------------------------------------

def gen_eig(kd, ko, m):
    """Eigenpairs of K W = M W Lambda with W^T M W = I, sorted by (Re, Im) of lambda.

    K is the complex-symmetric tridiagonal (kd, ko), M = diag(m).  Eigenvectors
    come from numpy's dense eigen-solver on M^{-1} K and are scaled by the
    principal square root of w^T M w (after M-orthogonalisation, see below).
    """
    K = tridiag_dense(kd, ko)
    m = np.asarray(m)
    lam, V = np.linalg.eig(K / m[:, None])
    order = np.lexsort((lam.imag, lam.real))
    lam, V = lam[order], V[:, order]
    # Eigenvectors of distinct eigenvalues are M-orthogonal in exact arithmetic;
    # a dense solver leaves an O(eps / gap) defect for nearly equal eigenvalues
    # (the PML axes have such pairs).  Modified Gram-Schmidt in the bilinear
    # form <a, b> = a^T M b restores W^T M W = I without changing the span of
    # any cluster.
    W = V.copy()
    for j in range(W.shape[1]):
        for _ in range(2):
            c = W[:, :j].T @ (m * W[:, j])
            W[:, j] -= W[:, :j] @ c
        W[:, j] /= np.sqrt(np.sum(W[:, j] * m * W[:, j]))
    return lam, W


def axis_blocks(n, ifaces):
    """(start, size) of the interior-node runs between interfaces p_1 < ... < p_{B-1}."""
    edges = [-1] + [int(p) for p in ifaces] + [n]
    return [(edges[b] + 1, edges[b + 1] - edges[b] - 1) for b in range(len(edges) - 1)]


def block_eig(h, start, size):
    """Eigenpairs of the block pencil P K P, P M P (Dirichlet at the block's bounding nodes)."""
    kd, ko = stiffness(h)
    m = dual_lengths(h)
    sl = slice(start, start + size)
    return gen_eig(kd[sl], ko[start:start + size - 1], m[sl])


# ---------------------------------------------------------------------------
# Mode-space z solves: Eq. (fdmtrprjfr) / Eq. (fdmtrprjfrerr)
# ---------------------------------------------------------------------------

def mode_solve(tzd, tzo, sz, s, rhs):
    """Solve (Tz + s_lm S_z) x = rhs for every mode.

    s   : (Mm, Ml) mode shifts lambda_l + mu_m.
    rhs : (R, Nz, Mm, Ml).
    Each system is a complex tridiagonal solved by pivoted banded LU.
    """
    R, nz, Mm, Ml = rhs.shape
    out = np.empty_like(rhs)
    ab = np.zeros((3, nz), dtype=np.complex128)
    ab[0, 1:] = tzo
    ab[2, :-1] = tzo
    for m in range(Mm):
        for l in range(Ml):
            ab[1, :] = tzd + s[m, l] * sz
            out[:, :, m, l] = sla.solve_banded((1, 1), ab, rhs[:, :, m, l].T,
                                               check_finite=False).T
    return out


def fwd(Wx, Wy, b):
    """(Wx^T (x) Wy^T (x) I) b per plane: out[r,k,m,l] = sum_ij Wx[i,l] Wy[j,m] b[r,k,j,i]."""
    return np.einsum("il,jm,rkji->rkml", Wx, Wy, b, optimize=True)


def inv(Wx, Wy, t):
    """(Wx (x) Wy (x) I) t per plane: out[r,k,j,i] = sum_lm Wx[i,l] Wy[j,m] t[r,k,m,l]."""
    return np.einsum("il,jm,rkml->rkji", Wx, Wy, t, optimize=True)


# ---------------------------------------------------------------------------
# O-BLK: the seven steps of the algorithm in Sec. 2
# ---------------------------------------------------------------------------

def iface_mask(P: Problem):
    nz, ny, nx = P.shape
    mask = np.zeros((ny, nx), dtype=bool)
    mask[:, P.x_iface] = True
    mask[P.y_iface, :] = True
    return mask


def block_solve_weighted(P: Problem, b, A=None, stages=None):
    """x = A^{-1} b by the block algorithm of Sec. 2 (b already weighted, e.g. b = M f).

    Follows the paper's seven steps in order; `stages`, if a dict, receives the
    intermediate quantities (v, r, w on the interfaces, ...) for stage tests.
    """
    if A is None:
        A, _ = assemble(P)
    R, nz, ny, nx = b.shape
    tzd, tzo, mz, sz = z_coefficients(P)
    xb, yb = axis_blocks(nx, P.x_iface), axis_blocks(ny, P.y_iface)
    ex = [block_eig(P.hx, s0, n) for s0, n in xb]
    ey = [block_eig(P.hy, s0, n) for s0, n in yb]
    mask = iface_mask(P)

    # Steps 1-3: per block, f~ = W^T b, v~ from the mode systems, v by the inverse transform.
    vt = {}
    v = np.zeros_like(b)
    for bx, (x0, nbx) in enumerate(xb):
        for by, (y0, nby) in enumerate(yb):
            lx, Wx = ex[bx]
            ly, Wy = ey[by]
            ft = fwd(Wx, Wy, b[:, :, y0:y0 + nby, x0:x0 + nbx])              # step 1
            s = lx[None, :] + ly[:, None]
            vt[bx, by] = mode_solve(tzd, tzo, sz, s, ft)                      # step 2
            v[:, :, y0:y0 + nby, x0:x0 + nbx] = inv(Wx, Wy, vt[bx, by])       # step 3
    # Step 4: r = b - A v, supported on the interfaces.
    r_full = b - apply_A(P, v, A)
    r = np.where(mask[None, None], r_full, 0.0)
    # Step 5: w on the interfaces from the global eigen-transform.
    kxd, kxo = stiffness(P.hx)
    kyd, kyo = stiffness(P.hy)
    lgx, Wgx = gen_eig(kxd, kxo, dual_lengths(P.hx))
    lgy, Wgy = gen_eig(kyd, kyo, dual_lengths(P.hy))
    rt = fwd(Wgx, Wgy, r)
    wt = mode_solve(tzd, tzo, sz, lgx[None, :] + lgy[:, None], rt)
    w_iface = np.where(mask[None, None], inv(Wgx, Wgy, wt), 0.0)
    # Step 6: per block, w~ from A_int w = -A_{int,iface} w_iface.
    g = -apply_A(P, w_iface, A)
    u = w_iface.copy()
    for bx, (x0, nbx) in enumerate(xb):
        for by, (y0, nby) in enumerate(yb):
            lx, Wx = ex[bx]
            ly, Wy = ey[by]
            gt = fwd(Wx, Wy, g[:, :, y0:y0 + nby, x0:x0 + nbx])
            s = lx[None, :] + ly[:, None]
            wtb = mode_solve(tzd, tzo, sz, s, gt)
            # Step 7: u = W (v~ + w~) inside the block; u = w on the interfaces.
            u[:, :, y0:y0 + nby, x0:x0 + nbx] = inv(Wx, Wy, vt[bx, by] + wtb)
    if stages is not None:
        stages.update(v=v, r_full=r_full, r=r, w_iface=w_iface, g=g,
                      eig_x=ex, eig_y=ey, eig_gx=(lgx, Wgx), eig_gy=(lgy, Wgy))
    return u


def block_solve(P: Problem, f, A=None, stages=None):
    """u = A^{-1} (M f) by the block algorithm (O-BLK)."""
    return block_solve_weighted(P, weighted_rhs(P, f), A, stages)


# ---------------------------------------------------------------------------
# Adjoint and layer gradient (derived from the symmetry of Eq. (fdmtr))
# ---------------------------------------------------------------------------

def adjoint_solve(P: Problem, g, A=None, method="blk"):
    """lambda = A^{-H} g.  A is complex symmetric, so A^H = conj(A) and
    lambda = conj(A^{-1} conj(g)); g is already in the weighted space."""
    solver = block_solve_weighted if method == "blk" else solve_direct
    return np.conj(solver(P, np.conj(g), A))


def layer_gradient(P: Problem, u, lam):
    """G_L = sum_rhs sum_{k in L} hhat^z_k sum_ij conj(lam_ijk) hhat^x_i hhat^y_j u_ijk.

    This is <lam, (dA/dk^2_L) u> up to sign: dA/dk^2_L = -Mx (x) My (x) diag(hhat^z 1_{k in L}),
    so for J = 1/2 sum |P u - d|^2 the derivative is dJ = Re(G_L dk^2_L),
    i.e. dJ/dRe k^2_L = Re G_L and dJ/dIm k^2_L = -Im G_L.
    """
    mx, my, mz = dual_lengths(P.hx), dual_lengths(P.hy), dual_lengths(P.hz)
    prod = np.conj(lam) * u * my[None, None, :, None] * mx[None, None, None, :]
    p_k = prod.sum(axis=(0, 2, 3)) * mz
    nl = len(P.z_begin) - 1
    return np.array([p_k[P.z_begin[L]:P.z_begin[L + 1]].sum() for L in range(nl)])


def rhs_gradient(P: Problem, lam):
    """M^H lam: the gradient in f of a real objective J(u) whose adjoint state is lam.

    The solve is u = A^{-1} M f with M = Mz (x) My (x) Mx diagonal (Eq. (fdmtr)), so
    du = A^{-1} M df and the adjoint of that map sends lam = A^{-H} g to M^H lam, i.e.
    conj(hhat^x_i hhat^y_j hhat^z_k) lam_ijk.  With g = dJ/du* in PyTorch's scaling
    (g = P^T (P u - d) for J = 1/2 sum |P u - d|^2) the result gr satisfies
    dJ/dRe f = Re gr and dJ/dIm f = Im gr.
    """
    mx, my, mz = dual_lengths(P.hx), dual_lengths(P.hy), dual_lengths(P.hz)
    w = mz[:, None, None] * my[None, :, None] * mx[None, None, :]
    return np.conj(w)[None] * lam


def misfit(u, rec_flat, d_obs):
    """J = 1/2 sum_s sum_rec |u_s(rec) - d_s,rec|^2 and the adjoint source g_s = P^T (P u_s - d_s)."""
    R = u.shape[0]
    flat = u.reshape(R, -1)
    res = flat[:, rec_flat] - d_obs
    J = 0.5 * float(np.sum(np.abs(res) ** 2))
    g = np.zeros_like(flat)
    g[:, rec_flat] = res
    return J, g.reshape(u.shape)


def misfit_gradient(P: Problem, f, rec_flat, d_obs, method="blk"):
    """J and G (per layer) through one forward and one adjoint solve per RHS."""
    A, _ = assemble(P)
    solver = block_solve if method == "blk" else solve
    u = solver(P, f, A)
    J, g = misfit(u, rec_flat, d_obs)
    lam = adjoint_solve(P, g, A, method)
    return J, layer_gradient(P, u, lam), u, lam


# ---------------------------------------------------------------------------
# Layered medium with a local perturbation (Sec. 1: the layered solve as a fast
# preconditioner for media with embedded inhomogeneities)
# ---------------------------------------------------------------------------

def solve_perturbed(P: Problem, f, dk2, A=None):
    """u of -div(sigma grad u) - (k^2(z) + dk2(x, y, z)) u = f by sparse LU.

    dk2 is node-based, shape (Nz, Ny, Nx).  The perturbation adds -dk2 to the k^2 term of
    every node, i.e. subtracts diag(M dk2) from A (the k^2 term of Eq. (fdmtr) is
    -k^2 times the control-volume weight):  (A - diag(M dk2)) u = M f.
    """
    if A is None:
        A, mdiag = assemble(P)
    else:
        mdiag = np.kron(dual_lengths(P.hz), np.kron(dual_lengths(P.hy), dual_lengths(P.hx)))
    Ap = (A - sp.diags(mdiag * np.asarray(dk2, dtype=np.complex128).ravel())).tocsc()
    return solve_direct(P, weighted_rhs(P, f), Ap)


def residual_perturbed(P: Problem, u, f, dk2, A=None):
    """Per-RHS ||M f - (A - diag(M dk2)) u|| / ||M f||."""
    if A is None:
        A, _ = assemble(P)
    b = weighted_rhs(P, f)
    r = b - apply_A(P, u, A) + weighted_rhs(P, dk2[None] * u)
    R = u.shape[0]
    return (np.linalg.norm(r.reshape(R, -1), axis=1) / np.linalg.norm(b.reshape(R, -1), axis=1))

