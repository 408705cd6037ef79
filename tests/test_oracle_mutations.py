"""Plant plausible mistakes in the CPU oracle and check that a pin catches each one.

Every mutation is applied with monkeypatch to the oracle module only (on the
CPU); the pins are the functions of `oracle_pins`.
"""
import numpy as np
import pytest

from oracle import hz_oracle as O
from paper_1909_01299_gb300 import workloads as W
from tests import oracle_pins as pins

_orig = {name: getattr(O, name) for name in
         ["stiffness", "dual_lengths", "fwd", "inv", "z_coefficients", "mode_solve", "apply_A",
          "gen_eig", "sigma_half", "weighted_rhs", "adjoint_solve", "layer_gradient", "axis_blocks",
          "residual", "residual_perturbed", "rhs_gradient"]}


def _any_pin_fails():
    """Run the pins with their bounds; True if at least one is violated."""
    checks = [
        (lambda: pins.sine_eigenpair_error(9, 0.7), 1e-13),
        (lambda: pins.eigen_identity_error(W.rim_axis(12, rim_nodes=4, pml_nodes=2)), 1e-12),
        (lambda: pins.stencil_error(W.tiny_pml(5, 4, 6, 2, 2, sigma=True, rim=1, pml=1)), 1e-14),
        (lambda: pins.quadratic_error(W.tiny_pml(9, 8, 7, 2, 2), "blk"), 1e-12),
        (lambda: pins.quadratic_error(W.tiny_pml(9, 8, 7, 2, 2), "lu"), 1e-12),
        (lambda: pins.single_mode_error(blocks=(2, 2)), 1e-12),
        (lambda: pins.blk_vs_lu_error(W.tiny_pml(9, 8, 7, 2, 2, sigma=True)), 1e-12),
        (lambda: pins.adjoint_error(W.tiny_pml(9, 8, 7, 2, 2)), 1e-12),
        (lambda: pins.residual_error(W.tiny_pml(6, 5, 4, 2, 2, rim=1, pml=1)), 1e-12),
        (lambda: pins.residual_perturbed_error(W.tiny_pml(6, 5, 4, 2, 2, rim=1, pml=1, nrhs=2)), 1e-11),
        (lambda: pins.rhs_gradient_fd_error(W.tiny_pml(9, 8, 6, 2, 2, rim=3, pml=2, nrhs=2)), 1e-6),
    ]
    for fn, bound in checks:
        try:
            err = fn()
        except Exception:
            return True
        if not np.isfinite(err) or err > bound:
            return True
    return False


def test_unmutated_oracle_passes_all_pins():
    assert not _any_pin_fails()


def _mut_stiffness_sign(h, s_half=None):
    d, o = _orig["stiffness"](h, s_half)
    return d, -o


def _mut_stiffness_index(h, s_half=None):
    h = np.asarray(h, dtype=np.complex128)
    s = np.ones(len(h)) if s_half is None else np.asarray(s_half)
    flux = s / h
    return flux[:-1] + flux[1:], -flux[:-2]          # off-diagonal taken from the wrong step


def _mut_dual_lengths(h):
    return np.asarray(h)[:-1].copy()                   # no averaging of the two steps


def _mut_fwd_transposed(Wx, Wy, b):
    return _orig["fwd"](Wx, Wy.T, b) if Wy.shape[0] == Wy.shape[1] else _orig["fwd"](Wx, Wy, b)


def _mut_inv_transposed(Wx, Wy, t):
    return _orig["inv"](Wx.T, Wy, t)                    # W^T where W belongs


def _mut_z_k2_sign(P):
    tzd, tzo, mz, sz = _orig["z_coefficients"](P)
    k2n = P.node_values(P.k2)
    return tzd + 2 * k2n * mz, tzo, mz, sz


def _mut_mode_shift_mass(tzd, tzo, sz, s, rhs):
    return _orig["mode_solve"](tzd, tzo, np.ones_like(sz), s, rhs)   # shift without S_z


def _mut_gen_eig_conj(kd, ko, m):
    lam, Wm = _orig["gen_eig"](kd, ko, m)
    return lam, np.conj(Wm)


def _mut_sigma_arith(sig_nodes):
    s = np.asarray(sig_nodes, dtype=np.float64)
    out = np.empty(len(s) + 1)
    out[0], out[-1] = s[0], s[-1]
    out[1:-1] = s[:-1]                                  # upper node's sigma instead of the mean
    return out


def _mut_weighted_rhs(P, f):
    mx, my = O.dual_lengths(P.hx), O.dual_lengths(P.hy)
    return f * my[None, None, :, None] * mx[None, None, None, :]   # M_z dropped


def _mut_adjoint_no_conj(P, g, A=None, method="blk"):
    solver = O.block_solve_weighted if method == "blk" else O.solve_direct
    return solver(P, g, A)


def _mut_blocks_take_interface(n, ifaces):
    blocks = _orig["axis_blocks"](n, ifaces)
    if len(blocks) > 1:                                 # the first block swallows its interface node
        blocks[0] = (blocks[0][0], blocks[0][1] + 1)
    return blocks


def _mut_block_offdiag_shift(h, start, size):
    kd, ko = O.stiffness(h)
    m = O.dual_lengths(h)
    sl = slice(start, start + size)
    return O.gen_eig(kd[sl], np.roll(ko[start:start + size - 1], 1), m[sl])   # couplings one step along


def _mut_iface_mask_x_only(P):
    nz, ny, nx = P.shape
    mask = np.zeros((ny, nx), dtype=bool)
    mask[:, P.x_iface] = True                           # the y interfaces forgotten
    return mask


def _mut_residual_without_M(P, u, f, A=None):
    # the unweighted residual f - M^{-1} A u over ||f||
    _, mdiag = O.assemble(P)
    R = u.shape[0]
    r = f.reshape(R, -1) - O.apply_A(P, u, A).reshape(R, -1) / mdiag[None]
    return np.linalg.norm(r, axis=1) / np.linalg.norm(f.reshape(R, -1), axis=1)


def _mut_residual_f_denominator(P, u, f, A=None):
    # ||M f - A u|| over ||f|| instead of ||M f||
    R = u.shape[0]
    r = O.weighted_rhs(P, f) - O.apply_A(P, u, A)
    return np.linalg.norm(r.reshape(R, -1), axis=1) / np.linalg.norm(f.reshape(R, -1), axis=1)


def _mut_residual_pooled(P, u, f, A=None):
    # one norm over all right-hand sides, repeated per RHS
    r = O.weighted_rhs(P, f) - O.apply_A(P, u, A)
    return np.full(u.shape[0], np.linalg.norm(r) / np.linalg.norm(O.weighted_rhs(P, f)))


def _mut_residual_perturbed_dk2_sign(P, u, f, dk2, A=None):
    return _orig["residual_perturbed"](P, u, f, -np.asarray(dk2), A)


def _mut_residual_perturbed_dk2_unweighted(P, u, f, dk2, A=None):
    # dk2 u added without the control-volume weight
    R = u.shape[0]
    b = O.weighted_rhs(P, f)
    r = b - O.apply_A(P, u, A) + dk2[None] * u
    return np.linalg.norm(r.reshape(R, -1), axis=1) / np.linalg.norm(b.reshape(R, -1), axis=1)


def _mut_rhs_gradient_no_conj(P, lam):
    return np.conj(_orig["rhs_gradient"](P, np.conj(lam)))         # M lam instead of M^H lam


def _mut_rhs_gradient_no_weight(P, lam):
    return lam.copy()                                                # M dropped


MUTATIONS = {
    "rhs_gradient_without_conjugate": ("rhs_gradient", _mut_rhs_gradient_no_conj),
    "rhs_gradient_without_M": ("rhs_gradient", _mut_rhs_gradient_no_weight),
    "residual_without_M": ("residual", _mut_residual_without_M),
    "residual_f_denominator": ("residual", _mut_residual_f_denominator),
    "residual_pooled_over_rhs": ("residual", _mut_residual_pooled),
    "residual_perturbed_dk2_sign": ("residual_perturbed", _mut_residual_perturbed_dk2_sign),
    "residual_perturbed_dk2_unweighted": ("residual_perturbed", _mut_residual_perturbed_dk2_unweighted),
    "block_takes_its_interface_node": ("axis_blocks", _mut_blocks_take_interface),
    "block_offdiag_one_step_along": ("block_eig", _mut_block_offdiag_shift),
    "interfaces_x_only": ("iface_mask", _mut_iface_mask_x_only),
    "stiffness_offdiag_sign": ("stiffness", _mut_stiffness_sign),
    "stiffness_offdiag_index": ("stiffness", _mut_stiffness_index),
    "dual_lengths_not_averaged": ("dual_lengths", _mut_dual_lengths),
    "forward_transform_transposed": ("fwd", _mut_fwd_transposed),
    "inverse_transform_transposed": ("inv", _mut_inv_transposed),
    "k2_sign": ("z_coefficients", _mut_z_k2_sign),
    "mode_shift_without_Sz": ("mode_solve", _mut_mode_shift_mass),
    "eigenvectors_conjugated": ("gen_eig", _mut_gen_eig_conj),
    "sigma_half_node": ("sigma_half", _mut_sigma_arith),
    "rhs_without_Mz": ("weighted_rhs", _mut_weighted_rhs),
    "adjoint_without_conjugation": ("adjoint_solve", _mut_adjoint_no_conj),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(O, attr, fn)
    assert _any_pin_fails(), f"no pin caught the planted mistake {name}"


def test_gradient_without_conjugation_is_caught(monkeypatch):
    # layer gradient: dropping conj(lambda) breaks the finite-difference agreement
    def bad(P, u, lam):
        return _orig["layer_gradient"](P, u, np.conj(lam))
    monkeypatch.setattr(O, "layer_gradient", bad)
    w = W.tiny_pml(9, 8, 9, 2, 2, nrhs=1)
    rng = np.random.default_rng(11)
    rec = rng.choice(w.nx * w.ny * w.nz, 4, replace=False)
    d_obs = O.solve(O.Problem.from_workload(w, k2=w.k2 * 1.1), w.f).reshape(1, -1)[:, rec]
    P = O.Problem.from_workload(w)
    _, G, _, _ = O.misfit_gradient(P, w.f, rec, d_obs)
    eps = 1e-6

    def J_at(k2):
        u = O.solve(O.Problem.from_workload(w, k2=k2), w.f)
        return O.misfit(u, rec, d_obs)[0]
    e = np.zeros(len(w.k2), complex)
    e[0] = eps
    fd = (J_at(w.k2 + e) - J_at(w.k2 - e)) / (2 * eps)
    assert abs(G[0].real - fd) > 1e-6 * abs(fd)


@pytest.mark.parametrize("mistake", ["sign", "no_weight", "transposed"])
def test_perturbed_solve_mistakes_are_caught(mistake, monkeypatch):
    # plausible slips in the perturbed operator: the perturbation added with the wrong
    # sign, without the control-volume weight, or laid out transposed
    orig = O.solve_perturbed

    def bad(P, f, dk2, A=None):
        d = np.asarray(dk2)
        if mistake == "sign":
            d = -d
        elif mistake == "no_weight":
            mdiag = np.kron(O.dual_lengths(P.hz), np.kron(O.dual_lengths(P.hy), O.dual_lengths(P.hx)))
            d = d / mdiag.reshape(d.shape)
        else:
            d = np.ascontiguousarray(np.swapaxes(d, 1, 2)).reshape(d.shape)
        return orig(P, f, d, A)
    monkeypatch.setattr(O, "solve_perturbed", bad)
    w = W.tiny_pml(9, 8, 6, 2, 2, rim=2, pml=1, nrhs=2)
    assert pins.perturbed_bruteforce_error(w) > 1e-8
