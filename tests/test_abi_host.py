"""The C ABI library on the CPU: it loads, exports every declared symbol, and its
host-side eigen-solver (used by every plan) meets the closed forms and identities."""
import os
import re

import numpy as np
import pytest

from paper_1909_01299_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hz():
    from paper_1909_01299_gb300 import build
    build.build()
    from paper_1909_01299_gb300 import hz as mod
    return mod


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hz.h")).read()
    return sorted(set(re.findall(r"\b(hz_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(hz):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(hz._lib, n), n
    assert set(names) == set(hz.SIGNATURES), "binding signatures and header disagree"


def test_status_strings(hz):
    for code in range(9):
        assert hz._lib.hz_status_str(code).decode()


def _axis_ops(h):
    h = np.asarray(h, complex)
    flux = 1.0 / h
    return flux[:-1] + flux[1:], -flux[1:-1], 0.5 * (h[:-1] + h[1:])


def test_plan_eigensolver_closed_form(hz):
    for n, h in [(9, 0.7), (32, 1.0), (80, 1.0)]:
        kd, ko, m = _axis_ops(np.full(n + 1, h))
        lam, Wm, res = hz.tridiag_eig(kd, ko, m)
        mm = np.arange(1, n + 1)
        ref = 4.0 / h ** 2 * np.sin(mm * np.pi / (2 * (n + 1))) ** 2
        assert np.max(np.abs(lam - ref)) < 1e-12 * ref.max()
        i = np.arange(1, n + 1)
        Wref = np.sqrt(2.0 / ((n + 1) * h)) * np.sin(np.outer(i, mm) * np.pi / (n + 1))
        sign = np.sign((Wm * Wref).sum(axis=0).real)
        assert np.max(np.abs(Wm * sign - Wref)) < 1e-12
        assert res < 1e-13
        assert np.all(Wm.imag == 0)        # real steps give exactly real tables


@pytest.mark.parametrize("case", ["pml160", "pml160_blk0", "pml192", "ramp"])
def test_plan_eigensolver_identities(hz, case):
    if case.startswith("pml160"):
        h = W.rim_axis(128)
        if case.endswith("blk0"):
            kd, ko, m = _axis_ops(h)
            kd, ko, m = kd[:79], ko[:78], m[:79]
        else:
            kd, ko, m = _axis_ops(h)
    elif case == "pml192":
        kd, ko, m = _axis_ops(W.rim_axis(160))
    else:
        kd, ko, m = _axis_ops(W.ramp_z(200))
    lam, Wm, res = hz.tridiag_eig(kd, ko, m)
    K = np.diag(kd) + np.diag(ko, 1) + np.diag(ko, -1)
    M = np.diag(m)
    e1 = np.linalg.norm(K @ Wm - M @ Wm @ np.diag(lam)) / (np.linalg.norm(K) * np.linalg.norm(Wm))
    e2 = np.max(np.abs(Wm.T @ M @ Wm - np.eye(len(kd))))
    assert e1 < 1e-13 and e2 < 1e-11, (e1, e2)
    assert res < 1e-11


def test_plan_eigenvalues_match_independent_solver(hz):
    # the oracle's numpy-based pairs, computed without any code of the library
    from oracle import hz_oracle as O
    h = W.rim_axis(128)
    kd, ko, m = _axis_ops(h)
    lam, _, _ = hz.tridiag_eig(kd, ko, m)
    lam_o, _ = O.gen_eig(kd, ko, m)
    assert np.max(np.abs(np.sort_complex(lam) - np.sort_complex(lam_o))) < 1e-10 * np.abs(lam_o).max()


def test_plan_create_rejects_bad_arguments_without_touching_the_device(hz):
    # argument validation happens before any device call
    with pytest.raises(hz.HzError) as e:
        hz.Plan(np.ones(5), np.ones(5), np.ones(5), [0, 2], [0.1], stream=_NoStream())
    assert e.value.code == 1
    with pytest.raises(hz.HzError):
        hz.Plan(np.ones(5), np.ones(5), np.ones(5), [0, 4], [0.1], x_iface=[0], stream=_NoStream())


class _NoStream:
    cuda_stream = 0


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 9, 11, 14, 15, 19, 23, 24, 29, 31, 35, 39, 47, 63, 79, 80, 95, 99, 119, 127])
def test_fast_sine_transform_matches_the_definition(hz, n):
    # the plan's FFT-based sine transform (host twin of the GPU kernel) against the DST-I sum
    # out = S sum_j x_j sin(pi j m / (n + 1)) with the symmetric-modes-first column order
    rng = np.random.default_rng(n)
    N = n + 1
    ns = (n + 1) // 2
    modes = np.array([2 * c + 1 if c < ns else 2 * (c - ns) + 2 for c in range(n)])
    Sm = np.sin(np.pi * np.outer(np.arange(1, N), np.arange(1, N)) / N)   # [j-1][m-1]
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    S = 0.37
    # forward: natural nodes in, modes out in the symmetric-first order
    ref_f = S * (x @ Sm)[modes - 1]
    got_f = hz.sine_transform_host(x, 1, S)
    assert np.max(np.abs(got_f - ref_f)) <= 1e-13 * np.max(np.abs(ref_f))
    # inverse: modes in (symmetric-first order), natural nodes out
    X = np.empty(n, complex)
    X[modes - 1] = x
    ref_i = S * (Sm @ X)
    got_i = hz.sine_transform_host(x, 2, S)
    assert np.max(np.abs(got_i - ref_i)) <= 1e-13 * np.max(np.abs(ref_i))


@pytest.mark.parametrize("n", [1, 6, 12, 128, 160])
def test_fast_sine_transform_rejects_unsupported_lengths(hz, n):
    # n + 1 with a prime factor above 5 (7, 13, 161 = 7 x 23), n + 1 > 128, or n < 2
    with pytest.raises(hz.HzError) as e:
        hz.sine_transform_host(np.ones(n, complex), 1, 1.0)
    assert e.value.code == 1


def test_plan_setters_reject_a_null_plan(hz):
    # every per-plan kernel choice returns HZ_ERR_ARG (1) for a NULL plan, without a device
    lib = hz._lib
    assert lib.hz_plan_set_z_sweep(None, 1) == 1
    assert lib.hz_plan_set_dense_tile_rows(None, 16) == 1
    assert lib.hz_plan_set_fast_sine(None, 1) == 1
    assert lib.hz_plan_set_real_tables(None, 1) == 1
