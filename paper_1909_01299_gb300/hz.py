"""Thin Python binding of the hz C ABI (include/hz.h).

Argument marshalling only: every step of the solve runs in the CUDA library
libhz.so.  PyTorch supplies device memory and the stream; tensors must be
contiguous complex128 of shape (nrhs, Nz, Ny, Nx) on the plan's device.
Importing this module loads the library and fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhz.so")

HZ_FP64, HZ_MIXED, HZ_MIXED_TF32 = 0, 1, 2
_PRECISION = {"fp64": HZ_FP64, "mixed": HZ_MIXED, "mixed_3xtf32": HZ_MIXED, "mixed_tf32": HZ_MIXED_TF32}


class c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class hz_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_void_p), ("hy", ctypes.c_void_p), ("hz", ctypes.c_void_p)]


class hz_layers(ctypes.Structure):
    _fields_ = [("nlayers", ctypes.c_int), ("z_begin", ctypes.c_void_p), ("k2", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p)]


class hz_blocks(ctypes.Structure):
    _fields_ = [("nbx", ctypes.c_int), ("nby", ctypes.c_int), ("x_iface", ctypes.c_void_p),
                ("y_iface", ctypes.c_void_p)]


class hz_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rtol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class hz_info(ctypes.Structure):
    _fields_ = [("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("min_abs_pivot", ctypes.c_double), ("plan_ms", ctypes.c_double),
                ("eig_max_residual", ctypes.c_double), ("device_bytes", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("nbx", ctypes.c_int), ("nby", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("fast_sine", ctypes.c_int), ("real_tables", ctypes.c_int),
                ("z_sweep", ctypes.c_int)]


# Every symbol declared in include/hz.h, with its ctypes signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "hz_plan_create": (ctypes.c_int, [ctypes.POINTER(hz_grid), ctypes.POINTER(hz_layers),
                                      ctypes.POINTER(hz_blocks), ctypes.POINTER(hz_options),
                                      ctypes.POINTER(_P)]),
    "hz_plan_set_frequency": (ctypes.c_int, [_P, ctypes.c_double]),
    "hz_plan_set_k2": (ctypes.c_int, [_P, _P]),
    "hz_plan_set_options": (ctypes.c_int, [_P, ctypes.POINTER(hz_options)]),
    "hz_plan_set_fast_sine": (ctypes.c_int, [_P, ctypes.c_int]),
    "hz_plan_set_real_tables": (ctypes.c_int, [_P, ctypes.c_int]),
    "hz_plan_set_z_sweep": (ctypes.c_int, [_P, ctypes.c_int]),
    "hz_plan_set_dense_tile_rows": (ctypes.c_int, [_P, ctypes.c_int]),
    "hz_sine_transform_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P]),
    "hz_plan_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "hz_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "hz_solve_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "hz_solve_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "hz_grad_layers": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "hz_solve_perturbed": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, _P, _P]),
    "hz_grad_rhs": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "hz_residual": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "hz_residual_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "hz_get_info": (ctypes.c_int, [_P, ctypes.POINTER(hz_info)]),
    "hz_plan_destroy": (ctypes.c_int, [_P]),
    "hz_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "hz_set_stage_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "hz_get_stage_times": (ctypes.c_int, [_P, _P, _P]),
    "hz_tridiag_eig": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, _P,
                                      ctypes.POINTER(ctypes.c_double)]),
    "hz_batch_create": (ctypes.c_int, [ctypes.c_int, _P, _P, ctypes.c_int, ctypes.POINTER(_P)]),
    "hz_batch_solve": (ctypes.c_int, [_P, _P, _P, _P]),
    "hz_batch_autotune": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "hz_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_int)]),
    "hz_batch_destroy": (ctypes.c_int, [_P]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"hz CUDA library not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class HzError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_lib.hz_status_str(code).decode()} (status {code})")


def _check(code: int, where: str):
    if code != 0:
        raise HzError(code, where)


def _c128_array(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def tridiag_eig(kd, ko, m):
    """Host eigen-solver of the plan: K W = M W Lambda, W^T M W = I (complex symmetric)."""
    kd, ko, m = _c128_array(kd), _c128_array(ko), _c128_array(m)
    n = len(kd)
    lam = np.empty(n, np.complex128)
    W = np.empty((n, n), np.complex128)
    res = ctypes.c_double()
    _check(_lib.hz_tridiag_eig(n, kd.ctypes.data, ko.ctypes.data if n > 1 else None, m.ctypes.data,
                               lam.ctypes.data, W.ctypes.data, ctypes.byref(res)), "hz_tridiag_eig")
    return lam, W, res.value


def sine_transform_host(x, direction: int, scale: float) -> np.ndarray:
    """Host-only: the plan's fast sine transform of one row (hz_sine_transform_host)."""
    x = _c128_array(x)
    out = np.empty_like(x)
    _check(_lib.hz_sine_transform_host(len(x), int(direction), float(scale), x.ctypes.data, out.ctypes.data),
           "hz_sine_transform_host")
    return out


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Plan:
    """A solver plan (hz_plan_create): grid, layers, blocks and options.

    precision: "fp64" (DFMA transforms) or "mixed" (= "mixed_3xtf32"; FP32 transforms, the bulk
    ones as three TF32 products on the tensor cores, FP64 z solves, interface solves and
    refinement to `rtol`) or "mixed_tf32" (one TF32 product per bulk transform).
    """

    def __init__(self, hx, hy, hz, z_begin, k2, sigma=None, x_iface=None, y_iface=None,
                 nbx: Optional[int] = None, nby: Optional[int] = None, precision: str = "fp64",
                 rtol: float = 1e-8, max_refine: int = 10, stream=None):
        self._keep = []
        hx, hy, hz = _c128_array(hx), _c128_array(hy), _c128_array(hz)
        zb = np.ascontiguousarray(np.asarray(z_begin, dtype=np.int32))
        k2 = _c128_array(k2)
        self.nx, self.ny, self.nz = len(hx) - 1, len(hy) - 1, len(hz) - 1
        self.nlayers = len(k2)
        self.z_begin = zb.copy()
        g = hz_grid(self.nx, self.ny, self.nz, hx.ctypes.data, hy.ctypes.data, hz.ctypes.data)
        sig = None if sigma is None else np.ascontiguousarray(np.asarray(sigma, dtype=np.float64))
        lay = hz_layers(self.nlayers, zb.ctypes.data, k2.ctypes.data, None if sig is None else sig.ctypes.data)
        xi = None if x_iface is None else np.ascontiguousarray(np.asarray(x_iface, dtype=np.int32))
        yi = None if y_iface is None else np.ascontiguousarray(np.asarray(y_iface, dtype=np.int32))
        nbx = (len(xi) + 1 if xi is not None else 1) if nbx is None else nbx
        nby = (len(yi) + 1 if yi is not None else 1) if nby is None else nby
        blk = hz_blocks(nbx, nby, None if xi is None or len(xi) == 0 else xi.ctypes.data,
                        None if yi is None or len(yi) == 0 else yi.ctypes.data)
        self.precision = precision
        self._opts = hz_options(_PRECISION[precision], rtol, max_refine, _stream_handle(stream))
        h = _P()
        _check(_lib.hz_plan_create(ctypes.byref(g), ctypes.byref(lay), ctypes.byref(blk),
                                   ctypes.byref(self._opts), ctypes.byref(h)), "hz_plan_create")
        self._h = h
        self.hx, self.hy, self.hz = hx, hy, hz

    @classmethod
    def from_workload(cls, w, precision: Optional[str] = None, **kw):
        return cls(w.hx, w.hy, w.hz, w.z_begin, w.k2, w.sigma, w.x_iface, w.y_iface,
                   nbx=len(w.x_iface) + 1, nby=len(w.y_iface) + 1,
                   precision=precision or w.precision, **kw)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.hz_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration ------------------------------------------------------
    def set_options(self, precision=None, rtol=None, max_refine=None, stream=None):
        if precision is not None:
            self.precision = precision
            self._opts.precision = _PRECISION[precision]
        if rtol is not None:
            self._opts.rtol = rtol
        if max_refine is not None:
            self._opts.max_refine = max_refine
        self._opts.cuda_stream = _stream_handle(stream)
        _check(_lib.hz_plan_set_options(self._h, ctypes.byref(self._opts)), "hz_plan_set_options")

    def autotune(self, nrhs: int) -> dict:
        """hz_plan_autotune: pick the fastest kernel variants for nrhs right-hand sides."""
        c = ctypes.c_int()
        _check(_lib.hz_plan_autotune(self._h, int(nrhs), ctypes.byref(c)), "hz_plan_autotune")
        return {"z_sweep": c.value % 10, "tensor_cores": (c.value // 10) % 10 == 1,
                "fast_sine": (c.value // 100) % 10 == 1, "real_tables": (c.value // 1000) % 10 == 1,
                "dense_tile_rows": {1: 16, 2: 64}.get(c.value // 10000, 0)}

    def set_real_tables(self, enable: bool):
        """Mixed path: real block tables through the real-table tensor-core kernel (True, the
        default) or the interleaved complex GEMM (False) (hz_plan_set_real_tables)."""
        _check(_lib.hz_plan_set_real_tables(self._h, int(bool(enable))), "hz_plan_set_real_tables")

    def set_z_sweep(self, variant: int):
        """z sweep variant (hz_plan_set_z_sweep): 1 or 2 right-hand sides per thread, 3 z in
        register chunks (few modes, long z), 0 (default) chosen per launch."""
        _check(_lib.hz_plan_set_z_sweep(self._h, int(variant)), "hz_plan_set_z_sweep")

    def set_dense_tile_rows(self, rows: int):
        """Data rows per CTA of the dense CUDA-core transforms (hz_plan_set_dense_tile_rows):
        16, 64, or 0 (default) chosen by launch size."""
        _check(_lib.hz_plan_set_dense_tile_rows(self._h, int(rows)), "hz_plan_set_dense_tile_rows")

    def set_fast_sine(self, enable: int):
        """Uniform blocks by the FFT-based sine transform (hz_plan_set_fast_sine): 0 dense
        everywhere, 1 (default) the FP64 path, 2 also the mixed path (in FP32)."""
        _check(_lib.hz_plan_set_fast_sine(self._h, int(enable)), "hz_plan_set_fast_sine")

    def set_frequency(self, omega: float):
        _check(_lib.hz_plan_set_frequency(self._h, float(omega)), "hz_plan_set_frequency")

    def set_k2(self, k2):
        k2 = _c128_array(k2)
        assert len(k2) == self.nlayers
        _check(_lib.hz_plan_set_k2(self._h, k2.ctypes.data), "hz_plan_set_k2")

    def info(self) -> dict:
        i = hz_info()
        _check(_lib.hz_get_info(self._h, ctypes.byref(i)), "hz_get_info")
        return {f: getattr(i, f) for f, _ in hz_info._fields_}

    STAGES = ["fwd", "pass_a", "edges", "iface_residual", "global", "pass_b", "inv", "iface_out",
              "residual"]

    def set_stage_timing(self, enable: bool):
        _check(_lib.hz_set_stage_timing(self._h, int(enable)), "hz_set_stage_timing")

    def stage_times(self) -> dict:
        ms = np.zeros(len(self.STAGES), np.float64)
        n = np.zeros(len(self.STAGES), np.int64)
        _check(_lib.hz_get_stage_times(self._h, ms.ctypes.data, n.ctypes.data), "hz_get_stage_times")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.STAGES)}

    # -- solves -------------------------------------------------------------
    def _check_tensor(self, t):
        import torch
        if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
            raise ValueError("expected a contiguous complex128 CUDA tensor")
        if t.dim() != 4 or tuple(t.shape[1:]) != (self.nz, self.ny, self.nx):
            raise ValueError(f"expected shape (nrhs, {self.nz}, {self.ny}, {self.nx}), got {tuple(t.shape)}")
        return t.shape[0]

    def solve(self, f, out=None):
        """u = A^{-1} (M f) for device tensors (hz_solve)."""
        import torch
        R = self._check_tensor(f)
        u = torch.empty_like(f) if out is None else out
        _check(_lib.hz_solve(self._h, f.data_ptr(), u.data_ptr(), R), "hz_solve")
        return u

    def solve_host(self, f_host, out=None):
        """hz_solve_host on host arrays (numpy or CPU tensors); returns a numpy array."""
        f = _c128_array(f_host) if not hasattr(f_host, "data_ptr") else f_host
        if hasattr(f, "data_ptr"):
            u = np.empty(tuple(f.shape), np.complex128) if out is None else out
            ptr_f = f.data_ptr()
        else:
            u = np.empty_like(f) if out is None else out
            ptr_f = f.ctypes.data
        ptr_u = u.data_ptr() if hasattr(u, "data_ptr") else u.ctypes.data
        _check(_lib.hz_solve_host(self._h, ptr_f, ptr_u, f.shape[0]), "hz_solve_host")
        return u

    def solve_adjoint(self, g, out=None):
        """lam = A^{-H} g (hz_solve_adjoint); g is in the weighted space."""
        import torch
        R = self._check_tensor(g)
        lam = torch.empty_like(g) if out is None else out
        _check(_lib.hz_solve_adjoint(self._h, g.data_ptr(), lam.data_ptr(), R), "hz_solve_adjoint")
        return lam

    def solve_perturbed(self, dk2, f, rtol: float = 1e-8, max_iter: int = 200, restart: int = 20, out=None):
        """u of the layered medium with a local k^2 perturbation dk2 (device complex128 of shape
        (Nz, Ny, Nx)), by GMRES around this plan's layered solve (hz_solve_perturbed).
        Returns (u, iterations, per-RHS true relative residual)."""
        import torch
        R = self._check_tensor(f)
        if tuple(dk2.shape) != (self.nz, self.ny, self.nx) or dk2.dtype != torch.complex128 or not dk2.is_cuda \
                or not dk2.is_contiguous():
            raise ValueError("dk2 must be a contiguous CUDA complex128 tensor of shape (nz, ny, nx)")
        u = torch.empty_like(f) if out is None else out
        it = ctypes.c_int()
        rel = np.empty(R, np.float64)
        code = _lib.hz_solve_perturbed(self._h, dk2.data_ptr(), f.data_ptr(), u.data_ptr(), R, rtol, max_iter,
                                       restart, ctypes.byref(it), rel.ctypes.data)
        _check(code, "hz_solve_perturbed")
        return u, it.value, rel

    def grad_layers(self, u, lam) -> np.ndarray:
        R = self._check_tensor(u)
        self._check_tensor(lam)
        G = np.empty(self.nlayers, np.complex128)
        _check(_lib.hz_grad_layers(self._h, u.data_ptr(), lam.data_ptr(), R, G.ctypes.data), "hz_grad_layers")
        return G

    def grad_rhs(self, lam, out=None):
        """M^H lam: the gradient in f of a real objective whose adjoint state is lam (hz_grad_rhs)."""
        import torch
        R = self._check_tensor(lam)
        gf = torch.empty_like(lam) if out is None else out
        _check(_lib.hz_grad_rhs(self._h, lam.data_ptr(), gf.data_ptr(), R), "hz_grad_rhs")
        return gf

    def residual(self, f, u) -> np.ndarray:
        R = self._check_tensor(f)
        out = np.empty(R, np.float64)
        _check(_lib.hz_residual(self._h, f.data_ptr(), u.data_ptr(), R, out.ctypes.data), "hz_residual")
        return out


def residual_noalloc(plan: Plan, f, u) -> np.ndarray:
    """hz_residual_noalloc: the residual check that allocates no device memory.

    For callers that cannot allocate device memory at the time of the check
    (allocation-free serving or real-time loops, frameworks that own all device
    memory); nrhs <= 64; the plan's device must be the current one; calls that
    overlap on the GPU must be serialised (they share one fixed scratch array).
    """
    R = plan._check_tensor(f)
    plan._check_tensor(u)
    out = np.empty(R, np.float64)
    _check(_lib.hz_residual_noalloc(plan._h, f.data_ptr(), u.data_ptr(), R, out.ctypes.data),
           "hz_residual_noalloc")
    return out


class Batch:
    """hz_batch_*: many (plan, nrhs) solves captured once and replayed as one CUDA graph.

    plans: one Plan per (model, frequency); nrhs: RHS count per plan.  The batch keeps
    references to the plans so they outlive it.
    """

    def __init__(self, plans, nrhs, lanes: int = 0):
        self.plans = list(plans)
        self.nrhs = [int(r) for r in nrhs]
        hs = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        rs = (ctypes.c_int * len(self.nrhs))(*self.nrhs)
        h = _P()
        _check(_lib.hz_batch_create(len(self.plans), ctypes.cast(hs, _P), ctypes.cast(rs, _P), int(lanes),
                                    ctypes.byref(h)), "hz_batch_create")
        self._h = h

    def _ptrs(self, fs, us):
        for p, f, u, R in zip(self.plans, fs, us, self.nrhs):
            assert p._check_tensor(f) == R and p._check_tensor(u) == R
        fa = (ctypes.c_void_p * len(fs))(*[f.data_ptr() for f in fs])
        ua = (ctypes.c_void_p * len(us))(*[u.data_ptr() for u in us])
        return fa, ua

    def solve(self, fs, us) -> np.ndarray:
        """u_i = A_i^{-1} M f_i for every item; returns each item's max relative residual."""
        fa, ua = self._ptrs(fs, us)
        rel = np.empty(len(fs), np.float64)
        _check(_lib.hz_batch_solve(self._h, ctypes.cast(fa, _P), ctypes.cast(ua, _P), rel.ctypes.data),
               "hz_batch_solve")
        return rel

    def autotune(self, fs, us) -> int:
        fa, ua = self._ptrs(fs, us)
        lanes = ctypes.c_int()
        _check(_lib.hz_batch_autotune(self._h, ctypes.cast(fa, _P), ctypes.cast(ua, _P), ctypes.byref(lanes)),
               "hz_batch_autotune")
        return lanes.value

    def info(self) -> dict:
        ms, n, lanes = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_int()
        _check(_lib.hz_batch_info(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(lanes)), "hz_batch_info")
        return {"last_ms": ms.value, "launches_per_replay": n.value, "lanes": lanes.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.hz_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HzSolve:
    """torch.autograd.Function wrapper: u = A(k2)^{-1} M f, differentiable in k2 and f.

    Usage: u = HzSolve.apply(k2, f, plan) with k2 a complex128 tensor (nlayers,)
    on the CPU (it sets the plan's layer k^2) and f a CUDA tensor.  The backward
    pass runs one adjoint solve lam = A^{-H} grad_u and returns
    k2.grad = conj(G) (G from hz_grad_layers; PyTorch's convention for complex
    leaves of real losses) and f.grad = M^H lam (hz_grad_rhs).
    """

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, k2, f, plan):
                plan.set_k2(k2.detach().cpu().numpy())
                u = plan.solve(f.contiguous())
                ctx.plan = plan
                ctx.save_for_backward(u)
                return u

            @staticmethod
            def backward(ctx, grad_u):
                (u,) = ctx.saved_tensors
                plan = ctx.plan
                lam = plan.solve_adjoint(grad_u.contiguous())
                G = plan.grad_layers(u, lam)
                gk = torch.from_numpy(np.conj(G))
                gf = plan.grad_rhs(lam)
                return gk, gf, None

        return _F

    _cache = None

    @classmethod
    def apply(cls, k2, f, plan):
        if cls._cache is None:
            cls._cache = cls._fn()
        return cls._cache.apply(k2, f, plan)
