"""Error measures of the GPU parity tests."""
import numpy as np


def rel(a, b):
    """Relative L2 error of a against b.  For arrays of right-hand sides (nrhs, Nz, Ny, Nx)
    it is the largest per-RHS error, so that no right-hand side with a small norm can hide
    behind a larger one."""
    a, b = np.asarray(a), np.asarray(b)
    if a.ndim == 4:
        assert a.shape == b.shape, (a.shape, b.shape)
        return max(float(np.linalg.norm(a[r] - b[r]) / np.linalg.norm(b[r])) for r in range(a.shape[0]))
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
