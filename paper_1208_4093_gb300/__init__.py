"""GB300-native hierarchical master-slave solver for triangle-lattice trusses.

The solver (Xu, Liu, Dong: global equilibrium over incremental modes plus
local relaxation of every set) runs in hand-written sm_103a CUDA kernels
behind the C ABI of include/hms.h; ``capi`` is its Python binding and
``Solver`` a small convenience wrapper.  PyTorch is used only for device
memory when callers pass CUDA tensors.
"""
from __future__ import annotations

import numpy as np

from . import capi
from .capi import HMS_FP64, HMS_MIXED, HmsError  # noqa: F401

__all__ = ["capi", "Solver", "HMS_FP64", "HMS_MIXED", "HmsError"]


class Solver:
    """One lattice problem on one GPU: owns a context and a problem handle."""

    def __init__(self, nx, ny, set_sx, set_sy, *, ea=None, ea_uniform=1.0, fixed=None,
                 fix_bottom_edge=1, bar_length=1.0, precision=HMS_FP64, tol=1e-8, max_iter=1000,
                 coarse_solves=0, batch=0, profile=0, device=0):
        self.nx, self.ny = nx, ny
        self.ctx = capi.hms_context_create(device)
        try:
            self.pr = capi.hms_problem_create(
                self.ctx, nx, ny, set_sx, set_sy, bar_length=bar_length, ea=ea, ea_uniform=ea_uniform,
                fixed=fixed, fix_bottom_edge=fix_bottom_edge, precision=precision, tol=tol,
                max_iter=max_iter, coarse_solves=coarse_solves, batch=batch, profile=profile)
        except Exception:
            capi.hms_context_destroy(self.ctx)
            raise
        self.max_iter = max_iter

    @property
    def ndof(self):
        return 2 * self.nx * self.ny

    def solve(self, loads, u0=None, allow_no_convergence=False):
        """loads: [2N] or [nrhs, 2N] float64 (host).  Returns (u, hist, iters)."""
        p = np.ascontiguousarray(loads, dtype=np.float64)
        single = p.ndim == 1
        p = p.reshape(-1, self.ndof)
        u = np.empty_like(p)
        hist = np.full((p.shape[0], self.max_iter + 1, 3), np.nan)
        iters = np.zeros(p.shape[0], dtype=np.int32)
        capi.hms_solve(self.ctx, self.pr, p, u, u0=u0, hist=hist, iters=iters,
                       allow_no_convergence=allow_no_convergence)
        if single:
            return u[0], hist[0], int(iters[0])
        return u, hist, iters

    def close(self):
        if getattr(self, "pr", None) is not None:
            capi.hms_problem_destroy(self.pr)
            self.pr = None
        if getattr(self, "ctx", None) is not None:
            capi.hms_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
