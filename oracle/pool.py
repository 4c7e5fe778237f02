"""The oracle's per-set relaxation on several host cores (test infrastructure only).

The sets of Eq. 12 relax independently from the same residual (Sec. 3: one
slave process per set), so ``PoolFactors`` spreads them over worker
processes: worker k factors and relaxes the sets I with I mod W = k (its own
``hms.LocalFactors`` restricted to them).  The residual and the increment
live in shared memory: each worker reads r and writes delta on its own sets'
DOFs, so the parts need no adding and the result equals
``LocalFactors.relax`` exactly.  Workers are started with the 'spawn' method,
so they never inherit a CUDA context, and use one BLAS thread each.  The
arithmetic is that of ``hms`` unchanged; only where it runs differs.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

_W = {}


def _init(nx, ny, ea, fixed, L, sx, sy, overlap, k, w, r_name, d_name):
    from . import hms, truss
    tr = truss.Truss(nx, ny, ea, fixed, L)
    g = hms.SetGrid(nx, ny, sx, sy)
    lf = hms.LocalFactors(tr, g, overlap, sets=range(k, g.M, w))
    rs = shared_memory.SharedMemory(name=r_name)
    ds = shared_memory.SharedMemory(name=d_name)
    n = tr.ndof
    _W.update(lf=lf, rs=rs, ds=ds, r=np.ndarray((n,), np.float64, rs.buf), d=np.ndarray((n,), np.float64, ds.buf))


def _ready(_):
    return "lf" in _W


def _relax(_):
    """delta on this worker's sets, from r, into the shared increment."""
    import scipy.linalg as sla
    lf, r, d = _W["lf"], _W["r"], _W["d"]
    for dofs, dr, pos, cb in zip(lf.dofs, lf.region, lf.pos, lf.factors):
        if cb is not None:
            d[dofs] = sla.cho_solve_banded((cb, True), r[dr])[pos]
    return True


class PoolFactors:
    """Drop-in for ``hms.LocalFactors`` (its ``relax``) over ``workers`` processes."""

    TIMEOUT = 1800  # seconds a worker may take for its setup or one relaxation

    def __init__(self, nx, ny, sx, sy, ea=None, fixed=None, L=1.0, overlap=0, workers=None):
        self.workers = max(1, int(workers or os.cpu_count() or 1))
        n = 2 * nx * ny
        self.rs = shared_memory.SharedMemory(create=True, size=8 * n)
        self.ds = shared_memory.SharedMemory(create=True, size=8 * n)
        self.r = np.ndarray((n,), np.float64, self.rs.buf)
        self.d = np.ndarray((n,), np.float64, self.ds.buf)
        ctx = mp.get_context("spawn")
        self.pools = []
        # one BLAS thread per worker: the workers themselves fill the cores
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            for k in range(self.workers):
                self.pools.append(ctx.Pool(1, initializer=_init, initargs=(
                    nx, ny, ea, fixed, L, sx, sy, overlap, k, self.workers, self.rs.name, self.ds.name)))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        # wait until every worker has its factors (a worker that died makes
        # this raise instead of waiting for ever)
        if not all(p.apply_async(_ready, (0,)).get(timeout=self.TIMEOUT) for p in self.pools):
            self.close()
            raise RuntimeError("oracle pool workers failed to start")

    def relax(self, r: np.ndarray) -> np.ndarray:
        self.r[:] = r
        self.d[:] = 0.0
        jobs = [p.apply_async(_relax, (0,)) for p in self.pools]
        for j in jobs:
            j.get(timeout=self.TIMEOUT)
        return self.d.copy()

    def close(self):
        for p in self.pools:
            p.terminate()
            p.join()
        self.pools = []
        for s in (getattr(self, "rs", None), getattr(self, "ds", None)):
            if s is not None:
                s.close()
                s.unlink()
        self.rs = self.ds = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
