"""Shared helpers for the GPU tests (import only from test modules)."""
import numpy as np
import pytest

_ff = None


def ff():
    """The built binding; builds the library on first use."""
    global _ff
    if _ff is None:
        import torch
        if not torch.cuda.is_available():
            pytest.fail("GPU test needs CUDA")
        from paper_1909_05098_gb300.build import build
        build()
        from paper_1909_05098_gb300 import fedfem
        _ff = fedfem
    return _ff


def run_gpu(problem, dt, n_steps, precision, order=None, kernel=None, T0=None, T_lo=None, T_hi=None):
    f = ff()
    kw = {}
    if order is not None:
        kw["order"] = order
    if kernel is not None:
        kw["kernel"] = kernel
    s = f.Solver(problem, precision=precision, T_lo=T_lo, T_hi=T_hi, **kw)
    try:
        if T0 is not None:
            s.init(T0)
        if n_steps:
            s.step(dt, n_steps)
        done = s.sync()
        assert done == n_steps
        return s.temperature(), s.info()
    finally:
        s.close()


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
