"""Error and summary statistics used by the paper's verification tables.

Oracle code (test infrastructure only).  Eq. 20 is the relative L2 error
sqrt(sum (T_ref - T)^2 / sum T_ref^2); Tables 1-5 report min, max, median,
RMS and the quartiles of the reference, the proposed result and their
difference.
"""
from __future__ import annotations

import numpy as np


def eq20_error(T_ref, T) -> float:
    T_ref = np.asarray(T_ref, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    return float(np.sqrt(np.sum((T_ref - T) ** 2) / np.sum(T_ref ** 2)))


def table_stats(x) -> dict:
    x = np.asarray(x, dtype=np.float64)
    return {"min": float(x.min()), "max": float(x.max()), "median": float(np.median(x)),
            "rms": float(np.sqrt(np.mean(x ** 2))),
            "q1": float(np.percentile(x, 25)), "q3": float(np.percentile(x, 75))}
