"""Helpers shared by the GPU parity tests (no decoding arithmetic here)."""
import numpy as np
from scipy.stats import beta

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I

FP32_TOL = 1e-3      # |APP_gpu - APP_oracle| <= 1e-3 * max(1, |APP_oracle|)


def rel_err(a, ref):
    return np.abs(np.asarray(a, np.float64) - ref) / np.maximum(1.0, np.abs(ref))


def clopper_pearson(k: int, n: int, conf: float = 0.95):
    a = 1.0 - conf
    lo = 0.0 if k == 0 else beta.ppf(a / 2, k, n - k + 1)
    hi = 1.0 if k == n else beta.ppf(1 - a / 2, k + 1, n - k)
    return lo, hi


_codes = {}


def oracle_code(name):
    if name not in _codes:
        B, Z = I.load_code(name)
        _codes[name] = O.QCCode(B, Z)
    return _codes[name]
