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


# Binary16 message storage (FP16 forms).  GPU and oracle both round every stored message to
# binary16, from an FP32 and an FP64 value respectively, so a message near a rounding
# boundary can round one binary16 ulp apart.  At the first flooding iteration every message
# depends on the channel LLRs only: each posterior then differs by at most 2 half-ulps of
# every incoming message beyond the FP32 tolerance, and a band of `mult` half-ulps (4 for
# flooding) holds on every codeword.  After that, and within the first layered iteration, a
# changed posterior feeds later checks whose messages may cross further rounding boundaries:
# the flips cascade.  The FP64 oracle itself, fed LLRs perturbed by 1e-6 relative, moves a
# few codewords by tens of half-ulps while the rest stay within 1-3.  These cascades stay
# inside their codeword, so beyond the first flooding iteration the band (4 half-ulps for
# flooding, 8 for layered) must hold on all but F16_CASCADE_FRAC of the codewords; a
# systematic error (a slot, a barrier group, a refill wave) would move far more of them.
F16_CASCADE_FRAC = 0.02


def binary16_band(oc, layered: bool, L, T: int, mult: float, X: float = 80.0):
    """(ref, band): the FP64 oracle (clamp X) with binary16 message storage after T
    iterations (no early exit) and the per-element band FP32_TOL * max(1, |ref|) + mult
    half-ulps of the sum of the incoming message magnitudes."""
    orc = oc.spa_layered if layered else oc.spa_flood
    ref, _, _, R = orc(L, T, early_exit=False, X=X, fp16_msgs=True, return_messages=True)
    band = FP32_TOL * np.maximum(1.0, np.abs(ref)) + mult * 2.0 ** -11 * oc.incoming_message_sum(R)
    return ref, band


def codewords_outside(app, ref, band) -> int:
    """Codewords (rows) with at least one element outside the band."""
    return int((np.abs(np.asarray(app, np.float64) - ref) > band).any(axis=1).sum())


def assert_binary16_close(app, ref, band, strict: bool, what=""):
    """Every codeword within the band (strict: the first flooding iteration), else all but
    F16_CASCADE_FRAC of them."""
    out = codewords_outside(app, ref, band)
    limit = 0 if strict else int(F16_CASCADE_FRAC * len(ref))
    assert out <= limit, (what, out, len(ref))
