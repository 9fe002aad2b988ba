"""ctypes front end of the plain-C LDPC oracle (``ldpc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg.  The decoding library never imports it.

Every routine takes and returns numpy arrays; codes are given either as a QC base
matrix plus lifting Z (``QCCode``) or as an explicit CSR parity-check matrix (``Code``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_OK = 0


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP when available, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_num_threads.restype = C.c_int
    return _lib


class use_library:
    """Context manager: route every oracle call through another build of ldpc_oracle.c
    (the mutation tests load deliberately broken copies this way)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _lib = C.CDLL(self.path)
        _lib.orc_num_threads.restype = C.c_int
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != ORC_OK:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Code:
    """Parity-check matrix in CSR form: check m joins variables ci[rp[m]:rp[m+1]] (ascending).

    ``layers`` (optional) are the check-index boundaries of the layered schedule.
    """

    def __init__(self, M: int, N: int, rp, ci, layers=None):
        self.M, self.N = int(M), int(N)
        self.rp = np.ascontiguousarray(rp, dtype=np.int32)
        self.ci = np.ascontiguousarray(ci, dtype=np.int32)
        self.E = int(self.rp[-1])
        self.layers = None if layers is None else np.ascontiguousarray(layers, dtype=np.int32)

    @classmethod
    def from_dense(cls, H, layers=None):
        H = np.asarray(H) != 0
        M, N = H.shape
        rp = [0]
        ci = []
        for m in range(M):
            cols = np.nonzero(H[m])[0]
            ci.extend(int(c) for c in cols)
            rp.append(len(ci))
        return cls(M, N, rp, ci, layers)

    def dense(self) -> np.ndarray:
        H = np.zeros((self.M, self.N), dtype=np.uint8)
        for m in range(self.M):
            H[m, self.ci[self.rp[m]:self.rp[m + 1]]] = 1
        return H

    def syndrome_weight(self, c) -> np.ndarray:
        c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.uint8)
        w = np.zeros(c.shape[0], dtype=np.int32)
        _check(lib().orc_syndrome_batch(C.c_int(self.M), C.c_int(self.N), _p(self.rp), _p(self.ci), _p(c),
                                        C.c_int64(c.shape[0]), _p(w)), "syndrome")
        return w

    def spa_flood(self, L, max_iter: int, early_exit: bool = True, X: float = 80.0, fp16_msgs: bool = False,
                  nthreads: int = 0, return_messages: bool = False):
        """FP64 flooding sum-product.  L fp32 [B, N] -> (app f64 [B, N], bits u8, iters i32)
        (+ the last messages R f64 [B, E] in CSR edge order when return_messages)."""
        L = np.ascontiguousarray(np.atleast_2d(L), dtype=np.float32)
        B = L.shape[0]
        app = np.empty((B, self.N), dtype=np.float64)
        bits = np.empty((B, self.N), dtype=np.uint8)
        iters = np.empty(B, dtype=np.int32)
        R = np.empty((B, self.E), dtype=np.float64) if return_messages else None
        _check(lib().orc_spa_flood(C.c_int(self.M), C.c_int(self.N), _p(self.rp), _p(self.ci), _p(L),
                                   C.c_int64(B), C.c_int(max_iter), C.c_int(int(early_exit)), C.c_double(X),
                                   C.c_int(int(fp16_msgs)), _p(app), _p(bits), _p(iters),
                                   None if R is None else _p(R), C.c_int(nthreads)),
               "spa_flood")
        return (app, bits, iters, R) if return_messages else (app, bits, iters)

    def spa_layered(self, L, max_iter: int, early_exit: bool = True, X: float = 80.0, fp16_msgs: bool = False,
                    nthreads: int = 0, return_messages: bool = False):
        """FP64 layered sum-product over ``self.layers``: same inputs and outputs as spa_flood."""
        if self.layers is None:
            raise ValueError("code has no layer boundaries")
        L = np.ascontiguousarray(np.atleast_2d(L), dtype=np.float32)
        B = L.shape[0]
        app = np.empty((B, self.N), dtype=np.float64)
        bits = np.empty((B, self.N), dtype=np.uint8)
        iters = np.empty(B, dtype=np.int32)
        R = np.empty((B, self.E), dtype=np.float64) if return_messages else None
        _check(lib().orc_spa_layered(C.c_int(self.M), C.c_int(self.N), _p(self.rp), _p(self.ci),
                                     C.c_int(len(self.layers) - 1), _p(self.layers), _p(L), C.c_int64(B),
                                     C.c_int(max_iter), C.c_int(int(early_exit)), C.c_double(X),
                                     C.c_int(int(fp16_msgs)), _p(app), _p(bits), _p(iters),
                                     None if R is None else _p(R), C.c_int(nthreads)),
               "spa_layered")
        return (app, bits, iters, R) if return_messages else (app, bits, iters)

    def incoming_message_sum(self, R):
        """sum_m |R_mn| per variable n, for messages R [B, E] in CSR edge order."""
        out = np.zeros((R.shape[0], self.N))
        np.add.at(out.T, self.ci, np.abs(R).T)
        return out

    def nms_layered(self, q, max_iter: int, early_exit: bool = True, alpha_num: int = 3, alpha_shift: int = 2,
                    msg_sat: int = 31, app_sat: int = 127, nthreads: int = 0):
        """Integer layered normalised min-sum.  q int8 [B, N] -> (app i32, bits u8, iters i32)."""
        if self.layers is None:
            raise ValueError("code has no layer boundaries")
        q = np.ascontiguousarray(np.atleast_2d(q), dtype=np.int8)
        B = q.shape[0]
        app = np.empty((B, self.N), dtype=np.int32)
        bits = np.empty((B, self.N), dtype=np.uint8)
        iters = np.empty(B, dtype=np.int32)
        _check(lib().orc_nms_layered(C.c_int(self.M), C.c_int(self.N), _p(self.rp), _p(self.ci),
                                     C.c_int(len(self.layers) - 1), _p(self.layers), _p(q), C.c_int64(B),
                                     C.c_int(max_iter), C.c_int(int(early_exit)), C.c_int(alpha_num),
                                     C.c_int(alpha_shift), C.c_int(msg_sat), C.c_int(app_sat), _p(app), _p(bits),
                                     _p(iters), C.c_int(nthreads)), "nms_layered")
        return app, bits, iters

    def nms_layered_real(self, L, max_iter: int, alpha: float = 0.75):
        if self.layers is None:
            raise ValueError("code has no layer boundaries")
        L = np.ascontiguousarray(np.atleast_2d(L), dtype=np.float64)
        B = L.shape[0]
        app = np.empty((B, self.N), dtype=np.float64)
        _check(lib().orc_nms_layered_real(C.c_int(self.M), C.c_int(self.N), _p(self.rp), _p(self.ci),
                                          C.c_int(len(self.layers) - 1), _p(self.layers), _p(L), C.c_int64(B),
                                          C.c_int(max_iter), C.c_double(alpha), _p(app), C.c_int(0)),
               "nms_layered_real")
        return app

    def ml_decode(self, L):
        L = np.ascontiguousarray(np.atleast_2d(L), dtype=np.float32)
        B = L.shape[0]
        bits = np.empty((B, self.N), dtype=np.uint8)
        size = C.c_int32(0)
        _check(lib().orc_ml_decode(C.c_int(self.M), C.c_int(self.N), _p(self.rp), _p(self.ci), _p(L),
                                   C.c_int64(B), _p(bits), C.byref(size)), "ml_decode")
        return bits, int(size.value)


class QCCode(Code):
    """A code lifted from a QC base matrix by the oracle's own expansion; layers = block rows."""

    def __init__(self, base, Z: int):
        self.base = np.ascontiguousarray(base, dtype=np.int32)
        mb, nb = self.base.shape
        self.mb, self.nb, self.Z = mb, nb, int(Z)
        nnz = int(lib().orc_qc_nnz(_p(self.base), C.c_int(mb), C.c_int(nb), C.c_int(Z)))
        if nnz < 0:
            raise ValueError("base matrix entry outside [-1, Z)")
        rp = np.zeros(mb * Z + 1, dtype=np.int32)
        ci = np.zeros(nnz * Z, dtype=np.int32)
        _check(lib().orc_qc_expand(_p(self.base), C.c_int(mb), C.c_int(nb), C.c_int(Z), _p(rp), _p(ci)), "qc_expand")
        super().__init__(mb * Z, nb * Z, rp, ci, layers=np.arange(0, mb * Z + 1, Z, dtype=np.int32))
        self.K = (nb - mb) * Z

    def encode(self, u):
        u = np.ascontiguousarray(np.atleast_2d(u), dtype=np.uint8)
        B = u.shape[0]
        c = np.empty((B, self.N), dtype=np.uint8)
        _check(lib().orc_encode_qc(_p(self.base), C.c_int(self.mb), C.c_int(self.nb), C.c_int(self.Z), _p(u),
                                   C.c_int64(B), _p(c)), "encode_qc")
        return c


def quantize(L, scale: float = 2.0, sat: int = 31):
    L = np.ascontiguousarray(L, dtype=np.float32)
    out = np.empty(L.shape, dtype=np.int8)
    _check(lib().orc_quantize(_p(L), C.c_int64(L.size), C.c_float(scale), C.c_int(sat), _p(out)), "quantize")
    return out


def phi(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    _check(lib().orc_phi(_p(x), C.c_int64(x.size), _p(out)), "phi")
    return out


def round_binary16(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    _check(lib().orc_round_binary16(_p(x), C.c_int64(x.size), _p(out)), "round_binary16")
    return out
