"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each ``pin_*`` function takes the oracle module (``oracle.oracle`` or a copy loaded
from a deliberately broken build) and raises AssertionError when the oracle disagrees
with the fact it is pinned to:

* the paper's worked example (Sec. II, Eq. 1: the (10,5) H-matrix in tests/golden);
* closed forms (the tanh rule for the first sum-product iteration, phi(ln 3) = ln 2,
  the degree-2 check, hand-derived integer min-sum steps);
* brute force (bitwise MAP marginals on cycle-free codes, ML over the enumerated codebook);
* invariants (H.c = 0 on encoded words, all-zero-codeword symmetry);
* library routines for special cases (numpy's IEEE binary16 rounding).
"""
from __future__ import annotations

import os

import numpy as np

from paper_1812_06545_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------- helpers (independent of the oracle)

def eq1_H() -> np.ndarray:
    rows = []
    with open(os.path.join(GOLDEN, "eq1_H.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                rows.append([int(x) for x in ln.split()])
    return np.array(rows, dtype=np.uint8)


def dense_lift(B: np.ndarray, Z: int) -> np.ndarray:
    """H from a base matrix by placing np.roll(I_Z, s, axis=1) blocks: row r has its one
    in column (r + s) mod Z."""
    mb, nb = B.shape
    H = np.zeros((mb * Z, nb * Z), dtype=np.uint8)
    eye = np.eye(Z, dtype=np.uint8)
    for i in range(mb):
        for j in range(nb):
            if B[i, j] >= 0:
                H[i * Z:(i + 1) * Z, j * Z:(j + 1) * Z] = np.roll(eye, int(B[i, j]), axis=1)
    return H


def gf2_rank(H: np.ndarray) -> int:
    A = (np.asarray(H) & 1).astype(np.uint8).copy()
    r = 0
    for c in range(A.shape[1]):
        piv = np.nonzero(A[r:, c])[0]
        if len(piv) == 0:
            continue
        p = r + piv[0]
        A[[r, p]] = A[[p, r]]
        for i in range(A.shape[0]):
            if i != r and A[i, c]:
                A[i] ^= A[r]
        r += 1
        if r == A.shape[0]:
            break
    return r


def codebook(H: np.ndarray) -> np.ndarray:
    """All x in {0,1}^N with H x = 0 (N <= 20), by enumeration."""
    M, N = H.shape
    x = ((np.arange(1 << N)[:, None] >> np.arange(N)[None, :]) & 1).astype(np.uint8)
    ok = ((x.astype(np.int64) @ H.T.astype(np.int64)) % 2 == 0).all(axis=1)
    return x[ok]


def map_llr(H: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Exact bitwise MAP posterior LLRs by marginalising over the codebook:
    p(c | y) ~ exp(sum_n (1 - 2 c_n) L_n / 2)."""
    cb = codebook(H)
    s = ((1.0 - 2.0 * cb) * L[None, :]).sum(axis=1) / 2.0
    out = np.empty(H.shape[1])
    for n in range(H.shape[1]):
        a, b = s[cb[:, n] == 0], s[cb[:, n] == 1]
        out[n] = np.logaddexp.reduce(a) - np.logaddexp.reduce(b)
    return out


def random_tree_H(rng: np.random.Generator, n_target: int) -> np.ndarray:
    """A cycle-free Tanner graph: each new check joins one existing variable and 1-3 new ones."""
    checks = []
    n = 1
    while n < n_target:
        v = int(rng.integers(0, n))
        k = int(min(rng.integers(1, 4), n_target - n))
        checks.append([v] + list(range(n, n + k)))
        n += k
    H = np.zeros((len(checks), n), dtype=np.uint8)
    for m, vs in enumerate(checks):
        H[m, vs] = 1
    return H


def tanh_rule_first_iteration(H: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Posterior after one sum-product iteration from Q = L:
    APP_n = L_n + sum_m 2 atanh( prod_{n' in N(m), n' != n} tanh(L_n' / 2) )."""
    app = L.astype(np.float64).copy()
    for m in range(H.shape[0]):
        vs = np.nonzero(H[m])[0]
        for n in vs:
            others = [k for k in vs if k != n]
            app[n] += 2.0 * np.arctanh(np.prod(np.tanh(L[others] / 2.0)))
    return app


# ----------------------------------------------------------------- pins: code model and encoder

def pin_eq1_code(O):
    H = eq1_H()
    assert H.shape == (5, 10)
    assert (H.sum(axis=1) == 4).all() and (H.sum(axis=0) == 2).all()
    # any two checks share exactly one variable: no 4-cycles
    ov = H.astype(int) @ H.T.astype(int)
    assert (ov[~np.eye(5, dtype=bool)] == 1).all()
    assert gf2_rank(H) == 4                       # the five rows sum to zero over GF(2)
    code = O.Code.from_dense(H)
    assert (code.dense() == H).all()
    cb = codebook(H)
    assert len(cb) == 64                          # 2^(10 - 4)
    _, size = code.ml_decode(np.ones((1, 10), np.float32))
    assert size == 64
    assert (code.syndrome_weight(cb) == 0).all()
    assert (code.syndrome_weight(np.eye(10, dtype=np.uint8)) == 2).all()   # column weight 2


def pin_qc_expand(O):
    for name in ["qc12x24_z27_s1", "qc4x24_z81_s3"]:
        B, Z = I.load_code(name)
        code = O.QCCode(B, Z)
        assert (code.dense() == dense_lift(B, Z)).all(), name
    # Z = 1: the Eq. 1 code as a base matrix
    H = eq1_H()
    Bq = np.where(H == 1, 0, -1).astype(np.int32)
    assert (O.QCCode(Bq, 1).dense() == H).all()
    # shifts 0 and Z-1
    Bs = np.array([[0, 6, -1], [6, -1, 0]], dtype=np.int32)
    assert (O.QCCode(Bs, 7).dense() == dense_lift(Bs, 7)).all()


def pin_encoder(O):
    rng = np.random.default_rng(5)
    for name in ["qc12x24_z27_s1", "qc12x24_z81_s2", "qc4x24_z81_s3", "qc8x24_z54_s45", "qc6x24_z27_s42"]:
        B, Z = I.load_code(name)
        code = O.QCCode(B, Z)
        u = rng.integers(0, 2, size=(64, code.K), dtype=np.uint8)
        c = code.encode(u)
        H = dense_lift(B, Z).astype(np.int64)
        assert ((c.astype(np.int64) @ H.T) % 2 == 0).all(), name
        assert (c[:, :code.K] == u).all()
        assert (c == I.encode(B, Z, u)).all()


# ----------------------------------------------------------------- pins: sum-product

def pin_phi(O):
    x = np.array([1e-3, 0.1, np.log(3.0), 1.0, 5.0, 20.0, 40.0, 79.0])
    p = O.phi(x)
    assert abs(p[2] - np.log(2.0)) < 1e-15               # tanh(ln(3)/2) = 1/2
    # -ln tanh(x/2) = ln((1 + t)/(1 - t)) = 2 atanh(t) with t = exp(-x)
    assert np.allclose(p, 2.0 * np.arctanh(np.exp(-x)), rtol=1e-12, atol=0)
    assert np.allclose(O.phi(p), x, rtol=1e-9)           # phi is an involution


def pin_spa_first_iteration(O):
    H = eq1_H()
    code = O.Code.from_dense(H)
    rng = np.random.default_rng(1)
    L = (2.0 + 1.5 * rng.standard_normal((16, 10))).astype(np.float32)
    app, _, it = code.spa_flood(L, 1, early_exit=False)
    assert (it == 1).all()
    for b in range(L.shape[0]):
        ref = tanh_rule_first_iteration(H, L[b].astype(np.float64))
        assert np.allclose(app[b], ref, rtol=1e-9, atol=1e-9)


def pin_spa_degree2(O):
    code = O.Code.from_dense(np.array([[1, 1]], np.uint8))
    L = np.array([[3.5, -1.25], [0.5, 7.0], [-60.0, -2.0]], np.float32)
    app, _, _ = code.spa_flood(L, 1, early_exit=False)
    # a degree-2 check passes the other edge's message unchanged: R_0 = L_1, R_1 = L_0
    s = L.astype(np.float64).sum(axis=1)
    assert np.allclose(app, np.stack([s, s], axis=1), rtol=1e-11, atol=1e-11)


def pin_spa_erasure_readings(O):
    # an erased input (L = 0) at a degree-3 check, first iteration, both schedules.  Readings:
    # sgn(0) = +1, and |Q| is clamped from below to phi(X) before phi, so an erasure
    # contributes phi(phi(X)) = X to a check's sum instead of an infinite phi(0).
    #  * toward the erased variable: the tanh rule on the other two, 2 atanh(tanh(a/2) tanh(b/2));
    #  * toward the others: the sign of the other non-erased input (times +1 for the erasure)
    #    and a magnitude that the erasure's X pushes down to at most phi(X) ~ 2 e^-X, but
    #    not to zero.
    a, b, X = 2.5, -1.5, 80.0
    L = np.array([[0.0, a, b]], np.float32)
    H = np.array([[1, 1, 1]], np.uint8)
    code = O.Code.from_dense(H, layers=_per_check_layers(H))
    tiny = 2.0 * np.exp(-X) * (1.0 + 1e-9)
    for run in (code.spa_flood, code.spa_layered):
        _, _, _, R = run(L, 1, early_exit=False, X=X, return_messages=True)
        r0, r1, r2 = R[0]
        want0 = 2.0 * np.arctanh(np.tanh(a / 2.0) * np.tanh(b / 2.0))
        assert abs(r0 - want0) <= 1e-12 * abs(want0), (run.__name__, r0, want0)
        assert -tiny <= r1 < 0.0, (run.__name__, r1)   # sign of b; erasure counts +1
        assert 0.0 < r2 <= tiny, (run.__name__, r2)    # sign of a
    # an erasure at each of two checks of a degree-2 variable stays an erasure for that check
    # only: the other check still passes its degree-2 partner's value unchanged
    H2 = np.array([[1, 1, 0], [0, 1, 1]], np.uint8)
    code2 = O.Code.from_dense(H2, layers=_per_check_layers(H2))
    L2 = np.array([[0.0, 0.0, 3.0]], np.float32)
    app, _, _ = code2.spa_flood(L2, 1, early_exit=False, X=X)
    assert abs(app[0, 1] - 3.0) <= 1e-12 * 3.0, app         # from check 1; check 0 adds ~phi(X)
    assert 0.0 < app[0, 0] <= tiny, app                     # from check 0: the erased partner
    # a check of 11 erasures: each message is phi(10 X), which is 0 in double precision
    # (e^-800 underflows), so every posterior stays exactly 0 and decides 0 (R1: APP = 0 -> 0)
    H3 = np.ones((1, 11), np.uint8)
    code3 = O.Code.from_dense(H3, layers=_per_check_layers(H3))
    for run in (code3.spa_flood, code3.spa_layered):
        app3, bits3, _ = run(np.zeros((1, 11), np.float32), 1, early_exit=False, X=X)
        assert (app3 == 0.0).all() and (bits3 == 0).all(), (run.__name__, app3, bits3)


def pin_spa_tree_map(O):
    rng = np.random.default_rng(7)
    for trial in range(12):
        H = random_tree_H(rng, int(rng.integers(4, 15)))
        N = H.shape[1]
        L = (rng.choice([-1.0, 1.0], N) + rng.standard_normal(N)).astype(np.float32)
        assert np.abs(L).sum() < 75.0
        code = O.Code.from_dense(H)
        app, _, _ = code.spa_flood(L[None], 2 * N, early_exit=False)
        ref = map_llr(H, L.astype(np.float64))
        assert np.allclose(app[0], ref, rtol=1e-9, atol=1e-9), (trial, app[0], ref)


def pin_spa_symmetry(O):
    B, Z = I.load_code("qc12x24_z27_s1")
    code = O.QCCode(B, Z)
    _, _, c, _ = I.make_frames("qc12x24_z27_s1", 16, 2.0, 101, 102)
    L0 = I.awgn_llr(np.zeros_like(c), 2.0, 0.5, 102)      # all-zero codeword through the channel
    s = (1.0 - 2.0 * c).astype(np.float32)
    L = L0 * s                                              # the same channel seen from codeword c
    a0, b0, i0 = code.spa_flood(L0, 8, early_exit=True)
    a1, b1, i1 = code.spa_flood(L, 8, early_exit=True)
    assert np.array_equal(a1, a0 * s)
    assert np.array_equal(b1, b0 ^ c)
    assert np.array_equal(i1, i0)


def pin_spa_ml_high_snr(O):
    H = eq1_H()
    code = O.Code.from_dense(H)
    cb = codebook(H)
    rng = np.random.default_rng(3)
    c = cb[rng.integers(0, len(cb), 400)]
    L = I.awgn_llr(c, 7.0, 0.6, 33)
    _, bits, _ = code.spa_flood(L, 20, early_exit=True)
    ml, _ = code.ml_decode(L)
    agree = (bits == ml).all(axis=1).mean()
    ok = (bits == c).all(axis=1).mean()
    assert agree >= 0.995 and ok >= 0.99, (agree, ok)
    # ML is a lower bound on the frame error rate of any decoder at low SNR
    L2 = I.awgn_llr(c, 0.0, 0.6, 34)
    _, bits2, _ = code.spa_flood(L2, 20, early_exit=True)
    ml2, _ = code.ml_decode(L2)
    assert (ml2 != c).any(axis=1).mean() <= (bits2 != c).any(axis=1).mean() + 0.02


def pin_spa_iterations_and_clamp(O):
    B, Z = I.load_code("qc12x24_z27_s1")
    code = O.QCCode(B, Z)
    # noiseless channel: the codeword satisfies H at once -> one iteration
    u = I.info_bits(4, code.K, 9)
    c = I.encode(B, Z, u)
    L = (4.0 * (1.0 - 2.0 * c)).astype(np.float32)
    _, bits, it = code.spa_flood(L, 20, early_exit=True)
    assert (it == 1).all() and (bits == c).all()
    _, _, it = code.spa_flood(L, 7, early_exit=False)
    assert (it == 7).all()
    # huge LLRs: the clamp keeps |R| <= X, no inf/nan
    Lh = (1000.0 * (1.0 - 2.0 * c)).astype(np.float32)
    app, bits, _ = code.spa_flood(Lh, 3, early_exit=False, X=80.0)
    assert np.isfinite(app).all() and (bits == c).all()
    dv = code.dense().sum(axis=0)
    assert (np.abs(app - Lh) <= 80.0 * dv + 1e-9).all()


def pin_spa_clamp_closed_form(O):
    # every |Q| beyond X is clamped to X, so a check of degree d sends
    # phi((d - 1) phi(X)) = X - ln(d - 1) (to O(e^-2X)) with the sign of the others' product
    code = O.Code.from_dense(np.array([[1, 1, 1, 1]], np.uint8))
    L = np.array([[200.0, 300.0, -400.0, 500.0]], np.float32)
    for X in (80.0, 30.0):
        app, _, _ = code.spa_flood(L, 1, early_exit=False, X=X)
        sgn = np.array([-1.0, -1.0, 1.0, -1.0])
        assert np.allclose(app[0] - L[0], sgn * (X - np.log(3.0)), rtol=0, atol=1e-9), (X, app)


def pin_binary16(O):
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(4000) * 20, rng.standard_normal(1000) * 1e-5,
                        np.array([0.0, 65504.0, 65519.9, 1e-8, 2.0 ** -24, 3 * 2.0 ** -25, 1.0 + 2.0 ** -11])])
    ref = x.astype(np.float16).astype(np.float64)       # numpy: IEEE round to nearest even
    assert np.array_equal(O.round_binary16(x), ref)


def pin_spa_fp16_messages(O):
    # messages rounded to binary16 change the posterior by at most the rounding of each R
    H = eq1_H()
    code = O.Code.from_dense(H)
    rng = np.random.default_rng(2)
    L = (2.0 + 1.5 * rng.standard_normal((8, 10))).astype(np.float32)
    a64, _, _ = code.spa_flood(L, 1, early_exit=False)
    a16, _, _ = code.spa_flood(L, 1, early_exit=False, fp16_msgs=True)
    R64 = a64 - L
    assert np.all(np.abs(a16 - a64) <= 2 * 2.0 ** -11 * np.abs(R64) + 1e-12)
    assert not np.array_equal(a16, a64)


# ----------------------------------------------------------------- pins: layered sum-product

def _per_check_layers(H):
    return np.arange(H.shape[0] + 1, dtype=np.int32)


def pin_spa_layered_path_sweep(O):
    # repetition code on a path: check k joins x_k and x_{k+1}, one check per layer in
    # order.  A degree-2 check passes the other edge's value unchanged, so one layered
    # iteration carries the running sum forward: APP_k = L_0 + ... + L_{min(k+1, n-1)}
    # (flooding would give L_{k-1} + L_k + L_{k+1} instead).
    n = 12
    H = np.zeros((n - 1, n), np.uint8)
    for k in range(n - 1):
        H[k, k] = H[k, k + 1] = 1
    code = O.Code.from_dense(H, layers=_per_check_layers(H))
    rng = np.random.default_rng(21)
    L = rng.uniform(-3.0, 3.0, (4, n)).astype(np.float32)
    app, _, it = code.spa_layered(L, 1, early_exit=False)
    cs = np.cumsum(L.astype(np.float64), axis=1)
    ref = np.concatenate([cs[:, 1:], cs[:, -1:]], axis=1)
    assert np.allclose(app, ref, rtol=1e-10, atol=1e-10), (app, ref)
    assert (it == 1).all()


def pin_spa_layered_tree_map(O):
    # on a cycle-free graph the layered schedule converges to the exact bitwise MAP
    rng = np.random.default_rng(17)
    for trial in range(10):
        H = random_tree_H(rng, int(rng.integers(4, 15)))
        N = H.shape[1]
        L = (rng.choice([-1.0, 1.0], N) + rng.standard_normal(N)).astype(np.float32)
        assert np.abs(L).sum() < 75.0
        code = O.Code.from_dense(H, layers=_per_check_layers(H))
        app, _, _ = code.spa_layered(L[None], 2 * N, early_exit=False)
        ref = map_llr(H, L.astype(np.float64))
        assert np.allclose(app[0], ref, rtol=1e-9, atol=1e-9), (trial, app[0], ref)


def pin_spa_layered_posterior_invariant(O):
    # every check update removes its old message and adds the new one, so at any point
    # APP_n = L_n + sum_m R_mn; binary16 storage leaves every message a binary16 value
    B, Z = I.load_code("qc12x24_z27_s1")
    code = O.QCCode(B, Z)
    _, _, _, L = I.make_frames("qc12x24_z27_s1", 6, 1.5, 201, 202)
    for fp16 in (False, True):
        app, _, _, R = code.spa_layered(L, 3, early_exit=False, fp16_msgs=fp16, return_messages=True)
        tot = L.astype(np.float64).copy()
        np.add.at(tot.T, code.ci, R.T)
        assert np.allclose(app, tot, rtol=1e-9, atol=1e-9)
        if fp16:
            assert np.array_equal(R, R.astype(np.float16).astype(np.float64))
            app64, _, _ = code.spa_layered(L, 3, early_exit=False)
            assert not np.array_equal(app, app64) and np.allclose(app, app64, rtol=0.05, atol=0.05)


def pin_spa_layered_symmetry(O):
    B, Z = I.load_code("qc12x24_z27_s1")
    code = O.QCCode(B, Z)
    _, _, c, _ = I.make_frames("qc12x24_z27_s1", 16, 2.0, 111, 112)
    L0 = I.awgn_llr(np.zeros_like(c), 2.0, 0.5, 112)
    s = (1.0 - 2.0 * c).astype(np.float32)
    a0, b0, i0 = code.spa_layered(L0, 8, early_exit=True)
    a1, b1, i1 = code.spa_layered(L0 * s, 8, early_exit=True)
    assert np.array_equal(a1, a0 * s)
    assert np.array_equal(b1, b0 ^ c)
    assert np.array_equal(i1, i0)
    # noiseless channel: one iteration, decisions = the codeword
    u = I.info_bits(4, code.K, 9)
    cw = I.encode(B, Z, u)
    _, bits, it = code.spa_layered((4.0 * (1.0 - 2.0 * cw)).astype(np.float32), 20, early_exit=True)
    assert (it == 1).all() and (bits == cw).all()


def pin_spa_layered_clamp_closed_form(O):
    # one check of degree 4, |L| far beyond X: each message is X - ln 3 (as for flooding)
    H = np.array([[1, 1, 1, 1]], np.uint8)
    code = O.Code.from_dense(H, layers=_per_check_layers(H))
    L = np.array([[200.0, 300.0, -400.0, 500.0]], np.float32)
    for X in (80.0, 30.0):
        app, _, _ = code.spa_layered(L, 1, early_exit=False, X=X)
        sgn = np.array([-1.0, -1.0, 1.0, -1.0])
        assert np.allclose(app[0] - L[0], sgn * (X - np.log(3.0)), rtol=0, atol=1e-9), (X, app)


def pin_spa_layered_converges_faster(O):
    # the layered schedule reuses updated posteriors within an iteration; on a QC code it
    # needs markedly fewer iterations than flooding at no worse frame error rate (Sec. II)
    B, Z = I.load_code("qc12x24_z27_s1")
    code = O.QCCode(B, Z)
    _, _, c, L = I.make_frames("qc12x24_z27_s1", 192, 2.0, 301, 302)
    _, bf, itf = code.spa_flood(L, 20, early_exit=True)
    _, bl, itl = code.spa_layered(L, 20, early_exit=True)
    assert itl.mean() < 0.7 * itf.mean(), (itl.mean(), itf.mean())
    assert (bl != c).any(axis=1).sum() <= (bf != c).any(axis=1).sum() + 2


# ----------------------------------------------------------------- pins: integer layered min-sum

def pin_quantize(O):
    L = np.array([1.25, 1.75, -1.25, 20.0, -0.2, 0.25, 0.75, -15.6, 15.4, -100.0], np.float32)
    q = O.quantize(L, 2.0, 31)
    assert q.tolist() == [2, 4, -2, 31, 0, 0, 2, -31, 31, -31]


def _nms_code(H, layers):
    from oracle import oracle as _  # noqa: F401  (layers carried by Code)
    return H, np.asarray(layers, np.int32)


def pin_nms_hand_values(O):
    # degree-2 check, q = [10, -7]: R_0 = -(3*7 >> 2) = -5, R_1 = +(3*10 >> 2) = +7
    c2 = O.Code.from_dense(np.array([[1, 1]], np.uint8), layers=[0, 1])
    app, bits, _ = c2.nms_layered(np.array([[10, -7]], np.int8), 1, early_exit=False)
    assert app.tolist() == [[5, 0]] and bits.tolist() == [[0, 0]]
    # degree-3 check with a tie at the minimum, q = [4, -4, 9]: min1 = min2 = 4, S = 1
    c3 = O.Code.from_dense(np.array([[1, 1, 1]], np.uint8), layers=[0, 1])
    app, _, _ = c3.nms_layered(np.array([[4, -4, 9]], np.int8), 1, early_exit=False)
    assert app.tolist() == [[1, -1, 6]]


def pin_nms_layer_order(O):
    # checks {0,1} and {0,2} in two layers: layer 1 must see the APP_0 written by layer 0.
    H = np.array([[1, 1, 0], [1, 0, 1]], np.uint8)
    code = O.Code.from_dense(H, layers=[0, 1, 2])
    app, bits, it = code.nms_layered(np.array([[2, 8, -6]], np.int8), 1, early_exit=False)
    # layer 0: Q=[2,8] -> R=[+6,+1], APP0=8, APP1=9; layer 1: Q=[8,-6] -> R=[-4,+6], APP0=4, APP2=0
    assert app.tolist() == [[4, 9, 0]]
    _, _, it = code.nms_layered(np.array([[2, 8, -6]], np.int8), 5, early_exit=True)
    assert it.tolist() == [1]


def pin_nms_saturation(O):
    H = np.array([[1, 1, 0], [1, 0, 1]], np.uint8)
    code = O.Code.from_dense(H, layers=[0, 1, 2])
    q = np.array([[20, 30, 30]], np.int8)
    # it 1: layer 0 Q=[20,30] -> R=[22,15], APP=[42,45]; layer 1 Q0 = sat(42) = 31, Q2 = 30
    #       -> R=[22,23], APP=[53,45,53].  it 2: layer 0 Q=[31,30] -> APP=[53,53,53]
    app, _, _ = code.nms_layered(q, 1, early_exit=False)
    assert app.tolist() == [[53, 45, 53]]
    app, _, _ = code.nms_layered(q, 2, early_exit=False)
    assert app.tolist() == [[53, 53, 53]]
    app, _, _ = code.nms_layered(q, 1, early_exit=False, app_sat=40)
    assert app.tolist() == [[40, 40, 40]]


def pin_nms_real_crosscheck(O):
    # with saturation out of reach, the integer rule equals sgn * floor(0.75 * min over others)
    B, Z = I.load_code("qc4x24_z27_s43")
    code = O.QCCode(B, Z)
    _, _, c, L = I.make_frames("qc4x24_z27_s43", 24, 3.0, 5, 6)
    q = O.quantize(L, 2.0, 31)
    big = 1 << 24
    for T in (1, 2, 4):
        ai, _, _ = code.nms_layered(q, T, early_exit=False, msg_sat=big, app_sat=big)
        ar = code.nms_layered_real(q.astype(np.float64), T, 0.75)
        assert np.array_equal(ai.astype(np.float64), ar), T


def pin_nms_symmetry(O):
    B, Z = I.load_code("qc4x24_z81_s3")
    code = O.QCCode(B, Z)
    _, _, c, _ = I.make_frames("qc4x24_z81_s3", 32, 3.5, 7, 8)
    L0 = I.awgn_llr(np.zeros_like(c), 3.5, code.K / code.N, 8)
    s = (1 - 2 * c.astype(np.int32))
    q0 = O.quantize(L0, 2.0, 31)
    q1 = O.quantize(L0 * s.astype(np.float32), 2.0, 31)
    assert np.array_equal(q1.astype(np.int32), q0.astype(np.int32) * s)   # rint is odd-symmetric
    a0, b0, i0 = code.nms_layered(q0, 10, early_exit=False)
    a1, b1, i1 = code.nms_layered(q1, 10, early_exit=False)
    assert np.array_equal(a1, a0 * s)
    nz = a0 != 0                       # hard decision 0 at APP = 0 breaks the symmetry there
    assert np.array_equal(b1[nz], (b0 ^ c)[nz])


def pin_nms_ml_high_snr(O):
    H = eq1_H()
    cb = codebook(H)
    code = O.Code.from_dense(H, layers=np.arange(6))
    rng = np.random.default_rng(4)
    c = cb[rng.integers(0, len(cb), 400)]
    L = I.awgn_llr(c, 8.0, 0.6, 44)
    q = O.quantize(L, 2.0, 31)
    _, bits, _ = code.nms_layered(q, 10, early_exit=True)
    ml, _ = code.ml_decode(L)
    assert (bits == ml).all(axis=1).mean() >= 0.99
    assert (bits == c).all(axis=1).mean() >= 0.99


def pin_ml_decode(O):
    H = eq1_H()
    code = O.Code.from_dense(H)
    cb = codebook(H)
    rng = np.random.default_rng(8)
    L = rng.standard_normal((50, 10)).astype(np.float32) * 2
    ml, _ = code.ml_decode(L)
    score = (1.0 - 2.0 * cb) @ L.astype(np.float64).T          # [|C|, B]
    ref = cb[np.argmax(score, axis=0)]
    assert np.array_equal(ml, ref)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
