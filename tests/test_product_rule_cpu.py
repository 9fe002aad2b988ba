"""The sum-product check rule in the product (tanh) domain, as the on-chip decoders evaluate it,
against the FP64 oracle's phi-domain rule (Sec. II): a CPU restatement in FP32 numpy.

The decoders write R'_k = prod sgn * min(X, phi(sum_{j != k} phi(a_j))) as ln(alpha_k / beta_k),
where d_j = e^-a_j and the pair (alpha, beta) of the other edges follows
(alpha, beta) <- (alpha + d beta, beta + d alpha) from (1, 0).  Both forms are the same
function; these tests check that the FP32 evaluation keeps the relative accuracy the oracle
tolerances need at the extremes (|Q| -> 0, |Q| past the clamp, many reliable edges), in
the prefix / suffix form (rows up to degree 8) and in the grouped form (wider rows), and
that the clamp [phi(X), X] maps onto the exponent as stated.
"""
import numpy as np
import pytest

from oracle import oracle as O

F = np.float32
LOG2E = F(1.4426950408889634)
LN2 = F(0.6931471805599453)


def pair_mul(a1, b1, a2, b2):
    return (b1 * b2 + a1 * a2).astype(F), (b1 * a2 + a1 * b2).astype(F)


def step(a, b, d):
    """One more edge's map applied to the pair (alpha, beta)."""
    return (a + d * b).astype(F), (b + d * a).astype(F)


def factors(q, X):
    """d = e^-a with a = |Q| clamped to [phi(X), X], through the base-2 exponent."""
    Xb = F(X) * LOG2E
    Pb = F(O.phi(np.array([X]))[0] * np.log2(np.e))
    arg = np.minimum(np.maximum(-np.abs(q) * LOG2E, -Xb), -Pb).astype(F)
    return np.exp2(arg).astype(F)


def exclusive_pairs_prefix_suffix(d):
    """(alpha_k, beta_k) of the other edges of each row from prefix and suffix maps."""
    B, D = d.shape
    one, zero = np.ones(B, F), np.zeros(B, F)
    sa, sb = [None] * (D + 1), [None] * (D + 1)
    sa[D], sb[D] = one, zero
    for k in range(D - 1, -1, -1):
        sa[k], sb[k] = step(sa[k + 1], sb[k + 1], d[:, k])
    al, be = np.empty_like(d), np.empty_like(d)
    pa, pb = one, zero
    for k in range(D):
        al[:, k], be[:, k] = pair_mul(pa, pb, sa[k + 1], sb[k + 1])
        pa, pb = step(pa, pb, d[:, k])
    return al, be


def exclusive_pairs_grouped(d, G=8):
    """The grouped form of wide rows: each group's product, then per group the product of
    the other groups as the prefix start, and prefix / suffix maps inside the group."""
    B, D = d.shape
    groups = [d[:, g:g + G] for g in range(0, D, G)]
    one, zero = np.ones(B, F), np.zeros(B, F)
    prod = []
    for gd in groups:
        a, b = one, zero
        for i in range(gd.shape[1]):
            a, b = step(a, b, gd[:, i])
        prod.append((a, b))
    al, be = np.empty_like(d), np.empty_like(d)
    for g, gd in enumerate(groups):
        pa, pb = one, zero
        first = True
        for h, (a, b) in enumerate(prod):
            if h == g:
                continue
            pa, pb = (a, b) if first else pair_mul(pa, pb, a, b)
            first = False
        n = gd.shape[1]
        sa, sb = [None] * (n + 1), [None] * (n + 1)
        sa[n], sb[n] = one, zero
        for i in range(n - 1, -1, -1):
            sa[i], sb[i] = step(sa[i + 1], sb[i + 1], gd[:, i])
        for i in range(n):
            al[:, g * G + i], be[:, g * G + i] = pair_mul(pa, pb, sa[i + 1], sb[i + 1])
            pa, pb = step(pa, pb, gd[:, i])
    return al, be


def product_rule(q, X, grouped):
    d = factors(q, X)
    al, be = exclusive_pairs_grouped(d) if grouped else exclusive_pairs_prefix_suffix(d)
    mag = ((np.log2(al) - np.log2(be)) * LN2).astype(F)
    neg = np.signbit(q) & (q != 0)  # sgn(0) = +1, as the oracle reads it
    others = (neg.sum(axis=1, keepdims=True) - neg) % 2 == 1
    return np.where(others, -mag, mag)


def oracle_rule(q, X):
    """The oracle's messages after one flooding iteration of a single check (R = 0, Q = L)."""
    B, D = q.shape
    oc = O.Code(1, D, [0, D], list(range(D)))
    _, _, _, R = oc.spa_flood(q, 1, early_exit=False, X=X, return_messages=True)
    return R


def extreme_inputs(D, B, seed):
    rng = np.random.default_rng(seed)
    q = rng.normal(2.0, 3.0, (B, D)).astype(F)
    pick = rng.random((B, D))
    q[pick < 0.08] = F(0.0)                                                 # erasures
    q[(pick >= 0.08) & (pick < 0.14)] = rng.choice([-1, 1], ((pick >= 0.08) & (pick < 0.14)).sum()) * F(1e-6)
    big = (pick >= 0.14) & (pick < 0.30)
    q[big] = rng.choice([-1, 1], big.sum()) * rng.uniform(20.0, 120.0, big.sum()).astype(F)  # past the clamp too
    q[: B // 8] = rng.uniform(30.0, 75.0, (B // 8, D)).astype(F)             # every edge reliable
    return q


@pytest.mark.parametrize("D", [2, 3, 5, 7, 8, 12, 19, 24])
@pytest.mark.parametrize("X", [80.0, 6.0, 2.5])
def test_product_rule_matches_the_oracle(D, X):
    q = extreme_inputs(D, 4000, 100 + D)
    ref = oracle_rule(q, X)
    got = product_rule(q, X, grouped=D > 8)
    err = np.abs(got.astype(np.float64) - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 2e-6, (D, X, float(err.max()))
    # signs agree wherever the message is above FP32 resolution: next to a nearly erased edge
    # (|Q| ~ 1e-6) alpha ~ beta and lg2 alpha - lg2 beta rounds to +-2e-7, either sign, an
    # absolute error inside the bound above
    sure = np.abs(ref) > 1e-5
    assert np.array_equal(np.signbit(got)[sure], np.signbit(ref)[sure]), (D, X)


@pytest.mark.parametrize("D", [12, 20])
def test_grouped_and_prefix_suffix_forms_agree(D):
    q = extreme_inputs(D, 2000, 7 + D)
    a = product_rule(q, 80.0, grouped=True)
    b = product_rule(q, 80.0, grouped=False)
    assert np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))) <= 2e-6


def test_result_never_exceeds_the_clamp():
    # phi(sum of the others' phi) <= the others' smallest clamped |Q| <= X: the decoders
    # apply no clamp to the result, which rounding may exceed only by an ulp
    for X in (80.0, 6.0, 2.5):
        q = extreme_inputs(8, 4000, 3)
        got = np.abs(product_rule(q, X, grouped=False))
        assert got.max() <= X * (1 + 4e-7), (X, float(got.max()))


def test_the_textbook_tanh_product_would_fail_here():
    # the same rule through P = prod tanh(a_j / 2) and ln((1 + P) / (1 - P)) loses 1 - P to
    # cancellation when every other edge is reliable: the pair form exists because of this
    q = np.full((1, 6), 18.0, F)
    ref = oracle_rule(q, 80.0)
    t = np.tanh(q.astype(F) / F(2)).astype(F)
    P = (np.prod(t) / t).astype(F)
    naive = np.log(((1 + P) / (1 - P)).astype(F)).astype(F)
    good = product_rule(q, 80.0, grouped=False)
    assert not np.all(np.isfinite(naive)) or np.max(np.abs(naive - ref)) > 1e-2
    assert np.max(np.abs(good - ref) / np.maximum(1.0, np.abs(ref))) <= 2e-6
