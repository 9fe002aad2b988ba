"""The binary16 identities behind the two-codewords-per-thread integer min-sum kernel,
checked exhaustively on the CPU in numpy float16 (every operation rounds to binary16,
round-to-nearest-even, as the packed half-precision instructions do).

The kernel computes the integer layered normalised min-sum with packed half-precision
instructions; this is exact only because every step below lands on the same integer as the
integer definition for every input the parameters allow.  A fused multiply-add rounds once,
so it is modelled by the exact product-sum (float64 here, exact for these magnitudes)
rounded once to float16."""
import numpy as np

H = np.float16


def fma16(a, b, c):
    return H(np.float64(a) * np.float64(b) + np.float64(c))


def admitted(alpha_num, alpha_shift, msg_sat, app_sat=127):
    """The parameter sets for which the kernel is used (the host's exactness condition)."""
    if not (1 <= msg_sat <= 127 and msg_sat <= app_sat <= 127 and 0 <= alpha_shift <= 10 and alpha_num >= 0):
        return False
    if (alpha_num * msg_sat) >> alpha_shift > 127:
        return False
    return 2 * alpha_num * msg_sat + (1 << alpha_shift) <= 2047


def test_scaled_minimum_is_the_integer_floor():
    # floor(alpha_num * m / 2^shift) as round(alpha m - delta) at spacing 1 (+1536, -1536),
    # for every admitted (alpha_num, shift, msg_sat) and every m in [0, msg_sat]
    checked = 0
    for shift in range(0, 8):
        for num in range(0, 40):
            for sat in (1, 7, 15, 31, 63, 100, 127):
                if not admitted(num, shift, sat):
                    continue
                alpha = H(num / 2 ** shift)
                ndelta = H(1.0 / 2 ** (shift + 1) - 0.5)
                assert float(alpha) == num / 2 ** shift and float(ndelta) == 1.0 / 2 ** (shift + 1) - 0.5
                for m in range(0, sat + 1):
                    y = fma16(H(m), alpha, ndelta)
                    z = H(H(y + H(1536)) + H(-1536))
                    assert float(z) == (num * m) >> shift, (num, shift, sat, m)
                    checked += 1
    assert checked > 10000


def test_check_node_input_saturation():
    # Q = sat(APP - R, msg_sat) as ((APP - (1024 + R + 128)) + 1152) then min/max, for every
    # APP in [-127, 127] and R in [-127, 127]; a zero Q is +0 (sign bit = [Q < 0])
    app = np.arange(-127, 128)
    r = np.arange(-127, 128)
    A, R = np.meshgrid(app, r, indexing="ij")
    rb = (1024 + R + 128).astype(H)
    for sat in (15, 31, 63, 127):
        q = (A.astype(H) - rb).astype(H)
        q = (q + H(1152)).astype(H)
        q = np.maximum(np.minimum(q, H(sat)), H(-sat))
        assert np.array_equal(q.astype(np.int64), np.clip(A - R, -sat, sat))
        assert not np.signbit(q[q == 0]).any()


def test_message_bytes_round_trip():
    # R in [-127, 127]: 1024 + (R + 128) has the byte R + 128 in the low mantissa bits under
    # the exponent of 1024 (bits 0x64__), and R + 1152 narrows back to that byte
    for R in range(-127, 128):
        b = R + 128
        widened = np.array([0x6400 | b], np.uint16).view(H)[0]
        assert float(widened) == 1024 + b and float(widened) - 1152 == R
        narrowed = np.array([H(R) + H(1152)], H).view(np.uint16)[0]
        assert narrowed >> 8 == 0x64 and (narrowed & 0xFF) == b
    # R = -0 (a zero magnitude given the check's negative sign) narrows to the byte of +0
    assert np.array([H(-0.0) + H(1152)], H).view(np.uint16)[0] & 0xFF == 128


def test_posterior_update_never_yields_negative_zero():
    # APP = Q + R with |Q| <= msg_sat and R = +-floor(alpha min): exact, and +0 when it cancels
    # (also for R = -0), so the sign bit of APP is the hard decision [APP < 0]
    q = np.arange(-127, 128).astype(H)
    for R in list(range(-127, 128)) + [-0.0]:
        s = (q + H(R)).astype(H)
        assert np.array_equal(s.astype(np.float64), q.astype(np.float64) + R)
        assert not np.signbit(s[s == 0]).any()


def test_admitted_parameter_sets_include_the_defaults():
    assert admitted(3, 2, 31)                      # alpha = 0.75, messages in [-31, 31]
    assert admitted(7, 3, 31, 63) and admitted(1, 0, 63) and admitted(3, 2, 15, 15)
    assert not admitted(9, 4, 127)                 # 2 * 9 * 127 + 16 > 2047: the one-per-thread kernel
    assert not admitted(15, 3, 127)                # a message magnitude above 127
