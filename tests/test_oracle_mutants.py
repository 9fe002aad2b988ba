"""Each plausible mistake planted in a copy of the oracle must fail at least one pin.

The mistakes are planted in a temporary copy of ldpc_oracle.c, compiled on the CPU and
loaded in place of the real oracle; the pins are the same functions test_oracle_pins runs.
"""
import os
import subprocess

import pytest

from oracle import oracle as O
from tests import oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "ldpc_oracle.c")

# (name, text to replace, replacement, which occurrence)
MUTANTS = [
    ("spa_sign_flipped", "double r = sgn * mag;", "double r = -sgn * mag;", 0),
    ("spa_self_in_sum", "if (k2 == k) continue;\n                                if (Q[k2] < 0.0) sgn = -sgn;",
     "if (Q[k2] < 0.0) sgn = -sgn;", 0),
    ("spa_no_extrinsic", "Q[k] = app[ci[e0 + k]] - R[e0 + k];", "Q[k] = app[ci[e0 + k]];", 0),
    ("spa_vn_drops_channel", "for (int n = 0; n < N; n++) app[n] = (double)Lb[n];\n                    for (int m = 0;",
     "for (int n = 0; n < N; n++) app[n] = 0.0;\n                    for (int m = 0;", 0),
    ("spa_exit_inverted", "if (early_exit && syndrome_weight(M, rp, ci, hd) == 0) {",
     "if (early_exit && syndrome_weight(M, rp, ci, hd) != 0) {", 0),
    ("spa_hard_decision", "hd[n] = app[n] < 0.0;", "hd[n] = app[n] > 0.0;", 0),
    ("spa_no_upper_clamp", "if (a > X) a = X;", "", 0),
    ("phi_log_not_log1p", "return log1p(2.0 / expm1(x));", "return log(2.0 / expm1(x));", 0),
    ("nms_alpha_shift", "int32_t magp = (alpha_num * mag) >> alpha_shift;",
     "int32_t magp = (alpha_num * mag) >> (alpha_shift - 1);", 0),
    ("nms_no_min2_update", "} else if (a < min2) {", "} else if (0) {", 0),
    ("nms_sign_not_extrinsic", "int32_t neg = S ^ (Q[k] < 0);", "int32_t neg = S;", 0),
    ("nms_no_msg_sat", "Q[k] = sat(app[ci[e0 + k]] - R[e0 + k], msg_sat);", "Q[k] = app[ci[e0 + k]] - R[e0 + k];", 0),
    ("nms_no_app_sat", "app[ci[e0 + k]] = sat(Q[k] + R[e0 + k], app_sat);", "app[ci[e0 + k]] = Q[k] + R[e0 + k];", 0),
    ("nms_min_swapped", "int32_t mag = (k == arg) ? min2 : min1;", "int32_t mag = (k == arg) ? min1 : min2;", 0),
    ("nms_exit_inverted", "if (early_exit && syndrome_weight(M, rp, ci, hd) == 0) {",
     "if (early_exit && syndrome_weight(M, rp, ci, hd) != 0) {", 2),
    ("nms_layers_reversed", "for (int l = 0; l < nl; l++) {\n                        for (int m = lp[l];",
     "for (int l = nl - 1; l >= 0; l--) {\n                        for (int m = lp[l];", 1),
    # layered sum-product (second occurrence of the lines it shares with the flooding routine)
    ("spal_sign_flipped", "double r = sgn * mag;", "double r = -sgn * mag;", 1),
    ("spal_no_extrinsic", "Q[k] = app[ci[e0 + k]] - R[e0 + k];", "Q[k] = app[ci[e0 + k]];", 1),
    ("spal_app_from_channel", "app[ci[e0 + k]] = Q[k] + Rn[k];", "app[ci[e0 + k]] = (double)Lb[ci[e0 + k]] + Rn[k];", 0),
    ("spal_messages_not_kept", "R[e0 + k] = Rn[k];\n", "\n", 0),
    ("spal_layers_reversed", "for (int l = 0; l < nl; l++) {\n                        for (int m = lp[l];",
     "for (int l = nl - 1; l >= 0; l--) {\n                        for (int m = lp[l];", 0),
    ("spal_fp16_ignored", "Rn[k] = fp16_msgs ? round_binary16(r) : r;", "Rn[k] = r;", 0),
    ("spal_no_upper_clamp", "if (a > X) a = X;", "", 1),
    ("spal_exit_inverted", "if (early_exit && syndrome_weight(M, rp, ci, hd) == 0) {",
     "if (early_exit && syndrome_weight(M, rp, ci, hd) != 0) {", 1),
    ("spal_hard_decision", "hd[n] = app[n] < 0.0;", "hd[n] = app[n] > 0.0;", 1),
    ("encoder_p1_shift", "p[1 * Z + r] = lam[r] ^ p[(r + s_top) % Z];", "p[1 * Z + r] = lam[r] ^ p[r];", 0),
    ("encoder_transposed_shift", "lam[i * Z + r] ^= ub[j * Z + (r + s) % Z] & 1;",
     "lam[i * Z + r] ^= ub[j * Z + (r + Z - s) % Z] & 1;", 0),
    ("qc_shift_direction", "ci[e++] = j * Z + (r + s) % Z;", "ci[e++] = j * Z + (r + Z - s) % Z;", 0),
    ("quantize_round_half_away", "float r = rintf(p);", "float r = roundf(p);", 0),
    ("binary16_precision", "int q = e - 11;", "int q = e - 10;", 0),
    ("ml_correlation_sign", "corr += ((cb[i] >> n) & 1u) ? -(double)Lb[n] : (double)Lb[n];",
     "corr += ((cb[i] >> n) & 1u) ? (double)Lb[n] : -(double)Lb[n];", 0),
    # readings at an erased input (Q = 0): the lower clamp and sgn(0) = +1, both schedules
    ("spa_no_lower_clamp", "if (a < phiX) a = phiX;", "", 0),
    ("spa_sign_of_zero", "if (Q[k2] < 0.0) sgn = -sgn;", "if (Q[k2] <= 0.0) sgn = -sgn;", 0),
    ("spal_no_lower_clamp", "if (a < phiX) a = phiX;", "", 1),
    ("spal_sign_of_zero", "if (Q[k2] < 0.0) sgn = -sgn;", "if (Q[k2] <= 0.0) sgn = -sgn;", 1),
    ("spa_messages_not_kept", "for (int e = 0; e < E; e++) R[e] = Rn[e];", "", 0),
    ("spa_channel_doubled", "for (int n = 0; n < N; n++) app[n] = (double)Lb[n];\n                    for (int m = 0;",
     "for (int n = 0; n < N; n++) app[n] = 2.0 * (double)Lb[n];\n                    for (int m = 0;", 0),
    ("syndrome_or_not_xor", "for (int e = rp[m]; e < rp[m + 1]; e++) par ^= c[ci[e]] & 1;",
     "for (int e = rp[m]; e < rp[m + 1]; e++) par |= c[ci[e]] & 1;", 0),
    ("nms_min1_never_set", "if (a < min1) {", "if (0) {", 0),
    # a posterior of exactly 0 decides 0 (R1), in all three decoders; a tie at the minimum
    # leaves min2 = min1
    ("spa_hd_zero_is_one", "hd[n] = app[n] < 0.0;", "hd[n] = app[n] <= 0.0;", 0),
    ("spal_hd_zero_is_one", "hd[n] = app[n] < 0.0;", "hd[n] = app[n] <= 0.0;", 1),
    ("nms_hd_zero_is_one", "hd[n] = app[n] < 0;", "hd[n] = app[n] <= 0;", 0),
    ("nms_min2_skips_tie", "} else if (a < min2) {", "} else if (a < min2 && a != min1) {", 0),
    # binary16 message storage and the exclusive magnitude sum of the flooding routine
    ("spa_fp16_ignored", "Rn[e0 + k] = fp16_msgs ? round_binary16(r) : r;", "Rn[e0 + k] = r;", 0),
    ("binary16_round_away", "double r = nearbyint(ldexp(a, -q));", "double r = round(ldexp(a, -q));", 0),
    ("binary16_no_subnormal_floor", "if (q < -24) q = -24;", "", 0),
    ("binary16_overflow_threshold", "if (a >= 65520.0) return copysign(INFINITY, x);",
     "if (a > 65504.0) return copysign(INFINITY, x);", 0),
    ("spa_magnitude_includes_self",
     "if (k2 == k) continue;\n                                if (Q[k2] < 0.0) sgn = -sgn;\n                                double a = fabs(Q[k2]);",
     "if (Q[k2] < 0.0 && k2 != k) sgn = -sgn;\n                                double a = fabs(Q[k2]);", 0),
]


def _plant(src, old, new, occ):
    idx = -1
    for _ in range(occ + 1):
        idx = src.find(old, idx + 1)
        assert idx >= 0, f"mutation site not found: {old!r}"
    return src[:idx] + new + src[idx + len(old):]


@pytest.mark.parametrize("name,old,new,occ", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new, occ):
    src = open(SRC).read()
    mutant = _plant(src, old, new, occ)
    assert mutant != src
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(mutant)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", str(c), "-o", str(so), "-lm"],
                   check=True, capture_output=True)
    failed = []
    with O.use_library(str(so)):
        for pin in P.ALL_PINS:
            try:
                pin(O)
            except (AssertionError, RuntimeError, ValueError, FloatingPointError):
                failed.append(pin.__name__)
                break  # one catching pin is enough
    assert failed, f"no pin caught mutant {name}"
