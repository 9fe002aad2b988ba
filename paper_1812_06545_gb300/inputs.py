"""Seeded synthetic inputs for the LDPC decoder: codes, codewords and channel LLRs.

This module is the one place both sides of every parity check draw their inputs from:
the CUDA path (tests, bench) and the CPU oracle (tests, CPU baseline).  It holds none of
the decoding arithmetic (no check-node, variable-node, posterior or syndrome logic):

* ``SplitMix64`` - the published 64-bit mixing generator (Steele, Lea & Flood, 2014),
  used only to draw the quasi-cyclic base matrices;
* ``qc_base_matrix`` - the seeded QC base-matrix recipe: a dual-diagonal ("staircase")
  parity half in the style of IEEE 802.11n and info columns of degree 3 or 4 with
  cyclic shifts uniform in [0, Z).  The paper (Sec. II, Eq. 1) defines a code by its
  H-matrix only; the quasi-cyclic lifting is this library's reading;
* ``encode`` - systematic encoding of that recipe by dual-diagonal back-substitution,
  used only to produce transmitted codewords;
* ``awgn_llr`` - BPSK (bit 0 -> +1) over AWGN, channel LLR L = 2y/sigma^2 stored as fp32.

The committed base files under ``codes/`` were written by ``write_code_files``; tests
check that the generator still reproduces them byte for byte.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

CODES_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "codes")

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a Weyl sequence fed to a 64-bit mixer."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Integer uniform in [0, n) by multiply-shift of the top 32 bits."""
        return ((self.next() >> 32) * n) >> 32


def _code_seed(seed: int, mb: int, nb: int, Z: int) -> int:
    return ((seed << 32) ^ (mb << 24) ^ (nb << 12) ^ Z) & _M64


def qc_base_matrix(mb: int, nb: int, Z: int, seed: int) -> np.ndarray:
    """Seeded QC base matrix, shape (mb, nb), entries -1 (zero block) or a shift in [0, Z).

    Parity half (block columns kb..nb-1, kb = nb - mb):
      column kb     : shift 1 at row 0, shift 0 at row mb//2, shift 1 at row mb-1 (mod Z);
      column kb + c : shift 0 at rows c-1 and c, for c = 1..mb-1 (the staircase).
    Info columns j < kb: degree 3 or 4 (one draw, uniform), distinct rows drawn by a
    partial Fisher-Yates shuffle, then one shift uniform in [0, Z) per chosen row in draw
    order.  4-cycles are not filtered.
    """
    if mb < 3 or nb <= mb or Z < 1:
        raise ValueError("recipe needs mb >= 3, nb > mb, Z >= 1")
    kb = nb - mb
    B = -np.ones((mb, nb), dtype=np.int32)
    B[0, kb] = 1 % Z
    B[mb // 2, kb] = 0
    B[mb - 1, kb] = 1 % Z
    for c in range(1, mb):
        B[c - 1, kb + c] = 0
        B[c, kb + c] = 0
    rng = SplitMix64(_code_seed(seed, mb, nb, Z))
    for j in range(kb):
        d = 3 + (rng.next() >> 63)
        d = min(d, mb)
        rows = list(range(mb))
        for i in range(d):
            k = i + rng.below(mb - i)
            rows[i], rows[k] = rows[k], rows[i]
        for i in rows[:d]:
            B[i, j] = rng.below(Z)
    return B


def code_name(mb: int, nb: int, Z: int, seed: int) -> str:
    return f"qc{mb}x{nb}_z{Z}_s{seed}"


def format_base(B: np.ndarray, Z: int, header: str = "") -> str:
    mb, nb = B.shape
    lines = []
    if header:
        lines += ["# " + h for h in header.splitlines()]
    lines.append("# entries: -1 = zero block, s >= 0 = identity cyclically shifted so that")
    lines.append("# row r of the block has its one in column (r + s) mod Z")
    lines.append(f"{mb} {nb} {Z}")
    for i in range(mb):
        lines.append(" ".join(f"{int(v):3d}" for v in B[i]))
    return "\n".join(lines) + "\n"


def parse_base(text: str):
    """Parse a base-matrix text file -> (B int32 [mb, nb], Z)."""
    rows = [ln.split() for ln in text.splitlines() if ln.strip() and not ln.lstrip().startswith("#")]
    mb, nb, Z = (int(x) for x in rows[0])
    B = np.array([[int(x) for x in r] for r in rows[1:]], dtype=np.int32)
    if B.shape != (mb, nb):
        raise ValueError(f"base shape {B.shape} != header ({mb}, {nb})")
    return B, Z


def load_code(name: str):
    with open(os.path.join(CODES_DIR, name + ".txt")) as f:
        return parse_base(f.read())


# The seeded codes used by the workloads below.  (mb, nb, Z, seed).
CODE_SPECS = {
    "qc12x24_z27_s1": (12, 24, 27, 1),     # rate 1/2, N = 648
    "qc12x24_z81_s2": (12, 24, 81, 2),     # rate 1/2, N = 1944
    "qc4x24_z81_s3": (4, 24, 81, 3),       # rate 5/6, N = 1944
    "qc34x68_z384_s5": (34, 68, 384, 5),   # rate 1/2, N = 26112 (large code)
    # rate-1/2 codes at the frame lengths of the paper's throughput figures (Sec. IV:
    # 576 .. 8000 bits; 1944 is qc12x24_z81_s2 above)
    "qc12x24_z24_s6": (12, 24, 24, 6),     # N = 576
    "qc16x32_z32_s7": (16, 32, 32, 7),     # N = 1024
    "qc12x24_z50_s8": (12, 24, 50, 8),     # N = 1200
    "qc12x24_z96_s9": (12, 24, 96, 9),     # N = 2304
    "qc10x20_z200_s10": (10, 20, 200, 10),  # N = 4000
    "qc20x40_z200_s11": (20, 40, 200, 11),  # N = 8000
}
# Mixed-code family: Z in {27, 54, 81} x rate {1/2, 2/3, 3/4, 5/6}, seeds 40 + i.
for _i, (_Z, _mb) in enumerate([(z, m) for z in (27, 54, 81) for m in (12, 8, 6, 4)]):
    CODE_SPECS[code_name(_mb, 24, _Z, 40 + _i)] = (_mb, 24, _Z, 40 + _i)


def write_code_files(out_dir: str = CODES_DIR) -> list[str]:
    """(Re)write every committed base file from the recipe.  Returns the names written."""
    os.makedirs(out_dir, exist_ok=True)
    names = []
    for name, (mb, nb, Z, seed) in CODE_SPECS.items():
        B = qc_base_matrix(mb, nb, Z, seed)
        hdr = (f"{name}: seeded QC-LDPC base matrix, mb={mb} nb={nb} Z={Z} seed={seed}\n"
               f"written by paper_1812_06545_gb300.inputs.write_code_files (dual-diagonal parity half,\n"
               f"info columns of degree 3-4, shifts uniform in [0, Z); 4-cycles not filtered)")
        with open(os.path.join(out_dir, name + ".txt"), "w") as f:
            f.write(format_base(B, Z, hdr))
        names.append(name)
    return names


def encode(B: np.ndarray, Z: int, u: np.ndarray) -> np.ndarray:
    """Systematic codewords [u | p_0 .. p_{mb-1}] for the dual-diagonal recipe.

    u: uint8 [n, K] with K = (nb - mb) * Z.  Block-row sums over GF(2):
    lam_i = sum_j P^{s_ij} u_j;  p_0 = sum_i lam_i;  p_1 = lam_0 + P^{s_top} p_0;
    p_{i+1} = lam_i + p_i (+ P^{s_mid} p_0 at the middle row).  The last block row is
    asserted to close.  (P^s x)[r] = x[(r + s) mod Z].
    """
    mb, nb = B.shape
    kb = nb - mb
    u = np.ascontiguousarray(u, dtype=np.uint8)
    n = u.shape[0]
    if u.shape[1] != kb * Z:
        raise ValueError("info length mismatch")
    mid = mb // 2
    s_top, s_mid, s_bot = int(B[0, kb]), int(B[mid, kb]), int(B[mb - 1, kb])
    stair_ok = all(B[c - 1, kb + c] == 0 and B[c, kb + c] == 0 for c in range(1, mb))
    col0 = [i for i in range(mb) if B[i, kb] >= 0]
    if not stair_ok or col0 != [0, mid, mb - 1] or s_top != s_bot:
        raise ValueError("base matrix does not have the dual-diagonal parity half")

    def shift(x, s):
        return np.roll(x, -s, axis=-1) if s else x

    ub = u.reshape(n, kb, Z)
    lam = np.zeros((n, mb, Z), dtype=np.uint8)
    for i in range(mb):
        for j in range(kb):
            s = int(B[i, j])
            if s >= 0:
                lam[:, i, :] ^= shift(ub[:, j, :], s)
    p = np.zeros((n, mb, Z), dtype=np.uint8)
    p0 = np.bitwise_xor.reduce(lam, axis=1)
    p[:, 0] = p0
    p[:, 1] = lam[:, 0] ^ shift(p0, s_top)
    for i in range(1, mb - 1):
        p[:, i + 1] = lam[:, i] ^ p[:, i] ^ (shift(p0, s_mid) if i == mid else 0)
    if np.any(lam[:, mb - 1] ^ shift(p0, s_bot) ^ p[:, mb - 1]):
        raise AssertionError("last block row does not close")
    return np.concatenate([u, p.reshape(n, mb * Z)], axis=1)


def info_bits(n: int, K: int, seed: int) -> np.ndarray:
    """Uniform random info bits, uint8 [n, K], numpy PCG64(seed)."""
    return np.random.Generator(np.random.PCG64(seed)).integers(0, 2, size=(n, K), dtype=np.uint8)


def sigma2_for(ebn0_db: float, rate: float) -> float:
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def awgn_llr(c: np.ndarray, ebn0_db: float, rate: float, seed: int, chunk: int = 4096) -> np.ndarray:
    """BPSK x = 1 - 2c over AWGN, y = x + sigma*n, L = 2y/sigma^2 as fp32 [n, N].

    sigma^2 = 1 / (2 R 10^(EbN0/10)).  Noise is numpy PCG64(seed) standard normals drawn
    in row-major order (drawn in row chunks; the stream is the same as one draw).
    """
    s2 = sigma2_for(ebn0_db, rate)
    sig = np.sqrt(s2)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty(c.shape, dtype=np.float32)
    for a in range(0, c.shape[0], chunk):
        cc = c[a:a + chunk]
        y = (1.0 - 2.0 * cc) + sig * rng.standard_normal(cc.shape)
        out[a:a + chunk] = (2.0 / s2) * y
    return out


@dataclass
class Workload:
    """A named decode workload: code, batch size, Eb/N0 points and seeds."""
    name: str
    code: str
    batch: int
    ebn0_db: list
    info_seed: int
    noise_seeds: list
    max_iter: int
    early_exit: bool
    note: str = ""
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    # Plain FP32 flooding SPA, 10 fixed iterations, no early exit.
    "flood_n648_b128": Workload("flood_n648_b128", "qc12x24_z27_s1", 128, [2.0], 11, [12], 10, False,
                                "rate 1/2, N=648, 128 codewords at Eb/N0 = 2.0 dB"),
    # FP32 (and FP16-storage) flooding SPA, early exit, max 20, Eb/N0 1.0..2.5 dB step 0.25.
    "flood_n1944_b8192_sweep": Workload("flood_n1944_b8192_sweep", "qc12x24_z81_s2", 8192,
                                        [1.0 + 0.25 * i for i in range(7)], 20, [21 + i for i in range(7)],
                                        20, True, "rate 1/2, N=1944, 8192 codewords per Eb/N0 point"),
    # int8 layered normalised min-sum, max 10 iterations, early exit.
    "layered_i8_n1944_r56_b65536": Workload("layered_i8_n1944_r56_b65536", "qc4x24_z81_s3", 65536, [4.0], 30,
                                            [31], 10, True, "rate 5/6, N=1944, 65536 codewords at 4.0 dB"),
}


MIXED_FAMILY = sorted(n for n in CODE_SPECS if n.endswith(tuple(f"_s{s}" for s in range(40, 52))))


def operating_points() -> dict:
    """Eb/N0 per mixed-family code at which the FP64 oracle's frame error rate is about
    1e-2 (committed data; see its 'written_by' field)."""
    import json

    with open(os.path.join(CODES_DIR, "operating_points.json")) as f:
        return {k: v["ebn0_db"] for k, v in json.load(f)["points"].items()}


def mixed_batch(n_total: int = 20000, seed: int = 40):
    """The mixed-code workload: n_total codewords, each drawn uniformly from the 12 codes
    Z in {27, 54, 81} x rate {1/2, 2/3, 3/4, 5/6} (seeded multinomial), every code at its
    operating point.  Returns [(code name, c uint8 [n, N], L fp32 [n, N])] in family order."""
    ops = operating_points()
    counts = np.random.Generator(np.random.PCG64(seed)).multinomial(n_total, [1 / len(MIXED_FAMILY)] * len(MIXED_FAMILY))
    out = []
    for i, (name, n) in enumerate(zip(MIXED_FAMILY, counts)):
        _, _, c, L = make_frames(name, int(n), ops[name], seed * 100 + i, seed * 100 + 50 + i)
        out.append((name, c, L))
    return out


def llr_scale_for(rate: float, ebn0_db: float, sat: int = 31) -> float:
    """Quantiser scale s of the int8 layered min-sum (q = sat(rint(s L))): the power of two
    nearest to sat / (4 E|L|), so that saturation sits at about four mean channel LLRs.
    E|L| = 2/sigma^2 = 4 R Eb/N0 for BPSK/AWGN.  (A parameter choice, measured on the oracle:
    on the rate-5/6 code at 4.0 dB, s = 1 / 2 / 4 give FER 0.002 / 0.0085 / 0.79; on the
    rate-1/2 code at 2.5 dB, 0.16 / 0.0048 / 0.19.)"""
    mean = 4.0 * rate * 10.0 ** (ebn0_db / 10.0)
    return float(2.0 ** round(np.log2(sat / (4.0 * mean))))


def make_frames(code: str, n: int, ebn0_db: float, info_seed: int, noise_seed: int):
    """Encode n random-info codewords of ``code`` and pass them through BPSK/AWGN.

    Returns (B, Z, c uint8 [n, N], L fp32 [n, N]).
    """
    B, Z = load_code(code)
    mb, nb = B.shape
    K = (nb - mb) * Z
    u = info_bits(n, K, info_seed)
    c = encode(B, Z, u)
    L = awgn_llr(c, ebn0_db, K / (nb * Z), noise_seed)
    return B, Z, c, L


if __name__ == "__main__":
    for nm in write_code_files():
        print("wrote", nm)
