"""Host-side checks of the CUDA library that need no GPU: it loads, exports every symbol
the header declares, and rejects bad input before touching the device."""
import os
import re

import numpy as np
import pytest

from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ldpc_[a-z_0-9]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_lists_functions():
    names = header_functions()
    assert "ldpc_decode_batch" in names and "ldpc_code_create" in names and len(names) >= 12


def test_library_exports_every_header_symbol():
    lib = ldpc.lib()
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params():
    p = ldpc.ldpc_default_params()
    assert (p.sched, p.algo, p.msg, p.max_iter, p.early_exit) == (0, 0, 0, 20, 1)
    assert p.phi_clamp == 80.0 and (p.nms_alpha_num, p.nms_alpha_shift) == (3, 2)
    assert (p.msg_sat, p.app_sat, p.llr_scale, p.impl) == (31, 127, 2.0, 0)
    with pytest.raises(TypeError):
        ldpc.ldpc_default_params(bogus=1)


@pytest.mark.parametrize("base,Z,msg", [
    ([[0, 1, -1]], 1, "outside"),                          # shift >= Z
    ([[0, -1, -1], [0, 0, 0]], 4, "nonzero blocks"),        # a row with one block
    ([[0, 0], [0, 0]], 4, "mb < nb"),                       # mb >= nb
    ([[0, 0, -1]], 4, "empty"),                             # empty block column
    ([[0, -2, 0]], 4, "outside"),                           # entry below -1
    ([[0, 0, 0]], 0, "Z must be"),                          # Z out of range
])
def test_code_create_rejects_bad_base(base, Z, msg):
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_code_create(np.array(base), Z)
    assert ei.value.status == ldpc.LDPC_EINVAL and msg in str(ei.value)


def test_inputs_reproduce_committed_codes(tmp_path):
    names = I.write_code_files(str(tmp_path))
    for nm in names:
        assert (tmp_path / (nm + ".txt")).read_text() == open(os.path.join(I.CODES_DIR, nm + ".txt")).read(), nm


def test_recipe_structure():
    for nm, (mb, nb, Z, seed) in I.CODE_SPECS.items():
        B, Zf = I.load_code(nm)
        assert B.shape == (mb, nb) and Zf == Z
        info = B[:, : nb - mb] >= 0
        assert set(info.sum(axis=0)) <= {3, 4}
        assert ((B >= -1) & (B < Z)).all()


def test_quantiser_scale_rule():
    # the power of two nearest to 31 / (4 E|L|), E|L| = 4 R Eb/N0: the scales the oracle
    # measurements chose for the two workloads of the int8 form, and monotone in the channel
    from paper_1812_06545_gb300 import inputs as I
    assert I.llr_scale_for(5 / 6, 4.0) == 1.0
    assert I.llr_scale_for(0.5, 2.5) == 2.0
    scales = [I.llr_scale_for(0.5, eb) for eb in np.arange(0.0, 8.0, 0.25)]
    assert all(a >= b for a, b in zip(scales, scales[1:]))
    assert all(np.log2(s) == round(np.log2(s)) for s in scales)


def test_quantiser_scale_rule_against_the_oracle():
    # on the rate-5/6 code at 4.0 dB the rule's scale (1) beats the default (2): fewer frame
    # errors of the bit-exact integer min-sum on the same frames
    from oracle import oracle as O
    from paper_1812_06545_gb300 import inputs as I
    B, Z = I.load_code("qc4x24_z81_s3")
    oc = O.QCCode(B, Z)
    _, _, c, L = I.make_frames("qc4x24_z81_s3", 1500, 4.0, 17, 18)
    fer = {}
    for s in (1.0, 2.0):
        _, bits, _ = oc.nms_layered(O.quantize(L, s, 31), 10)
        fer[s] = (bits != c).any(axis=1).mean()
    assert fer[I.llr_scale_for(5 / 6, 4.0)] < fer[2.0], fer
