"""Posterior parity at full occupancy: batches that fill every slot of every CTA (and refill
them), in the launch configuration the benchmark times, compared element by element with
the FP64 oracle after iterations 1, 2 and 3 (early exit off), through the C ABI.

The slot decoders take codewords from a work counter, so which codeword lands in which
slot of which CTA is decided at run time.  Every codeword of the batch is therefore
compared, which covers every slot position (first and last slot of every CTA, every
barrier group) and the refilled slots of the second wave."""
import numpy as np
import pytest
import torch

from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import FP32_TOL, assert_binary16_close, binary16_band, oracle_code, rel_err

pytestmark = pytest.mark.gpu

HEADLINE = "qc12x24_z81_s2"
BIG = "qc34x68_z384_s5"
_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


def decode_app(name, form, L, dev, T):
    code = gpu_code(name)
    bits, iters, app = ldpc.decode(code, ldpc.params_for(form, max_iter=T, early_exit=0),
                                   torch.from_numpy(L).to(dev), app=True)
    torch.cuda.synchronize()
    return app.cpu().numpy(), bits.cpu().numpy(), iters.cpu().numpy()


# (form, code, codewords, Eb/N0, binary16 tolerance multiplier: 0 = FP32 tolerance only)
CASES = [("flood_f32", HEADLINE, 8192, 1.5, 0), ("flood_f16", HEADLINE, 8192, 1.5, 4),
         ("layered_f32", HEADLINE, 8192, 1.5, 0), ("layered_f16", HEADLINE, 8192, 1.5, 8),
         ("flood_f16", BIG, 200, 1.9, 4), ("flood_f32", BIG, 160, 1.9, 0)]


@pytest.mark.parametrize("form,name,n,eb,h16", CASES)
def test_posterior_every_codeword_full_occupancy(cuda_dev, form, name, n, eb, h16):
    # the N = 1944 headline code: 8192 codewords fill the 152 CTAs' slots (7 FP32 slots, 12
    # paired FP16 slots in barrier groups, 7 / 12 layered slots) several times over; the
    # N = 26112 code: more codewords than its 76 two-SM clusters
    _, _, c, L = I.make_frames(name, n, eb, 301, 302)
    oc = oracle_code(name)
    layered = form.startswith("layered")
    orc = oc.spa_layered if layered else oc.spa_flood
    for T in (1, 2, 3):
        app, bits, iters = decode_app(name, form, L, cuda_dev, T)
        assert (iters == T).all()
        assert np.array_equal(bits, (app < 0).astype(np.uint8))
        if h16:
            # binary16 band: every codeword after the first flooding iteration, all but the
            # few in which rounding flips cascade otherwise
            ref, band = binary16_band(oc, layered, L, T, h16)
            assert_binary16_close(app, ref, band, strict=T == 1 and not layered, what=(form, name, T))
        else:
            ref, _, _ = orc(L, T, early_exit=False)
            err = rel_err(app, ref)
            bad = np.argwhere(err > FP32_TOL)
            assert bad.size == 0, (form, name, T, bad[:5], err.max())


@pytest.mark.parametrize("form", ["flood_f32", "layered_f32"])
def test_decisions_far_from_zero_match_the_oracle(cuda_dev, form):
    # wherever the oracle's posterior is farther from 0 than the tolerance, the hard decision
    # cannot differ: checked on every bit of the full batch after 3 iterations
    name = HEADLINE
    _, _, c, L = I.make_frames(name, 8192, 2.0, 303, 304)
    app, bits, _ = decode_app(name, form, L, cuda_dev, 3)
    oc = oracle_code(name)
    ref, rbits, _ = (oc.spa_layered if form.startswith("layered") else oc.spa_flood)(L, 3, early_exit=False)
    clear = np.abs(ref) > FP32_TOL * np.maximum(1.0, np.abs(ref))
    assert np.array_equal(bits[clear], rbits[clear])
