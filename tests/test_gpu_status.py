"""The device input status word (ldpc_stream_check): bad channel input is flagged by the
decoding kernels themselves, for every form, without a host pass over the data."""
import numpy as np
import pytest
import torch

from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "stream_f32", "plain_f32", "layered_f32", "layered_f16",
                                  "layered_i8", "layered_i8_group"])
def test_non_finite_llr_is_flagged(cuda_dev, form):
    B, Z = I.load_code("qc12x24_z27_s1")
    code = ldpc.Code(B, Z)
    _, _, c, L = I.make_frames("qc12x24_z27_s1", 64, 2.5, 1, 2)
    p = ldpc.params_for(form, max_iter=5)
    ldpc.ldpc_stream_flags()                           # drain anything left by earlier tests
    x = torch.from_numpy(L).to(cuda_dev)
    ldpc.decode(code, p, x)
    assert ldpc.ldpc_stream_check() == 0               # clean input: no flag
    for bad in (float("nan"), float("inf"), -float("inf")):
        y = x.clone()
        y[17, 100] = bad
        ldpc.decode(code, p, y)
        with pytest.raises(ldpc.LdpcError) as ei:
            ldpc.ldpc_stream_check()
        assert ei.value.status == ldpc.LDPC_EINVAL
        assert ldpc.ldpc_stream_check() == 0           # taking the word cleared it
    # the flag is set at load time only: the other codewords still decode
    y = x.clone()
    y[3, 5] = float("nan")
    bits, iters, _ = ldpc.decode(code, p, y)
    assert ldpc.ldpc_stream_flags() == 1
    ok = [i for i in range(64) if i != 3]
    ref_bits, ref_iters, _ = ldpc.decode(code, p, x)
    assert torch.equal(bits[ok], ref_bits[ok]) and torch.equal(iters[ok], ref_iters[ok])
    assert ldpc.ldpc_stream_check() == 0


@pytest.mark.parametrize("form", ["layered_i8", "layered_i8_group"])
def test_int8_llr_out_of_range_is_flagged(cuda_dev, form):
    B, Z = I.load_code("qc4x24_z81_s3")
    code = ldpc.Code(B, Z)
    _, _, c, L = I.make_frames("qc4x24_z81_s3", 40, 4.0, 3, 4)
    q = np.clip(np.rint(2.0 * L), -31, 31).astype(np.int8)
    p = ldpc.params_for(form, max_iter=5)
    x = torch.from_numpy(q).to(cuda_dev)
    ldpc.decode(code, p, x)
    assert ldpc.ldpc_stream_check() == 0
    y = x.clone()
    y[7, 9] = 100                                       # > msg_sat = 31: saturated and flagged
    bits, _, _ = ldpc.decode(code, p, y)
    assert ldpc.ldpc_stream_flags() == 2
    y[7, 9] = 31
    bits2, _, _ = ldpc.decode(code, p, y)
    assert torch.equal(bits, bits2)                     # saturation = the in-range value
    assert ldpc.ldpc_stream_check() == 0
