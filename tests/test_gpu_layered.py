"""Layered int8 normalised min-sum on the GPU against the integer oracle: bit-exact
posterior, hard decisions and iteration counts, through the C ABI."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import oracle_code

pytestmark = pytest.mark.gpu

_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


def run(code, x, dev, form="layered_i8", **kw):
    p = ldpc.params_for(form, **kw)
    bits, iters, app = ldpc.decode(code, p, torch.from_numpy(x).to(dev), app=True)
    torch.cuda.synchronize()
    return app.cpu().numpy().astype(np.int32), bits.cpu().numpy(), iters.cpu().numpy()


def assert_exact(got, ref):
    ga, gb, gi = got
    ra, rb, ri = ref
    assert np.array_equal(gi, ri), np.nonzero(gi != ri)[0][:10]
    assert np.array_equal(ga, ra)
    assert np.array_equal(gb, rb)


@pytest.mark.parametrize("form", ["layered_i8", "layered_i8_group"])
@pytest.mark.parametrize("eb,early", [(4.0, 1), (3.0, 1), (3.0, 0)])
def test_rate56_bit_exact_int8_input(cuda_dev, form, eb, early):
    # persistent slots (AUTO) and the fixed group-per-CTA kernel, bit-exact alike
    name = "qc4x24_z81_s3"
    _, _, c, L = I.make_frames(name, 1003, eb, 30, 31)
    q = O.quantize(L, 2.0, 31)
    got = run(gpu_code(name), q, cuda_dev, form, max_iter=10, early_exit=early)
    assert_exact(got, oracle_code(name).nms_layered(q, 10, early_exit=bool(early)))


def test_fp32_input_quantised_in_kernel(cuda_dev):
    name = "qc4x24_z81_s3"
    _, _, c, L = I.make_frames(name, 500, 4.0, 32, 33)
    L[0, :8] = [1.25, 1.75, -1.25, 20.0, -0.2, 0.25, 0.75, -15.6]     # rounding ties and saturation
    for scale in (2.0, 1.0, 4.0):
        got = run(gpu_code(name), L, cuda_dev, max_iter=10, llr_scale=scale)
        q = O.quantize(L, scale, 31)
        assert_exact(got, oracle_code(name).nms_layered(q, 10, early_exit=True))


@pytest.mark.parametrize("name", sorted(n for n in I.CODE_SPECS if n.endswith(tuple(f"_s{s}" for s in range(40, 52)))))
def test_mixed_code_family_bit_exact(cuda_dev, name):
    mb = I.CODE_SPECS[name][0]
    rate = 1 - mb / 24
    _, _, c, L = I.make_frames(name, 450, 2.0 + 4 * (rate - 0.5), 40, 41)
    q = O.quantize(L, 2.0, 31)
    got = run(gpu_code(name), q, cuda_dev, max_iter=8)
    assert_exact(got, oracle_code(name).nms_layered(q, 8, early_exit=True))


def test_saturation_parameters(cuda_dev):
    name = "qc6x24_z54_s46"
    _, _, c, L = I.make_frames(name, 200, 3.0, 42, 43)
    # the first three run on two codewords per thread in packed half precision (exact for
    # them); alpha = 9/16 at msg_sat = 127 is not exact there and runs one codeword per thread
    for msg_sat, app_sat, an, ash in ((15, 15, 3, 2), (31, 63, 7, 3), (63, 127, 1, 0), (127, 127, 9, 4)):
        q = O.quantize(L, 2.0, msg_sat)
        got = run(gpu_code(name), q, cuda_dev, max_iter=6, msg_sat=msg_sat, app_sat=app_sat, nms_alpha_num=an,
                  nms_alpha_shift=ash)
        ref = oracle_code(name).nms_layered(q, 6, True, an, ash, msg_sat, app_sat)
        assert_exact(got, ref)


@pytest.mark.parametrize("form", ["layered_i8", "layered_i8_group"])
def test_large_code_z384(cuda_dev, form):
    name = "qc34x68_z384_s5"
    _, _, c, L = I.make_frames(name, 5, 2.5, 50, 51)
    q = O.quantize(L, 2.0, 31)
    got = run(gpu_code(name), q, cuda_dev, form, max_iter=10)
    assert_exact(got, oracle_code(name).nms_layered(q, 10, early_exit=True))


@pytest.mark.parametrize("form", ["layered_i8", "layered_i8_group"])
@pytest.mark.parametrize("name,n,eb", [("qc10x20_z200_s10", 400, 2.75), ("qc20x40_z200_s11", 300, 2.5)])
def test_paper_frame_lengths_z200(cuda_dev, form, name, n, eb):
    # the paper's frame lengths N = 4000 and 8000 (Sec. IV) with Z = 200 (lanes not a multiple
    # of 32, seven warps per slot), fp32 LLRs quantised in the kernel, 10 iterations
    _, _, c, L = I.make_frames(name, n, eb, 52, 53)
    scale = I.llr_scale_for(0.5, eb)
    got = run(gpu_code(name), L, cuda_dev, form, max_iter=10, llr_scale=scale)
    q = O.quantize(L, scale, 31)
    assert_exact(got, oracle_code(name).nms_layered(q, 10, early_exit=True))


def test_eq1_code_z1(cuda_dev):
    H = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "eq1_H.txt"))
    base = np.where(H == 1, 0, -1).astype(np.int32)
    code = ldpc.Code(base, 1)
    oc = O.QCCode(base, 1)
    rng = np.random.default_rng(1)
    q = rng.integers(-31, 32, size=(77, 10)).astype(np.int8)
    got = run(code, q, cuda_dev, max_iter=5)
    assert_exact(got, oc.nms_layered(q, 5, early_exit=True))


def test_batch_invariance(cuda_dev):
    name = "qc4x24_z81_s3"
    _, _, c, L = I.make_frames(name, 4000, 3.0, 70, 71)
    q = O.quantize(L, 2.0, 31)
    ga, gb, gi = run(gpu_code(name), q, cuda_dev, max_iter=10)
    for i in (0, 11, 12, 1999, 3999):
        a1, b1, i1 = run(gpu_code(name), q[i:i + 1].copy(), cuda_dev, max_iter=10)
        assert np.array_equal(a1[0], ga[i]) and i1[0] == gi[i]


def test_full_size_sampled(cuda_dev):
    # 65536 codewords of the rate-5/6 code at 4.0 dB, decoded in one launch as the
    # benchmark does; 512 sampled codewords decoded one by one by the oracle.
    name = "qc4x24_z81_s3"
    _, _, c, L = I.make_frames(name, 65536, 4.0, 30, 31)
    q = O.quantize(L, 2.0, 31)
    ga, gb, gi = run(gpu_code(name), q, cuda_dev, max_iter=10)
    idx = np.sort(np.random.default_rng(9).choice(65536, 512, replace=False))
    idx = np.concatenate([idx, [0, 65535]])
    ra, rb, ri = oracle_code(name).nms_layered(q[idx], 10, early_exit=True)
    assert_exact((ga[idx], gb[idx], gi[idx]), (ra, rb, ri))


def test_single_and_empty(cuda_dev):
    name = "qc4x24_z81_s3"
    code = gpu_code(name)
    _, _, c, L = I.make_frames(name, 1, 3.0, 60, 61)
    q = O.quantize(L, 2.0, 31)
    assert_exact(run(code, q, cuda_dev, max_iter=10), oracle_code(name).nms_layered(q, 10, True))
    bits, iters, _ = ldpc.decode(code, ldpc.params_for("layered_i8"),
                                 torch.empty((0, code.N), dtype=torch.int8, device=cuda_dev))
    assert bits.shape[0] == 0
