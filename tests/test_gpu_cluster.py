"""The cluster decoder (one codeword per two-SM thread-block cluster, flooding sum-product)
against the FP64 oracle, through the C ABI: the N = 26112 code that does not fit one SM
(chosen automatically), and small codes of every kernel shape when asked for explicitly."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import FP32_TOL, assert_binary16_close, binary16_band, clopper_pearson, oracle_code, rel_err

pytestmark = pytest.mark.gpu
BIG = "qc34x68_z384_s5"

_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


def run(name, form, L, dev, **kw):
    bits, iters, app = ldpc.decode(gpu_code(name), ldpc.params_for(form, **kw), torch.from_numpy(L).to(dev),
                                   app=True)
    torch.cuda.synchronize()
    return app.cpu().numpy(), bits.cpu().numpy(), iters.cpu().numpy()


@pytest.mark.parametrize("form,name,n,eb", [("flood_f32", BIG, 9, 1.5), ("cluster_f32", "qc12x24_z27_s1", 37, 2.0),
                                            ("cluster_f32", "qc8x24_z54_s45", 21, 2.5),
                                            ("cluster_f32", "qc4x24_z27_s43", 19, 3.5)])
def test_fp32_posterior_first_three_iterations(cuda_dev, form, name, n, eb):
    # AUTO picks the cluster decoder for the N = 26112 code (one codeword exceeds an SM);
    # the small codes cover the degree <= 8, <= 16 and <= 32 kernel shapes
    _, _, c, L = I.make_frames(name, n, eb, 61, 62)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, bits, iters = run(name, form, L, cuda_dev, max_iter=T, early_exit=0)
        ref, _, _ = oc.spa_flood(L, T, early_exit=False)
        assert rel_err(app, ref).max() <= FP32_TOL, (name, T, rel_err(app, ref).max())
        assert (iters == T).all() and np.array_equal(bits, (app < 0).astype(np.uint8))


@pytest.mark.parametrize("form,name", [("flood_f16", BIG), ("cluster_f16", "qc12x24_z81_s2")])
def test_fp16_messages_first_three_iterations(cuda_dev, form, name):
    _, _, c, L = I.make_frames(name, 60, 1.75, 63, 64)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, _, _ = run(name, form, L, cuda_dev, max_iter=T, early_exit=0)
        ref, band = binary16_band(oc, False, L, T, 4)
        assert_binary16_close(app, ref, band, strict=T == 1, what=(name, T))


def test_large_code_early_exit_and_fer(cuda_dev):
    # 256 codewords of the N = 26112 code at 1.9 dB (in its waterfall: some frames converge,
    # some do not), early exit, max 20: decisions and iteration counts against the FP64
    # oracle; FER inside its 95 % interval
    _, _, c, L = I.make_frames(BIG, 256, 1.9, 65, 66)
    app, bits, iters = run(BIG, "flood_f32", L, cuda_dev, max_iter=20, early_exit=1)
    _, rbits, riters = oracle_code(BIG).spa_flood(L, 20, early_exit=True)
    same = (bits == rbits).all(axis=1)
    assert same.mean() >= 0.99, same.mean()
    conv = riters < 20
    assert (conv & same).sum() >= 20
    assert (iters[conv & same] == riters[conv & same]).mean() >= 0.99
    fer_g, fer_o = int((bits != c).any(axis=1).sum()), int((rbits != c).any(axis=1).sum())
    lo, hi = clopper_pearson(fer_o, len(c))
    assert lo <= fer_g / len(c) <= hi, (fer_g, fer_o)


def test_cluster_matches_streaming_and_batch_invariance(cuda_dev):
    _, _, c, L = I.make_frames(BIG, 300, 1.9, 67, 68)
    a1, b1, i1 = run(BIG, "flood_f32", L, cuda_dev, max_iter=20, early_exit=1)
    a2, b2, i2 = run(BIG, "stream_f32", L, cuda_dev, max_iter=20, early_exit=1)
    conv = (i1 < 20) & (i2 < 20)
    assert np.array_equal(b1[conv], b2[conv]) and np.array_equal(i1[conv], i2[conv])
    for i in (0, 77, 299):
        a3, _, i3 = run(BIG, "flood_f32", L[i:i + 1].copy(), cuda_dev, max_iter=20, early_exit=1)
        assert np.array_equal(a3[0], a1[i]) and i3[0] == i1[i]


def test_eq1_code_and_unsupported(cuda_dev):
    H = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "eq1_H.txt"))
    base = np.where(H == 1, 0, -1).astype(np.int32)
    code = ldpc.Code(base, 1)
    oc = O.QCCode(base, 1)
    L = (1.5 + 2.0 * np.random.default_rng(2).standard_normal((13, code.N))).astype(np.float32)
    _, _, app = ldpc.decode(code, ldpc.params_for("cluster_f32", max_iter=3, early_exit=0),
                            torch.from_numpy(L).to(cuda_dev), app=True)
    ref, _, _ = oc.spa_flood(L, 3, early_exit=False)
    assert rel_err(app.cpu().numpy(), ref).max() <= FP32_TOL
    # the integer min-sum and the layered sum-product do not run on the cluster decoder
    small = gpu_code("qc12x24_z27_s1")
    x = torch.zeros((2, small.N), device=cuda_dev)
    b = torch.empty((2, small.N), dtype=torch.uint8, device=cuda_dev)
    i = torch.empty((2,), dtype=torch.int32, device=cuda_dev)
    for form in ("layered_i8", "layered_f32"):
        with pytest.raises(ldpc.LdpcError) as ei:
            ldpc.ldpc_decode_batch(small.handle, ldpc.params_for(form, impl=ldpc.LDPC_IMPL_CLUSTER), x, 0, 2, b, i)
        assert ei.value.status == ldpc.LDPC_ENOTSUP
