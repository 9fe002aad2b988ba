"""Layered sum-product on the GPU (FP32 and FP16 message storage) against the FP64 layered
oracle, through the C ABI."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import FP32_TOL, assert_binary16_close, binary16_band, clopper_pearson, oracle_code, rel_err

pytestmark = pytest.mark.gpu

# check degrees <= 8 (exact bodies, messages held), <= 16 and <= 32 (bucketed bodies,
# register-lean form); batch sizes are not multiples of the slots of one CTA.
CASES = [("qc12x24_z81_s2", 260, 1.5), ("qc12x24_z27_s1", 300, 2.0), ("qc8x24_z54_s45", 140, 2.5),
         ("qc4x24_z27_s43", 130, 3.5), ("qc4x24_z81_s3", 97, 3.5),
         # the paper's frame lengths N = 4000 and 8000 (Sec. IV), Z = 200
         ("qc10x20_z200_s10", 170, 2.0), ("qc20x40_z200_s11", 160, 2.0)]

_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


def run(name, form, L, dev, **kw):
    code = gpu_code(name)
    bits, iters, app = ldpc.decode(code, ldpc.params_for(form, **kw), torch.from_numpy(L).to(dev), app=True)
    torch.cuda.synchronize()
    return app.cpu().numpy(), bits.cpu().numpy(), iters.cpu().numpy()


@pytest.mark.parametrize("name,n,eb", CASES)
def test_fp32_posterior_first_three_iterations(cuda_dev, name, n, eb):
    _, _, c, L = I.make_frames(name, n, eb, 31, 32)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, bits, iters = run(name, "layered_f32", L, cuda_dev, max_iter=T, early_exit=0)
        ref, _, _ = oc.spa_layered(L, T, early_exit=False)
        err = rel_err(app, ref)
        assert err.max() <= FP32_TOL, (name, T, err.max())
        assert (iters == T).all()
        assert np.array_equal(bits, (app < 0).astype(np.uint8))


@pytest.mark.parametrize("name,n,eb", CASES)
def test_fp16_messages_first_three_iterations(cuda_dev, name, n, eb):
    # the oracle rounds every message to binary16 before adding it to the posterior, as the
    # kernel does; FP32 and FP64 values on either side of a rounding boundary may round one
    # binary16 ulp apart.  Under the layered schedule a flip also reaches the checks of later
    # layers of the same iteration through the posterior it changed: the band is 8 half-ulps
    # of every incoming message on top of the fp32 tolerance, on all but the few codewords in
    # which flips cascade (the oracle itself, fed LLRs perturbed by 1e-6 relative, moves such
    # a codeword by tens of half-ulps)
    _, _, c, L = I.make_frames(name, n, eb, 33, 34)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, _, _ = run(name, "layered_f16", L, cuda_dev, max_iter=T, early_exit=0)
        ref, band = binary16_band(oc, True, L, T, 8)
        assert_binary16_close(app, ref, band, strict=False, what=(name, T))


@pytest.mark.parametrize("form", ["layered_f32", "layered_f16"])
def test_early_exit_and_fer_full_size(cuda_dev, form):
    # 8192 codewords of the rate-1/2 N=1944 code per point at 1.25 and 1.75 dB, early exit,
    # max 20 iterations, in the launch configuration the benchmark times: GPU FER inside the
    # oracle's 95 % Clopper-Pearson interval; FP32 decisions identical to FP64 on >= 99.99 %
    # of codewords; FP16 identical wherever both decoders converged
    name = "qc12x24_z81_s2"
    oc = oracle_code(name)
    f16 = form.endswith("f16")
    mism = tot = 0
    for eb, seed in ((1.25, 41), (1.75, 43)):
        _, _, c, L = I.make_frames(name, 8192, eb, 40, seed)
        app, bits, iters = run(name, form, L, cuda_dev, max_iter=20, early_exit=1)
        _, rbits, riters = oc.spa_layered(L, 20, early_exit=True, fp16_msgs=f16)
        same = (bits == rbits).all(axis=1)
        mism += int((~same).sum())
        tot += len(same)
        fer_g = int((bits != c).any(axis=1).sum())
        fer_o = int((rbits != c).any(axis=1).sum())
        lo, hi = clopper_pearson(fer_o, len(c))
        assert lo <= fer_g / len(c) <= hi, (form, eb, fer_g, fer_o)
        conv = riters < 20
        # a binary16 rounding flip can move the iteration in which the syndrome first clears
        # by one without changing the decisions: FP16 is held to 99.5 %, FP32 to 99.9 %
        agree = (iters[conv & same] == riters[conv & same]).mean()
        assert agree >= (0.995 if f16 else 0.999), (form, eb, agree)
        if f16:
            both = conv & (iters < 20)
            assert (same[both]).mean() >= 0.9999, (eb, int((~same[both]).sum()))
    if not f16:
        assert mism <= 1e-4 * tot, (form, mism, tot)


def test_fewer_iterations_than_flooding(cuda_dev):
    # the point of the layered schedule (Sec. II): markedly fewer iterations at no worse FER
    name = "qc12x24_z81_s2"
    _, _, c, L = I.make_frames(name, 4096, 1.75, 45, 46)
    _, bl, il = run(name, "layered_f32", L, cuda_dev, max_iter=20, early_exit=1)
    _, bf, itf = run(name, "flood_f32", L, cuda_dev, max_iter=20, early_exit=1)
    assert il.mean() < 0.7 * itf.mean(), (il.mean(), itf.mean())
    assert (bl != c).any(axis=1).sum() <= (bf != c).any(axis=1).sum()


@pytest.mark.parametrize("form", ["layered_f32", "layered_f16"])
def test_batch_invariance(cuda_dev, form):
    name = "qc12x24_z81_s2"
    _, _, c, L = I.make_frames(name, 3000, 1.5, 47, 48)
    app_all, _, it_all = run(name, form, L, cuda_dev, max_iter=20, early_exit=1)
    for i in (0, 6, 7, 1499, 2999):
        app1, _, it1 = run(name, form, L[i:i + 1].copy(), cuda_dev, max_iter=20, early_exit=1)
        assert np.array_equal(app1[0], app_all[i]) and it1[0] == it_all[i]


def test_eq1_code_z1_and_small_lifting(cuda_dev):
    H = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "eq1_H.txt"))
    base = np.where(H == 1, 0, -1).astype(np.int32)
    rng = np.random.default_rng(1)
    for B, Z in ((base, 1), (np.array([[0, 6, -1, 3], [6, 0, 6, -1], [-1, 6, 0, 0]], np.int32), 7)):
        code = ldpc.Code(B, Z)
        oc = O.QCCode(B, Z)
        L = (1.5 + 2.0 * rng.standard_normal((37, code.N))).astype(np.float32)
        for T in (1, 4):
            _, _, app = ldpc.decode(code, ldpc.params_for("layered_f32", max_iter=T, early_exit=0),
                                    torch.from_numpy(L).to(cuda_dev), app=True)
            ref, _, _ = oc.spa_layered(L, T, early_exit=False)
            assert rel_err(app.cpu().numpy(), ref).max() <= FP32_TOL


def test_single_empty_and_unsupported(cuda_dev):
    name = "qc12x24_z27_s1"
    code = gpu_code(name)
    p = ldpc.params_for("layered_f32", max_iter=6)
    bits, _, _ = ldpc.decode(code, p, torch.empty((0, code.N), dtype=torch.float32, device=cuda_dev))
    assert bits.shape == (0, code.N)
    _, _, c, L = I.make_frames(name, 1, 2.5, 49, 50)
    app, bits, iters = run(name, "layered_f32", L, cuda_dev, max_iter=6, early_exit=1)
    ref, rbits, riters = oracle_code(name).spa_layered(L, 6, early_exit=True)
    assert rel_err(app, ref).max() <= FP32_TOL and np.array_equal(iters, riters)
    x = torch.zeros((2, code.N), device=cuda_dev)
    b = torch.empty((2, code.N), dtype=torch.uint8, device=cuda_dev)
    i = torch.empty((2,), dtype=torch.int32, device=cuda_dev)
    for bad, status in ((dict(impl=ldpc.LDPC_IMPL_PLAIN), ldpc.LDPC_ENOTSUP),
                        (dict(impl=ldpc.LDPC_IMPL_STREAMING), ldpc.LDPC_ENOTSUP),
                        (dict(msg=ldpc.LDPC_MSG_I8), ldpc.LDPC_ENOTSUP),
                        (dict(phi_clamp=0.5), ldpc.LDPC_EINVAL)):
        with pytest.raises(ldpc.LdpcError) as ei:
            ldpc.ldpc_decode_batch(code.handle, ldpc.params_for("layered_f32", **bad), x, 0, 2, b, i)
        assert ei.value.status == status
    with pytest.raises(ldpc.LdpcError) as ei:   # int8 LLRs are for the min-sum form
        ldpc.ldpc_decode_batch(code.handle, p, x.to(torch.int8), ldpc.LDPC_LLR_I8, 2, b, i)
    assert ei.value.status == ldpc.LDPC_EINVAL
    big = gpu_code("qc34x68_z384_s5")           # N = 26112: one slot exceeds shared memory
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_workspace_size(big.handle, p, 1)
    assert ei.value.status == ldpc.LDPC_ENOTSUP


def test_multi_request_launch_matches_lone_decodes(cuda_dev):
    names = ["qc12x24_z81_s2", "qc12x24_z27_s1", "qc4x24_z81_s3"]
    p = ldpc.params_for("layered_f16", max_iter=20)
    reqs, refs, outs = [], [], []
    for k, name in enumerate(names):
        code = gpu_code(name)
        _, _, c, L = I.make_frames(name, 150 + 37 * k, 2.0, 51 + k, 61 + k)
        Lt = torch.from_numpy(L).to(cuda_dev)
        b = torch.empty((len(L), code.N), dtype=torch.uint8, device=cuda_dev)
        it = torch.empty((len(L),), dtype=torch.int32, device=cuda_dev)
        reqs.append((code.handle, Lt, len(L), b, it, None))
        outs.append((b, it))
        refs.append(ldpc.decode(code, p, Lt))
    ldpc.ldpc_decode_multi(reqs, p, ldpc.LDPC_LLR_F32)
    torch.cuda.synchronize()
    for (b, it), (rb, rit, _) in zip(outs, refs):
        assert torch.equal(b, rb) and torch.equal(it, rit)
