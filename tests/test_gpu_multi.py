"""Mixed-code persistent launches (ldpc_decode_multi) through the C ABI: every request
decodes exactly as it does alone."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import F16_CASCADE_FRAC, FP32_TOL, binary16_band, codewords_outside, oracle_code, rel_err

pytestmark = pytest.mark.gpu

FAMILY = sorted(n for n in I.CODE_SPECS if n.endswith(tuple(f"_s{s}" for s in range(40, 52))))
_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


def frames(name, n, seed):
    mb = I.CODE_SPECS[name][0]
    rate = 1 - mb / 24
    return I.make_frames(name, n, 1.5 + 3.0 * (rate - 0.5), seed, seed + 1)


def outputs(code, n, dev):
    return (torch.empty((n, code.N), dtype=torch.uint8, device=dev), torch.empty((n,), dtype=torch.int32, device=dev),
            torch.empty((n, code.N), dtype=torch.float32, device=dev))


@pytest.mark.parametrize("form", ["flood_f16", "flood_f32"])
def test_mixed_codes_equal_alone(cuda_dev, form):
    p = ldpc.params_for(form, max_iter=20)
    reqs, refs, outs = [], [], []
    sizes = [0, 1, 37, 300, 129, 64, 512, 7, 250, 3, 90, 200]
    for i, name in enumerate(FAMILY):
        code = gpu_code(name)
        n = sizes[i % len(sizes)]
        _, _, c, L = frames(name, n, 100 + i)
        x = torch.from_numpy(L).to(cuda_dev)
        o = outputs(code, n, cuda_dev)
        reqs.append((code.handle, x, n, o[0], o[1], o[2]))
        outs.append(o)
        refs.append(ldpc.decode(code, p, x, app=True) if n else None)
    # a second request of the first non-empty code, to share a group
    code = gpu_code(FAMILY[1])
    _, _, c, L = frames(FAMILY[1], 100, 999)
    x = torch.from_numpy(L).to(cuda_dev)
    o = outputs(code, 100, cuda_dev)
    reqs.append((code.handle, x, 100, o[0], o[1], o[2]))
    outs.append(o)
    refs.append(ldpc.decode(code, p, x, app=True))
    ldpc.ldpc_decode_multi(reqs, p)
    torch.cuda.synchronize()
    for (h, x, n, *_), o, ref in zip(reqs, outs, refs):
        if n == 0:
            continue
        assert torch.equal(o[0], ref[0]) and torch.equal(o[1], ref[1]) and torch.equal(o[2], ref[2])


def test_mixed_codes_single_code_many_requests(cuda_dev):
    name = "qc12x24_z81_s2"
    code = gpu_code(name)
    p = ldpc.params_for("flood_f32", max_iter=20)
    _, _, c, L = I.make_frames(name, 3000, 1.75, 5, 6)
    x = torch.from_numpy(L).to(cuda_dev)
    ref = ldpc.decode(code, p, x, app=True)
    outs = outputs(code, 3000, cuda_dev)
    cuts = [0, 1000, 1001, 2500, 3000]
    reqs = [(code.handle, x[a:b], b - a, outs[0][a:b], outs[1][a:b], outs[2][a:b]) for a, b in zip(cuts, cuts[1:])]
    ldpc.ldpc_decode_multi(reqs, p)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], ref[0]) and torch.equal(outs[1], ref[1]) and torch.equal(outs[2], ref[2])


def test_mixed_launch_argument_errors(cuda_dev):
    code = gpu_code(FAMILY[0])
    x = torch.zeros((4, code.N), device=cuda_dev)
    o = outputs(code, 4, cuda_dev)
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_decode_multi([(code.handle, x, 4, o[0], o[1], None)], ldpc.params_for("stream_f32"))
    assert ei.value.status == ldpc.LDPC_ENOTSUP
    with pytest.raises(ldpc.LdpcError):
        ldpc.ldpc_decode_multi([(code.handle, x, 4, None, o[1], None)], ldpc.params_for("flood_f32"))
    ldpc.ldpc_decode_multi([], ldpc.params_for("flood_f32"))


def test_mixed_launch_with_a_cluster_sized_code(cuda_dev):
    # a code whose codeword exceeds one SM joins a mixed launch: it runs on the cluster
    # decoder in a launch of its own, the others in the shared persistent launch; every
    # request decodes exactly as alone
    p = ldpc.params_for("flood_f16", max_iter=20)
    names = [FAMILY[0], "qc34x68_z384_s5", FAMILY[5]]
    reqs, outs, refs = [], [], []
    for k, name in enumerate(names):
        code = gpu_code(name)
        _, _, c, L = I.make_frames(name, 37 + 11 * k, 2.0, 71 + k, 81 + k)
        Lt = torch.from_numpy(L).to(cuda_dev)
        o = outputs(code, len(L), cuda_dev)
        reqs.append((code.handle, Lt, len(L), o[0], o[1], None))
        outs.append(o)
        refs.append(ldpc.decode(code, p, Lt))
    ldpc.ldpc_decode_multi(reqs, p)
    torch.cuda.synchronize()
    for o, (rb, ri, _) in zip(outs, refs):
        assert torch.equal(o[0], rb) and torch.equal(o[1], ri)


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "layered_f32", "layered_f16", "layered_i8"])
def test_mixed_launch_against_the_oracle(cuda_dev, form):
    # One ldpc_decode_multi call over all 12 family codes (request sizes 1..512, ragged)
    # against the oracle, code by code: the sum-product forms after 3 iterations without early
    # exit, element by element within the FP32 tolerance; the FP16 forms within the binary16
    # band (4 half-ulps of every incoming message for flooding, 8 for layered) on all but the
    # few codewords in which rounding flips cascade; the int8 min-sum bit-exact (posterior,
    # decisions, iteration counts) at max 10 with early exit
    i8 = form == "layered_i8"
    layered = form.startswith("layered")
    p = ldpc.params_for(form, max_iter=10 if i8 else 3, early_exit=1 if i8 else 0)
    sizes = [1, 37, 300, 129, 64, 512, 7, 250, 3, 90, 200, 33]
    reqs, outs, Ls = [], [], []
    for i, name in enumerate(FAMILY):
        code = gpu_code(name)
        n = sizes[i]
        _, _, c, L = frames(name, n, 700 + i)
        x = torch.from_numpy(L).to(cuda_dev)
        o = outputs(code, n, cuda_dev)
        reqs.append((code.handle, x, n, o[0], o[1], o[2]))
        outs.append(o)
        Ls.append(L)
    ldpc.ldpc_decode_multi(reqs, p)
    torch.cuda.synchronize()
    outside = 0
    for name, L, o in zip(FAMILY, Ls, outs):
        oc = oracle_code(name)
        app, bits, iters = (t.cpu().numpy() for t in (o[2], o[0], o[1]))
        if i8:
            q = O.quantize(L, 2.0, 31)
            ra, rb, ri = oc.nms_layered(q, 10, early_exit=True)
            assert np.array_equal(iters, ri) and np.array_equal(app.astype(np.int32), ra), name
            assert np.array_equal(bits, rb), name
            continue
        assert (iters == 3).all()
        orc = oc.spa_layered if layered else oc.spa_flood
        if form.endswith("f16"):
            ref, band = binary16_band(oc, layered, L, 3, 8 if layered else 4)
            outside += codewords_outside(app, ref, band)
        else:
            ref, _, _ = orc(L, 3, early_exit=False)
            assert rel_err(app, ref).max() <= FP32_TOL, (form, name, rel_err(app, ref).max())
    # binary16 rounding flips that cascade: at most a few codewords of the launch
    assert outside <= F16_CASCADE_FRAC * sum(sizes), (form, outside)


def test_layered_i8_many_requests_per_code_one_launch_each(cuda_dev):
    # The packed int8 min-sum takes every request of one code into one launch (one work
    # sequence over the requests' codewords): requests of two codes, interleaved in the call,
    # cut at ragged points (one of a single codeword); every request bit-exact against the
    # decode of the whole batch alone and against the integer oracle.
    p = ldpc.params_for("layered_i8", max_iter=10)
    specs = [("qc4x24_z81_s3", 3000, 3.5, [0, 1000, 1001, 2500, 3000]),
             ("qc8x24_z54_s45", 900, 2.75, [0, 450, 899, 900])]
    reqs, checks = [], []
    for name, n, eb, cuts in specs:
        code = gpu_code(name)
        _, _, c, L = I.make_frames(name, n, eb, 121, 122)
        x = torch.from_numpy(L).to(cuda_dev)
        whole = ldpc.decode(code, p, x, app=True)
        o = outputs(code, n, cuda_dev)
        parts = [(code.handle, x[a:b], b - a, o[0][a:b], o[1][a:b], o[2][a:b]) for a, b in zip(cuts, cuts[1:])]
        reqs.append(parts)
        checks.append((name, L, o, whole))
    mixed = [q for pair in zip(reqs[0], reqs[1] + [None] * 4) for q in pair if q is not None]
    ldpc.ldpc_decode_multi(mixed, p)
    torch.cuda.synchronize()
    for name, L, o, whole in checks:
        assert torch.equal(o[0], whole[0]) and torch.equal(o[1], whole[1]) and torch.equal(o[2], whole[2]), name
        ra, rb, ri = oracle_code(name).nms_layered(O.quantize(L, 2.0, 31), 10, early_exit=True)
        assert np.array_equal(o[1].cpu().numpy(), ri) and np.array_equal(o[0].cpu().numpy(), rb), name
        assert np.array_equal(o[2].cpu().numpy().astype(np.int32), ra), name


def test_large_code_requests_share_a_launch(cuda_dev):
    # requests of the N = 26112 code (too large for the slot decoders): the FP16 flooding
    # requests share one cluster-decoder launch and the int8 min-sum requests one launch of the
    # one-codeword-per-thread kernel; every request equals its lone decode, and the int8 ones
    # the integer oracle bit for bit
    name = "qc34x68_z384_s5"
    code = gpu_code(name)
    _, _, c, L = I.make_frames(name, 23, 2.25, 131, 132)
    x = torch.from_numpy(L).to(cuda_dev)
    cuts = [0, 5, 6, 23]
    for form in ("flood_f16", "layered_i8"):
        p = ldpc.params_for(form, max_iter=10 if form == "layered_i8" else 20)
        whole = ldpc.decode(code, p, x, app=True)
        o = outputs(code, len(L), cuda_dev)
        reqs = [(code.handle, x[a:b], b - a, o[0][a:b], o[1][a:b], o[2][a:b]) for a, b in zip(cuts, cuts[1:])]
        ldpc.ldpc_decode_multi(reqs, p)
        torch.cuda.synchronize()
        assert torch.equal(o[0], whole[0]) and torch.equal(o[1], whole[1]) and torch.equal(o[2], whole[2]), form
        if form == "layered_i8":
            ra, rb, ri = oracle_code(name).nms_layered(O.quantize(L, 2.0, 31), 10, early_exit=True)
            assert np.array_equal(o[0].cpu().numpy(), rb) and np.array_equal(o[1].cpu().numpy(), ri)
            assert np.array_equal(o[2].cpu().numpy().astype(np.int32), ra)
