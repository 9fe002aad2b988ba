"""Mixed-code persistent launches (ldpc_decode_multi) through the C ABI: every request
decodes exactly as it does alone."""
import numpy as np
import pytest
import torch

from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc

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
