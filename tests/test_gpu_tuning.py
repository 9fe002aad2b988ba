"""Autotuned schedules and CUDA-graph capture of the decode calls, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import FP32_TOL, assert_binary16_close, binary16_band, oracle_code, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "layered_i8"])
def test_autotune_picks_a_schedule_and_decodes_correctly(cuda_dev, form):
    name = "qc12x24_z81_s2" if form != "layered_i8" else "qc4x24_z81_s3"
    B, Z = I.load_code(name)
    code = ldpc.Code(B, Z)
    p = ldpc.params_for(form, max_iter=20 if form != "layered_i8" else 10)
    _, _, c, L = I.make_frames(name, 2048, 2.0 if form != "layered_i8" else 4.0, 3, 4)
    x = torch.from_numpy(L).to(cuda_dev)
    choice, ms = ldpc.ldpc_autotune(code.handle, p, x, ldpc.LDPC_LLR_F32, 2048)
    assert choice in (1, 2, 3)
    assert all(m > 0 for m in ms if m >= 0) and sum(m > 0 for m in ms) >= 2
    assert ms[choice - 1] == min(m for m in ms if m > 0)
    if form == "layered_i8":
        return  # every layered schedule is bit-exact (test_gpu_layered)
    _, _, _, L3 = I.make_frames(name, 300, 1.5, 5, 6)
    bits, iters, app = ldpc.decode(code, ldpc.params_for(form, max_iter=3, early_exit=0),
                                   torch.from_numpy(L3).to(cuda_dev), app=True)
    torch.cuda.synchronize()
    if form.endswith("f16"):
        ref, band = binary16_band(oracle_code(name), False, L3, 3, 4)
        assert_binary16_close(app.cpu().numpy(), ref, band, strict=False, what=form)
    else:
        ref, _, _ = oracle_code(name).spa_flood(L3, 3, early_exit=False)
        assert rel_err(app.cpu().numpy(), ref).max() <= FP32_TOL


@pytest.mark.parametrize("form", ["stream_f32", "flood_f32", "layered_i8"])
def test_cuda_graph_capture_and_replay(cuda_dev, form):
    name = "qc12x24_z81_s2" if form != "layered_i8" else "qc4x24_z81_s3"
    B, Z = I.load_code(name)
    code = ldpc.Code(B, Z)
    n = 600
    p = ldpc.params_for(form, max_iter=12)
    x = torch.empty((n, code.N), dtype=torch.float32, device=cuda_dev)
    bits = torch.empty((n, code.N), dtype=torch.uint8, device=cuda_dev)
    iters = torch.empty((n,), dtype=torch.int32, device=cuda_dev)
    app = torch.empty((n, code.N), dtype=torch.float32, device=cuda_dev)
    wsb = max(ldpc.ldpc_workspace_size(code.handle, p, n), 256)
    ws = torch.empty(wsb, dtype=torch.uint8, device=cuda_dev)
    _, _, _, L0 = I.make_frames(name, n, 2.0, 1, 2)
    x.copy_(torch.from_numpy(L0))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # eager warm-up (kernel attributes set outside the capture)
        ldpc.ldpc_decode_batch(code.handle, p, x, 0, n, bits, iters, app, ws, wsb, side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ldpc.ldpc_decode_batch(code.handle, p, x, 0, n, bits, iters, app, ws, wsb, torch.cuda.current_stream())
    for seed in (11, 12):
        _, _, _, L = I.make_frames(name, n, 1.75, seed, seed + 1)
        x.copy_(torch.from_numpy(L))
        g.replay()
        torch.cuda.synchronize()
        rb, ri, ra = ldpc.decode(code, p, torch.from_numpy(L).to(cuda_dev), app=True)
        torch.cuda.synchronize()
        assert torch.equal(bits, rb) and torch.equal(iters, ri) and torch.equal(app, ra)
