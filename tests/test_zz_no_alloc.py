"""The static-scratch decode entry point against the allocating one.

ldpc_decode_batch_static serves callers that cannot allocate device memory while they
decode (for instance a real-time receive chain that reserves everything at start-up): its
scratch is a fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import FP32_TOL, rel_err

pytestmark = pytest.mark.gpu


def _decode_static(code, p, x, dev):
    n = x.shape[0]
    bits = torch.empty((n, code.N), dtype=torch.uint8, device=dev)
    iters = torch.empty((n,), dtype=torch.int32, device=dev)
    app = torch.empty((n, code.N), dtype=torch.float32, device=dev)
    ldpc.ldpc_decode_batch_static(code.handle, p, x, n, bits, iters, app, torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    return bits.cpu().numpy(), iters.cpu().numpy(), app.cpu().numpy()


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "stream_f32"])
def test_static_scratch_matches_allocating_entry_point(cuda_dev, form):
    B, Z = I.load_code("qc12x24_z81_s2")
    code = ldpc.Code(B, Z)
    p = ldpc.params_for(form, max_iter=20)
    # two calls in a row with different batches: the second must not see the first's state
    for n, eb, seed in ((700, 1.5, 101), (333, 2.0, 102)):
        _, _, c, L = I.make_frames("qc12x24_z81_s2", n, eb, seed, seed + 1)
        x = torch.from_numpy(L).to(cuda_dev)
        rb, ri, ra = ldpc.decode(code, p, x, app=True)
        torch.cuda.synchronize()
        sb, si, sa = _decode_static(code, p, x, cuda_dev)
        assert rel_err(sa, ra.cpu().numpy()).max() <= FP32_TOL
        assert np.array_equal(si, ri.cpu().numpy())
        assert np.array_equal(sb, rb.cpu().numpy())


def _pool_used_high(dev_index: int):
    """High-water mark of the device's default stream-ordered memory pool (driver API), reset
    to the current use; None if the driver library cannot be reached."""
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError:
        return None
    d, pool, v = ctypes.c_int(), ctypes.c_void_p(), ctypes.c_uint64()
    if cu.cuDeviceGet(ctypes.byref(d), dev_index) or cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), d):
        return None
    return cu, pool, v


def _used_high(h):
    cu, pool, v = h
    assert cu.cuMemPoolGetAttribute(pool, 8, ctypes.byref(v)) == 0   # CU_MEMPOOL_ATTR_USED_MEM_HIGH
    return v.value


def _reset_used_high(h):
    cu, pool, v = h
    v.value = 0
    assert cu.cuMemPoolSetAttribute(pool, 8, ctypes.byref(v)) == 0


@pytest.mark.parametrize("form", ["flood_f32", "stream_f32"])
def test_static_scratch_allocates_nothing_after_the_first_call(cuda_dev, form):
    # the first call on the device reserves the array (lazy module loading); after it, a call
    # leaves the device's free memory and the stream-ordered pool's high-water mark unchanged
    # (the allocating entry point would take its scratch from that pool)
    B, Z = I.load_code("qc12x24_z81_s2")
    code = ldpc.Code(B, Z)
    p = ldpc.params_for(form, max_iter=20)
    n = 500
    _, _, c, L = I.make_frames("qc12x24_z81_s2", n, 1.75, 121, 122)
    x = torch.from_numpy(L).to(cuda_dev)
    bits = torch.empty((n, code.N), dtype=torch.uint8, device=cuda_dev)
    iters = torch.empty((n,), dtype=torch.int32, device=cuda_dev)
    app = torch.empty((n, code.N), dtype=torch.float32, device=cuda_dev)
    stream = torch.cuda.current_stream(cuda_dev)
    ldpc.ldpc_decode_batch_static(code.handle, p, x, n, bits, iters, app, stream)
    torch.cuda.synchronize()
    ref = bits.clone(), iters.clone()
    pool = _pool_used_high(cuda_dev.index or 0)
    if pool:
        _reset_used_high(pool)
        high0 = _used_high(pool)
    free0 = torch.cuda.mem_get_info(cuda_dev)[0]
    bits.zero_()
    ldpc.ldpc_decode_batch_static(code.handle, p, x, n, bits, iters, app, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(cuda_dev)[0] == free0
    if pool:
        assert _used_high(pool) == high0
    assert torch.equal(bits, ref[0]) and torch.equal(iters, ref[1])


def test_static_scratch_rejects_batches_beyond_the_array(cuda_dev):
    # the streaming kernels' scratch grows with the batch (tiles of 128 codewords)
    B, Z = I.load_code("qc12x24_z81_s2")
    code = ldpc.Code(B, Z)
    p = ldpc.params_for("stream_f32")
    assert ldpc.ldpc_workspace_size(code.handle, p, 896) <= ldpc.LDPC_STATIC_SCRATCH_BYTES
    assert ldpc.ldpc_workspace_size(code.handle, p, 897) > ldpc.LDPC_STATIC_SCRATCH_BYTES
    x = torch.zeros((897, code.N), device=cuda_dev)
    b = torch.empty((897, code.N), dtype=torch.uint8, device=cuda_dev)
    i = torch.empty((897,), dtype=torch.int32, device=cuda_dev)
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_decode_batch_static(code.handle, p, x, 897, b, i)
    assert ei.value.status == ldpc.LDPC_ENOMEM and "static array" in str(ei.value)
