"""Flooding sum-product on the GPU (FP32 and FP16 message storage, and the plain FP32
comparator) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import (FP32_TOL, F16_CASCADE_FRAC, assert_binary16_close, binary16_band, clopper_pearson,
                               oracle_code, rel_err)

pytestmark = pytest.mark.gpu

# codes covering the three kernel shapes: check degree <= 8 (4 codewords per lane),
# <= 16 (2 per lane) and <= 32 (1 per lane); batch sizes leave a ragged last tile.
CASES = [("qc12x24_z81_s2", 260, 1.5), ("qc12x24_z27_s1", 300, 2.0), ("qc8x24_z54_s45", 140, 2.5),
         ("qc4x24_z27_s43", 130, 3.5), ("qc10x20_z200_s10", 170, 2.0)]

_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


def run(name, form, L, dev, **kw):
    code = gpu_code(name)
    p = ldpc.params_for(form, **kw)
    bits, iters, app = ldpc.decode(code, p, torch.from_numpy(L).to(dev), app=True)
    torch.cuda.synchronize()
    return app.cpu().numpy(), bits.cpu().numpy(), iters.cpu().numpy()


@pytest.mark.parametrize("form", ["flood_f32", "stream_f32", "plain_f32"])
@pytest.mark.parametrize("name,n,eb", CASES)
def test_fp32_posterior_first_three_iterations(cuda_dev, form, name, n, eb):
    _, _, c, L = I.make_frames(name, n, eb, 3, 4)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, bits, iters = run(name, form, L, cuda_dev, max_iter=T, early_exit=0)
        ref, rbits, _ = oc.spa_flood(L, T, early_exit=False)
        err = rel_err(app, ref)
        assert err.max() <= FP32_TOL, (form, name, T, err.max())
        assert (iters == T).all()
        assert np.array_equal(bits, (app < 0).astype(np.uint8))


@pytest.mark.parametrize("form", ["flood_f16", "stream_f16"])
@pytest.mark.parametrize("name,n,eb", CASES)
def test_fp16_messages_first_three_iterations(cuda_dev, form, name, n, eb):
    # The oracle models half-precision message storage (messages rounded to binary16).
    # Beyond the fp32 tolerance the two may differ by the rounding of each incoming message
    # (FP32 vs FP64 values on either side of a binary16 rounding boundary): a band of 4
    # binary16 half-ulps (2^-11 relative) of every incoming message, on every codeword after
    # the first iteration, and on all but a few codewords (rounding flips that cascade) after
    # the second and third
    _, _, c, L = I.make_frames(name, n, eb, 5, 6)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, _, _ = run(name, form, L, cuda_dev, max_iter=T, early_exit=0)
        ref, band = binary16_band(oc, False, L, T, 4)
        assert_binary16_close(app, ref, band, strict=T == 1, what=(name, T))


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "stream_f32", "layered_f32"])
@pytest.mark.parametrize("name,n,eb", [("qc12x24_z81_s2", 400, 2.0), ("qc8x24_z54_s45", 300, 2.5)])
@pytest.mark.parametrize("X", [2.5, 6.0])
def test_small_phi_clamp(cuda_dev, form, name, n, eb, X):
    # a clamp X whose lower end phi(X) is far from 0 (phi(2.5) = 0.165, phi(6) = 0.005):
    # both ends of [phi(X), X] bind on many messages, so a decoder that drops either end
    # of the clamp, or applies it to the wrong quantity, leaves the tolerance
    _, _, c, L = I.make_frames(name, n, eb, 91, 92)
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, _, _ = run(name, form, L, cuda_dev, max_iter=T, early_exit=0, phi_clamp=X)
        if form.endswith("f16"):
            ref, band = binary16_band(oc, False, L, T, 4, X=X)
            assert_binary16_close(app, ref, band, strict=T == 1, what=(name, T, X))
            continue
        orc = oc.spa_layered if form.startswith("layered") else oc.spa_flood
        ref, _, _ = orc(L, T, early_exit=False, X=X)
        err = rel_err(app, ref)
        assert err.max() <= FP32_TOL, (form, name, T, X, err.max())


@pytest.mark.parametrize("form", ["flood_f32", "stream_f32", "plain_f32", "layered_f32"])
def test_erased_inputs(cuda_dev, form):
    # 10 % of the LLRs erased (exactly 0, some of them -0.0): a zero |Q| is clamped up to
    # phi(X) and counts as positive, so the check's other messages are at most phi(X) ~ 4e-35
    # (0 in FP32); iterations 1-3 within the FP32 tolerance of the oracle, no NaN anywhere
    name = "qc12x24_z81_s2"
    _, _, c, L = I.make_frames(name, 300, 2.5, 81, 82)
    rng = np.random.default_rng(83)
    er = rng.random(L.shape) < 0.1
    L[er] = 0.0
    L[er & (rng.random(L.shape) < 0.5)] = -0.0
    oc = oracle_code(name)
    for T in (1, 2, 3):
        app, _, _ = run(name, form, L, cuda_dev, max_iter=T, early_exit=0)
        assert np.isfinite(app).all(), (form, T)
        orc = oc.spa_layered if form.startswith("layered") else oc.spa_flood
        ref, _, _ = orc(L, T, early_exit=False)
        err = rel_err(app, ref)
        assert err.max() <= FP32_TOL, (form, T, err.max())


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "stream_f32", "stream_f16", "plain_f32"])
def test_early_exit_and_fer_full_size(cuda_dev, form):
    # 8192 codewords of the rate-1/2 N=1944 code, early exit, max 20 iterations, at 1.5
    # and 2.0 dB, in the launch configuration the benchmark times: the GPU frame error rate
    # inside the oracle's 95 % Clopper-Pearson interval; FP32 hard decisions identical to the
    # FP64 oracle on >= 99.99 % of codewords.  Half-precision storage is held to the FER
    # interval and to identical decisions wherever both decoders converged (where neither
    # converges, 20 iterations of the non-converging dynamics amplify the binary16 rounding).
    name = "qc12x24_z81_s2"
    oc = oracle_code(name)
    f16 = form.endswith("f16")
    mism = tot = 0
    for eb, seed in ((1.5, 23), (2.0, 25)):
        _, _, c, L = I.make_frames(name, 8192, eb, 20, seed)
        app, bits, iters = run(name, form, L, cuda_dev, max_iter=20, early_exit=1)
        _, rbits, riters = oc.spa_flood(L, 20, early_exit=True, fp16_msgs=f16)
        same = (bits == rbits).all(axis=1)
        mism += int((~same).sum())
        tot += len(same)
        fer_g = int((bits != c).any(axis=1).sum())
        fer_o = int((rbits != c).any(axis=1).sum())
        lo, hi = clopper_pearson(fer_o, len(c))
        assert lo <= fer_g / len(c) <= hi, (form, eb, fer_g, fer_o)
        conv = riters < 20
        assert (iters[conv & same] == riters[conv & same]).mean() >= 0.999
        if f16:
            both = conv & (iters < 20)
            assert (same[both]).mean() >= 0.9999, (eb, int((~same[both]).sum()))
    if not f16:
        assert mism <= 1e-4 * tot, (form, mism, tot)


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16", "stream_f32"])
def test_batch_invariance(cuda_dev, form):
    # a codeword decodes to the same bits, posterior and iteration count alone and in a
    # batch (whatever slot or tile position it lands in)
    name = "qc12x24_z81_s2"
    _, _, c, L = I.make_frames(name, 3000, 1.75, 7, 8)
    app_all, _, it_all = run(name, form, L, cuda_dev, max_iter=20, early_exit=1)
    for i in (0, 127, 128, 1499, 2999):
        app1, _, it1 = run(name, form, L[i:i + 1].copy(), cuda_dev, max_iter=20, early_exit=1)
        assert np.array_equal(app1[0], app_all[i]) and it1[0] == it_all[i]


@pytest.mark.parametrize("name,slots,eb", [("qc16x32_z32_s7", 20, 2.0), ("qc12x24_z24_s6", 40, 2.0),
                                            ("qc12x24_z81_s2", 12, 1.75)])
def test_paired_slots_in_barrier_groups(cuda_dev, name, slots, eb):
    # A batch that fills every CTA's FP16 slots, so that the paired slots run in independent
    # barrier groups: one-warp groups for Z = 32, groups of four thread slots in three whole
    # warps for Z = 24, two groups of three for Z = 81.  Batches of two codewords per SM
    # run one group per CTA.  Every codeword's arithmetic is its own, so the grouped decode
    # must equal, bit for bit, the decode of the same codewords in such small batches (early
    # exit on: slots finish at different iterations and refill at different times).  The
    # first iteration also follows the FP16-message oracle on every codeword.
    n = 152 * slots
    _, _, c, L = I.make_frames(name, n, eb, 71, 72)
    oc = oracle_code(name)
    app, _, _ = run(name, "flood_f16", L, cuda_dev, max_iter=1, early_exit=0)
    ref, band = binary16_band(oc, False, L, 1, 4)
    assert_binary16_close(app, ref, band, strict=True, what=name)
    app_all, bits_all, it_all = run(name, "flood_f16", L, cuda_dev, max_iter=20, early_exit=1)
    assert len(np.unique(it_all)) > 1  # codewords finish at different iterations
    chunk = 2 * 152
    for a in range(0, n, chunk):
        app1, bits1, it1 = run(name, "flood_f16", L[a:a + chunk].copy(), cuda_dev, max_iter=20, early_exit=1)
        assert np.array_equal(app1, app_all[a:a + chunk]), (name, a)
        assert np.array_equal(bits1, bits_all[a:a + chunk]) and np.array_equal(it1, it_all[a:a + chunk])


def test_small_and_empty_batches(cuda_dev):
    name = "qc12x24_z27_s1"
    code = gpu_code(name)
    p = ldpc.params_for("flood_f32", max_iter=5)
    empty = torch.empty((0, code.N), dtype=torch.float32, device=cuda_dev)
    bits, iters, _ = ldpc.decode(code, p, empty)
    assert bits.shape == (0, code.N)
    _, _, c, L = I.make_frames(name, 1, 2.5, 9, 10)
    app, bits, iters = run(name, "flood_f32", L, cuda_dev, max_iter=5, early_exit=1)
    ref, rbits, riters = oracle_code(name).spa_flood(L, 5, early_exit=True)
    assert rel_err(app, ref).max() <= FP32_TOL and np.array_equal(iters, riters)


def test_slot_and_streaming_paths_agree(cuda_dev):
    # the on-chip slot decoder and the HBM-streaming kernels compute the same iteration;
    # they differ only in summation order, so decisions and iteration counts agree
    name = "qc12x24_z81_s2"
    _, _, c, L = I.make_frames(name, 4096, 2.0, 13, 14)
    a1, b1, i1 = run(name, "flood_f32", L, cuda_dev, max_iter=20, early_exit=1)
    a2, b2, i2 = run(name, "stream_f32", L, cuda_dev, max_iter=20, early_exit=1)
    conv = (i1 < 20) & (i2 < 20)
    assert np.array_equal(b1[conv], b2[conv]) and np.array_equal(i1[conv], i2[conv])
    assert (b1 == b2).all(axis=1).mean() >= 0.999


def test_eq1_code_z1_and_extreme_shifts(cuda_dev):
    H = np.loadtxt(__import__("os").path.join(__import__("os").path.dirname(__file__), "golden", "eq1_H.txt"))
    base = np.where(H == 1, 0, -1).astype(np.int32)
    rng = np.random.default_rng(0)
    for B, Z in ((base, 1), (np.array([[0, 6, -1, 3], [6, 0, 6, -1], [-1, 6, 0, 0]], np.int32), 7)):
        code = ldpc.Code(B, Z)
        oc = O.QCCode(B, Z)
        L = (1.5 + 2.0 * rng.standard_normal((37, code.N))).astype(np.float32)
        for T in (1, 3):
            for form in ("flood_f32", "stream_f32"):
                bits, iters, app = ldpc.decode(code, ldpc.params_for(form, max_iter=T, early_exit=0),
                                               torch.from_numpy(L).to(cuda_dev), app=True)
                ref, _, _ = oc.spa_flood(L, T, early_exit=False)
                assert rel_err(app.cpu().numpy(), ref).max() <= FP32_TOL


def test_multistream_host_path_matches_device_path(cuda_dev):
    name = "qc12x24_z81_s2"
    code = gpu_code(name)
    _, _, c, L = I.make_frames(name, 1000, 1.75, 11, 12)
    p = ldpc.params_for("flood_f32", max_iter=20)
    bits_d, it_d, _ = ldpc.decode(code, p, torch.from_numpy(L).to(cuda_dev))
    torch.cuda.synchronize()
    Lh = torch.from_numpy(L).pin_memory()
    bh = torch.empty((1000, code.N), dtype=torch.uint8).pin_memory()
    ih = torch.empty((1000,), dtype=torch.int32).pin_memory()
    ldpc.ldpc_decode_host(code.handle, p, Lh, 1000, bh, ih, n_streams=3, chunk_cw=200)
    assert np.array_equal(bh.numpy(), bits_d.cpu().numpy()) and np.array_equal(ih.numpy(), it_d.cpu().numpy())


def test_argument_errors(cuda_dev):
    code = gpu_code("qc12x24_z27_s1")
    x = torch.zeros((4, code.N), device=cuda_dev)
    b = torch.empty((4, code.N), dtype=torch.uint8, device=cuda_dev)
    i = torch.empty((4,), dtype=torch.int32, device=cuda_dev)
    for bad in (dict(max_iter=0), dict(phi_clamp=0.5), dict(msg=ldpc.LDPC_MSG_I8), dict(early_exit=2)):
        with pytest.raises(ldpc.LdpcError):
            ldpc.ldpc_decode_batch(code.handle, ldpc.params_for("flood_f32", **bad), x, 0, 4, b, i)
    with pytest.raises(ldpc.LdpcError):
        ldpc.ldpc_decode_batch(code.handle, ldpc.params_for("flood_f32"), x, 0, 4, None, i)
    p = ldpc.params_for("flood_f32")
    need = ldpc.ldpc_workspace_size(code.handle, p, 4)
    ws = torch.empty(need // 4 + 64, dtype=torch.int32, device=cuda_dev)
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_decode_batch(code.handle, p, x, 0, 4, b, i, None, ws, need - 1)
    assert ei.value.status == ldpc.LDPC_ENOMEM
    ldpc.ldpc_decode_batch(code.handle, p, x, 0, 4, b, i, None, ws, need)
    torch.cuda.synchronize()


@pytest.mark.parametrize("form", ["flood_f32", "flood_f16"])
def test_multistream_host_path_against_the_oracle(cuda_dev, form):
    # Sec. III-C: W = 3 streams, each chunk copied in, decoded and copied out on its own
    # stream.  (1) Three iterations without early exit: every decision at a bit whose oracle
    # posterior lies outside the tolerance band around 0 equals the oracle's.  (2) The
    # full-size workload (8192 codewords at 1.5 and 2.0 dB, early exit, max 20) through the
    # host path: decisions and iteration counts against the oracle, FER inside its 95 %
    # interval, as for the device path.
    name = "qc12x24_z81_s2"
    code = gpu_code(name)
    oc = oracle_code(name)
    f16 = form.endswith("f16")

    def host_decode(L, p):
        n = L.shape[0]
        Lh = torch.from_numpy(L).pin_memory()
        bh = torch.empty((n, code.N), dtype=torch.uint8).pin_memory()
        ih = torch.empty((n,), dtype=torch.int32).pin_memory()
        ldpc.ldpc_decode_host(code.handle, p, Lh, n, bh, ih, n_streams=3, chunk_cw=700)
        return bh.numpy().copy(), ih.numpy().copy()

    _, _, c, L = I.make_frames(name, 2100, 1.75, 111, 112)
    bits, iters = host_decode(L, ldpc.params_for(form, max_iter=3, early_exit=0))
    assert (iters == 3).all()
    if f16:
        ref, band = binary16_band(oc, False, L, 3, 4)
    else:
        ref, _, _ = oc.spa_flood(L, 3, early_exit=False)
        band = FP32_TOL * np.maximum(1.0, np.abs(ref))
    rbits = (ref < 0).astype(np.uint8)
    clear = np.abs(ref) > band
    wrong = ((bits != rbits) & clear).any(axis=1).sum()
    assert wrong <= (F16_CASCADE_FRAC * len(L) if f16 else 0), (form, wrong)
    mism = tot = 0
    for eb, seed in ((1.5, 23), (2.0, 25)):
        _, _, c, L = I.make_frames(name, 8192, eb, 20, seed)
        bits, iters = host_decode(L, ldpc.params_for(form, max_iter=20, early_exit=1))
        _, rbits, riters = oc.spa_flood(L, 20, early_exit=True, fp16_msgs=f16)
        same = (bits == rbits).all(axis=1)
        mism += int((~same).sum())
        tot += len(same)
        fer_g, fer_o = int((bits != c).any(axis=1).sum()), int((rbits != c).any(axis=1).sum())
        lo, hi = clopper_pearson(fer_o, len(c))
        assert lo <= fer_g / len(c) <= hi, (form, eb, fer_g, fer_o)
        conv = riters < 20
        assert (iters[conv & same] == riters[conv & same]).mean() >= 0.999
        if f16:
            both = conv & (iters < 20)
            assert same[both].mean() >= 0.9999, (eb, int((~same[both]).sum()))
    if not f16:
        assert mism <= 1e-4 * tot, (form, mism, tot)
