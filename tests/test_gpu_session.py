"""The serving loop (ldpc_session) through the C ABI: continuous batching, admission by
memory budget, host-side failure injection, bounded waits and cancellation.  Failures are
made on the host (an injected allocation failure, a paused dispatcher): no GPU fault."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1812_06545_gb300 import inputs as I
from paper_1812_06545_gb300 import ldpc
from tests.gpu_helpers import clopper_pearson, oracle_code

pytestmark = pytest.mark.gpu

_gcodes = {}


def gpu_code(name):
    if name not in _gcodes:
        B, Z = I.load_code(name)
        _gcodes[name] = ldpc.Code(B, Z)
    return _gcodes[name]


class Job:
    def __init__(self, name, form, n, seed):
        self.name, self.form, self.n = name, form, n
        self.code = gpu_code(name)
        self.p = ldpc.params_for(form, max_iter=10 if form == "layered_i8" else 20)
        eb = I.operating_points().get(name, 2.0)
        _, _, self.c, L = I.make_frames(name, n, eb, seed, seed + 1)
        self.llr = torch.from_numpy(L).pin_memory()
        self.bits = torch.empty((n, self.code.N), dtype=torch.uint8).pin_memory()
        self.iters = torch.empty((n,), dtype=torch.int32).pin_memory()

    def reference(self, dev):
        b, i, _ = ldpc.decode(self.code, self.p, self.llr.to(dev))
        torch.cuda.synchronize()
        return b.cpu().numpy(), i.cpu().numpy()

    def submit(self, sess):
        return ldpc.ldpc_session_submit(sess, self.code.handle, self.p, self.llr, self.n, self.bits, self.iters)


def session(**cfg):
    return ldpc.ldpc_session_create(ldpc.ldpc_session_default_config(**cfg))


def test_same_alone_and_in_the_mix(cuda_dev):
    rng = np.random.default_rng(3)
    family = I.MIXED_FAMILY + ["qc12x24_z81_s2"]
    target = Job("qc8x24_z54_s45", "flood_f16", 300, 77)
    ref_b, ref_i = target.reference(cuda_dev)
    s = session(max_inflight=3)
    try:
        rid = target.submit(s)
        st, _ = ldpc.ldpc_session_wait(s, rid, 30.0)
        assert st == ldpc.LDPC_OK
        alone_b, alone_i = target.bits.numpy().copy(), target.iters.numpy().copy()
        assert np.array_equal(alone_b, ref_b) and np.array_equal(alone_i, ref_i)
        target.bits.zero_()
        jobs = [Job(family[int(rng.integers(len(family)))], str(rng.choice(["flood_f16", "layered_i8", "flood_f32"])),
                    int(rng.integers(1, 400)), 1000 + k) for k in range(40)]
        ids = []
        for k, j in enumerate(jobs):
            ids.append((j, j.submit(s)))
            if k == 17:
                ids.append((target, target.submit(s)))
        for j, rid in ids:
            st, lat = ldpc.ldpc_session_wait(s, rid, 60.0)
            assert st == ldpc.LDPC_OK and lat > 0
        assert np.array_equal(target.bits.numpy(), alone_b) and np.array_equal(target.iters.numpy(), alone_i)
        for j in jobs:
            b, i = j.reference(cuda_dev)
            assert np.array_equal(j.bits.numpy(), b) and np.array_equal(j.iters.numpy(), i), (j.name, j.form)
        stats = ldpc.ldpc_session_stats_get(s)
        assert stats.completed == len(ids) + 1 and stats.failed == 0 and stats.launches < len(ids) + 1
        check_against_oracle(jobs + [target])
    finally:
        ldpc.ldpc_session_destroy(s)


def check_against_oracle(jobs):
    """Every served request against the oracle: the int8 min-sum bit-exact (decisions and
    iteration counts); the sum-product forms, aggregated over all requests of a form, with
    identical decisions on >= 99.99 % of the codewords (FP16: wherever both decoders
    converged), the same iteration count on >= 99.9 % of the converged codewords with identical
    decisions (FP16: 99.5 %, a binary16 rounding flip can move the iteration in which the
    syndrome first clears by one), and a frame error rate inside the oracle's 95 % interval."""
    # per form: decision mismatches, codewords compared, iteration mismatches, converged,
    # GPU frame errors, oracle frame errors, codewords
    stats = {"flood_f32": [0] * 7, "flood_f16": [0] * 7}
    for j in jobs:
        oc = oracle_code(j.name)
        L = j.llr.numpy()
        bits, iters = j.bits.numpy(), j.iters.numpy()
        if j.form == "layered_i8":
            _, rb, ri = oc.nms_layered(O.quantize(L, 2.0, 31), 10, early_exit=True)
            assert np.array_equal(bits, rb) and np.array_equal(iters, ri), j.name
            continue
        f16 = j.form == "flood_f16"
        _, rb, ri = oc.spa_flood(L, 20, early_exit=True, fp16_msgs=f16)
        same = (bits == rb).all(axis=1)
        conv = ri < 20
        st = stats[j.form]
        st[2] += int((iters[conv & same] != ri[conv & same]).sum())
        st[3] += int((conv & same).sum())
        if f16:
            same = same[conv & (iters < 20)]
        st[0] += int((~same).sum())
        st[1] += len(same)
        st[4] += int((bits != j.c).any(axis=1).sum())
        st[5] += int((rb != j.c).any(axis=1).sum())
        st[6] += j.n
    for form, (mism, tot, imism, nconv, eg, eo, n) in stats.items():
        if n == 0:
            continue
        assert mism <= 1e-4 * tot, (form, mism, tot)
        assert imism <= (5e-3 if form == "flood_f16" else 1e-3) * nconv, (form, imism, nconv)
        lo, hi = clopper_pearson(eo, n)
        assert lo <= eg / n <= hi, (form, eg, eo, n)


def test_admission_by_memory_budget(cuda_dev):
    budget = 24 << 20
    s = session(hbm_budget_bytes=budget, max_inflight=4)
    try:
        jobs = [Job("qc12x24_z81_s2", "flood_f16", 900, 50 + k) for k in range(12)]   # ~8.8 MB each
        ids = [(j, j.submit(s)) for j in jobs]
        for j, rid in ids:
            assert ldpc.ldpc_session_wait(s, rid, 60.0)[0] == ldpc.LDPC_OK
        stats = ldpc.ldpc_session_stats_get(s)
        assert stats.peak_bytes <= budget and stats.launches >= 4 and stats.completed == 12
        b, i = jobs[5].reference(cuda_dev)
        assert np.array_equal(jobs[5].bits.numpy(), b)
        big = Job("qc12x24_z81_s2", "flood_f16", 3000, 9)
        with pytest.raises(ldpc.LdpcError) as ei:
            big.submit(s)
        assert ei.value.status == ldpc.LDPC_ENOMEM
    finally:
        ldpc.ldpc_session_destroy(s)


def test_injected_allocation_failure(cuda_dev):
    s = session(fail_alloc_after=3, max_inflight=1, max_batch=1)
    try:
        jobs = [Job("qc12x24_z27_s40", "flood_f32", 50, 60 + k) for k in range(5)]
        ids = [(j, j.submit(s)) for j in jobs]
        res = [ldpc.ldpc_session_wait(s, rid, 30.0)[0] for _, rid in ids]
        assert res == [0, 0, ldpc.LDPC_ENOMEM, 0, 0]
        b, i = jobs[4].reference(cuda_dev)
        assert np.array_equal(jobs[4].bits.numpy(), b)
        st = ldpc.ldpc_session_stats_get(s)
        assert st.failed == 1 and st.completed == 4
    finally:
        ldpc.ldpc_session_destroy(s)


def test_pause_timeout_cancel(cuda_dev):
    s = session(start_paused=1)
    try:
        jobs = [Job("qc4x24_z81_s51", "layered_i8", 20, 80 + k) for k in range(3)]
        ids = [j.submit(s) for j in jobs]
        st, _ = ldpc.ldpc_session_wait(s, ids[0], 0.2)
        assert st == ldpc.LDPC_ETIMEDOUT
        state, rc, _ = ldpc.ldpc_session_poll(s, ids[1])
        assert state == ldpc.LDPC_REQ_QUEUED
        assert ldpc.ldpc_session_cancel(s, ids[1]) == ldpc.LDPC_OK
        state, rc, _ = ldpc.ldpc_session_poll(s, ids[1])
        assert state == ldpc.LDPC_REQ_CANCELLED
        ldpc.ldpc_session_pause(s, False)
        for k in (0, 2):
            assert ldpc.ldpc_session_wait(s, ids[k], 30.0)[0] == ldpc.LDPC_OK
            b, i = jobs[k].reference(cuda_dev)
            assert np.array_equal(jobs[k].bits.numpy(), b)
        with pytest.raises(ldpc.LdpcError):
            ldpc.ldpc_session_poll(s, ids[0])  # collected by the wait above
    finally:
        ldpc.ldpc_session_destroy(s)


def test_large_code_request_decodes_alone(cuda_dev):
    s = session(hbm_budget_bytes=1 << 30)
    try:
        j = Job("qc34x68_z384_s5", "flood_f16", 4, 90)
        rid = j.submit(s)
        assert ldpc.ldpc_session_wait(s, rid, 60.0)[0] == ldpc.LDPC_OK
        b, i = j.reference(cuda_dev)
        assert np.array_equal(j.bits.numpy(), b) and np.array_equal(j.iters.numpy(), i)
    finally:
        ldpc.ldpc_session_destroy(s)


def test_two_waiters_on_one_request(cuda_dev):
    # two host threads wait for the same request: the first to wake collects it, the other
    # learns at once that it was collected (LDPC_EINVAL) instead of waiting out its timeout
    import threading
    import time

    s = session(start_paused=1)
    try:
        j = Job("qc12x24_z27_s40", "flood_f32", 40, 95)
        rid = j.submit(s)
        res = []

        def waiter():
            t0 = time.perf_counter()
            st, _ = ldpc.ldpc_session_wait(s, rid, 30.0)
            res.append((st, time.perf_counter() - t0))

        ts = [threading.Thread(target=waiter) for _ in range(2)]
        for t in ts:
            t.start()
        time.sleep(0.3)
        ldpc.ldpc_session_pause(s, False)
        for t in ts:
            t.join(60.0)
        assert sorted(r[0] for r in res) == [ldpc.LDPC_EINVAL, ldpc.LDPC_OK], res
        assert max(r[1] for r in res) < 20.0, res
        b, i = j.reference(cuda_dev)
        assert np.array_equal(j.bits.numpy(), b)
    finally:
        ldpc.ldpc_session_destroy(s)
