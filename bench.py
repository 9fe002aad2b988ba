#!/usr/bin/env python3
"""Throughput benchmark of the GB300 LDPC decoder.

One step = one pass of the decoding path over the FP32 flooding sum-product sweep
workload: 7 batches of 8192 codewords of the seeded rate-1/2 QC code (N = 1944, K = 972),
one per Eb/N0 in 1.0..2.5 dB (0.25 dB steps), early exit after at most 20 iterations:
interleave, check-node and variable-node phases with the fused syndrome, deinterleave.
Metric: decoded info Gbit/s (K x codewords / time).  Also timed on the same inputs: the
FP16-message form and the plain FP32 comparator; and the int8 layered min-sum form on its
own workload (65536 codewords of the rate-5/6 code at 4.0 dB).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank decodes its own batches (weak scaling, no data-path collective);
timing is bracketed by a barrier and synchronize on both sides and the maximum over
ranks is reported by rank 0 as one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded info Gbit/s and p99 latency at equal FER vs plain FP32 flooding SPA, 1 GB300"
WORKLOAD = "flood_n1944_b8192_sweep"
LAYERED_WORKLOAD = "layered_i8_n1944_r56_b65536"
_CSRC = os.path.join(ROOT, "paper_1812_06545_gb300", "csrc")
# the files each profiled kernel is compiled from: a stored ncu traffic figure is used only
# while their combined hash is unchanged
CN_SOURCES = ("flood_kernels.cu", "ldpc_internal.h")
SLOTS_SOURCES = ("flood_slots.cu", "slot_common.cuh", "ldpc_internal.h")


def strip_comments(src: str) -> str:
    """C/C++ source without its comments and blank lines (string and character literals kept),
    so that a comment-only edit leaves the hash of the compiled code unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(ln.rstrip() for ln in "".join(out).splitlines() if ln.strip())


def source_sha256(names):
    """Hash of the comment-stripped sources a kernel is compiled from."""
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(_CSRC, n), encoding="utf-8") as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()


def stored_traffic(kernel, sources):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None when the
    kernel's sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            ent = json.load(f).get(kernel)
        if ent and ent.get("source_sha256") == source_sha256(sources):
            return ent.get("bytes_per_launch_full_size")
    except (OSError, ValueError):
        pass
    return None


def streaming_roofline(ldpc, iters_np, steps, N, E, T, hbm_peak, peak_src):
    """HBM roofline of the streaming check-node kernel from the library's event timing and
    the iteration counts (CN(t) runs while t <= iters + 1, VN(t) while t <= iters)."""
    n_cn, cn_ms = ldpc.ldpc_profile_read("check_node")
    n_vn, vn_ms = ldpc.ldpc_profile_read("variable_node")
    cn_bytes = vn_bytes = 0
    for it in iters_np:
        last_cn = np.where(it < T, it + 1, T)
        for t in range(1, T + 1):
            cn_bytes += int((last_cn >= t).sum()) * (4 * N + 4 * E + (4 * E if t >= 2 else 0))
            vn_bytes += int((it >= t).sum()) * (4 * E + 8 * N)
    cn_gbs = steps * cn_bytes / (cn_ms * 1e-3) / 1e9 if cn_ms > 0 else None
    vn_gbs = steps * vn_bytes / (vn_ms * 1e-3) / 1e9 if vn_ms > 0 else None
    traffic = stored_traffic("k_flood_cn", CN_SOURCES)
    return {"bound": "hbm", "kernel": "k_flood_cn (check-node phase)", "achieved": cn_gbs, "peak": hbm_peak,
            "unit": "GB/s", "frac": (cn_gbs / hbm_peak) if cn_gbs else None, "peak_source": peak_src,
            "frac_of_nominal_7900": (cn_gbs / 7900.0) if cn_gbs else None,
            "traffic": traffic, "launches": n_cn, "avg_launch_ms": cn_ms / max(n_cn, 1),
            "algorithmic_bytes_per_cw_iteration": 4 * N + 8 * E,
            "variable_node": {"achieved": vn_gbs, "frac": (vn_gbs / hbm_peak) if vn_gbs else None,
                              "launches": n_vn, "avg_launch_ms": vn_ms / max(n_vn, 1),
                              "algorithmic_bytes_per_cw_iteration": 4 * E + 8 * N}}


# ------------------------------------------------------------------ replicas (N > 1)

def reduce_max(dist, x: float, device=None) -> float:
    """The maximum of x over all ranks (x itself without a process group): the job's time is
    the slowest rank's."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbps(world: int, codewords_per_rank: int, K: int, seconds_max: float) -> float:
    """Information Gbit/s of the whole job: the codewords every rank decoded (weak scaling, the
    same work per rank) over the slowest rank's time."""
    return world * codewords_per_rank * K / seconds_max / 1e9


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--streams", type=int, default=4, help="streams of the end-to-end host path")
    ap.add_argument("--no-forms", action="store_true", help="time only the headline form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample budget")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--serve-seconds", type=float, default=1.5, help="arrival window per offered rate")
    ap.add_argument("--no-paper-shape", action="store_true", help="skip the frame-length / stream sweep")
    ap.add_argument("--no-equal-fer", action="store_true", help="skip the equal-FER throughput comparison")
    ap.add_argument("--fer-frames", type=int, default=400000, help="frames per equal-FER point")
    ap.add_argument("--details", default=os.environ.get("LDPC_BENCH_DETAILS") or
                    os.path.join(tempfile.gettempdir(), "ldpc_bench_details.json"),
                    help="file that receives every section of the run (the last stdout line is a summary)")
    return ap.parse_args()


# ------------------------------------------------------------------ inputs

def workload_frames(name: str, rank: int = 0):
    """[(ebn0, c uint8 [n, N], L fp32 [n, N])] for a named workload (rank-offset noise seeds)."""
    from paper_1812_06545_gb300 import inputs as I

    w = I.WORKLOADS[name]
    out = []
    for eb, ns in zip(w.ebn0_db, w.noise_seeds):
        B, Z, c, L = I.make_frames(w.code, w.batch, eb, w.info_seed + 1000 * rank, ns + 1000 * rank)
        out.append((eb, c, L))
    return w, B, Z, out


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary); LDPC_CLOCKS_DIR keeps them
        out = os.environ.get("LDPC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"ldpc_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"unavailable": "nvidia-smi not available"}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"unavailable": "no samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample_rate(frames, code_name: str, max_iter: int, budget_s: float, threads: int = 0):
    """Time the FP64 oracle on a bounded sample of every batch: returns (info bits/s,
    description, cores used, frame errors, frames)."""
    from oracle import oracle as O
    from paper_1812_06545_gb300 import inputs as I

    B, Z = I.load_code(code_name)
    oc = O.QCCode(B, Z)
    cores = threads or O.num_threads()
    # calibrate on 8 codewords of the hardest batch, then size the per-batch sample
    t0 = time.perf_counter()
    oc.spa_flood(frames[0][2][:8], max_iter, True, nthreads=threads)
    per_cw = max((time.perf_counter() - t0) / 8, 1e-5)
    n = int(max(8, min(len(frames[0][2]), budget_s / (per_cw * len(frames)))))
    t0 = time.perf_counter()
    errs = 0
    obits = []
    for eb, c, L in frames:
        _, bits, _ = oc.spa_flood(L[:n], max_iter, True, nthreads=threads)
        errs += int((bits != c[:n]).any(axis=1).sum())
        obits.append(bits)
    dt = time.perf_counter() - t0
    rate = n * len(frames) * oc.K / dt
    return rate, f"first {n} codewords of each of the {len(frames)} Eb/N0 batches ({n * len(frames)} codewords)", \
        cores, errs, n * len(frames), obits


# ------------------------------------------------------------------ serving loop

def run_serving(ldpc, dev, window_s: float):
    """Poisson arrivals of requests of 1..512 codewords, each of one code drawn uniformly from
    the 12-code family plus the N = 26112 code, half FP16 sum-product and half int8 layered
    min-sum, into one ldpc_session.  A closed-loop burst first measures the session's
    capacity; the offered rate is then swept as fractions of it.  Latency is the session's
    own submission-to-completion stamp."""
    import torch

    from paper_1812_06545_gb300 import inputs as I

    rng = np.random.default_rng(5)
    names = I.MIXED_FAMILY + ["qc34x68_z384_s5"]
    ops = I.operating_points()
    pool = []
    for k, name in enumerate(names):
        B, Z = I.load_code(name)
        code = ldpc.Code(B, Z)
        n = 512
        _, _, c, L = I.make_frames(name, n, ops.get(name, 2.0), 500 + k, 600 + k)
        pool.append((code, torch.from_numpy(L).pin_memory(), torch.empty((n, code.N), dtype=torch.uint8).pin_memory(),
                     torch.empty((n,), dtype=torch.int32).pin_memory()))
    forms = {"flood_f16": ldpc.params_for("flood_f16", max_iter=20),
             "layered_i8": ldpc.params_for("layered_i8", max_iter=10)}
    cfg = ldpc.ldpc_session_default_config(hbm_budget_bytes=16 << 30, max_inflight=4)
    sess = ldpc.ldpc_session_create(cfg)

    def draw():
        k = int(rng.integers(len(pool)))
        n = int(rng.integers(1, 513))
        form = "flood_f16" if rng.random() < 0.5 else "layered_i8"
        return k, n, form

    def submit(k, n, form):
        code, L, bits, it = pool[k]
        o = int(rng.integers(0, 513 - n))
        return ldpc.ldpc_session_submit(sess, code.handle, forms[form], L[o:o + n], n, bits[o:o + n],
                                        it[o:o + n]), code.K * n

    failed = [0]

    def collect(ids):
        # latency and information bits of the requests that decoded; a failed request counts
        # against the run (the serving section is marked invalid) and adds no bits or latency
        lat, bits_done = [], 0
        for rid, kb in ids:
            st, t = ldpc.ldpc_session_wait(sess, rid, 120.0)
            if st == 0:
                lat.append(t)
                bits_done += kb
            else:
                failed[0] += 1
        return lat, bits_done

    try:
        for _ in range(2):  # warm-up (tables, attributes, pinned-memory paths)
            collect([submit(*draw()) for _ in range(32)])
        burst = [draw() for _ in range(1500)]
        t0 = time.perf_counter()
        ids = [submit(*d) for d in burst]
        lat, kb = collect(ids)
        t_cap = time.perf_counter() - t0
        cap_rps = len(lat) / t_cap
        cap_gbps = kb / t_cap / 1e9
        out = {"workload": "requests of 1-512 codewords, code uniform over 12 family codes + N=26112 code, "
                           "half FP16 SPA / half int8 layered NMS, Poisson arrivals",
               "session": {"hbm_budget_bytes": cfg.hbm_budget_bytes, "max_inflight": cfg.max_inflight,
                           "max_batch": cfg.max_batch},
               "capacity": {"requests_per_s": cap_rps, "info_gbps": cap_gbps, "burst_requests": len(burst)},
               "sweep": []}
        for frac in (0.25, 0.5, 0.75, 0.9, 1.0, 1.2):
            rate = frac * cap_rps
            ids = []
            t0 = time.perf_counter()
            t_next = t0
            while True:
                now = time.perf_counter()
                if now - t0 >= window_s:
                    break
                if now < t_next:
                    continue
                ids.append(submit(*draw()))
                t_next += rng.exponential(1.0 / rate)
            lat, kb = collect(ids)
            t_all = time.perf_counter() - t0
            lat_ms = np.array(lat) * 1e3
            out["sweep"].append({"offered_fraction": frac, "offered_rps": rate, "requests": len(ids),
                                 "achieved_info_gbps": kb / t_all / 1e9,
                                 "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99))})
        sat = [x for x in out["sweep"] if x["offered_fraction"] == 1.0][0]
        out["at_saturation"] = {"achieved_info_gbps": sat["achieved_info_gbps"], "p50_ms": sat["p50_ms"],
                                "p99_ms": sat["p99_ms"]}
        st = ldpc.ldpc_session_stats_get(sess)
        out["stats"] = {"launches": st.launches, "completed": st.completed, "failed": st.failed,
                        "peak_bytes": st.peak_bytes}
        out["failed_requests"] = failed[0]
        out["valid"] = failed[0] == 0
        if failed[0]:
            print(f"serving: {failed[0]} requests failed; the serving numbers are not valid", file=sys.stderr)
        return out
    finally:
        ldpc.ldpc_session_destroy(sess)


# ------------------------------------------------------------------ mixed codes (one launch)

def run_mixed(ldpc, dev, rank, world, steps, warmup, max_over_ranks, barrier, n_total: int = 20000):
    """20000 codewords, each of a code drawn uniformly from the 12-code family (Z in {27, 54,
    81} x rate {1/2, 2/3, 3/4, 5/6}), every code at its FER ~1e-2 operating point, FP16
    messages, max 20 iterations: one persistent ldpc_decode_multi launch per step.  Before
    timing, ldpc_autotune picks each code's schedule on a sample of its own frames.  Timed
    twice: eager calls, and replays of a CUDA graph that captured the call."""
    import torch

    from paper_1812_06545_gb300 import inputs as I

    stream = torch.cuda.current_stream(dev)
    mixed = I.mixed_batch(n_total, 40 + rank)
    mp = ldpc.params_for("flood_f16", max_iter=20)
    mreqs, mK, tuned = [], 0, {}
    for name, c, L in mixed:
        mb_, mZ = I.load_code(name)
        mc = ldpc.Code(mb_, mZ)
        x = torch.from_numpy(L).to(dev)
        o = (torch.empty((len(L), mc.N), dtype=torch.uint8, device=dev),
             torch.empty((len(L),), dtype=torch.int32, device=dev))
        if len(L):
            choice, tms = ldpc.ldpc_autotune(mc.handle, mp, x, ldpc.LDPC_LLR_F32, len(L), stream)
            tuned[name] = {"choice": {1: "slots x1", 2: "slots x2", 3: "streaming"}.get(choice, str(choice)),
                           "ms": [float(t) for t in tms]}
        mreqs.append((mc, x, len(L), o[0], o[1], c))
        mK += mc.K * len(L)
    mws = torch.empty(ldpc.ldpc_multi_workspace_size(), dtype=torch.uint8, device=dev)
    margs = [(q[0].handle, q[1], q[2], q[3], q[4], None) for q in mreqs]

    def launch(st):
        ldpc.ldpc_decode_multi(margs, mp, ldpc.LDPC_LLR_F32, mws, mws.numel(), st)

    def timed(fn):
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1))

    for _ in range(max(warmup, 1)):
        launch(stream)
    eager_ms = timed(lambda: launch(stream))
    eager_bits = [q[3].clone() for q in mreqs]
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        launch(side)
    torch.cuda.synchronize()
    for q in mreqs:
        q[3].zero_()
    for _ in range(max(warmup, 1)):
        g.replay()
    graph_ms = timed(g.replay)
    same = all(torch.equal(q[3], b) for q, b in zip(mreqs, eager_bits))
    n = sum(q[2] for q in mreqs)
    errs = sum(int((q[3].cpu().numpy() != q[5]).any(axis=1).sum()) for q in mreqs)
    per_code = {name: float((q[3].cpu().numpy() != q[5]).any(axis=1).mean()) if q[2] else None
                for (name, _, _), q in zip(mixed, mreqs)}
    return {"workload": f"mixed_12codes_b{n_total} (Z in {{27,54,81}} x rate {{1/2,2/3,3/4,5/6}}, each code at "
                        "its FER~1e-2 operating point, FP16 messages, max 20 iterations)",
            "api": "graph replay of one ldpc_decode_multi launch per step (eager calls timed beside it)",
            "value": world * steps * mK / (graph_ms * 1e-3) / 1e9, "graph_info_gbps": world * steps * mK / (graph_ms * 1e-3) / 1e9,
            "eager_info_gbps": world * steps * mK / (eager_ms * 1e-3) / 1e9, "ms_per_launch_graph": graph_ms / steps,
            "ms_per_launch_eager": eager_ms / steps, "graph_equals_eager": bool(same), "codewords": n,
            "fer": errs / n, "fer_per_code": per_code, "autotuned": tuned,
            "frames": [(name, q[1], q[3], q[5]) for (name, _, _), q in zip(mixed, mreqs)]}


def mixed_oracle_check(frames, per_code: int, budget_s: float):
    """FER of the FP64 oracle and of the mixed launch on the first codewords of every code of
    the mixed batch (the same frames), and the share of identical decisions."""
    from oracle import oracle as O
    from paper_1812_06545_gb300 import inputs as I

    t0 = time.perf_counter()
    go = oo = same = tot = 0
    for name, x, bits, c in frames:
        if time.perf_counter() - t0 > budget_s:
            break
        n = min(per_code, x.shape[0])
        if n == 0:
            continue
        B, Z = I.load_code(name)
        _, ob, _ = O.QCCode(B, Z).spa_flood(x[:n].cpu().numpy(), 20, True, fp16_msgs=True)
        gb = bits[:n].cpu().numpy()
        go += int((gb != c[:n]).any(axis=1).sum())
        oo += int((ob != c[:n]).any(axis=1).sum())
        same += int((gb == ob).all(axis=1).sum())
        tot += n
    return {"codewords": tot, "gpu_fer": go / max(tot, 1), "oracle_fer": oo / max(tot, 1),
            "identical_decisions": same / max(tot, 1), "oracle": "FP64 flooding SPA with binary16 message storage"}


# ------------------------------------------------------------------ the summary line

SUMMARY_LIMIT = 2400     # bytes of the last stdout line


def _sig(x, digits: int = 4):
    """x with every float rounded to `digits` significant digits (non-finite -> None)."""
    if isinstance(x, float):
        if x != x or x in (float("inf"), float("-inf")):
            return None
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: _sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_sig(v, digits) for v in x]
    return x


def summary_line(line: dict, details_path: str) -> dict:
    """The run's last stdout line: the required keys and the headline figure of every section,
    rounded, within SUMMARY_LIMIT bytes.  The optional sections join in priority order (serving,
    the equal-FER ratios, the forms), each only if the line still fits; every section in full
    is in the details file."""
    out = {k: line[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                                "higher_is_better", "scaling", "vs_baseline", "dtype", "data")}
    cfg = line["config"]
    out["config"] = {"workload": cfg["workload"], "code": cfg["code"], "N": cfg["N"], "K": cfg["K"],
                     "batch": cfg["batch"], "ebn0_db": "1.0-2.5 step 0.25", "max_iter": cfg["max_iter"],
                     "early_exit": True, "parallelism": cfg["parallelism"], "l2": "inputs larger than L2"}
    rf = line["roofline"]
    out["roofline"] = {"bound": rf["bound"], "kernel": "k_flood_slots", "achieved": rf["achieved"],
                       "peak": rf["peak"], "unit": rf["unit"], "frac": rf["frac"], "traffic": rf["traffic"],
                       "peak_source": "SFU rates measured live: 1/(1/ex2+2/lg2) edge updates/s (product-domain "
                                      "check rule)"}
    if rf.get("frac_of_phi_rule_ceiling") is not None:
        # the same throughput against the ceiling of the phi-domain rule, 1/(2/ex2+4/lg2)
        out["roofline"]["frac_of_phi_rule_ceiling"] = rf["frac_of_phi_rule_ceiling"]
    out["latency_ms"] = {"p50": line["latency_ms"]["p50"], "p99": line["latency_ms"]["p99"]}
    e2e = line["e2e"]
    out["e2e"] = {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "streams")}
    for k in ("gpu_launches", "avg_iterations", "coded_bit_iterations_per_s"):
        out[k] = line[k]
    clk = line.get("clocks") or {}
    out["clocks"] = {k: clk[k] for k in ("sm_mhz", "sm_max_mhz", "reasons") if k in clk} or clk
    if "cpu_baseline" in line:
        cb = line["cpu_baseline"]
        out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        d = cb.get("fer_delta_vs_oracle", {})
        out["cpu_baseline"]["fer_delta_max"] = {f: max(abs(v["delta"]) for v in r["per_ebn0"].values())
                                                for f, r in d.items()}
        if "mixed_f16" in cb:
            out["cpu_baseline"]["mixed_fer_delta"] = cb["mixed_f16"]["gpu_fer"] - cb["mixed_f16"]["oracle_fer"]
    opt = []
    sv = line.get("serving")
    if sv:
        opt.append(("serving", {"capacity_gbps": sv["capacity"]["info_gbps"], **sv["at_saturation"],
                                "p99_ms_quarter_load": sv["sweep"][0]["p99_ms"], "valid": sv["valid"]}))
    ef = line.get("equal_fer")
    if ef:
        eq = {}
        for c in ef["codes"]:
            eq[c["code"]] = {"ebn0_star_db": c["ebn0_star_db"], "plain_f32_gbps": c["reference"]["info_gbps"]}
            for r in c["forms"]:
                eq[c["code"]][r["form"]] = [r["ratio_vs_plain_f32"], r.get("ratio_vs_flood_f32"),
                                            r["fer_within_10pct"]]
        opt.append(("equal_fer", eq))
    f = line.get("forms")
    if f:
        gb = {k: f[k]["value"] for k in ("flood_f16", "layered_f32", "layered_f16", "stream_f32", "stream_f16",
                                          "plain_f32", "layered_i8") if k in f}
        if "mixed_f16" in f:
            gb["mixed_f16_graph"] = f["mixed_f16"]["graph_info_gbps"]
            gb["mixed_f16_eager"] = f["mixed_f16"]["eager_info_gbps"]
        if "large_code" in f:
            gb["n26112_f16"] = f["large_code"]["cluster_f16"]["value"]
        extra = {"stream_f32_hbm_frac": f.get("stream_f32", {}).get("roofline", {}).get("frac"),
                 "layered_i8_gedge_s": f.get("layered_i8", {}).get("edge_updates_per_s", 0) / 1e9,
                 "layered_i8_alu_frac": f.get("layered_i8", {}).get("roofline", {}).get("frac")}
        opt.append(("forms_gbps", gb))
        opt.append(("forms_extra", extra))
    out["details"] = details_path
    out = _sig(out)
    opt = [(k, _sig(v)) for k, v in opt]
    for k, v in opt:                 # in priority order; a section that would not fit is left out
        trial = dict(out, **{k: v})
        if len(json.dumps(trial)) <= SUMMARY_LIMIT:
            out = trial
    return out


# ------------------------------------------------------------------ reference arm (the oracle)

# rate-1/2 codes at the frame lengths of the paper's throughput figures (Sec. IV)
PAPER_SHAPE_CODES = ["qc12x24_z24_s6", "qc16x32_z32_s7", "qc12x24_z50_s8", "qc12x24_z81_s2", "qc12x24_z96_s9",
                     "qc10x20_z200_s10", "qc20x40_z200_s11"]


def run_paper_shape(ldpc, dev, reps: int = 3):
    """Throughput over frame length for a fixed number of layered iterations (5 and 10, no
    early exit), the shape of the paper's Sec. IV measurements: end to end through the host
    API (pinned LLRs in, decisions out, copies included) with W = 1 and W = 3 streams, and the
    device-resident decode alone.  2^24 coded bits per run at 2.0 dB, each row with its FER.
    At 2.0 dB the int8 min-sum fails most frames of the long codes, so every code also gets an
    int8 row at its own operating point: the lowest Eb/N0 on a 0.25 dB grid from 2.0 dB at
    which 10 iterations give FER <= 1e-2 (noise drawn on the device, seeded)."""
    import torch

    from paper_1812_06545_gb300 import inputs as I

    out = []
    stream = torch.cuda.current_stream(dev)

    def device_llr(c_dev, rate, eb, seed):
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        s2 = 1.0 / (2.0 * rate * 10.0 ** (eb / 10.0))
        y = (1.0 - 2.0 * c_dev.float()) + (s2 ** 0.5) * torch.randn(c_dev.shape, generator=g, device=dev)
        return (2.0 / s2) * y

    for name in PAPER_SHAPE_CODES:
        B, Z = I.load_code(name)
        code = ldpc.Code(B, Z)
        n = (1 << 24) // code.N
        rate = code.K / code.N
        _, _, c, L = I.make_frames(name, n, 2.0, 71, 72)
        Lh = torch.from_numpy(L).pin_memory()
        bh = torch.empty((n, code.N), dtype=torch.uint8).pin_memory()
        ih = torch.empty((n,), dtype=torch.int32).pin_memory()
        Ld = Lh.to(dev)
        c_dev = torch.from_numpy(c).to(dev)
        bd = torch.empty((n, code.N), dtype=torch.uint8, device=dev)
        idv = torch.empty((n,), dtype=torch.int32, device=dev)
        chunk = (n + 11) // 12

        def device_rate(p, x):
            wsb = ldpc.ldpc_workspace_size(code.handle, p, n)
            ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
            times = []
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ldpc.ldpc_decode_batch(code.handle, p, x, ldpc.LDPC_LLR_F32, n, bd, idv, None, ws, wsb, stream)
                e1.record(stream)
                e1.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1) * 1e-3)
            return n * code.K / float(np.median(times)) / 1e9, float((bd != c_dev).any(dim=1).float().mean())

        def host_rates(p, Lhost, row):
            for W in (1, 3):
                times = []
                for r in range(reps + 1):
                    t0 = time.perf_counter()
                    ldpc.ldpc_decode_host(code.handle, p, Lhost, n, bh, ih, n_streams=W, chunk_cw=chunk)
                    if r:
                        times.append(time.perf_counter() - t0)
                row[f"e2e_info_gbps_w{W}"] = n * code.K / float(np.median(times)) / 1e9
            row["fer"] = float((bh.numpy() != c).any(axis=1).mean())

        for form in ("layered_f32", "layered_i8"):
            for T in (5, 10):
                kw = {"llr_scale": I.llr_scale_for(rate, 2.0)} if form == "layered_i8" else {}
                p = ldpc.params_for(form, max_iter=T, early_exit=0, **kw)
                gbps, _ = device_rate(p, Ld)
                row = {"code": name, "N": code.N, "K": code.K, "codewords": n, "form": form, "iterations": T,
                       "ebn0_db": 2.0, "device_info_gbps": gbps}
                host_rates(p, Lh, row)
                out.append(row)
        # int8 at its own operating point (FER <= 1e-2 at 10 iterations)
        eb = 2.0
        while eb <= 6.0:
            p = ldpc.params_for("layered_i8", max_iter=10, early_exit=0, llr_scale=I.llr_scale_for(rate, eb))
            x = device_llr(c_dev, rate, eb, 7300 + int(eb * 100))
            gbps, fer = device_rate(p, x)
            if fer <= 1e-2:
                row = {"code": name, "N": code.N, "K": code.K, "codewords": n, "form": "layered_i8",
                       "iterations": 10, "ebn0_db": eb, "operating_point": "FER <= 1e-2", "device_info_gbps": gbps}
                host_rates(p, x.cpu().pin_memory(), row)
                out.append(row)
                break
            eb += 0.25
        ldpc.ldpc_release_host_buffers()
        del code
    return {"what": "info Gbit/s over frame length, fixed layered iterations (no early exit), 2^24 coded bits per "
                    "run at 2.0 dB, plus an int8 row per code at its FER <= 1e-2 operating point; e2e through "
                    "ldpc_decode_host with W streams (12 chunks), device = decode of HBM-resident LLRs; fer "
                    "of every row beside its throughput", "rows": out}


def run_equal_fer(ldpc, dev, n_frames: int = 400000, chunk: int = 50000):
    """Throughput at equal frame error rate.  For each code: E* = the Eb/N0 where FP32
    flooding (max 20 iterations, early exit) has FER 1e-3 (sweep, then log-FER interpolated
    in dB); at E* the plain FP32 comparator is measured on n_frames frames, and every other
    form gets the smallest max_iter on a ladder whose FER is within 10 % of the comparator's;
    its throughput there over the comparator's is the ratio.  Frames: codewords from an
    encoded pool of 8192, BPSK/AWGN noise drawn on the device (seeded), the same frames for
    every form at a point.  Device-resident decode timed with CUDA events."""
    import torch

    from paper_1812_06545_gb300 import inputs as I

    stream = torch.cuda.current_stream(dev)
    ladder = (4, 5, 6, 8, 10, 12, 15, 20, 30, 50)

    def frames(pool, rate, eb, seed, n):
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        idx = torch.arange(n, device=dev) % pool.shape[0]
        x = 1.0 - 2.0 * pool[idx].float()
        s2 = 1.0 / (2.0 * rate * 10.0 ** (eb / 10.0))
        y = x + (s2 ** 0.5) * torch.randn(x.shape, generator=g, device=dev)
        return (2.0 / s2) * y, idx

    def measure(code, pool, rate, form, eb, max_iter, n, seed0):
        kw = {"llr_scale": I.llr_scale_for(rate, eb)} if form == "layered_i8" else {}
        p = ldpc.params_for(form, max_iter=max_iter, early_exit=1, **kw)
        errs, ms, it_sum = 0, 0.0, 0
        for k in range(0, n, chunk):
            m = min(chunk, n - k)
            L, idx = frames(pool, rate, eb, seed0 + k // chunk, m)
            bits = torch.empty((m, code.N), dtype=torch.uint8, device=dev)
            iters = torch.empty((m,), dtype=torch.int32, device=dev)
            wsb = ldpc.ldpc_workspace_size(code.handle, p, m)
            ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ldpc.ldpc_decode_batch(code.handle, p, L, ldpc.LDPC_LLR_F32, m, bits, iters, None, ws, wsb, stream)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            errs += int((bits != pool[idx]).any(dim=1).sum())
            it_sum += int(iters.sum())
        return {"fer": errs / n, "errors": errs, "frames": n, "max_iter": max_iter, "avg_iterations": it_sum / n,
                "info_gbps": n * code.K / (ms * 1e-3) / 1e9}

    out = []
    for name, forms in (("qc12x24_z81_s2", ("flood_f32", "flood_f16", "layered_f32", "layered_f16", "layered_i8")),
                        ("qc4x24_z81_s3", ("flood_f32", "flood_f16", "layered_f32", "layered_i8"))):
        B, Z, c, _ = I.make_frames(name, 8192, 3.0, 81, 82)
        code = ldpc.Code(B, Z)
        pool = torch.from_numpy(c).to(dev)
        rate = code.K / code.N
        # E*: FER of FP32 flooding over a coarse sweep (n_frames / 4 frames per point)
        pts = []
        eb = 1.5 if rate < 0.6 else 3.0
        while eb < 8.0:
            r = measure(code, pool, rate, "flood_f32", eb, 20, n_frames // 4, 1000)
            pts.append((eb, r["fer"]))
            if r["fer"] < 1e-3:
                if len(pts) > 1:
                    break
                pts, eb = [], eb - 1.0          # started above E*: restart lower
                continue
            eb += 0.25
        (e_a, f_a), (e_b, f_b) = pts[-2], pts[-1]
        if f_b > 0 and f_a > 0:
            e_star = e_a + (np.log(1e-3) - np.log(f_a)) / (np.log(f_b) - np.log(f_a)) * (e_b - e_a)
        else:
            e_star = e_b
        ref = measure(code, pool, rate, "plain_f32", e_star, 20, n_frames, 2000)
        ref["form"] = "plain_f32"
        rows = []
        for form in forms:
            best = None
            for T in ladder:
                r = measure(code, pool, rate, form, e_star, T, n_frames, 2000)
                best = r
                if r["fer"] <= 1.1 * ref["fer"]:
                    break
            best["form"] = form
            best["fer_within_10pct"] = bool(best["fer"] <= 1.1 * ref["fer"])
            best["ratio_vs_plain_f32"] = best["info_gbps"] / ref["info_gbps"]
            if not best["fer_within_10pct"]:
                # context for a form that cannot match the comparator's FER at E*: the Eb/N0 at
                # which it reaches FER 1e-3 itself (max_iter as on the ladder's last rung)
                eb2, prev = e_star, (e_star, best["fer"])
                while eb2 < e_star + 2.0:
                    eb2 += 0.1
                    r2 = measure(code, pool, rate, form, eb2, best["max_iter"], n_frames // 4, 3000)
                    if r2["fer"] <= 1e-3:
                        f0, f1 = max(prev[1], 1e-9), max(r2["fer"], 1e-9)
                        own = prev[0] + (np.log(1e-3) - np.log(f0)) / (np.log(f1) - np.log(f0)) * (eb2 - prev[0]) \
                            if f1 < f0 else eb2
                        best["own_ebn0_star_db"] = float(own)
                        best["snr_gap_db"] = float(own - e_star)
                        break
                    prev = (eb2, r2["fer"])
            rows.append(best)
        f32 = [r for r in rows if r["form"] == "flood_f32"]
        for r in rows:
            r["ratio_vs_flood_f32"] = r["info_gbps"] / f32[0]["info_gbps"] if f32 else None
        out.append({"code": name, "N": code.N, "K": code.K, "ebn0_star_db": float(e_star),
                    "sweep_fp32_flooding": [{"ebn0_db": e, "fer": f} for e, f in pts], "reference": ref,
                    "forms": rows})
        del code
    return {"what": "info Gbit/s at equal FER: E* where FP32 flooding (max 20, early exit) has FER 1e-3; each "
                    "form at the smallest max_iter whose FER is within 10 % of the plain FP32 comparator's at E*; ratios against "
                    "the plain comparator and against the optimised FP32 flooding decoder",
            "codes": out}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1812_06545_gb300 import inputs as I
    from oracle import oracle as O

    O.build()
    w, B, Z, frames = workload_frames(WORKLOAD)
    oc = O.QCCode(B, Z)
    # size each step for ~2 s of CPU work
    t0 = time.perf_counter()
    oc.spa_flood(frames[0][2][:8], w.max_iter, True)
    per_cw = max((time.perf_counter() - t0) / 8, 1e-5)
    n = int(max(4, min(w.batch, 2.0 / (per_cw * len(frames)))))
    for _ in range(args.warmup):
        for eb, c, L in frames:
            oc.spa_flood(L[:n], w.max_iter, True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for eb, c, L in frames:
            oc.spa_flood(L[:n], w.max_iter, True)
    dt = time.perf_counter() - t0
    value = args.steps * n * len(frames) * oc.K / dt / 1e9
    sample = f"first {n} codewords of each of the {len(frames)} Eb/N0 batches per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "FP64 flooding sum-product (CPU oracle)", "code": w.code,
                       "batch": w.batch, "ebn0_db": w.ebn0_db, "max_iter": w.max_iter, "early_exit": True},
            "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm

def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_1812_06545_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()
    from paper_1812_06545_gb300 import ldpc

    def barrier():
        if dist:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(dist, x, dev)

    # ---------------- inputs resident in HBM before timing
    w, B, Z, frames = workload_frames(WORKLOAD, rank)
    code = ldpc.Code(B, Z)
    xs = [torch.from_numpy(L).to(dev) for _, _, L in frames]
    n_per_batch = w.batch
    stream = torch.cuda.current_stream(dev)

    def params(form):
        return ldpc.params_for(form, max_iter=w.max_iter, early_exit=1 if w.early_exit else 0)

    def run_form(form, steps, warmup, profile=False, lat=None):
        p = params(form)
        bits = [torch.empty((n_per_batch, code.N), dtype=torch.uint8, device=dev) for _ in xs]
        iters = [torch.empty((n_per_batch,), dtype=torch.int32, device=dev) for _ in xs]
        wsb = ldpc.ldpc_workspace_size(code.handle, p, n_per_batch)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)

        def step(events=None):
            for i, x in enumerate(xs):
                if events is not None:
                    events[i][0].record(stream)
                ldpc.ldpc_decode_batch(code.handle, p, x, ldpc.LDPC_LLR_F32, n_per_batch, bits[i], iters[i], None,
                                       ws, wsb, stream)
                if events is not None:
                    events[i][1].record(stream)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        if profile:
            ldpc.ldpc_profile_reset()
            ldpc.ldpc_profile_enable(True)
        ldpc.ldpc_launch_count_reset()
        evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in xs] for _ in range(steps)] \
            if lat is not None else None
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for k in range(steps):
            step(evs[k] if evs else None)
        s1.record(stream)
        torch.cuda.synchronize()
        launches = ldpc.ldpc_launch_count()
        barrier()
        torch.cuda.synchronize()
        if profile:
            ldpc.ldpc_profile_enable(False)
        ms = s0.elapsed_time(s1)
        if lat is not None:
            lat.extend(e[0].elapsed_time(e[1]) for st in evs for e in st)
        return ms, launches, bits, iters

    # ---------------- headline: FP32 flooding sum-product
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    lat = []
    ms, launches, bits, iters = run_form("flood_f32", args.steps, args.warmup, profile=True, lat=lat)
    clocks = sampler.stop() if sampler else None
    ms_max = max_over_ranks(ms)
    units = world * args.steps * len(xs) * n_per_batch
    value = whole_job_gbps(world, args.steps * len(xs) * n_per_batch, code.K, ms_max * 1e-3)

    # FER and iteration statistics of the last timed step
    fer = {}
    iters_np = []
    for (eb, c, _), b, it in zip(frames, bits, iters):
        bn = b.cpu().numpy()
        fer[f"{eb:.2f}"] = float((bn != c).any(axis=1).mean())
        iters_np.append(it.cpu().numpy())

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    N, E, T = code.N, code.E, w.max_iter

    # roofline of the slot decoder (the headline form's only kernel): compute-bound; in the
    # product (tanh) domain every edge update needs one exponential (of |Q|) and the
    # logarithm of one ratio (of the other edges' pair: two logarithms, or a logarithm and
    # a reciprocal; rcp.approx runs at the lg2 rate), on the special-function units whose
    # throughput is measured live.  The phi-domain rule (two phi per edge update, each an
    # exponential and the logarithm of a ratio) has half this ceiling.
    n_sl, sl_ms = ldpc.ldpc_profile_read("slots")
    edge_updates = args.steps * E * int(sum(int(it.sum()) for it in iters_np))
    ex2_s, lg2_s = ldpc.ldpc_sfu_throughput(stream)
    sfu_peak = 1.0 / (1.0 / ex2_s + 2.0 / lg2_s) / 1e9                  # Gedge/s
    sfu_peak_phi = 1.0 / (2.0 / ex2_s + 4.0 / lg2_s) / 1e9
    achieved = edge_updates / (sl_ms * 1e-3) / 1e9 if sl_ms > 0 else None
    traffic = stored_traffic("k_flood_slots", SLOTS_SOURCES)
    roofline = {"bound": "alu", "kernel": "k_flood_slots (on-chip flooding slot decoder)", "achieved": achieved,
                "peak": sfu_peak, "unit": "Gedge/s", "frac": (achieved / sfu_peak) if achieved else None,
                "frac_of_phi_rule_ceiling": (achieved / sfu_peak_phi) if achieved else None,
                "peak_source": (f"derived from the special-function throughput measured live on this GPU "
                                f"(ex2 {ex2_s / 1e12:.2f} T/s = {ex2_s / n_sm / (sm_mhz * 1e6):.1f}/clk/SM, lg2 "
                                f"{lg2_s / 1e12:.2f} T/s = {lg2_s / n_sm / (sm_mhz * 1e6):.1f}/clk/SM at {sm_mhz:.0f} MHz): "
                                f"1 / (1/ex2 + 2/lg2) edge updates per second: the product-domain check rule, "
                                f"one exponential and the logarithm of one ratio (two lg2-rate operations) per "
                                f"edge update; the phi-domain rule's ceiling is {sfu_peak_phi:.1f}"),
                "traffic": traffic, "launches": n_sl, "avg_launch_ms": sl_ms / max(n_sl, 1),
                "algorithmic_work": "edge updates = E x iterations run, summed over codewords"}
    # the same throughput against the HBM limit of a flooding decoder that streams its state
    # through HBM (R read and written, APP and L once per phase: 12E + 12N bytes per
    # codeword-iteration at FP32): how close the on-chip design runs to that design's ceiling
    cw_it_s = edge_updates / E / (sl_ms * 1e-3) if sl_ms > 0 else None
    hbm_limit = hbm_peak * 1e9 / (12 * E + 12 * N)
    roofline["streaming_hbm_equivalent"] = {
        "codeword_iterations_per_s": cw_it_s, "hbm_bound_limit_per_s": hbm_limit,
        "frac": (cw_it_s / hbm_limit) if cw_it_s else None,
        "what": "codeword-iterations/s of the slot decoder over the HBM-bound limit of the streaming flooding "
                "design (12E + 12N bytes per codeword-iteration at the measured copy bandwidth); the slot "
                "decoder itself moves only the LLRs and decisions"}

    line = {"metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "flooding sum-product, FP32 messages (on-chip slot decoder)",
                       "code": w.code,
                       "N": code.N, "K": code.K, "batch": n_per_batch, "ebn0_db": w.ebn0_db,
                       "max_iter": w.max_iter, "early_exit": True, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (7 x 63.7 MB LLR batches per step)"},
            "latency_ms": {"what": "one 8192-codeword decode call", "p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99))},
            "avg_iterations": float(np.mean(np.concatenate(iters_np))), "fer": fer,
            "edge_updates_per_batch": {f"{eb:.2f}": E * int(it.sum()) for eb, it in zip(w.ebn0_db, iters_np)},
            "coded_bit_iterations_per_s": world * args.steps * N * float(sum(int(it.sum()) for it in iters_np)) /
                                          (ms_max * 1e-3),
            "roofline": roofline, "gpu_launches": launches, "clocks": clocks}

    gpu_bits = {"flood_f32": [b.cpu().numpy() for b in bits]}

    # ---------------- other forms on the same inputs
    if not args.no_forms:
        forms = {}
        # on-chip forms: special-function roofline of their slot kernel (same peak as above)
        sfu_family = {"flood_f16": "slots", "layered_f32": "layered_spa", "layered_f16": "layered_spa"}
        for form in ("flood_f16", "layered_f32", "layered_f16", "stream_f32", "stream_f16", "plain_f32"):
            prof = form.startswith("stream") or form in sfu_family
            fms, fl, fb, fi = run_form(form, args.steps, args.warmup, profile=prof)
            fms = max_over_ranks(fms)
            fv = units * code.K / (fms * 1e-3) / 1e9
            fi_np = [x.cpu().numpy() for x in fi]
            if form == "flood_f16":
                gpu_bits[form] = [b.cpu().numpy() for b in fb]
            ffer = {f"{eb:.2f}": float((b.cpu().numpy() != c).any(axis=1).mean()) for (eb, c, _), b in zip(frames, fb)}
            forms[form] = {"value": fv, "ms_per_step": fms / args.steps, "fer": ffer, "gpu_launches": fl,
                           "avg_iterations": float(np.mean(np.concatenate(fi_np)))}
            if form.startswith("stream"):
                forms[form]["roofline"] = streaming_roofline(ldpc, fi_np, args.steps, N, E, T, hbm_peak, peak_src)
            elif form in sfu_family:
                fn, fk_ms = ldpc.ldpc_profile_read(sfu_family[form])
                fach = args.steps * E * int(sum(int(it.sum()) for it in fi_np)) / (fk_ms * 1e-3) / 1e9 \
                    if fk_ms > 0 else None
                forms[form]["roofline"] = {"bound": "alu", "achieved": fach, "peak": sfu_peak, "unit": "Gedge/s",
                                           "frac": (fach / sfu_peak) if fach else None, "launches": fn,
                                           "avg_launch_ms": fk_ms / max(fn, 1)}
        plain = forms["plain_f32"]["value"]
        forms["flood_f32"] = {"value": value, "vs_plain_f32": value / plain}
        for f in ("flood_f16", "layered_f32", "layered_f16", "stream_f32", "stream_f16"):
            forms[f]["vs_plain_f32"] = forms[f]["value"] / plain
        # the small latency case: 128 codewords of the N=648 code, 10 fixed iterations, the
        # plain comparator beside the slot decoder (whole decode state L2-resident)
        sw, SB, SZ, sframes = workload_frames("flood_n648_b128", rank)
        scode = ldpc.Code(SB, SZ)
        sx = torch.from_numpy(sframes[0][2]).to(dev)
        small = {"workload": "flood_n648_b128 (128 codewords, N=648 rate 1/2, 2.0 dB, 10 fixed iterations)"}
        for form in ("plain_f32", "flood_f32", "layered_f32"):
            sp = ldpc.params_for(form, max_iter=sw.max_iter, early_exit=0)
            sb = torch.empty((sw.batch, scode.N), dtype=torch.uint8, device=dev)
            si = torch.empty((sw.batch,), dtype=torch.int32, device=dev)
            swsb = ldpc.ldpc_workspace_size(scode.handle, sp, sw.batch)
            sws = torch.empty(max(swsb, 256), dtype=torch.uint8, device=dev)
            lat_us = []
            for k in range(60):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ldpc.ldpc_decode_batch(scode.handle, sp, sx, ldpc.LDPC_LLR_F32, sw.batch, sb, si, None, sws, swsb,
                                       stream)
                e1.record(stream)
                e1.synchronize()
                if k >= 10:
                    lat_us.append(e0.elapsed_time(e1) * 1e3)
            small[form] = {"p50_us": float(np.percentile(lat_us, 50)), "p99_us": float(np.percentile(lat_us, 99)),
                           "info_gbps": sw.batch * scode.K / (np.percentile(lat_us, 50) * 1e-6) / 1e9}
        forms["small_latency"] = small
        # the N = 26112 code (one codeword exceeds an SM): the cluster decoder, against the
        # streaming kernels it replaces for such codes
        bB, bZ = I.load_code("qc34x68_z384_s5")
        bcode = ldpc.Code(bB, bZ)
        _, _, bc, bL = I.make_frames("qc34x68_z384_s5", 2048, 2.0, 91 + 1000 * rank, 92 + 1000 * rank)
        bx = torch.from_numpy(bL).to(dev)
        large = {"workload": "2048 codewords of the N=26112 rate-1/2 code (qc34x68_z384_s5) at 2.0 dB, <= 20 iterations"}
        for form in ("flood_f16", "stream_f16"):
            bp = ldpc.params_for(form, max_iter=20)
            bb = torch.empty((2048, bcode.N), dtype=torch.uint8, device=dev)
            bi = torch.empty((2048,), dtype=torch.int32, device=dev)
            for _ in range(args.warmup):
                ldpc.ldpc_decode_batch(bcode.handle, bp, bx, ldpc.LDPC_LLR_F32, 2048, bb, bi, None, None, 0, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                ldpc.ldpc_decode_batch(bcode.handle, bp, bx, ldpc.LDPC_LLR_F32, 2048, bb, bi, None, None, 0, stream)
            e1.record(stream)
            e1.synchronize()
            bms = e0.elapsed_time(e1) / 3
            large["cluster_f16" if form == "flood_f16" else "stream_f16"] = {
                "value": 2048 * bcode.K / (bms * 1e-3) / 1e9, "ms_per_decode": bms,
                "avg_iterations": float(bi.float().mean()),
                "fer": float((bb.cpu().numpy() != bc).any(axis=1).mean()),
                "edge_updates_per_s": bcode.E * float(bi.sum()) / (bms * 1e-3)}
        forms["large_code"] = large
        # the autotuner's candidate times on the headline code (a separate code object, so no
        # other section sees the pick): one or two codewords per thread in the slot decoder,
        # or the streaming kernels, on the 1.0 dB batch of 8192 codewords
        acode = ldpc.Code(B, Z)
        tuned = {}
        for form in ("flood_f32", "flood_f16"):
            choice, tms = ldpc.ldpc_autotune(acode.handle, params(form), xs[0], ldpc.LDPC_LLR_F32, n_per_batch, stream)
            tuned[form] = {"choice": {1: "slots x1", 2: "slots x2", 3: "streaming"}.get(choice, str(choice)),
                           "ms_slots_x1": float(tms[0]), "ms_slots_x2": float(tms[1]), "ms_streaming": float(tms[2])}
        forms["autotune_headline_code"] = tuned
        del acode
        # int8 layered min-sum on its own workload (rate 5/6, 65536 codewords, 4.0 dB)
        lw, LB, LZ, lframes = workload_frames(LAYERED_WORKLOAD, rank)
        lcode = ldpc.Code(LB, LZ)
        lx = torch.from_numpy(lframes[0][2]).to(dev)        # fp32 LLRs; quantised inside the kernel
        lp = ldpc.params_for("layered_i8", max_iter=lw.max_iter,
                             llr_scale=I.llr_scale_for(lcode.K / lcode.N, lw.ebn0_db[0]))
        lbits = torch.empty((lw.batch, lcode.N), dtype=torch.uint8, device=dev)
        lit = torch.empty((lw.batch,), dtype=torch.int32, device=dev)
        for _ in range(args.warmup):
            ldpc.ldpc_decode_batch(lcode.handle, lp, lx, ldpc.LDPC_LLR_F32, lw.batch, lbits, lit, None, None, 0, stream)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ldpc.ldpc_profile_reset()
        ldpc.ldpc_profile_enable(True)
        e0.record(stream)
        for _ in range(args.steps):
            ldpc.ldpc_decode_batch(lcode.handle, lp, lx, ldpc.LDPC_LLR_F32, lw.batch, lbits, lit, None, None, 0, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ldpc.ldpc_profile_enable(False)
        lms = max_over_ranks(e0.elapsed_time(e1))
        lv = world * args.steps * lw.batch * lcode.K / (lms * 1e-3) / 1e9
        lit_np = lit.cpu().numpy()
        # mixed codes in one persistent launch: 20000 codewords over 12 codes (FP16 messages),
        # schedules autotuned per code, the launch captured in a CUDA graph and replayed
        mixed = run_mixed(ldpc, dev, rank, world, args.steps, args.warmup, max_over_ranks, barrier)
        mixed_frames = mixed.pop("frames")
        forms["mixed_f16"] = mixed
        i8_eps = float(lcode.E * lit_np.sum() * args.steps / (lms * 1e-3))
        # integer-issue roofline of the min-sum (the survey's definition): every SM retires 128
        # int32 lane operations per clock and an edge update takes about 13.5 of them (sub,
        # saturate, abs, min1/min2 tracking, sign xor; select, scale, sign, add, saturate); the
        # packed binary16 kernel does two codewords per lane operation, so its own ceiling is
        # twice this one
        i8_peak = n_sm * 128 * sm_mhz * 1e6 / 13.5
        forms["layered_i8"] = {"workload": LAYERED_WORKLOAD, "code": lw.code, "value": lv,
                               "ms_per_decode": lms / args.steps, "avg_iterations": float(lit_np.mean()),
                               "fer": {f"{lw.ebn0_db[0]:.2f}": float((lbits.cpu().numpy() != lframes[0][1])
                                                                     .any(axis=1).mean())},
                               "edge_updates_per_s": i8_eps,
                               "roofline": {"bound": "alu", "kernel": "k_layered_pairs", "achieved": i8_eps / 1e9,
                                            "peak": i8_peak / 1e9, "unit": "Gedge/s", "frac": i8_eps / i8_peak,
                                            "frac_of_packed_ceiling": i8_eps / (2 * i8_peak),
                                            "peak_source": f"{n_sm} SMs x 128 int32 lanes per clock x {sm_mhz:.0f} MHz "
                                                           f"/ 13.5 integer operations per edge update"}}
        line["forms"] = forms

    # ---------------- end to end through the C ABI with host buffers
    Lh = torch.from_numpy(np.concatenate([L for _, _, L in frames])).pin_memory()
    ntot = Lh.shape[0]
    bh = torch.empty((ntot, code.N), dtype=torch.uint8).pin_memory()
    ih = torch.empty((ntot,), dtype=torch.int32).pin_memory()
    p32 = params("flood_f32")
    chunk = 4096
    for _ in range(max(1, args.warmup)):
        ldpc.ldpc_decode_host(code.handle, p32, Lh, ntot, bh, ih, args.streams, chunk)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ldpc.ldpc_decode_host(code.handle, p32, Lh, ntot, bh, ih, args.streams, chunk)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    barrier()
    e2e = {"value": world * args.steps * ntot * code.K / e2e_s / 1e9, "unit": "Gbit/s",
           "h2d_bytes_per_step": int(Lh.numel() * 4), "d2h_bytes_per_step": int(bh.numel() + ih.numel() * 4),
           "streams": args.streams, "chunk_codewords": chunk, "api": "ldpc_decode_host"}
    ok = all(np.array_equal(bh[i * n_per_batch:(i + 1) * n_per_batch].numpy(), bits[i].cpu().numpy())
             for i in range(len(xs)))
    e2e["matches_device_path"] = bool(ok)
    line["e2e"] = e2e
    ldpc.ldpc_release_host_buffers()

    # ---------------- serving loop: Poisson arrivals of mixed requests (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_serving:
        line["serving"] = run_serving(ldpc, dev, args.serve_seconds)

    # ---------------- equal-FER comparison (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_equal_fer:
        line["equal_fer"] = run_equal_fer(ldpc, dev, args.fer_frames)

    # ---------------- paper-shape sweep: frame length x iterations x streams (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_paper_shape:
        line["paper_shape"] = run_paper_shape(ldpc, dev)

    # ---------------- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sample, cores, errs, nfr, obits = oracle_sample_rate(frames, w.code, w.max_iter, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate / 1e9, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "fer_sample": errs / nfr}
        # the flooding forms against the FP64 oracle on the same sampled codewords: FER delta
        # per Eb/N0 point and the share of identical decisions
        deltas = {}
        for form, gb in gpu_bits.items():
            per = {}
            same = tot = 0
            for (eb, c, _), ob, g in zip(frames, obits, gb):
                n = ob.shape[0]
                fo = float((ob != c[:n]).any(axis=1).mean())
                fg = float((g[:n] != c[:n]).any(axis=1).mean())
                per[f"{eb:.2f}"] = {"oracle_fer": fo, "gpu_fer": fg, "delta": fg - fo}
                same += int((g[:n] == ob).all(axis=1).sum())
                tot += n
            deltas[form] = {"per_ebn0": per, "identical_decisions": same / tot}
        line["cpu_baseline"]["fer_delta_vs_oracle"] = deltas
    if rank == 0:
        if not args.no_forms and not args.no_cpu_baseline and "cpu_baseline" in line:
            line["cpu_baseline"]["mixed_f16"] = mixed_oracle_check(mixed_frames, 64, 6.0)
        try:
            with open(args.details, "w") as f:
                json.dump(line, f, indent=1)
        except OSError as ex:
            print(f"bench: could not write {args.details}: {ex}", file=sys.stderr)
        print(json.dumps(summary_line(line, args.details)))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
