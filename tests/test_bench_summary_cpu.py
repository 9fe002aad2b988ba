"""The benchmark's last stdout line: a compact JSON object carrying every required key, small
enough that a reader keeping only the tail of the output still gets all of it."""
import json

import bench


def full_line():
    per = {f"{1.0 + 0.25 * i:.2f}": {"oracle_fer": 0.123456789, "gpu_fer": 0.123456789, "delta": 0.00137551}
           for i in range(7)}
    rows = [{"form": f, "ratio_vs_plain_f32": 12.3456789, "ratio_vs_flood_f32": 1.23456789, "fer_within_10pct": True,
             "info_gbps": 16.5, "fer": 1e-3, "max_iter": 12} for f in
            ("flood_f32", "flood_f16", "layered_f32", "layered_f16", "layered_i8")]
    roof = {"frac": 0.33512345678}
    return {
        "metric": "decoded info Gbit/s and p99 latency at equal FER vs plain FP32 flooding SPA, 1 GB300",
        "value": 4.98123456789, "unit": "Gbit/s", "n_gpus": 1, "steps": 20, "warmup": 5, "ms_per_step": 11.1923456789,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "flood_n1944_b8192_sweep", "form": "x" * 80, "code": "qc12x24_z81_s2", "N": 1944,
                   "K": 972, "batch": 8192, "ebn0_db": [1.0 + 0.25 * i for i in range(7)], "max_iter": 20,
                   "early_exit": True, "parallelism": "replicas x1", "l2": "y" * 60},
        "latency_ms": {"what": "z" * 40, "p50": 1.6312345678, "p99": 2.0412345678},
        "avg_iterations": 6.93456789, "fer": {k: 0.1 for k in per}, "coded_bit_iterations_per_s": 1.2345678e12,
        "roofline": {"bound": "alu", "kernel": "k" * 40, "achieved": 388.123456789, "peak": 998.123456789,
                     "unit": "Gedge/s", "frac": 0.3891234567, "peak_source": "p" * 300, "traffic": 64512345.0,
                     "launches": 140, "avg_launch_ms": 1.59012345, "algorithmic_work": "w" * 80,
                     "streaming_hbm_equivalent": {"frac": 0.95, "what": "q" * 200}},
        "gpu_launches": 140, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 55, "reasons": []},
        "forms": {**{f: {"value": 5.75123456789, "fer": {k: 0.1 for k in per}, "roofline": roof} for f in
                     ("flood_f16", "layered_f32", "layered_f16", "stream_f32", "stream_f16", "plain_f32")},
                  "layered_i8": {"value": 32.91234567, "edge_updates_per_s": 4.18123456e11,
                                 "roofline": {"frac": 0.2161234}},
                  "mixed_f16": {"graph_info_gbps": 7.4123456, "eager_info_gbps": 7.3412345},
                  "large_code": {"cluster_f16": {"value": 2.75123456}}},
        "e2e": {"value": 4.9712345678, "unit": "Gbit/s", "h2d_bytes_per_step": 445906944,
                "d2h_bytes_per_step": 111706112, "streams": 4, "chunk_codewords": 4096, "api": "ldpc_decode_host"},
        "serving": {"capacity": {"info_gbps": 4.412345678}, "sweep": [{"p99_ms": 2.8123456}],
                    "at_saturation": {"achieved_info_gbps": 4.41234567, "p50_ms": 16.123456, "p99_ms": 89.123456},
                    "valid": True},
        "equal_fer": {"codes": [{"code": c, "ebn0_star_db": 2.5212345, "reference": {"info_gbps": 1.0123456},
                                 "forms": rows} for c in ("qc12x24_z81_s2", "qc4x24_z81_s3")]},
        "paper_shape": {"rows": [{"code": "c" * 16, "fer": 0.5} for _ in range(35)]},
        "cpu_baseline": {"value": 0.0012549223217810522, "unit": "Gbit/s", "cores": 16, "kind": "oracle",
                         "sample": "first 727 codewords of each of the 7 Eb/N0 batches (5089 codewords)",
                         "fer_sample": 0.31, "fer_delta_vs_oracle": {f: {"per_ebn0": per, "identical_decisions": 1.0}
                                                                     for f in ("flood_f32", "flood_f16")},
                         "mixed_f16": {"gpu_fer": 0.0112345, "oracle_fer": 0.0104567}},
    }


REQUIRED = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks")


def test_summary_line_is_compact_and_complete():
    line = full_line()
    s = bench.summary_line(line, "/tmp/ldpc_bench_details.json")
    text = json.dumps(s)
    assert len(text) <= bench.SUMMARY_LIMIT, len(text)
    back = json.loads(text)
    for k in REQUIRED:
        assert k in back, k
    assert back["config"]["workload"] == "flood_n1944_b8192_sweep"
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in back["roofline"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in back["cpu_baseline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in back["e2e"], k
    assert abs(back["value"] - 4.981) < 1e-9 and back["latency_ms"]["p99"] == 2.041
    # the headline sections survive at this size
    for k in ("forms_gbps", "equal_fer", "serving"):
        assert k in back, k
    assert back["cpu_baseline"]["fer_delta_max"]["flood_f16"] == 0.001376


def test_summary_drops_optional_sections_before_required_keys():
    line = full_line()
    c0 = line["equal_fer"]["codes"][0]
    line["equal_fer"]["codes"] = [dict(c0, code=f"qc12x24_z81_s{k}") for k in range(12)]  # far too many rows
    s = bench.summary_line(line, "/tmp/d.json")
    assert len(json.dumps(s)) <= bench.SUMMARY_LIMIT
    assert "equal_fer" not in s and "forms_gbps" in s
    assert s["serving"]["p99_ms"] == 89.12           # the metric's p99 is kept longest
    for k in REQUIRED:
        assert k in s, k


def test_sig_rounds_floats_only():
    assert bench._sig({"a": [1.23456789, 7, "x"], "b": float("nan")}) == {"a": [1.235, 7, "x"], "b": None}


def test_source_hash_ignores_comments_only():
    a = 'int f(int x) { // add one\n  return x + 1; /* done */ }\nconst char *s = "// not a comment";\n'
    b = '/* header */\nint f(int x) {\n  return x + 1; }\nconst char *s = "// not a comment";\n'
    c = 'int f(int x) { return x + 2; }\nconst char *s = "// not a comment";\n'
    assert bench.strip_comments(a).replace(" ", "").replace("\n", "") == \
        bench.strip_comments(b).replace(" ", "").replace("\n", "")
    assert '"// not a comment"' in bench.strip_comments(a)
    assert bench.strip_comments(a) != bench.strip_comments(c)
