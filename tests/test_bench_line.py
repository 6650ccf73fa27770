"""The benchmark's stdout line (CPU): from a full measurement record, `compact_line` keeps every key the
benchmark contract names (metric, value, unit, n_gpus, steps, warmup, ms_per_step, higher_is_better, scaling,
vs_baseline, dtype, data, config, roofline with achieved / peak / frac / traffic, cpu_baseline, e2e with the
copied bytes, clocks, gpu_launches) and the metric's other parts (backward / forward, batched vs plain, the
vegetation workload's rate, roofline and end-to-end figure), in a line short enough to be kept whole by a
reader of its last 2 kB."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def detail_record():
    rf = {"bound": "alu", "kernel": "k_accum (specular accumulator)", "achieved": 23.3, "peak": 80.5, "unit": "TFLOP/s",
          "frac": 0.289, "traffic": 39.9e6}
    return {
        "metric": "Mrays/s (closest + any-hit segments/s; spectra <=1e-4 rel-L2 vs oracle)", "value": 528.1,
        "unit": "Mrays/s", "n_gpus": 1, "steps": 10, "warmup": 3, "ms_per_step": 11.37, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (float-float r and phase)", "data": "synthetic",
        "config": {"workload": "clutter: 202570 triangles, 1000000 rays x 5 bounces, 32 mics, 512 bins 20-80 kHz, "
                               "diffraction on", "triangles": 202570, "rays": 1000000, "bounces": 5, "mics": 32,
                   "bins": 512, "diffraction": True, "step": "simulate (scene prebuilt)",
                   "l2": "flushed between steps (256 MiB write)", "parallelism": "1 pose(s), one per GPU"},
        "mic_spectra_per_s": 2812.0,
        "roofline": rf,
        "roofline_diffraction": dict(rf, bound="tensor", kernel="k_accum_diff_mma (diffraction)", frac=0.112,
                                     peak=1863.0, traffic=21.4e6),
        "cpu_baseline": {"value": 0.083, "unit": "Mrays/s", "cores": 16, "kind": "oracle", "sample": "long text",
                         "seconds": 1.3, "sample_short": "1/61 of the rays and diffraction samples, 1.3 s"},
        "e2e": {"value": 514.2, "unit": "Mrays/s", "h2d_bytes_per_step": 12000412, "d2h_bytes_per_step": 393216,
                "ms_per_step": 11.7},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 300},
        "gpu_launches": 730,
        "adjoint": {"gradient workload (shoebox)": {"bwd_over_fwd": 0.95}, "clutter workload": {"bwd_over_fwd": 1.74}},
        "batched": {"speedup": 2.2, "batched_ms": 213.2, "plain_ms": 468.0},
        "batched_directional": {"speedup": 5.55, "batched_ms": 16.1, "plain_ms": 89.3},
        "vegetation": {"value": 357.5, "ms_per_step": 81.8, "roofline": dict(rf, kernel="k_accum_narrow x"),
                       "e2e": {"value": 354.4, "unit": "Mrays/s", "h2d_bytes_per_step": 57473620,
                               "d2h_bytes_per_step": 49152}},
    }


def test_compact_line_keeps_the_contract():
    bench = load_bench()
    line = bench.compact_line(detail_record())
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < 2048, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in line, k
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    assert abs(line["roofline"]["frac"] - 0.289) < 1e-9
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in line["cpu_baseline"], k
    assert line["cpu_baseline"]["kind"] == "oracle"
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in line["clocks"], k
    assert line["bwd_over_fwd"] == {"gradient": 0.95, "clutter": 1.74}
    assert line["batched_vs_plain"]["speedup"] == 2.2 and line["batched_vs_plain_bat"]["speedup"] == 5.55
    assert line["vegetation"]["roofline"]["kernel"] == "k_accum_narrow" and "e2e" in line["vegetation"]
    assert "workload" in line["config"] and "model" not in line["config"]


def test_compact_line_without_the_extras():
    """A run with the extra measurements switched off still prints the contract's keys."""
    bench = load_bench()
    d = detail_record()
    for k in ("adjoint", "batched", "batched_directional", "vegetation", "roofline_diffraction"):
        d[k] = None
    d["cpu_baseline"] = None
    line = bench.compact_line(d)
    assert line["cpu_baseline"] is None and "roofline" in line and "e2e" in line
    assert "bwd_over_fwd" not in line and "vegetation" not in line
