"""The benchmark's last stdout line is short enough to survive a truncated log tail
and carries every key the measurement contract names (no GPU needed)."""
import json
import math

import bench


def _tte(arms, targets):
    return {f"{t:g}": {a: {"ms": 1.0 + k + 10 * t, "extrapolated": k == 0} for k, a in enumerate(arms)}
            for t in targets}


def _fake():
    line = {"metric": bench.METRIC, "value": 3.3812345678e9, "unit": "packets/s", "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 19.8612345, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": bench.workload_config(1 << 26),
            "roofline": {"bound": "alu", "achieved": 14.2912345, "peak": 40.2712345, "unit": "Tops/s",
                         "frac": 0.35512345, "traffic": 80123456.0, "kernel": "k_trace_single<float>",
                         "kernel_ms": 19.8412345, "per_unit": "10 ops per cell visit x 422.34 cells per packet",
                         "peak_basis": "152 SMs x 128 lanes x 2070 MHz (measured max clock)"},
            "e2e": {"value": 3.3112345e9, "unit": "packets/s", "h2d_bytes_per_step": 67108864,
                    "d2h_bytes_per_step": 1572864},
            "gpu_launches": 40, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 400}}
    gens = ["sobol", "sobol_owen", "niederreiter", "faure", "halton", "hammersley", "mc_philox"]
    sec = {"multiple_scattering": {"packets_per_s": 1.87e8, "path": "wavefront", "roofline": {"frac": 0.1261234}},
           "batched": {"packets_per_s": 2.2512345e9, "speedup_at_equal_images": 1.01312345,
                       "time_to_error": {"speedup": 1.5123}},
           "observers": {"speedup": 3.112345, "identical_images": True},
           "time_to_error_learned_vs_plain": {"time_to_error_ms": _tte(["plain_qmc", "learned_qmc", "mc_philox"],
                                                                       (0.05, 0.03, 0.01, 0.001))},
           "cpu_baseline": {"value": 2245756.126, "unit": "packets/s", "cores": 16, "kind": "oracle",
                            "sample": "first 25970350 packets of the workload (same Sobol points), FP64 C oracle, "
                                      "16 threads, 11.6 s",
                            "sample_short": "first 25970350 packets, 16 threads",
                            "single_core": {"value": 119789.0146, "unit": "packets/s", "sample": "x"}}}
    for k in ("disk", "disk_pole", "shell", "fractal"):
        sec[f"time_to_error_qmc_vs_mc_{k}"] = {"time_to_error_ms": _tte(gens, (0.05, 0.02, 0.01, 0.003))}
    return line, sec


def test_headline_is_short_and_complete():
    line, sec = _fake()
    h = bench.headline(line, sec)
    text = json.dumps(h, separators=(",", ":"))  # as bench.py prints it
    assert len(text) <= 1400, len(text)  # the recorded log tail keeps 1500 bytes
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
              "config", "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches"):
        assert k in h, k
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in h["roofline"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in h["cpu_baseline"], k
    assert h["value"] > 0 and math.isfinite(h["value"])
    assert json.loads(text)["sections"]["learned_vs_plain_at_rms"]


def test_speedup_summary_and_rounding():
    tte = {"0.01": {"a": {"ms": 10.0, "extrapolated": False}, "b": {"ms": 4.0, "extrapolated": True}},
           "0.05": {"a": {"ms": None, "extrapolated": True}, "b": {"ms": 1.0, "extrapolated": False}}}
    sp, ex = bench._speedups(tte, "a", "b")
    assert sp == {"0.01": 2.5} and ex == ["0.01"]
    assert bench._sig(3.38123456e9, 4) == 3.381e9
    assert bench._sig(None) is None and bench._sig(0) == 0
